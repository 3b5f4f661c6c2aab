"""GPU parity of the full Frank-Wolfe solve (Algorithm 2, Sect. 5.1) at the
512 x 512, M = 200k w-stacked workload the benchmark times, against the FP64
oracle's solve stored in tests/golden/medium_512_w_solve.json (written by the
committed script beside it, which runs only the oracle).

Checked: identical final support, objective within 1e-4 relative, weights
within 1e-3 relative L2 (the reweighting stops early, Sect. 5.1), the final
certificate equal to the oracle's certificate of the returned image at 4096
seeded pixels within 1e-5 relative L2, and per iteration the pruned support
and the active set as INDEX SETS: they may differ only by pixels the oracle
lists as borderline (certificate within the FP32 operator error, 1e-5
max|mu|, of the selection threshold; the reading of non-unique FP32 ties).
The tensor-core Gram is also compared on the oracle's first active set (the
benchmark's first contraction, 873 atoms at M = 200k) on sampled entries.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import operators
from tests.helpers import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "medium_512_w_solve.json")
SCRIPT = os.path.join(HERE, "golden", "make_medium_512_solve.py")


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


@pytest.fixture(scope="module")
def golden():
    g = json.load(open(GOLDEN))
    assert g["script_sha256"] == hashlib.sha256(open(SCRIPT, "rb").read()).hexdigest(), \
        "the golden file was written by another version of its script"
    return g


@pytest.fixture(scope="module")
def problem(golden):
    """The workload and its complex64 visibilities, formed exactly as the golden
    script forms them (oracle forward operator + seeded noise)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", SCRIPT)
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    from paper_2406_01342_gb300 import synth
    wl = synth.WORKLOADS[golden["workload"]]()
    V = mk.visibilities(wl)
    assert abs(float(np.vdot(V, V).real) - golden["V_sumsq"]) <= 1e-12 * golden["V_sumsq"]
    return wl, V


@pytest.mark.parametrize("reweight", [0, 2])
def test_solve_matches_oracle_at_benchmark_size(abi, golden, problem, reweight):
    """The default solve (the cost model picks the Gram form here) and the
    solve with every reweighting in operator form."""
    wl, V = problem
    lam = golden["lambda"]
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    # lambda_max by the GPU certificate agrees with the oracle's
    assert abs(abi.pc_lambda_max(plan, Vd) - golden["lambda_max"]) <= 1e-5 * golden["lambda_max"]
    res = abi.pc_solve(plan, Vd, lam, golden["delta"], reweight=reweight)
    idx = res["idx"].cpu().numpy()
    x = res["x"].cpu().numpy().astype(np.float64)
    assert res["converged"]
    assert idx.tolist() == golden["support"], (idx.tolist(), golden["support"])
    assert abs(res["objective"] - golden["objective"]) <= 1e-4 * golden["objective"]
    assert rel_l2(x, np.array(golden["x"])) <= 1e-3
    assert res["iterations"] == golden["iterations"]
    # the final certificate is the oracle's certificate of the returned image
    pix = np.array(golden["mu_pixels"], dtype=np.int64)
    mu_ref = operators.certificate(wl.uvw, wl.N, wl.fov, V, lam, idx, x, pix)
    assert rel_l2(res["mu"].cpu().numpy().ravel()[pix], mu_ref) <= 1e-5


def test_per_iteration_index_sets_match_oracle(abi, golden, problem):
    """After k reweightings the GPU's pruned support equals the oracle's up to
    borderline pixels; the next active set, formed from the GPU's own state by
    its certificate and selection calls, likewise."""
    wl, V = problem
    lam, delta = golden["lambda"], golden["delta"]
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    hist = golden["history"]
    border = set()
    for k, h in enumerate(hist):
        border |= set(h["borderline"])
        res = abi.pc_solve(plan, Vd, lam, delta, max_fw=k + 1)
        assert len(res["history"]) == k + 1
        g = res["history"][k]
        assert abs(g["n_active"] - h["n_active"]) <= len(h["borderline"]), (k, g, h["n_active"])
        sup = set(res["idx"].cpu().numpy().tolist())
        diff = sup ^ set(h["support"])
        assert diff <= border, (k, sorted(diff - border))
        if k + 1 < len(hist):
            mu, _, _ = abi.pc_certificate(plan, Vd, res["idx"], res["x"], lam)
            nxt = abi.pc_select(plan, mu, 1.0 - delta, res["idx"], 65536).cpu().numpy()
            diff = set(nxt.tolist()) ^ set(hist[k + 1]["active"])
            assert diff <= border | set(hist[k + 1]["borderline"]), (k + 1, sorted(diff))


def test_tensor_core_gram_on_the_oracle_first_active_set(abi, golden, problem):
    """The benchmark's first contraction: the oracle's first active set (all new
    atoms, clustered around the sources) against M = 200k visibilities, 16
    sampled atoms' 136 distinct G entries and their b entries, each within 1e-5
    of its Cauchy-Schwarz bound."""
    from tests.test_gpu_large import gram_errors
    wl, V = problem
    idx = np.array(golden["history"][0]["active"], dtype=np.int32)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vs = V.astype(np.complex64)
    G, b = abi.pc_gram(plan, to_dev(Vs), to_dev(idx), mode=2)
    G = G.cpu().numpy().astype(np.float64)
    b = b.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(53)
    sub = np.sort(np.concatenate([np.arange(8), rng.choice(np.arange(8, idx.size), 8, replace=False)]))
    eG, eb = gram_errors(wl, G, b, Vs, idx, sub)
    assert eG <= 1e-5, eG
    assert eb <= 1e-5, eb
