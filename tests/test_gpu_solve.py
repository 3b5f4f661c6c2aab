"""GPU parity of the Frank-Wolfe solve (Algorithm 2) and its sub-solver against
the FP64 oracle: identical supports, objective within 1e-4 relative, the final
certificate equal (1e-5 relative L2) to the oracle's certificate at the
returned image."""
import numpy as np
import pytest

from oracle import lasso, operators, pfw
from tests.helpers import rel_l2, to_dev, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


def _compare(abi, wl, V, lam, delta, rule="R2", positive=False, **opts):
    Vs = V.astype(np.complex64).astype(np.complex128)
    ref = pfw.solve(wl.uvw, wl.N, wl.fov, Vs, lam, delta, rule=rule, positive=positive)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    res = abi.pc_solve(plan, to_dev(V.astype(np.complex64)), lam, delta,
                       select_rule=1 if rule == "R1" else 2, positivity=int(positive), **opts)
    idx = res["idx"].cpu().numpy()
    x = res["x"].cpu().numpy().astype(np.float64)
    assert idx.tolist() == ref.idx.tolist(), (idx, ref.idx)
    assert abs(res["objective"] - ref.objective) <= 1e-4 * ref.objective
    assert res["converged"] and ref.converged
    # per-iteration active sets follow the oracle's, up to the pixels whose
    # certificate lies within the FP32 operator error (1e-5 max|mu|) of the
    # selection threshold (the oracle counts them)
    assert len(res["history"]) == len(ref.history)
    for g, o in zip(res["history"], ref.history):
        assert abs(g["n_active"] - o["n_active"]) <= o["n_borderline"], (g, o)
        assert abs(g["n_support"] - o["n_support"]) <= o["n_borderline"], (g, o)
    # the final certificate is the certificate of the returned image
    mu_ref = operators.certificate(wl.uvw, wl.N, wl.fov, Vs, lam, idx, x)
    assert rel_l2(res["mu"].cpu().numpy().ravel(), mu_ref) <= 1e-5
    assert rel_l2(x, ref.x) <= 1e-3
    return res, ref


def test_solve_tiny_coplanar(abi):
    wl, V = workload("tiny_64_coplanar")
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V.astype(np.complex64).astype(np.complex128))
    _compare(abi, wl, V, wl.alpha * lmax, wl.delta)


def test_solve_wide_field_w(abi):
    wl, V = workload("small_wide_w")
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V.astype(np.complex64).astype(np.complex128))
    _compare(abi, wl, V, 0.05 * lmax, wl.delta)


def test_solve_rule_r1(abi):
    wl, V = workload("tiny_64_coplanar")
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V.astype(np.complex64).astype(np.complex128))
    _compare(abi, wl, V, wl.alpha * lmax, 0.9, rule="R1")


@pytest.mark.parametrize("rule", ["R2", "R1"])
def test_repeated_solves_on_one_plan_start_fresh(abi, rule):
    """A solve leaves nothing behind that the next solve on the same plan
    sees: the second and third solves repeat the first one's Frank-Wolfe
    iterations (the first active set holds only what the first exploration
    selects, not the previous solve's support) and its result."""
    wl, V = workload("tiny_64_coplanar")
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    lmax = abi.pc_lambda_max(plan, Vd)
    opts = {"select_rule": 1, "lambda_max": lmax} if rule == "R1" else {}
    delta = 0.9 if rule == "R1" else wl.delta
    runs = [abi.pc_solve(plan, Vd, wl.alpha * lmax, delta, **opts) for _ in range(3)]
    first = [h["n_active"] for h in runs[0]["history"]]
    assert len(runs[0]["history"]) > 1
    for r in runs[1:]:
        assert [h["n_active"] for h in r["history"]] == first
        assert r["idx"].cpu().numpy().tolist() == runs[0]["idx"].cpu().numpy().tolist()
        assert abs(r["objective"] - runs[0]["objective"]) <= 1e-6 * runs[0]["objective"]


def test_lambda_above_lambda_max_gives_zero(abi):
    wl, V = workload("tiny_64_coplanar")
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    lmax = abi.pc_lambda_max(plan, Vd)
    res = abi.pc_solve(plan, Vd, lmax * 1.001, wl.delta)
    assert res["idx"].numel() == 0 and res["converged"]
    assert abs(res["objective"] - 0.5 * res["sumsq_V"]) <= 1e-12 * res["sumsq_V"]


@pytest.mark.parametrize("n_rand", [30, 60, 150, 290])
def test_apgd_matches_oracle_subsolver(abi, n_rand):
    """Restricted LASSO by the APGD kernels vs the oracle's FISTA on the same
    support: about 36 atoms (one warp), 66 and 156 (one CTA), 296 (cluster)."""
    wl, V = workload("small_wide_w")
    Vs = V.astype(np.complex64).astype(np.complex128)
    lam = 0.05 * operators.lambda_max(wl.uvw, wl.N, wl.fov, Vs)
    idx = np.sort(np.random.default_rng(9).choice(wl.N * wl.N, n_rand, replace=False))
    idx = np.union1d(idx, wl.sky_idx)
    l, m, n = operators.pixel_lmn(wl.N, wl.fov, idx)
    A = operators.phase_block(wl.uvw, l, m, n)
    G = np.real(A.conj().T @ A).astype(np.float32)
    b = np.real(A.conj().T @ Vs).astype(np.float32)
    x_ref, it_ref, L_ref = lasso.apgd(A, Vs, lam, np.zeros(idx.size), 1e-7, 50_000)
    x = torch.zeros(idx.size, dtype=torch.float32, device="cuda")
    x, it, L = abi.pc_apgd(to_dev(G), to_dev(b), lam, 1e-7, 50_000, x)
    assert abs(L - L_ref) <= 1e-4 * L_ref
    xg = x.cpu().numpy()
    assert rel_l2(xg, x_ref) <= 1e-3
    assert set(np.nonzero(xg)[0]) == set(np.nonzero(x_ref)[0])


def test_solve_host_buffers(abi):
    """pc_solve_host: host uvw / V in, host support out, same result as the device path."""
    wl, V = workload("tiny_64_coplanar")
    res = abi.pc_solve_host(wl.uvw, V.astype(np.complex64), wl.N, wl.fov, wl.alpha, wl.delta)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    lam = wl.alpha * abi.pc_lambda_max(plan, Vd)
    dev = abi.pc_solve(plan, Vd, lam, wl.delta)
    assert res["idx"].tolist() == dev["idx"].cpu().numpy().tolist()
    assert np.allclose(res["x"], dev["x"].cpu().numpy(), rtol=1e-5, atol=0)


def test_tensor_core_and_fp32_gram_give_the_same_solve(abi):
    """The 512 x 512, M = 200k benchmark workload: the solve with the tensor-core
    support contraction and with the FP32 one end on the same support and objective."""
    wl, V = workload("medium_512_w")
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    lam = wl.alpha * abi.pc_lambda_max(plan, Vd)
    a = abi.pc_solve(plan, Vd, lam, wl.delta, gram_mode=1)
    b = abi.pc_solve(plan, Vd, lam, wl.delta, gram_mode=2)
    assert a["idx"].cpu().numpy().tolist() == b["idx"].cpu().numpy().tolist()
    assert abs(a["objective"] - b["objective"]) <= 1e-6 * a["objective"]
    assert a["converged"] and b["converged"]


@pytest.mark.parametrize("name,frac", [("tiny_64_coplanar", None), ("small_wide_w", 0.05)])
def test_solve_operator_form_reweighting(abi, name, frac):
    """The reweighting in operator form (reweight = 2: monotone FISTA whose
    gradient Re Phi_S^H (Phi_S x - V) goes through degridding and gridding on
    every iteration, no Gram matrix) reaches the oracle's solve: same final
    support, per-iteration active sets, objective within 1e-4, weights within
    1e-3 and the final certificate within 1e-5."""
    wl, V = workload(name)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V.astype(np.complex64).astype(np.complex128))
    res, ref = _compare(abi, wl, V, (frac if frac else wl.alpha) * lmax, wl.delta, reweight=2)
    assert all(h["lanczos_steps"] > 0 for h in res["history"] if h["n_active"] > 0)


def test_operator_and_gram_forms_agree_at_benchmark_size(abi):
    """The 512 x 512, M = 200k benchmark workload solved with the Gram-form
    reweighting (tensor-core contraction) and with the operator form end on
    the same support and objective (the cost model picks the Gram form here)."""
    wl, V = workload("medium_512_w")
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    lam = wl.alpha * abi.pc_lambda_max(plan, Vd)
    a = abi.pc_solve(plan, Vd, lam, wl.delta, reweight=1)
    b = abi.pc_solve(plan, Vd, lam, wl.delta, reweight=2)
    c = abi.pc_solve(plan, Vd, lam, wl.delta)
    assert a["idx"].cpu().numpy().tolist() == b["idx"].cpu().numpy().tolist()
    assert abs(a["objective"] - b["objective"]) <= 1e-6 * a["objective"]
    assert c["idx"].cpu().numpy().tolist() == a["idx"].cpu().numpy().tolist()
    assert a["converged"] and b["converged"]


@pytest.mark.parametrize("N", [600, 1100])
def test_operator_form_on_large_grids_matches_the_gram_form(abi, N):
    """On grids of side 2048 and 4096 the operator form's FFT passes run on
    the one-CTA kernels and transform only the image rows that hold active
    atoms: the solve still ends on the Gram form's support and objective."""
    wl, V = workload("small_wide_w", N=N)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    assert abi.pc_plan_info(plan)["grid_side"] in (2048, 4096)
    Vd = to_dev(V.astype(np.complex64))
    # the wide-field layout's main lobes span ~15 pixels here: lambda = 0.5
    # lambda_max keeps the active sets to the lobes (hundreds of atoms)
    lam = 0.5 * abi.pc_lambda_max(plan, Vd)
    a = abi.pc_solve(plan, Vd, lam, wl.delta, reweight=1)
    b = abi.pc_solve(plan, Vd, lam, wl.delta, reweight=2)
    assert a["converged"] and b["converged"]
    assert a["idx"].cpu().numpy().tolist() == b["idx"].cpu().numpy().tolist()
    # the two forms take their FISTA step from different Lanczos estimates
    # (tolerance 1e-5 on the Gram, 1e-3 on the operator) and stop on the
    # relative-change test at eps_min = 1e-5, so their last iterates sit that
    # far apart on the same support
    assert abs(a["objective"] - b["objective"]) <= 1e-5 * a["objective"]
    # the supports here are a few neighbouring pixels of one lobe (two at N =
    # 1100): the objective is flat along directions that move flux between
    # them, so the early stop fixes only their sum (the total flux) tightly
    xa, xb = a["x"].cpu().numpy().astype(np.float64), b["x"].cpu().numpy().astype(np.float64)
    assert abs(xa.sum() - xb.sum()) <= 1e-3 * abs(xa).sum()


# ---------------------------------------------------------------- positivity (remark of Sect. 5.1)

def _signed_workload(name):
    """The workload with its brightest source made negative (so the constraint binds)."""
    from oracle import operators as ops
    wl, _ = workload(name)
    flux = wl.sky_flux.copy()
    flux[int(np.argmax(flux))] *= -1.0
    V = ops.forward(wl.uvw, wl.N, wl.fov, wl.sky_idx, flux) + wl.noise
    return wl, V


@pytest.mark.parametrize("name,frac", [("tiny_64_coplanar", None), ("small_wide_w", 0.05)])
def test_solve_positivity(abi, name, frac):
    """Non-negative solve: candidates only at positive certificate values, the
    reweighting with x >= 0; same support, objective and certificate as the
    oracle's positive solve; every weight positive."""
    wl, V = _signed_workload(name)
    Vs = V.astype(np.complex64).astype(np.complex128)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    lmax_pos = abi.pc_lambda_max_positive(plan, to_dev(V.astype(np.complex64)))
    ref_lmax = operators.lambda_max_positive(wl.uvw, wl.N, wl.fov, Vs)
    assert abs(lmax_pos - ref_lmax) <= 1e-5 * ref_lmax
    assert ref_lmax < operators.lambda_max(wl.uvw, wl.N, wl.fov, Vs)
    lam = (frac if frac else wl.alpha) * ref_lmax
    res, ref = _compare(abi, wl, V, lam, wl.delta, positive=True)
    assert (res["x"].cpu().numpy() > 0).all() and (ref.x > 0).all()


def test_solve_positivity_rule_r1(abi):
    wl, V = _signed_workload("tiny_64_coplanar")
    Vs = V.astype(np.complex64).astype(np.complex128)
    lam = wl.alpha * operators.lambda_max_positive(wl.uvw, wl.N, wl.fov, Vs)
    _compare(abi, wl, V, lam, 0.9, rule="R1", positive=True)


def test_solve_positivity_operator_form(abi):
    wl, V = _signed_workload("small_wide_w")
    Vs = V.astype(np.complex64).astype(np.complex128)
    lam = 0.05 * operators.lambda_max_positive(wl.uvw, wl.N, wl.fov, Vs)
    res, ref = _compare(abi, wl, V, lam, wl.delta, positive=True, reweight=2)
    assert (res["x"].cpu().numpy() > 0).all()


def test_apgd_positive_matches_oracle_subsolver(abi):
    wl, V = _signed_workload("small_wide_w")
    Vs = V.astype(np.complex64).astype(np.complex128)
    lam = 0.05 * operators.lambda_max_positive(wl.uvw, wl.N, wl.fov, Vs)
    idx = np.sort(np.random.default_rng(9).choice(wl.N * wl.N, 60, replace=False))
    idx = np.union1d(idx, wl.sky_idx)
    l, m, n = operators.pixel_lmn(wl.N, wl.fov, idx)
    A = operators.phase_block(wl.uvw, l, m, n)
    G = np.real(A.conj().T @ A).astype(np.float32)
    b = np.real(A.conj().T @ Vs).astype(np.float32)
    x_ref, it_ref, L_ref = lasso.apgd(A, Vs, lam, np.zeros(idx.size), 1e-7, 50_000, positive=True)
    x = torch.zeros(idx.size, dtype=torch.float32, device="cuda")
    x, it, L = abi.pc_apgd(to_dev(G), to_dev(b), lam, 1e-7, 50_000, x, positive=True)
    xg = x.cpu().numpy()
    assert (xg >= 0).all()
    assert abs(L - L_ref) <= 1e-4 * L_ref
    assert rel_l2(xg, x_ref) <= 1e-3
    assert set(np.nonzero(xg)[0]) == set(np.nonzero(x_ref)[0])


def test_pooled_memory_reuse_and_trim(abi):
    """Plans and solves draw device memory from the library's pool: building,
    solving and destroying plans repeatedly gives the same result (support
    identical; weights and objective up to the order of atomic additions), and
    pc_trim_memory returns the cached memory without disturbing a later solve."""
    wl, V = workload("small_wide_w")
    Vd = to_dev(V.astype(np.complex64))
    first = None
    for rep in range(3):
        plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
        lam = 0.05 * abi.pc_lambda_max(plan, Vd)
        res = abi.pc_solve(plan, Vd, lam, wl.delta)
        got = (res["idx"].cpu().numpy().tolist(), res["x"].cpu().numpy(), res["objective"])
        if first is None:
            first = got
        assert got[0] == first[0]
        assert np.allclose(got[1], first[1], rtol=1e-5, atol=0)
        assert abs(got[2] - first[2]) <= 1e-7 * first[2]
        del plan
        if rep == 1:
            abi.pc_trim_memory()
    r = abi.pc_solve_host(wl.uvw, V.astype(np.complex64), wl.N, wl.fov, 0.05, wl.delta)
    assert r["idx"].tolist() == first[0]


def test_resume_from_the_oracle_state_finishes_the_oracle_run(abi):
    """Resume (checkpoint of Algorithm 2; the resume state's reading): started
    from the oracle's support and weights after its iteration j - 1, at
    init_k = j, the GPU solve runs the oracle's remaining iterations (same
    iteration indices, active sets within the borderline pixels) and ends on
    the oracle's final support and objective (1e-4)."""
    wl, V = workload("small_wide_w")
    Vs = V.astype(np.complex64).astype(np.complex128)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, Vs)
    lam = 0.05 * lmax
    ref = pfw.solve(wl.uvw, wl.N, wl.fov, Vs, lam, wl.delta)
    assert len(ref.history) >= 3
    j = 2
    h = ref.history[j - 1]
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    res = abi.pc_solve(plan, to_dev(V.astype(np.complex64)), lam, wl.delta,
                       init_idx=to_dev(h["support"].astype(np.int32)), init_x=to_dev(h["x"].astype(np.float32)),
                       init_k=j)
    assert res["idx"].cpu().numpy().tolist() == ref.idx.tolist()
    assert abs(res["objective"] - ref.objective) <= 1e-4 * ref.objective
    assert res["converged"] and res["iterations"] == ref.iterations
    assert [g["k"] for g in res["history"]] == [o["k"] for o in ref.history[j:]]
    for g, o in zip(res["history"], ref.history[j:]):
        assert abs(g["n_active"] - o["n_active"]) <= o["n_borderline"], (g, o)


def test_warm_start_at_the_solution_stops_after_one_iteration(abi):
    """Started from its own converged (S, x) the solve stops after one
    iteration (relative improvement below the tolerance) on the same support,
    its objective not above the starting one (FP32 rounding aside)."""
    wl, V = workload("tiny_64_coplanar")
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    lam = wl.alpha * abi.pc_lambda_max(plan, Vd)
    cold = abi.pc_solve(plan, Vd, lam, wl.delta)
    warm = abi.pc_solve(plan, Vd, lam, wl.delta, init_idx=cold["idx"].clone(), init_x=cold["x"].clone())
    assert warm["converged"] and len(warm["history"]) == 1
    assert warm["idx"].cpu().tolist() == cold["idx"].cpu().tolist()
    assert warm["objective"] <= cold["objective"] * (1 + 1e-5)


def test_resume_state_is_checked(abi):
    """An invalid resume state is an argument error (checked before the first
    iteration): pixels not strictly ascending or outside the image, a
    non-finite weight, a negative weight under positivity, init_k outside
    [0, max_fw)."""
    wl, V = workload("tiny_64_coplanar")
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    Vd = to_dev(V.astype(np.complex64))
    lam = wl.alpha * abi.pc_lambda_max(plan, Vd)
    NN = wl.N * wl.N
    bad = [(np.array([5, 3], np.int32), np.array([1.0, 1.0], np.float32), {}),
           (np.array([3, 3], np.int32), np.array([1.0, 1.0], np.float32), {}),
           (np.array([3, NN], np.int32), np.array([1.0, 1.0], np.float32), {}),
           (np.array([3, 5], np.int32), np.array([1.0, np.inf], np.float32), {}),
           (np.array([3, 5], np.int32), np.array([1.0, -1.0], np.float32), {"positivity": 1}),
           (np.array([3, 5], np.int32), np.array([1.0, 1.0], np.float32), {"init_k": 100})]
    for idx, x, kw in bad:
        with pytest.raises(abi.PcError) as e:
            abi.pc_solve(plan, Vd, lam, wl.delta, init_idx=to_dev(idx), init_x=to_dev(x), **kw)
        assert e.value.status == abi.PC_ERR_INVALID_ARG, (idx, x, kw)
    # the plan is still usable
    assert abi.pc_solve(plan, Vd, lam, wl.delta)["converged"]
