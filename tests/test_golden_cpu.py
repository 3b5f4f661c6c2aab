"""The stored FP64 oracle solve of the 512 x 512, M = 200k workload
(tests/golden/medium_512_w_solve.json) against what the paper fixes, on the
CPU: it was written by the committed script as it stands, it converged, its
objective never increased over the Frank-Wolfe iterations (Algorithm 2), and
its final certificate satisfies the optimality conditions of Sect. 4.2 on the
stored pixels (|mu| <= 1 up to the early-stopped reweighting, mu = sign(x) on
the support). The GPU parity tests (tests/test_gpu_golden.py) compare the
CUDA path with it."""
import hashlib
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "medium_512_w_solve.json")
SCRIPT = os.path.join(HERE, "golden", "make_medium_512_solve.py")


def _golden():
    return json.load(open(GOLDEN))


def test_golden_was_written_by_the_committed_script():
    g = _golden()
    assert g["script_sha256"] == hashlib.sha256(open(SCRIPT, "rb").read()).hexdigest()
    assert g["workload"] == "medium_512_w" and g["N"] == 512 and g["M"] == 200_000


def test_golden_is_a_converged_oracle_solve():
    g = _golden()
    assert g["converged"] and g["iterations"] == len(g["history"])
    F = [0.5 * g["V_sumsq"]] + [h["objective"] for h in g["history"]]
    assert all(b <= a for a, b in zip(F, F[1:]))
    assert abs(g["lambda"] - g["alpha"] * g["lambda_max"]) <= 1e-12 * g["lambda"]
    # every support is inside that iteration's active set, the last is the result
    for h in g["history"]:
        assert set(h["support"]) <= set(h["active"])
        assert len(h["active"]) == h["n_active"] and len(h["support"]) == h["n_support"]
    assert g["history"][-1]["support"] == g["support"]


def test_golden_certificate_meets_the_optimality_conditions():
    g = _golden()
    pix = np.array(g["mu_pixels"])
    mu = np.array(g["mu"])
    S = np.array(g["support"])
    x = np.array(g["x"])
    on = np.searchsorted(pix, S)
    assert np.array_equal(pix[on], S)                  # the support is among the stored pixels
    assert np.all(np.sign(mu[on]) == np.sign(x))
    assert np.abs(np.abs(mu[on]) - 1.0).max() <= 1e-2
    assert g["mu_inf"] <= 1.0 + 1e-2
    assert np.abs(mu).max() <= g["mu_inf"] + 1e-12
