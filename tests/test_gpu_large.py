"""GPU parity at the full sizes of the 2048 x 2048 (M = 2M, ~17 w-planes) and
4096 x 4096 (M = 10M) configurations: the operators on seeded samples of
pixels and visibilities that the FP64 oracle computes one by one, and
invariants of the full solve that hold at any size (the oracle cannot solve
these sizes).

The adjoint is checked on seeded white-noise visibilities (no method
arithmetic involved in the input), the forward on a seeded random support.
"""
import numpy as np
import pytest

from oracle import operators
from paper_2406_01342_gb300 import synth
from tests.helpers import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


@pytest.mark.parametrize("name,n_pix", [("large_2048_w", 40), ("fine_4096_w", 16)])
def test_operators_full_size_sampled(abi, name, n_pix):
    wl = synth.WORKLOADS[name]()
    assert wl.M in (2_000_000, 10_000_000)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    info = abi.pc_plan_info(plan)
    assert info["n_planes"] > 8                      # several plane groups per tile
    rng = np.random.default_rng(31)
    V = synth.unit_complex_noise(wl.M, rng).astype(np.complex64)
    img = abi.pc_adjoint_grid(plan, to_dev(V)).cpu().numpy().ravel()
    N = wl.N
    corners = np.array([0, N - 1, (N - 1) * N, N * N - 1, (N // 2) * N + N // 2])
    pix = np.union1d(np.sort(rng.choice(N * N, n_pix, replace=False)), corners)
    ref = operators.adjoint(wl.uvw, N, wl.fov, V.astype(np.complex128), pix)
    assert rel_l2(img[pix], ref) <= TOL
    # forward on a random 300-atom support, sampled visibilities
    idx = np.sort(rng.choice(N * N, 300, replace=False)).astype(np.int32)
    x = rng.uniform(-1.0, 2.0, 300).astype(np.float32)
    y = abi.pc_forward_sparse(plan, to_dev(idx), to_dev(x)).cpu().numpy()
    ks = np.sort(rng.choice(wl.M, 4000, replace=False))
    yref = operators.forward(wl.uvw[ks], N, wl.fov, idx, x.astype(np.float64))
    assert rel_l2(y[ks], yref) <= TOL


def _physical_vis(abi, plan, wl):
    """Noisy visibilities of the workload's sky, formed with the GPU forward
    operator (no oracle value is involved in these solve tests)."""
    y = abi.pc_forward_sparse(plan, to_dev(wl.sky_idx.astype(np.int32)),
                              to_dev(wl.sky_flux.astype(np.float32)))
    p_sig = float((y.abs() ** 2).mean())
    sigma = np.sqrt(p_sig * 10.0 ** (-wl.snr_db / 10.0))
    return y + to_dev((sigma * wl.noise).astype(np.complex64))


@pytest.mark.parametrize("name", ["large_2048_w", "fine_4096_w"])
def test_full_size_solve_invariants(abi, name):
    """Algorithm 2 at full size: converges at the 1e-4 stop rule, the objective
    never increases and ends below F(0) = ||V||^2 / 2, the certificate of the
    returned image is ~1 in magnitude on its support (optimality, Sect. 4.2)
    and the brightest true sources are in the support."""
    wl = synth.WORKLOADS[name]()
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    V = _physical_vis(abi, plan, wl)
    lam = wl.alpha * abi.pc_lambda_max(plan, V)
    res = abi.pc_solve(plan, V, lam, wl.delta)
    assert res["converged"]
    F = [0.5 * res["sumsq_V"]] + [h["objective"] for h in res["history"]]
    assert all(b <= a * (1 + 1e-7) for a, b in zip(F, F[1:]))
    assert res["objective"] < 0.5 * res["sumsq_V"]
    idx = res["idx"].cpu().numpy()
    x = res["x"].cpu().numpy()
    assert idx.size > 0 and np.isfinite(x).all() and (np.diff(idx) > 0).all()
    mu = res["mu"].cpu().numpy().ravel()
    assert np.abs(np.abs(mu[idx]) - 1.0).max() <= 0.05
    assert np.all(np.sign(mu[idx]) == np.sign(x))
    bright = wl.sky_idx[np.argsort(wl.sky_flux)[-10:]]
    assert np.isin(bright, idx).all()
