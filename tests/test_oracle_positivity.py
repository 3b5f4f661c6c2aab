"""Pins of the oracle's positivity-constrained variant (the remarks on a
positivity constraint in Sect. 4.1 and 5.1: candidates only at positive values
of the residual image, reweighting with x >= 0), against what the mathematics
fixes independently of the oracle: exhaustive enumeration over {0, +1}^n
patterns, a separately written coordinate descent, the one-sided optimality
conditions and the positive lambda_max.
"""
import math

import numpy as np
import pytest

from oracle import lasso, operators, pfw
from paper_2406_01342_gb300 import synth


def _random_uvw(rng, M, umax, wmax):
    u = rng.uniform(-umax, umax, M)
    v = rng.uniform(-umax, umax, M)
    w = rng.uniform(-wmax, wmax, M)
    return np.stack([u, v, w], axis=1)


def _signed_tiny_problem(seed, N=3, M=12, fov_deg=40.0, wmax=3.0):
    """3 x 3 sky with one positive and one negative source (so the constrained
    and unconstrained minimisers differ)."""
    rng = np.random.default_rng(seed)
    fov = math.radians(fov_deg)
    uvw = _random_uvw(rng, M, 3.0, wmax)
    idx = np.arange(N * N)
    x_true = np.zeros(N * N)
    p, q = rng.choice(N * N, 2, replace=False)
    x_true[p] = rng.uniform(1, 3)
    x_true[q] = -rng.uniform(1, 3)
    V = operators.forward(uvw, N, fov, idx, x_true)
    V = V + 0.05 * np.abs(V).mean() * (rng.normal(size=M) + 1j * rng.normal(size=M))
    return uvw, N, fov, V


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_positive_pfw_matches_brute_force_on_3x3(seed):
    """Exact non-negative LASSO by enumerating all 2^9 supports, an independent
    positive coordinate descent and the positive PFW agree; the unconstrained
    minimiser of the same data has a negative entry (the constraint is active)."""
    uvw, N, fov, V = _signed_tiny_problem(seed)
    lmax_pos = operators.lambda_max_positive(uvw, N, fov, V)
    lam = 0.15 * lmax_pos
    l, m, n = operators.pixel_lmn(N, fov, np.arange(N * N))
    A = operators.phase_block(uvw, l, m, n)
    x_bf = lasso.brute_force(A, V, lam, positive=True)
    x_cd = lasso.coordinate_descent(A, V, lam, positive=True)
    res = pfw.solve(uvw, N, fov, V, lam, delta=0.01, tol=1e-13, eps0=1e-13, eps_min=1e-13,
                    apgd_max_iter=200_000, positive=True)
    x_pfw = np.zeros(N * N)
    x_pfw[res.idx] = res.x
    scale = np.abs(x_bf).max()
    assert np.count_nonzero(x_bf) >= 1 and (x_bf >= 0).all()
    assert np.allclose(x_cd, x_bf, atol=1e-8 * scale)
    assert np.allclose(x_pfw, x_bf, atol=1e-7 * scale)
    assert (res.x > 0).all()
    assert set(res.idx.tolist()) == set(np.nonzero(x_bf)[0].tolist())
    x_free = lasso.brute_force(A, V, lam)
    assert x_free.min() < 0.0


def test_positive_select_rules():
    """R2 positive keeps mu >= 1 - delta only (never a negative pixel); R1 positive
    with delta = 1 keeps exactly the positive argmax."""
    eta = np.array([-5.0, 0.2, 3.0, -3.5, 2.99, 0.0])
    assert pfw.select_r2(eta / 3.0, 0.01, positive=True).tolist() == [2, 4]
    assert pfw.select_r2(eta / 3.0, 0.01).tolist() == [0, 2, 3, 4]
    assert pfw.select_r1(eta, 0, 0.0, positive=True).tolist() == [2]
    assert pfw.select_r1(eta, 0, 0.0).tolist() == [0]


@pytest.fixture(scope="module")
def tight_positive():
    wl = synth.tiny_coplanar()
    V = operators.forward(wl.uvw, wl.N, wl.fov, wl.sky_idx, wl.sky_flux) + wl.noise
    lmax_pos = operators.lambda_max_positive(wl.uvw, wl.N, wl.fov, V)
    lam = wl.alpha * lmax_pos
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, wl.delta, tol=1e-12, eps0=1e-12, eps_min=1e-12,
                    apgd_max_iter=100_000, positive=True)
    return wl, V, lmax_pos, lam, res


def test_positive_kkt_conditions_at_convergence(tight_positive):
    """One-sided optimality: max mu <= 1 on the grid, mu = 1 on the support,
    x > 0, and the duality gap with the dual constraint Phi* theta <= lambda vanishes."""
    wl, V, lmax_pos, lam, res = tight_positive
    mu = res.mu.ravel()
    assert mu.max() <= 1 + 1e-6
    assert (res.x > 0).all()
    assert np.allclose(mu[res.idx], 1.0, atol=1e-6)
    gap = pfw.duality_gap(wl.uvw, wl.N, wl.fov, V, lam, res.idx, res.x, positive=True)
    assert -1e-9 * res.objective <= gap <= 1e-8 * res.objective


def test_positive_lambda_max_gives_zero():
    """With a dominant negative source ||Phi* V||_inf > max Phi* V; at
    lambda >= max(Phi* V) the non-negative solution is exactly 0, just below it is not."""
    wl = synth.tiny_coplanar(M=400, N=32)
    flux = wl.sky_flux.copy()
    flux[0] = -3.0 * np.abs(flux).max()
    V = operators.forward(wl.uvw, wl.N, wl.fov, wl.sky_idx, flux)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V)
    lmax_pos = operators.lambda_max_positive(wl.uvw, wl.N, wl.fov, V)
    assert lmax_pos < lmax
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lmax_pos * (1 + 1e-9), delta=0.01, positive=True)
    assert res.idx.size == 0 and res.objective == 0.5 * float(np.vdot(V, V).real)
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lmax_pos * 0.95, delta=0.01, positive=True)
    assert res.idx.size >= 1 and (res.x > 0).all()


def test_positive_solve_monotone_and_close_to_tight(tight_positive):
    """Default stopping rule: monotone objective, within 1e-4 of the tight optimum."""
    wl, V, lmax_pos, lam, tight = tight_positive
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, wl.delta, positive=True)
    F = [0.5 * float(np.vdot(V, V).real)] + [h["objective"] for h in res.history]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(F, F[1:]))
    assert abs(res.objective - tight.objective) <= 1e-4 * tight.objective
