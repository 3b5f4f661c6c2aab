"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

Each test checks the oracle against something other than its own formula:
an identity (adjoint pair), a library routine in a special case (numpy.fft on
the uv lattice), a closed form (single atom, lambda_max), an independent
solver (brute force over sign patterns, coordinate descent) or an optimality
condition of the LASSO (Sect. 4.2: |mu| <= 1, mu = sign(x) on the support).
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


def _vis(wl):
    Vc = operators.forward(wl.uvw, wl.N, wl.fov, wl.sky_idx, wl.sky_flux)
    sig = synth.noise_sigma(float(np.mean(np.abs(Vc) ** 2)), wl.snr_db)
    return Vc + sig * wl.noise


# ------------------------------------------------------------ operators (Sect. 2.2)

def test_adjoint_identity_wide_field():
    """Re<Phi x, y> == <x, Phi* y> (the adjoint equation of Sect. 2.2) with w != 0."""
    rng = np.random.default_rng(1)
    N, fov = 12, math.radians(30.0)
    uvw = _random_uvw(rng, 37, 40.0, 25.0)
    idx = np.arange(N * N)
    x = rng.normal(size=N * N)
    y = rng.normal(size=37) + 1j * rng.normal(size=37)
    lhs = np.real(np.vdot(y, operators.forward(uvw, N, fov, idx, x)))
    rhs = float(x @ operators.adjoint(uvw, N, fov, y))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def _lattice_case(N=16, fov=math.radians(40.0), M=60, seed=2):
    rng = np.random.default_rng(seed)
    dl = fov / N
    a = rng.integers(-N // 2, N // 2, M)
    b = rng.integers(-N // 2, N // 2, M)
    uvw = np.stack([a / (N * dl), b / (N * dl), np.zeros(M)], axis=1)
    return rng, N, fov, a, b, uvw


def test_lattice_adjoint_is_inverse_fft():
    """w = 0 and (u, v) on the lattice 1/(N dl): Phi* is a 2-D inverse DFT times 1/n."""
    rng, N, fov, a, b, uvw = _lattice_case()
    h = rng.normal(size=a.size) + 1j * rng.normal(size=a.size)
    H = np.zeros((N, N), dtype=complex)
    np.add.at(H, (a % N, b % N), h)
    ref = np.fft.fftshift(np.real(N * N * np.fft.ifft2(H)))
    _, _, n = operators.pixel_lmn(N, fov, np.arange(N * N))
    got = operators.adjoint(uvw, N, fov, h).reshape(N, N) * n.reshape(N, N)
    assert np.allclose(got, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    # n is far from 1 at this field of view, so a dropped 1/n cannot pass
    assert n.min() < 0.97


def test_lattice_forward_is_fft():
    """w = 0 lattice: Phi x = 2-D DFT of x / n sampled at (a, b)."""
    rng, N, fov, a, b, uvw = _lattice_case(seed=3)
    x = rng.normal(size=N * N)
    _, _, n = operators.pixel_lmn(N, fov, np.arange(N * N))
    F = np.fft.fft2(np.fft.ifftshift((x / n).reshape(N, N)))
    ref = F[a % N, b % N]
    got = operators.forward(uvw, N, fov, np.arange(N * N), x)
    assert np.allclose(got, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_point_source_dirty_image_is_shifted_psf_coplanar():
    """Van Cittert-Zernike case (w = 0, Sect. 2.1 remark): n_p n_q Phi*Phi delta_p [q] is the
    PSF sum_k cos(2 pi (u_k dl_pq + v_k dm_pq)), a function of the offset q - p only."""
    rng = np.random.default_rng(4)
    N, fov = 16, math.radians(30.0)
    uvw = _random_uvw(rng, 50, 30.0, 0.0)
    p = 3 * N + 5
    l, m, n = operators.pixel_lmn(N, fov, np.arange(N * N))
    img = operators.adjoint(uvw, N, fov, operators.forward(uvw, N, fov, [p], [1.0]))
    psf = np.cos(2 * np.pi * (np.outer(uvw[:, 0], l - l[p]) + np.outer(uvw[:, 1], m - m[p]))).sum(0)
    assert np.allclose(img * n * n[p], psf, atol=1e-10 * np.abs(psf).max())


def test_point_source_not_shift_invariant_with_w():
    """With w != 0 the same product differs from the shifted PSF (the w-term, Sect. 2.1)."""
    rng = np.random.default_rng(5)
    N, fov = 16, math.radians(30.0)
    uvw = _random_uvw(rng, 50, 30.0, 30.0)
    p = 3 * N + 5
    l, m, n = operators.pixel_lmn(N, fov, np.arange(N * N))
    img = operators.adjoint(uvw, N, fov, operators.forward(uvw, N, fov, [p], [1.0]))
    psf = np.cos(2 * np.pi * (np.outer(uvw[:, 0], l - l[p]) + np.outer(uvw[:, 1], m - m[p]))).sum(0)
    assert np.max(np.abs(img * n * n[p] - psf)) > 1e-2 * np.abs(psf).max()
    assert abs(img[p] * n[p] ** 2 - uvw.shape[0]) < 1e-9 * uvw.shape[0]   # zero offset is still M


def test_phase_reduction_keeps_large_arguments_exact():
    """The turn reduction must not change the operator: compare with an unreduced
    exponential at small baselines where the unreduced argument is exact enough."""
    rng = np.random.default_rng(6)
    N, fov = 8, math.radians(10.0)
    uvw = _random_uvw(rng, 20, 5.0, 5.0)
    idx = np.arange(N * N)
    x = rng.normal(size=N * N)
    l, m, n = operators.pixel_lmn(N, fov, idx)
    direct = np.exp(-2j * np.pi * (np.outer(uvw[:, 0], l) + np.outer(uvw[:, 1], m)
                                   + np.outer(uvw[:, 2], n - 1))) @ (x / n)
    assert np.allclose(operators.forward(uvw, N, fov, idx, x), direct, atol=1e-12 * np.abs(direct).max())


# ------------------------------------------------------------ LASSO facts (Sect. 4, 5.3)

def test_single_atom_closed_form():
    """One atom a: argmin 1/2||V - a x||^2 + lam|x| = soft(Re(a^H V), lam) / ||a||^2."""
    rng = np.random.default_rng(7)
    a = (rng.normal(size=(30, 1)) + 1j * rng.normal(size=(30, 1)))
    V = rng.normal(size=30) + 1j * rng.normal(size=30)
    c = float(np.real(np.vdot(a[:, 0], V)))
    for lam in (0.3 * abs(c), 0.9 * abs(c), 1.2 * abs(c)):
        ref = np.sign(c) * max(abs(c) - lam, 0.0) / float(np.sum(np.abs(a) ** 2))
        x, _, _ = lasso.apgd(a, V, lam, np.zeros(1), 1e-14, 100_000)
        assert abs(x[0] - ref) <= 1e-10 * max(1.0, abs(ref))


def test_lipschitz_is_top_eigenvalue():
    """The step-size constant is 1.01 x the top eigenvalue of Re(A^H A), checked
    against the power method (an independent computation) and the Rayleigh bound."""
    rng = np.random.default_rng(8)
    A = rng.normal(size=(40, 7)) + 1j * rng.normal(size=(40, 7))
    v = np.ones(7)
    for _ in range(2000):
        v = lasso.gram_apply(A, v)
        v /= np.linalg.norm(v)
    ev = float(v @ lasso.gram_apply(A, v))
    L = lasso.lipschitz(A)
    assert abs(L - 1.01 * ev) <= 1e-9 * ev
    x = rng.normal(size=7)
    assert float(x @ lasso.gram_apply(A, x)) <= L / 1.01 * float(x @ x) * (1 + 1e-12)


def _tiny_problem(seed, N=3, M=12, fov_deg=40.0, wmax=3.0):
    rng = np.random.default_rng(seed)
    fov = math.radians(fov_deg)
    uvw = _random_uvw(rng, M, 3.0, wmax)
    idx = np.arange(N * N)
    x_true = np.zeros(N * N)
    x_true[rng.choice(N * N, 2, replace=False)] = rng.uniform(1, 3, 2)
    V = operators.forward(uvw, N, fov, idx, x_true)
    V = V + 0.05 * np.abs(V).mean() * (rng.normal(size=M) + 1j * rng.normal(size=M))
    return uvw, N, fov, V


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_pfw_matches_brute_force_on_3x3(seed):
    """Tiny grids: the PFW solution equals the exact LASSO minimiser found by
    enumerating all 3^9 sign patterns, and an independent coordinate descent."""
    uvw, N, fov, V = _tiny_problem(seed)
    lmax = operators.lambda_max(uvw, N, fov, V)
    lam = 0.15 * lmax
    l, m, n = operators.pixel_lmn(N, fov, np.arange(N * N))
    A = operators.phase_block(uvw, l, m, n)
    x_bf = lasso.brute_force(A, V, lam)
    x_cd = lasso.coordinate_descent(A, V, lam)
    res = pfw.solve(uvw, N, fov, V, lam, delta=0.01, tol=1e-13, eps0=1e-13, eps_min=1e-13,
                    apgd_max_iter=200_000)
    x_pfw = np.zeros(N * N)
    x_pfw[res.idx] = res.x
    scale = np.abs(x_bf).max()
    assert np.count_nonzero(x_bf) >= 1
    assert np.allclose(x_cd, x_bf, atol=1e-8 * scale)
    assert np.allclose(x_pfw, x_bf, atol=1e-7 * scale)
    assert set(res.idx.tolist()) == set(np.nonzero(x_bf)[0].tolist())


def test_lambda_at_lambda_max_gives_zero():
    """Sect. 5.3: for lambda >= lambda_max = ||Phi* V||_inf the solution is exactly 0."""
    wl = synth.tiny_coplanar(M=400, N=32)
    V = _vis(wl)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V)
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lmax * (1 + 1e-9), delta=0.01)
    assert res.idx.size == 0 and res.objective == 0.5 * float(np.vdot(V, V).real)
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lmax * 0.95, delta=0.01)
    assert res.idx.size >= 1


@pytest.fixture(scope="module")
def tight_tiny():
    wl = synth.tiny_coplanar()
    V = _vis(wl)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V)
    lam = wl.alpha * lmax
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, wl.delta, tol=1e-12, eps0=1e-12, eps_min=1e-12,
                    apgd_max_iter=100_000)
    return wl, V, lmax, lam, res


def test_kkt_conditions_at_convergence(tight_tiny):
    """Sect. 4.2: ||mu||_inf <= 1 and mu = sign(x) on the support; the duality gap vanishes."""
    wl, V, lmax, lam, res = tight_tiny
    mu = res.mu.ravel()
    assert np.abs(mu).max() <= 1 + 1e-6
    assert np.allclose(mu[res.idx], np.sign(res.x), atol=1e-6)
    gap = pfw.duality_gap(wl.uvw, wl.N, wl.fov, V, lam, res.idx, res.x)
    assert -1e-9 * res.objective <= gap <= 1e-8 * res.objective


def test_alpha_identity(tight_tiny):
    """Sect. 5.3: at convergence ||Phi*(V - Phi x)||_inf / ||Phi* V||_inf = alpha."""
    wl, V, lmax, lam, res = tight_tiny
    ratio = np.abs(res.mu).max() * lam / lmax
    assert abs(ratio - wl.alpha) <= 1e-6 * wl.alpha


def test_default_solve_is_monotone_and_close_to_tight(tight_tiny):
    """The objective never increases over Frank-Wolfe iterations, and the default
    stopping rule (1e-4 relative improvement) lands within 1e-4 of the tight optimum."""
    wl, V, lmax, lam, tight = tight_tiny
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, wl.delta)
    F = [0.5 * float(np.vdot(V, V).real)] + [h["objective"] for h in res.history]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(F, F[1:]))
    assert abs(res.objective - tight.objective) <= 1e-4 * tight.objective
    assert res.converged


def test_rule_r1_classic_fw_and_same_optimum(tight_tiny):
    """R1 with delta = 1 adds only the argmax (classic Frank-Wolfe); R1 and R2 reach
    the same LASSO optimum."""
    wl, V, lmax, lam, tight = tight_tiny
    eta = operators.adjoint(wl.uvw, wl.N, wl.fov, V)
    sel = pfw.select_r1(eta, 0, 0.0)
    assert sel.tolist() == [int(np.argmax(np.abs(eta)))]
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, delta=0.9, rule="R1", tol=1e-12, eps0=1e-12,
                    eps_min=1e-12, apgd_max_iter=100_000)
    assert abs(res.objective - tight.objective) <= 1e-9 * tight.objective
    assert res.idx.tolist() == tight.idx.tolist()


def test_wide_field_solve_invariants():
    """Wide-field case (w-term on): monotone objective and |mu| <= 1 + eps at stop."""
    wl = synth.small_wide_field()
    V = _vis(wl)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V)
    res = pfw.solve(wl.uvw, wl.N, wl.fov, V, 0.05 * lmax, wl.delta, tol=1e-10, eps0=1e-10, eps_min=1e-10,
                    apgd_max_iter=100_000)
    F = [0.5 * float(np.vdot(V, V).real)] + [h["objective"] for h in res.history]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(F, F[1:]))
    assert np.abs(res.mu).max() <= 1 + 1e-5
    assert np.allclose(res.mu.ravel()[res.idx], np.sign(res.x), atol=1e-5)


@pytest.mark.parametrize("rule,delta", [("R2", None), ("R1", 0.9)])
def test_resume_from_a_saved_state_repeats_the_rest_of_the_run(rule, delta):
    """Checkpoint / resume: the state of Algorithm 2 at the start of iteration
    j is (j, S_j, I_j). A solve resumed from the state an uninterrupted run
    recorded at the end of its iteration j - 1 repeats that run's iterations
    j, j + 1, ... (same active sets and supports, same objectives, same stop),
    for both selection rules (R1's threshold and the eps_k schedule depend on
    k). A resume that got the iteration index, the first stop test's F or the
    residual of the saved image wrong would leave the recorded path."""
    wl = synth.tiny_coplanar()
    V = _vis(wl)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V)
    lam = wl.alpha * lmax
    d = wl.delta if delta is None else delta
    cold = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, d, rule=rule, lmax=lmax)
    assert len(cold.history) >= 4
    j = 2
    h = cold.history[j - 1]
    warm = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, d, rule=rule, lmax=lmax, S0=h["support"], x0=h["x"], k0=j)
    assert len(warm.history) == len(cold.history) - j
    for a, b in zip(cold.history[j:], warm.history):
        assert a["k"] == b["k"]
        assert a["active"].tolist() == b["active"].tolist()
        assert a["support"].tolist() == b["support"].tolist()
        assert b["objective"] == pytest.approx(a["objective"], rel=1e-12)
        assert b["rel_improvement"] == pytest.approx(a["rel_improvement"], rel=1e-9, abs=1e-15)
        assert b["apgd_iterations"] == a["apgd_iterations"] and b["eps"] == a["eps"]
    assert warm.idx.tolist() == cold.idx.tolist() and warm.converged == cold.converged
    assert warm.iterations == cold.iterations
    assert warm.objective == pytest.approx(cold.objective, rel=1e-12)


def test_warm_start_at_the_solution_stops_after_one_iteration():
    """Started from a converged solve's (S, x), the first iteration's relative
    improvement is below the tolerance: the solve stops there with the same
    support, and its objective is not above the starting one."""
    wl = synth.tiny_coplanar()
    V = _vis(wl)
    lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, V)
    lam = wl.alpha * lmax
    cold = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, wl.delta)
    warm = pfw.solve(wl.uvw, wl.N, wl.fov, V, lam, wl.delta, S0=cold.idx, x0=cold.x)
    assert warm.converged and len(warm.history) == 1
    assert warm.idx.tolist() == cold.idx.tolist()
    assert warm.objective <= cold.objective * (1 + 1e-12)
