"""Pins of the synthesis-dictionary oracle (Sect. 4.3 and the diffuse
experiment of Sect. 6) to facts other than its own formulas: the kernel's
closed form and unit l1 norm, scipy's 2-D convolution and correlation for Psi
and Psi*, the adjoint identities, the reduction of a one-scale sigma = 0
dictionary to the pixel problem, lambda_max, an independent coordinate-descent
LASSO on a tiny grid and the optimality conditions of Sect. 4.2."""
import math

import numpy as np
import pytest

from oracle import dictionary, lasso, operators, pfw

signal = pytest.importorskip("scipy.signal")


def _uvw(rng, M, umax, wmax):
    return np.stack([rng.uniform(-umax, umax, M), rng.uniform(-umax, umax, M),
                     rng.uniform(-wmax, wmax, M)], axis=1)


def test_kernel_closed_form():
    assert dictionary.kernel(0.0).tolist() == [[1.0]]
    for s in (2.0, 5.0, 8.0, 1.3):
        g = dictionary.kernel(s)
        K = int(math.floor(2 * s))
        assert g.shape == (2 * K + 1, 2 * K + 1)
        assert abs(g.sum() - 1.0) <= 1e-14 and np.all(g > 0)
        c = g[K, K]
        # g[n, m] / g[0, 0] = exp(-(n^2 + m^2) / sigma^2)
        assert g[K, K + 1] / c == pytest.approx(math.exp(-1.0 / s ** 2), rel=1e-14)
        assert g[0, 2 * K] / c == pytest.approx(math.exp(-2.0 * K * K / s ** 2), rel=1e-12)
        assert np.array_equal(g, g.T) and np.array_equal(g, g[::-1, :])


def test_synthesis_is_scipy_same_convolution():
    d = dictionary.Dictionary(24)
    rng = np.random.default_rng(11)
    theta = rng.normal(size=d.n_atoms) * (rng.random(d.n_atoms) < 0.05)
    img = dictionary.synthesize(d, theta).reshape(24, 24)
    ref = sum(gm * signal.convolve2d(th, g, mode="same")
              for th, g, gm in zip(theta.reshape(4, 24, 24), d.kernels(), d.gammas))
    assert np.allclose(img, ref, rtol=0, atol=1e-13)


def test_analysis_is_scipy_same_correlation_and_adjoint():
    d = dictionary.Dictionary(20, sigmas=(0.0, 1.5, 3.0), gammas=(1.0, 0.7, 2.0))
    rng = np.random.default_rng(12)
    z = rng.normal(size=400)
    out = dictionary.analyze(d, z).reshape(3, 20, 20)
    for i, (g, gm) in enumerate(zip(d.kernels(), d.gammas)):
        assert np.allclose(out[i], gm * signal.correlate2d(z.reshape(20, 20), g, mode="same"),
                           rtol=0, atol=1e-13)
    theta = rng.normal(size=d.n_atoms)
    lhs = float(dictionary.synthesize(d, theta) @ z)
    rhs = float(theta @ dictionary.analyze(d, z))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_single_atom_image_and_border_crop():
    N = 40
    d = dictionary.Dictionary(N)
    for i, (x0, y0) in [(1, (20, 21)), (2, (19, 5)), (3, (0, 0)), (0, (39, 17))]:
        a = i * N * N + x0 * N + y0
        e = np.zeros(d.n_atoms)
        e[a] = 1.0
        img = dictionary.synthesize(d, e).reshape(N, N)
        g = dictionary.kernel(d.sigmas[i]) * d.gammas[i]
        K = g.shape[0] // 2
        big = np.zeros((N + 2 * K, N + 2 * K))
        big[x0:x0 + 2 * K + 1, y0:y0 + 2 * K + 1] = g
        assert np.array_equal(img, big[K:K + N, K:K + N])
        inside = K <= x0 < N - K and K <= y0 < N - K
        assert (abs(img.sum() - d.gammas[i]) <= 1e-13) == inside   # no renormalisation at the border
        pix, w = dictionary.atom_pixels(d, a)
        assert np.array_equal(np.sort(pix), np.nonzero(img.ravel())[0])
        assert np.allclose(img.ravel()[pix], w, rtol=0, atol=0)


def test_composite_operator_adjoint_and_columns():
    rng = np.random.default_rng(13)
    N, fov = 16, math.radians(20.0)
    uvw = _uvw(rng, 41, 20.0, 10.0)
    d = dictionary.Dictionary(N)
    atoms = np.sort(rng.choice(d.n_atoms, 30, replace=False))
    theta = rng.normal(size=30)
    y = dictionary.forward(uvw, fov, d, atoms, theta)
    A = dictionary.columns(uvw, fov, d, atoms)
    assert np.allclose(A @ theta, y, rtol=0, atol=1e-12 * np.abs(y).max())
    h = rng.normal(size=41) + 1j * rng.normal(size=41)
    full = np.zeros(d.n_atoms)
    full[atoms] = theta
    lhs = float(np.real(np.vdot(h, y)))
    rhs = float(full @ dictionary.adjoint(uvw, fov, d, h))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
    # a sigma = 0 atom is the pixel's column of Phi
    a0 = atoms[0] % (N * N)
    ref = operators.forward(uvw, N, fov, [a0], [1.0])
    assert np.allclose(dictionary.columns(uvw, fov, d, [a0])[:, 0], ref, rtol=0, atol=1e-15)


def _small_problem(seed, N=16, M=120):
    rng = np.random.default_rng(seed)
    fov = math.radians(10.0)
    uvw = _uvw(rng, M, 0.6 / (fov / N) / 2, 5.0)
    d = dictionary.Dictionary(N)
    atoms = np.array([2 * N * N + 8 * N + 7, 1 * N * N + 3 * N + 12, 5 * N + 5])
    theta = np.array([2.0, 1.0, 0.5])
    V = dictionary.forward(uvw, fov, d, atoms, theta)
    V = V + 0.01 * np.abs(V).max() * (rng.normal(size=M) + 1j * rng.normal(size=M))
    return uvw, fov, d, V, atoms


def test_one_scale_point_dictionary_is_the_pixel_problem():
    rng = np.random.default_rng(14)
    N, fov = 12, math.radians(8.0)
    uvw = _uvw(rng, 90, 0.5 / (fov / N), 3.0)
    V = operators.forward(uvw, N, fov, [30, 77], [3.0, -1.5]) + 0.05 * (rng.normal(size=90) + 0j)
    d = dictionary.Dictionary(N, sigmas=(0.0,), gammas=(1.0,))
    lam = 0.2 * dictionary.lambda_max(uvw, fov, d, V)
    assert dictionary.lambda_max(uvw, fov, d, V) == pytest.approx(operators.lambda_max(uvw, N, fov, V),
                                                                  rel=1e-14)
    a = dictionary.solve(uvw, fov, d, V, lam, tol=1e-4)
    b = pfw.solve(uvw, N, fov, V, lam, tol=1e-4)
    assert a.idx.tolist() == b.idx.tolist()
    assert a.objective == pytest.approx(b.objective, rel=1e-12)


def test_lambda_max_gives_zero_and_below_it_does_not():
    uvw, fov, d, V, _ = _small_problem(15)
    lmax = dictionary.lambda_max(uvw, fov, d, V)
    r = dictionary.solve(uvw, fov, d, V, lmax * (1 + 1e-9), max_fw=3)
    assert r.idx.size == 0 and r.objective == pytest.approx(0.5 * float(np.vdot(V, V).real))
    r = dictionary.solve(uvw, fov, d, V, 0.9 * lmax, max_fw=3)
    assert r.idx.size > 0


def test_solve_matches_coordinate_descent_and_optimality():
    """Tiny grid (8 x 8, 4 scales = 256 atoms): the PFW solve reaches the
    objective of an independent coordinate-descent LASSO on the full
    dictionary, and its certificate satisfies |eta| <= 1 with eta = sign(theta)
    on the support (Sect. 4.2)."""
    rng = np.random.default_rng(16)
    N, fov, M = 8, math.radians(6.0), 60
    uvw = _uvw(rng, M, 0.5 / (fov / N), 2.0)
    d = dictionary.Dictionary(N, sigmas=(0.0, 1.0, 1.5, 2.0))
    V = dictionary.forward(uvw, fov, d, [1 * 64 + 27, 3 * 64 + 36], [1.5, 1.0])
    V = V + 0.02 * np.abs(V).max() * (rng.normal(size=M) + 1j * rng.normal(size=M))
    lam = 0.05 * dictionary.lambda_max(uvw, fov, d, V)
    r = dictionary.solve(uvw, fov, d, V, lam, tol=1e-10, eps_min=1e-12, max_fw=200,
                         apgd_max_iter=200_000)
    A = dictionary.columns(uvw, fov, d, np.arange(d.n_atoms))
    x_cd = lasso.coordinate_descent(A, V, lam)
    f_cd = lasso.objective(A, V, lam, x_cd)
    assert r.objective == pytest.approx(f_cd, rel=1e-7)
    eta = r.eta.ravel()
    assert np.max(np.abs(eta)) <= 1 + 1e-4
    assert np.allclose(eta[r.idx], np.sign(r.theta), atol=1e-4)


def test_extended_source_prefers_a_wide_atom():
    """Data dominated by one sigma = 5 atom (two weaker atoms of other scales,
    1 % noise): the solve puts most of that atom's flux on sigma = 5 atoms,
    its largest coefficient on that scale at (or next to) the true pixel."""
    uvw, fov, d, V, atoms = _small_problem(17)
    lam = 0.05 * dictionary.lambda_max(uvw, fov, d, V)
    r = dictionary.solve(uvw, fov, d, V, lam, tol=1e-5)
    N2 = d.N * d.N
    scales = r.idx // N2
    assert np.any(scales == 2)
    flux2 = np.abs(r.theta[scales == 2]).sum()
    assert flux2 >= 0.5 * 2.0
    best = r.idx[np.argmax(np.abs(r.theta))]
    bx, by = divmod(int(best % N2), d.N)
    assert best // N2 == 2 and abs(bx - 8) <= 1 and abs(by - 7) <= 1


def test_positive_solve_matches_positive_coordinate_descent():
    """Positivity variant (remark of Sect. 5.1) on the dictionary: theta >= 0,
    lambda_max = max(0, max Psi* Phi* V), same optimum as a non-negative
    coordinate descent."""
    rng = np.random.default_rng(18)
    N, fov, M = 8, math.radians(6.0), 60
    uvw = _uvw(rng, M, 0.5 / (fov / N), 2.0)
    d = dictionary.Dictionary(N, sigmas=(0.0, 1.0, 2.0))
    V = dictionary.forward(uvw, fov, d, [64 + 20, 2 * 64 + 43], [1.0, 2.0])
    V = V + 0.02 * np.abs(V).max() * (rng.normal(size=M) + 1j * rng.normal(size=M))
    lmax = dictionary.lambda_max(uvw, fov, d, V, positive=True)
    assert lmax == pytest.approx(max(0.0, dictionary.adjoint(uvw, fov, d, V).max()), rel=0)
    lam = 0.1 * lmax
    r = dictionary.solve(uvw, fov, d, V, lam, tol=1e-10, eps_min=1e-12, max_fw=200,
                         apgd_max_iter=200_000, positive=True)
    assert np.all(r.theta > 0)
    A = dictionary.columns(uvw, fov, d, np.arange(d.n_atoms))
    x_cd = lasso.coordinate_descent(A, V, lam, positive=True)
    assert r.objective == pytest.approx(lasso.objective(A, V, lam, x_cd), rel=1e-7)
    assert np.max(r.eta) <= 1 + 1e-4
