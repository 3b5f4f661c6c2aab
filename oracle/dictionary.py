"""Synthesis-form LASSO over a multi-scale Gaussian dictionary in FP64 (test
infrastructure only).

Sect. 4.3 writes the image as I = Psi theta and solves

    argmin_theta 1/2 ||V - Phi Psi theta||^2 + lambda ||theta||_1,

and the diffuse experiment of Sect. 6 builds Psi from scaled Gaussian kernels
g_i = gamma_i g~_i, g~_i[n, m] proportional to exp(-(n^2 + m^2) / sigma_i^2)
on |n|, |m| <= 2 sigma_i, normalised to unit l1 norm, sigma = (0, 2, 5, 8),
gamma_i = 1.2^i. lambda_max is taken with Psi as well.

Readings (the paper leaves these open):

  * sigma = 0 is the point-source atom: a single pixel of weight 1;
  * the crop is the square |n|, |m| <= floor(2 sigma);
  * Psi places g_i centred on the atom's pixel and drops what falls outside
    the N x N image (zero-padded, "same"-size convolution, no renormalisation
    at the border); Psi* is the matching correlation restricted to the image;
  * coefficient index a = i N^2 + p (scale-major, p the raster pixel index);
  * ||theta||_1 is the plain l1 norm (gamma_i lives inside the atoms).

Everything is a direct restatement: shift-and-add for Psi and Psi*, the
measurement operator of operators.py on the synthesised pixels for Phi Psi,
and the Frank-Wolfe loop of pfw.py over the coefficient atoms.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import operators, pfw

SIGMAS = (0.0, 2.0, 5.0, 8.0)
GAMMAS = tuple(1.2 ** i for i in range(4))


def kernel(sigma: float) -> np.ndarray:
    """g~ for one scale: (2K+1) x (2K+1), K = floor(2 sigma), unit sum."""
    if sigma == 0.0:
        return np.ones((1, 1))
    K = int(np.floor(2.0 * sigma))
    n = np.arange(-K, K + 1, dtype=np.float64)
    g = np.exp(-(n[:, None] ** 2 + n[None, :] ** 2) / sigma ** 2)
    return g / g.sum()


@dataclasses.dataclass
class Dictionary:
    N: int
    sigmas: tuple = SIGMAS
    gammas: tuple = GAMMAS

    @property
    def n_scales(self) -> int:
        return len(self.sigmas)

    @property
    def n_atoms(self) -> int:
        return self.n_scales * self.N * self.N

    def kernels(self):
        return [kernel(s) for s in self.sigmas]


def atom_pixels(d: Dictionary, a: int):
    """Raster pixels and weights gamma_i g~_i of atom a, inside the image."""
    N = d.N
    i, p = divmod(int(a), N * N)
    x0, y0 = divmod(p, N)
    g = kernel(d.sigmas[i])
    K = g.shape[0] // 2
    pix, wts = [], []
    for n in range(-K, K + 1):
        for m in range(-K, K + 1):
            x, y = x0 + n, y0 + m
            if 0 <= x < N and 0 <= y < N:
                pix.append(x * N + y)
                wts.append(d.gammas[i] * g[n + K, m + K])
    return np.array(pix, dtype=np.int64), np.array(wts)


def synthesize(d: Dictionary, theta) -> np.ndarray:
    """Psi theta: the N x N image (raster vector) of the coefficients theta (n_atoms,)."""
    N = d.N
    theta = np.asarray(theta, dtype=np.float64).reshape(d.n_scales, N, N)
    img = np.zeros((N, N))
    for i, g in enumerate(d.kernels()):
        K = g.shape[0] // 2
        for n in range(-K, K + 1):
            for m in range(-K, K + 1):
                # img[x + n, y + m] += gamma g[n, m] theta_i[x, y] for in-image targets
                xs = slice(max(0, -n), min(N, N - n))
                ys = slice(max(0, -m), min(N, N - m))
                xt = slice(max(0, n), min(N, N + n))
                yt = slice(max(0, m), min(N, N + m))
                img[xt, yt] += d.gammas[i] * g[n + K, m + K] * theta[i][xs, ys]
    return img.ravel()


def analyze(d: Dictionary, z) -> np.ndarray:
    """Psi* z for an N x N image z (raster vector): (n_atoms,), scale-major."""
    N = d.N
    z = np.asarray(z, dtype=np.float64).reshape(N, N)
    out = np.zeros((d.n_scales, N, N))
    for i, g in enumerate(d.kernels()):
        K = g.shape[0] // 2
        for n in range(-K, K + 1):
            for m in range(-K, K + 1):
                # out_i[x, y] += gamma g[n, m] z[x + n, y + m] for in-image sources
                xo = slice(max(0, -n), min(N, N - n))
                yo = slice(max(0, -m), min(N, N - m))
                xs = slice(max(0, n), min(N, N + n))
                ys = slice(max(0, m), min(N, N + m))
                out[i][xo, yo] += d.gammas[i] * g[n + K, m + K] * z[xs, ys]
    return out.ravel()


_PIXEL_MATRIX_MAX = 1 << 23   # entries of Phi on every pixel worth building once


def columns(uvw, fov, d: Dictionary, atoms) -> np.ndarray:
    """Columns of Phi Psi for the atoms (M x len(atoms), complex128): each is
    Phi applied to the atom's image, sum_p w_p Phi[:, p] over its footprint.
    On small problems Phi is built once on every pixel and its columns reused."""
    atoms = np.asarray(atoms, dtype=np.int64)
    M, N = uvw.shape[0], d.N
    A = np.zeros((M, atoms.size), dtype=np.complex128)
    P = None
    if atoms.size > 1 and M * N * N <= _PIXEL_MATRIX_MAX:
        P = operators.phase_block(uvw, *operators.pixel_lmn(N, fov, np.arange(N * N)))
    for c, a in enumerate(atoms):
        pix, wts = atom_pixels(d, a)
        A[:, c] = P[:, pix] @ wts if P is not None else operators.forward(uvw, N, fov, pix, wts)
    return A


def forward(uvw, fov, d: Dictionary, atoms, theta) -> np.ndarray:
    """Phi Psi theta for coefficients theta on the atoms (complex128, (M,))."""
    full = np.zeros(d.n_atoms)
    full[np.asarray(atoms, dtype=np.int64)] = np.asarray(theta, dtype=np.float64)
    img = synthesize(d, full)
    nz = np.nonzero(img)[0]
    return operators.forward(uvw, d.N, fov, nz, img[nz])


def adjoint(uvw, fov, d: Dictionary, h) -> np.ndarray:
    """Psi* Phi* h on every atom (n_atoms,)."""
    return analyze(d, operators.adjoint(uvw, d.N, fov, h))


def lambda_max(uvw, fov, d: Dictionary, V, positive=False) -> float:
    """Smallest lambda with theta = 0 optimal: ||Psi* Phi* V||_inf (max(0, max)
    under positivity)."""
    eta = adjoint(uvw, fov, d, V)
    return max(0.0, float(eta.max())) if positive else float(np.max(np.abs(eta)))


@dataclasses.dataclass
class SynthesisResult:
    idx: np.ndarray          # int64 sorted atom indices (a = scale N^2 + pixel)
    theta: np.ndarray        # float64 coefficients on idx
    eta: np.ndarray          # final certificate Psi* Phi* r / lambda, (n_scales, N, N)
    objective: float
    iterations: int
    converged: bool
    lambda_: float
    history: list


def solve(uvw, fov, d: Dictionary, V, lam, delta=0.01, rule="R2", tol=1e-5, max_fw=100,
          eps0=1e-2, eps_min=1e-5, apgd_max_iter=10_000, lmax=None, positive=False) -> SynthesisResult:
    """Algorithm 2 on the synthesis-form LASSO (stop 1e-5 as in the diffuse
    experiment of Sect. 6)."""
    V = np.asarray(V, dtype=np.complex128)
    if lmax is None:
        lmax = lambda_max(uvw, fov, d, V, positive)
    S, x, r, F, iters, converged, history = pfw.frank_wolfe(
        V, lam, lambda res: adjoint(uvw, fov, d, res), lambda S_: columns(uvw, fov, d, S_), lmax,
        delta, rule, tol, max_fw, eps0, eps_min, apgd_max_iter, positive)
    eta = adjoint(uvw, fov, d, r).reshape(d.n_scales, d.N, d.N) / lam
    return SynthesisResult(S, x, eta, F, iters, converged, lam, history)
