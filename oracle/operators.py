"""Direct-sum measurement operator and adjoint in FP64 (test infrastructure only).

Sect. 2.2 of the paper: the image is an N x N real array on a uniform grid of
direction cosines (l_i, m_j), n = sqrt(1 - l^2 - m^2). The discrete forward
operator (degridding) is

    Phi(I)[k] = sum_{i,j} I[i,j] / n_ij * exp(-j 2 pi (u_k l_i + v_k m_j)) * W(l_i, m_j; w_k),
    W(l, m; w) = exp(-j 2 pi w (n(l, m) - 1))                          (Sect. 2.1)

and its adjoint (gridding) is

    Phi*(h)[i,j] = Re{ sum_k h_k / n_ij * exp(+j 2 pi (u_k l_i + v_k m_j)) * conj(W(l_i, m_j; w_k)) }.

Pixel geometry (the paper only says "uniform fine grid"): dl = fov / N,
l_i = (i - N//2) dl, m_j = (j - N//2) dl, raster index p = i N + j.

These are plain direct sums over all visibilities and the requested pixels.
Arrays are processed in chunks only to bound memory; the order of operations
within a sum is numpy's.
"""
from __future__ import annotations

import numpy as np

_CHUNK = 1 << 22   # complex entries per temporary phase block


def pixel_lmn(N: int, fov: float, idx):
    """(l, m, n) of raster indices idx on the N x N grid with full side fov."""
    idx = np.asarray(idx, dtype=np.int64)
    dl = fov / N
    i, j = np.divmod(idx, N)
    l = (i - N // 2) * dl
    m = (j - N // 2) * dl
    n = np.sqrt(1.0 - l * l - m * m)
    return l, m, n


def phase_block(uvw: np.ndarray, l, m, n) -> np.ndarray:
    """Matrix with entries exp(-j 2 pi (u_k l_p + v_k m_p + w_k (n_p - 1))) / n_p.

    Rows are visibilities k, columns pixels p. The phase is formed in turns and
    reduced to [-1/2, 1/2] before the exponential, so the float64 argument of
    exp stays small (an exact reduction up to the rounding of the turn count).
    """
    u, v, w = uvw[:, 0], uvw[:, 1], uvw[:, 2]
    turns = np.outer(u, l) + np.outer(v, m) + np.outer(w, n - 1.0)
    turns -= np.round(turns)
    return np.exp(-2j * np.pi * turns) / n[None, :]


def forward(uvw: np.ndarray, N: int, fov: float, idx, x) -> np.ndarray:
    """Phi restricted to the support idx with weights x: returns complex128 (M,)."""
    idx = np.asarray(idx, dtype=np.int64)
    x = np.asarray(x, dtype=np.float64)
    M = uvw.shape[0]
    out = np.zeros(M, dtype=np.complex128)
    if idx.size == 0:
        return out
    l, m, n = pixel_lmn(N, fov, idx)
    step = max(1, _CHUNK // max(1, idx.size))
    for k0 in range(0, M, step):
        A = phase_block(uvw[k0:k0 + step], l, m, n)
        out[k0:k0 + step] = A @ x
    return out


def adjoint(uvw: np.ndarray, N: int, fov: float, h, idx=None) -> np.ndarray:
    """Phi*(h) at raster indices idx (all N*N pixels, raster order, when idx is None)."""
    h = np.asarray(h, dtype=np.complex128)
    if idx is None:
        idx = np.arange(N * N, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    M = uvw.shape[0]
    out = np.empty(idx.size, dtype=np.float64)
    if idx.size == 0:
        return out
    step = max(1, _CHUNK // max(1, M))
    for p0 in range(0, idx.size, step):
        l, m, n = pixel_lmn(N, fov, idx[p0:p0 + step])
        A = phase_block(uvw, l, m, n)            # M x P block of Phi
        out[p0:p0 + step] = np.real(A.conj().T @ h)
    return out


def dirty_image(uvw, N, fov, V) -> np.ndarray:
    """Phi*(V) as an N x N array (natural weighting, Sect. 2.2)."""
    return adjoint(uvw, N, fov, V).reshape(N, N)


def lambda_max(uvw, N, fov, V) -> float:
    """lambda_max = ||Phi* V||_inf (Sect. 5.3): the smallest lambda with x = 0 optimal."""
    return float(np.max(np.abs(adjoint(uvw, N, fov, V))))


def lambda_max_positive(uvw, N, fov, V) -> float:
    """max(0, max_p Phi*(V)_p): the smallest lambda for which x = 0 is optimal
    when the image is constrained to be non-negative (the positivity remark of
    Sect. 4.1): the optimality condition at 0 is Phi*(V) <= lambda."""
    return max(0.0, float(np.max(adjoint(uvw, N, fov, V))))


def residual(uvw, N, fov, V, idx, x) -> np.ndarray:
    """r = V - Phi x for a sparse image (support idx, weights x)."""
    return np.asarray(V, dtype=np.complex128) - forward(uvw, N, fov, idx, x)


def objective(uvw, N, fov, V, lam, idx, x) -> float:
    """LASSO objective 1/2 ||V - Phi x||^2 + lambda ||x||_1 (Sect. 4.1)."""
    r = residual(uvw, N, fov, V, idx, x)
    return 0.5 * float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(x)))


def certificate(uvw, N, fov, V, lam, idx, x, pix=None) -> np.ndarray:
    """Empirical dual certificate mu = Phi*(V - Phi x) / lambda (Sect. 4.2)."""
    r = residual(uvw, N, fov, V, idx, x)
    return adjoint(uvw, N, fov, r, pix) / lam
