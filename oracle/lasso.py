"""Restricted LASSO sub-solvers in FP64 (test infrastructure only).

Step 2 of Algorithm 2 solves the LASSO (Sect. 4.1)

    min_x  1/2 ||V - A x||^2 + lambda ||x||_1,   x real, A = Phi restricted to a support,

with an accelerated proximal-gradient method (APGD / FISTA, Beck & Teboulle
2009, cited in Sect. 4.4), stopped early with an accuracy that tightens over
the Frank-Wolfe iterations (Sect. 5.1). The paper gives no constants, so this
module fixes them (the same readings are used by the GPU path):

  * step 1/L with L = 1.01 x the largest eigenvalue of Re(A^H A), the Hessian
    of the data term (here by a dense symmetric eigensolver);
  * the monotone FISTA variant (Beck & Teboulle 2009, "MFISTA"): the proximal
    point z is accepted only if it does not increase the objective;
  * stop when the proximal-gradient step ||z - y||_2 <= eps ||z||_2, or after
    max_iter iterations.

coordinate_descent and brute_force are independent LASSO solvers used only to
pin apgd and the Frank-Wolfe loop on tiny problems.

positive=True solves the positivity-constrained variant (the remarks on a
positivity constraint in Sect. 4.1 and 5.1): x >= 0, the proximal map of
t ||.||_1 + indicator(x >= 0) is max(z - t, 0).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def soft(z, t):
    """Proximal map of t ||.||_1 (soft thresholding)."""
    return np.sign(z) * np.maximum(np.abs(z) - t, 0.0)


def prox(z, t, positive=False):
    """Proximal map of t ||.||_1, plus the indicator of x >= 0 when positive."""
    return np.maximum(z - t, 0.0) if positive else soft(z, t)


def objective(A, V, lam, x) -> float:
    r = V - A @ x
    return 0.5 * float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(x)))


def gram_apply(A, v):
    """Re(A^H A) v, the Hessian of the data term applied to a real vector."""
    return np.real(A.conj().T @ (A @ v))


def lipschitz(A) -> float:
    """1.01 x the largest eigenvalue of Re(A^H A) (exact, numpy.linalg.eigvalsh)."""
    s = A.shape[1]
    if s == 0:
        return 1.0
    ev = float(np.linalg.eigvalsh(np.real(A.conj().T @ A))[-1])
    return 1.01 * ev if ev > 0.0 else 1.0


def apgd(A, V, lam, x0, eps, max_iter=10_000, L=None, positive=False):
    """Monotone FISTA on the restricted LASSO. Returns (x, iterations, L)."""
    if L is None:
        L = lipschitz(A)
    x = np.array(x0, dtype=np.float64)
    Fx = objective(A, V, lam, x)
    y = x.copy()
    t = 1.0
    it = 0
    for it in range(1, max_iter + 1):
        grad = np.real(A.conj().T @ (A @ y - V))
        z = prox(y - grad / L, lam / L, positive)
        Fz = objective(A, V, lam, z)
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        x_next = z if Fz <= Fx else x
        if Fz <= Fx:
            Fx = Fz
        step = float(np.linalg.norm(z - y))
        y = x_next + (t / t_next) * (z - x_next) + ((t - 1.0) / t_next) * (x_next - x)
        x = x_next
        t = t_next
        if step <= eps * float(np.linalg.norm(z)):
            break
    return x, it, L


def coordinate_descent(A, V, lam, tol=1e-14, max_sweeps=100_000, positive=False):
    """Cyclic coordinate descent (independent solver for pins)."""
    s = A.shape[1]
    x = np.zeros(s)
    col2 = np.sum(np.abs(A) ** 2, axis=0)
    r = V.astype(np.complex128).copy()
    for _ in range(max_sweeps):
        change = 0.0
        for j in range(s):
            rj = r + A[:, j] * x[j]
            c = float(np.real(np.vdot(A[:, j], rj)))
            if positive:
                xj = max(c - lam, 0.0) / col2[j]
            else:
                xj = np.sign(c) * max(abs(c) - lam, 0.0) / col2[j]
            if xj != x[j]:
                change = max(change, abs(xj - x[j]))
                r = rj - A[:, j] * xj
                x[j] = xj
        if change <= tol * max(1.0, float(np.max(np.abs(x)))):
            break
    return x


def brute_force(A, V, lam, positive=False):
    """Exact LASSO by enumerating sign patterns s in {-1, 0, +1}^n (tiny n only;
    {0, +1}^n when positive).

    For a pattern with support T: solve G_TT x_T = b_T - lam s_T with
    G = Re(A^H A), b = Re(A^H V); keep x if sign(x_T) = s_T and the
    off-support optimality |b - G x| <= lam (b - G x <= lam when positive)
    holds. Returns the feasible x with the smallest objective.
    """
    n = A.shape[1]
    G = np.real(A.conj().T @ A)
    b = np.real(A.conj().T @ V)
    best, best_f = np.zeros(n), objective(A, V, lam, np.zeros(n))
    for pattern in itertools.product((0, 1) if positive else (-1, 0, 1), repeat=n):
        s = np.array(pattern, dtype=np.float64)
        T = np.nonzero(s)[0]
        if T.size == 0:
            continue
        try:
            xT = np.linalg.solve(G[np.ix_(T, T)], b[T] - lam * s[T])
        except np.linalg.LinAlgError:
            continue
        if np.any(np.sign(xT) != s[T]):
            continue
        x = np.zeros(n)
        x[T] = xT
        g = b - G @ x
        off = np.setdiff1d(np.arange(n), T)
        viol = g[off] if positive else np.abs(g[off])
        if off.size and np.max(viol) > lam * (1 + 1e-12):
            continue
        f = objective(A, V, lam, x)
        if f < best_f:
            best, best_f = x, f
    return best
