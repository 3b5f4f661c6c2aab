"""Polyatomic Frank-Wolfe (Algorithm 2) in FP64 (test infrastructure only).

Steps per iteration k = 0, 1, 2, ... (Algorithm 2 with Sect. 5.1):

  0. dirty residual    eta_k = Phi*(V - Phi I_k)     (on every pixel)
  1a. exploration      I_{k+1} = select(eta_k)
  1b. active set       S_{k+1} = S_k u I_{k+1}        (kept in ascending raster order)
  2.  reweighting      I_{k+1} = argmin over supp in S_{k+1} of the LASSO, by APGD
                       warm-started from I_k (0 on the new atoms), early-stopped at eps_k
  3.  pruning          S_{k+1} = supp(I_{k+1})
  4.  stop             relative objective improvement (F_k - F_{k+1}) / F_k < tol

Readings where the paper gives no value (the GPU path uses the same ones):

  * select rule "R2" (default): I = {p : |mu_k[p]| >= 1 - delta}, mu_k = eta_k / lambda,
    the empirical dual certificate (Sect. 4.2 / 4.1);
    select rule "R1" (the literal exploration set of Algorithm 2):
    I = {p : |eta_k[p]| >= ||eta_k||_inf - 2 Delta / (k + 2)}, Delta = (1 - delta) lambda_max;
  * eps_k = max(eps_min, eps0 * 2^-k), eps0 = 1e-2, eps_min = 1e-5;
  * objective F_k = 1/2 ||V - Phi I_k||^2 + lambda ||I_k||_1, F_0 = 1/2 ||V||^2;
  * tol = 1e-4 (Sect. 6.1), at most max_fw iterations.

Resume (checkpoint / warm start): the state of Algorithm 2 at the start of
iteration k is (k, S_k, I_k); S0, x0, k0 give it, and the loop then runs
exactly as it would have from there (F_prev = F(x0) for the first stop test,
eps_k and the R1 threshold at k = k0, ...). S0 = x0 = None, k0 = 0 is the
cold start.

positive=True is the positivity-constrained variant (remark in Sect. 5.1):
candidates only at positive values of the certificate (R2: mu >= 1 - delta;
R1: eta >= max(eta) - 2 Delta/(k + 2) with eta > 0, Delta from
lambda_max_positive), and the reweighting with x >= 0.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import lasso, operators


@dataclasses.dataclass
class SolveResult:
    idx: np.ndarray          # int64 sorted support (raster indices)
    x: np.ndarray            # float64 weights on the support
    mu: np.ndarray           # final certificate, N x N
    objective: float
    iterations: int
    converged: bool
    lambda_: float
    history: list


def select_r2(mu: np.ndarray, delta: float, positive: bool = False) -> np.ndarray:
    """Pixels whose certificate magnitude (its value, when positive) reaches
    1 - delta (ascending raster order)."""
    a = mu if positive else np.abs(mu)
    return np.nonzero(a >= 1.0 - delta)[0]


def select_r1(eta: np.ndarray, k: int, Delta: float, positive: bool = False) -> np.ndarray:
    """Exploration set of Algorithm 2: |eta| >= ||eta||_inf - 2 Delta / (k + 2);
    when positive, eta >= max(eta) - 2 Delta / (k + 2) among the pixels with eta > 0."""
    if positive:
        return np.nonzero((eta > 0.0) & (eta >= eta.max() - 2.0 * Delta / (k + 2)))[0]
    a = np.abs(eta)
    return np.nonzero(a >= a.max() - 2.0 * Delta / (k + 2))[0]


def eps_schedule(k: int, eps0: float = 1e-2, eps_min: float = 1e-5) -> float:
    return max(eps_min, eps0 * 2.0 ** (-k))


def duality_gap(uvw, N, fov, V, lam, idx, x, positive=False) -> float:
    """F(x) - D(theta) with the dual-feasible scaling theta = r min(1, lambda / ||Phi* r||_inf)
    (lambda / max(Phi* r) when positive: the dual constraint is then Phi* theta <= lambda).

    D(theta) = 1/2 ||V||^2 - 1/2 ||V - theta||^2 is the LASSO dual objective
    (complex data as a real vector space with inner product Re<.,.>).
    """
    V = np.asarray(V, dtype=np.complex128)
    r = operators.residual(uvw, N, fov, V, idx, x)
    eta = operators.adjoint(uvw, N, fov, r)
    g = np.max(eta) if positive else np.max(np.abs(eta))
    theta = r * min(1.0, lam / g) if g > 0 else r
    F = 0.5 * float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(x)))
    D = 0.5 * float(np.vdot(V, V).real) - 0.5 * float(np.vdot(V - theta, V - theta).real)
    return F - D


def frank_wolfe(V, lam, eta_all, columns, lmax, delta=0.01, rule="R2", tol=1e-4, max_fw=100,
                eps0=1e-2, eps_min=1e-5, apgd_max_iter=10_000, positive=False, S0=None, x0=None, k0=0):
    """Algorithm 2 over an abstract set of atoms (pixels, or the atoms of a
    synthesis dictionary, Sect. 4.3): eta_all(r) is Phi_A*(r) on every atom,
    columns(S) the columns of the measurement operator of the atoms S (sorted).
    (S0, x0, k0): the state to resume from (see the top of the file).
    Returns (S, x, r, F, iterations, converged, history)."""
    V = np.asarray(V, dtype=np.complex128)
    Delta = (1.0 - delta) * lmax
    S = np.zeros(0, dtype=np.int64)
    x = np.zeros(0)
    r = V.copy()
    if S0 is not None and len(S0):
        S = np.asarray(S0, dtype=np.int64)
        x = np.asarray(x0, dtype=np.float64)
        assert S.shape == x.shape and np.all(np.diff(S) > 0)
        r = V - columns(S) @ x
        F_prev = 0.5 * float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(x)))
    else:
        F_prev = 0.5 * float(np.vdot(V, V).real)
    history = []
    converged = False
    k = k0
    for k in range(k0, max_fw):
        eta = eta_all(r)                                          # dirty residual, all atoms
        if rule == "R2":
            new = select_r2(eta / lam, delta, positive)
            thr_mu = 1.0 - delta
        elif rule == "R1":
            new = select_r1(eta, k, Delta, positive)
            top = eta.max() if positive else np.abs(eta).max()
            thr_mu = (top - 2.0 * Delta / (k + 2)) / lam
        else:
            raise ValueError(rule)
        # diagnostic (no effect on the iteration): atoms whose candidate value
        # lies within 1e-5 max|mu| of the threshold, where an FP32 evaluation of
        # the certificate may legitimately take the other side
        cand = eta / lam if positive else np.abs(eta) / lam
        border = np.nonzero(np.abs(cand - thr_mu) <= 1e-5 * np.abs(eta).max() / lam)[0]
        n_border = int(border.size)
        n_new = int(np.setdiff1d(new, S).size)
        S_next = np.union1d(S, new).astype(np.int64)            # sorted, unique
        x0 = np.zeros(S_next.size)
        if S.size:
            x0[np.searchsorted(S_next, S)] = x                   # warm start on old atoms
        A = columns(S_next)                                       # operator restricted to S_next
        eps = eps_schedule(k, eps0, eps_min)
        xs, n_it, L = lasso.apgd(A, V, lam, x0, eps, apgd_max_iter, positive=positive)
        keep = xs != 0.0                                          # pruning
        S, x = S_next[keep], xs[keep]
        r = V - A[:, keep] @ x
        F = 0.5 * float(np.vdot(r, r).real) + lam * float(np.sum(np.abs(x)))
        rel = (F_prev - F) / F_prev if F_prev > 0 else 0.0
        history.append(dict(k=k, n_new=n_new,
                            n_active=int(S_next.size), n_support=int(S.size),
                            mu_inf=float(np.max(eta if positive else np.abs(eta)) / lam),
                            objective=F,
                            rel_improvement=rel, apgd_iterations=int(n_it), L=float(L),
                            eps=eps, n_borderline=n_border,
                            active=S_next.copy(), support=S.copy(), x=x.copy(), borderline=border))
        F_prev = F
        if rel < tol:
            converged = True
            break
    return S, x, r, F_prev, k + 1, converged, history


def solve(uvw, N, fov, V, lam, delta=0.01, rule="R2", tol=1e-4, max_fw=100,
          eps0=1e-2, eps_min=1e-5, apgd_max_iter=10_000, lmax=None, positive=False,
          S0=None, x0=None, k0=0) -> SolveResult:
    V = np.asarray(V, dtype=np.complex128)
    if lmax is None:
        lmax = (operators.lambda_max_positive if positive else operators.lambda_max)(uvw, N, fov, V)

    def columns(S):
        l, m, n = operators.pixel_lmn(N, fov, S)
        return operators.phase_block(uvw, l, m, n)

    S, x, r, F, iters, converged, history = frank_wolfe(
        V, lam, lambda r: operators.adjoint(uvw, N, fov, r), columns, lmax, delta, rule, tol, max_fw,
        eps0, eps_min, apgd_max_iter, positive, S0, x0, k0)
    mu = operators.adjoint(uvw, N, fov, r).reshape(N, N) / lam
    return SolveResult(S, x, mu, F, iters, converged, lam, history)
