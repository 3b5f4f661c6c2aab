"""Thin Python binding of the C ABI in include/polyclean.h (ctypes).

Every function here only marshals arguments: torch CUDA tensors are passed as
device pointers, the stream is the current torch stream unless given. All
arithmetic runs in the CUDA kernels of libpolyclean.so. The library must be
built (paper_2406_01342_gb300.build.build()); there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

PC_ABI_VERSION = 5
PC_OK = 0
PC_ERR_INVALID_ARG = -1
PC_ERR_OOM = -2
PC_ERR_CUDA = -3
PC_ERR_NOT_CONVERGED = -4
PC_ERR_TIMEOUT = -5
PC_ERR_NUMERIC = -6
PC_ERR_CAPACITY = -7

# Every function the header declares (checked by the CPU test-suite).
EXPORTS = [
    "pc_plan_create", "pc_plan", "pc_plan_destroy", "pc_plan_info", "pc_forward_sparse",
    "pc_adjoint_sparse", "pc_adjoint_grid", "pc_lambda_max", "pc_certificate", "pc_select",
    "pc_gram", "pc_apgd", "pc_solve", "pc_solve_host", "pc_profile_begin", "pc_profile_end",
    "pc_last_error", "pc_abi_version", "pc_adjoint_sparse_noalloc", "pc_lambda_max_positive",
    "pc_profile_begin_classes", "pc_server_create", "pc_server_submit", "pc_server_wait",
    "pc_server_destroy", "pc_plan_tuning_info", "pc_dict_adjoint", "pc_dict_forward_sparse",
    "pc_dict_lambda_max", "pc_solve_synthesis", "pc_forward_grid", "pc_trim_memory", "pc_plan_reach",
]


class PcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[status {status}] {msg}")
        self.status = status


class pc_plan_opts(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("kernel_width", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("max_planes", ctypes.c_int32),
                ("grid_mode", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("fft_kernel", ctypes.c_int32)]


class pc_plan_tuning(ctypes.Structure):
    _fields_ = [("tuned", ctypes.c_int32), ("grid_mode", ctypes.c_int32),
                ("grid_piece", ctypes.c_int32), ("fft_rows_per_cta", ctypes.c_int32),
                ("grid_us", ctypes.c_double), ("fft_rows_us", ctypes.c_double),
                ("fft_cols_planes", ctypes.c_int32), ("fft_warp", ctypes.c_int32),
                ("fft_cols_us", ctypes.c_double), ("degrid_piece", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("degrid_us", ctypes.c_double)]


class pc_server_opts(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("max_jobs", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("batch_apgd", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class pc_job_times(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_double), ("admitted", ctypes.c_double),
                ("finished", ctypes.c_double)]


class pc_solve_opts(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("select_rule", ctypes.c_int32),
                ("max_fw", ctypes.c_int32), ("apgd_max_iter", ctypes.c_int32),
                ("gram_mode", ctypes.c_int32), ("positivity", ctypes.c_int32),
                ("tol", ctypes.c_double), ("eps0", ctypes.c_double),
                ("eps_min", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("reweight", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("init_idx", ctypes.c_void_p), ("init_x", ctypes.c_void_p),
                ("init_S", ctypes.c_int32), ("init_k", ctypes.c_int32)]


PC_DICT_MAX_SCALES = 8


class pc_dictionary(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("n_scales", ctypes.c_int32),
                ("sigma", ctypes.c_double * PC_DICT_MAX_SCALES),
                ("gamma", ctypes.c_double * PC_DICT_MAX_SCALES)]


def make_dictionary(sigmas=(0.0, 2.0, 5.0, 8.0), gammas=None) -> pc_dictionary:
    """Multi-scale Gaussian dictionary; gammas default to 1.2^i."""
    if gammas is None:
        gammas = [1.2 ** i for i in range(len(sigmas))]
    d = pc_dictionary()
    d.version = PC_ABI_VERSION
    d.n_scales = len(sigmas)
    for i, (s, g) in enumerate(zip(sigmas, gammas)):
        d.sigma[i] = float(s)
        d.gamma[i] = float(g)
    return d


class pc_iter_record(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_new", ctypes.c_int32), ("n_active", ctypes.c_int32),
                ("n_support", ctypes.c_int32), ("apgd_iterations", ctypes.c_int32),
                ("lanczos_steps", ctypes.c_int32), ("mu_inf", ctypes.c_double),
                ("objective", ctypes.c_double), ("rel_improvement", ctypes.c_double),
                ("lipschitz", ctypes.c_double)]


class pc_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("kernels", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class pc_solve_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("n_support", ctypes.c_int32), ("n_history", ctypes.c_int32),
                ("objective", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("mu_inf", ctypes.c_double), ("sumsq_V", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
_F = ctypes.c_float


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libpolyclean.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2406_01342_gb300.build.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "pc_plan_create": (_I32, [_P, _I64, _I32, _D, _P, _P, ctypes.POINTER(_P)]),
        "pc_plan": (_I32, [_P, _I64, _I32, _D, _P, _P, ctypes.POINTER(_P)]),
        "pc_plan_destroy": (None, [_P]),
        "pc_plan_tuning_info": (_I32, [_P, ctypes.POINTER(pc_plan_tuning)]),
        "pc_plan_reach": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
        "pc_plan_info": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                ctypes.POINTER(_I64), ctypes.POINTER(_I32), ctypes.POINTER(_D)]),
        "pc_forward_sparse": (_I32, [_P, _P, _P, _I32, _P, _P]),
        "pc_adjoint_sparse": (_I32, [_P, _P, _P, _I32, _P, _P]),
        "pc_adjoint_grid": (_I32, [_P, _P, _P, _P]),
        "pc_forward_grid": (_I32, [_P, _P, _P, _P]),
        "pc_lambda_max": (_I32, [_P, _P, ctypes.POINTER(_D), _P]),
        "pc_lambda_max_positive": (_I32, [_P, _P, ctypes.POINTER(_D), _P]),
        "pc_certificate": (_I32, [_P, _P, _P, _P, _I32, _D, _P, ctypes.POINTER(_D),
                                  ctypes.POINTER(_D), _P]),
        "pc_select": (_I32, [_P, _P, _F, _P, _I32, _P, _I32, ctypes.POINTER(_I32), _P]),
        "pc_gram": (_I32, [_P, _P, _P, _I32, _P, _I32, _P, _I32, _P]),
        "pc_apgd": (_I32, [_P, _I32, _P, _I32, _D, _D, _I32, _I32, _P, ctypes.POINTER(_I32),
                           ctypes.POINTER(_D), _P]),
        "pc_solve": (_I32, [_P, _P, _D, _D, _P, _P, _P, _I32, _P, ctypes.POINTER(pc_solve_stats),
                            _P, _I32, _P]),
        "pc_solve_host": (_I32, [_P, _P, _I64, _I32, _D, _D, _D, _P, _P, _P, _I32,
                                 ctypes.POINTER(pc_solve_stats), _P]),
        "pc_dict_adjoint": (_I32, [_P, ctypes.POINTER(pc_dictionary), _P, _D, _P, _P]),
        "pc_dict_forward_sparse": (_I32, [_P, ctypes.POINTER(pc_dictionary), _P, _P, _I32, _P, _P]),
        "pc_dict_lambda_max": (_I32, [_P, ctypes.POINTER(pc_dictionary), _P, _I32, ctypes.POINTER(_D), _P]),
        "pc_solve_synthesis": (_I32, [_P, ctypes.POINTER(pc_dictionary), _P, _D, _D, _P, _P, _P, _I32, _P,
                                      ctypes.POINTER(pc_solve_stats), _P, _I32, _P]),
        "pc_adjoint_sparse_noalloc": (_I32, [_P, _I64, _I32, _D, _P, _P, _I32, _P, _P]),
        "pc_profile_begin": (_I32, []),
        "pc_profile_begin_classes": (_I32, [ctypes.c_char_p]),
        "pc_server_create": (_I32, [_P, ctypes.POINTER(_P)]),
        "pc_server_submit": (_I32, [_P, _P, _P, _I64, _I32, _D, _D, _D, _P, ctypes.POINTER(_I64)]),
        "pc_server_wait": (_I32, [_P, _I64, _P, _P, _I32, ctypes.POINTER(pc_solve_stats),
                                  ctypes.POINTER(pc_job_times)]),
        "pc_server_destroy": (None, [_P]),
        "pc_profile_end": (_I32, [ctypes.POINTER(pc_kernel_time), _I32, ctypes.POINTER(_I32)]),
        "pc_last_error": (ctypes.c_char_p, []),
        "pc_abi_version": (_I32, []),
        "pc_trim_memory": (_I32, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, allow=(PC_OK,)) -> int:
    if status not in allow:
        raise PcError(status, load().pc_last_error().decode(errors="replace"))
    return status


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev(t: torch.Tensor | None, dtype, name: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owns a pc_plan_t handle (destroyed with the object)."""

    def __init__(self, handle, M: int, N: int, fov: float):
        self.handle = handle
        self.M, self.N, self.fov = M, N, fov

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().pc_plan_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def pc_plan_create(uvw: torch.Tensor, N: int, fov: float, kernel_width: int = 0, tile: int = 0,
                   max_planes: int = 0, stream=None, grid_mode: int = 0, autotune: int = 0,
                   fft_kernel: int = 0) -> Plan:
    lib = load()
    opts = pc_plan_opts(PC_ABI_VERSION, kernel_width, tile, max_planes, grid_mode, autotune, fft_kernel)
    h = _P()
    M = int(uvw.shape[0])
    _check(lib.pc_plan_create(_dev(uvw, torch.float64, "uvw") if M else None, M, N, float(fov),
                              ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
    return Plan(h, M, N, fov)


def pc_plan_info(plan: Plan) -> dict:
    g, t, p = _I32(), _I32(), _I32()
    ns, w = _I64(), _I32()
    dw = _D()
    _check(load().pc_plan_info(plan.handle, ctypes.byref(g), ctypes.byref(t), ctypes.byref(p),
                               ctypes.byref(ns), ctypes.byref(w), ctypes.byref(dw)))
    return dict(grid_side=g.value, tile=t.value, n_planes=p.value, n_slots=ns.value,
                kernel_width=w.value, dw=dw.value)


def pc_plan_reach(plan: Plan) -> dict:
    """Reachable grid rows and 32-column groups of each w-plane."""
    r, c = _I32(), _I32()
    _check(load().pc_plan_reach(plan.handle, ctypes.byref(r), ctypes.byref(c)))
    return dict(rows=r.value, col_groups=c.value)


def pc_plan_tuning_info(plan: Plan) -> dict:
    t = pc_plan_tuning()
    _check(load().pc_plan_tuning_info(plan.handle, ctypes.byref(t)))
    return dict(tuned=bool(t.tuned), grid_mode=t.grid_mode, grid_piece=t.grid_piece,
                fft_rows_per_cta=t.fft_rows_per_cta, grid_us=t.grid_us, fft_rows_us=t.fft_rows_us,
                fft_cols_planes=t.fft_cols_planes, fft_cols_us=t.fft_cols_us,
                fft_warp=t.fft_warp, degrid_piece=t.degrid_piece, degrid_us=t.degrid_us)


def pc_forward_sparse(plan: Plan, idx: torch.Tensor, x: torch.Tensor, y: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    if y is None:
        y = torch.empty(plan.M, dtype=torch.complex64, device=idx.device)
    S = int(idx.numel())
    _check(load().pc_forward_sparse(plan.handle, _dev(idx, torch.int32, "idx"),
                                    _dev(x, torch.float32, "x"), S, _dev(y, torch.complex64, "y"),
                                    _stream(stream)))
    return y


def pc_adjoint_sparse(plan: Plan, y: torch.Tensor, idx: torch.Tensor, out: torch.Tensor | None = None,
                      stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(idx.numel(), dtype=torch.float32, device=idx.device)
    _check(load().pc_adjoint_sparse(plan.handle, _dev(y, torch.complex64, "y"),
                                    _dev(idx, torch.int32, "idx"), int(idx.numel()),
                                    _dev(out, torch.float32, "out"), _stream(stream)))
    return out


def pc_adjoint_grid(plan: Plan, y: torch.Tensor, img: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    if img is None:
        img = torch.empty(plan.N, plan.N, dtype=torch.float32, device=y.device)
    _check(load().pc_adjoint_grid(plan.handle, _dev(y, torch.complex64, "y"),
                                  _dev(img, torch.float32, "img"), _stream(stream)))
    return img


def pc_forward_grid(plan: Plan, img: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Phi(img) for a dense N x N float32 image (degridding)."""
    if y is None:
        y = torch.empty(plan.M, dtype=torch.complex64, device=img.device)
    _check(load().pc_forward_grid(plan.handle, _dev(img, torch.float32, "img"), _dev(y, torch.complex64, "y"),
                                  _stream(stream)))
    return y


def pc_lambda_max(plan: Plan, V: torch.Tensor, stream=None) -> float:
    out = _D()
    _check(load().pc_lambda_max(plan.handle, _dev(V, torch.complex64, "V"), ctypes.byref(out),
                                _stream(stream)))
    return out.value


def pc_lambda_max_positive(plan: Plan, V: torch.Tensor, stream=None) -> float:
    out = _D()
    _check(load().pc_lambda_max_positive(plan.handle, _dev(V, torch.complex64, "V"),
                                         ctypes.byref(out), _stream(stream)))
    return out.value


def pc_certificate(plan: Plan, V: torch.Tensor, idx: torch.Tensor, x: torch.Tensor, lam: float,
                   mu: torch.Tensor | None = None, stream=None):
    if mu is None:
        mu = torch.empty(plan.N, plan.N, dtype=torch.float32, device=V.device)
    mi, ss = _D(), _D()
    _check(load().pc_certificate(plan.handle, _dev(V, torch.complex64, "V"),
                                 _dev(idx, torch.int32, "idx"), _dev(x, torch.float32, "x"),
                                 int(idx.numel()), float(lam), _dev(mu, torch.float32, "mu"),
                                 ctypes.byref(mi), ctypes.byref(ss), _stream(stream)))
    return mu, mi.value, ss.value


def pc_select(plan: Plan, mu: torch.Tensor, thr: float, prev_idx: torch.Tensor, cap: int,
              stream=None) -> torch.Tensor:
    out = torch.empty(max(cap, 1), dtype=torch.int32, device=mu.device)
    n = _I32()
    _check(load().pc_select(plan.handle, _dev(mu, torch.float32, "mu"), float(thr),
                            _dev(prev_idx, torch.int32, "prev_idx"), int(prev_idx.numel()),
                            _dev(out, torch.int32, "out"), int(cap), ctypes.byref(n),
                            _stream(stream)))
    return out[: n.value]


def pc_gram(plan: Plan, V: torch.Tensor | None, idx: torch.Tensor, mode: int = 0, stream=None):
    S = int(idx.numel())
    G = torch.empty(S, S, dtype=torch.float32, device=idx.device)
    b = torch.empty(S, dtype=torch.float32, device=idx.device) if V is not None else None
    _check(load().pc_gram(plan.handle, _dev(V, torch.complex64, "V"), _dev(idx, torch.int32, "idx"),
                          S, _dev(G, torch.float32, "G"), S, _dev(b, torch.float32, "b"),
                          int(mode), _stream(stream)))
    return G, b


def pc_apgd(G: torch.Tensor, b: torch.Tensor, lam: float, eps: float, max_iter: int,
            x: torch.Tensor, stream=None, positive: bool = False):
    S = int(b.numel())
    it = _I32()
    L = _D()
    _check(load().pc_apgd(_dev(G, torch.float32, "G"), int(G.stride(0)), _dev(b, torch.float32, "b"),
                          S, float(lam), float(eps), int(max_iter), int(bool(positive)),
                          _dev(x, torch.float32, "x"), ctypes.byref(it), ctypes.byref(L),
                          _stream(stream)))
    return x, it.value, L.value


def _solve_opts(select_rule=0, max_fw=0, apgd_max_iter=0, tol=0.0, eps0=0.0, eps_min=0.0,
                lambda_max=0.0, gram_mode=0, positivity=0, reweight=0, init_idx=None, init_x=None,
                init_k=0):
    S = 0 if init_idx is None else int(init_idx.numel())
    if S and (init_x is None or int(init_x.numel()) != S):
        raise ValueError("init_x must hold one weight per init_idx entry")
    return pc_solve_opts(PC_ABI_VERSION, select_rule, max_fw, apgd_max_iter, gram_mode,
                         int(positivity), tol, eps0, eps_min, lambda_max, int(reweight), 0,
                         _dev(init_idx, torch.int32, "init_idx") if S else None,
                         _dev(init_x, torch.float32, "init_x") if S else None, S, int(init_k))


def pc_solve(plan: Plan, V: torch.Tensor, lam: float, delta: float, cap: int = 65536,
             want_mu: bool = True, history: int = 256, stream=None, **opts) -> dict:
    dev = V.device
    idx = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    x = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
    mu = torch.empty(plan.N, plan.N, dtype=torch.float32, device=dev) if want_mu else None
    st = pc_solve_stats()
    hist = (pc_iter_record * max(history, 1))()
    o = _solve_opts(**opts)
    status = load().pc_solve(plan.handle, _dev(V, torch.complex64, "V"), float(lam), float(delta),
                             ctypes.byref(o), _dev(idx, torch.int32, "idx"),
                             _dev(x, torch.float32, "x"), int(cap),
                             _dev(mu, torch.float32, "mu") if mu is not None else None,
                             ctypes.byref(st), hist, int(history), _stream(stream))
    _check(status, allow=(PC_OK, PC_ERR_NOT_CONVERGED))
    n = st.n_support
    recs = [dict(k=h.k, n_new=h.n_new, n_active=h.n_active, n_support=h.n_support,
                 apgd_iterations=h.apgd_iterations, lanczos_steps=h.lanczos_steps,
                 mu_inf=h.mu_inf, objective=h.objective,
                 rel_improvement=h.rel_improvement, lipschitz=h.lipschitz)
            for h in hist[: st.n_history]]
    return dict(idx=idx[:n], x=x[:n], mu=mu, status=st.status, iterations=st.iterations,
                objective=st.objective, lam=st.lambda_, mu_inf=st.mu_inf, sumsq_V=st.sumsq_V,
                converged=st.status == PC_OK, history=recs)


def pc_dict_adjoint(plan: Plan, dictionary: pc_dictionary, h: torch.Tensor, scale: float = 1.0,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """scale * Psi* Phi* h on every coefficient, shape (n_scales, N, N)."""
    if out is None:
        out = torch.empty(dictionary.n_scales, plan.N, plan.N, dtype=torch.float32, device=h.device)
    _check(load().pc_dict_adjoint(plan.handle, ctypes.byref(dictionary), _dev(h, torch.complex64, "h"),
                                  float(scale), _dev(out, torch.float32, "out"), _stream(stream)))
    return out


def pc_dict_forward_sparse(plan: Plan, dictionary: pc_dictionary, idx: torch.Tensor, theta: torch.Tensor,
                           y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Phi Psi theta for coefficients theta on the ascending coefficient indices idx."""
    if y is None:
        y = torch.empty(plan.M, dtype=torch.complex64, device=idx.device)
    _check(load().pc_dict_forward_sparse(plan.handle, ctypes.byref(dictionary), _dev(idx, torch.int32, "idx"),
                                         _dev(theta, torch.float32, "theta"), int(idx.numel()),
                                         _dev(y, torch.complex64, "y"), _stream(stream)))
    return y


def pc_dict_lambda_max(plan: Plan, dictionary: pc_dictionary, V: torch.Tensor, positive: bool = False,
                       stream=None) -> float:
    out = _D()
    _check(load().pc_dict_lambda_max(plan.handle, ctypes.byref(dictionary), _dev(V, torch.complex64, "V"),
                                     int(bool(positive)), ctypes.byref(out), _stream(stream)))
    return out.value


def pc_solve_synthesis(plan: Plan, dictionary: pc_dictionary, V: torch.Tensor, lam: float, delta: float,
                       cap: int = 65536, want_eta: bool = True, history: int = 256, stream=None,
                       **opts) -> dict:
    """Synthesis-form solve over the dictionary; idx are coefficient indices
    (scale * N^2 + pixel), theta their coefficients."""
    dev = V.device
    idx = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    th = torch.empty(max(cap, 1), dtype=torch.float32, device=dev)
    eta = (torch.empty(dictionary.n_scales, plan.N, plan.N, dtype=torch.float32, device=dev)
           if want_eta else None)
    st = pc_solve_stats()
    hist = (pc_iter_record * max(history, 1))()
    o = _solve_opts(**opts)
    status = load().pc_solve_synthesis(plan.handle, ctypes.byref(dictionary), _dev(V, torch.complex64, "V"),
                                       float(lam), float(delta), ctypes.byref(o),
                                       _dev(idx, torch.int32, "idx"), _dev(th, torch.float32, "theta"),
                                       int(cap), _dev(eta, torch.float32, "eta") if eta is not None else None,
                                       ctypes.byref(st), hist, int(history), _stream(stream))
    _check(status, allow=(PC_OK, PC_ERR_NOT_CONVERGED))
    n = st.n_support
    recs = [dict(k=h.k, n_new=h.n_new, n_active=h.n_active, n_support=h.n_support,
                 apgd_iterations=h.apgd_iterations, lanczos_steps=h.lanczos_steps,
                 mu_inf=h.mu_inf, objective=h.objective,
                 rel_improvement=h.rel_improvement, lipschitz=h.lipschitz)
            for h in hist[: st.n_history]]
    return dict(idx=idx[:n], theta=th[:n], eta=eta, status=st.status, iterations=st.iterations,
                objective=st.objective, lam=st.lambda_, mu_inf=st.mu_inf, sumsq_V=st.sumsq_V,
                converged=st.status == PC_OK, history=recs)


def pc_solve_host(uvw, V, N: int, fov: float, alpha: float, delta: float, cap: int = 65536,
                  stream=None, **opts) -> dict:
    """uvw: (M, 3) float64 and V: (M,) complex64 CPU tensors or numpy arrays (host memory)."""
    import numpy as np
    uvw_np = np.ascontiguousarray(np.asarray(uvw, dtype=np.float64))
    V_np = np.ascontiguousarray(np.asarray(V, dtype=np.complex64))
    M = int(uvw_np.shape[0])
    idx = np.empty(max(cap, 1), dtype=np.int32)
    x = np.empty(max(cap, 1), dtype=np.float32)
    st = pc_solve_stats()
    o = _solve_opts(**opts)
    status = load().pc_solve_host(uvw_np.ctypes.data, V_np.ctypes.data, M, int(N), float(fov),
                                  float(alpha), float(delta), ctypes.byref(o), idx.ctypes.data,
                                  x.ctypes.data, int(cap), ctypes.byref(st), _stream(stream))
    _check(status, allow=(PC_OK, PC_ERR_NOT_CONVERGED))
    n = st.n_support
    return dict(idx=idx[:n].copy(), x=x[:n].copy(), status=st.status, iterations=st.iterations,
                objective=st.objective, lam=st.lambda_, mu_inf=st.mu_inf,
                converged=status == PC_OK)


def pc_profile_begin(classes: str | None = None) -> None:
    """Start per-kernel-class event timing: every class, or only the
    comma-separated classes named (e.g. "gram_tc")."""
    if classes:
        _check(load().pc_profile_begin_classes(classes.encode()))
    else:
        _check(load().pc_profile_begin())


def pc_profile_end() -> dict:
    """{kernel class: (launcher calls, kernels, total_ms)} recorded since pc_profile_begin()."""
    recs = (pc_kernel_time * 32)()
    n = _I32()
    _check(load().pc_profile_end(recs, 32, ctypes.byref(n)))
    return {r.name.decode(): (int(r.launches), int(r.kernels), float(r.total_ms))
            for r in recs[: min(n.value, 32)]}


def pc_adjoint_sparse_noalloc(uvw: torch.Tensor, N: int, fov: float, y: torch.Tensor,
                              idx: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """Allocation-free Phi*(y) at the pixels idx, written into the caller's `out`
    (no plan; the library allocates nothing, see include/polyclean.h)."""
    M = int(uvw.shape[0])
    _check(load().pc_adjoint_sparse_noalloc(
        _dev(uvw, torch.float64, "uvw") if M else None, M, int(N), float(fov),
        _dev(y, torch.complex64, "y") if M else None, _dev(idx, torch.int32, "idx"),
        int(idx.numel()), _dev(out, torch.float32, "out"), _stream(stream)))
    return out


class Server:
    """Continuous-batching request loop of the library (pc_server_*): submit
    imaging requests from the host at any time, collect each result with wait()."""

    def __init__(self, max_jobs: int = 8, memory_budget: int = 0, batch_apgd: int = 1):
        lib = load()
        o = pc_server_opts(PC_ABI_VERSION, max_jobs, memory_budget, batch_apgd, 0)
        h = _P()
        _check(lib.pc_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    def submit(self, uvw, V, N: int, fov: float, alpha: float, delta: float, **opts) -> int:
        import numpy as np
        uvw_np = np.ascontiguousarray(np.asarray(uvw, dtype=np.float64))
        V_np = np.ascontiguousarray(np.asarray(V, dtype=np.complex64))
        o = _solve_opts(**opts)
        jid = _I64()
        _check(load().pc_server_submit(self.handle, uvw_np.ctypes.data, V_np.ctypes.data,
                                       int(V_np.shape[0]), int(N), float(fov), float(alpha),
                                       float(delta), ctypes.byref(o), ctypes.byref(jid)))
        return jid.value

    def wait(self, job: int, cap: int = 1 << 20) -> dict:
        import numpy as np
        idx = np.empty(max(cap, 1), dtype=np.int32)
        x = np.empty(max(cap, 1), dtype=np.float32)
        st = pc_solve_stats()
        tm = pc_job_times()
        status = load().pc_server_wait(self.handle, int(job), idx.ctypes.data, x.ctypes.data, int(cap),
                                       ctypes.byref(st), ctypes.byref(tm))
        _check(status, allow=(PC_OK, PC_ERR_NOT_CONVERGED))
        n = st.n_support
        return dict(idx=idx[:n].copy(), x=x[:n].copy(), status=st.status, iterations=st.iterations,
                    objective=st.objective, lam=st.lambda_, converged=status == PC_OK,
                    submitted=tm.submitted, admitted=tm.admitted, finished=tm.finished,
                    latency=tm.finished - tm.submitted)

    def close(self):
        if getattr(self, "handle", None):
            load().pc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pc_trim_memory() -> None:
    """Return the library's cached device and pinned memory to the system."""
    _check(load().pc_trim_memory())
