"""GPU parity of the operators (the forward and adjoint equations of Sect. 2.2,
the certificate of Sect. 4.2, lambda_max of Sect. 5.3) against the FP64 oracle.

Tolerance: relative L2 error <= 1e-5 for every operator output (FP32 kernels
against FP64 direct sums), as the accuracy target of the hot path states.
"""
import math

import numpy as np
import pytest

from oracle import operators
from tests.helpers import rel_l2, to_dev, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


CASES = [("tiny_64_coplanar", {}), ("small_wide_w", {}), ("medium_512_w", {"M": 20_000})]


def _plan(abi, wl, **kw):
    return abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov, **kw)


@pytest.mark.parametrize("name,kw", CASES)
def test_plan_geometry(abi, name, kw):
    wl, V = workload(name, **kw)
    plan = _plan(abi, wl)
    info = abi.pc_plan_info(plan)
    assert info["grid_side"] >= 2 * wl.N and info["grid_side"] % info["tile"] == 0
    assert wl.M <= info["n_slots"] <= 4 * wl.M
    if np.all(wl.uvw[:, 2] == 0):
        assert info["n_planes"] == 1
    else:
        assert info["n_planes"] > info["kernel_width"]


@pytest.mark.parametrize("name,kw", CASES)
def test_forward_sparse(abi, name, kw):
    wl, V = workload(name, **kw)
    plan = _plan(abi, wl)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(wl.N * wl.N, 37, replace=False)).astype(np.int32)
    x = rng.normal(size=37).astype(np.float32)
    y = abi.pc_forward_sparse(plan, to_dev(idx), to_dev(x)).cpu().numpy()
    ref = operators.forward(wl.uvw, wl.N, wl.fov, idx, x.astype(np.float64))
    assert rel_l2(y, ref) <= TOL


@pytest.mark.parametrize("grid_mode", [1, 2, 3])
@pytest.mark.parametrize("name,kw", CASES)
def test_adjoint_grid(abi, name, kw, grid_mode):
    """Gridding on FP32 CUDA cores (1), on the tensor cores with split-FP16
    operands (2; w-stacked plans) and on FP32 CUDA cores over plane windows
    with one CTA per tile (3; w-stacked plans), then FFT and epilogue, against
    the direct sum."""
    wl, V = workload(name, **kw)
    plan = _plan(abi, wl, grid_mode=grid_mode)
    img = abi.pc_adjoint_grid(plan, to_dev(V.astype(np.complex64))).cpu().numpy().ravel()
    if wl.N <= 64:
        pix = np.arange(wl.N * wl.N)
    else:
        pix = np.sort(np.random.default_rng(4).choice(wl.N * wl.N, 2048, replace=False))
    ref = operators.adjoint(wl.uvw, wl.N, wl.fov, V.astype(np.complex64).astype(np.complex128), pix)
    assert rel_l2(img[pix], ref) <= TOL


@pytest.mark.parametrize("name,kw", [("small_wide_w", {"N": 200}), ("small_wide_w", {"N": 256}),
                                     ("small_wide_w", {"N": 300}), ("diffuse_256", {}),
                                     ("medium_512_w", {"M": 20_000}),
                                     ("tiny_64_coplanar", {"N": 256}), ("tiny_64_coplanar", {"N": 512})])
def test_fft_kernels(abi, name, kw):
    """The FFT passes of the adjoint on one warp per row in registers (the
    default at G = 512 and 1024) and on shared-memory Stockham stages
    (fft_kernel = 1): each meets the tolerance against the direct sum on the
    image's border rows and columns and on random pixels, and the two agree
    on the whole image. N = 200 and 300 leave part of the kept band empty;
    the coplanar cases (one plane, no w-screen) put eight image rows in each
    CTA of the second pass."""
    wl, V = workload(name, **kw)
    Vd = to_dev(V.astype(np.complex64))
    pw, ps = _plan(abi, wl), _plan(abi, wl, fft_kernel=1)
    assert abi.pc_plan_info(pw)["grid_side"] in (512, 1024)
    assert abi.pc_plan_tuning_info(pw)["fft_warp"] == 3
    assert abi.pc_plan_tuning_info(ps)["fft_warp"] == 0
    aw = abi.pc_adjoint_grid(pw, Vd).cpu().numpy().ravel()
    as_ = abi.pc_adjoint_grid(ps, Vd).cpu().numpy().ravel()
    N = wl.N
    border = np.concatenate([np.arange(N), (N - 1) * N + np.arange(N), np.arange(N) * N,
                             np.arange(N) * N + N - 1])
    pix = np.union1d(border, np.random.default_rng(5).choice(N * N, 1024, replace=False))
    ref = operators.adjoint(wl.uvw, N, wl.fov, V.astype(np.complex64).astype(np.complex128), pix)
    assert rel_l2(aw[pix], ref) <= TOL
    assert rel_l2(as_[pix], ref) <= TOL
    assert rel_l2(aw, as_) <= TOL


@pytest.mark.parametrize("grid_mode", [2, 3])
@pytest.mark.parametrize("name,kw", CASES)
def test_forward_grid(abi, name, kw, grid_mode):
    """Degridding (the type-2 non-uniform FFT of Sect. 5.2) of a dense random
    image against the direct sum of the forward equation (Sect. 2.2), on all
    visibilities or a seeded sample of them; grid_mode 3 interpolates over the
    plane windows (one thread per binned slot), 2 over the fixed plane groups
    (the coplanar case has one plane and takes the latter in both)."""
    wl, V = workload(name, **kw)
    plan = _plan(abi, wl, grid_mode=grid_mode)
    rng = np.random.default_rng(31)
    img = rng.normal(size=(wl.N, wl.N)).astype(np.float32)
    y = abi.pc_forward_grid(plan, to_dev(img)).cpu().numpy()
    ks = np.arange(wl.M) if wl.N * wl.N * wl.M <= 5e7 else np.sort(rng.choice(wl.M, 2000, replace=False))
    ref = operators.forward(wl.uvw[ks], wl.N, wl.fov, np.arange(wl.N * wl.N), img.ravel().astype(np.float64))
    assert rel_l2(y[ks], ref) <= TOL


@pytest.mark.parametrize("fft_kernel", [0, 1])
@pytest.mark.parametrize("name,kw", [("small_wide_w", {"N": 200}), ("small_wide_w", {"N": 300}),
                                     ("diffuse_256", {}), ("tiny_64_coplanar", {"N": 256})])
def test_forward_grid_fft_kernels(abi, name, kw, fft_kernel):
    """Degridding with one-warp register FFTs (default at G = 512 and 1024)
    and with the Stockham passes (fft_kernel = 1), N = 200 and 300 leaving
    part of the length-G rows empty: against the direct sum on every
    visibility, and the adjoint identity with the same plan's gridding."""
    wl, _ = workload(name, **kw)
    plan = _plan(abi, wl, fft_kernel=fft_kernel)
    assert abi.pc_plan_tuning_info(plan)["fft_warp"] == (0 if fft_kernel else 3)
    rng = np.random.default_rng(33)
    img = rng.normal(size=(wl.N, wl.N)).astype(np.float32)
    y = abi.pc_forward_grid(plan, to_dev(img)).cpu().numpy()
    ks = np.sort(rng.choice(wl.M, min(wl.M, 3000), replace=False))
    ref = operators.forward(wl.uvw[ks], wl.N, wl.fov, np.arange(wl.N * wl.N), img.ravel().astype(np.float64))
    assert rel_l2(y[ks], ref) <= TOL
    h = (rng.normal(size=wl.M) + 1j * rng.normal(size=wl.M)).astype(np.complex64)
    g = abi.pc_adjoint_grid(plan, to_dev(h)).cpu().numpy().astype(np.float64)
    lhs = float(np.real(np.vdot(y.astype(np.complex128), h.astype(np.complex128))))
    rhs = float(np.sum(img.astype(np.float64) * g))
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(np.abs(y) ** 2) * np.sum(np.abs(h) ** 2))


BIG = [("small_wide_w", {"N": 600}), ("tiny_64_coplanar", {"N": 1024}), ("small_wide_w", {"N": 1100}),
       ("small_wide_w", {"N": 2100})]


@pytest.mark.parametrize("name,kw", BIG)
def test_fft_big_kernels(abi, name, kw):
    """The one-CTA FFT passes (the default at G = 2048, 4096 and 8192, with
    the pass-1 rows stored compactly) against the direct sum on the image's
    border rows and columns and random pixels, and against the shared-memory
    Stockham passes (fft_kernel = 1) on the whole image. N = 600, 1100 and
    2100 leave part of the kept band empty; the coplanar case has one plane."""
    wl, V = workload(name, **kw)
    Vd = to_dev(V.astype(np.complex64))
    pb, ps = _plan(abi, wl), _plan(abi, wl, fft_kernel=1)
    assert abi.pc_plan_info(pb)["grid_side"] in (2048, 4096, 8192)
    assert abi.pc_plan_tuning_info(pb)["fft_warp"] == 3
    assert abi.pc_plan_tuning_info(ps)["fft_warp"] == 0
    ab = abi.pc_adjoint_grid(pb, Vd).cpu().numpy().ravel()
    as_ = abi.pc_adjoint_grid(ps, Vd).cpu().numpy().ravel()
    N = wl.N
    border = np.concatenate([np.arange(N), (N - 1) * N + np.arange(N), np.arange(N) * N,
                             np.arange(N) * N + N - 1])
    pix = np.union1d(border, np.random.default_rng(5).choice(N * N, 1024, replace=False))
    ref = operators.adjoint(wl.uvw, N, wl.fov, V.astype(np.complex64).astype(np.complex128), pix)
    assert rel_l2(ab[pix], ref) <= TOL
    assert rel_l2(as_[pix], ref) <= TOL
    assert rel_l2(ab, as_) <= TOL


@pytest.mark.parametrize("name,kw", BIG)
def test_forward_grid_big(abi, name, kw):
    """Degridding through the one-CTA FFT passes: against the direct sum of
    the forward equation on sampled visibilities (a random image on a random
    fifth of the pixels), and the adjoint identity with the same plan's
    gridding."""
    wl, _ = workload(name, **kw)
    plan = _plan(abi, wl)
    rng = np.random.default_rng(34)
    NN = wl.N * wl.N
    on = np.sort(rng.choice(NN, NN // 5, replace=False))
    img = np.zeros(NN, dtype=np.float32)
    img[on] = rng.normal(size=on.size).astype(np.float32)
    img = img.reshape(wl.N, wl.N)
    y = abi.pc_forward_grid(plan, to_dev(img)).cpu().numpy()
    ks = np.sort(rng.choice(wl.M, 400 if wl.N <= 1100 else 120, replace=False))
    ref = operators.forward(wl.uvw[ks], wl.N, wl.fov, on, img.ravel()[on].astype(np.float64))
    assert rel_l2(y[ks], ref) <= TOL
    h = (rng.normal(size=wl.M) + 1j * rng.normal(size=wl.M)).astype(np.complex64)
    g = abi.pc_adjoint_grid(plan, to_dev(h)).cpu().numpy().astype(np.float64)
    lhs = float(np.real(np.vdot(y.astype(np.complex128), h.astype(np.complex128))))
    rhs = float(np.sum(img.astype(np.float64) * g))
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(np.abs(y) ** 2) * np.sum(np.abs(h) ** 2))


@pytest.mark.parametrize("grid_mode", [2, 3])
@pytest.mark.parametrize("name,kw", CASES)
def test_forward_grid_is_the_adjoint_of_adjoint_grid(abi, name, kw, grid_mode):
    """Re<Phi x, h> = <x, Phi* h> between the two NUFFT directions of one plan
    (they are built as exact adjoints: equal up to FP32 rounding)."""
    wl, _ = workload(name, **kw)
    plan = _plan(abi, wl, grid_mode=grid_mode)
    rng = np.random.default_rng(32)
    x = rng.normal(size=(wl.N, wl.N)).astype(np.float32)
    h = (rng.normal(size=wl.M) + 1j * rng.normal(size=wl.M)).astype(np.complex64)
    y = abi.pc_forward_grid(plan, to_dev(x)).cpu().numpy().astype(np.complex128)
    g = abi.pc_adjoint_grid(plan, to_dev(h)).cpu().numpy().astype(np.float64)
    lhs = float(np.real(np.vdot(y, h.astype(np.complex128))))
    rhs = float(np.sum(x.astype(np.float64) * g))
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(np.sum(np.abs(y) ** 2) * np.sum(np.abs(h) ** 2))


@pytest.mark.parametrize("name,kw", CASES[:2])
def test_adjoint_sparse(abi, name, kw):
    wl, V = workload(name, **kw)
    plan = _plan(abi, wl)
    idx = np.sort(np.random.default_rng(5).choice(wl.N * wl.N, 300, replace=False)).astype(np.int32)
    Vs = V.astype(np.complex64)
    out = abi.pc_adjoint_sparse(plan, to_dev(Vs), to_dev(idx)).cpu().numpy()
    ref = operators.adjoint(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128), idx)
    assert rel_l2(out, ref) <= TOL


def test_lambda_max_and_certificate(abi):
    wl, V = workload("small_wide_w")
    plan = _plan(abi, wl)
    Vs = V.astype(np.complex64)
    Vd = to_dev(Vs)
    lmax = abi.pc_lambda_max(plan, Vd)
    ref_lmax = operators.lambda_max(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128))
    assert abs(lmax - ref_lmax) <= TOL * ref_lmax
    lam = 0.1 * ref_lmax
    idx = wl.sky_idx.astype(np.int32)
    x = wl.sky_flux.astype(np.float32)
    mu, mu_inf, sumsq = abi.pc_certificate(plan, Vd, to_dev(idx), to_dev(x), lam)
    ref = operators.certificate(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128), lam, idx,
                                x.astype(np.float64))
    assert rel_l2(mu.cpu().numpy().ravel(), ref) <= TOL
    assert abs(mu_inf - np.abs(ref).max()) <= 1e-4 * np.abs(ref).max()
    r = operators.residual(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128), idx, x.astype(np.float64))
    assert abs(sumsq - np.vdot(r, r).real) <= 1e-5 * np.vdot(r, r).real


@pytest.mark.parametrize("mode,S,name,kw", [(1, 150, "small_wide_w", {}),
                                            (2, 150, "small_wide_w", {}),
                                            (2, 300, "medium_512_w", {"M": 20_000}),
                                            (2, 37, "tiny_64_coplanar", {})])
def test_gram_and_b(abi, mode, S, name, kw):
    """Support contraction: FP32 CUDA cores (mode 1) and split-FP16 tcgen05 tensor
    cores (mode 2), several tiles and a ragged tail, against the FP64 Gram."""
    wl, V = workload(name, **kw)
    plan = _plan(abi, wl)
    idx = np.sort(np.random.default_rng(6).choice(wl.N * wl.N, S, replace=False)).astype(np.int32)
    Vs = V.astype(np.complex64)
    G, b = abi.pc_gram(plan, to_dev(Vs), to_dev(idx), mode=mode)
    l, m, n = operators.pixel_lmn(wl.N, wl.fov, idx)
    A = operators.phase_block(wl.uvw, l, m, n)
    Gref = np.real(A.conj().T @ A)
    bref = np.real(A.conj().T @ Vs.astype(np.complex128))
    Gg = G.cpu().numpy()
    assert np.array_equal(Gg, Gg.T)
    assert rel_l2(Gg, Gref) <= TOL
    assert rel_l2(b.cpu().numpy(), bref) <= TOL


def test_select_is_exact(abi):
    """Exploration + union (Algorithm 2 steps 1a/1b): index work, bit-exact."""
    wl, V = workload("tiny_64_coplanar")
    plan = _plan(abi, wl)
    rng = np.random.default_rng(7)
    mu = rng.normal(size=(wl.N, wl.N)).astype(np.float32)
    prev = np.sort(rng.choice(wl.N * wl.N, 40, replace=False)).astype(np.int32)
    thr = np.float32(1.9)
    out = abi.pc_select(plan, to_dev(mu), float(thr), to_dev(prev), 4096).cpu().numpy()
    ref = np.union1d(np.nonzero(np.abs(mu.ravel()) >= thr)[0], prev)
    assert out.tolist() == ref.tolist()
    with pytest.raises(abi.PcError) as e:
        abi.pc_select(plan, to_dev(mu), float(thr), to_dev(prev), 10)
    assert e.value.status == abi.PC_ERR_CAPACITY


def test_empty_and_degenerate(abi):
    wl, V = workload("tiny_64_coplanar")
    # M = 0: every operator returns zeros
    empty = abi.pc_plan_create(torch.zeros(0, 3, dtype=torch.float64, device="cuda"), 32, 0.01)
    img = abi.pc_adjoint_grid(empty, torch.zeros(0, dtype=torch.complex64, device="cuda"))
    assert float(img.abs().max()) == 0.0
    plan = _plan(abi, wl)
    # empty support: Phi x = 0
    y = abi.pc_forward_sparse(plan, torch.zeros(0, dtype=torch.int32, device="cuda"),
                              torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert float(y.abs().max()) == 0.0
    # host pointers are rejected, never computed on the CPU
    with pytest.raises(ValueError):
        abi.pc_adjoint_grid(plan, torch.zeros(wl.M, dtype=torch.complex64))
    # invalid support (not ascending)
    with pytest.raises(abi.PcError) as e:
        abi.pc_forward_sparse(plan, to_dev(np.array([5, 3], np.int32)), to_dev(np.ones(2, np.float32)))
    assert e.value.status == abi.PC_ERR_INVALID_ARG
    with pytest.raises(abi.PcError):
        abi.pc_plan_create(to_dev(wl.uvw), 63, wl.fov)


@pytest.mark.parametrize("grid_mode", [1, 2, 3])
def test_full_size_medium_sampled(abi, grid_mode):
    """The 512 x 512, M = 200k workload timed by the benchmark: operators on
    seeded samples of pixels and visibilities (window gridding splits the
    heavy tiles near the uv origin into parts here)."""
    wl, V = workload("medium_512_w")
    plan = _plan(abi, wl, grid_mode=grid_mode)
    Vs = V.astype(np.complex64)
    img = abi.pc_adjoint_grid(plan, to_dev(Vs)).cpu().numpy().ravel()
    rng = np.random.default_rng(8)
    pix = np.sort(rng.choice(wl.N * wl.N, 1024, replace=False))
    pix = np.union1d(pix, wl.sky_idx)                      # include the brightest pixels
    ref = operators.adjoint(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128), pix)
    assert rel_l2(img[pix], ref) <= TOL
    y = abi.pc_forward_sparse(plan, to_dev(wl.sky_idx), to_dev(wl.sky_flux.astype(np.float32))).cpu().numpy()
    ks = np.sort(rng.choice(wl.M, 20_000, replace=False))
    yref = operators.forward(wl.uvw[ks], wl.N, wl.fov, wl.sky_idx, wl.sky_flux.astype(np.float32).astype(np.float64))
    assert rel_l2(y[ks], yref) <= TOL


def test_autotuned_plan(abi):
    """A plan with autotune = 1 times the gridding variants (tensor / CUDA
    cores x sub-problem size) and the FFT row pass on its own layout, keeps a
    valid choice, and its adjoint still meets the operator tolerance."""
    wl, V = workload("medium_512_w", M=60_000)
    plan = _plan(abi, wl, autotune=1)
    t = abi.pc_plan_tuning_info(plan)
    assert t["tuned"] and t["grid_mode"] in (1, 2, 3)
    assert t["grid_piece"] in ((1024, 4096, 16384, 65536) if t["grid_mode"] == 3 else (256, 512, 1024, 2048, 4096))
    assert t["fft_rows_per_cta"] in (1, 2, 4, 8, 16, 32)
    assert 0 < t["grid_us"] < 1e5 and 0 < t["fft_rows_us"] < 1e5
    assert t["fft_cols_planes"] in (1, 2, 4, 8) and 0 < t["fft_cols_us"] < 1e5
    assert t["fft_warp"] in (0, 1, 2, 3)
    if t["grid_mode"] == 3:
        assert t["degrid_piece"] in (2048, 4096, 8192, 16384) and 0 < t["degrid_us"] < 1e5
    else:
        assert t["degrid_piece"] == 0
    if t["fft_warp"] & 1:
        assert t["fft_rows_per_cta"] == 8
    if t["fft_warp"] & 2:
        assert t["fft_cols_planes"] == 1
    assert not abi.pc_plan_tuning_info(_plan(abi, wl))["tuned"]
    Vs = V.astype(np.complex64)
    img = abi.pc_adjoint_grid(plan, to_dev(Vs)).cpu().numpy().ravel()
    pix = np.union1d(np.sort(np.random.default_rng(9).choice(wl.N * wl.N, 1024, replace=False)), wl.sky_idx)
    ref = operators.adjoint(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128), pix)
    assert rel_l2(img[pix], ref) <= TOL
    # the degridding with the tuned choice: a random image on sampled visibilities
    rng = np.random.default_rng(10)
    x = rng.normal(size=(wl.N, wl.N)).astype(np.float32)
    y = abi.pc_forward_grid(plan, to_dev(x)).cpu().numpy()
    ks = np.sort(rng.choice(wl.M, 300, replace=False))
    yref = operators.forward(wl.uvw[ks], wl.N, wl.fov, np.arange(wl.N * wl.N), x.ravel().astype(np.float64))
    assert rel_l2(y[ks], yref) <= TOL
    with pytest.raises(abi.PcError) as e:
        _plan(abi, wl, autotune=2)
    assert e.value.status == abi.PC_ERR_INVALID_ARG


def test_tensor_core_bounded_wait_reports_timeout(abi):
    """Failure detection without a GPU fault: with its MMAs withheld (mode 3) the
    tensor-core kernel's bounded mbarrier wait expires, the kernel frees its
    tensor memory and returns, the host reports PC_ERR_TIMEOUT, and the context
    keeps working."""
    wl, V = workload("small_wide_w")
    plan = _plan(abi, wl)
    idx = np.sort(np.random.default_rng(6).choice(wl.N * wl.N, 150, replace=False)).astype(np.int32)
    with pytest.raises(abi.PcError) as e:
        abi.pc_gram(plan, to_dev(V.astype(np.complex64)), to_dev(idx), mode=3)
    assert e.value.status == abi.PC_ERR_TIMEOUT
    G, b = abi.pc_gram(plan, to_dev(V.astype(np.complex64)), to_dev(idx), mode=2)
    assert np.isfinite(G.cpu().numpy()).all()
