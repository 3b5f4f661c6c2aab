"""The allocation-free entry point pc_adjoint_sparse_noalloc, for callers that
cannot allocate device memory (fixed arenas, real-time pipelines, hosts that
forbid allocation while work is queued).

It is called through the C ABI on two consecutive calls (its shared scratch
array keeps the previous call's contents, so the second call checks that each
call clears what it reuses) and compared both with the FP64 oracle's direct
sum and with the plan-based pc_adjoint_sparse, within the operators'
tolerance (1e-5 relative L2). Also: NaN in exactly the slots whose index is
outside the image, zeros when there are no visibilities, a call on a side
stream, and the size limits. This file sorts last so a run that stops at the
first failure has already run every other test; it also passes alone in a
fresh process.
"""
import numpy as np
import pytest

from oracle import operators
from tests.helpers import rel_l2, to_dev, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


def test_noalloc_matches_oracle_and_plan_path_on_two_calls(abi):
    wl, V = workload("small_wide_w")
    uvw = to_dev(wl.uvw)
    Vs = V.astype(np.complex64)
    Vd = to_dev(Vs)
    plan = abi.pc_plan_create(uvw, wl.N, wl.fov)
    rng = np.random.default_rng(21)
    for call in range(2):
        S = 300 if call == 0 else 257          # the second call uses fewer pixels of the scratch
        idx_h = np.sort(rng.choice(wl.N * wl.N, S, replace=False)).astype(np.int32)
        idx = to_dev(idx_h)
        out = torch.full((S,), float("nan"), dtype=torch.float32, device="cuda")
        abi.pc_adjoint_sparse_noalloc(uvw, wl.N, wl.fov, Vd, idx, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        ref = operators.adjoint(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128), idx_h)
        assert rel_l2(got, ref) <= 1e-5, (call, rel_l2(got, ref))
        plan_out = abi.pc_adjoint_sparse(plan, Vd, idx).cpu().numpy()
        assert rel_l2(got, plan_out) <= 1e-5, (call, rel_l2(got, plan_out))


def test_noalloc_out_of_range_indices_give_nan_only_there(abi):
    wl, V = workload("tiny_64_coplanar")
    Vs = V.astype(np.complex64)
    NN = wl.N * wl.N
    idx_h = np.array([5, -1, 2080, NN, 4000, NN + 7, -300, 17], dtype=np.int32)
    bad = (idx_h < 0) | (idx_h >= NN)
    out = torch.zeros(idx_h.size, dtype=torch.float32, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):                # a non-default stream
        abi.pc_adjoint_sparse_noalloc(to_dev(wl.uvw), wl.N, wl.fov, to_dev(Vs), to_dev(idx_h), out,
                                      stream=side)
    side.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(np.isnan(got), bad)
    ref = operators.adjoint(wl.uvw, wl.N, wl.fov, Vs.astype(np.complex128), idx_h[~bad])
    assert rel_l2(got[~bad], ref) <= 1e-5


def test_noalloc_without_visibilities_gives_zeros(abi):
    idx = to_dev(np.array([0, 10, 4095], dtype=np.int32))
    out = torch.full((3,), 7.0, dtype=torch.float32, device="cuda")
    abi.pc_adjoint_sparse_noalloc(torch.zeros(0, 3, dtype=torch.float64, device="cuda"), 64, 0.01,
                                  torch.zeros(0, dtype=torch.complex64, device="cuda"), idx, out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0, 0.0]


def test_noalloc_rejects_more_pixels_than_its_scratch(abi):
    wl, V = workload("tiny_64_coplanar")
    S = 8193
    idx = torch.zeros(S, dtype=torch.int32, device="cuda")
    out = torch.zeros(S, dtype=torch.float32, device="cuda")
    with pytest.raises(abi.PcError) as e:
        abi.pc_adjoint_sparse_noalloc(to_dev(wl.uvw), wl.N, wl.fov, to_dev(V.astype(np.complex64)),
                                      idx, out)
    assert e.value.status == abi.PC_ERR_INVALID_ARG
    assert "at most 8192" in str(e.value)


def test_noalloc_rejects_more_visibilities_than_one_launch_takes(abi):
    """M beyond 65535 x 8192 is refused before any pointer is read."""
    import ctypes
    lib = abi.load()
    idx = to_dev(np.array([0], dtype=np.int32))
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    M = 65535 * 8192 + 1
    st = lib.pc_adjoint_sparse_noalloc(None, M, 64, 0.01, None, ctypes.c_void_p(idx.data_ptr()), 1,
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert st == abi.PC_ERR_INVALID_ARG
    assert b"at most" in lib.pc_last_error()
