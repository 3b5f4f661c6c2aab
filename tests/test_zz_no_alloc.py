"""The allocation-free entry point pc_adjoint_sparse_noalloc, for callers that
cannot allocate device memory (fixed arenas, real-time pipelines, hosts that
forbid allocation while work is queued).

It is called through the C ABI on two consecutive calls (its shared scratch
array keeps the previous call's contents, so the second call checks that each
call clears what it reuses) and compared with the plan-based pc_adjoint_sparse
within the operators' tolerance (1e-5 relative L2). This file sorts last so a
run that stops at the first failure has already run every other test; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest

from tests.helpers import rel_l2, to_dev, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


def test_noalloc_matches_plan_path_on_two_calls(abi):
    wl, V = workload("small_wide_w")
    uvw = to_dev(wl.uvw)
    Vd = to_dev(V.astype(np.complex64))
    plan = abi.pc_plan_create(uvw, wl.N, wl.fov)
    rng = np.random.default_rng(21)
    for call in range(2):
        S = 300 if call == 0 else 257          # the second call uses fewer pixels of the scratch
        idx = to_dev(np.sort(rng.choice(wl.N * wl.N, S, replace=False)).astype(np.int32))
        ref = abi.pc_adjoint_sparse(plan, Vd, idx).cpu().numpy()
        out = torch.full((S,), float("nan"), dtype=torch.float32, device="cuda")
        abi.pc_adjoint_sparse_noalloc(uvw, wl.N, wl.fov, Vd, idx, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) <= 1e-5, (call, rel_l2(got, ref))


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
