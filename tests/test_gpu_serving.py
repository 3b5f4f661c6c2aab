"""The serving loop (continuous batching of imaging requests): every result in
a mixed stream equals the result of the same request solved alone, admission
follows the memory budget, batched and per-job reweighting give the same
solves, and bad requests are refused."""
import numpy as np
import pytest

from tests.helpers import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


def _requests():
    """Requests of different grid and visibility sizes (visibilities from the
    oracle's forward model, so no request depends on the CUDA path)."""
    out = []
    for name, kw, opts in [("tiny_64_coplanar", {}, {}),
                           ("small_wide_w", {}, {}),
                           ("medium_512_w", {"M": 20_000}, {}),
                           ("tiny_64_coplanar", {}, {"positivity": 1}),
                           ("medium_512_w", {"M": 40_000}, {}),
                           ("small_wide_w", {}, {"select_rule": 1})]:
        wl, V = workload(name, **kw)
        delta = 0.9 if opts.get("select_rule") == 1 else wl.delta
        out.append((wl, V.astype(np.complex64), delta, opts))
    return out


def _same(a, b):
    assert a["idx"].tolist() == b["idx"].tolist()
    assert abs(a["objective"] - b["objective"]) <= 1e-6 * abs(b["objective"])
    assert np.allclose(a["x"], b["x"], rtol=1e-4, atol=1e-6 * np.abs(b["x"]).max(initial=0.0))


@pytest.mark.parametrize("batch_apgd", [1, 2])
def test_mixed_stream_equals_alone(abi, batch_apgd):
    reqs = _requests()
    alone = [abi.pc_solve_host(wl.uvw, V, wl.N, wl.fov, wl.alpha, delta, **opts)
             for wl, V, delta, opts in reqs]
    srv = abi.Server(max_jobs=3, batch_apgd=batch_apgd)
    try:
        ids = [srv.submit(wl.uvw, V, wl.N, wl.fov, wl.alpha, delta, **opts) for wl, V, delta, opts in reqs]
        got = [srv.wait(j) for j in ids]
    finally:
        srv.close()
    for g, a in zip(got, alone):
        _same(g, a)
        assert g["converged"] and g["finished"] >= g["admitted"] >= g["submitted"]
    # with three slots the later requests waited for earlier ones to finish
    assert max(g["admitted"] for g in got) >= min(g["finished"] for g in got)


def test_admission_follows_the_memory_budget(abi):
    """A budget smaller than any job admits one job at a time, in order."""
    reqs = _requests()[:3]
    srv = abi.Server(max_jobs=8, memory_budget=1)
    try:
        ids = [srv.submit(wl.uvw, V, wl.N, wl.fov, wl.alpha, delta, **opts) for wl, V, delta, opts in reqs]
        got = [srv.wait(j) for j in ids]
    finally:
        srv.close()
    for prev, nxt in zip(got, got[1:]):
        assert nxt["admitted"] >= prev["finished"]
    alone = abi.pc_solve_host(reqs[0][0].uvw, reqs[0][1], reqs[0][0].N, reqs[0][0].fov,
                              reqs[0][0].alpha, reqs[0][2])
    _same(got[0], alone)


def test_bad_requests_are_refused(abi):
    wl, V, delta, _ = _requests()[0]
    srv = abi.Server(max_jobs=2)
    try:
        with pytest.raises(abi.PcError) as e:
            srv.submit(wl.uvw, V, 63, wl.fov, wl.alpha, delta)          # odd N
        assert e.value.status == abi.PC_ERR_INVALID_ARG
        with pytest.raises(abi.PcError) as e:
            srv.submit(wl.uvw, V, wl.N, wl.fov, 1.5, delta)             # alpha > 1
        assert e.value.status == abi.PC_ERR_INVALID_ARG
        with pytest.raises(abi.PcError) as e:
            srv.wait(12345)
        assert e.value.status == abi.PC_ERR_INVALID_ARG
        j = srv.submit(wl.uvw, V, wl.N, wl.fov, wl.alpha, delta)
        assert srv.wait(j)["converged"]
        with pytest.raises(abi.PcError):
            srv.wait(j)                                                # collected already
    finally:
        srv.close()
