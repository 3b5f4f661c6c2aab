"""GPU parity at the full sizes of the 2048 x 2048 (M = 2M, ~17 w-planes) and
4096 x 4096 (M = 10M) configurations: the operators on seeded samples of
pixels and visibilities that the FP64 oracle computes one by one, and
invariants of the full solve that hold at any size (the oracle cannot solve
these sizes).

The adjoint is checked on seeded white-noise visibilities (no method
arithmetic involved in the input), the forward on a seeded random support.
"""
import numpy as np
import pytest

from oracle import operators
from paper_2406_01342_gb300 import synth
from tests.helpers import rel_l2, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def abi():
    from paper_2406_01342_gb300 import abi as _abi, build
    build.build()
    _abi.load()
    return _abi


@pytest.mark.parametrize("name,n_pix", [("large_2048_w", 40), ("fine_4096_w", 16)])
def test_operators_full_size_sampled(abi, name, n_pix):
    wl = synth.WORKLOADS[name]()
    assert wl.M in (2_000_000, 10_000_000)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    info = abi.pc_plan_info(plan)
    assert info["n_planes"] > 8                      # several plane groups per tile
    rng = np.random.default_rng(31)
    V = synth.unit_complex_noise(wl.M, rng).astype(np.complex64)
    img = abi.pc_adjoint_grid(plan, to_dev(V)).cpu().numpy().ravel()
    N = wl.N
    corners = np.array([0, N - 1, (N - 1) * N, N * N - 1, (N // 2) * N + N // 2])
    pix = np.union1d(np.sort(rng.choice(N * N, n_pix, replace=False)), corners)
    ref = operators.adjoint(wl.uvw, N, wl.fov, V.astype(np.complex128), pix)
    assert rel_l2(img[pix], ref) <= TOL
    # forward on a random 300-atom support, sampled visibilities
    idx = np.sort(rng.choice(N * N, 300, replace=False)).astype(np.int32)
    x = rng.uniform(-1.0, 2.0, 300).astype(np.float32)
    y = abi.pc_forward_sparse(plan, to_dev(idx), to_dev(x)).cpu().numpy()
    ks = np.sort(rng.choice(wl.M, 4000, replace=False))
    yref = operators.forward(wl.uvw[ks], N, wl.fov, idx, x.astype(np.float64))
    assert rel_l2(y[ks], yref) <= TOL
    # the same image through degridding (one-CTA FFT passes at these grid sizes)
    img = torch.zeros(N * N, dtype=torch.float32, device="cuda")
    img[torch.from_numpy(idx.astype(np.int64)).cuda()] = torch.from_numpy(x).cuda()
    y2 = abi.pc_forward_grid(plan, img.view(N, N)).cpu().numpy()
    assert rel_l2(y2[ks], yref) <= TOL


def _physical_vis(abi, plan, wl):
    """Noisy visibilities of the workload's sky, formed with the GPU forward
    operator (no oracle value is involved in these solve tests)."""
    y = abi.pc_forward_sparse(plan, to_dev(wl.sky_idx.astype(np.int32)),
                              to_dev(wl.sky_flux.astype(np.float32)))
    p_sig = float((y.abs() ** 2).mean())
    sigma = np.sqrt(p_sig * 10.0 ** (-wl.snr_db / 10.0))
    return y + to_dev((sigma * wl.noise).astype(np.complex64))


@pytest.mark.parametrize("name", ["large_2048_w", "fine_4096_w", "large_2048_blobs"])
def test_full_size_solve_invariants(abi, name):
    """Algorithm 2 at full size: converges at the 1e-4 stop rule, the objective
    never increases and ends below F(0) = ||V||^2 / 2, the certificate of the
    returned image is ~1 in magnitude on its support (optimality, Sect. 4.2)
    and the brightest true sources are in the support."""
    wl = synth.WORKLOADS[name]()
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    V = _physical_vis(abi, plan, wl)
    lmax = abi.pc_lambda_max(plan, V)
    lam = wl.alpha * lmax
    opts = {"select_rule": 1, "lambda_max": lmax} if wl.rule == "R1" else {}
    res = abi.pc_solve(plan, V, lam, wl.delta, **opts)
    assert res["converged"]
    F = [0.5 * res["sumsq_V"]] + [h["objective"] for h in res["history"]]
    assert all(b <= a * (1 + 1e-7) for a, b in zip(F, F[1:]))
    assert res["objective"] < 0.5 * res["sumsq_V"]
    idx = res["idx"].cpu().numpy()
    x = res["x"].cpu().numpy()
    assert idx.size > 0 and np.isfinite(x).all() and (np.diff(idx) > 0).all()
    mu = res["mu"].cpu().numpy().ravel()
    assert np.abs(np.abs(mu[idx]) - 1.0).max() <= 0.05
    assert np.all(np.sign(mu[idx]) == np.sign(x))
    if wl.rule == "R2":
        bright = wl.sky_idx[np.argsort(wl.sky_flux)[-10:]]
        assert np.isin(bright, idx).all()
    else:
        # diffuse sky: the support lies on the sky (a sparse subset of the
        # blobs' pixels and the point sources), mostly
        assert np.isin(idx, wl.sky_idx).mean() >= 0.5


@pytest.mark.parametrize("name", ["large_2048_blobs", "fine_4096_w"])
def test_full_size_solve_objective_against_the_plain_path(abi, name):
    """The default solve and the solve with every contraction in plain FP32
    (gram_mode 1: another rounding path through the same Algorithm 2) end
    within the 1e-4 relative stop tolerance of each other: a trajectory that
    stops early (a step size below the Lipschitz constant, a premature stop)
    shows up as a gap (3.4e-4 and 6.4e-4 were seen with a Lanczos start that
    could underestimate L)."""
    wl = synth.WORKLOADS[name]()
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    V = _physical_vis(abi, plan, wl)
    lmax = abi.pc_lambda_max(plan, V)
    lam = wl.alpha * lmax
    opts = {"select_rule": 1, "lambda_max": lmax} if wl.rule == "R1" else {}
    a = abi.pc_solve(plan, V, lam, wl.delta, want_mu=False, **opts)
    b = abi.pc_solve(plan, V, lam, wl.delta, want_mu=False, gram_mode=1, **opts)
    assert a["converged"] and b["converged"]
    assert abs(a["objective"] - b["objective"]) <= 1e-4 * b["objective"], (a["objective"], b["objective"],
                                                                          a["iterations"], b["iterations"])


def clustered_atoms(N: int, S: int, rng, n_clusters: int = 8) -> np.ndarray:
    """S distinct pixels in n_clusters square blocks around random centres (the
    shape of a Frank-Wolfe active set, which gathers around bright sources, so
    neighbouring atoms give Gram entries close to the diagonal), sorted."""
    side = int(np.ceil(np.sqrt(S / n_clusters))) + 1
    out = set()
    while len(out) < S:
        ci, cj = rng.integers(side, N - side, 2)
        for di in range(side):
            for dj in range(side):
                if len(out) < S:
                    out.add(int((ci + di) * N + cj + dj))
    return np.array(sorted(out), dtype=np.int32)


def gram_errors(wl, G, b, V, idx, sub):
    """Errors of the Gram entries G[sub][sub] and of b[sub] against the FP64
    oracle's columns (operators.phase_block), each normalised by its
    Cauchy-Schwarz bound: |dG_ij| / sqrt(G_ii G_jj) and |db_i| / (sqrt(G_ii) ||V||)."""
    l, m, n = operators.pixel_lmn(wl.N, wl.fov, idx[sub])
    A = np.empty((wl.M, sub.size), dtype=np.complex128)
    for c in range(sub.size):          # one column at a time keeps the temporaries small
        A[:, c] = operators.phase_block(wl.uvw, l[c:c + 1], m[c:c + 1], n[c:c + 1])[:, 0]
    Gref = np.real(A.conj().T @ A)
    bref = np.real(A.conj().T @ V.astype(np.complex128))
    d = np.sqrt(np.diag(Gref))
    eG = np.abs(G[np.ix_(sub, sub)] - Gref) / np.outer(d, d)
    eb = np.abs(b[sub] - bref) / (d * np.linalg.norm(V))
    return float(eG.max()), float(eb.max())


@pytest.mark.parametrize("name,S", [("medium_512_w", 873), ("large_2048_w", 512), ("fine_4096_w", 512),
                                    ("fine_4096_w", 100)])
def test_tensor_core_gram_sampled_at_full_size(abi, name, S):
    """The split-FP16 tensor-core contraction (pc_gram mode 2) at the
    visibility counts the solves use (M = 200k with 873 atoms, the first Gram of
    the benchmark's solve; M = 2M and 10M with 512; 100 atoms at 10M, a
    single row of A tiles as the solves' incremental Gram rows): 16 seeded
    atoms (two
    clusters' worth of neighbours among them), all their 136 distinct G entries
    and their b entries against the FP64 oracle, within 1e-5 of each entry's
    Cauchy-Schwarz bound. The accumulation drift of the tensor core grows with
    the number of MMA adds, which these sizes exercise (8192-visibility slices
    of 256-visibility sub-slices, phase-buffer chunks at 10M)."""
    wl = synth.WORKLOADS[name]()
    rng = np.random.default_rng(47)
    idx = clustered_atoms(wl.N, S, rng)
    V = synth.unit_complex_noise(wl.M, rng).astype(np.complex64)
    plan = abi.pc_plan_create(to_dev(wl.uvw), wl.N, wl.fov)
    G, b = abi.pc_gram(plan, to_dev(V), to_dev(idx), mode=2)
    G = G.cpu().numpy().astype(np.float64)
    b = b.cpu().numpy().astype(np.float64)
    assert np.array_equal(G, G.T)
    sub = np.sort(np.concatenate([np.arange(8), rng.choice(np.arange(8, S), 8, replace=False)]))
    eG, eb = gram_errors(wl, G, b, V, idx, sub)
    assert eG <= 1e-5, eG
    assert eb <= 1e-5, eb
