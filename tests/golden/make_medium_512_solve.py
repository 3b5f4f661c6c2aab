#!/usr/bin/env python
"""Writes medium_512_w_solve.json: the FP64 oracle's solve of the 512 x 512,
M = 200k w-stacked workload (the configuration the benchmark times), for the
GPU parity test of the full Frank-Wolfe solve (Algorithm 2, Sect. 5.1).

Only `oracle/` and the seeded input generator are used. The oracle runs as it
stands: `pfw.frank_wolfe` with the pixel atoms of `pfw.solve`; the dirty
residual on all N^2 pixels (`operators.adjoint`) is evaluated over pixel
chunks in a process pool (every chunk is the same direct sum, so the result
is the oracle's). Visibilities: V = Phi(sky) + sigma * noise with the
oracle's forward operator at the workload's SNR, rounded to complex64 (the
precision the GPU receives) and used in that form by both sides.

Stored: lambda, the final support and weights, the objective, per iteration
the active set, the pruned support and the pixels whose certificate lies
within 1e-5 max|mu| of the selection threshold (where an FP32 certificate may
legitimately fall on the other side), and the final certificate at 4096
seeded pixels plus the support. The file records the seeds and this
script's SHA-256; the test refuses a golden written by another version.

    python tests/golden/make_medium_512_solve.py [--workers K]

About an hour on 8 cores (each certificate is 5.2e10 phase evaluations).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "medium_512_w_solve.json")
WORKLOAD = "medium_512_w"
MU_SEED = 20260
MU_PIXELS = 4096

_W = {}


def _init(name: str) -> None:
    sys.path.insert(0, ROOT)
    from paper_2406_01342_gb300 import synth
    wl = synth.WORKLOADS[name]()
    _W.update(uvw=wl.uvw, N=wl.N, fov=wl.fov)


def _adjoint_chunk(args):
    from oracle import operators
    r, idx = args
    return operators.adjoint(_W["uvw"], _W["N"], _W["fov"], r, idx)


def script_sha256() -> str:
    return hashlib.sha256(open(os.path.abspath(__file__), "rb").read()).hexdigest()


def visibilities(wl):
    """V = Phi(sky) + sigma * noise (oracle forward operator), as complex64 values."""
    import numpy as np
    from oracle import operators
    from paper_2406_01342_gb300 import synth
    Vc = operators.forward(wl.uvw, wl.N, wl.fov, wl.sky_idx, wl.sky_flux)
    V = Vc + synth.noise_sigma(float(np.mean(np.abs(Vc) ** 2)), wl.snr_db) * wl.noise
    return V.astype(np.complex64).astype(np.complex128)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--workload", default=WORKLOAD, help="another workload (dry runs)")
    args = ap.parse_args()
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    sys.path.insert(0, ROOT)
    import numpy as np

    from oracle import operators, pfw
    from paper_2406_01342_gb300 import synth

    wl = synth.WORKLOADS[args.workload]()
    N, NN = wl.N, wl.N * wl.N
    V = visibilities(wl)
    chunks = np.array_split(np.arange(NN, dtype=np.int64), 8 * args.workers)
    pool = mp.get_context("spawn").Pool(args.workers, initializer=_init, initargs=(args.workload,))
    n_certs = [0]
    t0 = time.time()

    def eta_all(r):
        n_certs[0] += 1
        out = np.concatenate(pool.map(_adjoint_chunk, [(r, c) for c in chunks]))
        print(f"  certificate {n_certs[0]} ({time.time() - t0:.0f} s)", flush=True)
        return out

    def columns(S):
        l, m, n = operators.pixel_lmn(N, wl.fov, S)
        return operators.phase_block(wl.uvw, l, m, n)

    lmax = float(np.max(np.abs(eta_all(V))))
    lam = wl.alpha * lmax
    S, x, r, F, iters, converged, history = pfw.frank_wolfe(V, lam, eta_all, columns, lmax, wl.delta)
    mu = eta_all(r) / lam
    pool.close()
    pool.join()

    rng = np.random.default_rng(MU_SEED)
    pix = np.union1d(rng.choice(NN, MU_PIXELS, replace=False), S).astype(np.int64)
    hist = []
    for h in history:
        hist.append({k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in h.items()})
    golden = {
        "workload": args.workload, "seed": wl.seed, "mu_seed": MU_SEED, "script_sha256": script_sha256(),
        "N": N, "M": wl.M, "alpha": wl.alpha, "delta": wl.delta, "tol": 1e-4,
        "V_sumsq": float(np.vdot(V, V).real), "lambda_max": lmax, "lambda": lam,
        "support": S.tolist(), "x": x.tolist(), "objective": F, "iterations": iters,
        "converged": bool(converged), "history": hist,
        "mu_pixels": pix.tolist(), "mu": mu[pix].tolist(), "mu_inf": float(np.max(np.abs(mu))),
        "certificates": n_certs[0], "seconds": time.time() - t0,
    }
    with open(args.out, "w") as f:
        json.dump(golden, f, separators=(",", ":"))
    print(f"wrote {args.out}: {iters} iterations, support {S.size}, F = {F:.10g}")


if __name__ == "__main__":
    main()
