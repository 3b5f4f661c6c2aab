"""Shared helpers of the test-suite: seeded workloads with oracle visibilities."""
from __future__ import annotations

import functools

import numpy as np

from oracle import operators
from paper_2406_01342_gb300 import synth


def rel_l2(got, ref) -> float:
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


@functools.lru_cache(maxsize=None)
def workload(name: str, **kw):
    """(workload, V) with V = Phi(sky) + noise computed by the FP64 oracle."""
    wl = synth.WORKLOADS[name](**kw)
    Vc = operators.forward(wl.uvw, wl.N, wl.fov, wl.sky_idx, wl.sky_flux)
    V = Vc + synth.noise_sigma(float(np.mean(np.abs(Vc) ** 2)), wl.snr_db) * wl.noise
    return wl, V


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()
