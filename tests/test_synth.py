"""The seeded generators are deterministic and produce the documented shapes."""
import math

import numpy as np

from paper_2406_01342_gb300 import synth


def test_tiny_is_deterministic_and_shaped():
    a, b = synth.tiny_coplanar(), synth.tiny_coplanar()
    assert np.array_equal(a.uvw, b.uvw) and np.array_equal(a.noise, b.noise)
    assert a.uvw.shape == (2000, 3) and np.all(a.uvw[:, 2] == 0)
    R = 64.0 / (2 * a.N * a.dl)
    assert np.all(np.hypot(a.uvw[:, 0], a.uvw[:, 1]) <= R)
    assert a.sky_idx.size == 5 and np.all(np.diff(a.sky_idx) > 0)
    assert np.all((a.sky_flux >= 1) & (a.sky_flux <= 10))


def test_medium_layout_shape():
    wl = synth.medium_512(M=5000)
    assert wl.uvw.shape == (5000, 3)
    # baselines within 2 x 3 km at 100 MHz (3 m wavelength)
    assert np.max(np.linalg.norm(wl.uvw, axis=1)) <= 6000.0 / 2.99792458 + 1e-6
    assert np.abs(wl.uvw[:, 2]).max() > 10.0          # nonzero w
    assert wl.sky_idx.size == 50


def test_unit_noise_power():
    rng = np.random.default_rng(0)
    e = synth.unit_complex_noise(200_000, rng)
    assert abs(np.mean(np.abs(e) ** 2) - 1.0) < 0.01
    assert math.isclose(synth.noise_sigma(4.0, 20.0), 0.2)
