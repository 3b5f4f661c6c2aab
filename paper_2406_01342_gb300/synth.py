"""Seeded synthetic inputs shaped like the paper's workloads (Sect. 6, Table 1 and Table 3).

This module is the only code shared by the FP64 oracle and the CUDA path. It
draws random numbers and does array geometry (station layouts, Earth-rotation
baselines, pixel positions of point sources, unit noise). It holds none of the
imaging method's arithmetic: no measurement operator, no adjoint, no solver.
Each side forms the visibilities V = Phi(I) + sigma * noise with its own
operator, from the arrays produced here.

Conventions (shared by both sides, stated here once):
  * uvw: float64 array of shape (M, 3), row-major, in wavelengths.
  * Image: N x N, raster index p = i * N + j, i indexes l and j indexes m,
    with l_i = (i - N/2) * fov / N and m_j = (j - N/2) * fov / N (radians of
    direction cosine; the paper only says "uniform fine grid", Sect. 2.2).
  * Sky: sorted unique raster indices (int32) and fluxes (float64, Jy/pixel).
  * Noise: complex white Gaussian with E|e|^2 = 1 (each of Re, Im has variance 1/2);
    the caller scales it to the SNR it needs (Sect. 2.1, noise model).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0


@dataclasses.dataclass
class Workload:
    """One synthetic imaging problem."""

    name: str
    N: int                    # image side in pixels
    fov: float                # full side of the field of view, radians (direction cosine)
    uvw: np.ndarray           # (M, 3) float64, wavelengths
    sky_idx: np.ndarray       # (K,) int32 sorted raster indices of the true sources
    sky_flux: np.ndarray      # (K,) float64 fluxes
    noise: np.ndarray         # (M,) complex128 unit-power noise realisation
    snr_db: float             # SNR in dB: noise power = mean|V_clean|^2 * 10^(-snr/10)
    alpha: float              # lambda = alpha * lambda_max (Sect. 5.3)
    delta: float              # exploration quality parameter of the PFW select
    seed: int
    rule: str = "R2"          # exploration rule: "R2" |mu| >= 1 - delta, "R1" Algorithm 2's own set

    @property
    def M(self) -> int:
        return int(self.uvw.shape[0])

    @property
    def dl(self) -> float:
        return self.fov / self.N


def noise_sigma(v_clean_mean_power: float, snr_db: float) -> float:
    """Noise standard deviation for a target SNR: sigma^2 = P_signal * 10^(-SNR/10)."""
    return math.sqrt(v_clean_mean_power * 10.0 ** (-snr_db / 10.0))


# ---------------------------------------------------------------- layouts

def stations_uniform_disk(n_stations: int, radius_m: float, rng: np.random.Generator) -> np.ndarray:
    """Station (east, north, up) positions in metres, uniform in a disk, up = 0."""
    r = radius_m * np.sqrt(rng.random(n_stations))
    th = 2.0 * np.pi * rng.random(n_stations)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n_stations)], axis=1)


def earth_rotation_uvw(enu_m: np.ndarray, lat_rad: float, dec_rad: float,
                       hour_angles_rad: np.ndarray, freq_hz: float) -> np.ndarray:
    """Baseline (u, v, w) tracks in wavelengths for every station pair i < j and hour angle.

    Textbook Earth-rotation synthesis (Thompson, Moran & Swenson, ch. 4): local
    ENU baseline -> equatorial XYZ at latitude lat, then the rotation by hour
    angle H and declination dec. Output rows are ordered (time, baseline).
    """
    n = enu_m.shape[0]
    ii, jj = np.triu_indices(n, k=1)
    b = enu_m[jj] - enu_m[ii]                                   # (B, 3) east, north, up
    e, nn, up = b[:, 0], b[:, 1], b[:, 2]
    X = -math.sin(lat_rad) * nn + math.cos(lat_rad) * up
    Y = e
    Z = math.cos(lat_rad) * nn + math.sin(lat_rad) * up
    H = hour_angles_rad[:, None]
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    u = np.sin(H) * X + np.cos(H) * Y
    v = -sd * np.cos(H) * X + sd * np.sin(H) * Y + cd * Z
    w = cd * np.cos(H) * X - cd * np.sin(H) * Y + sd * Z
    lam = C_LIGHT / freq_hz
    return np.stack([u.ravel(), v.ravel(), w.ravel()], axis=1) / lam


def gaussian_radial_uv(M: int, R: float, rng: np.random.Generator) -> np.ndarray:
    """Coplanar (w = 0) uv points: radius |N(0, R/2)| redrawn until <= R, angle U[0, 2pi)."""
    r = np.abs(rng.normal(0.0, R / 2.0, M))
    bad = r > R
    while bad.any():
        r[bad] = np.abs(rng.normal(0.0, R / 2.0, int(bad.sum())))
        bad = r > R
    th = 2.0 * np.pi * rng.random(M)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(M)], axis=1)


def subsample_rows(a: np.ndarray, M: int, rng: np.random.Generator) -> np.ndarray:
    """Seeded uniform subsample of exactly M rows (kept in their original order)."""
    if M >= a.shape[0]:
        return a.copy()
    keep = np.sort(rng.choice(a.shape[0], size=M, replace=False))
    return a[keep]


# ---------------------------------------------------------------- skies

def point_sources(N: int, K: int, rng: np.random.Generator, flux: str = "uniform",
                  lo: float = 1.0, hi: float = 10.0, margin: int = 0):
    """K distinct random pixels (raster order) with fluxes U[lo, hi] or exp(N(0, 1))."""
    side = N - 2 * margin
    cells = rng.choice(side * side, size=K, replace=False)
    i = cells // side + margin
    j = cells % side + margin
    idx = np.sort((i * N + j).astype(np.int64))
    if flux == "uniform":
        f = rng.uniform(lo, hi, K)
    elif flux == "lognormal":
        f = np.exp(rng.normal(0.0, 1.0, K))
    else:
        raise ValueError(flux)
    return idx.astype(np.int32), f.astype(np.float64)


def unit_complex_noise(M: int, rng: np.random.Generator) -> np.ndarray:
    return (rng.normal(size=M) + 1j * rng.normal(size=M)) / math.sqrt(2.0)


# ---------------------------------------------------------------- named workloads

def gaussian_blobs(N: int, n_blobs: int, rng: np.random.Generator, width_px=(5.0, 50.0),
                   peak=(0.1, 1.0), floor: float = 1e-3):
    """Elliptical Gaussian blobs: axis FWHMs U[width_px], random orientation,
    centres in the inner 80 % of the image, peak brightness U[peak] per pixel;
    pixels below `floor` x peak are dropped. Returns (sorted raster indices,
    brightness per pixel), overlapping blobs summed."""
    img = {}
    for _ in range(n_blobs):
        fa, fb = rng.uniform(width_px[0], width_px[1], 2)
        sa, sb = fa / 2.3548200450309493, fb / 2.3548200450309493
        th = rng.uniform(0.0, np.pi)
        ci, cj = rng.uniform(0.1 * N, 0.9 * N, 2)
        pk = rng.uniform(peak[0], peak[1])
        r = int(math.ceil(max(sa, sb) * math.sqrt(2.0 * math.log(1.0 / floor)))) + 1
        i0, i1 = max(0, int(ci) - r), min(N, int(ci) + r + 1)
        j0, j1 = max(0, int(cj) - r), min(N, int(cj) + r + 1)
        ii, jj = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), indexing="ij")
        di, dj = ii - ci, jj - cj
        u = di * math.cos(th) + dj * math.sin(th)
        v = -di * math.sin(th) + dj * math.cos(th)
        val = pk * np.exp(-0.5 * ((u / sa) ** 2 + (v / sb) ** 2))
        for p, b in zip((ii * N + jj)[val >= floor * pk].ravel(), val[val >= floor * pk].ravel()):
            img[int(p)] = img.get(int(p), 0.0) + float(b)
    idx = np.array(sorted(img), dtype=np.int64)
    return idx, np.array([img[int(p)] for p in idx], dtype=np.float64)


def merge_skies(idx_a, f_a, idx_b, f_b):
    """Union of two sparse skies (sorted indices), values summed where they meet."""
    idx = np.union1d(idx_a, idx_b)
    f = np.zeros(idx.size)
    f[np.searchsorted(idx, idx_a)] += f_a
    f[np.searchsorted(idx, idx_b)] += f_b
    return idx, f


def _rngs(seed: int):
    ss = np.random.SeedSequence(seed)
    layout, sky, noise, sub = ss.spawn(4)
    return (np.random.default_rng(layout), np.random.default_rng(sky),
            np.random.default_rng(noise), np.random.default_rng(sub))


def tiny_coplanar(seed: int = 1000, M: int = 2000, N: int = 64, fov_deg: float = 1.0,
                  n_src: int = 5) -> Workload:
    """64x64, FOV 1 deg, w = 0, M = 2000 Gaussian-radial (u, v) in a disk whose radius
    is 64 cells of the 2x oversampled grid (= 1 / (2 dl) wavelengths), 5 sources
    with fluxes U[1, 10], 20 dB SNR, alpha = 0.1, delta = 0.01."""
    r_lay, r_sky, r_noise, _ = _rngs(seed)
    fov = math.radians(fov_deg)
    dl = fov / N
    R = 64.0 / (2 * N * dl)            # 64 cells of the sigma=2 grid, cell = 1/(2 N dl)
    uvw = gaussian_radial_uv(M, R, r_lay)
    idx, f = point_sources(N, n_src, r_sky, "uniform", 1.0, 10.0)
    return Workload("tiny_64_coplanar", N, fov, uvw, idx, f, unit_complex_noise(M, r_noise),
                    20.0, 0.1, 0.01, seed)


def earth_rotation_workload(name: str, seed: int, N: int, fov_deg: float, n_stations: int,
                            radius_m: float, hours: float, dump_s: float, M: int,
                            n_src: int, snr_db: float, freq_hz: float = 100e6,
                            lat_deg: float = -30.0, dec_deg: float = -30.0,
                            alpha: float = 0.1, delta: float = 0.01,
                            flux: str = "lognormal") -> Workload:
    """Random station layout, Earth-rotation tracks symmetric about transit,
    seeded subsample to exactly M visibilities, log-normal point sources."""
    r_lay, r_sky, r_noise, r_sub = _rngs(seed)
    enu = stations_uniform_disk(n_stations, radius_m, r_lay)
    n_t = int(round(hours * 3600.0 / dump_s))
    H = (np.arange(n_t) - (n_t - 1) / 2.0) * dump_s * (2.0 * np.pi / 86164.0905)
    uvw = earth_rotation_uvw(enu, math.radians(lat_deg), math.radians(dec_deg), H, freq_hz)
    uvw = subsample_rows(uvw, M, r_sub)
    idx, f = point_sources(N, n_src, r_sky, flux)
    return Workload(name, N, math.radians(fov_deg), uvw, idx, f,
                    unit_complex_noise(uvw.shape[0], r_noise), snr_db, alpha, delta, seed)


def medium_512(seed: int = 1001, M: int = 200_000) -> Workload:
    """512x512, FOV 2 deg, 40 stations within 3 km, 4 h at 10 s dumps, nonzero w,
    seeded subsample to M = 200k, 50 log-normal point sources, 20 dB SNR."""
    return earth_rotation_workload("medium_512_w", seed, 512, 2.0, 40, 3000.0, 4.0, 10.0, M,
                                   50, 20.0)


def large_2048(seed: int = 1002, M: int = 2_000_000, blobs: bool = False) -> Workload:
    """2048x2048, FOV 5 deg, 60 stations within 5 km (baselines up to 10 km),
    Earth rotation to M = 2M, 200 log-normal point sources, 15 dB SNR; with
    blobs=True also 10 elliptical Gaussian blobs (FWHM 5-50 px, peak U[0.1, 1]
    per pixel), the diffuse part of the configuration, solved with the
    exploration rule of Algorithm 2 at delta = 0.9: on a diffuse sky at
    lambda = 0.1 lambda_max the normalised rule |mu| >= 1 - delta with delta =
    0.01 would put ~240k pixels into the first active set."""
    wl = earth_rotation_workload("large_2048_w", seed, 2048, 5.0, 60, 5000.0, 3.14, 10.0, M,
                                 200, 15.0)
    if blobs:
        rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(5)[4])
        bi, bf = gaussian_blobs(wl.N, 10, rng)
        wl.sky_idx, wl.sky_flux = merge_skies(wl.sky_idx, wl.sky_flux, bi, bf)
        wl.sky_idx = wl.sky_idx.astype(np.int32)
        wl.name = "large_2048_blobs"
        wl.rule, wl.delta = "R1", 0.9
    return wl


def fine_4096(seed: int = 1003, M: int = 10_000_000) -> Workload:
    """4096x4096, FOV 5 deg, 100 stations within 5.85 km, M = 10M, 500 log-normal sources."""
    return earth_rotation_workload("fine_4096_w", seed, 4096, 5.0, 100, 5850.0, 5.62, 10.0, M,
                                   500, 20.0)


def small_wide_field(seed: int = 1010, N: int = 64, fov_deg: float = 12.0, n_stations: int = 12,
                     radius_m: float = 300.0, hours: float = 2.0, dump_s: float = 120.0,
                     M: int | None = None, n_src: int = 6, snr_db: float = 20.0) -> Workload:
    """Small wide-field case with a strong w-term: the oracle solves it in seconds,
    and the GPU needs several w-planes for it."""
    n_b = n_stations * (n_stations - 1) // 2
    n_t = int(round(hours * 3600.0 / dump_s))
    return earth_rotation_workload("small_wide_w", seed, N, fov_deg, n_stations, radius_m,
                                   hours, dump_s, M if M is not None else n_b * n_t, n_src,
                                   snr_db)


def diffuse_workload(name: str, seed: int, N: int, fov_deg: float, n_stations: int, radius_m: float,
                     n_times: int, dump_s: float, M: int, n_blobs: int, width_px, n_src: int,
                     snr_db: float, alpha: float, delta: float = 0.01) -> Workload:
    """Diffuse sky for the synthesis-dictionary solve (Sect. 4.3): elliptical
    Gaussian blobs (pixels below 1 % of a blob's peak dropped) plus a few
    point sources with fluxes U[0.5, 2], observed by a random layout over
    n_times Earth-rotation dumps at 100 MHz, subsampled to M visibilities."""
    r_lay, r_sky, r_noise, r_sub = _rngs(seed)
    enu = stations_uniform_disk(n_stations, radius_m, r_lay)
    H = (np.arange(n_times) - (n_times - 1) / 2.0) * dump_s * (2.0 * np.pi / 86164.0905)
    uvw = earth_rotation_uvw(enu, math.radians(-30.0), math.radians(-30.0), H, 100e6)
    uvw = subsample_rows(uvw, M, r_sub)
    bi, bf = gaussian_blobs(N, n_blobs, r_sky, width_px, floor=1e-2)
    pi, pf = point_sources(N, n_src, r_sky, "uniform", 0.5, 2.0)
    idx, f = merge_skies(bi, bf, pi.astype(np.int64), pf)
    return Workload(name, N, math.radians(fov_deg), uvw, idx.astype(np.int32), f,
                    unit_complex_noise(uvw.shape[0], r_noise), snr_db, alpha, delta, seed)


def diffuse_256(seed: int = 1005, M: int = 31_600) -> Workload:
    """Shaped like the paper's diffuse experiment (Table 1, dataset III):
    256 x 256 at FOV 6.5 deg, 251 stations within 900 m (baselines up to
    ~1.8 km, ~600 wavelengths at 100 MHz), 11 dumps 2880 s apart, M = 31.6k
    visibilities; 6 blobs (FWHM 6-30 px) and 5 point sources, 20 dB SNR,
    lambda = 0.02 lambda_max (the paper's choice for the dictionary solve).
    delta = 0.98 goes with the exploration rule of Algorithm 2 (threshold
    ||eta||_inf - 2 Delta/(k+2)): with the normalised rule |eta| / lambda >=
    1 - delta a diffuse sky at this lambda puts about half of all coefficients
    into the first active set."""
    return diffuse_workload("diffuse_256", seed, 256, 6.5, 251, 900.0, 11, 2880.0, M, 6, (6.0, 30.0), 5,
                            20.0, 0.02, delta=0.98)


def small_diffuse(seed: int = 1011, N: int = 32, M: int = 1500) -> Workload:
    """Small diffuse case the oracle's dictionary solve finishes in seconds:
    32 x 32 at the pixel size of diffuse_256, 30 stations within 900 m, 11
    dumps, 3 blobs (FWHM 3-8 px) and 2 point sources, lambda = 0.05 lambda_max."""
    return diffuse_workload("small_diffuse", seed, N, 6.5 * N / 256, 30, 900.0, 11, 2880.0, M, 3, (3.0, 8.0),
                            2, 20.0, 0.05)


def serving_stream(seed: int = 1004, n_requests: int = 64, rate_hz: float = 4.0):
    """The mixed request stream of the serving configuration: Poisson arrivals
    at rate_hz, grids drawn from {256, 512, 1024, 2048}^2, M log-uniform in
    [1e4, 1e6], 5-200 log-normal point sources, 20 dB SNR, alpha = 0.1,
    delta = 0.01. Grids up to 512 use the 40-station / 3 km layout at FOV 2 deg,
    larger grids the 60-station / 5 km layout at FOV 5 deg. Returns a list of
    (arrival time in seconds, Workload)."""
    ss = np.random.SeedSequence(seed)
    r_arr, r_req = (np.random.default_rng(s) for s in ss.spawn(2))
    t = np.cumsum(r_arr.exponential(1.0 / rate_hz, n_requests))
    out = []
    for i in range(n_requests):
        N = int(r_req.choice([256, 512, 1024, 2048]))
        M = int(round(10.0 ** r_req.uniform(4.0, 6.0)))
        K = int(r_req.integers(5, 201))
        sub_seed = int(r_req.integers(0, 2 ** 31 - 1))
        if N <= 512:
            wl = earth_rotation_workload(f"stream_{i}_{N}", sub_seed, N, 2.0, 40, 3000.0, 4.0, 10.0, M,
                                         K, 20.0)
        else:
            wl = earth_rotation_workload(f"stream_{i}_{N}", sub_seed, N, 5.0, 60, 5000.0, 3.14, 10.0, M,
                                         K, 20.0)
        out.append((float(t[i]), wl))
    return out


WORKLOADS = {
    "tiny_64_coplanar": tiny_coplanar,
    "medium_512_w": medium_512,
    "large_2048_w": large_2048,
    "large_2048_blobs": lambda: large_2048(blobs=True),
    "fine_4096_w": fine_4096,
    "small_wide_w": small_wide_field,
    "diffuse_256": diffuse_256,
    "small_diffuse": small_diffuse,
}
