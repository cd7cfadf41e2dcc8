"""Seeded synthetic inputs for the visibility-prediction workloads.

This module only draws inputs: antenna layouts, baseline (u, v, w) tracks,
channel lists, sky-component tables, gains and data. It holds none of the
measurement-equation arithmetic (no phases, envelopes, spectra or Hermite
functions); both the FP64 oracle and the CUDA library consume what it makes.

Recipes (all angles in radians, lengths in metres, frequencies in Hz):

* Array: ENU antenna positions, heights N(0, 2 m), latitude -26.70 deg (an
  MWA-like site).  ``layout="disc"`` draws uniformly in a disc; ``"mwa"`` draws
  half the tiles uniformly within 100 m and half within 750 m (dense core plus
  a 1.5 km footprint); ``max_baseline`` rescales the horizontal layout so the
  longest baseline has that length.
* (u, v, w): the textbook ENU -> local equatorial XYZ -> (H, dec) rotation in
  FP64; the baseline vector is X[ant2] - X[ant1] with ant1 < ant2, baselines
  ordered (0,1), (0,2), ..., (A-2, A-1); the hour angle advances by ``dt_s``
  seconds of sidereal time per step.
* Sky: (l, m) uniform in a disc of radius sin(fov); flux log-uniform in
  [0.1, 10] Jy; spectral index N(-0.8, 0.2); reference frequency 180 MHz.
  Gaussian FWHMs log-uniform 1-10 arcmin (major >= minor), PA uniform [0, pi).
  Shapelet coefficients C[n1, n2] ~ N(0, 1) exp(-(n1 + n2)/5) for
  n1 + n2 <= n_max, optionally keeping only the ``keep`` largest |C| (the
  paper's truncation rule with |C| in place of the beam-convolved flux), then
  scaled to unit l1 norm (a stand-in for the paper's division of the
  coefficients by the integrated flux, which would need the basis itself).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ARCMIN = math.pi / (180.0 * 60.0)
DEG = math.pi / 180.0
MWA_LAT = -26.70 * DEG
SIDEREAL_DAY_S = 86400.0  # "8 s of sidereal time" -> 2*pi*8/86400 rad of hour angle


@dataclass
class Obs:
    """An observation: baseline tracks and channels (host, FP64)."""
    n_ant: int
    n_time: int
    n_chan: int
    uvw: np.ndarray        # [T, B, 3] float64, metres
    freq: np.ndarray       # [F] float64, Hz
    ant1: np.ndarray       # [B] int32
    ant2: np.ndarray       # [B] int32
    dec0: float            # phase-centre declination (rad)
    enu: np.ndarray = None  # [A, 3] antenna positions (kept for tests)
    ha: np.ndarray = None   # [T] hour angle of the phase centre (rad)
    lat: float = MWA_LAT

    @property
    def n_base(self) -> int:
        return int(self.ant1.shape[0])

    @property
    def n_rows(self) -> int:
        return self.n_time * self.n_base

    @property
    def n_vis(self) -> int:
        return self.n_rows * self.n_chan


@dataclass
class Sky:
    """Component tables, points first, then Gaussians, then shapelets (host)."""
    n_point: int
    n_gauss: int
    n_shape: int
    l: np.ndarray          # [N] float64
    m: np.ndarray          # [N] float64
    flux: np.ndarray       # [N] float64, Jy at nu_ref
    alpha: np.ndarray      # [N] float64
    nu_ref: np.ndarray     # [N] float64, Hz
    g_maj: np.ndarray      # [n_gauss] FWHM rad
    g_min: np.ndarray      # [n_gauss] FWHM rad
    g_pa: np.ndarray       # [n_gauss] rad, E of N
    s_beta1: np.ndarray    # [n_shape] rad
    s_beta2: np.ndarray    # [n_shape] rad
    s_pa: np.ndarray       # [n_shape] rad
    s_nmax: np.ndarray     # [n_shape] int32
    s_off: np.ndarray      # [n_shape + 1] int32 offsets into the coefficient triples
    s_n1: np.ndarray       # [nnz] int32
    s_n2: np.ndarray       # [nnz] int32
    s_coeff: np.ndarray    # [nnz] float64

    @property
    def n_comp(self) -> int:
        return self.n_point + self.n_gauss + self.n_shape


def enu_layout(rng: np.random.Generator, n_ant: int, layout: str = "mwa",
               diameter: float = 1000.0, max_baseline: float | None = None) -> np.ndarray:
    if layout == "disc":
        r = 0.5 * diameter * np.sqrt(rng.uniform(size=n_ant))
    elif layout == "mwa":
        half = n_ant // 2
        r = np.concatenate([100.0 * np.sqrt(rng.uniform(size=half)),
                            750.0 * np.sqrt(rng.uniform(size=n_ant - half))])
    else:
        raise ValueError(layout)
    th = rng.uniform(0.0, 2.0 * math.pi, size=n_ant)
    e, n = r * np.cos(th), r * np.sin(th)
    if max_baseline is not None:
        d = np.hypot(e[:, None] - e[None, :], n[:, None] - n[None, :]).max()
        e, n = e * (max_baseline / d), n * (max_baseline / d)
    u = rng.normal(0.0, 2.0, size=n_ant)
    return np.stack([e, n, u], axis=1)


def enu_to_xyz(enu: np.ndarray, lat: float) -> np.ndarray:
    """Local ENU -> local equatorial XYZ (X to H=0 on the equator, Z to the pole)."""
    e, n, u = enu[:, 0], enu[:, 1], enu[:, 2]
    x = -math.sin(lat) * n + math.cos(lat) * u
    y = e
    z = math.cos(lat) * n + math.sin(lat) * u
    return np.stack([x, y, z], axis=1)


def xyz_to_uvw_matrix(ha: float, dec: float) -> np.ndarray:
    """Rotation taking an XYZ baseline to (u, v, w) for a phase centre at hour angle ha, declination dec."""
    sh, ch, sd, cd = math.sin(ha), math.cos(ha), math.sin(dec), math.cos(dec)
    return np.array([[sh, ch, 0.0],
                     [-sd * ch, sd * sh, cd],
                     [cd * ch, -cd * sh, sd]])


def baselines(n_ant: int):
    a1, a2 = np.triu_indices(n_ant, k=1)
    return a1.astype(np.int32), a2.astype(np.int32)


def make_obs(seed: int, n_ant: int, n_time: int, freq: np.ndarray, layout: str = "mwa",
             diameter: float = 1000.0, max_baseline: float | None = None,
             dec0: float | None = None, ha0: float = 0.0, dt_s: float = 8.0,
             lat: float = MWA_LAT) -> Obs:
    rng = np.random.default_rng(seed)
    enu = enu_layout(rng, n_ant, layout, diameter, max_baseline)
    xyz = enu_to_xyz(enu, lat)
    a1, a2 = baselines(n_ant)
    bxyz = xyz[a2] - xyz[a1]                    # baseline vector = X[ant2] - X[ant1]
    dec0 = lat if dec0 is None else dec0        # default: zenith at ha0 = 0
    ha = ha0 + np.arange(n_time) * (2.0 * math.pi * dt_s / SIDEREAL_DAY_S)
    uvw = np.stack([bxyz @ xyz_to_uvw_matrix(h, dec0).T for h in ha], axis=0)
    return Obs(n_ant=n_ant, n_time=n_time, n_chan=len(freq), uvw=np.ascontiguousarray(uvw),
               freq=np.asarray(freq, dtype=np.float64), ant1=a1, ant2=a2, dec0=float(dec0),
               enu=enu, ha=ha, lat=lat)


def uniform_channels(f0: float, df: float, n: int) -> np.ndarray:
    return f0 + df * np.arange(n, dtype=np.float64)


def _disc_lm(rng, n, fov):
    r = math.sin(fov) * np.sqrt(rng.uniform(size=n))
    th = rng.uniform(0.0, 2.0 * math.pi, size=n)
    return r * np.cos(th), r * np.sin(th)


def shapelet_coeffs(rng: np.random.Generator, nmax: int, keep: int | None = None):
    n1, n2 = [], []
    for s in range(nmax + 1):          # triangle n1 + n2 <= nmax, ordered by s = n1 + n2
        for b in range(s + 1):
            n1.append(s - b)
            n2.append(b)
    n1 = np.array(n1, dtype=np.int32)
    n2 = np.array(n2, dtype=np.int32)
    c = rng.normal(size=n1.size) * np.exp(-(n1 + n2) / 5.0)
    if keep is not None and keep < c.size:
        idx = np.sort(np.argsort(-np.abs(c), kind="stable")[:keep])
        n1, n2, c = n1[idx], n2[idx], c[idx]
    c = c / np.abs(c).sum()
    return n1, n2, c


def make_sky(seed: int, n_point: int, n_gauss: int, n_shape: int = 0, fov: float = 20 * DEG,
             shape_nmax=10, shape_beta=(5 * ARCMIN, 5 * ARCMIN), shape_keep=None,
             shape_lm=None, nu_ref: float = 180e6) -> Sky:
    """Draw a sky; ``shape_beta`` is a (lo, hi) range for beta1 and beta2 (uniform)."""
    rng = np.random.default_rng(seed)
    n = n_point + n_gauss + n_shape
    l, m = _disc_lm(rng, n, fov)
    if shape_lm is not None and n_shape:
        sl = np.asarray(shape_lm, dtype=np.float64).reshape(n_shape, 2)
        l[n_point + n_gauss:], m[n_point + n_gauss:] = sl[:, 0], sl[:, 1]
    flux = 10.0 ** rng.uniform(-1.0, 1.0, size=n)
    alpha = rng.normal(-0.8, 0.2, size=n)
    nref = np.full(n, nu_ref)
    w = np.exp(rng.uniform(math.log(1.0), math.log(10.0), size=(n_gauss, 2))) * ARCMIN
    g_maj, g_min = w.max(axis=1), w.min(axis=1)
    g_pa = rng.uniform(0.0, math.pi, size=n_gauss)
    nmaxs = np.broadcast_to(np.asarray(shape_nmax, dtype=np.int32), (n_shape,)).copy()
    b = rng.uniform(shape_beta[0], shape_beta[1], size=(n_shape, 2))
    s_pa = rng.uniform(0.0, math.pi, size=n_shape)
    offs, N1, N2, CC = [0], [], [], []
    for s in range(n_shape):
        a, bb, c = shapelet_coeffs(rng, int(nmaxs[s]), shape_keep)
        N1.append(a), N2.append(bb), CC.append(c)
        offs.append(offs[-1] + c.size)
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    return Sky(n_point, n_gauss, n_shape, l, m, flux, alpha, nref, g_maj, g_min, g_pa,
               b[:, 0].copy(), b[:, 1].copy(), s_pa, nmaxs, np.array(offs, dtype=np.int32),
               cat(N1, np.int32), cat(N2, np.int32), cat(CC, np.float64))


def make_gains(seed: int, n_ant: int, n_tg: int = 1, n_fg: int = 1, sigma: float = 0.05) -> np.ndarray:
    """Complex gains [Tg, Fg, A] = 1 + N(0, sigma) + i N(0, sigma)."""
    rng = np.random.default_rng(seed)
    g = 1.0 + rng.normal(0, sigma, size=(n_tg, n_fg, n_ant)) + 1j * rng.normal(0, sigma, size=(n_tg, n_fg, n_ant))
    return g.astype(np.complex128)


def complex_noise(seed: int, shape, sigma: float) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.normal(0, sigma, size=shape) + 1j * rng.normal(0, sigma, size=shape)).astype(np.complex128)


# ---------------------------------------------------------------------------------------------
# The five workloads.  Sizes follow the paper's simulations (MWA Phase I / II, 8 s / 80 kHz,
# Fornax A modelled with two n_max ~ 80 shapelets beside a ~40k-component CLEAN-like model).
# ---------------------------------------------------------------------------------------------

def tiny(seed: int = 1):
    """8 antennas in a 1 km disc, zenith, 1 step, 4 channels 167-197 MHz; 10 P + 2 G + 1 S (n_max 10)."""
    obs = make_obs(seed, 8, 1, np.array([167e6, 177e6, 187e6, 197e6]), layout="disc", diameter=1000.0)
    sky = make_sky(seed + 100, 10, 2, 1, fov=10 * DEG, shape_nmax=10, shape_beta=(5 * ARCMIN, 5 * ARCMIN))
    return obs, sky


def mwa(seed: int = 2, n_point: int = 20000, n_gauss: int = 5000, n_time: int = 14, n_chan: int = 384):
    """128 tiles (8128 baselines), 14 steps at 8 s, 384 x 80 kHz from 167 MHz; 20k P + 5k G within 20 deg."""
    obs = make_obs(seed, 128, n_time, uniform_channels(167e6, 80e3, n_chan), layout="mwa")
    sky = make_sky(seed + 100, n_point, n_gauss, 0, fov=20 * DEG)
    return obs, sky


def fornax(seed: int = 3, n_time: int = 14, n_chan: int = 384, keep: int = 1500, nmax: int = 80):
    """Same array stretched to a 5 km maximum baseline, dec0 = -37.2 deg; 2 shapelets at n_max 80."""
    obs = make_obs(seed, 128, n_time, uniform_channels(167e6, 80e3, n_chan), layout="mwa",
                   max_baseline=5000.0, dec0=-37.2 * DEG)
    sky = make_sky(seed + 100, 0, 0, 2, fov=1 * DEG, shape_nmax=nmax, shape_beta=(3 * ARCMIN, 15 * ARCMIN),
                   shape_keep=keep, shape_lm=[(-0.004, 0.001), (0.005, -0.002)])
    return obs, sky


def fornax_clean(seed: int = 3, n_time: int = 14, n_chan: int = 384, n_point: int = 30000, n_gauss: int = 10000):
    """The 40,000-component point/Gaussian model that stands beside the shapelet model (within 1 deg)."""
    obs, _ = fornax(seed, n_time, n_chan)
    sky = make_sky(seed + 200, n_point, n_gauss, 0, fov=1 * DEG)
    return obs, sky


def adjoint(seed: int = 4):
    """64 tiles (2016 baselines) x 64 channels x 4 steps; 500 points + 1 shapelet at n_max 40."""
    obs = make_obs(seed, 64, 4, uniform_channels(167e6, 80e3, 64), layout="mwa")
    sky = make_sky(seed + 100, 500, 0, 1, fov=20 * DEG, shape_nmax=40, shape_beta=(5 * ARCMIN, 10 * ARCMIN),
                   shape_lm=[(0.01, -0.02)])
    return obs, sky


def sub_obs(obs: Obs, rows: np.ndarray) -> np.ndarray:
    """(u, v, w) of selected flattened rows (row = t * B + b) as [R, 3]."""
    return np.ascontiguousarray(obs.uvw.reshape(-1, 3)[rows])
