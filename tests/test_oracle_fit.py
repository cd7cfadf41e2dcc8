"""Pins of the oracle's visibility-space shapelet fit (CPU): exact recovery of known coefficients from
noiseless data with gains and fixed points/Gaussians present, and the design matrix against finite
differences of the prediction (linearity in the coefficients)."""
import numpy as np

import oracle
import synth


def problem(seed=3, n_ant=6, nmax=(4,)):
    obs = synth.make_obs(seed, n_ant, 2, synth.uniform_channels(167e6, 0.5e6, 5), layout="mwa", max_baseline=2500.0)
    sky = synth.make_sky(seed + 1, 3, 2, len(nmax), fov=5 * synth.DEG, shape_nmax=np.array(nmax),
                         shape_beta=(4 * synth.ARCMIN, 8 * synth.ARCMIN))
    rows = np.arange(obs.n_rows)
    gains = synth.make_gains(seed + 2, obs.n_ant, obs.n_time, 1, 0.05)
    G = oracle.gain_product(rows // obs.n_base, rows % obs.n_base, obs.ant1, obs.ant2, gains, obs.n_chan)
    return obs, sky, G


def test_exact_coefficients_recovered():
    obs, sky, G = problem()
    uvw = obs.uvw.reshape(-1, 3)
    D = G * oracle.predict(uvw, obs.freq, obs.dec0, sky)
    c = oracle.fit_shapelet_coeffs(uvw, obs.freq, obs.dec0, sky, G, D)
    np.testing.assert_allclose(c, sky.s_coeff, rtol=0, atol=1e-9 * np.abs(sky.s_coeff).max())


def test_design_columns_are_the_linear_response():
    obs, sky, G = problem(5, nmax=(3, 2))
    uvw = obs.uvw.reshape(-1, 3)
    A = oracle.fit_design(uvw, obs.freq, obs.dec0, sky, G)
    rng = np.random.default_rng(1)
    d = rng.normal(size=A.shape[1])
    s1 = sky.__class__(**sky.__dict__)
    n_pg = sky.n_point + sky.n_gauss
    base = sky.s_coeff.copy()
    flux = sky.flux.copy()
    s1.flux = flux.copy()
    s1.flux[:n_pg] = 0.0
    s1.s_coeff = base + d
    v1 = G * oracle.predict(uvw, obs.freq, obs.dec0, s1)
    s1.s_coeff = base
    v0 = G * oracle.predict(uvw, obs.freq, obs.dec0, s1)
    np.testing.assert_allclose((v1 - v0).ravel(), A @ d, rtol=0, atol=1e-10 * np.abs(A @ d).max())
