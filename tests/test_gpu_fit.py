"""Visibility-space shapelet fitting (CGLS over the library's forward contraction and coefficient
adjoint) against the oracle's dense least squares, with gains and fixed points/Gaussians present."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wn():
    import paper_2005_09316_b300 as wn
    return wn


@pytest.fixture(scope="module")
def ctx(wn):
    c = wn.Context(0)
    yield c
    c.close()


def problem(seed, n_ant=10, n_time=2, n_chan=12, nmax=(6,), noise=0.0):
    obs = synth.make_obs(seed, n_ant, n_time, synth.uniform_channels(167e6, 0.5e6, n_chan), layout="mwa",
                         max_baseline=2500.0, dec0=-30 * synth.DEG)
    sky = synth.make_sky(seed + 1, 5, 3, len(nmax), fov=6 * synth.DEG, shape_nmax=np.array(nmax),
                         shape_beta=(4 * synth.ARCMIN, 8 * synth.ARCMIN))
    sky.flux[sky.n_point + sky.n_gauss:] = 4.0
    rows = np.arange(obs.n_rows)
    gains = synth.make_gains(seed + 2, obs.n_ant, obs.n_time, 1, 0.05)
    G = oracle.gain_product(rows // obs.n_base, rows % obs.n_base, obs.ant1, obs.ant2, gains, obs.n_chan)
    uvw = obs.uvw.reshape(-1, 3)
    D = G * oracle.predict(uvw, obs.freq, obs.dec0, sky) + synth.complex_noise(seed + 3, (obs.n_rows, obs.n_chan), noise)
    return obs, sky, gains, G, D


def gpu_fit(wn, ctx, obs, sky, gains, D, n_iter=400, tol=1e-7):
    d = wn.obs_to_device(obs)
    start = sky.__class__(**sky.__dict__)
    start.s_coeff = np.zeros_like(sky.s_coeff)          # fit from zero
    m = ctx.upload(start)
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    dd = torch.as_tensor(D.astype(np.complex64).reshape(obs.n_time, obs.n_base, obs.n_chan)).cuda()
    c, info = ctx.fit_shapelets(d, m, gd, dd, n_iter=n_iter, tol=tol)
    flags = ctx.device_errors()
    # the model now predicts with the fitted coefficients
    v = ctx.predict(d, m).cpu().numpy()
    m.free()
    return c.cpu().numpy(), info, flags, v


def test_noiseless_coefficients_recovered(wn, ctx):
    """One shapelet at n_max 6 is well conditioned on this array: the coefficients come back."""
    obs, sky, gains, G, D = problem(11, nmax=(6,))
    c, info, flags, _ = gpu_fit(wn, ctx, obs, sky, gains, D)
    assert flags == 0
    assert info["resid2"] <= 1e-6 * info["resid2_start"], info
    err = np.abs(c - sky.s_coeff).max() / np.abs(sky.s_coeff).max()
    assert err <= 2e-3, (err, info)


def test_two_shapelets_fit_the_data_like_the_oracle(wn, ctx):
    """Two shapelets (n_max 4 and 8): high orders are poorly sampled by a 10-antenna array, so the
    least-squares coefficients are ill-determined, but the fitted visibilities are unique; they match
    the data and the oracle's least-squares model."""
    obs, sky, gains, G, D = problem(12, nmax=(4, 8))
    c, info, flags, vfit = gpu_fit(wn, ctx, obs, sky, gains, D)
    assert flags == 0
    uvw = obs.uvw.reshape(-1, 3)
    ref = oracle.fit_shapelet_coeffs(uvw, obs.freq, obs.dec0, sky, G, D)
    fitted = sky.__class__(**sky.__dict__)
    fitted.s_coeff = ref
    vref = oracle.predict(uvw, obs.freq, obs.dec0, fitted)
    assert np.abs(vfit.reshape(vref.shape) - vref).max() <= 2e-3 * np.abs(vref).max()
    assert info["resid2"] <= 1e-6 * info["resid2_start"], info


def _design(obs, sky, G):
    """The oracle's design matrix of the shapelet coefficients (gains applied), one column per
    coefficient, and the data less the fixed points and Gaussians: V = V_pg + A c (eq:shape-env is
    linear in the coefficients)."""
    uvw = obs.uvw.reshape(-1, 3)
    n = len(sky.s_coeff)
    cols = []
    for k in range(n):
        s2 = sky.__class__(**sky.__dict__)
        s2.flux = np.array(sky.flux, float).copy()
        s2.flux[:sky.n_point + sky.n_gauss] = 0.0
        e = np.zeros(n)
        e[k] = 1.0
        s2.s_coeff = e
        cols.append((G * oracle.predict(uvw, obs.freq, obs.dec0, s2)).ravel())
    pg = sky.__class__(**sky.__dict__)
    pg.flux = np.array(sky.flux, float).copy()
    pg.flux[sky.n_point + sky.n_gauss:] = 0.0
    return np.array(cols).T, (G * oracle.predict(uvw, obs.freq, obs.dec0, pg)).ravel()


def test_noisy_fit_matches_oracle_least_squares(wn, ctx):
    """n_max 7 (36 coefficients) under noise.  The least-squares problem has condition number about 280,
    so its coefficients are determined only to about cond^2 times the FP32 rounding of the products
    (~1e-7): the fit must reach the oracle's least-squares objective within 1e-4, and its coefficients
    must equal the oracle's within 1e-2 of the largest."""
    obs, sky, gains, G, D = problem(21, nmax=(7,), noise=0.5)
    c, info, flags, vfit = gpu_fit(wn, ctx, obs, sky, gains, D)
    assert flags == 0
    uvw = obs.uvw.reshape(-1, 3)
    ref = oracle.fit_shapelet_coeffs(uvw, obs.freq, obs.dec0, sky, G, D)
    A, vpg = _design(obs, sky, G)
    b = D.ravel() - vpg
    f_gpu = np.sum(np.abs(b - A @ c) ** 2)
    f_ref = np.sum(np.abs(b - A @ ref) ** 2)
    assert f_gpu <= f_ref * (1 + 1e-4), (f_gpu, f_ref, info)
    err = np.abs(c - ref).max() / np.abs(ref).max()
    assert err <= 1e-2, (err, info)
    # the model keeps the fitted coefficients
    fitted = sky.__class__(**sky.__dict__)
    fitted.s_coeff = ref
    vref = oracle.predict(uvw, obs.freq, obs.dec0, fitted)
    assert np.abs(vfit.reshape(vref.shape) - vref).max() <= 2e-3 * np.abs(vref).max()


def test_rejects_a_model_without_shapelets(wn, ctx):
    obs, sky, gains, G, D = problem(31)
    d = wn.obs_to_device(obs)
    pg = synth.make_sky(5, 4, 2, 0)
    m = ctx.upload(pg)
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    dd = torch.as_tensor(D.astype(np.complex64).reshape(obs.n_time, obs.n_base, obs.n_chan)).cuda()
    with pytest.raises(wn.WnError) as e:
        ctx.fit_shapelets(d, m, gd, dd, coeff=torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert e.value.code == wn.WN_EINVAL
    m.free()
