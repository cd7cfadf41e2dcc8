"""Gain calibration (Sec. 5.1, eq:peeling-iter) on the GPU against the oracle's loop: the same gauge,
the same number of iterations, gains compared element by element; exact recovery of known gains;
a 128-antenna problem with a predicted model; the calibrate-then-peel chain; the degenerate case."""
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


def corrupted(seed, obs, I, noise):
    """Data V = g_true[ant1] conj(g_true[ant2]) I + noise with per-(t, f) gains g_true [T, F, A]."""
    rng = np.random.default_rng(seed)
    T, B, F = I.shape
    g = 1 + 0.05 * (rng.normal(size=(T, F, obs.n_ant)) + 1j * rng.normal(size=(T, F, obs.n_ant)))
    g1 = np.transpose(g[:, :, obs.ant1], (0, 2, 1))
    g2 = np.transpose(g[:, :, obs.ant2], (0, 2, 1))
    V = g1 * np.conj(g2) * I + noise * (rng.normal(size=I.shape) + 1j * rng.normal(size=I.shape))
    return g, V


def gpu_cal(wn, ctx, obs, I, V, n_iter=10):
    d = wn.obs_to_device(obs)
    It = torch.as_tensor(I.astype(np.complex64)).cuda()
    Vt = torch.as_tensor(V.astype(np.complex64)).cuda()
    g = ctx.calibrate(d, It, Vt, n_iter=n_iter)
    flags = ctx.device_errors()
    return g.cpu().numpy().astype(np.complex128), flags


def random_model(seed, obs):
    rng = np.random.default_rng(seed)
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("n_ant,n_time,n_chan", [(4, 1, 1), (8, 2, 3), (23, 1, 5), (48, 2, 2)])
def test_exact_gains_recovered(wn, ctx, n_ant, n_time, n_chan):
    obs = synth.make_obs(80 + n_ant, n_ant, n_time, synth.uniform_channels(167e6, 80e3, n_chan), layout="mwa")
    I = random_model(81, obs)
    g_true, V = corrupted(82, obs, I, 0.0)
    g, flags = gpu_cal(wn, ctx, obs, I, V)
    assert flags == 0
    want = g_true * np.exp(-1j * np.angle(g_true[:, :, :1]))  # gauge Im(g_0) = 0
    np.testing.assert_allclose(g, want, atol=2e-6, rtol=0)


@pytest.mark.parametrize("n_ant,noise", [(8, 0.3), (32, 0.5)])
def test_noisy_gains_match_oracle(wn, ctx, n_ant, noise):
    obs = synth.make_obs(90 + n_ant, n_ant, 2, synth.uniform_channels(167e6, 80e3, 3), layout="mwa")
    I = random_model(91, obs)
    _, V = corrupted(92, obs, I, noise)
    g, flags = gpu_cal(wn, ctx, obs, I, V)
    assert flags == 0
    ref = oracle.calibrate(obs.ant1, obs.ant2, n_ant, I, V, np.ones((2, 3, n_ant)), 10)
    np.testing.assert_allclose(g, ref, atol=1e-5, rtol=0)


def test_mwa_array_with_a_predicted_model(wn, ctx):
    """128 tiles (255 parameters per solve), a point/Gaussian model predicted by the library, data from
    known gains plus noise; a sample of (t, f) problems against the oracle."""
    obs, _ = synth.mwa(n_time=1)
    obs = synth.make_obs(5, 128, 1, synth.uniform_channels(167e6, 80e3, 8), layout="mwa")
    sky = synth.make_sky(6, 300, 60, 0)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    It = ctx.predict(d, m)
    I = It.cpu().numpy().astype(np.complex128)
    m.free()
    _, V = corrupted(7, obs, I, 0.05 * np.abs(I).mean())
    g, flags = gpu_cal(wn, ctx, obs, I, V)
    assert flags == 0
    for f in (0, 5):
        ref = oracle.calibrate(obs.ant1, obs.ant2, 128, I[:, :, f:f + 1], V[:, :, f:f + 1], np.ones((1, 1, 128)), 10)
        np.testing.assert_allclose(g[:, f:f + 1], ref, atol=2e-5, rtol=0)


def test_calibrate_then_peel_leaves_the_noise(wn, ctx):
    obs = synth.make_obs(11, 32, 2, synth.uniform_channels(167e6, 80e3, 16), layout="mwa")
    sky = synth.make_sky(12, 60, 10, 0)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    It = ctx.predict(d, m)
    I = It.cpu().numpy().astype(np.complex128)
    sigma = 1e-3 * np.abs(I).mean()
    _, V = corrupted(13, obs, I, sigma)
    Vt = torch.as_tensor(V.astype(np.complex64)).cuda()
    gains = ctx.calibrate(d, It, Vt)
    resid = ctx.peel_model(d, gains, Vt, It)
    r = resid.cpu().numpy()
    rms = np.sqrt(np.mean(np.abs(r) ** 2))
    assert rms < 1.6 * sigma * np.sqrt(2), (rms, sigma)     # the noise, to within the fit's degrees of freedom
    assert ctx.device_errors() == 0
    m.free()


def test_zero_model_sets_the_flag_and_keeps_the_gains(wn, ctx):
    obs = synth.make_obs(21, 6, 1, synth.uniform_channels(167e6, 80e3, 2), layout="mwa")
    d = wn.obs_to_device(obs)
    I = torch.zeros((1, obs.n_base, 2), dtype=torch.complex64, device="cuda")
    V = torch.ones((1, obs.n_base, 2), dtype=torch.complex64, device="cuda")
    g0 = torch.full((1, 2, obs.n_ant), 1 + 0.5j, dtype=torch.complex64, device="cuda")
    g = ctx.calibrate(d, I, V, g0.clone())
    assert ctx.device_errors() & wn.WN_DEVERR_CALIB
    assert torch.equal(g, g0)


def test_rejects_bad_arguments(wn, ctx):
    obs = synth.make_obs(31, 6, 1, synth.uniform_channels(167e6, 80e3, 2), layout="mwa")
    d = wn.obs_to_device(obs)
    I = torch.ones((1, obs.n_base, 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(wn.WnError) as e:
        ctx.calibrate(d, I, I, n_iter=0)
    assert e.value.code == wn.WN_EINVAL
    with pytest.raises(ValueError):
        ctx.calibrate(d, I, I[:, :, :1])
