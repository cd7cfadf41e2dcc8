"""wn_sky_update: a resident model re-packed in place from new parameter values equals a fresh upload of
those values bit for bit (predict, peel, the FP64 form and every gradient), and a gradient-descent fit
through the autograd loss on a resident model allocates nothing in the library per step."""
import copy

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wn():
    import paper_2005_09316_b300 as wn
    yield wn
    wn.debug_fail_allocs(0)


def _perturbed(sky, seed):
    rng = np.random.default_rng(seed)
    b = copy.deepcopy(sky)
    b.flux = sky.flux * (1 + 0.1 * rng.standard_normal(sky.flux.size))
    b.flux[3] = -b.flux[3]
    b.alpha = sky.alpha + 0.05 * rng.standard_normal(sky.alpha.size)
    b.l = sky.l + 1e-4 * rng.standard_normal(sky.l.size)
    b.m = sky.m + 1e-4 * rng.standard_normal(sky.m.size)
    b.g_maj = sky.g_maj * 1.1
    b.g_min = sky.g_min * 0.9
    b.g_pa = sky.g_pa + 0.2
    b.s_beta1 = sky.s_beta1 * 1.05
    b.s_beta2 = sky.s_beta2 * 0.95
    b.s_pa = sky.s_pa + 0.3
    b.s_coeff = sky.s_coeff * (1 + 0.2 * rng.standard_normal(sky.s_coeff.size))
    return b


def test_update_equals_fresh_upload(wn):
    ctx = wn.Context(0)
    obs = synth.make_obs(91, 20, 2, synth.uniform_channels(167e6, 80e3, 48), layout="mwa", dec0=-30 * synth.DEG)
    sky = synth.make_sky(92, 80, 30, 2, fov=8 * synth.DEG, shape_nmax=np.array([10, 24]))
    b = _perturbed(sky, 93)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    m.update(b)
    fresh = ctx.upload(b)
    assert torch.equal(ctx.predict(d, m), ctx.predict(d, fresh))
    gains = torch.as_tensor(synth.make_gains(94, obs.n_ant).astype(np.complex64)).cuda()
    data = torch.randn(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda",
                       generator=torch.Generator(device="cuda").manual_seed(5))
    assert torch.equal(ctx.peel(d, m, gains, data), ctx.peel(d, fresh, gains, data))
    ga, gb = ctx.predict_grad(d, m, gains, data), ctx.predict_grad(d, fresh, gains, data)
    for k, v in ga.items():
        if v is not None:
            assert torch.equal(v, gb[k]), k
    ctx.set_precision(wn.WN_PREC_FP64)
    assert torch.equal(ctx.predict(d, m), ctx.predict(d, fresh))
    ctx.set_precision(wn.WN_PREC_MIXED)
    # and it is the oracle's prediction of the new values
    ref = oracle.predict(obs.uvw.reshape(-1, 3), obs.freq, obs.dec0, b)
    got = ctx.predict(d, m).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    assert np.abs(got - ref).max() <= 2e-4 * np.abs(ref).max()
    assert ctx.device_errors() == 0
    m.free()
    fresh.free()
    ctx.close()


def test_update_refuses_other_counts_and_flags_bad_values(wn):
    ctx = wn.Context(0)
    sky = synth.make_sky(95, 10, 4, 1, shape_nmax=6)
    m = ctx.upload(sky)
    other = synth.make_sky(96, 11, 4, 1, shape_nmax=6)
    with pytest.raises(ValueError):
        m.update(other)
    bad = copy.deepcopy(sky)
    bad.l = bad.l.copy()
    bad.l[2] = 1.5                       # l^2 + m^2 >= 1: rejected on the device, not on the host
    m.update(bad)
    assert ctx.device_errors() & wn.WN_DEVERR_SKY
    m.update(sky)
    assert ctx.device_errors() == 0
    m.free()
    ctx.close()


def test_gradient_descent_fit_on_a_resident_model(wn):
    """20 Adam steps on the fluxes of 40 points and a shapelet's coefficients, through
    peel_loss with a resident model: the loss falls, the first loss equals that of the upload-per-call
    path, and no step allocates device memory in the library (every library allocation is armed to fail
    during the loop)."""
    from paper_2005_09316_b300.autograd import peel_loss
    ctx = wn.Context(0)
    obs = synth.make_obs(97, 24, 2, synth.uniform_channels(167e6, 80e3, 32), layout="mwa")
    truth = synth.make_sky(98, 40, 0, 1, fov=6 * synth.DEG, shape_nmax=12, shape_lm=[(0.01, 0.005)])
    truth.flux[40] = 20.0
    gains = synth.make_gains(99, obs.n_ant)
    V = oracle.predict(obs.uvw.reshape(-1, 3), obs.freq, obs.dec0, truth)
    rows = np.arange(obs.n_rows)
    G = oracle.gain_product(rows // obs.n_base, rows % obs.n_base, obs.ant1, obs.ant2, gains, obs.n_chan)
    data = (G * V + synth.complex_noise(100, V.shape, 0.01)).astype(np.complex64)
    start = copy.deepcopy(truth)
    start.flux = truth.flux * (1 + 0.3 * np.random.default_rng(101).standard_normal(truth.flux.size))
    start.s_coeff = truth.s_coeff * 0.5
    d = wn.obs_to_device(obs)
    sky = wn.sky_to_device(start)
    params = {k: sky[k].clone().requires_grad_(True) for k in ("flux", "s_coeff")}
    sky.update(params)
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    dd = torch.as_tensor(data.reshape(obs.n_time, obs.n_base, obs.n_chan)).cuda()
    resident = ctx.upload(start)
    l_upload = peel_loss(ctx, d, sky, gd, dd).item()
    opt = torch.optim.Adam([{"params": [params["flux"]], "lr": 0.1}, {"params": [params["s_coeff"]], "lr": 0.002}])
    losses = []
    for step in range(20):
        opt.zero_grad()
        loss = peel_loss(ctx, d, sky, gd, dd, model=resident)
        loss.backward()
        opt.step()
        losses.append(loss.item())
        if step == 0:
            assert losses[0] == pytest.approx(l_upload, rel=1e-12)
            wn.debug_fail_allocs(1 << 20)   # from the second step on, any library allocation fails
    wn.debug_fail_allocs(0)
    assert losses[-1] < 0.1 * losses[0], losses   # the same loop on the oracle reaches 0.037
    assert ctx.device_errors() == 0
    resident.free()
    ctx.close()
