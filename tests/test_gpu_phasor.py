"""GPU parity of the point/Gaussian prediction (mixed and FP64 forms) and the peels against the oracle.

Tolerances: the mixed-precision path (FP64 phase argument, FP32 phasors and sums) must reach
e_norm <= 1e-5 (normwise, relative to max |V|); the all-FP64 form is limited by the final
complex64 rounding of its output, e_norm <= 1e-6.  Element-wise errors (e_elem, over visibilities
above 1e-3 of the peak) are held to 1e-4 and 1e-6 respectively on the tiny sky, and to 3e-4 for the
mixed path where lanes run 16 channels.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import e_elem, e_norm, oracle_peel_rows, oracle_rows, sample_rows

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


def pg_only(sky):
    """The point/Gaussian part of a sky table."""
    n = sky.n_point + sky.n_gauss
    z = np.zeros(0)
    return synth.Sky(sky.n_point, sky.n_gauss, 0, sky.l[:n], sky.m[:n], sky.flux[:n], sky.alpha[:n], sky.nu_ref[:n],
                     sky.g_maj, sky.g_min, sky.g_pa, z, z, z, np.zeros(0, np.int32), np.zeros(1, np.int32),
                     np.zeros(0, np.int32), np.zeros(0, np.int32), z)


def run_predict(wn, ctx, obs, sky, prec=0):
    ctx.set_precision(prec)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    v = ctx.predict(d, m)
    torch.cuda.synchronize()
    m.free()
    ctx.set_precision(0)
    assert ctx.device_errors() == 0
    return v.cpu().numpy().reshape(obs.n_rows, obs.n_chan)


def small_obs(seed, n_ant, n_time, freq, **kw):
    return synth.make_obs(seed, n_ant, n_time, np.asarray(freq, dtype=np.float64), **kw)


@pytest.mark.parametrize("prec,tol_norm,tol_elem", [(0, 1e-5, 1e-4), (1, 1e-6, 1e-6)])
def test_tiny_points_gaussians(wn, ctx, prec, tol_norm, tol_elem):
    obs, sky = synth.tiny(1)
    sky = pg_only(sky)
    got = run_predict(wn, ctx, obs, sky, prec)
    ref = oracle_rows(obs, sky, np.arange(obs.n_rows))
    assert e_norm(got, ref) <= tol_norm
    assert e_elem(got, ref) <= tol_elem


@pytest.mark.parametrize("n_chan,uniform", [(384, True), (64, True), (100, True), (7, True), (1, True),
                                            (37, False), (130, False),
                                            # lane / channel configurations of the cost-model choice:
                                            (512, True), (16, True), (48, True), (256, True), (400, True),
                                            (700, False)])
def test_tiles_and_ragged_tails(wn, ctx, n_chan, uniform):
    """Component counts that span several 32-component tiles with a partial last tile, row counts that
    leave a ragged last CTA, channel counts that leave idle lanes, and non-uniform channel lists."""
    rng = np.random.default_rng(n_chan)
    if uniform:
        freq = synth.uniform_channels(150e6, 40e3 * (1 + n_chan % 3), n_chan)
    else:
        freq = np.sort(rng.uniform(140e6, 200e6, size=n_chan))
    obs = small_obs(n_chan, 13, 3, freq, layout="mwa", max_baseline=3000.0)
    sky = synth.make_sky(n_chan + 7, 77, 41, 0, fov=15 * synth.DEG)
    got = run_predict(wn, ctx, obs, sky, 0)
    ref = oracle_rows(obs, sky, np.arange(obs.n_rows))
    assert e_norm(got, ref) <= 1e-5
    # e_elem is reported beside the e_norm target.  Lanes of 16 channels (chosen for 400 and 512) run the
    # three-term phasor recurrence up to 8 steps from their start channel; its rounding error grows like
    # steps^2 / 2 ulp where the phasor barely turns, which shows on the smallest elements (1e-3 of the
    # maximum) as a few 1e-4 of their size
    assert e_elem(got, ref) <= 3e-4


@pytest.mark.parametrize("n_chan", [384, 512])
def test_phase_step_near_zero_and_half_turn(wn, ctx, n_chan):
    """The phasor recurrence across uniform channels is least accurate where the per-channel phase step
    delta is near 0 or a half turn (2 cos delta near +-2): its rounding then adds up coherently over the
    steps from a lane's start channel.  Rows are placed so that every component sees such a step (tau
    dnu / c within 1e-4 turn of 0, 1/2 or 1), and a sky of co-located components makes the errors of
    all terms add up in the same direction.  Lanes run 12 channels (384) and 16 (512)."""
    dnu, c = 100e3, 299792458.0
    freq = synth.uniform_channels(150e6, dnu, n_chan)
    rng = np.random.default_rng(n_chan)
    turns = np.array([0.0, 0.5, 1.0, 0.5, 0.0, 1.0, 0.5, 0.0])
    l0 = 0.3
    n_rows = 28
    targets = np.resize(turns, n_rows) + rng.uniform(-1e-4, 1e-4, n_rows)
    uvw = np.zeros((1, n_rows, 3))
    uvw[0, :, 0] = targets * c / dnu / l0           # tau = u l0 on these rows (m = 0, w = 0)
    uvw[0, :, 1] = rng.uniform(-0.5, 0.5, n_rows)   # a small v: components spread in m by < 1e-3
    ant1, ant2 = synth.baselines(8)
    obs = synth.Obs(n_ant=8, n_time=1, n_chan=n_chan, uvw=uvw, freq=freq, ant1=ant1, ant2=ant2, dec0=-0.47)
    sky = synth.make_sky(n_chan + 3, 60, 20, 0)
    sky.l[:] = l0 + rng.uniform(-1e-7, 1e-7, sky.l.size)
    sky.m[:] = rng.uniform(-1e-3, 1e-3, sky.m.size)
    sky.flux[:] = np.abs(sky.flux)
    got = run_predict(wn, ctx, obs, sky, 0)
    ref = oracle_rows(obs, sky, np.arange(obs.n_rows))
    assert e_norm(got, ref) <= 1e-5, e_norm(got, ref)
    assert e_elem(got, ref) <= 3e-4, e_elem(got, ref)


def test_negative_and_zero_flux_and_edge_positions(wn, ctx):
    obs = small_obs(5, 10, 2, synth.uniform_channels(160e6, 1e6, 24), layout="disc", diameter=2000.0)
    sky = synth.make_sky(6, 40, 20, 0, fov=60 * synth.DEG)
    sky.flux[::3] *= -1.0
    sky.flux[5] = 0.0
    sky.l[0], sky.m[0] = 0.0, 0.0
    sky.l[1], sky.m[1] = 0.7, -0.69            # far from the phase centre, n - 1 ~ -0.86
    got = run_predict(wn, ctx, obs, sky, 0)
    ref = oracle_rows(obs, sky, np.arange(obs.n_rows))
    assert e_norm(got, ref) <= 1e-5


def test_point_at_phase_centre_is_flux_on_every_baseline(wn, ctx):
    obs = small_obs(2, 16, 2, synth.uniform_channels(167e6, 80e3, 96))
    sky = synth.make_sky(3, 1, 0, 0)
    sky.l[0] = sky.m[0] = 0.0
    got = run_predict(wn, ctx, obs, sky, 0)
    want = sky.flux[0] * (obs.freq / sky.nu_ref[0]) ** sky.alpha[0]
    np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=2e-6, atol=0)


def test_zero_components_store_accumulate_and_peel(wn, ctx):
    obs, _ = synth.tiny(2)
    empty = synth.make_sky(0, 0, 0, 0)
    d = wn.obs_to_device(obs)
    m = ctx.upload(empty)
    v = ctx.predict(d, m)
    assert torch.count_nonzero(v).item() == 0
    data = torch.randn(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda")
    g = torch.ones(1, 1, obs.n_ant, dtype=torch.complex64, device="cuda")
    r = ctx.peel(d, m, g, data)
    assert torch.equal(r, data)
    acc = data.clone()
    ctx.predict(d, m, out=acc, accumulate=True)
    assert torch.equal(acc, data)
    m.free()


def test_fused_peel_matches_oracle_and_aliases(wn, ctx):
    obs, sky = synth.tiny(4)
    sky = pg_only(sky)
    rows = np.arange(obs.n_rows)
    V = oracle_rows(obs, sky, rows)
    data = V + synth.complex_noise(9, V.shape, 0.01)
    gains = synth.make_gains(10, obs.n_ant, obs.n_time, obs.n_chan)
    ref = oracle_peel_rows(obs, rows, gains, data, V)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    dd = torch.as_tensor(data.astype(np.complex64).reshape(obs.n_time, obs.n_base, obs.n_chan)).cuda()
    r = ctx.peel(d, m, gd, dd).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    assert np.max(np.abs(r - ref)) <= 1e-5 * np.max(np.abs(V))
    # in place: resid aliases data
    r2 = ctx.peel(d, m, gd, dd, out=dd).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    assert np.array_equal(r, r2)
    m.free()


def test_standalone_peel_matches_oracle(wn, ctx):
    obs = small_obs(8, 12, 3, synth.uniform_channels(170e6, 80e3, 33))  # odd channel count
    rows = np.arange(obs.n_rows)
    V = synth.complex_noise(1, (obs.n_rows, obs.n_chan), 3.0)
    data = synth.complex_noise(2, V.shape, 3.0)
    gains = synth.make_gains(3, obs.n_ant, 1, obs.n_chan, 0.2)
    ref = oracle_peel_rows(obs, rows, gains, data.astype(np.complex64), V.astype(np.complex64))
    d = wn.obs_to_device(obs)
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    Vd = torch.as_tensor(V.astype(np.complex64).reshape(shape)).cuda()
    Dd = torch.as_tensor(data.astype(np.complex64).reshape(shape)).cuda()
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    r = ctx.peel_model(d, gd, Dd, Vd).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    np.testing.assert_allclose(r, ref, rtol=0, atol=2e-6 * np.abs(ref).max())


def test_bad_antenna_index_is_flagged_not_dereferenced(wn, ctx):
    obs, sky = synth.tiny(5)
    obs.ant2 = obs.ant2.copy()
    obs.ant2[3] = obs.n_ant + 1000
    d = wn.obs_to_device(obs)
    m = ctx.upload(pg_only(sky))
    g = torch.ones(1, 1, obs.n_ant, dtype=torch.complex64, device="cuda")
    data = torch.zeros(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda")
    r = ctx.peel(d, m, g, data)
    flags = ctx.device_errors()
    assert flags & wn.WN_DEVERR_ANTENNA
    assert torch.isnan(r[0, 3]).all() and not torch.isnan(r[0, 2]).any()
    m.free()


def test_invalid_arguments_rejected_on_host(wn, ctx):
    obs, sky = synth.tiny(6)
    bad = synth.make_sky(1, 3, 0, 0)
    bad.l[1], bad.m[1] = 0.8, 0.7          # l^2 + m^2 >= 1
    with pytest.raises(wn.WnError) as e:
        ctx.upload(bad)
    assert e.value.code == wn.WN_EINVAL
    d = wn.obs_to_device(obs)
    m = ctx.upload(pg_only(sky))
    g = torch.ones(2, 1, obs.n_ant, dtype=torch.complex64, device="cuda")  # gains_t must be 1 or n_time (1)
    data = torch.zeros(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda")
    with pytest.raises(wn.WnError):
        ctx.peel(d, m, g, data)
    m.free()
    with pytest.raises(wn.WnError) as e:
        ctx.predict(d, m)
    assert e.value.code == wn.WN_ENOTFOUND


def test_bitwise_reproducible(wn, ctx):
    obs = small_obs(3, 20, 2, synth.uniform_channels(167e6, 80e3, 128))
    sky = synth.make_sky(4, 300, 100, 0)
    a = run_predict(wn, ctx, obs, sky, 0)
    b = run_predict(wn, ctx, obs, sky, 0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n_time,n_chan,uniform", [(2, 384, True), (1, 384, True), (2, 700, False), (3, 96, True)])
def test_split_tail_tiles_every_mode(wn, ctx, n_time, n_chan, uniform):
    """A 128-tile array at 1-3 time steps: 2 steps at 384 channels make 508 tiles of 32 rows and leave 64
    for a last wave of 148 CTAs, which the launch splits over component ranges and sums in a second
    kernel; 1 step leaves 106, too many for parts to shorten the tail (no split).  Rows from the whole
    tiles and from the split tail, in the store, accumulate and peel modes, against the oracle."""
    rng = np.random.default_rng(n_chan + n_time)
    freq = (synth.uniform_channels(167e6, 80e3, n_chan) if uniform
            else np.sort(rng.uniform(150e6, 190e6, size=n_chan)))
    obs = small_obs(40 + n_time, 128, n_time, freq, layout="mwa")
    sky = synth.make_sky(41, 380, 120, 0, fov=20 * synth.DEG)
    rows = np.unique(np.concatenate([np.arange(4), rng.choice(obs.n_rows, 6, replace=False),
                                     obs.n_rows - 1 - np.arange(6), obs.n_rows - 1700 - np.arange(3)]))
    rows = rows[(rows >= 0) & (rows < obs.n_rows)]
    V = oracle_rows(obs, sky, rows)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    rt = torch.as_tensor(rows).cuda()
    v = ctx.predict(d, m).reshape(obs.n_rows, obs.n_chan)
    assert e_norm(v[rt].cpu().numpy(), V) <= 1e-5
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    data = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    data.real.normal_(generator=torch.Generator(device="cuda").manual_seed(n_chan))
    acc = data.clone()
    ctx.predict(d, m, out=acc, accumulate=True)
    dat = data.reshape(obs.n_rows, obs.n_chan)[rt].cpu().numpy()
    got = acc.reshape(obs.n_rows, obs.n_chan)[rt].cpu().numpy()
    assert np.max(np.abs(got - (dat + V))) <= 1e-5 * np.max(np.abs(V))
    gains = synth.make_gains(n_chan, obs.n_ant, obs.n_time, 1)
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    r = ctx.peel(d, m, gd, data).reshape(obs.n_rows, obs.n_chan)[rt].cpu().numpy()
    ref = oracle_peel_rows(obs, rows, gains.astype(np.complex64), dat, V)
    assert np.max(np.abs(r - ref)) <= 1e-5 * np.max(np.abs(V))
    # the whole output is the same in every call (fixed summation order of the parts)
    v2 = ctx.predict(d, m).reshape(obs.n_rows, obs.n_chan)
    assert torch.equal(v, v2)
    assert ctx.device_errors() == 0
    m.free()


def test_split_tail_over_more_than_one_wave(wn, ctx):
    """72 antennas (2,556 baselines) x 1 step x 384 channels, 4,000 points + 1,000 Gaussians: 80 tiles of
    32 rows, all of them the tail, each split into 3 component ranges (240 CTAs, two waves on 148 SMs)
    and summed in part order.  Rows of every tile, in the store, accumulate and peel modes, against the
    oracle; the output is the same in every call."""
    obs = small_obs(72, 72, 1, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    sky = synth.make_sky(73, 4000, 1000, 0, fov=20 * synth.DEG)
    rng = np.random.default_rng(72)
    rows = np.unique(np.concatenate([np.arange(0, obs.n_rows, 32), rng.choice(obs.n_rows, 8, replace=False),
                                     [obs.n_rows - 1]]))
    V = oracle_rows(obs, sky, rows)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    rt = torch.as_tensor(rows).cuda()
    v = ctx.predict(d, m).reshape(obs.n_rows, obs.n_chan)
    assert e_norm(v[rt].cpu().numpy(), V) <= 1e-5
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    data = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    data.real.normal_(generator=torch.Generator(device="cuda").manual_seed(72))
    acc = data.clone()
    ctx.predict(d, m, out=acc, accumulate=True)
    dat = data.reshape(obs.n_rows, obs.n_chan)[rt].cpu().numpy()
    got = acc.reshape(obs.n_rows, obs.n_chan)[rt].cpu().numpy()
    assert np.max(np.abs(got - (dat + V))) <= 1e-5 * np.max(np.abs(V))
    gains = synth.make_gains(72, obs.n_ant, obs.n_time, 1)
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    r = ctx.peel(d, m, gd, data).reshape(obs.n_rows, obs.n_chan)[rt].cpu().numpy()
    ref = oracle_peel_rows(obs, rows, gains.astype(np.complex64), dat, V)
    assert np.max(np.abs(r - ref)) <= 1e-5 * np.max(np.abs(V))
    v2 = ctx.predict(d, m).reshape(obs.n_rows, obs.n_chan)
    assert torch.equal(v, v2)
    assert ctx.device_errors() == 0
    m.free()


def _sky_part(sky, idx_p, idx_g):
    """The points idx_p and Gaussians idx_g (indices within their groups) of a point/Gaussian sky."""
    P, G = sky.n_point, sky.n_gauss
    sel = np.concatenate([np.asarray(idx_p, int), P + np.asarray(idx_g, int)])
    z = np.zeros(0)
    return synth.Sky(len(idx_p), len(idx_g), 0, sky.l[sel], sky.m[sel], sky.flux[sel], sky.alpha[sel], sky.nu_ref[sel],
                     sky.g_maj[idx_g], sky.g_min[idx_g], sky.g_pa[idx_g], z, z, z, np.zeros(0, np.int32),
                     np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32), z)


def test_mwa_full_size_properties(wn, ctx):
    """Properties that hold at any size, over all 43.7 M visibilities and 25,000 components of the
    bench's workload: V(-uvw) = conj V(uvw), and V of the whole sky = the sum of V of two disjoint halves
    (every component tile, the split tail and the fixed-order sums included)."""
    obs, sky = synth.mwa()
    d = wn.obs_to_device(obs)
    dn = wn.obs_to_device(obs)
    dn.uvw.neg_()
    m = ctx.upload(sky)
    v = ctx.predict(d, m)
    vn = ctx.predict(dn, m)
    torch.cuda.synchronize()
    scale = v.abs().max().item()
    assert (vn - v.conj()).abs().max().item() <= 2e-6 * scale
    del vn
    m.free()
    rng = np.random.default_rng(8)
    pp, pg = rng.permutation(sky.n_point), rng.permutation(sky.n_gauss)
    a = _sky_part(sky, np.sort(pp[:12000]), np.sort(pg[:2000]))
    b = _sky_part(sky, np.sort(pp[12000:]), np.sort(pg[2000:]))
    ma, mb = ctx.upload(a), ctx.upload(b)
    va = ctx.predict(d, ma)
    ctx.predict(d, mb, out=va, accumulate=True)
    torch.cuda.synchronize()
    assert (va - v).abs().max().item() <= 2e-6 * scale
    assert ctx.device_errors() == 0
    ma.free()
    mb.free()


def test_mwa_full_size_sampled_rows(wn, ctx):
    """The 43.7 M-visibility, 25,000-component workload in the bench's launch configuration, checked
    on sampled rows (all channels, all components) against the oracle."""
    obs, sky = synth.mwa()
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    gains = synth.make_gains(5, obs.n_ant, 1, 1)
    data = torch.zeros(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda")
    data.real.normal_(generator=torch.Generator(device="cuda").manual_seed(1))
    gd = torch.as_tensor(gains.astype(np.complex64)).cuda()
    r = ctx.peel(d, m, gd, data)
    torch.cuda.synchronize()
    rows = sample_rows(obs, 24, seed=3)
    V = oracle_rows(obs, sky, rows)
    dat = data.reshape(obs.n_rows, obs.n_chan)[torch.as_tensor(rows).cuda()].cpu().numpy()
    ref = oracle_peel_rows(obs, rows, gains.astype(np.complex64), dat, V)
    got = r.reshape(obs.n_rows, obs.n_chan)[torch.as_tensor(rows).cuda()].cpu().numpy()
    # the residual's reference scale is the model's
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(V))
    assert ctx.device_errors() == 0
    m.free()


@pytest.mark.parametrize("n_chan", [64, 37])
def test_output_arrays_only_8_byte_aligned(wn, ctx, n_chan):
    """An output (and data) array that starts 8 bytes past a 16-byte boundary, as a complex64 view may:
    the coalesced epilogue then writes single channels instead of 16-byte pairs; predict and peel
    results equal those of aligned arrays bit for bit."""
    obs = small_obs(31, 24, 2, synth.uniform_channels(167e6, 80e3, n_chan), layout="mwa")
    sky = synth.make_sky(32, 300, 70, 0, fov=10 * synth.DEG)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    n = obs.n_vis
    ref = ctx.predict(d, m)
    buf = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")
    view = buf[1:].view(shape)
    assert view.data_ptr() % 16 == 8
    ctx.predict(d, m, out=view)
    assert torch.equal(view, ref)
    gains = torch.as_tensor(synth.make_gains(33, obs.n_ant).astype(np.complex64)).cuda()
    data = torch.randn(shape, dtype=torch.complex64, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    rref = ctx.peel(d, m, gains, data)
    dbuf = torch.zeros(n + 1, dtype=torch.complex64, device="cuda")
    dview = dbuf[1:].view(shape)
    dview.copy_(data)
    ctx.peel(d, m, gains, dview, out=view)
    assert torch.equal(view, rref)
    m.free()
    assert ctx.device_errors() == 0
