"""Host-side fault injection (no GPU fault): device allocations made to fail as out-of-memory by
wn_debug_fail_allocs.  Each call that needs the allocation returns WN_ENOMEM with a message, frees what
it had taken, and leaves its context usable: the same call then succeeds and its result matches a
context that never saw a failure."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wn():
    import paper_2005_09316_b300 as wn
    yield wn
    wn.debug_fail_allocs(0)


def expect_enomem(wn, fn, what):
    wn.debug_fail_allocs(1)
    with pytest.raises(wn.WnError) as ei:
        fn()
    wn.debug_fail_allocs(0)
    assert ei.value.code == wn.WN_ENOMEM and what in str(ei.value), str(ei.value)


def test_model_upload_and_workspaces_fail_cleanly(wn):
    ctx = wn.Context(0)
    obs, sky = synth.tiny(7)
    d = wn.obs_to_device(obs)
    expect_enomem(wn, lambda: ctx.upload(sky), "model allocation")
    m = ctx.upload(sky)                                   # the same upload, now with memory
    ref = ctx.predict(d, m).cpu().numpy()
    # the shapelet kernel's workspace: a fresh context has none yet
    ctx2 = wn.Context(0)
    m2 = ctx2.upload(sky)
    expect_enomem(wn, lambda: ctx2.predict(d, m2), "workspace")
    assert np.array_equal(ctx2.predict(d, m2).cpu().numpy(), ref)
    # the adjoint's workspace
    gains = torch.as_tensor(synth.make_gains(8, obs.n_ant).astype(np.complex64)).cuda()
    data = torch.as_tensor(ref.astype(np.complex64)).cuda() * 1.1
    ctx3 = wn.Context(0)
    m3 = ctx3.upload(sky)
    ctx3.predict(d, m3)                                   # the forward workspace exists; the adjoint's does not
    expect_enomem(wn, lambda: ctx3.predict_grad(d, m3, gains, data), "adjoint workspace")
    g_ok = ctx3.predict_grad(d, m3, gains, data)
    g_ref = ctx.predict_grad(d, m, gains, data)
    for k in ("flux", "l", "m", "s_coeff"):
        assert np.array_equal(g_ok[k].cpu().numpy(), g_ref[k].cpu().numpy()), k
    for c in (ctx, ctx2, ctx3):
        assert c.device_errors() == 0
    for mm in (m, m2, m3):
        mm.free()
    for c in (ctx, ctx2, ctx3):
        c.close()


def test_server_pool_and_calibration_workspace_fail_cleanly(wn):
    from paper_2005_09316_b300.serve import Server
    ctx = wn.Context(0)
    expect_enomem(wn, lambda: Server(ctx, n_streams=2, pool_bytes=1 << 26, max_inflight=4, max_rows=64, max_chan=16),
                  "server pool")
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 26, max_inflight=4, max_rows=64, max_chan=16)
    srv.close()
    obs = synth.make_obs(9, 12, 1, synth.uniform_channels(167e6, 80e3, 4), layout="mwa")
    d = wn.obs_to_device(obs)
    sky = synth.make_sky(10, 20, 5, 0)
    m = ctx.upload(sky)
    model = ctx.predict(d, m)
    g0 = torch.ones((obs.n_time, obs.n_chan, obs.n_ant), dtype=torch.complex64, device="cuda")
    expect_enomem(wn, lambda: ctx.calibrate(d, model, model * 1.01, g0.clone()), "calibration workspace")
    g = ctx.calibrate(d, model, model * 1.01, g0.clone())
    assert torch.isfinite(torch.view_as_real(g)).all()
    assert ctx.device_errors() == 0
    m.free()
    ctx.close()


def test_negative_count_is_rejected(wn):
    with pytest.raises(wn.WnError) as ei:
        wn.debug_fail_allocs(-1)
    assert ei.value.code == wn.WN_EINVAL
