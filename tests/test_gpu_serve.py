"""Continuous-batching server: results alone vs in a mix, admission by memory, overlap of batches,
cancellation and bounded waits (the waits are host-side; nothing here faults or hangs a GPU)."""
import numpy as np
import pytest

import synth
from helpers import e_norm

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


def uneven_requests(wn, ctx, n, seed=17, peel_every=2):
    """n requests of uneven size: 16-48 tiles, 1-4 steps, 32-160 channels, 100-2000 P/G, 0-2 shapelets."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        n_ant = int(rng.integers(16, 49))
        n_time = int(rng.integers(1, 5))
        n_chan = int(rng.integers(32, 161))
        obs = synth.make_obs(seed + i, n_ant, n_time, synth.uniform_channels(167e6, 80e3, n_chan), layout="mwa")
        n_pg = int(rng.integers(100, 2001))
        n_sh = int(rng.integers(0, 3))
        sky = synth.make_sky(seed + 100 + i, n_pg * 4 // 5, n_pg // 5, n_sh, fov=15 * synth.DEG,
                             shape_nmax=rng.integers(10, 31, size=max(1, n_sh))[:n_sh] if n_sh else 10)
        d = wn.obs_to_device(obs)
        m = ctx.upload(sky)
        gains = data = None
        if i % peel_every == 1:
            gains = torch.as_tensor(synth.make_gains(seed + 200 + i, n_ant).astype(np.complex64)).cuda()
            data = torch.randn(n_time, obs.n_base, n_chan, dtype=torch.complex64, device="cuda",
                               generator=torch.Generator(device="cuda").manual_seed(i))
        reqs.append((d, m, gains, data))
    return reqs


def solo(ctx, req):
    d, m, gains, data = req
    return (ctx.predict(d, m) if data is None else ctx.peel(d, m, gains, data)).cpu().numpy()


def test_same_alone_and_in_the_mix(wn, ctx):
    from paper_2005_09316_b300.serve import Server
    reqs = uneven_requests(wn, ctx, 10)
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=16, max_rows=4 * 1128, max_chan=160)
    # each request alone through the server
    alone = []
    for req in reqs:
        t = srv.submit(*req)
        srv.wait(t, 60)
        alone.append(srv.result_tensor(t, req[0]).cpu().numpy())
        srv.release(t)
    # all at once: batched together
    tickets = [srv.submit(*req) for req in reqs]
    mixed = []
    for t, req in zip(tickets, reqs):
        r = srv.wait(t, 60)
        assert r.state == 3
        mixed.append(srv.result_tensor(t, req[0]).cpu().numpy())
    batches = {srv.poll(t).batch for t in tickets}
    for t in tickets:
        srv.release(t)
    assert len(batches) < len(tickets), "requests were not batched together"
    for a, b, req in zip(alone, mixed, reqs):
        assert np.array_equal(a, b)                        # bit-identical alone and in the mix
        assert e_norm(b, solo(ctx, req)) <= 1e-5           # and the same as the single-request call
    srv.close()
    assert ctx.device_errors() == 0
    for req in reqs:
        req[1].free()


def test_admission_by_memory_and_refusal(wn, ctx):
    from paper_2005_09316_b300.serve import Server
    reqs = uneven_requests(wn, ctx, 6, seed=31, peel_every=3)
    largest = max(r[0].n_vis * 8 for r in reqs)
    pool = 2 * largest + 4096                      # room for about two requests at a time
    srv = Server(ctx, n_streams=2, pool_bytes=pool, max_inflight=8, max_rows=2 * 8128, max_chan=160)
    big = synth.make_obs(99, 128, 2, synth.uniform_channels(167e6, 80e3, 64))   # within the tables, not the pool
    assert big.n_vis * 8 > pool
    dbig = wn.obs_to_device(big)
    with pytest.raises(wn.WnError) as e:
        srv.submit(dbig, reqs[0][1])
    assert e.value.code == wn.WN_EBUSY
    tickets = [srv.submit(*r) for r in reqs]
    for t, r in zip(tickets, reqs):
        res = srv.wait(t, 60)
        assert res.state == 3
        got = srv.result_tensor(t, r[0]).cpu().numpy()
        srv.release(t)
        assert e_norm(got, solo(ctx, r)) <= 1e-5
    st = srv.stats()
    assert st["free_pool_bytes"] == (pool & ~255) and st["admitted"] == 0
    srv.close()
    for r in reqs:
        r[1].free()


def test_requests_arriving_during_batches_overlap(wn, ctx):
    from paper_2005_09316_b300.serve import Server, latency_summary, poisson_arrivals, run_stream
    obs = synth.make_obs(5, 64, 4, synth.uniform_channels(167e6, 80e3, 128))
    sky = synth.make_sky(6, 3000, 600, 0)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    srv = Server(ctx, n_streams=3, pool_bytes=1 << 30, max_inflight=32, max_rows=4 * 2016, max_chan=128)
    arrivals = poisson_arrivals(np.random.default_rng(17), 2000.0, 40)
    results, wall = run_stream(srv, [(d, m, None, None)] * 40, arrivals)
    st = srv.stats()
    assert st["max_batches_in_flight"] >= 2, st
    assert all(r.state == 3 for r in results)
    lat = latency_summary(results)
    assert lat["p99_ms"] >= lat["p50_ms"] > 0
    srv.close()
    m.free()


def test_cancel_and_bounded_wait(wn, ctx):
    from paper_2005_09316_b300.serve import Server
    reqs = uneven_requests(wn, ctx, 4, seed=51, peel_every=100)
    largest = max(r[0].n_vis * 8 for r in reqs)
    srv = Server(ctx, n_streams=1, pool_bytes=largest + 1024, max_inflight=1, max_rows=4 * 1128, max_chan=160)
    tickets = [srv.submit(*r) for r in reqs]
    # with one slot and room for one output at a time, the last request is still pending
    srv.cancel(tickets[-1])
    assert srv.poll(tickets[-1]).state == 4
    with pytest.raises(wn.WnError) as e:
        srv.wait(tickets[-1] + 1000, 0.0)
    assert e.value.code == wn.WN_ENOTFOUND
    for t in tickets[:-1]:
        assert srv.wait(t, 60).state == 3
        srv.release(t)
    srv.release(tickets[-1])
    srv.close()
    for r in reqs:
        r[1].free()


@pytest.mark.parametrize("peel", [False, True])
def test_large_request_in_component_ranges(wn, ctx, peel):
    """A request above the batch work budget is served in time slices over row tiles and component
    ranges (range 0 stores or peels, later ranges add or subtract); its result matches the single call."""
    from paper_2005_09316_b300.serve import Server
    obs = synth.make_obs(71, 128, 3, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    sky = synth.make_sky(72, 16000, 4000, 1, fov=15 * synth.DEG, shape_nmax=20)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    gains = data = None
    if peel:
        gains = torch.as_tensor(synth.make_gains(73, obs.n_ant).astype(np.complex64)).cuda()
        data = torch.randn(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda",
                           generator=torch.Generator(device="cuda").manual_seed(74))
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=4, max_rows=obs.n_rows, max_chan=384)
    t = srv.submit(d, m, gains, data)
    assert srv.wait(t, 120).state == 3
    got = srv.result_tensor(t, d).cpu().numpy()
    srv.release(t)
    st = srv.stats()
    srv.close()
    assert st["batches"] >= 4, st            # several launches: tile chunks of several component ranges
    ref = solo(ctx, (d, m, gains, data))
    assert e_norm(got, ref) <= 1e-5
    assert ctx.device_errors() == 0
    m.free()


def test_large_requests_start_least_work_first(wn, ctx):
    """Queued large requests start in order of estimated work, least first (one at a time here): with a
    large request running, a larger one and then a smaller one are submitted; the smaller starts first.
    Each result still matches the single call."""
    from paper_2005_09316_b300.serve import Server
    obs = synth.make_obs(81, 128, 4, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    d = wn.obs_to_device(obs)
    models = [ctx.upload(synth.make_sky(82 + i, n * 4 // 5, n // 5, 0, fov=15 * synth.DEG))
              for i, n in enumerate((20000, 20000, 8000))]
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=4, max_rows=obs.n_rows, max_chan=384)
    tickets = [srv.submit(d, m) for m in models]   # running, then larger, then smaller
    res = [srv.wait(t, 120) for t in tickets]
    assert all(r.state == 3 for r in res)
    got = [srv.result_tensor(t, d).cpu().numpy() for t in tickets]
    for t in tickets:
        srv.release(t)
    srv.close()
    assert res[2].t_launch < res[1].t_launch, [(r.t_submit, r.t_launch) for r in res]
    for g, m in zip(got, models):
        assert e_norm(g, ctx.predict(d, m).cpu().numpy()) <= 1e-5
    assert ctx.device_errors() == 0
    for m in models:
        m.free()


def test_policy_with_no_age_limit_starts_large_requests_in_submission_order(wn, ctx):
    """With the wait limit at 0 every queued large request counts as overdue, so they start in
    submission order: the same submissions as above, and now the larger (earlier) one starts first.
    Values outside the documented ranges are refused."""
    from paper_2005_09316_b300.serve import Server
    obs = synth.make_obs(81, 128, 4, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    d = wn.obs_to_device(obs)
    models = [ctx.upload(synth.make_sky(82 + i, n * 4 // 5, n // 5, 0, fov=15 * synth.DEG))
              for i, n in enumerate((20000, 20000, 8000))]
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=4, max_rows=obs.n_rows, max_chan=384)
    for bad in ((0, 1.0), (17, 1.0), (1, -1.0), (1, float("nan"))):
        with pytest.raises(wn.WnError):
            srv.set_policy(*bad)
    srv.set_policy(1, 0.0)
    tickets = [srv.submit(d, m) for m in models]
    res = [srv.wait(t, 120) for t in tickets]
    assert all(r.state == 3 for r in res)
    got = [srv.result_tensor(t, d).cpu().numpy() for t in tickets]
    for t in tickets:
        srv.release(t)
    srv.close()
    assert res[1].t_launch < res[2].t_launch, [(r.t_submit, r.t_launch) for r in res]
    for g, m in zip(got, models):
        assert e_norm(g, ctx.predict(d, m).cpu().numpy()) <= 1e-5
    assert ctx.device_errors() == 0
    for m in models:
        m.free()
