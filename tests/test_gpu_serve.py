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
def test_large_request_in_time_step_chunks(wn, ctx, peel):
    """Small-first order: a request above the batch work budget is served in chunks of whole time steps
    through the single-request kernels (each chunk applies the request's mode to its own rows, per-step
    data and gains offset to them); its result matches the single call."""
    from paper_2005_09316_b300.serve import SERVE_SMALL_FIRST, Server
    obs = synth.make_obs(71, 128, 5, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    sky = synth.make_sky(72, 16000, 4000, 1, fov=15 * synth.DEG, shape_nmax=20)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    gains = data = None
    if peel:
        gains = torch.as_tensor(synth.make_gains(73, obs.n_ant, obs.n_time, 1).astype(np.complex64)).cuda()
        data = torch.randn(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda",
                           generator=torch.Generator(device="cuda").manual_seed(74))
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=4, max_rows=obs.n_rows, max_chan=384)
    srv.set_order(SERVE_SMALL_FIRST)
    t = srv.submit(d, m, gains, data)
    assert srv.wait(t, 120).state == 3
    got = srv.result_tensor(t, d).cpu().numpy()
    srv.release(t)
    st = srv.stats()
    srv.close()
    assert st["batches"] >= 3, st            # several launches: chunks of the time steps
    ref = solo(ctx, (d, m, gains, data))
    assert e_norm(got, ref) <= 1e-5
    assert ctx.device_errors() == 0
    m.free()


def test_large_requests_start_least_work_first(wn, ctx):
    """Small-first order: queued large requests start in order of estimated work, least first (one at a
    time here): with a large request running, a larger one and then a smaller one are submitted; the
    smaller starts first.  Each result still matches the single call."""
    from paper_2005_09316_b300.serve import SERVE_SMALL_FIRST, Server
    obs = synth.make_obs(81, 128, 4, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    d = wn.obs_to_device(obs)
    models = [ctx.upload(synth.make_sky(82 + i, n * 4 // 5, n // 5, 0, fov=15 * synth.DEG))
              for i, n in enumerate((20000, 20000, 8000))]
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=4, max_rows=obs.n_rows, max_chan=384)
    srv.set_order(SERVE_SMALL_FIRST)
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
    """Small-first order with the wait limit at 0: every queued large request counts as overdue, so they
    start in submission order: the same submissions as above, and now the larger (earlier) one starts
    first.  Values outside the documented ranges are refused."""
    from paper_2005_09316_b300.serve import SERVE_SMALL_FIRST, Server
    obs = synth.make_obs(81, 128, 4, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    d = wn.obs_to_device(obs)
    models = [ctx.upload(synth.make_sky(82 + i, n * 4 // 5, n // 5, 0, fov=15 * synth.DEG))
              for i, n in enumerate((20000, 20000, 8000))]
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=4, max_rows=obs.n_rows, max_chan=384)
    for bad in ((0, 1.0), (17, 1.0), (1, -1.0), (1, float("nan"))):
        with pytest.raises(wn.WnError):
            srv.set_policy(*bad)
    srv.set_order(SERVE_SMALL_FIRST)
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


# ---------------------------------------------------------------------------------------------------
# Served results against the FP64 oracle (Sec. 5.1 peel, eq:env_visi_def), element by element on
# sampled rows.  Bound per result: max|G| (1e-5 max|V_pg| + 2e-4 max|V_sh|) + 1e-6 max|D|, i.e. the
# FP32 phasor path's and the bf16 hi+lo tensor path's tolerances on their parts of the model (each
# max over the oracle's visibilities of that part alone on the sampled rows), scaled by the gains for
# a peel, plus the complex64 rounding of the residual.
# ---------------------------------------------------------------------------------------------------

def _split(sky):
    import copy
    n_pg = sky.n_point + sky.n_gauss
    pg, sh = copy.deepcopy(sky), copy.deepcopy(sky)
    pg.flux = np.array(sky.flux, float).copy()
    sh.flux = np.array(sky.flux, float).copy()
    pg.flux[n_pg:] = 0.0
    sh.flux[:n_pg] = 0.0
    return pg, sh


def _host_request(wn, ctx, seed, n_ant, n_time, n_chan, n_pg, nmaxs, peel):
    obs = synth.make_obs(seed, n_ant, n_time, synth.uniform_channels(167e6, 80e3, n_chan), layout="mwa")
    sky = synth.make_sky(seed + 1, n_pg * 4 // 5, n_pg - n_pg * 4 // 5, len(nmaxs), fov=15 * synth.DEG,
                         shape_nmax=np.array(nmaxs) if nmaxs else 10)
    gains = data = None
    if peel:
        gains = synth.make_gains(seed + 2, n_ant).astype(np.complex64)
        data = synth.complex_noise(seed + 3, (obs.n_rows, n_chan), 1.0).astype(np.complex64)
    return {"obs": obs, "sky": sky, "gains": gains, "data": data, "d": wn.obs_to_device(obs), "m": ctx.upload(sky),
            "gd": None if gains is None else torch.as_tensor(gains).cuda(),
            "dd": None if data is None else torch.as_tensor(data.reshape(n_time, obs.n_base, n_chan)).cuda()}


def _check_against_oracle(srv, ticket, req, n_rows=8, seed=0):
    from helpers import oracle_peel_rows, oracle_rows, sample_rows
    obs = req["obs"]
    got = srv.result_tensor(ticket, req["d"]).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    rows = sample_rows(obs, n_rows, seed)
    pg, sh = _split(req["sky"])
    Vpg, Vsh = oracle_rows(obs, pg, rows), oracle_rows(obs, sh, rows)
    V = Vpg + Vsh
    bound = 1e-5 * np.abs(Vpg).max() + (2e-4 * np.abs(Vsh).max() if req["sky"].n_shape else 0.0)
    if req["data"] is None:
        ref = V
    else:
        ref = oracle_peel_rows(obs, rows, req["gains"], req["data"][rows], V)
        bound = bound * np.abs(req["gains"]).max() ** 2 + 1e-6 * np.abs(req["data"][rows]).max()
    err = np.abs(got[rows] - ref).max()
    assert err <= bound, (ticket, err, bound)
    return err


def test_mixed_stream_matches_oracle(wn, ctx):
    """Ten uneven requests (predict and peel, 0-2 shapelets) submitted at once: at least two share one
    batched persistent launch, and every served result equals the oracle's on sampled rows."""
    from paper_2005_09316_b300.serve import Server
    rng = np.random.default_rng(91)
    reqs = []
    for i in range(10):
        nm = [int(x) for x in rng.integers(5, 25, size=int(rng.integers(0, 3)))]
        reqs.append(_host_request(wn, ctx, 900 + 10 * i, int(rng.integers(16, 41)), int(rng.integers(1, 4)),
                                  int(rng.integers(32, 129)), int(rng.integers(100, 1500)), nm, peel=bool(i % 2)))
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=16, max_rows=3 * 780, max_chan=128)
    tickets = [srv.submit(r["d"], r["m"], r["gd"], r["dd"]) for r in reqs]
    for t in tickets:
        assert srv.wait(t, 60).state == 3
    batches = [srv.poll(t).batch for t in tickets]
    assert max(batches.count(b) for b in set(batches)) >= 2, batches   # a launch ran two requests or more
    assert srv.stats()["max_batch_requests"] >= 2
    for i, (t, r) in enumerate(zip(tickets, reqs)):
        _check_against_oracle(srv, t, r, seed=i)
        srv.release(t)
    srv.close()
    assert ctx.device_errors() == 0
    for r in reqs:
        r["m"].free()


@pytest.mark.parametrize("peel", [False, True])
def test_large_request_in_time_step_chunks_matches_oracle(wn, ctx, peel):
    """A request above the batch work budget (128 tiles x 3 steps x 384 ch, 16,000 P + 4,000 G + one
    n_max 20 shapelet) with five small requests submitted behind it, in both request orders (served in
    chunks of time steps small-first, in one launch in arrival order): every result equals the oracle's
    on sampled rows."""
    from paper_2005_09316_b300.serve import SERVE_ARRIVAL, SERVE_SMALL_FIRST, Server
    big = _host_request(wn, ctx, 71, 128, 3, 384, 20000, [20], peel)
    small = [_host_request(wn, ctx, 700 + 10 * i, 24, 2, 64, 400, [8] if i == 2 else [], peel=bool(i % 2))
             for i in range(5)]
    for order in (SERVE_SMALL_FIRST, SERVE_ARRIVAL):
        srv = Server(ctx, n_streams=3, pool_bytes=1 << 30, max_inflight=8, max_rows=big["obs"].n_rows,
                     max_chan=384)
        srv.set_order(order)
        tickets = [srv.submit(r["d"], r["m"], r["gd"], r["dd"]) for r in [big] + small]
        for t in tickets:
            assert srv.wait(t, 120).state == 3
        st = srv.stats()
        batches = [srv.poll(t).batch for t in tickets]
        if order == SERVE_SMALL_FIRST:
            assert st["batches"] >= 3, st                     # the large request ran in several launches
        else:
            assert batches.count(batches[0]) == 1, batches    # the large request: a launch of its own
        _check_against_oracle(srv, tickets[0], big, n_rows=10, seed=1)
        for i, (t, r) in enumerate(zip(tickets[1:], small)):
            _check_against_oracle(srv, t, r, seed=2 + i)
        for t in tickets:
            srv.release(t)
        srv.close()
    assert ctx.device_errors() == 0
    for r in [big] + small:
        r["m"].free()


def test_arrival_order_starts_large_requests_in_submission_order(wn, ctx):
    """The default (arrival) order: with a large request running, a larger one and then a smaller one are
    submitted, and they start in submission order whatever their size, each in one launch; results match
    the single call.  An unknown order is refused."""
    from paper_2005_09316_b300.serve import Server
    obs = synth.make_obs(81, 128, 4, synth.uniform_channels(167e6, 80e3, 384), layout="mwa")
    d = wn.obs_to_device(obs)
    models = [ctx.upload(synth.make_sky(82 + i, n * 4 // 5, n // 5, 0, fov=15 * synth.DEG))
              for i, n in enumerate((20000, 20000, 8000))]
    srv = Server(ctx, n_streams=2, pool_bytes=1 << 30, max_inflight=4, max_rows=obs.n_rows, max_chan=384)
    for bad in (-1, 2):
        with pytest.raises(wn.WnError):
            srv.set_order(bad)
    tickets = [srv.submit(d, m) for m in models]
    res = [srv.wait(t, 120) for t in tickets]
    assert all(r.state == 3 for r in res)
    got = [srv.result_tensor(t, d).cpu().numpy() for t in tickets]
    for t in tickets:
        srv.release(t)
    st = srv.stats()
    srv.close()
    assert res[0].t_launch <= res[1].t_launch < res[2].t_launch, [(r.t_submit, r.t_launch) for r in res]
    assert st["batches"] == 3, st
    for g, m in zip(got, models):
        assert e_norm(g, ctx.predict(d, m).cpu().numpy()) <= 1e-5
    assert ctx.device_errors() == 0
    for m in models:
        m.free()


def test_solo_requests_run_alone_and_match_the_oracle(wn, ctx):
    """Small requests that batching would not help run alone through the single-request kernels: one
    with few rows and channels but many components (a short grid of long tiles, 1 step x 1,830
    baselines x 88 ch x 13,000 P/G) and one of more than 1 ms of estimated work (2 steps x 2,016
    baselines x 128 ch x 8,000 P/G, peeled).  Each runs in a launch of its own, its result is the
    single-request call's bit for bit, and it equals the oracle's on sampled rows; three tiny
    requests submitted with them are served as before."""
    from paper_2005_09316_b300.serve import Server
    short = _host_request(wn, ctx, 1300, 61, 1, 88, 13000, [], peel=False)
    heavy = _host_request(wn, ctx, 1310, 64, 2, 128, 8000, [], peel=True)
    tiny = [_host_request(wn, ctx, 1320 + 10 * i, 24, 2, 64, 400, [6] if i == 1 else [], peel=bool(i % 2))
            for i in range(3)]
    reqs = [short, heavy] + tiny
    srv = Server(ctx, n_streams=3, pool_bytes=1 << 30, max_inflight=8, max_rows=2 * 2016, max_chan=128)
    tickets = [srv.submit(r["d"], r["m"], r["gd"], r["dd"]) for r in reqs]
    for t in tickets:
        assert srv.wait(t, 60).state == 3
    batches = [srv.poll(t).batch for t in tickets]
    for k in (0, 1):
        assert batches.count(batches[k]) == 1, batches     # a launch of its own
    for i, (t, r) in enumerate(zip(tickets, reqs)):
        _check_against_oracle(srv, t, r, seed=20 + i)
    for t, r in zip(tickets[:2], reqs[:2]):
        got = srv.result_tensor(t, r["d"]).cpu().numpy()
        assert np.array_equal(got, solo(ctx, (r["d"], r["m"], r["gd"], r["dd"])))
    for t in tickets:
        srv.release(t)
    srv.close()
    assert ctx.device_errors() == 0
    for r in reqs:
        r["m"].free()
