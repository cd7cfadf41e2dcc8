"""Pipe-rate microbenchmarks (wn_pipe_rates, wn_phasor_loop_rate, wn_mma_rate, wn_mma_rate_tf32): positive,
finite, and in the relations the roofline discussion relies on (packed f32x2 FMA does the same lane work
per second as scalar FMA; MUFU ex2 and FP64 FMA are much slower pipes on this part; a tcgen05 MMA is not
faster than the nominal tensor rate allows)."""
import math

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_pipe_rates():
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    r = ctx.pipe_rates()
    ctx.close()
    assert all(math.isfinite(v) and v > 0 for v in r.values()), r
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    derived = n_sm * 128 * 2.2e9  # FP32 lanes x a clock above any B300 boost clock
    assert r["ffma"] < derived, r
    assert 0.7 < r["ffma2"] / r["ffma"] < 1.4, r
    assert r["mufu_ex2"] < 0.5 * r["ffma"], r
    assert r["dfma"] < 0.25 * r["ffma"], r


def test_phasor_loop_rate_bounds_the_kernel():
    """The channel loop alone is at least as fast as the whole prediction (which adds records, barriers
    and I/O) and below the evaluations per second the FP32 pipe allows at the loop's 4 algorithmic lane
    operations each (a step of the phasor recurrence and the complex accumulate)."""
    import numpy as np

    import paper_2005_09316_b300 as wn
    import synth
    ctx = wn.Context(0)
    loop = ctx.phasor_loop_rate()
    ffma = ctx.pipe_rates()["ffma"]
    obs, sky = synth.mwa(n_time=2)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    out = torch.empty(obs.n_time, obs.n_base, obs.n_chan, dtype=torch.complex64, device="cuda")
    for _ in range(2):
        ctx.predict(d, m, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    ts = []
    for _ in range(3):
        e0.record()
        ctx.predict(d, m, out=out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    kernel = obs.n_vis * sky.n_comp / min(ts)
    m.free()
    ctx.close()
    assert math.isfinite(loop) and loop > 0
    assert kernel <= 1.05 * loop, (kernel, loop)
    assert loop < ffma / 4.0, (loop, ffma)
    assert np.isfinite(kernel)


def test_bounded_wait_gives_up_flags_and_leaves_the_context_usable():
    """The kernels' bounded-wait helper on an mbarrier nothing arrives at, with a 0.3 s limit: the kernel
    returns after about that long, the context reports WN_DEVERR_TIMEOUT (and clears it on reading), and a
    prediction afterwards still matches the oracle."""
    import time

    import numpy as np

    import oracle
    import paper_2005_09316_b300 as wn
    import synth
    ctx = wn.Context(0)
    assert ctx.device_errors() == 0
    t0 = time.perf_counter()
    ctx.selftest_timeout(0.3)
    dt = time.perf_counter() - t0
    assert ctx.device_errors() & wn.WN_DEVERR_TIMEOUT
    assert ctx.device_errors() == 0
    assert 0.2 < dt < 5.0, dt
    obs, sky = synth.tiny(3)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    v = ctx.predict(d, m).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    ref = oracle.predict(obs.uvw.reshape(-1, 3), obs.freq, obs.dec0, sky)
    assert np.abs(v - ref).max() <= 2e-4 * np.abs(ref).max()
    assert ctx.device_errors() == 0
    m.free()
    ctx.close()


def test_mma_rate_probe():
    """tcgen05 MMAs as the shapelet kernel issues them: an M = 128, N = 128, K = 16 bf16 instruction is
    2 * 128 * 128 * 16 flops, 64 SM clocks at the nominal 8,192 dense bf16 flops per SM clock, so the
    measured clocks per instruction cannot fall below that; N = 64 cannot take longer than N = 128.
    A 16-column TMEM load and its wait take tens of clocks, not hundreds."""
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    r = ctx.mma_rate()
    assert ctx.device_errors() == 0
    ctx.close()
    assert 62.0 <= r["clk_per_mma_n128"] <= 400.0, r
    assert 0.0 < r["clk_per_mma_n64"] <= r["clk_per_mma_n128"] + 1.0, r
    assert 0.0 < r["clk_tmem_ld16"] < 200.0 and 0.0 < r["clk_tmem_ld16_x8"] < 8 * 200.0, r


def test_mma_rate_probe_tf32():
    """The tf32 form of the same instruction (M = 128, N = 128, K = 8: the same operand bytes as the bf16
    one, half its flops): the nominal dense tf32 rate is half the bf16 rate per clock, so an instruction
    cannot take fewer clocks than the bf16 one's nominal 64; N = 64 is no slower than N = 128."""
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    r = ctx.mma_rate_tf32()
    assert ctx.device_errors() == 0
    ctx.close()
    assert 62.0 <= r["clk_per_mma_n128"] <= 400.0, r
    assert 0.0 < r["clk_per_mma_n64"] <= r["clk_per_mma_n128"] + 1.0, r


def test_tracing_leaves_results_unchanged():
    """With NVTX ranges on, the entry points give bit-identical results (the ranges are host-side only)."""
    import numpy as np

    import paper_2005_09316_b300 as wn
    import synth
    ctx = wn.Context(0)
    obs, sky = synth.tiny(5)
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    v0 = ctx.predict(d, m).cpu().numpy()
    ctx.set_trace(True)
    v1 = ctx.predict(d, m).cpu().numpy()
    m2 = ctx.upload(sky)
    v2 = ctx.predict(d, m2).cpu().numpy()
    ctx.set_trace(False)
    assert np.array_equal(v0, v1) and np.array_equal(v0, v2)
    assert ctx.device_errors() == 0
    m.free()
    m2.free()
    ctx.close()
