"""Benchmark: component-visibility evaluations per second of the fused predict + peel.

Workload (the paper's MWA Phase I simulation shape): 128 tiles (8128 baselines), 14 time steps,
384 x 80 kHz channels from 167 MHz, 20,000 points + 5,000 Gaussians within 20 deg; one step is
wn_peel over the whole observation (prediction of every visibility fused with
R = D - g_ant1 conj(g_ant2) V).  Inputs are seeded synthetic data of that shape (synth.mwa).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a bounded sample of
the same workload instead.  Under torchrun every rank runs the full workload on its own GPU
(independent observations, no collective: weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "comp-vis evals/s (mixed vs FP64 GPU) at stated error; % roofline; p50/p99"
UNIT = "comp-vis evals/s"
WORKLOAD = "mwa_phase1_predict_peel: 128 tiles (8128 baselines) x 14 steps x 384 ch, 20000 P + 5000 G"
# Algorithmic FP32-pipe operations per component-visibility evaluation of the phasor sum: one step
# of the three-term phasor recurrence across channels (1 FFMA for each of the real and imaginary
# parts) and one complex accumulate of amplitude x phasor (2 FFMA).
OPS_PER_EVAL = 4
FP32_LANES_PER_SM = 128


def traffic_record(name: str):
    """DRAM bytes per launch of a kernel from a committed ncu record in profiles/, or None when the kernel
    sources have changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    try:
        rec = json.load(open(path))
        m = hashlib.sha256()
        for p in rec["sources"]:
            m.update(open(os.path.join(ROOT, p), "rb").read())
        return rec["dram_bytes_per_launch"] if m.hexdigest() == rec["sources_sha256"] else None
    except Exception:
        return None


def k1_traffic():
    return traffic_record("k1_phasor_mwa_traffic.json")


def count_launches(step, torch):
    """The library's kernels that one step launches, counted from the CUDA activity trace of one extra
    untimed step (torch.profiler); returns (count, {kernel: launches}) or (None, reason)."""
    try:
        import warnings

        from torch.profiler import ProfilerActivity, profile
        torch.cuda.synchronize()
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            with profile(activities=[ProfilerActivity.CUDA]) as prof:
                step()
                torch.cuda.synchronize()
        names = {}
        for e in prof.key_averages():
            if "wn::" in e.key and e.count:
                short = e.key.split("wn::", 1)[1].split("(", 1)[0]
                names[short] = names.get(short, 0) + int(e.count)
        return (sum(names.values()) or None), names
    except Exception as exc:  # noqa: BLE001 - reported in the line, not fatal
        return None, f"unavailable: {type(exc).__name__}: {exc}"


def peaks():
    p = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
    return p


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            lines = [ln.split(",") for ln in open(self.path).read().strip().splitlines() if ln.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for f in lines:
            f = [x.strip() for x in f]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        os.unlink(self.path)
        return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_rate(obs, sky, target_s: float, rows_cap: int = 4096, seed: int = 0):
    """FP64 oracle evaluations/s on a sample of rows sized to ~target_s seconds."""
    import oracle
    rng = np.random.default_rng(seed)
    probe = rng.choice(obs.n_rows, size=2 * max(1, oracle.max_threads()), replace=False)
    t0 = time.perf_counter()
    oracle.predict(synth.sub_obs(obs, probe), obs.freq, obs.dec0, sky)
    dt = time.perf_counter() - t0
    n = int(min(rows_cap, max(len(probe), len(probe) * target_s / max(dt, 1e-6))))
    rows = np.sort(rng.choice(obs.n_rows, size=n, replace=False))
    t0 = time.perf_counter()
    oracle.predict(synth.sub_obs(obs, rows), obs.freq, obs.dec0, sky)
    dt = time.perf_counter() - t0
    evals = len(rows) * obs.n_chan * sky.n_comp
    return evals / dt, dict(rows=int(len(rows)), evals=int(evals), seconds=round(dt, 3))


def run_reference(args):
    """The FP64 CPU oracle, timed on a bounded sample of the workload per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    obs, sky = synth.mwa()
    rng = np.random.default_rng(7)
    n_rows = max(1, 2 * oracle.max_threads())
    rates, times = [], []
    for step in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(obs.n_rows, size=n_rows, replace=False))
        t0 = time.perf_counter()
        oracle.predict(synth.sub_obs(obs, rows), obs.freq, obs.dec0, sky)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            rates.append(n_rows * obs.n_chan * sky.n_comp / dt)
            times.append(dt)
    value = float(np.mean(rates))
    ms = 1e3 * float(np.mean(times))   # one step: the bounded sample this arm times
    ms_full = 1e3 * obs.n_vis * sky.n_comp / value
    sample = f"{n_rows} random rows x 384 ch x 25000 comps per step (of 113792 rows)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "ms_per_full_workload_step": ms_full,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def bench_shapelets(wn, ctx, local, P, torch):
    """Fornax-like peel: two n_max = 80 shapelets (1,500 coefficients each) over the 5 km observation,
    beside the equivalent 40,000-component point/Gaussian model (the paper's shapelet vs MS CLEAN cost)."""
    import oracle
    obs, sky = synth.fornax()
    d = wn.obs_to_device(obs, f"cuda:{local}")
    m = ctx.upload(sky)
    gains_np = synth.make_gains(7, obs.n_ant).astype(np.complex64)
    gains = torch.as_tensor(gains_np).cuda()
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    data = torch.randn(shape, dtype=torch.complex64, device=f"cuda:{local}",
                       generator=torch.Generator(device=f"cuda:{local}").manual_seed(5))
    out = torch.empty_like(data)

    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    ms = timed(lambda: ctx.peel(d, m, gains, data, out=out), 10)
    nnz = int(sky.s_off[-1])
    # the dense operands are sized by the highest order each shapelet's coefficients reach
    n_eff = [int(np.max(sky.s_n1[a:b] + sky.s_n2[a:b])) for a, b in zip(sky.s_off[:-1], sky.s_off[1:])]
    pads = [((n + 1 + 15) // 16 * 16, (2 * (n + 1) + 15) // 16 * 16) for n in n_eff]
    flops = sum(2.0 * obs.n_vis * kp * npad * 3 for kp, npad in pads)
    tf = flops / (ms * 1e-3) / 1e12
    tf_useful = 2.0 * nnz_all(sky) * obs.n_vis / (ms * 1e-3) / 1e12
    peak = float(P.get("bf16_tflops", 1800.0))
    rows = np.sort(np.random.default_rng(5).choice(obs.n_rows, size=16, replace=False))
    V = oracle.predict(synth.sub_obs(obs, rows), obs.freq, obs.dec0, sky)
    rt, rb = rows // obs.n_base, rows % obs.n_base
    idx = torch.as_tensor(rows).cuda()
    dat = data.reshape(obs.n_rows, obs.n_chan)[idx].cpu().numpy()
    ref = oracle.peel(rt, rb, obs.ant1, obs.ant2, obs.n_ant, gains_np, dat, V)
    got = out.reshape(obs.n_rows, obs.n_chan)[idx].cpu().numpy()
    err = float(np.abs(got - ref).max() / np.abs(V).max())
    # the same peel with the basis interpolated from the 1-D lookup table (Sec. 3.2) instead of the recurrence
    ctx.set_precision(0, wn.WN_SHAPE_LUT_BF16X3)
    ms_lut = timed(lambda: ctx.peel(d, m, gains, data, out=out), 10)
    got_lut = out.reshape(obs.n_rows, obs.n_chan)[idx].cpu().numpy()
    err_lut = float(np.abs(got_lut - ref).max() / np.abs(V).max())
    # the same peel with tf32 operands and one product (kind::tf32)
    ctx.set_precision(0, wn.WN_SHAPE_TF32)
    ms_tf32 = timed(lambda: ctx.peel(d, m, gains, data, out=out), 10)
    got_tf32 = out.reshape(obs.n_rows, obs.n_chan)[idx].cpu().numpy()
    err_tf32 = float(np.abs(got_tf32 - ref).max() / np.abs(V).max())
    # tf32 hi + lo operands, three products
    ctx.set_precision(0, wn.WN_SHAPE_TF32X3)
    ms_tf32x3 = timed(lambda: ctx.peel(d, m, gains, data, out=out), 10)
    got_x3 = out.reshape(obs.n_rows, obs.n_chan)[idx].cpu().numpy()
    err_x3 = float(np.abs(got_x3 - ref).max() / np.abs(V).max())
    ctx.set_precision(0, wn.WN_SHAPE_BF16X3)
    tf_tf32 = sum(2.0 * obs.n_vis * kp * npad for kp, npad in pads) / (ms_tf32 * 1e-3) / 1e12  # one product
    tf_x3 = 3.0 * sum(2.0 * obs.n_vis * kp * npad for kp, npad in pads) / (ms_tf32x3 * 1e-3) / 1e12
    peak_tf32, tf32_basis = measured_tf32_peak(torch)
    if peak_tf32 is None:
        peak_tf32, tf32_basis = peak / 2.0, "measured bf16 peak x the nominal tf32/bf16 ratio 1/2"
    try:  # the kernel's own instruction, timed alone: clocks per MMA of each kind at N = 128
        c16, c32 = ctx.mma_rate()["clk_per_mma_n128"], ctx.mma_rate_tf32()["clk_per_mma_n128"]
        mma_ratio = {"clk_bf16_k16": round(c16, 2), "clk_tf32_k8": round(c32, 2),
                     "tf32_over_bf16_flops": round(c16 / (2.0 * c32), 4)}
    except Exception as exc:  # noqa: BLE001 - reported, not fatal
        mma_ratio = f"unavailable: {exc}"
    m.free()
    # the equivalent multi-scale-CLEAN-like model on the same observation
    _, clean = synth.fornax_clean()
    mc = ctx.upload(clean)
    ms_clean = timed(lambda: ctx.peel(d, mc, gains, data, out=out), 2)
    mc.free()
    return {"workload": "fornax_peel: 128 tiles (5 km) x 14 x 384 ch, 2 shapelets n_max 80, 1500 coeffs each",
            "orders_present": n_eff, "k_pad_n_pad": pads,
            "ms_per_step": round(ms, 4), "shapelet_vis_per_s": obs.n_vis * sky.n_shape / (ms * 1e-3),
            "coeff_vis_per_s": nnz * obs.n_vis / (ms * 1e-3),
            "roofline": {"bound": "tensor", "achieved": round(tf, 2), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(tf / peak, 4),
                         "traffic": traffic_record("k2_shapelet_fornax_traffic.json"),
                         "traffic_unit": "bytes per launch (one launch sums both shapelets and writes the residual "
                                         "once; ncu dram__bytes_read + write, full size)",
                         "algorithmic_bytes": 16 * obs.n_vis,
                         "useful_achieved": round(tf_useful, 2), "useful_frac": round(tf_useful / peak, 4),
                         "note": "issued bf16 flops (2 k_pad n_pad x 3 products per visibility); useful: "
                                 "2 nnz per visibility"},
            "error": {"e_norm": err, "tolerance": 1e-3, "sample": "16 rows x 384 ch vs oracle peel"},
            "tf32": {"ms_per_step": round(ms_tf32, 4), "e_norm": err_tf32,
                     "roofline": {"bound": "tensor", "achieved": round(tf_tf32, 2), "peak": round(peak_tf32, 1),
                                  "unit": "TFLOP/s", "frac": round(tf_tf32 / peak_tf32, 4), "peak_basis": tf32_basis,
                                  "tcgen05_clocks": mma_ratio},
                     "note": "tf32 operands rounded to nearest, one product per visibility"},
            "tf32x3": {"ms_per_step": round(ms_tf32x3, 4), "e_norm": err_x3,
                       "roofline": {"bound": "tensor", "achieved": round(tf_x3, 2), "peak": round(peak_tf32, 1),
                                    "unit": "TFLOP/s", "frac": round(tf_x3 / peak_tf32, 4), "peak_basis": tf32_basis},
                       "note": "tf32 hi+lo operands, three products (hi*hi + hi*lo + lo*hi) per visibility"},
            "lookup_table_basis": {"ms_per_step": round(ms_lut, 4), "e_norm": err_lut,
                                   "note": "phi_n interpolated from a 1/256-spaced table in L2 instead of the recurrence"},
            "clean_model_40k_ms": round(ms_clean, 3), "clean_over_shapelet_time": round(ms_clean / ms, 2)}


def measured_tf32_peak(torch):
    """Dense tf32 tensor throughput of this GPU, measured as the bf16 peak is: cuBLAS through torch, an
    8192^3 float32 matmul with tf32 allowed (2 N^3 flops), best of 10 after warm-up."""
    try:
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        n = 8192
        a = torch.randn(n, n, device="cuda", dtype=torch.float32)
        b = torch.randn(n, n, device="cuda", dtype=torch.float32)
        for _ in range(3):
            a @ b
        torch.cuda.synchronize()
        best = float("inf")
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        for _ in range(10):
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        torch.backends.cuda.matmul.allow_tf32 = prev
        del a, b
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12, "measured: cuBLAS tf32 GEMM 8192^3 (torch, tf32 allowed), best of 10, this run"
    except Exception:  # noqa: BLE001 - fall back to the nominal ratio
        return None, None


def nnz_all(sky) -> int:
    return int(sky.s_off[-1]) if sky.n_shape else 0


def summary_block(line: dict) -> dict:
    """The sub-results in a few hundred bytes, so that a reader of the line's tail sees each of them."""
    def g(*path):
        d = line
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return float(f"{d:.4g}") if isinstance(d, float) else d

    def small_first():  # the serving stream under the small-first order with the 1 s wait limit
        for o in (line.get("serving") or {}).get("other_policies") or []:
            if o.get("order") == "small_first" and o.get("max_large_wait_s") == 1.0:
                c = o.get("p99_by_class") or {}
                return {"p50_ms": o.get("p50_ms"), "p99_ms": o.get("p99_ms"),
                        "small_p99_ms": (c.get("below_20ms") or {}).get("p99_ms"),
                        "large_p99_ms": (c.get("20ms_and_above") or {}).get("p99_ms")}
        return None
    return {
        "k1": {"evals_per_s": g("value"), "frac": g("roofline", "frac"), "e_norm": g("error", "e_norm"),
               "loop_bound_frac": g("roofline", "loop_bound", "frac")},
        "k2_fornax": {"ms": g("shapelet", "ms_per_step"), "issued_frac": g("shapelet", "roofline", "frac"),
                      "useful_frac": g("shapelet", "roofline", "useful_frac"), "e_norm": g("shapelet", "error", "e_norm"),
                      "tf32_ms": g("shapelet", "tf32", "ms_per_step"), "tf32x3_ms": g("shapelet", "tf32x3", "ms_per_step"),
                      "tf32x3_e_norm": g("shapelet", "tf32x3", "e_norm")},
        "k3_peel": {"gbs": g("standalone_peel", "achieved_gbs"), "frac": g("standalone_peel", "frac")},
        "k4_adjoint_ms": g("adjoint", "ms_per_step"), "fit_step_ms": g("adjoint", "autograd_fit_step_ms"),
        "k5_fp64": {"evals_per_s": g("fp64_gpu", "value"), "speedup": g("fp64_gpu", "speedup_mixed_over_fp64"),
                    "untuned_speedup": g("fp64_gpu_untuned", "speedup_mixed_over_untuned")},
        "k7_calib_ms": g("calibration", "ms"), "k8_fit_ms_per_iter": g("fit", "ms_per_iteration"),
        "serving": {"order": g("serving", "policy", "order"), "p50_ms": g("serving", "p50_ms"), "p99_ms": g("serving", "p99_ms"),
                    "one_at_a_time_p50_ms": g("serving", "one_at_a_time_p50_ms"),
                    "one_at_a_time_p99_ms": g("serving", "one_at_a_time_p99_ms"),
                    "large_p99_ms": g("serving", "p99_by_class", "20ms_and_above", "p99_ms"),
                    "large_one_at_a_time_p99_ms": g("serving", "p99_by_class", "20ms_and_above", "one_at_a_time_p99_ms"),
                    "small_p99_ms": g("serving", "p99_by_class", "below_20ms", "p99_ms"),
                    "small_one_at_a_time_p99_ms": g("serving", "p99_by_class", "below_20ms", "one_at_a_time_p99_ms"),
                    "max_batch_requests": g("serving", "max_batch_requests"),
                    "burst_gain": g("serving", "burst", "throughput_gain"),
                    "burst_max_batch_requests": g("serving", "burst", "max_batch_requests"),
                    "small_first": small_first()},
        "e2e": g("e2e", "value"), "cpu_baseline": g("cpu_baseline", "value"),
    }


def bench_calibration(wn, ctx, local, torch, n_iter=10):
    """Gain calibration (Sec. 5.1, eq:peeling-iter) of the MWA case: 14 x 384 (time, channel) problems of
    128 antennas (255 real parameters each), n_iter iterations, model from the library's prediction of
    2,000 points + 500 Gaussians, data from known per-(t, f) gains 1 + N(0, 0.05) plus noise."""
    import oracle
    obs, _ = synth.mwa()
    sky = synth.make_sky(102, 2000, 500, 0)
    d = wn.obs_to_device(obs, f"cuda:{local}")
    m = ctx.upload(sky)
    I = ctx.predict(d, m)
    m.free()
    rng = np.random.default_rng(23)
    T, B, F, A = obs.n_time, obs.n_base, obs.n_chan, obs.n_ant
    g_true = (1 + 0.05 * (rng.normal(size=(T, F, A)) + 1j * rng.normal(size=(T, F, A)))).astype(np.complex64)
    gt = torch.as_tensor(g_true).cuda()
    a1 = torch.as_tensor(obs.ant1.astype(np.int64)).cuda()
    a2 = torch.as_tensor(obs.ant2.astype(np.int64)).cuda()
    G = (gt[:, :, a1] * torch.conj(gt[:, :, a2])).permute(0, 2, 1)          # [T, B, F]
    sigma = 0.01 * float(I.abs().mean())
    gen = torch.Generator(device=f"cuda:{local}").manual_seed(24)
    noise = torch.complex(torch.randn(I.shape, generator=gen, device=I.device),
                          torch.randn(I.shape, generator=gen, device=I.device)) * sigma
    V = (G * I + noise).contiguous()
    g0 = torch.ones((T, F, A), dtype=torch.complex64, device=I.device)
    ctx.calibrate(d, I, V, g0.clone(), n_iter=n_iter)                        # warm-up
    ev = [torch.cuda.Event(True) for _ in range(2)]
    times = []
    for _ in range(3):
        g = g0.clone()
        torch.cuda.synchronize()
        ev[0].record()
        ctx.calibrate(d, I, V, g, n_iter=n_iter)
        ev[1].record()
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    flags = ctx.device_errors()
    ms = float(np.median(times))
    gg = g.cpu().numpy().astype(np.complex128)
    want = g_true.astype(np.complex128) * np.exp(-1j * np.angle(g_true[:, :, :1].astype(np.complex128)))
    resid = ctx.peel_model(d, g, V, I)
    rms = float(resid.abs().pow(2).mean().sqrt())
    # oracle on two (t, f) problems, same start and iteration count
    Ih, Vh = I.cpu().numpy().astype(np.complex128), V.cpu().numpy().astype(np.complex128)
    t0 = time.perf_counter()
    par = 0.0
    for (t, f) in ((0, 0), (T - 1, F // 2)):
        ref = oracle.calibrate(obs.ant1, obs.ant2, A, Ih[t:t + 1, :, f:f + 1], Vh[t:t + 1, :, f:f + 1],
                               np.ones((1, 1, A)), n_iter)
        par = max(par, float(np.abs(gg[t, f] - ref[0, 0]).max()))
    cpu_s = (time.perf_counter() - t0) / 2
    n = 2 * A - 1
    flops = T * F * n_iter * (n ** 3 / 3 + 2 * n * n + 60 * B)
    return {"workload": f"calibration: {T} x {F} (time, channel) problems, {A} antennas ({n} parameters), "
                        f"{n_iter} iterations, model 2000 P + 500 G, gains 1+N(0,0.05), noise 1% of |model|",
            "ms": round(ms, 3), "solves_per_s": T * F * n_iter / (ms * 1e-3),
            "achieved_tflops": round(flops / (ms * 1e-3) / 1e12, 3),
            "note": "FP32 normal equations (Cholesky n^3/3 + solves + accumulation) per solve; one problem per SM",
            "gain_error_max": float(np.abs(gg - want).max()), "parity_vs_oracle_max": par,
            "resid_rms_over_noise": round(rms / (sigma * np.sqrt(2)), 4), "device_errors": flags,
            "oracle_cpu_s_per_problem": round(cpu_s, 3)}


def bench_fit(wn, ctx, local, torch, n_iter=300, tol=1e-5):
    """Visibility-space fit of one n_max 40 shapelet (861 coefficients) with 500 fixed points, on 64 tiles
    x 4 steps x 64 channels: data = gains x model(true coefficients) + noise, fitted from zero."""
    obs, sky = synth.adjoint()
    rows = np.arange(obs.n_rows)
    gains_np = synth.make_gains(31, obs.n_ant).astype(np.complex64)
    d = wn.obs_to_device(obs, f"cuda:{local}")
    gd = torch.as_tensor(gains_np).cuda()
    m_true = ctx.upload(sky)
    clean = torch.zeros((obs.n_time, obs.n_base, obs.n_chan), dtype=torch.complex64, device=f"cuda:{local}")
    model = ctx.peel(d, m_true, gd, clean)                     # -G V
    m_true.free()
    sigma = 0.01 * float(model.abs().mean())
    gen = torch.Generator(device=f"cuda:{local}").manual_seed(32)
    data = (-model + sigma * torch.complex(torch.randn(model.shape, generator=gen, device=model.device),
                                           torch.randn(model.shape, generator=gen, device=model.device))).contiguous()
    start = sky.__class__(**sky.__dict__)
    start.s_coeff = np.zeros_like(sky.s_coeff)
    m = ctx.upload(start)
    ctx.fit_shapelets(d, m, gd, data, n_iter=5, tol=0.0)      # warm-up
    m.free()
    m = ctx.upload(start)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c, info = ctx.fit_shapelets(d, m, gd, data, n_iter=n_iter, tol=tol)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    fitted = ctx.peel(d, m, gd, clean)                        # -G V with the fitted coefficients
    m.free()
    cc = c.cpu().numpy()
    del rows
    return {"workload": "fit: 64 tiles x 4 x 64 ch, 500 P fixed + 1 shapelet n_max 40 (861 coefficients), "
                        "gains 1+N(0,0.05), noise 1% of |model|, CGLS from zero",
            "s": round(wall, 4), "iterations": info["iterations"], "ms_per_iteration": round(1e3 * wall / max(1, info["iterations"]), 3),
            "rel_normal_residual": info["rel_grad"], "resid2_over_noise2": info["resid2"] / (2 * sigma * sigma * obs.n_vis),
            "model_error_rel": float((fitted - model).abs().max() / model.abs().max()),
            "coeff_error_rel": float(np.abs(cc - sky.s_coeff).max() / np.abs(sky.s_coeff).max()),
            "note": "orders the array does not sample are unconstrained: the coefficients differ where the visibilities do not"}


def bench_truncation(wn, ctx, local, torch, fractions=(1.0, 0.999, 0.99, 0.95, 0.9, 0.8)):
    """Model truncation (Sec. 6.2) on the Fornax observation: GPU prediction time and model error against
    the full model as f_comp falls, for the 40,000-component point/Gaussian model and for the two
    n_max 80 shapelets.  Model error = max |V_f - V_full| / max |V_full| over every visibility."""
    from paper_2005_09316_b300 import truncate as tr
    obs, sky_s = synth.fornax()
    _, sky_c = synth.fornax_clean()
    d = wn.obs_to_device(obs, f"cuda:{local}")
    ev = [torch.cuda.Event(True) for _ in range(2)]
    out = {"workload": "fornax observation (128 tiles, 5 km, 14 x 384 ch): 40000 P/G model and 2 shapelets n_max 80"}
    for name, sky, reps in (("clean_40k", sky_c, 1), ("shapelets", sky_s, 3)):
        rows = []
        full = None
        for f in fractions:
            t, info = tr.truncate(sky, f)
            m = ctx.upload(t)
            v = ctx.predict(d, m)                      # warm-up, and the visibilities for the error
            torch.cuda.synchronize()
            ev[0].record()
            for _ in range(reps):
                ctx.predict(d, m, out=v)
            ev[1].record()
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / reps
            m.free()
            if full is None:
                full, vmax = v, float(v.abs().max())
                err = 0.0
            else:
                err = float((v - full).abs().max()) / vmax
            rows.append({"f_comp": f, "n_comp": info["n_comp"], "flux_fraction_kept": round(info["flux_fraction_kept"], 6),
                         "n_max": [int(x) for x in t.s_nmax] if t.n_shape else None,
                         "ms": round(ms, 3), "model_error": err})
        out[name] = rows
        del full
    return out


def bench_adjoint(wn, ctx, local, torch):
    """Adjoint (loss and every gradient) on 64 tiles x 4 steps x 64 channels, 500 points + 1 shapelet."""
    obs, sky = synth.adjoint()
    d = wn.obs_to_device(obs, f"cuda:{local}")
    m = ctx.upload(sky)
    gains = torch.as_tensor(synth.make_gains(9, obs.n_ant).astype(np.complex64)).cuda()
    data = torch.randn((obs.n_time, obs.n_base, obs.n_chan), dtype=torch.complex64, device=f"cuda:{local}",
                       generator=torch.Generator(device=f"cuda:{local}").manual_seed(9))
    resid = torch.empty_like(data)
    for _ in range(3):
        ctx.predict_grad(d, m, gains, data, resid=resid)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record()
    n = 5
    for _ in range(n):
        ctx.predict_grad(d, m, gains, data, resid=resid)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    m.free()
    # one gradient step of a fit through the autograd loss (forward + backward + optimiser update), with the
    # model re-packed in place (wn_sky_update) and with a model uploaded and freed per call; wall clock
    from paper_2005_09316_b300.autograd import peel_loss
    skyd = wn.sky_to_device(sky, f"cuda:{local}")
    params = {k: skyd[k].clone().requires_grad_(True) for k in ("flux", "s_coeff")}
    skyd.update(params)
    opt = torch.optim.SGD(params.values(), lr=0.0)
    resident = ctx.upload(sky)
    step_ms = {}
    def fit_steps(mdl, n):
        for _ in range(n):
            opt.zero_grad()
            peel_loss(ctx, d, skyd, gains, data, model=mdl).backward()
            opt.step()

    for name, mdl in (("resident_model", resident), ("upload_per_call", None)):
        fit_steps(mdl, 3)
        rounds = []
        for _ in range(5):  # host-driven steps: the median of five rounds of ten
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fit_steps(mdl, 10)
            torch.cuda.synchronize()
            rounds.append((time.perf_counter() - t0) / 10)
        step_ms[name] = round(1e3 * float(np.median(rounds)), 3)
    resident.free()
    return {"workload": "adjoint: 64 tiles (2016 baselines) x 4 x 64 ch, 500 P + 1 S (n_max 40)",
            "ms_per_step": round(ms, 4), "grad_evals_per_s": obs.n_vis * sky.n_comp / (ms * 1e-3),
            "autograd_fit_step_ms": step_ms}


def bench_serving(wn, ctx, local, torch, n_req=1000, n_templates=48, seed=17, policy=None, n_burst=256,
                  detail=None, order=None, extra_policies=((1, 1, 1.0), (1, 1, 0.3))):
    """Seeded Poisson stream of predict/peel requests of uneven size (16-128 tiles, 1-14 steps, 32-384
    channels, 100-50,000 P/G, 0-3 shapelets with n_max 10-80), models resident.  Requests are drawn
    uniformly from n_templates distinct (observation, sky, data) sets; the arrival rate is set for ~70%
    GPU busy from the measured one-at-a-time service times.  The one-at-a-time reference is measured: the
    same requests at the same arrival times run one after another through the single-request calls.  A
    burst phase submits n_burst requests of the sets that take under 5 ms alone at once, so that batches
    of several requests form, and compares the wall time with the same burst run one at a time.
    order: the request order (serve.SERVE_ARRIVAL or SERVE_SMALL_FIRST); None keeps the default (arrival).
    policy: (large requests in flight, wait limit in s) for Server.set_policy; None keeps the defaults.
    extra_policies: further (order, large requests in flight, wait limit) the same stream is played under
    (latencies only); by default small-first with the 1 s and the 0.3 s wait limits."""
    from paper_2005_09316_b300.serve import Server, latency_summary, poisson_arrivals, run_sequential, run_stream
    order_names = {0: "arrival", 1: "small_first"}
    rng = np.random.default_rng(seed)
    temps, models = [], []
    for i in range(n_templates):
        n_ant = int(round(np.exp(rng.uniform(np.log(16), np.log(128)))))
        n_time = int(rng.integers(1, 15))
        n_chan = int(rng.integers(32, 385))
        n_pg = int(round(np.exp(rng.uniform(np.log(100), np.log(50000)))))
        n_sh = int(rng.integers(0, 4))
        obs = synth.make_obs(seed + i, n_ant, n_time, synth.uniform_channels(167e6, 80e3, n_chan), layout="mwa")
        sky = synth.make_sky(seed + 1000 + i, n_pg * 4 // 5, n_pg - n_pg * 4 // 5, n_sh, fov=20 * synth.DEG,
                             shape_nmax=rng.integers(10, 81, size=max(n_sh, 1))[:n_sh] if n_sh else 10,
                             shape_beta=(3 * synth.ARCMIN, 15 * synth.ARCMIN))
        d = wn.obs_to_device(obs, f"cuda:{local}")
        m = ctx.upload(sky)
        models.append(m)
        gains = data = None
        if i % 2:
            gains = torch.as_tensor(synth.make_gains(seed + 2000 + i, n_ant).astype(np.complex64)).cuda()
            data = torch.randn((n_time, obs.n_base, n_chan), dtype=torch.complex64, device=f"cuda:{local}",
                               generator=torch.Generator(device=f"cuda:{local}").manual_seed(i))
        temps.append((d, m, gains, data))
    # one-at-a-time service time of each template (each alone, synchronously; median of 3), for the rate
    svc_t = []
    for d, m, gains, data in temps:
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            (ctx.predict(d, m) if data is None else ctx.peel(d, m, gains, data))
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        svc_t.append(float(np.median(ts)))
    pick = np.random.default_rng(seed + 1).integers(0, n_templates, size=n_req)
    reqs = [temps[k] for k in pick]
    svc = np.array([svc_t[k] for k in pick])
    mean_s = float(np.mean(svc))
    rate = 0.7 / mean_s
    arrivals = poisson_arrivals(np.random.default_rng(seed), rate, n_req)
    max_rows = max(r[0].n_rows for r in temps)

    def server():
        srv = Server(ctx, n_streams=6, pool_bytes=6 << 30, max_inflight=32, max_rows=max_rows, max_chan=384)
        if order is not None:
            srv.set_order(order)
        if policy is not None:
            srv.set_policy(*policy)
        return srv

    srv = server()
    results, wall = run_stream(srv, reqs, arrivals)
    st = srv.stats()
    srv.close()
    lat_seq, svc_seq, wall_seq = run_sequential(ctx, reqs, arrivals)
    seq_a = np.array(lat_seq)

    def classes(res):
        lat_a = np.array([r.latency for r in res])
        out = {}
        for name, sel in (("below_20ms", svc < 0.02), ("20ms_and_above", svc >= 0.02)):
            if not sel.any():  # a stream without requests of this class
                out[name] = {"n": 0}
                continue
            out[name] = {"n": int(sel.sum()), "p50_ms": round(1e3 * float(np.percentile(lat_a[sel], 50)), 3),
                         "p99_ms": round(1e3 * float(np.percentile(lat_a[sel], 99)), 3),
                         "one_at_a_time_p50_ms": round(1e3 * float(np.percentile(seq_a[sel], 50)), 3),
                         "one_at_a_time_p99_ms": round(1e3 * float(np.percentile(seq_a[sel], 99)), 3)}
        return out

    # the same stream under the other request order and policies (small first, 1 s and 0.3 s wait limits)
    others = []
    for pol in extra_policies:
        srv = server()
        srv.set_order(pol[0])
        srv.set_policy(pol[1], pol[2])
        res_p, _ = run_stream(srv, reqs, arrivals)
        st_p = srv.stats()
        srv.close()
        lat_p = latency_summary(res_p)
        others.append({"order": order_names[pol[0]], "max_large_inflight": pol[1], "max_large_wait_s": pol[2],
                       "p50_ms": round(lat_p["p50_ms"], 3),
                       "p99_ms": round(lat_p["p99_ms"], 3), "p99_by_class": classes(res_p),
                       "max_batch_requests": st_p["max_batch_requests"]})
    if detail is not None:  # per request: (template, service alone, server result, one-at-a-time latency)
        detail.extend(zip(pick.tolist(), svc.tolist(), results, lat_seq))
    total_evals = sum(r[0].n_vis * r[1].n_comp for r in reqs)
    lat = latency_summary(results)
    # p99 by request class (service time alone below / at or above 20 ms), each against the measured
    # one-at-a-time run of the same stream
    by_class = classes(results)
    # burst: n_burst requests of the sets under 5 ms alone, at once
    small = [k for k in range(n_templates) if svc_t[k] < 0.005]
    if not small:  # a stream without such sets: its fastest third
        small = sorted(range(n_templates), key=lambda k: svc_t[k])[:max(1, n_templates // 3)]
    bpick = np.random.default_rng(seed + 2).choice(small, size=n_burst)
    breqs = [temps[k] for k in bpick]
    bzero = np.zeros(n_burst)
    srv = server()
    bres, bwall = run_stream(srv, breqs, bzero)
    bst = srv.stats()
    srv.close()
    _, _, bwall_seq = run_sequential(ctx, breqs, bzero)
    bevals = sum(r[0].n_vis * r[1].n_comp for r in breqs)
    blat = latency_summary(bres)
    for m in models:
        m.free()
    return {"workload": f"serving: {n_req} Poisson requests drawn from {n_templates} uneven request sets "
                        "(16-128 tiles, 1-14 steps, 32-384 ch, 100-50000 P/G + 0-3 shapelets n_max 10-80)",
            "policy": {"order": order_names[0 if order is None else order],
                       "max_large_inflight": (policy or (1, 1.0))[0], "max_large_wait_s": (policy or (1, 1.0))[1]},
            "rate_hz": round(rate, 2), "mean_service_ms": round(1e3 * mean_s, 3),
            "p50_ms": round(lat["p50_ms"], 3), "p99_ms": round(lat["p99_ms"], 3),
            "one_at_a_time_p50_ms": round(1e3 * float(np.percentile(lat_seq, 50)), 3),
            "one_at_a_time_p99_ms": round(1e3 * float(np.percentile(lat_seq, 99)), 3),
            "one_at_a_time": "measured: the same stream run one request at a time through predict / peel",
            "p99_by_class": by_class,
            "other_policies": others,
            "service_alone_p50_ms": round(1e3 * float(np.percentile(svc_seq, 50)), 3),
            "service_alone_p99_ms": round(1e3 * float(np.percentile(svc_seq, 99)), 3),
            "throughput_evals_per_s": total_evals / wall, "wall_s": round(wall, 3),
            "one_at_a_time_throughput_evals_per_s": total_evals / wall_seq,
            "batches": st["batches"], "max_batches_in_flight": st["max_batches_in_flight"],
            "max_batch_requests": st["max_batch_requests"],
            "burst": {"requests": n_burst, "sets": "the request sets under 5 ms alone, all submitted at once",
                      "wall_s": round(bwall, 4), "one_at_a_time_wall_s": round(bwall_seq, 4),
                      "throughput_evals_per_s": bevals / bwall, "one_at_a_time_throughput_evals_per_s": bevals / bwall_seq,
                      "throughput_gain": round(bwall_seq / bwall, 3), "p50_ms": round(blat["p50_ms"], 3),
                      "p99_ms": round(blat["p99_ms"], 3), "batches": bst["batches"],
                      "max_batch_requests": bst["max_batch_requests"],
                      "max_batches_in_flight": bst["max_batches_in_flight"]}}


def run_case(case: str):
    """Small fixed cases for ncu captures (three warm-up calls, then one timed call)."""
    import torch
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    if case == "serve":          # K6: a reduced serving stream (200 requests drawn from 12 request sets)
        r = bench_serving(wn, ctx, 0, torch, n_req=200, n_templates=12)
        print(json.dumps({"case": case, "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "batches": r["batches"],
                          "wall_s": r["wall_s"], "device_errors": ctx.device_errors()}))
        return
    if case == "mwa_small":      # K1: 2 steps of the MWA array, 2,000 points + 500 Gaussians
        obs, _ = synth.mwa(n_time=2)
        sky = synth.make_sky(102, 2000, 500, 0)
    elif case == "fornax_small":  # K2: 2 steps of the Fornax array, 2 shapelets at n_max 80
        obs, sky = synth.fornax(n_time=2)
    elif case == "fornax":        # K2: the full Fornax peel (14 steps), for the one-pass traffic record
        obs, sky = synth.fornax()
    elif case == "adjoint":       # K4: the full adjoint workload
        obs, sky = synth.adjoint()
    elif case == "calib":         # K7: gain calibration, 128 tiles x 2 steps x 384 ch, 10 iterations
        obs, _ = synth.mwa(n_time=2)
        sky = synth.make_sky(102, 2000, 500, 0)
    else:                         # K3: standalone peel of the full MWA observation
        obs, sky = synth.mwa()
    d = wn.obs_to_device(obs)
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    gains = torch.as_tensor(synth.make_gains(5, obs.n_ant).astype(np.complex64)).cuda()
    data = torch.randn(shape, dtype=torch.complex64, device="cuda")
    if case == "peel":
        model = torch.randn(shape, dtype=torch.complex64, device="cuda")
        fn = lambda: ctx.peel_model(d, gains, data, model, out=out)  # noqa: E731
        work = 24 * obs.n_vis
    elif case == "calib":
        m = ctx.upload(sky)
        model = ctx.predict(d, m)
        data = model * 1.01
        g0 = torch.ones((obs.n_time, obs.n_chan, obs.n_ant), dtype=torch.complex64, device="cuda")
        fn = lambda: ctx.calibrate(d, model, data, g0.clone(), n_iter=10)  # noqa: E731
        work = obs.n_time * obs.n_chan * 10   # solves
    else:
        m = ctx.upload(sky)
        if case == "adjoint":
            fn = lambda: ctx.predict_grad(d, m, gains, data, resid=out)  # noqa: E731
        elif case == "fornax":    # the peel the bench's shapelet report times
            fn = lambda: ctx.peel(d, m, gains, data, out=out)  # noqa: E731
        else:
            fn = lambda: ctx.predict(d, m, out=out)  # noqa: E731
        work = obs.n_vis * sky.n_comp
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"case": case, "ms": ms, "work": work, "rate": work / (ms * 1e-3),
                      "device_errors": ctx.device_errors()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the shapelet, adjoint, calibration, truncation, fit and serving reports")
    ap.add_argument("--case", choices=["mwa_small", "fornax_small", "fornax", "adjoint", "peel", "calib", "serve"],
                    help="run one small fixed case for profiling instead of the benchmark")
    args = ap.parse_args()
    if args.case:
        return run_case(args.case)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2005_09316_b300 as wn

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    ctx = wn.Context(local)
    obs, sky = synth.mwa(seed=2 + rank)   # each rank: its own observation of the same shape
    d = wn.obs_to_device(obs, f"cuda:{local}")
    model = ctx.upload(sky)
    gains_np = synth.make_gains(5 + rank, obs.n_ant).astype(np.complex64)
    gains = torch.as_tensor(gains_np).cuda()
    shape = (obs.n_time, obs.n_base, obs.n_chan)
    gen = torch.Generator(device=f"cuda:{local}").manual_seed(11 + rank)
    data = torch.randn(shape, dtype=torch.complex64, device=f"cuda:{local}", generator=gen)
    resid = torch.empty_like(data)
    evals = obs.n_vis * sky.n_comp
    stream = torch.cuda.current_stream()

    def step():
        ctx.peel(d, model, gains, data, out=resid, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms = ev[0].elapsed_time(ev[-1]) / args.steps
    launches_per_step, launch_names = count_launches(step, torch)
    clocks = clk.summary()
    flags = ctx.device_errors()
    if flags:
        raise RuntimeError(f"device error flags {flags:#x}")
    if dist is not None:
        t = torch.tensor([ms], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = ws * evals / (ms * 1e-3)

    # ---------------- extras measured on rank 0 only ----------------
    extra = {}
    if rank == 0:
        P = peaks()
        sm_max = float(P.get("sm_max_mhz", 2032.0))
        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        peak_ops = n_sm * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12   # Top/s at the maximum SM clock
        achieved = OPS_PER_EVAL * evals / (ms * 1e-3) / 1e12
        extra["roofline"] = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_ops, 3),
                             "unit": "Top/s (FP32-pipe lane ops)", "frac": round(achieved / peak_ops, 4),
                             "traffic": k1_traffic(),
                             "traffic_unit": "bytes per launch (ncu dram__bytes_read + write, full size)",
                             "algorithmic_bytes": 16 * obs.n_vis + 24 * obs.n_rows,
                             "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (derived, not measured)",
                             "ops_per_eval": OPS_PER_EVAL}
        try:  # measured pipe rates (microbenchmarks in the library), for context beside the derived peak
            pr = ctx.pipe_rates()
            extra["roofline"]["measured_pipes_Tops"] = {k: round(v / 1e12, 3) for k, v in pr.items()}
            extra["roofline"]["frac_of_measured_ffma"] = round(achieved / (pr["ffma"] / 1e12), 4)
        except Exception as exc:  # noqa: BLE001 - reported, not fatal
            extra["roofline"]["measured_pipes_Tops"] = f"unavailable: {exc}"
        try:  # the kernel's own channel loop run alone: the bound its instruction mix sets
            lr = ctx.phasor_loop_rate()
            extra["roofline"]["loop_bound"] = {"value": lr, "unit": UNIT, "frac": round(value / ws / lr, 4),
                                               "what": "the kernel's channel loop alone (shared-memory components, "
                                                       "4 point tiles per Gaussian tile, no records/I/O/barriers)"}
        except Exception as exc:  # noqa: BLE001 - reported, not fatal
            extra["roofline"]["loop_bound"] = f"unavailable: {exc}"
        if clocks.get("sm_mhz"):
            extra["roofline"]["frac_at_sampled_clock"] = round(
                achieved / (n_sm * FP32_LANES_PER_SM * clocks["sm_mhz"] * 1e6 / 1e12), 4)

        # parity on sampled rows against the oracle (same launch configuration)
        import oracle
        rows = np.sort(np.random.default_rng(3).choice(obs.n_rows, size=16, replace=False))
        V = oracle.predict(synth.sub_obs(obs, rows), obs.freq, obs.dec0, sky)
        rt, rb = rows // obs.n_base, rows % obs.n_base
        dat = data.reshape(obs.n_rows, obs.n_chan)[torch.as_tensor(rows).cuda()].cpu().numpy()
        ref = oracle.peel(rt, rb, obs.ant1, obs.ant2, obs.n_ant, gains_np, dat, V)
        got = resid.reshape(obs.n_rows, obs.n_chan)[torch.as_tensor(rows).cuda()].cpu().numpy()
        err = np.abs(got - ref)
        extra["error"] = {"e_norm": float(err.max() / np.abs(V).max()),
                          "e_elem_model": float(np.max(err / np.maximum(np.abs(V), 1e-3 * np.abs(V).max()))),
                          "tolerance": 1e-5, "sample": "16 rows x 384 ch, residual vs oracle peel"}

        # the all-FP64 GPU form (speedup denominator): the per-component constants formed once per
        # component, as the mixed path forms them, on whole rows filling one wave of resident CTAs
        # (3 rows x 384 ch per SM: 9 CTAs of 128 threads per SM); the form that evaluates the printed
        # formulas per visibility (pow, the PA's cos and sin) beside it on a smaller sample
        import oracle

        def fp64_rate(prec, sub_rows, reps):
            sub = synth.Obs(obs.n_ant, 1, obs.n_chan, obs.uvw[:1, :sub_rows].copy(), obs.freq, obs.ant1[:sub_rows],
                            obs.ant2[:sub_rows], obs.dec0)
            ds = wn.obs_to_device(sub, f"cuda:{local}")
            ctx.set_precision(prec)
            o2 = torch.empty(1, sub_rows, obs.n_chan, dtype=torch.complex64, device=f"cuda:{local}")
            ctx.predict(ds, model, out=o2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            e0.record()
            for _ in range(reps):
                ctx.predict(ds, model, out=o2)
            e1.record()
            torch.cuda.synchronize()
            ctx.set_precision(wn.WN_PREC_MIXED)
            ms64 = e0.elapsed_time(e1) / reps
            Vs = oracle.predict(sub.uvw.reshape(-1, 3)[:8], sub.freq, sub.dec0, sky)
            e64 = float(np.abs(o2[0, :8].cpu().numpy() - Vs).max() / np.abs(Vs).max())
            return sub.n_vis * sky.n_comp / (ms64 * 1e-3), ms64, e64, sub.n_vis

        n_sm = torch.cuda.get_device_properties(local).multi_processor_count
        r64, ms64, e64, nv64 = fp64_rate(wn.WN_PREC_FP64, 3 * n_sm, 2)
        ru, msu, eu, nvu = fp64_rate(wn.WN_PREC_FP64_UNTUNED, 256, 1)
        extra["fp64_gpu"] = {"value": r64, "unit": UNIT, "speedup_mixed_over_fp64": value / ws / r64,
                             "e_norm": e64, "ms": round(ms64, 2),
                             "sample": f"{3 * n_sm} rows x 384 ch x 25000 comps ({nv64} visibilities, one wave)",
                             "form": "per-component constants hoisted (log-flux, alpha, Gaussian form); one FP64 "
                                     "sincospi and one exp2 per evaluation"}
        extra["fp64_gpu_untuned"] = {"value": ru, "unit": UNIT, "speedup_mixed_over_untuned": value / ws / ru,
                                     "e_norm": eu, "ms": round(msu, 2), "sample": f"256 rows x 384 ch x 25000 comps",
                                     "form": "printed formulas per evaluation (pow, cos/sin of the PA)"}

        # standalone streaming peel (HBM-bound): 24 bytes per visibility
        o3 = torch.empty_like(data)
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        for _ in range(3):
            ctx.peel_model(d, gains, data, resid, out=o3)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            ctx.peel_model(d, gains, data, resid, out=o3)
        e1.record()
        torch.cuda.synchronize()
        t_peel = e0.elapsed_time(e1) / 20 * 1e-3
        gbs = 24 * obs.n_vis / t_peel / 1e9
        hbm = float(P.get("hbm_gbs", 6400.0))
        extra["standalone_peel"] = {"achieved_gbs": round(gbs, 1), "peak_gbs": hbm, "frac": round(gbs / hbm, 4),
                                    "bytes_per_vis": 24, "ms": round(t_peel * 1e3, 4)}

        # end to end through the public API with host buffers (pinned), copies inside the timed region.
        # Two pipelines (each its own context, stream and device buffers) take alternate steps, so one
        # step's host<->device copies overlap the other's compute; a context's workspaces are per context.
        data_h = data.cpu().pin_memory()
        uvw_h = torch.as_tensor(obs.uvw).pin_memory()
        ctx2 = wn.Context(local)
        model2 = ctx2.upload(sky)
        pipes = []
        for c, mdl in ((ctx, model), (ctx2, model2)):
            pipes.append({"ctx": c, "model": mdl, "st": torch.cuda.Stream(), "d": wn.obs_to_device(obs, f"cuda:{local}"),
                          "data": torch.empty_like(data), "res": torch.empty(shape, dtype=torch.complex64).pin_memory()})
        torch.cuda.synchronize()

        def e2e_step(i):
            p = pipes[i % 2]
            with torch.cuda.stream(p["st"]):
                p["d"].uvw.copy_(uvw_h, non_blocking=True)
                p["data"].copy_(data_h, non_blocking=True)
                p["ctx"].peel(p["d"], p["model"], gains, p["data"], out=p["data"], stream=p["st"])
                p["res"].copy_(p["data"], non_blocking=True)

        for i in range(2):
            e2e_step(i)
        torch.cuda.synchronize()
        n_e2e = max(4, min(6, args.steps))
        t0 = time.perf_counter()
        for i in range(n_e2e):
            e2e_step(i)
        torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / n_e2e
        model2.free()
        ctx2.close()
        extra["e2e"] = {"value": evals / t_e2e, "unit": UNIT,
                        "h2d_bytes_per_step": int(data_h.numel() * 8 + uvw_h.numel() * 8),
                        "d2h_bytes_per_step": int(pipes[0]["res"].numel() * 8), "ms_per_step": round(t_e2e * 1e3, 3),
                        "pipeline": "2 contexts x 2 streams: each step's copies overlap the other step's compute"}

        # the long reports and the CPU baseline run at N = 1 only: a scaling run holds every GPU meanwhile
        if not args.no_extras and ws == 1:
            for key, fn in (("shapelet", lambda: bench_shapelets(wn, ctx, local, P, torch)),
                            ("adjoint", lambda: bench_adjoint(wn, ctx, local, torch)),
                            ("calibration", lambda: bench_calibration(wn, ctx, local, torch)),
                            ("truncation", lambda: bench_truncation(wn, ctx, local, torch)),
                            ("fit", lambda: bench_fit(wn, ctx, local, torch)),
                            ("serving", lambda: bench_serving(wn, ctx, local, torch))):
                try:
                    extra[key] = fn()
                except Exception as exc:  # an extra report must not hide the headline number
                    extra[key] = {"error": f"{type(exc).__name__}: {exc}"}

        if not args.no_cpu_baseline and ws == 1:
            rate, smp = oracle_rate(obs, sky, args.cpu_seconds)
            extra["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                                     "sample": f"{smp['rows']} random rows x 384 ch x 25000 comps "
                                               f"({smp['evals']} evals in {smp['seconds']} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_vis": obs.n_vis, "n_comp": sky.n_comp, "evals_per_step": evals,
                       "l2": "inputs > L2 each step (350 MB data in, 350 MB residual out); the 1.6 MB "
                             "component table stays L2-resident by design", "parallelism": f"replicas x{ws}"},
            "clocks": clocks, "gpu_launches": (args.steps * launches_per_step if launches_per_step else None),
            "gpu_launches_per_step": launch_names,
            "step_ms": {"min": min(per), "max": max(per)},
        }
        # the long reports first, then the headline keys, then a compact summary last (the line's tail)
        long_keys = ("truncation", "fit", "serving", "calibration", "shapelet", "adjoint")
        out = {k: extra[k] for k in long_keys if k in extra}
        out.update(line)
        out.update({k: v for k, v in extra.items() if k not in long_keys})
        if extra:
            out["summary"] = summary_block({**line, **extra})
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
