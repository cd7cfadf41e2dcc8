"""Continuous-batching serving of predict / peel requests (binding of the wn_server_* C ABI) and a
driver that replays a seeded Poisson stream of uneven requests and reports latency and throughput.

The scheduler itself is native (csrc/wn_serve.cu): admission by memory into a device pool, batches of
all newly admitted requests run by a persistent kernel replayed from a CUDA graph, several batches in
flight on separate streams.  This module only marshals arguments and measures.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import numpy as np

from . import Context, DeviceObs, Model, _check, load

REQ_PENDING, REQ_ADMITTED, REQ_RUNNING, REQ_DONE, REQ_CANCELLED, REQ_FAILED = range(6)
SERVE_ARRIVAL, SERVE_SMALL_FIRST = 0, 1   # request orders (wn_server_set_order)


@dataclass
class Result:
    ticket: int
    state: int
    vis_ptr: int
    t_submit: float
    t_admit: float
    t_launch: float
    t_done: float
    batch: int

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class Server:
    def __init__(self, ctx: Context, n_streams: int = 3, pool_bytes: int = 2 << 30, max_inflight: int = 32,
                 max_rows: int = 14 * 8128, max_chan: int = 384):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(load().wn_server_create(ctx.h, n_streams, pool_bytes, max_inflight, max_rows, max_chan,
                                       ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def close(self):
        if self.h:
            load().wn_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, obs: DeviceObs, model: Model, gains=None, data=None) -> int:
        o = obs.struct()
        t = ctypes.c_uint64()
        peel = data is not None
        _check(load().wn_server_submit(self.h, ctypes.byref(o), model.id, int(peel),
                                       gains.data_ptr() if peel else None, int(gains.shape[0]) if peel else 1,
                                       int(gains.shape[1]) if peel else 1, data.data_ptr() if peel else None,
                                       ctypes.byref(t)))
        self._keep[t.value] = (obs, gains, data)   # device arrays stay alive until release
        return t.value

    def _result(self, ticket, state, ptr, info) -> Result:
        return Result(ticket, state, ptr.value or 0, info[0], info[1], info[2], info[3], int(info[4]))

    def poll(self, ticket: int) -> Result:
        st, ptr, info = ctypes.c_int(), ctypes.c_void_p(), (ctypes.c_double * 5)()
        _check(load().wn_server_poll(self.h, ticket, ctypes.byref(st), ctypes.byref(ptr), info))
        return self._result(ticket, st.value, ptr, info)

    def wait(self, ticket: int, timeout: float = 60.0) -> Result:
        ptr, info = ctypes.c_void_p(), (ctypes.c_double * 5)()
        _check(load().wn_server_wait(self.h, ticket, float(timeout), ctypes.byref(ptr), info))
        return self.poll(ticket)

    def result_tensor(self, ticket: int, obs: DeviceObs, stream=None):
        """Copy a finished request's visibilities out of the pool into a new torch tensor."""
        import torch

        from . import _stream_handle
        out = torch.empty((obs.n_time, obs.n_base, obs.n_chan), dtype=torch.complex64,
                          device=f"cuda:{self.ctx.device}")
        _check(load().wn_server_copy(self.h, ticket, out.data_ptr(), _stream_handle(stream)))
        return out

    def release(self, ticket: int):
        _check(load().wn_server_release(self.h, ticket))
        self._keep.pop(ticket, None)

    def cancel(self, ticket: int):
        _check(load().wn_server_cancel(self.h, ticket))

    def set_policy(self, max_large_inflight: int = 1, max_large_wait_s: float = 1.0):
        """Admission of large requests: how many own a slot at once, and (small-first order) after how
        many seconds of waiting one starts ahead of any younger one (least estimated work first
        otherwise; 0 gives submission order)."""
        _check(load().wn_server_set_policy(self.h, int(max_large_inflight), float(max_large_wait_s)))

    def set_order(self, order: int = SERVE_ARRIVAL):
        """Request order: SERVE_ARRIVAL (default; submission order, small requests batched, large ones in
        one launch on the highest-priority stream) or SERVE_SMALL_FIRST (small requests first, large
        ones in time-step chunks)."""
        _check(load().wn_server_set_order(self.h, int(order)))

    def stats(self) -> dict:
        v = (ctypes.c_double * 6)()
        _check(load().wn_server_stats(self.h, v))
        return dict(batches=int(v[0]), max_batches_in_flight=int(v[1]), max_batch_requests=int(v[2]),
                    launched=int(v[3]), admitted=int(v[4]), free_pool_bytes=int(v[5]))


def percentile(xs, q) -> float:
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


def poisson_arrivals(rng: np.random.Generator, rate_hz: float, n: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def latency_summary(results) -> dict:
    lat = [r.latency for r in results]
    return {"p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "mean_ms": 1e3 * float(np.mean(lat)) if lat else float("nan"), "n": len(lat)}


def run_stream(server: Server, requests, arrivals, release=True, timeout=120.0):
    """Submit `requests` ((obs, model, gains, data) tuples) at the given arrival times (seconds from now)
    while a consumer thread collects (and releases) every result as soon as it completes, in any order;
    returns (results in submission order, wall seconds)."""
    import threading

    t0 = time.perf_counter()
    lock = threading.Lock()
    outstanding = {}          # ticket -> submission index
    results = {}
    errors = []
    submitted_all = threading.Event()

    def consume():
        deadline = None
        while True:
            with lock:
                items = list(outstanding.items())
            if not items and submitted_all.is_set():
                return
            progressed = False
            for t, i in items:
                try:
                    r = server.poll(t)
                except Exception as exc:  # surfaced after the join
                    errors.append(exc)
                    r = None
                if r is None or r.state in (REQ_DONE, REQ_FAILED, REQ_CANCELLED):
                    if r is not None:
                        results[i] = r
                        if release:
                            server.release(t)
                    with lock:
                        outstanding.pop(t, None)
                    progressed = True
            if not progressed:
                if items and deadline is None:
                    deadline = time.perf_counter() + timeout
                if deadline is not None and time.perf_counter() > deadline:
                    errors.append(TimeoutError("requests still outstanding"))
                    return
                time.sleep(2e-4)
            else:
                deadline = None

    th = threading.Thread(target=consume, daemon=True)
    th.start()
    for i, ((obs, model, gains, data), ta) in enumerate(zip(requests, arrivals)):
        while time.perf_counter() - t0 < ta:
            time.sleep(min(2e-4, max(0.0, ta - (time.perf_counter() - t0))))
        t = server.submit(obs, model, gains, data)
        with lock:
            outstanding[t] = i
    submitted_all.set()
    th.join()
    if errors:
        raise errors[0]
    return [results[i] for i in range(len(requests))], time.perf_counter() - t0


def run_sequential(ctx: Context, requests, arrivals):
    """The one-at-a-time reference, measured: the same requests at the same arrival times, each run alone
    through the single-request calls (predict, or peel when the request carries data) and waited for
    before the next starts, in arrival order.  Returns (latencies in s, service times in s, wall s)."""
    import torch

    lat, svc = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (obs, model, gains, data), ta in zip(requests, arrivals):
        while time.perf_counter() - t0 < ta:
            time.sleep(min(2e-4, max(0.0, ta - (time.perf_counter() - t0))))
        ts = time.perf_counter()
        if data is None:
            ctx.predict(obs, model)
        else:
            ctx.peel(obs, model, gains, data)
        torch.cuda.synchronize()
        te = time.perf_counter()
        svc.append(te - ts)
        lat.append(te - t0 - ta)
    return lat, svc, time.perf_counter() - t0
