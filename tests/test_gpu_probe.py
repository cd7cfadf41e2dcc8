"""Pipe-rate microbenchmarks (wn_pipe_rates): positive, finite, and in the relations the roofline
discussion relies on (packed f32x2 FMA does the same lane work per second as scalar FMA; MUFU ex2 and
FP64 FMA are much slower pipes on this part)."""
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
