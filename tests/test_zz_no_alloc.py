"""wn_predict_static, the allocation-free prediction, against wn_predict.

Callers that cannot allocate device memory at prediction time (a process whose memory is reserved by
another allocator, or a loop that cannot take cudaMalloc's implicit synchronisation) use
wn_predict_static: its shapelet launches take their per-row and per-channel tables from a fixed
4 MiB device array instead of the context's workspace.  This file sorts last so that a run stopping
at the first failure has already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synth
from helpers import e_norm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_predict_matches_predict_twice_in_a_row():
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    obs = synth.make_obs(31, 32, 3, synth.uniform_channels(167e6, 80e3, 96), layout="mwa", max_baseline=5000.0,
                         dec0=-37.2 * synth.DEG)
    sky = synth.make_sky(32, 40, 15, 2, fov=2 * synth.DEG, shape_nmax=np.array([20, 45]),
                         shape_beta=(3 * synth.ARCMIN, 12 * synth.ARCMIN))
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    ref = ctx.predict(d, m).cpu().numpy()
    for _ in range(2):
        got = ctx.predict_static(d, m).cpu().numpy()
        assert e_norm(got, ref) <= 2e-4
    # accumulate mode through the same entry point
    acc = ctx.predict_static(d, m, out=torch.as_tensor(ref).cuda(), accumulate=True).cpu().numpy()
    assert e_norm(acc, 2 * ref) <= 2e-4
    assert ctx.device_errors() == 0
    m.free()
    ctx.close()


def test_static_predict_rejects_observations_beyond_its_scratch():
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    obs = synth.make_obs(33, 128, 33, synth.uniform_channels(167e6, 80e3, 8), layout="mwa")  # 268,224 rows
    sky = synth.make_sky(34, 1, 0, 1, shape_nmax=np.array([4]))
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    with pytest.raises(wn.WnError) as e:
        ctx.predict_static(d, m)
    assert e.value.code == wn.WN_EINVAL and "static scratch" in str(e.value)
    m.free()
    ctx.close()


def test_static_predict_sums_shapelets_in_runs_that_fit_its_scratch():
    """105,664 rows: the fixed scratch holds two shapelets' row tables at a time, so three shapelets take
    two launches (the second adds to the first's output); the result matches wn_predict, which sums all
    three in one launch, and the oracle on sampled rows."""
    import oracle
    from helpers import sample_rows
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    obs = synth.make_obs(35, 128, 13, synth.uniform_channels(167e6, 80e3, 8), layout="mwa", max_baseline=3000.0)
    sky = synth.make_sky(36, 5, 2, 3, fov=2 * synth.DEG, shape_nmax=np.array([6, 14, 9]),
                         shape_beta=(3 * synth.ARCMIN, 12 * synth.ARCMIN))
    d = wn.obs_to_device(obs)
    m = ctx.upload(sky)
    ref = ctx.predict(d, m).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    got = ctx.predict_static(d, m).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    assert e_norm(got, ref) <= 1e-6
    rows = sample_rows(obs, 24, seed=3)
    V = oracle.predict(synth.sub_obs(obs, rows), obs.freq, obs.dec0, sky)
    assert e_norm(got[rows], V) <= 2e-4
    assert ctx.device_errors() == 0
    m.free()
    ctx.close()
