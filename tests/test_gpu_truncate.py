"""Truncation on the GPU (Sec. 6.2): the library's truncated model, predicted on the GPU, against the
oracle's prediction of the full model with the terms the oracle's own selection drops set to zero.

Tolerance: the two paths' bounds added, 1e-5 of max |V| of the points and Gaussians (FP32 phasor
path) plus 2e-4 of max |V| of the shapelets (bf16 hi+lo tensor path), each max taken over the oracle's
visibilities of that part alone."""
import numpy as np
import pytest

import oracle
import synth
from helpers import e_norm
from paper_2005_09316_b300 import truncate as tr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _parts(sky):
    """The oracle-side sky split into its point/Gaussian and shapelet parts (zero flux elsewhere)."""
    import copy
    n_pg = sky.n_point + sky.n_gauss
    pg, sh = copy.deepcopy(sky), copy.deepcopy(sky)
    pg.flux = np.array(sky.flux, float).copy()
    sh.flux = np.array(sky.flux, float).copy()
    pg.flux[n_pg:] = 0.0
    sh.flux[:n_pg] = 0.0
    return pg, sh


@pytest.mark.parametrize("f_comp", [0.5, 0.9, 0.99])
def test_truncated_model_matches_oracle(f_comp):
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    obs = synth.make_obs(51, 32, 2, synth.uniform_channels(167e6, 80e3, 48), layout="mwa")
    sky = synth.make_sky(52, 300, 100, 2, fov=10 * synth.DEG, shape_nmax=np.array([12, 20]))
    t, info = tr.truncate(sky, f_comp)
    assert 0 < info["n_comp"] < info["n_tot"]
    keep = oracle.truncation_keep(sky, f_comp)
    assert int(keep.sum()) == info["n_comp"]
    z = oracle.truncation_zeroed(sky, keep)
    uvw = obs.uvw.reshape(-1, 3)
    pg, sh = _parts(z)
    Vpg = oracle.predict(uvw, obs.freq, obs.dec0, pg)
    Vsh = oracle.predict(uvw, obs.freq, obs.dec0, sh)
    ref = Vpg + Vsh
    d = wn.obs_to_device(obs)
    mt = ctx.upload(t)
    got = ctx.predict(d, mt).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    tol = 1e-5 * np.abs(Vpg).max() + 2e-4 * np.abs(Vsh).max()
    assert np.abs(got - ref).max() <= tol, (np.abs(got - ref).max(), tol)
    # and the same as the full model with those terms zeroed, on the GPU (summation order only)
    mz = ctx.upload(z)
    vz = ctx.predict(d, mz).cpu().numpy().reshape(obs.n_rows, obs.n_chan)
    assert e_norm(got, vz) <= 2e-5
    assert ctx.device_errors() == 0
    mt.free()
    mz.free()
    ctx.close()
