"""Truncation on the GPU: predicting the truncated model equals predicting the full model with the
dropped components and basis functions set to zero (within FP32 summation order)."""
import copy

import numpy as np
import pytest

import synth
from helpers import e_norm
from paper_2005_09316_b300 import truncate as tr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("f_comp", [0.5, 0.9, 0.99])
def test_truncated_model_equals_zeroed_model(f_comp):
    import paper_2005_09316_b300 as wn
    ctx = wn.Context(0)
    obs = synth.make_obs(51, 32, 2, synth.uniform_channels(167e6, 80e3, 48), layout="mwa")
    sky = synth.make_sky(52, 300, 100, 2, fov=10 * synth.DEG, shape_nmax=np.array([12, 20]))
    t, info = tr.truncate(sky, f_comp)
    assert 0 < info["n_comp"] < info["n_tot"]
    # the same selection expressed as zeros in the full model
    w_pg, w_sh = tr.component_weights(sky)
    order, n = tr.n_keep(np.concatenate([w_pg, w_sh]), f_comp)
    keep = np.zeros(w_pg.size + w_sh.size, dtype=bool)
    keep[order[:n]] = True
    z = copy.deepcopy(sky)
    n_pg = sky.n_point + sky.n_gauss
    z.flux[:n_pg][~keep[:n_pg]] = 0.0
    z.s_coeff[~keep[n_pg:]] = 0.0
    d = wn.obs_to_device(obs)
    mt, mz = ctx.upload(t), ctx.upload(z)
    vt = ctx.predict(d, mt).cpu().numpy()
    vz = ctx.predict(d, mz).cpu().numpy()
    assert e_norm(vt, vz) <= 2e-5
    assert ctx.device_errors() == 0
    mt.free()
    mz.free()
    ctx.close()
