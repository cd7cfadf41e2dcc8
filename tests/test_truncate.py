"""Model truncation (Sec. 6.2): the selection rule on a hand-worked example, closed forms of the basis
l1 norms, and the kept set's properties on a random model (CPU)."""
import json
import math
import os

import numpy as np
import pytest

import synth
from paper_2005_09316_b300 import truncate as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "truncation_hand.json")


def test_hand_worked_selection():
    g = json.load(open(GOLDEN))
    w = np.array(g["weights"])
    for f, n, kept in g["cases"]:
        order, nk = tr.n_keep(w, f)
        assert nk == n, (f, nk)
        assert sorted(order[:nk].tolist()) == kept


def test_hermite_l1_closed_forms():
    l1 = tr.hermite_l1(4)
    # psi_0 is a unit-flux Gaussian; |phi_1| = sqrt(2) |t| e^{-t^2/2} integrates to 2 sqrt(2).  The trapezoid
    # rule meets the kinks of |phi_n| at its zeros, so the values are good to ~1e-8
    assert l1[0] == pytest.approx(1.0, abs=1e-9)
    assert l1[1] == pytest.approx(2.0 / math.sqrt(math.pi), abs=1e-7)
    # phi_2 = (2 t^2 - 1) e^{-t^2/2} / sqrt(2), zeros at +-z, z = 1/sqrt(2).  With
    # integral (1 - 2 t^2) e^{-t^2/2} dt = 2 t e^{-t^2/2} - integral e^{-t^2/2} dt,
    # the inner part is 4 z e^{-z^2/2} - sqrt(2 pi) erf(z / sqrt(2)), and the whole line gives sqrt(2 pi).
    z = 1.0 / math.sqrt(2.0)
    I_in = 4 * z * math.exp(-z * z / 2) - math.sqrt(2 * math.pi) * math.erf(z / math.sqrt(2))
    I_abs = math.sqrt(2 * math.pi) + 2 * I_in
    assert l1[2] == pytest.approx(I_abs / math.sqrt(2) / math.sqrt(2 * math.pi), abs=1e-7)


def test_kept_set_is_the_largest_within_the_flux_fraction():
    obs, sky = synth.tiny(5)
    sky = synth.make_sky(9, 40, 15, 3, fov=10 * synth.DEG, shape_nmax=np.array([6, 10, 14]))
    w_pg, w_sh = tr.component_weights(sky)
    w = np.concatenate([w_pg, w_sh])
    for f in (0.3, 0.7, 0.9, 0.99, 1.0):
        t, info = tr.truncate(sky, f)
        order, n = tr.n_keep(w, f)
        kept = np.sort(w[order[:n]])
        assert kept.sum() <= f * w.sum() * (1 + 1e-12)
        if n < w.size:
            assert kept.sum() + w[order[n]] > f * w.sum()
        assert info["n_comp"] == n
        assert t.n_point + t.n_gauss + int(t.s_off[-1]) == n
        assert info["flux_fraction_kept"] <= f + 1e-12
        # the table is consistent
        assert t.l.size == t.n_comp and t.g_maj.size == t.n_gauss and t.s_off.size == t.n_shape + 1
    t, _ = tr.truncate(sky, 1.0)
    assert t.n_point == sky.n_point and t.n_gauss == sky.n_gauss and int(t.s_off[-1]) == int(sky.s_off[-1])
