"""Pins of the oracle's model-truncation rule (Sec. 6.2) and of the basis-function weights it ranks,
and the library's host-side truncate() against it (CPU).

The weights' 1-D factor norms come from a Gauss-Legendre quadrature between the zeros of H_n; the
same quadrature must give the orthonormality integral of the Hermite functions (sqrt(pi) for the
peak-normalised phi_n) and the l1 norms that have closed forms."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from paper_2005_09316_b300 import truncate as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "truncation_hand.json")


def test_quadrature_gives_hermite_orthonormality():
    # integral phi_n(t)^2 dt = sqrt(pi) for phi_n = H_n e^{-t^2/2} / sqrt(2^n n!)
    for n in (0, 1, 2, 5, 17, 40, 80, 127):
        assert oracle.hermite_abs_moment(n, 2.0) == pytest.approx(math.sqrt(math.pi), rel=1e-12), n


def test_basis_l1_closed_forms():
    l1 = oracle.basis_l1(2)
    # n = 0: a unit-flux Gaussian; n = 1: sqrt(2) |t| e^{-t^2/2} integrates to 2 sqrt(2)
    assert l1[0] == pytest.approx(1.0, rel=1e-13)
    assert l1[1] == pytest.approx(2.0 / math.sqrt(math.pi), rel=1e-13)
    # n = 2: (2 t^2 - 1) e^{-t^2/2} / sqrt(2) changes sign at +-1/sqrt(2); integral (1 - 2t^2) e^{-t^2/2}
    # over |t| < z is 4 z e^{-z^2/2} - sqrt(2 pi) erf(z / sqrt(2)), and the whole line gives -sqrt(2 pi)
    z = 1.0 / math.sqrt(2.0)
    inner = 4 * z * math.exp(-z * z / 2) - math.sqrt(2 * math.pi) * math.erf(z / math.sqrt(2))
    assert l1[2] == pytest.approx((math.sqrt(2 * math.pi) + 2 * inner) / math.sqrt(2) / math.sqrt(2 * math.pi),
                                  rel=1e-13)


def _points(fluxes):
    n = len(fluxes)
    z = np.zeros(0)
    return synth.Sky(n, 0, 0, np.zeros(n), np.zeros(n), np.asarray(fluxes, float), np.zeros(n),
                     np.full(n, 180e6), z, z, z, z, z, z, np.zeros(0, np.int32), np.zeros(1, np.int32),
                     np.zeros(0, np.int32), np.zeros(0, np.int32), z)


def test_hand_worked_selection():
    """The golden's weights as point fluxes (signs flipped on two: the rule ranks |I_j|)."""
    g = json.load(open(GOLDEN))
    w = np.array(g["weights"])
    sky = _points(w * np.array([1, -1, 1, -1]))
    for f, n, kept in g["cases"]:
        keep = oracle.truncation_keep(sky, f)
        assert int(keep.sum()) == n, (f, keep)
        assert np.flatnonzero(keep).tolist() == kept


def test_shapelet_basis_weights():
    """One shapelet of flux -2 with C_00 = 0.5, C_10 = 0.25 and C_02 = -1: weights |S C| l1(n1) l1(n2)."""
    z1 = np.zeros(1)
    sky = synth.Sky(1, 0, 1, np.zeros(2), np.zeros(2), np.array([3.0, -2.0]), np.zeros(2), np.full(2, 180e6),
                    np.zeros(0), np.zeros(0), np.zeros(0), z1 + 1e-3, z1 + 1e-3, z1, np.array([2], np.int32),
                    np.array([0, 3], np.int32), np.array([0, 1, 0], np.int32), np.array([0, 0, 2], np.int32),
                    np.array([0.5, 0.25, -1.0]))
    l1 = oracle.basis_l1(2)
    w = oracle.truncation_weights(sky)
    np.testing.assert_allclose(w, [3.0, 1.0, 0.5 * l1[1], 2.0 * l1[2]], rtol=1e-15)
    # total 3 + 1 + 0.564 + 2.428 = 6.992; f = 0.8 keeps 3 and 2.428 (5.428 <= 5.594 < 6.428)
    assert oracle.truncation_keep(sky, 0.8).tolist() == [True, False, False, True]
    assert oracle.truncation_keep(sky, 1.0).all()
    assert not oracle.truncation_keep(sky, 0.0).any()


def test_package_l1_matches_oracle_quadrature():
    """The library's trapezoid over its own recurrence against the oracle's quadrature (relative 2e-6:
    the trapezoid meets the kinks of |phi_n| at its zeros)."""
    np.testing.assert_allclose(tr.hermite_l1(127), oracle.basis_l1(127), rtol=2e-6, atol=0)


def _kept_from_table(sky, t):
    """The keep mask that a truncated table implies, recovered by matching identities: components by
    their (l, m, flux), shapelet basis functions by (shapelet, n1, n2)."""
    n_pg = sky.n_point + sky.n_gauss
    keep = np.zeros(n_pg + (int(sky.s_off[-1]) if sky.n_shape else 0), dtype=bool)
    ids = {(float(a), float(b), float(c)): j for j, (a, b, c) in enumerate(zip(sky.l, sky.m, sky.flux))}
    for k in range(t.n_point + t.n_gauss):
        keep[ids[(float(t.l[k]), float(t.m[k]), float(t.flux[k]))]] = True
    for qt in range(t.n_shape):
        q = ids[(float(t.l[t.n_point + t.n_gauss + qt]), float(t.m[t.n_point + t.n_gauss + qt]),
                 float(t.flux[t.n_point + t.n_gauss + qt]))] - n_pg
        pos = {(int(a), int(b)): k for k, (a, b) in
               enumerate(zip(sky.s_n1[sky.s_off[q]:sky.s_off[q + 1]], sky.s_n2[sky.s_off[q]:sky.s_off[q + 1]]))}
        for k in range(int(t.s_off[qt]), int(t.s_off[qt + 1])):
            keep[n_pg + int(sky.s_off[q]) + pos[(int(t.s_n1[k]), int(t.s_n2[k]))]] = True
    return keep


@pytest.mark.parametrize("seed", [9, 10, 11])
def test_truncate_selects_the_oracle_set(seed):
    """truncate() keeps exactly the oracle's components and basis functions.  The cases are checked to be
    well posed first: no pair of weights, and no cumulative sum against the limit, closer than 2e-6
    relative (the library's l1 norms are within 7e-7 of the oracle's), so the two computations of the
    weights cannot disagree on the cut."""
    sky = synth.make_sky(seed, 60, 20, 3, fov=10 * synth.DEG, shape_nmax=np.array([6, 14, 30]))
    w = oracle.truncation_weights(sky)
    ws = np.sort(w)[::-1]
    for f in (0.3, 0.6, 0.9, 0.97, 0.995, 1.0):
        keep = oracle.truncation_keep(sky, f)
        n = int(keep.sum())
        cum = np.cumsum(ws)
        if 0 < n < w.size:
            assert (ws[n - 1] - ws[n]) > 2e-6 * ws[n - 1], "near-tie at the cut"
            assert abs(cum[n] - f * cum[-1]) > 2e-6 * cum[-1] and abs(cum[n - 1] - f * cum[-1]) > 2e-6 * cum[-1]
        t, info = tr.truncate(sky, f)
        assert info["n_comp"] == n
        got = _kept_from_table(sky, t)
        assert np.array_equal(got, keep), (f, np.flatnonzero(got != keep))
