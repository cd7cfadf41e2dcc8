"""Pins for the FP64 oracle: each check ties it to something other than itself.

Closed forms (a point at the phase centre), geometry computed a second way (delays from XYZ
baselines and source unit vectors), library routines (numpy's Hermite series and Gauss-Hermite
quadrature, torch's bfloat16 rounding, mpmath), brute-force 2-D DFTs of rendered images,
hand-worked values, and finite differences.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite as npherm

import oracle
import synth

C = 299792458.0
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def one_sky(kind, l=0.0, m=0.0, flux=1.0, alpha=0.0, nu_ref=180e6, maj=0.0, mn=0.0, pa=0.0,
            b1=0.0, b2=0.0, nmax=0, coeffs=((0, 0, 1.0),)):
    n = 1
    z = np.zeros(0)
    sk = synth.Sky(n_point=int(kind == "p"), n_gauss=int(kind == "g"), n_shape=int(kind == "s"),
                   l=np.array([l]), m=np.array([m]), flux=np.array([flux]), alpha=np.array([alpha]),
                   nu_ref=np.array([nu_ref]),
                   g_maj=np.array([maj]) if kind == "g" else z, g_min=np.array([mn]) if kind == "g" else z,
                   g_pa=np.array([pa]) if kind == "g" else z,
                   s_beta1=np.array([b1]) if kind == "s" else z, s_beta2=np.array([b2]) if kind == "s" else z,
                   s_pa=np.array([pa]) if kind == "s" else z,
                   s_nmax=np.array([nmax], dtype=np.int32) if kind == "s" else np.zeros(0, np.int32),
                   s_off=np.array([0, len(coeffs)], dtype=np.int32) if kind == "s" else np.array([0], np.int32),
                   s_n1=np.array([c[0] for c in coeffs], dtype=np.int32) if kind == "s" else np.zeros(0, np.int32),
                   s_n2=np.array([c[1] for c in coeffs], dtype=np.int32) if kind == "s" else np.zeros(0, np.int32),
                   s_coeff=np.array([c[2] for c in coeffs]) if kind == "s" else z)
    assert sk.n_comp == n
    return sk


def concat_sky(*skies):
    """Concatenate single-type skies into one table (points, then Gaussians, then shapelets)."""
    order = sorted(skies, key=lambda s: (s.n_point == 0, s.n_gauss == 0))
    cat = lambda f: np.concatenate([getattr(s, f) for s in order])
    offs = [0]
    for s in order:
        for k in range(s.n_shape):
            offs.append(offs[-1] + int(s.s_off[k + 1] - s.s_off[k]))
    return synth.Sky(sum(s.n_point for s in order), sum(s.n_gauss for s in order), sum(s.n_shape for s in order),
                     cat("l"), cat("m"), cat("flux"), cat("alpha"), cat("nu_ref"), cat("g_maj"), cat("g_min"),
                     cat("g_pa"), cat("s_beta1"), cat("s_beta2"), cat("s_pa"), cat("s_nmax").astype(np.int32),
                     np.array(offs, dtype=np.int32), cat("s_n1").astype(np.int32), cat("s_n2").astype(np.int32),
                     cat("s_coeff"))


# ------------------------------------------------------------------------------------------ points

def test_point_at_phase_centre_equals_spectrum_everywhere():
    obs, _ = synth.tiny()
    sky = one_sky("p", 0.0, 0.0, flux=3.5, alpha=-0.7, nu_ref=180e6)
    V = oracle.predict(obs.uvw.reshape(-1, 3), obs.freq, obs.dec0, sky)
    for f, nu in enumerate(obs.freq):
        s = oracle.spectrum(3.5, -0.7, 180e6, nu)
        assert np.all(V[:, f].imag == 0.0)
        assert np.all(V[:, f].real == s)


def test_spectrum_is_a_power_law_through_the_reference():
    assert oracle.spectrum(2.0, -0.8, 180e6, 180e6) == 2.0
    assert math.isclose(oracle.spectrum(2.0, -0.8, 180e6, 360e6), 2.0 * 2.0 ** -0.8, rel_tol=1e-15)
    nus = np.linspace(150e6, 210e6, 9)
    logs = np.log([oracle.spectrum(0.7, -1.3, 180e6, nu) for nu in nus])
    slope, icpt = np.polyfit(np.log(nus / 180e6), logs, 1)
    assert abs(slope + 1.3) < 1e-12 and abs(icpt - math.log(0.7)) < 1e-12


def test_n_minus_1_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for l, m in [(1e-9, -2e-9), (1e-4, 3e-5), (0.2, -0.3), (0.6, 0.5)]:
        exact = mp.sqrt(1 - mp.mpf(l) ** 2 - mp.mpf(m) ** 2) - 1
        got = oracle.n_minus_1(l, m)
        assert abs(got - float(exact)) <= 2e-16 * abs(float(exact))


def test_point_phase_is_the_geometric_delay():
    """u l + v m + w (n - 1) = b . (s - s0) with b the XYZ baseline, s, s0 unit vectors (no rotations)."""
    dec0 = -37.2 * synth.DEG
    obs = synth.make_obs(11, 6, 3, np.array([150e6, 200e6]), layout="mwa", max_baseline=5000.0, dec0=dec0,
                         ha0=-0.3, dt_s=600.0)
    xyz = synth.enu_to_xyz(obs.enu, obs.lat)
    b = xyz[obs.ant2] - xyz[obs.ant1]
    for dra, dd in [(0.05, 0.03), (-0.2, -0.1), (0.3, 0.25)]:
        dec = dec0 + dd
        l = math.cos(dec) * math.sin(dra)
        m = math.sin(dec) * math.cos(dec0) - math.cos(dec) * math.sin(dec0) * math.cos(dra)
        sky = one_sky("p", l, m, flux=1.0, alpha=0.0)
        V = oracle.predict(obs.uvw.reshape(-1, 3), obs.freq, obs.dec0, sky).reshape(obs.n_time, obs.n_base, -1)
        for t, h in enumerate(obs.ha):
            hs = h - dra                                   # H = LST - RA
            s = np.array([math.cos(dec) * math.cos(hs), -math.cos(dec) * math.sin(hs), math.sin(dec)])
            s0 = np.array([math.cos(dec0) * math.cos(h), -math.cos(dec0) * math.sin(h), math.sin(dec0)])
            tau = b @ (s - s0)
            for f, nu in enumerate(obs.freq):
                want = np.exp(-2j * math.pi * tau * nu / C)
                np.testing.assert_allclose(V[t, :, f], want, rtol=0, atol=2e-9)


def test_hermitian_symmetry_all_component_types():
    obs, sky = synth.tiny(5)
    uvw = obs.uvw.reshape(-1, 3)
    V = oracle.predict(uvw, obs.freq, obs.dec0, sky)
    Vn = oracle.predict(-uvw, obs.freq, obs.dec0, sky)
    np.testing.assert_allclose(Vn, np.conj(V), rtol=0, atol=1e-12 * np.abs(V).max())


# ---------------------------------------------------------------------------------------- Gaussian

def render_dft(img, l, m, uv):
    """Brute-force DFT with the e^{-2 pi i (u l + v m)} kernel of the measurement equation."""
    L, M = np.meshgrid(l, m, indexing="ij")
    out = []
    for u, v in uv:
        out.append(np.sum(img * np.exp(-2j * math.pi * (u * L + v * M))))
    return np.array(out)


def test_gaussian_envelope_is_one_at_origin():
    for maj, mn, pa in [(1e-3, 5e-4, 0.3), (3e-3, 3e-3, 2.0)]:
        assert oracle.gauss_env(0.0, 0.0, maj, mn, pa) == 1.0


@pytest.mark.parametrize("pa", [0.0, 0.6, 2.2])
def test_gaussian_matches_dft_of_rendered_image(pa):
    """eq:gauss-def rendered (x along PA, E of N), normalised to unit sum, then DFT'd by brute force."""
    maj, mn = 6.0 * synth.ARCMIN, 2.5 * synth.ARCMIN
    l0, m0 = 2.0e-3, -1.0e-3
    n = 257
    half = 4.0 * maj
    l = l0 + np.linspace(-half, half, n)
    m = m0 + np.linspace(-half, half, n)
    L, M = np.meshgrid(l - l0, m - m0, indexing="ij")
    x = L * math.sin(pa) + M * math.cos(pa)     # along the position angle (major axis)
    y = L * math.cos(pa) - M * math.sin(pa)
    img = np.exp(-4 * math.log(2) * (x ** 2 / maj ** 2 + y ** 2 / mn ** 2))
    img /= img.sum()
    rng = np.random.default_rng(0)
    uv = rng.uniform(-400, 400, size=(25, 2))
    dft = render_dft(img, l, m, uv)
    sky = one_sky("g", l0, m0, flux=1.0, alpha=0.0, maj=maj, mn=mn, pa=pa)
    uvw = np.column_stack([uv, np.zeros(len(uv))])          # w = 0: the flat-sky DFT
    V = oracle.predict(uvw, np.array([C]), 0.0, sky)[:, 0]  # nu = c: metres == wavelengths
    np.testing.assert_allclose(V, dft, rtol=0, atol=1e-9)


# ---------------------------------------------------------------------------------------- Hermite

def test_hermite_recurrence_matches_numpy_hermite_series():
    xs = [-7.5, -2.0, -0.3, 0.0, 0.7, 3.3, 9.0]
    for x in xs:
        phi = oracle.hermite(12, x)
        for n in range(13):
            c = np.zeros(n + 1)
            c[n] = 1.0
            want = npherm.hermval(x, c) * math.exp(-x * x / 2) / math.sqrt(2.0 ** n * math.factorial(n))
            assert abs(phi[n] - want) <= 1e-12 * max(1.0, abs(want))


def test_hermite_explicit_integer_coefficients():
    """H_3 = 8x^3 - 12x and H_4 = 16x^4 - 48x^2 + 12 written out."""
    for x in [0.4, -1.7, 2.9]:
        phi = oracle.hermite(4, x)
        g = math.exp(-x * x / 2)
        assert math.isclose(phi[3], (8 * x ** 3 - 12 * x) * g / math.sqrt(8 * 6), rel_tol=1e-13)
        assert math.isclose(phi[4], (16 * x ** 4 - 48 * x ** 2 + 12) * g / math.sqrt(16 * 24), rel_tol=1e-13)


def test_hermite_orthonormal_by_gauss_hermite_quadrature():
    """int phi_m phi_n dx = sqrt(pi) delta_mn for the peak-normalised functions, to n = 80."""
    nmax = 80
    xg, wg = npherm.hermgauss(120)
    P = np.array([oracle.hermite(nmax, x) for x in xg])        # [node, n]
    G = (P * (wg * np.exp(xg ** 2))[:, None]).T @ P
    np.testing.assert_allclose(G, math.sqrt(math.pi) * np.eye(nmax + 1), atol=1e-10)


def test_hermite_parity_and_large_argument():
    for x in [0.9, 5.0, 14.0]:
        a, b = oracle.hermite(40, x), oracle.hermite(40, -x)
        np.testing.assert_allclose(b, a * (-1.0) ** np.arange(41), rtol=1e-14, atol=1e-300)
    assert np.all(np.abs(oracle.hermite(127, 40.0)) < 1e-80)


# ---------------------------------------------------------------------------------------- shapelets

def image_basis(n, x, b):
    """Orthonormal image-space basis of eq:basis_1D with the normalisation [2^n sqrt(pi) n!]^-1/2."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return b ** -0.5 * (2.0 ** n * math.sqrt(math.pi) * math.factorial(n)) ** -0.5 * \
        npherm.hermval(x / b, c) * np.exp(-x ** 2 / (2 * b * b))


@pytest.mark.parametrize("n1,n2,pa", [(0, 0, 0.4), (1, 0, 0.0), (0, 1, 1.1), (2, 1, 2.5), (3, 2, 0.8), (1, 4, 1.9)])
def test_shapelet_matches_dft_of_rendered_basis(n1, n2, pa):
    """eq:basis_2D rendered with x along PA, DFT'd by brute force, equals
    2 sqrt(pi) sqrt(b1 b2) (-i)^(n1+n2) phi_n1(2 pi b1 kx) phi_n2(2 pi b2 ky), b = beta / (2 sqrt(2 ln 2)),
    i.e. the oracle's envelope for C[n1, n2] = 1 times 2 sqrt(pi b1 b2)."""
    beta1, beta2 = 5.0 * synth.ARCMIN, 3.0 * synth.ARCMIN
    b1, b2 = beta1 / (2 * math.sqrt(2 * math.log(2))), beta2 / (2 * math.sqrt(2 * math.log(2)))
    n = 256
    half = 12.0 * max(b1, b2)
    g = np.linspace(-half, half, n, endpoint=False)
    d = g[1] - g[0]
    L, M = np.meshgrid(g, g, indexing="ij")
    x = L * math.sin(pa) + M * math.cos(pa)
    y = L * math.cos(pa) - M * math.sin(pa)
    img = image_basis(n1, x, b1) * image_basis(n2, y, b2) * d * d
    rng = np.random.default_rng(n1 * 10 + n2)
    uv = rng.uniform(-900, 900, size=(20, 2))
    dft = render_dft(img, g, g, uv)
    sky = one_sky("s", 0.0, 0.0, flux=1.0, alpha=0.0, b1=beta1, b2=beta2, pa=pa, nmax=n1 + n2,
                  coeffs=((n1, n2, 1.0),))
    uvw = np.column_stack([uv, np.zeros(len(uv))])
    V = oracle.predict(uvw, np.array([C]), 0.0, sky)[:, 0]
    np.testing.assert_allclose(V * 2 * math.sqrt(math.pi * b1 * b2), dft, rtol=0, atol=1e-8)


def test_shapelet_00_equals_gaussian_at_centre():
    obs, _ = synth.tiny(7)
    maj, mn, pa = 7 * synth.ARCMIN, 3 * synth.ARCMIN, 0.9
    g = one_sky("g", 0.0, 0.0, flux=2.0, alpha=-0.5, maj=maj, mn=mn, pa=pa)
    s = one_sky("s", 0.0, 0.0, flux=2.0, alpha=-0.5, b1=maj, b2=mn, pa=pa, nmax=0)
    uvw = obs.uvw.reshape(-1, 3)
    Vg = oracle.predict(uvw, obs.freq, obs.dec0, g)
    Vs = oracle.predict(uvw, obs.freq, obs.dec0, s)
    np.testing.assert_allclose(Vs, Vg, rtol=1e-13, atol=1e-15)


def test_shapelet_00_off_centre_equals_gaussian_in_rotated_frame():
    """Off-centre, the shapelet envelope uses (u', v') of its own centre (Sec. 3.2)."""
    obs, _ = synth.tiny(8)
    l, m = 0.05, -0.08
    maj, mn, pa = 6 * synth.ARCMIN, 4 * synth.ARCMIN, 0.3
    s = one_sky("s", l, m, flux=1.0, alpha=0.0, b1=maj, b2=mn, pa=pa, nmax=0)
    uvw = obs.uvw.reshape(-1, 3)
    Vs = oracle.predict(uvw, obs.freq, obs.dec0, s)
    F = oracle.shapelet_frame(l, m, obs.dec0)
    for f, nu in enumerate(obs.freq):
        up = (uvw @ F.T) * nu / C
        u, v, w = (uvw * nu / C).T
        env = np.array([oracle.gauss_env(a, b, maj, mn, pa) for a, b in zip(up[:, 0], up[:, 1])])
        ph = np.exp(-2j * math.pi * (u * l + v * m + w * oracle.n_minus_1(l, m)))
        np.testing.assert_allclose(Vs[:, f], env * ph, rtol=1e-12, atol=1e-14)


def test_shapelet_frame_points_w_at_the_source_and_matches_textbook_uvw():
    dec0 = -30 * synth.DEG
    for dra, dd in [(0.0, 0.0), (0.1, -0.05), (-0.25, 0.2)]:
        dec = dec0 + dd
        l = math.cos(dec) * math.sin(dra)
        m = math.sin(dec) * math.cos(dec0) - math.cos(dec) * math.sin(dec0) * math.cos(dra)
        n = math.sqrt(1 - l * l - m * m)
        F = oracle.shapelet_frame(l, m, dec0)
        np.testing.assert_allclose(F @ F.T, np.eye(3), atol=1e-14)
        np.testing.assert_allclose(F @ np.array([l, m, n]), [0, 0, 1], atol=1e-14)
        if dra == 0.0 and dd == 0.0:
            np.testing.assert_allclose(F, np.eye(3), atol=1e-15)
        rng = np.random.default_rng(1)
        bxyz = rng.normal(size=(5, 3)) * 1000
        for h0 in [-0.4, 0.0, 0.7]:                      # frame is independent of the hour angle
            uvw0 = bxyz @ synth.xyz_to_uvw_matrix(h0, dec0).T
            uvwj = bxyz @ synth.xyz_to_uvw_matrix(h0 - dra, dec).T
            np.testing.assert_allclose(uvw0 @ F.T, uvwj, atol=1e-9)


# ---------------------------------------------------------------------------------------- packing

def test_p_tot_matches_paper_counts():
    g = json.load(open(os.path.join(GOLD, "paper_counts.json")))
    assert oracle.p_tot(g["p_max"]) * g["n_lobes"] == g["total_basis_functions"]
    assert g["ms_clean_points"] + g["ms_clean_gaussians"] == g["ms_clean_total"]
    n1, n2, _ = synth.shapelet_coeffs(np.random.default_rng(0), 86)
    assert n1.size == oracle.p_tot(86) and np.all(n1 + n2 <= 86)


def test_triangular_index_round_trip():
    for nmax in [0, 1, 10, 80, 127]:
        n1, n2, _ = synth.shapelet_coeffs(np.random.default_rng(0), nmax)
        k = oracle.tri_index(n1, n2)
        assert np.array_equal(np.sort(k), np.arange(oracle.p_tot(nmax)))
        a, b = oracle.tri_unindex(k)
        assert np.array_equal(a, n1) and np.array_equal(b, n2)


def test_parity_split_reassembles_the_phase():
    rng = np.random.default_rng(3)
    n1, n2, c = synth.shapelet_coeffs(rng, 9)
    re, im = oracle.parity_split(9, n1, n2, c)
    z = re + 1j * im
    for a, b, v in zip(n1, n2, c):
        assert z[a, b] == v * (-1j) ** int(a + b)
        assert (re[a, b] == 0.0) != ((a + b) % 2 == 0) or v == 0.0


def test_bf16_split_matches_torch_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(size=2000) * np.exp(rng.uniform(-30, 5, size=2000)), [0.0, 1.0, -0.5]])
    hi, lo = oracle.bf16_hi_lo(x)
    x32 = torch.tensor(x.astype(np.float32))
    thi = x32.to(torch.bfloat16)
    tlo = (x32 - thi.to(torch.float32)).to(torch.bfloat16)
    assert np.array_equal(hi, thi.view(torch.int16).numpy().view(np.uint16))
    assert np.array_equal(lo, tlo.view(torch.int16).numpy().view(np.uint16))
    rec = oracle.bf16_bits_to_f32(hi).astype(np.float64) + oracle.bf16_bits_to_f32(lo)
    assert np.all(np.abs(rec - x.astype(np.float32)) <= 2.0 ** -16 * np.abs(x.astype(np.float32)) + 1e-45)


# ---------------------------------------------------------------------------------------- peel

def test_peel_hand_worked_value():
    g = json.load(open(os.path.join(GOLD, "peel_hand.json")))
    gains = np.array([[[complex(*g["g_ant1"]), complex(*g["g_ant2"])]]])
    R = oracle.peel([0], [0], [0], [1], 2, gains, np.array([[complex(*g["data"])]]),
                    np.array([[complex(*g["model"])]]))
    assert R[0, 0] == complex(*g["resid"])


def test_peel_unit_gains_exact_model_is_zero_and_linear_in_data():
    obs, sky = synth.tiny(9)
    uvw = obs.uvw.reshape(-1, 3)
    V = oracle.predict(uvw, obs.freq, obs.dec0, sky)
    rows = np.arange(obs.n_rows)
    rt, rb = rows // obs.n_base, rows % obs.n_base
    ones = np.ones((1, 1, obs.n_ant), dtype=complex)
    assert np.all(oracle.peel(rt, rb, obs.ant1, obs.ant2, obs.n_ant, ones, V, V) == 0)
    g = synth.make_gains(3, obs.n_ant, 1, obs.n_chan)
    d1 = synth.complex_noise(1, V.shape, 1.0)
    d2 = synth.complex_noise(2, V.shape, 1.0)
    r1 = oracle.peel(rt, rb, obs.ant1, obs.ant2, obs.n_ant, g, d1, V)
    r2 = oracle.peel(rt, rb, obs.ant1, obs.ant2, obs.n_ant, g, d2, V)
    r12 = oracle.peel(rt, rb, obs.ant1, obs.ant2, obs.n_ant, g, d1 + d2, V)
    np.testing.assert_allclose(r12, r1 + r2 + oracle.gain_product(rt, rb, obs.ant1, obs.ant2, g, obs.n_chan) * V,
                               atol=1e-12)


# ---------------------------------------------------------------------------------------- gradient

def small_fit_problem(seed=21):
    obs = synth.make_obs(seed, 6, 2, synth.uniform_channels(167e6, 2e6, 3), layout="disc", diameter=800.0)
    p = synth.make_sky(seed + 1, 2, 2, 0, fov=5 * synth.DEG)
    s = one_sky("s", 0.01, -0.02, flux=1.7, alpha=-0.6, b1=8 * synth.ARCMIN, b2=5 * synth.ARCMIN, pa=0.7, nmax=5,
                coeffs=tuple((a, b, float(v)) for a, b, v in zip(*synth.shapelet_coeffs(np.random.default_rng(seed), 5))))
    sky = concat_sky(p, s)
    rows = np.arange(obs.n_rows)
    rt, rb = rows // obs.n_base, rows % obs.n_base
    gains = synth.make_gains(seed + 2, obs.n_ant, 1, 1, 0.1)
    data = synth.complex_noise(seed + 3, (obs.n_rows, obs.n_chan), 0.5)
    return obs, sky, rt, rb, gains, data


def _loss(obs, sky, rt, rb, gains, data):
    return oracle.loss(obs.uvw.reshape(-1, 3), obs.freq, obs.dec0, sky, rt, rb, obs.ant1, obs.ant2, obs.n_ant,
                       gains, data)


def test_gradient_matches_central_finite_differences():
    obs, sky, rt, rb, gains, data = small_fit_problem()
    uvw = obs.uvw.reshape(-1, 3)
    V = oracle.predict(uvw, obs.freq, obs.dec0, sky)
    G = oracle.gain_product(rt, rb, obs.ant1, obs.ant2, gains, obs.n_chan)
    W = np.conj(G) * (data - G * V)
    gr = oracle.grad(uvw, obs.freq, obs.dec0, sky, W)
    checks = [("flux", 1e-6), ("alpha", 1e-6), ("l", 1e-9), ("m", 1e-9), ("g_maj", 1e-9), ("g_min", 1e-9),
              ("g_pa", 1e-6), ("s_beta1", 1e-9), ("s_beta2", 1e-9), ("s_pa", 1e-6), ("s_coeff", 1e-6)]
    for name, h in checks:
        arr = getattr(sky, name)
        for i in range(arr.size):  # the shapelets' l and m too: their frame moves with them
            keep = arr[i]
            arr[i] = keep + h
            lp = _loss(obs, sky, rt, rb, gains, data)
            arr[i] = keep - h
            lm = _loss(obs, sky, rt, rb, gains, data)
            arr[i] = keep
            fd = (lp - lm) / (2 * h)
            an = gr[name][i]
            assert abs(an - fd) <= 2e-5 * max(1.0, abs(fd)), (name, i, an, fd)


def test_oracle_threads_do_not_change_results():
    obs, sky = synth.tiny(12)
    uvw = obs.uvw.reshape(-1, 3)
    a = oracle.predict(uvw, obs.freq, obs.dec0, sky, n_threads=1)
    b = oracle.predict(uvw, obs.freq, obs.dec0, sky, n_threads=4)
    assert np.array_equal(a, b)


def test_tf32_rounding_is_nearest_with_ties_away_from_zero():
    """oracle.f32_to_tf32_bits against its definition, without its formula: the result keeps 10 explicit
    mantissa bits (the 13 low bits clear); it is the tf32 value nearest the input, found here by
    comparing the two tf32 neighbours that bracket it; ties go away from zero."""
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        np.array([1.0, -1.0, 0.0, 3.0e-39, -2.5e-38])]).astype(np.float32)
    # exact ties: a tf32 value plus half its last-place unit
    base = (rng.standard_normal(200).astype(np.float32).view(np.uint32) & np.uint32(0xFFFFE000))
    ties = (base | np.uint32(0x1000)).view(np.float32)
    xs = np.concatenate([x, ties])
    got = oracle.f32_to_tf32_bits(xs)
    assert np.all(got & np.uint32(0x1FFF) == 0)
    b = xs.view(np.uint32)
    lo = (b & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)          # toward zero
    hi = ((b & np.uint32(0xFFFFE000)) + np.uint32(0x2000)).view(np.float32).astype(np.float64)  # away
    x64 = xs.astype(np.float64)
    d_lo, d_hi = np.abs(x64 - lo), np.abs(hi - x64)
    want = np.where(d_hi <= d_lo, hi, lo)   # nearest; at a tie (equal distance) the one away from zero
    assert np.array_equal(got.view(np.float32).astype(np.float64), want)


def test_tf32_split_operand_pair():
    """oracle.pack_coeff_tf32x3, from what the split must satisfy rather than its formula: hi is the one-
    product tf32 operand itself; both halves are tf32 values (13 low bits clear); and hi + lo reproduces the
    float32 coefficient to within the rounding of a 13-bit remainder to 11 bits (2^-21 of the value),
    i.e. about 21 significant bits, where hi alone keeps 11."""
    sky = synth.make_sky(21, 0, 0, 1, shape_nmax=30)
    n1, n2, c = sky.s_n1, sky.s_n2, sky.s_coeff * 1e3
    ne = int((n1 + n2).max())
    kp, npd = (ne + 1 + 15) // 16 * 16, (2 * (ne + 1) + 15) // 16 * 16
    hi, lo = oracle.pack_coeff_tf32x3(ne, n1, n2, c, kp, npd)
    assert np.array_equal(hi, oracle.pack_coeff_tf32(ne, n1, n2, c, kp, npd))
    assert np.all(hi & np.uint32(0x1FFF) == 0) and np.all(lo & np.uint32(0x1FFF) == 0)
    f = oracle.operand_dense(ne, n1, n2, c, kp, npd).astype(np.float32).astype(np.float64)
    both = hi.view(np.float32).astype(np.float64) + lo.view(np.float32).astype(np.float64)
    assert np.all(np.abs(both - f) <= 2.0 ** -21 * np.abs(f))
    only_hi = np.abs(hi.view(np.float32).astype(np.float64) - f)
    assert np.max(only_hi / np.maximum(np.abs(f), 1e-300)) > 2.0 ** -14    # hi alone is much coarser


def test_shapelet_frame_derivative_matches_finite_differences():
    """oracle.shapelet_frame_grad (chain rule through dec_j and RA_j) against central differences of
    oracle.shapelet_frame itself, off-centre and near the pole of the frame, at several declinations."""
    for l, m, dec0 in [(0.01, -0.02, -0.5), (0.2, 0.15, -1.1), (-0.3, 0.05, 0.3), (0.0, 0.0, -0.65), (0.05, 0.6, 0.1)]:
        fl, fm = oracle.shapelet_frame_grad(l, m, dec0)
        h = 1e-6
        dl = (oracle.shapelet_frame(l + h, m, dec0) - oracle.shapelet_frame(l - h, m, dec0)) / (2 * h)
        dm = (oracle.shapelet_frame(l, m + h, dec0) - oracle.shapelet_frame(l, m - h, dec0)) / (2 * h)
        assert np.max(np.abs(fl - dl)) <= 1e-8, (l, m, dec0, np.max(np.abs(fl - dl)))
        assert np.max(np.abs(fm - dm)) <= 1e-8, (l, m, dec0, np.max(np.abs(fm - dm)))


def test_rescaled_hermite_functions_and_operand():
    """The operand's scaling, pinned to what it must preserve.  (1) The rescaled functions g_n = k_n phi_n
    (oracle.herm_k) satisfy the two-operation recurrence g_(n+1) = e_n x g_n - g_(n-1) with
    e_n = sqrt(2/(n+1)) k_(n+1)/k_n, for n up to 127, against the oracle's plain basis; k_n stays within
    [1, 4].  (2) The contraction of the scaled operand with g(x) and g(y) equals the direct double sum
    of C (-i)^(n1+n2) phi_n1(x) phi_n2(y) (eq:shape-env)."""
    nmax = 127
    k = np.array([oracle.herm_k(n) for n in range(nmax + 2)])
    assert k[0] == 1.0 and k[1] == 1.0 and 1.0 <= k.min() and k.max() <= 4.0
    # k_(n+1) k_n ... the closed forms: k_2m = 2^m m! / sqrt((2m)!), k_(2m+1) = sqrt((2m+1)!) / (2^m m!)
    from math import factorial, sqrt
    for n in (2, 3, 10, 11, 40, 41):
        m = n // 2
        want = (2 ** m * factorial(m) / sqrt(factorial(2 * m)) if n % 2 == 0
                else sqrt(factorial(2 * m + 1)) / (2 ** m * factorial(m)))
        assert abs(k[n] - want) <= 1e-13 * want
    for x in (-7.3, -0.4, 0.0, 1.1, 5.0, 11.9):
        phi = oracle.hermite(nmax + 1, x)
        g = k * phi
        for n in range(1, nmax + 1):
            e = sqrt(2.0 / (n + 1)) * k[n + 1] / k[n]
            assert abs(g[n + 1] - (e * x * g[n] - g[n - 1])) <= 1e-11 * max(1.0, np.abs(g).max())
    sky = synth.make_sky(23, 0, 0, 1, shape_nmax=20)
    n1, n2, c = sky.s_n1, sky.s_n2, sky.s_coeff
    ne = int((n1 + n2).max())
    kp, npd = (ne + 1 + 15) // 16 * 16, (2 * (ne + 1) + 15) // 16 * 16
    D = oracle.operand_dense(ne, n1, n2, c, kp, npd)
    for x, y in ((0.3, -1.2), (2.5, 0.7), (-4.0, 3.3)):
        gx = k[:kp] * oracle.hermite(kp - 1, x)[:kp]
        gy = k[:ne + 1] * oracle.hermite(ne, y)[:ne + 1]
        T = D @ gx                                   # [n_pad]: Re, Im rows of each n2
        got = np.sum(T[0:2 * (ne + 1):2] * gy) + 1j * np.sum(T[1:2 * (ne + 1):2] * gy)
        px, py = oracle.hermite(ne, x), oracle.hermite(ne, y)
        want = sum(v * (-1j) ** (a + b) * px[a] * py[b] for a, b, v in zip(n1, n2, c))
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want))
