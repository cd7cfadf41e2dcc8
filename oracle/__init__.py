"""FP64 CPU oracle for direct measurement-equation prediction, peeling, its gradient, the gain
calibration loop and the model-truncation rule.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of bench.py, never by the library itself.

The arithmetic lives in ``wn_oracle.c`` (plain C, FP64, loops in the paper's order); this module
builds it with gcc, loads it with ctypes and marshals numpy arrays.  The calibration loop is numpy
(design matrix written out, numpy's solve for the normal equations).  The truncation rule of
Sec. 6.2 is plain Python over weights from a Gauss-Legendre quadrature of the Hermite functions.  It
also holds the oracle's own packers (triangular coefficient index, parity split of the (-i)^(n1+n2)
phase, the Hermite scales k_n the operand is divided by, bf16 hi/lo split, tf32 rounding), written from
the same definitions the CUDA packer follows, so the two can be compared bit for bit.

Parity pins (tests/test_oracle_pins.py) tie every function here to closed forms, library
routines, brute-force DFTs or finite differences; none is left unpinned.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

C_LIGHT = 299792458.0


def build(force: bool = False) -> str:
    """Compile wn_oracle.c into liboracle.so (gcc, -O2, OpenMP, strict IEEE arithmetic)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            d, i, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            _lib.or_n_minus_1.restype = d
            _lib.or_n_minus_1.argtypes = [d, d]
            _lib.or_spectrum.restype = d
            _lib.or_spectrum.argtypes = [d, d, d, d]
            _lib.or_gauss_env.restype = d
            _lib.or_gauss_env.argtypes = [d, d, d, d, d]
            _lib.or_hermite.restype = None
            _lib.or_hermite.argtypes = [i, d, P]
            _lib.or_shapelet_frame.restype = None
            _lib.or_shapelet_frame.argtypes = [d, d, d, P]
            _lib.or_shapelet_frame_grad.restype = None
            _lib.or_shapelet_frame_grad.argtypes = [d, d, d, P, P]
            _lib.or_max_threads.restype = i
            _lib.or_predict.restype = None
            _lib.or_predict.argtypes = [i, P, i, P, d, i, i, i] + [P] * 16 + [P, i]
            _lib.or_peel.restype = None
            _lib.or_peel.argtypes = [i, P, P, P, P, i, P, i, i, i, P, P, P]
            _lib.or_grad.restype = None
            _lib.or_grad.argtypes = [i, P, i, P, d, i, i, i] + [P] * 16 + [P, P, P, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def max_threads() -> int:
    return int(lib().or_max_threads())


def n_minus_1(l: float, m: float) -> float:
    return lib().or_n_minus_1(l, m)


def spectrum(s_ref, alpha, nu_ref, nu) -> float:
    return lib().or_spectrum(s_ref, alpha, nu_ref, nu)


def gauss_env(u, v, maj, mn, pa) -> float:
    return lib().or_gauss_env(u, v, maj, mn, pa)


def hermite(nmax: int, x: float) -> np.ndarray:
    out = np.zeros(nmax + 1)
    lib().or_hermite(nmax, float(x), _p(out))
    return out


def shapelet_frame(l: float, m: float, dec0: float) -> np.ndarray:
    out = np.zeros(9)
    lib().or_shapelet_frame(float(l), float(m), float(dec0), _p(out))
    return out.reshape(3, 3)


def shapelet_frame_grad(l: float, m: float, dec0: float):
    """(dF/dl, dF/dm) of shapelet_frame, 3 x 3 each, by the chain rule through the centre's declination
    and right ascension (the frame follows the shapelet's position)."""
    fl, fm = np.zeros(9), np.zeros(9)
    lib().or_shapelet_frame_grad(float(l), float(m), float(dec0), _p(fl), _p(fm))
    return fl.reshape(3, 3), fm.reshape(3, 3)


class _SkyArgs:
    """Keeps contiguous copies alive for the duration of a call."""

    def __init__(self, sky):
        self.keep = [_f64(sky.l), _f64(sky.m), _f64(sky.flux), _f64(sky.alpha), _f64(sky.nu_ref),
                     _f64(sky.g_maj), _f64(sky.g_min), _f64(sky.g_pa), _f64(sky.s_beta1), _f64(sky.s_beta2),
                     _f64(sky.s_pa), _i32(sky.s_nmax), _i32(sky.s_off), _i32(sky.s_n1), _i32(sky.s_n2),
                     _f64(sky.s_coeff)]
        # positional order of the C signature: l m s_ref alpha nu_ref g_maj g_min g_pa
        # s_b1 s_b2 s_pa s_nmax s_off s_n1 s_n2 s_c
        self.ptrs = [_p(a) for a in self.keep]


def predict(uvw_rows: np.ndarray, freq: np.ndarray, dec0: float, sky, n_threads: int = 0) -> np.ndarray:
    """Visibilities [R, F] complex128 for the rows of uvw_rows ([R, 3] metres)."""
    uvw_rows = _f64(uvw_rows).reshape(-1, 3)
    freq = _f64(freq)
    R, F = uvw_rows.shape[0], freq.shape[0]
    out = np.zeros((R, F, 2))
    sa = _SkyArgs(sky)
    lib().or_predict(R, _p(uvw_rows), F, _p(freq), float(dec0), int(sky.n_point), int(sky.n_gauss),
                     int(sky.n_shape), *sa.ptrs, _p(out), int(n_threads))
    return out[..., 0] + 1j * out[..., 1]


def peel(row_t, row_b, ant1, ant2, n_ant, gains, data, vis) -> np.ndarray:
    """R = D - g[ant1] conj(g[ant2]) V for rows (row_t, row_b); gains [Tg, Fg, A] complex."""
    row_t, row_b, ant1, ant2 = _i32(row_t), _i32(row_b), _i32(ant1), _i32(ant2)
    g = np.ascontiguousarray(gains, dtype=np.complex128)
    Tg, Fg = g.shape[0], g.shape[1]
    d = np.ascontiguousarray(data, dtype=np.complex128)
    v = np.ascontiguousarray(vis, dtype=np.complex128)
    R, F = d.shape
    out = np.zeros((R, F), dtype=np.complex128)
    lib().or_peel(R, _p(row_t), _p(row_b), _p(ant1), _p(ant2), int(n_ant), _p(g.view(np.float64)), Tg, Fg, F,
                  _p(d.view(np.float64)), _p(v.view(np.float64)), _p(out.view(np.float64)))
    return out


def gain_product(row_t, row_b, ant1, ant2, gains, n_chan) -> np.ndarray:
    """G[r, f] = g[ant1] conj(g[ant2]) by direct indexing (used to form W = conj(G) R)."""
    g = np.asarray(gains)
    Tg, Fg = g.shape[0], g.shape[1]
    t = np.zeros_like(row_t) if Tg == 1 else np.asarray(row_t)
    f = np.arange(n_chan) if Fg > 1 else np.zeros(n_chan, dtype=int)
    g1 = g[t[:, None], f[None, :], np.asarray(ant1)[row_b][:, None]]
    g2 = g[t[:, None], f[None, :], np.asarray(ant2)[row_b][:, None]]
    return g1 * np.conj(g2)


def grad(uvw_rows, freq, dec0, sky, W):
    """dL/dp for L = sum |D - G V|^2 given W = conj(G)(D - G V) ([R, F] complex)."""
    uvw_rows = _f64(uvw_rows).reshape(-1, 3)
    freq = _f64(freq)
    R, F = uvw_rows.shape[0], freq.shape[0]
    Wc = np.ascontiguousarray(W, dtype=np.complex128).reshape(R, F)
    g_comp = np.zeros((sky.n_comp, 4))
    g_gauss = np.zeros((sky.n_gauss, 3))
    g_shape = np.zeros((sky.n_shape, 3))
    g_coeff = np.zeros(int(sky.s_off[-1]) if sky.n_shape else 0)
    sa = _SkyArgs(sky)
    lib().or_grad(R, _p(uvw_rows), F, _p(freq), float(dec0), int(sky.n_point), int(sky.n_gauss),
                  int(sky.n_shape), *sa.ptrs, _p(Wc.view(np.float64)), _p(g_comp), _p(g_gauss),
                  _p(g_shape), _p(g_coeff))
    return dict(flux=g_comp[:, 0].copy(), alpha=g_comp[:, 1].copy(), l=g_comp[:, 2].copy(),
                m=g_comp[:, 3].copy(), g_maj=g_gauss[:, 0].copy(), g_min=g_gauss[:, 1].copy(),
                g_pa=g_gauss[:, 2].copy(), s_beta1=g_shape[:, 0].copy(), s_beta2=g_shape[:, 1].copy(),
                s_pa=g_shape[:, 2].copy(), s_coeff=g_coeff)


def loss(uvw_rows, freq, dec0, sky, row_t, row_b, ant1, ant2, n_ant, gains, data) -> float:
    """L = sum |D - G V|^2 over the given rows, V from the oracle."""
    V = predict(uvw_rows, freq, dec0, sky)
    R = peel(row_t, row_b, ant1, ant2, n_ant, gains, data, V)
    return float(np.sum(np.abs(R) ** 2))


# ------------------------------------------------------------------------------------------------
# The oracle's own packers.  The CUDA library packs on the device; these restate the same layout
# from its definition so the two can be compared bit for bit.
# ------------------------------------------------------------------------------------------------

def tri_index(n1, n2):
    """k(n1, n2) = s (s + 1) / 2 + n2 with s = n1 + n2: all pairs with n1 + n2 <= n_max, by s."""
    s = np.asarray(n1) + np.asarray(n2)
    return s * (s + 1) // 2 + np.asarray(n2)


def tri_unindex(k):
    k = np.asarray(k, dtype=np.int64)
    s = ((np.sqrt(8 * k + 1) - 1) // 2).astype(np.int64)
    s = np.where(s * (s + 1) // 2 > k, s - 1, s)
    s = np.where((s + 1) * (s + 2) // 2 <= k, s + 1, s)
    n2 = k - s * (s + 1) // 2
    return (s - n2).astype(np.int64), n2


def p_tot(nmax: int) -> int:
    """Number of basis functions with n1 + n2 <= n_max (Sec. 2)."""
    return (nmax + 2) * (nmax + 1) // 2


def parity_split(nmax, n1, n2, c):
    """C (-i)^(n1+n2) as two real matrices [n1][n2]: (C_re, C_im)."""
    re = np.zeros((nmax + 1, nmax + 1))
    im = np.zeros((nmax + 1, nmax + 1))
    for a, b, v in zip(np.asarray(n1), np.asarray(n2), np.asarray(c)):
        k = (a + b) % 4
        re[a, b] += v * (1.0, 0.0, -1.0, 0.0)[k]
        im[a, b] += v * (0.0, -1.0, 0.0, 1.0)[k]
    return re, im


def herm_k(n: int) -> float:
    """Scale k_n of the rescaled Hermite functions g_n = k_n phi_n that the device's contraction runs on:
    k_0 = k_1 = 1 and k_(n+1) = k_(n-1) sqrt((n+1)/n), which turns the normalised recurrence
    phi_(n+1) = sqrt(2/(n+1)) x phi_n - sqrt(n/(n+1)) phi_(n-1) into g_(n+1) = e_n x g_n - g_(n-1) with
    e_n = sqrt(2/(n+1)) k_(n+1) / k_n.  Formed in FP64 in this order (each step correctly rounded), as
    the device forms it."""
    km, k = 1.0, 1.0
    for m in range(1, n):
        kn = km * math.sqrt((m + 1) / m)
        km, k = k, kn
    return k


def operand_dense(nmax: int, n1, n2, c, k_pad: int, n_pad: int) -> np.ndarray:
    """The coefficient operand's values [n_pad][k_pad] in FP64: row 2*n2 holds Re(C (-i)^(n1+n2)) and row
    2*n2+1 the imaginary part, over n1 (the K index), each divided by k_n1 k_n2 (herm_k) so that the
    contraction with the rescaled functions g gives sum phi C phi; zero padding."""
    re, im = parity_split(nmax, n1, n2, c)
    k = np.array([herm_k(n) for n in range(nmax + 1)])
    kk = k[:, None] * k[None, :]
    re, im = re / kk, im / kk
    dense = np.zeros((n_pad, k_pad))
    for b in range(nmax + 1):
        dense[2 * b, :nmax + 1] = re[:, b]
        dense[2 * b + 1, :nmax + 1] = im[:, b]
    return dense


def f32_to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even float32 -> bfloat16 bit patterns (finite inputs)."""
    u = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


def bf16_hi_lo(x) -> tuple[np.ndarray, np.ndarray]:
    """hi = RN_bf16(float32(x)), lo = RN_bf16(float32(x) - hi): the split-precision operand pair."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    hi = f32_to_bf16_bits(x32)
    lo = f32_to_bf16_bits((x32 - bf16_bits_to_f32(hi)).astype(np.float32))
    return hi, lo


def f32_to_tf32_bits(x32) -> np.ndarray:
    """float32 values rounded to the nearest tf32 (10 explicit mantissa bits, ties away from zero), as
    float32 bit patterns: half the range of the 13 dropped bits is added to the magnitude, then they are
    cleared."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)


def pack_coeff_tf32(nmax: int, n1, n2, c, k_pad: int, n_pad: int) -> np.ndarray:
    """The dense B operand of pack_coeff_bf16 as tf32 bit patterns [n_pad][k_pad] (one element per entry,
    RN_tf32(float32(value))), for the tensor-core tf32 mode."""
    dense = operand_dense(nmax, n1, n2, c, k_pad, n_pad)
    return f32_to_tf32_bits(dense.astype(np.float32))


def tf32_bits_to_f32(b) -> np.ndarray:
    return np.asarray(b, dtype=np.uint32).view(np.float32)


def pack_coeff_tf32x3(nmax: int, n1, n2, c, k_pad: int, n_pad: int):
    """The split tf32 operand pair [n_pad][k_pad] as bit patterns: hi = RN_tf32(float32(value)) and
    lo = RN_tf32(float32(value) - hi), the difference taken in float32 (where it is exact)."""
    hi = pack_coeff_tf32(nmax, n1, n2, c, k_pad, n_pad)
    d32 = operand_dense(nmax, n1, n2, c, k_pad, n_pad).astype(np.float32)
    lo = f32_to_tf32_bits((d32 - tf32_bits_to_f32(hi)).astype(np.float32))
    return hi, lo


def pack_coeff_bf16(nmax: int, n1, n2, c, k_pad: int, n_pad: int):
    """Dense B operand of the shapelet contraction, as bf16 hi/lo bit patterns [n_pad][k_pad] of
    operand_dense: row 2*n2 holds Re(C (-i)^(n1+n2))[n1, n2] / (k_n1 k_n2) over n1 (the K index), row
    2*n2+1 the imaginary part."""
    return bf16_hi_lo(operand_dense(nmax, n1, n2, c, k_pad, n_pad))


# ------------------------------------------------------------------------------------------------
# Gain calibration (Sec. 5.1, eq:peeling-iter): per (time, channel), the linearised least squares for
# additive per-antenna gain errors e, iterated.  Model M_ij = g_i conj(g_j) I_ij; residual
# R_ij = V_ij - M_ij ~ e_i conj(g_j) I_ij + conj(e_j) g_i I_ij with the e e* term dropped.  Free
# parameters Re(e_i), Im(e_i); the conjugation shows up as sign flips on Im(e_j).  The overall phase
# of the gains is not determined by the data (g -> g e^{i phi} leaves M unchanged), so A^T A is
# singular as printed; the oracle fixes the gauge by holding Im(e_0) = 0 (antenna 0's column dropped),
# the same rule as the CUDA path.  numpy's solve is the library step for [A^T A]^{-1} A^T b.
# ------------------------------------------------------------------------------------------------

def calib_columns(n_ant: int):
    """Column of Re(e_i) and of Im(e_i) in the parameter vector x (Im(e_0) has none: -1)."""
    re = np.array([0] + [2 * i - 1 for i in range(1, n_ant)], dtype=np.int64)
    im = np.array([-1] + [2 * i for i in range(1, n_ant)], dtype=np.int64)
    return re, im


def calib_design(ant1, ant2, n_ant: int, I, V, g):
    """Design matrix A [2B, 2A-1] and residual vector b [2B] of one (time, channel) at gains g [A]:
    rows 2k, 2k+1 are Re and Im of R for baseline k = (i, j)."""
    ant1, ant2 = np.asarray(ant1), np.asarray(ant2)
    I, V, g = np.asarray(I, complex), np.asarray(V, complex), np.asarray(g, complex)
    B = ant1.size
    re, im = calib_columns(n_ant)
    gi, gj = g[ant1], g[ant2]
    R = V - gi * np.conj(gj) * I
    a = np.conj(gj) * I        # coefficient of e_i
    c = gi * I                 # coefficient of conj(e_j)
    A = np.zeros((2 * B, 2 * n_ant - 1))
    rows_re, rows_im = 2 * np.arange(B), 2 * np.arange(B) + 1
    # e_i a:  Re -> x_i Re a - y_i Im a ;  Im -> x_i Im a + y_i Re a
    A[rows_re, re[ant1]] += a.real
    A[rows_im, re[ant1]] += a.imag
    ok = im[ant1] >= 0
    A[rows_re[ok], im[ant1][ok]] += -a.imag[ok]
    A[rows_im[ok], im[ant1][ok]] += a.real[ok]
    # conj(e_j) c:  Re -> x_j Re c + y_j Im c ;  Im -> x_j Im c - y_j Re c
    A[rows_re, re[ant2]] += c.real
    A[rows_im, re[ant2]] += c.imag
    ok = im[ant2] >= 0
    A[rows_re[ok], im[ant2][ok]] += c.imag[ok]
    A[rows_im[ok], im[ant2][ok]] += -c.real[ok]
    b = np.empty(2 * B)
    b[0::2], b[1::2] = R.real, R.imag
    return A, b


def calib_step(ant1, ant2, n_ant: int, I, V, g):
    """One iteration: x = [A^T A]^{-1} A^T b, then g <- g + e.  Returns the new gains [A]."""
    A, b = calib_design(ant1, ant2, n_ant, I, V, g)
    x = np.linalg.solve(A.T @ A, A.T @ b)
    re, im = calib_columns(n_ant)
    e = x[re] + 1j * np.where(im >= 0, x[np.maximum(im, 0)], 0.0)
    return np.asarray(g, complex) + e


def calibrate(ant1, ant2, n_ant: int, I, V, g0, n_iter: int = 10):
    """Gains [T, F, A] fitted per (time, channel) by n_iter iterations from g0 [T, F, A];
    I (model) and V (data) are [T, B, F]."""
    I, V = np.asarray(I, complex), np.asarray(V, complex)
    g = np.array(g0, dtype=complex, copy=True)
    T, _, F = I.shape
    for t in range(T):
        for f in range(F):
            for _ in range(n_iter):
                g[t, f] = calib_step(ant1, ant2, n_ant, I[t, :, f], V[t, :, f], g[t, f])
    return g


# ------------------------------------------------------------------------------------------------
# Visibility-space least-squares fit of shapelet coefficients (the counterpart of the image-space fit
# of Sec. 2.2): V is linear in the coefficients, so column k of the design matrix is the (gain-applied)
# visibility of coefficient k alone at unit value; the model's points and Gaussians are a fixed part.
# numpy's lstsq is the library step for the real least-squares problem on stacked Re / Im parts.
# ------------------------------------------------------------------------------------------------

def _shapelet_only(sky, coeff):
    import copy
    s = copy.deepcopy(sky)
    n_pg = sky.n_point + sky.n_gauss
    s.flux = np.array(sky.flux, dtype=np.float64).copy()
    s.flux[:n_pg] = 0.0
    s.s_coeff = np.asarray(coeff, dtype=np.float64).copy()
    return s


def fit_design(uvw_rows, freq, dec0, sky, G):
    """Complex design matrix [R*F, nnz]: column k = G * V(shapelets with only coefficient k = 1)."""
    nnz = int(sky.s_off[-1])
    cols = []
    for k in range(nnz):
        e = np.zeros(nnz)
        e[k] = 1.0
        cols.append((G * predict(uvw_rows, freq, dec0, _shapelet_only(sky, e))).ravel())
    return np.stack(cols, axis=1)


def fit_shapelet_coeffs(uvw_rows, freq, dec0, sky, G, data):
    """Least-squares coefficients of |D - G (V_fixed + A C)|^2 over the given rows (G and D [R, F])."""
    import copy
    pg = copy.deepcopy(sky)
    pg.s_coeff = np.zeros(int(sky.s_off[-1]))          # the fixed part: points and Gaussians only
    b = (np.asarray(data) - G * predict(uvw_rows, freq, dec0, pg)).ravel()
    A = fit_design(uvw_rows, freq, dec0, sky, G)
    Ar = np.concatenate([A.real, A.imag], axis=0)
    br = np.concatenate([b.real, b.imag])
    return np.linalg.lstsq(Ar, br, rcond=None)[0]


# ------------------------------------------------------------------------------------------------
# Model truncation (Sec. 6.2, "Model truncation").  Each point/Gaussian component, and each shapelet
# basis function, carries an absolute flux |I_j|; after sorting them so that |I_j| > |I_{j+1}|, the
# truncated model keeps the first N_comp, N_comp being the largest count whose summed |I_j| does not
# exceed f_comp times the sum over the whole model.  With no restoring beam and no image here (the
# paper sums the beam-convolved basis image over the fitted pixels), the weight of basis function
# (n1, n2) of a shapelet of flux S is |S C_n1n2| times the l1 norms of its two image-space 1-D factors,
# each normalised so that the (0, 0) function has unit flux: (1 / sqrt(2 pi)) * integral |phi_n(t)| dt,
# with phi_n(t) = H_n(t) exp(-t^2 / 2) / sqrt(2^n n!) the peak-normalised Hermite function of the uv
# envelope (its image-space partner psi_n(x) = phi_n(x / b) / (sqrt(2 pi) b) transforms to
# (-i)^n phi_n(2 pi u b), so the norm does not depend on b).
#
# The integral is computed here independently of the library's recurrence: phi_n keeps one sign between
# consecutive zeros of H_n, so integral |phi_n|^p is a sum of Gauss-Legendre quadratures over those
# intervals (the zeros from numpy's Gauss-Hermite nodes, H_n from scipy's eval_hermite), plus the tail
# beyond the last zero in unit steps out to 40 past it.
# ------------------------------------------------------------------------------------------------

def hermite_abs_moment(n: int, p: float, order: int = 48) -> float:
    """integral over the real line of |phi_n(t)|^p dt (phi_n peak-normalised; even in t)."""
    import math

    import scipy.special as sp
    from numpy.polynomial.hermite import hermgauss
    from numpy.polynomial.legendre import leggauss
    x, w = leggauss(order)
    zeros = np.sort(hermgauss(n)[0]) if n > 0 else np.zeros(0)
    edges = [0.0] + [float(z) for z in zeros if z > 0.0]
    top = edges[-1] + 40.0
    edges += [float(v) for v in np.arange(edges[-1] + 1.0, top, 1.0)] + [top]
    lognorm = 0.5 * (n * math.log(2.0) + math.lgamma(n + 1.0))
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        t = 0.5 * (b - a) * x + 0.5 * (a + b)
        f = sp.eval_hermite(n, t) * np.exp(-0.5 * t * t - lognorm)
        total += 0.5 * (b - a) * float(np.sum(w * np.abs(f) ** p))
    return 2.0 * total          # |phi_n| is even


def basis_l1(nmax: int) -> np.ndarray:
    """Flux-normalised l1 norm of the 1-D image-space shapelet factor of order n = 0..nmax:
    (1 / sqrt(2 pi)) * integral |phi_n(t)| dt (1 for n = 0)."""
    return np.array([hermite_abs_moment(n, 1.0) for n in range(nmax + 1)]) / np.sqrt(2.0 * np.pi)


def truncation_weights(sky) -> np.ndarray:
    """|I_j| of every point/Gaussian component (|S_ref|), then of every shapelet basis function in
    coefficient-triple order (|S C_n1n2| l1(n1) l1(n2))."""
    n_pg = sky.n_point + sky.n_gauss
    w = [abs(float(sky.flux[j])) for j in range(n_pg)]
    if sky.n_shape:
        l1 = basis_l1(int(np.max(sky.s_nmax)))
        for q in range(sky.n_shape):
            S = float(sky.flux[n_pg + q])
            for k in range(int(sky.s_off[q]), int(sky.s_off[q + 1])):
                w.append(abs(S * float(sky.s_coeff[k])) * l1[int(sky.s_n1[k])] * l1[int(sky.s_n2[k])])
    return np.array(w, dtype=np.float64)


def truncation_keep(sky, f_comp: float) -> np.ndarray:
    """Boolean mask over truncation_weights(sky): True for the N_comp entries of largest |I_j| (ties
    keep the earlier entry), N_comp the largest count with cumulative |I| <= f_comp * total."""
    w = truncation_weights(sky)
    order = sorted(range(len(w)), key=lambda j: (-w[j], j))
    total = 0.0
    for j in order:             # summed in the same order as the running sum, so f_comp = 1 keeps all
        total += w[j]
    limit = f_comp * total
    keep = np.zeros(len(w), dtype=bool)
    running = 0.0
    for j in order:
        if running + w[j] > limit:
            break
        running += w[j]
        keep[j] = True
    return keep


def truncation_zeroed(sky, keep):
    """The full model with every dropped component's flux and every dropped basis function's
    coefficient set to zero: it predicts exactly what the truncated model predicts."""
    import copy
    z = copy.deepcopy(sky)
    n_pg = sky.n_point + sky.n_gauss
    z.flux = np.array(sky.flux, dtype=np.float64).copy()
    z.s_coeff = np.array(sky.s_coeff, dtype=np.float64).copy()
    z.flux[:n_pg][~keep[:n_pg]] = 0.0
    z.s_coeff[~keep[n_pg:]] = 0.0
    return z
