"""Model truncation (Sec. 6.2, "Model truncation"): drop the components, or shapelet basis functions,
that contribute the least absolute flux, keeping the N_comp largest whose summed |I_j| stays within a
fraction f_comp of the total.

- For a point or Gaussian component, I_j is its integrated flux density S_ref.
- For shapelet basis function (n1, n2) of a shapelet with flux S, the paper sums the absolute
  restoring-beam-convolved basis image over the fitted pixels. With no image and no restoring beam here,
  I_j is the absolute flux of the unconvolved image-space basis function: |S C_n1n2| times the l1 norms
  of its two 1-D factors.
  - Those factors are normalised so that the (0, 0) function has unit flux (the normalisation that makes
    B_00 the Gaussian of the same flux, Sec. 3.2).
  - Its 1-D factor psi_n(x) = phi_n(x / b) / (sqrt(2 pi) b) is the function whose Fourier transform is
    (-i)^n phi_n(2 pi u b), with phi_n the peak-normalised Hermite function of the uv envelope.
  - So the l1 norm of psi_n is (1 / sqrt(2 pi)) times the integral of |phi_n(t)| dt, independent of b.

Host-side preprocessing of a model before upload; the prediction itself is unchanged.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SKY_FIELDS = ("n_point", "n_gauss", "n_shape", "l", "m", "flux", "alpha", "nu_ref", "g_maj", "g_min", "g_pa",
              "s_beta1", "s_beta2", "s_pa", "s_nmax", "s_off", "s_n1", "s_n2", "s_coeff")


@dataclass
class SkyTable:
    """A host sky table with the wn_sky field names (points, then Gaussians, then shapelets)."""
    n_point: int
    n_gauss: int
    n_shape: int
    l: np.ndarray
    m: np.ndarray
    flux: np.ndarray
    alpha: np.ndarray
    nu_ref: np.ndarray
    g_maj: np.ndarray
    g_min: np.ndarray
    g_pa: np.ndarray
    s_beta1: np.ndarray
    s_beta2: np.ndarray
    s_pa: np.ndarray
    s_nmax: np.ndarray
    s_off: np.ndarray
    s_n1: np.ndarray
    s_n2: np.ndarray
    s_coeff: np.ndarray

    @property
    def n_comp(self) -> int:
        return self.n_point + self.n_gauss + self.n_shape


def hermite_l1(nmax: int, dt: float = 1e-3) -> np.ndarray:
    """(1 / sqrt(2 pi)) * integral |phi_n(t)| dt for n = 0..nmax (trapezoid rule on a grid that resolves
    the n_max oscillations and reaches far into the Gaussian tail), phi_n by the normalised recurrence
    phi_0 = e^{-t^2/2}, phi_{n+1} = sqrt(2/(n+1)) t phi_n - sqrt(n/(n+1)) phi_{n-1}."""
    half = np.sqrt(2.0 * nmax + 1.0) + 12.0
    t = np.arange(-half, half + dt / 2, dt)
    prev = np.zeros_like(t)
    cur = np.exp(-0.5 * t * t)
    out = np.empty(nmax + 1)
    for n in range(nmax + 1):
        a = np.abs(cur)
        out[n] = (a.sum() - 0.5 * (a[0] + a[-1])) * dt / np.sqrt(2.0 * np.pi)
        prev, cur = cur, np.sqrt(2.0 / (n + 1)) * t * cur - np.sqrt(n / (n + 1.0)) * prev
    return out


def component_weights(sky) -> tuple[np.ndarray, np.ndarray]:
    """|I_j| of every point/Gaussian component, then of every shapelet coefficient (triple order)."""
    n_pg = sky.n_point + sky.n_gauss
    w_pg = np.abs(np.asarray(sky.flux[:n_pg], dtype=np.float64))
    nnz = int(sky.s_off[-1]) if sky.n_shape else 0
    w_sh = np.zeros(nnz)
    if nnz:
        l1 = hermite_l1(int(np.max(sky.s_nmax)))
        for q in range(sky.n_shape):
            a, b = int(sky.s_off[q]), int(sky.s_off[q + 1])
            S = float(sky.flux[n_pg + q])
            w_sh[a:b] = np.abs(S * np.asarray(sky.s_coeff[a:b])) * l1[sky.s_n1[a:b]] * l1[sky.s_n2[a:b]]
    return w_pg, w_sh


def n_keep(weights: np.ndarray, f_comp: float) -> tuple[np.ndarray, int]:
    """Order of the weights, largest first (stable), and N_comp: the largest N with
    sum_{j<=N} |I_j| <= f_comp * sum_j |I_j| (a relative 1e-12 allows f_comp = 1 to keep everything)."""
    if not 0.0 <= f_comp <= 1.0:
        raise ValueError("f_comp must be in [0, 1]")
    order = np.argsort(-np.asarray(weights), kind="stable")
    if order.size == 0:
        return order, 0
    cum = np.cumsum(np.asarray(weights)[order])
    limit = f_comp * cum[-1] * (1.0 + 1e-12)
    return order, int(np.searchsorted(cum, limit, side="right"))


def truncate(sky, f_comp: float) -> tuple[SkyTable, dict]:
    """The truncated model: the N_comp components / basis functions of largest |I_j| over the whole model,
    in their original order.  A shapelet left with no coefficient is dropped; one that keeps some gets
    n_max = the largest retained n1 + n2 (its basis set shrinks, and with it the dense contraction).
    Returns (table, info)."""
    w_pg, w_sh = component_weights(sky)
    n_pg = w_pg.size
    order, n = n_keep(np.concatenate([w_pg, w_sh]), f_comp)
    keep = np.zeros(n_pg + w_sh.size, dtype=bool)
    keep[order[:n]] = True
    kpg, ksh = keep[:n_pg], keep[n_pg:]
    pts = np.flatnonzero(kpg[:sky.n_point])
    gss = np.flatnonzero(kpg[sky.n_point:n_pg])
    shp, off, n1, n2, cf = [], [0], [], [], []
    for q in range(sky.n_shape):
        a, b = int(sky.s_off[q]), int(sky.s_off[q + 1])
        sel = np.flatnonzero(ksh[a:b]) + a
        if sel.size == 0:
            continue
        shp.append(q)
        n1.append(np.asarray(sky.s_n1)[sel])
        n2.append(np.asarray(sky.s_n2)[sel])
        cf.append(np.asarray(sky.s_coeff)[sel])
        off.append(off[-1] + sel.size)
    comp = np.concatenate([pts, sky.n_point + gss, n_pg + np.asarray(shp, dtype=np.int64)]).astype(np.int64)
    gidx = gss
    sidx = np.asarray(shp, dtype=np.int64)
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    t = SkyTable(
        n_point=int(pts.size), n_gauss=int(gss.size), n_shape=len(shp),
        l=np.asarray(sky.l)[comp], m=np.asarray(sky.m)[comp], flux=np.asarray(sky.flux)[comp],
        alpha=np.asarray(sky.alpha)[comp], nu_ref=np.asarray(sky.nu_ref)[comp],
        g_maj=np.asarray(sky.g_maj)[gidx], g_min=np.asarray(sky.g_min)[gidx], g_pa=np.asarray(sky.g_pa)[gidx],
        s_beta1=np.asarray(sky.s_beta1)[sidx], s_beta2=np.asarray(sky.s_beta2)[sidx],
        s_pa=np.asarray(sky.s_pa)[sidx],
        s_nmax=np.asarray([int(np.max(a + b)) for a, b in zip(n1, n2)], dtype=np.int32),
        s_off=np.asarray(off, dtype=np.int32), s_n1=cat(n1, np.int32), s_n2=cat(n2, np.int32),
        s_coeff=cat(cf, np.float64))
    total = float(w_pg.sum() + w_sh.sum())
    kept = float(np.concatenate([w_pg, w_sh])[keep].sum())
    return t, {"n_comp": n, "n_tot": int(keep.size), "flux_fraction_kept": kept / total if total > 0 else 1.0}
