"""Shared helpers for the parity tests: error metrics and oracle sampling."""
import numpy as np

import oracle
import synth


def e_norm(got, ref) -> float:
    """max |V - V_ref| / max |V_ref| (normwise relative error)."""
    ref = np.asarray(ref)
    return float(np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def e_elem(got, ref, floor=1e-3) -> float:
    """max over |V_ref| >= floor * max|V_ref| of |V - V_ref| / |V_ref|."""
    ref = np.asarray(ref)
    a = np.abs(ref)
    mask = a >= floor * a.max()
    return float(np.max(np.abs(np.asarray(got) - ref)[mask] / a[mask]))


def oracle_rows(obs: synth.Obs, sky, rows, n_threads=0):
    """Oracle visibilities [len(rows), F] for flattened rows r = t * B + b."""
    return oracle.predict(synth.sub_obs(obs, rows), obs.freq, obs.dec0, sky, n_threads=n_threads)


def sample_rows(obs: synth.Obs, n: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n = min(n, obs.n_rows)
    rows = rng.choice(obs.n_rows, size=n, replace=False)
    rows[0] = 0
    if n > 1:
        rows[1] = obs.n_rows - 1  # the ragged tail
    return np.sort(rows)


def oracle_peel_rows(obs: synth.Obs, rows, gains, data_rows, vis_rows):
    rt, rb = rows // obs.n_base, rows % obs.n_base
    return oracle.peel(rt, rb, obs.ant1, obs.ant2, obs.n_ant, gains, data_rows, vis_rows)
