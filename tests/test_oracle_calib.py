"""Pins of the oracle's gain calibration loop (Sec. 5.1, eq:peeling-iter), on CPU.

- exact recovery: noiseless data made with known gains are fitted back, in the gauge Im(g_0) = 0;
- the design matrix is the Jacobian of the residual (finite differences, second-order error), which
  fixes every coefficient and the sign flips that stand for the conjugation;
- a model that already equals the data is a fixed point;
- with noise, the converged gains satisfy the normal equations (A^T b = 0): a stationary point of
  sum |R|^2."""
import numpy as np
import pytest

import oracle


def baselines(n_ant):
    a1, a2 = np.triu_indices(n_ant, 1)
    return a1.astype(np.int32), a2.astype(np.int32)


def problem(seed, n_ant=10, noise=0.0):
    rng = np.random.default_rng(seed)
    a1, a2 = baselines(n_ant)
    I = rng.normal(size=a1.size) + 1j * rng.normal(size=a1.size)
    g_true = 1 + 0.05 * (rng.normal(size=n_ant) + 1j * rng.normal(size=n_ant))
    V = g_true[a1] * np.conj(g_true[a2]) * I
    V = V + noise * (rng.normal(size=V.size) + 1j * rng.normal(size=V.size))
    return a1, a2, I, V, g_true


@pytest.mark.parametrize("seed,n_ant", [(1, 4), (2, 10), (3, 32)])
def test_exact_gains_are_recovered_in_the_fixed_gauge(seed, n_ant):
    a1, a2, I, V, g_true = problem(seed, n_ant)
    g = oracle.calibrate(a1, a2, n_ant, I[None, :, None], V[None, :, None], np.ones((1, 1, n_ant)), 10)[0, 0]
    want = g_true * np.exp(-1j * np.angle(g_true[0]))   # the gauge Im(g_0) = 0 (g_0 starts real)
    assert abs(g[0].imag) == 0.0
    np.testing.assert_allclose(g, want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g[a1] * np.conj(g[a2]), g_true[a1] * np.conj(g_true[a2]), rtol=0, atol=1e-12)


def test_design_matrix_is_the_jacobian_of_the_residual():
    a1, a2, I, V, _ = problem(4, 7, noise=0.1)
    rng = np.random.default_rng(5)
    g = 1 + 0.1 * (rng.normal(size=7) + 1j * rng.normal(size=7))
    A, b = oracle.calib_design(a1, a2, 7, I, V, g)
    re, im = oracle.calib_columns(7)
    for h in (1e-3, 1e-4):
        x = h * rng.normal(size=A.shape[1])
        e = x[re] + 1j * np.where(im >= 0, x[np.maximum(im, 0)], 0.0)
        _, b2 = oracle.calib_design(a1, a2, 7, I, V, g + e)
        # R(g) - R(g + e) = A x + O(|e|^2)
        err = np.linalg.norm((b - b2) - A @ x)
        assert err <= 50 * h * h * np.linalg.norm(x) / h, (h, err)
        assert np.linalg.norm(A @ x) > 100 * err


def test_model_equal_to_data_is_a_fixed_point():
    a1, a2, I, _, _ = problem(6, 9)
    g = 1 + 0.03 * np.arange(9) - 0.02j * np.arange(9)
    V = g[a1] * np.conj(g[a2]) * I
    np.testing.assert_array_equal(oracle.calib_step(a1, a2, 9, I, V, g), g)


def test_converged_gains_satisfy_the_normal_equations():
    a1, a2, I, V, _ = problem(7, 12, noise=0.2)
    g = oracle.calibrate(a1, a2, 12, I[None, :, None], V[None, :, None], np.ones((1, 1, 12)), 30)[0, 0]
    A, b = oracle.calib_design(a1, a2, 12, I, V, g)
    assert np.linalg.norm(A.T @ b) <= 1e-9 * np.linalg.norm(A.T) * np.linalg.norm(b)


def test_calibrate_runs_each_time_and_channel_separately():
    a1, a2, I, V, g_true = problem(8, 6)
    # channel 1 holds data made with other gains; each (t, f) is solved on its own
    rng = np.random.default_rng(9)
    g2 = 1 + 0.05 * (rng.normal(size=6) + 1j * rng.normal(size=6))
    V2 = g2[a1] * np.conj(g2[a2]) * I
    Is = np.stack([I, I], axis=1)[None]
    Vs = np.stack([V, V2], axis=1)[None]
    g = oracle.calibrate(a1, a2, 6, Is, Vs, np.ones((1, 2, 6)), 10)
    np.testing.assert_allclose(g[0, 0], g_true * np.exp(-1j * np.angle(g_true[0])), atol=1e-12)
    np.testing.assert_allclose(g[0, 1], g2 * np.exp(-1j * np.angle(g2[0])), atol=1e-12)
