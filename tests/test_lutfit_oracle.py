"""Pins of the LUT-fit reference (oracle/lutfit.py): interpolation is exact
on linear tables, the analytic gradient matches a numerical derivative of
the loss, the loss has its closed form on a constant table, and Adam drives
a problem generated from the model back to zero loss."""
import numpy as np
import pytest

from oracle import lutfit as lf


def _linear_tables():
    na, ng, nb = 6, 5, 12
    a0, da, g0, dg, drho = 0.2, 0.15, 0.0, 0.2, 0.5
    A = a0 + da * np.arange(na)[:, None, None]
    G = g0 + dg * np.arange(ng)[None, :, None]
    Rh = (np.arange(nb) + 0.5)[None, None, :] * drho
    p = 1.0 + 2.0 * A + 3.0 * G + 0.25 * Rh
    R = (0.1 + 0.5 * A + 0.2 * G)[:, :, 0]
    return lf.Tables(R, p, a0, da, g0, dg, drho)


def test_interpolation_is_exact_on_linear_tables():
    tab = _linear_tables()
    for a, g, rho in [(0.31, 0.27, 1.3), (0.9, 0.71, 4.9), (0.2, 0.0, 0.25)]:
        v, da, dg = tab.R_at(a, g)
        assert v == pytest.approx(0.1 + 0.5 * a + 0.2 * g, rel=1e-12)
        assert (da, dg) == pytest.approx((0.5, 0.2), rel=1e-12)
        v, da, dg, dr = tab.p_at(a, g, rho)
        assert v == pytest.approx(1 + 2 * a + 3 * g + 0.25 * rho, rel=1e-12)
        assert (da, dg, dr) == pytest.approx((2.0, 3.0, 0.25), rel=1e-12)


def _smooth_tables(seed=0):
    rng = np.random.default_rng(seed)
    na, ng, nb = 12, 10, 48
    a = np.linspace(0.0, 0.999, na)[:, None, None]
    g = np.linspace(0.0, 0.95, ng)[None, :, None]
    rho = (np.arange(nb) + 0.5)[None, None, :] * 0.25
    lam = 0.4 + 2.0 * (1 - a) + 0.5 * g
    p = (lam ** 2 / (2 * np.pi)) * np.exp(-lam * rho) * (1 + 0.05 * rng.uniform(size=(na, ng, nb)))
    R = (0.9 * a ** 3 * (1 - 0.3 * g))[:, :, 0]
    return lf.Tables(R, p, 0.0, 0.999 / (na - 1), 0.0, 0.95 / (ng - 1), 0.25)


def test_gradient_matches_numerical_derivative():
    tab = _smooth_tables()
    K = 3
    rng = np.random.default_rng(1)
    raw = rng.normal(size=4 * K) * 0.5
    r = np.linspace(0.05, 3.0, 24)
    P_mc = 0.3 * np.exp(-1.2 * r) + 1e-4
    L, g = lf.loss_grad(raw, K, tab, r, P_mc, 0.3)
    h = 1e-6
    for j in range(4 * K):
        e = np.zeros(4 * K); e[j] = h
        num = (lf.loss_grad(raw + e, K, tab, r, P_mc, 0.3)[0]
               - lf.loss_grad(raw - e, K, tab, r, P_mc, 0.3)[0]) / (2 * h)
        assert g[j] == pytest.approx(num, rel=1e-4, abs=1e-7), j


def test_loss_closed_form_on_constant_table():
    # constant tables: P_hat = sigma^2 c for K = 1, so every log error is
    # log(sigma^2 c / P_mc) and the RMSE is its absolute value
    na, ng, nb = 3, 3, 8
    c, Rv = 0.7, 0.25
    tab = lf.Tables(np.full((na, ng), Rv), np.full((na, ng, nb), c), 0.0, 0.5, 0.0, 0.4, 1.0)
    raw = np.array([0.3, -0.2, np.log(2.0), 0.0])
    r = np.linspace(0.5, 3.0, 10)
    P_mc = np.full(10, 0.9)
    L, _ = lf.loss_grad(raw, 1, tab, r, P_mc, 0.1)
    assert L == pytest.approx(abs(np.log(4.0 * c / 0.9)) + 5.0 * (Rv - 0.1) ** 2, rel=1e-12)


def test_adam_recovers_a_problem_generated_from_the_model():
    tab = _smooth_tables(2)
    K = 2
    truth = np.array([1.0, -0.5, 0.3, 0.8, np.log(1.5), np.log(0.6), 0.4, -0.4])
    r = np.linspace(0.05, 4.0, 32)
    a, g, s, w, _, _ = lf.unpack(truth, K, (0.0, 0.999), (0.0, 0.95))
    P_mc = np.array([sum(w[k] * s[k] ** 2 * tab.p_at(a[k], g[k], s[k] * ri)[0] for k in range(K))
                     for ri in r])
    R_mc = sum(w[k] * tab.R_at(a[k], g[k])[0] for k in range(K))
    assert lf.loss_grad(truth, K, tab, r, P_mc, R_mc)[0] == pytest.approx(0.0, abs=1e-12)
    start = truth + np.array([0.3, -0.3, 0.2, -0.2, 0.2, -0.2, 0.3, -0.3])
    L0 = lf.loss_grad(start, K, tab, r, P_mc, R_mc)[0]
    raw, L = lf.fit(start, K, tab, r, P_mc, R_mc, steps=400, lr=2e-2)
    assert L < 0.1 * L0
