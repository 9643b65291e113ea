"""Pins of the oracle's predictors (Section 3.2): Adams-Bashforth 4 and the regional MGS data-driven
correction.  Fixed by their mathematics: polynomial exactness, orthonormality, exact reproduction of
in-span queries and of linear recurrences, agreement with a Householder-QR least-squares solve, and the
column-drop rule."""
import numpy as np
import pytest

import oracle


def test_ab4_coefficients_and_cubic_exactness():
    assert sum(oracle.AB4_COEF) == 24.0
    dt = 0.013
    for t_prev in (0.0, 0.37, 2.0):
        ts = [t_prev - 3 * dt, t_prev - 2 * dt, t_prev - dt, t_prev]
        for deg in range(4):                                   # v = t^deg, u = t^{deg+1}/(deg+1)
            v_hist = [np.array([t ** deg]) for t in ts]
            u_prev = np.array([t_prev ** (deg + 1) / (deg + 1)])
            u_bar = oracle.adams_bashforth4(u_prev, v_hist, dt)
            exact = (t_prev + dt) ** (deg + 1) / (deg + 1)
            assert abs(u_bar[0] - exact) < 1e-13 * max(1.0, abs(exact))
    # degree 4 is not integrated exactly (AB4 has order 4)
    ts = [1.0 - 3 * dt, 1.0 - 2 * dt, 1.0 - dt, 1.0]
    u_bar = oracle.adams_bashforth4(np.array([1.0 / 5]), [np.array([t ** 4]) for t in ts], dt)
    assert abs(u_bar[0] - (1 + dt) ** 5 / 5) > 1e-12


def test_mgs_orthonormal_and_upper():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 12)) @ np.diag(np.logspace(0, -4, 12))
    U, P, kept = oracle.mgs_upper(X, 1e-10)
    assert kept.all()
    assert np.abs(P.T @ P - np.eye(12)).max() < 1e-12
    assert np.abs(np.tril(U, -1)).max() == 0.0
    assert np.abs(X @ U - P).max() < 1e-12


def test_mgs_equals_householder_least_squares():
    rng = np.random.default_rng(1)
    n, s = 500, 16
    X = rng.standard_normal((n, s))
    Y = rng.standard_normal((n, s))
    x = rng.standard_normal(n)
    y, w = oracle.mgs_predict(X, Y, x, tau=1e-10)
    Q, R = np.linalg.qr(X)                                    # Householder (LAPACK geqrf)
    w_ref = np.linalg.solve(R, Q.T @ x)
    cond = np.linalg.cond(X)
    assert np.abs(w - w_ref).max() <= cond * 1e-14 * np.abs(w_ref).max()
    assert np.abs(y - Y @ w_ref).max() <= cond * 1e-14 * np.abs(Y @ w_ref).max()


def test_in_span_query_is_exact():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((200, 8))
    Y = rng.standard_normal((200, 8))
    w_true = rng.standard_normal(8)
    y, w = oracle.mgs_predict(X, Y, X @ w_true, tau=1e-10)
    assert np.abs(w - w_true).max() < 1e-12
    assert np.abs(y - Y @ w_true).max() < 1e-11


def test_linear_recurrence_predicted_exactly():
    """If e^j = T e^{j-1} with rank(T) <= s, the regional predictor returns e^it exactly."""
    rng = np.random.default_rng(3)
    n, s = 120, 6
    Bm = rng.standard_normal((n, s))
    T = Bm @ (0.3 * rng.standard_normal((s, s))) @ np.linalg.pinv(Bm)   # rank s, acts inside span(Bm)
    e = [Bm @ rng.standard_normal(s)]
    for _ in range(s + 2):
        e.append(T @ e[-1])
    region = np.zeros(n, dtype=np.int64)
    y, W = oracle.regional_predict(e[:-1], region, 1, s, tau=1e-10)
    assert np.abs(y - e[-1]).max() < 1e-9 * np.abs(e[-1]).max()


def test_regions_are_independent_and_drop_rule():
    rng = np.random.default_rng(4)
    n, s = 90, 4
    hist = [rng.standard_normal(n) for _ in range(s + 1)]
    region = np.repeat(np.arange(3), 30)
    y, W = oracle.regional_predict(hist, region, 3, s)
    for R in range(3):
        idx = region == R
        yR, _ = oracle.regional_predict([h[idx] for h in hist], np.zeros(30, np.int64), 1, s)
        assert np.abs(y[idx] - yR).max() < 1e-13
    # a duplicated column is dropped and the prediction is unchanged
    X = rng.standard_normal((50, 3))
    Y = rng.standard_normal((50, 3))
    x = rng.standard_normal(50)
    X2 = np.concatenate([X, X[:, 1:2]], axis=1)
    Y2 = np.concatenate([Y, Y[:, 1:2]], axis=1)
    U, P, kept = oracle.mgs_upper(X2, 1e-6)
    assert kept.tolist() == [True, True, True, False]
    y1, _ = oracle.mgs_predict(X, Y, x)
    y2, _ = oracle.mgs_predict(X2, Y2, x)
    assert np.abs(y1 - y2).max() < 1e-12
    # zero history (wave not arrived) -> zero prediction
    yz, _ = oracle.regional_predict([np.zeros(n)] * (s + 1), region, 3, s)
    assert np.all(yz == 0.0)


def test_early_steps_use_fewer_pairs():
    rng = np.random.default_rng(5)
    n = 40
    region = np.zeros(n, np.int64)
    y0, _ = oracle.regional_predict([rng.standard_normal(n)], region, 1, 8)
    assert np.all(y0 == 0.0)                                    # one correction: no pair yet
    h = [rng.standard_normal(n) for _ in range(3)]
    y, W = oracle.regional_predict(h, region, 1, 8)
    assert np.count_nonzero(W[0]) <= 2
