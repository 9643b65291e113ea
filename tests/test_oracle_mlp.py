"""Pins of the oracle's learned-proposal network (FP64, CPU): GELU closed forms, gradients by central finite
differences, the closed form of Adam's first step, targets against an SVD least-squares solve, and the
sample builder on a small case."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp_oracle as mo
from paper_2409_20380_gb300 import workload as wl
from helpers import small_mesh


def test_gelu_closed_forms():
    # Phi(1) = 0.841344746068543 (standard normal table), Phi(-1) = 1 - Phi(1), Phi(0) = 1/2
    assert mo.gelu(np.array(0.0)) == 0.0
    assert abs(mo.gelu(np.array(1.0)) - 0.841344746068543) < 1e-15
    assert abs(mo.gelu(np.array(-1.0)) + (1.0 - 0.841344746068543)) < 1e-15
    assert abs(mo.gelu(np.array(12.0)) - 12.0) < 1e-15 and abs(mo.gelu(np.array(-12.0))) < 1e-15
    assert abs(mo.gelu_grad(np.array(0.0)) - 0.5) < 1e-16
    x = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (mo.gelu(x + h) - mo.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mo.gelu_grad(x)).max() < 1e-9


def test_param_layout():
    assert mo.n_params() == 256 * 64 + 256 + 256 * 256 + 256 + 32 * 256 + 32 == 90656
    th = wl.mlp_init_weights(0)
    assert th.shape == (90656,)
    W1, b1, W2, b2, W3, b3 = mo.unpack(th)
    assert W1.shape == (256, 64) and W3.shape == (32, 256)
    assert np.all(b1 == 0) and np.all(b3 == 0)
    assert np.abs(W1).max() <= math.sqrt(6 / 64) and np.abs(W2).max() <= math.sqrt(6 / 256)
    assert np.array_equal(mo.pack(mo.unpack(th)), th)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    th = wl.mlp_init_weights(3) * 0.5
    th[16384:16384 + 256] = rng.normal(0, 0.1, 256)          # nonzero biases
    X = rng.normal(0, 1, (24, 64))
    X[:, 36:] = 0.0
    T = rng.normal(0, 1, (24, 32))
    L, g = mo.loss_and_grad(th, X, T)
    idx = np.concatenate([rng.choice(mo.n_params(), 300, replace=False),
                          [0, 16383, 16384, 16639, 90655, 90655 - 32]])
    for i in idx:
        h = 1e-5 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mo.loss(tp, X, T) - mo.loss(tm, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * np.abs(g).max()), (i, fd, g[i])


def test_output_layer_special_case():
    """With W3 = 0 the network outputs b3; the loss and the b3 gradient have closed forms."""
    rng = np.random.default_rng(2)
    th = wl.mlp_init_weights(1)
    W1, b1, W2, b2, W3, b3 = mo.unpack(th)
    W3[:] = 0.0
    b3[:] = rng.normal(0, 1, 32)
    th = mo.pack([W1, b1, W2, b2, W3, b3])
    X = rng.normal(0, 1, (10, 64))
    T = rng.normal(0, 1, (10, 32))
    L, g = mo.loss_and_grad(th, X, T)
    assert abs(L - np.mean((b3[None, :] - T) ** 2)) < 1e-14
    gb3 = g[-32:]
    assert np.abs(gb3 - 2.0 * (b3 - T.mean(axis=0)) / 32.0).max() < 1e-14
    assert np.all(g[:16384 + 256 + 65536 + 256] == 0.0)       # nothing flows back through W3 = 0


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so every coordinate moves by
    lr * g / (|g| + eps): lr * sign(g) up to eps."""
    rng = np.random.default_rng(4)
    th = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    g[3] = 0.0
    t1, m, v = mo.adam_step(th, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    step = th - t1
    assert np.allclose(step, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert step[3] == 0.0
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_reduces_loss_on_a_teacher_task():
    rng = np.random.default_rng(5)
    teacher = wl.mlp_init_weights(7) * 0.3
    X = rng.normal(0, 1, (512, 64))
    X[:, 36:] = 0
    T, _ = mo.forward(teacher, X)
    th = wl.mlp_init_weights(0)
    batches = [rng.choice(512, 64, replace=False) for _ in range(150)]
    th2, losses = mo.train(th, X, T, batches, lr=1e-3)
    assert mo.loss(th2, X, T) < 0.2 * mo.loss(th, X, T)


def test_best_coefficients_vs_svd_least_squares():
    rng = np.random.default_rng(6)
    Y = rng.normal(0, 1, (300, 12))
    e = rng.normal(0, 1, 300)
    c = mo.best_coefficients(Y, e)
    ref = np.linalg.lstsq(Y, e, rcond=None)[0]
    assert np.abs(c - ref).max() < 1e-12 * np.abs(ref).max() * np.linalg.cond(Y)
    # rank deficient: a repeated column is dropped, the residual is still the least-squares minimum
    Yd = np.concatenate([Y, Y[:, 2:3]], axis=1)
    cd = mo.best_coefficients(Yd, e)
    assert cd[-1] == 0.0
    assert abs(np.linalg.norm(Yd @ cd - e) - np.linalg.norm(Y @ ref - e)) < 1e-10


def test_age_order_and_features():
    c = np.array([1.0, 2.0, 3.0])                             # oldest .. newest
    a = mo.to_age_order(c)
    assert list(a[:4]) == [3.0, 2.0, 1.0, 0.0]
    assert np.array_equal(mo.from_age_order(a, 3), c)
    x = mo.features([0.5, 0.25, 0.125], [0.25, 0.25, 0.25], 2.0, 8.0, c)
    assert np.allclose(x[:4], [0.125, 0.0, -0.0625, 1.0])
    # asinh(t) = log(t + sqrt(t^2 + 1))
    assert np.allclose(x[4:8], [math.log(3 + math.sqrt(10)), math.log(2 + math.sqrt(5)), math.log(1 + math.sqrt(2)), 0])
    assert np.all(x[36:] == 0)
    assert abs(mo.features([0, 0, 0], [0, 0, 0], 1.0, 5.0, [1e300])[4] - 691.4686750787736) < 1e-9


def test_target_clip():
    assert list(mo.target([1.0, 5.0], [0.5, 1.0])[:3]) == [4.0, 0.5, 0.0]
    assert np.all(mo.target([1.0, 500.0], [0.0, 0.0]) == 0.0)
    assert np.all(mo.target([np.inf, 1.0], [0.0, 0.0]) == 0.0)


def test_step_samples_small_case():
    """Targets of a developed step: Y c* reproduces e^it in every region at least as well as the
    predictor's own coefficients (c* is the least-squares optimum in the same basis)."""
    m = small_mesh(6, 5, 4)
    tp = wl.config2_time_params()
    sysm, A = oracle.build_system(m, tp)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    reg = wl.region_map(m, 64)
    src = wl.random_source(m, wl.rng_for(9, 0, 0, 2))
    sim = oracle.CaseSimulator(sysm, A, Binv, src, predictor="dd", s_max=8, region_of_node=reg)
    R = sim.n_regions
    cents = mo.region_centroids(m.xyz, reg, R)
    L = mo.domain_extent(m.xyz)
    for _ in range(14):
        sim.step()
        X, T = mo.step_samples(sim, m.xyz[src.node], cents, L, src.f0)
    n = sim.last_npairs
    assert n == 8 and X.shape == (R, 64) and T.shape == (R, 32)
    Y = np.stack(sim.E_hist[-(n + 1):-1], axis=1)
    e = sim.E_hist[-1]
    for r in range(R):
        idx = np.nonzero(sim.region_of_dof == r)[0]
        c = mo.from_age_order(np.sinh(X[r, 4:36]), n)
        cs = c + mo.from_age_order(T[r], n)
        assert np.linalg.norm(Y[idx] @ cs - e[idx]) <= np.linalg.norm(Y[idx] @ c - e[idx]) * (1 + 1e-9) + 1e-300
        assert np.allclose(X[r, :3], (m.xyz[src.node] - cents[r]) / L)


# ---------------------------------------------------------------------------------------------------------
# Residual-space loss (L6)
# ---------------------------------------------------------------------------------------------------------

def _explicit_rel_residual(Y, e, c, d_age):
    """||Y (c + d) - e||^2 / ||e||^2 with d given in age order, written out directly from the vectors."""
    n = Y.shape[1]
    d_slot = np.array([d_age[n - 1 - a] for a in range(n)])
    return float(np.sum((Y @ (c + d_slot) - e) ** 2) / np.sum(e ** 2))


def _lstsq_floor(Y, e):
    """min_c ||Y c - e||^2 / ||e||^2 by an SVD least-squares solve (independent of MGS)."""
    c, *_ = np.linalg.lstsq(Y, e, rcond=None)
    return float(np.sum((Y @ c - e) ** 2) / np.sum(e ** 2))


@pytest.mark.parametrize("rank_deficient", [False, True])
def test_residual_sample_reproduces_the_relative_residual(rank_deficient):
    """||W d - w||^2 plus the least-squares floor equals the relative residual ||Y (c + d) - e||^2 / ||e||^2
    of the proposed correction, for any d; also with a column of Y repeated (the drop rule removes it)."""
    rng = np.random.default_rng(11)
    n, rows = 7, 60
    Y = rng.normal(0, 1, (rows, n)) * np.logspace(0, -3, n)
    if rank_deficient:
        Y[:, 4] = Y[:, 1]
    e = Y @ rng.normal(0, 1, n) + 0.05 * rng.normal(0, 1, rows)
    c = rng.normal(0, 1, n)
    W, w = mo.residual_sample(Y, e, c)
    assert np.allclose(W, np.triu(W)) and np.all(np.diag(W)[:n] >= 0.0)
    assert np.all(W[n:, :] == 0.0) and np.all(W[:, n:] == 0.0) and np.all(w[n:] == 0.0)
    floor = _lstsq_floor(Y, e)
    for trial in range(5):
        d = rng.normal(0, 1, 32) * (0.0 if trial == 0 else 1.0)
        lhs = float(np.sum((W @ d - w) ** 2)) + floor
        rhs = _explicit_rel_residual(Y, e, c, d)
        assert abs(lhs - rhs) <= 1e-10 * rhs, (trial, lhs, rhs)
    # the least-squares coefficients make the residual-space term vanish
    cs = mo.best_coefficients(Y, e)
    d_opt = mo.to_age_order(cs - c)
    assert np.sum((W @ d_opt - w) ** 2) <= 1e-20 + 1e-12 * np.sum(w ** 2)


def test_residual_packing_round_trip():
    rng = np.random.default_rng(12)
    W = np.triu(rng.normal(0, 1, (32, 32)))
    w = rng.normal(0, 1, 32)
    S = mo.pack_residual(W, w)
    assert S.shape == (mo.N_RES,) and mo.N_RES == 528 + 32
    W2, w2 = mo.unpack_residual(S)
    assert np.array_equal(W2[0], W) and np.array_equal(w2[0], w)


def test_residual_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(13)
    th = wl.mlp_init_weights(4) * 0.5
    th[-32:] = rng.normal(0, 0.1, 32)
    X = rng.normal(0, 1, (16, 64))
    X[:, 36:] = 0.0
    S = np.stack([mo.pack_residual(np.triu(rng.normal(0, 1, (32, 32))), rng.normal(0, 1, 32)) for _ in range(16)])
    L, g = mo.loss_and_grad_residual(th, X, S)
    assert abs(L - mo.loss_residual(th, X, S)) <= 1e-14 * L
    idx = np.concatenate([rng.choice(mo.n_params(), 200, replace=False), [0, 16384, 90655, 90655 - 32]])
    for i in idx:
        h = 1e-5 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mo.loss_residual(tp, X, S) - mo.loss_residual(tm, X, S)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * np.abs(g).max()), (i, fd, g[i])


def test_residual_loss_identity_weights_is_the_squared_error():
    """With W = I and w = t the L6 loss is the sum over the 32 outputs of (d - t)^2, i.e. 32 x the MSE."""
    rng = np.random.default_rng(14)
    th = wl.mlp_init_weights(5)
    X = rng.normal(0, 1, (8, 64))
    T = rng.normal(0, 1, (8, 32))
    S = np.stack([mo.pack_residual(np.eye(32), t) for t in T])
    L1, g1 = mo.loss_and_grad_residual(th, X, S)
    L0, g0 = mo.loss_and_grad(th, X, T)
    assert abs(L1 - 32.0 * L0) <= 1e-12 * L1
    assert np.abs(g1 - 32.0 * g0).max() <= 1e-12 * np.abs(g1).max()


def test_residual_step_samples_small_case():
    """Residual-space samples of a developed oracle step: a zero network's loss, summed over the regions, is
    the relative error of the case's plain guess of the correction above the least-squares floors,
    (||Y c - e||^2 - floors) / ||e||^2."""
    m = small_mesh(6, 5, 4)
    tp = wl.config2_time_params()
    sysm, A = oracle.build_system(m, tp)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    reg = wl.region_map(m, 64)
    src = wl.random_source(m, wl.rng_for(9, 0, 0, 2))
    sim = oracle.CaseSimulator(sysm, A, Binv, src, predictor="dd", s_max=8, region_of_node=reg)
    R = sim.n_regions
    cents = mo.region_centroids(m.xyz, reg, R)
    L = mo.domain_extent(m.xyz)
    for _ in range(14):
        sim.step()
    X, S = mo.step_samples_residual(sim, m.xyz[src.node], cents, L, src.f0)
    n = sim.last_npairs
    assert n == 8 and S.shape == (R, mo.N_RES)
    Y = np.stack(sim.E_hist[-(n + 1):-1], axis=1)
    e = sim.E_hist[-1]
    Wb, wb = mo.unpack_residual(S)
    y_case = np.zeros_like(e)
    for r in range(R):
        idx = np.nonzero(sim.region_of_dof == r)[0]
        y_case[idx] = Y[idx] @ sim.last_W[r, :n]
    D = float(e @ e)
    err2 = float(np.sum((y_case - e) ** 2))         # the plain guess's squared error, written out
    assert abs(mo.plain_error2(Y, e, sim.last_W, n, sim.region_of_dof, R) - err2) <= 1e-12 * err2
    zero, rel, floor = 0.0, 0.0, 0.0
    for r in range(R):
        idx = np.nonzero(sim.region_of_dof == r)[0]
        c = sim.last_W[r, :n]
        ze = float(np.sum(wb[r] ** 2))
        er2 = float(e[idx] @ e[idx])
        re = _explicit_rel_residual(Y[idx], e[idx], c, np.zeros(32)) * er2 / D
        fl = _lstsq_floor(Y[idx], e[idx]) * er2 / D
        assert abs(ze + fl - re) <= 1e-8 * re + 1e-14, (r, ze, re)
        zero, rel, floor = zero + ze, rel + re, floor + fl
    assert abs(rel - err2 / D) <= 1e-10 * rel
    assert zero + floor <= rel * (1.0 + 1e-8) and zero >= 0.0
