"""Pins of the oracle's Newmark step (Section 3.1, Eq. GE:DIS and Eq. timestep with readings R1-R3).

Average-acceleration Newmark (beta = 1/4, gamma = 1/2) has closed-form properties that fail for a wrong
coefficient or sign: a single-DOF oscillator advances by the exact rotation angle 2 atan(w dt / 2), and
an undamped, unforced system conserves E = 1/2 v^T M v + 1/2 u^T K u exactly.  A planted mistake (the
'+ 4/dt v' acceleration sign as printed) is shown to be caught."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2409_20380_gb300 import workload as wl


def _sdof(m, k, c=0.0, dt=0.1):
    M = sp.csr_matrix([[m]])
    K = sp.csr_matrix([[k]])
    s = oracle.System(M=M, K=K, free=np.array([0]), dt=dt, a0=c / m if m else 0.0, a1=0.0)
    return s


def _run_sdof(s, u0, n, update=None):
    update = update or oracle.newmark_update
    A = s.reduce(s.A_full).toarray()
    u = np.array([u0])
    v = np.zeros(1)
    a = -(s.K @ u) / s.M.toarray()[0, 0]                       # consistent initial acceleration
    out = [u[0]]
    for _ in range(n):
        b = oracle.newmark_rhs(s, np.zeros(1), u, v, a)
        du = np.linalg.solve(A, b)
        u, v, a = update(u, v, a, du, s.dt)
        out.append(u[0])
    return np.array(out)


def test_sdof_exact_rotation_angle():
    m, k, dt = 2.0, 50.0, 0.07
    w = math.sqrt(k / m)
    s = _sdof(m, k, dt=dt)
    u = _run_sdof(s, 1.0, 200)
    theta = 2.0 * math.atan(w * dt / 2.0)                       # trapezoidal rule phase per step
    n = np.arange(201)
    assert np.abs(u - np.cos(n * theta)).max() < 1e-12


def test_planted_plus_sign_breaks_sdof():
    """The printed '+ 4/dt v' in the acceleration update does not give the trapezoidal rotation."""
    def wrong_update(u, v, a, du, dt):
        v_new = -v + 2.0 / dt * du
        a_new = -a + 4.0 / dt * v + 4.0 / dt ** 2 * du
        return u + du, v_new, a_new
    m, k, dt = 2.0, 50.0, 0.07
    s = _sdof(m, k, dt=dt)
    u = _run_sdof(s, 1.0, 200, update=wrong_update)
    theta = 2.0 * math.atan(math.sqrt(k / m) * dt / 2.0)
    assert np.abs(u - np.cos(np.arange(201) * theta)).max() > 1e-3


def _small_system(dt=0.01, a0=0.0, a1=0.0):
    m = wl.layered_mesh(3, 3, 2, 0.25, layer_tops=[0.25], base_lame=[(4.0, 2.0), (2.0, 1.0)])
    tp = wl.TimeParams(dt=dt, a0=a0, a1=a1)
    sysm, A = oracle.build_system(m, tp)
    return m, sysm, A


def _free_vibration(sysm, A, u0, n, update):
    free = sysm.free
    Ared = A.toarray()
    Mr = sysm.reduce(sysm.M).toarray()
    u = u0.copy()
    v = np.zeros_like(u)
    a = np.zeros_like(u)
    a[free] = np.linalg.solve(Mr, -(sysm.K @ u)[free])
    E = [oracle.energy(sysm, u, v)]
    for _ in range(n):
        b = oracle.newmark_rhs(sysm, np.zeros_like(u), u, v, a)[free]
        du = np.zeros_like(u)
        du[free] = np.linalg.solve(Ared, b)
        u, v, a = update(u, v, a, du, sysm.dt)
        E.append(oracle.energy(sysm, u, v))
    return np.array(E)


def test_undamped_energy_conserved():
    m, sysm, A = _small_system()
    rng = np.random.default_rng(1)
    u0 = np.zeros(3 * m.n_nodes)
    u0[sysm.free] = rng.standard_normal(sysm.free.size) * 1e-3
    E = _free_vibration(sysm, A, u0, 100, oracle.newmark_update)
    assert np.abs(E / E[0] - 1.0).max() < 1e-12


def test_planted_plus_sign_breaks_energy():
    def wrong_update(u, v, a, du, dt):
        return u + du, -v + 2.0 / dt * du, -a + 4.0 / dt * v + 4.0 / dt ** 2 * du
    m, sysm, A = _small_system()
    rng = np.random.default_rng(1)
    u0 = np.zeros(3 * m.n_nodes)
    u0[sysm.free] = rng.standard_normal(sysm.free.size) * 1e-3
    E = _free_vibration(sysm, A, u0, 20, wrong_update)
    assert np.abs(E / E[0] - 1.0).max() > 1e-3


def test_forced_energy_balance():
    """Undamped forced trapezoidal rule: E^n - E^{n-1} = 1/2 (f^n + f^{n-1})^T (u^n - u^{n-1})."""
    m, sysm, A = _small_system()
    src = wl.random_source(m, np.random.default_rng(5), f0=5.0)
    free = sysm.free
    Ared = A.toarray()
    n = 3 * m.n_nodes
    u, v, a = np.zeros(n), np.zeros(n), np.zeros(n)
    f_prev = oracle.point_force(n, src, 0.0)
    Mr = sysm.reduce(sysm.M).toarray()
    a[free] = np.linalg.solve(Mr, f_prev[free])
    for it in range(1, 60):
        f = oracle.point_force(n, src, it * sysm.dt)
        b = oracle.newmark_rhs(sysm, f, u, v, a)[free]
        du = np.zeros(n)
        du[free] = np.linalg.solve(Ared, b)
        E0 = oracle.energy(sysm, u, v)
        u, v, a = oracle.newmark_update(u, v, a, du, sysm.dt)
        E1 = oracle.energy(sysm, u, v)
        work = 0.5 * (f + f_prev)[free] @ du[free]
        assert abs((E1 - E0) - work) <= 1e-10 * max(abs(E1), abs(work), 1e-300)
        f_prev = f


def test_ricker_closed_form():
    f0, t0 = 5.0, 0.24
    assert abs(oracle.ricker(t0, f0, t0, 2.5) - 2.5) < 1e-15
    tz = t0 + 1.0 / (math.sqrt(2.0) * math.pi * f0)             # zero crossings of the Mexican hat
    assert abs(oracle.ricker(tz, f0, t0)) < 1e-15
    assert abs(oracle.ricker(2 * t0 - tz, f0, t0)) < 1e-15
    assert abs(oracle.ricker(t0 + 0.1, f0, t0) - oracle.ricker(t0 - 0.1, f0, t0)) < 1e-15


def test_damping_matrix_is_rayleigh():
    m, sysm, A = _small_system(dt=0.01, a0=0.3, a1=0.002)
    dt = sysm.dt
    A2 = sysm.reduce((4 / dt ** 2 + 2 * 0.3 / dt) * sysm.M + (1 + 2 * 0.002 / dt) * sysm.K)
    assert abs(A - A2).max() < 1e-9 * abs(A).max()
