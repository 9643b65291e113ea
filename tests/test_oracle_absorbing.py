"""Pins of the oracle's absorbing side boundaries (R22: Lysmer-Kuhlemeyer dashpots lumped to the faces'
corners) and of the random-impulse load (R23).

* Closed form: on a homogeneous box the node blocks of the four vertical sides sum to
  rho (2 Ly Lz diag(c_p, c_s, c_s) + 2 Lx Lz diag(c_s, c_p, c_s)) -- each side's area times rho c_p in its
  normal direction and rho c_s in the tangential ones.
* Energy: average-acceleration Newmark with C = C_b (no Rayleigh damping, no load) satisfies
  E^n - E^{n-1} = -dt vbar^T C_b vbar exactly, vbar = (v^n + v^{n-1}) / 2, E = 1/2 v^T M v + 1/2 u^T K u.  It pins
  the factor 2/dt with which C enters A and the C v term of the right-hand side; a planted 1/dt fails.
* The impulse load of a step is the sum of the impulses of that step at their nodes."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2409_20380_gb300 import workload as wl


def _box(Hx=3, Hy=4, Hz=2, h=0.25, lame=(4.0, 2.0)):
    return wl.layered_mesh(Hx, Hy, Hz, h, layer_tops=[], base_lame=[lame])


def test_dashpot_closed_form_on_a_homogeneous_box():
    m = _box()
    faces = wl.side_faces(m)
    Hx, Hy, Hz = m.dims
    assert faces.shape == (2 * 2 * (Hx * Hz + Hy * Hz), 3)       # two triangles per hex face
    B = oracle.lysmer_dashpots(m.xyz, m.conn, m.mat_id, m.lam_mu_rho, faces).toarray()
    lam, mu, rho = m.lam_mu_rho[0]
    cp, cs = math.sqrt((lam + 2 * mu) / rho), math.sqrt(mu / rho)
    Lx, Ly, Lz = Hx * m.h, Hy * m.h, Hz * m.h
    ref = rho * (2 * Ly * Lz * np.diag([cp, cs, cs]) + 2 * Lx * Lz * np.diag([cs, cp, cs]))
    S = sum(B[3 * n:3 * n + 3, 3 * n:3 * n + 3] for n in range(m.n_nodes))
    assert np.abs(S - ref).max() <= 1e-13 * np.abs(ref).max()
    on_side = np.zeros(m.n_nodes, dtype=bool)
    on_side[faces.ravel()] = True
    for n in range(m.n_nodes):
        blk = B[3 * n:3 * n + 3, 3 * n:3 * n + 3]
        assert np.array_equal(blk, blk.T)
        assert np.linalg.eigvalsh(blk).min() >= -1e-15
        if not on_side[n]:
            assert np.all(blk == 0.0)
    # only diagonal node blocks
    Bd = sp.block_diag([B[3 * n:3 * n + 3, 3 * n:3 * n + 3] for n in range(m.n_nodes)]).toarray()
    assert np.array_equal(B, Bd)


def test_dashpot_rejects_an_interior_face():
    m = _box()
    tet = m.conn[len(m.conn) // 2]
    # an interior face of a tet in the middle of the box is shared by two elements
    interior = None
    for k in range(4):
        tri = np.delete(tet, k)
        if not np.all(np.isin(tri, wl.side_faces(m).ravel())):
            interior = tri
            break
    with pytest.raises(ValueError):
        oracle.lysmer_dashpots(m.xyz, m.conn, m.mat_id, m.lam_mu_rho, interior[None, :])


def _free_vibration_energy(mesh, dt, n_steps, cb_factor_in_A=2.0):
    """Undamped, unforced Newmark steps with the side dashpots, from a seeded initial displacement; returns the
    energies and the dissipation terms dt vbar^T C_b vbar of each step."""
    tp = wl.TimeParams(dt=dt, a0=0.0, a1=0.0)
    sysm, A = oracle.build_system(mesh, tp, absorbing_faces=wl.side_faces(mesh))
    if cb_factor_in_A != 2.0:      # a planted mistake: C_b entering A with a wrong factor
        A = sysm.reduce(4.0 / dt ** 2 * sysm.M + cb_factor_in_A / dt * sysm.Cb + sysm.K)
    free = sysm.free
    Ad = A.toarray()
    rng = np.random.default_rng(5)
    n = 3 * mesh.n_nodes
    u = np.zeros(n)
    u[free] = rng.normal(0, 1e-3, free.size)
    v = np.zeros(n)
    a = np.zeros(n)
    a[free] = np.linalg.solve(sysm.reduce(sysm.M).toarray(), -(sysm.K @ u)[free])
    E, D = [oracle.energy(sysm, u, v)], []
    for _ in range(n_steps):
        b = oracle.newmark_rhs(sysm, np.zeros(n), u, v, a)[free]
        du = np.zeros(n)
        du[free] = np.linalg.solve(Ad, b)
        u2, v2, a2 = oracle.newmark_update(u, v, a, du, dt)
        vbar = 0.5 * (v + v2)
        D.append(dt * vbar @ (sysm.Cb @ vbar))
        u, v, a = u2, v2, a2
        E.append(oracle.energy(sysm, u, v))
    return np.array(E), np.array(D)


def test_energy_balance_with_dashpots():
    m = _box(3, 3, 2, 0.25)
    E, D = _free_vibration_energy(m, 0.02, 40)
    dE = np.diff(E)
    assert np.all(D > 0.0) and np.all(dE < 0.0)                 # the dashpots only take energy out
    assert np.abs(dE + D).max() <= 1e-10 * E[0], np.abs(dE + D).max() / E[0]
    assert E[-1] < 0.9 * E[0]


def test_planted_dashpot_factor_breaks_the_energy_balance():
    m = _box(3, 3, 2, 0.25)
    E, D = _free_vibration_energy(m, 0.02, 40, cb_factor_in_A=1.0)
    assert np.abs(np.diff(E) + D).max() > 1e-3 * E[0]


def test_impulse_load():
    m = _box(4, 4, 2, 0.25)
    imp = wl.random_impulses(m, wl.rng_for(6, 0, 0, 4), n_points=7, last_step=5)
    surf = wl.surface_nodes(m)
    assert imp.nodes.size == 7 and np.all(np.isin(imp.nodes, surf)) and len(set(imp.nodes)) == 7
    assert np.all((imp.steps >= 1) & (imp.steps <= 5))
    n = 3 * m.n_nodes
    total = np.zeros(n)
    for it in range(0, 8):
        f = oracle.impulse_force(n, imp, it)
        for k in range(imp.nodes.size):
            node = imp.nodes[k]
            if imp.steps[k] == it:
                assert np.array_equal(f[3 * node:3 * node + 3], imp.forces[k])
        mask = np.zeros(n, dtype=bool)
        for k in np.nonzero(imp.steps == it)[0]:
            mask[3 * imp.nodes[k]:3 * imp.nodes[k] + 3] = True
        assert np.all(f[~mask] == 0.0)
        total += f
    ref = np.zeros(n)
    for k in range(imp.nodes.size):
        ref[3 * imp.nodes[k]:3 * imp.nodes[k] + 3] += imp.forces[k]
    assert np.array_equal(total, ref)
    assert np.all(oracle.case_force(n, imp, 3, 0.01) == oracle.impulse_force(n, imp, 3))
