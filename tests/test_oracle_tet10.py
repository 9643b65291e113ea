"""Pins of the tet10 oracle (Section 3.1's 10-node tetrahedron) against facts fixed by the mathematics,
independent of the oracle's own formulas:

* two integration routes agree (4-point Gauss rule and monomial-by-monomial exact integration);
* element stiffness symmetric, positive semi-definite, exactly six zero modes (rigid-body motions);
* rigid-body modes lie in the null space of the assembled K;
* patch test: a linear displacement field gives zero nodal forces at interior nodes, and its strain energy
  equals the closed form V (lambda tr(eps)^2 / 2 + mu eps:eps) for a homogeneous body;
* a linear field has the same strain energy as with the tet4 oracle on the corner mesh;
* consistent mass: the textbook coefficients (rho V / 420) (6, 32, 1, -4, -6, 16, 8) and total mass rho V.
"""
import numpy as np
import pytest

import oracle
from oracle import tet10_oracle as t10
from paper_2409_20380_gb300 import workload as wl


def _mesh(nx=3, ny=2, nz=2, perturb=0.0, homogeneous=False, seed=0):
    if homogeneous:
        m = wl.layered_mesh(nx, ny, nz, 0.5, layer_tops=[], base_lame=[(3.0, 1.5)])
    else:
        m = wl.layered_mesh(nx, ny, nz, 0.5, layer_tops=[0.5], base_lame=[(4.0, 2.0), (2.0, 1.0)])
    if perturb:
        rng = np.random.default_rng(seed)
        interior = np.all((m.xyz > 1e-9) & (m.xyz < m.xyz.max(axis=0) - 1e-9), axis=1)
        m.xyz[interior] += perturb * 0.5 * (rng.random((interior.sum(), 3)) - 0.5)
    return m, wl.tet10_mesh(m)


def test_tet10_mesh_edge_nodes_are_midpoints():
    m, m10 = _mesh(perturb=0.2)
    for k, (a, b) in enumerate(wl.TET10_EDGES):
        mid = 0.5 * (m10.xyz[m10.conn[:, a]] + m10.xyz[m10.conn[:, b]])
        assert np.allclose(m10.xyz[m10.conn[:, 4 + k]], mid, atol=1e-15)
    # each distinct edge gets one node: Euler-style count on the structured Kuhn mesh
    edges = set()
    for e in m.conn:
        for a, b in wl.TET10_EDGES:
            edges.add((min(e[a], e[b]), max(e[a], e[b])))
    assert m10.n_nodes == m.n_nodes + len(edges)


def test_quadrature_matches_exact_integration():
    _, m10 = _mesh(perturb=0.3)
    K, _ = t10.tet10_element_matrices(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    Kx = t10.tet10_element_stiffness_exact(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    assert np.abs(K - Kx).max() <= 1e-13 * np.abs(K).max()


def test_element_stiffness_symmetric_psd_six_zero_modes():
    _, m10 = _mesh(perturb=0.3)
    K, M = t10.tet10_element_matrices(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    for e in range(0, K.shape[0], 7):
        assert np.abs(K[e] - K[e].T).max() <= 1e-13 * np.abs(K[e]).max()
        ev = np.linalg.eigvalsh(K[e])
        assert ev.min() > -1e-12 * ev.max()
        assert np.sum(ev < 1e-10 * ev.max()) == 6
        assert np.linalg.eigvalsh(M[e]).min() > 0.0


def test_rigid_body_modes_in_null_space():
    _, m10 = _mesh(perturb=0.3)
    K, _ = t10.assemble10(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    x = m10.xyz
    scale = abs(K).sum(axis=1).max()
    for mode in range(6):
        u = np.zeros_like(x)
        if mode < 3:
            u[:, mode] = 1.0
        else:
            w = np.zeros(3)
            w[mode - 3] = 1.0
            u = np.cross(w, x)
        assert np.abs(K @ u.reshape(-1)).max() <= 1e-12 * scale


def test_patch_test_linear_field():
    m, m10 = _mesh(nx=3, ny=3, nz=3, perturb=0.3, homogeneous=True)
    K, _ = t10.assemble10(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    Bg = np.array([[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [0.2, 0.1, -0.25]])
    u = m10.xyz @ Bg.T
    f = (K @ u.reshape(-1)).reshape(-1, 3)
    lo, hi = m10.xyz.min(axis=0), m10.xyz.max(axis=0)
    interior = np.all((m10.xyz > lo + 1e-9) & (m10.xyz < hi - 1e-9), axis=1)
    assert interior.sum() > 0
    assert np.abs(f[interior]).max() <= 1e-12 * np.abs(f).max()
    # strain energy of the homogeneous body in closed form
    lam, mu = m10.lam_mu_rho[0, 0], m10.lam_mu_rho[0, 1]
    eps = 0.5 * (Bg + Bg.T)
    V = np.prod(hi - lo)
    w_exact = V * (0.5 * lam * np.trace(eps) ** 2 + mu * np.sum(eps * eps))
    w = 0.5 * u.reshape(-1) @ (K @ u.reshape(-1))
    assert abs(w - w_exact) <= 1e-12 * w_exact


def test_linear_field_energy_matches_tet4():
    m, m10 = _mesh(perturb=0.3)
    K10, _ = t10.assemble10(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    _, K4 = oracle.assemble(m.xyz, m.conn, m.mat_id, m.lam_mu_rho)
    Bg = np.array([[0.1, 0.2, -0.3], [0.0, -0.4, 0.2], [0.3, 0.1, 0.5]])
    u10 = (m10.xyz @ Bg.T).reshape(-1)
    u4 = (m.xyz @ Bg.T).reshape(-1)
    e10, e4 = u10 @ (K10 @ u10), u4 @ (K4 @ u4)
    assert abs(e10 - e4) <= 1e-12 * abs(e4)


def test_mass_textbook_coefficients_and_total():
    m = t10.mass_coefficients() * 420.0
    assert m[0, 0] == pytest.approx(6.0) and m[4, 4] == pytest.approx(32.0)
    assert m[0, 1] == pytest.approx(1.0)
    assert m[0, 4] == pytest.approx(-4.0)      # corner 0 and edge (0,1): adjacent
    assert m[0, 5] == pytest.approx(-6.0)      # corner 0 and edge (1,2): opposite
    assert m[4, 6] == pytest.approx(16.0)      # edges (0,1) and (0,2) share a corner
    assert m[4, 9] == pytest.approx(8.0)       # edges (0,1) and (2,3) are opposite
    _, m10 = _mesh(perturb=0.3)
    _, M = t10.assemble10(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    ones = np.zeros(3 * m10.n_nodes)
    ones[0::3] = 1.0
    g, V = t10.corner_geometry(m10.xyz, m10.conn)
    rho = m10.lam_mu_rho[m10.mat_id, 2]
    assert ones @ (M @ ones) == pytest.approx(float(np.sum(rho * V)), rel=1e-13)
