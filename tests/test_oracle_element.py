"""Pins of the oracle's element matrices and assembly (Section 3.1, Eq. GE:ORG discretised by tets).

Each check is fixed by mathematics, not by the oracle itself: a hand-derived single-tet closed form, the
patch test, rigid-body null space, symmetry/definiteness, and total mass."""
import os

import numpy as np
import pytest

import oracle
from paper_2409_20380_gb300 import workload as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden", "unit_tet_lame2_3.txt")


def _unit_tet():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    conn = np.array([[0, 1, 2, 3]], dtype=np.int32)
    return xyz, conn


def test_unit_tet_closed_form():
    xyz, conn = _unit_tet()
    Ke, Me = oracle.tet4_element_matrices(xyz, conn, np.zeros(1, np.int32), np.array([[2.0, 3.0, 1.0]]))
    d = {"x": 0, "y": 1, "z": 2}
    n = 0
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        m, a, i, b, j, num, den = line.split()
        r, c = 3 * int(a) + d[i], 3 * int(b) + d[j]
        val = float(num) / float(den)
        got = (Ke if m == "K" else Me)[0, r, c]
        assert abs(got - val) < 1e-14, (line, got, val)
        n += 1
    assert n >= 16


def _random_tets(n, seed=0):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((n, 4, 3))
    det = np.linalg.det(P[:, 1:] - P[:, :1])
    P[det < 0, 2], P[det < 0, 3] = P[det < 0, 3].copy(), P[det < 0, 2].copy()
    xyz = P.reshape(-1, 3)
    conn = np.arange(4 * n, dtype=np.int32).reshape(n, 4)
    props = np.stack([rng.uniform(0.5, 5, n), rng.uniform(0.5, 5, n), rng.uniform(0.5, 2, n)], axis=1)
    return xyz, conn, np.arange(n, dtype=np.int32), props


def test_element_symmetry_definiteness_rank():
    xyz, conn, mid, props = _random_tets(50)
    Ke, Me = oracle.tet4_element_matrices(xyz, conn, mid, props)
    assert np.abs(Ke - Ke.transpose(0, 2, 1)).max() < 1e-12 * np.abs(Ke).max()
    assert np.abs(Me - Me.transpose(0, 2, 1)).max() == 0.0
    for e in range(50):
        ev = np.linalg.eigvalsh(Ke[e])
        tol = 1e-10 * ev.max()
        assert ev.min() > -tol                                  # PSD
        assert (ev > tol).sum() == 6                            # 12 DOF - 6 rigid modes
        assert np.linalg.eigvalsh(Me[e]).min() > 0.0            # SPD


def _mesh(Hx=3, Hy=2, Hz=2, h=0.5, perturb=0.0):
    m = wl.layered_mesh(Hx, Hy, Hz, h, layer_tops=[0.5], base_lame=[(4.0, 2.0), (2.0, 1.0)])
    if perturb:
        rng = np.random.default_rng(3)
        inner = wl.interior_nodes(m)
        m.xyz[inner] += perturb * h * rng.uniform(-1, 1, (inner.size, 3))
    return m


@pytest.mark.parametrize("perturb", [0.0, 0.2])
def test_rigid_body_modes_in_null_space(perturb):
    m = _mesh(perturb=perturb)
    M, K = oracle.assemble(m.xyz, m.conn, m.mat_id, m.lam_mu_rho)
    N = m.n_nodes
    x = m.xyz
    modes = []
    for i in range(3):
        t = np.zeros((N, 3))
        t[:, i] = 1.0
        modes.append(t.ravel())
    for w in np.eye(3):
        modes.append(np.cross(w, x).ravel())                     # infinitesimal rotation
    scale = abs(K).max() * np.abs(x).max()
    for u in modes:
        assert np.abs(K @ u).max() < 1e-12 * scale


@pytest.mark.parametrize("perturb", [0.0, 0.25])
def test_patch_test_linear_field(perturb):
    """A linear displacement u = G x + c has constant stress: interior nodal forces vanish."""
    m = _mesh(4, 3, 3, 0.5, perturb)
    m.mat_id[:] = 0                                              # patch test needs one material
    _, K = oracle.assemble(m.xyz, m.conn, m.mat_id, m.lam_mu_rho)
    rng = np.random.default_rng(7)
    G = rng.standard_normal((3, 3))
    c = rng.standard_normal(3)
    u = (m.xyz @ G.T + c).ravel()
    f = (K @ u).reshape(-1, 3)
    inner = wl.interior_nodes(m)
    assert inner.size > 0
    assert np.abs(f[inner]).max() < 1e-11 * np.abs(f).max()
    # boundary forces are not all zero (the field is loaded through the surface)
    assert np.abs(f).max() > 1e-3


def test_total_mass():
    m = _mesh(3, 3, 2, 0.5)
    m.lam_mu_rho[:, 2] = [1.7, 2.3]
    M, _ = oracle.assemble(m.xyz, m.conn, m.mat_id, m.lam_mu_rho)
    ex = np.zeros(3 * m.n_nodes)
    ex[0::3] = 1.0
    vol = m.h ** 3 / 6.0
    rho = m.lam_mu_rho[m.mat_id, 2]
    assert abs(ex @ (M @ ex) - (rho * vol).sum()) < 1e-12 * (rho * vol).sum()
    assert abs(M - M.T).max() < 1e-15 * abs(M).max()


def test_kuhn_split_volume_and_conformity():
    m = _mesh(3, 2, 2, 0.5)
    P = m.xyz[m.conn]
    vol = np.linalg.det(P[:, 1:] - P[:, :1]) / 6.0
    assert vol.min() > 0.0
    assert abs(vol.sum() - 3 * 2 * 2 * 0.5 ** 3) < 1e-13
    # conforming: every interior triangular face is shared by exactly two tets
    faces = np.sort(np.concatenate([m.conn[:, [0, 1, 2]], m.conn[:, [0, 1, 3]], m.conn[:, [0, 2, 3]],
                                    m.conn[:, [1, 2, 3]]]), axis=1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert counts.max() == 2
    boundary_faces = (counts == 1).sum()
    assert boundary_faces == 2 * 2 * (3 * 2 + 3 * 2 + 2 * 2)     # two triangles per boundary quad
