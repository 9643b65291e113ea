"""Pins of the oracle's Algorithm 1 (3x3 block-Jacobi PCG) and its Dirichlet elimination.

Fixed by linear algebra: dense direct solves on tiny meshes, one-iteration convergence when the
preconditioner is the exact inverse, finite termination, and the zero right-hand side."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2409_20380_gb300 import workload as wl


def _tiny(H):
    m = wl.layered_mesh(H, H, H, 1.0 / H, layer_tops=[0.5], base_lame=[(4.0, 2.0), (2.0, 1.0)])
    sysm, A = oracle.build_system(m, wl.TimeParams(dt=0.05, a0=0.01, a1=0.001))
    return m, sysm, A


@pytest.mark.parametrize("H", [1, 2, 3])
def test_cg_matches_dense_direct_solve(H):
    m, sysm, A = _tiny(H)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    rng = np.random.default_rng(H)
    b = rng.standard_normal(A.shape[0])
    x_ref = np.linalg.solve(A.toarray(), b)
    res = oracle.block_jacobi_cg(A, Binv, b, np.zeros_like(b), eps=1e-13)
    assert np.linalg.norm(res.x - x_ref) <= 1e-11 * np.linalg.norm(x_ref)
    assert res.relres < 1e-13
    # Dirichlet elimination: the reduced operator equals the full one restricted to free DOFs
    Afull = sysm.A_full.toarray()
    assert np.array_equal(A.toarray(), Afull[np.ix_(sysm.free, sysm.free)])


def test_block_jacobi_inverse_blocks():
    m, sysm, A = _tiny(2)
    Binv = oracle.block_jacobi_inverse(A, sysm.free).toarray()
    Ad = A.toarray()
    node = sysm.free // 3
    for nd in np.unique(node)[:20]:
        idx = np.nonzero(node == nd)[0]
        blk = Ad[np.ix_(idx, idx)]
        assert np.abs(Binv[np.ix_(idx, idx)] @ blk - np.eye(idx.size)).max() < 1e-12
        other = np.setdiff1d(np.arange(Ad.shape[0]), idx)
        assert np.abs(Binv[np.ix_(idx, other)]).max() == 0.0


def test_exact_preconditioner_one_iteration():
    """If A is 3x3-block diagonal, B^{-1} = A^{-1} and Algorithm 1 stops after one iteration."""
    rng = np.random.default_rng(0)
    nb = 40
    blocks = []
    for _ in range(nb):
        Q = rng.standard_normal((3, 3))
        blocks.append(Q @ Q.T + 3 * np.eye(3))
    A = sp.csr_matrix(sp.block_diag([sp.csr_matrix(b) for b in blocks]))
    free = np.arange(3 * nb)
    Binv = oracle.block_jacobi_inverse(A, free)
    b = rng.standard_normal(3 * nb)
    res = oracle.block_jacobi_cg(A, Binv, b, np.zeros(3 * nb), eps=1e-12)
    assert res.iters == 1
    assert res.relres < 1e-13


def test_finite_termination_24_dof():
    m, sysm, A = _tiny(1)            # 1 hex: 8 nodes, bottom 4 fixed -> 12 free DOFs
    n = A.shape[0]
    assert n == 12
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    b = np.random.default_rng(2).standard_normal(n)
    res = oracle.block_jacobi_cg(A, Binv, b, np.zeros(n), eps=1e-12)
    assert res.iters <= n + 2
    # a 24-DOF system: two free layers of a 1x1x2 column
    m2 = wl.layered_mesh(1, 1, 2, 0.5, layer_tops=[0.5], base_lame=[(4.0, 2.0), (2.0, 1.0)])
    s2, A2 = oracle.build_system(m2, wl.TimeParams(dt=0.5))
    assert A2.shape[0] == 24
    B2 = oracle.block_jacobi_inverse(A2, s2.free)
    b2 = np.random.default_rng(3).standard_normal(24)
    r2 = oracle.block_jacobi_cg(A2, B2, b2, np.zeros(24), eps=1e-12)
    assert r2.iters <= 24 + 2 and r2.relres < 1e-12


def test_zero_rhs_and_good_guess():
    m, sysm, A = _tiny(2)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    n = A.shape[0]
    res = oracle.block_jacobi_cg(A, Binv, np.zeros(n), np.ones(n))
    assert res.iters == 0 and np.all(res.x == 0.0)
    b = np.random.default_rng(4).standard_normal(n)
    x = np.linalg.solve(A.toarray(), b)
    res2 = oracle.block_jacobi_cg(A, Binv, b, x, eps=1e-8)
    assert res2.iters == 0
