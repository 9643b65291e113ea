"""pcg_solve on the GPU (Algorithm 1 with the EBE product; FP64, and FP32-inner / FP64-refined) against
the oracle: the certified residual is recomputed here from the oracle's CSR matrix, and the solution is
compared with a sparse direct solve.

Bounds: a solve certified at ||b - A x|| / ||b|| < eps has relative error at most kappa(A) * eps; with
eps = 1e-12 the GPU solution must match the direct solve to 1e-9 (kappa of these systems < 1e3)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import from_cases, small_mesh, to_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    build.build()
    fem.lib()
    return torch


def _setup(dims, r, perturb=0.1, seed=0):
    m = small_mesh(*dims, perturb=perturb)
    tp = wl.TimeParams()
    sysm, A = oracle.build_system(m, tp)
    rng = np.random.default_rng(seed)
    bs = []
    for _ in range(r):
        b = np.zeros(3 * m.n_nodes)
        b[sysm.free] = rng.standard_normal(sysm.free.size)
        bs.append(b)
    return m, tp, sysm, A, bs


@pytest.mark.parametrize("precision", [fem.FEM_FP64, fem.FEM_FP32_INNER])
@pytest.mark.parametrize("dims,r", [((7, 5, 4), 1), ((9, 6, 5), 4), ((8, 8, 6), 16)])
def test_pcg_certified_and_matches_direct(torch_dev, precision, dims, r):
    torch = torch_dev
    m, tp, sysm, A, bs = _setup(dims, r, seed=r)
    h = fem.fem_mesh_create(m, tp)
    try:
        for tol in (1e-8, 1e-12):
            b = torch.tensor(from_cases(bs, m.n_nodes, r), device="cuda")
            x = torch.zeros_like(b)
            opts = fem.fem_opts_default(precision=precision, tol=tol)
            st, iters, relres = fem.pcg_solve(h, b, x, r, opts)
            xs = to_cases(x.cpu().numpy(), m.n_nodes, r)
            for c in range(r):
                bf = bs[c][sysm.free]
                xf = xs[c][sysm.free]
                cert = np.linalg.norm(bf - A @ xf) / np.linalg.norm(bf)
                assert cert < tol, (tol, c, cert)
                assert abs(relres[c] - cert) <= 1e-3 * tol + 1e-6 * cert
                assert np.all(xs[c][m.fixed_dof == 1] == 0.0)
                if tol == 1e-12:
                    x_ref = spla.spsolve(A.tocsc(), bf)
                    assert np.linalg.norm(xf - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
                assert 0 < iters[c] < 2000
    finally:
        fem.fem_mesh_destroy(h)


def test_pcg_iterations_match_oracle(torch_dev):
    """Same algorithm, same start: FP64 iteration counts agree with the oracle's Algorithm 1."""
    torch = torch_dev
    m, tp, sysm, A, bs = _setup((8, 7, 6), 4, seed=5)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    h = fem.fem_mesh_create(m, tp)
    try:
        b = torch.tensor(from_cases(bs, m.n_nodes, 4), device="cuda")
        x = torch.zeros_like(b)
        st, iters, relres = fem.pcg_solve(h, b, x, 4, fem.fem_opts_default(tol=1e-8, check_every=1))
        for c in range(4):
            res = oracle.block_jacobi_cg(A, Binv, bs[c][sysm.free], np.zeros(sysm.free.size), eps=1e-8)
            assert abs(int(iters[c]) - res.iters) <= 1, (iters[c], res.iters)
    finally:
        fem.fem_mesh_destroy(h)


def test_pcg_edge_cases(torch_dev):
    torch = torch_dev
    m, tp, sysm, A, bs = _setup((5, 4, 3), 4, seed=9)
    h = fem.fem_mesh_create(m, tp)
    try:
        # zero right-hand side for some cases: x = 0, 0 iterations (guess ignored)
        bs[1][:] = 0.0
        bs[3][:] = 0.0
        b = torch.tensor(from_cases(bs, m.n_nodes, 4), device="cuda")
        x = torch.ones_like(b)
        st, iters, relres = fem.pcg_solve(h, b, x, 4, fem.fem_opts_default())
        xs = to_cases(x.cpu().numpy(), m.n_nodes, 4)
        assert iters[1] == 0 and iters[3] == 0
        assert np.all(xs[1] == 0.0) and np.all(xs[3] == 0.0)
        assert iters[0] > 0 and relres[0] < 1e-8
        # exact guess: no iterations
        x2 = x.clone()
        st, iters2, _ = fem.pcg_solve(h, b, x2, 4, fem.fem_opts_default(tol=1e-6))
        assert iters2[0] == 0
        # iteration limit reported
        x3 = torch.zeros_like(b)
        st, it3, rr3 = fem.pcg_solve(h, b, x3, 4, fem.fem_opts_default(maxit=2), raise_on_error=False)
        assert st == fem.FEM_ERR_NOT_CONVERGED
        st, it4, rr4 = fem.pcg_solve(h, b, torch.zeros_like(b), 4,
                                     fem.fem_opts_default(maxit=2, precision=fem.FEM_FP32_INNER),
                                     raise_on_error=False)
        assert st == fem.FEM_ERR_NOT_CONVERGED
        with pytest.raises(fem.FemError):
            fem.pcg_solve(h, b, x, 4, fem.fem_opts_default(tol=-1.0))
    finally:
        fem.fem_mesh_destroy(h)
