"""Tet10 EBE product on the GPU (the paper's element, Section 3.1; Eq. eqebefem with 30 x 30 element
operators formed on the fly) against the tet10 oracle's assembled CSR matrices, element by element of the
output, for 1..32 interleaved cases, FP64 and FP32.

Tolerances: FP64 differs from the CSR product only by summation order (1e-13 of the vector's largest
entry); FP32 records and arithmetic give ~1e-7 relative per entry, bounded here by 5e-6 (the tet10
operator's entries span a wider range than the tet4 ones: edge/corner couplings of both signs)."""
import numpy as np
import pytest

from oracle import tet10_oracle as t10
from paper_2409_20380_gb300 import fem
from paper_2409_20380_gb300 import workload as wl
from helpers import from_cases, random_free_vectors, small_mesh, to_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2409_20380_gb300 import build
    build.build()
    fem.lib()
    assert torch.cuda.is_available()
    return torch


CASES = [((3, 2, 2), 1, 0.0), ((5, 4, 3), 4, 0.2), ((6, 5, 4), 16, 0.1), ((2, 2, 1), 32, 0.0)]


@pytest.mark.parametrize("dims,r,perturb", CASES)
@pytest.mark.parametrize("coef", ["A", "M", "K"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ebe10_matches_csr(torch_dev, dims, r, perturb, coef, precision):
    torch = torch_dev
    m10 = wl.tet10_mesh(small_mesh(*dims, perturb=perturb))
    K, M = t10.assemble10(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    tp = wl.TimeParams()
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    aM, aK = {"A": (cM, cK), "M": (1.0, 0.0), "K": (0.0, 1.0)}[coef]
    ref_mat = aM * M + aK * K
    h = fem.fem_mesh10_create(m10)
    try:
        dt = torch.float64 if precision == "fp64" else torch.float32
        ps = random_free_vectors(m10, r, seed=11 + r)
        if precision == "fp32":
            ps = [x.astype(np.float32).astype(np.float64) for x in ps]
        p = torch.tensor(from_cases(ps, m10.n_nodes, r), device="cuda", dtype=dt)
        q = torch.full_like(p, 5.0)                      # stale contents must be overwritten
        ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
        fem.fem_ebe10_apply(h, p, q, r, aM, aK, ptq)
        torch.cuda.synchronize()
        qs = to_cases(q.cpu().double().numpy(), m10.n_nodes, r)
        fixed = m10.fixed_dof == 1
        tol = 1e-13 if precision == "fp64" else 5e-6
        for c in range(r):
            ref = ref_mat @ ps[c]
            ref[fixed] = 0.0
            assert np.all(qs[c][fixed] == 0.0)
            err = np.abs(qs[c] - ref).max() / np.abs(ref).max()
            assert err < tol, (c, err)
            d_ref = ps[c] @ (ref_mat @ ps[c])
            assert abs(ptq[c].item() - d_ref) <= tol * abs(d_ref)
    finally:
        fem.fem_mesh10_destroy(h)


def test_ebe10_argument_errors(torch_dev):
    torch = torch_dev
    m10 = wl.tet10_mesh(small_mesh(2, 2, 1))
    bad = wl.Mesh10(m10.xyz, m10.conn.copy(), m10.mat_id, m10.lam_mu_rho, m10.fixed_dof)
    bad.conn[0, 5] = m10.n_nodes                         # node id out of range
    with pytest.raises(fem.FemError) as ei:
        fem.fem_mesh10_create(bad)
    assert ei.value.status == fem.FEM_ERR_ARG
    h = fem.fem_mesh10_create(m10)
    try:
        p = torch.zeros(m10.n_nodes * 3 * 3, dtype=torch.float64, device="cuda")
        with pytest.raises(fem.FemError) as ei:
            fem.fem_ebe10_apply(h, p, p.clone(), 3, 1.0, 1.0)   # n_rhs not a power of two
        assert ei.value.status == fem.FEM_ERR_ARG
    finally:
        fem.fem_mesh10_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dims,r", [((3, 3, 2), 1), ((4, 3, 3), 4)])
def test_pcg10_matches_direct_solve_and_oracle_iterations(torch_dev, dims, r, precision):
    """The tet10 PCG (Algorithm 1 with 3x3 block Jacobi) against a sparse direct solve of the oracle's
    reduced system; in FP64 also against the oracle's literal Algorithm 1 (iteration counts within one);
    FP32-inner / FP64-refined to the same certified tolerance."""
    import scipy.sparse.linalg as spla
    import oracle
    torch = torch_dev
    m10 = wl.tet10_mesh(small_mesh(*dims, perturb=0.15))
    K, M = t10.assemble10(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    tp = wl.TimeParams()
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    A = (cM * M + cK * K).tocsr()
    free = np.nonzero(m10.fixed_dof == 0)[0]
    A_red = A[free][:, free].tocsr()
    Binv = oracle.block_jacobi_inverse(A_red, free)
    bs = random_free_vectors(m10, r, seed=21 + r)
    h = fem.fem_mesh10_create(m10)
    try:
        b = torch.tensor(from_cases(bs, m10.n_nodes, r), device="cuda")
        x = torch.zeros_like(b)
        tol = 1e-10
        prec = fem.FEM_FP64 if precision == "fp64" else fem.FEM_FP32_INNER
        iters, relres = fem.pcg10_solve(h, b, x, r, cM, cK, tol=tol, precision=prec)
        xs = to_cases(x.cpu().numpy(), m10.n_nodes, r)
        for c in range(r):
            ref = spla.spsolve(A_red.tocsc(), bs[c][free])
            assert np.abs(xs[c][free] - ref).max() <= 1e-8 * np.abs(ref).max()
            assert np.all(xs[c][m10.fixed_dof == 1] == 0.0)
            true_rel = np.linalg.norm(bs[c][free] - A_red @ xs[c][free]) / np.linalg.norm(bs[c][free])
            assert true_rel < tol and relres[c] < tol
            if precision == "fp64":
                res = oracle.block_jacobi_cg(A_red, Binv, bs[c][free], np.zeros(free.size), eps=tol)
                assert abs(int(iters[c]) - res.iters) <= 1, (iters[c], res.iters)
    finally:
        fem.fem_mesh10_destroy(h)
