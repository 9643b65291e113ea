"""The time-stepping solver on 10-node tetrahedra, the paper's element (Section 3.1), against the oracle.

The oracle's system is assembled from its own tet10 element matrices (exact integration, oracle/
tet10_oracle.py); its Newmark right-hand side, certification, update and predictors are the same functions
the linear-tet step tests use (Section 3.1, Algorithm 1, Section 3.2), so every GPU step is checked as there:
b to 1e-12, the increment certified with the oracle's CSR A, the Newmark update to rounding, and the
predictor from the GPU's own history.  The products of a tet10 mesh (the element kernel in FP64 and FP32,
the FP64 split products and the assembled blocks of the certification) are checked against the oracle's
CSR matrices directly."""
import numpy as np
import pytest

import oracle
from oracle import tet10_oracle as t10
from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import from_cases, random_free_vectors, small_mesh, to_cases
from test_gpu_step import _run_and_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    build.build()
    fem.lib()
    return torch


def tet10_system(m10, tp):
    """(System, reduced A) of a tet10 mesh from the oracle's tet10 assembly."""
    K, M = t10.assemble10(m10.xyz, m10.conn, m10.mat_id, m10.lam_mu_rho)
    free = np.nonzero(m10.fixed_dof == 0)[0]
    sysm = oracle.System(M=M.tocsr(), K=K.tocsr(), free=free, dt=tp.dt, a0=tp.a0, a1=tp.a1)
    return sysm, sysm.reduce(sysm.A_full)


def tet10_case(dims, perturb=0.0, n_cases=2, seed=0):
    m4 = small_mesh(*dims, perturb=perturb)
    m10, new_id = wl.tet10_mesh_ordered(m4)
    srcs = []
    for c in range(n_cases):
        s = wl.random_source(m4, wl.rng_for(9, seed, c), f0=5.0)
        s.node = int(new_id[s.node])
        srcs.append(s)
    return m4, m10, srcs


@pytest.mark.parametrize("dims,r,perturb", [((3, 3, 2), 1, 0.0), ((4, 3, 3), 4, 0.15), ((5, 4, 3), 8, 0.1)])
def test_tet10_mesh_products_match_csr(torch_dev, dims, r, perturb):
    """fem_ebe_apply (FP64 and FP32, both product forms), fem_mesh_split_product (all four forms) and
    fem_ebe_apply_noalloc on a fem_mesh_create_tet10 mesh against the oracle's CSR M and K."""
    torch = torch_dev
    m4 = small_mesh(*dims, perturb=perturb)
    m10, _ = wl.tet10_mesh_ordered(m4)
    tp = wl.TimeParams()
    sysm, _ = tet10_system(m10, tp)
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    h = fem.fem_mesh_create_tet10(m10, tp)
    fixed = m10.fixed_dof == 1
    try:
        ps = random_free_vectors(m10, r, seed=5 + r)
        p64 = torch.tensor(from_cases(ps, m10.n_nodes, r), device="cuda")
        ps32 = [x.astype(np.float32).astype(np.float64) for x in ps]
        p32 = torch.tensor(from_cases(ps32, m10.n_nodes, r), device="cuda", dtype=torch.float32)
        for variant in (0, 8):
            fem.fem_mesh_tune(h, variant, 0)
            for prec, p, vs, tol in ((fem.FEM_FP64, p64, ps, 1e-13), (fem.FEM_FP32_INNER, p32, ps32, 5e-6)):
                q = torch.full_like(p, 7.0)
                ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
                fem.fem_ebe_apply(h, p, q, r, cM, cK, ptq, precision=prec)
                torch.cuda.synchronize()
                qs = to_cases(q.cpu().double().numpy(), m10.n_nodes, r)
                for c in range(r):
                    ref = (cM * sysm.M + cK * sysm.K) @ vs[c]
                    ref[fixed] = 0.0
                    err = np.abs(qs[c] - ref).max() / np.abs(ref).max()
                    assert err < tol, (variant, prec, c, err)
                    assert abs(ptq[c].item() - vs[c] @ ref) <= 10 * tol * abs(vs[c]) @ abs(ref), (variant, prec, c)
        fem.fem_mesh_tune(h, 0, 0)
        for mode in (0, 1, 2, 3):
            qM, qK = torch.full_like(p64, 3.0), torch.full_like(p64, 3.0)
            fem.fem_mesh_split_product(h, mode, p64, qM, qK, r)
            torch.cuda.synchronize()
            gM = to_cases(qM.cpu().numpy(), m10.n_nodes, r)
            gK = to_cases(qK.cpu().numpy(), m10.n_nodes, r)
            tol = 1e-13 if mode in (0, 1, 2) else 1e-12
            for c in range(r):
                for got, mat in ((gM[c], sysm.M), (gK[c], sysm.K)):
                    ref = mat @ ps[c]
                    ref[fixed] = 0.0
                    assert np.all(got[fixed] == 0.0)
                    assert np.abs(got - ref).max() / np.abs(ref).max() < tol, (mode, c)
        q = torch.full_like(p64, 7.0)
        ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
        fem.fem_ebe_apply_noalloc(h, p64, q, r, cM, cK, ptq)
        torch.cuda.synchronize()
        qs = to_cases(q.cpu().numpy(), m10.n_nodes, r)
        for c in range(r):
            ref = (cM * sysm.M + cK * sysm.K) @ ps[c]
            ref[fixed] = 0.0
            assert np.abs(qs[c] - ref).max() / np.abs(ref).max() < 1e-13
            assert abs(ptq[c].item() - ps[c] @ ref) <= 1e-12 * abs(ps[c]) @ abs(ref)
    finally:
        fem.fem_mesh_destroy(h)


@pytest.mark.parametrize("precision,predictor,graph", [("fp64", "ab4", 0), ("fp64", "dd", 0),
                                                       ("mixed", "dd", 0), ("mixed", "dd", 1)])
def test_step10_matches_oracle(torch_dev, precision, predictor, graph):
    """25 steps of 2 cases on a 4x3x3-hex box split into 10-node tets (perturbed nodes), every step checked
    against the oracle; with the data-driven predictor (s = 8, regions of 48 nodes) the prediction is
    recomputed from the GPU's own history and checked too."""
    m4, m10, srcs = tet10_case((4, 3, 3), perturb=0.1)
    tp = wl.TimeParams()
    system = tet10_system(m10, tp)
    opts = fem.fem_opts_default(precision=fem.FEM_FP64 if precision == "fp64" else fem.FEM_FP32_INNER,
                                predictor=fem.FEM_PRED_AB4 if predictor == "ab4" else fem.FEM_PRED_DD, s_max=8,
                                tol=1e-8, use_graph=graph)
    regions = wl.region_map10(m10, m4.h, 48) if predictor == "dd" else None
    iters, stats = _run_and_check(m10, tp, srcs, opts, 25, system=system, create=fem.fem_mesh_create_tet10,
                                  regions=regions)
    assert np.all(iters > 0)


def test_step10_dd_reduces_iterations(torch_dev):
    """On quadratic tets as on linear ones the data-driven correction (Section 3.2) takes fewer CG iterations
    than Adams-Bashforth alone over the same 60 certified steps."""
    m4, m10, srcs = tet10_case((5, 4, 3), n_cases=2, seed=1)
    tp = wl.TimeParams()
    its = {}
    for pred in (fem.FEM_PRED_AB4, fem.FEM_PRED_DD):
        h = fem.fem_mesh_create_tet10(m10, tp)
        fem.fem_mesh_set_regions(h, wl.region_map10(m10, m4.h, 64))
        bt = fem.fem_batch_create(fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=pred, s_max=8,
                                                       tol=1e-8))
        try:
            for s in srcs:
                fem.fem_case_add(bt, h, s)
            st, it, rr = fem.fem_step(bt, 60, len(srcs))
            assert st == fem.FEM_OK and np.all(rr < 1e-8)
            its[pred] = int(it.sum())
        finally:
            fem.fem_batch_destroy(bt)
            fem.fem_mesh_destroy(h)
    assert its[fem.FEM_PRED_DD] < its[fem.FEM_PRED_AB4], its


def test_tet10_mesh_rejects_linear_only_features(torch_dev):
    m4, m10, _ = tet10_case((3, 3, 2))
    tp = wl.TimeParams()
    h = fem.fem_mesh_create_tet10(m10, tp)
    try:
        for call in (lambda: fem.fem_mesh_tune(h, 5, 0),
                     lambda: fem.fem_mesh_autotune(h, fem.FEM_FP32_INNER, 4),
                     lambda: fem.fem_mesh_set_absorbing(h, np.array([[0, 1, 2]], dtype=np.int32))):
            with pytest.raises(fem.FemError) as ei:
                call()
            assert ei.value.status == fem.FEM_ERR_ARG
    finally:
        fem.fem_mesh_destroy(h)
