"""Variant 9: the FP32 product with per-hex element matrices in FP16 on the tensor cores (the element data in
reduced precision, form 1 of the mixed-precision solver), against the oracle's assembled CSR matrices.

Tolerance: the hex matrix entries and the scaled inputs are rounded to FP16 (relative 2^-11 each) and the
products accumulate in FP32, so an output row differs from the exact row by at most ~2 x 2^-11 of the row's
sum of absolute terms (|A| |p|)_i; bounded here by 2e-3 of it.  The same rows must differ from the exact
ones by more than FP32 rounding somewhere (1e-6), which shows that the FP16 path ran.  Products it does not
apply to (other case counts, coefficients other than the mesh's, FP64) fall back to the FP32 / FP64 kernels
and keep their tolerances.  Steps with the FP16 inner product stay certified below tol by the oracle's CSR A."""
import numpy as np
import pytest

import oracle
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


def _coefs(tp):
    return 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt, 1.0 + 2.0 * tp.a1 / tp.dt


# (dims, cases, perturbation): 8 and 16 cases; boxes of 12 .. 756 hexes (one and many 64-hex tiles, a
# ragged last tile), straight and perturbed geometry
TC_CASES = [((7, 5, 4), 8, 0.2), ((9, 6, 5), 16, 0.1), ((3, 2, 2), 16, 0.0), ((12, 9, 7), 8, 0.15),
            ((4, 4, 4), 8, 0.0)]


@pytest.mark.parametrize("dims,r,perturb", TC_CASES)
def test_tc_product_matches_csr(torch_dev, dims, r, perturb):
    torch = torch_dev
    m = small_mesh(*dims, perturb=perturb)
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    cM, cK = _coefs(tp)
    A = cM * sysm.M + cK * sysm.K
    absA = abs(A)
    h = fem.fem_mesh_create(m, tp)
    try:
        fem.fem_mesh_tune(h, 9, 0)
        ps = random_free_vectors(m, r, seed=40 + r)
        ps = [x.astype(np.float32).astype(np.float64) for x in ps]
        p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda", dtype=torch.float32)
        q = torch.full_like(p, 7.0)
        ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
        fem.fem_ebe_apply(h, p, q, r, cM, cK, ptq)
        torch.cuda.synchronize()
        qs = to_cases(q.cpu().double().numpy(), m.n_nodes, r)
        fixed = m.fixed_dof == 1
        worst = 0.0
        for c in range(r):
            ref = A @ ps[c]
            ref[fixed] = 0.0
            assert np.all(qs[c][fixed] == 0.0)
            scale = absA @ np.abs(ps[c]) + 1e-300
            err = np.abs(qs[c] - ref)[~fixed] / scale[~fixed]
            assert err.max() < 2e-3, (c, err.max())
            worst = max(worst, err.max())
            own = float(ps[c] @ qs[c])                 # p^T q of the product's own output
            assert abs(ptq[c].item() - own) <= 1e-5 * abs(own), (c, ptq[c].item(), own)
            exact = float(ps[c] @ (A @ ps[c]))
            assert abs(ptq[c].item() - exact) <= 2e-3 * float(np.abs(ps[c]) @ (absA @ np.abs(ps[c])))
        assert worst > 1e-6, worst                    # FP16 rounding visible: the tensor-core path ran
    finally:
        fem.fem_mesh_destroy(h)


@pytest.mark.parametrize("r,coef,prec", [(4, "A", "fp32"), (32, "A", "fp32"), (8, "M", "fp32"), (8, "A", "fp64")])
def test_tc_falls_back_where_it_does_not_apply(torch_dev, r, coef, prec):
    """4 or 32 cases, coefficients other than the mesh's, or an FP64 product: the FP32 / FP64 kernels run
    with their own tolerances (2e-6, 1e-13 of the largest entry)."""
    torch = torch_dev
    m = small_mesh(7, 5, 4, perturb=0.1)
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    cM, cK = _coefs(tp)
    aM, aK, mat = (cM, cK, cM * sysm.M + cK * sysm.K) if coef == "A" else (1.0, 0.0, sysm.M)
    h = fem.fem_mesh_create(m, tp)
    try:
        fem.fem_mesh_tune(h, 9, 0)
        ps = random_free_vectors(m, r, seed=3)
        dt = torch.float32 if prec == "fp32" else torch.float64
        if prec == "fp32":
            ps = [x.astype(np.float32).astype(np.float64) for x in ps]
        p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda", dtype=dt)
        q = torch.full_like(p, 7.0)
        fem.fem_ebe_apply(h, p, q, r, aM, aK)
        torch.cuda.synchronize()
        qs = to_cases(q.cpu().double().numpy(), m.n_nodes, r)
        fixed = m.fixed_dof == 1
        tol = 2e-6 if prec == "fp32" else 1e-13
        for c in range(r):
            ref = mat @ ps[c]
            ref[fixed] = 0.0
            assert np.abs(qs[c] - ref).max() / np.abs(ref).max() < tol
    finally:
        fem.fem_mesh_destroy(h)


@pytest.mark.parametrize("graph", [0, 1])
def test_tc_inner_product_steps_certified(torch_dev, graph):
    """The benchmark's solver settings on a 16 x 16 x 12 box of the large recipe, 8 cases, with the inner CG
    products on the tensor cores: every step certified by the oracle's CSR A, the right-hand side, the
    Newmark update and the predictor checked as in the linear-tet step tests, and the CG iterations within
    15% of the FP32 inner product's on the same steps."""
    mesh = wl.config4_mesh(16, 16, 12)
    tp = wl.config4_time_params()
    srcs = wl.config4_sources(mesh, 8)
    its = {}
    for ip in (fem.FEM_INNER_FP32, fem.FEM_INNER_TC):
        opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16,
                                    cert_df=3, snapshot_format=2, use_graph=graph, inner_product=ip)
        it, _ = _run_and_check(mesh, tp, srcs, opts, 40, region_nodes=1024, b_tol=1e-11)
        its[ip] = int(it.sum())
    assert its[fem.FEM_INNER_TC] <= 1.15 * its[fem.FEM_INNER_FP32], its


def test_tc_inner_product_option_checked(torch_dev):
    with pytest.raises(fem.FemError) as ei:
        fem.fem_batch_create(fem.fem_opts_default(precision=fem.FEM_FP32_INNER, inner_product=2))
    assert ei.value.status == fem.FEM_ERR_ARG


def test_tc_pass_selection(torch_dev):
    """A refinement pass takes the FP16 products only when every active case asks its inner solve for a
    reduction of 1e-3 or less: from rest (the predictor not yet trained, initial residuals near 1) passes run
    the FP32 products, later ones the FP16 products (eager steps, where the profile tells the two apart; the
    predictor's correction product is the one FP32 product a step otherwise has)."""
    mesh = wl.config4_mesh(16, 16, 12)
    tp = wl.config4_time_params()
    srcs = wl.config4_sources(mesh, 8)
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16,
                                cert_df=3, snapshot_format=2, use_graph=0, inner_product=fem.FEM_INNER_TC)
    h = fem.fem_mesh_create(mesh, tp)
    fem.fem_mesh_set_regions(h, wl.region_map(mesh, 1024))
    bt = fem.fem_batch_create(opts)
    try:
        for s in srcs:
            fem.fem_case_add(bt, h, s)
        fem.fem_batch_profile(bt, 1)
        n = 60
        st, it, rel = fem.fem_step(bt, n, len(srcs))
        prof = fem.fem_batch_profile(bt, 0)
        assert np.all(rel < opts.tol)
        assert prof["ebe16_launches"] > 0, prof
        assert prof["ebe32_launches"] > n, prof
    finally:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)
