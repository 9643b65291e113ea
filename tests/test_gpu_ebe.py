"""EBE product on the GPU (Section 3.2, Eq. eqebefem / eqmebefem) against the oracle's assembled CSR
matrices, element by element of the output, for 1..32 interleaved cases, FP64 and FP32 element data.

Tolerances: FP64 results differ from the CSR product only by summation order (relative 1e-13 of the
vector norm); FP32 element records and arithmetic give ~1e-7 relative per entry, bounded here by 2e-6."""
import numpy as np
import pytest

import oracle
from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import from_cases, random_free_vectors, small_mesh, to_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    build.build()
    fem.lib()
    assert torch.cuda.is_available()
    return torch


CASES = [((7, 5, 4), 1, 0.0), ((7, 5, 4), 4, 0.2), ((9, 6, 5), 16, 0.1), ((3, 2, 2), 32, 0.0), ((12, 9, 7), 8, 0.15)]
# (ebe_variant, hex_per_tile): generic element kernel; tiled hex kernel and staged tiled hex kernel with
# automatic and small tiles (140..756 hexes over 64-hex tiles: several tiles and a ragged last one); 7 (hex
# element matrices) applies to FP32 products with the mesh's coefficients and falls back to 5 (then 3) else;
# 8 is the assembled 3x3-block (CRS-style) product
VARIANTS = [(1, 0), (2, 0), (2, 64), (3, 0), (3, 64), (4, 0), (4, 64), (5, 0), (5, 64), (6, 0), (6, 64), (7, 0),
            (7, 64), (8, 0)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dims,r,perturb", CASES)
@pytest.mark.parametrize("coef", ["A", "M", "K"])
def test_ebe_fp64_matches_csr(torch_dev, dims, r, perturb, coef, variant):
    torch = torch_dev
    m = small_mesh(*dims, perturb=perturb)
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    aM, aK, ref_mat = {"A": (cM, cK, sysm.A_full), "M": (1.0, 0.0, sysm.M), "K": (0.0, 1.0, sysm.K)}[coef]
    h = fem.fem_mesh_create(m, tp)
    try:
        assert fem.fem_mesh_info(h)["has_hex_patches"] == 1
        fem.fem_mesh_tune(h, *variant)
        ps = random_free_vectors(m, r, seed=r)
        p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda")
        q = torch.full_like(p, 7.0)                      # stale contents must be overwritten
        ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
        fem.fem_ebe_apply(h, p, q, r, aM, aK, ptq)
        torch.cuda.synchronize()
        qs = to_cases(q.cpu().numpy(), m.n_nodes, r)
        fixed = m.fixed_dof == 1
        for c in range(r):
            ref = ref_mat @ ps[c]
            ref[fixed] = 0.0
            assert np.all(qs[c][fixed] == 0.0)
            err = np.abs(qs[c] - ref).max() / np.abs(ref).max()
            assert err < 1e-13, (c, err)
            d_ref = ps[c] @ (ref_mat @ ps[c])
            assert abs(ptq[c].item() - d_ref) <= 1e-13 * abs(d_ref)
    finally:
        fem.fem_mesh_destroy(h)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("dims,r,perturb", CASES)
def test_ebe_fp32_matches_csr(torch_dev, dims, r, perturb, variant):
    torch = torch_dev
    m = small_mesh(*dims, perturb=perturb)
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    h = fem.fem_mesh_create(m, tp)
    try:
        fem.fem_mesh_tune(h, *variant)
        ps = random_free_vectors(m, r, seed=3 * r)
        p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda", dtype=torch.float32)
        q = torch.empty_like(p)
        ptq = torch.zeros(r, dtype=torch.float64, device="cuda")
        fem.fem_ebe_apply(h, p, q, r, cM, cK, ptq)
        torch.cuda.synchronize()
        qs = to_cases(q.cpu().double().numpy(), m.n_nodes, r)
        p32 = [x.astype(np.float32).astype(np.float64) for x in ps]
        for c in range(r):
            ref = sysm.A_full @ p32[c]
            ref[m.fixed_dof == 1] = 0.0
            err = np.abs(qs[c] - ref).max() / np.abs(ref).max()
            assert err < 2e-6, (c, err)
            d_ref = p32[c] @ (sysm.A_full @ p32[c])
            assert abs(ptq[c].item() - d_ref) <= 2e-6 * abs(d_ref)
    finally:
        fem.fem_mesh_destroy(h)


def test_ebe_edge_cases(torch_dev):
    torch = torch_dev
    m = small_mesh(2, 2, 1)
    tp = wl.TimeParams()
    h = fem.fem_mesh_create(m, tp)
    try:
        p = torch.zeros(m.n_nodes * 3 * 4, dtype=torch.float64, device="cuda")
        q = torch.ones_like(p)
        fem.fem_ebe_apply(h, p, q, 4, 1.0, 1.0)
        torch.cuda.synchronize()
        assert torch.count_nonzero(q).item() == 0
        with pytest.raises(fem.FemError) as ei:
            fem.fem_ebe_apply(h, p, q, 3, 1.0, 1.0)
        assert ei.value.status == fem.FEM_ERR_ARG
    finally:
        fem.fem_mesh_destroy(h)
    # invalid meshes are rejected with an argument error
    bad = small_mesh(2, 2, 1)
    bad.conn = bad.conn.copy()
    bad.conn[0, [2, 3]] = bad.conn[0, [3, 2]]              # negative orientation
    with pytest.raises(fem.FemError) as ei:
        fem.fem_mesh_create(bad, tp)
    assert ei.value.status == fem.FEM_ERR_ARG
    bad2 = small_mesh(2, 2, 1)
    bad2.conn = bad2.conn.copy()
    bad2.conn[5, 1] = bad2.n_nodes                        # node id out of range
    with pytest.raises(fem.FemError):
        fem.fem_mesh_create(bad2, tp)


def test_ebe_mesh_without_hex_patches(torch_dev):
    """Elements in shuffled order do not form hex patches: the generic kernel serves, with the same result."""
    torch = torch_dev
    m = small_mesh(6, 5, 4, perturb=0.1)
    perm = np.random.default_rng(0).permutation(m.n_elems)
    m.conn = np.ascontiguousarray(m.conn[perm])
    m.mat_id = np.ascontiguousarray(m.mat_id[perm])
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    h = fem.fem_mesh_create(m, tp)
    try:
        assert fem.fem_mesh_info(h)["has_hex_patches"] == 0
        with pytest.raises(fem.FemError):
            fem.fem_mesh_tune(h, 2, 0)
        ps = random_free_vectors(m, 4, seed=1)
        p = torch.tensor(from_cases(ps, m.n_nodes, 4), device="cuda")
        for variant in (0, 8):      # generic element kernel; assembled blocks (any mesh)
            fem.fem_mesh_tune(h, variant, 0)
            q = torch.empty_like(p)
            fem.fem_ebe_apply(h, p, q, 4, 1.0, 1.0)
            torch.cuda.synchronize()
            qs = to_cases(q.cpu().numpy(), m.n_nodes, 4)
            for c in range(4):
                ref = (sysm.M + sysm.K) @ ps[c]
                ref[m.fixed_dof == 1] = 0.0
                assert np.abs(qs[c] - ref).max() <= 1e-13 * np.abs(ref).max(), variant
    finally:
        fem.fem_mesh_destroy(h)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("r", [1, 8, 32])
def test_autotuned_product_matches_csr(torch_dev, precision, r):
    """The autotuner picks one of the implementations, and the product it selects keeps parity."""
    torch = torch_dev
    m = small_mesh(12, 9, 7, perturb=0.1)
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    h = fem.fem_mesh_create(m, tp)
    try:
        prec = fem.FEM_FP32_INNER if precision == "fp32" else fem.FEM_FP64
        v, hpt, ms = fem.fem_mesh_autotune(h, prec, r)
        assert (v, hpt) in [(1, 0), (2, 64), (2, 128), (2, 256), (2, 512), (3, 64), (3, 128), (3, 256), (4, 64),
                            (4, 128), (5, 64), (5, 128), (6, 64), (6, 128), (6, 256), (7, 64), (8, 0)] and ms > 0
        dt = torch.float32 if precision == "fp32" else torch.float64
        ps = random_free_vectors(m, r, seed=5 + r)
        p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda", dtype=dt)
        q = torch.empty_like(p)
        fem.fem_ebe_apply(h, p, q, r, cM, cK)
        torch.cuda.synchronize()
        qs = to_cases(q.cpu().double().numpy(), m.n_nodes, r)
        pr = [x.astype(np.float32).astype(np.float64) for x in ps] if precision == "fp32" else ps
        tol = 2e-6 if precision == "fp32" else 1e-13
        for c in range(r):
            ref = sysm.A_full @ pr[c]
            ref[m.fixed_dof == 1] = 0.0
            assert np.abs(qs[c] - ref).max() / np.abs(ref).max() < tol
    finally:
        fem.fem_mesh_destroy(h)
