"""Split certification products M p and K p on the GPU against the oracle's assembled CSR matrices (Section
3.1, tet4 consistent mass and stiffness), for the four forms: element by element or assembled 3x3 blocks,
each in FP64 or in double-float arithmetic.  FP64 forms match to 1e-13 of the largest entry (summation
order only); double-float forms to 1e-12 (48-bit significands)."""
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
    return torch


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("dims,r,perturb,shuffle", [((7, 5, 4), 1, 0.0, False), ((9, 6, 5), 16, 0.15, False),
                                                    ((3, 2, 2), 32, 0.0, False), ((6, 5, 4), 4, 0.1, True),
                                                    ((5, 4, 3), 2, 0.1, False), ((8, 7, 6), 8, 0.1, False)])
def test_split_product_matches_csr(torch_dev, mode, dims, r, perturb, shuffle):
    torch = torch_dev
    m = small_mesh(*dims, perturb=perturb)
    if shuffle:      # elements in random order: no hex patches, pattern from arbitrary connectivity
        perm = np.random.default_rng(0).permutation(m.n_elems)
        m.conn = np.ascontiguousarray(m.conn[perm])
        m.mat_id = np.ascontiguousarray(m.mat_id[perm])
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    h = fem.fem_mesh_create(m, tp)
    try:
        ps = random_free_vectors(m, r, seed=7 + r)
        p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda")
        qM = torch.full_like(p, 3.0)
        qK = torch.full_like(p, 3.0)
        fem.fem_mesh_split_product(h, mode, p, qM, qK, r)
        torch.cuda.synchronize()
        gM = to_cases(qM.cpu().numpy(), m.n_nodes, r)
        gK = to_cases(qK.cpu().numpy(), m.n_nodes, r)
        tol = 1e-13 if mode in (0, 2) else 1e-12
        fixed = m.fixed_dof == 1
        for c in range(r):
            for got, mat in ((gM[c], sysm.M), (gK[c], sysm.K)):
                ref = mat @ ps[c]
                ref[fixed] = 0.0
                assert np.all(got[fixed] == 0.0)
                err = np.abs(got - ref).max() / np.abs(ref).max()
                assert err < tol, (mode, c, err)
    finally:
        fem.fem_mesh_destroy(h)


def test_split_product_rejects_bad_mode(torch_dev):
    torch = torch_dev
    m = small_mesh(2, 2, 1)
    h = fem.fem_mesh_create(m, wl.TimeParams())
    try:
        p = torch.zeros(m.n_nodes * 3, dtype=torch.float64, device="cuda")
        with pytest.raises(fem.FemError) as ei:
            fem.fem_mesh_split_product(h, 4, p, p.clone(), p.clone(), 1)
        assert ei.value.status == fem.FEM_ERR_ARG
    finally:
        fem.fem_mesh_destroy(h)


def test_split_product_double_float_wide_range(torch_dev):
    """Inputs spanning 1e-15 .. 1e10 (the double-float split is done by integer bit operations): the
    double-float assembled product matches the FP64 one to 1e-12 of the row's sum of absolute terms.  (FP32
    pairs carry 48 bits down to about 1e-31; values far below that lose relative accuracy.)"""
    torch = torch_dev
    m = small_mesh(6, 5, 4, perturb=0.1)
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    rng = np.random.default_rng(11)
    r = 4
    ps = []
    for c in range(r):
        v = rng.standard_normal(3 * m.n_nodes) * 10.0 ** rng.uniform(-15, 10, 3 * m.n_nodes)
        v[m.fixed_dof == 1] = 0.0
        ps.append(v)
    h = fem.fem_mesh_create(m, tp)
    try:
        p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda")
        out = {}
        for mode in (2, 3):
            qM, qK = torch.empty_like(p), torch.empty_like(p)
            fem.fem_mesh_split_product(h, mode, p, qM, qK, r)
            out[mode] = (to_cases(qM.cpu().numpy(), m.n_nodes, r), to_cases(qK.cpu().numpy(), m.n_nodes, r))
        absK = abs(sysm.K)
        absM = abs(sysm.M)
        for c in range(r):
            scaleK = absK @ np.abs(ps[c]) + 1e-300
            scaleM = absM @ np.abs(ps[c]) + 1e-300
            assert np.all(np.abs(out[3][1][c] - out[2][1][c]) <= 1e-12 * scaleK)
            assert np.all(np.abs(out[3][0][c] - out[2][0][c]) <= 1e-12 * scaleM)
    finally:
        fem.fem_mesh_destroy(h)


@pytest.mark.parametrize("r", [2, 8])
def test_split_product_unaligned_views(torch_dev, r):
    """Vectors that start 8 bytes past a 16-byte boundary (views into larger buffers): the double-float form
    that reads and writes case pairs with 16-byte accesses is not taken for them, and the result still matches
    the oracle's CSR to 1e-12."""
    torch = torch_dev
    m = small_mesh(6, 5, 4, perturb=0.1)
    tp = wl.TimeParams()
    sysm, _ = oracle.build_system(m, tp)
    h = fem.fem_mesh_create(m, tp)
    try:
        ps = random_free_vectors(m, r, seed=3 + r)
        n = m.n_nodes * 3 * r
        base = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        p = base[1:]
        p.copy_(torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda"))
        outs = torch.full((2, n + 1), 3.0, dtype=torch.float64, device="cuda")
        qM, qK = outs[0, 1:], outs[1, 1:]
        assert p.data_ptr() % 16 == 8 and qM.data_ptr() % 16 == 8
        fem.fem_mesh_split_product(h, 3, p, qM, qK, r)
        torch.cuda.synchronize()
        gM = to_cases(qM.cpu().numpy(), m.n_nodes, r)
        gK = to_cases(qK.cpu().numpy(), m.n_nodes, r)
        fixed = m.fixed_dof == 1
        for c in range(r):
            for got, mat in ((gM[c], sysm.M), (gK[c], sysm.K)):
                ref = mat @ ps[c]
                ref[fixed] = 0.0
                err = np.abs(got - ref).max() / np.abs(ref).max()
                assert err < 1e-12, (c, err)
    finally:
        fem.fem_mesh_destroy(h)
