"""The allocation-free EBE entry point (fem_ebe_apply_noalloc) against the allocating one.

Callers that cannot allocate device memory (memory owned by another allocator under a fixed budget, or
loops that cannot take cudaMalloc's synchronisation) use fem_ebe_apply_noalloc, whose reduction scratch is
a fixed array inside the library.  Its products and p^T q values must equal fem_ebe_apply's within the
tolerances of the EBE parity tests (FP64: 1e-13 relative; FP32: 2e-6), on two calls in a row (the
second call reuses the scratch the first one left behind).  This file is named to be collected last."""
import numpy as np
import pytest

from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import from_cases, random_free_vectors, small_mesh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype_name,tol,r", [("float64", 1e-13, 16), ("float32", 2e-6, 16), ("float64", 1e-13, 1)])
def test_noalloc_matches_allocating_entry_point(dtype_name, tol, r):
    import torch
    build.build()
    fem.lib()
    dtype = getattr(torch, dtype_name)
    m = small_mesh(9, 6, 5, perturb=0.1)
    tp = wl.TimeParams()
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    h = fem.fem_mesh_create(m, tp)
    try:
        for call in range(2):
            ps = random_free_vectors(m, r, seed=100 + call)
            p = torch.tensor(from_cases(ps, m.n_nodes, r), device="cuda", dtype=dtype)
            q_ref = torch.empty_like(p)
            ptq_ref = torch.zeros(r, dtype=torch.float64, device="cuda")
            fem.fem_ebe_apply(h, p, q_ref, r, cM, cK, ptq_ref)
            q = torch.full_like(p, 3.0)
            ptq = torch.full((r,), -1.0, dtype=torch.float64, device="cuda")
            fem.fem_ebe_apply_noalloc(h, p, q, r, cM, cK, ptq)
            torch.cuda.synchronize()
            qa, qb = q.double().cpu().numpy(), q_ref.double().cpu().numpy()
            assert np.abs(qa - qb).max() <= tol * np.abs(qb).max(), call
            pa, pb = ptq.cpu().numpy(), ptq_ref.cpu().numpy()
            assert np.all(np.abs(pa - pb) <= tol * np.abs(pb)), (call, pa, pb)
        with pytest.raises(fem.FemError) as ei:
            fem.fem_ebe_apply_noalloc(h, p, q, 64, cM, cK, ptq)
        assert ei.value.status == fem.FEM_ERR_ARG
    finally:
        fem.fem_mesh_destroy(h)
