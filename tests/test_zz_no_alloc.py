"""The allocation-free EBE entry point (fem_ebe_apply_noalloc) against the allocating one.

Callers that cannot allocate device memory (memory owned by another allocator under a fixed budget, or
loops that cannot take cudaMalloc's synchronisation) use fem_ebe_apply_noalloc, whose reduction scratch is
a fixed array inside the library.  Its products and p^T q values must equal fem_ebe_apply's within the
tolerances of the EBE parity tests (FP64: 1e-13 relative; FP32: 2e-6), on two calls in a row (the
second call reuses the scratch the first one left behind).  The entry point is called on a fresh mesh
before any allocating entry point touches that mesh, and the device's free memory must not drop across
those calls.  This file is named to be collected last."""
import numpy as np
import pytest

from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import from_cases, random_free_vectors, small_mesh

pytestmark = pytest.mark.gpu


def _coeffs():
    tp = wl.TimeParams()
    return tp, 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt, 1.0 + 2.0 * tp.a1 / tp.dt


def _warm_up_scratch(torch):
    """One call on a throw-away mesh: the one-time per-device set-up (the scratch's address, loading the
    kernels) happens here, so later calls can be checked for allocations."""
    tp, cM, cK = _coeffs()
    m = small_mesh(3, 3, 3)
    h = fem.fem_mesh_create(m, tp)
    try:
        for dt in (torch.float64, torch.float32):
            p = torch.zeros(m.n_nodes * 3, device="cuda", dtype=dt)
            q = torch.empty_like(p)
            ptq = torch.zeros(1, dtype=torch.float64, device="cuda")
            fem.fem_ebe_apply_noalloc(h, p, q, 1, cM, cK, ptq)
            fem.fem_ebe_apply_noalloc(h, p, q, 1, cM, cK, None)
        torch.cuda.synchronize()
    finally:
        fem.fem_mesh_destroy(h)


@pytest.mark.parametrize("dtype_name,tol,r,with_ptq", [("float64", 1e-13, 16, True), ("float32", 2e-6, 16, True),
                                                       ("float64", 1e-13, 1, True), ("float32", 2e-6, 1, True),
                                                       ("float32", 2e-6, 8, False)])
def test_noalloc_matches_allocating_entry_point(dtype_name, tol, r, with_ptq):
    import torch
    build.build()
    fem.lib()
    dtype = getattr(torch, dtype_name)
    _warm_up_scratch(torch)
    tp, cM, cK = _coeffs()
    m = small_mesh(9, 6, 5, perturb=0.1)
    h = fem.fem_mesh_create(m, tp)
    try:
        # inputs and outputs of both calls, allocated up front (by the caller, as the entry point expects)
        ps = [torch.tensor(from_cases(random_free_vectors(m, r, seed=100 + k), m.n_nodes, r), device="cuda",
                           dtype=dtype) for k in range(2)]
        qs = [torch.full_like(ps[0], 3.0) for _ in range(2)]
        ptqs = [torch.full((r,), -1.0, dtype=torch.float64, device="cuda") if with_ptq else None for _ in range(2)]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for k in range(2):    # two calls in a row on the fresh mesh, before any allocating entry point
            fem.fem_ebe_apply_noalloc(h, ps[k], qs[k], r, cM, cK, ptqs[k])
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 >= free0, f"device free memory dropped by {free0 - free1} bytes"
        assert fem.fem_last_error() == ""
        for k in range(2):
            q_ref = torch.empty_like(ps[k])
            ptq_ref = torch.zeros(r, dtype=torch.float64, device="cuda")
            fem.fem_ebe_apply(h, ps[k], q_ref, r, cM, cK, ptq_ref)
            torch.cuda.synchronize()
            qa, qb = qs[k].double().cpu().numpy(), q_ref.double().cpu().numpy()
            assert np.abs(qa - qb).max() <= tol * np.abs(qb).max(), k
            if with_ptq:
                pa, pb = ptqs[k].cpu().numpy(), ptq_ref.cpu().numpy()
                assert np.all(np.abs(pa - pb) <= tol * np.abs(pb)), (k, pa, pb)
        with pytest.raises(fem.FemError) as ei:
            fem.fem_ebe_apply_noalloc(h, ps[0], qs[0], 64, cM, cK, ptqs[0])
        assert ei.value.status == fem.FEM_ERR_ARG
        # a successful call clears the message the failed one left
        fem.fem_ebe_apply_noalloc(h, ps[0], qs[0], r, cM, cK, ptqs[0])
        assert fem.fem_last_error() == ""
    finally:
        fem.fem_mesh_destroy(h)
