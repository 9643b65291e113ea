"""The FEM_ERR_TIMEOUT path of the bounded device-side waits.

The staged EBE kernels wait for their bulk tile copies with a bounded number of tries (fem_opts.wait_budget);
a wait that gives up sets a flag the host reads after the work, and the call reports FEM_ERR_TIMEOUT.  The
kernel then still drains its copies with a second bounded wait, so the GPU context stays usable.  A budget
of 0 makes every wait that has not completed at its first check report, which exercises that path without
any fault: the next call with the default budget must run normally.
"""
import numpy as np
import pytest

from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import small_mesh

pytestmark = pytest.mark.gpu


def _batch(h, mesh, opts, n):
    bt = fem.fem_batch_create(opts)
    for c in range(n):
        fem.fem_case_add(bt, h, wl.random_source(mesh, wl.rng_for(77, 0, c), f0=6.0))
    return bt


@pytest.mark.parametrize("use_graph", [0, 1])
def test_zero_wait_budget_reports_timeout_then_recovers(use_graph):
    import torch
    build.build()
    fem.lib()
    mesh = small_mesh(8, 6, 5)
    tp = wl.TimeParams()
    h = fem.fem_mesh_create(mesh, tp)
    try:
        opts0 = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_AB4, wait_budget=0,
                                     use_graph=use_graph)
        bt = _batch(h, mesh, opts0, 4)
        with pytest.raises(fem.FemError) as ei:
            for _ in range(3):      # from rest the first steps may have b = 0 (no product launched)
                fem.fem_step(bt, 2, 4)
        assert ei.value.status == fem.FEM_ERR_TIMEOUT
        fem.fem_batch_destroy(bt)
        # the context is intact: the same work with the default budget runs and is certified
        opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_AB4, use_graph=use_graph)
        assert opts.wait_budget == 1 << 20
        bt = _batch(h, mesh, opts, 4)
        st, iters, relres = fem.fem_step(bt, 6, 4)
        assert st == fem.FEM_OK and np.all(relres < 1e-8) and np.all(iters > 0)
        fem.fem_batch_destroy(bt)
        torch.cuda.synchronize()
    finally:
        fem.fem_mesh_destroy(h)


def test_zero_wait_budget_in_pcg_solve():
    import torch
    build.build()
    fem.lib()
    mesh = small_mesh(8, 6, 5)
    tp = wl.TimeParams()
    h = fem.fem_mesh_create(mesh, tp)
    try:
        r = 4
        rng = np.random.default_rng(3)
        b = rng.standard_normal((mesh.n_nodes, 3, r))
        b[mesh.fixed_dof.reshape(-1, 3).astype(bool)] = 0.0
        b = torch.tensor(b.reshape(-1), device="cuda")
        x = torch.zeros_like(b)
        opts0 = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, wait_budget=0)
        with pytest.raises(fem.FemError) as ei:
            fem.pcg_solve(h, b, x, r, opts0)
        assert ei.value.status == fem.FEM_ERR_TIMEOUT
        x.zero_()
        _, its, rr = fem.pcg_solve(h, b, x, r, fem.fem_opts_default(precision=fem.FEM_FP32_INNER))
        assert np.all(rr < 1e-8)
        with pytest.raises(fem.FemError) as ei:
            fem.pcg_solve(h, b, x, r, fem.fem_opts_default(wait_budget=-1))
        assert ei.value.status == fem.FEM_ERR_ARG
        torch.cuda.synchronize()
    finally:
        fem.fem_mesh_destroy(h)
