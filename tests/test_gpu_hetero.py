"""The paper's heterogeneous scheme (Algorithm 3): the data-driven correction computed on the host CPU from a
host copy of the stored corrections while the GPU steps the other case set, s balanced after each step.

Every step of every case is certified with the oracle's CSR A, and every region's host prediction is checked
against the oracle's MGS on the same stored values (consistency with the reported coefficients, the
least-squares objective, element by element where the kept columns are well-conditioned), with the pair
count the balancing chose.  The balance stays within [1, s_max]."""
import numpy as np
import pytest

import oracle
from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import small_mesh
from test_gpu_step import PredStats, check_guard, check_prediction, guarded_correction, stored_value

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    build.build()
    fem.lib()
    return torch


@pytest.mark.parametrize("precision,fmt", [("mixed", 2), ("fp64", 0)])
def test_host_predictor_steps(torch_dev, precision, fmt):
    mesh = small_mesh(8, 7, 6, h=1.0 / 64)
    tp = wl.config2_time_params()
    srcs = [wl.random_source(mesh, wl.rng_for(95, 0, c)) for c in range(4)]
    s_max = 8
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER if precision == "mixed" else fem.FEM_FP64,
                                predictor=fem.FEM_PRED_DD, s_max=s_max, snapshot_format=fmt, cpu_predictor=1)
    sysm, A = oracle.build_system(mesh, tp)
    N = mesh.n_nodes
    regions = wl.region_map(mesh, 64)
    n_reg = int(regions.max()) + 1
    reg_dof = np.repeat(regions, 3)[sysm.free]
    h = fem.fem_mesh_create(mesh, tp)
    fem.fem_mesh_set_regions(h, regions)
    bt = fem.fem_batch_create(opts)
    try:
        for s in srcs:
            fem.fem_case_add(bt, h, s)
        st = {c: dict(u=np.zeros(3 * N), v=np.zeros(3 * N), a=np.zeros(3 * N), vh=[np.zeros(3 * N)] * 4, E=[])
              for c in range(4)}
        stats = PredStats()
        absA = abs(A)
        total = np.zeros(4)
        for it in range(1, 41):
            stat, iters, relres = fem.fem_step(bt, 1, 4)
            total += iters
            for c in range(4):
                S = st[c]
                u = fem.fem_case_get(bt, c, fem.FEM_FIELD_U, N)
                v = fem.fem_case_get(bt, c, fem.FEM_FIELD_V, N)
                a = fem.fem_case_get(bt, c, fem.FEM_FIELD_A, N)
                du = fem.fem_case_get(bt, c, fem.FEM_FIELD_DU, N)
                guess = fem.fem_case_get(bt, c, fem.FEM_FIELD_GUESS, N)
                f = oracle.point_force(3 * N, srcs[c], it * tp.dt)
                b_ref = oracle.newmark_rhs(sysm, f, S["u"], S["v"], S["a"])
                nb = np.linalg.norm(b_ref[sysm.free])
                cert = np.linalg.norm(b_ref[sysm.free] - A @ du[sysm.free]) / nb
                assert cert < 1e-8, (it, c, cert)
                u_ab = oracle.adams_bashforth4(S["u"], S["vh"], tp.dt)
                du_ab = u_ab - S["u"]
                coef, n_pairs = fem.predictor_coefficients(bt, c, n_reg, s_max)
                assert n_pairs <= s_max
                y = (guess - du_ab)[sysm.free]
                floor = 1e-13 * max(np.abs(du_ab).max(), 1e-300)
                if n_pairs == 0:
                    assert np.abs(y).max() <= floor or it <= 2
                else:
                    y, kind = guarded_correction(bt, c, y, S["E"], reg_dof, n_reg, coef, n_pairs, floor, stats,
                                                 where=(it, c))
                    check_guard(kind, A, absA, b_ref[sysm.free], du_ab[sysm.free], y, where=(it, c))
                    check_prediction(S["E"], reg_dof, n_reg, y, coef, n_pairs, opts, floor, stats, where=(it, c),
                                     s_used=n_pairs)
                S["E"].append(stored_value(du[sysm.free] - du_ab[sysm.free], fmt))
                if len(S["E"]) > s_max + 1:
                    S["E"].pop(0)
                S["vh"] = S["vh"][1:] + [v.copy()]
                S["u"], S["v"], S["a"] = u, v, a
        stats.assert_ok()
        assert stats.n > 0
        for c in range(4):
            bal = fem.fem_batch_predictor_balance(bt, c)
            assert 1 <= bal["s"] <= s_max and bal["predict_total_ms"] > 0.0
    finally:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)


def test_host_predictor_arguments(torch_dev):
    with pytest.raises(fem.FemError):
        fem.fem_batch_create(fem.fem_opts_default(cpu_predictor=1))                    # needs the DD predictor
    with pytest.raises(fem.FemError):
        fem.fem_batch_create(fem.fem_opts_default(predictor=fem.FEM_PRED_DD, cpu_predictor=1, snapshot_format=1))
