"""fem_step on the GPU against the oracle, step by step (Section 3.1 Newmark stepping, Algorithm 1 solve,
Section 3.2 predictors).

After every GPU step the oracle recomputes, from the GPU's previous state (u, v, a), the right-hand side
b (must match to 1e-12 relative), certifies the GPU's increment (||b - A du|| / ||b|| < tol, with the
oracle's CSR A), checks the Newmark update exactly, and recomputes the predictor output from the GPU's own
history (Adams-Bashforth to 1e-13; the regional data-driven correction to the Gram-vs-MGS rounding bound
derived from the condition number of each region's snapshot matrix)."""
import numpy as np
import pytest

import oracle
from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import small_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    build.build()
    fem.lib()
    return torch


def _run_and_check(mesh, tp, sources, opts, n_steps, region_nodes=None, check_pred=True, b_tol=1e-12):
    sysm, A = oracle.build_system(mesh, tp)
    N = mesh.n_nodes
    h = fem.fem_mesh_create(mesh, tp)
    regions = None
    if region_nodes:
        regions = wl.region_map(mesh, region_nodes)
        fem.fem_mesh_set_regions(h, regions)
    bt = fem.fem_batch_create(opts)
    nc = len(sources)
    try:
        for s in sources:
            fem.fem_case_add(bt, h, s)
        st = {c: dict(u=np.zeros(3 * N), v=np.zeros(3 * N), a=np.zeros(3 * N), vh=[np.zeros(3 * N)] * 4, E=[])
              for c in range(nc)}
        total_iters = np.zeros(nc, dtype=np.int64)
        worst_pred = 0.0
        reg_dof = np.repeat(regions, 3)[sysm.free] if regions is not None else None
        for it in range(1, n_steps + 1):
            stat, iters, relres = fem.fem_step(bt, 1, nc)
            total_iters += iters
            for c in range(nc):
                S = st[c]
                u = fem.fem_case_get(bt, c, fem.FEM_FIELD_U, N)
                v = fem.fem_case_get(bt, c, fem.FEM_FIELD_V, N)
                a = fem.fem_case_get(bt, c, fem.FEM_FIELD_A, N)
                du = fem.fem_case_get(bt, c, fem.FEM_FIELD_DU, N)
                b = fem.fem_case_get(bt, c, fem.FEM_FIELD_B, N)
                guess = fem.fem_case_get(bt, c, fem.FEM_FIELD_GUESS, N)
                f = oracle.point_force(3 * N, sources[c], it * tp.dt)
                b_ref = oracle.newmark_rhs(sysm, f, S["u"], S["v"], S["a"])
                b_ref[mesh.fixed_dof == 1] = 0.0
                nb = np.linalg.norm(b_ref)
                assert np.linalg.norm(b - b_ref) <= b_tol * nb, (it, c, np.linalg.norm(b - b_ref) / nb)
                cert = np.linalg.norm(b_ref[sysm.free] - A @ du[sysm.free]) / nb
                assert cert < opts.tol, (it, c, cert)
                assert abs(relres[c] - cert) <= 1e-3 * opts.tol + 1e-6 * cert
                u_ref, v_ref, a_ref = oracle.newmark_update(S["u"], S["v"], S["a"], du, tp.dt)
                for got, ref in ((u, u_ref), (v, v_ref), (a, a_ref)):
                    assert np.abs(got - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300)
                # predictor from the GPU's own history
                u_ab = oracle.adams_bashforth4(S["u"], S["vh"], tp.dt)
                du_ab = (u_ab - S["u"])
                if check_pred:
                    if opts.predictor == fem.FEM_PRED_AB4 or regions is None:
                        assert np.abs(guess - du_ab).max() <= 1e-13 * max(np.abs(du_ab).max(), 1e-300)
                    else:
                        # the oracle predicts from the snapshots as stored (format 3 rounds them to ~2^-32)
                        E_st = [_hl_stored(e) for e in S["E"]] if opts.snapshot_format == 3 else S["E"]
                        y_ref, W = oracle.regional_predict(E_st, reg_dof, int(regions.max()) + 1, opts.s_max,
                                                           opts.tau)
                        y_gpu = (guess - du_ab)[sysm.free]
                        if y_ref is None:
                            y_ref = np.zeros_like(y_gpu)
                        floor = 1e-13 * max(np.abs(du_ab).max(), 1e-300)     # AB4 rounding in y_gpu
                        worst_pred = max(worst_pred, _pred_err(E_st, reg_dof, y_gpu, y_ref, opts.s_max, floor))
                S["E"].append(du[sysm.free] - du_ab[sysm.free])
                if len(S["E"]) > opts.s_max + 1:
                    S["E"].pop(0)
                S["vh"] = S["vh"][1:] + [v.copy()]
                S["u"], S["v"], S["a"] = u, v, a
        assert worst_pred <= 1.0, worst_pred
        return total_iters, worst_pred
    finally:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)


def _hl_stored(v):
    """The value a snapshot slot of format 3 holds for the FP64 value v: hi = v truncated to 24 significant
    bits, lo = v - hi truncated to 24 bits and rounded to the nearest-even BF16, values below 2^-126
    flushed (the GPU reads the pair back as hi + lo)."""
    mask = ~np.uint64((1 << 29) - 1)
    tiny = 2.0 ** -126
    hi = (np.ascontiguousarray(v, dtype=np.float64).view(np.uint64) & mask).view(np.float64)
    hi = np.where(np.abs(v) < tiny, 0.0, hi)
    lo = (np.ascontiguousarray(v - hi).view(np.uint64) & mask).view(np.float64)
    lo = np.where(np.abs(lo) < tiny, 0.0, lo)
    u = lo.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    lo_bf = u.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.abs(v) < tiny, 0.0, hi + lo_bf)


def _pred_err(E, reg_dof, y_gpu, y_ref, s_max, floor):
    """max over regions of |y_gpu - y_ref| / bound, bound = 10 cond(X)^2 eps scale + floor: the rounding
    bound of a least-squares solve through the normal equations (the GPU's Gram route) against MGS (the
    oracle).  It is a bound on the whole prediction once cond(X) reaches ~1e8 (early steps, when the
    stored corrections are nearly collinear): there the column-drop decisions the Gram pivots take are no
    longer resolvable in FP64 and the check keeps only the prediction's size in bounds.  The floor is the
    rounding of the Adams-Bashforth part that y_gpu = guess - du_AB carries."""
    npairs = min(s_max, len(E) - 1)
    if npairs <= 0:
        assert np.abs(y_gpu).max() <= floor
        return 0.0
    X = np.stack(E[-(npairs + 1):-1], axis=1)
    worst = 0.0
    for R in range(int(reg_dof.max()) + 1):
        idx = reg_dof == R
        XR = X[idx]
        scale = max(np.abs(y_ref[idx]).max(), np.abs(E[-1][idx]).max(), 1e-300)
        sv = np.linalg.svd(XR, compute_uv=False)
        cond = sv[0] / sv[-1] if sv[-1] > 0 else np.inf
        bound = 10.0 * min(cond, 1e9) ** 2 * 2.2e-16 * scale + 1e-14 * scale + floor
        worst = max(worst, np.abs(y_gpu[idx] - y_ref[idx]).max() / bound)
    return worst


def test_step_cfg1_fp64_ab4(torch_dev):
    mesh = wl.config1_mesh()
    tp = wl.TimeParams()
    opts = fem.fem_opts_default(tol=1e-8)
    _run_and_check(mesh, tp, wl.config1_sources(1), opts, 100)


def test_step_multicase_dd_fp64_snapshots(torch_dev):
    mesh = small_mesh(8, 7, 6)
    tp = wl.TimeParams()
    srcs = [wl.random_source(mesh, wl.rng_for(91, 0, c), f0=6.0) for c in range(4)]
    opts_ab = fem.fem_opts_default(tol=1e-8, predictor=fem.FEM_PRED_AB4)
    it_ab, _ = _run_and_check(mesh, tp, srcs, opts_ab, 40)
    opts_dd = fem.fem_opts_default(tol=1e-8, predictor=fem.FEM_PRED_DD, s_max=8, snapshot_format=2)
    it_dd, worst = _run_and_check(mesh, tp, srcs, opts_dd, 40, region_nodes=64)
    assert it_dd.sum() < it_ab.sum(), (it_dd, it_ab)


def test_step_multicase_dd_fp32_bf16_snapshots(torch_dev):
    """Snapshots stored as an FP32 value plus its BF16-rounded residual (about 2^-32 relative): the
    prediction matches the oracle's prediction from the same stored values within the FP64 rounding bound,
    still saves iterations against AB4 and takes no more than 5% over double-float storage."""
    mesh = small_mesh(8, 7, 6)
    tp = wl.TimeParams()
    srcs = [wl.random_source(mesh, wl.rng_for(91, 0, c), f0=6.0) for c in range(4)]
    opts_ab = fem.fem_opts_default(tol=1e-8, predictor=fem.FEM_PRED_AB4)
    it_ab, _ = _run_and_check(mesh, tp, srcs, opts_ab, 40)
    opts_df = fem.fem_opts_default(tol=1e-8, predictor=fem.FEM_PRED_DD, s_max=8, snapshot_format=2)
    it_df, _ = _run_and_check(mesh, tp, srcs, opts_df, 40, region_nodes=64)
    opts_hl = fem.fem_opts_default(tol=1e-8, predictor=fem.FEM_PRED_DD, s_max=8, snapshot_format=3)
    it_hl, _ = _run_and_check(mesh, tp, srcs, opts_hl, 40, region_nodes=64)
    assert it_hl.sum() < it_ab.sum(), (it_hl, it_ab)
    assert it_hl.sum() <= 1.05 * it_df.sum() + 2, (it_hl, it_df)


@pytest.mark.parametrize("refresh,cert_df", [(200, 0), (7, 0), (200, 1), (7, 1), (200, 2), (200, 3), (7, 3)])
def test_step_mixed_precision_dd(torch_dev, refresh, cert_df):
    """FP32-inner steps keep K u, M v, K v, M a and A v by recurrences: b must still match the oracle's b
    recomputed from the state, with or without periodic direct refreshes of those products.  With native
    FP64 certification products (element by element or assembled) the bound is FP64 rounding (1e-12); with
    double-float products (2^-47 relative error per operation, accumulated over 40 recurrence steps) it is
    1e-11."""
    mesh = small_mesh(8, 7, 6)
    tp = wl.TimeParams()
    srcs = [wl.random_source(mesh, wl.rng_for(92, 0, c), f0=4.0) for c in range(3)]   # padded to 4 lanes
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=8,
                                snapshot_format=1, refresh_every=refresh, cert_df=cert_df)
    _run_and_check(mesh, tp, srcs, opts, 40, region_nodes=64, check_pred=False,
                   b_tol=1e-11 if cert_df in (1, 3) else 1e-12)


def test_step_mixed_precision_ab4_cfg1(torch_dev):
    mesh = wl.config1_mesh()
    tp = wl.TimeParams()
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, cert_df=0)
    _run_and_check(mesh, tp, wl.config1_sources(1), opts, 100)


def test_step_mixed_precision_dd_medium_dt(torch_dev):
    """The medium workload's time step (dt = 0.004) with FP64 snapshots and the double-float assembled
    certification product."""
    mesh = small_mesh(10, 8, 6, h=1.0 / 64)
    tp = wl.config2_time_params()
    srcs = [wl.random_source(mesh, wl.rng_for(93, 0, c)) for c in range(4)]
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16, cert_df=3)
    _run_and_check(mesh, tp, srcs, opts, 60, region_nodes=64, check_pred=False, b_tol=1e-11)


def test_step_matches_independent_oracle_run(torch_dev):
    """GPU and oracle time histories, each solved to 1e-12, agree to 1e-9 after 50 steps."""
    mesh = wl.config1_mesh()
    tp = wl.TimeParams()
    src = wl.config1_sources(1)[0]
    sysm, A = oracle.build_system(mesh, tp)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    sim = oracle.CaseSimulator(sysm, A, Binv, src, predictor="ab4", eps=1e-12)
    for _ in range(50):
        sim.step()
    h = fem.fem_mesh_create(mesh, tp)
    bt = fem.fem_batch_create(fem.fem_opts_default(tol=1e-12))
    try:
        fem.fem_case_add(bt, h, src)
        fem.fem_step(bt, 50, 1)
        u = fem.fem_case_get(bt, 0, fem.FEM_FIELD_U, mesh.n_nodes)
        assert np.linalg.norm(u - sim.u) <= 1e-9 * np.linalg.norm(sim.u)
        assert fem.fem_batch_steps(bt) == 50
    finally:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)
