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


def _run_and_check(mesh, tp, sources, opts, n_steps, region_nodes=None, check_pred=True, b_tol=1e-12,
                   system=None, create=None, regions=None, eager_steps=()):
    """Steps the batch one step at a time and checks every step against the oracle; returns (iterations per
    case, predictor check statistics).  system (the oracle's (System, reduced A)), create (the mesh
    constructor) and regions (a node -> region map) default to the linear-tet ones.  Steps listed in
    eager_steps run eagerly (profiling on) inside a graph-step run."""
    sysm, A = system if system is not None else oracle.build_system(mesh, tp)
    N = mesh.n_nodes
    h = (create or fem.fem_mesh_create)(mesh, tp)
    if region_nodes and regions is None:
        regions = wl.region_map(mesh, region_nodes)
    if regions is not None:
        fem.fem_mesh_set_regions(h, regions)
    bt = fem.fem_batch_create(opts)
    nc = len(sources)
    try:
        for s in sources:
            fem.fem_case_add(bt, h, s)
        st = {c: dict(u=np.zeros(3 * N), v=np.zeros(3 * N), a=np.zeros(3 * N), vh=[np.zeros(3 * N)] * 4, E=[])
              for c in range(nc)}
        total_iters = np.zeros(nc, dtype=np.int64)
        stats = PredStats()
        absA = None
        reg_dof = np.repeat(regions, 3)[sysm.free] if regions is not None else None
        n_reg = int(regions.max()) + 1 if regions is not None else 0
        for it in range(1, n_steps + 1):
            if it in eager_steps:
                fem.fem_batch_profile(bt, 1)
            stat, iters, relres = fem.fem_step(bt, 1, nc)
            if it in eager_steps:
                fem.fem_batch_profile(bt, 0)
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
                # a few ulps of the largest term of each update formula (u + du; 2/dt du - v;
                # 4/dt^2 du - 4/dt v - a)
                dmax = np.abs(du).max()
                scales = (max(np.abs(S["u"]).max(), dmax), max(2.0 / tp.dt * dmax, np.abs(S["v"]).max()),
                          max(4.0 / tp.dt ** 2 * dmax, 4.0 / tp.dt * np.abs(S["v"]).max(), np.abs(S["a"]).max()))
                for got, ref, sc in ((u, u_ref, scales[0]), (v, v_ref, scales[1]), (a, a_ref, scales[2])):
                    assert np.abs(got - ref).max() <= 1e-13 * max(np.abs(ref).max(), sc, 1e-300), (it, c)
                # predictor from the GPU's own history
                u_ab = oracle.adams_bashforth4(S["u"], S["vh"], tp.dt)
                du_ab = (u_ab - S["u"])
                if check_pred:
                    if opts.predictor == fem.FEM_PRED_AB4 or regions is None:
                        assert np.abs(guess - du_ab).max() <= 1e-13 * max(np.abs(du_ab).max(), 1e-300)
                    else:
                        coef, n_pairs = fem.predictor_coefficients(bt, c, n_reg, opts.s_max)
                        y_gpu = (guess - du_ab)[sysm.free]
                        floor = 1e-13 * max(np.abs(du_ab).max(), 1e-300)     # AB4 rounding in y_gpu
                        y_gpu, kind = guarded_correction(bt, c, y_gpu, S["E"], reg_dof, n_reg, coef, n_pairs,
                                                         floor, stats, where=(it, c))
                        if n_pairs > 0 and opts.pred_guard and opts.precision == fem.FEM_FP32_INNER:
                            if absA is None:
                                absA = abs(A)
                            check_guard(kind, A, absA, b_ref[sysm.free], du_ab[sysm.free], y_gpu, where=(it, c))
                        check_prediction(S["E"], reg_dof, n_reg, y_gpu, coef, n_pairs, opts, floor, stats,
                                         where=(it, c))
                S["E"].append(stored_value(du[sysm.free] - du_ab[sysm.free], opts.snapshot_format))
                if len(S["E"]) > opts.s_max + 1:
                    S["E"].pop(0)
                S["vh"] = S["vh"][1:] + [v.copy()]
                S["u"], S["v"], S["a"] = u, v, a
        if check_pred and opts.predictor == fem.FEM_PRED_DD and regions is not None and \
                opts.precision == fem.FEM_FP32_INNER:
            assert sum(fem.fem_case_stats(bt, c)["fallbacks"] for c in range(nc)) == stats.guess.get(2, 0)
        stats.assert_ok()
        return total_iters, stats
    finally:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)


def _trunc24(v):
    """v truncated to 24 significant bits (as the GPU's integer-pipe split does); |v| < 2^-126 -> 0."""
    mask = ~np.uint64((1 << 29) - 1)
    t = (np.ascontiguousarray(v, dtype=np.float64).view(np.uint64) & mask).view(np.float64)
    return np.where(np.abs(v) < 2.0 ** -126, 0.0, t)


def stored_value(v, fmt):
    """The value a snapshot slot of format fmt holds for the FP64 value v (the GPU predicts from these):
    0 FP64 as is; 1 FP32 rounded to nearest; 2 double-float pair hi = v truncated to 24 significant bits,
    lo = the remainder truncated to 24 bits; 3 hi as in 2 and lo rounded to the nearest-even BF16.  Values
    below 2^-126 are flushed in formats 2 and 3 (the GPU reads a pair back as hi + lo)."""
    v = np.asarray(v, dtype=np.float64)
    if fmt == 0:
        return v.copy()
    if fmt == 1:
        return v.astype(np.float32).astype(np.float64)
    tiny = 2.0 ** -126
    hi = _trunc24(v)
    lo = _trunc24(v - hi)
    if fmt == 3:
        u = lo.astype(np.float32).view(np.uint32).astype(np.uint64)
        u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
        lo = u.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.abs(v) < tiny, 0.0, hi + lo)


# Relative rounding of one Gram entry as the GPU accumulates it, per snapshot format: FP64 FMAs; FP32
# products with compensated FP32 sums; double-float products and sums (formats 2 and 3).
GRAM_EPS = {0: 2.0 ** -52, 1: 2.0 ** -23, 2: 2.0 ** -46, 3: 2.0 ** -46}
# Unit of the stored value per format.  The test forms the corrections e = du - du_AB from its own
# Adams-Bashforth increment, which differs from the GPU's by FP64 rounding; where that difference crosses a
# rounding boundary of the storage format, the modelled stored value and the GPU's differ by one unit.
STORE_EPS = {0: 2.0 ** -52, 1: 2.0 ** -24, 2: 2.0 ** -48, 3: 2.0 ** -32}


class PredStats:
    """Per (step, case, region) outcomes of check_prediction (and the guess guard's choices)."""

    def __init__(self):
        self.guess = {}         # case-steps by initial guess kind (fem_case_stats_t.guess)
        self.n = 0              # regions checked
        self.elementwise = 0    # also checked element by element (well-conditioned kept columns)
        self.ambiguous = 0      # a column's drop decision is within rounding of the threshold
        self.worst = {"consistency": 0.0, "objective": 0.0, "elementwise": 0.0}
        self.fail = []

    def note(self, kind, ratio, where):
        self.worst[kind] = max(self.worst[kind], ratio)
        if not ratio <= 1.0:
            self.fail.append((kind, ratio, where))

    def assert_ok(self):
        assert not self.fail, self.fail[:5]
        assert self.ambiguous <= max(2, 0.02 * self.n), (self.ambiguous, self.n)


def check_prediction(E, reg_dof, n_reg, y_gpu, coef, n_pairs, opts, floor, stats, where=None, s_used=None):
    """Checks the GPU's regional correction y_gpu (and its coefficients coef [n_reg][s_max]) against the
    oracle's modified Gram-Schmidt on the stored corrections E (oldest first, E[-1] = the query e^{it-1}).

    Per region R, with X_R, Y_R the stored pairs and x_R the query:
      consistency  y_gpu_R = Y_R c_gpu to the combination's rounding;
      objective    ||X_R c_gpu - x_R|| <= ||X_R w_ref - x_R|| + 30 eps_G (cond_k sigma_max ||w_ref|| + ||x_R||):
                   c_gpu solves the same least-squares problem as MGS's w_ref, up to the first-order effect of
                   the Gram's rounding eps_G on the residual (cond_k, sigma_max: condition number and norm of the
                   columns MGS keeps).  This holds however ill-conditioned X_R is, where the coefficients
                   themselves are not determined;
      elementwise  where cond_k <= 1e6: |y_gpu - y_ref| <= 10 eps_G cond_k^2 max|Y_R| ||w_ref||_1 + floor (the
                   normal equations' rounding bound on the coefficients, carried through Y_R).
    A column whose orthogonalised norm ratio lies within a factor 3 of tau may be kept by one side and
    dropped by the other (the Gram pivot's rounding at the threshold): such a region is counted as ambiguous
    and its objective is bounded by MGS's residual with those columns dropped."""
    n = min(opts.s_max if s_used is None else s_used, len(E) - 1) if E else 0
    assert n_pairs == max(n, 0), (n_pairs, n, where)
    if n <= 0:
        assert np.abs(y_gpu).max() <= floor, where
        return
    X = np.stack(E[-(n + 1):-1], axis=1)
    Y = np.stack(E[-n:], axis=1)
    xq = E[-1]
    eps = GRAM_EPS[opts.snapshot_format]
    tau = opts.tau
    for R in range(n_reg):
        idx = np.nonzero(reg_dof == R)[0]
        if idx.size == 0:
            continue
        stats.n += 1
        XR, YR, xR, yg = X[idx], Y[idx], xq[idx], y_gpu[idx]
        cg = coef[R, :n]
        # consistency of the prediction with the reported coefficients (the combination's arithmetic:
        # FP32 for FP32 snapshots, double-float or FP64 otherwise)
        comb = np.abs(YR).max() * np.abs(cg).sum()
        err = np.abs(yg - YR @ cg).max()
        ceps = (4e-6 if opts.snapshot_format == 1 else 1e-12) + 4.0 * STORE_EPS[opts.snapshot_format]
        stats.note("consistency", err / (ceps * comb + floor + 1e-300), where + (R,) if where else R)
        # the oracle: MGS with the drop rule, and each column's orthogonalised norm ratio
        U, P, kept = oracle.mgs_upper(XR, tau)
        w_ref = U @ (P.T @ xR)
        y_ref = YR @ w_ref
        rho = np.zeros(n)
        for j in range(n):
            nj = np.linalg.norm(XR[:, j])
            prev = P[:, :j][:, kept[:j]]
            vj = XR[:, j] - prev @ (prev.T @ XR[:, j]) if prev.size else XR[:, j]
            rho[j] = np.linalg.norm(vj) / nj if nj > 0 else 0.0
        amb = (rho > tau / 3) & (rho < 3 * tau)
        res_g = np.linalg.norm(XR @ cg - xR)
        if amb.any():
            stats.ambiguous += 1
            Xd = XR.copy()
            Xd[:, amb] = 0.0
            Ud, Pd, kd = oracle.mgs_upper(Xd, tau)
            res_ref = max(np.linalg.norm(XR @ (U @ (P.T @ xR)) - xR), np.linalg.norm(Xd @ (Ud @ (Pd.T @ xR)) - xR))
            kept = kept & ~amb
        else:
            res_ref = np.linalg.norm(XR @ w_ref - xR)
        Xk = XR[:, kept]
        if Xk.shape[1]:
            sv = np.linalg.svd(Xk, compute_uv=False)
            cond_k = sv[0] / sv[-1] if sv[-1] > 0 else np.inf
            smax = sv[0]
        else:
            cond_k, smax = 1.0, 0.0
        xn = np.linalg.norm(xR)
        seps = 4.0 * STORE_EPS[opts.snapshot_format]
        bound = (30.0 * eps * (min(cond_k, 1e12) * smax * np.linalg.norm(w_ref) + xn) + 1e-14 * xn + floor +
                 seps * (np.linalg.norm(XR) * np.abs(cg).sum() + xn))
        stats.note("objective", max(res_g - res_ref, 0.0) / bound, where + (R,) if where else R)
        if cond_k <= 1e6 and not amb.any():
            stats.elementwise += 1
            bnd = ((10.0 * eps * cond_k ** 2 + seps * cond_k) * np.abs(YR).max() * np.abs(w_ref).sum() +
                   1e-13 * np.abs(y_ref).max() + floor)
            stats.note("elementwise", np.abs(yg - y_ref).max() / bnd, where + (R,) if where else R)


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
    for fmt in (0, 2):
        opts_dd = fem.fem_opts_default(tol=1e-8, predictor=fem.FEM_PRED_DD, s_max=8, snapshot_format=fmt)
        it_dd, stats = _run_and_check(mesh, tp, srcs, opts_dd, 40, region_nodes=64)
        assert it_dd.sum() < it_ab.sum(), (fmt, it_dd, it_ab)
        assert stats.n > 0


def test_step_multicase_dd_fp32_bf16_snapshots(torch_dev):
    """Snapshots stored as an FP32 value plus its BF16-rounded residual (about 2^-32 relative): the
    prediction solves the least-squares problem of the stored values, still saves iterations against AB4
    and takes no more than 5% over double-float storage."""
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
    1e-11.  The predictor (FP32 snapshots) is checked against the oracle's MGS on the stored values."""
    mesh = small_mesh(8, 7, 6)
    tp = wl.TimeParams()
    srcs = [wl.random_source(mesh, wl.rng_for(92, 0, c), f0=4.0) for c in range(3)]   # padded to 4 lanes
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=8,
                                snapshot_format=1, refresh_every=refresh, cert_df=cert_df)
    _run_and_check(mesh, tp, srcs, opts, 40, region_nodes=64, b_tol=1e-11 if cert_df in (1, 3) else 1e-12)


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
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16,
                                cert_df=3, snapshot_format=0)
    _run_and_check(mesh, tp, srcs, opts, 60, region_nodes=64, b_tol=1e-11)


@pytest.mark.parametrize("s_max", [16, 32])
def test_step_benchmark_settings(torch_dev, s_max):
    """The benchmark's solver settings on a smaller box of the large recipe: dt = 0.004, h = 1/64, 16 cases
    in one group, FP32-inner solver, double-float snapshot ring, regions of 1024 nodes, the double-float
    assembled certification product, graph steps.  Every step is certified by the oracle's CSR A, and every
    region of every step's prediction is checked against the oracle's MGS (consistency and least-squares
    objective; element by element where the kept columns are well-conditioned)."""
    mesh = wl.config4_mesh(16, 16, 12)
    tp = wl.config4_time_params()
    srcs = wl.config4_sources(mesh, 16)
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=s_max,
                                cert_df=3, snapshot_format=2, use_graph=1)
    it, stats = _run_and_check(mesh, tp, srcs, opts, s_max + 24, region_nodes=1024, b_tol=1e-11)
    assert stats.n >= 16 * (s_max + 20) * 3 and stats.elementwise > 0, (stats.n, stats.elementwise)


@pytest.mark.parametrize("margin", [0.5, 0.9])
def test_step_inner_margin(torch_dev, margin):
    """Inner FP32 solves aimed at a larger fraction of the tolerance (fem_opts.inner_margin): every step is
    still certified below tol by the oracle's CSR A (a case that ends at or above tol takes another
    refinement pass), and the CG iterations do not exceed those of an aim of 0.1 on the same steps."""
    mesh = wl.config4_mesh(16, 16, 12)
    tp = wl.config4_time_params()
    srcs = wl.config4_sources(mesh, 8)
    its = {}
    for m in (0.1, margin):
        opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16,
                                    cert_df=3, snapshot_format=2, use_graph=1, inner_margin=m)
        it, _ = _run_and_check(mesh, tp, srcs, opts, 40, region_nodes=1024, b_tol=1e-11)
        its[m] = int(it.sum())
    assert its[margin] <= its[0.1], its


@pytest.mark.parametrize("graph", [0, 1])
def test_step_guess_guard(torch_dev, graph):
    """The guess guard (fem_opts.pred_guard) with the benchmark's solver settings on a 16 x 16 x 12 box of the
    large recipe, 8 cases, 40 steps from rest: every step certified by the oracle's CSR A, every choice
    between the data-driven and the Adams-Bashforth guess checked against the oracle's residuals of both
    (check_guard), the coefficients of dropped corrections still checked against the oracle's MGS, and the
    library's count of dropped corrections equal to the steps seen with the Adams-Bashforth guess.  With the
    guard off no correction is dropped."""
    mesh = wl.config4_mesh(16, 16, 12)
    tp = wl.config4_time_params()
    srcs = wl.config4_sources(mesh, 8)
    res = {}
    for guard in (0, 1):
        opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16,
                                    cert_df=3, snapshot_format=2, use_graph=graph, pred_guard=guard)
        it, stats = _run_and_check(mesh, tp, srcs, opts, 40, region_nodes=1024, b_tol=1e-11)
        res[guard] = (int(it.sum()), dict(stats.guess))
    print("guess guard", graph, res)
    assert res[0][1].get(2, 0) == 0, res
    assert res[1][1].get(2, 0) > 0, res


def test_graph_steps_around_eager_steps(torch_dev):
    """Graph steps form the next step's Adams-Bashforth increment at their tail; a graph step after eager
    steps forms its own before the launch.  Graph steps interleaved with eager ones (profiling on) on the
    benchmark's settings: every step certified, every guess checked against the oracle's Adams-Bashforth
    increment and regional correction."""
    mesh = wl.config4_mesh(16, 16, 12)
    tp = wl.config4_time_params()
    srcs = wl.config4_sources(mesh, 8)
    opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16,
                                cert_df=3, snapshot_format=2, use_graph=1)
    _run_and_check(mesh, tp, srcs, opts, 30, region_nodes=1024, b_tol=1e-11, eager_steps={1, 9, 10, 17, 25})


def test_pred_guard_option_checked(torch_dev):
    for g in (-1, 2):
        with pytest.raises(fem.FemError) as ei:
            fem.fem_batch_create(fem.fem_opts_default(precision=fem.FEM_FP32_INNER, pred_guard=g))
        assert ei.value.status == fem.FEM_ERR_ARG


def test_inner_margin_out_of_range_rejected(torch_dev):
    for m in (0.0, 1.0, -0.5):
        with pytest.raises(fem.FemError) as ei:
            fem.fem_batch_create(fem.fem_opts_default(precision=fem.FEM_FP32_INNER, inner_margin=m))
        assert ei.value.status == fem.FEM_ERR_ARG


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


def guarded_correction(bt, c, y_gpu, E, reg_dof, n_reg, coef, n_pairs, floor, stats, where=None):
    """The correction the prediction checks apply to, and the step's initial guess kind.  Where the guess
    guard dropped the case's correction (kind 2) the guess is the Adams-Bashforth one (y_gpu = 0 to its
    rounding floor) and the checks apply to the correction the coefficients give, Y_R c_R on each region."""
    kind = fem.fem_case_stats(bt, c)["guess"]
    stats.guess[kind] = stats.guess.get(kind, 0) + 1
    if kind != 2:
        return y_gpu, kind
    assert np.abs(y_gpu).max() <= floor, where
    n = n_pairs
    if n <= 0:
        return y_gpu, kind
    Y = np.stack(E[-n:], axis=1)
    y = np.zeros_like(y_gpu)
    for R in range(n_reg):
        idx = np.nonzero(reg_dof == R)[0]
        y[idx] = Y[idx] @ coef[R, :n]
    return y, kind


def check_guard(kind, A, absA, b, du_ab, y, where=None):
    """The guard's choice against the oracle's residuals (free DOFs): the Adams-Bashforth guess's
    r_ab = b - A du_ab and the data-driven one's r_ab - A y.  Kind 2 (correction dropped) needs
    ||r_ab|| <= ||r_ab - A y||, kind 1 the reverse, each up to the GPU's rounding: FP32 residual values
    (1e-6 of the norms), the FP32 product of y in FP32 (4e-6 of || |A| |y| ||) and the FP64 recurrence
    products (1e-10 of ||b||)."""
    if kind not in (1, 2):
        return
    r_ab = b - A @ du_ab
    n_ab = np.linalg.norm(r_ab)
    n_dd = np.linalg.norm(r_ab - A @ y)
    slack = 4e-6 * np.linalg.norm(absA @ np.abs(y)) + 1e-6 * (n_ab + n_dd) + 1e-10 * np.linalg.norm(b)
    if kind == 2:
        assert n_ab <= n_dd + slack, (where, n_ab, n_dd, slack)
    else:
        assert n_dd <= n_ab + slack, (where, n_ab, n_dd, slack)
