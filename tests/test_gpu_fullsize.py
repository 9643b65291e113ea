"""The benchmark's workload at its full size, in the configuration bench.py times, checked on sampled outputs.

Workload: the large recipe's 256 x 256 x 128 box (50,331,648 tets, 8,520,321 nodes, five layers and the
basin), 8 cases on one mesh; FP32-inner / FP64-certified PCG with the packed staged EBE kernel at 8 cases,
the data-driven predictor with s = 16 on regions of 1024 nodes, double-float snapshot ring and certification
product, graph steps (the library defaults bench.py runs with).

The oracle cannot assemble or solve this system inside a test, so it computes sampled outputs one by one:
the rows of M and K at sampled nodes come from its tet4 element matrices of the elements around each
node (Section 3.1), and the regional correction of sampled regions from its MGS on those regions' stored
corrections (Section 3.2).  Checked:
  * the EBE product q = (cM M + cK K) p at sampled rows, FP32 (the inner solve's kernel) and FP64;
  * the symmetry of A through the product, p1^T (A p2) = p2^T (A p1), a property at any size;
  * every step of 30 graph steps from rest: b at sampled rows (Eq. GE:DIS, increment form); the
    certificate's residual b - A du at sampled rows against the certified bound tol ||b||; the Newmark
    update at sampled DOFs; the Adams-Bashforth increment and the data-driven correction on the sampled
    regions against the oracle's (consistency, least-squares objective, element by element where the kept
    columns are well-conditioned)."""
import numpy as np
import pytest

import oracle
from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from test_gpu_step import PredStats, check_prediction, guarded_correction, stored_value

pytestmark = pytest.mark.gpu

DIMS = (256, 256, 128)
NC = 8


class RowSampler:
    """Rows of M and K at sampled nodes from the oracle's element matrices of the elements around them."""

    def __init__(self, mesh, nodes):
        self.nodes = np.unique(np.asarray(nodes, dtype=np.int64))
        inc = np.nonzero(np.isin(mesh.conn, self.nodes).any(axis=1))[0]
        conn = mesh.conn[inc].astype(np.int64)
        Ke, Me = oracle.tet4_element_matrices(mesh.xyz, conn, mesh.mat_id[inc], mesh.lam_mu_rho)
        self.support = np.unique(conn)                       # nodes whose values the rows read
        loc = {int(n): i for i, n in enumerate(self.support)}
        row_of = {int(n): i for i, n in enumerate(self.nodes)}
        ns, nn = self.nodes.size, self.support.size
        self.M = np.zeros((ns * 3, nn * 3))
        self.K = np.zeros((ns * 3, nn * 3))
        for e in range(conn.shape[0]):
            for a in range(4):
                r = row_of.get(int(conn[e, a]))
                if r is None:
                    continue
                for b in range(4):
                    c = loc[int(conn[e, b])]
                    self.M[3 * r:3 * r + 3, 3 * c:3 * c + 3] += Me[e, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
                    self.K[3 * r:3 * r + 3, 3 * c:3 * c + 3] += Ke[e, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
        fixed = mesh.fixed_dof.reshape(-1, 3)
        self.row_free = (fixed[self.nodes] == 0).reshape(-1)
        self.sup_dofs = (3 * self.support[:, None] + np.arange(3)).reshape(-1)
        self.row_dofs = (3 * self.nodes[:, None] + np.arange(3)).reshape(-1)


def gather(torch, v, N, dofs):
    """Values of the DOFs `dofs` of every case from a [N][3][r] device vector: host array [r][len(dofs)]."""
    idx = torch.as_tensor(dofs, device=v.device)
    return v.view(N * 3, NC)[idx].T.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def big():
    import torch
    build.build()
    fem.lib()
    mesh = wl.config4_mesh(*DIMS)
    tp = wl.config4_time_params()
    srcs = wl.config4_sources(mesh, NC)
    regions = wl.region_map(mesh, 1024)
    h = fem.fem_mesh_create(mesh, tp)
    fem.fem_mesh_set_regions(h, regions)
    rng = np.random.default_rng(20380)
    interior = wl.interior_nodes(mesh)
    sample = np.concatenate([[s.node for s in srcs], rng.choice(interior, 24, replace=False),
                             rng.integers(0, mesh.n_nodes, 16)])
    rows = RowSampler(mesh, sample)
    yield dict(torch=torch, mesh=mesh, tp=tp, srcs=srcs, regions=regions, h=h, rows=rows)
    fem.fem_mesh_destroy(h)


def test_fullsize_product_sampled_rows_and_symmetry(big):
    torch, mesh, tp, h, rows = big["torch"], big["mesh"], big["tp"], big["h"], big["rows"]
    N = mesh.n_nodes
    cM = 4.0 / tp.dt ** 2 + 2.0 * tp.a0 / tp.dt
    cK = 1.0 + 2.0 * tp.a1 / tp.dt
    free = torch.as_tensor(mesh.fixed_dof == 0, device="cuda").repeat_interleave(NC)
    g = torch.Generator(device="cuda").manual_seed(7)
    p64 = torch.randn(N * 3 * NC, device="cuda", dtype=torch.float64, generator=g) * free
    A_rows = cM * rows.M + cK * rows.K
    for prec, p, tol in ((fem.FEM_FP32_INNER, p64.float(), 2e-6), (fem.FEM_FP64, p64, 1e-13)):
        q = torch.full_like(p, 9.0)
        ptq = torch.zeros(NC, dtype=torch.float64, device="cuda")
        fem.fem_ebe_apply(h, p, q, NC, cM, cK, ptq, precision=prec)
        torch.cuda.synchronize()
        ps = gather(torch, p, N, rows.sup_dofs)            # the product's own inputs (FP32-rounded for FP32)
        qs = gather(torch, q, N, rows.row_dofs)
        for c in range(NC):
            ref = A_rows @ ps[c]
            scale = np.abs(A_rows) @ np.abs(ps[c])          # the row's sum of absolute terms
            ref[~rows.row_free] = 0.0
            assert np.all(qs[c][~rows.row_free] == 0.0), (prec, c)
            err = np.abs(qs[c] - ref)[rows.row_free] / scale[rows.row_free]
            assert err.max() < tol, (prec, c, err.max())
            # the fused p^T q equals the sum over the product's own output
            full = float((p.double().view(-1, NC)[:, c] * q.double().view(-1, NC)[:, c]).sum())
            assert abs(ptq[c].item() - full) <= (1e-5 if prec == fem.FEM_FP32_INNER else 1e-12) * abs(full)
    # symmetry: p1^T A p2 = p2^T A p1 (FP64 products)
    p2 = torch.randn(N * 3 * NC, device="cuda", dtype=torch.float64, generator=g) * free
    q1, q2 = torch.empty_like(p64), torch.empty_like(p64)
    fem.fem_ebe_apply(h, p64, q1, NC, cM, cK)
    fem.fem_ebe_apply(h, p2, q2, NC, cM, cK)
    for c in range(NC):
        a = float((p64.view(-1, NC)[:, c] * q2.view(-1, NC)[:, c]).sum())
        b = float((p2.view(-1, NC)[:, c] * q1.view(-1, NC)[:, c]).sum())
        assert abs(a - b) <= 1e-11 * float((p64.abs().view(-1, NC)[:, c] * q2.abs().view(-1, NC)[:, c]).sum())


def test_fullsize_steps_sampled(big):
    """30 graph steps of the benchmark's configuration from rest, every step checked at the sampled rows,
    DOFs and regions."""
    torch, mesh, tp, h, rows = big["torch"], big["mesh"], big["tp"], big["h"], big["rows"]
    srcs, regions = big["srcs"], big["regions"]
    N, dt = mesh.n_nodes, tp.dt
    opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=16, tol=1e-8,
                                cert_df=3, snapshot_format=2, use_graph=1)
    # sampled regions: those of the first three sources (where the corrections are not zero) and one more
    sreg = sorted({int(regions[s.node]) for s in srcs[:3]} | {int(regions[rows.nodes[-1]])} - {-1})
    reg_nodes = np.nonzero(np.isin(regions, sreg))[0]
    reg_dofs_all = (3 * reg_nodes[:, None] + np.arange(3)).reshape(-1)
    reg_free = mesh.fixed_dof[reg_dofs_all] == 0
    reg_dofs = reg_dofs_all[reg_free]
    local = {R: i for i, R in enumerate(sreg)}           # sampled regions renumbered 0 .. len(sreg) - 1
    reg_of_dof = np.array([local[int(R)] for R in np.repeat(regions[reg_nodes], 3)[reg_free]])
    n_reg = int(regions.max()) + 1
    # DOFs read each step: the rows' support, the sampled rows, the sampled regions
    dofs = np.unique(np.concatenate([rows.sup_dofs, rows.row_dofs, reg_dofs]))
    pos = {int(d): i for i, d in enumerate(dofs)}
    sup_i = np.array([pos[int(d)] for d in rows.sup_dofs])
    row_i = np.array([pos[int(d)] for d in rows.row_dofs])
    reg_i = np.array([pos[int(d)] for d in reg_dofs])
    src_rows = [{k: int(np.nonzero(rows.row_dofs == 3 * s.node + k)[0][0]) for k in range(3)
                 if (rows.row_dofs == 3 * s.node + k).any()} for s in srcs]
    bt = fem.fem_batch_create(opts)
    buf = torch.empty(N * 3, dtype=torch.float64, device="cuda")
    fields = {}

    def read(what):
        out = np.zeros((NC, dofs.size))
        idx = torch.as_tensor(dofs, device="cuda")
        for c in range(NC):
            fem.fem_case_get(bt, c, what, N, out=buf)
            out[c] = buf[idx].cpu().numpy()
        return out

    try:
        for s in srcs:
            fem.fem_case_add(bt, h, s)
        zero = np.zeros((NC, dofs.size))
        prev = dict(u=zero, v=zero, a=zero)
        vh = [zero] * 4
        E = [[] for _ in range(NC)]
        stats = PredStats()
        for it in range(1, 31):
            st, iters, relres = fem.fem_step(bt, 1, NC)
            assert st == fem.FEM_OK and np.all(relres < opts.tol), (it, relres)
            cur = {k: read(w) for k, w in (("u", fem.FEM_FIELD_U), ("v", fem.FEM_FIELD_V), ("a", fem.FEM_FIELD_A),
                                           ("du", fem.FEM_FIELD_DU), ("b", fem.FEM_FIELD_B),
                                           ("guess", fem.FEM_FIELD_GUESS))}
            bnorm = [None] * NC
            if it % 10 == 0:
                for c in range(NC):
                    fem.fem_case_get(bt, c, fem.FEM_FIELD_B, N, out=buf)
                    bnorm[c] = float(torch.linalg.norm(buf))
            for c in range(NC):
                # b at the sampled rows: f + M (a + (4/dt + a0) v) + K (a1 v - u), from the previous state
                m_in = prev["a"][c] + (4.0 / dt + tp.a0) * prev["v"][c]
                k_in = tp.a1 * prev["v"][c] - prev["u"][c]
                b_ref = rows.M @ m_in[sup_i] + rows.K @ k_in[sup_i]
                s = srcs[c]
                for k, r in src_rows[c].items():
                    b_ref[r] += oracle.ricker(it * dt, s.f0, s.t0, s.amp) * s.direction[k]
                b_ref[~rows.row_free] = 0.0
                b_g = cur["b"][c][row_i]
                scale = np.abs(rows.M) @ np.abs(m_in[sup_i]) + np.abs(rows.K) @ np.abs(k_in[sup_i]) + np.abs(b_ref)
                assert np.all(np.abs(b_g - b_ref) <= 1e-11 * scale.max() + 1e-300), (it, c)
                # certificate at the sampled rows: |b - A du| <= tol ||b|| (the certified relative residual)
                cM = 4.0 / dt ** 2 + 2.0 * tp.a0 / dt
                cK = 1.0 + 2.0 * tp.a1 / dt
                r_rows = b_g - (cM * rows.M + cK * rows.K) @ cur["du"][c][sup_i]
                if bnorm[c] is not None:
                    assert np.abs(r_rows[rows.row_free]).max() <= opts.tol * bnorm[c], (it, c)
                # Newmark update at the sampled DOFs (a few ulps of each formula's largest term)
                du = cur["du"][c]
                u0, v0, a0 = prev["u"][c], prev["v"][c], prev["a"][c]
                u_ref, v_ref, a_ref = oracle.newmark_update(u0, v0, a0, du, dt)
                dmax = np.abs(du).max()
                scales = (max(np.abs(u0).max(), dmax), max(2.0 / dt * dmax, np.abs(v0).max()),
                          max(4.0 / dt ** 2 * dmax, 4.0 / dt * np.abs(v0).max(), np.abs(a0).max()))
                for name, ref, sc in (("u", u_ref, scales[0]), ("v", v_ref, scales[1]), ("a", a_ref, scales[2])):
                    assert np.abs(cur[name][c] - ref).max() <= 1e-13 * max(np.abs(ref).max(), sc, 1e-300), (it, c, name)
                # predictor on the sampled regions: Adams-Bashforth from the GPU's history, then the regional
                # correction against the oracle's MGS on the stored corrections
                u_ab = oracle.adams_bashforth4(prev["u"][c], [x[c] for x in vh], dt)
                du_ab = u_ab - prev["u"][c]
                y_gpu = (cur["guess"][c] - du_ab)[reg_i]
                coef, n_pairs = fem.predictor_coefficients(bt, c, n_reg, opts.s_max)
                floor = 1e-13 * max(np.abs(du_ab).max(), 1e-300)
                y_gpu, _ = guarded_correction(bt, c, y_gpu, E[c], reg_of_dof, len(sreg), coef[sreg], n_pairs, floor,
                                              stats, where=(it, c))
                check_prediction(E[c], reg_of_dof, len(sreg), y_gpu, coef[sreg], n_pairs, opts, floor, stats,
                                 where=(it, c))
                E[c].append(stored_value(du[reg_i] - du_ab[reg_i], opts.snapshot_format))
                if len(E[c]) > opts.s_max + 1:
                    E[c].pop(0)
            vh = vh[1:] + [cur["v"]]
            prev = dict(u=cur["u"], v=cur["v"], a=cur["a"])
        stats.assert_ok()
        assert stats.n > 0 and stats.elementwise > 0, (stats.n, stats.elementwise)
    finally:
        fem.fem_batch_destroy(bt)
