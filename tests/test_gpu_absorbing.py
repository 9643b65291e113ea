"""Absorbing side boundaries (Lysmer-Kuhlemeyer dashpots on listed faces) and random surface impulses on the GPU
against the FP64 oracle (oracle/fem_oracle.py: lysmer_dashpots, impulse_force, build_system with
absorbing_faces).

* pcg_solve on A = cM M + cK K + (2/dt) C_b: the certified residual recomputed with the oracle's A, and the
  iteration count of the oracle's Algorithm 1 with the same block-Jacobi preconditioner (within one).
* fem_step with impulse cases on a mesh with absorbing sides, step by step: b against the oracle's right-hand
  side (C = a0 M + a1 K + C_b, f = the step's impulses), every increment certified with the oracle's A, the
  Newmark update; FP64 solver, and FP32-inner solver with graph steps and the data-driven predictor.
* Argument errors: a face that is not a boundary face, impulses before step 1."""
import numpy as np
import pytest

import oracle
from paper_2409_20380_gb300 import build, fem
from paper_2409_20380_gb300 import workload as wl
from helpers import from_cases, small_mesh, to_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    build.build()
    fem.lib()
    return torch


def _interior_face(m):
    """A face shared by two elements."""
    seen = set()
    for e in range(m.n_elems):
        nd = [int(v) for v in m.conn[e]]
        for k in range(4):
            key = tuple(sorted(nd[:k] + nd[k + 1:]))
            if key in seen:
                return np.array(key, dtype=np.int32)
            seen.add(key)
    raise AssertionError("no interior face")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pcg_with_dashpots_matches_oracle(torch_dev, precision):
    torch = torch_dev
    m = small_mesh(8, 6, 5, h=1.0 / 16)
    tp = wl.TimeParams(dt=0.01)
    faces = wl.side_faces(m)
    sysm, A = oracle.build_system(m, tp, absorbing_faces=faces)
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    h = fem.fem_mesh_create(m, tp)
    try:
        fem.fem_mesh_set_absorbing(h, faces)
        r = 4
        rng = np.random.default_rng(7)
        bs = [rng.standard_normal(3 * m.n_nodes) * (m.fixed_dof == 0) for _ in range(r)]
        b = torch.tensor(from_cases(bs, m.n_nodes, r), device="cuda")
        x = torch.zeros_like(b)
        opts = fem.fem_opts_default(tol=1e-10, precision=fem.FEM_FP64 if precision == "fp64" else fem.FEM_FP32_INNER)
        _, iters, relres = fem.pcg_solve(h, b, x, r, opts)
        xs = to_cases(x.cpu().numpy(), m.n_nodes, r)
        for c in range(r):
            bc = bs[c][sysm.free]
            cert = np.linalg.norm(bc - A @ xs[c][sysm.free]) / np.linalg.norm(bc)
            assert cert < 1e-10, (c, cert)
            if precision == "fp64":
                ref = oracle.block_jacobi_cg(A, Binv, bc, np.zeros_like(bc), eps=1e-10)
                assert abs(int(iters[c]) - ref.iters) <= 1, (c, iters[c], ref.iters)
        # the dashpots are part of A: without them the same solution is not certified
        sys0, A0 = oracle.build_system(m, tp)
        c0 = np.linalg.norm(bs[0][sysm.free] - A0 @ xs[0][sysm.free]) / np.linalg.norm(bs[0][sysm.free])
        assert c0 > 1e-6
        # removing them restores the plain system
        fem.fem_mesh_set_absorbing(h, None)
        x.zero_()
        fem.pcg_solve(h, b, x, r, opts)
        xs = to_cases(x.cpu().numpy(), m.n_nodes, r)
        c1 = np.linalg.norm(bs[0][sysm.free] - A0 @ xs[0][sysm.free]) / np.linalg.norm(bs[0][sysm.free])
        assert c1 < 1e-10
        with pytest.raises(fem.FemError) as ei:
            fem.fem_mesh_set_absorbing(h, _interior_face(m)[None, :])
        assert ei.value.status == fem.FEM_ERR_ARG
    finally:
        fem.fem_mesh_destroy(h)


def _impulse_cases(m, n_cases, seed):
    return [wl.random_impulses(m, wl.rng_for(seed, 0, c, 4), n_points=12, last_step=10) for c in range(n_cases)]


@pytest.mark.parametrize("mode", ["fp64_ab4", "mixed_dd_graph", "mixed_dd_eager"])
def test_step_with_impulses_and_absorbing_sides(torch_dev, mode):
    m = small_mesh(8, 7, 6, h=1.0 / 32)
    tp = wl.TimeParams(dt=0.004)
    faces = wl.side_faces(m)
    sysm, A = oracle.build_system(m, tp, absorbing_faces=faces)
    imps = _impulse_cases(m, 3, 61)
    N = m.n_nodes
    if mode == "fp64_ab4":
        opts = fem.fem_opts_default(tol=1e-8)
    else:
        opts = fem.fem_opts_default(tol=1e-8, precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=8,
                                    use_graph=1 if mode == "mixed_dd_graph" else 0, refresh_every=7)
    h = fem.fem_mesh_create(m, tp)
    fem.fem_mesh_set_absorbing(h, faces)
    fem.fem_mesh_set_regions(h, wl.region_map(m, 64))
    bt = fem.fem_batch_create(opts)
    try:
        for imp in imps:
            fem.fem_case_add_impulses(bt, h, imp)
        st = [dict(u=np.zeros(3 * N), v=np.zeros(3 * N), a=np.zeros(3 * N)) for _ in imps]
        n_steps = 24
        energy_ok = 0
        for it in range(1, n_steps + 1):
            stat, iters, relres = fem.fem_step(bt, 1, len(imps))
            for c, imp in enumerate(imps):
                S = st[c]
                u = fem.fem_case_get(bt, c, fem.FEM_FIELD_U, N)
                v = fem.fem_case_get(bt, c, fem.FEM_FIELD_V, N)
                a = fem.fem_case_get(bt, c, fem.FEM_FIELD_A, N)
                du = fem.fem_case_get(bt, c, fem.FEM_FIELD_DU, N)
                b = fem.fem_case_get(bt, c, fem.FEM_FIELD_B, N)
                f = oracle.impulse_force(3 * N, imp, it)
                b_ref = oracle.newmark_rhs(sysm, f, S["u"], S["v"], S["a"])
                b_ref[m.fixed_dof == 1] = 0.0
                nb = np.linalg.norm(b_ref)
                if nb == 0.0:
                    assert np.abs(b).max() == 0.0 and np.abs(du).max() == 0.0
                else:
                    assert np.linalg.norm(b - b_ref) <= 1e-11 * nb, (it, c, np.linalg.norm(b - b_ref) / nb)
                    cert = np.linalg.norm(b_ref[sysm.free] - A @ du[sysm.free]) / nb
                    assert cert < 1e-8, (it, c, cert)
                u_ref, v_ref, a_ref = oracle.newmark_update(S["u"], S["v"], S["a"], du, tp.dt)
                dmax = np.abs(du).max()
                for got, ref, sc in ((u, u_ref, max(np.abs(S["u"]).max(), dmax)),
                                     (v, v_ref, max(2 / tp.dt * dmax, np.abs(S["v"]).max())),
                                     (a, a_ref, max(4 / tp.dt ** 2 * dmax, 4 / tp.dt * np.abs(S["v"]).max(),
                                                    np.abs(S["a"]).max()))):
                    assert np.abs(got - ref).max() <= 1e-13 * max(np.abs(ref).max(), sc, 1e-300), (it, c)
                S["u"], S["v"], S["a"] = u, v, a
                energy_ok += 1
        assert energy_ok == n_steps * len(imps)
    finally:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)


def test_impulse_arguments(torch_dev):
    m = small_mesh(4, 4, 3)
    h = fem.fem_mesh_create(m, wl.TimeParams())
    bt = fem.fem_batch_create(fem.fem_opts_default())
    try:
        bad = wl.Impulses(nodes=np.array([1], dtype=np.int32), steps=np.array([0], dtype=np.int32),
                          forces=np.ones((1, 3)))
        with pytest.raises(fem.FemError) as ei:
            fem.fem_case_add_impulses(bt, h, bad)
        assert ei.value.status == fem.FEM_ERR_ARG
        bad = wl.Impulses(nodes=np.array([m.n_nodes], dtype=np.int32), steps=np.array([1], dtype=np.int32),
                          forces=np.ones((1, 3)))
        with pytest.raises(fem.FemError) as ei:
            fem.fem_case_add_impulses(bt, h, bad)
        assert ei.value.status == fem.FEM_ERR_ARG
    finally:
        fem.fem_batch_destroy(bt)
        fem.fem_mesh_destroy(h)
