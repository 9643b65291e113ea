"""Graph steps (use_graph = 1): the FP32-inner step captured once as a CUDA graph with device-side control
must reproduce the eager step (same kernels, decisions moved from the host to the device).  The EBE
products accumulate with floating-point atomics, whose order varies from run to run, so two eager runs
already differ in the last bits; the graph run must stay within the same envelope: fields within a
relative 1e-7 of the eager run (both certified at 1e-8), iteration counts equal up to one per step,
and every step certified.  Covered: data-driven predictor, periodic refresh, double-float
certification, external loads, AB4, fused uneven meshes."""
import numpy as np
import pytest

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


def _run(meshes, srcs, n_steps, use_graph, loads=None, **kw):
    tp = wl.config2_time_params()
    opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=kw.pop("predictor", fem.FEM_PRED_DD),
                                s_max=8, tol=1e-8, use_graph=use_graph, **kw)
    hs = []
    for m in meshes:
        h = fem.fem_mesh_create(m, tp)
        fem.fem_mesh_set_regions(h, wl.region_map(m, 64))
        hs.append(h)
    bt = fem.fem_batch_create(opts)
    nc = len(srcs)
    try:
        for k, s in enumerate(srcs):
            fem.fem_case_add(bt, hs[k % len(hs)], s)
        its, rrs = [], []
        chunk = 7
        done = 0
        while done < n_steps:
            k = min(chunk, n_steps - done)
            if loads is not None:
                for j in range(k):          # loads are per step: one step per call
                    fem.fem_batch_set_loads(bt, loads[done + j])
                    st, it, rr = fem.fem_step(bt, 1, nc)
                    its.append(it.copy())
                    rrs.append(rr.copy())
            else:
                st, it, rr = fem.fem_step(bt, k, nc)
                its.append(it.copy())
                rrs.append(rr.copy())
            assert st == fem.FEM_OK
            done += k
        n_nodes = sum(meshes[k % len(meshes)].n_nodes for k in range(nc))
        out = {}
        for name, what in (("u", fem.FEM_FIELD_U), ("v", fem.FEM_FIELD_V), ("a", fem.FEM_FIELD_A)):
            f = np.empty(3 * n_nodes)
            fem.fem_batch_get_field(bt, what, f)
            out[name] = f
        stats = [fem.fem_case_stats(bt, c) for c in range(nc)]
        return out, np.array(its), np.array(rrs), stats
    finally:
        fem.fem_batch_destroy(bt)
        for h in hs:
            fem.fem_mesh_destroy(h)


def _same(a, b):
    for k in a[0]:
        d = np.linalg.norm(a[0][k] - b[0][k]) / max(np.linalg.norm(a[0][k]), 1e-300)
        assert d <= 1e-7, (k, d)
    assert np.abs(a[1] - b[1]).max() <= 7          # per call of up to 7 steps: at most one iteration per step
    assert abs(int(a[1].sum()) - int(b[1].sum())) <= 0.02 * a[1].sum() + 2
    assert np.all(a[2] < 1e-8) and np.all(b[2] < 1e-8)
    for s1, s2 in zip(a[3], b[3]):
        assert s1["steps"] == s2["steps"] and s1["status"] == s2["status"] == 0
        assert s1["relres"] < 1e-8 and s2["relres"] < 1e-8


@pytest.mark.parametrize("refresh_every,cert_df", [(0, 0), (9, 0), (9, 1), (9, 3)])
def test_graph_step_equals_eager_multi_rhs(torch_dev, refresh_every, cert_df):
    m = small_mesh(8, 6, 5, h=1.0 / 64)
    srcs = [wl.random_source(m, wl.rng_for(93, 0, c, 2)) for c in range(3)]
    eager = _run([m], srcs, 40, 0, refresh_every=refresh_every, cert_df=cert_df)
    graph = _run([m], srcs, 40, 1, refresh_every=refresh_every, cert_df=cert_df)
    _same(eager, graph)


def test_graph_step_equals_eager_ab4(torch_dev):
    m = small_mesh(6, 5, 4, h=1.0 / 64)
    srcs = [wl.random_source(m, wl.rng_for(94, 0, c, 2)) for c in range(2)]
    _same(_run([m], srcs, 20, 0, predictor=fem.FEM_PRED_AB4), _run([m], srcs, 20, 1, predictor=fem.FEM_PRED_AB4))


def test_graph_step_equals_eager_external_loads(torch_dev):
    m = small_mesh(6, 5, 4, h=1.0 / 64)
    srcs = [wl.random_source(m, wl.rng_for(95, 0, c, 2)) for c in range(2)]
    tp = wl.config2_time_params()
    loads = np.zeros((25, 2, 3))
    for k in range(25):
        for c, s in enumerate(srcs):
            loads[k, c] = 0.7 * wl.ricker_load(s, (k + 1) * tp.dt)     # different from the sources' own
    _same(_run([m], srcs, 25, 0, loads=loads), _run([m], srcs, 25, 1, loads=loads))


def test_graph_step_equals_eager_fused_meshes(torch_dev):
    meshes = [small_mesh(*d, h=1.0 / 64) for d in [(6, 5, 4), (9, 6, 5), (5, 7, 3)]]
    srcs = [wl.random_source(m, wl.rng_for(96, k, 0, 2)) for k, m in enumerate(meshes)]
    eager = _run(meshes, srcs, 30, 0, fuse_meshes=1, cert_df=3)
    graph = _run(meshes, srcs, 30, 1, fuse_meshes=1, cert_df=3)
    _same(eager, graph)


def test_async_field_reads_match_sync(torch_dev):
    """fem_batch_get_field_async: each step's field, staged on the device and copied on the copy stream
    while the next step runs, equals the synchronous read of that step (alternating pinned buffers), and
    fused groups read the same way."""
    torch = torch_dev
    for fuse in (0, 1):
        meshes = [small_mesh(6, 5, 4, h=1.0 / 64), small_mesh(5, 6, 3, h=1.0 / 64)] if fuse else \
            [small_mesh(6, 5, 4, h=1.0 / 64)]
        tp = wl.config2_time_params()
        opts = fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD, s_max=8, tol=1e-8,
                                    fuse_meshes=fuse)
        hs = []
        for m in meshes:
            h = fem.fem_mesh_create(m, tp)
            fem.fem_mesh_set_regions(h, wl.region_map(m, 64))
            hs.append(h)
        bt = fem.fem_batch_create(opts)
        srcs = [wl.random_source(meshes[k % len(meshes)], wl.rng_for(97, k, 0, 2)) for k in range(3)]
        try:
            for k, s in enumerate(srcs):
                fem.fem_case_add(bt, hs[k % len(hs)], s)
            n_tot = 3 * sum(meshes[k % len(meshes)].n_nodes for k in range(len(srcs)))
            bufs = [torch.empty(n_tot, dtype=torch.float64).pin_memory() for _ in range(2)]
            ref = []
            for k in range(6):
                fem.fem_step(bt, 1, len(srcs))
                sync = np.empty(n_tot)
                fem.fem_batch_get_field(bt, fem.FEM_FIELD_U, sync)
                ref.append(sync)
                fem.fem_batch_get_field_async(bt, fem.FEM_FIELD_U, bufs[k % 2])
            fem.fem_batch_sync(bt)
            assert np.array_equal(bufs[0].numpy(), ref[4]) and np.array_equal(bufs[1].numpy(), ref[5])
            assert np.abs(ref[5]).max() > 0.0
        finally:
            fem.fem_batch_destroy(bt)
            for h in hs:
                fem.fem_mesh_destroy(h)


def test_step_async_matches_step(torch_dev):
    """fem_step_async queues graph steps without host waits; after fem_batch_sync the fields match a run
    of fem_step within the run-to-run envelope, the statistics of the queued steps reach the next
    fem_step's outputs, and the status is reported by fem_batch_sync."""
    m = small_mesh(6, 5, 4, h=1.0 / 64)
    tp = wl.config2_time_params()
    srcs = [wl.random_source(m, wl.rng_for(98, 0, c, 2)) for c in range(3)]

    def run(async_steps):
        h = fem.fem_mesh_create(m, tp)
        fem.fem_mesh_set_regions(h, wl.region_map(m, 64))
        bt = fem.fem_batch_create(fem.fem_opts_default(precision=fem.FEM_FP32_INNER, predictor=fem.FEM_PRED_DD,
                                                       s_max=8, tol=1e-8))
        try:
            for s in srcs:
                fem.fem_case_add(bt, h, s)
            if async_steps:
                for _ in range(24):
                    fem.fem_step_async(bt, 1)
                assert fem.fem_batch_sync(bt) == fem.FEM_OK
                st, it, rr = fem.fem_step(bt, 1, len(srcs))     # its outputs include the queued steps
            else:
                st, it, rr = fem.fem_step(bt, 25, len(srcs))
            u = np.empty(3 * m.n_nodes * len(srcs))
            fem.fem_batch_get_field(bt, fem.FEM_FIELD_U, u)
            assert fem.fem_batch_steps(bt) == 25
            return st, it, rr, u
        finally:
            fem.fem_batch_destroy(bt)
            fem.fem_mesh_destroy(h)

    a, b = run(True), run(False)
    assert a[0] == b[0] == fem.FEM_OK
    assert np.abs(a[1] - b[1]).max() <= 25 and abs(int(a[1].sum()) - int(b[1].sum())) <= 0.02 * b[1].sum() + 2
    assert np.all(a[2] < 1e-8) and np.all(b[2] < 1e-8)
    assert np.linalg.norm(a[3] - b[3]) <= 1e-7 * np.linalg.norm(b[3])
