"""Whole time-history runs of the oracle on the 8x8x8-hex unit box (3072 tets, 729 nodes).

Every step must be certified at ||b - A du|| / ||b|| < 1e-8 (Algorithm 1's tolerance, Section 3.3), with
the residual recomputed here from the assembled matrix; and the data-driven predictor must lower the
iteration count against Adams-Bashforth, more so with more stored steps (the qualitative trend of
Section 3.3: 154 -> 59/51/43 iterations for s = 8/16/32)."""
import numpy as np
import pytest

import oracle
from paper_2409_20380_gb300 import workload as wl


@pytest.fixture(scope="module")
def cfg1():
    m = wl.config1_mesh()
    sysm, A = oracle.build_system(m, wl.TimeParams())
    Binv = oracle.block_jacobi_inverse(A, sysm.free)
    return m, sysm, A, Binv, wl.config1_sources(1)[0]


def _run(cfg1, predictor, s_max=16, steps=100, region_nodes=128):
    m, sysm, A, Binv, src = cfg1
    sim = oracle.CaseSimulator(sysm, A, Binv, src, predictor=predictor, s_max=s_max,
                               region_of_node=wl.region_map(m, region_nodes))
    recs = []
    for _ in range(steps):
        u_prev, v_prev, a_prev = sim.u.copy(), sim.v.copy(), sim.a.copy()
        rec = sim.step()
        f = oracle.point_force(3 * m.n_nodes, src, rec.it * sysm.dt)
        b = oracle.newmark_rhs(sysm, f, u_prev, v_prev, a_prev)[sysm.free]
        nb = np.linalg.norm(b)
        cert = np.linalg.norm(b - A @ rec.du) / nb
        assert cert < 1e-8, (rec.it, cert)
        recs.append(rec)
    return recs


def test_case_certified_and_predictor_gain(cfg1):
    ab = _run(cfg1, "ab4")
    dd4 = _run(cfg1, "dd", s_max=4)
    dd16 = _run(cfg1, "dd", s_max=16)
    n_ab = sum(r.iters for r in ab)
    n4 = sum(r.iters for r in dd4)
    n16 = sum(r.iters for r in dd16)
    assert n16 <= n4 < n_ab
    # same solution whatever the initial guess (to the certified tolerance)
    du_ab = ab[-1].du
    assert np.linalg.norm(dd16[-1].du - du_ab) < 1e-6 * np.linalg.norm(du_ab)
