"""Shared test helpers: layout conversions between the library's [node][3][case] vectors and the oracle's
per-case DOF vectors, and small seeded meshes."""
import numpy as np

from paper_2409_20380_gb300 import workload as wl


def small_mesh(Hx=7, Hy=5, Hz=4, h=None, sigma=0.3, seed_mesh=11, perturb=0.0):
    h = h if h is not None else 1.0 / 8
    zt = Hz * h
    m = wl.layered_mesh(Hx, Hy, Hz, h, layer_tops=[zt / 3, 2 * zt / 3],
                        base_lame=[(8.0, 4.0), (4.0, 2.0), (2.0, 1.0)], sigma=sigma,
                        rng=wl.rng_for(90, seed_mesh, 0, 1))
    if perturb:
        rng = np.random.default_rng(seed_mesh)
        inner = wl.interior_nodes(m)
        m.xyz[inner] += perturb * h * rng.uniform(-1, 1, (inner.size, 3))
    return m


def to_cases(v, n_nodes, r):
    """[N*3*r] flat -> list of r full-length (3N) vectors."""
    a = np.asarray(v).reshape(n_nodes, 3, r)
    return [a[:, :, c].reshape(-1).copy() for c in range(r)]


def from_cases(vs, n_nodes, r):
    """list of r full-length vectors -> [N*3*r] flat."""
    out = np.zeros((n_nodes, 3, r))
    for c, v in enumerate(vs):
        out[:, :, c] = np.asarray(v).reshape(n_nodes, 3)
    return out.reshape(-1)


def random_free_vectors(mesh, r, seed=0):
    rng = np.random.default_rng(seed)
    vs = []
    for _ in range(r):
        v = rng.standard_normal(3 * mesh.n_nodes)
        v[mesh.fixed_dof == 1] = 0.0
        vs.append(v)
    return vs
