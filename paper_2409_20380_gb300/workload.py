"""Seeded synthetic inputs for the time-evolution FE cases (mesh, materials, sources, regions).

This module only *generates inputs*: node coordinates, tetrahedral connectivity, per-element material
ids with their Lame parameters and density, the Dirichlet mask, Ricker point-source parameters and the
node -> region map used by the regional predictor.  It contains none of the method's arithmetic (no
element matrices, no time integration, no solver, no predictor); both the CUDA path and the CPU oracle
consume what it returns.

The workloads stand in for the paper's ground models (Section 3.1: layered ground, random impulse inputs at
surface points, bottom fixed), which are not public: a unit-spaced hex grid split into six linear tets per
hex (Kuhn/Freudenthal split along the (0,0,0)->(1,1,1) diagonal, the same in every hex, hence conforming),
horizontally layered log-normal materials (soft over stiff, like sediment over bedrock), an optional
low-velocity basin inclusion, and one Ricker-wavelet point force per case at a random interior node in a
random direction.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

# Six Kuhn tets of the unit hex: vertex chains 0 -> e_a -> e_a + e_b -> (1,1,1) for every permutation
# (a, b, c) of the axes.  Corner index bits: bit0 = x, bit1 = y, bit2 = z.
_KUHN = []
for perm in itertools.permutations(range(3)):
    c0 = 0
    c1 = c0 | (1 << perm[0])
    c2 = c1 | (1 << perm[1])
    c3 = 7
    # parity of the permutation decides orientation; odd permutations swap the last two vertices
    inv = sum(1 for i in range(3) for j in range(i + 1, 3) if perm[i] > perm[j])
    _KUHN.append((c0, c1, c3, c2) if inv % 2 else (c0, c1, c2, c3))
KUHN_TETS = np.array(_KUHN, dtype=np.int64)  # [6][4] corner ids


@dataclasses.dataclass
class Mesh:
    """A tet4 mesh with per-element materials and a per-DOF Dirichlet mask."""
    xyz: np.ndarray          # [N][3] float64
    conn: np.ndarray         # [E][4] int32, positively oriented
    mat_id: np.ndarray       # [E] int32
    lam_mu_rho: np.ndarray   # [n_mat][3] float64
    fixed_dof: np.ndarray    # [3N] uint8 (1 = Dirichlet, value 0)
    dims: tuple              # (Hx, Hy, Hz) hex counts
    h: float                 # hex edge length

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]

    @property
    def n_elems(self) -> int:
        return self.conn.shape[0]


@dataclasses.dataclass
class Source:
    """Ricker point force: amp * (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2) along `direction`."""
    node: int
    direction: np.ndarray    # [3] unit vector
    f0: float
    t0: float
    amp: float = 1.0


@dataclasses.dataclass
class TimeParams:
    dt: float = 0.01
    beta: float = 0.25
    gamma: float = 0.5
    a0: float = 0.01         # Rayleigh mass-proportional damping
    a1: float = 0.001        # Rayleigh stiffness-proportional damping


def rng_for(config: int, mesh_id: int = 0, case_id: int = 0, stream: int = 0) -> np.random.Generator:
    """Independent reproducible stream per (config, mesh, case, purpose)."""
    return np.random.default_rng(np.random.SeedSequence([20380, config, mesh_id, case_id, stream]))


def _morton3(ix, iy, iz, bits=21):
    code = np.zeros(ix.shape, dtype=np.uint64)
    for b in range(bits):
        code |= ((ix >> b) & 1).astype(np.uint64) << np.uint64(3 * b)
        code |= ((iy >> b) & 1).astype(np.uint64) << np.uint64(3 * b + 1)
        code |= ((iz >> b) & 1).astype(np.uint64) << np.uint64(3 * b + 2)
    return code


def structured_grid(Hx: int, Hy: int, Hz: int, h: float):
    """Node coordinates and Kuhn-split connectivity of an Hx x Hy x Hz hex grid.

    Nodes are numbered in Morton (Z-curve) order of their integer grid position and elements hex by hex
    in Morton order of the hex, the six tets of a hex consecutive -- the locality-preserving numbering a
    mesher's reordering step would hand to an FE solver.
    """
    nx, ny, nz = Hx + 1, Hy + 1, Hz + 1
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    node_order = np.argsort(_morton3(i, j, k), kind="stable")
    new_id = np.empty(node_order.size, dtype=np.int64)
    new_id[node_order] = np.arange(node_order.size)
    xyz = np.stack([i[node_order] * h, j[node_order] * h, k[node_order] * h], axis=1).astype(np.float64)
    hk, hj, hi = np.meshgrid(np.arange(Hz), np.arange(Hy), np.arange(Hx), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    hex_order = np.argsort(_morton3(hi, hj, hk), kind="stable")
    base = (hi + nx * (hj + ny * hk))[hex_order].astype(np.int64)        # [H] lower corner (lexicographic)
    corner_off = np.array([(c & 1) + nx * (((c >> 1) & 1) + ny * ((c >> 2) & 1)) for c in range(8)],
                          dtype=np.int64)
    conn_lex = base[:, None, None] + corner_off[KUHN_TETS][None, :, :]   # [H][6][4]
    return xyz, new_id[conn_lex].reshape(-1, 4).astype(np.int32)


def _element_centroid_z(xyz, conn):
    return xyz[conn, 2].mean(axis=1)


def layered_mesh(Hx, Hy, Hz, h, layer_tops, base_lame, rho=1.0, sigma=0.0, rng=None, basin=None) -> Mesh:
    """Horizontally layered materials assigned by element centroid depth.

    layer_tops: increasing z-coordinates of the layer interfaces from the bottom (len = n_layers - 1).
    base_lame:  (lambda, mu) per layer, listed bottom -> top.
    sigma:      log-normal scatter: each layer's (lambda, mu) times exp(sigma * xi), xi ~ N(0,1), one xi per
                layer shared by lambda and mu (Poisson ratio kept).
    basin:      optional (cx, cy, ax, ay, az, mu_factor): half-ellipsoid at the top surface whose elements
                get mu scaled by mu_factor (one extra material per layer it cuts).
    """
    xyz, conn = structured_grid(Hx, Hy, Hz, h)
    zc = _element_centroid_z(xyz, conn)
    layer = np.searchsorted(np.asarray(layer_tops, dtype=np.float64), zc, side="right").astype(np.int32)
    n_layers = len(base_lame)
    lmr = []
    for li in range(n_layers):
        lam, mu = base_lame[li]
        if sigma > 0.0:
            s = math.exp(sigma * rng.standard_normal())
            lam, mu = lam * s, mu * s
        lmr.append((lam, mu, rho))
    mat_id = layer.copy()
    if basin is not None:
        cx, cy, ax, ay, az, fac = basin
        ztop = Hz * h
        cen = xyz[conn].mean(axis=1)
        inside = ((cen[:, 0] - cx) / ax) ** 2 + ((cen[:, 1] - cy) / ay) ** 2 + ((cen[:, 2] - ztop) / az) ** 2 < 1.0
        for li in range(n_layers):
            lam, mu, r = lmr[li]
            lmr.append((lam, mu * fac, r))
        mat_id = np.where(inside, layer + n_layers, layer).astype(np.int32)
    fixed = np.zeros(xyz.shape[0] * 3, dtype=np.uint8)
    bottom = np.nonzero(xyz[:, 2] == 0.0)[0]
    fixed[3 * bottom] = 1
    fixed[3 * bottom + 1] = 1
    fixed[3 * bottom + 2] = 1
    return Mesh(xyz=xyz, conn=conn, mat_id=mat_id, lam_mu_rho=np.asarray(lmr, dtype=np.float64),
                fixed_dof=fixed, dims=(Hx, Hy, Hz), h=h)


def interior_nodes(mesh: Mesh) -> np.ndarray:
    """Nodes strictly inside the box (on no boundary face)."""
    Hx, Hy, Hz = mesh.dims
    q = np.rint(mesh.xyz / mesh.h).astype(np.int64)
    m = ((q[:, 0] > 0) & (q[:, 0] < Hx) & (q[:, 1] > 0) & (q[:, 1] < Hy) & (q[:, 2] > 0) & (q[:, 2] < Hz))
    return np.nonzero(m)[0]


def random_source(mesh: Mesh, rng: np.random.Generator, f0=None, f0_range=(2.0, 8.0)) -> Source:
    nodes = interior_nodes(mesh)
    node = int(nodes[rng.integers(0, nodes.size)])
    d = rng.standard_normal(3)
    d = d / np.linalg.norm(d)
    if f0 is None:
        f0 = float(rng.uniform(*f0_range))
    return Source(node=node, direction=d, f0=float(f0), t0=1.2 / float(f0), amp=1.0)


@dataclasses.dataclass
class Impulses:
    """Random impulse inputs of one case: at node nodes[k], the force forces[k] during time step steps[k]
    (steps >= 1), nothing at other steps."""
    nodes: np.ndarray        # [n] int32
    steps: np.ndarray        # [n] int32
    forces: np.ndarray       # [n][3] float64


def surface_nodes(mesh: Mesh) -> np.ndarray:
    """Free nodes of the top face (z = Hz h)."""
    Hz = mesh.dims[2]
    q = np.rint(mesh.xyz[:, 2] / mesh.h).astype(np.int64)
    free = mesh.fixed_dof.reshape(-1, 3).max(axis=1) == 0
    return np.nonzero((q == Hz) & free)[0]


def random_impulses(mesh: Mesh, rng: np.random.Generator, n_points: int, last_step: int) -> Impulses:
    """Impulses at n_points distinct random surface nodes, each once, at a random step in [1, last_step], with
    an amplitude ~ N(0, 1) along a random unit direction."""
    cand = surface_nodes(mesh)
    nodes = rng.choice(cand, size=min(n_points, cand.size), replace=False).astype(np.int32)
    n = nodes.size
    steps = rng.integers(1, last_step + 1, size=n).astype(np.int32)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    forces = rng.standard_normal(n)[:, None] * d
    return Impulses(nodes=nodes, steps=steps, forces=forces)


def side_faces(mesh: Mesh) -> np.ndarray:
    """[n][3] int32 node triples of the element faces lying in the four vertical sides of the box (x = 0,
    x = Lx, y = 0, y = Ly): where the workloads with absorbing sides put them (the bottom is fixed, the top
    free)."""
    Hx, Hy, _ = mesh.dims
    q = np.rint(mesh.xyz / mesh.h).astype(np.int64)
    out = []
    for k in range(4):
        tri = np.delete(mesh.conn, k, axis=1)                       # [E][3] faces opposite corner k
        qt = q[tri]                                                 # [E][3][3]
        on = np.zeros(tri.shape[0], dtype=bool)
        for ax, val in ((0, 0), (0, Hx), (1, 0), (1, Hy)):
            on |= np.all(qt[:, :, ax] == val, axis=1)
        out.append(tri[on])
    return np.ascontiguousarray(np.concatenate(out, axis=0), dtype=np.int32)


def region_map(mesh: Mesh, region_nodes: int = 1024) -> np.ndarray:
    """Node -> region id: free nodes in Morton order of their grid position, cut into runs of
    `region_nodes`; nodes whose three DOFs are all fixed get -1 (they carry no unknowns)."""
    q = np.rint(mesh.xyz / mesh.h).astype(np.int64)
    code = _morton3(q[:, 0], q[:, 1], q[:, 2])
    free_node = mesh.fixed_dof.reshape(-1, 3).min(axis=1) == 0
    order = np.argsort(code, kind="stable")
    order = order[free_node[order]]
    reg = np.full(mesh.n_nodes, -1, dtype=np.int32)
    reg[order] = (np.arange(order.size) // region_nodes).astype(np.int32)
    return reg


# --------------------------------------------------------------------------------------------------------
# The benchmark workloads.  Sizes follow the five configurations the method is exercised on; every
# random draw is seeded by (config, mesh, case).
# --------------------------------------------------------------------------------------------------------

def config1_mesh() -> Mesh:
    """Unit box, 8^3 hexes, h = 1/8: two layers, (4,2) below z = 0.5 and (2,1) above, rho = 1."""
    return layered_mesh(8, 8, 8, 1.0 / 8, layer_tops=[0.5], base_lame=[(4.0, 2.0), (2.0, 1.0)])


def config1_sources(n_cases: int = 1):
    m = config1_mesh()
    return [random_source(m, rng_for(1, 0, c), f0=5.0) for c in range(n_cases)]


def config2_mesh(Hx=64, Hy=64, Hz=32, mesh_id=0, h=1.0 / 64) -> Mesh:
    """Three equal layers, base (8,4)/(4,2)/(2,1) bottom -> top, log-normal sigma = 0.3 per layer."""
    zt = Hz * h
    return layered_mesh(Hx, Hy, Hz, h, layer_tops=[zt / 3.0, 2.0 * zt / 3.0],
                        base_lame=[(8.0, 4.0), (4.0, 2.0), (2.0, 1.0)], sigma=0.3,
                        rng=rng_for(2, mesh_id, 0, 1))


def config2_time_params() -> TimeParams:
    """dt = 0.004 for the h = 1/64 meshes: S-wave Courant number c_s dt / h = 0.36-0.7 and 12-30 steps per
    period over the sources' band, the regime of the paper's runs (dt = 0.005 with 2.5 m elements), where the
    Adams-Bashforth initial error is O(1e-3).  Damping as in the unit-box configuration."""
    return TimeParams(dt=0.004, a0=0.01, a1=0.001)


def config2_sources(mesh: Mesh, n_cases: int = 16, config: int = 2, first_case: int = 0):
    return [random_source(mesh, rng_for(config, 0, first_case + c, 2)) for c in range(n_cases)]


def config3_dims(n_meshes: int = 64):
    rng = rng_for(3, 0, 0, 3)
    return [(int(rng.integers(24, 65)), int(rng.integers(24, 65)), int(rng.integers(24, 49)))
            for _ in range(n_meshes)]


def config3_mesh(mesh_id: int, dims) -> Mesh:
    Hx, Hy, Hz = dims
    h = 1.0 / 64
    zt = Hz * h
    return layered_mesh(Hx, Hy, Hz, h, layer_tops=[zt / 3.0, 2.0 * zt / 3.0],
                        base_lame=[(8.0, 4.0), (4.0, 2.0), (2.0, 1.0)], sigma=0.3,
                        rng=rng_for(3, mesh_id, 0, 1))


def config4_mesh(Hx=256, Hy=256, Hz=128, h=1.0 / 64) -> Mesh:
    """Five seeded layers plus a half-ellipsoid low-velocity basin (mu x 0.3) at the surface.

    The full configuration is the 256 x 256 x 128 hex box (4 x 4 x 2, 50,331,648 tets, 8,520,321 nodes).  Smaller
    dims give the same recipe scaled to the box: layer interfaces at the same depth fractions, the basin's
    centre at the same fractions of the top face and its semi-axes scaled by the box's extent (by Lx / 4,
    Ly / 4 and Lz / 2), with the same seeded draws."""
    rng = rng_for(4, 0, 0, 1)
    zt = Hz * h
    tops = [zt * f for f in (0.2, 0.4, 0.6, 0.8)]
    base = [(16.0, 8.0), (12.0, 6.0), (8.0, 4.0), (4.0, 2.0), (2.0, 1.0)]
    Lx, Ly = Hx * h, Hy * h
    basin = (rng.uniform(0.25 * Lx, 0.75 * Lx), rng.uniform(0.25 * Ly, 0.75 * Ly),
             rng.uniform(0.5, 1.5) * Lx / 4.0, rng.uniform(0.5, 1.5) * Ly / 4.0, rng.uniform(0.3, 1.0) * zt / 2.0,
             0.3)
    return layered_mesh(Hx, Hy, Hz, h, layer_tops=tops, base_lame=base, sigma=0.3, rng=rng, basin=basin)


def config4_time_params() -> TimeParams:
    """The large box has the medium meshes' spacing h = 1/64, so the same dt = 0.004 and damping."""
    return TimeParams(dt=0.004, a0=0.01, a1=0.001)


def config4_sources(mesh: Mesh, n_cases: int = 8, first_case: int = 0):
    """Ricker point forces at seeded interior nodes, f0 ~ U[2, 8], seeded unit directions."""
    return [random_source(mesh, rng_for(4, 0, first_case + c, 2)) for c in range(n_cases)]


def ricker_load(src: Source, t: float) -> np.ndarray:
    """Point-force vector [3] that source `src` applies at time t (a case's load input at its node)."""
    arg = (math.pi * src.f0 * (t - src.t0)) ** 2
    return src.amp * (1.0 - 2.0 * arg) * math.exp(-arg) * np.asarray(src.direction, dtype=np.float64)


# --------------------------------------------------------------------------------------------------------
# Learned proposal: initial network weights (seeded draws only; the network itself lives elsewhere).
# --------------------------------------------------------------------------------------------------------

MLP_LAYERS = (64, 256, 256, 32)


def mlp_init_weights(seed: int = 0) -> np.ndarray:
    """He-uniform draws for the 64-256-256-32 network, flat in the order W1 [256][64], b1 [256],
    W2 [256][256], b2 [256], W3 [32][256], b3 [32]: W ~ U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)), b = 0."""
    rng = np.random.default_rng(np.random.SeedSequence([20380, 5, 0, seed, 9]))
    parts = []
    for i in range(3):
        fan_in, fan_out = MLP_LAYERS[i], MLP_LAYERS[i + 1]
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)


def config5_sources(mesh: Mesh, n_train: int = 200, n_eval: int = 32):
    """Training and held-out sources on the medium mesh; the two seed ranges are disjoint."""
    train = [random_source(mesh, rng_for(5, 0, c, 2)) for c in range(n_train)]
    held = [random_source(mesh, rng_for(5, 0, 100000 + c, 2)) for c in range(n_eval)]
    return train, held


# --------------------------------------------------------------------------------------------------------
# 10-node tetrahedra (the paper's element, Section 3.1): the tet4 mesh with a node added at the midpoint of
# every edge.  Local order: corners 0-3, then the edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).
# --------------------------------------------------------------------------------------------------------
TET10_EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))


@dataclasses.dataclass
class Mesh10:
    """A straight-sided tet10 mesh: corners of the tet4 mesh plus edge midpoints."""
    xyz: np.ndarray          # [N10][3] float64 (the tet4 nodes first, then one node per edge)
    conn: np.ndarray         # [E][10] int32
    mat_id: np.ndarray       # [E] int32
    lam_mu_rho: np.ndarray   # [n_mat][3] float64
    fixed_dof: np.ndarray    # [3 N10] uint8 (an edge node is fixed where both ends are)

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]

    @property
    def n_elems(self) -> int:
        return self.conn.shape[0]


def tet10_mesh(mesh: Mesh) -> Mesh10:
    """Mid-edge nodes for every distinct edge of the tet4 mesh (numbered after the corner nodes in order of
    first appearance)."""
    conn4 = mesh.conn.astype(np.int64)
    E, N = conn4.shape[0], mesh.n_nodes
    pairs = np.stack([np.stack([conn4[:, a], conn4[:, b]], axis=1) for a, b in TET10_EDGES], axis=1)   # [E][6][2]
    lo, hi = pairs.min(axis=2), pairs.max(axis=2)
    key = (lo * N + hi).reshape(-1)
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")            # edges numbered by first appearance
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    edge_id = rank[inv].reshape(E, 6)
    ulo, uhi = (uniq // N)[order], (uniq % N)[order]
    xyz = np.concatenate([mesh.xyz, 0.5 * (mesh.xyz[ulo] + mesh.xyz[uhi])], axis=0)
    conn = np.concatenate([conn4, N + edge_id], axis=1).astype(np.int32)
    f4 = mesh.fixed_dof.reshape(N, 3)
    fe = f4[ulo] & f4[uhi]
    fixed = np.concatenate([f4, fe], axis=0).reshape(-1).astype(np.uint8)
    return Mesh10(np.ascontiguousarray(xyz), np.ascontiguousarray(conn), mesh.mat_id.copy(),
                  mesh.lam_mu_rho.copy(), np.ascontiguousarray(fixed))


def tet10_mesh_ordered(mesh: Mesh) -> tuple[Mesh10, np.ndarray]:
    """tet10_mesh(mesh) with all nodes, corner and edge alike, renumbered in Morton order of their position on
    the grid of spacing h/2 (a mesher's reordering step; it makes the predictor's regions contiguous node
    ranges).  Returns the mesh and the new id of each node of `mesh`."""
    m10 = tet10_mesh(mesh)
    q = np.rint(2.0 * m10.xyz / mesh.h).astype(np.int64)
    order = np.argsort(_morton3(q[:, 0], q[:, 1], q[:, 2]), kind="stable")    # old id at each new position
    new_id = np.empty_like(order)
    new_id[order] = np.arange(order.size)
    fixed = m10.fixed_dof.reshape(-1, 3)[order].reshape(-1)
    out = Mesh10(np.ascontiguousarray(m10.xyz[order]), np.ascontiguousarray(new_id[m10.conn].astype(np.int32)),
                 m10.mat_id, m10.lam_mu_rho, np.ascontiguousarray(fixed))
    return out, new_id[:mesh.n_nodes]


def region_map10(m10: Mesh10, h: float, region_nodes: int = 1024) -> np.ndarray:
    """region_map for a tet10 mesh: free nodes in Morton order of their position on the grid of spacing h/2,
    cut into runs of `region_nodes`; fully fixed nodes get -1."""
    q = np.rint(2.0 * m10.xyz / h).astype(np.int64)
    code = _morton3(q[:, 0], q[:, 1], q[:, 2])
    free_node = m10.fixed_dof.reshape(-1, 3).min(axis=1) == 0
    order = np.argsort(code, kind="stable")
    order = order[free_node[order]]
    reg = np.full(m10.n_nodes, -1, dtype=np.int32)
    reg[order] = (np.arange(order.size) // region_nodes).astype(np.int32)
    return reg
