"""FP64 CPU oracle for the time-evolution FE solve -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this module.  It shares no
code with the CUDA path: it builds the global matrices by plain assembly of textbook tet4 element matrices
(B^T D B in Voigt notation and the consistent mass), eliminates Dirichlet DOFs from a scipy CSR matrix,
and runs the paper's algorithms literally, one case at a time:

* Section 3.1, Eq. (GE:DIS) and Eq. (timestep): Newmark-beta (beta = 1/4, gamma = 1/2) time stepping of the
  linear elastodynamics equation with Rayleigh damping C = a0 M + a1 K.
* Algorithm 1: conjugate gradients with a 3x3 block-Jacobi preconditioner.
* Section 3.2: the Adams-Bashforth predictor of the initial solution.
* Section 3.2, last paragraphs: the data-driven predictor -- modified Gram-Schmidt of the stored inputs X,
  P = X U orthonormal, c = P^T x, y = Y U c -- applied independently per region.

Readings of the paper where it is silent or garbled (each one is listed with its reason in the design notes):
  R1  A = 4M/dt^2 + 2C/dt + K (Newmark beta = 1/4, gamma = 1/2); the printed Eq. (GE:DIS) drops the factors.
  R2  The unknown is the increment du = u^it - u^{it-1}; b = f^it - K u^{it-1} + C v^{it-1}
      + M (a^{it-1} + 4/dt v^{it-1}).  The tolerance of Algorithm 1 applies to this b.
  R3  a^it = -a^{it-1} - 4/dt v^{it-1} + 4/dt^2 du (minus sign; average-acceleration Newmark).
  R4  C = a0 M + a1 K (Rayleigh).            R5  consistent tet4 mass rho V/20 (1 + delta_ab) I3.
  R8  predictor pairs x_j = e^{j-1}, y_j = e^j with e = u - u_AB; query x = e^{it-1}; k < s pairs early on.
  R9  MGS drops column j when its orthogonalised norm <= tau * its original norm.
  R11 rest initial conditions; velocities before step 1 are zero in the Adams-Bashforth formula.
  R12 Ricker source w(t) = amp (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t = it * dt.
  R13 ||b|| = 0 gives du = 0 with 0 iterations.
  R14 on exit Algorithm 1's recursive residual is replaced by the true residual; iteration continues
      while that true residual is above the tolerance (up to maxit).
  R22 absorbing side boundaries (Section 3.1 names them without a form): viscous dashpots of Lysmer and
      Kuhlemeyer, traction t = -rho (c_p (v.n) n + c_s (v - (v.n) n)) on the boundary faces the caller lists,
      lumped to the face's corners (a third of the face's area each).  They add the node-block matrix C_b to
      the damping: C = a0 M + a1 K + C_b.
  R23 the paper's random inputs (impulses with random amplitudes and uniform spectra, in random directions,
      at randomly selected surface points): each point receives one force impulse during one time step, a
      random amplitude times a random unit direction, at a random step (a one-step pulse has a flat spectrum
      up to the step's Nyquist frequency).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

# --------------------------------------------------------------------------------------------------------
# Element matrices (Section 3.1: linear elasticity, Eq. GE:ORG, discretised with tetrahedral elements).
# The paper uses 10-node tets; the workloads here use 4-node tets (12 x 12 element matrices).
# --------------------------------------------------------------------------------------------------------


def tet4_shape_gradients(P: np.ndarray):
    """P: [E][4][3] vertex coordinates.  Returns (grad [E][4][3], volume [E]).

    x = x0 + J xi with J = [x1-x0, x2-x0, x3-x0] (columns); N_a = xi_a (a = 1..3), N_0 = 1 - sum xi, so
    grad N_a is row a of J^{-1} and grad N_0 = -(sum of the others).  Volume = det(J) / 6.
    """
    J = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)   # [E][3][3]
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                                            # rows = grad N_1..3
    g = np.empty((P.shape[0], 4, 3))
    g[:, 1:, :] = Jinv
    g[:, 0, :] = -Jinv.sum(axis=1)
    return g, detJ / 6.0


def strain_displacement(g: np.ndarray) -> np.ndarray:
    """Voigt B matrix [E][6][12]; strain order (xx, yy, zz, yz, xz, xy) with engineering shear."""
    E = g.shape[0]
    B = np.zeros((E, 6, 12))
    for a in range(4):
        gx, gy, gz = g[:, a, 0], g[:, a, 1], g[:, a, 2]
        c = 3 * a
        B[:, 0, c + 0] = gx
        B[:, 1, c + 1] = gy
        B[:, 2, c + 2] = gz
        B[:, 3, c + 1] = gz
        B[:, 3, c + 2] = gy
        B[:, 4, c + 0] = gz
        B[:, 4, c + 2] = gx
        B[:, 5, c + 0] = gy
        B[:, 5, c + 1] = gx
    return B


def isotropic_D(lam: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Voigt elasticity matrix [E][6][6] of an isotropic material."""
    E = lam.shape[0]
    D = np.zeros((E, 6, 6))
    for i in range(3):
        for j in range(3):
            D[:, i, j] = lam
        D[:, i, i] = lam + 2.0 * mu
        D[:, 3 + i, 3 + i] = mu
    return D


def tet4_element_matrices(xyz, conn, mat_id, lam_mu_rho):
    """Stiffness K_e = V B^T D B and consistent mass M_e = rho V / 20 (1 + delta_ab) (x) I3 (R5).

    Returns (Ke [E][12][12], Me [E][12][12]); local DOF order 3a + i (node a, direction i)."""
    P = xyz[conn]                                    # [E][4][3]
    g, V = tet4_shape_gradients(P)
    props = lam_mu_rho[mat_id]
    lam, mu, rho = props[:, 0], props[:, 1], props[:, 2]
    B = strain_displacement(g)
    D = isotropic_D(lam, mu)
    DB = np.einsum("ekl,elj->ekj", D, B)
    Ke = V[:, None, None] * np.einsum("eki,ekj->eij", B, DB)
    mass_pattern = (np.ones((4, 4)) + np.eye(4)) / 20.0
    Me = (rho * V)[:, None, None] * np.kron(mass_pattern, np.eye(3))[None, :, :]
    return Ke, Me


def assemble(xyz, conn, mat_id, lam_mu_rho, chunk=200000):
    """Global CSR M and K (3N x 3N) by summing element matrices into rows/cols 3*node + i."""
    N = xyz.shape[0]
    n = 3 * N
    Ms, Ks = [], []
    for s in range(0, conn.shape[0], chunk):
        c = conn[s:s + chunk]
        Ke, Me = tet4_element_matrices(xyz, c, mat_id[s:s + chunk], lam_mu_rho)
        dof = (3 * c[:, :, None].astype(np.int64) + np.arange(3)[None, None, :]).reshape(-1, 12)
        rows = np.broadcast_to(dof[:, :, None], Ke.shape).ravel()
        cols = np.broadcast_to(dof[:, None, :], Ke.shape).ravel()
        Ks.append(sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr())
        Ms.append(sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(n, n)).tocsr())
    K = Ks[0]
    M = Ms[0]
    for k in Ks[1:]:
        K = K + k
    for m in Ms[1:]:
        M = M + m
    return M.tocsr(), K.tocsr()


# --------------------------------------------------------------------------------------------------------
# The implicit Newmark system (Section 3.1, Eq. GE:DIS / timestep, readings R1-R4).
# --------------------------------------------------------------------------------------------------------


def lysmer_dashpots(xyz, conn, mat_id, lam_mu_rho, faces):
    """R22: the 3N x 3N dashpot matrix C_b (a symmetric 3 x 3 block per node) of the absorbing boundary faces
    [n][3] (node triples).  Each face must be a face of exactly one element; its outward unit normal n points
    away from that element's fourth node; with the element's (lambda, mu, rho), c_p = sqrt((lambda + 2 mu) /
    rho), c_s = sqrt(mu / rho), each of the face's corners gets (area / 3) rho (c_p n n^T + c_s (I - n n^T))."""
    N = xyz.shape[0]
    owner = {}
    for e in range(conn.shape[0]):
        nd = [int(v) for v in conn[e]]
        for k in range(4):
            tri = tuple(sorted(nd[:k] + nd[k + 1:]))
            owner.setdefault(tri, []).append((e, nd[k]))
    rows, cols, vals = [], [], []
    for f in np.asarray(faces):
        key = tuple(sorted(int(v) for v in f))
        own = owner.get(key, [])
        if len(own) != 1:
            raise ValueError(f"face {key} is not a boundary face of exactly one element")
        e, opp = own[0]
        p0, p1, p2 = xyz[key[0]], xyz[key[1]], xyz[key[2]]
        nrm = np.cross(p1 - p0, p2 - p0)
        area = 0.5 * np.linalg.norm(nrm)
        n = nrm / np.linalg.norm(nrm)
        if n @ (xyz[opp] - p0) > 0.0:
            n = -n
        lam, mu, rho = lam_mu_rho[mat_id[e]]
        cp, cs = math.sqrt((lam + 2.0 * mu) / rho), math.sqrt(mu / rho)
        blk = area / 3.0 * rho * (cp * np.outer(n, n) + cs * (np.eye(3) - np.outer(n, n)))
        for node in key:
            for i in range(3):
                for j in range(3):
                    rows.append(3 * node + i)
                    cols.append(3 * node + j)
                    vals.append(blk[i, j])
    return sp.coo_matrix((vals, (rows, cols)), shape=(3 * N, 3 * N)).tocsr()


@dataclasses.dataclass
class System:
    """Assembled operators of one mesh, with Dirichlet DOFs eliminated (reduced system on `free`)."""
    M: sp.csr_matrix          # full 3N x 3N
    K: sp.csr_matrix
    free: np.ndarray          # indices of free DOFs
    dt: float
    a0: float
    a1: float
    Cb: sp.csr_matrix = None  # R22 dashpots of absorbing boundaries (None: none)

    @property
    def C(self):
        C = self.a0 * self.M + self.a1 * self.K                          # R4
        return C + self.Cb if self.Cb is not None else C

    @property
    def A_full(self):
        dt = self.dt
        return 4.0 / dt ** 2 * self.M + 2.0 / dt * self.C + self.K         # R1

    def reduce(self, Mat):
        return Mat[self.free][:, self.free].tocsr()


def build_system(mesh, tp, absorbing_faces=None) -> tuple[System, sp.csr_matrix]:
    """Assemble M, K (and the R22 dashpots of the listed boundary faces, if given); return (System, reduced A)."""
    M, K = assemble(mesh.xyz, mesh.conn, mesh.mat_id, mesh.lam_mu_rho)
    free = np.nonzero(mesh.fixed_dof == 0)[0]
    Cb = None
    if absorbing_faces is not None:
        Cb = lysmer_dashpots(mesh.xyz, mesh.conn, mesh.mat_id, mesh.lam_mu_rho, absorbing_faces)
    sysm = System(M=M, K=K, free=free, dt=tp.dt, a0=tp.a0, a1=tp.a1, Cb=Cb)
    return sysm, sysm.reduce(sysm.A_full)


def ricker(t, f0, t0, amp=1.0):
    """R12: Ricker wavelet."""
    arg = (math.pi * f0 * (t - t0)) ** 2
    return amp * (1.0 - 2.0 * arg) * math.exp(-arg)


def point_force(n_dof, src, t):
    """Full-length force vector of one Ricker point source at time t."""
    f = np.zeros(n_dof)
    w = ricker(t, src.f0, src.t0, src.amp)
    f[3 * src.node:3 * src.node + 3] = w * np.asarray(src.direction)
    return f


def impulse_force(n_dof, imp, it):
    """R23: full-length force vector of step `it` of a set of impulses (imp.nodes, imp.steps, imp.forces)."""
    f = np.zeros(n_dof)
    for k in np.nonzero(np.asarray(imp.steps) == it)[0]:
        node = int(imp.nodes[k])
        f[3 * node:3 * node + 3] += imp.forces[k]
    return f


def case_force(n_dof, src, it, dt):
    """The load of step `it`: a Ricker point source (R12) at t = it dt, or a set of impulses (R23)."""
    if hasattr(src, "steps"):
        return impulse_force(n_dof, src, it)
    return point_force(n_dof, src, it * dt)


def newmark_rhs(sysm: System, f, u, v, a):
    """R2: b = f - K u + C v + M (a + 4/dt v), full length (reduce with [free])."""
    dt = sysm.dt
    return f - sysm.K @ u + sysm.C @ v + sysm.M @ (a + 4.0 / dt * v)


def newmark_update(u, v, a, du, dt):
    """Eq. (timestep) with R3: returns (u_new, v_new, a_new)."""
    v_new = -v + 2.0 / dt * du
    a_new = -a - 4.0 / dt * v + 4.0 / dt ** 2 * du
    return u + du, v_new, a_new


# --------------------------------------------------------------------------------------------------------
# Algorithm 1: block-Jacobi preconditioned CG.
# --------------------------------------------------------------------------------------------------------


def block_jacobi_inverse(A_red: sp.csr_matrix, free: np.ndarray):
    """B^{-1} of Algorithm 1: the inverse of each node's diagonal block (the 3x3 block of its free DOFs,
    smaller where some of the node's DOFs are fixed), returned as a block-diagonal CSR matrix."""
    node = free // 3
    starts = np.r_[0, np.nonzero(np.diff(node))[0] + 1]     # a node's free DOFs are consecutive
    sizes = np.diff(np.r_[starts, node.size])
    blk_of = np.repeat(np.arange(starts.size), sizes)
    pos = np.arange(node.size) - starts[blk_of]
    coo = A_red.tocoo()
    same = blk_of[coo.row] == blk_of[coo.col]
    blocks = np.zeros((starts.size, 3, 3))
    blocks[blk_of[coo.row[same]], pos[coo.row[same]], pos[coo.col[same]]] = coo.data[same]
    for k in range(3):                                       # identity padding of absent DOFs
        blocks[sizes <= k, k, k] = 1.0
    inv = np.linalg.inv(blocks)
    rows, cols, vals = [], [], []
    for i in range(3):
        for j in range(3):
            m = (sizes > i) & (sizes > j)
            rows.append(starts[m] + i)
            cols.append(starts[m] + j)
            vals.append(inv[m, i, j])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=A_red.shape).tocsr()


@dataclasses.dataclass
class CGResult:
    x: np.ndarray
    iters: int
    relres: float             # true residual ||f - A x|| / ||f|| at exit
    history: list


def block_jacobi_cg(A, Binv, f, x_bar, eps=1e-8, maxit=10000, true_residual_exit=True):
    """Algorithm 1, literally: x = CG(A, f, x_bar) with z = B^{-1} r.  R13, R14 at exit."""
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return CGResult(np.zeros_like(f), 0, 0.0, [0.0])
    x = x_bar.copy()
    r = f - A @ x
    beta = 0.0
    i = 1
    hist = [np.linalg.norm(r) / nf]
    p = np.zeros_like(f)
    rho_b = 1.0
    while i <= maxit:
        if np.linalg.norm(r) / nf < eps:
            if not true_residual_exit:
                break
            r = f - A @ x                       # R14: replace by the true residual and re-test
            if np.linalg.norm(r) / nf < eps:
                break
        z = Binv @ r
        rho_a = z @ r
        if i > 1:
            beta = rho_a / rho_b
        p = z + beta * p
        q = A @ p
        alpha = rho_a / (p @ q)
        rho_b = rho_a
        r = r - alpha * q
        x = x + alpha * p
        i += 1
        hist.append(np.linalg.norm(r) / nf)
    rel = np.linalg.norm(f - A @ x) / nf
    return CGResult(x, i - 1, rel, hist)


# --------------------------------------------------------------------------------------------------------
# Predictors (Section 3.2).
# --------------------------------------------------------------------------------------------------------

AB4_COEF = (-9.0, 37.0, -59.0, 55.0)


def adams_bashforth4(u_prev, v_hist, dt):
    """u_bar = u^{it-1} + dt/24 (-9 v^{it-4} + 37 v^{it-3} - 59 v^{it-2} + 55 v^{it-1});
    v_hist = [v^{it-4}, v^{it-3}, v^{it-2}, v^{it-1}]."""
    acc = np.zeros_like(u_prev)
    for c, v in zip(AB4_COEF, v_hist):
        acc = acc + c * v
    return u_prev + dt / 24.0 * acc


def mgs_upper(X: np.ndarray, tau: float):
    """Modified Gram-Schmidt on the columns of X.  Returns (U [s][s] upper triangular, P = X U with
    orthonormal kept columns, kept mask).  Column j is dropped (R9) when its orthogonalised norm is
    <= tau times its original norm; a dropped column has zero columns in U and P."""
    n, s = X.shape
    U = np.zeros((s, s))
    P = np.zeros((n, s))
    kept = np.zeros(s, dtype=bool)
    for j in range(s):
        v = X[:, j].copy()
        u = np.zeros(s)
        u[j] = 1.0
        for k in range(j):
            if not kept[k]:
                continue
            coef = P[:, k] @ v            # modified GS: project the running vector
            v = v - coef * P[:, k]
            u = u - coef * U[:, k]
        nv = np.linalg.norm(v)
        n0 = np.linalg.norm(X[:, j])
        if n0 == 0.0 or nv <= tau * n0:
            continue
        P[:, j] = v / nv
        U[:, j] = u / nv
        kept[j] = True
    return U, P, kept


def mgs_predict(X, Y, x, tau=1e-6):
    """y = Y U c with c = P^T x (Section 3.2).  Returns (y, w) where w = U c are the coefficients of
    the prediction in the stored-snapshot basis (y = Y w)."""
    if X.shape[1] == 0:
        return np.zeros(Y.shape[0]), np.zeros(0)
    U, P, kept = mgs_upper(X, tau)
    c = P.T @ x
    w = U @ c
    return Y @ w, w


def regional_predict(E_hist, region_of_dof, n_regions, s, tau=1e-6):
    """Data-driven correction per region (R8, R10).

    E_hist: list of past corrections [e^{it-k-1}, ..., e^{it-1}] (reduced-DOF vectors), k <= s pairs.
    Returns (y_hat, W) with y_hat the predicted e^{it} and W [n_regions][s] the per-region coefficients.
    """
    npairs = min(s, len(E_hist) - 1)
    y = np.zeros(E_hist[-1].shape[0]) if E_hist else None
    W = np.zeros((n_regions, s))
    if npairs <= 0:
        return (y if y is not None else None), W
    cols = E_hist[-(npairs + 1):]
    X_all = np.stack(cols[:-1], axis=1)          # x_j = e^{j-1}
    Y_all = np.stack(cols[1:], axis=1)           # y_j = e^{j}
    xq = cols[-1]                                # query x = e^{it-1}
    for R in range(n_regions):
        idx = np.nonzero(region_of_dof == R)[0]
        if idx.size == 0:
            continue
        yR, w = mgs_predict(X_all[idx], Y_all[idx], xq[idx], tau)
        y[idx] = yR
        W[R, :npairs] = w
    return y, W


# --------------------------------------------------------------------------------------------------------
# Time loop (Algorithm 2 with the predictor of Algorithm 3), one case.
# --------------------------------------------------------------------------------------------------------


@dataclasses.dataclass
class StepRecord:
    it: int
    iters: int
    relres: float
    init_relres: float
    du: np.ndarray            # reduced increment


class CaseSimulator:
    """Newmark time stepping of one case with the paper's predictor and Algorithm 1 solver."""

    def __init__(self, sysm: System, A_red, Binv, src, predictor="ab4", s_max=32, region_of_node=None,
                 tau=1e-6, eps=1e-8, maxit=10000):
        self.sysm, self.A, self.Binv, self.src = sysm, A_red, Binv, src
        n = sysm.M.shape[0]
        self.u = np.zeros(n)
        self.v = np.zeros(n)
        self.a = np.zeros(n)
        self.v_hist = [np.zeros(n) for _ in range(4)]      # R11
        self.E_hist = []                                   # reduced corrections e^j
        self.predictor, self.s_max, self.tau = predictor, s_max, tau
        self.eps, self.maxit = eps, maxit
        self.it = 0
        if region_of_node is not None:
            reg = np.repeat(region_of_node, 3)[sysm.free]
            self.region_of_dof = reg
            self.n_regions = int(reg.max()) + 1
        else:
            self.region_of_dof, self.n_regions = None, 0

    def guess(self):
        """Initial increment du_bar = (AB4 + data-driven correction) - u^{it-1}, reduced."""
        dt = self.sysm.dt
        free = self.sysm.free
        u_ab = adams_bashforth4(self.u, self.v_hist, dt)
        du_ab = (u_ab - self.u)[free]
        self.last_W, self.last_npairs = None, 0
        if self.predictor == "dd" and self.region_of_dof is not None:
            y, W = regional_predict(self.E_hist, self.region_of_dof, self.n_regions, self.s_max, self.tau)
            self.last_W, self.last_npairs = W, max(0, min(self.s_max, len(self.E_hist) - 1))
            if y is not None:
                return du_ab + y, du_ab
        return du_ab, du_ab

    def step(self, du_bar_override=None):
        self.it += 1
        sysm = self.sysm
        t = self.it * sysm.dt
        f = case_force(sysm.M.shape[0], self.src, self.it, sysm.dt)
        b_full = newmark_rhs(sysm, f, self.u, self.v, self.a)
        b = b_full[sysm.free]
        du_bar, du_ab = self.guess()
        if du_bar_override is not None:
            du_bar = du_bar_override
        nb = np.linalg.norm(b)
        init_rel = np.linalg.norm(b - self.A @ du_bar) / nb if nb > 0 else 0.0
        res = block_jacobi_cg(self.A, self.Binv, b, du_bar, self.eps, self.maxit)
        du = np.zeros_like(self.u)
        du[sysm.free] = res.x
        self.u, self.v, self.a = newmark_update(self.u, self.v, self.a, du, sysm.dt)
        self.v_hist = self.v_hist[1:] + [self.v.copy()]
        self.E_hist.append(res.x - du_ab)                  # e^it = u^it - u_AB^it (reduced)
        if len(self.E_hist) > self.s_max + 1:
            self.E_hist.pop(0)
        return StepRecord(self.it, res.iters, res.relres, init_rel, res.x)


def energy(sysm: System, u, v):
    """E = 1/2 v^T M v + 1/2 u^T K u."""
    return 0.5 * v @ (sysm.M @ v) + 0.5 * u @ (sysm.K @ u)
