"""FP64 CPU oracle for the 10-node tetrahedron (the paper's element, Section 3.1) -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module; it shares no code with the CUDA path.  Straight-sided tet10 with
barycentric coordinates L_0..L_3 (grad L_a = g_a, constant on the element; g_0 = -(g_1 + g_2 + g_3)):

  corner a:    N_a  = L_a (2 L_a - 1),          grad N_a  = (4 L_a - 1) g_a
  edge (a, b): N_ab = 4 L_a L_b,                grad N_ab = 4 (L_a g_b + L_b g_a)

with the local order corners 0-3, edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).

* Stiffness K_e = int B^T D B dV: the gradients are linear, so the integrand is quadratic and the 4-point
  Gauss rule on the tetrahedron (barycentric points (a, b, b, b) and permutations, a = (5 + 3 sqrt 5) / 20,
  b = (5 - sqrt 5) / 20, weights V / 4) is exact.  `tet10_element_stiffness_exact` integrates the same
  products monomial by monomial instead (a second, independent route used as a pin).
* Consistent mass M_e = rho int N_i N_j dV I3, integrated exactly with
  int_T L_0^p L_1^q L_2^r L_3^s dV = 6 V p! q! r! s! / (p + q + r + s + 3)!.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np
import scipy.sparse as sp

from .fem_oracle import isotropic_D, tet4_shape_gradients

EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))


def shape_polys():
    """Each N_i as {exponent tuple (p, q, r, s): coefficient} in the barycentric coordinates."""
    polys = []
    for a in range(4):
        e2 = [0, 0, 0, 0]
        e2[a] = 2
        e1 = [0, 0, 0, 0]
        e1[a] = 1
        polys.append({tuple(e2): Fraction(2), tuple(e1): Fraction(-1)})
    for a, b in EDGES:
        e = [0, 0, 0, 0]
        e[a] += 1
        e[b] += 1
        polys.append({tuple(e): Fraction(4)})
    return polys


def monomial_integral(exps) -> Fraction:
    """int_T prod L_k^{e_k} dV / V."""
    num = 6 * math.prod(math.factorial(e) for e in exps)
    return Fraction(num, math.factorial(sum(exps) + 3))


def poly_mul(p1, p2):
    out = {}
    for e1, c1 in p1.items():
        for e2, c2 in p2.items():
            e = tuple(x + y for x, y in zip(e1, e2))
            out[e] = out.get(e, 0) + c1 * c2
    return out


def mass_coefficients() -> np.ndarray:
    """m[i][j] = int N_i N_j dV / V (exact rationals, returned as float64)."""
    P = shape_polys()
    m = np.zeros((10, 10))
    for i in range(10):
        for j in range(10):
            m[i, j] = float(sum(c * monomial_integral(e) for e, c in poly_mul(P[i], P[j]).items()))
    return m


_A = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
_B = (5.0 - math.sqrt(5.0)) / 20.0
GAUSS4 = [tuple(_A if k == q else _B for k in range(4)) for q in range(4)]


def shape_gradients(g: np.ndarray, L) -> np.ndarray:
    """g: [E][4][3] barycentric gradients; L: one barycentric point.  Returns [E][10][3]."""
    out = np.empty((g.shape[0], 10, 3))
    for a in range(4):
        out[:, a] = (4.0 * L[a] - 1.0) * g[:, a]
    for k, (a, b) in enumerate(EDGES):
        out[:, 4 + k] = 4.0 * (L[a] * g[:, b] + L[b] * g[:, a])
    return out


def voigt_B(dN: np.ndarray) -> np.ndarray:
    """[E][6][30] strain-displacement matrix (xx, yy, zz, yz, xz, xy; engineering shear)."""
    E = dN.shape[0]
    B = np.zeros((E, 6, 30))
    for i in range(10):
        dx, dy, dz = dN[:, i, 0], dN[:, i, 1], dN[:, i, 2]
        c = 3 * i
        B[:, 0, c] = dx
        B[:, 1, c + 1] = dy
        B[:, 2, c + 2] = dz
        B[:, 3, c + 1] = dz
        B[:, 3, c + 2] = dy
        B[:, 4, c] = dz
        B[:, 4, c + 2] = dx
        B[:, 5, c] = dy
        B[:, 5, c + 1] = dx
    return B


def corner_geometry(xyz, conn10):
    return tet4_shape_gradients(xyz[conn10[:, :4]])


def tet10_element_matrices(xyz, conn10, mat_id, lam_mu_rho):
    """(K_e [E][30][30], M_e [E][30][30]) by the 4-point rule and the exact mass integrals."""
    g, V = corner_geometry(xyz, conn10)
    lmr = lam_mu_rho[mat_id]
    D = isotropic_D(lmr[:, 0], lmr[:, 1])
    K = np.zeros((conn10.shape[0], 30, 30))
    for L in GAUSS4:
        B = voigt_B(shape_gradients(g, L))
        K += 0.25 * V[:, None, None] * np.einsum("eki,ekl,elj->eij", B, D, B)
    m = mass_coefficients()
    M = (lmr[:, 2] * V)[:, None, None] * np.kron(m, np.eye(3))[None]
    return K, M


def tet10_element_stiffness_exact(xyz, conn10, mat_id, lam_mu_rho):
    """K_e integrated monomial by monomial (no quadrature): grad N_i = sum_a c_ia(L) g_a with c linear in L,
    so B^T D B is a quadratic polynomial in L whose monomials integrate exactly."""
    g, V = corner_geometry(xyz, conn10)
    lmr = lam_mu_rho[mat_id]
    D = isotropic_D(lmr[:, 0], lmr[:, 1])
    # grad N_i = sum_a sum_k C[i][a][k] L_k g_a (+ constant D0[i][a] g_a)
    lin = np.zeros((10, 4, 4))      # coefficient of L_k g_a
    const = np.zeros((10, 4))       # coefficient of g_a
    for a in range(4):
        lin[a, a, a] = 4.0
        const[a, a] = -1.0
    for k, (a, b) in enumerate(EDGES):
        lin[4 + k, b, a] = 4.0
        lin[4 + k, a, b] = 4.0
    # int L_k dV / V = 1/4; int L_k L_l dV / V = (1 + delta_kl) / 20
    I1 = np.full(4, 0.25)
    I2 = (np.ones((4, 4)) + np.eye(4)) / 20.0
    # the gradient field as [E][10][3] = const part + sum_k L_k part_k
    G0 = np.einsum("ia,eax->eix", const, g)
    Gk = np.einsum("iak,eax->keix", lin, g)        # [4][E][10][3]
    K = np.zeros((conn10.shape[0], 30, 30))
    terms = [(G0, G0, 1.0)]
    for k in range(4):
        terms.append((G0, Gk[k], I1[k]))
        terms.append((Gk[k], G0, I1[k]))
    for k in range(4):
        for l in range(4):
            terms.append((Gk[k], Gk[l], I2[k, l]))
    for Ga, Gb, w in terms:
        Ba, Bb = voigt_B(Ga), voigt_B(Gb)
        K += w * V[:, None, None] * np.einsum("eki,ekl,elj->eij", Ba, D, Bb)
    return K


def assemble10(xyz, conn10, mat_id, lam_mu_rho):
    """Global (K, M) as scipy CSR, 3 DOFs per node in node-major order."""
    Ke, Me = tet10_element_matrices(xyz, conn10, mat_id, lam_mu_rho)
    dof = (3 * conn10[:, :, None] + np.arange(3)[None, None, :]).reshape(conn10.shape[0], 30)
    rows = np.repeat(dof, 30, axis=1).reshape(-1)
    cols = np.tile(dof, (1, 30)).reshape(-1)
    n = 3 * xyz.shape[0]
    K = sp.csr_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n))
    M = sp.csr_matrix((Me.reshape(-1), (rows, cols)), shape=(n, n))
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M
