// Element-by-element product for 10-node tetrahedra, the paper's element (Section 3.1; the EBE of
// Section 3.2 / Eq. eqebefem applied to quadratic tets).  Straight-sided elements: the barycentric
// gradients g_a are constant on a tet, so the element record is the tet4 one of its corners (g_1..g_3,
// lambda V, mu V, rho V / 20) and the quadratic shape-function gradients are formed on the fly,
//   corner a:    grad N_a  = (4 L_a - 1) g_a,       edge (a, b): grad N_ab = 4 (L_a g_b + L_b g_a),
// at the four points of the degree-2 Gauss rule (exact for the stiffness, whose integrand is quadratic):
//   (K p)_i = sum_q V/4 sigma(G_q) grad N_i(L_q),  G_q = sum_j p_j (x) grad N_j(L_q),
//   sigma(G) = lambda tr(G) I + mu (G + G^T),
// both sums taken through the four corner gradients (about 180 operations a point instead of 450).
// The consistent mass (M p)_i = rho V sum_j m_ij p_j with m_ij = int N_i N_j dV / V: generated on the host
// from int L_0^a L_1^b L_2^c L_3^d dV = 6 V a! b! c! d! / (a + b + c + d + 3)! for the preconditioner's
// diagonal, applied in the product through the seven distinct values of 420 m_ij.
// Local order: corners 0-3, edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).  One thread per (element,
// case); sums scatter with global atomics (Dirichlet rows masked afterwards).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fem_internal.cuh"

namespace fem {

namespace {

// edge s joins corners edge_a(s) and edge_b(s)
__host__ __device__ constexpr int edge_a(int s) { return s == 0 ? 0 : s == 1 ? 1 : s == 2 ? 0 : s == 3 ? 0 : s == 4 ? 1 : 2; }
__host__ __device__ constexpr int edge_b(int s) { return s == 0 ? 1 : s == 1 ? 2 : s == 2 ? 2 : s == 3 ? 3 : s == 4 ? 3 : 3; }
// the edge sharing no corner with edge s
__host__ __device__ constexpr int edge_opp(int s) { return s == 0 ? 5 : s == 1 ? 3 : s == 2 ? 4 : s == 3 ? 1 : s == 4 ? 2 : 0; }

struct Mass10 {
  double m64[55];   // upper triangle of m_ij, row-major
};

// Exact m_ij = int N_i N_j dV / V by expanding N_i N_j into barycentric monomials.
void mass10_host(double out[10][10]) {
  // N_i as up to two terms c * L^e (exponents over L_0..L_3)
  struct Term {
    double c;
    int e[4];
  };
  std::vector<std::vector<Term>> N(10);
  for (int a = 0; a < 4; ++a) {
    Term t2{2.0, {0, 0, 0, 0}}, t1{-1.0, {0, 0, 0, 0}};
    t2.e[a] = 2;
    t1.e[a] = 1;
    N[a] = {t2, t1};
  }
  for (int k = 0; k < 6; ++k) {
    Term t{4.0, {0, 0, 0, 0}};
    t.e[edge_a(k)] += 1;
    t.e[edge_b(k)] += 1;
    N[4 + k] = {t};
  }
  auto fact = [](int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
  };
  for (int i = 0; i < 10; ++i)
    for (int j = 0; j < 10; ++j) {
      double s = 0.0;
      for (const Term& a : N[i])
        for (const Term& b : N[j]) {
          int e[4], deg = 0;
          double num = 6.0;
          for (int k = 0; k < 4; ++k) {
            e[k] = a.e[k] + b.e[k];
            deg += e[k];
            num *= fact(e[k]);
          }
          s += a.c * b.c * num / fact(deg + 3);
        }
      out[i][j] = s;
    }
}

__host__ __device__ constexpr int tri(int i, int j) { return i <= j ? i * 10 - i * (i - 1) / 2 + (j - i) : tri(j, i); }


template <typename T> struct Rec10;
template <> struct Rec10<float> {
  static __device__ __forceinline__ const float* get(const float* r32, const double*) { return r32; }
};
template <> struct Rec10<double> {
  static __device__ __forceinline__ const double* get(const float*, const double* r64) { return r64; }
};

// I: index type of the vector offsets (32-bit when N * 3 * rpad fits: one multiply-add an address)
template <typename T, bool DOT, typename I>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 2 : 1) k_ebe10(int64_t E, int rpad, int rshift, const int32_t* __restrict__ conn,
                                                   const float* __restrict__ rec32, const double* __restrict__ rec64,
                                                   const T* __restrict__ p, T* __restrict__ q, T aM, T aK,
                                                   Reducer red, double* ptq_out, CgCase* sc,
                                                   const int* gate) {
  if (gate && *gate == 0) return;
  const T* __restrict__ recs = Rec10<T>::get(rec32, rec64);
  // barycentric coordinates of the four Gauss points: (A, B, B, B) and its permutations
  const T GA = (T)0.5854101966249685, GB = (T)0.1381966011250105;
  double dot = 0.0;
  const int64_t total = E << rshift;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < total; it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = it >> rshift;
    const int c = (int)(it & (rpad - 1));
    I off[10];   // offset of node i's first value of case c
#pragma unroll
    for (int i = 0; i < 10; ++i) off[i] = (I)__ldg(conn + e * 10 + i) * (I)(3 * rpad) + (I)c;
    T P[10][3], Q[10][3];
#pragma unroll
    for (int i = 0; i < 10; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        P[i][k] = __ldg(p + off[i] + (I)(k * rpad));
        Q[i][k] = (T)0;
      }
    const T* r = recs + e * kRec;
    T g[4][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g[1][k] = r[k], g[2][k] = r[3 + k], g[3][k] = r[6 + k];
      g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
    }
    const T lam = aK * r[9] * (T)0.25, mu = aK * r[10] * (T)0.25, rv = aM * r[11] * (T)20;   // V/4 weights
    // At a Gauss point grad N_i = sum_a c_ia g_a (c linear in L), so both contractions run through the four
    // corners: G = sum_a W_a (x) g_a with W_a = sum_i c_ia p_i, and the forces sum_a c_ia (sigma g_a):
    //   W_a = (4 L_a - 1) p_a + 4 sum_{edges (a, b)} L_b p_ab,
    //   f_a += (4 L_a - 1) T_a,   f_ab += 4 (L_a T_b + L_b T_a),   T_a = sigma g_a.
#pragma unroll
    for (int qp = 0; qp < 4; ++qp) {   // (unrolled: the points' coefficients are constants)
      T L[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) L[a] = a == qp ? GA : GB;
      T W[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) W[a][k] = ((T)4 * L[a] - (T)1) * P[a][k];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int a = edge_a(e), b = edge_b(e);
        const T lb4 = (T)4 * L[b], la4 = (T)4 * L[a];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          W[a][k] += lb4 * P[4 + e][k];
          W[b][k] += la4 * P[4 + e][k];
        }
      }
      T G[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) G[k][j] = W[0][k] * g[0][j] + W[1][k] * g[1][j] + W[2][k] * g[2][j] + W[3][k] * g[3][j];
      const T ltr = lam * (G[0][0] + G[1][1] + G[2][2]);
      T S[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[k][j] = mu * (G[k][j] + G[j][k]) + (k == j ? ltr : (T)0);
      T Tg[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) Tg[a][k] = S[k][0] * g[a][0] + S[k][1] * g[a][1] + S[k][2] * g[a][2];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) Q[a][k] += ((T)4 * L[a] - (T)1) * Tg[a][k];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int a = edge_a(e), b = edge_b(e);
        const T la4 = (T)4 * L[a], lb4 = (T)4 * L[b];
#pragma unroll
        for (int k = 0; k < 3; ++k) Q[4 + e][k] += la4 * Tg[b][k] + lb4 * Tg[a][k];
      }
    }
    // consistent mass through its structure: 420 m_ij = 6 / 1 (corner diagonal / other corner), -4 / -6
    // (corner and an edge through it / the others), 32 / 16 / 8 (edge diagonal / an edge sharing a corner /
    // the opposite edge), so with the corner and edge sums Sc, Se:
    //   corner a:      5 p_a + Sc - 6 Se + 2 (sum of a's three edges)
    //   edge (a, b):  -6 Sc + 2 (p_a + p_b) + 16 Se + 16 p_ab - 8 p_opposite
    const T rv420 = rv * (T)(1.0 / 420.0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T Sc = (P[0][k] + P[1][k]) + (P[2][k] + P[3][k]);
      const T Se = (P[4][k] + P[5][k]) + (P[6][k] + P[7][k]) + (P[8][k] + P[9][k]);
      const T base_c = Sc - (T)6 * Se, base_e = (T)16 * Se - (T)6 * Sc;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T Ea = (T)0;
#pragma unroll
        for (int e = 0; e < 6; ++e)
          if (edge_a(e) == a || edge_b(e) == a) Ea += P[4 + e][k];
        Q[a][k] += rv420 * ((T)5 * P[a][k] + base_c + (T)2 * Ea);
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int a = edge_a(e), b = edge_b(e), o = edge_opp(e);
        Q[4 + e][k] += rv420 * (base_e + (T)2 * (P[a][k] + P[b][k]) + (T)16 * P[4 + e][k] - (T)8 * P[4 + o][k]);
      }
    }
    T hd = (T)0;   // (the element's p^T q in the product's precision, one conversion an element: FP64
                   // conversions and adds run on GB300's narrow FP64 pipe)
#pragma unroll
    for (int i = 0; i < 10; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (DOT) hd += P[i][k] * Q[i][k];
        atomicAdd(q + off[i] + (I)(k * rpad), Q[i][k]);
      }
    if (DOT) dot += (double)hd;
  }
  if (DOT) {
    double v[1] = {dot};
    if (block_reduce_last<1>(v, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);   // (and the CG step length)
  }
}

// Node diagonal 3x3 blocks of aM M + aK K (xx yy zz xy xz yz), element by element: at the Gauss points
// K_ii = V/4 sum_q [lambda d d^T + mu (|d|^2 I + d d^T)] with d = grad N_i, and M_ii = rho V m_ii I.
__global__ void k_diag10(int64_t E, const int32_t* __restrict__ conn, const double* __restrict__ rec, double aM,
                         double aK, Mass10 mc, double* __restrict__ D) {
  const double GA = 0.5854101966249685, GB = 0.1381966011250105;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const double* r = rec + e * kRec;
    double g[4][3];
    for (int k = 0; k < 3; ++k) {
      g[1][k] = r[k], g[2][k] = r[3 + k], g[3][k] = r[6 + k];
      g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
    }
    const double lam = aK * r[9] * 0.25, mu = aK * r[10] * 0.25, rv = aM * r[11] * 20.0;
    for (int i = 0; i < 10; ++i) {
      double b[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int qp = 0; qp < 4; ++qp) {
        double L[4];
        for (int a = 0; a < 4; ++a) L[a] = a == qp ? GA : GB;
        double d[3];
        if (i < 4) {
          for (int k = 0; k < 3; ++k) d[k] = (4.0 * L[i] - 1.0) * g[i][k];
        } else {
          const int a = edge_a(i - 4), bb = edge_b(i - 4);
          for (int k = 0; k < 3; ++k) d[k] = 4.0 * (L[a] * g[bb][k] + L[bb] * g[a][k]);
        }
        const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double lm = lam + mu;
        b[0] += lm * d[0] * d[0] + mu * dd, b[1] += lm * d[1] * d[1] + mu * dd, b[2] += lm * d[2] * d[2] + mu * dd;
        b[3] += lm * d[0] * d[1], b[4] += lm * d[0] * d[2], b[5] += lm * d[1] * d[2];
      }
      const double mi = rv * mc.m64[tri(i, i)];
      b[0] += mi, b[1] += mi, b[2] += mi;
      double* dn = D + (int64_t)conn[e * 10 + i] * 6;
      for (int k = 0; k < 6; ++k) atomicAdd(dn + k, b[k]);
    }
  }
}

// The assembled operators of a tet10 mesh (the certification product's 3x3-block stiffness and scalar mass on
// the node pattern): one thread per element adds its 100 node-pair blocks,
//   K_ij = sum_q V/4 [lambda d_i d_j^T + mu d_j d_i^T + mu (d_i . d_j) I],  d_i = grad N_i at Gauss point q,
//   M_ij = rho V m_ij,
// the same operators the product applies (exact Gauss rule for the stiffness, exact mass coefficients).
__device__ __forceinline__ void grad10(const double (&g)[4][3], const double (&L)[4], int i, double (&d)[3]) {
  if (i < 4) {
    for (int k = 0; k < 3; ++k) d[k] = (4.0 * L[i] - 1.0) * g[i][k];
  } else {
    const int a = edge_a(i - 4), b = edge_b(i - 4);
    for (int k = 0; k < 3; ++k) d[k] = 4.0 * (L[a] * g[b][k] + L[b] * g[a][k]);
  }
}

__global__ void k_bcsr_assemble10(int64_t E, const int32_t* __restrict__ conn, const double* __restrict__ rec,
                                  Mass10 mc, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                  double* __restrict__ Kb, double* __restrict__ Mb, int* __restrict__ missing) {
  const double GA = 0.5854101966249685, GB = 0.1381966011250105;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const double* r = rec + e * kRec;
    double g[4][3];
    for (int k = 0; k < 3; ++k) {
      g[1][k] = r[k], g[2][k] = r[3 + k], g[3][k] = r[6 + k];
      g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
    }
    const double lam = r[9] * 0.25, mu = r[10] * 0.25, rv = r[11] * 20.0;
    int nd[10];
    for (int i = 0; i < 10; ++i) nd[i] = conn[e * 10 + i];
    for (int i = 0; i < 10; ++i) {
      const int lo = row_ptr[nd[i]], hi = row_ptr[nd[i] + 1];
      for (int j = 0; j < 10; ++j) {
        int jj = -1;
        for (int t = lo; t < hi; ++t)
          if (col[t] == nd[j]) {
            jj = t;
            break;
          }
        if (jj < 0) {
          atomicExch(missing, 1);
          continue;
        }
        double kb[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int qp = 0; qp < 4; ++qp) {
          double L[4], di[3], dj[3];
          for (int a = 0; a < 4; ++a) L[a] = a == qp ? GA : GB;
          grad10(g, L, i, di);
          grad10(g, L, j, dj);
          const double dd = di[0] * dj[0] + di[1] * dj[1] + di[2] * dj[2];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              kb[a * 3 + b] += lam * di[a] * dj[b] + mu * dj[a] * di[b] + (a == b ? mu * dd : 0.0);
        }
        for (int u = 0; u < 9; ++u) atomicAdd(Kb + (int64_t)jj * 9 + u, kb[u]);
        atomicAdd(Mb + jj, rv * mc.m64[tri(i, j)]);
      }
    }
  }
}

Mass10 mass10_table() {
  static Mass10 mc = [] {
    Mass10 t{};
    double mm[10][10];
    mass10_host(mm);
    for (int i = 0; i < 10; ++i)
      for (int j = i; j < 10; ++j) t.m64[tri(i, j)] = mm[i][j];
    return t;
  }();
  return mc;
}

__global__ void k_corner_conn(int64_t E, const int32_t* __restrict__ conn10, int4* __restrict__ conn4) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
    conn4[e] = make_int4(conn10[e * 10], conn10[e * 10 + 1], conn10[e * 10 + 2], conn10[e * 10 + 3]);
}

int lg2i(int r) {
  int s = 0;
  while ((1 << s) < r) ++s;
  return s;
}

}  // namespace

// The products of the time-stepping solver on a tet10 mesh: q = aM M pm + aK K pk (pk null: the same p for
// both, with p^T q and the CG step length fused when red is given; gate as the tet4 kernels'), Dirichlet
// rows of q zeroed.
template <typename T>
cudaError_t launch_ebe10_gated(int64_t E, int64_t N, int rpad, const int32_t* conn10, const float* rec32,
                               const double* rec64, const uint8_t* fm, const T* pm, const T* pk, T* q, double aM,
                               double aK, const Reducer* red, CgCase* sc, double* ptq, const int* gate,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(q, 0, sizeof(T) * (size_t)N * 3 * rpad, s);
  if (e != cudaSuccess) return e;
  const int rs = lg2i(rpad);
  const bool i32 = N * 3 * rpad < ((int64_t)1 << 31);
  const Reducer none{nullptr, nullptr, nullptr};
  auto run = [&](const T* p, T a_m, T a_k, bool dot) {
    const int grid = grid_for(E << rs, dot ? red_grid_cap() : -1);
    auto fn = dot ? (i32 ? k_ebe10<T, true, int32_t> : k_ebe10<T, true, int64_t>)
                  : (i32 ? k_ebe10<T, false, int32_t> : k_ebe10<T, false, int64_t>);
    fn<<<grid, kBlock, 0, s>>>(E, rpad, rs, conn10, rec32, rec64, p, q, a_m, a_k, dot ? *red : none,
                               dot ? ptq : nullptr, dot ? sc : nullptr, gate);
    return cudaGetLastError();
  };
  if (pk) {
    e = run(pm, (T)aM, (T)0, false);
    if (e == cudaSuccess) e = run(pk, (T)0, (T)aK, false);
  } else {
    e = run(pm, (T)aM, (T)aK, red != nullptr);
  }
  if (e == cudaSuccess) e = launch_mask<T>(N, rpad, fm, q, s);
  return e;
}
template cudaError_t launch_ebe10_gated<float>(int64_t, int64_t, int, const int32_t*, const float*, const double*,
                                               const uint8_t*, const float*, const float*, float*, double, double,
                                               const Reducer*, CgCase*, double*, const int*, cudaStream_t);
template cudaError_t launch_ebe10_gated<double>(int64_t, int64_t, int, const int32_t*, const float*, const double*,
                                                const uint8_t*, const double*, const double*, double*, double, double,
                                                const Reducer*, CgCase*, double*, const int*, cudaStream_t);

cudaError_t launch_diag10(int64_t E, const int32_t* conn10, const double* rec64, double aM, double aK, double* D,
                          cudaStream_t s) {
  k_diag10<<<grid_for(E), kBlock, 0, s>>>(E, conn10, rec64, aM, aK, mass10_table(), D);
  return cudaGetLastError();
}

cudaError_t launch_bcsr_assemble10(int64_t E, const int32_t* conn10, const double* rec64, const int32_t* row_ptr,
                                   const int32_t* col, int64_t nnz, double* Kb, double* Mb, float2* KMd, int* missing,
                                   cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(Kb, 0, sizeof(double) * 9 * (size_t)nnz, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Mb, 0, sizeof(double) * (size_t)nnz, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(missing, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_bcsr_assemble10<<<grid_for(E), kBlock, 0, s>>>(E, conn10, rec64, mass10_table(), row_ptr, col, Kb, Mb, missing);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_to_kmd(nnz, Kb, Mb, KMd, s);
}

}  // namespace fem

using namespace fem;

struct fem_mesh10 {
  int64_t N = 0, E = 0;
  int device = 0;
  int32_t* conn = nullptr;    // [E][10]
  float* rec32 = nullptr;     // [E][12] records of the corner tets
  double* rec64 = nullptr;
  uint8_t* fm = nullptr;      // [N] free-DOF bits
  double* partial = nullptr;  // reduction scratch
  unsigned* counter = nullptr;
  double* out = nullptr;
  Mass10 mc{};
  ~fem_mesh10() {
    cudaFree(conn); cudaFree(rec32); cudaFree(rec64); cudaFree(fm); cudaFree(partial); cudaFree(counter); cudaFree(out);
  }
};

extern "C" {

fem_status fem_mesh10_create(int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn10,
                             const int32_t* mat_id, int n_mat, const double* lam_mu_rho, const uint8_t* fixed_dof,
                             void* stream, fem_mesh10** out) {
  if (!out) return set_error(FEM_ERR_ARG, "out is null");
  *out = nullptr;
  if (!xyz || !conn10 || !mat_id || !lam_mu_rho || !fixed_dof) return set_error(FEM_ERR_ARG, "null input pointer");
  if (n_nodes < 10 || n_elems < 1 || n_mat < 1) return set_error(FEM_ERR_ARG, "empty mesh");
  if (n_nodes > INT32_MAX) return set_error(FEM_ERR_ARG, "node ids must fit int32");
  for (int64_t i = 0; i < n_elems * 10; ++i)
    if (conn10[i] < 0 || conn10[i] >= n_nodes) return set_error(FEM_ERR_ARG, "connectivity out of range");
  cudaStream_t s = (cudaStream_t)stream;
  fem_mesh10* m = new fem_mesh10();
  m->N = n_nodes, m->E = n_elems;
  cudaGetDevice(&m->device);
  double* d_xyz = nullptr;
  int32_t* d_mat = nullptr;
  double* d_lmr = nullptr;
  int4* d_c4 = nullptr;
  int* d_err = nullptr;
  std::vector<uint8_t> fm(n_nodes);
  for (int64_t n = 0; n < n_nodes; ++n)
    fm[n] = (uint8_t)((fixed_dof[3 * n] ? 0 : 1) | (fixed_dof[3 * n + 1] ? 0 : 2) | (fixed_dof[3 * n + 2] ? 0 : 4));
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  al((void**)&m->conn, sizeof(int32_t) * 10 * n_elems);
  al((void**)&m->rec32, sizeof(float) * kRec * n_elems);
  al((void**)&m->rec64, sizeof(double) * kRec * n_elems);
  al((void**)&m->fm, n_nodes);
  al((void**)&m->partial, sizeof(double) * kMaxRedBlocks * 3 * kMaxCases);
  al((void**)&m->counter, sizeof(unsigned));
  al((void**)&m->out, sizeof(double) * 3 * kMaxCases);
  al((void**)&d_xyz, sizeof(double) * 3 * n_nodes);
  al((void**)&d_mat, sizeof(int32_t) * n_elems);
  al((void**)&d_lmr, sizeof(double) * 3 * n_mat);
  al((void**)&d_c4, sizeof(int4) * n_elems);
  al((void**)&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->conn, conn10, sizeof(int32_t) * 10 * n_elems, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->fm, fm.data(), n_nodes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_xyz, xyz, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mat, mat_id, sizeof(int32_t) * n_elems, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_lmr, lam_mu_rho, sizeof(double) * 3 * n_mat, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->counter, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_corner_conn<<<grid_for(n_elems), kBlock, 0, s>>>(n_elems, m->conn, d_c4);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_elem_setup(n_elems, n_nodes, d_xyz, d_c4, d_mat, n_mat, d_lmr, m->rec64, m->rec32, d_err, s);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_xyz); cudaFree(d_mat); cudaFree(d_lmr); cudaFree(d_c4); cudaFree(d_err);
  if (e != cudaSuccess || h_err) {
    cudaGetLastError();
    delete m;
    if (e != cudaSuccess) return set_error(FEM_ERR_CUDA, std::string("tet10 mesh: ") + cudaGetErrorString(e));
    return set_error(FEM_ERR_ARG, h_err & 2 ? "degenerate or inverted corner tet" : "bad material id");
  }
  double mm[10][10];
  mass10_host(mm);
  for (int i = 0; i < 10; ++i)
    for (int j = i; j < 10; ++j) {
      m->mc.m64[tri(i, j)] = mm[i][j];
    }
  *out = m;
  return FEM_OK;
}

fem_status fem_mesh10_destroy(fem_mesh10* m) {
  delete m;
  return FEM_OK;
}

fem_status fem_ebe10_apply(fem_mesh10* m, int precision, const void* p_dev, void* q_dev, int n_rhs, double alpha_M,
                           double alpha_K, double* ptq_dev, void* stream) {
  if (!m || !p_dev || !q_dev) return set_error(FEM_ERR_ARG, "null argument");
  if (n_rhs < 1 || n_rhs > kMaxRpad || (n_rhs & (n_rhs - 1))) return set_error(FEM_ERR_ARG, "n_rhs must be 1, 2, 4, 8, 16 or 32");
  if (precision != FEM_FP64 && precision != FEM_FP32_INNER) return set_error(FEM_ERR_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  const int rs = lg2i(n_rhs);
  const int64_t items = m->E << rs;
  int grid = grid_for(items, red_grid_cap());
  const Reducer red{m->partial, m->counter, m->out};
  const bool dot = ptq_dev != nullptr;
  const size_t bytes = (precision == FEM_FP64 ? 8 : 4) * (size_t)m->N * 3 * n_rhs;
  cudaError_t e = cudaMemsetAsync(q_dev, 0, bytes, s);
  if (e == cudaSuccess) {
    const bool i32 = m->N * 3 * n_rhs < ((int64_t)1 << 31);
    if (precision == FEM_FP64) {
      auto fn = dot ? (i32 ? k_ebe10<double, true, int32_t> : k_ebe10<double, true, int64_t>)
                    : (i32 ? k_ebe10<double, false, int32_t> : k_ebe10<double, false, int64_t>);
      fn<<<grid, kBlock, 0, s>>>(m->E, n_rhs, rs, m->conn, m->rec32, m->rec64, (const double*)p_dev, (double*)q_dev,
                                 alpha_M, alpha_K, red, ptq_dev, nullptr, nullptr);
    } else {
      auto fn = dot ? (i32 ? k_ebe10<float, true, int32_t> : k_ebe10<float, true, int64_t>)
                    : (i32 ? k_ebe10<float, false, int32_t> : k_ebe10<float, false, int64_t>);
      fn<<<grid, kBlock, 0, s>>>(m->E, n_rhs, rs, m->conn, m->rec32, m->rec64, (const float*)p_dev, (float*)q_dev,
                                 (float)alpha_M, (float)alpha_K, red, ptq_dev, nullptr, nullptr);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = precision == FEM_FP64 ? launch_mask<double>(m->N, n_rhs, m->fm, (double*)q_dev, s)
                              : launch_mask<float>(m->N, n_rhs, m->fm, (float*)q_dev, s);
  if (e != cudaSuccess) return set_error(FEM_ERR_CUDA, std::string("tet10 product: ") + cudaGetErrorString(e));
  return FEM_OK;
}

// Plain FP64 block-Jacobi PCG (Algorithm 1) on the tet10 system (alpha_M M + alpha_K K) x = b, the
// product being the tet10 EBE; the same device-side per-case CG kernels as the tet4 solver.
fem_status pcg10_solve(fem_mesh10* m, int precision, const double* b_dev, double* x_dev, int n_rhs, double alpha_M,
                       double alpha_K, double tol, int maxit, void* stream, int* iters_out, double* relres_out) {
  if (!m || !b_dev || !x_dev) return set_error(FEM_ERR_ARG, "null argument");
  if (precision != FEM_FP64 && precision != FEM_FP32_INNER) return set_error(FEM_ERR_ARG, "unknown precision");
  if (n_rhs < 1 || n_rhs > kMaxRpad || (n_rhs & (n_rhs - 1))) return set_error(FEM_ERR_ARG, "n_rhs must be 1, 2, 4, 8, 16 or 32");
  if (!(tol > 0.0) || maxit < 1) return set_error(FEM_ERR_ARG, "tol must be > 0 and maxit >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const int rpad = n_rhs, rs = lg2i(n_rhs);
  const size_t n = (size_t)m->N * 3 * rpad;
  double *D = nullptr, *b64 = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  float* b32 = nullptr;
  CgCase *sc = nullptr, *outer = nullptr;
  int *n_active = nullptr, *err = nullptr;
  float *r32 = nullptr, *x32 = nullptr, *rr32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;
  const bool mixed = precision == FEM_FP32_INNER;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  al((void**)&D, sizeof(double) * 6 * m->N);
  al((void**)&b64, sizeof(double) * 6 * m->N);
  al((void**)&b32, sizeof(float) * 6 * m->N);
  al((void**)&r, sizeof(double) * n);
  al((void**)&z, sizeof(double) * n);
  al((void**)&p, sizeof(double) * n);
  al((void**)&q, sizeof(double) * n);
  al((void**)&sc, sizeof(CgCase) * rpad);
  al((void**)&n_active, sizeof(int));
  al((void**)&err, sizeof(int));
  if (mixed) {
    al((void**)&outer, sizeof(CgCase) * rpad);
    for (float** v : {&r32, &x32, &rr32, &z32, &p32, &q32}) al((void**)v, sizeof(float) * n);
  }
  MeshView mv{m->N, m->E, nullptr, m->rec64, m->rec32, b64, b32, m->fm, nullptr, 0};
  const Reducer red{m->partial, m->counter, m->out};
  const int grid = grid_for(m->E << rs, red_grid_cap());
  auto product32 = [&](const float* in, float* out) {   // FP32 product with p^T q and the step length
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(float) * n, s);
    if (e != cudaSuccess) return;
    k_ebe10<float, true, int64_t><<<grid, kBlock, 0, s>>>(m->E, rpad, rs, m->conn, m->rec32, m->rec64, in, out,
                                                          (float)alpha_M, (float)alpha_K, red, nullptr, sc,
                                                          n_active);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_mask<float>(m->N, rpad, m->fm, out, s);
  };
  auto product = [&](const double* in, double* out, bool dot) {
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(double) * n, s);
    if (e != cudaSuccess) return;
    if (dot)
      k_ebe10<double, true, int64_t><<<grid, kBlock, 0, s>>>(m->E, rpad, rs, m->conn, m->rec32, m->rec64, in, out,
                                                             alpha_M, alpha_K, red, nullptr, sc, n_active);
    else
      k_ebe10<double, false, int64_t><<<grid, kBlock, 0, s>>>(m->E, rpad, rs, m->conn, m->rec32, m->rec64, in, out,
                                                              alpha_M, alpha_K, red, nullptr, nullptr, nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_mask<double>(m->N, rpad, m->fm, out, s);
  };
  if (e == cudaSuccess) e = cudaMemsetAsync(D, 0, sizeof(double) * 6 * m->N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_diag10<<<grid_for(m->E, wide_grid_cap()), kBlock, 0, s>>>(m->E, m->conn, m->rec64, alpha_M, alpha_K, m->mc, D);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_binv(m->N, D, m->fm, b64, b32, err, s);
  if (mixed) {
    // FP32-inner / FP64-outer refinement (the tet4 solver's form 1): r64 = b - A64 x (FP64 tet10 product),
    // inner FP32 PCG on A32 d = r64 from zero to the per-case target the outer residual sets, x += d
    if (e == cudaSuccess) e = launch_norm_b_gated<double>(mv, rpad, b_dev, red, outer, nullptr, tol, s);
    if (e == cudaSuccess) e = launch_zero_b0_t<double>(mv, rpad, x_dev, outer, s);
    std::vector<CgCase> ho(rpad);
    const double inner_tol = 1e-6;
    for (int outer_it = 0; outer_it <= 40 && e == cudaSuccess; ++outer_it) {
      product(x_dev, q, false);
      if (e == cudaSuccess) e = launch_outer_resid(mv, rpad, b_dev, q, r32, red, outer, n_active, tol, inner_tol,
                                                              0.1 * tol, s);
      int h_active = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h_active, n_active, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ho.data(), outer, sizeof(CgCase) * rpad, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess || h_active == 0) break;
      int used = 0;
      for (int c = 0; c < rpad; ++c) used = std::max(used, ho[c].iters);
      if (used >= maxit || outer_it == 40) break;
      if (e == cudaSuccess) e = launch_norm_b_gated<float>(mv, rpad, r32, red, sc, outer, inner_tol, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(x32, 0, sizeof(float) * n, s);
      if (e == cudaSuccess)
        e = launch_resid<float>(mv, rpad, r32, nullptr, x32, rr32, z32, 1, red, sc, n_active, inner_tol, maxit - used, s);
      for (int issued = 0; e == cudaSuccess && issued <= maxit - used + 64;) {
        for (int k = 0; k < 8 && e == cudaSuccess; ++k) {
          e = launch_dir_gated<float>(mv, rpad, z32, p32, sc, n_active, s);
          product32(p32, q32);
          if (e == cudaSuccess)
            e = launch_update<float>(mv, rpad, p32, q32, x32, rr32, z32, red, sc, n_active, inner_tol, maxit - used, s);
        }
        issued += 8;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_active, n_active, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (h_active == 0) break;
      }
      if (e == cudaSuccess) e = launch_refine_counts(mv, rpad, rpad, x_dev, x32, outer, sc, s);
    }
  } else {
    if (e == cudaSuccess) e = launch_norm_b_gated<double>(mv, rpad, b_dev, red, sc, nullptr, tol, s);
    // the guess is zeroed on Dirichlet DOFs (and for b = 0) before its residual is formed
    if (e == cudaSuccess) e = launch_zero_b0_t<double>(mv, rpad, x_dev, sc, s);
    product(x_dev, q, false);
    if (e == cudaSuccess) e = launch_resid<double>(mv, rpad, b_dev, q, x_dev, r, z, 1, red, sc, n_active, tol, maxit, s);
    int h_active = 1, issued = 0, checks = 0;
    while (e == cudaSuccess) {
      for (int k = 0; k < 8 && e == cudaSuccess; ++k) {
        e = launch_dir_gated<double>(mv, rpad, z, p, sc, n_active, s);
        product(p, q, true);
        if (e == cudaSuccess) e = launch_update<double>(mv, rpad, p, q, x_dev, r, z, red, sc, n_active, tol, maxit, s);
      }
      issued += 8;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h_active, n_active, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      if (h_active == 0) {
        // the recursive residual says converged: confirm with the true one (and resume if it is not)
        product(x_dev, q, false);
        if (e == cudaSuccess) e = launch_resid<double>(mv, rpad, b_dev, q, x_dev, r, z, 0, red, sc, n_active, tol, maxit, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_active, n_active, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || h_active == 0 || ++checks > 16) break;
      }
      if (issued > maxit + 64) break;
    }
  }
  std::vector<CgCase> h(rpad);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), mixed ? outer : sc, sizeof(CgCase) * rpad, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(D); cudaFree(b64); cudaFree(b32); cudaFree(r); cudaFree(z); cudaFree(p); cudaFree(q); cudaFree(sc);
  cudaFree(n_active); cudaFree(err); cudaFree(outer);
  for (float* v : {r32, x32, rr32, z32, p32, q32}) cudaFree(v);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(FEM_ERR_CUDA, std::string("tet10 solve: ") + cudaGetErrorString(e));
  }
  if (h_err) return set_error(FEM_ERR_ARG, "a node's diagonal block is not positive definite");
  fem_status worst = FEM_OK;
  for (int c = 0; c < rpad; ++c) {
    if (iters_out) iters_out[c] = h[c].iters;
    if (relres_out) relres_out[c] = h[c].relres;
    if (h[c].status != FEM_OK) worst = (fem_status)h[c].status;
    else if (h[c].active) worst = FEM_ERR_NOT_CONVERGED;
  }
  if (worst != FEM_OK) return set_error(worst, "tet10 solve: a case did not converge");
  return FEM_OK;
}

}  // extern "C"
