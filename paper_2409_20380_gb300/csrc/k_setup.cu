// Mesh setup on the GPU: element records for the EBE product (Section 3.2, Eq. eqebefem) and the 3x3
// block-Jacobi preconditioner of Algorithm 1.
#include "fem_internal.cuh"

#include <mutex>
#include <vector>
#include <algorithm>
#include <unordered_map>

namespace fem {

// One full wave of resident blocks for grid-stride kernels: SMs x blocks of `fn` that fit on one SM (the
// occupancy query is made once per kernel).
int grid_resident(const void* fn, int block, int64_t items) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  int waves;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(fn);
    if (it == cache.end()) {
      int per_sm = 1;
      const int nsm = sm_count();
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      it = cache.emplace(fn, nsm * per_sm).first;
    }
    waves = it->second;
  }
  int64_t g = (items + block - 1) / block;
  if (g < 1) g = 1;
  if (g > waves) g = waves;
  return (int)g;
}

int sm_count() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 1;
    }
    it = cache.emplace(dev, n).first;
  }
  return it->second;
}
int vec_grid_cap() { return std::min(3 * sm_count(), kMaxRedBlocks); }
int red_grid_cap() { return std::min(8 * sm_count(), kMaxRedBlocks); }
int wide_grid_cap() { return 16 * sm_count(); }

int grid_for(int64_t items, int cap) {
  if (cap < 0) cap = red_grid_cap();
  int64_t g = (items + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Linear tet: x = x0 + J xi, J = [e1 e2 e3] (columns).  The gradients of N1..N3 are the rows of J^{-1}:
// (e2 x e3, e3 x e1, e1 x e2) / det J; N0's is minus their sum; volume = det J / 6.
__global__ void k_elem_setup(int64_t E, int64_t N, const double* __restrict__ xyz, const int4* __restrict__ conn,
                             const int32_t* __restrict__ mat, int n_mat, const double* __restrict__ lmr,
                             double* __restrict__ rec64, float* __restrict__ rec32, int* err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int4 c = conn[e];
    const int nd[4] = {c.x, c.y, c.z, c.w};
    bool bad = false;
    for (int a = 0; a < 4; ++a) bad |= (nd[a] < 0 || nd[a] >= N);
    const int mi = mat[e];
    bad |= (mi < 0 || mi >= n_mat);
    if (bad) {
      atomicOr(err, 1);
      continue;
    }
    double x[4][3];
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) x[a][k] = xyz[(int64_t)nd[a] * 3 + k];
    double e1[3], e2[3], e3[3];
    for (int k = 0; k < 3; ++k) {
      e1[k] = x[1][k] - x[0][k];
      e2[k] = x[2][k] - x[0][k];
      e3[k] = x[3][k] - x[0][k];
    }
    const double c23[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2], e2[0] * e3[1] - e2[1] * e3[0]};
    const double c31[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
    const double c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double det = e1[0] * c23[0] + e1[1] * c23[1] + e1[2] * c23[2];
    if (!(det > 0.0) || !isfinite(det)) {
      atomicOr(err, 2);
      continue;
    }
    const double inv = 1.0 / det;
    const double V = det / 6.0;
    double r[kRec];
    for (int k = 0; k < 3; ++k) {
      r[0 + k] = c23[k] * inv;
      r[3 + k] = c31[k] * inv;
      r[6 + k] = c12[k] * inv;
    }
    r[9] = lmr[mi * 3 + 0] * V;
    r[10] = lmr[mi * 3 + 1] * V;
    r[11] = lmr[mi * 3 + 2] * V / 20.0;
    for (int j = 0; j < kRec; ++j) {
      rec64[e * kRec + j] = r[j];
      rec32[e * kRec + j] = (float)r[j];
    }
  }
}

// Diagonal 3x3 block of A_e at local node a:
//   K_e[a i, a j] = V (lambda g_ai g_aj + mu g_aj g_ai + mu delta_ij |g_a|^2),  M_e[a i, a j] = 2 rho V/20 delta_ij.
__global__ void k_diag_blocks(MeshView m, double aM, double aK, double* __restrict__ D) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.E; e += (int64_t)gridDim.x * blockDim.x) {
    const double* r = m.rec64 + e * kRec;
    double g[4][3];
    for (int k = 0; k < 3; ++k) {
      g[1][k] = r[k];
      g[2][k] = r[3 + k];
      g[3][k] = r[6 + k];
      g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
    }
    const double lam = aK * r[9], mu = aK * r[10], ms = aM * 2.0 * r[11];
    const int4 c = m.conn[e];
    const int nd[4] = {c.x, c.y, c.z, c.w};
    for (int a = 0; a < 4; ++a) {
      const double gg = g[a][0] * g[a][0] + g[a][1] * g[a][1] + g[a][2] * g[a][2];
      const double lm = lam + mu;
      double* d = D + (int64_t)nd[a] * 6;
      atomicAdd(d + 0, lm * g[a][0] * g[a][0] + mu * gg + ms);
      atomicAdd(d + 1, lm * g[a][1] * g[a][1] + mu * gg + ms);
      atomicAdd(d + 2, lm * g[a][2] * g[a][2] + mu * gg + ms);
      atomicAdd(d + 3, lm * g[a][0] * g[a][1]);
      atomicAdd(d + 4, lm * g[a][0] * g[a][2]);
      atomicAdd(d + 5, lm * g[a][1] * g[a][2]);
    }
  }
}

// Inverse of each node's block restricted to its free DOFs (fixed rows/cols -> identity, inverted by the
// adjugate, then zeroed), so that z = B^{-1} r is zero on Dirichlet DOFs.
__global__ void k_binv(int64_t N, const double* __restrict__ D, const uint8_t* __restrict__ fm,
                       double* __restrict__ b64, float* __restrict__ b32, int* err) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t f = fm[n];
    double a[3][3];
    const double* d = D + n * 6;
    a[0][0] = d[0]; a[1][1] = d[1]; a[2][2] = d[2];
    a[0][1] = a[1][0] = d[3];
    a[0][2] = a[2][0] = d[4];
    a[1][2] = a[2][1] = d[5];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        if (!dof_free(f, i) || !dof_free(f, j)) a[i][j] = (i == j) ? 1.0 : 0.0;
    const double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    const double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    const double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    const double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
    if (!(det > 0.0) || !isfinite(det)) {
      atomicOr(err, 4);
      for (int j = 0; j < 6; ++j) { b64[n * 6 + j] = 0.0; b32[n * 6 + j] = 0.f; }
      continue;
    }
    const double id = 1.0 / det;
    double inv[3][3];
    inv[0][0] = c00 * id;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        if (!dof_free(f, i) || !dof_free(f, j)) {
          if (i <= j) inv[i][j] = 0.0;
        }
    const double o[6] = {inv[0][0], inv[1][1], inv[2][2], inv[0][1], inv[0][2], inv[1][2]};
    for (int j = 0; j < 6; ++j) {
      b64[n * 6 + j] = o[j];
      b32[n * 6 + j] = (float)o[j];
    }
  }
}

cudaError_t launch_elem_setup(int64_t E, int64_t N, const double* xyz, const int4* conn, const int32_t* mat,
                              int n_mat, const double* lmr, double* rec64, float* rec32, int* err_flag,
                              cudaStream_t s) {
  k_elem_setup<<<grid_for(E, wide_grid_cap()), kBlock, 0, s>>>(E, N, xyz, conn, mat, n_mat, lmr, rec64, rec32, err_flag);
  return cudaGetLastError();
}

cudaError_t launch_diag_blocks(const MeshView& m, double aM, double aK, double* D, cudaStream_t s) {
  k_diag_blocks<<<grid_for(m.E, wide_grid_cap()), kBlock, 0, s>>>(m, aM, aK, D);
  return cudaGetLastError();
}

cudaError_t launch_binv(int64_t N, const double* D, const uint8_t* freemask, double* binv64, float* binv32,
                        int* err_flag, cudaStream_t s) {
  k_binv<<<grid_for(N, wide_grid_cap()), kBlock, 0, s>>>(N, D, freemask, binv64, binv32, err_flag);
  return cudaGetLastError();
}

// Per-node element-wise absolute row sums: for local node a and component i of element e,
// sum_b sum_k |K^e_ab[i][k]| with K^e_ab = lambdaV g_a g_b^T + muV (g_a . g_b) I + muV g_b g_a^T, and
// sum_b |M^e_ab| = 5 rho V / 20 (M^e_ab = rho V / 20 (1 + delta_ab) I).
__global__ void k_abs_rows(MeshView m, double* __restrict__ mrow, double* __restrict__ krow) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.E; e += (int64_t)gridDim.x * blockDim.x) {
    const double* r = m.rec64 + e * kRec;
    double g[4][3];
    for (int k = 0; k < 3; ++k) {
      g[1][k] = r[k];
      g[2][k] = r[3 + k];
      g[3][k] = r[6 + k];
      g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
    }
    const double lam = r[9], mu = r[10], ms = r[11];
    const int4 cn = m.conn[e];
    const int nd[4] = {cn.x, cn.y, cn.z, cn.w};
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        double ks = 0.0;
        for (int b = 0; b < 4; ++b) {
          const double gab = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
          for (int k = 0; k < 3; ++k) ks += fabs(lam * g[a][i] * g[b][k] + mu * g[b][i] * g[a][k] + (i == k ? mu * gab : 0.0));
        }
        atomicAdd(krow + (int64_t)nd[a] * 3 + i, ks);
        atomicAdd(mrow + (int64_t)nd[a] * 3 + i, 5.0 * fabs(ms));
      }
  }
}

cudaError_t elem_abs_row_bounds(const MeshView& m, double* abs_m, double* abs_k, cudaStream_t s) {
  double *mrow = nullptr, *krow = nullptr;
  const size_t n = (size_t)m.N * 3;
  cudaError_t e = cudaMalloc(&mrow, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&krow, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMemsetAsync(mrow, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(krow, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) {
    k_abs_rows<<<grid_for(m.E), kBlock, 0, s>>>(m, mrow, krow);
    e = cudaGetLastError();
  }
  std::vector<double> hm(n), hk(n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hm.data(), mrow, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hk.data(), krow, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(mrow);
  cudaFree(krow);
  if (e != cudaSuccess) return e;
  double bm = 0.0, bk = 0.0;
  for (size_t i = 0; i < n; ++i) bm = std::max(bm, hm[i]), bk = std::max(bk, hk[i]);
  *abs_m = bm;
  *abs_k = bk;
  return cudaSuccess;
}

}  // namespace fem
