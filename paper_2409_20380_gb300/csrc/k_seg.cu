// Kernels of fused groups: several meshes concatenated into one node/element numbering, one case per mesh
// (rpad = 1), solved as one system whose Algorithm 1 scalars stay per case.  The case of node n is
// m.seg[n]; per-case sums go through shared-memory accumulators (seg_add) and one grid reduction.
// Loops run in whole rounds of the block so that every lane takes part in the warp-level aggregation.
#include "fem_internal.cuh"

namespace fem {

template <typename T> __device__ __forceinline__ const T* binv_of_s(const MeshView& m);
template <> __device__ __forceinline__ const double* binv_of_s<double>(const MeshView& m) { return m.binv64; }
template <> __device__ __forceinline__ const float* binv_of_s<float>(const MeshView& m) { return m.binv32; }

__device__ __forceinline__ void count_active_seg(const CgCase* sc, int ncase, int* n_active) {
  if (threadIdx.x == 0 && n_active) {
    int n = 0;
    for (int c = 0; c < ncase; ++c) n += sc[c].active;
    *n_active = n;
  }
}

__device__ __forceinline__ void zero_acc(double* acc, int n) {
  for (int t = threadIdx.x; t < n; t += blockDim.x) acc[t] = 0.0;
  __syncthreads();
}

template <typename T>
__global__ void k_norm_b_seg(MeshView m, const T* __restrict__ b, Reducer red, CgCase* sc, const CgCase* gate,
                             double tol) {
  extern __shared__ double acc[];
  const int nc = m.nseg;
  zero_acc(acc, nc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < m.N; base += stride) {
    const int64_t n = base + threadIdx.x;
    double v[1] = {0.0};
    int c = 0;
    if (n < m.N) {
      c = m.seg[n];
      const uint8_t f = m.freemask[n];
      for (int k = 0; k < 3; ++k)
        if (dof_free(f, k)) {
          const double x = (double)b[n * 3 + k];
          v[0] += x * x;
        }
    }
    seg_add<1>(acc, nc, c, v);
  }
  if (block_reduce_last_seg<1>(acc, nc, red)) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      CgCase& s = sc[c];
      s.bb = (gate && !gate[c].active) ? 0.0 : red.out[c];
      s.rho = s.pq = s.rr = s.alpha = s.beta = s.relres = s.relres0 = 0.0;
      s.active = 0;
      s.iters = 0;
      s.outer = 0;
      const double t = (gate && gate[c].inner_tol > 0.0) ? gate[c].inner_tol : tol;
      s.tol2 = t * t;
      s.status = isfinite(s.bb) ? FEM_OK : FEM_ERR_NONFINITE;
      s.phase = 0;
    }
  }
}

// r = b - q (q null: zero), masked; z = B^{-1} r; first solve start (x = 0 for b = 0 cases).
template <typename T>
__global__ void k_resid_seg(MeshView m, const T* __restrict__ b, const T* __restrict__ q, T* __restrict__ x,
                            T* __restrict__ r, T* __restrict__ z, Reducer red, CgCase* sc, int* n_active) {
  extern __shared__ double acc[];
  const int nc = m.nseg;
  zero_acc(acc, 2 * nc);
  const T* __restrict__ bi = binv_of_s<T>(m);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < m.N; base += stride) {
    const int64_t n = base + threadIdx.x;
    double v[2] = {0.0, 0.0};
    int c = 0;
    if (n < m.N) {
      c = m.seg[n];
      const uint8_t f = m.freemask[n];
      const bool zero_b = sc[c].bb == 0.0;
      T rv[3];
      for (int k = 0; k < 3; ++k) {
        const int64_t id = n * 3 + k;
        T val = b[id] - (q ? q[id] : (T)0);
        if (!dof_free(f, k) || zero_b) val = (T)0;
        rv[k] = val;
        r[id] = val;
        if (zero_b || !dof_free(f, k)) x[id] = (T)0;
      }
      const T* B = bi + n * 6;
      const T z0 = B[0] * rv[0] + B[3] * rv[1] + B[4] * rv[2];
      const T z1 = B[3] * rv[0] + B[1] * rv[1] + B[5] * rv[2];
      const T z2 = B[4] * rv[0] + B[5] * rv[1] + B[2] * rv[2];
      z[n * 3 + 0] = z0;
      z[n * 3 + 1] = z1;
      z[n * 3 + 2] = z2;
      v[0] = (double)(z0 * rv[0] + z1 * rv[1] + z2 * rv[2]);
      v[1] = (double)(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    }
    seg_add<2>(acc, nc, c, v);
  }
  if (block_reduce_last_seg<2>(acc, nc, red)) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      CgCase& s = sc[c];
      const double zrc = red.out[c], rrc = red.out[nc + c];
      s.rho = zrc;
      s.rr = rrc;
      s.beta = 0.0;
      s.phase = 0;
      s.relres = s.bb > 0.0 ? sqrt(rrc / s.bb) : 0.0;
      s.relres0 = s.relres;
      if (!isfinite(rrc) || !isfinite(zrc)) s.status = FEM_ERR_NONFINITE;
      s.active = (s.status == FEM_OK && s.bb > 0.0 && rrc >= s.tol2 * s.bb) ? 1 : 0;
    }
    __syncthreads();
    count_active_seg(sc, nc, n_active);
  }
}

template <typename T>
__global__ void k_dir_seg(MeshView m, const T* __restrict__ z, T* __restrict__ p, const CgCase* sc,
                          const int* n_active) {
  if (*n_active == 0) return;
  const int64_t total = m.N * 3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const CgCase& s = sc[m.seg[i / 3]];
    if (!s.active) continue;
    p[i] = z[i] + (T)(s.phase ? s.beta : 0.0) * p[i];
  }
}

template <typename T>
__global__ void k_update_seg(MeshView m, const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ x,
                             T* __restrict__ r, T* __restrict__ z, Reducer red, CgCase* sc, int* n_active, int maxit) {
  if (*n_active == 0) return;
  extern __shared__ double acc[];
  const int nc = m.nseg;
  zero_acc(acc, 2 * nc);
  const T* __restrict__ bi = binv_of_s<T>(m);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < m.N; base += stride) {
    const int64_t n = base + threadIdx.x;
    double v[2] = {0.0, 0.0};
    int c = 0;
    if (n < m.N) {
      c = m.seg[n];
      const uint8_t f = m.freemask[n];
      const T alpha = (T)sc[c].alpha;
      T rv[3];
      for (int k = 0; k < 3; ++k) {
        const int64_t id = n * 3 + k;
        T rk = r[id];
        if (alpha != (T)0) {
          x[id] += alpha * p[id];
          if (dof_free(f, k)) rk -= alpha * q[id];
          r[id] = rk;
        }
        rv[k] = rk;
      }
      const T* B = bi + n * 6;
      const T z0 = B[0] * rv[0] + B[3] * rv[1] + B[4] * rv[2];
      const T z1 = B[3] * rv[0] + B[1] * rv[1] + B[5] * rv[2];
      const T z2 = B[4] * rv[0] + B[5] * rv[1] + B[2] * rv[2];
      z[n * 3 + 0] = z0;
      z[n * 3 + 1] = z1;
      z[n * 3 + 2] = z2;
      v[0] = (double)(z0 * rv[0] + z1 * rv[1] + z2 * rv[2]);
      v[1] = (double)(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    }
    seg_add<2>(acc, nc, c, v);
  }
  if (block_reduce_last_seg<2>(acc, nc, red)) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      CgCase& s = sc[c];
      if (!s.active) continue;
      const double zrc = red.out[c], rrc = red.out[nc + c];
      s.beta = zrc / s.rho;
      s.rho = zrc;
      s.rr = rrc;
      s.iters += 1;
      s.phase = 1;
      s.relres = sqrt(rrc / s.bb);
      if (!isfinite(zrc) || !isfinite(rrc)) {
        s.status = FEM_ERR_NONFINITE;
        s.active = 0;
      } else if (rrc < s.tol2 * s.bb) {
        s.active = 0;
      } else if (s.iters >= maxit) {
        s.active = 0;
        s.status = FEM_ERR_NOT_CONVERGED;
      }
    }
    __syncthreads();
    count_active_seg(sc, nc, n_active);
  }
}

// Residual of the guess from the recurrences (fused form of k_r0; ALT: the guess guard's norms of the
// Adams-Bashforth guess's residual r0 + A y and the per-case choice, as in k_r0).
template <bool ALT>
__global__ void k_r0_seg(MeshView m, double h, const double* __restrict__ b, const double* __restrict__ Av4,
                         const double* __restrict__ Av3, const double* __restrict__ Av2, const double* __restrict__ Av1,
                         const float* __restrict__ qy, float* __restrict__ r32, Reducer red, CgCase* outer,
                         int* n_active, double tol, double inner_floor, double aim, Ring4 avr, const StepCtl* ctl,
                         int* fallbacks) {
  if (ctl) {   // A v^{it-4} .. A v^{it-1} in ring slots it .. it+3 (mod 4)
    const int it = ctl->it;
    Av4 = avr.p[it & 3], Av3 = avr.p[(it + 1) & 3], Av2 = avr.p[(it + 2) & 3], Av1 = avr.p[(it + 3) & 3];
  }
  constexpr int NQ = ALT ? 3 : 2;
  extern __shared__ double acc[];
  const int nc = m.nseg;
  zero_acc(acc, NQ * nc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < m.N; base += stride) {
    const int64_t n = base + threadIdx.x;
    double v[NQ];
    for (int q = 0; q < NQ; ++q) v[q] = 0.0;
    int c = 0;
    if (n < m.N) {
      c = m.seg[n];
      const uint8_t f = m.freemask[n];
      for (int k = 0; k < 3; ++k) {
        const int64_t id = n * 3 + k;
        double val = 0.0;
        float qv = 0.f;
        const double bv = b[id];
        if (dof_free(f, k)) {
          val = bv - h * (-9.0 * Av4[id] + 37.0 * Av3[id] - 59.0 * Av2[id] + 55.0 * Av1[id]);
          if (qy) {
            qv = qy[id];
            val -= f2d(qv);
          }
        }
        const float rf = d2f(val);
        r32[id] = rf;
        v[0] += bv * bv;
        v[1] += val * val;
        if (ALT) {
          const float fa = dof_free(f, k) ? rf + qv : 0.f;
          v[NQ - 1] += (double)(fa * fa);
        }
      }
    }
    seg_add<NQ>(acc, nc, c, v);
  }
  if (block_reduce_last_seg<NQ>(acc, nc, red)) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      CgCase& s = outer[c];
      const double bbc = red.out[c];
      double rrc = red.out[nc + c];
      s.guess = qy ? 1 : 0;
      if (ALT) {
        const double rra = red.out[2 * nc + c];
        if (bbc > 0.0 && isfinite(rra) && (!isfinite(rrc) || rra < rrc * (1.0 - 1e-6))) {
          rrc = rra;
          s.guess = 2;
          if (fallbacks) fallbacks[c] += 1;
        }
      }
      s.rho = s.pq = s.alpha = s.beta = 0.0;
      s.iters = 0;
      s.outer = 0;
      s.phase = 0;
      s.bb = bbc;
      s.rr = rrc;
      s.relres = bbc > 0.0 ? sqrt(rrc / bbc) : 0.0;
      s.relres0 = s.relres;
      s.status = (isfinite(bbc) && isfinite(rrc)) ? FEM_OK : FEM_ERR_NONFINITE;
      s.active = (s.status == FEM_OK && bbc > 0.0 && rrc >= tol * tol * bbc) ? 1 : 0;
      s.inner_tol = inner_target(aim, s.relres, inner_floor);
    }
    __syncthreads();
    count_active_seg(outer, nc, n_active);
  }
}

__global__ void k_cert_seg(MeshView m, double cM, double cK, const double* __restrict__ b,
                           const double* __restrict__ qM, const double* __restrict__ qK, float* __restrict__ r32,
                           Reducer red, CgCase* outer, int* n_active, double tol, double inner_floor, double aim) {
  extern __shared__ double acc[];
  const int nc = m.nseg;
  zero_acc(acc, nc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < m.N; base += stride) {
    const int64_t n = base + threadIdx.x;
    double v[1] = {0.0};
    int c = 0;
    if (n < m.N) {
      c = m.seg[n];
      const uint8_t f = m.freemask[n];
      for (int k = 0; k < 3; ++k) {
        const int64_t id = n * 3 + k;
        const double val = dof_free(f, k) ? b[id] - (cM * qM[id] + cK * qK[id]) : 0.0;
        r32[id] = d2f(val);
        v[0] += val * val;
      }
    }
    seg_add<1>(acc, nc, c, v);
  }
  if (block_reduce_last_seg<1>(acc, nc, red)) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      CgCase& s = outer[c];
      const double rrc = red.out[c];
      s.rr = rrc;
      s.relres = s.bb > 0.0 ? sqrt(rrc / s.bb) : 0.0;
      s.outer += 1;
      if (!isfinite(rrc)) s.status = FEM_ERR_NONFINITE;
      s.active = (s.status == FEM_OK && s.bb > 0.0 && rrc >= tol * tol * s.bb) ? 1 : 0;
      s.inner_tol = inner_target(aim, s.relres, inner_floor);
    }
    __syncthreads();
    count_active_seg(outer, nc, n_active);
  }
}

// ---- launchers ----
static int seg_grid(int64_t items) {
  int64_t g = (items + kVecBlock - 1) / kVecBlock;
  if (g < 1) g = 1;
  if (g > vec_grid_cap()) g = vec_grid_cap();
  return (int)g;
}

template <typename T>
cudaError_t launch_norm_b_seg(const MeshView& m, const T* b, Reducer red, CgCase* sc, const CgCase* gate, double tol,
                              cudaStream_t s) {
  k_norm_b_seg<T><<<seg_grid(m.N), kVecBlock, sizeof(double) * m.nseg, s>>>(m, b, red, sc, gate, tol);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_resid_seg(const MeshView& m, const T* b, const T* q, T* x, T* r, T* z, Reducer red, CgCase* sc,
                             int* n_active, cudaStream_t s) {
  k_resid_seg<T><<<seg_grid(m.N), kVecBlock, sizeof(double) * 2 * m.nseg, s>>>(m, b, q, x, r, z, red, sc, n_active);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dir_seg(const MeshView& m, const T* z, T* p, const CgCase* sc, const int* n_active, cudaStream_t s) {
  k_dir_seg<T><<<grid_for(m.N * 3), kBlock, 0, s>>>(m, z, p, sc, n_active);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_update_seg(const MeshView& m, const T* p, const T* q, T* x, T* r, T* z, Reducer red, CgCase* sc,
                              int* n_active, int maxit, cudaStream_t s) {
  k_update_seg<T><<<seg_grid(m.N), kVecBlock, sizeof(double) * 2 * m.nseg, s>>>(m, p, q, x, r, z, red, sc, n_active,
                                                                                 maxit);
  return cudaGetLastError();
}
cudaError_t launch_r0_seg(const MeshView& m, double dt, const double* b, const double* Av4, const double* Av3,
                          const double* Av2, const double* Av1, const float* qy, float* r32, Reducer red,
                          CgCase* outer, int* n_active, double tol, double inner_floor, double aim, cudaStream_t s,
                          Ring4 avr, const StepCtl* ctl, bool guard, int* fallbacks) {
  if (guard && qy) {
    k_r0_seg<true><<<seg_grid(m.N), kVecBlock, sizeof(double) * 3 * m.nseg, s>>>(
        m, dt / 24.0, b, Av4, Av3, Av2, Av1, qy, r32, red, outer, n_active, tol, inner_floor, aim, avr, ctl, fallbacks);
  } else {
    k_r0_seg<false><<<seg_grid(m.N), kVecBlock, sizeof(double) * 2 * m.nseg, s>>>(
        m, dt / 24.0, b, Av4, Av3, Av2, Av1, qy, r32, red, outer, n_active, tol, inner_floor, aim, avr, ctl, nullptr);
  }
  return cudaGetLastError();
}
cudaError_t launch_cert_seg(const MeshView& m, double cM, double cK, const double* b, const double* qM, const double* qK,
                            float* r32, Reducer red, CgCase* outer, int* n_active, double tol, double inner_floor,
                            double aim, cudaStream_t s) {
  k_cert_seg<<<seg_grid(m.N), kVecBlock, sizeof(double) * m.nseg, s>>>(m, cM, cK, b, qM, qK, r32, red, outer,
                                                                        n_active, tol, inner_floor, aim);
  return cudaGetLastError();
}

#define INST(T)                                                                                                      \
  template cudaError_t launch_norm_b_seg<T>(const MeshView&, const T*, Reducer, CgCase*, const CgCase*, double,      \
                                            cudaStream_t);                                                           \
  template cudaError_t launch_resid_seg<T>(const MeshView&, const T*, const T*, T*, T*, T*, Reducer, CgCase*, int*,  \
                                           cudaStream_t);                                                            \
  template cudaError_t launch_dir_seg<T>(const MeshView&, const T*, T*, const CgCase*, const int*, cudaStream_t);    \
  template cudaError_t launch_update_seg<T>(const MeshView&, const T*, const T*, T*, T*, T*, Reducer, CgCase*, int*,  \
                                            int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace fem
