// Vector kernels of Algorithm 1 (block-Jacobi PCG) on [N][3][rpad] data, fused so that each iteration
// makes three passes: direction (p = z + beta p), EBE (q = A p with p^T q fused), and the update
// (x += alpha p, r -= alpha q, z = B^{-1} r, (z, r), (r, r)).  Per-case scalars live on the device and
// are advanced by the last block of each reducing kernel, so the host only polls the active count.
#include "fem_internal.cuh"

namespace fem {

template <typename T> struct Acc { using type = double; };
template <> struct Acc<float> { using type = float; };

template <typename T> __device__ __forceinline__ const T* binv_of(const MeshView& m);
template <> __device__ __forceinline__ const double* binv_of<double>(const MeshView& m) { return m.binv64; }
template <> __device__ __forceinline__ const float* binv_of<float>(const MeshView& m) { return m.binv32; }

static int vec_grid(int64_t items) {
  int64_t g = (items + kVecBlock - 1) / kVecBlock;
  if (g < 1) g = 1;
  if (g > vec_grid_cap()) g = vec_grid_cap();
  return (int)g;
}

static int log2i(int r) {
  int s = 0;
  while ((1 << s) < r) ++s;
  return s;
}

__device__ __forceinline__ void count_active(const CgCase* sc, int rpad, int* n_active) {
  if (threadIdx.x == 0 && n_active) {
    int n = 0;
    for (int c = 0; c < rpad; ++c) n += sc[c].active;
    *n_active = n;
  }
}

// bb = ||b||^2 over free DOFs; resets the case state.  gate (optional): a case whose gate is inactive is
// treated as b = 0.
template <typename T>
__global__ void __launch_bounds__(kVecBlock, 3) k_norm_b(MeshView m, int rpad, int rshift, const T* __restrict__ b,
                                                   Reducer red, CgCase* sc, const CgCase* gate, double tol) {
  typename Acc<T>::type acc = 0;
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T v = b[(n * 3 + k) * rpad + c];
      if (dof_free(f, k)) acc += v * v;
    }
  }
  double v[1] = {(double)acc};
  if (block_reduce_last<1>(v, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
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

// r = b - q (q may be null: zero), masked; first: x = 0 for cases with b = 0.  z = B^{-1} r.
// Tail (first): start the iteration.  Tail (re-check): true-residual test of cases that stopped on the
// recursive residual; they resume if the true residual is above tol.
template <typename T>
__global__ void __launch_bounds__(kVecBlock, 3) k_resid(MeshView m, int rpad, int rshift, const T* __restrict__ b,
                                                  const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                                                  T* __restrict__ z, int first, Reducer red, CgCase* sc,
                                                  int* n_active, double tol, int maxit) {
  const T* __restrict__ bi = binv_of<T>(m);
  typename Acc<T>::type zr = 0, rr = 0;
  const int64_t total = m.N << rshift;
  const bool zero_case = sc[(blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & (rpad - 1)].bb == 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
    const bool zero_b = first && zero_case;
    T rv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t id = (n * 3 + k) * rpad + c;
      T v = b[id] - (q ? q[id] : (T)0);
      if (!dof_free(f, k) || zero_b) v = (T)0;
      rv[k] = v;
      r[id] = v;
      if (zero_b || !dof_free(f, k)) x[id] = (T)0;
    }
    const T* B = bi + n * 6;
    const T z0 = B[0] * rv[0] + B[3] * rv[1] + B[4] * rv[2];
    const T z1 = B[3] * rv[0] + B[1] * rv[1] + B[5] * rv[2];
    const T z2 = B[4] * rv[0] + B[5] * rv[1] + B[2] * rv[2];
    z[(n * 3 + 0) * rpad + c] = z0;
    z[(n * 3 + 1) * rpad + c] = z1;
    z[(n * 3 + 2) * rpad + c] = z2;
    zr += z0 * rv[0] + z1 * rv[1] + z2 * rv[2];
    rr += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
  }
  double v[2] = {(double)zr, (double)rr};
  if (block_reduce_last<2>(v, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
      CgCase& s = sc[c];
      const double zrc = red.out[c], rrc = red.out[rpad + c];
      const double thr = s.tol2 * s.bb;
      if (first) {
        s.rho = zrc;
        s.rr = rrc;
        s.beta = 0.0;
        s.phase = 0;
        s.relres = s.bb > 0.0 ? sqrt(rrc / s.bb) : 0.0;
        s.relres0 = s.relres;
        if (!isfinite(rrc) || !isfinite(zrc)) s.status = FEM_ERR_NONFINITE;
        s.active = (s.status == FEM_OK && s.bb > 0.0 && rrc >= thr) ? 1 : 0;
      } else if (s.status == FEM_OK && !s.active && s.bb > 0.0) {
        s.rr = rrc;
        s.relres = sqrt(rrc / s.bb);
        if (rrc >= thr) {
          if (s.iters >= maxit) {
            s.status = FEM_ERR_NOT_CONVERGED;
          } else {
            s.beta = (s.phase && s.rho != 0.0) ? zrc / s.rho : 0.0;
            s.rho = zrc;
            s.active = 1;
          }
        }
      }
    }
    __syncthreads();
    count_active(sc, rpad, n_active);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_dir(MeshView m, int rpad, int rshift, const T* __restrict__ z,
                                                T* __restrict__ p, const CgCase* sc, const int* n_active) {
  if (*n_active == 0) return;
  const int64_t total = (m.N * 3) << rshift;
  // the grid stride is a multiple of rpad: every thread serves one case
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & (rpad - 1));
  const CgCase s = sc[c];
  if (!s.active) return;
  const T beta = (T)(s.phase ? s.beta : 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

template <typename T>
__global__ void __launch_bounds__(kVecBlock, 3) k_update(MeshView m, int rpad, int rshift, const T* __restrict__ p,
                                                   const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                                                   T* __restrict__ z, Reducer red, CgCase* sc, int* n_active,
                                                   double tol, int maxit) {
  if (*n_active == 0) return;
  const T* __restrict__ bi = binv_of<T>(m);
  typename Acc<T>::type zr = 0, rr = 0;
  const int64_t total = m.N << rshift;
  const T alpha = (T)sc[(blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & (rpad - 1)].alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
    T rv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t id = (n * 3 + k) * rpad + c;
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
    z[(n * 3 + 0) * rpad + c] = z0;
    z[(n * 3 + 1) * rpad + c] = z1;
    z[(n * 3 + 2) * rpad + c] = z2;
    zr += z0 * rv[0] + z1 * rv[1] + z2 * rv[2];
    rr += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
  }
  double v[2] = {(double)zr, (double)rr};
  if (block_reduce_last<2>(v, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
      CgCase& s = sc[c];
      if (s.active) {
        const double zrc = red.out[c], rrc = red.out[rpad + c];
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
    }
    __syncthreads();
    count_active(sc, rpad, n_active);
  }
}

// Deferred-update form of the iteration (the FP32 inner solves, which do not test the true residual): the
// direction pass forms z = B^{-1} r itself and applies the previous step's x += alpha p while it reads p,
// so the update pass reads only q and r and stores only r (z is never stored): 8 vector passes an
// iteration instead of 10.  A case that has stopped keeps its last alpha until a later direction pass or
// the final refinement (k_refine_pending) applies it; the product's tail then zeroes it.
template <typename T>
__global__ void __launch_bounds__(kVecBlock, 3) k_dir_defer(MeshView m, int rpad, int rshift, const T* __restrict__ r,
                                                      T* __restrict__ p, T* __restrict__ x, const CgCase* sc,
                                                      const int* n_active) {
  if (*n_active == 0) return;
  // the grid stride is a multiple of rpad: every thread serves one case
  const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & (rpad - 1));
  const bool act = sc[c].active != 0;
  const T alpha = (T)sc[c].alpha;
  if (!act && alpha == (T)0) return;
  const T beta = (T)(sc[c].phase ? sc[c].beta : 0.0);
  const T* __restrict__ bi = binv_of<T>(m);
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int64_t id0 = n * 3 * rpad + c;
    T pv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      pv[k] = p[id0 + k * rpad];
      if (alpha != (T)0) x[id0 + k * rpad] += alpha * pv[k];
    }
    if (act) {
      const T r0 = r[id0], r1 = r[id0 + rpad], r2 = r[id0 + 2 * rpad];
      const T* B = bi + n * 6;
      p[id0] = B[0] * r0 + B[3] * r1 + B[4] * r2 + beta * pv[0];
      p[id0 + rpad] = B[3] * r0 + B[1] * r1 + B[5] * r2 + beta * pv[1];
      p[id0 + 2 * rpad] = B[4] * r0 + B[5] * r1 + B[2] * r2 + beta * pv[2];
    }
  }
}

// r -= alpha q on free DOFs; (B^{-1} r, r) and (r, r) reduced; the same per-case tail as k_update.
template <typename T>
__global__ void __launch_bounds__(kVecBlock, 2) k_update_defer(MeshView m, int rpad, int rshift,
                                                         const T* __restrict__ q, T* __restrict__ r, Reducer red,
                                                         CgCase* sc, int* n_active, int maxit) {
  if (*n_active == 0) return;
  const T* __restrict__ bi = binv_of<T>(m);
  typename Acc<T>::type zr = 0, rr = 0;
  const int64_t total = m.N << rshift;
  const T alpha = (T)sc[(blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & (rpad - 1)].alpha;
  // two items an iteration (the grid stride apart: the same case), all their loads -- r, q, the free-DOF
  // bits and B^-1 -- issued before either is updated: two memory round trips' worth of bytes in flight
  struct Item {
    T rv[3], qv[3], B[6];
    uint8_t f;
    int64_t id0;
  };
  auto load = [&](int64_t i, Item& it) {
    const int64_t n = i >> rshift;
    it.id0 = n * 3 * rpad + (int)(i & (rpad - 1));
    it.f = m.freemask[n];
#pragma unroll
    for (int k = 0; k < 3; ++k) it.rv[k] = r[it.id0 + k * rpad];
    if (alpha != (T)0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) it.qv[k] = q[it.id0 + k * rpad];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) it.B[k] = bi[n * 6 + k];
  };
  auto apply = [&](Item& it) {
    if (alpha != (T)0) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (dof_free(it.f, k)) {
          it.rv[k] -= alpha * it.qv[k];
          r[it.id0 + k * rpad] = it.rv[k];
        }
    }
    const T* B = it.B;
    const T* rv = it.rv;
    const T z0 = B[0] * rv[0] + B[3] * rv[1] + B[4] * rv[2];
    const T z1 = B[3] * rv[0] + B[1] * rv[1] + B[5] * rv[2];
    const T z2 = B[4] * rv[0] + B[5] * rv[1] + B[2] * rv[2];
    zr += z0 * rv[0] + z1 * rv[1] + z2 * rv[2];
    rr += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += 2 * stride) {
    Item a, b;
    const bool two = i + stride < total;
    load(i, a);
    if (two) load(i + stride, b);
    apply(a);
    if (two) apply(b);
  }
  double v[2] = {(double)zr, (double)rr};
  if (block_reduce_last<2>(v, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
      CgCase& s = sc[c];
      if (s.active) {
        const double zrc = red.out[c], rrc = red.out[rpad + c];
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
    }
    __syncthreads();
    count_active(sc, rpad, n_active);
  }
}

// ---- mixed precision: FP64 outer residual -> FP32 inner right-hand side; FP64 refinement update ----
__global__ void __launch_bounds__(kVecBlock, 3) k_outer_resid(MeshView m, int rpad, int rshift, const double* __restrict__ b,
                                                        const double* __restrict__ q, float* __restrict__ r32,
                                                        Reducer red, CgCase* outer, int* n_active, double tol,
                                                        double inner_max, double aim) {
  double rr = 0.0;
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t id = (n * 3 + k) * rpad + c;
      const double v = dof_free(f, k) ? b[id] - q[id] : 0.0;
      r32[id] = d2f(v);
      rr += v * v;
    }
  }
  double v[1] = {rr};
  if (block_reduce_last<1>(v, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
      CgCase& s = outer[c];
      const double rrc = red.out[c];
      s.rr = rrc;
      s.relres = s.bb > 0.0 ? sqrt(rrc / s.bb) : 0.0;
      if (s.outer == 0) s.relres0 = s.relres;
      s.outer += 1;
      if (!isfinite(rrc)) s.status = FEM_ERR_NONFINITE;
      s.active = (s.status == FEM_OK && s.bb > 0.0 && rrc >= tol * tol * s.bb) ? 1 : 0;
      s.inner_tol = inner_target(aim, s.relres, inner_max);
    }
    __syncthreads();
    count_active(outer, rpad, n_active);
  }
}

// x += d (FP64 accumulation of the FP32 correction); block 0 adds the inner iteration counts.
__global__ void k_refine(int64_t n_items, int ncase, double* __restrict__ x, const float* __restrict__ d,
                         CgCase* outer, const CgCase* inner) {
  if (blockIdx.x == 0 && threadIdx.x < ncase) {
    outer[threadIdx.x].iters += inner[threadIdx.x].iters;
    if (inner[threadIdx.x].status == FEM_ERR_BREAKDOWN || inner[threadIdx.x].status == FEM_ERR_NONFINITE)
      outer[threadIdx.x].status = inner[threadIdx.x].status;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_items; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += f2d(d[i]);
}

// The same after a deferred-update inner solve: x += d + alpha_c p (each case's pending last step).
__global__ void k_refine_pending(int64_t n_items, int rpad, int ncase, double* __restrict__ x,
                                 const float* __restrict__ d, const float* __restrict__ p, CgCase* outer,
                                 const CgCase* inner) {
  if (blockIdx.x == 0 && threadIdx.x < ncase) {
    outer[threadIdx.x].iters += inner[threadIdx.x].iters;
    if (inner[threadIdx.x].status == FEM_ERR_BREAKDOWN || inner[threadIdx.x].status == FEM_ERR_NONFINITE)
      outer[threadIdx.x].status = inner[threadIdx.x].status;
  }
  // the grid stride is a multiple of rpad: every thread serves one case
  // two consecutive values (cases c, c + 1) a thread by vector accesses; the grid stride is a multiple of
  // rpad / 2 pairs, so a thread's pair of cases is fixed
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int c0 = (int)((2 * t0) & (rpad - 1));
  const float a0 = (float)inner[c0].alpha, a1 = (float)inner[rpad > 1 ? c0 + 1 : c0].alpha;
  if (rpad > 1) {
    for (int64_t t = t0; t < (n_items >> 1); t += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = 2 * t;
      const float2 dv = *reinterpret_cast<const float2*>(d + i), pv = *reinterpret_cast<const float2*>(p + i);
      double2 xv = *reinterpret_cast<const double2*>(x + i);
      xv.x += f2d(a0 != 0.0f ? fmaf(a0, pv.x, dv.x) : dv.x);
      xv.y += f2d(a1 != 0.0f ? fmaf(a1, pv.y, dv.y) : dv.y);
      *reinterpret_cast<double2*>(x + i) = xv;
    }
  } else {
    for (int64_t i = t0; i < n_items; i += (int64_t)gridDim.x * blockDim.x)
      x[i] += f2d(a0 != 0.0f ? fmaf(a0, p[i], d[i]) : d[i]);
  }
}

// x = 0 on Dirichlet DOFs and for cases whose right-hand side is zero (||b|| = 0 gives x = 0).
template <typename T>
__global__ void k_zero_b0(MeshView m, int rpad, int rshift, T* __restrict__ x, const CgCase* __restrict__ sc) {
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
    const bool z = sc[c].bb == 0.0;
    for (int k = 0; k < 3; ++k)
      if (z || !dof_free(f, k)) x[(n * 3 + k) * rpad + c] = (T)0;
  }
}

// ---- launchers ----
template <typename T>
cudaError_t launch_zero_b0_t(const MeshView& m, int rpad, T* x, const CgCase* sc, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_zero_b0<T><<<grid_for(m.N << rs), kBlock, 0, s>>>(m, rpad, rs, x, sc);
  return cudaGetLastError();
}
template cudaError_t launch_zero_b0_t<double>(const MeshView&, int, double*, const CgCase*, cudaStream_t);
template cudaError_t launch_zero_b0_t<float>(const MeshView&, int, float*, const CgCase*, cudaStream_t);

template <typename T>
cudaError_t launch_norm_b_gated(const MeshView& m, int rpad, const T* b, Reducer red, CgCase* sc,
                                const CgCase* gate, double tol, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_norm_b<T><<<vec_grid(m.N << rs), kVecBlock, 0, s>>>(m, rpad, rs, b, red, sc, gate, tol);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resid(const MeshView& m, int rpad, const T* b, const T* q, T* x, T* r, T* z, int first,
                         Reducer red, CgCase* sc, int* n_active, double tol, int maxit, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_resid<T><<<vec_grid(m.N << rs), kVecBlock, 0, s>>>(m, rpad, rs, b, q, x, r, z, first, red, sc, n_active, tol, maxit);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dir_gated(const MeshView& m, int rpad, const T* z, T* p, const CgCase* sc, const int* n_active,
                             cudaStream_t s) {
  const int rs = log2i(rpad);
  k_dir<T><<<grid_for((m.N * 3) << rs), kBlock, 0, s>>>(m, rpad, rs, z, p, sc, n_active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(const MeshView& m, int rpad, const T* p, const T* q, T* x, T* r, T* z, Reducer red,
                          CgCase* sc, int* n_active, double tol, int maxit, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_update<T><<<vec_grid(m.N << rs), kVecBlock, 0, s>>>(m, rpad, rs, p, q, x, r, z, red, sc, n_active, tol, maxit);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dir_defer(const MeshView& m, int rpad, const T* r, T* p, T* x, const CgCase* sc,
                             const int* n_active, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_dir_defer<T><<<vec_grid(m.N << rs), kVecBlock, 0, s>>>(m, rpad, rs, r, p, x, sc, n_active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_defer(const MeshView& m, int rpad, const T* q, T* r, Reducer red, CgCase* sc,
                                int* n_active, int maxit, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_update_defer<T><<<grid_resident((const void*)k_update_defer<T>, kVecBlock, m.N << rs), kVecBlock, 0, s>>>(m, rpad, rs, q, r, red, sc, n_active, maxit);
  return cudaGetLastError();
}
template cudaError_t launch_dir_defer<float>(const MeshView&, int, const float*, float*, float*, const CgCase*,
                                             const int*, cudaStream_t);
template cudaError_t launch_update_defer<float>(const MeshView&, int, const float*, float*, Reducer, CgCase*, int*,
                                                int, cudaStream_t);

cudaError_t launch_refine_pending(const MeshView& m, int rpad, int ncase, double* x, const float* d32,
                                  const float* p32, CgCase* outer, const CgCase* inner, cudaStream_t s) {
  const int64_t n = m.N * 3 * rpad;
  k_refine_pending<<<grid_for(n), kBlock, 0, s>>>(n, rpad, ncase, x, d32, p32, outer, inner);
  return cudaGetLastError();
}

cudaError_t launch_outer_resid(const MeshView& m, int rpad, const double* b, const double* q, float* r32,
                               Reducer red, CgCase* outer, int* n_active, double tol, double inner_max, double aim,
                               cudaStream_t s) {
  const int rs = log2i(rpad);
  k_outer_resid<<<vec_grid(m.N << rs), kVecBlock, 0, s>>>(m, rpad, rs, b, q, r32, red, outer, n_active, tol, inner_max,
                                                          aim);
  return cudaGetLastError();
}

cudaError_t launch_refine_counts(const MeshView& m, int rpad, int ncase, double* x, const float* d32, CgCase* outer,
                                 const CgCase* inner, cudaStream_t s) {
  const int64_t n = m.N * 3 * rpad;
  k_refine<<<grid_for(n), kBlock, 0, s>>>(n, ncase, x, d32, outer, inner);
  return cudaGetLastError();
}

#define INST(T)                                                                                                   \
  template cudaError_t launch_norm_b_gated<T>(const MeshView&, int, const T*, Reducer, CgCase*, const CgCase*,    \
                                              double, cudaStream_t);                                              \
  template cudaError_t launch_resid<T>(const MeshView&, int, const T*, const T*, T*, T*, T*, int, Reducer,        \
                                       CgCase*, int*, double, int, cudaStream_t);                                 \
  template cudaError_t launch_dir_gated<T>(const MeshView&, int, const T*, T*, const CgCase*, const int*,         \
                                           cudaStream_t);                                                         \
  template cudaError_t launch_update<T>(const MeshView&, int, const T*, const T*, T*, T*, T*, Reducer, CgCase*,   \
                                        int*, double, int, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace fem
