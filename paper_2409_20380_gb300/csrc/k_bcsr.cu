// Assembled operators for the FP64 certification product: the stiffness K as a 3x3-block CSR matrix and
// the consistent mass M as a scalar CSR matrix on the same node pattern, assembled on the GPU from the
// FP64 element records (the factorised form K_ab = V [lambda g_a g_b^T + mu (g_a . g_b) I + mu g_b g_a^T],
// M_ab = rho V / 20 (1 + delta_ab) I of the element apply).  Applied to r cases at once, one block row
// serves all r right-hand sides, so a product issues ~4x fewer FP64 operations than recomputing the element
// operators; the double-float variant (values and inputs as FP32 pairs, error-free transforms) runs the
// arithmetic on the FP32 pipe instead of GB300's narrow FP64 pipe.
#include "fem_internal.cuh"

namespace fem {

namespace {

__device__ __forceinline__ int find_col(const int32_t* __restrict__ col, int lo, int hi, int c) {
  for (int j = lo; j < hi; ++j)
    if (col[j] == c) return j;
  return -1;
}

// One thread per element: its 16 node-pair blocks added to the assembled matrices.
__global__ void k_bcsr_assemble(MeshView m, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                double* __restrict__ Kb, double* __restrict__ Mb, int* __restrict__ missing) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.E; e += (int64_t)gridDim.x * blockDim.x) {
    const int4 cn = m.conn[e];
    const int nd[4] = {cn.x, cn.y, cn.z, cn.w};
    const double* r = m.rec64 + e * kRec;
    double g[4][3];
    for (int k = 0; k < 3; ++k) {
      g[1][k] = r[k];
      g[2][k] = r[3 + k];
      g[3][k] = r[6 + k];
      g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
    }
    const double lam = r[9], mu = r[10], ms = r[11];
    for (int a = 0; a < 4; ++a) {
      const int lo = row_ptr[nd[a]], hi = row_ptr[nd[a] + 1];
      for (int b = 0; b < 4; ++b) {
        const int j = find_col(col, lo, hi, nd[b]);
        if (j < 0) {
          atomicExch(missing, 1);
          continue;
        }
        const double gab = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 3; ++k) {
            const double v = lam * g[a][i] * g[b][k] + mu * g[b][i] * g[a][k] + (i == k ? mu * gab : 0.0);
            atomicAdd(Kb + (int64_t)j * 9 + i * 3 + k, v);
          }
        atomicAdd(Mb + j, a == b ? 2.0 * ms : ms);
      }
    }
  }
}

// FP64 values -> (hi, lo) FP32 pairs with hi + lo = v to 2^-47 relative (integer-pipe split).
__global__ void k_to_df(int64_t n, const double* __restrict__ v, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = d2df(v[i]);
  }
}

// The 80-byte double-float block records: KMd[10 j + 0..8] = pairs of Kb[9 j + 0..8], KMd[10 j + 9] = Mb[j].
__global__ void k_to_kmd(int64_t nnz, const double* __restrict__ Kb, const double* __restrict__ Mb,
                         float2* __restrict__ KMd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 10 * nnz; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / 10;
    const int r = (int)(i - 10 * j);
    KMd[i] = d2df(r < 9 ? Kb[9 * j + r] : Mb[j]);
  }
}

// acc (sh + sl) += (ah + al)(bh + bl): the product's rounding error by FMA, the sum's by two-sum; the low
// word is renormalised only at the end (its own FP32 rounding is ~2^-24 of a quantity ~2^-24 smaller).
__device__ __forceinline__ void df_fma_acc(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// qM = M p, qK = K p for r cases, one thread per (node row, case); rows of Dirichlet DOFs are zero.  I is
// the index type of the vector offsets (32-bit when N * 3 * rpad fits).  A block record is 5 aligned
// 16-byte loads.
template <typename I>
__global__ void __launch_bounds__(256) k_bcsr_split_df(int64_t N, int rpad, int rshift, const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col, const float4* __restrict__ KM,
                                                       const uint8_t* __restrict__ fm, const float2* __restrict__ p,
                                                       double* __restrict__ qM, double* __restrict__ qK) {
  const int64_t total = N << rshift;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const I n = (I)(t >> rshift);
    const int c = (int)(t & (rpad - 1));
    float kh[3] = {0.f, 0.f, 0.f}, kl[3] = {0.f, 0.f, 0.f}, mh[3] = {0.f, 0.f, 0.f}, ml[3] = {0.f, 0.f, 0.f};
    const int lo = __ldg(row_ptr + n), hi = __ldg(row_ptr + n + 1);
    const float2* pc = p + c;
    const I r3 = (I)(3 * rpad);
    for (int j = lo; j < hi; ++j) {
      const I cn = (I)__ldg(col + j);
      float2 pv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) pv[k] = __ldg(pc + cn * r3 + (I)(k * rpad));
      const float4* rec = KM + (int64_t)j * 5;
      const float4 q0 = __ldg(rec), q1 = __ldg(rec + 1), q2 = __ldg(rec + 2), q3 = __ldg(rec + 3), q4 = __ldg(rec + 4);
      const float2 a[10] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                            make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w),
                            make_float2(q3.x, q3.y), make_float2(q3.z, q3.w), make_float2(q4.x, q4.y),
                            make_float2(q4.z, q4.w)};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        df_fma_acc(mh[i], ml[i], a[9].x, a[9].y, pv[i].x, pv[i].y);
#pragma unroll
        for (int k = 0; k < 3; ++k) df_fma_acc(kh[i], kl[i], a[i * 3 + k].x, a[i * 3 + k].y, pv[k].x, pv[k].y);
      }
    }
    const uint8_t f = fm[n];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t id = ((int64_t)n * 3 + i) * rpad + c;
      const bool fr = dof_free(f, i);
      qM[id] = fr ? f2d(mh[i]) + f2d(ml[i]) : 0.0;
      qK[id] = fr ? f2d(kh[i]) + f2d(kl[i]) : 0.0;
    }
  }
}

// Two cases a thread (rpad >= 2): the same arithmetic as k_bcsr_split_df in paired FP32 instructions (one
// instruction applies an operation to both cases), so each block record's loads and the loop's address work
// also serve two cases.  The input comes pair-packed: p2[(node * 3 + k) * rpad / 2 + pair] = (hi of case
// 2 pair, hi of case 2 pair + 1, lo of case 2 pair, lo of case 2 pair + 1).
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ void df2_fma_acc(float2& sh, float2& sl, float2 ah, float2 al, float2 bh, float2 bl) {
  const float2 p = __fmul2_rn(ah, bh);
  float2 e = __ffma2_rn(ah, bh, __fmul2_rn(p, make_float2(-1.f, -1.f)));
  e = __ffma2_rn(ah, bl, e);
  e = __ffma2_rn(al, bh, e);
  const float2 s = __fadd2_rn(sh, p);
  const float2 bb = sub2(s, sh);
  const float2 err = __fadd2_rn(sub2(sh, sub2(s, bb)), sub2(p, bb));
  sh = s;
  sl = __fadd2_rn(sl, __fadd2_rn(err, e));
}

template <typename I>
__global__ void __launch_bounds__(256) k_bcsr_split_df2(int64_t N, int rpad, int hshift, const int32_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col, const float4* __restrict__ KM,
                                                        const uint8_t* __restrict__ fm, const float4* __restrict__ p2,
                                                        double* __restrict__ qM, double* __restrict__ qK) {
  const int hpad = rpad >> 1;
  const int64_t total = N << hshift;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const I n = (I)(t >> hshift);
    const int cp = (int)(t & (hpad - 1));
    const float2 z = make_float2(0.f, 0.f);
    float2 kh[3] = {z, z, z}, kl[3] = {z, z, z}, mh[3] = {z, z, z}, ml[3] = {z, z, z};
    const int lo = __ldg(row_ptr + n), hi = __ldg(row_ptr + n + 1);
    const float4* pc = p2 + cp;
    const I r3 = (I)(3 * hpad);
    for (int j = lo; j < hi; ++j) {
      const I cn = (I)__ldg(col + j);
      float2 bh[3], bl[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float4 v = __ldg(pc + cn * r3 + (I)(k * hpad));
        bh[k] = make_float2(v.x, v.y);
        bl[k] = make_float2(v.z, v.w);
      }
      const float4* rec = KM + (int64_t)j * 5;
      const float4 q0 = __ldg(rec), q1 = __ldg(rec + 1), q2 = __ldg(rec + 2), q3 = __ldg(rec + 3), q4 = __ldg(rec + 4);
      const float ah[10] = {q0.x, q0.z, q1.x, q1.z, q2.x, q2.z, q3.x, q3.z, q4.x, q4.z};
      const float al[10] = {q0.y, q0.w, q1.y, q1.w, q2.y, q2.w, q3.y, q3.w, q4.y, q4.w};
      const float2 mvh = bc2(ah[9]), mvl = bc2(al[9]);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        df2_fma_acc(mh[i], ml[i], mvh, mvl, bh[i], bl[i]);
#pragma unroll
        for (int k = 0; k < 3; ++k) df2_fma_acc(kh[i], kl[i], bc2(ah[i * 3 + k]), bc2(al[i * 3 + k]), bh[k], bl[k]);
      }
    }
    const uint8_t f = fm[n];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t id = ((int64_t)n * 3 + i) * rpad + 2 * cp;
      const bool fr = dof_free(f, i);
      *reinterpret_cast<double2*>(qM + id) = fr ? make_double2(f2d(mh[i].x) + f2d(ml[i].x), f2d(mh[i].y) + f2d(ml[i].y))
                                               : make_double2(0.0, 0.0);
      *reinterpret_cast<double2*>(qK + id) = fr ? make_double2(f2d(kh[i].x) + f2d(kl[i].x), f2d(kh[i].y) + f2d(kl[i].y))
                                               : make_double2(0.0, 0.0);
    }
  }
}

// FP64 values of case pairs -> pair-packed double-float inputs of k_bcsr_split_df2.
__global__ void k_to_df2(int64_t n_pairs, const double2* __restrict__ v, float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pairs; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = v[i];
    const float2 a = d2df(x.x), b = d2df(x.y);
    out[i] = make_float4(a.x, b.x, a.y, b.y);
  }
}

// The same product in native FP64.
__global__ void __launch_bounds__(256) k_bcsr_split_f64(int64_t N, int rpad, int rshift,
                                                        const int32_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col, const double* __restrict__ Kb,
                                                        const double* __restrict__ Mb, const uint8_t* __restrict__ fm,
                                                        const double* __restrict__ p, double* __restrict__ qM,
                                                        double* __restrict__ qK) {
  const int64_t total = N << rshift;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t >> rshift;
    const int c = (int)(t & (rpad - 1));
    double ka[3] = {0.0, 0.0, 0.0}, ma[3] = {0.0, 0.0, 0.0};
    const int lo = __ldg(row_ptr + n), hi = __ldg(row_ptr + n + 1);
    for (int j = lo; j < hi; ++j) {
      const int64_t cn = __ldg(col + j);
      double pv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) pv[k] = __ldg(p + (cn * 3 + k) * rpad + c);
      const double mv = __ldg(Mb + j);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        ma[i] = fma(mv, pv[i], ma[i]);
#pragma unroll
        for (int k = 0; k < 3; ++k) ka[i] = fma(__ldg(Kb + (int64_t)j * 9 + i * 3 + k), pv[k], ka[i]);
      }
    }
    const uint8_t f = fm[n];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t id = (n * 3 + i) * rpad + c;
      const bool fr = dof_free(f, i);
      qM[id] = fr ? ma[i] : 0.0;
      qK[id] = fr ? ka[i] : 0.0;
    }
  }
}

int lg2(int r) {
  int s = 0;
  while ((1 << s) < r) ++s;
  return s;
}

// q = (aM M + aK K) p with the assembled operators (variant 8: the CRS-style product the paper compares the
// EBE with, Section 3.3), one thread per (node row, case), K p and M p accumulated apart and combined once.
// FP64 products read the FP64 blocks; FP32 products read the high words of the (hi, lo) block records (the
// FP32 rounding of the FP64 values).  Dirichlet rows of q are zero; DOT fuses p^T q per case.
template <typename T, bool DOT>
__global__ void __launch_bounds__(256) k_bcsr_apply(int64_t N, int rpad, int rshift, const int32_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col, const double* __restrict__ Kb,
                                                    const double* __restrict__ Mb, const float4* __restrict__ KM,
                                                    const uint8_t* __restrict__ fm, const T* __restrict__ p,
                                                    T* __restrict__ q, T aM, T aK, Reducer red, CgCase* sc,
                                                    double* ptq_out, const int* gate) {
  if (gate && *gate == 0) return;
  double dot = 0.0;
  const int64_t total = N << rshift;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t >> rshift;
    const int c = (int)(t & (rpad - 1));
    T kp[3] = {0, 0, 0}, mp[3] = {0, 0, 0};
    const int lo = __ldg(row_ptr + n), hi = __ldg(row_ptr + n + 1);
    for (int j = lo; j < hi; ++j) {
      const int64_t cn = __ldg(col + j);
      T pv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) pv[k] = __ldg(p + (cn * 3 + k) * rpad + c);
      T K[9], Mv;
      if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int u = 0; u < 9; ++u) K[u] = __ldg(Kb + j * 9 + u);
        Mv = __ldg(Mb + j);
      } else {
        const float4* rec = KM + j * 5;
        const float4 q0 = __ldg(rec), q1 = __ldg(rec + 1), q2 = __ldg(rec + 2), q3 = __ldg(rec + 3), q4 = __ldg(rec + 4);
        K[0] = q0.x, K[1] = q0.z, K[2] = q1.x, K[3] = q1.z, K[4] = q2.x, K[5] = q2.z, K[6] = q3.x, K[7] = q3.z;
        K[8] = q4.x, Mv = q4.z;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        mp[i] += Mv * pv[i];
        kp[i] += K[3 * i] * pv[0] + K[3 * i + 1] * pv[1] + K[3 * i + 2] * pv[2];
      }
    }
    const uint8_t f = fm[n];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int64_t id = (n * 3 + i) * rpad + c;
      const T v = dof_free(f, i) ? aM * mp[i] + aK * kp[i] : (T)0;
      q[id] = v;
      if (DOT) dot += (double)(p[id] * v);
    }
  }
  if (DOT) {
    double v[1] = {dot};
    if (block_reduce_last<1>(v, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);
  }
}

int grid_of(int64_t items) {
  int64_t g = (items + 255) / 256;
  if (g > wide_grid_cap()) g = wide_grid_cap();
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_bcsr_assemble(const MeshView& m, const int32_t* row_ptr, const int32_t* col, int64_t nnz,
                                 double* Kb, double* Mb, float2* KMd, int* missing, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(Kb, 0, sizeof(double) * 9 * (size_t)nnz, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Mb, 0, sizeof(double) * (size_t)nnz, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(missing, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_bcsr_assemble<<<grid_of(m.E), 256, 0, s>>>(m, row_ptr, col, Kb, Mb, missing);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_to_kmd<<<grid_of(10 * nnz), 256, 0, s>>>(nnz, Kb, Mb, KMd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bcsr_apply(const MeshView& m, int rpad, const int32_t* row_ptr, const int32_t* col,
                              const double* Kb, const double* Mb, const float2* KMd, const T* p, T* q, double aM,
                              double aK, const Reducer* red, CgCase* sc, double* ptq_out, const int* gate,
                              cudaStream_t s) {
  if (!row_ptr || m.seg) return cudaErrorInvalidValue;
  const int rs = lg2(rpad);
  int grid = grid_of(m.N << rs);
  if (grid > red_grid_cap()) grid = red_grid_cap();
  const float4* km = reinterpret_cast<const float4*>(KMd);
  Reducer rd = red ? *red : Reducer{nullptr, nullptr, nullptr};
  if (red)
    k_bcsr_apply<T, true><<<grid, 256, 0, s>>>(m.N, rpad, rs, row_ptr, col, Kb, Mb, km, m.freemask, p, q, (T)aM,
                                               (T)aK, rd, sc, ptq_out, gate);
  else
    k_bcsr_apply<T, false><<<grid, 256, 0, s>>>(m.N, rpad, rs, row_ptr, col, Kb, Mb, km, m.freemask, p, q, (T)aM,
                                                (T)aK, rd, nullptr, nullptr, gate);
  return cudaGetLastError();
}
template cudaError_t launch_bcsr_apply<double>(const MeshView&, int, const int32_t*, const int32_t*, const double*,
                                               const double*, const float2*, const double*, double*, double, double,
                                               const Reducer*, CgCase*, double*, const int*, cudaStream_t);
template cudaError_t launch_bcsr_apply<float>(const MeshView&, int, const int32_t*, const int32_t*, const double*,
                                              const double*, const float2*, const float*, float*, double, double,
                                              const Reducer*, CgCase*, double*, const int*, cudaStream_t);

cudaError_t launch_to_kmd(int64_t nnz, const double* Kb, const double* Mb, float2* KMd, cudaStream_t s) {
  k_to_kmd<<<grid_of(10 * nnz), 256, 0, s>>>(nnz, Kb, Mb, KMd);
  return cudaGetLastError();
}

cudaError_t launch_to_df(int64_t n, const double* v, float2* out, cudaStream_t s) {
  k_to_df<<<grid_of(n), 256, 0, s>>>(n, v, out);
  return cudaGetLastError();
}

cudaError_t launch_bcsr_split(const MeshView& m, int rpad, const int32_t* row_ptr, const int32_t* col,
                              const double* Kb, const double* Mb, const float2* KMd, const double* p, float2* p_df,
                              double* qM, double* qK, cudaStream_t s) {
  const int rs = lg2(rpad);
  const int64_t items = m.N << rs;
  const bool al16 = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(qM) |
                      reinterpret_cast<uintptr_t>(qK) | reinterpret_cast<uintptr_t>(p_df)) & 15u) == 0;
  if (p_df && rpad >= 2 && al16) {   // double-float, two cases a thread (16-byte accesses of case pairs)
    const int64_t n_pairs = m.N * 3 * (rpad / 2);
    k_to_df2<<<grid_of(n_pairs), 256, 0, s>>>(n_pairs, reinterpret_cast<const double2*>(p),
                                              reinterpret_cast<float4*>(p_df));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float4* km = reinterpret_cast<const float4*>(KMd);
    const float4* p2 = reinterpret_cast<const float4*>(p_df);
    const int64_t items2 = m.N << (rs - 1);
    if (n_pairs < ((int64_t)1 << 31))
      k_bcsr_split_df2<int32_t><<<grid_of(items2), 256, 0, s>>>(m.N, rpad, rs - 1, row_ptr, col, km, m.freemask, p2, qM, qK);
    else
      k_bcsr_split_df2<int64_t><<<grid_of(items2), 256, 0, s>>>(m.N, rpad, rs - 1, row_ptr, col, km, m.freemask, p2, qM, qK);
  } else if (p_df) {   // double-float: inputs split once per value, then the product on the FP32 pipe
    cudaError_t e = launch_to_df(m.N * 3 * rpad, p, p_df, s);
    if (e != cudaSuccess) return e;
    const float4* km = reinterpret_cast<const float4*>(KMd);
    if (m.N * 3 * rpad < ((int64_t)1 << 31))
      k_bcsr_split_df<int32_t><<<grid_of(items), 256, 0, s>>>(m.N, rpad, rs, row_ptr, col, km, m.freemask, p_df, qM, qK);
    else
      k_bcsr_split_df<int64_t><<<grid_of(items), 256, 0, s>>>(m.N, rpad, rs, row_ptr, col, km, m.freemask, p_df, qM, qK);
  } else {
    k_bcsr_split_f64<<<grid_of(items), 256, 0, s>>>(m.N, rpad, rs, row_ptr, col, Kb, Mb, m.freemask, p, qM, qK);
  }
  return cudaGetLastError();
}

}  // namespace fem
