// Matrix-free element-by-element product (Section 3.2, Eq. eqebefem / eqmebefem):
//   q = sum_e P_e^T ((aM M_e + aK K_e) (P_e p))   for r cases interleaved as [node][3][r].
// One thread per (element, case): the r threads of an element read the same element record (broadcast)
// and consecutive case values of each node (coalesced), which is the block random access of the
// multi-RHS form.  Element apply in factorised form:
//   G = sum_b p_b g_b^T,  sigma = lambda tr(G) I + mu (G + G^T),  (K_e p)_a = V sigma g_a,
//   (M_e p)_a = rho V / 20 (p_a + sum_b p_b).
// This generic kernel scatters with global atomics; fixed DOFs are left to the consumer to mask.
#include <cuda_fp16.h>

#include "fem_internal.cuh"

#include <mutex>
#include <unordered_map>

namespace fem {

template <typename T> __device__ __forceinline__ const T* rec_of(const MeshView& m);
template <> __device__ __forceinline__ const double* rec_of<double>(const MeshView& m) { return m.rec64; }
template <> __device__ __forceinline__ const float* rec_of<float>(const MeshView& m) { return m.rec32; }

// Same for fused groups: cases 0..nc-1, totals in red.out[c].
__device__ __forceinline__ void ebe_tail_seg(const Reducer& red, CgCase* sc, double* ptq_out, int nc) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const double pq = red.out[c];
    if (ptq_out) ptq_out[c] = pq;
    if (sc) {
      CgCase& s = sc[c];
      s.pq = pq;
      if (s.active) {
        if (!(pq > 0.0) || !isfinite(pq)) {
          s.active = 0;
          s.status = FEM_ERR_BREAKDOWN;
          s.alpha = 0.0;
        } else {
          s.alpha = s.rho / pq;
        }
      } else {
        s.alpha = 0.0;
      }
    }
  }
}

static int log2i(int r) {
  int s = 0;
  while ((1 << s) < r) ++s;
  return s;
}

template <typename T, bool TWO, bool DOT>
__global__ void __launch_bounds__(kBlock) k_ebe_atomic(MeshView m, int rpad, int rshift, const T* __restrict__ pm,
                                                       const T* __restrict__ pk, T* __restrict__ q, T aM, T aK,
                                                       Reducer red, CgCase* sc, double* ptq_out,
                                                       const int* gate_active) {
  if (gate_active && *gate_active == 0) return;
  const T* __restrict__ rec = rec_of<T>(m);
  T dot = 0;
  const int64_t total = m.E << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const int4 cn = __ldg(m.conn + e);
    const int64_t nd[4] = {cn.x, cn.y, cn.z, cn.w};
    const T* re = rec + e * kRec;
    T g[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) g[j] = re[j];
    const T lam = aK * re[9], mu = aK * re[10], ms = aM * re[11];
    T P[4][3], PK[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        P[a][k] = pm[(nd[a] * 3 + k) * rpad + c];
        PK[a][k] = TWO ? pk[(nd[a] * 3 + k) * rpad + c] : P[a][k];
      }
    // displacement gradient G_ij = sum_{b=1..3} (p_b - p_0)_i g_b,j
    T G[3][3];
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) {
      const T d1 = PK[1][i2] - PK[0][i2], d2 = PK[2][i2] - PK[0][i2], d3 = PK[3][i2] - PK[0][i2];
#pragma unroll
      for (int j = 0; j < 3; ++j) G[i2][j] = d1 * g[j] + d2 * g[3 + j] + d3 * g[6 + j];
    }
    const T tr = G[0][0] + G[1][1] + G[2][2];
    T S[3][3];
    const T mu2 = mu + mu;
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) S[i2][i2] = lam * tr + mu2 * G[i2][i2];
    S[0][1] = S[1][0] = mu * (G[0][1] + G[1][0]);
    S[0][2] = S[2][0] = mu * (G[0][2] + G[2][0]);
    S[1][2] = S[2][1] = mu * (G[1][2] + G[2][1]);
    T Q[4][3];
#pragma unroll
    for (int b = 1; b < 4; ++b)
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
        Q[b][i2] = S[i2][0] * g[(b - 1) * 3 + 0] + S[i2][1] * g[(b - 1) * 3 + 1] + S[i2][2] * g[(b - 1) * 3 + 2];
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) Q[0][i2] = -(Q[1][i2] + Q[2][i2] + Q[3][i2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T sum = P[0][k] + P[1][k] + P[2][k] + P[3][k];
#pragma unroll
      for (int a = 0; a < 4; ++a) Q[a][k] += ms * (P[a][k] + sum);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (DOT) dot += P[a][k] * Q[a][k];
        atomicAdd(q + (nd[a] * 3 + k) * rpad + c, Q[a][k]);
      }
  }
  if (DOT) {
    double v[1] = {(double)dot};
    if (block_reduce_last<1>(v, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);
  }
}

template <typename T>
cudaError_t launch_ebe_gated(const MeshView& m, int rpad, const T* pm, const T* pk, T* q, double aM, double aK,
                             const Reducer* red, CgCase* sc, double* ptq_out, const int* gate, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(q, 0, sizeof(T) * (size_t)m.N * 3 * rpad, s);
  if (err != cudaSuccess) return err;
  const int rs = log2i(rpad);
  const int grid = grid_for(m.E << rs, red ? vec_grid_cap() : red_grid_cap());
  Reducer rd = red ? *red : Reducer{nullptr, nullptr, nullptr};
  if (pk) {
    k_ebe_atomic<T, true, false><<<grid, kBlock, 0, s>>>(m, rpad, rs, pm, pk, q, (T)aM, (T)aK, rd, nullptr, nullptr, gate);
  } else if (red) {
    k_ebe_atomic<T, false, true><<<grid, kBlock, 0, s>>>(m, rpad, rs, pm, pm, q, (T)aM, (T)aK, rd, sc, ptq_out, gate);
  } else {
    k_ebe_atomic<T, false, false><<<grid, kBlock, 0, s>>>(m, rpad, rs, pm, pm, q, (T)aM, (T)aK, rd, nullptr, nullptr, gate);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ebe(const MeshView& m, int rpad, const T* pm, const T* pk, T* q, double aM, double aK,
                       const Reducer* red, CgCase* sc, double* ptq_out, cudaStream_t s) {
  return launch_ebe_gated<T>(m, rpad, pm, pk, q, aM, aK, red, sc, ptq_out, nullptr, s);
}

template cudaError_t launch_ebe<double>(const MeshView&, int, const double*, const double*, double*, double, double,
                                        const Reducer*, CgCase*, double*, cudaStream_t);
template cudaError_t launch_ebe<float>(const MeshView&, int, const float*, const float*, float*, double, double,
                                       const Reducer*, CgCase*, double*, cudaStream_t);
template cudaError_t launch_ebe_gated<double>(const MeshView&, int, const double*, const double*, double*, double,
                                              double, const Reducer*, CgCase*, double*, const int*, cudaStream_t);
template cudaError_t launch_ebe_gated<float>(const MeshView&, int, const float*, const float*, float*, double, double,
                                             const Reducer*, CgCase*, double*, const int*, cudaStream_t);

// Zeroes Dirichlet DOFs of a [N][3][rpad] vector.
template <typename T>
__global__ void k_mask(int64_t N, int rpad, int rshift, const uint8_t* __restrict__ fm, T* __restrict__ v) {
  const int64_t total = N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = fm[n];
    if (f == 7) continue;
    for (int k = 0; k < 3; ++k)
      if (!dof_free(f, k)) v[(n * 3 + k) * rpad + c] = (T)0;
  }
}

template <typename T>
cudaError_t launch_mask(int64_t N, int rpad, const uint8_t* fm, T* v, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_mask<T><<<grid_for(N << rs), kBlock, 0, s>>>(N, rpad, rs, fm, v);
  return cudaGetLastError();
}
template cudaError_t launch_mask<double>(int64_t, int, const uint8_t*, double*, cudaStream_t);
template cudaError_t launch_mask<float>(int64_t, int, const uint8_t*, float*, cudaStream_t);


// ------------------------------------------------------------------------------------------------------
// Tiled hex-patch EBE.  One thread per (hex, case): the hex's eight corner values of its case are gathered
// once, its six tets are applied with register accumulation into the eight corners (the tet corner slots
// are compile-time constants, kHexTet), and the 24 corner sums are added into a shared-memory accumulator
// of the tile's nodes.  The flush stores nodes only this tile touches and adds (global red) the others;
// q must be zero beforehand for those.  Dirichlet DOFs of q are written as zero.
// ------------------------------------------------------------------------------------------------------
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  __device__ __forceinline__ static void load12(const float* __restrict__ src, float (&r)[12]) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const float4 a = __ldg(s4), b = __ldg(s4 + 1), c = __ldg(s4 + 2);
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
  }
};
template <> struct Vec4<double> {
  __device__ __forceinline__ static void load12(const double* __restrict__ src, double (&r)[12]) {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double2 v = __ldg(s2 + i);
      r[2 * i] = v.x;
      r[2 * i + 1] = v.y;
    }
  }
};

template <typename T, int A0, int A1, int A2, int A3>
__device__ __forceinline__ void tet_acc(const T* __restrict__ re, T aM, T aK, const T (&P)[8][3], T (&Q)[8][3]) {
  T r[12];
  Vec4<T>::load12(re, r);
  const T lam = aK * r[9], mu = aK * r[10], ms = aM * r[11];
  T G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T d1 = P[A1][i] - P[A0][i], d2 = P[A2][i] - P[A0][i], d3 = P[A3][i] - P[A0][i];
#pragma unroll
    for (int j = 0; j < 3; ++j) G[i][j] = d1 * r[j] + d2 * r[3 + j] + d3 * r[6 + j];
  }
  const T tr = G[0][0] + G[1][1] + G[2][2];
  const T mu2 = mu + mu;
  T S[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) S[i][i] = lam * tr + mu2 * G[i][i];
  S[0][1] = S[1][0] = mu * (G[0][1] + G[1][0]);
  S[0][2] = S[2][0] = mu * (G[0][2] + G[2][0]);
  S[1][2] = S[2][1] = mu * (G[1][2] + G[2][1]);
  T F[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int i = 0; i < 3; ++i) F[b][i] = S[i][0] * r[3 * b] + S[i][1] * r[3 * b + 1] + S[i][2] * r[3 * b + 2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T sum = P[A0][k] + P[A1][k] + P[A2][k] + P[A3][k];
    Q[A0][k] += ms * (P[A0][k] + sum) - (F[0][k] + F[1][k] + F[2][k]);
    Q[A1][k] += ms * (P[A1][k] + sum) + F[0][k];
    Q[A2][k] += ms * (P[A2][k] + sum) + F[1][k];
    Q[A3][k] += ms * (P[A3][k] + sum) + F[2][k];
  }
}

template <typename T, bool DOT, bool SEG>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 2 : 1) k_ebe_hex(HexTiles ht, MeshView m, int rpad, int rshift,
                                                    const T* __restrict__ p, T* __restrict__ q, T aM, T aK,
                                                    Reducer red, CgCase* sc, double* ptq_out, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* qs = reinterpret_cast<T*>(smem_raw);
  int* snode = reinterpret_cast<int*>(smem_raw + sizeof(T) * (size_t)ht.nloc_max * 3 * rpad);
  // fused groups: per-case p^T q accumulators after the node list (8-byte aligned)
  double* sacc = reinterpret_cast<double*>(smem_raw + ((sizeof(T) * (size_t)ht.nloc_max * 3 * rpad +
                                                        sizeof(int) * (size_t)ht.nloc_max + 7) & ~(size_t)7));
  constexpr bool seg = DOT && SEG;
  if (seg) {
    for (int t = threadIdx.x; t < m.nseg; t += blockDim.x) sacc[t] = 0.0;
    __syncthreads();
  }
  const T* __restrict__ rec = rec_of<T>(m);
  double dot = 0.0;
  const int per_node = 3 * rpad;
  for (int tile = blockIdx.x; tile < ht.n_tiles; tile += gridDim.x) {
    const int n0 = ht.tile_node_off[tile], nl = ht.tile_node_off[tile + 1] - n0;
    const int h0 = ht.tile_hex_off[tile], nh = ht.tile_hex_off[tile + 1] - h0;
    for (int i = threadIdx.x; i < nl * per_node; i += blockDim.x) qs[i] = (T)0;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) snode[i] = ht.tile_nodes[n0 + i];
    __syncthreads();
    T tdot = 0;
    const int items = nh << rshift;
    const int rounds_end = seg ? ((items + blockDim.x - 1) / blockDim.x) * blockDim.x : items;
    for (int it = threadIdx.x; it < rounds_end; it += blockDim.x) {
      if (it >= items) {   // idle lane of the last round (fused groups aggregate per warp)
        double z1[1] = {0.0};
        seg_add<1>(sacc, m.nseg, 0, z1);
        continue;
      }
      const int hl = it >> rshift, c = it & (rpad - 1);
      const int64_t hx = h0 + hl;
      const uint4 lw = __ldg(ht.hex_local + hx);
      int ls[8] = {(int)(lw.x & 0xffff), (int)(lw.x >> 16), (int)(lw.y & 0xffff), (int)(lw.y >> 16),
                   (int)(lw.z & 0xffff), (int)(lw.z >> 16), (int)(lw.w & 0xffff), (int)(lw.w >> 16)};
      T P[8][3], Q[8][3];
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) {
        const int64_t g = snode[ls[sl]] & 0x0fffffff;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          P[sl][k] = p[(g * 3 + k) * rpad + c];
          Q[sl][k] = (T)0;
        }
      }
      const T* re = rec + hx * 6 * kRec;
      tet_acc<T, kHexTet[0][0], kHexTet[0][1], kHexTet[0][2], kHexTet[0][3]>(re + 0 * kRec, aM, aK, P, Q);
      tet_acc<T, kHexTet[1][0], kHexTet[1][1], kHexTet[1][2], kHexTet[1][3]>(re + 1 * kRec, aM, aK, P, Q);
      tet_acc<T, kHexTet[2][0], kHexTet[2][1], kHexTet[2][2], kHexTet[2][3]>(re + 2 * kRec, aM, aK, P, Q);
      tet_acc<T, kHexTet[3][0], kHexTet[3][1], kHexTet[3][2], kHexTet[3][3]>(re + 3 * kRec, aM, aK, P, Q);
      tet_acc<T, kHexTet[4][0], kHexTet[4][1], kHexTet[4][2], kHexTet[4][3]>(re + 4 * kRec, aM, aK, P, Q);
      tet_acc<T, kHexTet[5][0], kHexTet[5][1], kHexTet[5][2], kHexTet[5][3]>(re + 5 * kRec, aM, aK, P, Q);
      T hdot = 0;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (DOT) hdot += P[sl][k] * Q[sl][k];
          atomicAdd(qs + ls[sl] * per_node + k * rpad + c, Q[sl][k]);
        }
      if (seg) {
        double v1[1] = {(double)hdot};
        seg_add<1>(sacc, m.nseg, m.seg[snode[ls[0]] & 0x0fffffff], v1);
      } else {
        tdot += hdot;
      }
    }
    dot += (double)tdot;
    __syncthreads();
    for (int i = threadIdx.x; i < nl * per_node; i += blockDim.x) {
      const int l = i / per_node, rem = i - l * per_node;
      const int k = rem >> rshift;
      const int raw = snode[l];
      const int64_t g = raw & 0x0fffffff;
      const bool fixed = !dof_free((uint8_t)((raw >> 28) & 7), k);
      T* dst = q + g * per_node + rem;
      if (raw < 0) {
        if (!fixed) atomicAdd(dst, qs[i]);
      } else {
        *dst = fixed ? (T)0 : qs[i];
      }
    }
    __syncthreads();
  }
  if (DOT) {
    if (seg) {
      if (block_reduce_last_seg<1>(sacc, m.nseg, red)) ebe_tail_seg(red, sc, ptq_out, m.nseg);
    } else {
      double v[1] = {dot};
      if (block_reduce_last<1>(v, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);
    }
  }
}

template <typename T>
cudaError_t launch_ebe_hex(const HexTiles& ht, const MeshView& m, int rpad, const T* p, T* q, double aM, double aK,
                           const Reducer* red, CgCase* sc, double* ptq_out, const int* gate, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(q, 0, sizeof(T) * (size_t)m.N * 3 * rpad, s);
  if (err != cudaSuccess) return err;
  const int rs = log2i(rpad);
  const size_t smem = ((sizeof(T) * (size_t)ht.nloc_max * 3 * rpad + sizeof(int) * (size_t)ht.nloc_max + 7) & ~(size_t)7) +
                      (m.seg ? sizeof(double) * (size_t)m.nseg : 0);
  const int nsm = sm_count();
  int per_sm = 1;
  auto kfn = red ? (m.seg ? k_ebe_hex<T, true, true> : k_ebe_hex<T, true, false>) : k_ebe_hex<T, false, false>;
  err = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBlock, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int grid = nsm * per_sm;
  if (grid > ht.n_tiles) grid = ht.n_tiles;
  if (grid > red_grid_cap()) grid = red_grid_cap();
  Reducer rd = red ? *red : Reducer{nullptr, nullptr, nullptr};
  kfn<<<grid, kBlock, smem, s>>>(ht, m, rpad, rs, p, q, (T)aM, (T)aK, rd, red ? sc : nullptr, red ? ptq_out : nullptr,
                                 gate);
  return cudaGetLastError();
}
template cudaError_t launch_ebe_hex<double>(const HexTiles&, const MeshView&, int, const double*, double*, double,
                                            double, const Reducer*, CgCase*, double*, const int*, cudaStream_t);
template cudaError_t launch_ebe_hex<float>(const HexTiles&, const MeshView&, int, const float*, float*, double,
                                           double, const Reducer*, CgCase*, double*, const int*, cudaStream_t);

template <typename T> struct SVec4;
template <> struct SVec4<float> {
  __device__ __forceinline__ static void load12(const float* src, float (&r)[12]) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const float4 a = s4[0], b = s4[1], c = s4[2];
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
  }
};
template <> struct SVec4<double> {
  __device__ __forceinline__ static void load12(const double* src, double (&r)[12]) {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double2 v = s2[i];
      r[2 * i] = v.x;
      r[2 * i + 1] = v.y;
    }
  }
};

template <typename T, int A0, int A1, int A2, int A3>
__device__ __forceinline__ void tet_acc_s(const T* re, T aM, T aK, const T (&P)[8][3], T (&Q)[8][3]) {
  T r[12];
  SVec4<T>::load12(re, r);
  const T lam = aK * r[9], mu = aK * r[10], ms = aM * r[11];
  T G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T d1 = P[A1][i] - P[A0][i], d2 = P[A2][i] - P[A0][i], d3 = P[A3][i] - P[A0][i];
#pragma unroll
    for (int j = 0; j < 3; ++j) G[i][j] = d1 * r[j] + d2 * r[3 + j] + d3 * r[6 + j];
  }
  const T tr = G[0][0] + G[1][1] + G[2][2];
  const T mu2 = mu + mu;
  T S[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) S[i][i] = lam * tr + mu2 * G[i][i];
  S[0][1] = S[1][0] = mu * (G[0][1] + G[1][0]);
  S[0][2] = S[2][0] = mu * (G[0][2] + G[2][0]);
  S[1][2] = S[2][1] = mu * (G[1][2] + G[2][1]);
  T F[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int i = 0; i < 3; ++i) F[b][i] = S[i][0] * r[3 * b] + S[i][1] * r[3 * b + 1] + S[i][2] * r[3 * b + 2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T sum = P[A0][k] + P[A1][k] + P[A2][k] + P[A3][k];
    Q[A0][k] += ms * (P[A0][k] + sum) - (F[0][k] + F[1][k] + F[2][k]);
    Q[A1][k] += ms * (P[A1][k] + sum) + F[0][k];
    Q[A2][k] += ms * (P[A2][k] + sum) + F[1][k];
    Q[A3][k] += ms * (P[A3][k] + sum) + F[2][k];
  }
}

// Two cases per thread on Blackwell's paired FP32 pipe operations (one instruction, two lanes of values):
// the cases of a node are adjacent in memory, so a pair loads as one float2 and every operation of the
// element arithmetic is the same for both; the element records are shared and broadcast to both halves.
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// The tet_acc_s arithmetic for a pair of cases.
template <int A0, int A1, int A2, int A3>
__device__ __forceinline__ void tet_acc_p(const float* re, float aM, float aK, const float2 (&P)[8][3],
                                          float2 (&Q)[8][3]) {
  float r[12];
  SVec4<float>::load12(re, r);
  const float2 lam = bc2(aK * r[9]), mu = bc2(aK * r[10]), ms = bc2(aM * r[11]);
  float2 G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float2 d1 = sub2(P[A1][i], P[A0][i]), d2 = sub2(P[A2][i], P[A0][i]), d3 = sub2(P[A3][i], P[A0][i]);
#pragma unroll
    for (int j = 0; j < 3; ++j) G[i][j] = fma2(d3, bc2(r[6 + j]), fma2(d2, bc2(r[3 + j]), mul2(d1, bc2(r[j]))));
  }
  const float2 tr = add2(add2(G[0][0], G[1][1]), G[2][2]);
  const float2 mu2 = add2(mu, mu);
  const float2 ltr = mul2(lam, tr);
  float2 S[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) S[i][i] = fma2(mu2, G[i][i], ltr);
  S[0][1] = S[1][0] = mul2(mu, add2(G[0][1], G[1][0]));
  S[0][2] = S[2][0] = mul2(mu, add2(G[0][2], G[2][0]));
  S[1][2] = S[2][1] = mul2(mu, add2(G[1][2], G[2][1]));
  float2 F[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      F[b][i] = fma2(S[i][2], bc2(r[3 * b + 2]), fma2(S[i][1], bc2(r[3 * b + 1]), mul2(S[i][0], bc2(r[3 * b]))));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 sum = add2(add2(P[A0][k], P[A1][k]), add2(P[A2][k], P[A3][k]));
    const float2 fs = add2(add2(F[0][k], F[1][k]), F[2][k]);
    Q[A0][k] = fma2(ms, add2(P[A0][k], sum), sub2(Q[A0][k], fs));
    Q[A1][k] = fma2(ms, add2(P[A1][k], sum), add2(Q[A1][k], F[0][k]));
    Q[A2][k] = fma2(ms, add2(P[A2][k], sum), add2(Q[A2][k], F[1][k]));
    Q[A3][k] = fma2(ms, add2(P[A3][k], sum), add2(Q[A3][k], F[2][k]));
  }
}

// One hex for a pair of cases, corner offsets o[] into the staged tile.  The six tets are visited around
// the cycle of their middle corners (the diagonal corners 0 and 3 are in all six), so each middle corner's
// values are loaded just before its first tet and its sums leave for the tile accumulator right after its
// second; corner 2, which closes the cycle, leaves after the first tet and is loaded again for the last,
// so at most four corners are live at once (instead of all eight held through the hex).
template <bool DOT>
__device__ __forceinline__ void hex_acc_p(const float* ps, int* qs, const int (&o)[8], int rpad, const float* re,
                                          float aM, float aK, float2 sinv, float2& hd) {
  float2 P[8][3], Q[8][3];
  auto ld = [&](int sl) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      P[sl][k] = *reinterpret_cast<const float2*>(ps + o[sl] + k * rpad);
      Q[sl][k] = make_float2(0.f, 0.f);
    }
  };
  // corner sums leave in fixed point: Q scaled by the tile's power of two sinv, rounded to integers and
  // added by native integer shared-memory atomics (a float atomic add on shared memory is a compare-and-
  // swap loop)
  auto fl = [&](int sl) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (DOT) hd = fma2(P[sl][k], Q[sl][k], hd);
      int* d = qs + o[sl] + k * rpad;
      const float2 v = mul2(Q[sl][k], sinv);
      atomicAdd(d, __float2int_rn(v.x));
      atomicAdd(d + 1, __float2int_rn(v.y));
    }
  };
  static_assert(kHexTet[0][1] == 1 && kHexTet[0][2] == 2 && kHexTet[1][3] == 4 && kHexTet[4][1] == 7 &&
                    kHexTet[5][3] == 6 && kHexTet[3][1] == 5,
                "the visiting order follows the corner table");
  ld(0), ld(3), ld(1), ld(2);
  tet_acc_p<kHexTet[0][0], kHexTet[0][1], kHexTet[0][2], kHexTet[0][3]>(re + 0 * kRec, aM, aK, P, Q);
  fl(2);
  ld(4);
  tet_acc_p<kHexTet[1][0], kHexTet[1][1], kHexTet[1][2], kHexTet[1][3]>(re + 1 * kRec, aM, aK, P, Q);
  fl(1);
  ld(7);
  tet_acc_p<kHexTet[4][0], kHexTet[4][1], kHexTet[4][2], kHexTet[4][3]>(re + 4 * kRec, aM, aK, P, Q);
  fl(4);
  ld(6);
  tet_acc_p<kHexTet[5][0], kHexTet[5][1], kHexTet[5][2], kHexTet[5][3]>(re + 5 * kRec, aM, aK, P, Q);
  fl(7);
  ld(5);
  tet_acc_p<kHexTet[3][0], kHexTet[3][1], kHexTet[3][2], kHexTet[3][3]>(re + 3 * kRec, aM, aK, P, Q);
  fl(6);
  ld(2);
  tet_acc_p<kHexTet[2][0], kHexTet[2][1], kHexTet[2][2], kHexTet[2][3]>(re + 2 * kRec, aM, aK, P, Q);
  fl(5), fl(2), fl(0), fl(3);
}

// ------------------------------------------------------------------------------------------------------
// TMA-staged tiled hex kernel.  Tile t's element records (one contiguous block) and its nodes' values of
// p (3 x rpad contiguous values per node) are brought into shared memory by bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier), double-buffered: while tile t is computed,
// the copies of tile t+1 are in flight.  The per-hex arithmetic then reads only shared memory.  Waits are
// bounded; a wait that gives up sets g_tma_timeout (the results are then not valid and the caller reports
// FEM_ERR_TIMEOUT).  Needs 3 x rpad x sizeof(T) to be a multiple of 16 bytes (rpad >= 4 for FP32).
// ------------------------------------------------------------------------------------------------------
__device__ int g_tma_timeout = 0;
// Tries of the reporting wait (fem_opts.wait_budget, set by the host before a solve; device-wide).
constexpr int kDrainTries = 1 << 20;
__device__ int g_wait_budget = kDrainTries;

struct StagedLayout {
  size_t bar, qs, ps0, ps1, rec0, rec1, node0, node1, loc0, loc1, acc, total;
};
template <typename T>
__host__ __device__ inline StagedLayout staged_layout(int nloc_max, int rpad, int hex_per_tile, int nseg) {
  auto up = [](size_t x) { return (x + 127) & ~(size_t)127; };
  StagedLayout L;
  const size_t vals = up((size_t)nloc_max * 3 * rpad * sizeof(T));
  const size_t recs = up(sizeof(T) * (size_t)hex_per_tile * 6 * kRec);
  const size_t nodes = up(sizeof(int) * (size_t)nloc_max);
  L.bar = 0;
  L.qs = 512;   // head: 2 mbarriers, then (packed kernel) per-case |p| maxima x2 and scales
  L.ps0 = L.qs + vals;
  L.ps1 = L.ps0 + vals;
  L.rec0 = L.ps1 + vals;
  L.rec1 = L.rec0 + recs;
  L.node0 = L.rec1 + recs;
  L.node1 = L.node0 + nodes;
  L.loc0 = L.loc1 = L.node1 + nodes;   // (corner tables are not staged in this variant)
  L.acc = L.node1 + nodes;
  L.total = L.acc + sizeof(double) * (size_t)nseg;
  return L;
}

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }
__device__ __forceinline__ uint64_t gmem_u64(const void* ptr) {
  uint64_t g;
  asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(ptr));
  return g;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(gmem_u64(src)), "r"(bytes), "r"(bar)
               : "memory");
}
// Bounded wait for phase `parity` of the barrier; false if it did not complete.  Each try may suspend the
// thread for up to 1 us (instead of spinning on the issue slots the other block of the SM computes with);
// at most `tries` tries (2^20: about a second).  The kernels first wait with the budget g_wait_budget and
// report a wait that gives up; they then wait again with kDrainTries, so that no bulk copy is still in
// flight when the block moves on to its next tile or exits.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int tries = kDrainTries) {
  for (int i = 0; i < tries; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <typename T, bool DOT, bool SEG, int PK>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4 && PK != 2) ? 2 : 1) k_ebe_hex_staged(
    HexTiles ht, MeshView m, int rpad, int rshift, const T* __restrict__ p, T* __restrict__ q, T aM, T aK, Reducer red,
    CgCase* sc, double* ptq_out, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const StagedLayout L = staged_layout<T>(ht.nloc_max, rpad, ht.hex_per_tile, SEG ? m.nseg : 0);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + L.bar);
  T* qs = reinterpret_cast<T*>(smem_raw + L.qs);
  // buffer b of each double-buffered section (selected arithmetically: no local-memory pointer arrays)
  auto psb = [&](int b) { return reinterpret_cast<T*>(smem_raw + (b ? L.ps1 : L.ps0)); };
  auto srb = [&](int b) { return reinterpret_cast<T*>(smem_raw + (b ? L.rec1 : L.rec0)); };
  auto snb = [&](int b) { return reinterpret_cast<int*>(smem_raw + (b ? L.node1 : L.node0)); };
  double* sacc = reinterpret_cast<double*>(smem_raw + L.acc);
  constexpr bool seg = DOT && SEG;
  const int per_node = 3 * rpad;
  const uint32_t node_bytes = (uint32_t)(per_node * sizeof(T));
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (seg)
    for (int t = threadIdx.x; t < m.nseg; t += blockDim.x) sacc[t] = 0.0;
  __syncthreads();
  const T* __restrict__ rec = rec_of<T>(m);
  // node ids of a tile (each thread owns tile nodes threadIdx.x and threadIdx.x + kBlock)
  auto load_nodes = [&](int t, int (&nd)[2]) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int l = threadIdx.x + j * kBlock;
      nd[j] = 0;
      if (t < ht.n_tiles) {
        const int n0 = ht.tile_node_off[t];
        if (l < ht.tile_node_off[t + 1] - n0) nd[j] = ht.tile_nodes[n0 + l];
      }
    }
  };
  // bulk copies of tile t into buffer b (the buffer's previous readers have passed a block barrier)
  auto issue = [&](int t, int b, const int (&nd)[2]) {
    const int n0 = ht.tile_node_off[t], nl = ht.tile_node_off[t + 1] - n0;
    const int h0 = ht.tile_hex_off[t], nh = ht.tile_hex_off[t + 1] - h0;
    const uint32_t bar = smem_u32(mbar + b);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
      const uint32_t rbytes = (uint32_t)(nh * 6 * kRec * sizeof(T));
      mbar_expect_tx(bar, rbytes + (uint32_t)nl * node_bytes);
      bulk_g2s(smem_u32(srb(b)), rec + (int64_t)h0 * 6 * kRec, rbytes, bar);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int l = threadIdx.x + j * kBlock;
      if (l < nl) {
        snb(b)[l] = nd[j];
        bulk_g2s(smem_u32(psb(b) + (int64_t)l * per_node), p + (int64_t)(nd[j] & 0x0fffffff) * per_node, node_bytes,
                 bar);
      }
    }
  };
  double dot = 0.0, dot1 = 0.0;   // (packed: dot1 is the second case of the thread's pair)
  constexpr bool pk = PK != 0;
  int nd_next[2], nd_after[2];
  const int t0 = blockIdx.x;
  {
    int nd0[2];
    load_nodes(t0, nd0);
    load_nodes(t0 + gridDim.x, nd_next);
    if (t0 < ht.n_tiles) issue(t0, 0, nd0);
  }
  // packed: fixed-point tile sums.  Per tile and case c the scale is 2^(30 - E_c) with 2^E_c >= bound_c =
  // (|aM| abs_m + |aK| abs_k) max |p_c| over the tile's nodes, which bounds every partial sum of element
  // contributions to a tile node's row: the integer sums stay below 2^30, and the rounding of the sums is
  // below 2^-31 bound_c per contribution.  spm[2][32]: the per-case maxima (|p| bit patterns, ordered as
  // integers), one buffer per tile parity; sfwd[32]: 2^(E_c - 30), the factors back to floating point.
  int* spm = reinterpret_cast<int*>(smem_raw + 32);
  float* sfwd = reinterpret_cast<float*>(smem_raw + 288);
  const float bco = fabsf((float)aM) * ht.abs_m + fabsf((float)aK) * ht.abs_k;
  if constexpr (pk) {   // the tile accumulator starts zeroed; each flush zeroes what it reads
    for (int i = threadIdx.x; i < (ht.nloc_max * per_node) >> 2; i += blockDim.x)
      reinterpret_cast<float4*>(qs)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if ((int)threadIdx.x < 2 * 32) spm[threadIdx.x] = 0;
  }
  // packed: the case pairs with an active case (inner iterations; all pairs otherwise), nap of them, laid
  // on napw >= nap item slots (a power of two, so a thread's slot, and pair, is fixed); a converged pair's
  // product is not needed (its step length is zero)
  uint32_t pmask = 0;
  int nap = 0, napw = 1, lgw = 0, mypair = -1;
  if constexpr (pk) {
    const int npair = rpad >> 1;
    if (DOT && sc) {
      for (int pr = 0; pr < npair; ++pr)
        if (sc[2 * pr].active || sc[2 * pr + 1].active) pmask |= 1u << pr;
    } else {
      pmask = npair >= 32 ? 0xffffffffu : ((1u << npair) - 1u);
    }
    nap = __popc(pmask);
    while (napw < nap) napw <<= 1, ++lgw;
    const int slot = threadIdx.x & (napw - 1);
    if (slot < nap) {   // the slot-th active pair
      uint32_t m = pmask;
      for (int q = 0; q < slot; ++q) m &= m - 1;
      mypair = __ffs(m) - 1;
    }
  }
  for (int k = 0;; ++k) {
    const int t = t0 + k * gridDim.x;
    if (t >= ht.n_tiles) break;
    const int b = k & 1;
    const int tn = t + gridDim.x;
    if (tn < ht.n_tiles) issue(tn, b ^ 1, nd_next);
    if constexpr (!PK) load_nodes(tn + gridDim.x, nd_after);
    const int n0 = ht.tile_node_off[t], nl = ht.tile_node_off[t + 1] - n0;
    const int h0 = ht.tile_hex_off[t], nh = ht.tile_hex_off[t + 1] - h0;
    if constexpr (!pk) {   // (the packed flush leaves the accumulator zeroed behind it)
      for (int i = threadIdx.x; i < nl * per_node; i += blockDim.x) qs[i] = (T)0;
    }
    const uint32_t bar = smem_u32(mbar + b);
    if (!mbar_wait(bar, (uint32_t)((k >> 1) & 1), g_wait_budget)) {
      atomicExch(&g_tma_timeout, 1);
      mbar_wait(bar, (uint32_t)((k >> 1) & 1));   // second bounded wait for the copies still in flight
    }
    __syncthreads();
    const T* ps = psb(b);
    const T* sr = srb(b);
    const int* snode = snb(b);
    float2 sinv = make_float2(1.f, 1.f);
    if constexpr (pk) {
      // per-case largest |p| of the staged tile (a thread's values all belong to case threadIdx.x mod rpad)
      const float* pf = reinterpret_cast<const float*>(ps);
      float mx = 0.f;
      for (int i = threadIdx.x; i < nl * per_node; i += blockDim.x) mx = fmaxf(mx, fabsf(pf[i]));
      for (int off = 16; off >= rpad; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      int* spm_b = spm + (b << 5);
      if ((int)(threadIdx.x & 31) < rpad) atomicMax(spm_b + (threadIdx.x & 31), __float_as_int(mx));
      if ((int)threadIdx.x < rpad) spm[((b ^ 1) << 5) + threadIdx.x] = 0;   // the next tile's buffer
      __syncthreads();
      // E_c: the exponent field of bound_c gives bound_c < 2^(field - 126)
      auto expo = [&](int c) {
        const uint32_t f = (__float_as_uint(bco * __int_as_float(spm_b[c])) >> 23) & 0xffu;
        return f == 0u ? -126 : (int)f - 126;
      };
      auto pow2 = [](int e) { return __uint_as_float((uint32_t)min(max(e + 127, 1), 254) << 23); };
      if (mypair >= 0) sinv = make_float2(pow2(30 - expo(2 * mypair)), pow2(30 - expo(2 * mypair + 1)));
      if ((int)threadIdx.x < rpad) sfwd[threadIdx.x] = pow2(expo(threadIdx.x) - 30);
    }
    if constexpr (pk) {
      // items (hex, active-pair slot); a thread's slot and pair are fixed (blockDim.x is a multiple of napw)
      const int items = mypair >= 0 ? nh << lgw : 0;
      const int c0 = mypair << 1;
      float2 tdot2 = make_float2(0.f, 0.f);
      uint4 lw_next = (int)threadIdx.x < items ? __ldg(ht.hex_local + h0 + (threadIdx.x >> lgw)) : make_uint4(0, 0, 0, 0);
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int hl = it >> lgw;
        const uint4 lw = lw_next;
        if (it + (int)blockDim.x < items) lw_next = __ldg(ht.hex_local + h0 + ((it + blockDim.x) >> lgw));
        const int o[8] = {(int)(lw.x & 0xffff) * per_node + c0, (int)(lw.x >> 16) * per_node + c0,
                          (int)(lw.y & 0xffff) * per_node + c0, (int)(lw.y >> 16) * per_node + c0,
                          (int)(lw.z & 0xffff) * per_node + c0, (int)(lw.z >> 16) * per_node + c0,
                          (int)(lw.w & 0xffff) * per_node + c0, (int)(lw.w >> 16) * per_node + c0};
        hex_acc_p<DOT>(reinterpret_cast<const float*>(ps), reinterpret_cast<int*>(qs), o, rpad,
                       reinterpret_cast<const float*>(sr) + hl * 6 * kRec, (float)aM, (float)aK, sinv, tdot2);
      }
      dot += (double)tdot2.x;
      dot1 += (double)tdot2.y;
      load_nodes(tn + gridDim.x, nd_after);   // (after the items: fewer registers live through them)
    } else {
    T tdot = 0;
    const int items = nh << rshift;
    const int rounds_end = seg ? ((items + blockDim.x - 1) / blockDim.x) * blockDim.x : items;
    // the corner table of the thread's next item is loaded one item ahead
    uint4 lw_next = (int)threadIdx.x < items ? __ldg(ht.hex_local + h0 + (threadIdx.x >> rshift)) : make_uint4(0, 0, 0, 0);
    for (int it = threadIdx.x; it < rounds_end; it += blockDim.x) {
      if (it >= items) {
        double z1[1] = {0.0};
        seg_add<1>(sacc, m.nseg, 0, z1);
        continue;
      }
      const int hl = it >> rshift, c = it & (rpad - 1);
      const uint4 lw = lw_next;
      if (it + (int)blockDim.x < items) lw_next = __ldg(ht.hex_local + h0 + ((it + blockDim.x) >> rshift));
      int ls[8] = {(int)(lw.x & 0xffff), (int)(lw.x >> 16), (int)(lw.y & 0xffff), (int)(lw.y >> 16),
                   (int)(lw.z & 0xffff), (int)(lw.z >> 16), (int)(lw.w & 0xffff), (int)(lw.w >> 16)};
      T P[8][3], Q[8][3];
#pragma unroll
      for (int sl = 0; sl < 8; ++sl)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          P[sl][kk] = ps[ls[sl] * per_node + (kk << rshift) + c];
          Q[sl][kk] = (T)0;
        }
      const T* re = sr + hl * 6 * kRec;
      tet_acc_s<T, kHexTet[0][0], kHexTet[0][1], kHexTet[0][2], kHexTet[0][3]>(re + 0 * kRec, aM, aK, P, Q);
      tet_acc_s<T, kHexTet[1][0], kHexTet[1][1], kHexTet[1][2], kHexTet[1][3]>(re + 1 * kRec, aM, aK, P, Q);
      tet_acc_s<T, kHexTet[2][0], kHexTet[2][1], kHexTet[2][2], kHexTet[2][3]>(re + 2 * kRec, aM, aK, P, Q);
      tet_acc_s<T, kHexTet[3][0], kHexTet[3][1], kHexTet[3][2], kHexTet[3][3]>(re + 3 * kRec, aM, aK, P, Q);
      tet_acc_s<T, kHexTet[4][0], kHexTet[4][1], kHexTet[4][2], kHexTet[4][3]>(re + 4 * kRec, aM, aK, P, Q);
      tet_acc_s<T, kHexTet[5][0], kHexTet[5][1], kHexTet[5][2], kHexTet[5][3]>(re + 5 * kRec, aM, aK, P, Q);
      T hdot = 0;
#pragma unroll
      for (int sl = 0; sl < 8; ++sl)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          if (DOT) hdot += P[sl][kk] * Q[sl][kk];
          atomicAdd(qs + ls[sl] * per_node + (kk << rshift) + c, Q[sl][kk]);
        }
      if (seg) {
        double v1[1] = {(double)hdot};
        seg_add<1>(sacc, m.nseg, m.seg[snode[ls[0]] & 0x0fffffff], v1);
      } else {
        tdot += hdot;
      }
    }
    dot += (double)tdot;
    }
    __syncthreads();
    if constexpr (pk) {
      // float4 pieces of the tile accumulator (four cases of one component of one node)
      const int sh4 = rshift - 2;
      const int f4 = per_node >> 2;
      for (int i = threadIdx.x; i < nl * f4; i += blockDim.x) {
        const int l = (i >> sh4) / 3, kk = (i - l * f4) >> sh4;
        const int raw = snode[l];
        const int64_t g = raw & 0x0fffffff;
        const bool fixed = !dof_free((uint8_t)((raw >> 28) & 7), kk);
        float4* dst = reinterpret_cast<float4*>(q + g * per_node) + (i - l * f4);
        const int4 vi = reinterpret_cast<const int4*>(qs)[i];
        const int c4 = (i << 2) & (rpad - 1);   // the four cases of this piece: c4 .. c4 + 3
        const float4 v = make_float4((float)vi.x * sfwd[c4], (float)vi.y * sfwd[c4 + 1], (float)vi.z * sfwd[c4 + 2],
                                     (float)vi.w * sfwd[c4 + 3]);
        reinterpret_cast<int4*>(qs)[i] = make_int4(0, 0, 0, 0);
        if (raw < 0) {
          if (!fixed) atomicAdd(dst, v);
        } else {
          *dst = fixed ? make_float4(0.f, 0.f, 0.f, 0.f) : v;
        }
      }
    } else
    for (int i = threadIdx.x; i < nl * per_node; i += blockDim.x) {
      const int l = (i >> rshift) / 3, rem = i - l * per_node;
      const int kk = rem >> rshift;
      const int raw = snode[l];
      const int64_t g = raw & 0x0fffffff;
      const bool fixed = !dof_free((uint8_t)((raw >> 28) & 7), kk);
      T* dst = q + g * per_node + rem;
      if (raw < 0) {
        if (!fixed) atomicAdd(dst, qs[i]);
      } else {
        *dst = fixed ? (T)0 : qs[i];
      }
    }
    __syncthreads();
    nd_next[0] = nd_after[0];
    nd_next[1] = nd_after[1];
  }
  if (DOT) {
    if (seg) {
      if (block_reduce_last_seg<1>(sacc, m.nseg, red)) ebe_tail_seg(red, sc, ptq_out, m.nseg);
    } else if constexpr (pk) {
      // slot sums over the warp's hexes, then over the warps (through the idle record buffer), then thread
      // c < rpad takes case c (the layout of the block reduction); converged pairs give 0
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      double d0 = dot, d1 = dot1;
      for (int off = napw; off < 32; off <<= 1) {
        d0 += __shfl_xor_sync(0xffffffffu, d0, off);
        d1 += __shfl_xor_sync(0xffffffffu, d1, off);
      }
      double* spair = reinterpret_cast<double*>(smem_raw + L.rec0);   // [warp][16 slots][2]
      __syncthreads();
      if (lane < napw) {
        spair[(warp * 16 + lane) * 2] = d0;
        spair[(warp * 16 + lane) * 2 + 1] = d1;
      }
      __syncthreads();
      double vc = 0.0;
      if ((int)threadIdx.x < rpad) {
        const int pr = threadIdx.x >> 1;
        if ((pmask >> pr) & 1u) {
          const int sl = __popc(pmask & ((1u << pr) - 1u));
          for (int w = 0; w < nw; ++w) vc += spair[(w * 16 + sl) * 2 + (threadIdx.x & 1)];
        }
      }
      double v[1] = {vc};
      if (block_reduce_last<1>(v, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);
    } else {
      double v[1] = {dot};
      if (block_reduce_last<1>(v, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);
    }
  }
}

// ------------------------------------------------------------------------------------------------------
// Case-major staged variant: the same TMA double-buffered tiles, but each warp applies 32 hexes of ONE case,
// so a case whose inner solve has converged (sc[c].active == 0) skips its warps entirely (the product of a
// converged case is not used: its step length is zero).  Node rows in shared memory are padded to PN
// values (PN = 4 mod 8 for FP32, PN = 2 mod 4 for FP64: 16-byte rows) so that lanes reading different nodes spread
// over the banks.  One block of 512 threads per SM.  Per-case p^T q sums go through shared memory.
// ------------------------------------------------------------------------------------------------------
constexpr int kBlockCM = 512;

template <typename T>
__host__ __device__ inline int cm_stride(int rpad) {
  int pn = 3 * rpad;
  if (sizeof(T) == 4) {
    while (pn % 8 != 4) ++pn;
  } else {
    while (pn % 4 != 2) ++pn;
  }
  return pn;
}

template <typename T>
__host__ __device__ inline StagedLayout cm_layout(int nloc_max, int rpad, int hex_per_tile, int nseg) {
  auto up = [](size_t x) { return (x + 127) & ~(size_t)127; };
  StagedLayout L;
  const size_t vals = up((size_t)nloc_max * cm_stride<T>(rpad) * sizeof(T));
  const size_t recs = up(sizeof(T) * (size_t)hex_per_tile * 6 * kRec);
  const size_t nodes = up(sizeof(int) * (size_t)nloc_max);
  L.bar = 0;
  L.qs = 128;
  L.ps0 = L.qs + vals;
  L.ps1 = L.ps0 + vals;
  L.rec0 = L.ps1 + vals;
  L.rec1 = L.rec0 + recs;
  L.node0 = L.rec1 + recs;
  L.node1 = L.node0 + nodes;
  L.loc0 = L.node1 + nodes;
  L.loc1 = L.loc0 + up(sizeof(uint4) * (size_t)hex_per_tile);
  L.acc = L.loc1 + up(sizeof(uint4) * (size_t)hex_per_tile);
  L.total = L.acc + sizeof(double) * (size_t)nseg;
  return L;
}

template <typename T, bool DOT>
__global__ void __launch_bounds__(kBlockCM, 1) k_ebe_hex_cm(HexTiles ht, MeshView m, int rpad, int rshift,
                                                            const T* __restrict__ p, T* __restrict__ q, T aM, T aK,
                                                            Reducer red, CgCase* sc, double* ptq_out, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const StagedLayout L = cm_layout<T>(ht.nloc_max, rpad, ht.hex_per_tile, 0);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + L.bar);
  T* qs = reinterpret_cast<T*>(smem_raw + L.qs);
  auto psb = [&](int b) { return reinterpret_cast<T*>(smem_raw + (b ? L.ps1 : L.ps0)); };
  auto srb = [&](int b) { return reinterpret_cast<T*>(smem_raw + (b ? L.rec1 : L.rec0)); };
  auto snb = [&](int b) { return reinterpret_cast<int*>(smem_raw + (b ? L.node1 : L.node0)); };
  auto lcb = [&](int b) { return reinterpret_cast<uint4*>(smem_raw + (b ? L.loc1 : L.loc0)); };
  const int per_node = 3 * rpad;
  const int PN = cm_stride<T>(rpad);
  const uint32_t node_bytes = (uint32_t)(per_node * sizeof(T));
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init(smem_u32(mbar + 1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // cases whose product is needed: all, unless the solve state says a case has converged
  unsigned live = 0xffffffffu;
  if (DOT && sc)
    for (int c = 0; c < rpad; ++c)
      if (!sc[c].active) live &= ~(1u << c);
  const T* __restrict__ rec = rec_of<T>(m);
  auto load_node = [&](int t) {
    int nd = 0;
    if (t < ht.n_tiles) {
      const int n0 = ht.tile_node_off[t];
      if ((int)threadIdx.x < ht.tile_node_off[t + 1] - n0) nd = ht.tile_nodes[n0 + threadIdx.x];
    }
    return nd;
  };
  auto issue = [&](int t, int b, int nd) {
    const int n0 = ht.tile_node_off[t], nl = ht.tile_node_off[t + 1] - n0;
    const int h0 = ht.tile_hex_off[t], nh = ht.tile_hex_off[t + 1] - h0;
    const uint32_t bar = smem_u32(mbar + b);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
      const uint32_t rbytes = (uint32_t)(nh * 6 * kRec * sizeof(T));
      const uint32_t lbytes = (uint32_t)(nh * sizeof(uint4));
      mbar_expect_tx(bar, rbytes + lbytes + (uint32_t)nl * node_bytes);
      bulk_g2s(smem_u32(srb(b)), rec + (int64_t)h0 * 6 * kRec, rbytes, bar);
      bulk_g2s(smem_u32(lcb(b)), ht.hex_local + h0, lbytes, bar);
    }
    const int l = threadIdx.x;
    if (l < nl) {
      snb(b)[l] = nd;
      bulk_g2s(smem_u32(psb(b) + (int64_t)l * PN), p + (int64_t)(nd & 0x0fffffff) * per_node, node_bytes, bar);
    }
  };
  __shared__ double sdot[kMaxRpad];
  if (DOT && threadIdx.x < kMaxRpad) sdot[threadIdx.x] = 0.0;
  const int t0 = blockIdx.x;
  int nd_next = load_node(t0 + gridDim.x);
  issue(t0, 0, load_node(t0));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0;; ++k) {
    const int t = t0 + k * gridDim.x;
    if (t >= ht.n_tiles) break;
    const int b = k & 1;
    const int tn = t + gridDim.x;
    if (tn < ht.n_tiles) issue(tn, b ^ 1, nd_next);
    const int nd_after = load_node(tn + gridDim.x);
    const int n0 = ht.tile_node_off[t], nl = ht.tile_node_off[t + 1] - n0;
    const int h0 = ht.tile_hex_off[t], nh = ht.tile_hex_off[t + 1] - h0;
    for (int i = threadIdx.x; i < nl * PN; i += blockDim.x) qs[i] = (T)0;
    const uint32_t bar = smem_u32(mbar + b);
    if (!mbar_wait(bar, (uint32_t)((k >> 1) & 1), g_wait_budget)) {
      atomicExch(&g_tma_timeout, 1);
      mbar_wait(bar, (uint32_t)((k >> 1) & 1));
    }
    __syncthreads();
    const T* ps = psb(b);
    const T* sr = srb(b);
    const int* snode = snb(b);
    const uint4* hexl = lcb(b);
    // warp-group g applies hexes 32 (g / rpad) .. +31 of case g % rpad
    const int groups = ((nh + 31) >> 5) << rshift;
    for (int gw = warp; gw < groups; gw += kBlockCM / 32) {
      const int c = gw & (rpad - 1);
      if (!((live >> c) & 1u)) continue;
      const int hl = ((gw >> rshift) << 5) + lane;
      T hdot = 0;
      if (hl < nh) {
        const uint4 lw = hexl[hl];
        int ls[8] = {(int)(lw.x & 0xffff), (int)(lw.x >> 16), (int)(lw.y & 0xffff), (int)(lw.y >> 16),
                     (int)(lw.z & 0xffff), (int)(lw.z >> 16), (int)(lw.w & 0xffff), (int)(lw.w >> 16)};
        T P[8][3], Q[8][3];
#pragma unroll
        for (int sl = 0; sl < 8; ++sl)
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            P[sl][kk] = ps[ls[sl] * PN + (kk << rshift) + c];
            Q[sl][kk] = (T)0;
          }
        const T* re = sr + hl * 6 * kRec;
        tet_acc_s<T, kHexTet[0][0], kHexTet[0][1], kHexTet[0][2], kHexTet[0][3]>(re + 0 * kRec, aM, aK, P, Q);
        tet_acc_s<T, kHexTet[1][0], kHexTet[1][1], kHexTet[1][2], kHexTet[1][3]>(re + 1 * kRec, aM, aK, P, Q);
        tet_acc_s<T, kHexTet[2][0], kHexTet[2][1], kHexTet[2][2], kHexTet[2][3]>(re + 2 * kRec, aM, aK, P, Q);
        tet_acc_s<T, kHexTet[3][0], kHexTet[3][1], kHexTet[3][2], kHexTet[3][3]>(re + 3 * kRec, aM, aK, P, Q);
        tet_acc_s<T, kHexTet[4][0], kHexTet[4][1], kHexTet[4][2], kHexTet[4][3]>(re + 4 * kRec, aM, aK, P, Q);
        tet_acc_s<T, kHexTet[5][0], kHexTet[5][1], kHexTet[5][2], kHexTet[5][3]>(re + 5 * kRec, aM, aK, P, Q);
#pragma unroll
        for (int sl = 0; sl < 8; ++sl)
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            if (DOT) hdot += P[sl][kk] * Q[sl][kk];
            atomicAdd(qs + ls[sl] * PN + (kk << rshift) + c, Q[sl][kk]);
          }
      }
      if (DOT) {   // the warp's lanes share one case: one shared-memory add per warp
        for (int off = 16; off > 0; off >>= 1) hdot += __shfl_xor_sync(0xffffffffu, hdot, off);
        if (lane == 0) atomicAdd(sdot + c, (double)hdot);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nl * per_node; i += blockDim.x) {
      const int l = (i >> rshift) / 3, rem = i - l * per_node;
      const int kk = rem >> rshift;
      const int raw = snode[l];
      const int64_t g = raw & 0x0fffffff;
      const bool fixed = !dof_free((uint8_t)((raw >> 28) & 7), kk);
      T* dst = q + g * per_node + rem;
      const T v = qs[l * PN + rem];
      if (raw < 0) {
        if (!fixed) atomicAdd(dst, v);
      } else {
        *dst = fixed ? (T)0 : v;
      }
    }
    __syncthreads();
    nd_next = nd_after;
  }
  if (DOT) {
    // block partials are per case: the lanes of the reduction hold case c in lane c
    if (block_reduce_last_seg<1>(sdot, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);
  }
}

template <typename T>
size_t ebe_hex_staged_smem(const HexTiles& ht, const MeshView& m, int rpad) {
  if ((3 * rpad * sizeof(T)) % 16 != 0 || ht.nloc_max > 2 * kBlock) return ~(size_t)0;   // not applicable
  return staged_layout<T>(ht.nloc_max, rpad, ht.hex_per_tile, m.seg ? m.nseg : 0).total;
}
template size_t ebe_hex_staged_smem<float>(const HexTiles&, const MeshView&, int);
template size_t ebe_hex_staged_smem<double>(const HexTiles&, const MeshView&, int);

template <typename T>
cudaError_t launch_ebe_hex_staged(const HexTiles& ht, const MeshView& m, int rpad, const T* p, T* q, double aM,
                                  double aK, const Reducer* red, CgCase* sc, double* ptq_out, const int* gate,
                                  cudaStream_t s, int packed) {
  const size_t smem = ebe_hex_staged_smem<T>(ht, m, rpad);
  if (smem == ~(size_t)0 || (reinterpret_cast<uintptr_t>(p) & 15) != 0) return cudaErrorInvalidValue;
  cudaError_t err = cudaMemsetAsync(q, 0, sizeof(T) * (size_t)m.N * 3 * rpad, s);
  if (err != cudaSuccess) return err;
  const int rs = log2i(rpad);
  const int nsm = sm_count();
  int per_sm = 1;
  // packed pairs: FP32 only, one case per lane of the node row (not fused groups), a 16-byte aligned output
  // (the tile flush writes float4 pieces); 1: registers capped for two blocks per SM, 2: one block per SM
  const int pk = (sizeof(T) == 4 && !m.seg && rpad >= 4 && (reinterpret_cast<uintptr_t>(q) & 15) == 0) ? packed : 0;
  auto kfn = red ? (m.seg ? k_ebe_hex_staged<T, true, true, 0> : k_ebe_hex_staged<T, true, false, 0>)
                 : k_ebe_hex_staged<T, false, false, 0>;
  if constexpr (sizeof(T) == 4) {
    if (pk == 1) kfn = red ? k_ebe_hex_staged<T, true, false, 1> : k_ebe_hex_staged<T, false, false, 1>;
    if (pk == 2) kfn = red ? k_ebe_hex_staged<T, true, false, 2> : k_ebe_hex_staged<T, false, false, 2>;
  }
  err = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBlock, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int grid = nsm * per_sm;
  if (grid > ht.n_tiles) grid = ht.n_tiles;
  if (grid > red_grid_cap()) grid = red_grid_cap();
  Reducer rd = red ? *red : Reducer{nullptr, nullptr, nullptr};
  kfn<<<grid, kBlock, smem, s>>>(ht, m, rpad, rs, p, q, (T)aM, (T)aK, rd, red ? sc : nullptr, red ? ptq_out : nullptr,
                                 gate);
  return cudaGetLastError();
}
template cudaError_t launch_ebe_hex_staged<double>(const HexTiles&, const MeshView&, int, const double*, double*,
                                                   double, double, const Reducer*, CgCase*, double*, const int*,
                                                   cudaStream_t, int);
template cudaError_t launch_ebe_hex_staged<float>(const HexTiles&, const MeshView&, int, const float*, float*, double,
                                                  double, const Reducer*, CgCase*, double*, const int*, cudaStream_t,
                                                  int);

// ------------------------------------------------------------------------------------------------------
// Hex element matrices (variant 7).  The six Kuhn tets of a hex are summed once into the hex's symmetric
// 24 x 24 operator A_h = aM M_h + aK K_h (in FP64 from the FP64 records, stored FP32), so a product applies
// each hex as one dense 24 x 24 block: 576 multiply-adds a case, with no per-tet strain and stress
// intermediates, at 1200 bytes of matrix a hex instead of 288 of tet records.  Per tet with gradients g_a
// (g_0 = -(g_1 + g_2 + g_3)), lambda V, mu V and rho V / 20:
//   K_ab = lambda V g_a g_b^T + mu V ((g_a . g_b) I + g_b g_a^T),   M_ab = rho V / 20 (1 + delta_ab) I.
// Storage: per hex the upper block triangle by corner rows -- for corner a the diagonal block as
// (xx, xy, xz, yy, yz, zz), then the blocks (a, b > a) row-major -- 300 values; hexes 2j and 2j + 1 are
// interleaved value by value, so one float2 holds an entry of both and a thread applies a PAIR OF HEXES to
// one case with paired FP32 operations on natural pairs (no broadcast operands).
// ------------------------------------------------------------------------------------------------------
__host__ __device__ constexpr int hm_row_off(int a) { return 6 * a + 9 * (7 * a - a * (a - 1) / 2); }
static_assert(hm_row_off(8) == kHexMatVals, "300 values a hex");

__global__ void k_hexmat_build(int64_t H, const double* __restrict__ rec, double aM, double aK,
                               float* __restrict__ out) {
  constexpr int T[6][4] = {{0, 1, 2, 3}, {0, 1, 3, 4}, {0, 5, 3, 2}, {0, 5, 6, 3}, {0, 7, 4, 3}, {0, 7, 3, 6}};
  const int64_t n = H * 36;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t h = w / 36;
    int bi = (int)(w - h * 36), a = 0;
    while (bi >= 8 - a) bi -= 8 - a, ++a;
    const int b = a + bi;
    double B[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int t = 0; t < 6; ++t) {
      int la = -1, lb = -1;
      for (int k = 0; k < 4; ++k) {
        if (T[t][k] == a) la = k;
        if (T[t][k] == b) lb = k;
      }
      if (la < 0 || lb < 0) continue;
      const double* r = rec + (h * 6 + t) * kRec;
      double ga[3], gb[3];
      for (int i = 0; i < 3; ++i) {
        ga[i] = la == 0 ? -(r[i] + r[3 + i] + r[6 + i]) : r[3 * (la - 1) + i];
        gb[i] = lb == 0 ? -(r[i] + r[3 + i] + r[6 + i]) : r[3 * (lb - 1) + i];
      }
      const double lam = aK * r[9], mu = aK * r[10], ms = aM * r[11] * (la == lb ? 2.0 : 1.0);
      const double gg = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
          B[i][k] += lam * ga[i] * gb[k] + mu * (gb[i] * ga[k] + (i == k ? gg : 0.0)) + (i == k ? ms : 0.0);
    }
    float* o = out + (h >> 1) * (2 * kHexMatVals) + (h & 1);
    if (a == b) {
      const int e = hm_row_off(a);
      const double d[6] = {B[0][0], B[0][1], B[0][2], B[1][1], B[1][2], B[2][2]};
      for (int j = 0; j < 6; ++j) o[2 * (e + j)] = (float)d[j];
    } else {
      const int e = hm_row_off(a) + 6 + 9 * (b - a - 1);
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) o[2 * (e + 3 * i + k)] = (float)B[i][k];
    }
  }
}

cudaError_t launch_hexmat_build(int64_t n_hex, const double* rec64, double aM, double aK, float* out,
                                cudaStream_t s) {
  const int64_t pairs = (n_hex + 1) / 2;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * 2 * kHexMatVals * (size_t)pairs, s);   // odd tail
  if (e != cudaSuccess || n_hex == 0) return e;
  k_hexmat_build<<<grid_for(n_hex * 36, wide_grid_cap()), kBlock, 0, s>>>(n_hex, rec64, aM, aK, out);
  return cudaGetLastError();
}

constexpr int kHmChunk = 32;   // hexes a staged chunk (16 interleaved pairs, 38.4 KB)

struct HexMatLayout {
  size_t qs, node, m0, m1, total;
};
__host__ __device__ inline HexMatLayout hexmat_layout(int nloc_max, int rpad) {
  auto up = [](size_t x) { return (x + 127) & ~(size_t)127; };
  HexMatLayout L;
  L.qs = 512;   // head: 2 mbarriers, per-case |p| maxima and scales
  L.node = L.qs + up((size_t)nloc_max * 3 * rpad * sizeof(int));
  L.m0 = L.node + up(sizeof(int) * (size_t)nloc_max);
  L.m1 = L.m0 + up(sizeof(float) * 2 * kHexMatVals * (kHmChunk / 2));
  L.total = L.m1 + up(sizeof(float) * 2 * kHexMatVals * (kHmChunk / 2));
  return L;
}

// Product q = A p with the hex matrices, r cases, FP32.  Tiles as in the staged kernel (its node list, the
// fixed-point tile accumulator and flush); the chunks of 32 hexes' matrices come by bulk asynchronous copies,
// double-buffered (the copy of chunk j + 1 runs while chunk j is applied); p is gathered straight from
// global memory (it is L2-resident: the search-direction pass has just written it).  Items are (hex pair,
// active case slot); a thread's case is fixed.  The matrix is applied row by row (corner a's three sums
// live at a time, then added to the tile accumulator), each stored off-diagonal block serving two rows.
// Measured slower than the tet form on the medium workload (167 against 105 us): the shared-memory loads
// of the matrix (one vector load a value pair for two lanes' worth of distinct data) and the gathers
// leave it latency-bound at 1.9 k instructions an item, 35% issue; applying each stored block to both of
// its corners from registers instead (one block of 8 warps per SM) measured 197 us.
template <bool DOT>
__global__ void __launch_bounds__(kBlock, 2) k_ebe_hexmat(HexTiles ht, const float* __restrict__ hm, int rpad,
                                                          const float* __restrict__ p, float* __restrict__ q,
                                                          float aM, float aK, Reducer red, CgCase* sc,
                                                          double* ptq_out, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const HexMatLayout L = hexmat_layout(ht.nloc_max, rpad);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);
  int* spm = reinterpret_cast<int*>(smem_raw + 32);          // [32] per-case largest |p| (bit patterns)
  float* sfwd = reinterpret_cast<float*>(smem_raw + 160);    // [32] 2^(E_c - 30)
  int* qs = reinterpret_cast<int*>(smem_raw + L.qs);
  int* snode = reinterpret_cast<int*>(smem_raw + L.node);
  auto smb = [&](int b) { return reinterpret_cast<const float4*>(smem_raw + (b ? L.m1 : L.m0)); };
  const int per_node = 3 * rpad;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < (ht.nloc_max * per_node) >> 2; i += blockDim.x)
    reinterpret_cast<int4*>(qs)[i] = make_int4(0, 0, 0, 0);
  if ((int)threadIdx.x < 32) spm[threadIdx.x] = 0;
  // active cases (inner iterations; all otherwise) on napw >= nac slots, a power of two: a thread's slot,
  // and case, are fixed (blockDim.x is a multiple of napw)
  uint32_t cmask = rpad >= 32 ? 0xffffffffu : ((1u << rpad) - 1u);
  if (DOT && sc) {
    cmask = 0;
    for (int c = 0; c < rpad; ++c)
      if (sc[c].active) cmask |= 1u << c;
  }
  const int nac = __popc(cmask);
  int napw = 1, lgw = 0, myc = -1;
  while (napw < nac) napw <<= 1, ++lgw;
  {
    const int slot = threadIdx.x & (napw - 1);
    if (slot < nac) {
      uint32_t mm = cmask;
      for (int k = 0; k < slot; ++k) mm &= mm - 1;
      myc = __ffs(mm) - 1;
    }
  }
  __syncthreads();
  const float bco = fabsf(aM) * ht.abs_m + fabsf(aK) * ht.abs_k;
  // chunk sequence of this block: tiles t0, t0 + grid, ..., each in chunks of kHmChunk hexes
  const int t0 = blockIdx.x;
  auto n_chunks = [&](int t) { return (ht.tile_hex_off[t + 1] - ht.tile_hex_off[t] + kHmChunk - 1) / kHmChunk; };
  auto issue = [&](int t, int ch, int b) {   // chunk ch of tile t into buffer b (its readers are past a barrier)
    const int hb = ht.tile_hex_off[t] + ch * kHmChunk;
    const int he = min(hb + kHmChunk, ht.tile_hex_off[t + 1]);
    const uint32_t bytes = (uint32_t)(sizeof(float) * 2 * kHexMatVals * ((he - hb + 1) >> 1));
    const uint32_t bar = smem_u32(mbar + b);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, bytes);
      bulk_g2s(smem_u32(smb(b)), hm + (int64_t)(hb >> 1) * (2 * kHexMatVals), bytes, bar);
    }
  };
  if (t0 < ht.n_tiles) issue(t0, 0, 0);
  double dsum = 0.0;
  int j = 0;   // chunk counter (buffer j & 1, phase (j >> 1) & 1)
  for (int t = t0; t < ht.n_tiles; t += gridDim.x) {
    const int n0 = ht.tile_node_off[t], nl = ht.tile_node_off[t + 1] - n0;
    const int h0 = ht.tile_hex_off[t], h1 = ht.tile_hex_off[t + 1];
    for (int l = threadIdx.x; l < nl; l += blockDim.x) snode[l] = ht.tile_nodes[n0 + l];
    __syncthreads();
    {
      // per-case largest |p| over the tile's nodes: float4 pieces, a thread's four cases fixed
      const int f4 = per_node >> 2, cq = rpad >> 2;
      float4 mx = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int i = threadIdx.x; i < nl * f4; i += blockDim.x) {
        const int l = i / f4;
        const float4 v = __ldg(reinterpret_cast<const float4*>(p + (int64_t)(snode[l] & 0x0fffffff) * per_node) +
                               (i - l * f4));
        mx.x = fmaxf(mx.x, fabsf(v.x)), mx.y = fmaxf(mx.y, fabsf(v.y));
        mx.z = fmaxf(mx.z, fabsf(v.z)), mx.w = fmaxf(mx.w, fabsf(v.w));
      }
      for (int off = cq; off < 32; off <<= 1) {
        mx.x = fmaxf(mx.x, __shfl_xor_sync(0xffffffffu, mx.x, off));
        mx.y = fmaxf(mx.y, __shfl_xor_sync(0xffffffffu, mx.y, off));
        mx.z = fmaxf(mx.z, __shfl_xor_sync(0xffffffffu, mx.z, off));
        mx.w = fmaxf(mx.w, __shfl_xor_sync(0xffffffffu, mx.w, off));
      }
      const int lane = threadIdx.x & 31;
      if (lane < cq) {
        const int c = 4 * (lane % cq);
        atomicMax(spm + c, __float_as_int(mx.x));
        atomicMax(spm + c + 1, __float_as_int(mx.y));
        atomicMax(spm + c + 2, __float_as_int(mx.z));
        atomicMax(spm + c + 3, __float_as_int(mx.w));
      }
    }
    __syncthreads();
    // E_c from the exponent field of bound_c (bound_c < 2^(field - 126)); scale 2^(30 - E_c)
    auto expo = [&](int c) {
      const uint32_t f = (__float_as_uint(bco * __int_as_float(spm[c])) >> 23) & 0xffu;
      return f == 0u ? -126 : (int)f - 126;
    };
    auto pow2 = [](int e) { return __uint_as_float((uint32_t)min(max(e + 127, 1), 254) << 23); };
    const float sv = myc >= 0 ? pow2(30 - expo(myc)) : 1.f;
    const float2 sinv = make_float2(sv, sv);
    if ((int)threadIdx.x < rpad) sfwd[threadIdx.x] = pow2(expo(threadIdx.x) - 30);
    const int nch = n_chunks(t);
    for (int ch = 0; ch < nch; ++ch, ++j) {
      const int b = j & 1;
      // the next chunk: this tile's next, else the first of the block's next tile
      {
        int tn = t, cn = ch + 1;
        if (cn == nch) tn = t + gridDim.x, cn = 0;
        if (tn < ht.n_tiles) issue(tn, cn, b ^ 1);
      }
      const uint32_t bar = smem_u32(mbar + b);
      if (!mbar_wait(bar, (uint32_t)((j >> 1) & 1), g_wait_budget)) {
        atomicExch(&g_tma_timeout, 1);
        mbar_wait(bar, (uint32_t)((j >> 1) & 1));   // second bounded wait for the copy still in flight
      }
      const float4* m4b = smb(b);
      const int hb = h0 + ch * kHmChunk;
      const int he = min(hb + kHmChunk, h1);
      const int npair = (he - hb + 1) >> 1;
      const int items = myc >= 0 ? npair << lgw : 0;
      float2 hd = make_float2(0.f, 0.f);
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int pr = it >> lgw;
        const int hA = hb + 2 * pr;
        const bool hasB = hA + 1 < he;
        const uint4 lA = __ldg(ht.hex_local + hA);
        const uint4 lB = hasB ? __ldg(ht.hex_local + hA + 1) : lA;
        auto loc = [](const uint4& w, int s) -> int {
          const uint32_t v = s < 2 ? w.x : s < 4 ? w.y : s < 6 ? w.z : w.w;
          return (int)((s & 1) ? (v >> 16) : (v & 0xffffu));
        };
        float2 P[8][3];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const float* pa = p + (int64_t)(snode[loc(lA, s)] & 0x0fffffff) * per_node + myc;
          const float* pb = p + (int64_t)(snode[loc(lB, s)] & 0x0fffffff) * per_node + myc;
#pragma unroll
          for (int k = 0; k < 3; ++k) P[s][k] = make_float2(__ldg(pa + k * rpad), __ldg(pb + k * rpad));
        }
        const float4* m4 = m4b + pr * (kHexMatVals / 2);
        auto M = [&](int e) -> float2 {
          const float4 v = m4[e >> 1];
          return (e & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
        };
        // row a of A: blocks (a, b >= a) as stored, blocks (b < a, a) transposed (the stored block read
        // again: the symmetric storage halves the matrix bytes, and only corner a's sums are live)
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          float2 Q[3];
          {
            const int e0 = hm_row_off(a);
            const float2 xx = M(e0), xy = M(e0 + 1), xz = M(e0 + 2), yy = M(e0 + 3), yz = M(e0 + 4), zz = M(e0 + 5);
            Q[0] = fma2(xz, P[a][2], fma2(xy, P[a][1], mul2(xx, P[a][0])));
            Q[1] = fma2(yz, P[a][2], fma2(yy, P[a][1], mul2(xy, P[a][0])));
            Q[2] = fma2(zz, P[a][2], fma2(yz, P[a][1], mul2(xz, P[a][0])));
          }
#pragma unroll
          for (int bb = 0; bb < 8; ++bb) {
            if (bb == a) continue;
            const int lo = bb < a ? bb : a, hi = bb < a ? a : bb;
            const int eb = hm_row_off(lo) + 6 + 9 * (hi - lo - 1);
            float2 B[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int k = 0; k < 3; ++k) B[i][k] = bb > a ? M(eb + 3 * i + k) : M(eb + 3 * k + i);
#pragma unroll
            for (int i = 0; i < 3; ++i)
              Q[i] = fma2(B[i][2], P[bb][2], fma2(B[i][1], P[bb][1], fma2(B[i][0], P[bb][0], Q[i])));
          }
          // corner a's sums: fixed point into the tile accumulator
          int* da = qs + loc(lA, a) * per_node + myc;
          int* db = qs + loc(lB, a) * per_node + myc;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (DOT) hd = fma2(P[a][k], Q[k], hd);
            const float2 v = mul2(Q[k], sinv);
            atomicAdd(da + k * rpad, __float2int_rn(v.x));
            if (hasB) atomicAdd(db + k * rpad, __float2int_rn(v.y));
          }
        }
      }
      if (DOT) dsum += (double)hd.x + (double)hd.y;
      __syncthreads();   // buffer b's readers are done; the tile accumulator is complete after the last chunk
    }
    // flush: float4 pieces of the tile accumulator (four cases of one component of one node)
    {
      const int sh4 = __ffs(rpad) - 3;
      const int f4 = per_node >> 2;
      for (int i = threadIdx.x; i < nl * f4; i += blockDim.x) {
        const int l = (i >> sh4) / 3, kk = (i - l * f4) >> sh4;
        const int raw = snode[l];
        const int64_t g = raw & 0x0fffffff;
        const bool fixed = !dof_free((uint8_t)((raw >> 28) & 7), kk);
        float4* dst = reinterpret_cast<float4*>(q + g * per_node) + (i - l * f4);
        const int4 vi = reinterpret_cast<const int4*>(qs)[i];
        const int c4 = (i << 2) & (rpad - 1);
        const float4 v = make_float4((float)vi.x * sfwd[c4], (float)vi.y * sfwd[c4 + 1], (float)vi.z * sfwd[c4 + 2],
                                     (float)vi.w * sfwd[c4 + 3]);
        reinterpret_cast<int4*>(qs)[i] = make_int4(0, 0, 0, 0);
        if (raw < 0) {
          if (!fixed) atomicAdd(dst, v);
        } else {
          *dst = fixed ? make_float4(0.f, 0.f, 0.f, 0.f) : v;
        }
      }
      if ((int)threadIdx.x < 32) spm[threadIdx.x] = 0;   // (its readers passed the chunk barriers)
    }
    __syncthreads();
  }
  if (DOT) {
    // case totals: lanes of one case slot are napw apart in a warp; warps through shared memory one slot at
    // a time would cost a barrier each, so each warp's slot sums go to a [warp][slot] table in the (idle)
    // matrix buffer, then thread c < rpad adds its case's column
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double d = dsum;
    for (int off = napw; off < 32; off <<= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    double* tab = reinterpret_cast<double*>(smem_raw + L.m0);   // [warp][32 slots]
    if (lane < napw) tab[warp * 32 + lane] = d;
    __syncthreads();
    double vc = 0.0;
    if ((int)threadIdx.x < rpad && ((cmask >> threadIdx.x) & 1u)) {
      const int sl = __popc(cmask & ((1u << threadIdx.x) - 1u));
      for (int w = 0; w < nw; ++w) vc += tab[w * 32 + sl];
    }
    double v[1] = {vc};
    if (block_reduce_last<1>(v, rpad, red)) ebe_tail(red, sc, ptq_out, rpad);
  }
}

size_t ebe_hexmat_smem(const HexTiles& ht, const MeshView& m, int rpad) {
  if (m.seg || rpad < 4 || rpad > 32 || ht.hex_per_tile % kHmChunk != 0) return ~(size_t)0;   // not applicable
  return hexmat_layout(ht.nloc_max, rpad).total;
}

cudaError_t launch_ebe_hexmat(const HexTiles& ht, const MeshView& m, const float* hm, int rpad, const float* p,
                              float* q, double aM, double aK, const Reducer* red, CgCase* sc, double* ptq_out,
                              const int* gate, cudaStream_t s) {
  const size_t smem = ebe_hexmat_smem(ht, m, rpad);
  if (smem == ~(size_t)0 || !hm || (reinterpret_cast<uintptr_t>(p) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(q) & 15) != 0)
    return cudaErrorInvalidValue;
  cudaError_t err = cudaMemsetAsync(q, 0, sizeof(float) * (size_t)m.N * 3 * rpad, s);
  if (err != cudaSuccess) return err;
  const int nsm = sm_count();
  int per_sm = 1;
  auto kfn = red ? k_ebe_hexmat<true> : k_ebe_hexmat<false>;
  err = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBlock, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int grid = nsm * per_sm;
  if (grid > ht.n_tiles) grid = ht.n_tiles;
  if (grid > red_grid_cap()) grid = red_grid_cap();
  Reducer rd = red ? *red : Reducer{nullptr, nullptr, nullptr};
  kfn<<<grid, kBlock, smem, s>>>(ht, hm, rpad, p, q, (float)aM, (float)aK, rd, red ? sc : nullptr,
                                 red ? ptq_out : nullptr, gate);
  return cudaGetLastError();
}

template <typename T>
size_t ebe_hex_cm_smem(const HexTiles& ht, const MeshView& m, int rpad) {
  if ((3 * rpad * sizeof(T)) % 16 != 0 || ht.nloc_max > kBlockCM || m.seg) return ~(size_t)0;   // not applicable
  return cm_layout<T>(ht.nloc_max, rpad, ht.hex_per_tile, 0).total;
}
template size_t ebe_hex_cm_smem<float>(const HexTiles&, const MeshView&, int);
template size_t ebe_hex_cm_smem<double>(const HexTiles&, const MeshView&, int);

template <typename T>
cudaError_t launch_ebe_hex_cm(const HexTiles& ht, const MeshView& m, int rpad, const T* p, T* q, double aM, double aK,
                              const Reducer* red, CgCase* sc, double* ptq_out, const int* gate, cudaStream_t s) {
  const size_t smem = ebe_hex_cm_smem<T>(ht, m, rpad);
  if (smem == ~(size_t)0 || (reinterpret_cast<uintptr_t>(p) & 15) != 0) return cudaErrorInvalidValue;
  cudaError_t err = cudaMemsetAsync(q, 0, sizeof(T) * (size_t)m.N * 3 * rpad, s);
  if (err != cudaSuccess) return err;
  const int rs = log2i(rpad);
  const int nsm = sm_count();
  auto kfn = red ? k_ebe_hex_cm<T, true> : k_ebe_hex_cm<T, false>;
  err = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int grid = nsm;
  if (grid > ht.n_tiles) grid = ht.n_tiles;
  Reducer rd = red ? *red : Reducer{nullptr, nullptr, nullptr};
  kfn<<<grid, kBlockCM, smem, s>>>(ht, m, rpad, rs, p, q, (T)aM, (T)aK, rd, red ? sc : nullptr,
                                   red ? ptq_out : nullptr, gate);
  return cudaGetLastError();
}
template cudaError_t launch_ebe_hex_cm<double>(const HexTiles&, const MeshView&, int, const double*, double*, double,
                                               double, const Reducer*, CgCase*, double*, const int*, cudaStream_t);
template cudaError_t launch_ebe_hex_cm<float>(const HexTiles&, const MeshView&, int, const float*, float*, double,
                                              double, const Reducer*, CgCase*, double*, const int*, cudaStream_t);

// Tries of the staged kernels' reporting wait for the launches ordered after this on s.
// (Each device starts with the default; the copy is skipped while the device already holds the value.)
cudaError_t ebe_set_wait_budget(int tries, cudaStream_t s) {
  static std::mutex mu;
  static std::unordered_map<int, int> held;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = held.find(dev);
  if (it != held.end() ? it->second == tries : tries == kDrainTries) return cudaSuccess;
  e = cudaMemcpyToSymbolAsync(g_wait_budget, &tries, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) held[dev] = tries;
  return e;
}

// Reads (and clears) the flag set when a staged kernel's bounded wait for its copies gave up.
cudaError_t ebe_tma_timeout(int* flag) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_tma_timeout, sizeof(int));
  if (e == cudaSuccess && *flag) e = cudaMemcpyToSymbol(g_tma_timeout, &zero, sizeof(int));
  return e;
}

// Split FP64 product for the certification pass: qM = M p and qK = K p in one pass over the elements (the
// increment's two products feed the recurrences of the right-hand side).  Generic element kernel.
__global__ void __launch_bounds__(kBlock) k_ebe_split(MeshView m, int rpad, int rshift, const double* __restrict__ p,
                                                      double* __restrict__ qM, double* __restrict__ qK) {
  const int64_t total = m.E << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const int4 cn = __ldg(m.conn + e);
    const int64_t nd[4] = {cn.x, cn.y, cn.z, cn.w};
    double r[12];
    Vec4<double>::load12(m.rec64 + e * kRec, r);
    double P[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) P[a][k] = p[(nd[a] * 3 + k) * rpad + c];
    double G[3][3];
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) {
      const double d1 = P[1][i2] - P[0][i2], d2 = P[2][i2] - P[0][i2], d3 = P[3][i2] - P[0][i2];
#pragma unroll
      for (int j = 0; j < 3; ++j) G[i2][j] = d1 * r[j] + d2 * r[3 + j] + d3 * r[6 + j];
    }
    const double lam = r[9], mu = r[10], ms = r[11];
    const double tr = G[0][0] + G[1][1] + G[2][2];
    double S[3][3];
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) S[i2][i2] = lam * tr + 2.0 * mu * G[i2][i2];
    S[0][1] = S[1][0] = mu * (G[0][1] + G[1][0]);
    S[0][2] = S[2][0] = mu * (G[0][2] + G[2][0]);
    S[1][2] = S[2][1] = mu * (G[1][2] + G[2][1]);
    double F[4][3];
#pragma unroll
    for (int b = 1; b < 4; ++b)
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
        F[b][i2] = S[i2][0] * r[(b - 1) * 3] + S[i2][1] * r[(b - 1) * 3 + 1] + S[i2][2] * r[(b - 1) * 3 + 2];
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) F[0][i2] = -(F[1][i2] + F[2][i2] + F[3][i2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double sum = P[0][k] + P[1][k] + P[2][k] + P[3][k];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        atomicAdd(qK + (nd[a] * 3 + k) * rpad + c, F[a][k]);
        atomicAdd(qM + (nd[a] * 3 + k) * rpad + c, ms * (P[a][k] + sum));
      }
    }
  }
}

cudaError_t launch_ebe_split(const MeshView& m, int rpad, const double* p, double* qM, double* qK, cudaStream_t s) {
  const size_t bytes = sizeof(double) * (size_t)m.N * 3 * rpad;
  cudaError_t err = cudaMemsetAsync(qM, 0, bytes, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(qK, 0, bytes, s);
  if (err != cudaSuccess) return err;
  const int rs = log2i(rpad);
  k_ebe_split<<<grid_for(m.E << rs), kBlock, 0, s>>>(m, rpad, rs, p, qM, qK);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
// Split product in double-float arithmetic (value = hi + lo, two FP32 numbers; 48-bit significand).
// GB300 issues FP32 at 64x its FP64 rate, so the certification product (q = M p and K p, needed to ~1e-12
// of ||b||) runs as error-free FP32 transforms instead of FP64 instructions.  Records are split once into
// (hi, lo) pairs; p is split on load; element contributions are converted back to FP64 and scattered with
// FP64 atomics.  __fadd_rn/__fmul_rn keep the transforms from being contracted into FMAs.
// ------------------------------------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl df_fast(float a, float b) {   // requires |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast(s.hi, e);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast(p, e);
}
__device__ __forceinline__ dfl df_from(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }

__global__ void __launch_bounds__(kBlock) k_ebe_split_df(MeshView m, const float* __restrict__ rec_df, int rpad,
                                                         int rshift, const double* __restrict__ p,
                                                         double* __restrict__ qM, double* __restrict__ qK) {
  const int64_t total = m.E << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const int4 cn = __ldg(m.conn + e);
    const int64_t nd[4] = {cn.x, cn.y, cn.z, cn.w};
    const float* re = rec_df + e * 24;
    dfl g[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) g[j] = {__ldg(re + 2 * j), __ldg(re + 2 * j + 1)};
    dfl P[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) P[a][k] = df_from(p[(nd[a] * 3 + k) * rpad + c]);
    dfl G[3][3];
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) {
      const dfl d1 = df_sub(P[1][i2], P[0][i2]), d2 = df_sub(P[2][i2], P[0][i2]), d3 = df_sub(P[3][i2], P[0][i2]);
#pragma unroll
      for (int j = 0; j < 3; ++j)
        G[i2][j] = df_add(df_add(df_mul(d1, g[j]), df_mul(d2, g[3 + j])), df_mul(d3, g[6 + j]));
    }
    const dfl lam = g[9], mu = g[10], ms = g[11];
    const dfl tr = df_add(df_add(G[0][0], G[1][1]), G[2][2]);
    const dfl ltr = df_mul(lam, tr);
    const dfl mu2 = df_add(mu, mu);
    dfl S[3][3];
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) S[i2][i2] = df_add(ltr, df_mul(mu2, G[i2][i2]));
    S[0][1] = S[1][0] = df_mul(mu, df_add(G[0][1], G[1][0]));
    S[0][2] = S[2][0] = df_mul(mu, df_add(G[0][2], G[2][0]));
    S[1][2] = S[2][1] = df_mul(mu, df_add(G[1][2], G[2][1]));
    dfl F[4][3];
#pragma unroll
    for (int b = 1; b < 4; ++b)
#pragma unroll
      for (int i2 = 0; i2 < 3; ++i2)
        F[b][i2] = df_add(df_add(df_mul(S[i2][0], g[(b - 1) * 3]), df_mul(S[i2][1], g[(b - 1) * 3 + 1])),
                          df_mul(S[i2][2], g[(b - 1) * 3 + 2]));
#pragma unroll
    for (int i2 = 0; i2 < 3; ++i2) F[0][i2] = df_neg(df_add(df_add(F[1][i2], F[2][i2]), F[3][i2]));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const dfl sum = df_add(df_add(P[0][k], P[1][k]), df_add(P[2][k], P[3][k]));
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        atomicAdd(qK + (nd[a] * 3 + k) * rpad + c, df_to(F[a][k]));
        atomicAdd(qM + (nd[a] * 3 + k) * rpad + c, df_to(df_mul(ms, df_add(P[a][k], sum))));
      }
    }
  }
}

__global__ void k_split_records(int64_t n, const double* __restrict__ rec64, float* __restrict__ rec_df) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = rec64[i];
    const float hi = (float)x;
    rec_df[2 * i] = hi;
    rec_df[2 * i + 1] = (float)(x - (double)hi);
  }
}

cudaError_t launch_split_records(int64_t E, const double* rec64, float* rec_df, cudaStream_t s) {
  k_split_records<<<grid_for(E * kRec, wide_grid_cap()), kBlock, 0, s>>>(E * kRec, rec64, rec_df);
  return cudaGetLastError();
}

cudaError_t launch_ebe_split_df(const MeshView& m, const float* rec_df, int rpad, const double* p, double* qM,
                                double* qK, cudaStream_t s) {
  const size_t bytes = sizeof(double) * (size_t)m.N * 3 * rpad;
  cudaError_t err = cudaMemsetAsync(qM, 0, bytes, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(qK, 0, bytes, s);
  if (err != cudaSuccess) return err;
  const int rs = log2i(rpad);
  k_ebe_split_df<<<grid_for(m.E << rs), kBlock, 0, s>>>(m, rec_df, rpad, rs, p, qM, qK);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------------
// Hex element matrices in FP16 on the tensor cores (variant 9; the inner FP32 solve's CG products).
// Per hex the symmetric 24 x 24 operator A_h = aM M_h + aK K_h (the six Kuhn tets summed in FP64, as for
// variant 7) in component-major DOF order (rows: x-components of corner slots 0..7, then y, then z), scaled
// by a power of two so that its largest entry lies in [2^13, 2^14), rounded to FP16.  Of its nine 8 x 8
// component blocks the six upper ones (xx, xy, xz, yy, yz, zz) are stored row-major (128 bytes each), then
// the FP32 factor 2^-scale back and padding: 784-byte records.  A tile's records, corner tables and node
// rows of p arrive by bulk copies; the tile's per-case largest |p| sets a power-of-two scale of p into FP16
// range.  A warp applies a hex to 8 cases with four mma.sync (m16n8k16 over the x and y columns, m16n8k8
// over the z columns, for output rows 0..15 and 16..23); the A fragments come from four ldmatrix, the
// lower blocks as transposes (.trans) of the stored upper ones.  With the component-major order a lane's B
// operand needs only corner slots 2tq and 2tq + 1, and its outputs are the three components of corner slot
// gq.  Sums go to the tile accumulator in the packed kernel's fixed point; p^T q is taken at the flush from
// the tile's sums and its FP32 values of p.  FP16 operands carry ~2.4e-4 of relative error into a product
// (FP32 accumulation): a refinement pass takes this product only when its reduction targets are 1e-3 or
// coarser, and the FP64 certification removes the rest.  Blocks of 256 threads (two an SM with 64-hex tiles at 8 cases, three with 32-hex tiles at 16):
// the node rows are double-buffered, the records single-buffered (the next tile's records are requested
// once the hexes of this one are done).
// ------------------------------------------------------------------------------------------------------
constexpr int kHm16Bytes = kHm16RecBytes;
constexpr int kTcBlock = 256;
static_assert(kHm16Bytes % 16 == 0 && kHm16Bytes >= 6 * 128 + 4, "six 8 x 8 FP16 blocks and the factor");

// Block (a, b) of the hex operator (corner slots a, b): B[i][k] = A[(i, a), (k, b)].
__device__ void hex_block(const double* __restrict__ rec, int64_t h, int a, int b, double aM, double aK,
                          double (&B)[3][3]) {
  constexpr int T[6][4] = {{0, 1, 2, 3}, {0, 1, 3, 4}, {0, 5, 3, 2}, {0, 5, 6, 3}, {0, 7, 4, 3}, {0, 7, 3, 6}};
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) B[i][k] = 0.0;
  for (int t = 0; t < 6; ++t) {
    int la = -1, lb = -1;
    for (int k = 0; k < 4; ++k) {
      if (T[t][k] == a) la = k;
      if (T[t][k] == b) lb = k;
    }
    if (la < 0 || lb < 0) continue;
    const double* r = rec + (h * 6 + t) * kRec;
    double ga[3], gb[3];
    for (int i = 0; i < 3; ++i) {
      ga[i] = la == 0 ? -(r[i] + r[3 + i] + r[6 + i]) : r[3 * (la - 1) + i];
      gb[i] = lb == 0 ? -(r[i] + r[3 + i] + r[6 + i]) : r[3 * (lb - 1) + i];
    }
    const double lam = aK * r[9], mu = aK * r[10], ms = aM * r[11] * (la == lb ? 2.0 : 1.0);
    const double gg = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k)
        B[i][k] += lam * ga[i] * gb[k] + mu * (gb[i] * ga[k] + (i == k ? gg : 0.0)) + (i == k ? ms : 0.0);
  }
}

// Stored component blocks (bi <= bj) in record order: xx, xy, xz, yy, yz, zz.
__host__ __device__ constexpr int cblk(int bi, int bj) { return bi == 0 ? bj : bi == 1 ? 2 + bj : 5; }

// One thread per hex: the largest entry first, then the scaled FP16 entries.
__global__ void k_hexmat16_build(int64_t H, const double* __restrict__ rec, double aM, double aK,
                                 unsigned char* __restrict__ out) {
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < H; h += (int64_t)gridDim.x * blockDim.x) {
    double mx = 0.0, B[3][3];
    for (int a = 0; a < 8; ++a)
      for (int b = a; b < 8; ++b) {
        hex_block(rec, h, a, b, aM, aK, B);
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 3; ++k) mx = fmax(mx, fabs(B[i][k]));
      }
    int e = 0;
    frexp(mx, &e);                                  // mx < 2^e
    const double sc = mx > 0.0 ? ldexp(1.0, 14 - e) : 1.0;
    __half* o = reinterpret_cast<__half*>(out + h * kHm16Bytes);
    // entry (r, c) of component block (bi, bj) is A[(bi, r), (bj, c)] = B_rc[bi][bj] with B_cr = B_rc^T
    for (int a = 0; a < 8; ++a)
      for (int b = a; b < 8; ++b) {
        hex_block(rec, h, a, b, aM, aK, B);
        for (int bi = 0; bi < 3; ++bi)
          for (int bj = bi; bj < 3; ++bj) {
            __half* blk = o + 64 * cblk(bi, bj);
            blk[8 * a + b] = __float2half_rn((float)(B[bi][bj] * sc));   // (row a, col b)
            blk[8 * b + a] = __float2half_rn((float)(B[bj][bi] * sc));   // (row b, col a) = B_ba[bi][bj]
          }
      }
    *reinterpret_cast<float*>(out + h * kHm16Bytes + 768) = mx > 0.0 ? (float)ldexp(1.0, e - 14) : 1.0f;
    for (int j = 772; j < kHm16Bytes; j += 4) *reinterpret_cast<float*>(out + h * kHm16Bytes + j) = 0.0f;
  }
}

cudaError_t launch_hexmat16_build(int64_t n_hex, const double* rec64, double aM, double aK, unsigned char* out,
                                  cudaStream_t s) {
  if (n_hex == 0) return cudaSuccess;
  k_hexmat16_build<<<grid_for(n_hex, wide_grid_cap()), kBlock, 0, s>>>(n_hex, rec64, aM, aK, out);
  return cudaGetLastError();
}

struct TcLayout {
  size_t qs, ps0, ps1, hm, loc0, loc1, node0, node1, total;
};
__host__ __device__ inline TcLayout tc_layout(int nloc_max, int rpad, int hex_per_tile) {
  auto up = [](size_t x) { return (x + 127) & ~(size_t)127; };
  TcLayout L;
  const size_t vals = up((size_t)nloc_max * 3 * rpad * sizeof(float));
  const size_t nodes = up(sizeof(int) * (size_t)nloc_max);
  const size_t locs = up((size_t)hex_per_tile * 16);
  L.qs = 1024;   // head: 2 mbarriers, per-case |p| maxima x2, back factors, dot sums
  L.ps0 = L.qs + vals;
  L.ps1 = L.ps0 + vals;
  L.hm = L.ps1 + vals;
  L.loc0 = L.hm + up((size_t)hex_per_tile * kHm16Bytes);
  L.loc1 = L.loc0 + locs;
  L.node0 = L.loc1 + locs;
  L.node1 = L.node0 + nodes;
  L.total = L.node1 + nodes;
  return L;
}

__device__ __forceinline__ void mma_f16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                              uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_f16_1688(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2t(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x1t(uint32_t addr, uint32_t& r0) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x1.trans.shared.b16 {%0}, [%1];\n" : "=r"(r0) : "r"(addr));
}
__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <bool DOT, int R>
__global__ void __launch_bounds__(kTcBlock, R == 8 ? 2 : 3) k_ebe_hex_tc(HexTiles ht, MeshView m, const float* __restrict__ p,
                                                         float* __restrict__ q, const unsigned char* __restrict__ hm,
                                                         float aM, float aK, Reducer red, CgCase* sc,
                                                         double* ptq_out, const int* gate) {
  if (gate && *gate == 0) return;
  constexpr int rpad = R, per_node = 3 * R, f4 = per_node / 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const TcLayout L = tc_layout(ht.nloc_max, R, ht.hex_per_tile);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);
  int* spm = reinterpret_cast<int*>(smem_raw + 32);          // [2][32] per-case max |p| bits, per tile parity
  float* sfwd = reinterpret_cast<float*>(smem_raw + 288);    // [32] fixed point back to FP32
  double* sdot = reinterpret_cast<double*>(smem_raw + 768);  // [32] p^T q sums of the block
  int* qs = reinterpret_cast<int*>(smem_raw + L.qs);
  unsigned char* hs = smem_raw + L.hm;
  auto psb = [&](int b) { return reinterpret_cast<float*>(smem_raw + (b ? L.ps1 : L.ps0)); };
  auto slb = [&](int b) { return reinterpret_cast<const uint32_t*>(smem_raw + (b ? L.loc1 : L.loc0)); };
  auto snb = [&](int b) { return reinterpret_cast<int*>(smem_raw + (b ? L.node1 : L.node0)); };
  constexpr uint32_t node_bytes = (uint32_t)(per_node * sizeof(float));
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < ht.nloc_max * f4; i += kTcBlock) reinterpret_cast<int4*>(qs)[i] = make_int4(0, 0, 0, 0);
  if (tid < 64) spm[tid] = 0;
  if (tid < 32) sdot[tid] = 0.0;
  __syncthreads();
  // node rows and corner tables of tile t into buffer b (bytes of the tile's records counted too: they are
  // requested by request_records once the record buffer is free)
  auto issue = [&](int t, int b) {
    const int n0 = ht.tile_node_off[t], nl = ht.tile_node_off[t + 1] - n0;
    const int h0 = ht.tile_hex_off[t], nh = ht.tile_hex_off[t + 1] - h0;
    const uint32_t bar = smem_u32(mbar + b);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
      const uint32_t lbytes = (uint32_t)(nh * 16);
      mbar_expect_tx(bar, (uint32_t)(nh * kHm16Bytes) + lbytes + (uint32_t)nl * node_bytes);
      bulk_g2s(smem_u32(slb(b)), ht.hex_local + h0, lbytes, bar);
    }
    for (int l = tid; l < nl; l += kTcBlock) {
      const int nd = ht.tile_nodes[n0 + l];
      snb(b)[l] = nd;
      bulk_g2s(smem_u32(psb(b) + l * per_node), p + (int64_t)(nd & 0x0fffffff) * per_node, node_bytes, bar);
    }
  };
  auto request_records = [&](int t, int b) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
      const int h0 = ht.tile_hex_off[t], nh = ht.tile_hex_off[t + 1] - h0;
      bulk_g2s(smem_u32(hs), hm + (int64_t)h0 * kHm16Bytes, (uint32_t)(nh * kHm16Bytes), smem_u32(mbar + b));
    }
  };
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int nwarp = kTcBlock / 32;
  const int gq = lane >> 2, tq = lane & 3;
  // ldmatrix row addresses of the lane (byte offsets in a record): x4 {xx, xy, yy, xz}, x2 {yz, zz},
  // x2.trans {xy, xz} (giving yx, zx), x1.trans {yz} (giving zy)
  const int r16 = (lane & 7) * 16;
  const uint32_t o_x4 = (uint32_t)(128 * ((lane >> 3) == 0 ? 0 : (lane >> 3) == 1 ? 1 : (lane >> 3) == 2 ? 3 : 2) + r16);
  const uint32_t o_x2 = (uint32_t)(128 * ((lane & 8) ? 5 : 4) + r16);
  const uint32_t o_t2 = (uint32_t)(128 * ((lane & 8) ? 2 : 1) + r16);
  const uint32_t o_t1 = (uint32_t)(128 * 4 + r16);
  const uint32_t hs_u32 = smem_u32(hs);
  const float bco = fabsf(aM) * ht.abs_m + fabsf(aK) * ht.abs_k;
  auto pow2 = [](int e) { return __uint_as_float((uint32_t)min(max(e + 127, 1), 254) << 23); };
  float4 tdot = make_float4(0.f, 0.f, 0.f, 0.f);
  double dd[4] = {0.0, 0.0, 0.0, 0.0};
  const int t0 = blockIdx.x;
  if (t0 < ht.n_tiles) {
    issue(t0, 0);
    request_records(t0, 0);
  }
  for (int k = 0;; ++k) {
    const int t = t0 + k * gridDim.x;
    if (t >= ht.n_tiles) break;
    const int b = k & 1;
    const int tn = t + gridDim.x;
    if (tn < ht.n_tiles) issue(tn, b ^ 1);
    const int n0 = ht.tile_node_off[t], nl = ht.tile_node_off[t + 1] - n0;
    const int h0 = ht.tile_hex_off[t], nh = ht.tile_hex_off[t + 1] - h0;
    const uint32_t bar = smem_u32(mbar + b);
    if (!mbar_wait(bar, (uint32_t)((k >> 1) & 1), g_wait_budget)) {
      atomicExch(&g_tma_timeout, 1);
      mbar_wait(bar, (uint32_t)((k >> 1) & 1));   // second bounded wait for the copies still in flight
    }
    const float* ps = psb(b);
    const uint32_t* sl = slb(b);
    const int* snode = snb(b);
    // per-case largest |p| of the staged tile (a thread's values all belong to case tid mod R)
    {
      float mx = 0.f;
      for (int i = tid; i < nl * per_node; i += kTcBlock) mx = fmaxf(mx, fabsf(ps[i]));
      for (int off = 16; off >= R; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      if (lane < R) atomicMax(spm + (b << 5) + lane, __float_as_int(mx));
    }
    __syncthreads();
    const int* spm_b = spm + (b << 5);
    // per case: E (the fixed-point bound 2^E), ep (max |p| < 2^ep); p enters FP16 as p 2^(14 - ep), sums
    // leave to fixed point by 2^(30 - E - (14 - ep))
    auto expo_b = [&](int c) {
      const uint32_t fb = (__float_as_uint(bco * __int_as_float(spm_b[c])) >> 23) & 0xffu;
      return fb == 0u ? -126 : (int)fb - 126;
    };
    auto expo_p = [&](int c) {
      const uint32_t fp = ((uint32_t)spm_b[c] >> 23) & 0xffu;
      return fp == 0u ? -126 : (int)fp - 126;
    };
    float s_in[R / 8], f_out0[R / 8], f_out1[R / 8];
#pragma unroll
    for (int nt = 0; nt < R / 8; ++nt) {
      const int cn = nt * 8 + gq, c = nt * 8 + 2 * tq;
      s_in[nt] = pow2(14 - expo_p(cn));
      f_out0[nt] = pow2(30 - expo_b(c) - 14 + expo_p(c));
      f_out1[nt] = pow2(30 - expo_b(c + 1) - 14 + expo_p(c + 1));
    }
    if (tid < R) {
      sfwd[tid] = pow2(expo_b(tid) - 30);
      spm[((b ^ 1) << 5) + tid] = 0;   // the next tile's maxima
    }
    for (int hl = warp; hl < nh; hl += nwarp) {
      const uint32_t wb = sl[4 * hl + tq], wo = sl[4 * hl + (gq >> 1)];
      const float* p0 = ps + (int)(wb & 0xffffu) * per_node;
      const float* p1 = ps + (int)(wb >> 16) * per_node;
      int* dst = qs + (int)((wo >> ((gq & 1) << 4)) & 0xffffu) * per_node;
      const uint32_t rb = hs_u32 + (uint32_t)(hl * kHm16Bytes);
      const float hu = *reinterpret_cast<const float*>(hs + hl * kHm16Bytes + 768);
      uint32_t xx, xy, yy, xz, yz, zz, yx, zx, zy;
      ldsm_x4(rb + o_x4, xx, xy, yy, xz);
      ldsm_x2(rb + o_x2, yz, zz);
      ldsm_x2t(rb + o_t2, yx, zx);
      ldsm_x1t(rb + o_t1, zy);
#pragma unroll
      for (int nt = 0; nt < R / 8; ++nt) {
        const int cn = nt * 8 + gq;   // the case of the lane's B operand
        const float s = s_in[nt];
        const uint32_t b0 = pack_f16(p0[cn] * s, p1[cn] * s);
        const uint32_t b1 = pack_f16(p0[R + cn] * s, p1[R + cn] * s);
        const uint32_t b2 = pack_f16(p0[2 * R + cn] * s, p1[2 * R + cn] * s);
        float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
        mma_f16_16816(d0, xx, yx, xy, yy, b0, b1);   // rows x, y; columns x, y
        mma_f16_1688(d0, xz, yz, b2);                // rows x, y; columns z
        mma_f16_16816(d1, zx, 0u, zy, 0u, b0, b1);   // rows z; columns x, y
        mma_f16_1688(d1, zz, 0u, b2);                // rows z; columns z
        // rows gq (x), gq + 8 (y), 16 + gq (z) of corner slot gq; columns: cases c, c + 1
        const int c = nt * 8 + 2 * tq;
        const float g0 = hu * f_out0[nt], g1 = hu * f_out1[nt];
        atomicAdd(dst + c, __float2int_rn(d0[0] * g0));
        atomicAdd(dst + c + 1, __float2int_rn(d0[1] * g1));
        atomicAdd(dst + R + c, __float2int_rn(d0[2] * g0));
        atomicAdd(dst + R + c + 1, __float2int_rn(d0[3] * g1));
        atomicAdd(dst + 2 * R + c, __float2int_rn(d1[0] * g0));
        atomicAdd(dst + 2 * R + c + 1, __float2int_rn(d1[1] * g1));
      }
    }
    __syncthreads();
    if (tn < ht.n_tiles) request_records(tn, b ^ 1);   // the record buffer is free: the next tile's records
    // flush: float4 pieces (four cases of one component of one node) to the output; p^T q from the tile's
    // sums and its FP32 values of p (a thread's four cases are fixed: 4 kTcBlock is a multiple of R)
    for (int i = tid; i < nl * f4; i += kTcBlock) {
      const int l = i / f4, kk = (i - l * f4) / (R / 4);
      const int raw = snode[l];
      const int64_t g = raw & 0x0fffffff;
      const bool fixed = !dof_free((uint8_t)((raw >> 28) & 7), kk);
      float4* dstg = reinterpret_cast<float4*>(q + g * per_node) + (i - l * f4);
      const int4 vi = reinterpret_cast<const int4*>(qs)[i];
      const int c4 = (i << 2) & (R - 1);
      const float4 v = make_float4((float)vi.x * sfwd[c4], (float)vi.y * sfwd[c4 + 1], (float)vi.z * sfwd[c4 + 2],
                                   (float)vi.w * sfwd[c4 + 3]);
      reinterpret_cast<int4*>(qs)[i] = make_int4(0, 0, 0, 0);
      if (DOT && !fixed) {
        const float4 pv = reinterpret_cast<const float4*>(ps)[i];
        tdot.x = fmaf(pv.x, v.x, tdot.x), tdot.y = fmaf(pv.y, v.y, tdot.y);
        tdot.z = fmaf(pv.z, v.z, tdot.z), tdot.w = fmaf(pv.w, v.w, tdot.w);
      }
      if (raw < 0) {
        if (!fixed) atomicAdd(dstg, v);
      } else {
        *dstg = fixed ? make_float4(0.f, 0.f, 0.f, 0.f) : v;
      }
    }
    if (DOT) {
      dd[0] += (double)tdot.x, dd[1] += (double)tdot.y, dd[2] += (double)tdot.z, dd[3] += (double)tdot.w;
      tdot = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
  }
  if (DOT) {
    const int c4 = (tid << 2) & (R - 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicAdd(sdot + c4 + j, dd[j]);
    __syncthreads();
    double v[1] = {tid < R ? sdot[tid] : 0.0};
    if (block_reduce_last<1>(v, R, red)) ebe_tail(red, sc, ptq_out, R);
  }
}

size_t ebe_hex_tc_smem(const HexTiles& ht, int rpad) {
  if (ht.hex_per_tile > 64 || (rpad != 8 && rpad != 16)) return ~(size_t)0;
  return tc_layout(ht.nloc_max, rpad, ht.hex_per_tile).total;
}

cudaError_t launch_ebe_hex_tc(const HexTiles& ht, const MeshView& m, const unsigned char* hm16, int rpad,
                              const float* p, float* q, double aM, double aK, const Reducer* red, CgCase* sc,
                              double* ptq_out, const int* gate, cudaStream_t s) {
  const size_t smem = ebe_hex_tc_smem(ht, rpad);
  if (smem == ~(size_t)0 || ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15) != 0 || m.seg)
    return cudaErrorInvalidValue;
  cudaError_t err = cudaMemsetAsync(q, 0, sizeof(float) * (size_t)m.N * 3 * rpad, s);
  if (err != cudaSuccess) return err;
  auto kfn = rpad == 8 ? (red ? k_ebe_hex_tc<true, 8> : k_ebe_hex_tc<false, 8>)
                       : (red ? k_ebe_hex_tc<true, 16> : k_ebe_hex_tc<false, 16>);
  err = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1;
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kTcBlock, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) per_sm = 1;
  int grid = sm_count() * per_sm;
  if (grid > ht.n_tiles) grid = ht.n_tiles;
  if (grid > red_grid_cap()) grid = red_grid_cap();
  Reducer rd = red ? *red : Reducer{nullptr, nullptr, nullptr};
  kfn<<<grid, kTcBlock, smem, s>>>(ht, m, p, q, hm16, (float)aM, (float)aK, rd, red ? sc : nullptr,
                                   red ? ptq_out : nullptr, gate);
  return cudaGetLastError();
}

}  // namespace fem
