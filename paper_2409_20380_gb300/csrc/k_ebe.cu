// Matrix-free element-by-element product (Section 3.2, Eq. eqebefem / eqmebefem):
//   q = sum_e P_e^T ((aM M_e + aK K_e) (P_e p))   for r cases interleaved as [node][3][r].
// One thread per (element, case): the r threads of an element read the same element record (broadcast)
// and consecutive case values of each node (coalesced), which is the block random access of the
// multi-RHS form.  Element apply in factorised form:
//   G = sum_b p_b g_b^T,  sigma = lambda tr(G) I + mu (G + G^T),  (K_e p)_a = V sigma g_a,
//   (M_e p)_a = rho V / 20 (p_a + sum_b p_b).
// This generic kernel scatters with global atomics; fixed DOFs are left to the consumer to mask.
#include "fem_internal.cuh"

namespace fem {

template <typename T> __device__ __forceinline__ const T* rec_of(const MeshView& m);
template <> __device__ __forceinline__ const double* rec_of<double>(const MeshView& m) { return m.rec64; }
template <> __device__ __forceinline__ const float* rec_of<float>(const MeshView& m) { return m.rec32; }

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
    if (block_reduce_last<1>(v, rpad, red)) {
      if (threadIdx.x < rpad) {
        const int c = threadIdx.x;
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
  }
}

static int log2i(int r) {
  int s = 0;
  while ((1 << s) < r) ++s;
  return s;
}

template <typename T>
cudaError_t launch_ebe_gated(const MeshView& m, int rpad, const T* pm, const T* pk, T* q, double aM, double aK,
                             const Reducer* red, CgCase* sc, double* ptq_out, const int* gate, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(q, 0, sizeof(T) * (size_t)m.N * 3 * rpad, s);
  if (err != cudaSuccess) return err;
  const int rs = log2i(rpad);
  const int grid = grid_for(m.E << rs);
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

}  // namespace fem
