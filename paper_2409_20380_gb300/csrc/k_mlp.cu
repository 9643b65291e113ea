// Learned proposal (the learned form of the data-driven predictor of Section 3.2): a 64 -> 256 -> 256 -> 32
// multilayer perceptron with GELU, BF16 weights and activations and FP32 accumulation on the tensor cores,
// forward and backward passes, Adam, and the kernels that tie it to the time step: input features per
// (region, case), the proposal's coefficient correction, the per-case choice between the proposal and the
// plain data-driven guess (smaller initial residual wins), and the collection of training samples.
//
// Parameter layout (FP32 master copy, also the gradient layout): W1 [256][64], b1 [256], W2 [256][256],
// b2 [256], W3 [32][256], b3 [32].  Layer l computes Z_l = A_{l-1} W_l^T + b_l, A_l = GELU(Z_l) (l < 3).
#include <cuda_bf16.h>

#include <cmath>
#include <mutex>
#include <string>

#include "fem_internal.cuh"

using namespace fem;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int kL0 = 64, kL1 = 256, kL2 = 256, kL3 = 32;
// A residual-space sample: the upper triangle of W (row by row) and w, in age order.
constexpr int kNTri = kL3 * (kL3 + 1) / 2;
constexpr int kNRes = kNTri + kL3;
static_assert(kNRes == FEM_MLP_RES, "residual sample size");
constexpr int64_t kOffW1 = 0;
constexpr int64_t kOffB1 = kOffW1 + (int64_t)kL1 * kL0;
constexpr int64_t kOffW2 = kOffB1 + kL1;
constexpr int64_t kOffB2 = kOffW2 + (int64_t)kL2 * kL1;
constexpr int64_t kOffW3 = kOffB2 + kL2;
constexpr int64_t kOffB3 = kOffW3 + (int64_t)kL3 * kL2;
constexpr int64_t kNParams = kOffB3 + kL3;
static_assert(kNParams == 90656, "parameter count of the 64-256-256-32 network");

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ------------------------------------------------------------------------------------------------------
// C = A B^T on the tensor cores.  A [M][K] and B [N][K] are BF16 with K contiguous; FP32 accumulation.
// M % 64 == 0, N % 32 == 0, K % 32 == 0, lda/ldb % 8 == 0 (16-byte rows of the staged tiles).  A CTA of
// 4 warps computes a 64 x 32 tile; warp w owns rows 16w..16w+15 and all 32 columns (4 m16n8 tiles).
// With gridDim.z > 1 (split contraction, plain epilogue only) CTA z sums its share of K and adds it into C,
// which the caller has zeroed.
// ------------------------------------------------------------------------------------------------------
enum { EPI_BIAS = 0, EPI_GELU = 1, EPI_GELU_BWD = 2, EPI_PLAIN = 3 };

struct GemmArgs {
  int M, N, K;
  const bf16* A;
  int lda;
  const bf16* B;
  int ldb;
  float* C;            // optional FP32 output C[m * c_rs + n * c_cs]
  int64_t c_rs, c_cs;
  const float* bias;   // [N] (EPI_BIAS, EPI_GELU)
  const float* zin;    // pre-activation zin[m * ldz + n] (EPI_GELU_BWD)
  int ldz;
  bf16* act;           // optional BF16 output act[m * ld_act + n]
  int ld_act;
  bf16* actT;          // optional BF16 output actT[n * ld_actT + m]
  int ld_actT;
  int m_valid;         // EPI_GELU_BWD: rows >= m_valid are written as zero
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_tn(GemmArgs g) {
  __shared__ __align__(16) bf16 As[64][40];   // 80-byte rows: 16-byte aligned, conflict-free fragment reads
  __shared__ __align__(16) bf16 Bs[32][40];
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
  float acc[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[j][e] = 0.0f;
  const int kper = g.K / (int)gridDim.z, kbeg = (int)blockIdx.z * kper;
  for (int k0 = kbeg; k0 < kbeg + kper; k0 += 32) {
#pragma unroll
    for (int v = tid; v < 256; v += 128) {
      const int r = v >> 2, cv = (v & 3) * 8;
      *reinterpret_cast<uint4*>(&As[r][cv]) =
          *reinterpret_cast<const uint4*>(g.A + (int64_t)(m0 + r) * g.lda + k0 + cv);
    }
    {
      const int r = tid >> 2, cv = (tid & 3) * 8;
      *reinterpret_cast<uint4*>(&Bs[r][cv]) =
          *reinterpret_cast<const uint4*>(g.B + (int64_t)(n0 + r) * g.ldb + k0 + cv);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      const int ar = warp * 16 + gq;
      const uint32_t a0 = *reinterpret_cast<const uint32_t*>(&As[ar][kk + tq * 2]);
      const uint32_t a1 = *reinterpret_cast<const uint32_t*>(&As[ar + 8][kk + tq * 2]);
      const uint32_t a2 = *reinterpret_cast<const uint32_t*>(&As[ar][kk + 8 + tq * 2]);
      const uint32_t a3 = *reinterpret_cast<const uint32_t*>(&As[ar + 8][kk + 8 + tq * 2]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[j * 8 + gq][kk + tq * 2]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[j * 8 + gq][kk + 8 + tq * 2]);
        mma_bf16_16816(acc[j], a0, a1, a2, a3, b0, b1);
      }
    }
    __syncthreads();
  }
  // accumulator (j, e): row gq + 8 (e >> 1) of the warp's 16, column 8 j + 2 tq + (e & 1)
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = m0 + warp * 16 + gq + 8 * (e >> 1);
      const int c = n0 + j * 8 + tq * 2 + (e & 1);
      float v = acc[j][e];
      float out = v, a = v;
      if (EPI == EPI_BIAS || EPI == EPI_GELU) {
        out = v + g.bias[c];
        a = EPI == EPI_GELU ? gelu_f(out) : out;
      } else if (EPI == EPI_GELU_BWD) {
        out = r < g.m_valid ? v * gelu_grad_f(g.zin[(int64_t)r * g.ldz + c]) : 0.0f;
        a = out;
      }
      if (g.C) {
        float* dst = g.C + (int64_t)r * g.c_rs + (int64_t)c * g.c_cs;
        if (gridDim.z > 1)
          atomicAdd(dst, out);
        else
          *dst = out;
      }
      if (g.act) g.act[(int64_t)r * g.ld_act + c] = __float2bfloat16_rn(a);
      if (g.actT) g.actT[(int64_t)c * g.ld_actT + r] = __float2bfloat16_rn(a);
    }
}

template <int EPI>
cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M % 64 || g.N % 32 || g.K % 32 || g.lda % 8 || g.ldb % 8) return cudaErrorInvalidValue;
  dim3 grid(g.M / 64, g.N / 32, 1);
  // A contraction long against the output (the weight gradients: K = the batch) is split so that the grid
  // covers the SMs twice, each share at least 8 of the 32-wide K steps; C (dense M x N) is zeroed first.
  if (EPI == EPI_PLAIN && g.C && !g.act && !g.actT &&
      ((g.c_rs == g.N && g.c_cs == 1) || (g.c_rs == 1 && g.c_cs == g.M))) {
    const int steps = g.K / 32, tiles = (int)(grid.x * grid.y), want = 2 * sm_count();
    int ks = 1;
    for (int d = 2; d <= steps / 8 && tiles * ks < want; ++d)
      if (steps % d == 0) ks = d;
    if (ks > 1) {
      cudaError_t e = cudaMemsetAsync(g.C, 0, sizeof(float) * (size_t)g.M * g.N, s);
      if (e != cudaSuccess) return e;
      grid.z = ks;
    }
  }
  k_gemm_tn<EPI><<<grid, 128, 0, s>>>(g);
  return cudaGetLastError();
}

GemmArgs gargs(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb) {
  GemmArgs g{};
  g.M = M, g.N = N, g.K = K, g.A = A, g.lda = lda, g.B = B, g.ldb = ldb;
  g.m_valid = M;
  return g;
}

// x rows (optionally gathered through idx) -> BF16 [Mpad][64] and its transpose [64][Mpad]; pad rows zero.
__global__ void k_stage(const float* __restrict__ x, const int32_t* __restrict__ idx, int64_t n_src, int64_t B,
                        int64_t Mpad, bf16* __restrict__ X0, bf16* __restrict__ X0T, int* __restrict__ bad) {
  const int64_t total = Mpad * kL0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / kL0;
    const int c = (int)(i % kL0);
    float v = 0.0f;
    if (r < B) {
      const int64_t sr = idx ? (int64_t)idx[r] : r;
      if (sr >= 0 && sr < n_src)
        v = x[sr * kL0 + c];
      else if (c == 0)
        atomicExch(bad, 1);     // sample index outside [0, n_src): the row is zero, the call reports it
    }
    const bf16 b = __float2bfloat16_rn(v);
    X0[i] = b;
    if (X0T) X0T[(int64_t)c * Mpad + r] = b;
  }
}

// dL/dout of the mean squared error, in FP32 and BF16 (row-major and transposed); pad rows zero.
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ t, const int32_t* __restrict__ idx,
                       int64_t n_src, int64_t B, int64_t Mpad, float* __restrict__ dzf, bf16* __restrict__ dzb,
                       bf16* __restrict__ dzT, double* __restrict__ loss_acc) {
  const float scale = 2.0f / ((float)B * kL3);
  double sq = 0.0;
  const int64_t total = Mpad * kL3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / kL3;
    const int j = (int)(i % kL3);
    float d = 0.0f;
    const int64_t sr = r < B ? (idx ? (int64_t)idx[r] : r) : -1;
    if (sr >= 0 && sr < n_src) {
      const float diff = out[i] - t[sr * kL3 + j];
      d = scale * diff;
      sq += (double)diff * diff;
    }
    dzf[i] = d;
    dzb[i] = __float2bfloat16_rn(d);
    dzT[(int64_t)j * Mpad + r] = __float2bfloat16_rn(d);
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0 && sq != 0.0) atomicAdd(loss_acc, sq);
}

// dL/dout of the residual-space loss, one warp per row: with the row's sample (W upper triangular, w),
// r = W d - w, loss += ||r||^2, dL/dd = 2 W^T r / B; FP32 and BF16 (row-major and transposed); pad rows zero.
__global__ void __launch_bounds__(256) k_loss_res(const float* __restrict__ out, const float* __restrict__ smp,
                                                  const int32_t* __restrict__ idx, int64_t n_src, int64_t B,
                                                  int64_t Mpad, float* __restrict__ dzf, bf16* __restrict__ dzb,
                                                  bf16* __restrict__ dzT, double* __restrict__ loss_acc) {
  __shared__ float sd[8][kL3], sr[8][kL3];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const float scale = 2.0f / (float)B;
  for (int64_t r = (int64_t)blockIdx.x * 8 + wp; r < Mpad; r += (int64_t)gridDim.x * 8) {
    const int64_t sr_ = r < B ? (idx ? (int64_t)idx[r] : r) : -1;
    const bool valid = sr_ >= 0 && sr_ < n_src;
    float g = 0.0f;
    if (valid) {
      const float* S = smp + sr_ * kNRes;
      sd[wp][lane] = out[r * kL3 + lane];
      __syncwarp();
      // r_i = sum_{j >= i} W_ij d_j - w_i  (lane i; row i of the packed triangle starts at 32 i - i (i - 1) / 2)
      const int off = lane * kL3 - lane * (lane - 1) / 2;
      float ri = -S[kNTri + lane];
      for (int j = lane; j < kL3; ++j) ri = fmaf(S[off + j - lane], sd[wp][j], ri);
      sr[wp][lane] = ri;
      double sq = (double)ri * ri;
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) atomicAdd(loss_acc, sq);
      __syncwarp();
      // g_j = scale sum_{i <= j} W_ij r_i  (lane j)
      for (int i = 0; i <= lane; ++i) g = fmaf(S[i * kL3 - i * (i - 1) / 2 + lane - i], sr[wp][i], g);
      g *= scale;
      __syncwarp();
    }
    dzf[r * kL3 + lane] = g;
    dzb[r * kL3 + lane] = __float2bfloat16_rn(g);
    dzT[(int64_t)lane * Mpad + r] = __float2bfloat16_rn(g);
  }
}

// Bias gradient: column sums of dz [Mpad][N] (fixed order: deterministic).
__global__ void k_colsum(const float* __restrict__ dz, int64_t Mpad, int N, float* __restrict__ out) {
  __shared__ float part[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + tx;
  float s = 0.0f;
  for (int64_t r = ty; r < Mpad; r += 8) s += dz[r * N + c];
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0) {
    float t = 0.0f;
    for (int k = 0; k < 8; ++k) t += part[k][tx];
    out[c] = t;
  }
}

__global__ void k_adam(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// BF16 copies of the weight matrices used by the products: W_l [N][K] and, for the backward products,
// W_l^T [K][N] (layers 2 and 3).
__global__ void k_pack(const float* __restrict__ th, bf16* W1, bf16* W2, bf16* W2T, bf16* W3, bf16* W3T) {
  const int64_t n1 = (int64_t)kL1 * kL0, n2 = (int64_t)kL2 * kL1, n3 = (int64_t)kL3 * kL2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1 + n2 + n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n1) {
      W1[i] = __float2bfloat16_rn(th[kOffW1 + i]);
    } else if (i < n1 + n2) {
      const int64_t j = i - n1, n = j / kL1, k = j % kL1;
      const bf16 b = __float2bfloat16_rn(th[kOffW2 + j]);
      W2[j] = b;
      W2T[k * kL2 + n] = b;
    } else {
      const int64_t j = i - n1 - n2, n = j / kL2, k = j % kL2;
      const bf16 b = __float2bfloat16_rn(th[kOffW3 + j]);
      W3[j] = b;
      W3T[k * kL3 + n] = b;
    }
  }
}

int grid_of(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : (g > wide_grid_cap() ? wide_grid_cap() : g));
}

}  // namespace

// ------------------------------------------------------------------------------------------------------
// The network object.
// ------------------------------------------------------------------------------------------------------
struct fem_mlp {
  int device = 0;
  cudaStream_t s = nullptr;
  float *th = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  int64_t t = 0;                       // Adam steps taken
  bf16 *W1 = nullptr, *W2 = nullptr, *W2T = nullptr, *W3 = nullptr, *W3T = nullptr;
  int64_t cap = 0;                     // rows of the activation workspace (multiple of 64)
  bf16 *X0 = nullptr, *X0T = nullptr, *A1 = nullptr, *A1T = nullptr, *A2 = nullptr, *A2T = nullptr;
  bf16 *dZ3b = nullptr, *dZ3T = nullptr, *dZ2b = nullptr, *dZ2T = nullptr, *dZ1T = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *OUT = nullptr, *dZ3f = nullptr, *dZ2f = nullptr, *dZ1f = nullptr;
  double* loss_acc = nullptr;
  int* bad = nullptr;                  // set by a kernel that met a sample index out of range
  std::mutex mu;

  void free_ws() {
    for (void* p : {(void*)X0, (void*)X0T, (void*)A1, (void*)A1T, (void*)A2, (void*)A2T, (void*)dZ3b, (void*)dZ3T,
                    (void*)dZ2b, (void*)dZ2T, (void*)dZ1T, (void*)Z1, (void*)Z2, (void*)OUT, (void*)dZ3f,
                    (void*)dZ2f, (void*)dZ1f})
      if (p) cudaFree(p);
    X0 = X0T = A1 = A1T = A2 = A2T = dZ3b = dZ3T = dZ2b = dZ2T = dZ1T = nullptr;
    Z1 = Z2 = OUT = dZ3f = dZ2f = dZ1f = nullptr;
    cap = 0;
  }
  ~fem_mlp() {
    free_ws();
    for (void* p : {(void*)th, (void*)m, (void*)v, (void*)grad, (void*)W1, (void*)W2, (void*)W2T, (void*)W3,
                    (void*)W3T, (void*)loss_acc, (void*)bad})
      if (p) cudaFree(p);
  }
};

namespace {

#define CE(x)                                 \
  do {                                        \
    cudaError_t e_ = (x);                     \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

template <typename T>
cudaError_t alloc_n(T** p, int64_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (size_t)(n > 0 ? n : 1));
}

cudaError_t ensure_cap(fem_mlp* n, int64_t rows) {
  const int64_t need = ((rows + 63) / 64) * 64;
  if (need <= n->cap) return cudaSuccess;
  // the old workspace may still be read by work queued on another stream
  CE(cudaDeviceSynchronize());
  n->free_ws();
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, int64_t k) {
    if (e == cudaSuccess) e = alloc_n(p, k);
  };
  A(&n->X0, need * kL0); A(&n->X0T, need * kL0);
  A(&n->A1, need * kL1); A(&n->A1T, need * kL1); A(&n->A2, need * kL2); A(&n->A2T, need * kL2);
  A(&n->dZ3b, need * kL3); A(&n->dZ3T, need * kL3); A(&n->dZ2b, need * kL2); A(&n->dZ2T, need * kL2);
  A(&n->dZ1T, need * kL1);
  A(&n->Z1, need * kL1); A(&n->Z2, need * kL2); A(&n->OUT, need * kL3);
  A(&n->dZ3f, need * kL3); A(&n->dZ2f, need * kL2); A(&n->dZ1f, need * kL1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    n->free_ws();
    return e;
  }
  n->cap = need;
  return cudaSuccess;
}

cudaError_t pack_weights(fem_mlp* n, cudaStream_t s) {
  k_pack<<<grid_of(90112), 256, 0, s>>>(n->th, n->W1, n->W2, n->W2T, n->W3, n->W3T);
  return cudaGetLastError();
}


// Forward over B rows of x (gathered through idx if given).  training: keep pre-activations and the
// transposed activations for the backward pass.  The output stays in n->OUT [Mpad][32].
cudaError_t forward(fem_mlp* n, const float* x, const int32_t* idx, int64_t n_src, int64_t B, bool training,
                    cudaStream_t s) {
  CE(ensure_cap(n, B));
  const int64_t Mp = ((B + 63) / 64) * 64;
  const int M = (int)Mp;
  k_stage<<<grid_of(Mp * kL0), 256, 0, s>>>(x, idx, n_src, B, Mp, n->X0, training ? n->X0T : nullptr, n->bad);
  CE(cudaGetLastError());
  GemmArgs g1 = gargs(M, kL1, kL0, n->X0, kL0, n->W1, kL0);
  g1.bias = n->th + kOffB1;
  g1.C = training ? n->Z1 : nullptr, g1.c_rs = kL1, g1.c_cs = 1;
  g1.act = n->A1, g1.ld_act = kL1;
  g1.actT = training ? n->A1T : nullptr, g1.ld_actT = M;
  CE(gemm<EPI_GELU>(g1, s));
  GemmArgs g2 = gargs(M, kL2, kL1, n->A1, kL1, n->W2, kL1);
  g2.bias = n->th + kOffB2;
  g2.C = training ? n->Z2 : nullptr, g2.c_rs = kL2, g2.c_cs = 1;
  g2.act = n->A2, g2.ld_act = kL2;
  g2.actT = training ? n->A2T : nullptr, g2.ld_actT = M;
  CE(gemm<EPI_GELU>(g2, s));
  GemmArgs g3 = gargs(M, kL3, kL2, n->A2, kL2, n->W3, kL2);
  g3.bias = n->th + kOffB3;
  g3.C = n->OUT, g3.c_rs = kL3, g3.c_cs = 1;
  CE(gemm<EPI_BIAS>(g3, s));
  return cudaSuccess;
}

// Backward of the mean squared error against t (rows gathered through idx) after forward(training):
// gradient into n->grad, sum of squared errors added to n->loss_acc.
cudaError_t backward(fem_mlp* n, const float* t, const int32_t* idx, int64_t n_src, int64_t B, cudaStream_t s,
                     bool residual = false) {
  const int64_t Mp = ((B + 63) / 64) * 64;
  const int M = (int)Mp;
  if (residual)
    k_loss_res<<<(int)std::min<int64_t>((Mp + 7) / 8, 4096), 256, 0, s>>>(n->OUT, t, idx, n_src, B, Mp, n->dZ3f,
                                                                          n->dZ3b, n->dZ3T, n->loss_acc);
  else
    k_loss<<<grid_of(Mp * kL3), 256, 0, s>>>(n->OUT, t, idx, n_src, B, Mp, n->dZ3f, n->dZ3b, n->dZ3T, n->loss_acc);
  CE(cudaGetLastError());
  // dW3 [32][256] = dZ3^T A2, computed as its transpose (256 x 32, contraction over the batch)
  GemmArgs w3 = gargs(kL2, kL3, M, n->A2T, M, n->dZ3T, M);
  w3.C = n->grad + kOffW3, w3.c_rs = 1, w3.c_cs = kL2;
  CE(gemm<EPI_PLAIN>(w3, s));
  k_colsum<<<kL3 / 32, 256, 0, s>>>(n->dZ3f, Mp, kL3, n->grad + kOffB3);
  CE(cudaGetLastError());
  // dZ2 = (dZ3 W3) * GELU'(Z2)
  GemmArgs d2 = gargs(M, kL2, kL3, n->dZ3b, kL3, n->W3T, kL3);
  d2.zin = n->Z2, d2.ldz = kL2, d2.m_valid = (int)B;
  d2.C = n->dZ2f, d2.c_rs = kL2, d2.c_cs = 1;
  d2.act = n->dZ2b, d2.ld_act = kL2;
  d2.actT = n->dZ2T, d2.ld_actT = M;
  CE(gemm<EPI_GELU_BWD>(d2, s));
  GemmArgs w2 = gargs(kL2, kL1, M, n->dZ2T, M, n->A1T, M);
  w2.C = n->grad + kOffW2, w2.c_rs = kL1, w2.c_cs = 1;
  CE(gemm<EPI_PLAIN>(w2, s));
  k_colsum<<<kL2 / 32, 256, 0, s>>>(n->dZ2f, Mp, kL2, n->grad + kOffB2);
  CE(cudaGetLastError());
  // dZ1 = (dZ2 W2) * GELU'(Z1)
  GemmArgs d1 = gargs(M, kL1, kL2, n->dZ2b, kL2, n->W2T, kL2);
  d1.zin = n->Z1, d1.ldz = kL1, d1.m_valid = (int)B;
  d1.C = n->dZ1f, d1.c_rs = kL1, d1.c_cs = 1;
  d1.actT = n->dZ1T, d1.ld_actT = M;
  CE(gemm<EPI_GELU_BWD>(d1, s));
  GemmArgs w1 = gargs(kL1, kL0, M, n->dZ1T, M, n->X0T, M);
  w1.C = n->grad + kOffW1, w1.c_rs = kL0, w1.c_cs = 1;
  CE(gemm<EPI_PLAIN>(w1, s));
  k_colsum<<<kL1 / 32, 256, 0, s>>>(n->dZ1f, Mp, kL1, n->grad + kOffB1);
  return cudaGetLastError();
}

cudaError_t adam(fem_mlp* n, double lr, cudaStream_t s) {
  n->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = (float)(1.0 - std::pow(b1, (double)n->t)), bc2 = (float)(1.0 - std::pow(b2, (double)n->t));
  k_adam<<<grid_of(kNParams), 256, 0, s>>>(n->th, n->m, n->v, n->grad, kNParams, (float)lr, (float)b1, (float)b2,
                                           1e-8f, bc1, bc2);
  CE(cudaGetLastError());
  return pack_weights(n, s);
}

// ------------------------------------------------------------------------------------------------------
// Kernels of the time step.
// ------------------------------------------------------------------------------------------------------

// Input features of row R * rpad + c: (source - centroid_R) / L, (f0 - 5) / 3, asinh of the predictor's
// coefficients in age order (newest pair first), zeros.  Pad rows up to Mpad are zero.
__global__ void k_features(PredView p, int n_pairs, const float4* __restrict__ case_src,
                           const float* __restrict__ centroid, float inv_extent, int64_t Mpad, float* __restrict__ F) {
  const int64_t rows = (int64_t)p.n_regions * p.rpad;
  const int64_t total = Mpad * kL0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / kL0;
    const int j = (int)(i % kL0);
    float v = 0.0f;
    if (row < rows) {
      const int R = (int)(row / p.rpad), c = (int)(row % p.rpad);
      if (j < 3) {
        const float4 sp = case_src[c];
        const float s3[3] = {sp.x, sp.y, sp.z};
        v = (s3[j] - centroid[R * 3 + j]) * inv_extent;
      } else if (j == 3) {
        v = case_src[c].w;
      } else if (j < 4 + n_pairs) {
        const int a = n_pairs - 1 - (j - 4);
        const double c = p.w[row * kMaxSlots + a];
        v = isfinite(c) ? (float)asinh(c) : 0.0f;     // bounded input for nearly collinear snapshots
      }
    }
    F[i] = v;
  }
}

// Coefficient correction of the proposal in slot order (column a of Y is e^{it-n+a}):  dw_a = out[n-1-a].
__global__ void k_coef_delta(int64_t rows, int n_pairs, const float* __restrict__ out, double* __restrict__ dw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * kMaxSlots;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / kMaxSlots;
    const int a = (int)(i % kMaxSlots);
    dw[i] = a < n_pairs ? (double)out[row * kL3 + (n_pairs - 1 - a)] : 0.0;
  }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// Per case: squared norm of the proposal's initial residual r0 - A dy (free DOFs); the proposal is taken
// where it is smaller than the plain guess's.  The last block updates the case's solver state.
__global__ void __launch_bounds__(kVecBlock) k_choose(MeshView m, int rpad, int rshift, const float* __restrict__ r32,
                                                      const float* __restrict__ qd, Reducer red, CgCase* outer,
                                                      int* n_active, double tol, double inner_max, double aim,
                                                      int ncase, int* __restrict__ choose,
                                                      long long* __restrict__ counts) {
  double rr = 0.0;
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!dof_free(f, k)) continue;
      const int64_t id = (n * 3 + k) * rpad + c;
      const double v = (double)r32[id] - (double)qd[id];
      rr += v * v;
    }
  }
  double vals[1] = {rr};
  if (block_reduce_last<1>(vals, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
      CgCase& s = outer[c];
      const double rrc = red.out[c];
      const bool take = c < ncase && s.status == FEM_OK && s.bb > 0.0 && isfinite(rrc) && rrc < s.rr;
      choose[c] = take ? 1 : 0;
      if (take) {
        s.rr = rrc;
        s.relres = sqrt(rrc / s.bb);
        s.relres0 = s.relres;
        s.active = rrc >= tol * tol * s.bb ? 1 : 0;
        s.inner_tol = inner_target(aim, s.relres, inner_max);
      }
      if (c < ncase && s.bb > 0.0) atomicAdd(reinterpret_cast<unsigned long long*>(counts + (take ? 0 : 1)), 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int na = 0;
      for (int c = 0; c < rpad; ++c) na += outer[c].active;
      *n_active = na;
    }
  }
}

__global__ void k_apply(int64_t n, int rpad, const int* __restrict__ choose, float* __restrict__ r32,
                        const float* __restrict__ qd, double* __restrict__ guess, const double* __restrict__ dy) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!choose[i & (rpad - 1)]) continue;
    r32[i] -= qd[i];
    guess[i] += dy[i];
  }
}

// Training samples of one step: features F (computed at prediction time) and targets c* - c in age
// order, for the real cases; rows are appended at row0 in (region, case) order.  A target with a
// non-finite entry or one above kTargetClip in magnitude is written as zero (no correction).
constexpr double kTargetClip = 100.0;

__global__ void k_collect(int n_regions, int rpad, int ncase, int n_pairs, const float* __restrict__ F,
                          const double* __restrict__ w_best, const double* __restrict__ w_pred, int64_t row0,
                          float* __restrict__ x_out, float* __restrict__ t_out) {
  const int64_t rows = (int64_t)n_regions * ncase;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * (kL0 + 1);
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / (kL0 + 1);
    const int j = (int)(i % (kL0 + 1));
    const int R = (int)(row / ncase), c = (int)(row % ncase);
    const int64_t src = (int64_t)R * rpad + c;
    if (j < kL0) {
      x_out[(row0 + row) * kL0 + j] = F[src * kL0 + j];
    } else {
      float t[kL3];
      bool ok = true;
#pragma unroll
      for (int k = 0; k < kL3; ++k) {
        double d = 0.0;
        if (k < n_pairs) {
          const int a = n_pairs - 1 - k;
          d = w_best[src * kMaxSlots + a] - w_pred[src * kMaxSlots + a];
        }
        ok = ok && isfinite(d) && fabs(d) <= kTargetClip;
        t[k] = (float)d;
      }
#pragma unroll
      for (int k = 0; k < kL3; ++k) t_out[(row0 + row) * kL3 + k] = ok ? t[k] : 0.0f;
    }
  }
}

// Per case c: ||e||^2 of the step's correction over all regions, sum_R G_R[new][new] (one block per case,
// fixed summation order).
__global__ void __launch_bounds__(256) k_case_e2(PredView p, int slot_new, double* __restrict__ e2) {
  __shared__ double part[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int R = threadIdx.x; R < p.n_regions; R += blockDim.x)
    acc += p.gram[(((int64_t)R * p.rpad + c) * kMaxSlots + slot_new) * kMaxSlots + slot_new];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) e2[c] = part[0];
}

// Residual-space training samples of one step (one warp per region and real case): the features F of the
// step's prediction, and (W, w) of the region's share ||Y_R (c + d) - e_R||^2 / ||e||^2 of the relative error
// of the case's corrected guess of the correction, from the ring Gram after e = e^it is pushed (||e||^2 of the
// whole case from k_case_e2).  In age order (index k: the pair whose output is e^{it-1-k}) the Gram of Y_R is
// factored R^T R by the same right-looking Cholesky with the column-drop rule as the predictor (pivot <=
// tau^2 G_kk drops column k: its row of R is zero); then z = R^{-T} Y_R^T e_R, W = R / ||e||,
// w = (z - R c) / ||e||.  A sample of a case with ||e|| = 0, or with a non-finite value, is zero.
__global__ void __launch_bounds__(32) k_collect_res(PredView p, const int* __restrict__ y_slots, int n, int slot_new,
                                                    double tau, int ncase, const double* __restrict__ e2case,
                                                    const float* __restrict__ F, int64_t row0,
                                                    float* __restrict__ x_out, float* __restrict__ s_out) {
  const int R = blockIdx.x / ncase, c = blockIdx.x % ncase;
  const int lane = threadIdx.x;
  constexpr int LD = kMaxSlots;
  __shared__ double L[kMaxSlots * LD];
  __shared__ double inv[kMaxSlots];
  const int64_t src = (int64_t)R * p.rpad + c;
  const int64_t row = row0 + (int64_t)R * ncase + c;
  for (int j = lane; j < kL0; j += 32) x_out[row * kL0 + j] = F[src * kL0 + j];
  const double* G = p.gram + src * kMaxSlots * kMaxSlots;
  const int yk = lane < n ? y_slots[n - 1 - lane] : 0;
  for (int i = 0; i < n; ++i) {
    const int yi = __shfl_sync(0xffffffffu, yk, i);
    if (lane < n) L[i * LD + lane] = G[yi * kMaxSlots + yk];
  }
  const double rhs = lane < n ? G[yk * kMaxSlots + slot_new] : 0.0;
  const double d0 = lane < n ? G[yk * kMaxSlots + yk] : 0.0;
  const double E = e2case[c];
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const double djj = L[j * LD + j];
    const double d0j = __shfl_sync(0xffffffffu, d0, j);
    const bool keep = d0j > 0.0 && djj > tau * tau * d0j && isfinite(djj);
    const double ip = keep ? rsqrt(djj) : 0.0;
    __syncwarp();
    if (lane > j && lane < n) L[lane * LD + j] = keep ? L[lane * LD + j] * ip : 0.0;
    if (lane == j) {
      L[j * LD + j] = keep ? djj * ip : 0.0;
      inv[j] = ip;
    }
    __syncwarp();
    if (keep && lane > j && lane < n) {   // lane i updates row i of the trailing block: L_ik -= L_ij L_kj
      const double lij = L[lane * LD + j];
      for (int k = j + 1; k <= lane; ++k) L[lane * LD + k] = fma(-lij, L[k * LD + j], L[lane * LD + k]);
    }
    __syncwarp();
  }
  double z = rhs;   // forward substitution R^T z = Y^T e (dropped columns give 0)
  for (int j = 0; j < n; ++j) {
    const double zr = __shfl_sync(0xffffffffu, z, j);
    const double zj = inv[j] != 0.0 ? zr * inv[j] : 0.0;
    if (lane == j) z = zj;
    if (lane > j && lane < n) z -= L[lane * LD + j] * zj;
  }
  const double ck = lane < n ? p.w[src * kMaxSlots + (n - 1 - lane)] : 0.0;
  double v = z;     // v_i = z_i - sum_{j >= i} R_ij c_j with R_ij = L_ji
  for (int j = 0; j < n; ++j) {
    const double cj = __shfl_sync(0xffffffffu, ck, j);
    if (lane <= j && lane < n) v -= L[j * LD + lane] * cj;
  }
  double sc = (E > 0.0 && isfinite(E)) ? rsqrt(E) : 0.0;
  if (__any_sync(0xffffffffu, !isfinite(v * sc))) sc = 0.0;
  float* so = s_out + row * kNRes;
  for (int i = 0; i < kL3; ++i) {
    const int off = i * kL3 - i * (i - 1) / 2;
    for (int j = i + lane; j < kL3; j += 32)
      so[off + j - i] = (sc != 0.0 && i < n && j < n) ? (float)(L[j * LD + i] * sc) : 0.0f;
  }
  so[kNTri + lane] = (sc != 0.0 && lane < n) ? (float)(v * sc) : 0.0f;
}

}  // namespace

// ------------------------------------------------------------------------------------------------------
// Internal entry points used by the time step.
// ------------------------------------------------------------------------------------------------------
namespace fem {

cudaError_t mlp_features(const PredView& p, int n_pairs, const float4* case_src, const float* centroid,
                         float inv_extent, float* F, cudaStream_t s) {
  const int64_t Mp = (((int64_t)p.n_regions * p.rpad + 63) / 64) * 64;
  k_features<<<grid_of(Mp * kL0), 256, 0, s>>>(p, n_pairs, case_src, centroid, inv_extent, Mp, F);
  return cudaGetLastError();
}

cudaError_t mlp_propose(fem_mlp* net, const float* F, int64_t rows, int n_pairs, double* dw, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(net->mu);
  CE(forward(net, F, nullptr, rows, rows, false, s));
  k_coef_delta<<<grid_of(rows * kMaxSlots), 256, 0, s>>>(rows, n_pairs, net->OUT, dw);
  return cudaGetLastError();
}

cudaError_t mlp_to_f32(int64_t n, const double* x, float* y, cudaStream_t s) {
  k_to_f32<<<grid_of(n), 256, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

cudaError_t mlp_choose(const MeshView& m, int rpad, const float* r32, const float* qd, Reducer red, CgCase* outer,
                       int* n_active, double tol, double inner_max, double aim, int ncase, int* choose,
                       long long* counts, cudaStream_t s) {
  int rs = 0;
  while ((1 << rs) < rpad) ++rs;
  int64_t items = m.N << rs;
  int grid = (int)((items + kVecBlock - 1) / kVecBlock);
  if (grid > vec_grid_cap()) grid = vec_grid_cap();
  if (grid < 1) grid = 1;
  k_choose<<<grid, kVecBlock, 0, s>>>(m, rpad, rs, r32, qd, red, outer, n_active, tol, inner_max, aim, ncase,
                                      choose, counts);
  return cudaGetLastError();
}

cudaError_t mlp_apply(int64_t n, int rpad, const int* choose, float* r32, const float* qd, double* guess,
                      const double* dy, cudaStream_t s) {
  k_apply<<<grid_of(n), 256, 0, s>>>(n, rpad, choose, r32, qd, guess, dy);
  return cudaGetLastError();
}

cudaError_t mlp_collect(int n_regions, int rpad, int ncase, int n_pairs, const float* F, const double* w_best,
                        const double* w_pred, int64_t row0, float* x_out, float* t_out, cudaStream_t s) {
  const int64_t rows = (int64_t)n_regions * ncase;
  k_collect<<<grid_of(rows * (kL0 + 1)), 256, 0, s>>>(n_regions, rpad, ncase, n_pairs, F, w_best, w_pred, row0,
                                                        x_out, t_out);
  return cudaGetLastError();
}

cudaError_t mlp_collect_res(const PredView& p, const int* y_slots, int n_pairs, int slot_new, double tau, int ncase,
                            const float* F, int64_t row0, float* x_out, float* s_out, double* e2, cudaStream_t s) {
  k_case_e2<<<ncase, 256, 0, s>>>(p, slot_new, e2);
  k_collect_res<<<p.n_regions * ncase, 32, 0, s>>>(p, y_slots, n_pairs, slot_new, tau, ncase, e2, F, row0, x_out,
                                                   s_out);
  return cudaGetLastError();
}

int mlp_device(const fem_mlp* n) { return n->device; }

}  // namespace fem

// ------------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------------
#define MCU(x)                                                                                 \
  do {                                                                                         \
    cudaError_t e_ = (x);                                                                      \
    if (e_ != cudaSuccess) {                                                                   \
      cudaGetLastError();                                                                      \
      return set_error(FEM_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_));           \
    }                                                                                          \
  } while (0)

extern "C" {

fem_status fem_mlp_create(const float* params, void* stream, fem_mlp** out) {
  if (!params || !out) return set_error(FEM_ERR_ARG, "fem_mlp_create: null argument");
  *out = nullptr;
  fem_mlp* n = new fem_mlp();
  n->s = (cudaStream_t)stream;
  cudaGetDevice(&n->device);
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, int64_t k) {
    if (e == cudaSuccess) e = alloc_n(p, k);
  };
  A(&n->th, kNParams); A(&n->m, kNParams); A(&n->v, kNParams); A(&n->grad, kNParams);
  A(&n->W1, (int64_t)kL1 * kL0); A(&n->W2, (int64_t)kL2 * kL1); A(&n->W2T, (int64_t)kL2 * kL1);
  A(&n->W3, (int64_t)kL3 * kL2); A(&n->W3T, (int64_t)kL3 * kL2); A(&n->loss_acc, 1); A(&n->bad, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete n;
    return set_error(FEM_ERR_OOM, "fem_mlp_create: device allocation failed");
  }
  e = cudaMemcpyAsync(n->th, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, n->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, sizeof(float) * kNParams, n->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, sizeof(float) * kNParams, n->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->bad, 0, sizeof(int), n->s);
  if (e == cudaSuccess) e = pack_weights(n, n->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete n;
    return set_error(FEM_ERR_CUDA, std::string("fem_mlp_create: ") + cudaGetErrorString(e));
  }
  *out = n;
  return FEM_OK;
}

fem_status fem_mlp_destroy(fem_mlp* n) {
  if (!n) return FEM_OK;
  cudaStreamSynchronize(n->s);
  delete n;
  return FEM_OK;
}

fem_status fem_mlp_get_params(fem_mlp* n, float* params) {
  if (!n || !params) return set_error(FEM_ERR_ARG, "fem_mlp_get_params: null argument");
  MCU(cudaMemcpyAsync(params, n->th, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, n->s));
  MCU(cudaStreamSynchronize(n->s));
  return FEM_OK;
}

fem_status fem_mlp_forward(fem_mlp* n, const float* x_dev, int64_t B, float* out_dev) {
  if (!n || (B > 0 && (!x_dev || !out_dev)) || B < 0) return set_error(FEM_ERR_ARG, "fem_mlp_forward: bad argument");
  if (B == 0) return FEM_OK;
  std::lock_guard<std::mutex> lk(n->mu);
  MCU(forward(n, x_dev, nullptr, B, B, false, n->s));
  MCU(cudaMemcpyAsync(out_dev, n->OUT, sizeof(float) * kL3 * B, cudaMemcpyDeviceToDevice, n->s));
  return FEM_OK;
}


static fem_status mlp_loss_grad_any(fem_mlp* n, const float* x_dev, const float* t_dev, int64_t B, float* grad_dev,
                                    double* loss_out, bool residual) {
  clear_error();
  if (!n || !x_dev || !t_dev || B <= 0) return set_error(FEM_ERR_ARG, "fem_mlp_loss_grad: bad argument");
  std::lock_guard<std::mutex> lk(n->mu);
  MCU(cudaMemsetAsync(n->loss_acc, 0, sizeof(double), n->s));
  MCU(forward(n, x_dev, nullptr, B, B, true, n->s));
  MCU(backward(n, t_dev, nullptr, B, B, n->s, residual));
  if (grad_dev) MCU(cudaMemcpyAsync(grad_dev, n->grad, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, n->s));
  double acc = 0.0;
  MCU(cudaMemcpyAsync(&acc, n->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, n->s));
  MCU(cudaStreamSynchronize(n->s));
  if (loss_out) *loss_out = residual ? acc / (double)B : acc / ((double)B * kL3);
  return FEM_OK;
}

static fem_status mlp_train_any(fem_mlp* n, const float* x_dev, const float* t_dev, int64_t n_samples,
                                const int32_t* order_dev, int n_updates, int batch, double lr, double* loss_out,
                                bool residual) {
  clear_error();
  if (!n || !x_dev || !t_dev || !order_dev || n_samples <= 0 || n_updates < 0 || batch <= 0 || !(lr > 0.0))
    return set_error(FEM_ERR_ARG, "fem_mlp_train: bad argument");
  std::lock_guard<std::mutex> lk(n->mu);
  MCU(cudaMemsetAsync(n->bad, 0, sizeof(int), n->s));
  for (int u = 0; u < n_updates; ++u) {
    const int32_t* idx = order_dev + (int64_t)u * batch;
    if (loss_out) MCU(cudaMemsetAsync(n->loss_acc, 0, sizeof(double), n->s));
    MCU(forward(n, x_dev, idx, n_samples, batch, true, n->s));
    MCU(backward(n, t_dev, idx, n_samples, batch, n->s, residual));
    if (loss_out) {
      double acc = 0.0;
      MCU(cudaMemcpyAsync(&acc, n->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, n->s));
      MCU(cudaStreamSynchronize(n->s));
      loss_out[u] = residual ? acc / (double)batch : acc / ((double)batch * kL3);
    }
    MCU(adam(n, lr, n->s));
  }
  int bad = 0;
  MCU(cudaMemcpyAsync(&bad, n->bad, sizeof(int), cudaMemcpyDeviceToHost, n->s));
  MCU(cudaStreamSynchronize(n->s));
  if (bad) return set_error(FEM_ERR_ARG, "fem_mlp_train: a sample index was outside [0, n_samples)");
  return FEM_OK;
}

fem_status fem_mlp_loss_grad(fem_mlp* n, const float* x_dev, const float* t_dev, int64_t B, float* grad_dev,
                             double* loss_out) {
  return mlp_loss_grad_any(n, x_dev, t_dev, B, grad_dev, loss_out, false);
}

fem_status fem_mlp_loss_grad_residual(fem_mlp* n, const float* x_dev, const float* s_dev, int64_t B, float* grad_dev,
                                      double* loss_out) {
  return mlp_loss_grad_any(n, x_dev, s_dev, B, grad_dev, loss_out, true);
}

fem_status fem_mlp_train(fem_mlp* n, const float* x_dev, const float* t_dev, int64_t n_samples,
                         const int32_t* order_dev, int n_updates, int batch, double lr, double* loss_out) {
  return mlp_train_any(n, x_dev, t_dev, n_samples, order_dev, n_updates, batch, lr, loss_out, false);
}

fem_status fem_mlp_train_residual(fem_mlp* n, const float* x_dev, const float* s_dev, int64_t n_samples,
                                  const int32_t* order_dev, int n_updates, int batch, double lr, double* loss_out) {
  return mlp_train_any(n, x_dev, s_dev, n_samples, order_dev, n_updates, batch, lr, loss_out, true);
}

}  // extern "C"
