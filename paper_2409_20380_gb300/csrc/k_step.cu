// Time-stepping kernels (Section 3.1, Eq. GE:DIS and Eq. timestep, in increment form) and the
// predictors of Section 3.2: Adams-Bashforth 4 and the regional data-driven correction.
// All vectors are [N][3][rpad] FP64 unless stated.
#include "fem_internal.cuh"

#include <type_traits>

namespace fem {

// Snapshot storage: FP64, FP32, double-float pairs (hi, lo FP32 with hi + lo = e to 2^-48 relative; the
// same 8 bytes as FP64, read and combined on the FP32 pipe), or SnapHL: the FP32 value and its residual
// rounded to BF16 in two planes of one slot (6 bytes a value, e to about 2^-32 relative, read as a
// double-float pair).  A slot holds `stride` values (a multiple of 8, so both planes start on 16 bytes);
// slot j starts snap_bytes<E> * stride * j bytes into the ring.
struct SnapHL {
  float h;
};
template <typename E> struct SnapVal { typedef E V; };
template <> struct SnapVal<SnapHL> { typedef float2 V; };
template <typename E> constexpr int snap_bytes() { return (int)sizeof(E); }
template <> constexpr int snap_bytes<SnapHL>() { return 6; }

__device__ __forceinline__ uint16_t f2bf_rn(float x) {   // round to nearest even (finite inputs)
  const uint32_t u = __float_as_uint(x);
  return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ void store_snap(double* p, int64_t, int64_t i, double v) { p[i] = v; }
__device__ __forceinline__ void store_snap(float* p, int64_t, int64_t i, double v) { p[i] = (float)v; }
__device__ __forceinline__ void store_snap(float2* p, int64_t, int64_t i, double v) { p[i] = d2df(v); }
__device__ __forceinline__ void store_snap(SnapHL* p, int64_t stride, int64_t i, double v) {
  const float2 hl = d2df(v);
  reinterpret_cast<float*>(p)[i] = hl.x;
  reinterpret_cast<uint16_t*>(reinterpret_cast<float*>(p) + stride)[i] = f2bf_rn(hl.y);
}
// Values i and i + 1 (i even) stored with one vector access per plane.
__device__ __forceinline__ void store_snap2(double* p, int64_t, int64_t i, double v0, double v1) {
  *reinterpret_cast<double2*>(p + i) = make_double2(v0, v1);
}
__device__ __forceinline__ void store_snap2(float* p, int64_t, int64_t i, double v0, double v1) {
  *reinterpret_cast<float2*>(p + i) = make_float2((float)v0, (float)v1);
}
__device__ __forceinline__ void store_snap2(float2* p, int64_t, int64_t i, double v0, double v1) {
  const float2 a = d2df(v0), b = d2df(v1);
  *reinterpret_cast<float4*>(p + i) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store_snap2(SnapHL* p, int64_t stride, int64_t i, double v0, double v1) {
  const float2 a = d2df(v0), b = d2df(v1);
  float* h = reinterpret_cast<float*>(p);
  *reinterpret_cast<float2*>(h + i) = make_float2(a.x, b.x);
  *reinterpret_cast<uint32_t*>(reinterpret_cast<uint16_t*>(h + stride) + i) =
      (uint32_t)f2bf_rn(a.y) | ((uint32_t)f2bf_rn(b.y) << 16);
}
template <typename E>
__device__ __forceinline__ typename SnapVal<E>::V load_snap(const E* p, int64_t, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ float2 load_snap<SnapHL>(const SnapHL* p, int64_t stride, int64_t i) {
  const float* h = reinterpret_cast<const float*>(p);
  return make_float2(h[i], bf2f(reinterpret_cast<const uint16_t*>(h + stride)[i]));
}
// Values i and i + 1 of a slot (i even) in one vector access per plane.
__device__ __forceinline__ void load_snap2(const double* p, int64_t, int64_t i, double& a, double& b) {
  const double2 t = *reinterpret_cast<const double2*>(p + i);
  a = t.x, b = t.y;
}
__device__ __forceinline__ void load_snap2(const float* p, int64_t, int64_t i, float& a, float& b) {
  const float2 t = *reinterpret_cast<const float2*>(p + i);
  a = t.x, b = t.y;
}
__device__ __forceinline__ void load_snap2(const float2* p, int64_t, int64_t i, float2& a, float2& b) {
  const float4 t = *reinterpret_cast<const float4*>(p + i);
  a = make_float2(t.x, t.y), b = make_float2(t.z, t.w);
}
__device__ __forceinline__ void load_snap2(const SnapHL* p, int64_t stride, int64_t i, float2& a, float2& b) {
  const float* h = reinterpret_cast<const float*>(p);
  const float2 hh = *reinterpret_cast<const float2*>(h + i);
  const uint32_t l = *reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint16_t*>(h + stride) + i);
  a = make_float2(hh.x, bf2f((uint16_t)(l & 0xffffu))), b = make_float2(hh.y, bf2f((uint16_t)(l >> 16)));
}
template <typename E> __device__ __forceinline__ E* snap_slot(E* ring, int64_t slot, int64_t stride) {
  return reinterpret_cast<E*>(reinterpret_cast<char*>(ring) + slot * stride * snap_bytes<E>());
}
template <typename E> __device__ __forceinline__ const E* snap_slot(const E* ring, int64_t slot, int64_t stride) {
  return reinterpret_cast<const E*>(reinterpret_cast<const char*>(ring) + slot * stride * snap_bytes<E>());
}


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

// Inputs of the fused right-hand-side EBE:  b = f + M m_in + K k_in  with
//   m_in = a + (4/dt + a0) v,  k_in = a1 v - u
// which equals f - K u + C v + M (a + 4/dt v) for C = a0 M + a1 K.
__global__ void k_rhs_prep(int64_t n, double c_mv, double a1, const double* __restrict__ u,
                           const double* __restrict__ v, const double* __restrict__ a, double* __restrict__ m_in,
                           double* __restrict__ k_in) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double vv = v[i];
    m_in[i] = a[i] + c_mv * vv;
    k_in[i] = a1 * vv - u[i];
  }
}

// Adds the Ricker point forces at time t and zeroes Dirichlet DOFs.
__global__ void k_rhs_finish(MeshView m, int rpad, int rshift, double* __restrict__ b, const RickerSrc* __restrict__ src,
                             const double* __restrict__ ext, double t) {
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
    const RickerSrc s = src[c];
    double fv[3] = {0.0, 0.0, 0.0};
    if (s.node == n) {
      if (ext) {
        for (int k = 0; k < 3; ++k) fv[k] = ext[c * 3 + k];
      } else {
        const double arg = (M_PI * s.f0 * (t - s.t0)) * (M_PI * s.f0 * (t - s.t0));
        const double w = s.amp * (1.0 - 2.0 * arg) * exp(-arg);
        for (int k = 0; k < 3; ++k) fv[k] = w * s.dir[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t id = (n * 3 + k) * rpad + c;
      b[id] = dof_free(f, k) ? b[id] + fv[k] : 0.0;
    }
  }
}

// du_AB = dt/24 (-9 v^{it-4} + 37 v^{it-3} - 59 v^{it-2} + 55 v^{it-1})   (Section 3.2)
// Weights times h (four FMAs a value: the FP64 pipe bounds this kernel), two values a thread by 16-byte
// accesses, then the odd last one.
__device__ __forceinline__ void ab4_body(int64_t n, double h, const double* __restrict__ v4,
                                         const double* __restrict__ v3, const double* __restrict__ v2,
                                         const double* __restrict__ v1, double* __restrict__ out) {
  const double w4 = -9.0 * h, w3 = 37.0 * h, w2 = -59.0 * h, w1 = 55.0 * h;
  auto ld = [](const double* x, int64_t i) { return *reinterpret_cast<const double2*>(x + i); };
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (n >> 1); t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 2 * t;
    const double2 a4 = ld(v4, i), a3 = ld(v3, i), a2 = ld(v2, i), a1 = ld(v1, i);
    *reinterpret_cast<double2*>(out + i) = make_double2(fma(w1, a1.x, fma(w2, a2.x, fma(w3, a3.x, w4 * a4.x))),
                                                        fma(w1, a1.y, fma(w2, a2.y, fma(w3, a3.y, w4 * a4.y))));
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    out[i] = fma(w1, v1[i], fma(w2, v2[i], fma(w3, v3[i], w4 * v4[i])));
  }
}

__global__ void k_ab4(int64_t n, double h, const double* __restrict__ v4, const double* __restrict__ v3,
                      const double* __restrict__ v2, const double* __restrict__ v1, double* __restrict__ out) {
  ab4_body(n, h, v4, v3, v2, v1, out);
}

// (ahead 1: for the step after the one the record holds, from the tail of the step graph or before it)
__global__ void k_ab4_ring(int64_t n, double h, Ring4 v, const StepCtl* __restrict__ ctl, double* __restrict__ out,
                           int ahead) {
  const int it = ctl->it + ahead;   // v^{it-4} .. v^{it-1} sit in slots it, it+1, it+2, it+3 (mod 4)
  ab4_body(n, h, v.p[it & 3], v.p[(it + 1) & 3], v.p[(it + 2) & 3], v.p[(it + 3) & 3], out);
}

__global__ void k_add(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = a[i] + b[i];
}

// u += du;  v^it = 2/dt du - v^{it-1};  a^it = 4/dt^2 du - 4/dt v^{it-1} - a^{it-1};
// snapshot e^it = du - du_AB (= u^it - u_AB^it).   v_prev and v_push may not alias.
template <typename E>
__global__ void k_newmark(int64_t n, double dt, const double* __restrict__ du, const double* __restrict__ du_ab,
                          double* __restrict__ u, const double* __restrict__ v_prev, double* __restrict__ a,
                          double* __restrict__ v_push, E* __restrict__ e_push, int64_t stride) {
  const double c2 = 2.0 / dt, c4 = 4.0 / dt, c44 = 4.0 / (dt * dt);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = du[i];
    const double vp = v_prev[i];
    u[i] += d;
    v_push[i] = c2 * d - vp;
    a[i] = c44 * d - c4 * vp - a[i];
    if (e_push) store_snap(e_push, stride, i, d - du_ab[i]);
  }
}

// ---- data-driven predictor ----
// Ring slot j of a group holds a past correction e (same layout as the state vectors).  Per region R
// (node range) and case c the Gram of stored corrections gram[R][c][i][j] = e_i . e_j is kept up to date
// by computing, after each push, the dots of the newest slot with every valid slot.

template <typename T> struct PredAcc;
template <> struct PredAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
};
template <> struct PredAcc<float2> {  // double-float: exact products by FMA, exact hi sums by two-sum
  float s = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    l = __fadd_rn(l, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double get() const { return f2d(s) + f2d(l); }
};
template <> struct PredAcc<float> {   // compensated FP32 summation of FP32 products
  float s = 0.f, comp = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float y = a * b - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)comp; }
};

// Partial sums carried through the block reduction: FP64 for FP64 / FP32 snapshots, (hi, lo) FP32 pairs for
// double-float snapshots (no FP64 conversion until one value per slot and case remains).
template <typename T> struct RedVal {
  double v;
  __device__ __forceinline__ static RedVal from(const PredAcc<T>& a) { return RedVal{a.get()}; }
  __device__ __forceinline__ void add(const RedVal& o) { v += o.v; }
  __device__ __forceinline__ RedVal shfl_xor(int off) const { return RedVal{__shfl_xor_sync(0xffffffffu, v, off)}; }
  __device__ __forceinline__ double get() const { return v; }
};
template <> struct RedVal<float2> {
  float h, l;
  __device__ __forceinline__ static RedVal from(const PredAcc<float2>& a) { return RedVal{a.s, a.l}; }
  __device__ __forceinline__ void add(const RedVal& o) {   // two-sum of the high words, low words added
    const float t = __fadd_rn(h, o.h);
    const float bb = __fsub_rn(t, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bb)), __fsub_rn(o.h, bb));
    h = t;
    l = __fadd_rn(__fadd_rn(l, o.l), err);
  }
  __device__ __forceinline__ RedVal shfl_xor(int off) const {
    return RedVal{__shfl_xor_sync(0xffffffffu, h, off), __shfl_xor_sync(0xffffffffu, l, off)};
  }
  __device__ __forceinline__ double get() const { return f2d(h) + f2d(l); }
};

// Region R is split into p.n_chunks node ranges; block (R, k, g) accumulates, for each valid slot j of its
// group g of kDotGrp slots, the partial dot of slot j with the newest slot over its range, per case:
// dpart[R][k][j][c].  Six slots a block (measured on the medium workload: 350 us a Gram row, against 412 us
// with 11 and 635 us with 17 slots a block: fewer ring streams at once per SM read faster).
constexpr int kDotGrp = 6;
constexpr int kDotGroups = (kMaxSlots + kDotGrp - 1) / kDotGrp;
template <typename E>
__global__ void __launch_bounds__(kBlock, 3) k_pred_dots(PredView p, int slot_new, uint64_t valid_mask,
                                                         const StepCtl* ctl) {
  typedef typename SnapVal<E>::V T;
  if (ctl) slot_new = ctl->slot_new, valid_mask = ctl->mask;
  const int rk = blockIdx.x / kDotGroups;   // the slot groups of one chunk are neighbours in the launch order,
  const int R = rk / p.n_chunks, k = rk % p.n_chunks;   // so their reads of the new slot's chunk share L2
  const int j0 = (blockIdx.x % kDotGroups) * kDotGrp;
  // a group with no stored slot (the ring holds s + 1 <= kMaxSlots slots) has nothing to add
  if (((valid_mask >> j0) & ((1ull << kDotGrp) - 1ull)) == 0ull) return;
  const int64_t lo = p.reg_lo[R], hi = p.reg_hi[R];
  const int64_t len = (hi - lo + p.n_chunks - 1) / p.n_chunks;
  const int64_t c_lo = lo + k * len, c_hi = c_lo + len < hi ? c_lo + len : hi;
  const int rpad = p.rpad;
  const E* ring = (const E*)p.ring;
  const int64_t st = p.slot_stride;
  const E* xn = snap_slot(ring, slot_new, st);
  const int64_t base = c_lo * 3 * rpad, cnt = c_hi > c_lo ? (c_hi - c_lo) * 3 * rpad : 0;
  __shared__ RedVal<T> sh[kBlock / 32][kDotGrp][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* out = p.dpart + ((int64_t)R * p.n_chunks + k) * kMaxSlots * rpad;
  if (std::is_same<E, SnapHL>::value && rpad >= 2) {
    // FP32 + BF16 snapshots: two consecutive values a thread (cases c, c + 1), so the two residual words
    // come in one 32-bit load (one value a thread, 2-byte loads, measured 3x slower); for the 8-byte
    // formats one value a thread is faster (350 us a Gram row against 578 us)
    PredAcc<T> acc0[kDotGrp], acc1[kDotGrp];
    for (int64_t i = 2 * (int64_t)threadIdx.x; i < cnt; i += 2 * (int64_t)blockDim.x) {
      T x0, x1;
      load_snap2(xn, st, base + i, x0, x1);
#pragma unroll
      for (int jj = 0; jj < kDotGrp; ++jj) {
        const int j = j0 + jj;
        if (j < kMaxSlots && ((valid_mask >> j) & 1ull)) {
          T y0, y1;
          load_snap2(snap_slot(ring, j, st), st, base + i, y0, y1);
          acc0[jj].add(y0, x0);
          acc1[jj].add(y1, x1);
        }
      }
    }
#pragma unroll
    for (int jj = 0; jj < kDotGrp; ++jj) {   // lanes holding the same case pair are rpad / 2 apart
      RedVal<T> v0 = RedVal<T>::from(acc0[jj]), v1 = RedVal<T>::from(acc1[jj]);
      for (int off = 16; off >= (rpad >> 1); off >>= 1) v0.add(v0.shfl_xor(off)), v1.add(v1.shfl_xor(off));
      if (lane < (rpad >> 1)) sh[warp][jj][2 * lane] = v0, sh[warp][jj][2 * lane + 1] = v1;
    }
  } else {
    PredAcc<T> acc[kDotGrp];
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      const T x = load_snap(xn, st, base + i);
#pragma unroll
      for (int jj = 0; jj < kDotGrp; ++jj) {
        const int j = j0 + jj;
        if (j < kMaxSlots && ((valid_mask >> j) & 1ull)) acc[jj].add(load_snap(snap_slot(ring, j, st), st, base + i), x);
      }
    }
#pragma unroll
    for (int jj = 0; jj < kDotGrp; ++jj) {
      RedVal<T> v = RedVal<T>::from(acc[jj]);
      for (int off = 16; off >= rpad; off >>= 1) v.add(v.shfl_xor(off));
      if (lane < rpad) sh[warp][jj][lane] = v;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kDotGrp * rpad; t += blockDim.x) {
    const int jj = t / rpad, c = t % rpad, j = j0 + jj;
    if (j < kMaxSlots && ((valid_mask >> j) & 1ull)) {
      RedVal<T> sum = sh[0][jj][c];
      for (int w = 1; w < nw; ++w) sum.add(sh[w][jj][c]);
      out[j * rpad + c] = sum.get();
    }
  }
}

// Sums the chunk partials in chunk order and writes row/column slot_new of each (region, case) Gram.
__global__ void k_pred_dots_finish(PredView p, int slot_new, uint64_t valid_mask, const StepCtl* ctl) {
  if (ctl) slot_new = ctl->slot_new, valid_mask = ctl->mask;
  const int R = blockIdx.x;
  for (int t = threadIdx.x; t < kMaxSlots * p.rpad; t += blockDim.x) {
    const int j = t / p.rpad, c = t % p.rpad;
    if (!((valid_mask >> j) & 1ull)) continue;
    double s = 0.0;
    for (int k = 0; k < p.n_chunks; ++k) s += p.dpart[(((int64_t)R * p.n_chunks + k) * kMaxSlots + j) * p.rpad + c];
    double* G = p.gram + ((int64_t)R * p.rpad + c) * kMaxSlots * kMaxSlots;
    G[slot_new * kMaxSlots + j] = s;
    G[j * kMaxSlots + slot_new] = s;
  }
}

// Per (region, case): least-squares coefficients w of the query (newest slot) on the X slots, by a
// pivot-free Cholesky of the Gram with the column-drop rule  pivot <= tau^2 G_jj  (the squared form of
// the modified Gram-Schmidt test ||v_j|| <= tau ||x_j||), then forward/back substitution.  One warp per
// system: the trailing updates of the factorisation are spread over the lanes (the FP64 pipe is the limit,
// so no lane idles through a column), the pivots are kept as reciprocals so the substitutions (lane i owns
// row i) multiply; rows padded to an odd length of doubles to spread shared-memory banks.
__global__ void k_pred_solve(PredView p, const int* __restrict__ x_slots, int n, int slot_new, double tau,
                             const StepCtl* ctl) {
  if (ctl) x_slots = ctl->xs, n = ctl->n_pairs, slot_new = ctl->slot_query;
  const int R = blockIdx.x / p.rpad, c = blockIdx.x % p.rpad;
  const int lane = threadIdx.x;
  constexpr int LD = kMaxSlots;                 // 33 doubles per row
  __shared__ double L[kMaxSlots * LD];
  __shared__ double inv[kMaxSlots];             // 1 / pivot, 0 for a dropped column
  __shared__ unsigned short tab[kMaxSlots * (kMaxSlots + 1) / 2];
  const double* G = p.gram + ((int64_t)R * p.rpad + c) * kMaxSlots * kMaxSlots;
  const int xi = lane < n ? x_slots[lane] : 0;
  for (int i = 0; i < n; ++i) {
    const int xs_i = __shfl_sync(0xffffffffu, xi, i);
    if (lane < n) L[i * LD + lane] = G[xs_i * kMaxSlots + xi];
  }
  // lower-triangle entries (i, k), k descending: the trailing block of column j is the prefix of length
  // (n - 1 - j)(n - j) / 2 (all entries with k > j)
  if (lane < n) {
    const int off = (n - 1 - lane) * (n - lane) / 2;
    for (int i = lane; i < n; ++i) tab[off + i - lane] = (unsigned short)((i << 8) | lane);
  }
  double rhs = lane < n ? G[xi * kMaxSlots + slot_new] : 0.0;
  const double d0 = lane < n ? G[xi * kMaxSlots + xi] : 0.0;
  __syncwarp();
  // right-looking Cholesky: column j scaled by 1 / pivot, then the trailing block updated with its
  // entries spread over the lanes (each entry still receives its updates in column order)
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
    if (keep) {
      const int T = (n - 1 - j) * (n - j) / 2;
      for (int t = lane; t < T; t += 32) {
        const int e = tab[t], i = e >> 8, k = e & 255;
        L[i * LD + k] = fma(-L[i * LD + j], L[k * LD + j], L[i * LD + k]);
      }
    }
    __syncwarp();
  }
  // forward substitution L y = rhs (column sweep), dropped columns give 0
  double y = rhs;
  for (int j = 0; j < n; ++j) {
    const double yj_raw = __shfl_sync(0xffffffffu, y, j);
    const double ij = inv[j];
    const double yj = ij != 0.0 ? yj_raw * ij : 0.0;
    if (lane == j) y = yj;
    if (lane > j && lane < n) y -= L[lane * LD + j] * yj;
  }
  // back substitution L^T w = y (row sweep from the bottom)
  double w = y;
  for (int j = n - 1; j >= 0; --j) {
    const double wj_raw = __shfl_sync(0xffffffffu, w, j);
    const double ij = inv[j];
    const double wj = ij != 0.0 ? wj_raw * ij : 0.0;
    if (lane == j) w = wj;
    if (lane < j) w -= L[j * LD + lane] * wj;
  }
  double* wo = p.w + ((int64_t)R * p.rpad + c) * kMaxSlots;
  wo[lane] = lane < n ? w : 0.0;
  if (lane == 0) wo[32] = 0.0;
}

// Accumulation of w * y for the combination kernels: FP64, FP32, or double-float (coefficients split into
// (hi, lo) pairs; products exact by FMA, hi sums exact by two-sum) for double-float snapshots.
template <typename T> struct CombAcc;
template <> struct CombAcc<double> {
  typedef double W;
  double s = 0.0;
  __device__ __forceinline__ static W wconv(double w) { return w; }
  __device__ __forceinline__ void add(W w, double y) { s = fma(w, y, s); }
  __device__ __forceinline__ void merge(const CombAcc& o) { s += o.s; }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ float getf() const { return d2f(s); }
};
template <> struct CombAcc<float> {
  typedef float W;
  float s = 0.f;
  __device__ __forceinline__ static W wconv(double w) { return (float)w; }
  __device__ __forceinline__ void add(W w, float y) { s = fmaf(w, y, s); }
  __device__ __forceinline__ void merge(const CombAcc& o) { s += o.s; }
  __device__ __forceinline__ double get() const { return (double)s; }
  __device__ __forceinline__ float getf() const { return s; }
};
template <> struct CombAcc<float2> {
  typedef float2 W;
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ static W wconv(double w) { return d2df(w); }
  __device__ __forceinline__ void add(W w, float2 y) {
    const float p = __fmul_rn(w.x, y.x);
    float e = __fmaf_rn(w.x, y.x, -p);
    e = __fmaf_rn(w.x, y.y, e);
    e = __fmaf_rn(w.y, y.x, e);
    const float t = __fadd_rn(h, p);
    const float bb = __fsub_rn(t, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    h = t;
    l = __fadd_rn(l, __fadd_rn(err, e));
  }
  __device__ __forceinline__ void merge(const CombAcc& o) {
    const float t = __fadd_rn(h, o.h);
    const float bb = __fsub_rn(t, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bb)), __fsub_rn(o.h, bb));
    h = t;
    l = __fadd_rn(__fadd_rn(l, o.l), err);
  }
  __device__ __forceinline__ double get() const { return f2d(h) + f2d(l); }
  __device__ __forceinline__ float getf() const { return __fadd_rn(h, l); }
};

// y_out += Y w over the region's node range: the coefficients [a][case] and slot offsets in shared memory.
// With y_base: y_out = y_base + Y w and corr32 = Y w in FP32 (the correction the guess's residual needs),
// and outside every region range y_out = y_base, corr32 = 0: the last chunk of region R also covers the
// nodes from its range's end to gap_hi[R] (the next range's start), block 0 the nodes before lead_hi.
// y_out2 (optional, with y_base) receives a second copy of y_out: the solver's starting iterate.
template <typename E>
__global__ void __launch_bounds__(kBlock, 5) k_pred_combine(PredView p, const int* __restrict__ y_slots, int n,
                                                         double* __restrict__ y_out, const double* __restrict__ y_base,
                                                         float* __restrict__ corr32, const int32_t* __restrict__ gap_hi,
                                                         int lead_hi, const StepCtl* ctl, double* __restrict__ y_out2) {
  if (ctl) y_slots = ctl->ys, n = ctl->n_pairs;
  typedef typename SnapVal<E>::V T;
  typedef typename CombAcc<T>::W W;
  const int R = blockIdx.x / p.n_chunks, k = blockIdx.x % p.n_chunks;
  const int64_t lo = p.reg_lo[R], hi = p.reg_hi[R];
  const int64_t len = (hi - lo + p.n_chunks - 1) / p.n_chunks;
  const int64_t c_lo = lo + k * len, c_hi = c_lo + len < hi ? c_lo + len : hi;
  const int rpad = p.rpad;
  const E* ring = (const E*)p.ring;
  const int64_t st = p.slot_stride;
  __shared__ W sw[kMaxSlots * kMaxRpad];
  __shared__ const E* sptr[kMaxSlots];
  for (int t = threadIdx.x; t < n * rpad; t += blockDim.x) {
    const int a = t / rpad, c = t % rpad;
    sw[t] = CombAcc<T>::wconv(p.w[((int64_t)R * rpad + c) * kMaxSlots + a]);
  }
  for (int a = threadIdx.x; a < n; a += blockDim.x) sptr[a] = snap_slot(ring, y_slots[a], st);
  __syncthreads();
  const int c = threadIdx.x & (rpad - 1);
  const int64_t base = c_lo * 3 * rpad, cnt = c_hi > c_lo ? (c_hi - c_lo) * 3 * rpad : 0;
  if (rpad >= 2) {
    // two consecutive values a thread (cases c0, c0 + 1), four slots' vector loads in flight
    const int c0 = (2 * threadIdx.x) & (rpad - 1);
    for (int64_t i = 2 * (int64_t)threadIdx.x; i < cnt; i += 2 * (int64_t)blockDim.x) {
      const int64_t gi = base + i;
      CombAcc<T> s0, s1;
      for (int a0 = 0; a0 < n; a0 += 4) {
        T y0[4], y1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (a0 + u < n) {
            load_snap2(sptr[a0 + u], st, gi, y0[u], y1[u]);
          } else {
            y0[u] = y1[u] = T{};
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (a0 + u < n) s0.add(sw[(a0 + u) * rpad + c0], y0[u]), s1.add(sw[(a0 + u) * rpad + c0 + 1], y1[u]);
      }
      if (y_base) {
        const double2 yb = *reinterpret_cast<const double2*>(y_base + gi);
        const double2 yo = make_double2(yb.x + s0.get(), yb.y + s1.get());
        *reinterpret_cast<double2*>(y_out + gi) = yo;
        if (y_out2) *reinterpret_cast<double2*>(y_out2 + gi) = yo;
        *reinterpret_cast<float2*>(corr32 + gi) = make_float2(s0.getf(), s1.getf());
      } else {
        double2 yo = *reinterpret_cast<const double2*>(y_out + gi);
        yo.x += s0.get();
        yo.y += s1.get();
        *reinterpret_cast<double2*>(y_out + gi) = yo;
      }
    }
  } else
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int64_t gi = base + i;
    CombAcc<T> s0, s1;
    // eight loads in flight per thread before their products are formed
    for (int a0 = 0; a0 < n; a0 += 8) {
      T y[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) y[u] = a0 + u < n ? load_snap(sptr[a0 + u], st, gi) : T{};
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        if (a0 + u < n) s0.add(sw[(a0 + u) * rpad + c], y[u]);
        if (a0 + u + 1 < n) s1.add(sw[(a0 + u + 1) * rpad + c], y[u + 1]);
      }
    }
    s0.merge(s1);
    if (y_base) {
      const double yo = y_base[gi] + s0.get();
      y_out[gi] = yo;
      if (y_out2) y_out2[gi] = yo;
      corr32[gi] = s0.getf();
    } else {
      y_out[gi] += s0.get();
    }
  }
  if (y_base) {
    auto copy = [&](int64_t e0, int64_t e1) {
      for (int64_t gi = e0 + threadIdx.x; gi < e1; gi += blockDim.x) {
        const double yb = y_base[gi];
        y_out[gi] = yb;
        if (y_out2) y_out2[gi] = yb;
        corr32[gi] = 0.0f;
      }
    };
    if (k == p.n_chunks - 1) copy(hi * 3 * rpad, (int64_t)gap_hi[R] * 3 * rpad);
    if (blockIdx.x == 0) copy(0, (int64_t)lead_hi * 3 * rpad);
  }
}

// Two combinations in one pass over the ring: y_out += Y w (the data-driven guess) and y2 = Y w2 (the
// learned proposal's correction of it).
template <typename E>
__global__ void __launch_bounds__(kBlock) k_pred_combine2(PredView p, const int* __restrict__ y_slots, int n,
                                                          double* __restrict__ y_out, const double* __restrict__ w2,
                                                          double* __restrict__ y2) {
  typedef typename SnapVal<E>::V T;
  typedef typename CombAcc<T>::W W;
  const int R = blockIdx.x / p.n_chunks, k = blockIdx.x % p.n_chunks;
  const int64_t lo = p.reg_lo[R], hi = p.reg_hi[R];
  const int64_t len = (hi - lo + p.n_chunks - 1) / p.n_chunks;
  const int64_t c_lo = lo + k * len, c_hi = c_lo + len < hi ? c_lo + len : hi;
  const int rpad = p.rpad;
  const E* ring = (const E*)p.ring;
  const int64_t st = p.slot_stride;
  __shared__ W sw[kMaxSlots * kMaxRpad];
  __shared__ W sw2[kMaxSlots * kMaxRpad];
  __shared__ const E* sptr[kMaxSlots];
  for (int t = threadIdx.x; t < n * rpad; t += blockDim.x) {
    const int a = t / rpad, c = t % rpad;
    const int64_t o = ((int64_t)R * rpad + c) * kMaxSlots + a;
    sw[t] = CombAcc<T>::wconv(p.w[o]);
    sw2[t] = CombAcc<T>::wconv(w2[o]);
  }
  for (int a = threadIdx.x; a < n; a += blockDim.x) sptr[a] = snap_slot(ring, y_slots[a], st);
  __syncthreads();
  const int c = threadIdx.x & (rpad - 1);
  const int64_t base = c_lo * 3 * rpad, cnt = c_hi > c_lo ? (c_hi - c_lo) * 3 * rpad : 0;
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int64_t gi = base + i;
    CombAcc<T> s0, t0;
    for (int a = 0; a < n; ++a) {
      const T y = load_snap(sptr[a], st, gi);
      s0.add(sw[a * rpad + c], y);
      t0.add(sw2[a * rpad + c], y);
    }
    y_out[gi] += s0.get();
    y2[gi] = t0.get();
  }
}

// dst[n*3 + k] = src[(n*3 + k)*rpad + c]
__global__ void k_extract_case(int64_t n3, int rpad, int c, const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i * rpad + c];
}

// dst[c][j] = src[j][c]: a thread reads one node component's row of cases (its neighbours the adjacent
// rows, so the reads stay in the same cache lines) and writes it out case by case, coalesced per case.
__global__ void k_extract_all(int64_t n3, int rpad, int n_cases, const double* __restrict__ src,
                              double* __restrict__ dst) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n3; j += (int64_t)gridDim.x * blockDim.x) {
    const double* row = src + j * rpad;
    for (int c = 0; c < n_cases; ++c) dst[c * n3 + j] = row[c];
  }
}

// ---- products kept by linear recurrences (FP32-inner steps) ----
// With K u, M v, K v maintained exactly (FP64) from the split products M du, K du of each certified
// increment, and with them the load-free part of the Newmark right-hand side
//   Pb = M a + (4/dt + a0) M v + a1 K v - K u,
// the right-hand side needs no EBE pass and reads one vector:  b = f + Pb.
__global__ void k_rhs_incr(MeshView m, int rpad, int rshift, const double* __restrict__ Pb, double* __restrict__ b,
                           const RickerSrc* __restrict__ src, const double* __restrict__ ext, double t,
                           const StepCtl* ctl) {
  if (ctl) {
    t = ctl->t;
    if (!ctl->use_ext) ext = nullptr;
  }
  // point load of case cs at node n (zero elsewhere)
  auto load_of = [&](int64_t n, int cs) -> double3 {
    if (src[cs].node != n) return make_double3(0.0, 0.0, 0.0);
    if (ext) return make_double3(ext[cs * 3], ext[cs * 3 + 1], ext[cs * 3 + 2]);
    const RickerSrc& s = src[cs];
    const double arg = (M_PI * s.f0 * (t - s.t0)) * (M_PI * s.f0 * (t - s.t0));
    const double w = s.amp * (1.0 - 2.0 * arg) * exp(-arg);
    return make_double3(w * s.dir[0], w * s.dir[1], w * s.dir[2]);
  };
  if (!m.seg && rpad >= 2) {
    // two cases (c, c + 1) a thread by 16-byte accesses
    const int rs1 = rshift - 1;
    const int64_t total = m.N << rs1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
      const int64_t n = i >> rs1;
      const int c = (int)(i & ((rpad >> 1) - 1)) << 1;
      const uint8_t f = m.freemask[n];
      double2 pb[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) pb[k] = *reinterpret_cast<const double2*>(Pb + (n * 3 + k) * rpad + c);
      const double3 g0 = load_of(n, c), g1 = load_of(n, c + 1);
      const double f0[3] = {g0.x, g0.y, g0.z}, f1[3] = {g1.x, g1.y, g1.z};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int64_t id = (n * 3 + k) * rpad + c;
        *reinterpret_cast<double2*>(b + id) =
            dof_free(f, k) ? make_double2(f0[k] + pb[k].x, f1[k] + pb[k].y) : make_double2(0.0, 0.0);
      }
    }
    return;
  }
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const int cs = m.seg ? m.seg[n] : c;            // case of this entry (fused groups: the node's mesh)
    const uint8_t f = m.freemask[n];
    const double3 g = load_of(n, cs);
    const double fv[3] = {g.x, g.y, g.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t id = (n * 3 + k) * rpad + c;
      b[id] = dof_free(f, k) ? fv[k] + Pb[id] : 0.0;
    }
  }
}

// Pb = Ma + c1 Mv + a1 Kv - Ku from directly computed products (the periodic refresh), in place of Ma.
__global__ void k_pb_form(int64_t n, double c1, double a1, double* __restrict__ Pb, const double* __restrict__ Mv,
                          const double* __restrict__ Kv, const double* __restrict__ Ku) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Pb[i] = Pb[i] + c1 * Mv[i] + a1 * Kv[i] - Ku[i];
}

// y32 = float(guess - du_ab): the data-driven part of the guess, for its FP32 product.
__global__ void k_corr_f32(int64_t n, const double* __restrict__ guess, const double* __restrict__ du_ab,
                           float* __restrict__ y32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y32[i] = d2f(guess[i] - du_ab[i]);
}

// Residual of the guess without an FP64 product:  r0 = b - A du_AB - A y  with
// A du_AB = dt/24 (-9 Av^{it-4} + 37 Av^{it-3} - 59 Av^{it-2} + 55 Av^{it-1}) exact (FP64 recurrences)
// and A y from the FP32 product of the small data-driven correction (qy, nullable).  Writes r32 and
// starts the outer (FP64) iteration state.
// The inner FP32 solve's starting state for a refinement pass whose right-hand side r32 a residual kernel
// has just written (zero initial guess, so its residual is r32 itself): the work of the separate norm and
// first-residual passes, from the sums the residual kernel already forms.  ||r32||^2 (rrc, summed in FP64)
// is both the right-hand side norm and the residual norm; zrc = (B^-1 r32, r32).  A case whose outer
// solve is inactive gets a zero right-hand side (inactive).
__device__ __forceinline__ void init_inner(CgCase& s, const CgCase& o, double rrc, double zrc) {
  s.bb = o.active ? rrc : 0.0;
  s.pq = s.alpha = s.beta = 0.0;
  s.iters = 0;
  s.outer = 0;
  s.phase = 0;
  s.tol2 = o.inner_tol * o.inner_tol;
  s.rho = zrc;
  s.rr = rrc;
  s.relres = s.bb > 0.0 ? 1.0 : 0.0;
  s.relres0 = s.relres;
  s.status = (isfinite(rrc) && isfinite(zrc)) ? FEM_OK : FEM_ERR_NONFINITE;
  s.active = (s.status == FEM_OK && s.bb > 0.0) ? 1 : 0;
}

// (B^-1 r, r) of one node's three values (FP32, B^-1 symmetric [xx yy zz xy xz yz]).
__device__ __forceinline__ float zr_node(const float* __restrict__ B, float r0, float r1, float r2) {
  const float z0 = B[0] * r0 + B[3] * r1 + B[4] * r2;
  const float z1 = B[3] * r0 + B[1] * r1 + B[5] * r2;
  const float z2 = B[4] * r0 + B[5] * r1 + B[2] * r2;
  return z0 * r0 + z1 * r1 + z2 * r2;
}

// ALT (a data-driven correction y whose product qy = A y is given, and the guess guard on): the same pass
// also forms the norms of the Adams-Bashforth guess's residual r0 + A y, in the FP32 values the guard's fix
// pass would write (r32 + qy, rounded once).  The last block keeps, per case, the guess with the smaller
// initial residual: a case whose correction makes the residual larger (an extrapolation that has gone
// astray at the onset of a wave) drops it (CgCase::guess = 2, fallbacks[c] += 1), and k_guard_fix then
// rewrites that case's r32 and guess.
template <bool ALT>
__global__ void __launch_bounds__(kVecBlock, 2) k_r0(MeshView m, int rpad, int rshift, double h, const double* __restrict__ b,
                                               const double* __restrict__ Av4, const double* __restrict__ Av3,
                                               const double* __restrict__ Av2, const double* __restrict__ Av1,
                                               const float* __restrict__ qy, float* __restrict__ r32, Reducer red,
                                               CgCase* outer, int* n_active, double tol, double inner_max,
                                               double aim, Ring4 avr, const StepCtl* ctl, CgCase* inner,
                                               int* fallbacks) {
  if (ctl) {   // A v^{it-4} .. A v^{it-1} in ring slots it .. it+3 (mod 4)
    const int it = ctl->it;
    Av4 = avr.p[it & 3], Av3 = avr.p[(it + 1) & 3], Av2 = avr.p[(it + 2) & 3], Av1 = avr.p[(it + 3) & 3];
  }
  double bb = 0.0, rr = 0.0, ra = 0.0;
  float zr = 0.f, za = 0.f;
  // the Adams-Bashforth weights times -h: four FMAs from b (the FP64 pipe bounds this kernel)
  const double w4 = 9.0 * h, w3 = -37.0 * h, w2 = 59.0 * h, w1 = -55.0 * h;
  const int64_t total = m.N << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i >> rshift;
    const int c = (int)(i & (rpad - 1));
    const uint8_t f = m.freemask[n];
    float rf[3], fa[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t id = (n * 3 + k) * rpad + c;
      double v = 0.0;
      float qv = 0.f;
      const double bv = b[id];
      if (dof_free(f, k)) {
        v = fma(w1, Av1[id], fma(w2, Av2[id], fma(w3, Av3[id], fma(w4, Av4[id], bv))));
        if (qy) {
          qv = qy[id];
          v -= f2d(qv);
        }
      }
      rf[k] = d2f(v);
      r32[id] = rf[k];
      bb += bv * bv;
      if (ALT) fa[k] = dof_free(f, k) ? rf[k] + qv : 0.f;
    }
    // the residual norms from the FP32 values, a node's three squares summed in FP32 (relative error ~1e-7;
    // the FP64 pipe, which bounds this kernel, takes one add a node instead of an FMA a value)
    rr += (double)fmaf(rf[2], rf[2], fmaf(rf[1], rf[1], rf[0] * rf[0]));
    if (ALT) ra += (double)fmaf(fa[2], fa[2], fmaf(fa[1], fa[1], fa[0] * fa[0]));
    if (inner) {
      zr += zr_node(m.binv32 + n * 6, rf[0], rf[1], rf[2]);
      if (ALT) za += zr_node(m.binv32 + n * 6, fa[0], fa[1], fa[2]);
    }
  }
  constexpr int NQ = ALT ? 5 : 3;
  double vals[NQ];
  vals[0] = bb, vals[1] = rr, vals[2] = (double)zr;
  if (ALT) vals[NQ - 2] = ra, vals[NQ - 1] = (double)za;
  if (block_reduce_last<NQ>(vals, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
      CgCase& s = outer[c];
      const double bbc = red.out[c];
      double rrc = red.out[rpad + c], zrc = red.out[2 * rpad + c];
      s.guess = qy ? 1 : 0;
      if (ALT) {
        // (a margin keeps a correction that changes the residual by rounding only)
        const double rra = red.out[3 * rpad + c];
        if (bbc > 0.0 && isfinite(rra) && (!isfinite(rrc) || rra < rrc * (1.0 - 1e-6))) {
          rrc = rra;
          zrc = red.out[4 * rpad + c];
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
      // estimate only: the certificate is the FP64 residual computed after the solve
      s.active = (s.status == FEM_OK && bbc > 0.0 && rrc >= tol * tol * bbc) ? 1 : 0;
      s.inner_tol = inner_target(aim, s.relres, inner_max);
      if (inner) init_inner(inner[c], s, rrc, zrc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int na = 0;
      for (int c = 0; c < rpad; ++c) na += outer[c].active;
      *n_active = na;
    }
  }
}

// The guess guard's fix pass: for each case whose correction k_r0 (or k_r0_seg) dropped (CgCase::guess ==
// 2), r32 += qy on free DOFs (the Adams-Bashforth guess's residual, the values whose norms were formed) and
// guess = x = du_AB.  Every block returns at once when no case dropped its correction, the usual case.
__global__ void k_guard_fix(MeshView m, int rpad, int rshift, const CgCase* __restrict__ outer,
                            const float* __restrict__ qy, float* __restrict__ r32, const double* __restrict__ du_ab,
                            double* __restrict__ guess, double* __restrict__ x) {
  __shared__ unsigned char drop[kMaxCases];
  __shared__ int any;
  const int nc = m.seg ? m.nseg : rpad;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    drop[c] = outer[c].guess == 2 ? 1 : 0;
    if (drop[c]) any = 1;
  }
  __syncthreads();
  if (!any) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (m.seg) {   // fused groups: one case a node, [N][3]
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < m.N; n += stride) {
      if (!drop[m.seg[n]]) continue;
      const uint8_t f = m.freemask[n];
      for (int k = 0; k < 3; ++k) {
        const int64_t id = n * 3 + k;
        if (dof_free(f, k)) r32[id] = r32[id] + qy[id];
        guess[id] = du_ab[id];
        if (x) x[id] = du_ab[id];
      }
    }
    return;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (m.N << rshift); i += stride) {
    const int c = (int)(i & (rpad - 1));
    if (!drop[c]) continue;
    const int64_t n = i >> rshift;
    const uint8_t f = m.freemask[n];
    for (int k = 0; k < 3; ++k) {
      const int64_t id = (n * 3 + k) * rpad + c;
      if (dof_free(f, k)) r32[id] = r32[id] + qy[id];
      guess[id] = du_ab[id];
      if (x) x[id] = du_ab[id];
    }
  }
}

// Certified FP64 residual from the split products:  r = b - (cM qM + cK qK);  r32 = float(r) for the next
// inner solve; cases at or above tol stay active.
__global__ void __launch_bounds__(kVecBlock, 2) k_cert(MeshView m, int rpad, int rshift, double cM, double cK,
                                                 const double* __restrict__ b, const double* __restrict__ qM,
                                                 const double* __restrict__ qK, float* __restrict__ r32, Reducer red,
                                                 CgCase* outer, int* n_active, double tol, double inner_max,
                                                 double aim, CgCase* inner) {
  double rr = 0.0;
  float zr = 0.f;
  const int64_t total = m.N << rshift;
  // two items an iteration (the grid stride apart), the loads of both issued first
  struct Item {
    double b[3], m[3], k[3];
    uint8_t f;
    int64_t n, id0;
  };
  auto load = [&](int64_t i, Item& it) {
    it.n = i >> rshift;
    it.id0 = it.n * 3 * rpad + (int)(i & (rpad - 1));
    it.f = m.freemask[it.n];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t id = it.id0 + k * rpad;
      it.b[k] = b[id], it.m[k] = qM[id], it.k[k] = qK[id];
    }
  };
  auto apply = [&](const Item& it) {
    float rf[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = dof_free(it.f, k) ? fma(-cK, it.k[k], fma(-cM, it.m[k], it.b[k])) : 0.0;
      rf[k] = d2f(v);
      r32[it.id0 + k * rpad] = rf[k];
      rr = fma(v, v, rr);
    }
    if (inner) zr += zr_node(m.binv32 + it.n * 6, rf[0], rf[1], rf[2]);
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += 2 * stride) {
    Item a, b2;
    const bool two = i + stride < total;
    load(i, a);
    if (two) load(i + stride, b2);
    apply(a);
    if (two) apply(b2);
  }
  double vals[2] = {rr, (double)zr};
  if (block_reduce_last<2>(vals, rpad, red)) {
    if (threadIdx.x < rpad) {
      const int c = threadIdx.x;
      CgCase& s = outer[c];
      const double rrc = red.out[c];
      s.rr = rrc;
      s.relres = s.bb > 0.0 ? sqrt(rrc / s.bb) : 0.0;
      s.outer += 1;
      if (!isfinite(rrc)) s.status = FEM_ERR_NONFINITE;
      s.active = (s.status == FEM_OK && s.bb > 0.0 && rrc >= tol * tol * s.bb) ? 1 : 0;
      s.inner_tol = inner_target(aim, s.relres, inner_max);
      if (inner) init_inner(inner[c], s, rrc, red.out[rpad + c]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int na = 0;
      for (int c = 0; c < rpad; ++c) na += outer[c].active;
      *n_active = na;
    }
  }
}

// Newmark update with the product recurrences (du, its products qM = M du, qK = K du):
//   u += du;  v' = 2/dt du - v;  a' = 4/dt^2 du - 4/dt v - a;
//   Ku += qK;  Mv' = 2/dt qM - Mv;  Kv' = 2/dt qK - Kv;  (Ma' = 4/dt^2 qM - 4/dt Mv - Ma, not stored: it
//   enters Pb' below);  Av' = cM Mv' + cK Kv' (pushed to the 4-deep ring);  e = du - du_AB (snapshot).
// P selects the part: 0 all of it; 1 the velocity side (v, M v, K v, A v, the snapshot: what the Gram row and
// the next step's Adams-Bashforth and guess residual read); 2 the state side (u, a, K u, Pb: what the next
// right-hand side reads), run after part 1 so that it may overlap the Gram row.  Part 2 finds M v already
// updated and uses  -4/dt Mv = 4/dt Mv' - (8/dt^2) qM  in the Pb recurrence.
template <typename E, int P>
__global__ void k_newmark_incr(int64_t n, double dt, double cM, double cK, double c1, double a1,
                               const double* __restrict__ du,
                               const double* __restrict__ du_ab, const double* __restrict__ qM,
                               const double* __restrict__ qK, double* __restrict__ u, const double* __restrict__ v_prev,
                               double* __restrict__ a, double* __restrict__ v_push, double* __restrict__ Ku,
                               double* __restrict__ Mv, double* __restrict__ Kv, double* __restrict__ Pb,
                               double* __restrict__ Av_push, E* __restrict__ e_push, Ring4 vr, Ring4 avr,
                               E* __restrict__ ring, int64_t slot_stride, const StepCtl* ctl) {
  if (ctl) {
    const int it = ctl->it;
    v_prev = vr.p[(it + 3) & 3];
    v_push = vr.p[it & 3];
    Av_push = avr.p[it & 3];
    e_push = ring ? snap_slot(ring, ctl->slot_new, slot_stride) : nullptr;
  }
  constexpr bool VEL = P != 2, STATE = P != 1;
  const double c2 = 2.0 / dt, c4 = 4.0 / dt, c44 = 4.0 / (dt * dt);
  // Pb' = Ma' + c1 Mv' + a1 Kv' - Ku' with the recurrences above substituted:
  //   Pb' = (4/dt^2 + 2 c1/dt) qM + (2 a1/dt - 1) qK - Pb - 4/dt Mv - 2 Ku   (Mv, Ku before the update)
  // (part 2: al2 qM + be qK - Pb + 4/dt Mv' - 2 Ku, al2 = al - 8/dt^2)
  const double al = c44 + c1 * c2, be = a1 * c2 - 1.0, al2 = al - c4 * c2;
  // two consecutive values a thread (vector loads and stores of every vector; n even), then a last odd one
  const int64_t npair = n >> 1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npair; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 2 * t;
    auto ld = [&](const double* x) { return *reinterpret_cast<const double2*>(x + i); };
    auto st = [&](double* x, double y0, double y1) { *reinterpret_cast<double2*>(x + i) = make_double2(y0, y1); };
    const double2 d = ld(du), vp = ld(v_prev), m_ = ld(qM), k_ = ld(qK), mv = ld(Mv);
    if (STATE) {
      const double2 uu = ld(u), aa = ld(a), ku = ld(Ku), pb = ld(Pb);
      st(u, uu.x + d.x, uu.y + d.y);
      st(a, c44 * d.x - c4 * vp.x - aa.x, c44 * d.y - c4 * vp.y - aa.y);
      st(Ku, ku.x + k_.x, ku.y + k_.y);
      if (P == 0) {
        st(Pb, al * m_.x + be * k_.x - (pb.x + c4 * mv.x + 2.0 * ku.x),
           al * m_.y + be * k_.y - (pb.y + c4 * mv.y + 2.0 * ku.y));
      } else {
        st(Pb, al2 * m_.x + be * k_.x - (pb.x - c4 * mv.x + 2.0 * ku.x),
           al2 * m_.y + be * k_.y - (pb.y - c4 * mv.y + 2.0 * ku.y));
      }
    }
    if (VEL) {
      const double2 kv = ld(Kv);
      st(v_push, c2 * d.x - vp.x, c2 * d.y - vp.y);
      const double mv2x = c2 * m_.x - mv.x, kv2x = c2 * k_.x - kv.x, mv2y = c2 * m_.y - mv.y, kv2y = c2 * k_.y - kv.y;
      st(Mv, mv2x, mv2y);
      st(Kv, kv2x, kv2y);
      st(Av_push, cM * mv2x + cK * kv2x, cM * mv2y + cK * kv2y);
      if (e_push) {
        const double2 ab = ld(du_ab);
        store_snap2(e_push, slot_stride, i, d.x - ab.x, d.y - ab.y);
      }
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    const double d = du[i], vp = v_prev[i], m_ = qM[i], k_ = qK[i], mv = Mv[i];
    if (STATE) {
      u[i] += d;
      a[i] = c44 * d - c4 * vp - a[i];
      const double ku = Ku[i];
      Ku[i] = ku + k_;
      Pb[i] = P == 0 ? al * m_ + be * k_ - (Pb[i] + c4 * mv + 2.0 * ku)
                     : al2 * m_ + be * k_ - (Pb[i] - c4 * mv + 2.0 * ku);
    }
    if (VEL) {
      v_push[i] = c2 * d - vp;
      const double kv = Kv[i];
      const double mv2 = c2 * m_ - mv, kv2 = c2 * k_ - kv;
      Mv[i] = mv2;
      Kv[i] = kv2;
      Av_push[i] = cM * mv2 + cK * kv2;
      if (e_push) store_snap(e_push, slot_stride, i, d - du_ab[i]);
    }
  }
}

// out = alpha x + beta y
__global__ void k_axpby(int64_t n, double alpha, const double* __restrict__ x, double beta,
                        const double* __restrict__ y, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = alpha * x[i] + beta * y[i];
}

// ---- launchers ----
cudaError_t launch_axpby(int64_t n, double alpha, const double* x, double beta, const double* y, double* out,
                         cudaStream_t s) {
  k_axpby<<<grid_for(n), kBlock, 0, s>>>(n, alpha, x, beta, y, out);
  return cudaGetLastError();
}

cudaError_t launch_extract_all(int64_t N, int rpad, int n_cases, const double* src, double* dst, cudaStream_t s) {
  k_extract_all<<<grid_for(N * 3, wide_grid_cap()), kBlock, 0, s>>>(N * 3, rpad, n_cases, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_extract_case(int64_t N, int rpad, int c, const double* src, double* dst, cudaStream_t s) {
  k_extract_case<<<grid_for(N * 3), kBlock, 0, s>>>(N * 3, rpad, c, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_rhs_prep(int64_t n, double dt, double a0, double a1, const double* u, const double* v,
                            const double* a, double* m_in, double* k_in, cudaStream_t s) {
  k_rhs_prep<<<grid_for(n), kBlock, 0, s>>>(n, 4.0 / dt + a0, a1, u, v, a, m_in, k_in);
  return cudaGetLastError();
}

cudaError_t launch_rhs_finish(const MeshView& m, int rpad, double* b, const RickerSrc* src, const double* ext,
                              double t, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_rhs_finish<<<grid_for(m.N << rs), kBlock, 0, s>>>(m, rpad, rs, b, src, ext, t);
  return cudaGetLastError();
}

cudaError_t launch_ab4(int64_t n, double dt, const double* v4, const double* v3, const double* v2, const double* v1,
                       double* du_ab, cudaStream_t s) {
  k_ab4<<<grid_for(n), kBlock, 0, s>>>(n, dt / 24.0, v4, v3, v2, v1, du_ab);
  return cudaGetLastError();
}

cudaError_t launch_ab4_ring(int64_t n, double dt, Ring4 v, const StepCtl* ctl, double* du_ab, cudaStream_t s,
                            int ahead) {
  k_ab4_ring<<<grid_for(n), kBlock, 0, s>>>(n, dt / 24.0, v, ctl, du_ab, ahead);
  return cudaGetLastError();
}

cudaError_t launch_add(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
  k_add<<<grid_for(n), kBlock, 0, s>>>(n, a, b, out);
  return cudaGetLastError();
}

cudaError_t launch_newmark_update(int64_t n, double dt, const double* du, const double* du_ab, double* u,
                                  const double* v_prev, double* a, double* v_push, void* e_push, int e_fmt,
                                  int64_t stride, cudaStream_t s) {
  if (e_fmt == 1)
    k_newmark<float><<<grid_for(n), kBlock, 0, s>>>(n, dt, du, du_ab, u, v_prev, a, v_push, (float*)e_push, stride);
  else if (e_fmt == 2)
    k_newmark<float2><<<grid_for(n), kBlock, 0, s>>>(n, dt, du, du_ab, u, v_prev, a, v_push, (float2*)e_push, stride);
  else if (e_fmt == 3)
    k_newmark<SnapHL><<<grid_for(n), kBlock, 0, s>>>(n, dt, du, du_ab, u, v_prev, a, v_push, (SnapHL*)e_push, stride);
  else
    k_newmark<double><<<grid_for(n), kBlock, 0, s>>>(n, dt, du, du_ab, u, v_prev, a, v_push, (double*)e_push, stride);
  return cudaGetLastError();
}

cudaError_t launch_rhs_incr(const MeshView& m, int rpad, const double* Pb, double* b, const RickerSrc* src,
                            const double* ext, double t, cudaStream_t s, const StepCtl* ctl) {
  const int rs = log2i(rpad);
  k_rhs_incr<<<grid_resident((const void*)k_rhs_incr, kBlock, m.N << rs), kBlock, 0, s>>>(m, rpad, rs, Pb, b, src, ext,
                                                                                          t, ctl);
  return cudaGetLastError();
}

cudaError_t launch_pb_form(int64_t n, double dt, double a0, double a1, double* Pb, const double* Mv, const double* Kv,
                           const double* Ku, cudaStream_t s) {
  k_pb_form<<<grid_for(n), kBlock, 0, s>>>(n, 4.0 / dt + a0, a1, Pb, Mv, Kv, Ku);
  return cudaGetLastError();
}

cudaError_t launch_corr_f32(int64_t n, const double* guess, const double* du_ab, float* y32, cudaStream_t s) {
  k_corr_f32<<<grid_for(n), kBlock, 0, s>>>(n, guess, du_ab, y32);
  return cudaGetLastError();
}

cudaError_t launch_r0(const MeshView& m, int rpad, double dt, const double* b, const double* Av4, const double* Av3,
                      const double* Av2, const double* Av1, const float* qy, float* r32, Reducer red, CgCase* outer,
                      int* n_active, double tol, double inner_max, double aim, cudaStream_t s, Ring4 avr,
                      const StepCtl* ctl, CgCase* inner, bool guard, int* fallbacks) {
  const int rs = log2i(rpad);
  if (guard && qy) {
    k_r0<true><<<grid_resident((const void*)k_r0<true>, kVecBlock, m.N << rs), kVecBlock, 0, s>>>(
        m, rpad, rs, dt / 24.0, b, Av4, Av3, Av2, Av1, qy, r32, red, outer, n_active, tol, inner_max, aim, avr, ctl,
        inner, fallbacks);
  } else {
    k_r0<false><<<grid_resident((const void*)k_r0<false>, kVecBlock, m.N << rs), kVecBlock, 0, s>>>(
        m, rpad, rs, dt / 24.0, b, Av4, Av3, Av2, Av1, qy, r32, red, outer, n_active, tol, inner_max, aim, avr, ctl,
        inner, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_guard_fix(const MeshView& m, int rpad, const CgCase* outer, const float* qy, float* r32,
                             const double* du_ab, double* guess, double* x, cudaStream_t s) {
  const int rs = log2i(rpad);
  k_guard_fix<<<grid_for(m.seg ? m.N : (m.N << rs)), kBlock, 0, s>>>(m, rpad, rs, outer, qy, r32, du_ab, guess, x);
  return cudaGetLastError();
}

cudaError_t launch_cert(const MeshView& m, int rpad, double cM, double cK, const double* b, const double* qM,
                        const double* qK, float* r32, Reducer red, CgCase* outer, int* n_active, double tol,
                        double inner_max, double aim, cudaStream_t s, CgCase* inner) {
  const int rs = log2i(rpad);
  k_cert<<<grid_resident((const void*)k_cert, kVecBlock, m.N << rs), kVecBlock, 0, s>>>(m, rpad, rs, cM, cK, b, qM, qK, r32, red, outer, n_active, tol,
                                                inner_max, aim, inner);
  return cudaGetLastError();
}

template <typename E, int P>
static void newmark_incr_t(int64_t n, double dt, double cM, double cK, double c1, double a1, const double* du,
                           const double* du_ab, const double* qM, const double* qK, double* u, const double* v_prev,
                           double* a, double* v_push, double* Ku, double* Mv, double* Kv, double* Pb, double* Av_push,
                           void* e_push, cudaStream_t s, Ring4 vr, Ring4 avr, void* ring, int64_t slot_stride,
                           const StepCtl* ctl) {
  const int grid = grid_resident((const void*)k_newmark_incr<E, P>, kBlock, n);
  k_newmark_incr<E, P><<<grid, kBlock, 0, s>>>(n, dt, cM, cK, c1, a1, du, du_ab, qM, qK, u, v_prev, a, v_push, Ku, Mv,
                                               Kv, Pb, Av_push, (E*)e_push, vr, avr, (E*)ring, slot_stride, ctl);
}

template <int P>
static void newmark_incr_p(int64_t n, double dt, double cM, double cK, double c1, double a1, const double* du,
                           const double* du_ab, const double* qM, const double* qK, double* u, const double* v_prev,
                           double* a, double* v_push, double* Ku, double* Mv, double* Kv, double* Pb, double* Av_push,
                           void* e_push, int e_fmt, cudaStream_t s, Ring4 vr, Ring4 avr, void* ring,
                           int64_t slot_stride, const StepCtl* ctl) {
#define NM_ARGS n, dt, cM, cK, c1, a1, du, du_ab, qM, qK, u, v_prev, a, v_push, Ku, Mv, Kv, Pb, Av_push, e_push, s, vr, \
                avr, ring, slot_stride, ctl
  if (e_fmt == 1)
    newmark_incr_t<float, P>(NM_ARGS);
  else if (e_fmt == 2)
    newmark_incr_t<float2, P>(NM_ARGS);
  else if (e_fmt == 3)
    newmark_incr_t<SnapHL, P>(NM_ARGS);
  else
    newmark_incr_t<double, P>(NM_ARGS);
#undef NM_ARGS
}

cudaError_t launch_newmark_incr_part(int64_t n, double dt, double cM, double cK, double a0, double a1,
                                     const double* du, const double* du_ab, const double* qM, const double* qK,
                                     double* u, const double* v_prev, double* a, double* v_push, double* Ku,
                                     double* Mv, double* Kv, double* Pb, double* Av_push, void* e_push, int e_fmt,
                                     cudaStream_t s, Ring4 vr, Ring4 avr, void* ring, int64_t slot_stride,
                                     const StepCtl* ctl, int part) {
  const double c1 = 4.0 / dt + a0;
  if (part == 1)
    newmark_incr_p<1>(n, dt, cM, cK, c1, a1, du, du_ab, qM, qK, u, v_prev, a, v_push, Ku, Mv, Kv, Pb, Av_push, e_push,
                      e_fmt, s, vr, avr, ring, slot_stride, ctl);
  else if (part == 2)
    newmark_incr_p<2>(n, dt, cM, cK, c1, a1, du, du_ab, qM, qK, u, v_prev, a, v_push, Ku, Mv, Kv, Pb, Av_push, e_push,
                      e_fmt, s, vr, avr, ring, slot_stride, ctl);
  else
    newmark_incr_p<0>(n, dt, cM, cK, c1, a1, du, du_ab, qM, qK, u, v_prev, a, v_push, Ku, Mv, Kv, Pb, Av_push, e_push,
                      e_fmt, s, vr, avr, ring, slot_stride, ctl);
  return cudaGetLastError();
}

cudaError_t launch_newmark_incr(int64_t n, double dt, double cM, double cK, double a0, double a1, const double* du,
                                const double* du_ab, const double* qM, const double* qK, double* u,
                                const double* v_prev, double* a, double* v_push, double* Ku, double* Mv, double* Kv,
                                double* Pb, double* Av_push, void* e_push, int e_fmt, cudaStream_t s, Ring4 vr,
                                Ring4 avr, void* ring, int64_t slot_stride, const StepCtl* ctl) {
  return launch_newmark_incr_part(n, dt, cM, cK, a0, a1, du, du_ab, qM, qK, u, v_prev, a, v_push, Ku, Mv, Kv, Pb,
                                  Av_push, e_push, e_fmt, s, vr, avr, ring, slot_stride, ctl, 0);
}

cudaError_t launch_pred_dots(const PredView& p, int slot_new, uint64_t valid_mask, cudaStream_t s,
                             const StepCtl* ctl) {
  if (p.n_regions == 0) return cudaSuccess;
  const dim3 grid(p.n_regions * p.n_chunks * kDotGroups);
  if (p.fmt == 1)
    k_pred_dots<float><<<grid, kBlock, 0, s>>>(p, slot_new, valid_mask, ctl);
  else if (p.fmt == 2)
    k_pred_dots<float2><<<grid, kBlock, 0, s>>>(p, slot_new, valid_mask, ctl);
  else if (p.fmt == 3)
    k_pred_dots<SnapHL><<<grid, kBlock, 0, s>>>(p, slot_new, valid_mask, ctl);
  else
    k_pred_dots<double><<<grid, kBlock, 0, s>>>(p, slot_new, valid_mask, ctl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pred_dots_finish<<<p.n_regions, 256, 0, s>>>(p, slot_new, valid_mask, ctl);
  return cudaGetLastError();
}

cudaError_t launch_pred_solve(const PredView& p, const int* x_slots, int n_pairs, int slot_new, double tau,
                              cudaStream_t s, const StepCtl* ctl) {
  if (p.n_regions == 0 || (!ctl && n_pairs <= 0)) return cudaSuccess;
  k_pred_solve<<<p.n_regions * p.rpad, 32, 0, s>>>(p, x_slots, n_pairs, slot_new, tau, ctl);
  return cudaGetLastError();
}

cudaError_t launch_pred_combine(const PredView& p, const int* y_slots, int n_pairs, double* y_out, cudaStream_t s,
                                const StepCtl* ctl, const double* y_base, float* corr32, const int32_t* gap_hi,
                                int lead_hi, double* y_out2) {
  if (p.n_regions == 0 || (!ctl && n_pairs <= 0 && !y_base)) return cudaSuccess;
  if (y_base && (!corr32 || !gap_hi)) return cudaErrorInvalidValue;
  const int grid = p.n_regions * p.n_chunks;
#define CMB_ARGS p, y_slots, n_pairs, y_out, y_base, corr32, gap_hi, lead_hi, ctl, y_base ? y_out2 : nullptr
  if (p.fmt == 1)
    k_pred_combine<float><<<grid, kBlock, 0, s>>>(CMB_ARGS);
  else if (p.fmt == 2)
    k_pred_combine<float2><<<grid, kBlock, 0, s>>>(CMB_ARGS);
  else if (p.fmt == 3)
    k_pred_combine<SnapHL><<<grid, kBlock, 0, s>>>(CMB_ARGS);
  else
    k_pred_combine<double><<<grid, kBlock, 0, s>>>(CMB_ARGS);
#undef CMB_ARGS
  return cudaGetLastError();
}

cudaError_t launch_pred_combine2(const PredView& p, const int* y_slots, int n_pairs, double* y_out, const double* w2,
                                 double* y2, cudaStream_t s) {
  if (p.n_regions == 0 || n_pairs <= 0) return cudaSuccess;
  const int grid = p.n_regions * p.n_chunks;
  if (p.fmt == 1)
    k_pred_combine2<float><<<grid, kBlock, 0, s>>>(p, y_slots, n_pairs, y_out, w2, y2);
  else if (p.fmt == 2)
    k_pred_combine2<float2><<<grid, kBlock, 0, s>>>(p, y_slots, n_pairs, y_out, w2, y2);
  else if (p.fmt == 3)
    k_pred_combine2<SnapHL><<<grid, kBlock, 0, s>>>(p, y_slots, n_pairs, y_out, w2, y2);
  else
    k_pred_combine2<double><<<grid, kBlock, 0, s>>>(p, y_slots, n_pairs, y_out, w2, y2);
  return cudaGetLastError();
}

}  // namespace fem
