// Absorbing side boundaries and random impulse loads (the paper's inputs and boundary treatment, Section 3.1).
//
// Absorbing boundaries: viscous dashpots of Lysmer and Kuhlemeyer on the boundary faces the caller lists (the
// paper applies absorbing boundary conditions to the sides of the domain).  Their damping
// C_b is one symmetric 3x3 block per boundary node, (area / 3) rho (c_p n n^T + c_s (I - n n^T)) summed over
// the node's faces, so it enters the Newmark system A = 4M/dt^2 + 2C/dt + K as (2/dt) C_b and the right-hand
// side as C_b v (Section 3.1, Eq. GE:DIS with C = a0 M + a1 K + C_b).  These kernels apply it to the few
// boundary nodes of a vector after the dense element-by-element work.
#include "fem_internal.cuh"

namespace fem {

namespace {

// q[node] (+)= coef C_b[node] p[node] for every listed boundary node and case, free DOFs only.  With DOT the
// per-case sum of p . (coef C_b p) is reduced and the last block adds it to the product's p^T q (and to the CG
// step length, as the element-by-element product's tail does).  With ctl (graph steps) p and q may come from
// the 4-deep history rings at the step read from ctl.
template <typename T, bool DOT>
__global__ void __launch_bounds__(kVecBlock) k_dashpot(int nb, const int32_t* __restrict__ node,
                                                       const T* __restrict__ cb, int rpad, int rshift, T coef,
                                                       const T* p, T* q, bool assign, const uint8_t* __restrict__ fm,
                                                       Ring4 pring, int poff, Ring4 qring, int qoff,
                                                       const StepCtl* ctl, Reducer red, CgCase* sc, double* ptq_out,
                                                       const int* gate) {
  if (gate && *gate == 0) return;
  if (ctl) {
    if (pring.p[0]) p = reinterpret_cast<const T*>(pring.p[(ctl->it + poff) & 3]);
    if (qring.p[0]) q = reinterpret_cast<T*>(qring.p[(ctl->it + qoff) & 3]);
  }
  double dot = 0.0;
  const int64_t total = (int64_t)nb << rshift;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i >> rshift);
    const int c = (int)(i & (rpad - 1));
    const int64_t n = node[b];
    const T* C = cb + (int64_t)b * 6;   // xx yy zz xy xz yz
    const uint8_t f = fm[n];
    const int64_t id = n * 3 * rpad + c;
    const T p0 = dof_free(f, 0) ? p[id] : (T)0, p1 = dof_free(f, 1) ? p[id + rpad] : (T)0,
            p2 = dof_free(f, 2) ? p[id + 2 * rpad] : (T)0;
    const T t[3] = {coef * (C[0] * p0 + C[3] * p1 + C[4] * p2), coef * (C[3] * p0 + C[1] * p1 + C[5] * p2),
                    coef * (C[4] * p0 + C[5] * p1 + C[2] * p2)};
    const T pv[3] = {p0, p1, p2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!dof_free(f, k)) continue;
      T* d = q + id + k * rpad;
      *d = assign ? t[k] : *d + t[k];
      if (DOT) dot += (double)pv[k] * (double)t[k];
    }
  }
  if constexpr (DOT) {
    double vals[1] = {dot};
    if (block_reduce_last<1>(vals, rpad, red) && threadIdx.x < rpad) {
      const int c = threadIdx.x;
      const double extra = red.out[c];
      if (ptq_out) ptq_out[c] += extra;
      if (sc) {
        CgCase& s = sc[c];
        s.pq += extra;
        if (s.active) {
          if (!(s.pq > 0.0) || !isfinite(s.pq)) {
            s.active = 0;
            s.status = FEM_ERR_BREAKDOWN;
            s.alpha = 0.0;
          } else {
            s.alpha = s.rho / s.pq;
          }
        }
      }
    }
  }
}

int lg2(int r) {
  int s = 0;
  while ((1 << s) < r) ++s;
  return s;
}

__global__ void k_add_node_blocks(int nb, const int32_t* __restrict__ node, const double* __restrict__ cb, double coef,
                                  double* __restrict__ D) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb * 6; i += gridDim.x * blockDim.x)
    D[(int64_t)node[i / 6] * 6 + i % 6] += coef * cb[i];
}

// Random impulse loads: a one-step force per entry, added in its step (entries of a step are contiguous).
// Two entries of one step may share a node and lane: atomic adds.
__global__ void k_impulses(Impulses im, int rpad, int it, const StepCtl* ctl, const uint8_t* __restrict__ fm,
                           double* __restrict__ b) {
  if (ctl) it = ctl->it;
  if (it < 1 || it > im.last) return;
  const int e0 = im.off[it], e1 = im.off[it + 1];
  for (int e = e0 + blockIdx.x * blockDim.x + threadIdx.x; e < e1; e += gridDim.x * blockDim.x) {
    const int64_t n = im.node[e];
    const uint8_t f = fm[n];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (dof_free(f, k)) atomicAdd(b + (n * 3 + k) * rpad + im.lane[e], im.f[3 * (int64_t)e + k]);
  }
}

}  // namespace

cudaError_t launch_add_node_blocks(const Absorb& ab, double coef, double* D, cudaStream_t s) {
  if (ab.nb == 0) return cudaSuccess;
  k_add_node_blocks<<<grid_for((int64_t)ab.nb * 6), kBlock, 0, s>>>(ab.nb, ab.node, ab.c64, coef, D);
  return cudaGetLastError();
}

cudaError_t launch_impulses(const Impulses& im, int rpad, int it, const StepCtl* ctl, const uint8_t* fm, double* b,
                            cudaStream_t s) {
  if (im.n == 0) return cudaSuccess;
  const int grid = (im.max_per_step + kBlock - 1) / kBlock;
  k_impulses<<<grid < 1 ? 1 : grid, kBlock, 0, s>>>(im, rpad, it, ctl, fm, b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dashpot(const Absorb& ab, int rpad, double coef, const T* p, T* q, bool assign,
                           const uint8_t* fm, const Reducer* red, CgCase* sc, double* ptq_out, const int* gate,
                           cudaStream_t s, Ring4 pring, int poff, Ring4 qring, int qoff, const StepCtl* ctl) {
  if (ab.nb == 0) return cudaSuccess;
  const T* cb = sizeof(T) == 8 ? reinterpret_cast<const T*>(ab.c64) : reinterpret_cast<const T*>(ab.c32);
  const int rs = lg2(rpad);
  const int64_t items = (int64_t)ab.nb << rs;
  int grid = (int)std::min<int64_t>((items + kVecBlock - 1) / kVecBlock, vec_grid_cap());
  if (grid < 1) grid = 1;
  if (red) {
    k_dashpot<T, true><<<grid, kVecBlock, 0, s>>>(ab.nb, ab.node, cb, rpad, rs, (T)coef, p, q, assign, fm, pring,
                                                   poff, qring, qoff, ctl, *red, sc, ptq_out, gate);
  } else {
    k_dashpot<T, false><<<grid, kVecBlock, 0, s>>>(ab.nb, ab.node, cb, rpad, rs, (T)coef, p, q, assign, fm, pring,
                                                    poff, qring, qoff, ctl, Reducer{nullptr, nullptr, nullptr},
                                                    nullptr, nullptr, gate);
  }
  return cudaGetLastError();
}
template cudaError_t launch_dashpot<float>(const Absorb&, int, double, const float*, float*, bool, const uint8_t*,
                                           const Reducer*, CgCase*, double*, const int*, cudaStream_t, Ring4, int,
                                           Ring4, int, const StepCtl*);
template cudaError_t launch_dashpot<double>(const Absorb&, int, double, const double*, double*, bool, const uint8_t*,
                                            const Reducer*, CgCase*, double*, const int*, cudaStream_t, Ring4, int,
                                            Ring4, int, const StepCtl*);

}  // namespace fem
