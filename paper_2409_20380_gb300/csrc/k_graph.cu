// Device-side control of a time step captured as one CUDA graph: the step record (step counter, time,
// predictor slots) and the conditions of the graph's loops.  The loops are those of the FP32-inner /
// FP64-certified solve: refinement passes (while any case is above tolerance), the inner PCG (while any
// case iterates).  Every decision the host would take between launches is taken here, so a step runs
// without a host round trip.
#include "fem_internal.cuh"

namespace fem {

namespace {

__device__ __forceinline__ int slot_of_d(int j, int n_slots) { return (j - 1) % n_slots; }

// it += 1 and everything that depends on it (one thread).
__global__ void k_step_begin(StepCtl* ctl, int n_slots, int s_max, double dt, int dd, long long n_fixed) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int it = ctl->it + 1;
  ctl->it = it;
  ctl->t = it * dt;
  int n_pairs = 0;
  if (dd && n_slots > 0) {
    const int n_e = min(it - 1, n_slots);
    n_pairs = min(s_max, n_e - 1);
    if (n_pairs < 0) n_pairs = 0;
  }
  ctl->n_pairs = n_pairs;
  for (int a = 0; a < kMaxSlots; ++a) {
    ctl->xs[a] = a < n_pairs ? slot_of_d(it - 1 - n_pairs + a, n_slots) : 0;
    ctl->ys[a] = a < n_pairs ? slot_of_d(it - n_pairs + a, n_slots) : 0;
  }
  ctl->slot_query = (n_slots > 0 && it >= 2) ? slot_of_d(it - 1, n_slots) : 0;
  ctl->slot_new = n_slots > 0 ? slot_of_d(it, n_slots) : 0;
  unsigned long long mask = 0ull;
  if (n_slots > 0) {
    const int n_e = min(it, n_slots);
    for (int j = it - n_e + 1; j <= it; ++j) mask |= 1ull << slot_of_d(j, n_slots);
  }
  ctl->mask = mask;
  ctl->pass = 0;
  ctl->issued = 0;
  ctl->launches += n_fixed;
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, unsigned value) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, value);
}

// Start of a refinement pass: cases still above tolerance after maxit inner iterations in total (or in the
// last allowed pass) are given up as not converged; the inner solve runs if any case is active.
__global__ void k_pass_begin(CgCase* outer, int ncase, int* n_active, int maxit, int max_pass, StepCtl* ctl,
                             cudaGraphConditionalHandle h_if, long long n_if) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int used = 0;
  for (int c = 0; c < ncase; ++c) used = max(used, outer[c].iters);
  int na = *n_active;
  if (na > 0 && (used >= maxit || ctl->pass == max_pass - 1)) {
    for (int c = 0; c < ncase; ++c)
      if (outer[c].active) outer[c].status = FEM_ERR_NOT_CONVERGED, outer[c].active = 0;
    na = 0;
    *n_active = 0;
  }
  if (na > 0) ctl->launches += n_if;
  cudaGraphSetConditional(h_if, na > 0 ? 1u : 0u);
}

__global__ void k_inner_start(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->issued = 0;
  cudaGraphSetConditional(h, *n_active > 0 ? 1u : 0u);
}

// Start of one of a pass's two inner loops (FP16 tensor-core products, want_tc 1; FP32 products, 0): the pass
// takes the tensor-core product only if every active case's reduction target is at least `floor`; the loop
// of the other product is skipped.
__global__ void k_inner_start_sel(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h,
                                  const CgCase* outer, int ncase, double floor, int want_tc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool tc = true;
  for (int c = 0; c < ncase; ++c)
    if (outer[c].active && outer[c].inner_tol < floor) tc = false;
  ctl->issued = 0;
  cudaGraphSetConditional(h, (*n_active > 0 && tc == (want_tc != 0)) ? 1u : 0u);
}

// After a chunk of inner iterations: continue while a case iterates, up to the issue limit.
__global__ void k_inner_cond(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, int chunk, int limit,
                             long long n_body) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->issued += chunk;
  ctl->launches += n_body;
  cudaGraphSetConditional(h, (*n_active > 0 && ctl->issued <= limit) ? 1u : 0u);
}

__global__ void k_pass_end(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, int max_pass,
                           long long n_body) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->pass += 1;
  ctl->launches += n_body;
  cudaGraphSetConditional(h, (*n_active > 0 && ctl->pass < max_pass) ? 1u : 0u);
}

// Per-case statistics of the step added to the accumulators the host reads after the last step.
__global__ void k_step_end(const CgCase* outer, int ncase, int* acc_iters, double* acc_relres, int* acc_status,
                           StepCtl* ctl) {
  for (int c = threadIdx.x; c < ncase; c += blockDim.x) {
    const CgCase& o = outer[c];
    acc_iters[c] += o.iters;
    acc_relres[c] = fmax(acc_relres[c], o.relres);
    if (o.status != FEM_OK && (acc_status[c] == FEM_OK || o.status < acc_status[c])) acc_status[c] = o.status;
  }
  if (threadIdx.x == 0) ctl->use_ext = 0;
}

}  // namespace

cudaError_t launch_step_begin(StepCtl* ctl, int n_slots, int s_max, double dt, int dd, long long n_fixed,
                              cudaStream_t s) {
  k_step_begin<<<1, 32, 0, s>>>(ctl, n_slots, s_max, dt, dd, n_fixed);
  return cudaGetLastError();
}

cudaError_t launch_set_cond(cudaGraphConditionalHandle h, unsigned value, cudaStream_t s) {
  k_set_cond<<<1, 32, 0, s>>>(h, value);
  return cudaGetLastError();
}

cudaError_t launch_pass_begin(CgCase* outer, int ncase, int* n_active, int maxit, int max_pass, StepCtl* ctl,
                              cudaGraphConditionalHandle h_if, long long n_if, cudaStream_t s) {
  k_pass_begin<<<1, 32, 0, s>>>(outer, ncase, n_active, maxit, max_pass, ctl, h_if, n_if);
  return cudaGetLastError();
}

cudaError_t launch_inner_start(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, cudaStream_t s) {
  k_inner_start<<<1, 32, 0, s>>>(n_active, ctl, h);
  return cudaGetLastError();
}

cudaError_t launch_inner_start_sel(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h,
                                   const CgCase* outer, int ncase, double floor, int want_tc, cudaStream_t s) {
  k_inner_start_sel<<<1, 32, 0, s>>>(n_active, ctl, h, outer, ncase, floor, want_tc);
  return cudaGetLastError();
}

cudaError_t launch_inner_cond(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, int chunk, int limit,
                              long long n_body, cudaStream_t s) {
  k_inner_cond<<<1, 32, 0, s>>>(n_active, ctl, h, chunk, limit, n_body);
  return cudaGetLastError();
}

cudaError_t launch_pass_end(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, int max_pass,
                            long long n_body, cudaStream_t s) {
  k_pass_end<<<1, 32, 0, s>>>(n_active, ctl, h, max_pass, n_body);
  return cudaGetLastError();
}

cudaError_t launch_step_end(const CgCase* outer, int ncase, int* acc_iters, double* acc_relres, int* acc_status,
                            StepCtl* ctl, cudaStream_t s) {
  k_step_end<<<1, 128, 0, s>>>(outer, ncase, acc_iters, acc_relres, acc_status, ctl);
  return cudaGetLastError();
}

}  // namespace fem
