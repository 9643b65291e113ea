// The paper's heterogeneous predictor (Algorithm 3, Section 2.2): the data-driven correction of one case set
// is computed on the host CPU from a host copy of its stored corrections, while the GPU solves the other case
// set; the number of stored pairs s is adjusted as the run goes so that the CPU's prediction time matches the
// GPU's solve time (Section 3.2, and the step-selection of Section 3.3).
//
// Per group (case set) the host keeps the snapshot ring in pinned memory ([n_slots][N][3][r] FP64), the
// per-(region, case) Gram of the stored corrections, and the prepared correction of the group's next step.
// After each step the GPU's new correction e^it is copied to the host; a worker thread then computes the Gram
// entries the next prediction needs and does not have yet (the new slot against the s pairs in use, and any
// older pair a grown s brings in), solves the least-squares problem of the next step per region (pivot-free
// Cholesky of the Gram with the column-drop rule, as the GPU predictor does) and combines the correction
// y = Y c, which the next step uploads.  The arithmetic is FP64 throughout.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <future>
#include <thread>
#include <vector>

#include "fem_internal.cuh"

namespace fem {

struct HostPred {
  int64_t n = 0;                 // values per vector (N * 3 * rpad)
  int rpad = 0, n_slots = 0, s_max = 0, R = 0, fmt = 0, threads = 1;
  double tau = 1e-6;
  std::vector<int32_t> lo, hi;   // region node ranges
  double* ring = nullptr;        // pinned [n_slots][n]
  void* stage = nullptr;         // pinned: the pushed slot as stored on the device (FP64 or double-float pairs)
  double* y = nullptr;           // pinned [n]: correction prepared for step y_step
  std::vector<double> gram;      // [R][rpad][kMaxSlots][kMaxSlots]
  std::vector<uint8_t> gvalid;   // [kMaxSlots][kMaxSlots]: the Gram entry of the slot pair is current
  std::vector<double> w_next;    // [R][rpad][kMaxSlots] coefficients of the prepared correction
  std::vector<double> w_used;    // the same for the last step that used one
  int y_step = -1, y_pairs = 0, used_pairs = 0;
  int s_cur = 0;
  double cpu_ms = 0.0, solve_ms = 0.0;   // last prediction task (wall), last GPU step of the group (wall)
  double cpu_ms_sum = 0.0, wait_ms_sum = 0.0;
  long long tasks = 0;
  cudaEvent_t ready = nullptr;
  std::future<void> task;
};

namespace {

// f(lo_r, hi_r, r) over the regions, split across the worker's threads.
template <typename F>
void for_regions(const HostPred& h, F f) {
  const int T = std::max(1, std::min(h.threads, h.R));
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t)
    th.emplace_back([&, t]() {
      for (int r = t; r < h.R; r += T) f(r);
    });
  for (int r = 0; r < h.R; r += T) f(r);
  for (auto& x : th) x.join();
}

int slot_of(const HostPred& h, int j) { return (j - 1) % h.n_slots; }   // correction e^j, j >= 1

// After step `it` pushed e^it: Gram row of the new slot, then the correction of step it + 1.
void task_body(HostPred* h, int it) {
  const auto t0 = std::chrono::steady_clock::now();
  const int sn = slot_of(*h, it);
  double* dst = h->ring + (int64_t)sn * h->n;
  const int n_e = std::min(it, h->n_slots);          // stored corrections e^{it - n_e + 1} .. e^it
  const int rp = h->rpad;
  const int n_pairs = std::max(0, std::min(h->s_cur, n_e - 1));
  std::vector<int> xs(n_pairs), ys(n_pairs);
  for (int a = 0; a < n_pairs; ++a) xs[a] = slot_of(*h, it - n_pairs + a), ys[a] = slot_of(*h, it - n_pairs + 1 + a);
  // the pushed slot's old entries are stale; the prediction needs the Gram of X and the query (Y is inside)
  for (int j = 0; j < kMaxSlots; ++j) h->gvalid[sn * kMaxSlots + j] = h->gvalid[j * kMaxSlots + sn] = 0;
  std::vector<int> need(xs);
  need.push_back(sn);
  std::vector<std::pair<int, int>> todo;
  for (size_t i = 0; i < need.size(); ++i)
    for (size_t j = i; j < need.size(); ++j)
      if (!h->gvalid[need[i] * kMaxSlots + need[j]]) todo.push_back({need[i], need[j]});
  for_regions(*h, [&](int r) {
    const int64_t b0 = (int64_t)h->lo[r] * 3 * rp, b1 = (int64_t)h->hi[r] * 3 * rp;
    // the region's part of the pushed slot into the ring (values outside every region are never read)
    if (h->fmt == 2) {
      const float* pr = static_cast<const float*>(h->stage);
      for (int64_t i = b0; i < b1; ++i) dst[i] = (double)pr[2 * i] + (double)pr[2 * i + 1];
    } else {
      std::memcpy(dst + b0, static_cast<const double*>(h->stage) + b0, sizeof(double) * (size_t)(b1 - b0));
    }
    double acc[kMaxRpad];
    for (const auto& pr : todo) {
      const double* a = h->ring + (int64_t)pr.first * h->n;
      const double* b = h->ring + (int64_t)pr.second * h->n;
      for (int c = 0; c < rp; ++c) acc[c] = 0.0;
      for (int64_t i = b0; i < b1; i += rp)
        for (int c = 0; c < rp; ++c) acc[c] += a[i + c] * b[i + c];
      for (int c = 0; c < rp; ++c) {
        double* G = h->gram.data() + ((int64_t)r * rp + c) * kMaxSlots * kMaxSlots;
        G[pr.first * kMaxSlots + pr.second] = acc[c];
        G[pr.second * kMaxSlots + pr.first] = acc[c];
      }
    }
    // least squares per case: X^T X w = X^T x (query x = e^it), right-looking Cholesky with the drop rule
    for (int c = 0; c < rp; ++c) {
      double* wo = h->w_next.data() + ((int64_t)r * rp + c) * kMaxSlots;
      for (int a = 0; a < kMaxSlots; ++a) wo[a] = 0.0;
      if (n_pairs == 0) continue;
      const double* G = h->gram.data() + ((int64_t)r * rp + c) * kMaxSlots * kMaxSlots;
      double L[kMaxSlots][kMaxSlots], ip[kMaxSlots], rhs[kMaxSlots], d0[kMaxSlots];
      for (int i = 0; i < n_pairs; ++i) {
        for (int k = 0; k < n_pairs; ++k) L[i][k] = G[xs[i] * kMaxSlots + xs[k]];
        rhs[i] = G[xs[i] * kMaxSlots + sn];
        d0[i] = G[xs[i] * kMaxSlots + xs[i]];
      }
      for (int j = 0; j < n_pairs; ++j) {
        const double djj = L[j][j];
        const bool keep = d0[j] > 0.0 && djj > h->tau * h->tau * d0[j] && std::isfinite(djj);
        ip[j] = keep ? 1.0 / std::sqrt(djj) : 0.0;
        for (int i = j + 1; i < n_pairs; ++i) L[i][j] = keep ? L[i][j] * ip[j] : 0.0;
        L[j][j] = keep ? djj * ip[j] : 0.0;
        if (keep)
          for (int i = j + 1; i < n_pairs; ++i)
            for (int k = j + 1; k <= i; ++k) L[i][k] -= L[i][j] * L[k][j];
      }
      double yv[kMaxSlots];
      for (int j = 0; j < n_pairs; ++j) {     // L y = rhs
        double v = rhs[j];
        for (int k = 0; k < j; ++k) v -= L[j][k] * yv[k];
        yv[j] = ip[j] != 0.0 ? v * ip[j] : 0.0;
      }
      for (int j = n_pairs - 1; j >= 0; --j) {   // L^T w = y
        double v = yv[j];
        for (int k = j + 1; k < n_pairs; ++k) v -= L[k][j] * wo[k];
        wo[j] = ip[j] != 0.0 ? v * ip[j] : 0.0;
      }
    }
    // y = Y w over the region (values outside every region stay zero)
    for (int64_t i = b0; i < b1; ++i) h->y[i] = 0.0;
    for (int a = 0; a < n_pairs; ++a) {
      const double* ya = h->ring + (int64_t)ys[a] * h->n;
      double wa[kMaxRpad];
      for (int c = 0; c < rp; ++c) wa[c] = h->w_next[((int64_t)r * rp + c) * kMaxSlots + a];
      for (int64_t i = b0; i < b1; i += rp)
        for (int c = 0; c < rp; ++c) h->y[i + c] += wa[c] * ya[i + c];
    }
  });
  for (const auto& pr : todo) h->gvalid[pr.first * kMaxSlots + pr.second] = h->gvalid[pr.second * kMaxSlots + pr.first] = 1;
  h->y_step = it + 1;
  h->y_pairs = n_pairs;
  h->cpu_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->cpu_ms_sum += h->cpu_ms;
  h->tasks += 1;
}

}  // namespace

cudaError_t hostpred_create(int64_t n, int rpad, int n_slots, int s_max, int fmt, double tau,
                            const std::vector<int32_t>& lo, const std::vector<int32_t>& hi, HostPred** out) {
  HostPred* h = new HostPred();
  h->n = n, h->rpad = rpad, h->n_slots = n_slots, h->s_max = s_max, h->fmt = fmt, h->tau = tau;
  h->R = (int)lo.size();
  h->lo = lo, h->hi = hi;
  h->s_cur = s_max;
  h->threads = std::max(1, std::min(64, (int)std::thread::hardware_concurrency()));
  h->gram.assign((size_t)h->R * rpad * kMaxSlots * kMaxSlots, 0.0);
  h->gvalid.assign((size_t)kMaxSlots * kMaxSlots, 0);
  h->w_next.assign((size_t)h->R * rpad * kMaxSlots, 0.0);
  h->w_used.assign((size_t)h->R * rpad * kMaxSlots, 0.0);
  cudaError_t e = cudaMallocHost((void**)&h->ring, sizeof(double) * (size_t)n * n_slots);
  if (e == cudaSuccess) e = cudaMallocHost(&h->stage, sizeof(double) * (size_t)n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->y, sizeof(double) * (size_t)n);
  if (e == cudaSuccess) std::memset(h->y, 0, sizeof(double) * (size_t)n);   // values outside every region stay 0
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ready, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    hostpred_destroy(h);
    return e;
  }
  *out = h;
  return cudaSuccess;
}

void hostpred_destroy(HostPred* h) {
  if (!h) return;
  if (h->task.valid()) h->task.wait();
  if (h->ring) cudaFreeHost(h->ring);
  if (h->stage) cudaFreeHost(h->stage);
  if (h->y) cudaFreeHost(h->y);
  if (h->ready) cudaEventDestroy(h->ready);
  delete h;
}

// After step `it` of the group: copy the pushed device slot to the host (ordered on s), then start the
// prediction task of step it + 1.  s is first adjusted from the last prediction and solve times.
cudaError_t hostpred_push(HostPred* h, const void* dev_slot, int it, double solve_ms, cudaStream_t s) {
  if (h->task.valid()) h->task.wait();
  h->solve_ms = solve_ms;
  if (h->tasks > 0) {   // balance: the prediction should take about as long as the solve it overlaps
    if (h->cpu_ms > solve_ms && h->s_cur > 1) h->s_cur -= 1;
    else if (h->cpu_ms < 0.7 * solve_ms && h->s_cur < h->s_max) h->s_cur += 1;
  }
  const size_t bytes = (h->fmt == 2 ? 2 * sizeof(float) : sizeof(double)) * (size_t)h->n;
  cudaError_t e = cudaMemcpyAsync(h->stage, dev_slot, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->ready, s);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev = h->ready;
  h->task = std::async(std::launch::async, [h, it, ev]() {
    cudaEventSynchronize(ev);
    task_body(h, it);
  });
  return cudaSuccess;
}

// The prepared correction of step `it` (waits for the task): host pointer and pair count, or nullptr if none.
const double* hostpred_take(HostPred* h, int it, int* n_pairs) {
  if (h->task.valid()) {
    const auto t0 = std::chrono::steady_clock::now();
    h->task.wait();
    h->task.get();
    h->wait_ms_sum += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  *n_pairs = 0;
  if (h->y_step != it || h->y_pairs == 0) return nullptr;
  *n_pairs = h->y_pairs;
  h->used_pairs = h->y_pairs;
  h->w_used = h->w_next;
  return h->y;
}

void hostpred_stats(const HostPred* h, int* s_cur, double* cpu_ms, double* solve_ms, double* cpu_sum, double* wait_sum,
                    long long* tasks) {
  *s_cur = h->s_cur, *cpu_ms = h->cpu_ms, *solve_ms = h->solve_ms, *cpu_sum = h->cpu_ms_sum,
  *wait_sum = h->wait_ms_sum, *tasks = h->tasks;
}

const double* hostpred_coefficients(const HostPred* h, int* n_pairs) {
  *n_pairs = h->used_pairs;
  return h->w_used.data();
}

}  // namespace fem
