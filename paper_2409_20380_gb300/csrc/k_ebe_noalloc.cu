// Allocation-free variant of the EBE product with its fused p^T q reduction.
//
// fem_ebe_apply() takes the scratch of its grid reduction (per-block partial sums, final sums, the
// last-block counter) from a workspace the library allocates with cudaMalloc on first use.  Some callers
// cannot allow that: code whose memory is owned by another allocator under a fixed budget, and
// latency-critical loops that cannot afford the implicit device synchronisation of cudaMalloc/cudaFree.
// fem_ebe_apply_noalloc() serves them: its scratch is the file-scope device array below, which exists
// once per GPU that loads the library and lives until the process exits.  It always runs the generic
// element kernel (one thread per element and case, global atomics): the tiled kernels fem_ebe_apply
// chooses keep per-mesh tile tables and tuning state that are built with allocations.  Its results equal
// fem_ebe_apply's to rounding (the FP32 atomic scatter order varies), not bit for bit.
#include <mutex>

#include "fem_internal.cuh"

namespace fem {

// Layout of the scratch: kMaxRedBlocks x kMaxRpad per-block partials, kMaxRpad final sums, one counter.
constexpr size_t kNaPartialBytes = sizeof(double) * (size_t)kMaxRedBlocks * kMaxRpad;
constexpr size_t kNaOutBytes = 256;                       // kMaxRpad doubles, padded to 256 bytes
constexpr size_t kNaCounterBytes = 256;
constexpr size_t kNaScratchBytes = kNaPartialBytes + kNaOutBytes + kNaCounterBytes;   // 311,808 bytes
static_assert(sizeof(double) * kMaxRpad <= kNaOutBytes, "final sums must fit their slot");

static __device__ __align__(256) unsigned char g_ebe_scratch[kNaScratchBytes];

constexpr int kNaMaxDevices = 64;
static std::mutex g_na_mu;
static void* g_na_addr[kNaMaxDevices];   // device address of g_ebe_scratch, per device (set up once)

// Device address of the scratch on the current device.  The host-side name g_ebe_scratch is only a
// stand-in: the address has to come from cudaGetSymbolAddress, once per device, with that device current.
static cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_ebe_scratch);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = p;
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_ebe_apply_noalloc(fem_mesh* m, int precision, const void* p_dev, void* q_dev, int n_rhs,
                                            double alpha_M, double alpha_K, double* ptq_dev, void* stream) {
  clear_error();
  if (!m || !p_dev || !q_dev) return set_error(FEM_ERR_ARG, "fem_ebe_apply_noalloc: null argument");
  if (!(n_rhs == 1 || n_rhs == 2 || n_rhs == 4 || n_rhs == 8 || n_rhs == 16 || n_rhs == 32))
    return set_error(FEM_ERR_ARG, "fem_ebe_apply_noalloc: n_rhs must be 1, 2, 4, 8, 16 or 32 (the scratch holds "
                                  "partial sums for at most 32 cases)");
  if (precision != FEM_FP64 && precision != FEM_FP32_INNER)
    return set_error(FEM_ERR_ARG, "fem_ebe_apply_noalloc: unknown precision");
  MeshView mv;
  int mesh_dev = 0;
  const int32_t* conn10 = nullptr;
  mesh_view_of(m, &mv, &mesh_dev, &conn10);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FEM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != mesh_dev)
    return set_error(FEM_ERR_ARG, "fem_ebe_apply_noalloc: the mesh's device must be the current device");
  if (dev < 0 || dev >= kNaMaxDevices) return set_error(FEM_ERR_ARG, "fem_ebe_apply_noalloc: device id too large");
  cudaStream_t s = (cudaStream_t)stream;
  Reducer red{nullptr, nullptr, nullptr};
  if (ptq_dev) {
    void* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess)
      return set_error(FEM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned char* b = (unsigned char*)base;
    red.partial = (double*)b;
    red.out = (double*)(b + kNaPartialBytes);
    red.counter = (unsigned*)(b + kNaPartialBytes + kNaOutBytes);
    // the last-block counter must start at zero (the scratch keeps whatever the previous call left)
    e = cudaMemsetAsync(red.counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return set_error(FEM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  if (conn10) {   // quadratic tets: their element kernel (the same scratch bound on the reduction's blocks)
    e = precision == FEM_FP64
            ? launch_ebe10_gated<double>(mv.E, mv.N, n_rhs, conn10, mv.rec32, mv.rec64, mv.freemask,
                                         (const double*)p_dev, nullptr, (double*)q_dev, alpha_M, alpha_K,
                                         ptq_dev ? &red : nullptr, nullptr, ptq_dev, nullptr, s)
            : launch_ebe10_gated<float>(mv.E, mv.N, n_rhs, conn10, mv.rec32, mv.rec64, mv.freemask,
                                        (const float*)p_dev, nullptr, (float*)q_dev, alpha_M, alpha_K,
                                        ptq_dev ? &red : nullptr, nullptr, ptq_dev, nullptr, s);
  } else if (precision == FEM_FP64) {
    e = launch_ebe<double>(mv, n_rhs, (const double*)p_dev, nullptr, (double*)q_dev, alpha_M, alpha_K,
                           ptq_dev ? &red : nullptr, nullptr, ptq_dev, s);
    if (e == cudaSuccess) e = launch_mask<double>(mv.N, n_rhs, mv.freemask, (double*)q_dev, s);
  } else {
    e = launch_ebe<float>(mv, n_rhs, (const float*)p_dev, nullptr, (float*)q_dev, alpha_M, alpha_K,
                          ptq_dev ? &red : nullptr, nullptr, ptq_dev, s);
    if (e == cudaSuccess) e = launch_mask<float>(mv.N, n_rhs, mv.freemask, (float*)q_dev, s);
  }
  if (e != cudaSuccess) return set_error(FEM_ERR_CUDA, std::string("fem_ebe_apply_noalloc: ") + cudaGetErrorString(e));
  return FEM_OK;
}
