// libfem C-ABI: host runtime around the kernels -- mesh setup, the PCG drivers (FP64 and FP32-inner /
// FP64-refined), and the batched time stepping of many cases (Section 3.1 time loop with the predictor
// of Section 3.2 and the solver of Algorithm 1; cases on one mesh form one multi-RHS system, Eq. eqmebefem).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fem_internal.cuh"

#include <array>
#include <unordered_map>

using namespace fem;


static thread_local std::string g_err;

static fem_status fail(fem_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(FEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CHK(call)                    \
  do {                               \
    fem_status st_ = (call);         \
    if (st_ != FEM_OK) return st_;   \
  } while (0)

template <typename T>
static fem_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(FEM_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  return FEM_OK;
}

template <typename T>
static void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Bytes of one stored snapshot value per snapshot_format: FP64, FP32, double-float pair, FP32 + BF16.
static size_t snap_bytes(int fmt) { return fmt == 1 ? 4 : fmt == 3 ? 6 : 8; }

static bool pow2_rhs(int r) { return r == 1 || r == 2 || r == 4 || r == 8 || r == 16 || r == 32; }

static int next_pow2(int r) {
  int p = 1;
  while (p < r) p <<= 1;
  return p;
}

// ------------------------------------------------------------------------------------------------------
// Event-based device-time profiler (CUDA events on the working stream, resolved at sync points).
// ------------------------------------------------------------------------------------------------------
enum ProfClass { P_EBE32 = 0, P_EBE64, P_VEC, P_PREDICT, P_RHS, P_SOLVE, P_UPDATE, P_EBE16, P_NCLASS };

struct Prof {
  bool on = false;       // counting launches and steps
  bool events = false;   // and timing kernel classes with events (forces eager steps)
  std::vector<cudaEvent_t> all, free_ev;
  struct Pair {
    int cls;
    cudaEvent_t a, b;
    bool closed;
    bool done;
  };
  std::vector<Pair> pend;
  double ms[P_NCLASS] = {};
  long long n[P_NCLASS] = {};
  long long launches = 0;
  int steps = 0;
  ~Prof() {
    for (auto e : all) cudaEventDestroy(e);
  }
  void reset() {
    for (int i = 0; i < P_NCLASS; ++i) {
      ms[i] = 0.0;
      n[i] = 0;
    }
    launches = 0;
    steps = 0;
  }
  cudaEvent_t get() {
    if (free_ev.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      all.push_back(e);
      return e;
    }
    cudaEvent_t e = free_ev.back();
    free_ev.pop_back();
    return e;
  }
  int begin(int cls, cudaStream_t s) {
    if (!on || !events) return -1;
    Pair p{cls, get(), get(), false, false};
    cudaEventRecord(p.a, s);
    pend.push_back(p);
    return (int)pend.size() - 1;
  }
  void end(int idx, cudaStream_t s) {
    if (idx < 0 || idx >= (int)pend.size()) return;
    cudaEventRecord(pend[idx].b, s);
    pend[idx].closed = true;
  }
  // Accumulates closed pairs (the stream has been synchronised); slots are recycled once none is open.
  void resolve() {
    bool any_open = false;
    for (auto& p : pend) {
      if (p.done) continue;
      if (!p.closed) {
        any_open = true;
        continue;
      }
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        ms[p.cls] += t;
        n[p.cls] += 1;
      }
      p.done = true;
    }
    cudaGetLastError();
    if (!any_open) {
      for (auto& p : pend) {
        free_ev.push_back(p.a);
        free_ev.push_back(p.b);
      }
      pend.clear();
    }
  }
};

// ------------------------------------------------------------------------------------------------------
// PCG workspace (scratch vectors, per-case scalars, reduction buffers) for one mesh and case count.
// ------------------------------------------------------------------------------------------------------
struct Workspace {
  int rpad = 0;
  int64_t n = 0;  // N * 3 * rpad
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  float *r32 = nullptr, *x32 = nullptr, *rr32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;
  CgCase* sc = nullptr;
  CgCase* outer = nullptr;
  double* partial = nullptr;
  unsigned* counter = nullptr;
  double* out = nullptr;
  int* n_active = nullptr;
  int* h_active = nullptr;   // pinned
  CgCase* h_sc = nullptr;    // pinned
  Prof* prof = nullptr;      // not owned; null = not profiled
  bool tc = false;           // FP32 CG products of the inner solve on the tensor cores (fem_opts.inner_product)
  void count(int k = 1) {
    if (prof && prof->on) prof->launches += k;
  }
  int pbeg(int cls, cudaStream_t s) { return prof ? prof->begin(cls, s) : -1; }
  void pend(int idx, cudaStream_t s) {
    if (prof) prof->end(idx, s);
  }
  void resolve() {
    if (prof && prof->on) prof->resolve();
  }
  ~Workspace() {
    dfree(r); dfree(z); dfree(p); dfree(q);
    dfree(r32); dfree(x32); dfree(rr32); dfree(z32); dfree(p32); dfree(q32);
    dfree(sc); dfree(outer); dfree(partial); dfree(counter); dfree(out); dfree(n_active);
    if (h_active) cudaFreeHost(h_active);
    if (h_sc) cudaFreeHost(h_sc);
  }
  Reducer red() const { return Reducer{partial, counter, out}; }
};

static fem_status ws_create(int64_t N, int rpad, Workspace** out) {
  Workspace* w = new Workspace();
  w->rpad = rpad;
  w->n = N * 3 * rpad;
  fem_status st = FEM_OK;
  if (st == FEM_OK) st = dalloc(&w->r, w->n);
  if (st == FEM_OK) st = dalloc(&w->z, w->n);
  if (st == FEM_OK) st = dalloc(&w->p, w->n);
  if (st == FEM_OK) st = dalloc(&w->q, w->n);
  if (st == FEM_OK) st = dalloc(&w->r32, w->n);
  if (st == FEM_OK) st = dalloc(&w->x32, w->n);
  if (st == FEM_OK) st = dalloc(&w->rr32, w->n);
  if (st == FEM_OK) st = dalloc(&w->z32, w->n);
  if (st == FEM_OK) st = dalloc(&w->p32, w->n);
  if (st == FEM_OK) st = dalloc(&w->q32, w->n);
  if (st == FEM_OK) st = dalloc(&w->sc, kMaxCases);
  if (st == FEM_OK) st = dalloc(&w->outer, kMaxCases);
  if (st == FEM_OK) st = dalloc(&w->partial, (size_t)kMaxRedBlocks * 3 * kMaxCases);
  if (st == FEM_OK) st = dalloc(&w->counter, 1);
  if (st == FEM_OK) st = dalloc(&w->out, 3 * kMaxCases);
  if (st == FEM_OK) st = dalloc(&w->n_active, 1);
  if (st != FEM_OK) {
    delete w;
    return st;
  }
  if (cudaMallocHost((void**)&w->h_active, sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&w->h_sc, sizeof(CgCase) * kMaxCases) != cudaSuccess) {
    cudaGetLastError();
    delete w;
    return fail(FEM_ERR_OOM, "cudaMallocHost failed");
  }
  cudaMemset(w->counter, 0, sizeof(unsigned));
  cudaMemset(w->p, 0, w->n * sizeof(double));
  cudaMemset(w->p32, 0, w->n * sizeof(float));
  cudaMemset(w->sc, 0, sizeof(CgCase) * kMaxCases);
  cudaMemset(w->outer, 0, sizeof(CgCase) * kMaxCases);
  *out = w;
  return FEM_OK;
}

// ------------------------------------------------------------------------------------------------------
struct fem_mesh {
  int64_t N = 0, E = 0;
  int npe = 4;                      // nodes per element: 4 (linear tets) or 10 (quadratic tets)
  int32_t* conn10 = nullptr;        // [E][10] (npe 10): corners, then the edges (0,1) (1,2) (0,2) (0,3) (1,3) (2,3)
  fem_time_params tp{};
  double cM = 0, cK = 0;
  int device = 0;
  double* xyz = nullptr;
  int4* conn = nullptr;
  int32_t* mat = nullptr;
  double* lmr = nullptr;
  double* rec64 = nullptr;
  float* rec32 = nullptr;
  float* rec_df = nullptr;         // [E][12][2] (hi, lo) split of rec64 for double-float products
  // assembled operators of the certification product (built on first use)
  int32_t* row_ptr = nullptr;       // [N + 1] node pattern (a node's neighbours through elements, itself included)
  int32_t* col = nullptr;           // [nnz]
  int64_t nnz = 0;
  double* Kb = nullptr;             // [nnz][3][3] stiffness blocks
  double* Mb = nullptr;             // [nnz] consistent-mass entries
  float2* KMd = nullptr;            // per block: the 9 (hi, lo) pairs of Kb, then the pair of Mb (80 bytes)
  double* D = nullptr;
  double* binv64 = nullptr;
  float* binv32 = nullptr;
  uint8_t* fm = nullptr;
  int n_regions = 0;
  float* reg_cent = nullptr;        // [R][3] centroid of each region's nodes (learned-proposal features)
  float inv_extent = 1.0f;          // 1 / largest edge of the bounding box
  int32_t* reg_lo = nullptr;
  int32_t* reg_hi = nullptr;
  std::vector<int32_t> h_reg_lo, h_reg_hi;   // host copies (the host predictor)
  // nodes outside every region range: [reg_hi[R], reg_gap[R]) follows region R, [0, reg_lead) precedes all
  int32_t* reg_gap = nullptr;
  int reg_lead = 0;
  std::vector<Workspace*> ws;
  // tiled hex-patch EBE (present when the elements come in Kuhn hex patches)
  bool hex = false;
  static constexpr int kNTile = 5;
  HexTiles tiles[kNTile];          // hex_per_tile 32, 64, 128, 256, 512
  std::vector<void*> tile_bufs;
  int ebe_variant = 0;             // 0 auto, 1 generic, 2 tiled hex, 3 staged, 4 case-major, 5/6 packed staged,
                                   // 7 hex element matrices, 8 assembled 3x3 blocks (CRS-style comparator)
  float* hexmat = nullptr;         // [ceil(H / 2)][300][2] hex matrices for (cM, cK) (built on first use)
  unsigned char* hm16 = nullptr;   // [H] 784-byte FP16 hex matrices for (cM, cK) (variant 9; built on first use)
  int hex_per_tile = 0;            // 0 auto
  // autotuned choice per (FP32 / FP64 product, log2 of the case count); variant 0 = not tuned
  struct Tuned {
    int variant = 0, hpt = 0;
  } tuned[2][6];
  // host copies of the inputs (used to fuse meshes into one system) and the region map
  std::vector<double> h_xyz, h_lmr;
  std::vector<int32_t> h_conn, h_mat, h_region, h_ab_faces;
  std::vector<uint8_t> h_fixed;
  // fused meshes: case of each node
  uint8_t* seg = nullptr;
  int nseg = 0;
  // dashpots of absorbing boundary faces (fem_mesh_set_absorbing)
  Absorb ab;
  int32_t* ab_node = nullptr;
  double* ab_c64 = nullptr;
  float* ab_c32 = nullptr;
  // Node pattern (host, threads over node ranges) and GPU assembly of the certification operators.
  fem_status ensure_bcsr(cudaStream_t s) {
    if (row_ptr) return FEM_OK;
    const int64_t n_nodes = N;
    std::vector<int64_t> inc_ptr(n_nodes + 1, 0);
    for (int32_t v : h_conn) inc_ptr[v + 1] += 1;
    for (int64_t n = 0; n < n_nodes; ++n) inc_ptr[n + 1] += inc_ptr[n];
    std::vector<int32_t> inc(h_conn.size());
    {
      std::vector<int64_t> pos(inc_ptr.begin(), inc_ptr.end() - 1);
      for (size_t i = 0; i < h_conn.size(); ++i) inc[pos[h_conn[i]]++] = (int32_t)(i / npe);
    }
    const int nt = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
    std::vector<int32_t> cnt(n_nodes);
    auto neighbours = [&](int64_t n, std::vector<int32_t>& buf) {
      buf.clear();
      for (int64_t k = inc_ptr[n]; k < inc_ptr[n + 1]; ++k)
        for (int a = 0; a < npe; ++a) buf.push_back(h_conn[(size_t)npe * inc[k] + a]);
      std::sort(buf.begin(), buf.end());
      buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
      if (buf.empty()) buf.push_back((int32_t)n);     // isolated node: diagonal slot only
    };
    auto par = [&](auto body) {
      std::vector<std::thread> th;
      for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
          std::vector<int32_t> buf;
          for (int64_t n = n_nodes * t / nt; n < n_nodes * (t + 1) / nt; ++n) body(n, buf);
        });
      for (auto& x : th) x.join();
    };
    par([&](int64_t n, std::vector<int32_t>& buf) {
      neighbours(n, buf);
      cnt[n] = (int32_t)buf.size();
    });
    std::vector<int32_t> rp(n_nodes + 1, 0);
    int64_t total = 0;
    for (int64_t n = 0; n < n_nodes; ++n) {
      rp[n] = (int32_t)total;
      total += cnt[n];
      if (total > INT32_MAX) return fail(FEM_ERR_ARG, "assembled pattern exceeds 2^31 entries");
    }
    rp[n_nodes] = (int32_t)total;
    std::vector<int32_t> cl(total);
    par([&](int64_t n, std::vector<int32_t>& buf) {
      neighbours(n, buf);
      std::copy(buf.begin(), buf.end(), cl.begin() + rp[n]);
    });
    int* missing = nullptr;
    fem_status st = FEM_OK;
    if (st == FEM_OK) st = dalloc(&row_ptr, (size_t)n_nodes + 1);
    if (st == FEM_OK) st = dalloc(&col, (size_t)total);
    if (st == FEM_OK) st = dalloc(&Kb, 9 * (size_t)total);
    if (st == FEM_OK) st = dalloc(&Mb, (size_t)total);
    if (st == FEM_OK) st = dalloc(&KMd, 10 * (size_t)total);
    if (st == FEM_OK) st = dalloc(&missing, 1);
    if (st != FEM_OK) {
      dfree(row_ptr); dfree(col); dfree(Kb); dfree(Mb); dfree(KMd); dfree(missing);
      return st;
    }
    nnz = total;
    int h_missing = 0;
    cudaError_t e = cudaMemcpyAsync(row_ptr, rp.data(), sizeof(int32_t) * (n_nodes + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(col, cl.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = npe == 10 ? launch_bcsr_assemble10(E, conn10, rec64, row_ptr, col, nnz, Kb, Mb, KMd, missing, s)
                    : launch_bcsr_assemble(view(), row_ptr, col, nnz, Kb, Mb, KMd, missing, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_missing, missing, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(missing);
    if (e != cudaSuccess || h_missing) {
      cudaGetLastError();
      dfree(row_ptr); dfree(col); dfree(Kb); dfree(Mb); dfree(KMd);
      row_ptr = nullptr;
      nnz = 0;
      return fail(e != cudaSuccess ? FEM_ERR_CUDA : FEM_ERR_ARG,
                  e != cudaSuccess ? std::string("assembly: ") + cudaGetErrorString(e) : "assembly: missing pattern slot");
    }
    return FEM_OK;
  }
  MeshView view() const { return MeshView{N, E, conn, rec64, rec32, binv64, binv32, fm, seg, nseg}; }
  // Hex element matrices for the mesh's own coefficients (cM, cK); built outside stream capture only.
  fem_status ensure_hexmat(cudaStream_t s) {
    if (hexmat || !hex) return FEM_OK;
    const int64_t H = E / 6;
    float* buf = nullptr;
    CHK(dalloc(&buf, (size_t)2 * kHexMatVals * (size_t)((H + 1) / 2)));
    cudaError_t e = launch_hexmat_build(H, rec64, cM, cK, buf, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      dfree(buf);
      return fail(FEM_ERR_CUDA, std::string("hex matrices: ") + cudaGetErrorString(e));
    }
    hexmat = buf;
    return FEM_OK;
  }
  fem_status ensure_hm16(cudaStream_t s) {
    if (hm16 || !hex) return FEM_OK;
    const int64_t H = E / 6;
    unsigned char* buf = nullptr;
    CHK(dalloc(&buf, (size_t)kHm16RecBytes * (size_t)H));
    cudaError_t e = launch_hexmat16_build(H, rec64, cM, cK, buf, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      dfree(buf);
      return fail(FEM_ERR_CUDA, std::string("FP16 hex matrices: ") + cudaGetErrorString(e));
    }
    hm16 = buf;
    return FEM_OK;
  }
  ~fem_mesh() {
    dfree(xyz); dfree(conn); dfree(conn10); dfree(mat); dfree(lmr); dfree(rec64); dfree(rec32); dfree(rec_df); dfree(D);
    dfree(row_ptr); dfree(col); dfree(Kb); dfree(Mb); dfree(KMd); dfree(hexmat); dfree(hm16);
    dfree(binv64); dfree(binv32); dfree(fm); dfree(reg_lo); dfree(reg_hi); dfree(reg_gap); dfree(seg); dfree(reg_cent);
    dfree(ab_node); dfree(ab_c64); dfree(ab_c32);
    for (auto* w : ws) delete w;
    for (void* b : tile_bufs) cudaFree(b);
  }
  // Tiling for a product on T with rpad cases: the largest tile whose accumulator fits the budget.
  // EBE implementation of a product on elements of elem_bytes with rpad cases: an explicit fem_mesh_tune
  // setting wins, else the autotuned choice for this precision and case count, else the staged tiled hex
  // kernel (two cases per thread for FP32 products) when the mesh has hex patches.
  void resolve(size_t elem_bytes, int rpad, int* variant, int* hpt) const {
    *variant = ebe_variant, *hpt = hex_per_tile;
    if (*variant == 0 && *hpt == 0) {
      int lg = 0;
      while ((1 << lg) < rpad && lg < 5) ++lg;
      const Tuned& t = tuned[elem_bytes == 4 ? 0 : 1][lg];
      if (t.variant) *variant = t.variant, *hpt = t.hpt;
    }
    if (*variant == 0) *variant = hex ? 5 : 1;       // packed staged tiles where they apply (else 3, 2, 1)
    if (!hex && *variant != 8) *variant = 1;
  }
  // Tiling for the resolved variant: the largest tile whose shared memory fits (or the requested size).
  const HexTiles* tiles_for(size_t elem_bytes, int rpad, int variant, int hpt) const {
    if (!hex || variant == 1) return nullptr;
    const HexTiles* best = nullptr;
    for (int i = 0; i < kNTile; ++i) {
      const HexTiles& t = tiles[i];
      if (t.n_tiles == 0) continue;
      if (hpt && t.hex_per_tile != hpt) continue;
      size_t need, budget;
      if (variant == 9) {
        need = elem_bytes == 4 ? ebe_hex_tc_smem(t, rpad) : ~(size_t)0;
        budget = 220 * 1024;
      } else if (variant == 7) {
        need = elem_bytes == 4 ? ebe_hexmat_smem(t, view(), rpad) : ~(size_t)0;
        budget = 110 * 1024;
      } else if (variant == 3 || variant == 5 || variant == 6) {   // (6: one block per SM)
        need = elem_bytes == 4 ? ebe_hex_staged_smem<float>(t, view(), rpad) : ebe_hex_staged_smem<double>(t, view(), rpad);
        budget = variant == 6 ? 220 * 1024 : 110 * 1024;
      } else if (variant == 4) {   // one block per SM
        need = elem_bytes == 4 ? ebe_hex_cm_smem<float>(t, view(), rpad) : ebe_hex_cm_smem<double>(t, view(), rpad);
        budget = 220 * 1024;
      } else {
        need = (size_t)t.nloc_max * (3 * rpad * elem_bytes + 4);
        budget = elem_bytes == 4 ? 100 * 1024 : 200 * 1024;
      }
      if (need <= budget || (hpt && need <= 220 * 1024)) best = &t;
    }
    return best;
  }
  fem_status workspace(int rpad, Workspace** out) {
    for (auto* w : ws)
      if (w->rpad == rpad) {
        *out = w;
        return FEM_OK;
      }
    Workspace* w = nullptr;
    CHK(ws_create(N, rpad, &w));
    ws.push_back(w);
    *out = w;
    return FEM_OK;
  }
};

// EBE product q = (aM M + aK K) p on the mesh: the tiled hex kernel when the mesh has hex patches and a
// tiling fits, else the generic element kernel (q masked on Dirichlet DOFs by the consumers).
template <typename T>
static cudaError_t ebe_elem_product(const fem_mesh* m, int rpad, const T* p, T* q, double aM, double aK,
                                    const Reducer* red, CgCase* sc, double* ptq, const int* gate, cudaStream_t s,
                                    bool tc = false) {
  int v, h;
  m->resolve(sizeof(T), rpad, &v, &h);
  if (tc || v == 9) {   // FP16 hex matrices on the tensor cores: FP32, the mesh's own coefficients, 8 or 16 cases
    if constexpr (sizeof(T) == 4) {
      // (tiles of 64 hexes for 8 cases, 32 for 16: measured fastest, 2.66 against 2.81 ms and 0.114 against
      // 0.131 ms on the large and medium boxes)
      const HexTiles* t = m->npe == 4 && !m->seg ? m->tiles_for(4, rpad, 9, rpad == 8 ? 64 : 32) : nullptr;
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      auto same = [](double x, double y) { return std::fabs(x - y) <= 1e-12 * std::fabs(y); };
      if (t && (rpad == 8 || rpad == 16) && same(aM, m->cM) && same(aK, m->cK) &&
          ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15) == 0 &&
          (m->hm16 || (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
                       const_cast<fem_mesh*>(m)->ensure_hm16(s) == FEM_OK)))
        return launch_ebe_hex_tc(*t, m->view(), m->hm16, rpad, p, q, aM, aK, red, sc, ptq, gate, s);
    }
    if (v == 9) v = m->hex ? 5 : 1, h = 0;
  }
  if (m->npe == 10 && v != 8)   // quadratic tets: the tet10 element kernel (or the assembled blocks, variant 8)
    return launch_ebe10_gated<T>(m->E, m->N, rpad, m->conn10, m->rec32, m->rec64, m->fm, p, nullptr, q, aM, aK, red,
                                 sc, ptq, gate, s);
  if (v == 8) {   // assembled 3x3 blocks (built outside stream capture only); not for fused groups
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!m->seg && (m->row_ptr || (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
                                   const_cast<fem_mesh*>(m)->ensure_bcsr(s) == FEM_OK)))
      return launch_bcsr_apply<T>(m->view(), rpad, m->row_ptr, m->col, m->Kb, m->Mb, m->KMd, p, q, aM, aK, red, sc,
                                  ptq, gate, s);
    if (m->npe == 10)
      return launch_ebe10_gated<T>(m->E, m->N, rpad, m->conn10, m->rec32, m->rec64, m->fm, p, nullptr, q, aM, aK,
                                   red, sc, ptq, gate, s);
    v = m->hex ? 5 : 1, h = 0;
  }
  if (v == 7) {   // hex element matrices: FP32, the mesh's own coefficients, no fused groups, aligned vectors
    if constexpr (sizeof(T) == 4) {
      const HexTiles* t = m->tiles_for(sizeof(T), rpad, 7, h);
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      // (coefficients equal to the mesh's to 1e-12: far below the FP32 matrices' own rounding)
      auto same = [](double x, double y) { return std::fabs(x - y) <= 1e-12 * std::fabs(y); };
      if (t && !m->seg && same(aM, m->cM) && same(aK, m->cK) &&
          ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(q)) & 15) == 0 &&
          (m->hexmat || (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
                         const_cast<fem_mesh*>(m)->ensure_hexmat(s) == FEM_OK)))
        return launch_ebe_hexmat(*t, m->view(), m->hexmat, rpad, p, q, aM, aK, red, sc, ptq, gate, s);
    }
    v = 5, h = 0;
  }
  if (v == 4) {   // case-major staged tiles (converged cases skipped); same requirements as 3, no fused groups
    const HexTiles* t = (reinterpret_cast<uintptr_t>(p) & 15) == 0 ? m->tiles_for(sizeof(T), rpad, 4, h) : nullptr;
    if (t) return launch_ebe_hex_cm<T>(*t, m->view(), rpad, p, q, aM, aK, red, sc, ptq, gate, s);
    v = 3, h = 0;
  }
  if ((v == 5 || v == 6) && (sizeof(T) != 4 || m->seg || rpad < 4)) v = 3;   // packed pairs: FP32, r >= 4 lanes
  if (v == 3 || v == 5 || v == 6) {   // staged copies need 16-byte rows (3 x rpad values), 16-byte aligned input
    const HexTiles* t = (reinterpret_cast<uintptr_t>(p) & 15) == 0 ? m->tiles_for(sizeof(T), rpad, v, h) : nullptr;
    if (t) return launch_ebe_hex_staged<T>(*t, m->view(), rpad, p, q, aM, aK, red, sc, ptq, gate, s, v == 3 ? 0 : v - 4);
    v = 2, h = 0;
  }
  if (const HexTiles* t = m->tiles_for(sizeof(T), rpad, v, h))
    return launch_ebe_hex<T>(*t, m->view(), rpad, p, q, aM, aK, red, sc, ptq, gate, s);
  return launch_ebe_gated<T>(m->view(), rpad, p, nullptr, q, aM, aK, red, sc, ptq, gate, s);
}

// A product of the solver: the element-by-element product and, with_ab on a mesh with absorbing faces, the
// dashpot term cB C_b p of A = cM M + cK K + cB C_b (its p^T q share added to the CG state).
template <typename T>
static cudaError_t ebe_product(const fem_mesh* m, int rpad, const T* p, T* q, double aM, double aK,
                               const Reducer* red, CgCase* sc, double* ptq, const int* gate, cudaStream_t s,
                               bool with_ab = false, bool tc = false) {
  cudaError_t e = ebe_elem_product<T>(m, rpad, p, q, aM, aK, red, sc, ptq, gate, s, tc);
  if (e == cudaSuccess && with_ab && m->ab.nb > 0)
    e = launch_dashpot<T>(m->ab, rpad, m->ab.cB, p, q, false, m->fm, red, sc, ptq, gate, s);
  return e;
}

// ------------------------------------------------------------------------------------------------------
// PCG drivers.
// ------------------------------------------------------------------------------------------------------
// Deferred x updates (launch_dir_defer) apply to the FP32 inner solves of multi-RHS groups; the caller then
// completes x with launch_refine_pending.
static bool defer_inner(const MeshView& mv) { return mv.seg == nullptr; }

template <typename T>
static fem_status pcg_core(fem_mesh* m, Workspace* w, const T* b, T* x, T* r, T* z, T* p, T* q, CgCase* sc,
                           bool zero_guess, bool true_check, double tol, int maxit, const CgCase* gate,
                           int check_every, cudaStream_t s) {
  const MeshView mv = m->view();
  const int rpad = w->rpad;
  const Reducer red = w->red();
  const int ebe_cls = sizeof(T) == 4 ? P_EBE32 : P_EBE64;
  const bool sg = mv.seg != nullptr;
  const bool defer = sizeof(T) == 4 && !true_check && defer_inner(mv);
  if (sg) {
    CU(launch_norm_b_seg<T>(mv, b, red, sc, gate, tol, s));
  } else {
    CU(launch_norm_b_gated<T>(mv, rpad, b, red, sc, gate, tol, s));
  }
  w->count();
  if (zero_guess) {
    CU(cudaMemsetAsync(x, 0, sizeof(T) * (size_t)w->n, s));
    if (sg) {
      CU(launch_resid_seg<T>(mv, b, nullptr, x, r, z, red, sc, w->n_active, s));
    } else {
      CU(launch_resid<T>(mv, rpad, b, nullptr, x, r, z, 1, red, sc, w->n_active, tol, maxit, s));
    }
    w->count();
  } else {
    if (sg) return fail(FEM_ERR_ARG, "fused groups solve from a zero inner guess only");
    // the guess is zeroed on Dirichlet DOFs (and for b = 0) before its residual is formed
    CU(launch_zero_b0_t<T>(mv, rpad, x, sc, s));
    int pi = w->pbeg(ebe_cls, s);
    CU(ebe_product<T>(m, rpad, x, q, m->cM, m->cK, nullptr, nullptr, nullptr, nullptr, s, true));
    w->pend(pi, s);
    CU(launch_resid<T>(mv, rpad, b, q, x, r, z, 1, red, sc, w->n_active, tol, maxit, s));
    w->count(3);
  }
  if (check_every < 1) check_every = 1;
  int issued = 0, rechecks = 0;
  for (;;) {
    for (int k = 0; k < check_every; ++k) {
      int p0 = w->pbeg(P_VEC, s);
      if (defer) {
        if constexpr (sizeof(T) == 4) CU(launch_dir_defer<float>(mv, rpad, r, p, x, sc, w->n_active, s));
      } else if (sg) {
        CU(launch_dir_seg<T>(mv, z, p, sc, w->n_active, s));
      } else {
        CU(launch_dir_gated<T>(mv, rpad, z, p, sc, w->n_active, s));
      }
      w->pend(p0, s);
      int p1 = w->pbeg(sizeof(T) == 4 && w->tc ? P_EBE16 : ebe_cls, s);
      CU(ebe_product<T>(m, rpad, p, q, m->cM, m->cK, &red, sc, nullptr, w->n_active, s, true, w->tc));
      w->pend(p1, s);
      int p2 = w->pbeg(P_VEC, s);
      if (defer) {
        if constexpr (sizeof(T) == 4) CU(launch_update_defer<float>(mv, rpad, q, r, red, sc, w->n_active, maxit, s));
      } else if (sg) {
        CU(launch_update_seg<T>(mv, p, q, x, r, z, red, sc, w->n_active, maxit, s));
      } else {
        CU(launch_update<T>(mv, rpad, p, q, x, r, z, red, sc, w->n_active, tol, maxit, s));
      }
      w->pend(p2, s);
      w->count(3);
    }
    issued += check_every;
    CU(cudaMemcpyAsync(w->h_active, w->n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    w->resolve();
    if (*w->h_active == 0) {
      if (!true_check) break;
      if (++rechecks > 32) break;
      // Algorithm 1 stops on the recursive residual; confirm with the true one and resume if needed.
      int pi = w->pbeg(ebe_cls, s);
      CU(ebe_product<T>(m, rpad, x, q, m->cM, m->cK, nullptr, nullptr, nullptr, nullptr, s, true));
      w->pend(pi, s);
      CU(launch_resid<T>(mv, rpad, b, q, x, r, z, 0, red, sc, w->n_active, tol, maxit, s));
      w->count(2);
      CU(cudaMemcpyAsync(w->h_active, w->n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      w->resolve();
      if (*w->h_active == 0) break;
    }
    if (issued > maxit + 64 * check_every) break;
  }
  return FEM_OK;
}

// Whether a refinement pass runs its inner CG products on the tensor cores (inner_product FEM_INNER_TC): only
// when every active case's reduction target is at least kTcFloor, what a product with FP16 operands (relative
// error ~2.4e-4) still delivers in one pass; a pass that asks more of some case takes the FP32 product, so the
// tensor cores never cost a refinement pass.
static bool tc_pass(const fem_opts& o, const fem_mesh* m, int rpad, const CgCase* h_sc, int ncase) {
  // (the tensor-core product exists for linear-tet hex-patch meshes, one multi-RHS group of 8 or 16 lanes)
  if (o.inner_product != FEM_INNER_TC || m->npe != 4 || m->seg || (rpad != 8 && rpad != 16)) return false;
  for (int c = 0; c < ncase; ++c)
    if (h_sc[c].active && h_sc[c].inner_tol < kTcFloor) return false;
  return true;
}

// FP32-inner / FP64-outer iterative refinement:  r64 = b - A64 x;  A32 d = r64 (inner PCG);  x += d.
static fem_status solve_mixed(fem_mesh* m, Workspace* w, const double* b, double* x, const fem_opts& o_in,
                              cudaStream_t s) {
  const fem_opts& o = o_in;
  w->tc = false;
  const MeshView mv = m->view();
  const int rpad = w->rpad;
  const Reducer red = w->red();
  CU(launch_norm_b_gated<double>(mv, rpad, b, red, w->outer, nullptr, o.tol, s));
  CU(launch_zero_b0_t<double>(mv, rpad, x, w->outer, s));
  w->count(2);
  const int kMaxOuter = 40;
  for (int outer_it = 0; outer_it <= kMaxOuter; ++outer_it) {
    int pi = w->pbeg(P_EBE64, s);
    CU(ebe_product<double>(m, rpad, x, w->q, m->cM, m->cK, nullptr, nullptr, nullptr, nullptr, s, true));
    w->pend(pi, s);
    CU(launch_outer_resid(mv, rpad, b, w->q, w->r32, red, w->outer, w->n_active, o.tol, o.inner_tol, o.inner_margin * o.tol, s));
    w->count(2);
    CU(cudaMemcpyAsync(w->h_active, w->n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(w->h_sc, w->outer, sizeof(CgCase) * rpad, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (*w->h_active == 0) break;
    int used = 0;
    if (outer_it == kMaxOuter) used = o.maxit;   // refinement stalled: report the active cases
    for (int c = 0; c < rpad; ++c) used = std::max(used, w->h_sc[c].iters);
    if (used >= o.maxit) {
      for (int c = 0; c < rpad; ++c) w->h_sc[c].status = w->h_sc[c].active ? FEM_ERR_NOT_CONVERGED : w->h_sc[c].status;
      CU(cudaMemcpyAsync(w->outer, w->h_sc, sizeof(CgCase) * rpad, cudaMemcpyHostToDevice, s));
      break;
    }
    w->tc = tc_pass(o, m, rpad, w->h_sc, rpad);
    CHK(pcg_core<float>(m, w, w->r32, w->x32, w->rr32, w->z32, w->p32, w->q32, w->sc, true, false, o.inner_tol,
                        o.maxit - used, w->outer, o.check_every, s));
    if (defer_inner(mv)) {
      CU(launch_refine_pending(mv, rpad, rpad, x, w->x32, w->p32, w->outer, w->sc, s));
    } else {
      CU(launch_refine_counts(mv, rpad, rpad, x, w->x32, w->outer, w->sc, s));
    }
    w->count();
  }
  w->resolve();
  return FEM_OK;
}

static fem_status solve_any(fem_mesh* m, Workspace* w, const double* b, double* x, const fem_opts& o,
                            cudaStream_t s, CgCase** result_dev) {
  if (o.precision == FEM_FP64) {
    CHK(pcg_core<double>(m, w, b, x, w->r, w->z, w->p, w->q, w->sc, false, true, o.tol, o.maxit, nullptr,
                         o.check_every, s));
    *result_dev = w->sc;
  } else {
    CHK(solve_mixed(m, w, b, x, o, s));
    *result_dev = w->outer;
  }
  return FEM_OK;
}

static fem_status check_opts(const fem_opts* o) {
  if (!o) return fail(FEM_ERR_ARG, "opts is null");
  if (o->precision != FEM_FP64 && o->precision != FEM_FP32_INNER) return fail(FEM_ERR_ARG, "unknown precision");
  if (!(o->tol > 0.0) || o->maxit < 1) return fail(FEM_ERR_ARG, "tol must be > 0 and maxit >= 1");
  if (o->precision == FEM_FP32_INNER && !(o->inner_tol > 0.0 && o->inner_tol < 1.0))
    return fail(FEM_ERR_ARG, "inner_tol must be in (0, 1)");
  if (o->predictor != FEM_PRED_AB4 && o->predictor != FEM_PRED_DD) return fail(FEM_ERR_ARG, "unknown predictor");
  if (o->s_max < 1 || o->s_max > kMaxSlots - 1) return fail(FEM_ERR_ARG, "s_max must be in [1, 32]");
  if (o->cert_df < 0 || o->cert_df > 3) return fail(FEM_ERR_ARG, "cert_df must be 0, 1, 2 or 3");
  if (o->snapshot_format < 0 || o->snapshot_format > 3) return fail(FEM_ERR_ARG, "snapshot_format must be 0 .. 3");
  if (o->wait_budget < 0) return fail(FEM_ERR_ARG, "wait_budget must be >= 0");
  if (o->precision == FEM_FP32_INNER && !(o->inner_margin > 0.0 && o->inner_margin < 1.0))
    return fail(FEM_ERR_ARG, "inner_margin must be in (0, 1)");
  if (o->inner_product != FEM_INNER_FP32 && o->inner_product != FEM_INNER_TC)
    return fail(FEM_ERR_ARG, "inner_product must be FEM_INNER_FP32 or FEM_INNER_TC");
  if (o->pred_guard != 0 && o->pred_guard != 1) return fail(FEM_ERR_ARG, "pred_guard must be 0 or 1");
  if (o->cpu_predictor) {
    if (o->predictor != FEM_PRED_DD) return fail(FEM_ERR_ARG, "cpu_predictor needs the data-driven predictor");
    if (o->snapshot_format != 0 && o->snapshot_format != 2)
      return fail(FEM_ERR_ARG, "cpu_predictor needs snapshot_format 0 or 2");
    if (o->fuse_meshes) return fail(FEM_ERR_ARG, "cpu_predictor does not combine with fuse_meshes");
  }
  return FEM_OK;
}

// ------------------------------------------------------------------------------------------------------
// Batch of cases.
// ------------------------------------------------------------------------------------------------------
struct Group {
  fem_mesh* mesh = nullptr;
  fem_mesh* owned_mesh = nullptr;   // fused groups: the virtual mesh (owned)
  std::vector<int64_t> node_off;    // fused groups: first node of each case's mesh, and the total
  int ncase = 0;                    // per-case arrays: rpad (multi-RHS group) or number of meshes (fused)
  int rpad = 0;
  std::vector<int> cases;
  std::vector<RickerSrc> hsrc;
  // random impulse loads per case lane (host, until the batch starts) and their device form
  struct HostImpulse {
    int32_t node, step;
    double f[3];
  };
  std::vector<std::vector<HostImpulse>> himp;
  Impulses imp;
  int32_t *imp_node = nullptr, *imp_lane = nullptr, *imp_off = nullptr;
  double* imp_f = nullptr;
  // the heterogeneous scheme: the host predictor and the device copy of its correction
  HostPred* hp = nullptr;
  double* ycpu = nullptr;
  int64_t n = 0;
  double *u = nullptr, *a = nullptr, *vh[4] = {nullptr, nullptr, nullptr, nullptr};
  double *b = nullptr, *x = nullptr, *du_ab = nullptr, *m_in = nullptr, *k_in = nullptr, *guess = nullptr;
  void* ring = nullptr;
  int n_slots = 0;
  int64_t snap_stride = 0;   // values per ring slot: n rounded up to a multiple of 8
  int n_regions = 0;            // regions the Gram buffers were sized for
  double* gram = nullptr;
  double* wcoef = nullptr;
  double* dpart = nullptr;
  int n_chunks = 1;
  int* slot_lists = nullptr;    // device [2][kMaxSlots]
  int* h_slots = nullptr;       // pinned [2][kMaxSlots]
  RickerSrc* src = nullptr;
  double* ext = nullptr;        // device [ncase][3]: external loads for the next step
  // FP32-inner steps: products kept by recurrences (K u, M v, K v, M a, ring of A v) and split products
  // (Pb = M a + (4/dt + a0) M v + a1 K v - K u: the right-hand side without the loads)
  double *Ku = nullptr, *Mv = nullptr, *Kv = nullptr, *Pb = nullptr, *Av[4] = {nullptr, nullptr, nullptr, nullptr};
  double *qM = nullptr, *qK = nullptr;
  float2* xdf = nullptr;          // (hi, lo) split of the product input for the double-float assembled product
  bool use_ext = false;
  // learned proposal and training-sample collection (allocated on first use)
  float* F = nullptr;             // features [Mpad][64] of this step's prediction, row R * rpad + c
  double* dw = nullptr;           // proposal's coefficient correction [R][rpad][kMaxSlots]
  double* wbest = nullptr;        // best coefficients of the solved correction [R][rpad][kMaxSlots]
  double* ydelta = nullptr;       // Y dw [n]
  int* choose = nullptr;          // [rpad] 1 = the case takes the proposal this step
  long long* counts = nullptr;    // [2] steps where cases took / rejected the proposal
  float4* case_src = nullptr;     // [rpad] source position and (f0 - 5) / 3
  double* e2case = nullptr;       // [ncase] ||e^it||^2 of each case (residual-space samples)
  int* fb = nullptr;              // [ncase] steps whose data-driven correction the guess guard dropped
  int last_npairs = 0;            // pairs used by this step's prediction
  bool featured = false;          // F holds this step's features
  bool proposed = false;          // ydelta holds this step's proposal
  // graph steps: the whole FP32-inner step captured once as a CUDA graph with device-side control
  StepCtl* ctl = nullptr;         // device step record
  int* acc_iters = nullptr;       // [ncase] inner iterations summed since the statistics were last read
  double* acc_relres = nullptr;   // [ncase] worst certified relres since then
  int* acc_status = nullptr;      // [ncase] worst status since then
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // capture streams (top level, bodies, fork)
  cudaEvent_t gev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr}; // forks / joins of the captured step
  int ab_ready = -1;              // step whose du_AB the last graph launch formed at its tail
  int* h_pin = nullptr;           // pinned: [0] = 1 (use_ext flag), [1] = step counter to upload
  int ctl_it = -1;                // step counter the device record holds (-1: unknown, upload first)
  bool graph_failed = false;      // capture or instantiation failed: eager steps from now on
  int graph_steps = 0;            // graph steps whose statistics are not read yet
  Workspace* ws = nullptr;
  int steps = 0;
  std::vector<int> iters_acc;
  std::vector<double> relres_max;
  std::vector<CgCase> last;     // per-lane solve statistics of the last step
  ~Group() {
    dfree(u); dfree(a);
    for (auto& v : vh) dfree(v);
    dfree(b); dfree(x); dfree(du_ab); dfree(m_in); dfree(k_in); dfree(guess);
    if (ring) cudaFree(ring);
    dfree(gram); dfree(wcoef); dfree(dpart); dfree(slot_lists); dfree(src); dfree(ext);
    dfree(Ku); dfree(Mv); dfree(Kv); dfree(Pb); dfree(qM); dfree(qK); dfree(xdf);
    for (auto& v : Av) dfree(v);
    dfree(F); dfree(dw); dfree(wbest); dfree(ydelta); dfree(choose); dfree(counts); dfree(case_src); dfree(e2case);
    dfree(fb);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& st : gs)
      if (st) cudaStreamDestroy(st);
    for (auto& ev : gev)
      if (ev) cudaEventDestroy(ev);
    dfree(ctl); dfree(acc_iters); dfree(acc_relres); dfree(acc_status);
    dfree(imp_node); dfree(imp_lane); dfree(imp_off); dfree(imp_f);
    hostpred_destroy(hp);
    dfree(ycpu);
    if (h_pin) cudaFreeHost(h_pin);
    if (h_slots) cudaFreeHost(h_slots);
    delete ws;
    delete owned_mesh;
  }
};

struct fem_batch {
  fem_opts opts{};
  Prof prof;
  cudaStream_t s = nullptr;
  std::vector<Group*> groups;
  std::vector<std::pair<int, int>> loc;   // case -> (group, lane)
  bool started = false;
  int steps = 0;
  fem_mlp* mlp = nullptr;              // learned proposal (caller-owned), or none
  float* col_x = nullptr;              // caller-owned sample buffers [capacity][64] / [capacity][32 or FEM_MLP_RES]
  bool col_res = false;                // residual-space samples (W, w) instead of coefficient targets
  float* col_t = nullptr;
  int64_t col_cap = 0, col_n = 0;
  bool col_full = false;
  // asynchronous field reads: two device staging buffers, copied to the host on their own stream
  cudaStream_t cs = nullptr;
  cudaEvent_t ready[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
  double* stage[2] = {nullptr, nullptr};
  int stage_k = 0;
  fem_status pending = FEM_OK;         // worst status of eagerly run steps queued by fem_step_async
  ~fem_batch() {
    for (auto* g : groups) delete g;
    if (cs) cudaStreamSynchronize(cs);
    for (int k = 0; k < 2; ++k) {
      if (stage[k]) cudaFree(stage[k]);
      if (ready[k]) cudaEventDestroy(ready[k]);
      if (done[k]) cudaEventDestroy(done[k]);
    }
    if (cs) cudaStreamDestroy(cs);
  }
};

static fem_status group_alloc(fem_batch* bt, Group* g) {
  fem_mesh* m = g->mesh;
  g->rpad = g->owned_mesh ? 1 : next_pow2((int)g->cases.size());
  g->ncase = g->owned_mesh ? (int)g->cases.size() : g->rpad;
  g->n = m->N * 3 * g->rpad;
  const size_t n = (size_t)g->n;
  CHK(dalloc(&g->u, n));
  CHK(dalloc(&g->a, n));
  for (auto& v : g->vh) CHK(dalloc(&v, n));
  CHK(dalloc(&g->b, n));
  CHK(dalloc(&g->x, n));
  CHK(dalloc(&g->du_ab, n));
  CHK(dalloc(&g->m_in, n));
  CHK(dalloc(&g->k_in, n));
  CHK(dalloc(&g->guess, n));
  CHK(dalloc(&g->fb, (size_t)kMaxCases));
  cudaStream_t s = bt->s;
  CU(cudaMemsetAsync(g->fb, 0, sizeof(int) * kMaxCases, s));
  CU(cudaMemsetAsync(g->u, 0, n * 8, s));
  CU(cudaMemsetAsync(g->a, 0, n * 8, s));
  for (auto& v : g->vh) CU(cudaMemsetAsync(v, 0, n * 8, s));
  CU(cudaMemsetAsync(g->x, 0, n * 8, s));
  CU(cudaMemsetAsync(g->guess, 0, n * 8, s));
  CU(cudaMemsetAsync(g->b, 0, n * 8, s));
  if (bt->opts.precision == FEM_FP32_INNER) {
    for (double** v : {&g->Ku, &g->Mv, &g->Kv, &g->Pb, &g->Av[0], &g->Av[1], &g->Av[2], &g->Av[3], &g->qM, &g->qK}) {
      CHK(dalloc(v, n));
      CU(cudaMemsetAsync(*v, 0, n * 8, s));
    }
    if (bt->opts.cert_df >= 2) CHK(m->ensure_bcsr(s));
    if (bt->opts.inner_product == FEM_INNER_TC && bt->opts.precision == FEM_FP32_INNER) CHK(m->ensure_hm16(s));
    if (bt->opts.cert_df == 3) CHK(dalloc(&g->xdf, n));
  }
  if (bt->opts.predictor == FEM_PRED_DD) {
    g->n_slots = bt->opts.s_max + 1;
    g->snap_stride = (n + 7) & ~(int64_t)7;
    const size_t ring_bytes = snap_bytes(bt->opts.snapshot_format) * (size_t)g->snap_stride * g->n_slots;
    cudaError_t e = cudaMalloc(&g->ring, ring_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g->ring = nullptr;
      return fail(FEM_ERR_OOM, "snapshot ring allocation failed");
    }
    CU(cudaMemsetAsync(g->ring, 0, ring_bytes, s));
    g->n_regions = m->n_regions;
    const int R = std::max(1, m->n_regions);
    CHK(dalloc(&g->gram, (size_t)R * g->rpad * kMaxSlots * kMaxSlots));
    CHK(dalloc(&g->wcoef, (size_t)R * g->rpad * kMaxSlots));
    // enough blocks for the dot/combine kernels to fill the GPU: about 8 per SM over all regions
    g->n_chunks = std::max(1, std::min(64, (8 * sm_count() + R - 1) / R));
    CHK(dalloc(&g->dpart, (size_t)R * g->n_chunks * kMaxSlots * g->rpad));
    CU(cudaMemsetAsync(g->gram, 0, sizeof(double) * (size_t)R * g->rpad * kMaxSlots * kMaxSlots, s));
    if (bt->opts.cpu_predictor && m->n_regions > 0) {
      CU(hostpred_create(g->snap_stride, g->rpad, g->n_slots, bt->opts.s_max, bt->opts.snapshot_format,
                         bt->opts.tau, m->h_reg_lo, m->h_reg_hi, &g->hp));
      CHK(dalloc(&g->ycpu, n));
    }
  }
  CHK(dalloc(&g->slot_lists, 2 * kMaxSlots));
  if (cudaMallocHost((void**)&g->h_slots, sizeof(int) * 2 * kMaxSlots) != cudaSuccess) {
    cudaGetLastError();
    return fail(FEM_ERR_OOM, "cudaMallocHost failed");
  }
  // one source and one external load per case: per column (multi-RHS group) or per mesh copy (fused)
  g->hsrc.resize(g->ncase);
  for (int l = (int)g->cases.size(); l < g->ncase; ++l) g->hsrc[l] = RickerSrc{-1, {0, 0, 0}, 1.0, 0.0, 0.0};
  CHK(dalloc(&g->src, g->ncase));
  CHK(dalloc(&g->ext, 3 * g->ncase));
  {   // impulse loads: entries sorted by step (counting sort), per step offsets
    int64_t ni = 0;
    int last = 0;
    g->himp.resize(g->ncase);
    for (const auto& v : g->himp)
      for (const auto& e : v) ni += 1, last = std::max(last, (int)e.step);
    if (ni > 0) {
      if (ni > INT32_MAX / 2) return fail(FEM_ERR_ARG, "too many impulses in one group");
      std::vector<int32_t> off((size_t)last + 2, 0), nd(ni), ln(ni);
      std::vector<double> f(3 * ni);
      for (const auto& v : g->himp)
        for (const auto& e : v) off[(size_t)e.step + 1] += 1;
      int mx = 0;
      for (int k = 1; k <= last + 1; ++k) mx = std::max(mx, off[k]), off[k] += off[k - 1];
      std::vector<int32_t> pos(off.begin(), off.end());
      for (int l = 0; l < (int)g->himp.size(); ++l)
        for (const auto& e : g->himp[l]) {
          const int32_t k = pos[e.step]++;
          nd[k] = e.node, ln[k] = l;
          for (int d = 0; d < 3; ++d) f[3 * (size_t)k + d] = e.f[d];
        }
      CHK(dalloc(&g->imp_node, (size_t)ni));
      CHK(dalloc(&g->imp_lane, (size_t)ni));
      CHK(dalloc(&g->imp_off, off.size()));
      CHK(dalloc(&g->imp_f, 3 * (size_t)ni));
      CU(cudaMemcpyAsync(g->imp_node, nd.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(g->imp_lane, ln.data(), sizeof(int32_t) * ni, cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(g->imp_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(g->imp_f, f.data(), sizeof(double) * 3 * ni, cudaMemcpyHostToDevice, s));
      CU(cudaStreamSynchronize(s));
      g->imp = Impulses{(int)ni, last, mx, g->imp_node, g->imp_lane, g->imp_f, g->imp_off};
    }
  }
  CU(cudaMemsetAsync(g->ext, 0, sizeof(double) * 3 * g->ncase, s));
  CU(cudaMemcpyAsync(g->src, g->hsrc.data(), sizeof(RickerSrc) * g->ncase, cudaMemcpyHostToDevice, s));
  CHK(ws_create(m->N, g->rpad, &g->ws));
  g->ws->prof = &bt->prof;
  g->iters_acc.assign(g->ncase, 0);
  g->relres_max.assign(g->ncase, 0.0);
  g->last.assign(g->ncase, CgCase{});
  return FEM_OK;
}

static PredView pred_view(const fem_batch* bt, const Group* g) {
  PredView p;
  p.n_regions = g->n_regions;
  p.reg_lo = g->mesh->reg_lo;
  p.reg_hi = g->mesh->reg_hi;
  p.rpad = g->rpad;
  p.n_slots = g->n_slots;
  p.slot_stride = g->snap_stride;
  p.ring = g->ring;
  p.fmt = bt->opts.snapshot_format;
  p.gram = g->gram;
  p.w = g->wcoef;
  p.n_chunks = g->n_chunks;
  p.dpart = g->dpart;
  return p;
}

static int slot_of(const Group* g, int j) { return (j - 1) % g->n_slots; }  // correction e^j, j >= 1

// Buffers of the learned proposal and of sample collection (first use).
static fem_status group_learn_alloc(fem_batch* bt, Group* g) {
  if (g->F) return FEM_OK;
  if (g->owned_mesh) return fail(FEM_ERR_ARG, "the learned proposal and sample collection need groups of one mesh");
  const int64_t rows = (int64_t)std::max(1, g->n_regions) * g->rpad;
  const int64_t mpad = ((rows + 63) / 64) * 64;
  CHK(dalloc(&g->F, (size_t)(mpad * 64)));
  CHK(dalloc(&g->dw, (size_t)(rows * kMaxSlots)));
  CHK(dalloc(&g->wbest, (size_t)(rows * kMaxSlots)));
  CHK(dalloc(&g->ydelta, (size_t)g->n));
  CHK(dalloc(&g->choose, (size_t)g->rpad));
  CHK(dalloc(&g->counts, 2));
  CHK(dalloc(&g->case_src, (size_t)g->rpad));
  CHK(dalloc(&g->e2case, (size_t)g->rpad));
  std::vector<float4> cs(g->rpad, make_float4(0.f, 0.f, 0.f, 0.f));
  const std::vector<double>& xyz = g->mesh->h_xyz;
  for (int l = 0; l < (int)g->cases.size(); ++l) {
    const RickerSrc& r = g->hsrc[l];
    if (r.node < 0) continue;
    cs[l] = make_float4((float)xyz[3 * (size_t)r.node], (float)xyz[3 * (size_t)r.node + 1],
                        (float)xyz[3 * (size_t)r.node + 2], (float)((r.f0 - 5.0) / 3.0));
  }
  cudaStream_t s = bt->s;
  CU(cudaMemcpyAsync(g->case_src, cs.data(), sizeof(float4) * g->rpad, cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(g->counts, 0, 2 * sizeof(long long), s));
  CU(cudaStreamSynchronize(s));
  return FEM_OK;
}

// Initial guess of the increment for step it = g->steps + 1 into `out`: AB4 (+ regional correction).
// learn: this is the time step's own prediction (features, learned proposal).
static fem_status group_predict(fem_batch* bt, Group* g, double* out, bool* corrected = nullptr, bool learn = false) {
  if (corrected) *corrected = false;
  if (learn) g->featured = g->proposed = false, g->last_npairs = 0;
  const int it = g->steps + 1;
  const double dt = g->mesh->tp.dt;
  auto vslot = [&](int j) { return g->vh[((j % 4) + 4) % 4]; };
  cudaStream_t s = bt->s;
  CU(launch_ab4(g->n, dt, vslot(it - 4), vslot(it - 3), vslot(it - 2), vslot(it - 1), g->du_ab, s));
  g->ws->count();
  CU(cudaMemcpyAsync(out, g->du_ab, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
  if (bt->opts.predictor != FEM_PRED_DD || g->n_regions == 0) return FEM_OK;
  if (g->mesh->n_regions != g->n_regions) return fail(FEM_ERR_STATE, "mesh regions changed after the batch started");
  if (g->hp) {   // heterogeneous scheme: the correction the host prepared for this step
    int np = 0;
    const double* yh = hostpred_take(g->hp, it, &np);
    if (!yh) return FEM_OK;
    CU(cudaMemcpyAsync(g->ycpu, yh, sizeof(double) * g->n, cudaMemcpyHostToDevice, s));
    CU(launch_add(g->n, g->du_ab, g->ycpu, out, s));
    g->ws->count();
    if (corrected) *corrected = true;
    return FEM_OK;
  }
  const int n_e = std::min(it - 1, g->n_slots);
  const int n_pairs = std::min(bt->opts.s_max, n_e - 1);
  if (n_pairs <= 0) return FEM_OK;
  // X: e^{it-1-n_pairs} .. e^{it-2};  Y: e^{it-n_pairs} .. e^{it-1};  query: e^{it-1}
  for (int a = 0; a < n_pairs; ++a) {
    g->h_slots[a] = slot_of(g, it - 1 - n_pairs + a);
    g->h_slots[kMaxSlots + a] = slot_of(g, it - n_pairs + a);
  }
  CU(cudaMemcpyAsync(g->slot_lists, g->h_slots, sizeof(int) * 2 * kMaxSlots, cudaMemcpyHostToDevice, s));
  const PredView pv = pred_view(bt, g);
  CU(launch_pred_solve(pv, g->slot_lists, n_pairs, slot_of(g, it - 1), bt->opts.tau, s));
  if (learn && (bt->mlp || bt->col_x)) {
    CHK(group_learn_alloc(bt, g));
    CU(mlp_features(pv, n_pairs, g->case_src, g->mesh->reg_cent, g->mesh->inv_extent, g->F, s));
    g->featured = true;
    g->last_npairs = n_pairs;
    g->ws->count();
  }
  if (learn && bt->mlp) {
    // learned proposal: coefficients c + net(features); its difference to the plain guess, Y dw, is kept
    CU(mlp_propose(bt->mlp, g->F, (int64_t)g->n_regions * g->rpad, n_pairs, g->dw, s));
    CU(cudaMemsetAsync(g->ydelta, 0, sizeof(double) * g->n, s));
    CU(launch_pred_combine2(pv, g->slot_lists + kMaxSlots, n_pairs, out, g->dw, g->ydelta, s));
    g->proposed = true;
    g->ws->count(6);
  } else {
    CU(launch_pred_combine(pv, g->slot_lists + kMaxSlots, n_pairs, out, s));
  }
  g->ws->count(2);
  if (corrected) *corrected = true;
  // the pinned slot list is reused next step: order the host write after this step's copy
  CU(cudaStreamSynchronize(s));
  return FEM_OK;
}

// The certification product qM = M p, qK = K p in the form opts.cert_df selects: 0 element-by-element FP64,
// 1 element-by-element double-float, 2 assembled blocks FP64, 3 assembled blocks double-float.
static cudaError_t split_product(const fem_mesh* m, int mode, int rpad, const double* p, float2* p_df, double* qM,
                                 double* qK, cudaStream_t s) {
  const MeshView mv = m->view();
  if (m->npe == 10 && (mode == 0 || mode == 1)) {   // quadratic tets: the FP64 element kernel, M and K apart
    cudaError_t e = launch_ebe10_gated<double>(m->E, m->N, rpad, m->conn10, m->rec32, m->rec64, m->fm, p, nullptr, qM,
                                               1.0, 0.0, nullptr, nullptr, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    return launch_ebe10_gated<double>(m->E, m->N, rpad, m->conn10, m->rec32, m->rec64, m->fm, p, nullptr, qK, 0.0,
                                      1.0, nullptr, nullptr, nullptr, nullptr, s);
  }
  if (mode == 1) return launch_ebe_split_df(mv, m->rec_df, rpad, p, qM, qK, s);
  if (mode == 2 || mode == 3)
    return launch_bcsr_split(mv, rpad, m->row_ptr, m->col, m->Kb, m->Mb, m->KMd, p, mode == 3 ? p_df : nullptr,
                             qM, qK, s);
  return launch_ebe_split(mv, rpad, p, qM, qK, s);
}

// Direct recomputation of the recurrence products from the state (bounds their rounding drift).
static fem_status group_refresh(fem_batch* bt, Group* g) {
  fem_mesh* m = g->mesh;
  const MeshView mv = m->view();
  cudaStream_t s = bt->s;
  const int it = g->steps;      // state after step it
  const int cm = bt->opts.cert_df;
  CU(split_product(m, cm, g->rpad, g->u, g->xdf, g->qM, g->qK, s));
  CU(cudaMemcpyAsync(g->Ku, g->qK, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
  CU(split_product(m, cm, g->rpad, g->a, g->xdf, g->Pb, g->qK, s));   // (M a into Pb, completed below)
  for (int j = it - 3; j <= it; ++j) {
    const int sl = ((j % 4) + 4) % 4;
    CU(split_product(m, cm, g->rpad, g->vh[sl], g->xdf, g->qM, g->qK, s));
    CU(launch_axpby(g->n, m->cM, g->qM, m->cK, g->qK, g->Av[sl], s));
    CU(launch_dashpot<double>(m->ab, g->rpad, m->ab.cB, g->vh[sl], g->Av[sl], false, m->fm, nullptr, nullptr, nullptr,
                              nullptr, s));
    if (j == it) {
      CU(cudaMemcpyAsync(g->Mv, g->qM, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
      CU(cudaMemcpyAsync(g->Kv, g->qK, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
    }
  }
  CU(launch_pb_form(g->n, m->tp.dt, m->tp.a0, m->tp.a1, g->Pb, g->Mv, g->Kv, g->Ku, s));
  g->ws->count(13);
  return FEM_OK;
}

// One step with the FP32-inner solver: right-hand side and the residual of the guess from the product
// recurrences (no FP64 product), inner FP32 PCG, and one FP64 certification product per refinement pass,
// whose split products M du, K du advance the recurrences.
static fem_status group_step_mixed(fem_batch* bt, Group* g, fem_status* worst) {
  const auto t_start = std::chrono::steady_clock::now();
  fem_mesh* m = g->mesh;
  const MeshView mv = m->view();
  cudaStream_t s = bt->s;
  const int it = g->steps + 1;
  const double dt = m->tp.dt;
  const fem_opts& o = bt->opts;
  Workspace* w = g->ws;
  w->tc = false;
  const Reducer red = w->red();
  auto vslot = [&](int j) { return g->vh[((j % 4) + 4) % 4]; };
  auto aslot = [&](int j) { return g->Av[((j % 4) + 4) % 4]; };
  const int every = o.refresh_every > 0 ? o.refresh_every : 200;
  if (it > 1 && (it - 1) % every == 0) CHK(group_refresh(bt, g));
  // 1. initial guess (Section 3.2)
  int ph = w->pbeg(P_PREDICT, s);
  bool corrected = false;
  CHK(group_predict(bt, g, g->guess, &corrected, true));
  w->pend(ph, s);
  // 2. right-hand side (Section 3.1, Eq. GE:DIS) from the recurrences
  ph = w->pbeg(P_RHS, s);
  CU(launch_rhs_incr(mv, g->rpad, g->Pb, g->b, g->src,
                     g->use_ext ? g->ext : nullptr, it * dt, s));
  // random impulses of this step, and the dashpots' C_b v of absorbing boundaries
  CU(launch_impulses(g->imp, g->rpad, it, nullptr, m->fm, g->b, s));
  CU(launch_dashpot<double>(m->ab, g->rpad, 1.0, vslot(it - 1), g->b, false, m->fm, nullptr, nullptr, nullptr, nullptr,
                            s));
  g->use_ext = false;
  w->pend(ph, s);
  w->count();
  // 3. residual of the guess: exact FP64 for the Adams-Bashforth part, FP32 product for the correction
  ph = w->pbeg(P_SOLVE, s);
  const float* qy = nullptr;
  if (corrected) {
    CU(launch_corr_f32(g->n, g->guess, g->du_ab, w->z32, s));
    int pe = w->pbeg(P_EBE32, s);
    CU(ebe_product<float>(m, g->rpad, w->z32, w->q32, m->cM, m->cK, nullptr, nullptr, nullptr, nullptr, s, true));
    w->pend(pe, s);
    qy = w->q32;
    w->count(2);
  }
  // the guess guard: a case whose correction leaves a larger residual than the Adams-Bashforth guess drops it
  // (not with a learned proposal, whose choice below is made against the corrected guess)
  const bool guard = qy && o.pred_guard && !g->proposed;
  if (mv.seg) {
    CU(launch_r0_seg(mv, dt, g->b, aslot(it - 4), aslot(it - 3), aslot(it - 2), aslot(it - 1), qy, w->r32, red,
                     w->outer, w->n_active, o.tol, o.inner_tol, o.inner_margin * o.tol, s, Ring4{}, nullptr, guard,
                     g->fb));
  } else {
    CU(launch_r0(mv, g->rpad, dt, g->b, aslot(it - 4), aslot(it - 3), aslot(it - 2), aslot(it - 1), qy, w->r32, red,
                 w->outer, w->n_active, o.tol, o.inner_tol, o.inner_margin * o.tol, s, Ring4{}, nullptr, nullptr,
                 guard, g->fb));
  }
  if (guard) {
    CU(launch_guard_fix(mv, g->rpad, w->outer, qy, w->r32, g->du_ab, g->guess, nullptr, s));
    w->count();
  }
  if (g->proposed) {
    // learned proposal: r0' = r0 - A32 (Y dw); a case takes it where its initial residual is smaller
    CU(mlp_to_f32(g->n, g->ydelta, w->z32, s));
    int pe = w->pbeg(P_EBE32, s);
    CU(ebe_product<float>(m, g->rpad, w->z32, w->q32, m->cM, m->cK, nullptr, nullptr, nullptr, nullptr, s, true));
    w->pend(pe, s);
    CU(mlp_choose(mv, g->rpad, w->r32, w->q32, red, w->outer, w->n_active, o.tol, o.inner_tol, o.inner_margin * o.tol, g->ncase, g->choose,
                  g->counts, s));
    CU(mlp_apply(g->n, g->rpad, g->choose, w->r32, w->q32, g->guess, g->ydelta, s));
    w->count(4);
  }
  CU(cudaMemcpyAsync(g->x, g->guess, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
  w->count();
  // 4. refinement passes: inner FP32 PCG (cases whose residual is above tol) + FP64 certification
  const int kMaxPass = 40;
  for (int pass = 0; pass < kMaxPass; ++pass) {
    CU(cudaMemcpyAsync(w->h_active, w->n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(w->h_sc, w->outer, sizeof(CgCase) * g->ncase, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    w->resolve();
    int used = 0;
    for (int c = 0; c < g->ncase; ++c) used = std::max(used, w->h_sc[c].iters);
    if (*w->h_active > 0) {
      if (used >= o.maxit || pass == kMaxPass - 1) {
        for (int c = 0; c < g->ncase; ++c)
          if (w->h_sc[c].active) w->h_sc[c].status = FEM_ERR_NOT_CONVERGED, w->h_sc[c].active = 0;
        CU(cudaMemcpyAsync(w->outer, w->h_sc, sizeof(CgCase) * g->ncase, cudaMemcpyHostToDevice, s));
      } else {
        w->tc = tc_pass(o, m, g->rpad, w->h_sc, g->ncase);
        CHK(pcg_core<float>(m, w, w->r32, w->x32, w->rr32, w->z32, w->p32, w->q32, w->sc, true, false, o.inner_tol,
                            o.maxit - used, w->outer, o.check_every, s));
        if (defer_inner(mv)) {
          CU(launch_refine_pending(mv, g->rpad, g->ncase, g->x, w->x32, w->p32, w->outer, w->sc, s));
        } else {
          CU(launch_refine_counts(mv, g->rpad, g->ncase, g->x, w->x32, w->outer, w->sc, s));
        }
        w->count();
      }
    } else if (pass > 0) {
      break;
    }
    int pe = w->pbeg(P_EBE64, s);
    CU(split_product(m, o.cert_df, g->rpad, g->x, g->xdf, g->qM, g->qK, s));
    // absorbing boundaries: the certificate's r = b - cM qM - cK qK takes the dashpot term in qK (undone below)
    CU(launch_dashpot<double>(m->ab, g->rpad, m->ab.cB / m->cK, g->x, g->qK, false, m->fm, nullptr, nullptr, nullptr,
                              nullptr, s));
    w->pend(pe, s);
    if (mv.seg) {
      CU(launch_cert_seg(mv, m->cM, m->cK, g->b, g->qM, g->qK, w->r32, red, w->outer, w->n_active, o.tol,
                         o.inner_tol, o.inner_margin * o.tol, s));
    } else {
      CU(launch_cert(mv, g->rpad, m->cM, m->cK, g->b, g->qM, g->qK, w->r32, red, w->outer, w->n_active, o.tol,
                     o.inner_tol, o.inner_margin * o.tol, s));
    }
    w->count(2);
  }
  CU(launch_dashpot<double>(m->ab, g->rpad, -m->ab.cB / m->cK, g->x, g->qK, false, m->fm, nullptr, nullptr, nullptr,
                            nullptr, s));
  w->pend(ph, s);
  CU(cudaMemcpyAsync(w->h_sc, w->outer, sizeof(CgCase) * g->ncase, cudaMemcpyDeviceToHost, s));
  // 5. Newmark update, product recurrences, snapshot push (Section 3.1, Eq. timestep)
  ph = w->pbeg(P_UPDATE, s);
  void* e_push = nullptr;
  const bool dd = o.predictor == FEM_PRED_DD && g->n_regions > 0;
  if (dd) {
    e_push = (char*)g->ring + snap_bytes(o.snapshot_format) * (size_t)g->snap_stride * slot_of(g, it);
  }
  CU(launch_newmark_incr(g->n, dt, m->cM, m->cK, m->tp.a0, m->tp.a1, g->x, g->du_ab, g->qM, g->qK, g->u,
                         vslot(it - 1), g->a, vslot(it), g->Ku, g->Mv, g->Kv, g->Pb, aslot(it), e_push,
                         o.snapshot_format, s, Ring4{}, Ring4{},
                         nullptr, g->snap_stride));
  CU(launch_dashpot<double>(m->ab, g->rpad, m->ab.cB, vslot(it), aslot(it), false, m->fm, nullptr, nullptr, nullptr,
                            nullptr, s));
  w->count();
  if (dd && g->hp) {   // heterogeneous scheme: the new correction to the host, the next prediction there
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    CU(hostpred_push(g->hp, e_push, it, ms, s));
  } else if (dd) {
    uint64_t mask = 0;
    const int n_e = std::min(it, g->n_slots);
    for (int j = it - n_e + 1; j <= it; ++j) mask |= 1ull << slot_of(g, j);
    CU(launch_pred_dots(pred_view(bt, g), slot_of(g, it), mask, s));
    w->count();
    // training samples: features of this step's prediction, targets from the solved correction e^it
    if (bt->col_x && g->featured && g->last_npairs > 0) {
      const int64_t rows = (int64_t)g->n_regions * g->ncase;
      if (bt->col_n + rows <= bt->col_cap) {
        if (bt->col_res) {
          CU(mlp_collect_res(pred_view(bt, g), g->slot_lists + kMaxSlots, g->last_npairs, slot_of(g, it), o.tau,
                             g->ncase, g->F, bt->col_n, bt->col_x, bt->col_t, g->e2case, s));
          w->count(2);
        } else {
          PredView pt = pred_view(bt, g);
          pt.w = g->wbest;
          CU(launch_pred_solve(pt, g->slot_lists + kMaxSlots, g->last_npairs, slot_of(g, it), o.tau, s));
          CU(mlp_collect(g->n_regions, g->rpad, g->ncase, g->last_npairs, g->F, g->wbest, g->wcoef, bt->col_n,
                         bt->col_x, bt->col_t, s));
          w->count(2);
        }
        bt->col_n += rows;
      } else {
        bt->col_full = true;
      }
    }
  }
  w->pend(ph, s);
  CU(cudaStreamSynchronize(s));
  w->resolve();
  for (int l = 0; l < g->ncase; ++l) g->last[l] = w->h_sc[l];
  for (int l = 0; l < (int)g->cases.size(); ++l) {
    const CgCase& c = w->h_sc[l];
    g->iters_acc[l] += c.iters;
    g->relres_max[l] = std::max(g->relres_max[l], c.relres);
    if (c.status != FEM_OK && (*worst == FEM_OK || c.status < *worst)) *worst = c.status;
  }
  g->steps = it;
  return FEM_OK;
}

// ------------------------------------------------------------------------------------------------------
// Graph steps.  The FP32-inner step of a group is captured once into a CUDA graph: its kernels read the
// step from a device record (StepCtl) and its loops (refinement passes, inner PCG) are conditional WHILE
// / IF nodes whose conditions the device sets, so a step is one graph launch with no host round trip.
// The periodic direct refresh of the recurrences runs between graph launches.
// ------------------------------------------------------------------------------------------------------
static const int kMaxPass = 40;

static cudaError_t cond_node(cudaStream_t s, cudaGraphConditionalNodeType type, unsigned dflt, unsigned flags,
                             cudaGraphConditionalHandle* h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  e = cudaGraphConditionalHandleCreate(h, graph, dflt, flags);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = *h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, graph, deps, nullptr, nd, &p);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaSuccess;
}

#define GE(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return e_;          \
  } while (0)

// Issues the launches of one step on the capture streams (nothing here synchronises).
static cudaError_t capture_step(fem_batch* bt, Group* g) {
  fem_mesh* m = g->mesh;
  const MeshView mv = m->view();
  Workspace* w = g->ws;
  const Reducer red = w->red();
  const fem_opts& o = bt->opts;
  w->tc = false;
  const double dt = m->tp.dt;
  const int rpad = g->rpad;
  const bool sg = mv.seg != nullptr;
  // FEM_INNER_TC: each pass's inner loop is captured twice, with the FP16 tensor-core product and with the
  // FP32 one; a start kernel runs the one the pass's reduction targets allow (tc_pass) and skips the other
  const bool sel = o.inner_product == FEM_INNER_TC && !sg;
  const bool dd = o.predictor == FEM_PRED_DD && g->n_regions > 0;
  const PredView pv = pred_view(bt, g);
  const Ring4 V{{g->vh[0], g->vh[1], g->vh[2], g->vh[3]}};
  const Ring4 AV{{g->Av[0], g->Av[1], g->Av[2], g->Av[3]}};
  StepCtl* ctl = g->ctl;
  const int ce = std::max(1, o.check_every);
  cudaStream_t s = g->gs[0], s2 = g->gs[1], s3 = g->gs[2], s4 = g->gs[3];
  const bool ab = m->ab.nb > 0;
  const long long n_fixed = 6 + (dd ? 6 + (o.pred_guard ? 1 : 0) : 0) + (g->imp.n > 0 ? 1 : 0) + (ab ? 3 + (dd ? 1 : 0) : 0),
                  n_pass = 4 + (ab ? 1 : 0), n_if = sg ? 4 : (sel ? 3 : 2), n_inner = (ab ? 4LL : 3LL) * ce + 1;
  // 1. step record; the per-region Gram solves (few warps per SM) run beside the right-hand side, which
  // does not depend on them
  GE(launch_step_begin(ctl, dd ? g->n_slots : 0, o.s_max, dt, dd ? 1 : 0, n_fixed, s));
  cudaStream_t sf = g->gs[4];
  GE(cudaEventRecord(g->gev[0], s));
  GE(cudaStreamWaitEvent(sf, g->gev[0], 0));
  // (du_AB of this step was formed at the tail of the previous step's graph, or just before this launch)
  // 2. right-hand side from the recurrences
  GE(launch_rhs_incr(mv, rpad, g->Pb, g->b, g->src, g->ext, 0.0, sf,
                     ctl));
  GE(launch_impulses(g->imp, rpad, 0, ctl, m->fm, g->b, sf));
  if (ab)
    GE(launch_dashpot<double>(m->ab, rpad, 1.0, nullptr, g->b, false, m->fm, nullptr, nullptr, nullptr, nullptr, sf, V,
                              -1, Ring4{}, 0, ctl));
  GE(cudaEventRecord(g->gev[1], sf));
  if (dd) GE(launch_pred_solve(pv, nullptr, 0, 0, o.tau, s, ctl));
  GE(cudaStreamWaitEvent(s, g->gev[1], 0));
  // guess = x = du_AB + Y w, and the correction Y w in FP32 for its residual
  if (dd) {
    GE(launch_pred_combine(pv, nullptr, 0, g->guess, s, ctl, g->du_ab, w->z32, m->reg_gap, m->reg_lead, g->x));
  } else {
    GE(cudaMemcpyAsync(g->guess, g->du_ab, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
    GE(cudaMemcpyAsync(g->x, g->du_ab, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
  }
  // 3. residual of the guess
  const float* qy = nullptr;
  if (dd) {
    GE(ebe_product<float>(m, rpad, w->z32, w->q32, m->cM, m->cK, nullptr, nullptr, nullptr, nullptr, s, true));
    qy = w->q32;
  }
  const bool guard = qy && o.pred_guard;
  if (sg) {
    GE(launch_r0_seg(mv, dt, g->b, nullptr, nullptr, nullptr, nullptr, qy, w->r32, red, w->outer, w->n_active, o.tol,
                     o.inner_tol, o.inner_margin * o.tol, s, AV, ctl, guard, g->fb));
  } else {
    GE(launch_r0(mv, rpad, dt, g->b, nullptr, nullptr, nullptr, nullptr, qy, w->r32, red, w->outer, w->n_active, o.tol,
                 o.inner_tol, o.inner_margin * o.tol, s, AV, ctl, w->sc, guard, g->fb));   // (and the inner solve's starting state)
  }
  if (guard) GE(launch_guard_fix(mv, rpad, w->outer, qy, w->r32, g->du_ab, g->guess, g->x, s));
  // 4. refinement passes: WHILE (pass 0, then while a case is above tol)
  cudaGraphConditionalHandle h_pass, h_if;
  cudaGraph_t b_pass, b_if, tmp;
  GE(cond_node(s, cudaGraphCondTypeWhile, 1, cudaGraphCondAssignDefault, &h_pass, &b_pass));
  GE(cudaStreamBeginCaptureToGraph(s2, b_pass, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  {
    // IF any case is active: inner FP32 PCG on the residual, then x += d
    cudaStreamCaptureStatus cs;
    cudaGraph_t gb = nullptr;
    GE(cudaStreamGetCaptureInfo(s2, &cs, nullptr, &gb, nullptr, nullptr, nullptr));
    GE(cudaGraphConditionalHandleCreate(&h_if, gb, 0, 0));
    GE(launch_pass_begin(w->outer, g->ncase, w->n_active, o.maxit, kMaxPass, ctl, h_if, n_if, s2));
    cudaGraphNodeParams pif{};
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    GE(cudaStreamGetCaptureInfo(s2, &cs, nullptr, &gb, &deps, nullptr, &nd));
    pif.type = cudaGraphNodeTypeConditional;
    pif.conditional.handle = h_if;
    pif.conditional.type = cudaGraphCondTypeIf;
    pif.conditional.size = 1;
    cudaGraphNode_t nif;
    GE(cudaGraphAddNode(&nif, gb, deps, nullptr, nd, &pif));
    GE(cudaStreamUpdateCaptureDependencies(s2, &nif, nullptr, 1, cudaStreamSetCaptureDependencies));
    b_if = pif.conditional.phGraph_out[0];
    GE(cudaStreamBeginCaptureToGraph(s3, b_if, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    {
      // multi-case groups: the residual kernel (r0 or cert) has started the inner solve on r32 in place
      if (sg) GE(launch_norm_b_seg<float>(mv, w->r32, red, w->sc, w->outer, o.inner_tol, s3));
      GE(cudaMemsetAsync(w->x32, 0, sizeof(float) * (size_t)w->n, s3));
      if (sg) GE(launch_resid_seg<float>(mv, w->r32, nullptr, w->x32, w->rr32, w->z32, red, w->sc, w->n_active, s3));
      // the inner PCG: WHILE a case iterates, chunks of ce iterations (want: -1 the loop always starts;
      // 1 / 0 it starts only if the pass does / does not take the tensor-core product)
      auto inner_loop = [&](bool tc_loop, int want) -> cudaError_t {
        cudaGraphConditionalHandle h_in;
        cudaGraph_t gi = nullptr, b_in = nullptr;
        GE(cudaStreamGetCaptureInfo(s3, &cs, nullptr, &gi, nullptr, nullptr, nullptr));
        GE(cudaGraphConditionalHandleCreate(&h_in, gi, 0, 0));
        if (want < 0) {
          GE(launch_inner_start(w->n_active, ctl, h_in, s3));
        } else {
          GE(launch_inner_start_sel(w->n_active, ctl, h_in, w->outer, g->ncase, kTcFloor, want, s3));
        }
        cudaGraphNodeParams pin{};
        GE(cudaStreamGetCaptureInfo(s3, &cs, nullptr, &gi, &deps, nullptr, &nd));
        pin.type = cudaGraphNodeTypeConditional;
        pin.conditional.handle = h_in;
        pin.conditional.type = cudaGraphCondTypeWhile;
        pin.conditional.size = 1;
        cudaGraphNode_t nin;
        GE(cudaGraphAddNode(&nin, gi, deps, nullptr, nd, &pin));
        GE(cudaStreamUpdateCaptureDependencies(s3, &nin, nullptr, 1, cudaStreamSetCaptureDependencies));
        b_in = pin.conditional.phGraph_out[0];
        GE(cudaStreamBeginCaptureToGraph(s4, b_in, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        for (int k = 0; k < ce; ++k) {
          if (sg) {
            GE(launch_dir_seg<float>(mv, w->z32, w->p32, w->sc, w->n_active, s4));
          } else {
            GE(launch_dir_defer<float>(mv, rpad, w->r32, w->p32, w->x32, w->sc, w->n_active, s4));
          }
          GE(ebe_product<float>(m, rpad, w->p32, w->q32, m->cM, m->cK, &red, w->sc, nullptr, w->n_active, s4, true,
                                tc_loop));
          if (sg) {
            GE(launch_update_seg<float>(mv, w->p32, w->q32, w->x32, w->rr32, w->z32, red, w->sc, w->n_active,
                                        o.maxit, s4));
          } else {
            GE(launch_update_defer<float>(mv, rpad, w->q32, w->r32, red, w->sc, w->n_active, o.maxit, s4));
          }
        }
        GE(launch_inner_cond(w->n_active, ctl, h_in, ce, o.maxit + 64 * ce, n_inner, s4));
        return cudaStreamEndCapture(s4, &tmp);
      };
      if (sel) {
        GE(inner_loop(true, 1));
        GE(inner_loop(false, 0));
      } else {
        GE(inner_loop(false, -1));
      }
      if (sg) {
        GE(launch_refine_counts(mv, rpad, g->ncase, g->x, w->x32, w->outer, w->sc, s3));
      } else {
        GE(launch_refine_pending(mv, rpad, g->ncase, g->x, w->x32, w->p32, w->outer, w->sc, s3));
      }
    }
    GE(cudaStreamEndCapture(s3, &tmp));
    // FP64 certification: split products of the increment, true residual, per-case stop test
    GE(split_product(m, o.cert_df, rpad, g->x, g->xdf, g->qM, g->qK, s2));
    if (ab)
      GE(launch_dashpot<double>(m->ab, rpad, m->ab.cB / m->cK, g->x, g->qK, false, m->fm, nullptr, nullptr, nullptr,
                                nullptr, s2));
    if (sg) {
      GE(launch_cert_seg(mv, m->cM, m->cK, g->b, g->qM, g->qK, w->r32, red, w->outer, w->n_active, o.tol, o.inner_tol, o.inner_margin * o.tol,
                         s2));
    } else {
      GE(launch_cert(mv, rpad, m->cM, m->cK, g->b, g->qM, g->qK, w->r32, red, w->outer, w->n_active, o.tol,
                     o.inner_tol, o.inner_margin * o.tol, s2, w->sc));
    }
    GE(launch_pass_end(w->n_active, ctl, h_pass, kMaxPass, n_pass, s2));
  }
  GE(cudaStreamEndCapture(s2, &tmp));
  if (ab)   // (the certification's dashpot term leaves qK: the recurrences advance by K du)
    GE(launch_dashpot<double>(m->ab, rpad, -m->ab.cB / m->cK, g->x, g->qK, false, m->fm, nullptr, nullptr, nullptr,
                              nullptr, s));
  // 5. Newmark update, recurrences, snapshot push, Gram row of the new snapshot, statistics.  With the
  // data-driven predictor the update runs in two parts: the velocity side first (the Gram row reads its
  // snapshot), then the state side on the fork stream beside the Gram row.
  const int n_part = dd ? 1 : 0;
  GE(launch_newmark_incr_part(g->n, dt, m->cM, m->cK, m->tp.a0, m->tp.a1, g->x, g->du_ab, g->qM, g->qK, g->u, nullptr,
                              g->a, nullptr, g->Ku, g->Mv, g->Kv, g->Pb, nullptr, nullptr, o.snapshot_format, s, V,
                              AV, dd ? g->ring : nullptr, g->snap_stride, ctl, n_part));
  // ... and the next step's Adams-Bashforth increment (it reads the velocity ring, now holding v^it; this
  // step's du_AB has been read) on a third stream
  GE(cudaEventRecord(g->gev[2], s));
  GE(cudaStreamWaitEvent(s4, g->gev[2], 0));
  GE(launch_ab4_ring(g->n, dt, V, ctl, g->du_ab, s4, 1));
  GE(cudaEventRecord(g->gev[4], s4));
  if (dd) {
    GE(cudaStreamWaitEvent(sf, g->gev[2], 0));
    GE(launch_newmark_incr_part(g->n, dt, m->cM, m->cK, m->tp.a0, m->tp.a1, g->x, g->du_ab, g->qM, g->qK, g->u,
                                nullptr, g->a, nullptr, g->Ku, g->Mv, g->Kv, g->Pb, nullptr, nullptr,
                                o.snapshot_format, sf, V, AV, nullptr, g->snap_stride, ctl, 2));
    GE(cudaEventRecord(g->gev[3], sf));
  }
  if (ab)
    GE(launch_dashpot<double>(m->ab, rpad, m->ab.cB, nullptr, nullptr, false, m->fm, nullptr, nullptr, nullptr, nullptr,
                              s, V, 0, AV, 0, ctl));
  if (dd) {
    GE(launch_pred_dots(pv, 0, 0, s, ctl));
    GE(cudaStreamWaitEvent(s, g->gev[3], 0));
  }
  GE(cudaStreamWaitEvent(s, g->gev[4], 0));
  GE(launch_step_end(w->outer, g->ncase, g->acc_iters, g->acc_relres, g->acc_status, ctl, s));
  return cudaSuccess;
}
#undef GE

static fem_status group_graph_build(fem_batch* bt, Group* g) {
  if (!g->ctl) {
    CHK(dalloc(&g->ctl, 1));
    CHK(dalloc(&g->acc_iters, (size_t)g->ncase));
    CHK(dalloc(&g->acc_relres, (size_t)g->ncase));
    CHK(dalloc(&g->acc_status, (size_t)g->ncase));
    if (cudaMallocHost((void**)&g->h_pin, 2 * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(FEM_ERR_OOM, "cudaMallocHost failed");
    }
    g->h_pin[0] = 1;
    CU(cudaMemsetAsync(g->ctl, 0, sizeof(StepCtl), bt->s));
    CU(cudaMemsetAsync(g->acc_iters, 0, sizeof(int) * g->ncase, bt->s));
    CU(cudaMemsetAsync(g->acc_relres, 0, sizeof(double) * g->ncase, bt->s));
    CU(cudaMemsetAsync(g->acc_status, 0, sizeof(int) * g->ncase, bt->s));
    for (auto& st : g->gs) CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto& ev : g->gev) CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CU(cudaStreamSynchronize(bt->s));
  }
  {   // operators built on first use are built before the capture (the graph only replays products)
    int v = 0, h = 0;
    g->mesh->resolve(sizeof(float), g->rpad, &v, &h);
    if (v == 7) CHK(g->mesh->ensure_hexmat(bt->s));
    if (v == 8) CHK(g->mesh->ensure_bcsr(bt->s));
  }
  Prof* saved = g->ws->prof;
  g->ws->prof = nullptr;
  cudaError_t e = cudaStreamBeginCapture(g->gs[0], cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = capture_step(bt, g);
  // after an error, end the nested body captures still open (streams 1-3 start their own captures; stream 4
  // only joins the top-level one, which ends with it)
  for (int k = 3; e != cudaSuccess && k >= 1; --k) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(g->gs[k], &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t t = nullptr;
      cudaStreamEndCapture(g->gs[k], &t);
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(g->gs[0], &graph);
  if (e == cudaSuccess) e = e2;
  g->ws->prof = saved;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->gexec, graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    g->gexec = nullptr;
    g->graph_failed = true;
    return fail(FEM_ERR_CUDA, std::string("step graph capture: ") + cudaGetErrorString(e));
  }
  g->graph = graph;
  return FEM_OK;
}

// One graph step: host-side refresh when due, the step counter uploaded if eager steps ran meanwhile,
// external loads flagged, one graph launch.
static fem_status group_step_graph(fem_batch* bt, Group* g) {
  const int it = g->steps + 1;
  const int every = bt->opts.refresh_every > 0 ? bt->opts.refresh_every : 200;
  if (it > 1 && (it - 1) % every == 0) CHK(group_refresh(bt, g));
  cudaStream_t s = bt->s;
  if (g->ctl_it != g->steps) {
    CU(cudaStreamSynchronize(s));           // h_pin[1] may still be read by an earlier upload
    g->h_pin[1] = g->steps;
    CU(cudaMemcpyAsync(&g->ctl->it, &g->h_pin[1], sizeof(int), cudaMemcpyHostToDevice, s));
  }
  if (g->use_ext) CU(cudaMemcpyAsync(&g->ctl->use_ext, &g->h_pin[0], sizeof(int), cudaMemcpyHostToDevice, s));
  g->use_ext = false;
  if (g->ab_ready != it) {   // the first graph step, or after eager steps: this step's du_AB before the graph
    const Ring4 V{{g->vh[0], g->vh[1], g->vh[2], g->vh[3]}};
    CU(launch_ab4_ring(g->n, g->mesh->tp.dt, V, g->ctl, g->du_ab, s, 1));
    g->ws->count();
  }
  CU(cudaGraphLaunch(g->gexec, s));
  g->steps = it;
  g->ctl_it = it;
  g->ab_ready = it + 1;
  g->graph_steps += 1;
  return FEM_OK;
}

// After graph steps: per-case statistics (accumulated on the device) and the last step's solver state.
static fem_status group_graph_stats(fem_batch* bt, Group* g, fem_status* worst) {
  if (g->graph_steps == 0) return FEM_OK;
  cudaStream_t s = bt->s;
  std::vector<int> it_acc(g->ncase), st_acc(g->ncase);
  std::vector<double> rr_acc(g->ncase);
  long long launches = 0;
  CU(cudaMemcpyAsync(it_acc.data(), g->acc_iters, sizeof(int) * g->ncase, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(rr_acc.data(), g->acc_relres, sizeof(double) * g->ncase, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(st_acc.data(), g->acc_status, sizeof(int) * g->ncase, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(&launches, &g->ctl->launches, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(g->ws->h_sc, g->ws->outer, sizeof(CgCase) * g->ncase, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  CU(cudaMemsetAsync(g->acc_iters, 0, sizeof(int) * g->ncase, s));
  CU(cudaMemsetAsync(g->acc_relres, 0, sizeof(double) * g->ncase, s));
  CU(cudaMemsetAsync(g->acc_status, 0, sizeof(int) * g->ncase, s));
  CU(cudaMemsetAsync(&g->ctl->launches, 0, sizeof(long long), s));
  for (int l = 0; l < g->ncase; ++l) g->last[l] = g->ws->h_sc[l];
  for (int l = 0; l < (int)g->cases.size(); ++l) {
    g->iters_acc[l] += it_acc[l];
    g->relres_max[l] = std::max(g->relres_max[l], rr_acc[l]);
    if (st_acc[l] != FEM_OK && (*worst == FEM_OK || st_acc[l] < *worst)) *worst = st_acc[l];
  }
  if (bt->prof.on) bt->prof.launches += launches;
  g->graph_steps = 0;
  return FEM_OK;
}

static bool graph_eligible(const fem_batch* bt, const Group* g) {
  return bt->opts.use_graph && bt->opts.precision == FEM_FP32_INNER && !bt->mlp && !bt->col_x && !g->hp &&
         !(bt->prof.on && bt->prof.events);
}

static fem_status group_step(fem_batch* bt, Group* g, fem_status* worst) {
  if (graph_eligible(bt, g)) {
    if (!g->gexec) CHK(group_graph_build(bt, g));     // use_graph was asked for: a failed capture is an error
    return group_step_graph(bt, g);
  }
  if (g->graph_steps) CHK(group_graph_stats(bt, g, worst));
  g->ctl_it = -1;
  if (bt->opts.precision == FEM_FP32_INNER) return group_step_mixed(bt, g, worst);
  if (g->owned_mesh) return fail(FEM_ERR_ARG, "fused meshes need the FP32-inner solver");
  const auto t_start = std::chrono::steady_clock::now();
  fem_mesh* m = g->mesh;
  const MeshView mv = m->view();
  cudaStream_t s = bt->s;
  const int it = g->steps + 1;
  const double dt = m->tp.dt;
  auto vslot = [&](int j) { return g->vh[((j % 4) + 4) % 4]; };
  Workspace* w = g->ws;
  // 1. initial guess (Section 3.2)
  int ph = w->pbeg(P_PREDICT, s);
  CHK(group_predict(bt, g, g->guess));
  w->pend(ph, s);
  // 2. Newmark right-hand side (Section 3.1, Eq. GE:DIS, increment form)
  ph = w->pbeg(P_RHS, s);
  CU(launch_rhs_prep(g->n, dt, m->tp.a0, m->tp.a1, g->u, vslot(it - 1), g->a, g->m_in, g->k_in, s));
  int pe = w->pbeg(P_EBE64, s);
  if (m->npe == 10) {
    CU(launch_ebe10_gated<double>(m->E, m->N, g->rpad, m->conn10, m->rec32, m->rec64, m->fm, g->m_in, g->k_in, g->b,
                                  1.0, 1.0, nullptr, nullptr, nullptr, nullptr, s));
  } else {
    CU(launch_ebe<double>(mv, g->rpad, g->m_in, g->k_in, g->b, 1.0, 1.0, nullptr, nullptr, nullptr, s));
  }
  w->pend(pe, s);
  CU(launch_rhs_finish(mv, g->rpad, g->b, g->src, g->use_ext ? g->ext : nullptr, it * dt, s));
  CU(launch_impulses(g->imp, g->rpad, it, nullptr, m->fm, g->b, s));
  CU(launch_dashpot<double>(m->ab, g->rpad, 1.0, vslot(it - 1), g->b, false, m->fm, nullptr, nullptr, nullptr, nullptr,
                            s));
  g->use_ext = false;
  w->pend(ph, s);
  w->count(3);
  // 3. certified solve of A du = b from the guess (Algorithm 1)
  ph = w->pbeg(P_SOLVE, s);
  CU(cudaMemcpyAsync(g->x, g->guess, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, s));
  CgCase* res = nullptr;
  CHK(solve_any(m, g->ws, g->b, g->x, bt->opts, s, &res));
  w->pend(ph, s);
  CU(cudaMemcpyAsync(g->ws->h_sc, res, sizeof(CgCase) * g->rpad, cudaMemcpyDeviceToHost, s));
  ph = w->pbeg(P_UPDATE, s);
  // 4. Newmark update and snapshot push (Section 3.1, Eq. timestep)
  void* e_push = nullptr;
  const bool dd = bt->opts.predictor == FEM_PRED_DD && g->n_regions > 0;
  if (dd) {
    e_push = (char*)g->ring + snap_bytes(bt->opts.snapshot_format) * (size_t)g->snap_stride * slot_of(g, it);
  }
  CU(launch_newmark_update(g->n, dt, g->x, g->du_ab, g->u, vslot(it - 1), g->a, vslot(it), e_push,
                           bt->opts.snapshot_format, g->snap_stride, s));
  w->count();
  if (dd && g->hp) {
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    CU(hostpred_push(g->hp, e_push, it, ms, s));
  } else if (dd) {
    uint64_t mask = 0;
    const int n_e = std::min(it, g->n_slots);
    for (int j = it - n_e + 1; j <= it; ++j) mask |= 1ull << slot_of(g, j);
    CU(launch_pred_dots(pred_view(bt, g), slot_of(g, it), mask, s));
    w->count();
  }
  w->pend(ph, s);
  CU(cudaStreamSynchronize(s));
  w->resolve();
  for (int l = 0; l < g->rpad; ++l) g->last[l] = g->ws->h_sc[l];
  for (int l = 0; l < (int)g->cases.size(); ++l) {
    const CgCase& c = g->ws->h_sc[l];
    g->iters_acc[l] += c.iters;
    g->relres_max[l] = std::max(g->relres_max[l], c.relres);
    if (c.status != FEM_OK && (*worst == FEM_OK || c.status < *worst)) *worst = c.status;
  }
  g->steps = it;
  return FEM_OK;
}

namespace fem {
fem_status set_error(fem_status s, const std::string& msg) { return fail(s, msg); }
void clear_error() { g_err.clear(); }
void mesh_view_of(const fem_mesh* m, MeshView* view, int* device, const int32_t** conn10) {
  *view = m->view();
  *device = m->device;
  *conn10 = m->npe == 10 ? m->conn10 : nullptr;
}
}  // namespace fem

// ------------------------------------------------------------------------------------------------------
// C-ABI
// ------------------------------------------------------------------------------------------------------
// Times every EBE implementation that applies to the mesh (generic element kernel; tiled hex kernel with
// 64/128/256/512 hexes per tile when its accumulator fits shared memory) on the product the inner solve
// uses (A p with the fused p^T A p), and keeps the fastest for this precision and case count.
template <typename T>
static fem_status autotune_t(fem_mesh* m, int rpad, cudaStream_t s, int* v_out, int* h_out, double* ms_out) {
  Workspace* w = nullptr;
  CHK(m->workspace(rpad, &w));
  const Reducer red = w->red();
  const size_t n = (size_t)m->N * 3 * rpad;
  T *p = nullptr, *q = nullptr;
  double* ptq = nullptr;
  CHK(dalloc(&p, n));
  CHK(dalloc(&q, n));
  CHK(dalloc(&ptq, (size_t)rpad));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fem_status st = FEM_OK;
  const int sv = m->ebe_variant, sh = m->hex_per_tile;
  int lg = 0;
  while ((1 << lg) < rpad) ++lg;
  std::vector<std::pair<int, int>> cand = {{1, 0}};
  if (m->hex) {
    for (int hpt : {64, 128, 256, 512}) cand.push_back({2, hpt});
    for (int hpt : {64, 128, 256}) cand.push_back({3, hpt});
    for (int hpt : {64, 128}) cand.push_back({4, hpt});
    if (sizeof(T) == 4 && rpad >= 4 && !m->seg) {
      for (int hpt : {64, 128}) cand.push_back({5, hpt});
      for (int hpt : {64, 128, 256}) cand.push_back({6, hpt});
      cand.push_back({7, 64});
    }
  }
  if (!m->seg) cand.push_back({8, 0});
  double best = 1e30;
  int bv = 1, bh = 0;
  cudaError_t e = cudaMemsetAsync(p, 0, n * sizeof(T), s);
  for (auto [v, hpt] : cand) {
    if (e != cudaSuccess) break;
    m->ebe_variant = v, m->hex_per_tile = hpt;
    if (v >= 2 && v <= 7) {
      const HexTiles* t = m->tiles_for(sizeof(T), rpad, v, hpt);
      if (!t || t->hex_per_tile != hpt) continue;   // this tiling does not fit
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      e = ebe_product<T>(m, rpad, p, q, m->cM, m->cK, &red, w->sc, ptq, nullptr, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    const int reps = 5;
    for (int k = 0; k < reps && e == cudaSuccess; ++k)
      e = ebe_product<T>(m, rpad, p, q, m->cM, m->cK, &red, w->sc, ptq, nullptr, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms / reps < best) best = ms / reps, bv = v, bh = hpt;
  }
  m->ebe_variant = sv, m->hex_per_tile = sh;
  if (e != cudaSuccess) {
    cudaGetLastError();
    st = fail(FEM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  } else {
    m->tuned[sizeof(T) == 4 ? 0 : 1][lg] = {bv, bh};
    if (v_out) *v_out = bv;
    if (h_out) *h_out = bh;
    if (ms_out) *ms_out = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(p);
  dfree(q);
  dfree(ptq);
  return st;
}

extern "C" {

const char* fem_last_error(void) { return g_err.c_str(); }

void fem_opts_default(fem_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = FEM_FP64;
  o->predictor = FEM_PRED_AB4;
  o->tol = 1e-8;
  o->maxit = 5000;
  o->s_max = 32;
  o->inner_tol = 1e-6;
  o->tau = 1e-6;
  o->snapshot_format = 2;
  o->check_every = 8;
  o->refresh_every = 200;
  o->cert_df = 3;
  o->fuse_meshes = 0;
  o->use_graph = 1;
  o->wait_budget = kDefaultWaitBudget;
  o->inner_margin = 0.5;
  o->inner_product = FEM_INNER_FP32;
  o->pred_guard = 1;
}

// Mesh set-up shared by the linear (npe 4) and quadratic (npe 10) tets: element records of the corner tets,
// block-Jacobi diagonal of the element type, and (linear tets in hex patches) the hex tiles.
static fem_status mesh_create(int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn_in, int npe,
                              const int32_t* mat_id, int n_mat, const double* lam_mu_rho, const uint8_t* fixed_dof,
                              const fem_time_params* tp, void* stream, fem_mesh** out) {
  g_err.clear();
  if (!out) return fail(FEM_ERR_ARG, "out is null");
  *out = nullptr;
  if (!xyz || !conn_in || !mat_id || !lam_mu_rho || !fixed_dof || !tp) return fail(FEM_ERR_ARG, "null input pointer");
  if (n_nodes < npe || n_elems < 1 || n_mat < 1) return fail(FEM_ERR_ARG, "empty mesh");
  if (n_nodes > INT32_MAX) return fail(FEM_ERR_ARG, "node ids must fit int32");
  std::vector<int32_t> corners;
  const int32_t* conn = conn_in;
  if (npe == 10) {   // the corner tets carry the element records; the edge nodes are checked here
    for (int64_t i = 0; i < 10 * n_elems; ++i)
      if (conn_in[i] < 0 || conn_in[i] >= n_nodes) return fail(FEM_ERR_ARG, "connectivity out of range");
    corners.resize(4 * (size_t)n_elems);
    for (int64_t e = 0; e < n_elems; ++e)
      for (int a = 0; a < 4; ++a) corners[4 * e + a] = conn_in[10 * e + a];
    conn = corners.data();
  }
  if (tp->beta != 0.25 || tp->gamma != 0.5) return fail(FEM_ERR_ARG, "only Newmark beta=1/4, gamma=1/2 is supported");
  if (!(tp->dt > 0.0)) return fail(FEM_ERR_ARG, "dt must be > 0");
  for (int i = 0; i < n_mat; ++i)
    if (!(lam_mu_rho[3 * i + 1] > 0.0) || !(lam_mu_rho[3 * i + 2] > 0.0) ||
        !(lam_mu_rho[3 * i] + 2.0 / 3.0 * lam_mu_rho[3 * i + 1] > 0.0))
      return fail(FEM_ERR_ARG, "material parameters must give a positive-definite elasticity tensor");
  cudaStream_t s = (cudaStream_t)stream;
  fem_mesh* m = new fem_mesh();
  cudaGetDevice(&m->device);
  m->h_xyz.assign(xyz, xyz + 3 * n_nodes);
  m->h_conn.assign(conn_in, conn_in + (size_t)npe * n_elems);
  m->npe = npe;
  m->h_mat.assign(mat_id, mat_id + n_elems);
  m->h_lmr.assign(lam_mu_rho, lam_mu_rho + 3 * n_mat);
  m->h_fixed.assign(fixed_dof, fixed_dof + 3 * n_nodes);
  m->N = n_nodes;
  m->E = n_elems;
  m->tp = *tp;
  m->cM = 4.0 / (tp->dt * tp->dt) + 2.0 * tp->a0 / tp->dt;
  m->cK = 1.0 + 2.0 * tp->a1 / tp->dt;
  std::vector<uint8_t> fm(n_nodes);
  for (int64_t n = 0; n < n_nodes; ++n)
    fm[n] = (uint8_t)((fixed_dof[3 * n] ? 0 : 1) | (fixed_dof[3 * n + 1] ? 0 : 2) | (fixed_dof[3 * n + 2] ? 0 : 4));
  fem_status st = FEM_OK;
  auto bail = [&](fem_status e) {
    delete m;
    return e;
  };
  if ((st = dalloc(&m->xyz, 3 * n_nodes)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->conn, n_elems)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->mat, n_elems)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->lmr, 3 * n_mat)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->rec64, kRec * n_elems)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->rec32, kRec * n_elems)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->rec_df, 2 * kRec * n_elems)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->D, 6 * n_nodes)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->binv64, 6 * n_nodes)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->binv32, 6 * n_nodes)) != FEM_OK) return bail(st);
  if ((st = dalloc(&m->fm, n_nodes)) != FEM_OK) return bail(st);
  int* d_err = nullptr;
  if ((st = dalloc(&d_err, 1)) != FEM_OK) return bail(st);
  cudaError_t e = cudaSuccess;
  auto cu = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  cu(cudaMemcpyAsync(m->xyz, xyz, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice, s));
  cu(cudaMemcpyAsync(m->conn, conn, sizeof(int4) * n_elems, cudaMemcpyHostToDevice, s));
  cu(cudaMemcpyAsync(m->mat, mat_id, sizeof(int32_t) * n_elems, cudaMemcpyHostToDevice, s));
  cu(cudaMemcpyAsync(m->lmr, lam_mu_rho, sizeof(double) * 3 * n_mat, cudaMemcpyHostToDevice, s));
  cu(cudaMemcpyAsync(m->fm, fm.data(), n_nodes, cudaMemcpyHostToDevice, s));
  cu(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  cu(cudaMemsetAsync(m->D, 0, sizeof(double) * 6 * n_nodes, s));
  cu(launch_elem_setup(n_elems, n_nodes, m->xyz, m->conn, m->mat, n_mat, m->lmr, m->rec64, m->rec32, d_err, s));
  if (npe == 10) {
    if (dalloc(&m->conn10, 10 * (size_t)n_elems) != FEM_OK) {
      cudaFree(d_err);
      return bail(FEM_ERR_OOM);
    }
    cu(cudaMemcpyAsync(m->conn10, conn_in, sizeof(int32_t) * 10 * n_elems, cudaMemcpyHostToDevice, s));
    cu(launch_diag10(n_elems, m->conn10, m->rec64, m->cM, m->cK, m->D, s));
  } else {
    cu(launch_diag_blocks(m->view(), m->cM, m->cK, m->D, s));
  }
  cu(launch_split_records(n_elems, m->rec64, m->rec_df, s));
  cu(launch_binv(n_nodes, m->D, m->fm, m->binv64, m->binv32, d_err, s));
  int h_err = 0;
  cu(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  cu(cudaStreamSynchronize(s));
  cudaFree(d_err);
  if (e != cudaSuccess) {
    delete m;
    return fail(FEM_ERR_CUDA, std::string("mesh setup: ") + cudaGetErrorString(e));
  }
  if (h_err & 1) return bail(fail(FEM_ERR_ARG, "connectivity or material id out of range"));
  if (h_err & 2) return bail(fail(FEM_ERR_ARG, "element with non-positive volume (conn must be positively oriented)"));
  if (h_err & 4) return bail(fail(FEM_ERR_ARG, "singular node diagonal block (node with no element?)"));
  // tile node entries carry the node id (bits 0-27), its three free-DOF bits (28-30) and whether another
  // tile shares the node (bit 31): the kernels' flush needs no separate mask load
  if (npe == 4 && n_nodes < (int64_t(1) << 28) && detect_hex_patches(conn, n_elems)) {
    const int sizes[fem_mesh::kNTile] = {32, 64, 128, 256, 512};
    bool ok = true;
    double abs_m = 0.0, abs_k = 0.0;   // scale bounds of the packed kernel's fixed-point tile sums
    {
      cudaError_t ce = elem_abs_row_bounds(m->view(), &abs_m, &abs_k, s);
      if (ce != cudaSuccess) return bail(fail(FEM_ERR_CUDA, std::string("row bounds: ") + cudaGetErrorString(ce)));
    }
    for (int i = 0; i < fem_mesh::kNTile && ok; ++i) {
      HexTilesHost th;
      if (!build_hex_tiles(conn, n_elems, n_nodes, sizes[i], &th)) continue;
      for (int& v : th.tile_nodes) {
        const uint32_t u = (uint32_t)v, node = u & 0x7fffffffu;
        v = (int)((u & 0x80000000u) | ((uint32_t)(fm[node] & 7u) << 28) | node);
      }
      int *d_hoff = nullptr, *d_noff = nullptr, *d_nodes = nullptr;
      uint4* d_loc = nullptr;
      ok = dalloc(&d_hoff, th.tile_hex_off.size()) == FEM_OK && dalloc(&d_noff, th.tile_node_off.size()) == FEM_OK &&
           dalloc(&d_nodes, th.tile_nodes.size()) == FEM_OK && dalloc(&d_loc, (size_t)th.n_hex) == FEM_OK;
      for (void* b : {(void*)d_hoff, (void*)d_noff, (void*)d_nodes, (void*)d_loc})
        if (b) m->tile_bufs.push_back(b);
      if (!ok) break;
      cudaError_t ce = cudaMemcpy(d_hoff, th.tile_hex_off.data(), sizeof(int) * th.tile_hex_off.size(), cudaMemcpyHostToDevice);
      if (ce == cudaSuccess) ce = cudaMemcpy(d_noff, th.tile_node_off.data(), sizeof(int) * th.tile_node_off.size(), cudaMemcpyHostToDevice);
      if (ce == cudaSuccess) ce = cudaMemcpy(d_nodes, th.tile_nodes.data(), sizeof(int) * th.tile_nodes.size(), cudaMemcpyHostToDevice);
      if (ce == cudaSuccess) ce = cudaMemcpy(d_loc, th.hex_local.data(), sizeof(uint16_t) * th.hex_local.size(), cudaMemcpyHostToDevice);
      if (ce != cudaSuccess) return bail(fail(FEM_ERR_CUDA, std::string("tile upload: ") + cudaGetErrorString(ce)));
      HexTiles& t = m->tiles[i];
      t.n_tiles = th.n_tiles;
      t.nloc_max = th.nloc_max;
      t.hex_per_tile = th.hex_per_tile;
      t.tile_hex_off = d_hoff;
      t.tile_node_off = d_noff;
      t.tile_nodes = d_nodes;
      t.hex_local = d_loc;
      // (rounded up to FP32 and given 1% more for the FP32 rounding of the records and products)
      t.abs_m = (float)(abs_m * 1.01);
      t.abs_k = (float)(abs_k * 1.01);
    }
    if (!ok) return bail(fail(FEM_ERR_OOM, "tile allocation failed"));
    m->hex = true;
  }
  *out = m;
  return FEM_OK;
}

fem_status fem_mesh_create(int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn,
                           const int32_t* mat_id, int n_mat, const double* lam_mu_rho, const uint8_t* fixed_dof,
                           const fem_time_params* tp, void* stream, fem_mesh** out) {
  return mesh_create(n_nodes, xyz, n_elems, conn, 4, mat_id, n_mat, lam_mu_rho, fixed_dof, tp, stream, out);
}

fem_status fem_mesh_create_tet10(int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn10,
                                 const int32_t* mat_id, int n_mat, const double* lam_mu_rho,
                                 const uint8_t* fixed_dof, const fem_time_params* tp, void* stream, fem_mesh** out) {
  return mesh_create(n_nodes, xyz, n_elems, conn10, 10, mat_id, n_mat, lam_mu_rho, fixed_dof, tp, stream, out);
}

fem_status fem_mesh_set_absorbing(fem_mesh* m, int64_t n_faces, const int32_t* faces, void* stream) {
  g_err.clear();
  if (!m) return fail(FEM_ERR_ARG, "mesh is null");
  if (n_faces < 0 || (n_faces > 0 && !faces)) return fail(FEM_ERR_ARG, "bad face list");
  if (m->seg) return fail(FEM_ERR_ARG, "a fused virtual mesh takes no absorbing faces");
  if (m->npe != 4) return fail(FEM_ERR_ARG, "absorbing faces are supported on linear-tet meshes only");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = m->N;
  // node -> elements incidence
  std::vector<int64_t> ip(N + 1, 0);
  for (int32_t v : m->h_conn) ip[v + 1] += 1;
  for (int64_t k = 0; k < N; ++k) ip[k + 1] += ip[k];
  std::vector<int32_t> inc(m->h_conn.size());
  {
    std::vector<int64_t> pos(ip.begin(), ip.end() - 1);
    for (size_t i = 0; i < m->h_conn.size(); ++i) inc[pos[m->h_conn[i]]++] = (int32_t)(i / 4);
  }
  std::unordered_map<int32_t, std::array<double, 6>> blk;
  for (int64_t f = 0; f < n_faces; ++f) {
    const int32_t a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
    if (a < 0 || a >= N || b < 0 || b >= N || c < 0 || c >= N || a == b || b == c || a == c)
      return fail(FEM_ERR_ARG, "absorbing face " + std::to_string(f) + ": bad node ids");
    int owner = -1, opp = -1, count = 0;
    for (int64_t k = ip[a]; k < ip[a + 1]; ++k) {
      const int32_t e = inc[k];
      const int32_t* nd = &m->h_conn[4 * (size_t)e];
      bool hb = false, hc = false;
      int other = -1;
      for (int j = 0; j < 4; ++j) {
        hb = hb || nd[j] == b;
        hc = hc || nd[j] == c;
        if (nd[j] != a && nd[j] != b && nd[j] != c) other = nd[j];
      }
      if (hb && hc) owner = e, opp = other, count += 1;
    }
    if (count != 1)
      return fail(FEM_ERR_ARG, "absorbing face " + std::to_string(f) + " is not a face of exactly one element");
    const double* X = m->h_xyz.data();
    double e1[3], e2[3], w[3], nrm[3];
    for (int d = 0; d < 3; ++d) e1[d] = X[3 * b + d] - X[3 * a + d], e2[d] = X[3 * c + d] - X[3 * a + d],
                                w[d] = X[3 * opp + d] - X[3 * a + d];
    nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double len = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    if (!(len > 0.0)) return fail(FEM_ERR_ARG, "absorbing face " + std::to_string(f) + " has zero area");
    double n[3] = {nrm[0] / len, nrm[1] / len, nrm[2] / len};
    if (n[0] * w[0] + n[1] * w[1] + n[2] * w[2] > 0.0) n[0] = -n[0], n[1] = -n[1], n[2] = -n[2];   // outward
    const int mid = m->h_mat[owner];
    const double lam = m->h_lmr[3 * mid], mu = m->h_lmr[3 * mid + 1], rho = m->h_lmr[3 * mid + 2];
    const double cp = std::sqrt((lam + 2.0 * mu) / rho), cs = std::sqrt(mu / rho);
    const double sc = 0.5 * len / 3.0 * rho;   // a third of the face's area, times rho
    const int ij[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int32_t node : {a, b, c}) {
      auto& B = blk[node];
      for (int q = 0; q < 6; ++q) {
        const int i = ij[q][0], j = ij[q][1];
        B[q] += sc * (cp * n[i] * n[j] + cs * ((i == j ? 1.0 : 0.0) - n[i] * n[j]));
      }
    }
  }
  std::vector<int32_t> nodes;
  nodes.reserve(blk.size());
  for (const auto& kv : blk) nodes.push_back(kv.first);
  std::sort(nodes.begin(), nodes.end());
  std::vector<double> c64(6 * nodes.size());
  std::vector<float> c32(6 * nodes.size());
  for (size_t k = 0; k < nodes.size(); ++k)
    for (int q = 0; q < 6; ++q) c64[6 * k + q] = blk[nodes[k]][q], c32[6 * k + q] = (float)c64[6 * k + q];
  dfree(m->ab_node); dfree(m->ab_c64); dfree(m->ab_c32);
  m->ab = Absorb{};
  if (!nodes.empty()) {
    CHK(dalloc(&m->ab_node, nodes.size()));
    CHK(dalloc(&m->ab_c64, c64.size()));
    CHK(dalloc(&m->ab_c32, c32.size()));
    CU(cudaMemcpyAsync(m->ab_node, nodes.data(), sizeof(int32_t) * nodes.size(), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(m->ab_c64, c64.data(), sizeof(double) * c64.size(), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(m->ab_c32, c32.data(), sizeof(float) * c32.size(), cudaMemcpyHostToDevice, s));
    m->ab = Absorb{(int)nodes.size(), m->ab_node, m->ab_c64, m->ab_c32, 2.0 / m->tp.dt};
  }
  // block-Jacobi diagonal of A = cM M + cK K + (2/dt) C_b, recomputed from scratch
  int* d_err = nullptr;
  CHK(dalloc(&d_err, 1));
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->D, 0, sizeof(double) * 6 * N, s);
  if (e == cudaSuccess) e = launch_diag_blocks(m->view(), m->cM, m->cK, m->D, s);
  if (e == cudaSuccess) e = launch_add_node_blocks(m->ab, m->ab.cB, m->D, s);
  if (e == cudaSuccess) e = launch_binv(N, m->D, m->fm, m->binv64, m->binv32, d_err, s);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_err);
  if (e != cudaSuccess) return fail(FEM_ERR_CUDA, std::string("fem_mesh_set_absorbing: ") + cudaGetErrorString(e));
  if (h_err) return fail(FEM_ERR_ARG, "singular node diagonal block");
  m->h_ab_faces.assign(faces, faces + 3 * n_faces);
  return FEM_OK;
}

fem_status fem_mesh_destroy(fem_mesh* m) {
  if (!m) return fail(FEM_ERR_ARG, "mesh is null");
  cudaDeviceSynchronize();
  delete m;
  return FEM_OK;
}

fem_status fem_mesh_tune(fem_mesh* m, int ebe_variant, int hex_per_tile) {
  g_err.clear();
  if (!m) return fail(FEM_ERR_ARG, "mesh is null");
  if (ebe_variant < 0 || ebe_variant > 9) return fail(FEM_ERR_ARG, "ebe_variant must be 0 .. 9");
  if (m->npe == 10 && ebe_variant != 0 && ebe_variant != 8)
    return fail(FEM_ERR_ARG, "a tet10 mesh takes variant 0 (its element kernel) or 8 (assembled blocks)");
  if (((ebe_variant >= 2 && ebe_variant <= 7) || ebe_variant == 9) && !m->hex)
    return fail(FEM_ERR_ARG, "the mesh has no hex patches: tiled kernel unavailable");
  if (hex_per_tile != 0 && hex_per_tile != 64 && hex_per_tile != 128 && hex_per_tile != 256 && hex_per_tile != 512)
    return fail(FEM_ERR_ARG, "hex_per_tile must be 0, 64, 128, 256 or 512");
  m->ebe_variant = ebe_variant;
  m->hex_per_tile = hex_per_tile;
  return FEM_OK;
}

fem_status fem_mesh_autotune(fem_mesh* m, int precision, int n_rhs, void* stream, int* ebe_variant_out,
                             int* hex_per_tile_out, double* ms_out) {
  g_err.clear();
  if (!m) return fail(FEM_ERR_ARG, "mesh is null");
  if (!pow2_rhs(n_rhs)) return fail(FEM_ERR_ARG, "n_rhs must be 1, 2, 4, 8, 16 or 32");
  if (m->npe != 4) return fail(FEM_ERR_ARG, "fem_mesh_autotune: linear-tet meshes only (fem_mesh_tune selects "
                                           "a tet10 mesh's product)");
  cudaStream_t s = (cudaStream_t)stream;
  CU(ebe_set_wait_budget(kDefaultWaitBudget, s));
  if (precision == FEM_FP64) return autotune_t<double>(m, n_rhs, s, ebe_variant_out, hex_per_tile_out, ms_out);
  if (precision == FEM_FP32_INNER) return autotune_t<float>(m, n_rhs, s, ebe_variant_out, hex_per_tile_out, ms_out);
  return fail(FEM_ERR_ARG, "unknown precision");
}

fem_status fem_mesh_split_product(fem_mesh* m, int mode, const double* p_dev, double* qM_dev, double* qK_dev,
                                  int n_rhs, void* stream) {
  g_err.clear();
  if (!m || !p_dev || !qM_dev || !qK_dev) return fail(FEM_ERR_ARG, "null argument");
  if (!pow2_rhs(n_rhs)) return fail(FEM_ERR_ARG, "n_rhs must be 1, 2, 4, 8, 16 or 32");
  if (mode < 0 || mode > 3) return fail(FEM_ERR_ARG, "mode must be 0, 1, 2 or 3");
  cudaStream_t s = (cudaStream_t)stream;
  float2* pdf = nullptr;
  if (mode >= 2) CHK(m->ensure_bcsr(s));
  if (mode == 3) CHK(dalloc(&pdf, (size_t)m->N * 3 * n_rhs));
  cudaError_t e = split_product(m, mode, n_rhs, p_dev, pdf, qM_dev, qK_dev, s);
  if (e == cudaSuccess && mode < 2) {   // the element forms leave Dirichlet rows to their consumers
    e = launch_mask<double>(m->N, n_rhs, m->fm, qM_dev, s);
    if (e == cudaSuccess) e = launch_mask<double>(m->N, n_rhs, m->fm, qK_dev, s);
  }
  if (pdf) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(pdf);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(FEM_ERR_CUDA, std::string("fem_mesh_split_product: ") + cudaGetErrorString(e));
  }
  return FEM_OK;
}

fem_status fem_mesh_info(const fem_mesh* m, int* has_hex_patches, int* ebe_variant, int* hex_per_tile) {
  if (!m) return fail(FEM_ERR_ARG, "mesh is null");
  if (has_hex_patches) *has_hex_patches = m->hex ? 1 : 0;
  if (ebe_variant) *ebe_variant = m->ebe_variant;
  if (hex_per_tile) *hex_per_tile = m->hex_per_tile;
  return FEM_OK;
}

fem_status fem_mesh_set_regions(fem_mesh* m, const int32_t* region_of_node) {
  g_err.clear();
  if (!m || !region_of_node) return fail(FEM_ERR_ARG, "null argument");
  int R = 0;
  for (int64_t n = 0; n < m->N; ++n) {
    if (region_of_node[n] < -1) return fail(FEM_ERR_ARG, "region id < -1");
    R = std::max(R, region_of_node[n] + 1);
  }
  std::vector<int32_t> lo(R, INT32_MAX), hi(R, -1);
  for (int64_t n = 0; n < m->N; ++n) {
    const int r = region_of_node[n];
    if (r < 0) continue;
    lo[r] = std::min<int32_t>(lo[r], (int32_t)n);
    hi[r] = std::max<int32_t>(hi[r], (int32_t)n + 1);
  }
  for (int r = 0; r < R; ++r) {
    if (hi[r] < 0) return fail(FEM_ERR_ARG, "empty region id " + std::to_string(r));
    for (int64_t n = lo[r]; n < hi[r]; ++n)
      if (region_of_node[n] != r && region_of_node[n] != -1)
        return fail(FEM_ERR_ARG, "region " + std::to_string(r) + " is not a contiguous node range");
  }
  dfree(m->reg_lo);
  dfree(m->reg_hi);
  dfree(m->reg_gap);
  dfree(m->reg_cent);
  m->n_regions = 0;
  m->h_region.assign(region_of_node, region_of_node + m->N);
  // region centroids and the domain extent (inputs of the learned proposal)
  std::vector<double> cs(3 * (size_t)R, 0.0), cnt(R, 0.0);
  double bmin[3] = {INFINITY, INFINITY, INFINITY}, bmax[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t n = 0; n < m->N; ++n) {
    for (int k = 0; k < 3; ++k) {
      bmin[k] = std::min(bmin[k], m->h_xyz[3 * n + k]);
      bmax[k] = std::max(bmax[k], m->h_xyz[3 * n + k]);
    }
    const int r = region_of_node[n];
    if (r < 0) continue;
    for (int k = 0; k < 3; ++k) cs[3 * (size_t)r + k] += m->h_xyz[3 * n + k];
    cnt[r] += 1.0;
  }
  std::vector<float> cf(3 * (size_t)R);
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < 3; ++k) cf[3 * (size_t)r + k] = (float)(cs[3 * (size_t)r + k] / cnt[r]);
  const double ext = std::max(bmax[0] - bmin[0], std::max(bmax[1] - bmin[1], bmax[2] - bmin[2]));
  m->inv_extent = ext > 0.0 ? (float)(1.0 / ext) : 1.0f;
  // node gaps between the ranges (ranges are disjoint): the gap after region r ends at the next range's start
  std::vector<int32_t> gap(R, (int32_t)m->N);
  {
    std::vector<int> order(R);
    for (int r = 0; r < R; ++r) order[r] = r;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return lo[x] < lo[y]; });
    for (int i = 0; i + 1 < R; ++i) gap[order[i]] = lo[order[i + 1]];
    m->reg_lead = R > 0 ? lo[order[0]] : 0;
  }
  CHK(dalloc(&m->reg_lo, R));
  CHK(dalloc(&m->reg_hi, R));
  CHK(dalloc(&m->reg_gap, R));
  CHK(dalloc(&m->reg_cent, 3 * (int64_t)R));
  CU(cudaMemcpy(m->reg_lo, lo.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(m->reg_hi, hi.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice));
  m->h_reg_lo = lo;
  m->h_reg_hi = hi;
  CU(cudaMemcpy(m->reg_gap, gap.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(m->reg_cent, cf.data(), sizeof(float) * 3 * R, cudaMemcpyHostToDevice));
  m->n_regions = R;
  return FEM_OK;
}

fem_status fem_ebe_apply(fem_mesh* m, int precision, const void* p_dev, void* q_dev, int n_rhs, double alpha_M,
                         double alpha_K, double* ptq_dev, void* stream) {
  g_err.clear();
  if (!m || !p_dev || !q_dev) return fail(FEM_ERR_ARG, "null argument");
  if (!pow2_rhs(n_rhs)) return fail(FEM_ERR_ARG, "n_rhs must be 1, 2, 4, 8, 16 or 32");
  cudaStream_t s = (cudaStream_t)stream;
  CU(ebe_set_wait_budget(kDefaultWaitBudget, s));
  Workspace* w = nullptr;
  CHK(m->workspace(n_rhs, &w));
  const Reducer red = w->red();
  const MeshView mv = m->view();
  if (precision == FEM_FP64) {
    CU(ebe_product<double>(m, n_rhs, (const double*)p_dev, (double*)q_dev, alpha_M, alpha_K,
                           ptq_dev ? &red : nullptr, nullptr, ptq_dev, nullptr, s));
    CU(launch_mask<double>(m->N, n_rhs, m->fm, (double*)q_dev, s));
  } else if (precision == FEM_FP32_INNER) {
    CU(ebe_product<float>(m, n_rhs, (const float*)p_dev, (float*)q_dev, alpha_M, alpha_K,
                          ptq_dev ? &red : nullptr, nullptr, ptq_dev, nullptr, s));
    CU(launch_mask<float>(m->N, n_rhs, m->fm, (float*)q_dev, s));
  } else {
    return fail(FEM_ERR_ARG, "unknown precision");
  }
  return FEM_OK;
}

fem_status pcg_solve(fem_mesh* m, const double* b_dev, double* x_dev, int n_rhs, const fem_opts* opts, void* stream,
                     int* iters_out, double* relres_out) {
  g_err.clear();
  if (!m || !b_dev || !x_dev) return fail(FEM_ERR_ARG, "null argument");
  if (!pow2_rhs(n_rhs)) return fail(FEM_ERR_ARG, "n_rhs must be 1, 2, 4, 8, 16 or 32");
  CHK(check_opts(opts));
  cudaStream_t s = (cudaStream_t)stream;
  CU(ebe_set_wait_budget(opts->wait_budget, s));
  Workspace* w = nullptr;
  CHK(m->workspace(n_rhs, &w));
  CgCase* res = nullptr;
  CHK(solve_any(m, w, b_dev, x_dev, *opts, s, &res));
  CU(cudaMemcpyAsync(w->h_sc, res, sizeof(CgCase) * n_rhs, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  {
    int tmo = 0;   // a staged EBE kernel whose bounded wait for its copies gave up: results not valid
    CU(ebe_tma_timeout(&tmo));
    if (tmo) return fail(FEM_ERR_TIMEOUT, "pcg_solve: an EBE kernel's wait for its tile copies timed out");
  }
  fem_status worst = FEM_OK;
  for (int c = 0; c < n_rhs; ++c) {
    if (iters_out) iters_out[c] = w->h_sc[c].iters;
    if (relres_out) relres_out[c] = w->h_sc[c].relres;
    const int st = w->h_sc[c].status;
    if (st != FEM_OK && (worst == FEM_OK || st < worst)) worst = st;
  }
  if (worst != FEM_OK) return fail(worst, "pcg_solve: a case did not converge or broke down");
  return FEM_OK;
}

fem_status fem_batch_create(const fem_opts* opts, void* stream, fem_batch** out) {
  g_err.clear();
  if (!out) return fail(FEM_ERR_ARG, "out is null");
  *out = nullptr;
  CHK(check_opts(opts));
  fem_batch* b = new fem_batch();
  b->opts = *opts;
  if (b->opts.check_every < 1) b->opts.check_every = 1;
  b->s = (cudaStream_t)stream;
  *out = b;
  return FEM_OK;
}

fem_status fem_batch_destroy(fem_batch* b) {
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  cudaStreamSynchronize(b->s);
  delete b;
  return FEM_OK;
}

static fem_status case_add(fem_batch* b, fem_mesh* m, int32_t src_node, const double dir[3], double f0, double t0,
                           double amp, int* case_id, Group** gout = nullptr) {
  Group* g = nullptr;
  if (b->opts.cpu_predictor) {   // two case sets per mesh, filled alternately (Algorithm 3's ping-pong)
    std::vector<Group*> sets;
    for (auto* gg : b->groups)
      if (gg->mesh == m) sets.push_back(gg);
    if (sets.size() >= 2) {
      g = sets[1]->cases.size() < sets[0]->cases.size() ? sets[1] : sets[0];
      if (g->cases.size() >= (size_t)kMaxRpad) return fail(FEM_ERR_ARG, "cpu_predictor: at most 64 cases per mesh");
    }
  } else {
    for (auto* gg : b->groups)
      if (gg->mesh == m && gg->cases.size() < (size_t)kMaxRpad) g = gg;
  }
  if (!g) {
    g = new Group();
    g->mesh = m;
    b->groups.push_back(g);
  }
  const int id = (int)b->loc.size();
  g->cases.push_back(id);
  g->hsrc.push_back(RickerSrc{src_node, {dir[0], dir[1], dir[2]}, f0, t0, amp});
  g->himp.resize(g->cases.size());
  b->loc.push_back({(int)(std::find(b->groups.begin(), b->groups.end(), g) - b->groups.begin()),
                    (int)g->cases.size() - 1});
  if (case_id) *case_id = id;
  if (gout) *gout = g;
  return FEM_OK;
}

fem_status fem_case_add(fem_batch* b, fem_mesh* m, int32_t src_node, const double dir[3], double f0, double t0,
                        double amp, int* case_id) {
  g_err.clear();
  if (!b || !m || !dir) return fail(FEM_ERR_ARG, "null argument");
  if (b->started) return fail(FEM_ERR_STATE, "cases must be added before the first fem_step");
  if (src_node < 0 || src_node >= m->N) return fail(FEM_ERR_ARG, "source node out of range");
  return case_add(b, m, src_node, dir, f0, t0, amp, case_id);
}

fem_status fem_case_add_impulses(fem_batch* b, fem_mesh* m, int64_t n, const int32_t* nodes, const int32_t* steps,
                                 const double* forces, int* case_id) {
  g_err.clear();
  if (!b || !m || n < 0 || (n > 0 && (!nodes || !steps || !forces))) return fail(FEM_ERR_ARG, "bad argument");
  if (b->started) return fail(FEM_ERR_STATE, "cases must be added before the first fem_step");
  for (int64_t k = 0; k < n; ++k) {
    if (nodes[k] < 0 || nodes[k] >= m->N) return fail(FEM_ERR_ARG, "impulse node out of range");
    if (steps[k] < 1) return fail(FEM_ERR_ARG, "impulse steps start at 1");
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(forces[3 * k + d])) return fail(FEM_ERR_ARG, "non-finite impulse force");
  }
  const double zero[3] = {0.0, 0.0, 0.0};
  Group* g = nullptr;
  int id = 0;
  // no Ricker point force: a zero amplitude (its node 0 receives nothing)
  CHK(case_add(b, m, 0, zero, 1.0, 0.0, 0.0, &id, &g));
  auto& v = g->himp[b->loc[id].second];
  v.reserve((size_t)n);
  for (int64_t k = 0; k < n; ++k)
    v.push_back(Group::HostImpulse{nodes[k], steps[k], {forces[3 * k], forces[3 * k + 1], forces[3 * k + 2]}});
  if (case_id) *case_id = id;
  return FEM_OK;
}

// Fuses every case of the batch into one system: each case gets its own copy of its mesh, all copies are
// concatenated into one virtual mesh (node, element, material and region numbering shifted), and the
// node -> case map makes the solver's scalars per case.  One set of launches then serves all cases.
static fem_status fuse_cases(fem_batch* b) {
  const int nc = (int)b->loc.size();
  if (nc > kMaxCases || nc > 255) return fail(FEM_ERR_ARG, "fuse_meshes supports at most 128 cases");
  std::vector<fem_mesh*> mesh_of(nc);
  std::vector<RickerSrc> src_of(nc);
  for (int c = 0; c < nc; ++c) {
    Group* g = b->groups[b->loc[c].first];
    mesh_of[c] = g->mesh;
    src_of[c] = g->hsrc[b->loc[c].second];
  }
  const fem_time_params tp = mesh_of[0]->tp;
  bool all_regions = true;
  int64_t N = 0, E = 0, nmat = 0;
  for (int c = 0; c < nc; ++c) {
    const fem_mesh* m = mesh_of[c];
    if (m->tp.dt != tp.dt || m->tp.a0 != tp.a0 || m->tp.a1 != tp.a1)
      return fail(FEM_ERR_ARG, "fused meshes must share dt and damping");
    if (m->ab.nb > 0) return fail(FEM_ERR_ARG, "fuse_meshes does not support absorbing faces");
    if (m->npe != 4) return fail(FEM_ERR_ARG, "fuse_meshes supports linear tets only");
    if (!b->groups[b->loc[c].first]->himp[b->loc[c].second].empty())
      return fail(FEM_ERR_ARG, "fuse_meshes does not support impulse loads");
    N += m->N;
    E += m->E;
    nmat += (int64_t)m->h_lmr.size() / 3;
    all_regions = all_regions && m->n_regions > 0;
  }
  std::vector<double> xyz, lmr;
  std::vector<int32_t> conn, mat, region;
  std::vector<uint8_t> fixed, seg;
  xyz.reserve(3 * N); conn.reserve(4 * E); mat.reserve(E); fixed.reserve(3 * N); seg.reserve(N);
  if (all_regions) region.reserve(N);
  std::vector<int64_t> node_off(nc + 1, 0);
  int32_t mat_off = 0, reg_off = 0;
  for (int c = 0; c < nc; ++c) {
    const fem_mesh* m = mesh_of[c];
    const int32_t noff = (int32_t)node_off[c];
    node_off[c + 1] = node_off[c] + m->N;
    xyz.insert(xyz.end(), m->h_xyz.begin(), m->h_xyz.end());
    for (int32_t v : m->h_conn) conn.push_back(v + noff);
    for (int32_t v : m->h_mat) mat.push_back(v + mat_off);
    lmr.insert(lmr.end(), m->h_lmr.begin(), m->h_lmr.end());
    fixed.insert(fixed.end(), m->h_fixed.begin(), m->h_fixed.end());
    seg.insert(seg.end(), (size_t)m->N, (uint8_t)c);
    if (all_regions) {
      int32_t rmax = -1;
      for (int32_t v : m->h_region) {
        region.push_back(v < 0 ? -1 : v + reg_off);
        rmax = std::max(rmax, v);
      }
      reg_off += rmax + 1;
    }
    mat_off += (int32_t)(m->h_lmr.size() / 3);
  }
  fem_mesh* vm = nullptr;
  CHK(fem_mesh_create(N, xyz.data(), E, conn.data(), mat.data(), (int)nmat, lmr.data(), fixed.data(), &tp, b->s, &vm));
  if (dalloc(&vm->seg, (size_t)N) != FEM_OK) {
    delete vm;
    return fail(FEM_ERR_OOM, "fused case map allocation failed");
  }
  vm->nseg = nc;
  cudaError_t e = cudaMemcpy(vm->seg, seg.data(), (size_t)N, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete vm;
    return fail(FEM_ERR_CUDA, std::string("fused case map upload: ") + cudaGetErrorString(e));
  }
  if (all_regions) {
    fem_status st = fem_mesh_set_regions(vm, region.data());
    if (st != FEM_OK) {
      delete vm;
      return st;
    }
  }
  Group* fg = new Group();
  fg->mesh = fg->owned_mesh = vm;
  fg->node_off = node_off;
  for (int c = 0; c < nc; ++c) {
    fg->cases.push_back(c);
    RickerSrc r = src_of[c];
    if (r.node >= 0) r.node += (int)node_off[c];
    fg->hsrc.push_back(r);
  }
  for (auto* g : b->groups) delete g;
  b->groups.assign(1, fg);
  for (int c = 0; c < nc; ++c) b->loc[c] = {0, c};
  return FEM_OK;
}

static fem_status batch_start(fem_batch* b) {
  if (b->started) return FEM_OK;
  if (b->loc.empty()) return fail(FEM_ERR_STATE, "batch has no cases");
  if (b->opts.fuse_meshes) {
    if (b->opts.precision != FEM_FP32_INNER) return fail(FEM_ERR_ARG, "fuse_meshes needs the FP32-inner solver");
    CHK(fuse_cases(b));
  }
  for (auto* g : b->groups) CHK(group_alloc(b, g));
  CU(cudaStreamSynchronize(b->s));
  b->started = true;
  return FEM_OK;
}

fem_status fem_step(fem_batch* b, int n_steps, int* iters_out, double* relres_out) {
  g_err.clear();
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  if (n_steps < 0) return fail(FEM_ERR_ARG, "n_steps < 0");
  CHK(batch_start(b));
  CU(ebe_set_wait_budget(b->opts.wait_budget, b->s));
  fem_status worst = FEM_OK;
  for (int k = 0; k < n_steps; ++k) {
    for (auto* g : b->groups) CHK(group_step(b, g, &worst));
    b->steps += 1;
    if (b->prof.on) b->prof.steps += 1;
  }
  for (auto* g : b->groups) CHK(group_graph_stats(b, g, &worst));
  {
    int tmo = 0;   // a staged EBE kernel whose bounded wait for its copies gave up: results not valid
    CU(ebe_tma_timeout(&tmo));
    if (tmo) return fail(FEM_ERR_TIMEOUT, "fem_step: an EBE kernel's wait for its tile copies timed out");
  }
  // the statistics since the last report (this call's steps and any queued by fem_step_async)
  for (size_t c = 0; c < b->loc.size(); ++c) {
    const Group* g = b->groups[b->loc[c].first];
    const int l = b->loc[c].second;
    if (iters_out) iters_out[c] = g->iters_acc[l];
    if (relres_out) relres_out[c] = g->relres_max[l];
  }
  for (auto* g : b->groups) {
    std::fill(g->iters_acc.begin(), g->iters_acc.end(), 0);
    std::fill(g->relres_max.begin(), g->relres_max.end(), 0.0);
  }
  if (b->pending != FEM_OK && (worst == FEM_OK || b->pending < worst)) worst = b->pending;
  b->pending = FEM_OK;
  if (worst != FEM_OK) return fail(worst, "fem_step: a case did not converge or broke down");
  return FEM_OK;
}

fem_status fem_step_async(fem_batch* b, int n_steps) {
  g_err.clear();
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  if (n_steps < 0) return fail(FEM_ERR_ARG, "n_steps < 0");
  CHK(batch_start(b));
  CU(ebe_set_wait_budget(b->opts.wait_budget, b->s));
  fem_status worst = FEM_OK;   // (steps that run eagerly report here; graph steps on the device)
  for (int k = 0; k < n_steps; ++k) {
    for (auto* g : b->groups) CHK(group_step(b, g, &worst));
    b->steps += 1;
    if (b->prof.on) b->prof.steps += 1;
  }
  if (worst != FEM_OK && (b->pending == FEM_OK || worst < b->pending)) b->pending = worst;
  return FEM_OK;
}

fem_status predictor_fit(fem_batch* b, int case_id) {
  g_err.clear();
  if (!b || case_id < 0 || case_id >= (int)b->loc.size()) return fail(FEM_ERR_ARG, "bad case id");
  CHK(batch_start(b));
  Group* g = b->groups[b->loc[case_id].first];
  if (b->opts.predictor != FEM_PRED_DD || g->n_regions == 0) return FEM_OK;
  const int it = g->steps;
  const int n_e = std::min(it, g->n_slots);
  uint64_t mask = 0;
  for (int j = it - n_e + 1; j <= it; ++j) mask |= 1ull << slot_of(g, j);
  for (int j = it - n_e + 1; j <= it; ++j) CU(launch_pred_dots(pred_view(b, g), slot_of(g, j), mask, b->s));
  CU(cudaStreamSynchronize(b->s));
  return FEM_OK;
}

fem_status predictor_predict(fem_batch* b, int case_id, double* x_guess_dev) {
  g_err.clear();
  if (!b || !x_guess_dev || case_id < 0 || case_id >= (int)b->loc.size()) return fail(FEM_ERR_ARG, "bad argument");
  CHK(batch_start(b));
  Group* g = b->groups[b->loc[case_id].first];
  CHK(group_predict(b, g, g->ws->q));
  const int l = b->loc[case_id].second;
  if (g->owned_mesh) {
    const int64_t n0 = g->node_off[l], n3 = 3 * (g->node_off[l + 1] - n0);
    CU(cudaMemcpyAsync(x_guess_dev, g->ws->q + 3 * n0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, b->s));
  } else {
    CU(launch_extract_case(g->mesh->N, g->rpad, l, g->ws->q, x_guess_dev, b->s));
  }
  CU(cudaStreamSynchronize(b->s));
  return FEM_OK;
}

fem_status predictor_coefficients(fem_batch* b, int case_id, double* coef_host, int* n_pairs_out) {
  g_err.clear();
  if (!b || !coef_host || case_id < 0 || case_id >= (int)b->loc.size()) return fail(FEM_ERR_ARG, "bad argument");
  Group* g = b->groups[b->loc[case_id].first];
  if (b->opts.predictor != FEM_PRED_DD || !g->wcoef || g->n_regions == 0)
    return fail(FEM_ERR_STATE, "predictor_coefficients: the batch has no data-driven predictor with regions");
  if (g->owned_mesh) return fail(FEM_ERR_STATE, "predictor_coefficients: not available for fused meshes");
  // the pairs of the last completed step's prediction (it = steps): X = e^{it-1-n} .. e^{it-2}
  const int it = g->steps;
  const int n_pairs = it >= 1 ? std::max(0, std::min(b->opts.s_max, std::min(it - 1, g->n_slots) - 1)) : 0;
  const int l = b->loc[case_id].second, R = g->n_regions, s = b->opts.s_max;
  std::vector<double> all((size_t)R * g->rpad * kMaxSlots);
  if (g->hp) {   // heterogeneous scheme: the host's coefficients and pair count of the last prediction used
    int np = 0;
    const double* wh = hostpred_coefficients(g->hp, &np);
    for (int r = 0; r < R; ++r)
      for (int a = 0; a < s; ++a) coef_host[(size_t)r * s + a] = a < np ? wh[((size_t)r * g->rpad + l) * kMaxSlots + a] : 0.0;
    if (n_pairs_out) *n_pairs_out = np;
    return FEM_OK;
  }
  CU(cudaMemcpyAsync(all.data(), g->wcoef, sizeof(double) * all.size(), cudaMemcpyDeviceToHost, b->s));
  CU(cudaStreamSynchronize(b->s));
  for (int r = 0; r < R; ++r)
    for (int a = 0; a < s; ++a)
      coef_host[(size_t)r * s + a] = a < n_pairs ? all[((size_t)r * g->rpad + l) * kMaxSlots + a] : 0.0;
  if (n_pairs_out) *n_pairs_out = n_pairs;
  return FEM_OK;
}

fem_status fem_case_get(fem_batch* b, int case_id, int what, double* dst, int on_device) {
  g_err.clear();
  if (!b || !dst || case_id < 0 || case_id >= (int)b->loc.size()) return fail(FEM_ERR_ARG, "bad argument");
  CHK(batch_start(b));
  Group* g = b->groups[b->loc[case_id].first];
  const double* src = nullptr;
  switch (what) {
    case FEM_FIELD_U: src = g->u; break;
    case FEM_FIELD_V: src = g->vh[((g->steps % 4) + 4) % 4]; break;
    case FEM_FIELD_A: src = g->a; break;
    case FEM_FIELD_DU: src = g->x; break;
    case FEM_FIELD_B: src = g->b; break;
    case FEM_FIELD_GUESS: src = g->guess; break;
    default: return fail(FEM_ERR_ARG, "unknown field");
  }
  const int l = b->loc[case_id].second;
  if (g->owned_mesh) {   // fused: the case's own node range of the virtual mesh
    const int64_t n0 = g->node_off[l], n3 = 3 * (g->node_off[l + 1] - n0);
    CU(cudaMemcpyAsync(dst, src + 3 * n0, sizeof(double) * n3, on_device ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyDeviceToHost, b->s));
    if (!on_device) CU(cudaStreamSynchronize(b->s));
    return FEM_OK;
  }
  if (on_device) {
    CU(launch_extract_case(g->mesh->N, g->rpad, l, src, dst, b->s));
  } else {
    double* tmp = g->ws->r;  // scratch, [N][3] fits
    CU(launch_extract_case(g->mesh->N, g->rpad, l, src, tmp, b->s));
    CU(cudaMemcpyAsync(dst, tmp, sizeof(double) * 3 * g->mesh->N, cudaMemcpyDeviceToHost, b->s));
    CU(cudaStreamSynchronize(b->s));
  }
  return FEM_OK;
}

fem_status fem_batch_set_loads(fem_batch* b, const double* loads) {
  g_err.clear();
  if (!b || !loads) return fail(FEM_ERR_ARG, "null argument");
  CHK(batch_start(b));
  if (b->groups.size() == 1) {  // one group holds the cases in id order: one copy
    Group* g = b->groups[0];
    CU(cudaMemcpyAsync(g->ext, loads, 3 * sizeof(double) * b->loc.size(), cudaMemcpyHostToDevice, b->s));
    g->use_ext = true;
    return FEM_OK;
  }
  for (size_t c = 0; c < b->loc.size(); ++c) {
    Group* g = b->groups[b->loc[c].first];
    const int l = b->loc[c].second;
    CU(cudaMemcpyAsync(g->ext + 3 * l, loads + 3 * c, 3 * sizeof(double), cudaMemcpyHostToDevice, b->s));
    g->use_ext = true;
  }
  return FEM_OK;
}

static fem_status learn_ok(const fem_batch* b) {
  if (b->opts.cpu_predictor) return fail(FEM_ERR_ARG, "the learned proposal needs the GPU predictor (cpu_predictor 0)");
  if (b->opts.precision != FEM_FP32_INNER) return fail(FEM_ERR_ARG, "the learned proposal needs FEM_FP32_INNER");
  if (b->opts.predictor != FEM_PRED_DD) return fail(FEM_ERR_ARG, "the learned proposal needs the data-driven predictor");
  if (b->opts.fuse_meshes) return fail(FEM_ERR_ARG, "the learned proposal needs groups of one mesh (no fuse_meshes)");
  return FEM_OK;
}

fem_status fem_batch_set_mlp(fem_batch* b, fem_mlp* net) {
  g_err.clear();
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  if (net) {
    CHK(learn_ok(b));
    int dev = 0;
    cudaGetDevice(&dev);
    if (mlp_device(net) != dev) return fail(FEM_ERR_ARG, "the network lives on another device");
  }
  b->mlp = net;
  return FEM_OK;
}

static fem_status batch_collect(fem_batch* b, float* x_dev, float* t_dev, int64_t capacity, bool residual) {
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  if (!x_dev) {
    b->col_x = b->col_t = nullptr;
    b->col_cap = 0;
    return FEM_OK;
  }
  if (!t_dev || capacity <= 0) return fail(FEM_ERR_ARG, "t_dev is null or capacity <= 0");
  CHK(learn_ok(b));
  b->col_x = x_dev;
  b->col_t = t_dev;
  b->col_res = residual;
  b->col_cap = capacity;
  b->col_n = 0;
  b->col_full = false;
  return FEM_OK;
}

fem_status fem_batch_collect(fem_batch* b, float* x_dev, float* t_dev, int64_t capacity) {
  g_err.clear();
  return batch_collect(b, x_dev, t_dev, capacity, false);
}

fem_status fem_batch_collect_residual(fem_batch* b, float* x_dev, float* s_dev, int64_t capacity) {
  g_err.clear();
  return batch_collect(b, x_dev, s_dev, capacity, true);
}

fem_status fem_batch_collected(fem_batch* b, int64_t* rows, int* full) {
  g_err.clear();
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  if (rows) *rows = b->col_n;
  if (full) *full = b->col_full ? 1 : 0;
  return FEM_OK;
}

fem_status fem_batch_proposal_counts(fem_batch* b, long long* taken, long long* rejected) {
  g_err.clear();
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  long long t = 0, r = 0;
  for (auto* g : b->groups) {
    if (!g->counts) continue;
    long long h[2] = {0, 0};
    CU(cudaMemcpyAsync(h, g->counts, sizeof(h), cudaMemcpyDeviceToHost, b->s));
    CU(cudaStreamSynchronize(b->s));
    t += h[0];
    r += h[1];
  }
  if (taken) *taken = t;
  if (rejected) *rejected = r;
  return FEM_OK;
}

// case c's field starts after the fields of cases 0..c-1 (each [n_nodes of its mesh][3])
static std::vector<int64_t> field_offsets(const fem_batch* b) {
  std::vector<int64_t> case_off(b->loc.size() + 1, 0);
  for (size_t c = 0; c < b->loc.size(); ++c) {
    const Group* g = b->groups[b->loc[c].first];
    const int l = b->loc[c].second;
    const int64_t nn = g->owned_mesh ? g->node_off[l + 1] - g->node_off[l] : g->mesh->N;
    case_off[c + 1] = case_off[c] + 3 * nn;
  }
  return case_off;
}

fem_status fem_batch_get_field(fem_batch* b, int what, double* dst, int on_device) {
  g_err.clear();
  if (!b || !dst) return fail(FEM_ERR_ARG, "null argument");
  CHK(batch_start(b));
  const std::vector<int64_t> case_off = field_offsets(b);
  for (auto* g : b->groups) {
    const double* src = nullptr;
    switch (what) {
      case FEM_FIELD_U: src = g->u; break;
      case FEM_FIELD_V: src = g->vh[((g->steps % 4) + 4) % 4]; break;
      case FEM_FIELD_A: src = g->a; break;
      case FEM_FIELD_DU: src = g->x; break;
      case FEM_FIELD_B: src = g->b; break;
      case FEM_FIELD_GUESS: src = g->guess; break;
      default: return fail(FEM_ERR_ARG, "unknown field");
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (g->owned_mesh) {
      for (size_t l = 0; l < g->cases.size(); ++l) {
        const int64_t n0 = g->node_off[l], n3 = 3 * (g->node_off[l + 1] - n0);
        CU(cudaMemcpyAsync(dst + case_off[g->cases[l]], src + 3 * n0, sizeof(double) * n3, kind, b->s));
      }
      continue;
    }
    const int64_t n3 = g->mesh->N * 3;
    double* tmp = g->ws->r;  // [rpad][N][3] scratch
    CU(launch_extract_all(g->mesh->N, g->rpad, (int)g->cases.size(), src, tmp, b->s));
    for (size_t l = 0; l < g->cases.size(); ++l)
      CU(cudaMemcpyAsync(dst + case_off[g->cases[l]], tmp + l * n3, sizeof(double) * n3, kind, b->s));
  }
  if (!on_device) CU(cudaStreamSynchronize(b->s));
  return FEM_OK;
}

fem_status fem_batch_get_field_async(fem_batch* b, int what, double* host_dst) {
  g_err.clear();
  if (!b || !host_dst) return fail(FEM_ERR_ARG, "null argument");
  CHK(batch_start(b));
  const std::vector<int64_t> case_off = field_offsets(b);
  const size_t total = (size_t)case_off.back();
  if (!b->cs) {
    CU(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      CU(cudaEventCreateWithFlags(&b->ready[k], cudaEventDisableTiming));
      CU(cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming));
      CHK(dalloc(&b->stage[k], total));
    }
  }
  const int k = b->stage_k;
  b->stage_k ^= 1;
  // the previous host copy out of stage[k] has finished before the field is staged there again
  CU(cudaStreamWaitEvent(b->s, b->done[k], 0));
  const Group* g0 = b->groups[0];
  bool direct = b->groups.size() == 1 && !g0->owned_mesh;   // one multi-case group, cases in lane order
  for (size_t c = 0; direct && c < b->loc.size(); ++c) direct = b->loc[c].second == (int)c;
  if (direct && (what == FEM_FIELD_U || what == FEM_FIELD_A || what == FEM_FIELD_DU)) {
    const double* src = what == FEM_FIELD_U ? g0->u : what == FEM_FIELD_A ? g0->a : g0->x;
    CU(launch_extract_all(g0->mesh->N, g0->rpad, (int)g0->cases.size(), src, b->stage[k], b->s));
  } else {
    CHK(fem_batch_get_field(b, what, b->stage[k], 1));
  }
  CU(cudaEventRecord(b->ready[k], b->s));
  CU(cudaStreamWaitEvent(b->cs, b->ready[k], 0));
  CU(cudaMemcpyAsync(host_dst, b->stage[k], sizeof(double) * total, cudaMemcpyDeviceToHost, b->cs));
  CU(cudaEventRecord(b->done[k], b->cs));
  return FEM_OK;
}

fem_status fem_batch_sync(fem_batch* b) {
  g_err.clear();
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  if (b->cs) CU(cudaStreamSynchronize(b->cs));
  CU(cudaStreamSynchronize(b->s));
  fem_status worst = b->pending;
  b->pending = FEM_OK;
  if (b->started) {
    for (auto* g : b->groups) CHK(group_graph_stats(b, g, &worst));
    int tmo = 0;
    CU(ebe_tma_timeout(&tmo));
    if (tmo) return fail(FEM_ERR_TIMEOUT, "fem_batch_sync: an EBE kernel's wait for its tile copies timed out");
  }
  if (worst != FEM_OK) return fail(worst, "fem_batch_sync: a case did not converge or broke down");
  return FEM_OK;
}

fem_status fem_batch_profile(fem_batch* b, int enable, fem_profile* out) {
  g_err.clear();
  if (!b) return fail(FEM_ERR_ARG, "batch is null");
  CU(cudaStreamSynchronize(b->s));
  b->prof.resolve();
  if (enable == 1 || enable == 2) {
    b->prof.reset();
    b->prof.on = true;
    b->prof.events = enable == 1;
  } else if (enable == 0) {
    b->prof.on = false;
    b->prof.events = false;
  }
  if (out) {
    std::memset(out, 0, sizeof(*out));
    const Prof& p = b->prof;
    out->steps = p.steps;
    out->kernel_launches = p.launches;
    out->ebe32_launches = p.n[P_EBE32];
    out->ebe32_ms = p.ms[P_EBE32];
    out->ebe64_launches = p.n[P_EBE64];
    out->ebe64_ms = p.ms[P_EBE64];
    out->cg_vec_launches = p.n[P_VEC];
    out->cg_vec_ms = p.ms[P_VEC];
    out->predict_ms = p.ms[P_PREDICT];
    out->rhs_ms = p.ms[P_RHS];
    out->solve_ms = p.ms[P_SOLVE];
    out->update_ms = p.ms[P_UPDATE];
    out->ebe16_launches = p.n[P_EBE16];
    out->ebe16_ms = p.ms[P_EBE16];
  }
  return FEM_OK;
}

fem_status fem_case_stats(fem_batch* b, int case_id, fem_case_stats_t* out) {
  g_err.clear();
  if (!b || !out || case_id < 0 || case_id >= (int)b->loc.size()) return fail(FEM_ERR_ARG, "bad argument");
  std::memset(out, 0, sizeof(*out));
  if (!b->started) return FEM_OK;
  const Group* g = b->groups[b->loc[case_id].first];
  const CgCase& c = g->last[b->loc[case_id].second];
  out->steps = g->steps;
  out->iters = c.iters;
  out->outer = b->opts.precision == FEM_FP64 ? 0 : c.outer;
  out->status = c.status;
  out->init_relres = c.relres0;
  out->relres = c.relres;
  out->guess = b->opts.precision == FEM_FP64 ? -1 : c.guess;
  if (g->fb) {
    CU(cudaMemcpyAsync(&out->fallbacks, g->fb + b->loc[case_id].second, sizeof(int), cudaMemcpyDeviceToHost, b->s));
    CU(cudaStreamSynchronize(b->s));
  }
  return FEM_OK;
}

fem_status fem_batch_predictor_balance(fem_batch* b, int case_id, int* s_current, double* predict_ms,
                                       double* solve_ms, double* predict_total_ms, double* wait_total_ms) {
  g_err.clear();
  if (!b || case_id < 0 || case_id >= (int)b->loc.size()) return fail(FEM_ERR_ARG, "bad case id");
  const Group* g = b->groups[b->loc[case_id].first];
  if (!g->hp) return fail(FEM_ERR_STATE, "the batch does not use the heterogeneous predictor");
  int sc = 0;
  double a = 0, c = 0, d = 0, e = 0;
  long long n = 0;
  hostpred_stats(g->hp, &sc, &a, &c, &d, &e, &n);
  if (s_current) *s_current = sc;
  if (predict_ms) *predict_ms = a;
  if (solve_ms) *solve_ms = c;
  if (predict_total_ms) *predict_total_ms = d;
  if (wait_total_ms) *wait_total_ms = e;
  return FEM_OK;
}

fem_status fem_batch_steps(const fem_batch* b, int* steps_out) {
  if (!b || !steps_out) return fail(FEM_ERR_ARG, "null argument");
  *steps_out = b->steps;
  return FEM_OK;
}

}  // extern "C"
