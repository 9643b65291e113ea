// Internal declarations shared by the libfem translation units (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fem.h"

namespace fem {

constexpr int kBlock = 256;              // threads per block of the element kernels
constexpr int kVecBlock = 512;           // threads per block of the reducing vector kernels
constexpr int kMaxRpad = 32;             // max cases per multi-RHS group (lanes of a node)
constexpr int kMaxCases = 128;           // max cases of a group (fused groups: one case per mesh)
constexpr int kMaxSlots = 33;            // predictor ring: s_max + 1 <= 33
constexpr int kDefaultWaitBudget = 1 << 20;   // tries (<= 1 us each) of a reporting device-side wait
// Smallest per-pass reduction target of an inner solve whose CG products take FP16 operands on the tensor
// cores (relative error ~2.4e-4 a product); a pass that asks a case for more runs FP32 products.
constexpr double kTcFloor = 1e-3;
constexpr int kMaxRedBlocks = 1216;     // rows of the per-block partial-sum buffers of reducing kernels

// Per-element record, 12 values: g1 (3), g2 (3), g3 (3) shape-function gradients of local nodes 1..3
// (g0 = -g1-g2-g3), lambda*V, mu*V, rho*V/20.
constexpr int kRec = 12;
constexpr int kHexMatVals = 300;          // stored values of a hex's symmetric 24 x 24 element matrix

// Hex-patch topology: slots of the four corners of each of the six tets of a hex, slots numbered by first
// appearance (the Kuhn split along the (0,0,0)-(1,1,1) diagonal gives exactly this table).
constexpr int kHexTet[6][4] = {{0, 1, 2, 3}, {0, 1, 3, 4}, {0, 5, 3, 2}, {0, 5, 6, 3}, {0, 7, 4, 3}, {0, 7, 3, 6}};

// Tiling of a hex-patch mesh (host copy).  tile_nodes carries bit 31 set for nodes other tiles touch too.
struct HexTilesHost {
  int hex_per_tile = 0;
  int64_t n_hex = 0;
  int n_tiles = 0;
  int nloc_max = 0;
  std::vector<int> tile_hex_off, tile_node_off, tile_nodes;
  std::vector<uint16_t> hex_local;   // [n_hex][8] tile-local corner index
};
struct HexTiles {                    // device view
  int n_tiles = 0;
  int nloc_max = 0;
  int hex_per_tile = 0;
  const int* tile_hex_off = nullptr;
  const int* tile_node_off = nullptr;
  const int* tile_nodes = nullptr;   // per entry: node id (bits 0-27), free-DOF bits (28-30), shared (31)
  const uint4* hex_local = nullptr;  // 8 x uint16 per hex
  // largest element-wise absolute row sums over the nodes: sum over the elements e of a node i and over j
  // of |M^e_ij| and |K^e_ij| (bounds on any partial sum of a product's element contributions to a row)
  float abs_m = 0.0f, abs_k = 0.0f;
};
bool detect_hex_patches(const int32_t* conn, int64_t E);
bool build_hex_tiles(const int32_t* conn, int64_t E, int64_t N, int hex_per_tile, HexTilesHost* out);

// Per-case CG scalars, device resident.
struct CgCase {
  double rho;      // (z, r) of the current residual
  double pq;       // (p, A p)
  double rr;       // (r, r)
  double bb;       // (b, b)
  double alpha;
  double beta;
  double relres;   // last certified / recursive relative residual
  int active;      // 1 while the case iterates
  int iters;
  int status;      // FEM_OK or a negative fem_status
  int phase;       // internal: 0 = before first direction
  double relres0;  // relative residual of the initial guess
  int outer;       // FP64 residual evaluations (refinement passes) of the solve
  int guess;       // outer state: the step's initial guess: 0 Adams-Bashforth (no correction), 1 with the
                   // data-driven correction, 2 correction dropped by the guess guard (larger residual)
  double tol2;     // squared relative tolerance of this case's (inner) solve; set when the solve starts
  double inner_tol;  // outer state: relative reduction the next inner solve is asked for
};

// Step-dependent values of a time step in device memory, so that one captured graph serves every step
// (the graph's kernels read the step from here instead of from launch arguments).  Written by the
// step-begin kernel; ring slot of correction e^j is (j - 1) mod n_slots.
struct StepCtl {
  int it;                        // step being computed (1-based)
  int n_pairs;                   // data-driven predictor pairs of this step (0: no correction)
  int slot_query;                // ring slot of e^{it-1}
  int slot_new;                  // ring slot of e^{it}
  unsigned long long mask;       // ring slots valid once e^it is pushed
  double t;                      // it * dt
  int use_ext;                   // external loads replace the point sources this step (set by the host)
  int pass;                      // refinement passes done in this step
  int issued;                    // inner iterations issued in this solve
  int pad_;
  long long launches;            // kernels the graph has run (for the launch count)
  int xs[33], ys[33];            // X and Y slot lists of the predictor
};
// The four buffers of a 4-deep history ring (vector of step j in p[j mod 4]).
struct Ring4 {
  double* p[4];
};

// Grid-wide deterministic per-case reduction: per-block partials + last-block final sum.
struct Reducer {
  double* partial;     // [kMaxRedBlocks][3 * kMaxCases]
  unsigned* counter;   // one counter, 0 between launches
  double* out;         // [3 * kMaxCases]
};

struct MeshView {
  int64_t N, E;
  const int4* conn;
  const double* rec64;
  const float* rec32;
  const double* binv64;   // [N][6] xx yy zz xy xz yz
  const float* binv32;
  const uint8_t* freemask;  // [N] bit k = DOF k free
  // Fused groups (several meshes concatenated, one case each): seg[n] is the case of node n, nseg the
  // number of cases.  seg == nullptr: the case of an entry is its lane (index % rpad).
  const uint8_t* seg = nullptr;
  int nseg = 0;
};

// Dashpots of absorbing boundary faces: per boundary node its symmetric 3x3 block (xx yy zz xy xz yz) of
// C_b, in FP64 and FP32; cB = 2/dt, the factor with which C_b enters A.
struct Absorb {
  int nb = 0;
  const int32_t* node = nullptr;
  const double* c64 = nullptr;
  const float* c32 = nullptr;
  double cB = 0.0;
};

// Random impulse loads of a group, sorted by step: entries off[it] .. off[it + 1] - 1 act in step it
// (1 <= it <= last); per entry the node, the case lane and the force [3].
struct Impulses {
  int n = 0, last = 0, max_per_step = 0;
  const int32_t* node = nullptr;
  const int32_t* lane = nullptr;
  const double* f = nullptr;
  const int32_t* off = nullptr;
};

struct RickerSrc {          // per case of a group
  int node;                 // -1: no source (padding lane)
  double dir[3];
  double f0, t0, amp;
};

// Accessors for translation units other than the C-ABI one: record the thread's error message and
// return `s`; clear it (every entry point does so on entry); the device view and device id of a mesh, and its
// tet10 connectivity (null for a linear-tet mesh).
fem_status set_error(fem_status s, const std::string& msg);
void clear_error();
void mesh_view_of(const fem_mesh* m, MeshView* view, int* device, const int32_t** conn10);

// ---- launchers (stream-ordered; return cudaGetLastError()) ----
// Multiprocessors of the current device (queried once per device) and the grid caps derived from them:
// reducing vector kernels 3 blocks per SM (few blocks keep the final reduction short), reducing element
// kernels 8 per SM, grid-stride kernels without reduction 16 per SM; the reducing caps never exceed the
// partial-sum buffers' kMaxRedBlocks rows.
int sm_count();
int vec_grid_cap();
int red_grid_cap();
int wide_grid_cap();
int grid_for(int64_t items, int cap = -1);   // cap < 0: red_grid_cap()
// Largest element-wise absolute row sums of M and K over the mesh's nodes (see HexTiles::abs_m).
cudaError_t elem_abs_row_bounds(const MeshView& m, double* abs_m, double* abs_k, cudaStream_t s);
// Grid of grid-stride kernel `fn` (blocks of `block` threads, no dynamic shared memory): at most one wave of
// the blocks that fit on the GPU at once, so no partial second wave.
int grid_resident(const void* fn, int block, int64_t items);

cudaError_t launch_elem_setup(int64_t E, int64_t N, const double* xyz, const int4* conn, const int32_t* mat,
                              int n_mat, const double* lmr, double* rec64, float* rec32, int* err_flag,
                              cudaStream_t s);
cudaError_t launch_diag_blocks(const MeshView& m, double aM, double aK, double* D, cudaStream_t s);
cudaError_t launch_binv(int64_t N, const double* D, const uint8_t* freemask, double* binv64, float* binv32,
                        int* err_flag, cudaStream_t s);

// q = (aM M + aK K) pm  (+ aK K pk - aK K pm when pk != nullptr: M acts on pm, K on pk).  q is zeroed
// first; Dirichlet DOFs of q are NOT masked (consumers mask).  If red != nullptr the per-case p^T q
// (element-wise p_e^T A_e p_e) is reduced into red->out[c] / ptq_out[c] and, if sc != nullptr, the CG
// step length alpha = rho / p^T A p is set.  gate: skip when *gate == 0.
template <typename T>
cudaError_t launch_ebe(const MeshView& m, int rpad, const T* pm, const T* pk, T* q, double aM, double aK,
                       const Reducer* red, CgCase* sc, double* ptq_out, cudaStream_t s);
template <typename T>
cudaError_t launch_ebe_gated(const MeshView& m, int rpad, const T* pm, const T* pk, T* q, double aM, double aK,
                             const Reducer* red, CgCase* sc, double* ptq_out, const int* gate, cudaStream_t s);
template <typename T>
cudaError_t launch_mask(int64_t N, int rpad, const uint8_t* fm, T* v, cudaStream_t s);
// Tiled hex-patch EBE: q = (aM M + aK K) p with Dirichlet DOFs of q zeroed; same reduction/tail options.
template <typename T>
cudaError_t launch_ebe_hex(const HexTiles& ht, const MeshView& m, int rpad, const T* p, T* q, double aM, double aK,
                           const Reducer* red, CgCase* sc, double* ptq_out, const int* gate, cudaStream_t s);

// CG vector kernels on [N][3][rpad] data of type T (scalars and reductions in FP64).
// Starts a solve: bb = ||b||^2, state reset; the case's tolerance is gate[c].inner_tol when given (> 0),
// else tol.
template <typename T>
cudaError_t launch_norm_b_gated(const MeshView& m, int rpad, const T* b, Reducer red, CgCase* sc,
                                const CgCase* gate, double tol, cudaStream_t s);
template <typename T>
cudaError_t launch_resid(const MeshView& m, int rpad, const T* b, const T* q, T* x, T* r, T* z,
                         int first, Reducer red, CgCase* sc, int* n_active, double tol, int maxit,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_dir_gated(const MeshView& m, int rpad, const T* z, T* p, const CgCase* sc, const int* n_active,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_update(const MeshView& m, int rpad, const T* p, const T* q, T* x, T* r, T* z,
                          Reducer red, CgCase* sc, int* n_active, double tol, int maxit, cudaStream_t s);

// Deferred-update iteration of the FP32 inner solves (no true-residual test): the direction pass forms
// z = B^{-1} r and applies the previous x += alpha p; the update pass only advances r.  x is complete
// after launch_refine_pending, which adds each case's last alpha p.
template <typename T>
cudaError_t launch_dir_defer(const MeshView& m, int rpad, const T* r, T* p, T* x, const CgCase* sc,
                             const int* n_active, cudaStream_t s);
template <typename T>
cudaError_t launch_update_defer(const MeshView& m, int rpad, const T* q, T* r, Reducer red, CgCase* sc,
                                int* n_active, int maxit, cudaStream_t s);
cudaError_t launch_refine_pending(const MeshView& m, int rpad, int ncase, double* x, const float* d32,
                                  const float* p32, CgCase* outer, const CgCase* inner, cudaStream_t s);

// Mixed precision helpers.
cudaError_t launch_outer_resid(const MeshView& m, int rpad, const double* b, const double* q,
                               float* r32, Reducer red, CgCase* outer, int* n_active, double tol,
                               double inner_max, double aim, cudaStream_t s);
cudaError_t launch_refine_counts(const MeshView& m, int rpad, int ncase, double* x, const float* d32, CgCase* outer,
                                 const CgCase* inner, cudaStream_t s);

// Fused groups (k_seg.cu): segmented forms of the CG and refinement kernels (rpad = 1, case = m.seg[node]).
template <typename T>
cudaError_t launch_norm_b_seg(const MeshView& m, const T* b, Reducer red, CgCase* sc, const CgCase* gate, double tol,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_resid_seg(const MeshView& m, const T* b, const T* q, T* x, T* r, T* z, Reducer red, CgCase* sc,
                             int* n_active, cudaStream_t s);
template <typename T>
cudaError_t launch_dir_seg(const MeshView& m, const T* z, T* p, const CgCase* sc, const int* n_active, cudaStream_t s);
template <typename T>
cudaError_t launch_update_seg(const MeshView& m, const T* p, const T* q, T* x, T* r, T* z, Reducer red, CgCase* sc,
                              int* n_active, int maxit, cudaStream_t s);
cudaError_t launch_r0_seg(const MeshView& m, double dt, const double* b, const double* Av4, const double* Av3,
                          const double* Av2, const double* Av1, const float* qy, float* r32, Reducer red,
                          CgCase* outer, int* n_active, double tol, double inner_floor, double aim, cudaStream_t s,
                          Ring4 avr = Ring4{}, const StepCtl* ctl = nullptr, bool guard = false,
                          int* fallbacks = nullptr);
cudaError_t launch_cert_seg(const MeshView& m, double cM, double cK, const double* b, const double* qM, const double* qK,
                            float* r32, Reducer red, CgCase* outer, int* n_active, double tol, double inner_floor,
                            double aim, cudaStream_t s);
// x = 0 on Dirichlet DOFs and for cases with ||b|| = 0.
template <typename T>
cudaError_t launch_zero_b0_t(const MeshView& m, int rpad, T* x, const CgCase* sc, cudaStream_t s);
cudaError_t launch_extract_case(int64_t N, int rpad, int c, const double* src, double* dst, cudaStream_t s);

// Time stepping (FP64 [N][3][rpad]).
cudaError_t launch_rhs_prep(int64_t n, double dt, double a0, double a1, const double* u, const double* v,
                            const double* a, double* m_in, double* k_in, cudaStream_t s);
// ext (nullable, device [rpad][3]): loads replacing the Ricker forces for this step.
cudaError_t launch_rhs_finish(const MeshView& m, int rpad, double* b, const RickerSrc* src, const double* ext,
                              double t, cudaStream_t s);
// dst[c][n*3 + k] = src[(n*3 + k)*rpad + c] for c < n_cases
cudaError_t launch_extract_all(int64_t N, int rpad, int n_cases, const double* src, double* dst, cudaStream_t s);
cudaError_t launch_ab4(int64_t n, double dt, const double* v4, const double* v3, const double* v2,
                       const double* v1, double* du_ab, cudaStream_t s);
// The same from the velocity ring with the step read from ctl (v^j in v.p[j mod 4]).
// (ahead 1: the increment of the step after the one ctl holds)
cudaError_t launch_ab4_ring(int64_t n, double dt, Ring4 v, const StepCtl* ctl, double* du_ab, cudaStream_t s,
                            int ahead = 0);
cudaError_t launch_add(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);
cudaError_t launch_newmark_update(int64_t n, double dt, const double* du, const double* du_ab, double* u,
                                  const double* v_prev, double* a, double* v_push, void* e_push, int e_fmt,
                                  int64_t stride, cudaStream_t s);

// FP32-inner steps with products kept by recurrences (see k_step.cu).
// b = f + Pb on free DOFs, Pb = M a + (4/dt + a0) M v + a1 K v - K u kept by launch_newmark_incr
cudaError_t launch_rhs_incr(const MeshView& m, int rpad, const double* Pb, double* b, const RickerSrc* src,
                            const double* ext, double t, cudaStream_t s, const StepCtl* ctl = nullptr);
// Pb <- Pb + (4/dt + a0) Mv + a1 Kv - Ku (Pb holding M a): the refresh's direct form of Pb
cudaError_t launch_pb_form(int64_t n, double dt, double a0, double a1, double* Pb, const double* Mv, const double* Kv,
                           const double* Ku, cudaStream_t s);
cudaError_t launch_corr_f32(int64_t n, const double* guess, const double* du_ab, float* y32, cudaStream_t s);
// inner != null (r0, cert): also start the inner FP32 solve of the pass on r32 (zero guess, its residual
// r32 itself): the inner case state as the norm and first-residual passes would leave it.
// guard (with qy, the product A y of the data-driven correction y): per case, the guess whose initial
// residual is smaller, the data-driven one or the Adams-Bashforth one (CgCase::guess; fallbacks[c], nullable,
// counts the cases' dropped corrections); launch_guard_fix then rewrites r32 and the guess of the cases that
// dropped theirs.
cudaError_t launch_r0(const MeshView& m, int rpad, double dt, const double* b, const double* Av4, const double* Av3,
                      const double* Av2, const double* Av1, const float* qy, float* r32, Reducer red, CgCase* outer,
                      int* n_active, double tol, double inner_max, double aim, cudaStream_t s,
                      Ring4 avr = Ring4{}, const StepCtl* ctl = nullptr, CgCase* inner = nullptr, bool guard = false,
                      int* fallbacks = nullptr);
cudaError_t launch_guard_fix(const MeshView& m, int rpad, const CgCase* outer, const float* qy, float* r32,
                             const double* du_ab, double* guess, double* x, cudaStream_t s);
cudaError_t launch_cert(const MeshView& m, int rpad, double cM, double cK, const double* b, const double* qM,
                        const double* qK, float* r32, Reducer red, CgCase* outer, int* n_active, double tol,
                        double inner_max, double aim, cudaStream_t s, CgCase* inner = nullptr);
// With ctl: v_prev, v_push, Av_push and the snapshot slot come from the rings (vr, avr, ring of slots of
// slot_stride elements) at the step read from ctl.
cudaError_t launch_newmark_incr(int64_t n, double dt, double cM, double cK, double a0, double a1, const double* du,
                                const double* du_ab, const double* qM, const double* qK, double* u,
                                const double* v_prev, double* a, double* v_push, double* Ku, double* Mv, double* Kv,
                                double* Pb, double* Av_push, void* e_push, int e_fmt, cudaStream_t s,
                                Ring4 vr = Ring4{}, Ring4 avr = Ring4{}, void* ring = nullptr,
                                int64_t slot_stride = 0, const StepCtl* ctl = nullptr);
// The same update in two parts: 1 the velocity side (v, M v, K v, A v, the snapshot), 2 the state side (u, a,
// K u, Pb), launched after part 1 (it reads the updated M v); 0 both, as launch_newmark_incr.
cudaError_t launch_newmark_incr_part(int64_t n, double dt, double cM, double cK, double a0, double a1,
                                     const double* du, const double* du_ab, const double* qM, const double* qK,
                                     double* u, const double* v_prev, double* a, double* v_push, double* Ku,
                                     double* Mv, double* Kv, double* Pb, double* Av_push, void* e_push, int e_fmt,
                                     cudaStream_t s, Ring4 vr, Ring4 avr, void* ring, int64_t slot_stride,
                                     const StepCtl* ctl, int part);
cudaError_t launch_axpby(int64_t n, double alpha, const double* x, double beta, const double* y, double* out,
                         cudaStream_t s);
// Split FP64 product: qM = M p and qK = K p in one pass (generic element kernel).
// Staged variant of the tiled hex kernel: each tile's node values and element records are brought into
// shared memory by bulk asynchronous (TMA) copies, double-buffered against the previous tile's compute.
// packed (FP32, not fused groups): each thread applies its hex to two cases with paired FP32 operations,
// 1 = registers capped for two blocks per SM, 2 = one block per SM; 0 = one case per thread.
template <typename T>
cudaError_t launch_ebe_hex_staged(const HexTiles& ht, const MeshView& m, int rpad, const T* p, T* q, double aM,
                                  double aK, const Reducer* red, CgCase* sc, double* ptq_out, const int* gate,
                                  cudaStream_t s, int packed = 0);
template <typename T>
size_t ebe_hex_staged_smem(const HexTiles& ht, const MeshView& m, int rpad);   // ~0 when not applicable
// Case-major staged variant: warps of 32 hexes of one case; converged cases (sc[c].active == 0) skipped.
template <typename T>
cudaError_t launch_ebe_hex_cm(const HexTiles& ht, const MeshView& m, int rpad, const T* p, T* q, double aM, double aK,
                              const Reducer* red, CgCase* sc, double* ptq_out, const int* gate, cudaStream_t s);
template <typename T>
size_t ebe_hex_cm_smem(const HexTiles& ht, const MeshView& m, int rpad);   // ~0 when not applicable
// Hex element matrices (variant 7): build the interleaved symmetric 24 x 24 matrices A_h = aM M_h + aK K_h
// of the mesh's hexes (n_hex, hex h = elements 6h .. 6h + 5, FP64 records) into out
// ([ceil(n_hex / 2)][300][2] floats), and the product q = A p with them (FP32, r cases, not fused groups).
cudaError_t launch_hexmat_build(int64_t n_hex, const double* rec64, double aM, double aK, float* out, cudaStream_t s);
// Variant 9: FP16 hex element matrices (784-byte records, one a hex) for the coefficients (aM, aK), and the
// FP32 product q = A p with them on the tensor cores (rpad 8 or 16; p^T q and the CG step length fused
// when red is given); smem ~0 when a tiling does not fit the kernel.
constexpr int kHm16RecBytes = 784;
cudaError_t launch_hexmat16_build(int64_t n_hex, const double* rec64, double aM, double aK, unsigned char* out,
                                  cudaStream_t s);
size_t ebe_hex_tc_smem(const HexTiles& ht, int rpad);
cudaError_t launch_ebe_hex_tc(const HexTiles& ht, const MeshView& m, const unsigned char* hm16, int rpad,
                              const float* p, float* q, double aM, double aK, const Reducer* red, CgCase* sc,
                              double* ptq_out, const int* gate, cudaStream_t s);
cudaError_t launch_ebe_hexmat(const HexTiles& ht, const MeshView& m, const float* hm, int rpad, const float* p,
                              float* q, double aM, double aK, const Reducer* red, CgCase* sc, double* ptq_out,
                              const int* gate, cudaStream_t s);
size_t ebe_hexmat_smem(const HexTiles& ht, const MeshView& m, int rpad);   // ~0 when not applicable
// q (+)= coef C_b p on the boundary nodes (free DOFs; assign: q = coef C_b p there).  red != nullptr: the
// per-case p . (coef C_b p) is added to ptq_out and to the CG state sc (p^T q and the step length), as the
// element-by-element product's tail does.  gate: skip when *gate == 0.  With ctl, p and q come from the rings
// pring / qring (when given) at step ctl->it + poff / + qoff.
template <typename T>
cudaError_t launch_dashpot(const Absorb& ab, int rpad, double coef, const T* p, T* q, bool assign,
                           const uint8_t* fm, const Reducer* red, CgCase* sc, double* ptq_out, const int* gate,
                           cudaStream_t s, Ring4 pring = Ring4{}, int poff = 0, Ring4 qring = Ring4{}, int qoff = 0,
                           const StepCtl* ctl = nullptr);
// D[node] += coef C_b[node] (node 3x3 diagonal blocks of A, before their inversion).
cudaError_t launch_add_node_blocks(const Absorb& ab, double coef, double* D, cudaStream_t s);
// b += the impulses of step `it` (or ctl->it) at their nodes and case lanes (free DOFs).
cudaError_t launch_impulses(const Impulses& im, int rpad, int it, const StepCtl* ctl, const uint8_t* fm, double* b,
                            cudaStream_t s);
// The heterogeneous predictor (hetero.cu): the data-driven correction of a group computed on the host.
struct HostPred;
cudaError_t hostpred_create(int64_t n, int rpad, int n_slots, int s_max, int fmt, double tau,
                            const std::vector<int32_t>& lo, const std::vector<int32_t>& hi, HostPred** out);
void hostpred_destroy(HostPred* h);
cudaError_t hostpred_push(HostPred* h, const void* dev_slot, int it, double solve_ms, cudaStream_t s);
const double* hostpred_take(HostPred* h, int it, int* n_pairs);
void hostpred_stats(const HostPred* h, int* s_cur, double* cpu_ms, double* solve_ms, double* cpu_sum,
                    double* wait_sum, long long* tasks);
const double* hostpred_coefficients(const HostPred* h, int* n_pairs);
// Reads and clears the flag a staged kernel sets when a bounded wait for its copies gave up.
cudaError_t ebe_tma_timeout(int* flag);
// Sets the number of tries (up to 1 us each) of the staged kernels' reporting wait (device-wide; ordered on s).
cudaError_t ebe_set_wait_budget(int tries, cudaStream_t s);
cudaError_t launch_ebe_split(const MeshView& m, int rpad, const double* p, double* qM, double* qK, cudaStream_t s);
// The same product in double-float arithmetic from (hi, lo) FP32 records rec_df [E][12][2].
cudaError_t launch_ebe_split_df(const MeshView& m, const float* rec_df, int rpad, const double* p, double* qM,
                                double* qK, cudaStream_t s);
cudaError_t launch_split_records(int64_t E, const double* rec64, float* rec_df, cudaStream_t s);

// Predictor (regions are node ranges [reg_lo[R], reg_hi[R])).
struct PredView {
  int n_regions;
  const int32_t* reg_lo;
  const int32_t* reg_hi;
  int rpad;
  int n_slots;             // ring size (s_max + 1)
  int64_t slot_stride;     // values per slot: N * 3 * rpad rounded up to a multiple of 8
  const void* ring;        // [n_slots] slots of [N][3][rpad] values, stored as fmt says
  int fmt;                 // snapshot storage: 0 FP64, 1 FP32, 2 double-float pairs, 3 FP32 + BF16 residual
  double* gram;            // [R][rpad][kMaxSlots][kMaxSlots]
  double* w;               // [R][rpad][kMaxSlots] coefficients in X order
  int n_chunks;            // node-range chunks per region (blocks per region of the dot/combine kernels)
  double* dpart;           // [R][n_chunks][kMaxSlots][rpad] partial dots
};
// valid_mask bit j = ring slot j holds a stored correction (64-bit: up to kMaxSlots = 33 slots).
// With ctl (graph steps) the slot lists, pair count, query/new slot and mask are read from ctl and the
// kernels are launched whatever the pair count (0 pairs: no correction).
cudaError_t launch_pred_dots(const PredView& p, int slot_new, uint64_t valid_mask, cudaStream_t s,
                             const StepCtl* ctl = nullptr);
cudaError_t launch_pred_solve(const PredView& p, const int* x_slots, int n_pairs, int slot_new, double tau,
                              cudaStream_t s, const StepCtl* ctl = nullptr);
cudaError_t launch_pred_combine(const PredView& p, const int* y_slots, int n_pairs, double* y_out, cudaStream_t s,
                                const StepCtl* ctl = nullptr, const double* y_base = nullptr,
                                float* corr32 = nullptr, const int32_t* gap_hi = nullptr, int lead_hi = 0,
                                double* y_out2 = nullptr);

// Assembled operators for the certification product (k_bcsr.cu): K as 3x3 blocks and M as scalars on the
// node pattern row_ptr/col.  assemble also writes the (hi, lo) FP32-pair copy KMd (per block the 9 pairs of
// the K block, then the pair of the M entry: 80 bytes); *missing = 1 if an element pair had no slot in the
// pattern.
cudaError_t launch_bcsr_assemble(const MeshView& m, const int32_t* row_ptr, const int32_t* col, int64_t nnz,
                                 double* Kb, double* Mb, float2* KMd, int* missing, cudaStream_t s);
// The 80-byte double-float block records KMd from the FP64 blocks Kb and mass entries Mb.
cudaError_t launch_to_kmd(int64_t nnz, const double* Kb, const double* Mb, float2* KMd, cudaStream_t s);
// 10-node tets (fem10.cu): the solver's products q = aM M pm + aK K pk (pk null: one input, p^T q and the CG
// step length fused when red is given), node diagonal blocks of aM M + aK K added into D, and the assembled
// operators of the certification product on a tet10 node pattern.
template <typename T>
cudaError_t launch_ebe10_gated(int64_t E, int64_t N, int rpad, const int32_t* conn10, const float* rec32,
                               const double* rec64, const uint8_t* fm, const T* pm, const T* pk, T* q, double aM,
                               double aK, const Reducer* red, CgCase* sc, double* ptq, const int* gate,
                               cudaStream_t s);
cudaError_t launch_diag10(int64_t E, const int32_t* conn10, const double* rec64, double aM, double aK, double* D,
                          cudaStream_t s);
cudaError_t launch_bcsr_assemble10(int64_t E, const int32_t* conn10, const double* rec64, const int32_t* row_ptr,
                                   const int32_t* col, int64_t nnz, double* Kb, double* Mb, float2* KMd, int* missing,
                                   cudaStream_t s);
// qM = M p, qK = K p (r cases, Dirichlet rows zero).  p_df != null: double-float arithmetic (p split into
// p_df first); else native FP64.
// q = (aM M + aK K) p with the assembled 3x3-block operators (EBE variant 8, the CRS-style comparator):
// FP64 blocks for FP64 products, the FP32 high words of KMd for FP32 ones; DOT (red != nullptr) fuses p^T q
// and the CG step length as the EBE products do.  Not for fused groups.
template <typename T>
cudaError_t launch_bcsr_apply(const MeshView& m, int rpad, const int32_t* row_ptr, const int32_t* col,
                              const double* Kb, const double* Mb, const float2* KMd, const T* p, T* q, double aM,
                              double aK, const Reducer* red, CgCase* sc, double* ptq_out, const int* gate,
                              cudaStream_t s);
cudaError_t launch_bcsr_split(const MeshView& m, int rpad, const int32_t* row_ptr, const int32_t* col,
                              const double* Kb, const double* Mb, const float2* KMd, const double* p, float2* p_df,
                              double* qM, double* qK, cudaStream_t s);

// Graph steps (k_graph.cu): device-side step control and the conditions of the graph's loops.
cudaError_t launch_step_begin(StepCtl* ctl, int n_slots, int s_max, double dt, int dd, long long n_fixed,
                              cudaStream_t s);
cudaError_t launch_set_cond(cudaGraphConditionalHandle h, unsigned value, cudaStream_t s);
cudaError_t launch_pass_begin(CgCase* outer, int ncase, int* n_active, int maxit, int max_pass, StepCtl* ctl,
                              cudaGraphConditionalHandle h_if, long long n_if, cudaStream_t s);
cudaError_t launch_inner_start(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_inner_start_sel(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h,
                                   const CgCase* outer, int ncase, double floor, int want_tc, cudaStream_t s);
cudaError_t launch_inner_cond(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, int chunk, int limit,
                              long long n_body, cudaStream_t s);
cudaError_t launch_pass_end(const int* n_active, StepCtl* ctl, cudaGraphConditionalHandle h, int max_pass,
                            long long n_body, cudaStream_t s);
cudaError_t launch_step_end(const CgCase* outer, int ncase, int* acc_iters, double* acc_relres, int* acc_status,
                            StepCtl* ctl, cudaStream_t s);
// y_out += Y w (as launch_pred_combine) and, in the same pass over the ring, y2 = Y w2.
cudaError_t launch_pred_combine2(const PredView& p, const int* y_slots, int n_pairs, double* y_out,
                                 const double* w2, double* y2, cudaStream_t s);

// Learned proposal (k_mlp.cu).  Rows of the network's batch are (region R, case c) -> R * rpad + c.
cudaError_t mlp_features(const PredView& p, int n_pairs, const float4* case_src, const float* centroid,
                         float inv_extent, float* F, cudaStream_t s);
cudaError_t mlp_propose(fem_mlp* net, const float* F, int64_t rows, int n_pairs, double* dw, cudaStream_t s);
cudaError_t mlp_to_f32(int64_t n, const double* x, float* y, cudaStream_t s);
cudaError_t mlp_choose(const MeshView& m, int rpad, const float* r32, const float* qd, Reducer red, CgCase* outer,
                       int* n_active, double tol, double inner_max, double aim, int ncase, int* choose,
                       long long* counts, cudaStream_t s);
cudaError_t mlp_apply(int64_t n, int rpad, const int* choose, float* r32, const float* qd, double* guess,
                      const double* dy, cudaStream_t s);
// Residual-space samples (features and the packed (W, w) of each region and case) from the ring Gram after the
// step's correction is pushed; y_slots: the step's Y slot list (device), slot_new: the pushed slot; e2: device
// scratch [ncase] for the cases' ||e||^2.
cudaError_t mlp_collect_res(const PredView& p, const int* y_slots, int n_pairs, int slot_new, double tau, int ncase,
                            const float* F, int64_t row0, float* x_out, float* s_out, double* e2, cudaStream_t s);
cudaError_t mlp_collect(int n_regions, int rpad, int ncase, int n_pairs, const float* F, const double* w_best,
                        const double* w_pred, int64_t row0, float* x_out, float* t_out, cudaStream_t s);
int mlp_device(const fem_mlp* n);

}  // namespace fem

// ---- device helpers ----
#ifdef __CUDACC__
namespace fem {

__device__ __forceinline__ bool dof_free(uint8_t fm, int k) { return (fm >> k) & 1; }

// Conversions between FP64 and double-float (hi, lo) FP32 pairs by integer bit operations.  GB300 executes
// double <-> float conversions on its narrow FP64 pipe; these use the integer pipe instead.
//   d2df: hi = x truncated to 24 significant bits, lo = the remainder truncated to 24 bits, so that
//         hi + lo = x to 2^-47 relative; |x| < 2^-126 maps to (0, 0); infinities and NaN keep the slow path.
//   f2d:  the exact FP64 value of a normal FP32 number; FP32 subnormals (|f| < 2^-126) map to 0.
__device__ __forceinline__ float2 d2df(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0x7ff) return make_float2((float)x, 0.0f);
  const int ef = e - 1023 + 127;
  if (ef <= 0) return make_float2(0.0f, 0.0f);
  if (ef >= 255) return make_float2((float)x, 0.0f);
  const uint64_t m = b & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((uint32_t)ef << 23) | (uint32_t)(m >> 29));
  const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFull);   // lo = rem * 2^(e - 1075)
  if (rem == 0u) return make_float2(hi, 0.0f);
  const int lz = __clz(rem);
  const int el = e - 1075 + (31 - lz) + 127;
  if (el <= 0) return make_float2(hi, 0.0f);
  const uint32_t mant = (uint32_t)((((uint64_t)rem << (lz + 1)) & 0xFFFFFFFFull) >> 9);
  return make_float2(hi, __uint_as_float(sign | ((uint32_t)el << 23) | mant));
}
// FP64 -> FP32 by truncation to 24 significant bits (integer pipe); |x| < 2^-126 maps to 0.
__device__ __forceinline__ float d2f(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const int ef = e - 1023 + 127;
  if (e == 0x7ff || ef >= 255) return (float)x;
  if (ef <= 0) return 0.0f;
  return __uint_as_float(((uint32_t)(b >> 32) & 0x80000000u) | ((uint32_t)ef << 23) |
                         (uint32_t)((b & 0xFFFFFFFFFFFFFull) >> 29));
}
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  if (e == 0xffu) return (double)f;
  return __longlong_as_double((long long)(((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                                          ((uint64_t)(u & 0x7fffffu) << 29)));
}

// Relative reduction asked of the next inner FP32 solve: just enough for one refinement pass to reach `aim`
// (a margin below the FP64 tolerance: aim / current relative residual), but no finer than `floor` (what FP32
// can deliver) and at least a halving.
__device__ __forceinline__ double inner_target(double aim, double relres, double floor) {
  double t = relres > 0.0 ? aim / relres : floor;
  if (t > 0.5) t = 0.5;
  if (t < floor) t = floor;
  return t;
}

// Number of cases the per-case arrays of a launch cover.
__host__ __device__ __forceinline__ int n_cases(const MeshView& m, int rpad) { return m.seg ? m.nseg : rpad; }

// Segmented accumulation for fused groups: per-case sums in shared memory acc[q * ncase + c].  Every lane
// of the warp must call it (invalid items pass value 0 and any case); a warp whose lanes all hold the same
// case reduces by shuffles and adds once.
template <int NQ>
__device__ __forceinline__ void seg_add(double* acc, int ncase, int c, const double (&v)[NQ]) {
  const int c0 = __shfl_sync(0xffffffffu, c, 0);
  if (__all_sync(0xffffffffu, c == c0)) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = v[q];
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if ((threadIdx.x & 31) == 0) atomicAdd(acc + q * ncase + c0, x);
    }
  } else {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (v[q] != 0.0) atomicAdd(acc + q * ncase + c, v[q]);
  }
}

// Grid-wide per-case sums of the shared accumulators acc[NQ * ncase] (all threads call it after the loop);
// returns true in the last block with red.out[q * ncase + c] holding the totals (fixed summation order
// over blocks).
template <int NQ>
__device__ __forceinline__ bool block_reduce_last_seg(double* acc, int ncase, const Reducer& red) {
  __shared__ bool am_last;
  const int V = NQ * ncase;
  __syncthreads();
  for (int t = threadIdx.x; t < V; t += blockDim.x) red.partial[(size_t)blockIdx.x * V + t] = acc[t];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(red.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  for (int t = threadIdx.x; t < V; t += blockDim.x) {
    double a0 = 0.0, a1 = 0.0;
    int b = 0;
    const int nb = (int)gridDim.x;
    for (; b + 1 < nb; b += 2) {
      a0 += __ldcg(red.partial + (size_t)b * V + t);
      a1 += __ldcg(red.partial + (size_t)(b + 1) * V + t);
    }
    if (b < nb) a0 += __ldcg(red.partial + (size_t)b * V + t);
    red.out[t] = a0 + a1;
  }
  if (threadIdx.x == 0) *red.counter = 0u;
  __syncthreads();
  return true;
}

// Last block of a product with the fused p^T q: publish it and set the CG step length alpha.
__device__ __forceinline__ void ebe_tail(const Reducer& red, CgCase* sc, double* ptq_out, int rpad) {
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

// Per-case sums over the grid.  Threads hold vals[q] for case c = threadIdx.x % rpad (the grid stride of
// every caller is a multiple of rpad).  Returns true in the last block to finish, after red.out[q*rpad+c]
// holds the grid totals (summed in a fixed order: deterministic).
template <int NQ>
__device__ __forceinline__ bool block_reduce_last(double (&vals)[NQ], int rpad, const Reducer& red) {
  __shared__ double sh[kVecBlock / 32][NQ][32];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double v = vals[q];
    for (int off = 16; off >= rpad; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane < rpad) sh[warp][q][lane] = v;
  }
  __syncthreads();
  const int V = NQ * rpad;
  if (threadIdx.x < V) {
    const int q = threadIdx.x / rpad, c = threadIdx.x % rpad;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w][q][c];
    red.partial[(size_t)blockIdx.x * V + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(red.counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double* flat = &sh[0][0][0];
  int S = blockDim.x / V;
  if (S * V > (kVecBlock / 32) * NQ * 32) S = (kVecBlock / 32) * NQ * 32 / V;
  if (threadIdx.x < S * V) {
    const int v = threadIdx.x % V, sl = threadIdx.x / V;
    // eight loads in flight per round so the L2 latency is paid few times; fixed assignment keeps the sum
    // deterministic
    double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int b = sl;
    const int nb = (int)gridDim.x;
    for (; b + 7 * S < nb; b += 8 * S) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = __ldcg(red.partial + (size_t)(b + u * S) * V + v);
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] += t[u];
    }
    for (int u = 0; b < nb; b += S, ++u) a[u & 7] += __ldcg(red.partial + (size_t)b * V + v);
    flat[sl * V + v] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
  __syncthreads();
  if (threadIdx.x < V) {
    double acc = 0.0;
    for (int sl = 0; sl < S; ++sl) acc += flat[sl * V + threadIdx.x];
    red.out[threadIdx.x] = acc;
  }
  if (threadIdx.x == 0) *red.counter = 0u;
  __syncthreads();
  return true;
}

}  // namespace fem
#endif
