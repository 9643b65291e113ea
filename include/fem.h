/*
 * libfem -- matrix-free element-by-element (EBE) solver for many time-evolution linear-elastic FE cases,
 * with the data-driven initial-guess predictor, for one NVIDIA GB300 GPU (sm_103a).
 *
 * The operations follow Ichimura et al., "Heterogeneous computing in a strongly-connected CPU-GPU
 * environment: fast multiple time-evolution equation-based modeling accelerated using data-driven
 * approach" (arXiv 2409.20380):
 *   - the target problem: many cases of A x^it = f^it solved sequentially in it (Section 2.1, Eq. 1);
 *   - the Newmark-beta system A = 4M/dt^2 + 2C/dt + K with C = a0 M + a1 K and its right-hand side
 *     (Section 3.1, Eq. GE:DIS), and the velocity/acceleration update (Section 3.1, Eq. timestep);
 *   - the EBE matrix-vector product q = sum_e P_e^T A_e P_e p, for r cases at once (Section 3.2,
 *     Eq. eqebefem and Eq. eqmebefem);
 *   - the 3x3 block-Jacobi preconditioned CG (Algorithm 1);
 *   - the Adams-Bashforth initial guess and the regional orthogonal-decomposition predictor (Section 3.2).
 * Elements are linear 4-node tetrahedra (12x12 element matrices); the paper's own runs use 10-node tets.
 *
 * Conventions for every entry point:
 *   - Return value: FEM_OK (0) or a negative fem_status; fem_last_error() gives a message (thread-local).
 *     No call aborts, traps or prints.
 *   - Host pointers (named *_host or documented as host) are read during the call and copied; the caller
 *     keeps ownership.  Device pointers (*_dev) are caller-owned device memory of the current device; the
 *     library never frees them.
 *   - Work is ordered on the CUDA stream passed as `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Calls that return per-case results to host memory synchronise that stream.
 *   - Multi-case nodal vectors use the layout [node][3][n_rhs] (component-major within a node, case
 *     fastest), i.e. value (node n, direction k, case c) is at index (n*3 + k)*n_rhs + c.  n_rhs must be
 *     1, 2, 4, 8, 16 or 32.
 *   - Dirichlet DOFs (fixed_dof = 1) hold zero in every solution; their entries of right-hand sides are
 *     ignored and their entries of matrix-vector products are returned as zero.
 */
#ifndef FEM_H_
#define FEM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fem_status;
enum {
  FEM_OK = 0,
  FEM_ERR_ARG = -1,            /* invalid argument (null pointer, size, layout, unsupported option) */
  FEM_ERR_OOM = -2,            /* device allocation failed */
  FEM_ERR_CUDA = -3,           /* a CUDA runtime call or kernel launch failed */
  FEM_ERR_NOT_CONVERGED = -4,  /* maxit reached before the certified tolerance */
  FEM_ERR_BREAKDOWN = -5,      /* p^T A p <= 0 or a non-finite CG scalar */
  FEM_ERR_NONFINITE = -6,      /* NaN/Inf in inputs or results */
  FEM_ERR_TIMEOUT = -7,        /* a bounded device-side wait expired */
  FEM_ERR_STATE = -8           /* call not valid in the object's current state */
};

/* Precision of the solve. */
enum {
  FEM_FP64 = 0,          /* every operation in FP64 (the plain method) */
  FEM_FP32_INNER = 1     /* FP32 EBE + preconditioner inside an inner PCG; FP64 outer residual,
                            dot-product accumulation and refinement update; certified in FP64 */
};

/* Product of the inner FP32 solve's CG iterations (FEM_FP32_INNER). */
enum {
  FEM_INNER_FP32 = 0,    /* the FP32 element-by-element kernels (the default) */
  FEM_INNER_TC = 1       /* per-hex 24 x 24 element matrices of A in FP16 (the element data in reduced precision),
                            applied on the tensor cores with FP32 accumulation: ~2.4e-4 relative error in a
                            product, so a refinement pass takes these products only when every active case's
                            reduction target is 1e-3 or coarser (its inner solve shrinks the residual by at most
                            a factor of 1000: a good initial guess); other passes take the FP32 kernels.  Hex-patch meshes, groups of 5..16 cases
                            (8 or 16 lanes; other groups keep the FP32 kernels); the predictor's correction and
                            all other products stay FP32/FP64 */
};

/* Initial-guess predictor used by fem_step. */
enum {
  FEM_PRED_AB4 = 0,      /* Adams-Bashforth 4 (Section 3.2) */
  FEM_PRED_DD = 1        /* Adams-Bashforth 4 + regional data-driven correction (Section 3.2) */
};

/* What fem_case_get returns. */
enum {
  FEM_FIELD_U = 0,       /* displacement u^it */
  FEM_FIELD_V = 1,       /* velocity v^it */
  FEM_FIELD_A = 2,       /* acceleration a^it */
  FEM_FIELD_DU = 3,      /* last solved increment du = u^it - u^{it-1} */
  FEM_FIELD_B = 4,       /* last right-hand side b (Section 3.1, Eq. GE:DIS in increment form) */
  FEM_FIELD_GUESS = 5    /* last initial guess of the increment handed to the solver */
};

typedef struct {
  double dt;             /* time increment */
  double beta;           /* Newmark beta; only 0.25 is supported */
  double gamma;          /* Newmark gamma; only 0.5 is supported */
  double a0, a1;         /* Rayleigh damping C = a0 M + a1 K */
} fem_time_params;

typedef struct {
  int precision;         /* FEM_FP64 or FEM_FP32_INNER */
  int predictor;         /* FEM_PRED_AB4 or FEM_PRED_DD */
  double tol;            /* certified relative residual ||b - A x|| / ||b|| (Algorithm 1's epsilon) */
  int maxit;             /* max CG iterations per solve (inner iterations summed in FEM_FP32_INNER) */
  int s_max;             /* max stored snapshot pairs s of the data-driven predictor (<= 32) */
  double inner_tol;      /* FEM_FP32_INNER: finest relative reduction asked of one inner FP32 solve; each
                            inner solve asks for just enough to reach inner_margin x tol,
                            but not less than this */
  double tau;            /* predictor column-drop threshold (relative orthogonalised norm) */
  int snapshot_format;   /* predictor snapshot storage: 0 = FP64; 1 = FP32 (half the memory; the prediction
                            loses the small orthogonal components FP32 rounds away); 2 = double-float pairs
                            (hi, lo FP32: FP64 size, 48-bit significand, arithmetic on the FP32 pipe);
                            3 = FP32 value and its residual rounded to BF16 (6 bytes, about 32-bit
                            significand, read as double-float pairs) */
  int check_every;       /* CG iterations between host-side convergence polls (>= 1) */
  int refresh_every;     /* FEM_FP32_INNER steps: every this many steps the products K u, M v, K v, M a and
                            A v^{it-3..it} that fem_step keeps by recurrence are recomputed directly
                            (0 = 200) */
  int cert_df;           /* FEM_FP32_INNER steps: form of the FP64-accurate certification product (the split
                            products M du, K du; see fem_mesh_split_product): 0 = element-by-element FP64,
                            1 = element-by-element double-float (FP32 pairs, 48-bit significand),
                            2 = assembled 3x3 blocks FP64, 3 = assembled 3x3 blocks double-float */
  int fuse_meshes;       /* 1 = solve all cases of the batch as one fused system (each case on its own mesh
                            copy; meshes of different sizes; one set of launches for all; at most 128 cases;
                            FEM_FP32_INNER only); 0 = one multi-RHS system per mesh */
  int use_graph;         /* FEM_FP32_INNER steps: 1 = each group's step is captured once as a CUDA graph
                            (device-side step counter, conditional loops for the refinement passes and the
                            inner PCG) and replayed with no host synchronisation between steps; statistics
                            are read once per fem_step call.  Steps with profiling on, a learned proposal or
                            sample collection run eagerly.  0 = eager launches with host-side control */
  int wait_budget;       /* bounded device-side waits (the staged EBE kernels' waits for their bulk tile copies):
                            tries of up to 1 us each before a wait gives up and the call reports
                            FEM_ERR_TIMEOUT (the kernel then still waits, bounded, for the copies in flight,
                            so none outlives it; results of a timed-out call are not to be used).  The value
                            is device-wide: fem_step, fem_step_async and pcg_solve set it before their work,
                            fem_ebe_apply and fem_mesh_autotune restore the default.  0 = a wait that has not
                            completed at once reports (a way to exercise the error path); default 1048576
                            (about a second); must be >= 0 */
  int cpu_predictor;     /* 1 = the paper's heterogeneous scheme (Algorithm 3): the data-driven correction is
                            computed on the host CPU from a pinned host copy of the stored corrections while the
                            GPU steps the other case set (the cases of a mesh are split into two sets), and s is
                            adjusted after every step toward equal prediction and solve times (s_max is the
                            ceiling).  Needs FEM_PRED_DD, regions, snapshot_format 0 or 2, no fuse_meshes and
                            no learned proposal; steps run eagerly.  0 = the predictor runs on the GPU */
  double inner_margin;   /* FEM_FP32_INNER: each inner FP32 solve is asked for the reduction that brings the
                            certified residual to inner_margin x tol (its FP32 recursive residual tracks the FP64
                            one to ~1e-7 of the pass's right-hand side), within [inner_tol, 0.5]; a case that
                            still ends at or above tol takes another refinement pass, so every step stays
                            certified below tol.  In (0, 1); default 0.5 (measured: 0.1 cost 3.5% more time on the
                            large workload for the same certificate) */
  int inner_product;     /* FEM_INNER_FP32 or FEM_INNER_TC (see above); the FP16 hex matrices (784 bytes a hex)
                            are built on the group's first step.  Default FEM_INNER_FP32 */
  int pred_guard;        /* FEM_FP32_INNER steps with FEM_PRED_DD: 1 = guess guard: per case, the step starts from
                            whichever guess has the smaller initial residual, the data-driven one (Adams-Bashforth
                            plus the regional correction) or the Adams-Bashforth one alone; the residual of the
                            latter comes from the same pass (the correction's FP32 product is formed anyway), so
                            the guard costs one more norm in that pass and a fix pass that returns at once unless a
                            case dropped its correction (fem_case_stats reports which guess a step used and how
                            often the correction was dropped).  Not applied to steps that take a learned
                            proposal.  0 = always the data-driven guess.  Default 1 */
} fem_opts;

/* Fills `o` with defaults: FP64, AB4, tol 1e-8, maxit 5000, s_max 32, inner_tol 1e-6, tau 1e-6,
 * snapshot_format 2, check_every 8, refresh_every 200, cert_df 3, fuse_meshes 0, use_graph 1,
 * wait_budget 1048576, cpu_predictor 0, inner_margin 0.5, inner_product FEM_INNER_FP32, pred_guard 1. */
void fem_opts_default(fem_opts* o);

typedef struct fem_mesh fem_mesh;    /* opaque: device copies of geometry, element records, preconditioner */
typedef struct fem_batch fem_batch;  /* opaque: per-case time-stepping state and predictor snapshots */

/*
 * Creates a mesh on the current device and precomputes, on the GPU, what the EBE operator needs
 * (Section 3.2, Eq. eqebefem): per-element shape-function gradients and volume-weighted material
 * coefficients, the node 3x3 diagonal blocks of A = (4/dt^2 + 2 a0/dt) M + (1 + 2 a1/dt) K and their
 * inverses (Algorithm 1's block-Jacobi B^{-1}; only the free DOFs of a node enter its block).
 *   xyz        [n_nodes][3] host, FP64 coordinates.
 *   conn       [n_elems][4] host, node ids of each linear tet, positively oriented (det > 0).
 *   mat_id     [n_elems] host, index into lam_mu_rho.
 *   lam_mu_rho [n_mat][3] host, (lambda, mu, rho) per material.
 *   fixed_dof  [3*n_nodes] host, 1 = Dirichlet (value 0), 0 = free.
 *   tp         time parameters (beta = 1/4, gamma = 1/2 only).
 * Errors: FEM_ERR_ARG for null pointers, ids out of range, non-positive volumes or unsupported Newmark
 * parameters; FEM_ERR_OOM / FEM_ERR_CUDA.  Synchronises `stream`.
 */
fem_status fem_mesh_create(int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn,
                           const int32_t* mat_id, int n_mat, const double* lam_mu_rho,
                           const uint8_t* fixed_dof, const fem_time_params* tp, void* stream,
                           fem_mesh** out);
/*
 * The same mesh object for 10-node tetrahedra, the paper's element (Section 3.1), so that the time-stepping
 * solver (fem_case_add, fem_step: Eq. GE:DIS, Algorithm 1, the predictors of Section 3.2) runs on quadratic
 * tets.  Straight-sided elements; local node order: corners 0-3, then the edge nodes of (0,1), (1,2), (0,2),
 * (0,3), (1,3), (2,3).  Arguments as fem_mesh_create's, with conn10 [n_elems][10] host int32 (the corner tet
 * positively oriented).  The products are the tet10 element-by-element kernel (stiffness by the 4-point Gauss
 * rule, exact for these elements; consistent mass by exact integration) in FP64 or FP32; the certification
 * product's assembled 3x3 blocks are assembled from the same operators (cert_df 2, 3), and cert_df 0 and 1
 * both take the FP64 element kernel.  The block-Jacobi B^{-1} comes from the tet10 node diagonal blocks.  Not
 * available on such a mesh: absorbing faces, fuse_meshes, fem_mesh_autotune (fem_mesh_tune selects variant 0,
 * the element kernel, or 8, the assembled blocks).  Predictor regions must be contiguous node ranges, as for
 * linear tets: number the nodes (corner and edge nodes alike) in an order with locality.
 * Errors: as fem_mesh_create's (every conn10 entry is range-checked on the host).
 */
fem_status fem_mesh_create_tet10(int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn10,
                                 const int32_t* mat_id, int n_mat, const double* lam_mu_rho,
                                 const uint8_t* fixed_dof, const fem_time_params* tp, void* stream,
                                 fem_mesh** out);
fem_status fem_mesh_destroy(fem_mesh* m);

/*
 * Absorbing boundary (the paper applies absorbing boundary conditions to the sides of the domain, Section 3.1;
 * the form is not given there): viscous dashpots of Lysmer and Kuhlemeyer on the listed boundary faces.  Each
 * face f of faces [n_faces][3] (host int32 node triples, copied) must be a face of exactly one element; with
 * its area, the outward unit normal n (away from that element's fourth node) and the element's material,
 * c_p = sqrt((lambda + 2 mu) / rho), c_s = sqrt(mu / rho), each of its three nodes gets the 3x3 damping block
 * (area / 3) rho (c_p n n^T + c_s (I - n n^T)).  The blocks form C_b, added to the damping:
 * C = a0 M + a1 K + C_b, so the system of every later solve and step is A = cM M + cK K + (2/dt) C_b and the
 * right-hand side gains C_b v (Section 3.1, Eq. GE:DIS); the block-Jacobi preconditioner includes (2/dt) C_b.
 * The element product entry points (fem_ebe_apply, fem_mesh_split_product) stay without it.  n_faces = 0
 * removes the dashpots; a new call replaces the previous faces.  Not for meshes of fuse_meshes batches.
 * Synchronises `stream`.  Errors: FEM_ERR_ARG (a face that is not on exactly one element, bad ids, zero area).
 */
fem_status fem_mesh_set_absorbing(fem_mesh* m, int64_t n_faces, const int32_t* faces, void* stream);

/*
 * Selects the EBE product implementation of a mesh (library tuning knob; the paper's EBE is one product,
 * Section 3.2, Eq. eqebefem).  ebe_variant: 0 = automatic, 1 = generic element kernel, 2 = tiled hex-patch
 * kernel (available when the elements come in groups of six tets splitting a hexahedron with the Kuhn
 * topology, which fem_mesh_create detects), 3 = the tiled hex kernel with each tile's node values and
 * element records staged in shared memory first by bulk asynchronous copies (double-buffered), 4 = as 3
 * with warps of one case each, so cases whose inner solve has converged are skipped, 5 = as 3 with each
 * thread applying its hex to two cases at once by paired FP32 operations (FP32 products of groups with
 * n_rhs >= 4; FP64 products and fused groups use 3), registers capped for two blocks per SM, 6 = as 5 with
 * one block per SM (variants 3-6 need 3 x n_rhs x element size to be a multiple of 16 bytes; otherwise 3,
 * then 2, then 1 is used), 7 = hex element matrices: each hex's six tets summed once into its symmetric
 * 24 x 24 matrix aM M_h + aK K_h (FP64 sums stored FP32, 1200 bytes a hex, built on first use, kept with
 * the mesh) and applied as dense blocks to pairs of hexes by paired FP32 operations, 64-hex tiles (FP32
 * products with the mesh's own Newmark coefficients and 16-byte aligned vectors, not fused groups;
 * otherwise 5 is used), 8 = not element by element: the assembled 3x3-block operators (the CRS-style
 * product the paper compares the EBE with, Section 3.3; built on first use and shared with the
 * certification product), FP64 blocks for FP64 products and their FP32 rounding for FP32 ones, any mesh,
 * not fused groups (those use 5, or 1 without hex patches).  hex_per_tile: 0 = automatic (largest tile
 * whose shared memory fits), or 64/128/256/512 hexes per tile.  Errors: FEM_ERR_ARG for other values or
 * variants 2-7 on a mesh without hex patches.
 */
fem_status fem_mesh_tune(fem_mesh* m, int ebe_variant, int hex_per_tile);

/*
 * Autotuner: times each EBE implementation that applies to the mesh on the inner solve's product
 * (q = A p with the fused p^T A p, n_rhs cases; FEM_FP32_INNER = FP32 product, FEM_FP64 = FP64 product):
 * the generic element kernel, the tiled hex kernel with 64/128/256/512 hexes per tile, the staged tiled
 * kernel with 64/128/256, the case-major staged kernel with 64/128 and the packed staged kernels with
 * 64/128/256 hexes per tile, where their shared memory fits.  The fastest is kept for that precision and n_rhs and used whenever
 * fem_mesh_tune is left at automatic (0, 0).  Outputs (nullable): the chosen variant and tile size, and its
 * time per product in ms.  Runs on `stream` and synchronises it; allocates two temporary vectors.
 */
fem_status fem_mesh_autotune(fem_mesh* m, int precision, int n_rhs, void* stream, int* ebe_variant_out,
                             int* hex_per_tile_out, double* ms_out);

/*
 * Split product qM = M p and qK = K p (Section 3.1: the mass and stiffness of Eq. GE:DIS, tet4 elements),
 * n_rhs cases in the [node][3][n_rhs] layout, FP64 in and out, Dirichlet rows zero.  This is the product
 * the FP32-inner solver certifies with and advances its recurrences by (b - cM qM - cK qK).  mode:
 *   0 = element by element in FP64 (the matrix-free form of Eq. eqebefem);
 *   1 = element by element in double-float arithmetic (records and inputs as FP32 pairs);
 *   2 = assembled operators in FP64: K as 3x3 blocks and M as scalars on the node pattern, assembled on the
 *       device from the same FP64 element records (built on first use and kept with the mesh);
 *   3 = the assembled operators in double-float arithmetic.
 * Modes 0 and 2 round like FP64; 1 and 3 to about 1e-14 of the largest term.  Modes 2/3 need
 * ~84 bytes x 15 x n_nodes of device memory for the operators.  Mode 3 allocates a temporary input copy.
 */
fem_status fem_mesh_split_product(fem_mesh* m, int mode, const double* p_dev, double* qM_dev, double* qK_dev,
                                  int n_rhs, void* stream);

/* Reports whether the mesh has hex patches and its current EBE variant and tile size (nullable outputs). */
fem_status fem_mesh_info(const fem_mesh* m, int* has_hex_patches, int* ebe_variant, int* hex_per_tile);

/*
 * Sets the predictor's regions (Section 3.2: the domain is divided into small regions, each predicted
 * independently).  region_of_node [n_nodes] host: region id >= 0, or -1 for a node with no free DOF.
 * The nodes of one region must form a contiguous node-id range (nodes with id -1 may sit inside it).
 * Errors: FEM_ERR_ARG if ids are out of range or a region is not contiguous.
 */
fem_status fem_mesh_set_regions(fem_mesh* m, const int32_t* region_of_node);

/*
 * Matrix-free EBE product (Section 3.2, Eq. eqebefem / eqmebefem), for n_rhs cases at once:
 *   q = sum_e P_e^T ((alpha_M M_e + alpha_K K_e) (P_e p)),  q = 0 on Dirichlet DOFs.
 * With alpha_M = 4/dt^2 + 2 a0/dt and alpha_K = 1 + 2 a1/dt this is q = A p.
 *   precision FEM_FP64: p_dev, q_dev are double*; FEM_FP32_INNER: float* (FP32 element records).
 *   p_dev, q_dev [n_nodes][3][n_rhs] device; p must be zero on Dirichlet DOFs; q is overwritten.
 *   ptq_dev      optional [n_rhs] device double*: receives p^T q per case, accumulated element by
 *                element (p_e^T A_e p_e) with FP64 reduction; NULL to skip.
 * Errors: FEM_ERR_ARG (null pointers, n_rhs), FEM_ERR_CUDA.
 */
fem_status fem_ebe_apply(fem_mesh* m, int precision, const void* p_dev, void* q_dev, int n_rhs,
                         double alpha_M, double alpha_K, double* ptq_dev, void* stream);

/*
 * Allocation-free variant of fem_ebe_apply (the paper has no counterpart: this is a library service).
 * Same arguments and errors as fem_ebe_apply, but it never allocates device memory (no cudaMalloc/cudaFree,
 * no allocating library routine).  It always runs the generic element kernel (one thread per element and
 * case, scatter by global atomics; the tet10 element kernel on a fem_mesh_create_tet10 mesh), not the tiled
 * or autotuned kernel fem_ebe_apply may choose, so it can be
 * slower, and its q and p^T q equal fem_ebe_apply's to rounding (FP32 atomics add in varying order), not bit
 * for bit.  It is meant for callers that cannot allocate:
 * code whose device memory is owned by another allocator under a fixed budget, and latency-critical loops
 * that cannot take the device-wide synchronisation cudaMalloc/cudaFree may cause.  The scratch of the
 * p^T q reduction is one fixed device array of 311,808 bytes inside the library (per-block partial sums
 * for up to 32 cases), present on every GPU that loads the library until the process exits.
 *   - n_rhs above 32 is rejected with FEM_ERR_ARG; the mesh's device must be the current device.
 *   - The first call with ptq_dev != NULL on a device looks up the array's device address (a one-time
 *     set-up per device); make that first call before any stream capture.
 *   - Every call uses the same array: calls whose kernels overlap on the GPU (e.g. on two streams without
 *     ordering between them) race and give wrong p^T q values.  Order such calls on one stream.
 *   - q is overwritten and the reduction counter is cleared by each call; nothing else needs zeroing.
 */
fem_status fem_ebe_apply_noalloc(fem_mesh* m, int precision, const void* p_dev, void* q_dev, int n_rhs,
                                 double alpha_M, double alpha_K, double* ptq_dev, void* stream);

/*
 * 10-node tetrahedra, the paper's element (Section 3.1): a separate mesh object for the EBE product of
 * quadratic tets (Section 3.2, Eq. eqebefem with 30 x 30 element operators formed on the fly).
 * Straight-sided elements; local node order: corners 0-3, then the edge nodes of (0,1), (1,2), (0,2),
 * (0,3), (1,3), (2,3).  Stiffness by the 4-point Gauss rule (exact for these elements), consistent mass
 * by exact integration.
 *   n_nodes, xyz     [n_nodes][3] host double, copied;  n_elems, conn10 [n_elems][10] host int32 (0-based);
 *   mat_id           [n_elems] host int32 in [0, n_mat);  lam_mu_rho [n_mat][3] host double (lambda, mu, rho);
 *   fixed_dof        [3 n_nodes] host uint8, 1 = Dirichlet;  stream: CUDA stream (NULL = default).
 *   out              receives the handle (owned by the caller; release with fem_mesh10_destroy).
 * Errors: FEM_ERR_ARG (null pointers, empty mesh, node ids out of range, a degenerate or inverted corner
 * tet, a bad material id), FEM_ERR_CUDA.  The call synchronises the stream.
 */
typedef struct fem_mesh10 fem_mesh10;
fem_status fem_mesh10_create(int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn10,
                             const int32_t* mat_id, int n_mat, const double* lam_mu_rho, const uint8_t* fixed_dof,
                             void* stream, fem_mesh10** out);
fem_status fem_mesh10_destroy(fem_mesh10* m);
/*
 * q = sum_e P_e^T ((alpha_M M_e + alpha_K K_e) (P_e p)) on the tet10 mesh, q = 0 on Dirichlet DOFs, for
 * n_rhs (1, 2, 4, ..., 32) cases; the same layout, precision choice and optional ptq_dev (p^T q per case,
 * element by element, FP64 reduction) as fem_ebe_apply.  Stream-ordered; calls on one mesh share its
 * reduction scratch, so calls whose kernels could overlap (two streams without ordering) must not share a
 * mesh.  Errors: FEM_ERR_ARG, FEM_ERR_CUDA.
 */
fem_status fem_ebe10_apply(fem_mesh10* m, int precision, const void* p_dev, void* q_dev, int n_rhs,
                           double alpha_M, double alpha_K, double* ptq_dev, void* stream);
/*
 * Block-Jacobi PCG (Algorithm 1) on the tet10 system (alpha_M M + alpha_K K) x = b for n_rhs cases, the
 * product being the tet10 EBE: each case iterates until ||b - A x|| / ||b|| < tol.  precision FEM_FP64:
 * plain FP64 PCG, confirmed with the true residual when the recursive one converges; FEM_FP32_INNER: the
 * FP64 residual r = b - A x (FP64 product), an inner FP32 PCG on A d = r from zero (FP32 product), x += d,
 * repeated until the FP64 residual meets tol (iterations counted over all inner solves).
 *   b_dev       [n_nodes][3][n_rhs] device double (zero on Dirichlet DOFs);
 *   x_dev       [n_nodes][3][n_rhs] device double, in: initial guess (zeroed on Dirichlet DOFs), out: solution;
 *   iters_out, relres_out  optional host [n_rhs]: iterations and final relative residual per case.
 * Allocates its work vectors per call and synchronises the stream.  Errors: FEM_ERR_ARG (arguments, a
 * singular diagonal block), FEM_ERR_NOT_CONVERGED (maxit reached), FEM_ERR_BREAKDOWN, FEM_ERR_NONFINITE,
 * FEM_ERR_CUDA.
 */
fem_status pcg10_solve(fem_mesh10* m, int precision, const double* b_dev, double* x_dev, int n_rhs,
                       double alpha_M, double alpha_K, double tol, int maxit, void* stream, int* iters_out,
                       double* relres_out);

/*
 * Solves A x = b for n_rhs cases (Algorithm 1: 3x3 block-Jacobi PCG with the EBE product), starting from
 * the guess in x_dev.  With opts->precision = FEM_FP32_INNER the solve is an FP64 iterative refinement
 * whose corrections come from an FP32 inner PCG.  Either way each case stops when its FP64 true residual
 * ||b - A x|| / ||b|| < opts->tol (a recursive residual below tol is re-checked against the true one and
 * the iteration continues if needed).  ||b|| = 0 gives x = 0 and 0 iterations.
 *   b_dev, x_dev [n_nodes][3][n_rhs] device doubles; x is in: guess, out: solution (0 on Dirichlet DOFs).
 *   iters_out    [n_rhs] host (nullable): CG iterations per case (inner iterations in FEM_FP32_INNER).
 *   relres_out   [n_rhs] host (nullable): certified FP64 relative residual per case.
 * Returns FEM_ERR_NOT_CONVERGED if some case hit maxit, FEM_ERR_BREAKDOWN on p^T A p <= 0.
 * Scratch vectors are allocated by the library (cached in the mesh).  Synchronises `stream`.
 */
fem_status pcg_solve(fem_mesh* m, const double* b_dev, double* x_dev, int n_rhs, const fem_opts* opts,
                     void* stream, int* iters_out, double* relres_out);

/* Creates an empty batch of cases; all later work of the batch is ordered on `stream`. */
fem_status fem_batch_create(const fem_opts* opts, void* stream, fem_batch** out);
fem_status fem_batch_destroy(fem_batch* b);

/*
 * Adds a case on mesh `m` starting at rest, loaded by a Ricker-wavelet point force
 *   f(t) = amp (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2) * dir   at node src_node,
 * evaluated at t = it * dt (the paper's runs use random impulses at surface points, Section 3.1).
 * Cases on the same mesh are solved together as one multi-RHS system (Section 3.2, Eq. eqmebefem), in
 * groups of at most 32.  Must be called before the first fem_step.  case_id receives the case index.
 */
fem_status fem_case_add(fem_batch* b, fem_mesh* m, int32_t src_node, const double dir[3], double f0,
                        double t0, double amp, int* case_id);

/*
 * Adds a case on mesh `m` starting at rest, loaded by random impulses (the paper's random inputs: impulse
 * waveforms of random amplitude and uniform spectrum in random directions at randomly selected surface
 * points, Section 3.1): impulse k acts during time step steps[k] (>= 1) only, as the force forces[k] [3] at node
 * nodes[k].  Several impulses may share a node and a step (they add).  Host arrays, copied:
 * nodes [n], steps [n] int32, forces [n][3] double.  Must be called before the first fem_step; not with
 * fuse_meshes.  Errors: FEM_ERR_ARG (ids out of range, steps < 1, non-finite forces), FEM_ERR_STATE.
 */
fem_status fem_case_add_impulses(fem_batch* b, fem_mesh* m, int64_t n, const int32_t* nodes, const int32_t* steps,
                                 const double* forces, int* case_id);

/*
 * Advances every case by n_steps time steps.  One step of a case (Section 3.1 and Algorithm 3's
 * per-case work on one device): Adams-Bashforth guess, data-driven correction (FEM_PRED_DD), Newmark
 * right-hand side b = f - K u + C v + M (a + 4/dt v), certified solve of A du = b, then
 * u += du, v = 2/dt du - v, a = 4/dt^2 du - 4/dt v_prev - a, and the snapshot push.
 *   iters_out   optional host [n_cases] int: CG iterations of each case summed over the n_steps.
 *   relres_out  optional host [n_cases] double: largest certified residual of each case over the steps.
 * Returns the worst per-step status (FEM_ERR_NOT_CONVERGED, FEM_ERR_BREAKDOWN) or FEM_OK.
 */
fem_status fem_step(fem_batch* b, int n_steps, int* iters_out, double* relres_out);

/*
 * fem_step without waiting for the GPU (a library service; the paper has none): queues n_steps on the
 * batch stream and returns (graph steps need no host round trip; steps that cannot run as a graph still
 * wait inside).  Statistics and status of these steps accumulate: fem_batch_sync returns their worst
 * status, and the next fem_step's iters_out / relres_out / status include them.
 */
fem_status fem_step_async(fem_batch* b, int n_steps);

/*
 * Refreshes the predictor of case `case_id` from its stored snapshots: recomputes the per-region Gram
 * matrices of the stored corrections from scratch (Section 3.2: the orthogonal decomposition of the
 * stored inputs X), replacing the incrementally updated ones.
 */
fem_status predictor_fit(fem_batch* b, int case_id);

/*
 * Writes the initial guess the predictor gives for the next step of case `case_id` (the increment
 * u_bar^{it+1} - u^it: Adams-Bashforth plus, with FEM_PRED_DD, the regional correction) into
 * x_guess_dev [n_nodes][3] device doubles.  Does not change the batch state.
 */
fem_status predictor_predict(fem_batch* b, int case_id, double* x_guess_dev);

/*
 * Coefficients of the data-driven correction of the last completed step of case `case_id` (Section 3.2: per
 * region R the prediction is y_R = Y_R c_R, c_R the least-squares coefficients of the query e^{it-1} on the
 * stored inputs X_R after the column-drop rule).  coef_host [n_regions][s_max] host doubles: entry a of a
 * region multiplies the a-th stored pair, oldest first (x_a = e^{it-1-n+a}, y_a = e^{it-n+a}); a dropped
 * column has coefficient 0; entries a >= n are 0.  n_pairs_out (nullable): n, the pairs the step used (0: no
 * correction).  With the learned proposal these are the plain predictor's coefficients.  Errors:
 * FEM_ERR_ARG; FEM_ERR_STATE for a batch without the data-driven predictor or regions, or fused meshes.
 * Synchronises the batch stream.
 */
fem_status predictor_coefficients(fem_batch* b, int case_id, double* coef_host, int* n_pairs_out);

/* Copies field `what` (FEM_FIELD_*) of case `case_id`, [n_nodes][3] doubles, to `dst` (device memory if
 * on_device != 0, else host memory; a host copy synchronises the batch stream). */
fem_status fem_case_get(fem_batch* b, int case_id, int what, double* dst, int on_device);

/*
 * Replaces, for the next fem_step only, the Ricker point force of every case by the force vectors in
 * loads [n_cases][3] (host, FP64; the load at each case's source node, i.e. the case's f^it of Section
 * 2.1, Eq. 1).  The copy to the device is ordered on the batch stream.
 */
fem_status fem_batch_set_loads(fem_batch* b, const double* loads);

/* Copies field `what` (FEM_FIELD_*) of every case to dst: the cases' [n_nodes][3] fields one after the
 * other in case order (n_nodes of each case's mesh; [n_cases][n_nodes][3] when all share one mesh).
 * Device memory if on_device != 0, else host memory (a host copy synchronises the batch stream). */
fem_status fem_batch_get_field(fem_batch* b, int what, double* dst, int on_device);

/*
 * Asynchronous form of fem_batch_get_field into host memory (a library service; the paper has none): the
 * field as it stands after the work queued so far is staged on the device (two staging buffers of the
 * field's size, allocated on first use and kept with the batch), and its copy to host_dst runs on the
 * batch's own copy stream, so it overlaps the steps queued next.  host_dst should be page-locked (else
 * the copy is not asynchronous); it is complete after fem_batch_sync, or after the next-but-one call of
 * this function (which reuses the staging buffer).  Same layout as fem_batch_get_field.
 */
fem_status fem_batch_get_field_async(fem_batch* b, int what, double* host_dst);

/* Waits until the batch stream and every asynchronous field copy have finished; returns the worst status
 * of the steps queued by fem_step_async since the last report (FEM_OK, FEM_ERR_NOT_CONVERGED, ...). */
fem_status fem_batch_sync(fem_batch* b);

/* Device-time profile of fem_step, measured with CUDA events on the batch stream. */
typedef struct {
  int steps;                         /* steps profiled */
  long long kernel_launches;         /* kernels the library launched */
  long long ebe32_launches;          /* FP32 EBE products (inner CG of FEM_FP32_INNER) */
  double ebe32_ms;
  long long ebe64_launches;          /* FP64 EBE products (FP64 CG, outer residuals, right-hand sides) */
  double ebe64_ms;
  long long cg_vec_launches;         /* CG direction + update kernels */
  double cg_vec_ms;
  double predict_ms, rhs_ms, solve_ms, update_ms;  /* phases of fem_step, summed over steps */
  long long ebe16_launches;          /* inner CG products with inner_product FEM_INNER_TC (FP16 hex matrices) */
  double ebe16_ms;
} fem_profile;

/* enable = 1: reset and start profiling (launch counts and per-class device times from CUDA events around
 * each launch; steps run eagerly); 2: reset and count launches and steps only (graph steps stay graphs);
 * 0: stop; -1: leave as is.  out (nullable) receives the totals accumulated so far. */
fem_status fem_batch_profile(fem_batch* b, int enable, fem_profile* out);

/* Statistics of the last completed step of one case. */
typedef struct {
  int steps;             /* completed steps of the case */
  int iters;             /* CG iterations of the last step (inner iterations summed in FEM_FP32_INNER) */
  int outer;             /* FP64 residual evaluations of the last step (FEM_FP32_INNER; 0 in FEM_FP64) */
  int status;            /* fem_status of the last step's solve */
  double init_relres;    /* ||b - A guess|| / ||b|| of the last step's initial guess (predictor quality) */
  double relres;         /* certified ||b - A du|| / ||b|| of the last step */
  int guess;             /* the last step's initial guess: 0 Adams-Bashforth, 1 data-driven (Adams-Bashforth plus
                            the regional correction), 2 Adams-Bashforth because the guess guard dropped the
                            correction (its residual was larger); -1 in FEM_FP64 (not tracked) */
  int fallbacks;         /* steps of the case whose correction the guess guard dropped */
} fem_case_stats_t;

fem_status fem_case_stats(fem_batch* b, int case_id, fem_case_stats_t* out);

/*
 * With opts.cpu_predictor: the balance of the heterogeneous scheme for the case set of case `case_id`:
 * s_current the pairs the next prediction uses, predict_ms the last host prediction's wall time, solve_ms the
 * last GPU step's wall time of the set, predict_total_ms / wait_total_ms the host prediction time and the time
 * the steps waited for it, summed (nullable outputs).  Errors: FEM_ERR_STATE without the scheme.
 */
fem_status fem_batch_predictor_balance(fem_batch* b, int case_id, int* s_current, double* predict_ms,
                                       double* solve_ms, double* predict_total_ms, double* wait_total_ms);

/* Number of completed steps of the batch. */
fem_status fem_batch_steps(const fem_batch* b, int* steps_out);

/* ---------------------------------------------------------------------------------------------------
 * Learned proposal: the learned form of the data-driven predictor (Section 3.2).  For every region R and
 * case, the predictor's coefficients c_R on the stored outputs Y_R (y_R = Y_R c_R) are corrected by a
 * network:  c_R + net(x_R),  x_R = [(source - centroid_R) / L, (f0 - 5) / 3, c_R in age order (newest pair
 * first), zeros] (64 inputs; L = largest edge of the mesh's bounding box).  The network is 64 -> 256 ->
 * 256 -> 32 with GELU (erf form) after the first two layers, BF16 weights and activations, FP32
 * accumulation on the tensor cores.  It is trained to the best coefficients in the same basis,
 * t_R = argmin ||Y_R c - e_R^it|| - c_R, from samples the time step itself collects.  In a step, a case
 * takes the proposal only if its initial residual is smaller than the plain guess's (PCG to the same
 * certified tolerance follows either way).
 *
 * Parameters: FP32 vector of FEM_MLP_N_PARAMS values in the order W1 [256][64], b1 [256], W2 [256][256],
 * b2 [256], W3 [32][256], b3 [32]; layer l computes z = W_l a + b_l.  Gradients use the same layout.
 * --------------------------------------------------------------------------------------------------- */
#define FEM_MLP_N_PARAMS 90656
#define FEM_MLP_IN 64
#define FEM_MLP_OUT 32
#define FEM_MLP_RES 560     /* values of one residual-space sample: 528 (upper triangle of W) + 32 (w) */
typedef struct fem_mlp fem_mlp;

/* Creates a network from host parameters (copied) on the current device; Adam moments start at zero.
 * `stream` orders the network's own calls (forward, gradient, training). */
fem_status fem_mlp_create(const float* params, void* stream, fem_mlp** out);
fem_status fem_mlp_destroy(fem_mlp* net);
/* Current FP32 master parameters -> host [FEM_MLP_N_PARAMS] (synchronises the network's stream). */
fem_status fem_mlp_get_params(fem_mlp* net, float* params);
/* out_dev [B][32] = net(x_dev [B][64]) (device buffers, FP32; inputs rounded to BF16 inside). */
fem_status fem_mlp_forward(fem_mlp* net, const float* x_dev, int64_t B, float* out_dev);
/* Mean squared error of net(x) against t over the B x 32 outputs and its gradient (grad_dev
 * [FEM_MLP_N_PARAMS] device FP32, may be NULL); the loss goes to *loss_out (host).  Synchronises. */
fem_status fem_mlp_loss_grad(fem_mlp* net, const float* x_dev, const float* t_dev, int64_t B, float* grad_dev,
                             double* loss_out);
/* n_updates Adam steps (lr, beta = 0.9 / 0.999, eps = 1e-8, bias-corrected) on minibatches of `batch` rows
 * of (x_dev [n_samples][64], t_dev [n_samples][32]); order_dev [n_updates][batch] (device int32) lists the
 * sample rows of each minibatch (the caller draws the shuffling).  loss_out: host [n_updates] losses before
 * each update, or NULL.  A row index outside [0, n_samples) returns FEM_ERR_ARG (that row counts as zero). */
fem_status fem_mlp_train(fem_mlp* net, const float* x_dev, const float* t_dev, int64_t n_samples,
                         const int32_t* order_dev, int n_updates, int batch, double lr, double* loss_out);

/*
 * The same with the residual-space loss, the error measure the proposal's acceptance decides on: the relative
 * error of a case's corrected guess, sum over regions R of ||Y_R (c_R + d_R) - e_R||^2 / ||e||^2 (e the case's
 * correction over all regions), d_R = net(x_R) in age order; each region's share is one sample.  Y_R's Gram is
 * factored R^T R (in age order, with the predictor's column-drop rule), so that the share is ||W d - w||^2 plus
 * a part d cannot change, W = R / ||e||, w = (R^{-T} Y_R^T e_R - R c_R) / ||e||.  A sample s_dev row holds
 * FEM_MLP_RES floats: the upper triangle of W row by row (W_ij, i <= j), then w.  Loss = mean over the samples
 * of ||W d - w||^2; otherwise as fem_mlp_loss_grad / fem_mlp_train.
 */
fem_status fem_mlp_loss_grad_residual(fem_mlp* net, const float* x_dev, const float* s_dev, int64_t B,
                                      float* grad_dev, double* loss_out);
fem_status fem_mlp_train_residual(fem_mlp* net, const float* x_dev, const float* s_dev, int64_t n_samples,
                                  const int32_t* order_dev, int n_updates, int batch, double lr, double* loss_out);

/* Uses `net` (NULL: none) for the learned proposal in the batch's next steps.  Needs FEM_FP32_INNER, the
 * data-driven predictor, regions and groups of one mesh (no fuse_meshes).  The caller keeps ownership and
 * must not train the network while the batch steps. */
fem_status fem_batch_set_mlp(fem_batch* b, fem_mlp* net);
/* Starts collecting training samples into caller-owned device buffers x_dev [capacity][64] and t_dev
 * [capacity][32] (NULL x_dev stops).  Every following step that made a data-driven prediction appends
 * n_regions x n_cases rows (region-major, then case) while they fit.  Same requirements as
 * fem_batch_set_mlp. */
fem_status fem_batch_collect(fem_batch* b, float* x_dev, float* t_dev, int64_t capacity);
/* As fem_batch_collect, but each sample's training data is the residual-space form (W, w) of
 * fem_mlp_train_residual: s_dev [capacity][FEM_MLP_RES], computed from the stored-snapshot Gram after the
 * step's correction e^it is pushed.  A region whose e_R is zero gives a zero sample. */
fem_status fem_batch_collect_residual(fem_batch* b, float* x_dev, float* s_dev, int64_t capacity);
/* Rows collected so far; *full = 1 if a step's rows no longer fit. */
fem_status fem_batch_collected(fem_batch* b, int64_t* rows, int* full);
/* Case-steps in which the learned proposal was taken / rejected (initial residual not smaller). */
fem_status fem_batch_proposal_counts(fem_batch* b, long long* taken, long long* rejected);

/* Message of the last error on this thread ("" if none). */
const char* fem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FEM_H_ */
