/* hn.h -- C ABI of the GB300 multigrid Poisson solver (HONEI paper, arXiv 0904.4152).
 *
 * The library solves the Q1 (bilinear, conforming) finite-element discretisation of
 *     -div(a grad u) = f   on the unit square, zero Dirichlet boundary on all or some
 *                          sides and free Neumann on the others          (Sec. 2.1, 6.2)
 * on a regular grid of refinement level L, i.e. n = 2^L + 1 nodes per side and N = n^2 unknowns
 * numbered in tensor-product order, node i = iy*n + ix with ix fastest (Sec. 2.1).  The matrix is
 * assembled fully into 9 bands at fixed positions (Sec. 2.1, Sec. 4.1) and solved by a geometric
 * multigrid V cycle with damped Jacobi pre/post smoothing and an exact or CG coarse solve,
 * optionally as the single-precision preconditioner of an FP64 defect-correction loop (Sec. 6.2),
 * or as the preconditioner of FP64 conjugate gradients (a solver plugged into another, Sec. 4.1).
 * Everything
 * runs on one GB300 GPU (sm_103a); data crosses the host-device boundary only at these calls.
 *
 * Conventions shared by every call:
 *  - Every function returning hn_status returns HN_OK (0) on success and never exits or aborts,
 *    also not when device memory runs out (Sec. 4.2 asks the same of an out-of-memory request).  hn_last_error()
 *    returns a message for the calling thread's last failure.
 *  - Explicit copy (Sec. 4.1): the library copies every input at call time and never keeps or
 *    aliases a caller pointer; outputs are written into caller buffers.  Handles are opaque and
 *    owned by the caller until passed to the matching *_destroy.
 *  - Vectors have length N over all (2^L+1)^2 nodes including the boundary.  Right-hand-side
 *    entries on Dirichlet nodes must be 0 (HN_ERR_ARG otherwise); solutions are 0 there.  Nodes
 *    on free Neumann sides (hn_band_create_bc) are unknowns like interior nodes.
 *  - Band layout: 9 bands, k = 0..8 <-> neighbour offset (dy, dx) = (k/3 - 1, k%3 - 1), band-major
 *    (band k occupies elements [k*N, (k+1)*N)), band_k[i] = A[i, i + dy*n + dx].  An entry is exactly
 *    0.0 where the neighbour is off the grid or either node lies on the Dirichlet boundary; boundary
 *    rows are identity rows (diagonal 1.0).
 *  - Thread safety: a handle is used by one thread at a time; different handles may be used from
 *    different threads.  hn_mg_solve_batch requires distinct handles.  The server is internally
 *    synchronised.
 */
#ifndef HN_H
#define HN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HN_OK = 0,
  HN_ERR_ARG = 1,            /* invalid argument (null pointer, level out of range, bad option) */
  HN_ERR_OOM = 2,            /* device or host allocation failed */
  HN_ERR_BUDGET = 3,         /* request exceeds the server's device-memory budget */
  HN_ERR_CUDA = 4,           /* a CUDA runtime call failed (message in hn_last_error) */
  HN_ERR_NOT_CONVERGED = 5,  /* cycle / outer-iteration cap reached before the tolerance */
  HN_ERR_NONFINITE = 6,      /* a norm became NaN or infinite (e.g. non-finite right-hand side) */
  HN_PENDING = 7,            /* server request accepted but not finished */
  HN_ERR_TIMEOUT = 8,        /* poll deadline passed */
  HN_ERR_STATE = 9           /* call not valid in the handle's current state */
} hn_status;

/* Precision of the solve (Sec. 6.2).  FP64: FP64 V cycles to the tolerance.  FP32_DC: FP64 defect
 * correction (defect b - A x, update and convergence norm in FP64 on the GPU) preconditioned by
 * FP32 V cycles (FP32 bands and vectors).  FP16BAND_DC: the same with the inner bands stored in
 * FP16 with one FP32 scale per band and level (FP32 arithmetic and vectors). */
typedef enum { HN_PREC_FP64 = 0, HN_PREC_FP32_DC = 1, HN_PREC_FP16BAND_DC = 2 } hn_precision;

/* Outer solver.  MG: V cycles to the tolerance (FP64), or the defect correction of the DC
 * precisions.  PCG: conjugate gradients in FP64 (x, residual, search direction, inner products
 * and convergence test in FP64 on the GPU), each step preconditioned by one V cycle from zero on
 * the current residual (Sec. 4.1: a solver plugged into another as its preconditioner), the cycle
 * in the hierarchy's precision (FP64, FP32, or FP32 with FP16 band storage; the residual is scaled
 * by 1 / ||previous residual|| before the cast).  PCG needs pre == post (a symmetric
 * preconditioner).  Convergence: recursively updated ||r|| / ||b|| <= tol. */
typedef enum { HN_SOLVER_MG = 0, HN_SOLVER_PCG = 1 } hn_solver;

/* Coarsest-level solver (Sec. 6.2 uses unpreconditioned CG).  EXACT: precomputed FP64 inverse of
 * the coarse operator on its unknowns.  CG: unpreconditioned conjugate gradients in FP64 from
 * x = 0 on the coarse unknowns, stopped at ||r|| <= 1e-13 ||b|| or after 2m + 10 steps for m
 * unknowns. */
typedef enum { HN_COARSE_EXACT = 0, HN_COARSE_CG = 1 } hn_coarse_solver;

typedef struct hn_band hn_band;      /* an assembled fine-level operator (device resident) */
typedef struct hn_mg hn_mg;          /* a multigrid hierarchy built from an hn_band (device) */
typedef struct hn_server hn_server;  /* continuous-batching solve server */

#define HN_MIN_LEVEL 2
#define HN_MAX_LEVEL 14

/* Boundary conditions per side of the square: a side in the mask is zero Dirichlet (its nodes
 * are eliminated), a side not in it is free Neumann (zero flux; its nodes are unknowns with the
 * rows of their 1 or 2 cells, the natural boundary condition).  The paper's accuracy test uses
 * Dirichlet on all sides (Sec. 6.2.1), its performance test mixes free Neumann and Dirichlet
 * sides (Sec. 6.2.2).  A corner is Dirichlet if either of its sides is. */
#define HN_DIRICHLET_BOTTOM 1u   /* y = 0 */
#define HN_DIRICHLET_RIGHT 2u    /* x = 1 */
#define HN_DIRICHLET_TOP 4u      /* y = 1 */
#define HN_DIRICHLET_LEFT 8u     /* x = 0 */
#define HN_DIRICHLET_ALL 15u

/* Assemble the Q1 stiffness matrix of -div(a grad u) at level L (HN_MIN_LEVEL..HN_MAX_LEVEL) on
 * the GPU (Sec. 2.1: full assembly, fixed band positions).  cell_coef: host array of (2^L)^2
 * per-cell coefficients a > 0, row-major by cell (ey, ex), cell (ex, ey) = [ex h, (ex+1) h] x
 * [ey h, (ey+1) h]; NULL means a = 1.  dirichlet_sides: a nonzero mask of HN_DIRICHLET_* sides
 * (at least one, so that the operator is definite).  Dirichlet nodes are eliminated symmetrically
 * (rows and columns zeroed, diagonal 1).  *out receives a new handle.  Errors: HN_ERR_ARG (L out
 * of range, out NULL, a coefficient not finite or <= 0, a mask outside 1..15), HN_ERR_OOM,
 * HN_ERR_CUDA. */
hn_status hn_band_create_bc(int L, const double* cell_coef, unsigned dirichlet_sides, hn_band** out);

/* hn_band_create_bc with all four sides Dirichlet. */
hn_status hn_band_create(int L, const double* cell_coef, hn_band** out);

/* Copy the 9 assembled FP64 bands to host memory: bands_out holds 9*N doubles in the band layout
 * above.  Errors: HN_ERR_ARG, HN_ERR_CUDA. */
hn_status hn_band_get(const hn_band* A, double* bands_out);

/* Level L and node count N of an operator (0 for a NULL handle). */
int hn_band_level(const hn_band* A);
long long hn_band_nodes(const hn_band* A);

void hn_band_destroy(hn_band* A);

typedef struct {
  int coarse_L;      /* coarsest level (2), solved by coarse_solver */
  int pre, post;     /* damped Jacobi steps before / after the coarse correction (2, 2).  pre >= 1,
                        pre + post even */
  int max_cycles;    /* cap on V cycles (FP64) or inner cycles in total (DC) (100) */
  int max_outer;     /* cap on defect-correction updates, or on PCG steps (50) */
  int inner_max;     /* cap on inner V cycles per defect-correction step (10) */
  double omega;      /* Jacobi damping (0.7) */
  double tol;        /* stop when ||b - A x||_2 / ||b||_2 <= tol, FP64 operator (1e-8) */
  double inner_tol;  /* inner cycles stop at relative inner residual <= inner_tol (1e-2) */
  hn_precision prec; /* HN_PREC_FP64 */
  void* stream;      /* cudaStream_t the solves run on; NULL = the library's own stream */
  unsigned dirichlet_sides;  /* boundary of the operators hn_mg_submit assembles
                                (HN_DIRICHLET_ALL); hn_mg_setup takes it from its operator */
  hn_solver solver;  /* HN_SOLVER_MG */
  hn_coarse_solver coarse_solver;  /* HN_COARSE_EXACT */
} hn_mg_opts;

typedef struct {
  int cycles;        /* V cycles run (inner cycles in DC modes; preconditioner cycles in PCG) */
  int outer_iters;   /* defect-correction updates applied (0 in FP64 MG mode); PCG steps */
  int inner_cycles;  /* inner V cycles (0 in FP64 mode) */
  int status;        /* hn_status of this solve */
  double relres;     /* final ||b - A x|| / ||b|| with the FP64 operator, FP64 arithmetic */
  long long setup_ns;/* time spent in hn_mg_setup for this hierarchy */
  long long solve_ns;/* wall time of the solve call (host clock, includes copies) */
} hn_mg_stats;

void hn_mg_opts_default(hn_mg_opts* opts);

/* Build the multigrid hierarchy of A on the device: coarse operators by re-discretisation with the
 * coarse cell coefficient equal to the mean of its 4 child cells, inner-precision copies of the
 * bands (FP32 cast, or FP16 codes with per-band scales), the coarse-level solver (the inverse, or
 * the dense coarse matrix for CG), and all work vectors (PCG: also FP64 residual, search
 * direction and its image).  A may be destroyed afterwards (its data are copied).  Errors: HN_ERR_ARG (bad
 * options, A NULL, coarse_L > level of A), HN_ERR_OOM, HN_ERR_CUDA. */
hn_status hn_mg_setup(const hn_band* A, const hn_mg_opts* opts, hn_mg** out);

/* Solve A x = b to the tolerance (Sec. 6.2).  b: N doubles.  x: N doubles; on entry the initial
 * guess (ignored and taken as 0 if x_is_guess is 0), on exit the solution.  device_ptrs = 1: b and
 * x are device pointers (16-byte aligned); 0: host pointers.  stats may be NULL.  Returns HN_OK,
 * HN_ERR_NOT_CONVERGED (x holds the last iterate), HN_ERR_NONFINITE, HN_ERR_ARG, HN_ERR_CUDA. */
hn_status hn_mg_solve(hn_mg* mg, const double* b, double* x, int x_is_guess, int device_ptrs,
                      hn_mg_stats* stats);

/* Solve count independent systems together: one launch per V-cycle phase covers every problem
 * (persistent kernels over a device work list), the per-iteration launch sequence is a CUDA
 * graph, and each problem stops on its own.  All handles must share precision, pre, post, omega,
 * coarse_L, solver and coarse solver, and may differ in level, coefficients and boundary.  b[j], x[j] as in hn_mg_solve (x zero guess).
 * stats: count entries or NULL.  Each problem's result is bit-identical to solving it alone.
 * Returns the first non-OK per-problem status, HN_OK if all converged. */
hn_status hn_mg_solve_batch(hn_mg* const* mgs, int count, const double* const* b,
                            double* const* x, int device_ptrs, hn_mg_stats* stats);

/* Device bytes held by a hierarchy (bands, vectors, scratch). */
size_t hn_mg_device_bytes(const hn_mg* mg);

void hn_mg_destroy(hn_mg* mg);

/* ---------------------------------------------------------------- single-kernel entry points
 * Run one kernel of the solver on one level of a hierarchy, for testing and measurement.  Vectors
 * are host arrays of N_l elements of the level's storage type: double for the FP64 hierarchy and
 * for the FP64 fine level of a DC hierarchy (inner = 0), float for the inner levels of a DC
 * hierarchy (inner = 1).  level is the refinement level l (coarse_L..L).
 *   HN_OP_SPMV        out = A_l in1
 *   HN_OP_DEFECT      out = in2 - A_l in1; *norm_out = ||out||_2 (FP64 accumulation)
 *   HN_OP_JACOBI      out = in1 + omega D^-1 (in2 - A_l in1)     (in1 = x, in2 = rhs)
 *   HN_OP_JACOBI_ZERO out = omega D^-1 in2                         (the step from x = 0)
 *   HN_OP_RESTRICT    out (level l-1) = R in1 (level l), R = P^T full weighting
 *   HN_OP_PROLONG_ADD out (level l) = in2 (level l) + P in1 (level l-1), bilinear
 *   HN_OP_COARSE      out = A_c^-1 in2 (level = coarse_L; by the hierarchy's coarse solver)
 * Errors: HN_ERR_ARG, HN_ERR_STATE (op not available for that precision/level), HN_ERR_CUDA. */
typedef enum {
  HN_OP_SPMV = 0, HN_OP_DEFECT = 1, HN_OP_JACOBI = 2, HN_OP_JACOBI_ZERO = 3,
  HN_OP_RESTRICT = 4, HN_OP_PROLONG_ADD = 5, HN_OP_COARSE = 6,
  HN_OP_PROLONG_JACOBI = 7   /* prolongation fused into a Jacobi step: hn_mg_time_kernel only */
} hn_op;
hn_status hn_mg_apply(hn_mg* mg, hn_op op, int level, int inner, const void* in1,
                      const void* in2, void* out, double* norm_out);

/* Allocation-free defect and norm (the paper has no counterpart; a service for callers that cannot
 * allocate device memory at the time of the call: code running while another thread captures a
 * CUDA graph in global mode, where cudaMalloc is not permitted; processes that hand out their
 * whole device-memory plan up front; latency-critical paths where cudaMalloc / cudaFree would
 * synchronize the device).  Computes r = b - A x and ||r||_2 for an operator from hn_band_create.
 * x, b, r: device pointers to N doubles, 16-byte aligned, caller-owned; r must not overlap x or b
 * (it is written while other threads still read their stencil neighbourhoods); norm: device
 * pointer to one double.  The operator's device must be the current device.  Runs on stream
 * (cudaStream_t, NULL = the legacy default stream) and returns without waiting; a caller that
 * launches while another thread captures a graph in global mode must pass a stream created with
 * cudaStreamNonBlocking, since the legacy default stream synchronizes with every blocking stream.
 * The only temporary (one partial sum per 128-node tile) is a fixed device array inside the library
 * (512 KiB, held by every GPU that loads the library until exit), so at most 8,388,608 nodes
 * (level 11) are accepted; larger operators get HN_ERR_ARG.  The call allocates nothing.  The first
 * call on a device looks up that array's address and should come before any stream capture.  All
 * calls share the array: calls that overlap on the GPU (e.g. on two streams) race and must be
 * ordered by the caller.  Errors: HN_ERR_ARG (null or misaligned pointer, r overlapping x or b,
 * the operator on another device, too many nodes), HN_ERR_CUDA. */
hn_status hn_band_defect_norm_static(const hn_band* A, const double* x, const double* b, double* r,
                                     double* norm, void* stream);

/* Copy the inner-precision bands of one level to the host: FP32 values (9*N_l floats) for an
 * FP32_DC hierarchy, or FP16 codes (9*N_l uint16) plus the 9 FP32 scales for FP16BAND_DC. */
hn_status hn_mg_get_inner_bands(const hn_mg* mg, int level, void* bands_out, float* scales_out);

/* -------------------------------------------------------------------------------- serving
 * A server owns two lanes (requests of levels below 10, and of levels 10 and up), each with a
 * worker thread, a FIFO queue and its own stream (the small requests' lane at the greatest stream
 * priority), two builder threads and a device-memory budget.  A request is admitted once a slot
 * (max_active, shared by the lanes) and budget room for its hierarchy are free; requests of one
 * lane are admitted in submission order, the lanes independently (under a budget too tight for
 * both, a large request waiting for memory can be overtaken by small ones).  Admitted requests
 * of a lane are solved together: every scheduler iteration of a lane runs one V-cycle phase
 * sequence over its active requests (continuous batching), beside the other lane's iterations;
 * finished requests leave, free their memory and let queued requests in.  All requests of a server share precision, pre, post, omega,
 * coarse_L, solver and coarse solver (taken from the first submit; HN_ERR_ARG for a request that
 * differs). */
hn_status hn_server_create(size_t budget_bytes, int max_active, hn_server** out);

/* Queue a solve of level L with cell coefficients (NULL = 1) and right-hand side b (host, N
 * doubles); both are copied (into page-locked buffers the server recycles).  *ticket identifies
 * the request.  HN_ERR_BUDGET if the request alone exceeds the budget; HN_ERR_ARG on bad input,
 * coefficients included (checked here, in the caller's thread, as hn_band_create_bc checks them);
 * HN_ERR_OOM if no page-locked host memory is left. */
hn_status hn_mg_submit(hn_server* srv, int L, const double* cell_coef, const double* b,
                       const hn_mg_opts* opts, unsigned long long* ticket);

/* Wait up to timeout_ns (0 = do not wait, < 0 = wait forever) for a request.  HN_PENDING if not
 * finished (timeout_ns == 0), HN_ERR_TIMEOUT if the deadline passed; otherwise the request's final
 * status, with x_out (host, N doubles, may be NULL) and stats filled and the request forgotten. */
hn_status hn_mg_poll(hn_server* srv, unsigned long long ticket, long long timeout_ns,
                     double* x_out, hn_mg_stats* stats);

typedef struct {
  long long submitted, completed, active, queued;
  long long iterations;        /* scheduler iterations run (both lanes) */
  size_t bytes_in_use, budget;
  /* time (ns) the builder threads spent building the hierarchies of admitted requests (on their
   * own streams, while the workers iterate the running requests), and the workers' time (summed
   * over the lanes, which run at the same time) spent waiting for iterations to finish, retiring
   * requests (their results come back on a copy stream while the next iteration runs), and
   * (re)building the schedule and starting requests */
  long long admit_ns, schedule_ns, iterate_ns, retire_ns;
} hn_server_info;
hn_status hn_server_query(hn_server* srv, hn_server_info* info);

/* Stop the workers after finishing active requests; queued requests are dropped. */
void hn_server_destroy(hn_server* srv);

/* Message describing the calling thread's last error ("" if none). */
const char* hn_last_error(void);

/* Library version string. */
const char* hn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HN_H */
