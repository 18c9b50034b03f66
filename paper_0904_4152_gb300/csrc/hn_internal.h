// Internal declarations of the hn library: device-side descriptors, the per-problem solver state
// machine, and the kernel launch wrappers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/hn.h"

namespace hn {

// ------------------------------------------------------------------------------ geometry
// A warp-tile is 128 consecutive nodes of the flat (padded) index range; each lane owns 4.
constexpr int kTile = 128;
constexpr int kLaneNodes = 4;
constexpr int kMaxLevel = HN_MAX_LEVEL;
constexpr int kMaxCoarse = 4;                       // coarse_L <= 4: at most 225 interior unknowns
constexpr int kMaxCoarseM = 289;   // unknowns of the coarsest level (17 x 17 at level 4)
constexpr int kSumGroup = 16384;   // tiles per group of a problem's norm partial sum

__host__ __device__ inline long long n_of_dev(int L) { return (1LL << L) + 1; }
inline long long n_of(int L) { return (1LL << L) + 1; }
inline long long N_of(int L) { return n_of(L) * n_of(L); }
inline long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }
// padded length of a level: multiple of the tile, and every row/tile index is in range
inline long long pitch_of(int L) { return round_up(N_of(L), kTile); }
// zero halo in front of / behind every vector, covers the +-(n+1) stencil reach of the padded
// range (multiple of 32 elements keeps every vector 256-byte aligned)
inline long long halo_of(int L) { return round_up(n_of(L) + 8, 32); }

enum Prec { P64 = 0, P32 = 1, P16 = 2 };
enum Solver { SOLVER_MG = 0, SOLVER_PCG = 1 };

// unpreconditioned CG on the coarsest level: stop at ||r|| <= kCoarseCgTol ||b|| or after
// coarse_cg_steps(m) steps (m unknowns)
constexpr double kCoarseCgTol = 1e-13;
__host__ __device__ inline int coarse_cg_steps(int m) { return 2 * m + 10; }

// ------------------------------------------------------------------- device descriptors
// One level of one problem.  Vectors and bands point at element 0 of pitch elements; a zero halo
// of halo_of(L) elements sits on either side of every array, so stencil windows of any padded row
// stay inside the allocation.
struct LevelDev {
  const void* band[9];   // double (FP64 hierarchy), float (FP32), __half (FP16 codes)
  const double* wdinv;   // FP64 hierarchy only: omega / diag, pitch doubles
  const float* wdf;      // FP32 / FP16 hierarchies: omega / diag in FP32, rounded as the band
                         // kernels round it (FP16: diag of the row-sum form), pitch floats
  void* x[2];            // iterate and its Jacobi ping-pong partner (double or float)
  void* rhs;             // right-hand side of this level (restricted defect, or the top rhs)
  void* r;               // defect of this level
  float scale[9];        // FP16 band scales
  int L, n, pitch;
  int bc;                // Dirichlet sides (HN_DIRICHLET_*), the same on every level
};

// node classes under the boundary mask bc: Dirichlet nodes are eliminated, all others (interior
// and free-Neumann boundary nodes) are unknowns
__host__ __device__ inline bool is_dirichlet(long long ix, long long iy, long long n, int bc) {
  return (iy == 0 && (bc & 1)) || (ix == n - 1 && (bc & 2)) || (iy == n - 1 && (bc & 4)) ||
         (ix == 0 && (bc & 8));
}
// the unknowns of a level form the rectangle of nodes x0..x0+nx-1, y0..y0+ny-1 (row-major)
struct UnknownRect { int x0, y0, nx, ny; };
__host__ __device__ inline UnknownRect unknown_rect(int n, int bc) {
  UnknownRect r;
  r.x0 = (bc & 8) ? 1 : 0;
  r.y0 = (bc & 1) ? 1 : 0;
  r.nx = ((bc & 2) ? n - 2 : n - 1) - r.x0 + 1;
  r.ny = ((bc & 4) ? n - 2 : n - 1) - r.y0 + 1;
  return r;
}

struct ProblemDev {
  int L;                 // finest level
  int coarse;            // coarsest level
  int m;                 // interior unknowns of the coarsest level
  int pad0;
  const double* cinv;    // m*m inverse of the coarsest block on its unknowns, row-major (for the
                         // CG coarse solver: the block itself)
  // FP64 fine-level data of the outer loop (x64, b64 alias the top level in FP64 MG mode)
  const double* band64[9];
  double* x64;           // solution
  double* b64;           // right-hand side
  double* r64;           // PCG: residual, search direction and its image A p (with zero halos)
  double* p64;
  double* q64;
  LevelDev lev[kMaxLevel + 1];   // indexed by level l in [coarse, L]
};

// per-problem state machine of a solve (device)
enum Phase {
  PH_DONE = 0,    // finished (status holds the outcome)
  PH_OUTER = 1,   // defect correction: needs the FP64 outer defect
  PH_INNER = 2,   // defect correction: running inner V cycles
  PH_UPDATE = 3,  // defect correction: inner solve finished, apply x += c / s
  PH_CYCLE = 4,   // FP64 multigrid: run a V cycle, then check
  PH_CHECK = 5,   // FP64 multigrid: check the initial guess before cycling
  PH_INIT = 6,    // starting: boundary check and ||b||
  PH_PRECOND = 7  // PCG: the preconditioner's V cycle on the scaled residual
};
// PCG uses PH_OUTER for its step (q = A p, alpha, x and r update, check; the initial residual
// when no cycle ran yet) and PH_UPDATE for the new direction (beta, p = z + beta p).

struct ProbState {
  int phase;             // Phase
  int status;            // hn_status once done; HN_PENDING while running
  int cycles, outer_iters, inner_cycles, inner_k;
  int zero_top;          // the top-level iterate is zero (first sweep skips reading it)
  int x_zero;            // the FP64 solution is still zero (outer defect = b)
  double bnorm;          // ||b||
  double dnorm;          // ||b - A x|| at the last outer defect / FP64 check
  double relres;         // dnorm / bnorm
  double s;              // scale applied to the defect before the cast to the inner precision
  double inv_s;          // 1 / s, formed once when s changes (an FP64 division per thread of a
                         // streaming kernel would cost more than the kernel's memory traffic)
  double inner_ref;      // ||scaled defect|| (reference of the inner relative residual)
  double inner_res;      // last inner residual norm
  double rho;            // PCG: (r, z) of the current direction
  double alpha;          // PCG: step length of the current step
  double beta;           // PCG: (r_new, z_new) / (r, z)
};

// solver parameters shared by every problem of an engine
// IF nodes of the device-side solve loop (closed-world graph only).  One iteration of the loop
// runs [IF outer: outer defect, control] [top-level first smoothing step, check] [IF cycle: rest
// of the V cycle] [IF update: update, control] summary.  The kernel that takes a phase decision
// sets the matching value (and its mirror in `taken`); the summary counts the launches the
// iteration ran and resets the values for the next one.
struct CondDev {
  unsigned long long h_cycle = 0, h_outer = 0, h_update = 0;   // cudaGraphConditionalHandle
  unsigned* taken = nullptr;              // [0] cycle, [1] outer, [2] update
  unsigned long long* launches = nullptr; // kernels launched by the loop's iterations
  unsigned n_base = 0, n_cycle = 0, n_outer = 0, n_update = 0;
  unsigned mask = 0;                      // handles that exist: bit w for taken[w]
};

struct Params {
  int prec, pre, post, coarse;
  int max_cycles, max_outer, inner_max, solver;
  int coarse_cg, pad;
  double omega, tol, inner_tol;
  CondDev cond;
};

// tile work list of one level: items[g] = (problem, tile of that problem's level).  The count is
// read from device memory so that a captured graph stays valid when the list is rewritten.
struct TileList {
  const int2* items;
  const int* count;
  // the same tiles grouped in chunks of up to kChunkTiles consecutive tiles of one problem,
  // items (problem, first tile, tiles, 0); used by the kernels that stage bands in shared memory
  const int4* chunks = nullptr;
  const int* chunk_count = nullptr;
  int chunk_cap = 0;        // host side: capacity of the chunk list
  // an engine of one problem also passes that problem's descriptors by value, so its kernels
  // start on the data without first loading the work list and the descriptor: solo_tiles > 0
  // tiles of level solo_d.L (solo_c: the next coarser level, solo_f: the next finer one), the
  // problem's finest level solo_L, problem slot 0
  int solo_tiles = 0;
  int solo_L = 0;
  LevelDev solo_d{}, solo_c{}, solo_f{};
};
constexpr int kChunkTiles = 8;

// ------------------------------------------------------------------------ launch wrappers
// setup kernels (k_setup.cu); band pointer sets are passed by value
struct BandPtrs64 { double* p[9]; };
struct BandPtrs64c { const double* p[9]; };
struct BandPtrs32 { float* p[9]; };
struct BandPtrs16 { __half* p[9]; };
// omega / diag of an FP32 or FP16 level into wdf (pitch floats)
cudaError_t launch_wdf(int L, int prec, const void* const* band, const float* scale, double omega,
                       float* wdf, cudaStream_t s);
cudaError_t launch_assemble(int L, const double* coef, const BandPtrs64& band, double* wdinv,
                            double omega, int bc, cudaStream_t s);
cudaError_t launch_coarsen_coef(int Lf, const double* af, double* ac, cudaStream_t s);
cudaError_t launch_band_to_f32(int L, const BandPtrs64c& src, const BandPtrs32& dst,
                               cudaStream_t s);
cudaError_t launch_band_to_f16(int L, const BandPtrs64c& src, unsigned long long* absmax9,
                               const BandPtrs16& dst, float* scales_dev, cudaStream_t s);

// solver kernels (k_cycle.cu).  All take the engine's device arrays.
struct EngineDev {
  const ProblemDev* P;   // problems
  ProbState* S;          // states
  const int* fine_off;   // first partial slot of each problem (fine-level tile list order)
  double* partial;       // one slot per fine-level tile
  double* partial2;      // second set (||b|| at start)
  int nprob;
  int pad;
  Params prm;
  unsigned int* active_host;   // mapped host word: problems not done after the iteration
  unsigned int* iter;          // iterations since the solve started (device)
  unsigned int iter_limit;     // beyond it every running problem stops as not converged
  int pdl;                     // launch with programmatic dependent launch (host-side flag)
  int* err;                    // device word: nonzero after a bounded wait gave up
  int staged;                  // host-side flag: large FP32/FP16 levels use the bulk-copy kernels
  int dsm;                     // host-side flag: the fused tail keeps its cluster levels in
                               // distributed shared memory when they fit
  int ctl_groups;              // blocks per problem of the control kernel (groups of the largest
                               // problem's norm partial sum)
  double* gsum;                // [nprob * ctl_groups] group sums of the control kernel
  unsigned* gticket;           // [nprob] blocks of a problem's control launch that finished
  unsigned* ticket;            // blocks of a first smoothing step with a fused check that finished
  unsigned long long* gbar;    // [3] grid barriers of the persistent kernels: arrivals of the
                               // down kernel, of the up kernel, barrier actions completed
};

// Launch wrappers for one step of the schedule; grid = CTAs of 256 threads.  level < 0 means
// "each problem's own finest level" (used with the fine work list).
// fuse_check (an engine of one problem whose norm is one group of partials, the first step of its
// finest level): the step also takes the lagged check, in place of a control launch
cudaError_t launch_jacobi(const EngineDev& E, TileList tl, int level, int want, int in_sel,
                          int first, int grid, cudaStream_t s, int fuse_check = 0);
cudaError_t launch_defect(const EngineDev& E, TileList tl, int level, int want, int in_sel,
                          int grid, cudaStream_t s);
cudaError_t launch_spmv(const EngineDev& E, TileList tl, int level, int want, int in_sel, int grid,
                        cudaStream_t s);
cudaError_t launch_check(const EngineDev& E, TileList fine, int want, int x_sel, int grid,
                         cudaStream_t s);
// first two smoothing steps: fused from a zero iterate (PRE12 alone), else step 1 (PRE12) and
// step 2 (PRE2B); pre_fuses(prec) tells whether the zero-iterate fusion exists for a precision
cudaError_t launch_pre12(const EngineDev& E, TileList tl, int level, int want, int grid,
                         cudaStream_t s, int fuse_check = 0);
cudaError_t launch_pre2b(const EngineDev& E, TileList tl, int level, int want, int grid,
                         cudaStream_t s);
bool pre_fuses(int prec);
// the V cycle on levels coarse..min(T, L) of every problem in phase `want`, one thread-block
// cluster of `cluster` blocks per problem slot
cudaError_t launch_tail(const EngineDev& E, int T, int want, int cluster, cudaStream_t s);
// one-time kernel attributes (cluster-size opt-in); call outside stream capture
cudaError_t prepare_kernels();

// the levels T+1..M of the V cycle in one cooperative launch each way (down: smoothing, defect,
// restriction and the lagged checks of problems whose finest level is there; up: prolongation
// and smoothing); lists: device copy of the engine's per-level tile lists
cudaError_t launch_mid(const EngineDev& E, const TileList* lists, int M, int T, int want, int up,
                       cudaStream_t s);

cudaError_t launch_restrict(const EngineDev& E, TileList tl_coarse, int fine_level, int want,
                            int grid, cudaStream_t s);
// Fused level sweeps of an engine of one problem (V(2,2) cycles): tiles of cx x cy coarse nodes,
// tx x ty of them over the coarse grid of the level, tile-local pitch P = 2 cx + 7 and R = 2 cy + 7
// rows in shared memory.  sweep_geom gives the tiles of level `level`, sweep_smem_bytes their
// shared memory.  launch_sweep_down: top = 1 on the problem's own finest level (after its first
// smoothing step), 0 on a level whose iterate starts at zero; launch_sweep_up: e_sel = the buffer
// of the coarse iterate (its result goes to buffer 1).
struct SweepGeom { int cx, cy, tx, ty, P, R; };
SweepGeom sweep_geom(int level);
size_t sweep_smem_bytes(int prec, const SweepGeom& g);
cudaError_t launch_sweep_down(const EngineDev& E, TileList tl, int level, int want, int top, cudaStream_t s);
cudaError_t launch_sweep_up(const EngineDev& E, TileList tl, int level, int want, int e_sel, cudaStream_t s);
// x_sel: bit 0 the fine buffer corrected in place, bit 1 the buffer of the coarse iterate
cudaError_t launch_prolong(const EngineDev& E, TileList tl, int level, int want, int x_sel,
                           int grid, cudaStream_t s);
// the prolongation into x[s] fused into the first post-smoothing step (result in x[1 - s]); s = bit 0
// of x_sel, bit 1 the buffer of the coarse iterate
cudaError_t launch_prolong_jacobi(const EngineDev& E, TileList tl, int level, int want, int x_sel,
                                  int grid, cudaStream_t s);
cudaError_t launch_coarse(const EngineDev& E, TileList tl, int want, int grid, cudaStream_t s);
// fuse: an engine of one problem whose fine norm is one group of partials takes the outer control
// step in the last block of the outer defect, and the control step after the update plus the
// end-of-iteration summary (WHILE handle h if use_handle) in the last block of the update
cudaError_t launch_outer_defect(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse = 0);
// PCG vector steps on each problem's finest level (FP64): q = A p with partials (p, q); x += alpha
// p, r -= alpha q with partials ||r||^2 and the scaled residual as the cycle's right-hand side;
// partials (r, z); p = z / s + beta p
cudaError_t launch_pcg_q(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse = 0);
// fuse (one problem): the kernels' last blocks take the control steps (pcg_x also the summary)
cudaError_t launch_pcg_x(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse = 0,
                         cudaGraphConditionalHandle h = 0, int use_handle = 0);
cudaError_t launch_pcg_dot(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse = 0);
cudaError_t launch_pcg_p(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse = 0);
cudaError_t launch_update(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse = 0,
                          cudaGraphConditionalHandle h = 0, int use_handle = 0);
cudaError_t launch_norm_b(const EngineDev& E, TileList fine, int grid, cudaStream_t s);
// kind: ControlKind; level: for CTRL_PRE, the finest level whose problems are checked
cudaError_t launch_control(const EngineDev& E, int kind, cudaStream_t s, int level = -1);
// end_of_iteration: clear the zero-iterate flag of running cycles (iteration graph only)
cudaError_t launch_summary(const EngineDev& E, cudaGraphConditionalHandle h, int use_handle,
                           int end_of_iteration, cudaStream_t s);
cudaError_t launch_boundary_check(const EngineDev& E, cudaStream_t s);

enum ControlKind {
  CTRL_INIT = 0, CTRL_CHECK = 1, CTRL_OUTER = 2, CTRL_POST = 4, CTRL_CHECK0 = 5,
  CTRL_PRE = 6,  // lagged convergence test after the first smoothing step of a cycle
  CTRL_PCG_ALPHA = 7,  // PCG: alpha = rho / (p, q)
  CTRL_PCG_BETA = 8    // PCG: rho' = (r, z), beta = rho' / rho
};

int sm_count();

}  // namespace hn
