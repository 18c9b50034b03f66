// Host-side engine of the hn library (internal): operators, hierarchies, and the batch engine
// that runs the V-cycle schedule over a set of hierarchies as CUDA graphs.
#pragma once

#include <chrono>
#include <cstdarg>
#include <string>
#include <vector>

#include "hn_internal.h"
#include "../../include/hn_profile.h"

namespace hn {

// thread-local error message + status helpers
hn_status set_error(hn_status st, const char* fmt, ...);
void clear_error();
const char* last_error();

#define HN_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return ::hn::set_error(e_ == cudaErrorMemoryAllocation ? HN_ERR_OOM : HN_ERR_CUDA, \
                             "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,  \
                             __LINE__);                                                  \
  } while (0)

#define HN_TRY(expr)                                    \
  do {                                                  \
    const hn_status hn_try_status_ = (expr);            \
    if (hn_try_status_ != HN_OK) return hn_try_status_; \
  } while (0)

inline long long now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch()).count();
}

// bump allocator over one device allocation (256-byte aligned pieces)
struct Bump {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* r = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return r;
  }
};

// Debug builds (HN_DEBUG_CHECKS=1): every device block the library allocates for an operator, a
// hierarchy or an engine carries kGuardBytes of a fixed pattern before and after it, checked by
// hn_debug_check_mg / hn_debug_check_band; release builds allocate the block alone.
#ifndef HN_DEBUG_CHECKS
#define HN_DEBUG_CHECKS 0
#endif
constexpr size_t kGuardBytes = HN_DEBUG_CHECKS ? 4096 : 0;
constexpr unsigned char kGuardByte = 0xC3;
// allocate bytes (+ guards) on the device: *base is what to free, *mem the usable block
hn_status guarded_alloc(size_t bytes, void** base, void** mem);
// the guards of a block from guarded_alloc are intact (always HN_OK in release builds)
hn_status guards_intact(const void* base, size_t bytes, const char* what);

// device bytes a hierarchy of fine level L needs (same arithmetic as its construction)
size_t hierarchy_bytes(int L, int coarse, int prec, int solver);

// kernel classes timed in profiling mode
enum KClass {
  KC_JACOBI = 0, KC_JACOBI_FIRST, KC_DEFECT, KC_RESTRICT, KC_PROLONG, KC_COARSE, KC_CHECK,
  KC_OUTER_DEFECT, KC_UPDATE, KC_CONTROL, KC_TAIL, KC_PCG_Q, KC_PCG_X, KC_PCG_DOT, KC_PCG_P,
  KC_PROLONG_JACOBI, KC_MID_DOWN, KC_MID_UP, KC_SWEEP_DOWN, KC_SWEEP_UP, KC_COUNT
};

// launch shape of the schedule: levels <= tail_level run fused in one cluster launch of
// `cluster` blocks per problem; levels above run as one launch per step
constexpr int kSweepMaxLevel = 9;   // largest level in fused sweeps under tuning sweep 1

struct Tuning {
  int tail_level = 7;
  int cluster = 16;
  int pdl = 2;      // programmatic dependent launch for launches of fewer blocks than SMs
  int staged = 0;   // stream the bands of large FP32/FP16 levels through shared memory by bulk
                    // copies (measured slower than the register path at L=12; off)
  int dsm = 1;      // fused tail: cluster levels in distributed shared memory when they fit
  int fuse_up = 0;  // levels above the tail: prolongation inside the first post-smoothing step
                    // (measured slower than the two kernels: 192 vs 157 us at L=12 FP32; off)
  int mid = 0;      // levels tail_level+1..mid run in the two persistent (cooperative) kernels
                    // of each cycle, levels above mid as one launch per step; 0: no persistent
                    // kernels (default: a grid barrier plus the memory latency of a step measured
                    // as long as a kernel boundary, ~3.5 us at L = 10, so they did not pay).
                    // Not combined with staged or fuse_up, which are per-step forms.
  int sweep = 1;    // an engine of one problem with V(2,2) cycles: the down part of each level
                    // between the tail and the finest, up to kSweepMaxLevel (smoothing, defect,
                    // restriction), and the up part (prolongation, smoothing) as one launch each
                    // over 2-D tiles with recomputed halos (k_sweep_down / k_sweep_up); 2: every
                    // level above the tail, with the finest level's steps after its first smoothing
                    // step.  Default 1 (measured at L = 9 / 10 / 12: FP32-inner DC -3.6 / -1.0 /
                    // -0.4 %, FP64 MG -11.5 / -2.3 / -0.3 %); 2 was slower from L = 10 up.
};

class Engine;

}  // namespace hn

namespace hn {
// output of the work-list kernel (engine.cu)
struct WorkListOut {
  int2* items[kMaxLevel + 1];
  int4* chunks[kMaxLevel + 1];
  int2* fine;
  int n[kMaxLevel + 1];              // members having level l
  int nt[kMaxLevel + 1];             // tiles of level l
  int nfine;                         // members
};
}  // namespace hn

struct hn_band {
  int L = 0;
  long long n = 0, N = 0, pitch = 0;
  void* mem = nullptr;
  double* band[9] = {};
  double* coef = nullptr;   // device cell coefficients, nullptr for a = 1
  unsigned bc = 15u;        // Dirichlet sides (HN_DIRICHLET_*); the others are free Neumann
  int device = 0;           // CUDA device the bands live on (current at creation)
  void* mem_base = nullptr; // the allocation of mem with its guards (nullptr: mem came from a caller)
  size_t mem_bytes = 0;
  ~hn_band();
};

struct hn_mg {
  int L = 0, coarse = 2, m = 0;
  hn_mg_opts opts{};
  hn::Params prm{};
  void* mem = nullptr;
  size_t bytes = 0;
  hn::ProblemDev host{};     // descriptor (device pointers)
  long long setup_ns = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  hn::Engine* solo = nullptr;
  hn::Tuning tuning{};        // launch shape chosen for this hierarchy (hn_mg_set_tuning)
  bool tuned = false;
  void* mem_base = nullptr;   // the allocation of mem with its guards (nullptr: mem came from a caller)
  ~hn_mg();
};

namespace hn {

// Device memory of the hierarchy: a block of exactly hierarchy_bytes() from the caller (mem) or
// a new allocation (mem == nullptr); the setup temporaries go to scratch when it holds
// hierarchy_tmp_bytes(), else to a transient allocation.
hn_status build_hierarchy(const hn_band* A, const hn_mg_opts& o, cudaStream_t stream, hn_mg* mg,
                          void* mem = nullptr, void* scratch = nullptr, size_t scratch_bytes = 0);
size_t hierarchy_tmp_bytes(int L, int c, int prec, bool has_coef);
// Q1 operator of level L (hn_band_create_bc without the input checks, on stream s, in mem of
// band_bytes() when given); check_band_inputs holds the checks.
hn_status check_band_inputs(int L, const double* cell_coef, unsigned dirichlet_sides);
size_t band_bytes(int L, bool has_coef);
hn_status build_band(int L, const double* cell_coef, unsigned bc, cudaStream_t s, void* mem,
                     hn_band** out);
hn_status validate_opts(const hn_mg_opts& o, int L);
Params params_from(const hn_mg_opts& o);

// A batch engine: up to `cap` problem slots solved together.
class Engine {
 public:
  Engine() = default;
  ~Engine();
  // cap: slots; Lmax: highest level the schedule covers; tiles_cap[l]: work-list capacity per
  // level (l = 0..kMaxLevel), fine_cap: fine-list capacity
  hn_status create(const Params& prm, int cap, int Lmax, const std::vector<long long>& tiles_cap,
                   long long fine_cap, cudaStream_t s);
  // assign hierarchies to slots (nullptr = empty slot) and rewrite the device work lists
  hn_status set_members(const std::vector<hn_mg*>& slots);
  // reset the state of the given slots for a new solve
  hn_status start(const std::vector<int>& slots, const std::vector<int>& have_guess);
  // closed-world solve of all members: device-side loop in one graph launch
  hn_status run_to_completion();
  // host-driven steps (serving / profiling)
  hn_status run_init();
  hn_status run_iteration(unsigned* active_out);
  // the same in two halves: launch (returns at once unless profiling) and wait for the result,
  // so that the caller can do host work while the iteration runs
  hn_status launch_iteration();
  hn_status finish_iteration(unsigned* active_out);
  hn_status read_states(std::vector<ProbState>& out);
  // the device error word (a bounded wait gave up); reset by start()
  hn_status read_error(int* err);
  // the device error word and the details a failed debug check recorded (source line, two indices)
  hn_status read_error_detail(int (&err)[4]);
  // the guards of the engine's device block (debug builds)
  hn_status check_guards() const;
  hn_status read_states_async(ProbState* host_dst);
  // single-kernel execution on slot 0 (hn_mg_apply)
  hn_status apply(int op, int level, int want, cudaStream_t s);
  hn_status apply_check_norm(cudaStream_t s);
  hn_status set_phase(int slot, int phase, int zero_top);

  void set_profiling(bool on);
  void set_iter_limit(unsigned lim) { E_.iter_limit = lim; graphsValid_ = false; }
  void set_tuning(const Tuning& t) {
    tune_ = t; E_.pdl = t.pdl; E_.staged = t.staged; E_.dsm = t.dsm; graphsValid_ = false;
  }
  const Tuning& tuning() const { return tune_; }
  // levels that may be some problem's finest level (their first smoothing step may start from a
  // nonzero iterate); all levels for the server
  void set_top_mask_all() { topMaskAll_ = true; graphsValid_ = false; }
  int kernel_times(hn_kernel_time* out, int max) const;

  long long last_launches() const { return lastLaunches_; }
  int cap() const { return cap_; }
  const Params& params() const { return prm_; }
  cudaStream_t stream() const { return s_; }

 private:
  hn_status capture_graphs();
  hn_status issue_init(cudaStream_t s, cudaGraphConditionalHandle h, int use_h);
  hn_status issue_iteration(cudaStream_t s, cudaGraphConditionalHandle h, int use_h);
  hn_status issue_vcycle(cudaStream_t s, int want);
  // IF node at the current end of stream s's capture; further launches go to its body (on aux_)
  hn_status open_if(cudaStream_t& s, int which);
  hn_status close_if(cudaStream_t& s, cudaStream_t outer);
  hn_status capture_solve(bool cond);
  void clear_marks();
  bool cond_on(int which) const { return condCapture_ && ((E_.prm.cond.mask >> which) & 1u); }
  int grid_for(long long tiles) const;
  hn_status mark(cudaStream_t s, int cls, int level, bool begin);
  void destroy_graphs();

  Params prm_{};
  int cap_ = 0, Lmax_ = 0;
  cudaStream_t s_ = nullptr;
  void* mem_ = nullptr;
  void* memBase_ = nullptr;      // mem_ with its guards
  size_t memBytes_ = 0;
  unsigned* hActive_ = nullptr;  // mapped pinned
  EngineDev E_{};
  ProblemDev* dP_ = nullptr;
  ProbState* dS_ = nullptr;
  int* dFineOff_ = nullptr;
  int* dCounts_ = nullptr;          // [kMaxLevel + 2]: per level, then the fine list
  int2* dItems_[kMaxLevel + 1] = {};
  int4* dChunks_[kMaxLevel + 1] = {};
  int* dChunkCounts_ = nullptr;
  long long chunkCap_[kMaxLevel + 1] = {};
  int* dErr_ = nullptr;
  int2* dFine_ = nullptr;
  long long itemCap_[kMaxLevel + 1] = {};
  long long fineCap_ = 0;
  TileList lists_[kMaxLevel + 1] = {};
  TileList fine_{};
  int grid_[kMaxLevel + 1] = {};
  TileList* dLists_ = nullptr;      // device copy of lists_ (read by the persistent kernels)
  TileList* hLists_ = nullptr;      // its pinned staging copy
  unsigned long long* dBar_ = nullptr;   // grid barriers of the persistent kernels
  int mid_top() const;              // top level of the persistent kernels (<= tail level: none)
  bool sweep_on() const;            // the fused level sweeps run (tuning sweep, and they apply)
  bool sweep_level(int l) const;    // level l's down / up parts run as fused sweeps
  bool fuse_control() const;        // the DC control steps fold into the outer defect and update
  // level l may be a member's own finest level (the server's engines: any level)
  bool is_top(int l) const { return topMaskAll_ || ((topMask_ >> l) & 1u); }
  int fineGrid_ = 1;
  int maxGrid_ = 1;
  std::vector<hn_mg*> members_;
  std::vector<int> hCounts_;
  // set_members' plan (device) and its pinned staging area: counts, fine offsets, plan, problems
  int* dPlan_ = nullptr;
  void* hStage_ = nullptr;
  cudaEvent_t upEv_ = nullptr;       // the last upload from the staging area
  size_t plan_ints() const { return (size_t)(kMaxLevel + 2) * cap_ + cap_ + 1; }
  size_t stage_probs_off() const {
    return (((size_t)(kMaxLevel + 2) + (kMaxLevel + 1) + cap_ + plan_ints()) * sizeof(int) + 255) & ~size_t(255);
  }
  size_t stage_bytes() const { return stage_probs_off() + sizeof(ProblemDev) * cap_; }
  cudaGraphExec_t gSolve_ = nullptr, gInit_ = nullptr, gIter_ = nullptr;
  bool graphsValid_ = false;
  int initLaunches_ = 0, iterLaunches_ = 0, counting_ = 0;
  Tuning tune_{};
  unsigned topMask_ = 0;
  bool topMaskAll_ = false;
  long long lastLaunches_ = 0;
  // IF nodes inside the closed-world loop (see CondDev)
  cudaStream_t aux_ = nullptr;
  bool condCapture_ = false, condUsed_ = false, pdlBarrier_ = false;
  cudaGraphConditionalHandle hCond_[2][3] = {};   // IF handles of the two halves of the loop body
  unsigned* dTaken_ = nullptr;
  unsigned long long* dLaunches_ = nullptr;
  // profiling
  bool profiling_ = false;
  struct Mark { cudaEvent_t b, e; int cls, level; long long bytes; };
  std::vector<Mark> marks_;
  std::vector<cudaEvent_t> openBegin_;
  struct Acc { double ms = 0; long long launches = 0; long long bytes = 0; };
  Acc acc_[KC_COUNT][kMaxLevel + 1];
  long long launch_bytes(int cls, int level) const;
  hn_status accumulate_marks();
};

}  // namespace hn
