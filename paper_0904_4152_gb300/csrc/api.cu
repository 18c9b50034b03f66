// C ABI of the hn library (include/hn.h, include/hn_profile.h): argument checking, explicit copies
// at the boundary (Sec. 4.1 explicit-copy containers), and dispatch to the engine.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>

#include "engine.h"
#include "../../include/hn_profile.h"
#include "../../include/hn_tune.h"
#include "../../include/hn_debug.h"

using namespace hn;

namespace {

struct OwnedStream {
  cudaStream_t s = nullptr;
  ~OwnedStream() { if (s) cudaStreamDestroy(s); }
};

// work-list capacities of a single hierarchy
void exact_caps(const std::vector<hn_mg*>& mgs, std::vector<long long>& caps, long long& fine) {
  caps.assign(kMaxLevel + 1, 0);
  fine = 0;
  for (hn_mg* mg : mgs) {
    for (int l = mg->coarse; l <= mg->L; ++l) caps[l] += pitch_of(l) / kTile;
    fine += pitch_of(mg->L) / kTile;
  }
}

// the engine's device error words after a solve: a bounded wait that gave up, or (debug builds) a
// failed index check
hn_status device_error(Engine& e) {
  int d[4] = {0, 0, 0, 0};
  HN_TRY(e.read_error_detail(d));
  switch (d[0]) {
    case 0: return HN_OK;
    case 3: return set_error(HN_ERR_CUDA, "a grid barrier of the persistent kernels timed out");
    case 5: return set_error(HN_ERR_STATE, "debug check failed (k_cycle.cu line %d, indices %d, %d)", d[1], d[2], d[3]);
    default: return set_error(HN_ERR_CUDA, "a bounded device wait for a bulk copy gave up");
  }
}

// name of the current GPU (the key of the launch-shape cache)
hn_status gpu_name(char* out, size_t cap) {
  int dev = 0;
  HN_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp p;
  HN_CUDA(cudaGetDeviceProperties(&p, dev));
  std::snprintf(out, cap, "%s", p.name);
  return HN_OK;
}

// top level of the persistent kernels among the autotuner's candidates
constexpr int kMidCandidate = 10;

// default launch shape of one problem: FP64 arithmetic is slow enough on this part that the
// fused tail pays from level 6 down (its levels then fit in distributed shared memory); the
// FP32/FP16 inner cycles fuse from level 5 down (block 0's shared memory alone), the levels
// above it up to 9 running as fused sweeps (autotuned at L = 10: 1.537 ms against >= 1.576 ms
// with the tail from level 7)
Tuning default_tuning(const Params& prm) {
  Tuning t;
  t.tail_level = prm.prec == P64 ? 6 : 5;
  return t;
}

hn_status ensure_solo(hn_mg* mg) {
  if (mg->solo) return HN_OK;
  std::vector<long long> caps;
  long long fine;
  exact_caps({mg}, caps, fine);
  std::unique_ptr<Engine> e(new Engine());
  HN_TRY(e->create(mg->prm, 1, mg->L, caps, fine, mg->stream));
  HN_TRY(e->set_members({mg}));
  e->set_tuning(mg->tuned ? mg->tuning : default_tuning(mg->prm));
  mg->solo = e.release();
  return HN_OK;
}

// cache of the last batch engine (same hierarchy list -> same work lists and graphs)
std::mutex g_batch_mu;
std::vector<hn_mg*> g_batch_key;
std::unique_ptr<Engine> g_batch_engine;

void forget_batch(hn_mg* mg) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (std::find(g_batch_key.begin(), g_batch_key.end(), mg) != g_batch_key.end()) {
    g_batch_engine.reset();
    g_batch_key.clear();
  }
}

// launch shape of a batch: the members' common tuned shape, else by batch size (many problems:
// one block per problem and a tail that fits in shared memory; few problems: the solo default)
Tuning batch_tuning(const std::vector<hn_mg*>& list) {
  bool same = list[0]->tuned;
  for (hn_mg* mg : list)
    same = same && mg->tuned && mg->tuning.tail_level == list[0]->tuning.tail_level &&
           mg->tuning.cluster == list[0]->tuning.cluster && mg->tuning.pdl == list[0]->tuning.pdl &&
           mg->tuning.staged == list[0]->tuning.staged && mg->tuning.dsm == list[0]->tuning.dsm &&
           mg->tuning.fuse_up == list[0]->tuning.fuse_up && mg->tuning.mid == list[0]->tuning.mid &&
           mg->tuning.sweep == list[0]->tuning.sweep;
  if (same) return list[0]->tuning;
  Tuning t;
  const int n = (int)list.size();
  if (n >= 32) { t.tail_level = 5; t.cluster = 1; }
  else if (n >= 8) { t.tail_level = 6; t.cluster = 4; }
  return t;
}

hn_status copy_in(double* dst, const double* src, long long N, int device_ptrs, cudaStream_t s) {
  HN_CUDA(cudaMemcpyAsync(dst, src, (size_t)N * 8,
                          device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return HN_OK;
}

hn_status copy_out(double* dst, const double* src, long long N, int device_ptrs, cudaStream_t s) {
  HN_CUDA(cudaMemcpyAsync(dst, src, (size_t)N * 8,
                          device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return HN_OK;
}

hn_status check_ptr(const void* p, int device_ptrs) {
  if (!p) return set_error(HN_ERR_ARG, "null vector pointer");
  if (device_ptrs && (reinterpret_cast<uintptr_t>(p) & 15))
    return set_error(HN_ERR_ARG, "device vectors must be 16-byte aligned");
  return HN_OK;
}

void fill_stats(const hn_mg* mg, const ProbState& st, long long t0, hn_mg_stats* out) {
  if (!out) return;
  out->cycles = st.cycles;
  out->outer_iters = st.outer_iters;
  out->inner_cycles = st.inner_cycles;
  out->status = st.status;
  out->relres = st.relres;
  out->setup_ns = mg->setup_ns;
  out->solve_ns = now_ns() - t0;
}

}  // namespace

extern "C" {

const char* hn_last_error(void) { return hn::last_error(); }
const char* hn_version(void) { return HN_DEBUG_CHECKS ? "hn 0.2 (sm_103a, debug checks)" : "hn 0.2 (sm_103a)"; }

int hn_debug_build(void) { return HN_DEBUG_CHECKS; }

hn_status hn_debug_check_mg(const hn_mg* mg) {
  clear_error();
  if (!mg) return set_error(HN_ERR_ARG, "null hierarchy");
  if (!HN_DEBUG_CHECKS) return set_error(HN_ERR_STATE, "library built without HN_DEBUG_CHECKS");
  if (mg->stream) HN_CUDA(cudaStreamSynchronize(mg->stream));
  HN_TRY(guards_intact(mg->mem_base, mg->bytes, "hierarchy block"));
  if (mg->solo) HN_TRY(mg->solo->check_guards());
  return HN_OK;
}

hn_status hn_debug_check_band(const hn_band* A) {
  clear_error();
  if (!A) return set_error(HN_ERR_ARG, "null operator");
  if (!HN_DEBUG_CHECKS) return set_error(HN_ERR_STATE, "library built without HN_DEBUG_CHECKS");
  return guards_intact(A->mem_base, A->mem_bytes, "operator block");
}

hn_status hn_debug_overwrite_guard(hn_mg* mg) {
  clear_error();
  if (!mg) return set_error(HN_ERR_ARG, "null hierarchy");
  if (!HN_DEBUG_CHECKS || !mg->mem_base)
    return set_error(HN_ERR_STATE, "no guarded hierarchy block (debug builds, library-allocated blocks)");
  if (mg->stream) HN_CUDA(cudaStreamSynchronize(mg->stream));
  HN_CUDA(cudaMemset(static_cast<char*>(mg->mem_base) + kGuardBytes + mg->bytes, 0, 1));
  return HN_OK;
}

hn_status hn_band_create(int L, const double* cell_coef, hn_band** out) {
  return hn_band_create_bc(L, cell_coef, HN_DIRICHLET_ALL, out);
}

hn_status hn_band_create_bc(int L, const double* cell_coef, unsigned dirichlet_sides, hn_band** out) {
  clear_error();
  if (!out) return set_error(HN_ERR_ARG, "out is NULL");
  *out = nullptr;
  HN_TRY(check_band_inputs(L, cell_coef, dirichlet_sides));
  OwnedStream os;
  HN_CUDA(cudaStreamCreateWithFlags(&os.s, cudaStreamNonBlocking));
  HN_TRY(build_band(L, cell_coef, dirichlet_sides, os.s, nullptr, out));
  return HN_OK;
}

hn_status hn_band_get(const hn_band* A, double* bands_out) {
  clear_error();
  if (!A || !bands_out) return set_error(HN_ERR_ARG, "null argument");
  for (int k = 0; k < 9; ++k)
    HN_CUDA(cudaMemcpy(bands_out + (size_t)k * A->N, A->band[k], (size_t)A->N * 8, cudaMemcpyDeviceToHost));
  return HN_OK;
}

int hn_band_level(const hn_band* A) { return A ? A->L : 0; }
long long hn_band_nodes(const hn_band* A) { return A ? A->N : 0; }
void hn_band_destroy(hn_band* A) { delete A; }

void hn_mg_opts_default(hn_mg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->coarse_L = 2;
  o->pre = 2;
  o->post = 2;
  o->max_cycles = 100;
  o->max_outer = 50;
  o->inner_max = 10;
  o->omega = 0.7;
  o->tol = 1e-8;
  o->inner_tol = 1e-2;
  o->prec = HN_PREC_FP64;
  o->stream = nullptr;
  o->dirichlet_sides = HN_DIRICHLET_ALL;
  o->solver = HN_SOLVER_MG;
  o->coarse_solver = HN_COARSE_EXACT;
}

hn_status hn_mg_setup(const hn_band* A, const hn_mg_opts* opts, hn_mg** out) {
  clear_error();
  if (!A || !out) return set_error(HN_ERR_ARG, "null argument");
  *out = nullptr;
  hn_mg_opts o;
  if (opts) o = *opts; else hn_mg_opts_default(&o);
  HN_TRY(validate_opts(o, A->L));
  const long long t0 = now_ns();
  std::unique_ptr<hn_mg> mg(new hn_mg());
  if (o.stream) {
    mg->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    HN_CUDA(cudaStreamCreateWithFlags(&mg->stream, cudaStreamNonBlocking));
    mg->own_stream = true;
  }
  HN_TRY(build_hierarchy(A, o, mg->stream, mg.get()));
  // a launch shape measured earlier for this key on this GPU (HN_TUNE_CACHE)
  if (const char* path = std::getenv("HN_TUNE_CACHE")) {
    char gpu[256];
    hn_tuning t;
    if (path[0] && gpu_name(gpu, sizeof gpu) == HN_OK &&
        hn_tune_cache_lookup(path, gpu, mg->L, (int)o.prec, (int)o.solver, (int)o.coarse_solver,
                             o.coarse_L, &t) == HN_OK) {
      Tuning tu;
      tu.tail_level = std::max(t.tail_level, mg->coarse);
      tu.cluster = t.cluster;
      tu.pdl = t.pdl;
      tu.staged = t.staged;
      tu.dsm = t.dsm;
      tu.fuse_up = t.fuse_up;
      tu.mid = t.mid;
      tu.sweep = t.sweep;
      mg->tuning = tu;
      mg->tuned = true;
    }
  }
  mg->setup_ns = now_ns() - t0;
  *out = mg.release();
  return HN_OK;
}

size_t hn_mg_device_bytes(const hn_mg* mg) { return mg ? mg->bytes : 0; }

void hn_mg_destroy(hn_mg* mg) {
  if (!mg) return;
  forget_batch(mg);
  if (mg->stream) cudaStreamSynchronize(mg->stream);
  delete mg;
}

hn_status hn_mg_solve(hn_mg* mg, const double* b, double* x, int x_is_guess, int device_ptrs,
                      hn_mg_stats* stats) {
  clear_error();
  if (!mg) return set_error(HN_ERR_ARG, "null hierarchy");
  HN_TRY(check_ptr(b, device_ptrs));
  HN_TRY(check_ptr(x, device_ptrs));
  const long long t0 = now_ns();
  HN_TRY(ensure_solo(mg));
  Engine& e = *mg->solo;
  cudaStream_t s = e.stream();
  const long long N = N_of(mg->L);
  ProblemDev& P = mg->host;
  HN_TRY(copy_in(P.b64, b, N, device_ptrs, s));
  if (x_is_guess) HN_TRY(copy_in(P.x64, x, N, device_ptrs, s));
  else HN_CUDA(cudaMemsetAsync(P.x64, 0, (size_t)N * 8, s));
  HN_TRY(e.start({0}, {x_is_guess ? 1 : 0}));
  HN_TRY(e.run_to_completion());
  std::vector<ProbState> st;
  HN_TRY(e.read_states(st));
  HN_TRY(device_error(e));
  if (st[0].status != HN_ERR_ARG) {
    if (st[0].status == HN_OK && st[0].bnorm == 0.0) HN_CUDA(cudaMemsetAsync(P.x64, 0, (size_t)N * 8, s));
    HN_TRY(copy_out(x, P.x64, N, device_ptrs, s));
    HN_CUDA(cudaStreamSynchronize(s));
  }
  fill_stats(mg, st[0], t0, stats);
  if (st[0].status == HN_ERR_ARG) return set_error(HN_ERR_ARG, "right-hand side is nonzero on the boundary");
  if (st[0].status == HN_ERR_NONFINITE) return set_error(HN_ERR_NONFINITE, "non-finite residual norm");
  if (st[0].status == HN_ERR_NOT_CONVERGED)
    return set_error(HN_ERR_NOT_CONVERGED, "not converged: relres %.3e after %d cycles", st[0].relres, st[0].cycles);
  return (hn_status)st[0].status;
}

hn_status hn_mg_solve_batch(hn_mg* const* mgs, int count, const double* const* b, double* const* x,
                            int device_ptrs, hn_mg_stats* stats) {
  clear_error();
  if (!mgs || !b || !x || count < 1) return set_error(HN_ERR_ARG, "bad batch arguments");
  const long long t0 = now_ns();
  std::vector<hn_mg*> list(mgs, mgs + count);
  for (int j = 0; j < count; ++j) {
    if (!list[j]) return set_error(HN_ERR_ARG, "null hierarchy %d", j);
    HN_TRY(check_ptr(b[j], device_ptrs));
    HN_TRY(check_ptr(x[j], device_ptrs));
    const Params& a = list[0]->prm;
    const Params& c = list[j]->prm;
    if (a.prec != c.prec || a.pre != c.pre || a.post != c.post || a.omega != c.omega ||
        a.coarse != c.coarse || a.solver != c.solver || a.coarse_cg != c.coarse_cg)
      return set_error(HN_ERR_ARG, "batch members must share precision, pre, post, omega, coarse_L, "
                                   "solver and coarse solver");
    for (int i = 0; i < j; ++i)
      if (list[i] == list[j]) return set_error(HN_ERR_ARG, "batch members must be distinct");
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (!g_batch_engine || g_batch_key != list) {
    g_batch_engine.reset();
    g_batch_key.clear();
    std::vector<long long> caps;
    long long fine;
    exact_caps(list, caps, fine);
    int Lmax = 0;
    for (hn_mg* mg : list) Lmax = std::max(Lmax, mg->L);
    // batch-wide iteration caps: the most generous member's (each problem keeps its own state)
    Params prm = list[0]->prm;
    for (hn_mg* mg : list) {
      prm.max_cycles = std::max(prm.max_cycles, mg->prm.max_cycles);
      prm.max_outer = std::max(prm.max_outer, mg->prm.max_outer);
    }
    std::unique_ptr<Engine> e(new Engine());
    HN_TRY(e->create(prm, count, Lmax, caps, fine, list[0]->stream));
    HN_TRY(e->set_members(list));
    e->set_tuning(batch_tuning(list));
    g_batch_engine = std::move(e);
    g_batch_key = list;
  }
  Engine& e = *g_batch_engine;
  {
    const Tuning t = batch_tuning(list);
    const Tuning& c = e.tuning();
    if (t.tail_level != c.tail_level || t.cluster != c.cluster || t.pdl != c.pdl || t.staged != c.staged ||
        t.dsm != c.dsm || t.fuse_up != c.fuse_up || t.mid != c.mid || t.sweep != c.sweep)
      e.set_tuning(t);
  }
  cudaStream_t s = e.stream();
  std::vector<int> slots(count), guess(count, 0);
  for (int j = 0; j < count; ++j) {
    slots[j] = j;
    ProblemDev& P = list[j]->host;
    const long long N = N_of(list[j]->L);
    HN_TRY(copy_in(P.b64, b[j], N, device_ptrs, s));
    HN_CUDA(cudaMemsetAsync(P.x64, 0, (size_t)N * 8, s));
  }
  HN_TRY(e.start(slots, guess));
  HN_TRY(e.run_to_completion());
  std::vector<ProbState> st;
  HN_TRY(e.read_states(st));
  HN_TRY(device_error(e));
  hn_status first_bad = HN_OK;
  for (int j = 0; j < count; ++j) {
    ProblemDev& P = list[j]->host;
    const long long N = N_of(list[j]->L);
    if (st[j].status != HN_ERR_ARG) {
      if (st[j].status == HN_OK && st[j].bnorm == 0.0) HN_CUDA(cudaMemsetAsync(P.x64, 0, (size_t)N * 8, s));
      HN_TRY(copy_out(x[j], P.x64, N, device_ptrs, s));
    }
    if (st[j].status != HN_OK && first_bad == HN_OK) first_bad = (hn_status)st[j].status;
  }
  HN_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < count; ++j) fill_stats(list[j], st[j], t0, stats ? stats + j : nullptr);
  if (first_bad != HN_OK) return set_error(first_bad, "at least one batch member did not converge cleanly");
  return HN_OK;
}

hn_status hn_mg_apply(hn_mg* mg, hn_op op, int level, int inner, const void* in1, const void* in2,
                      void* out, double* norm_out) {
  clear_error();
  if (!mg || !out) return set_error(HN_ERR_ARG, "null argument");
  if (level < mg->coarse || level > mg->L) return set_error(HN_ERR_ARG, "level out of range");
  const bool p64 = mg->prm.prec == P64;
  if ((inner != 0) == p64)
    return set_error(HN_ERR_STATE, "inner=%d does not match the hierarchy precision", inner);
  if ((op == HN_OP_RESTRICT || op == HN_OP_PROLONG_ADD) && level <= mg->coarse)
    return set_error(HN_ERR_ARG, "transfer needs a coarser level");
  if (op == HN_OP_COARSE && level != mg->coarse) return set_error(HN_ERR_ARG, "coarse op on the coarsest level only");
  if (norm_out && (op != HN_OP_DEFECT || level != mg->L))
    return set_error(HN_ERR_STATE, "norm only for the defect on the finest level");
  HN_TRY(ensure_solo(mg));
  Engine& e = *mg->solo;
  cudaStream_t s = e.stream();
  const size_t vs = p64 ? 8 : 4;
  const LevelDev& d = mg->host.lev[level];
  const size_t N = (size_t)N_of(level);
  auto put = [&](void* dst, const void* src, size_t n) -> hn_status {
    if (!src) return set_error(HN_ERR_ARG, "missing input vector");
    HN_CUDA(cudaMemcpyAsync(dst, src, n * vs, cudaMemcpyHostToDevice, s));
    return HN_OK;
  };
  const void* result = nullptr;
  size_t nres = N;
  HN_TRY(e.set_phase(0, PH_CYCLE, op == HN_OP_JACOBI_ZERO ? 1 : 0));
  switch (op) {
    case HN_OP_SPMV: HN_TRY(put(d.x[0], in1, N)); result = d.r; break;
    case HN_OP_DEFECT: HN_TRY(put(d.x[0], in1, N)); HN_TRY(put(d.rhs, in2, N)); result = d.r; break;
    case HN_OP_JACOBI: HN_TRY(put(d.x[0], in1, N)); HN_TRY(put(d.rhs, in2, N)); result = d.x[1]; break;
    case HN_OP_JACOBI_ZERO: HN_TRY(put(d.rhs, in2, N)); result = d.x[1]; break;
    case HN_OP_RESTRICT: {
      HN_TRY(put(d.r, in1, N));
      result = mg->host.lev[level - 1].rhs;
      nres = (size_t)N_of(level - 1);
      break;
    }
    case HN_OP_PROLONG_ADD:
      HN_TRY(put(mg->host.lev[level - 1].x[0], in1, (size_t)N_of(level - 1)));
      HN_TRY(put(d.x[0], in2, N));
      result = d.x[0];
      break;
    case HN_OP_COARSE: HN_TRY(put(d.rhs, in2, N)); result = d.x[0]; break;
    default: return set_error(HN_ERR_ARG, "unknown op %d", (int)op);
  }
  HN_TRY(e.apply(op, level, PH_CYCLE, s));
  HN_CUDA(cudaMemcpyAsync(out, result, nres * vs, cudaMemcpyDeviceToHost, s));
  HN_CUDA(cudaStreamSynchronize(s));
  if (norm_out) {
    std::vector<ProbState> st;
    HN_TRY(e.set_phase(0, PH_CHECK, 0));
    HN_TRY(e.apply_check_norm(s));
    HN_TRY(e.read_states(st));
    *norm_out = st[0].dnorm;
  }
  return HN_OK;
}

hn_status hn_mg_get_inner_bands(const hn_mg* mg, int level, void* bands_out, float* scales_out) {
  clear_error();
  if (!mg || !bands_out) return set_error(HN_ERR_ARG, "null argument");
  if (mg->prm.prec == P64) return set_error(HN_ERR_STATE, "FP64 hierarchy has no inner bands");
  if (level < mg->coarse || level > mg->L) return set_error(HN_ERR_ARG, "level out of range");
  const LevelDev& d = mg->host.lev[level];
  const size_t N = (size_t)N_of(level), es = mg->prm.prec == P32 ? 4 : 2;
  for (int k = 0; k < 9; ++k)
    HN_CUDA(cudaMemcpy(static_cast<char*>(bands_out) + k * N * es, d.band[k], N * es, cudaMemcpyDeviceToHost));
  if (scales_out)
    for (int k = 0; k < 9; ++k) scales_out[k] = d.scale[k];
  return HN_OK;
}

hn_status hn_mg_set_profiling(hn_mg* mg, int enable) {
  clear_error();
  if (!mg) return set_error(HN_ERR_ARG, "null hierarchy");
  HN_TRY(ensure_solo(mg));
  mg->solo->set_profiling(enable != 0);
  return HN_OK;
}

hn_status hn_mg_set_tuning(hn_mg* mg, const hn_tuning* t) {
  clear_error();
  if (!mg || !t) return set_error(HN_ERR_ARG, "null argument");
  const int c = t->cluster;
  if (t->tail_level < mg->coarse || t->tail_level > HN_MAX_LEVEL || !(c == 1 || c == 2 || c == 4 || c == 8 || c == 16))
    return set_error(HN_ERR_ARG, "tail_level in [coarse_L, %d], cluster in {1,2,4,8,16}", HN_MAX_LEVEL);
  HN_TRY(ensure_solo(mg));
  if (t->pdl < 0 || t->pdl > 3) return set_error(HN_ERR_ARG, "pdl must be 0, 1, 2 or 3");
  if (t->staged != 0 && t->staged != 1) return set_error(HN_ERR_ARG, "staged must be 0 or 1");
  if (t->dsm != 0 && t->dsm != 1) return set_error(HN_ERR_ARG, "dsm must be 0 or 1");
  if (t->fuse_up != 0 && t->fuse_up != 1) return set_error(HN_ERR_ARG, "fuse_up must be 0 or 1");
  if (t->mid < 0 || t->mid > HN_MAX_LEVEL) return set_error(HN_ERR_ARG, "mid must be in [0, %d]", HN_MAX_LEVEL);
  if (t->sweep < 0 || t->sweep > 2) return set_error(HN_ERR_ARG, "sweep must be 0, 1 or 2");
  Tuning tu;
  tu.tail_level = t->tail_level;
  tu.cluster = c;
  tu.pdl = t->pdl;
  tu.staged = t->staged;
  tu.dsm = t->dsm;
  tu.fuse_up = t->fuse_up;
  tu.mid = t->mid;
  tu.sweep = t->sweep;
  mg->solo->set_tuning(tu);
  mg->tuning = tu;
  mg->tuned = true;
  return HN_OK;
}

hn_status hn_mg_get_tuning(const hn_mg* mg, hn_tuning* t) {
  clear_error();
  if (!mg || !t) return set_error(HN_ERR_ARG, "null argument");
  const Tuning tu = mg->solo ? mg->solo->tuning() : (mg->tuned ? mg->tuning : default_tuning(mg->prm));
  t->tail_level = tu.tail_level;
  t->cluster = tu.cluster;
  t->pdl = tu.pdl;
  t->staged = tu.staged;
  t->dsm = tu.dsm;
  t->fuse_up = tu.fuse_up;
  t->mid = tu.mid;
  t->sweep = tu.sweep;
  return HN_OK;
}

hn_status hn_mg_autotune(hn_mg* mg, const double* b, int reps, hn_tuning* best, double* times_ms,
                         int cap) {
  clear_error();
  if (!mg || !b || reps < 1) return set_error(HN_ERR_ARG, "bad arguments");
  HN_TRY(ensure_solo(mg));
  const long long N = N_of(mg->L);
  double* x = nullptr;
  HN_CUDA(cudaMallocHost(reinterpret_cast<void**>(&x), (size_t)N * 8));
  struct Free { double* p; ~Free() { cudaFreeHost(p); } } fr{x};
  const int clusters[5] = {1, 2, 4, 8, 16};
  // the per-level forms: per-step launches, persistent kernels of the middle levels, fused sweeps
  const int mids[3] = {0, kMidCandidate, 0}, sweeps[3] = {0, 0, 1};
  double best_ms = 1e300;
  const Tuning cur = mg->solo->tuning();
  hn_tuning bt{cur.tail_level, cur.cluster, 2, 0, 1, 0, cur.mid, cur.sweep};
  cudaEvent_t e0, e1;
  HN_CUDA(cudaEventCreate(&e0));
  HN_CUDA(cudaEventCreate(&e1));
  struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
  const int tmax = std::min(mg->L, 9);
  for (int mi = 0; mi < 3; ++mi)
  for (int T = mg->coarse; T <= tmax; ++T)
    for (int ci = 0; ci < 5; ++ci) {
      hn_tuning t{T, clusters[ci], 2, 0, 1, 0, mids[mi], sweeps[mi]};
      HN_TRY(hn_mg_set_tuning(mg, &t));
      HN_TRY(hn_mg_solve(mg, b, x, 0, 0, nullptr));            // capture + warm-up
      HN_CUDA(cudaEventRecord(e0, mg->solo->stream()));
      for (int r = 0; r < reps; ++r) {
        hn_status st = hn_mg_solve(mg, b, x, 0, 0, nullptr);
        if (st != HN_OK && st != HN_ERR_NOT_CONVERGED) return st;
      }
      HN_CUDA(cudaEventRecord(e1, mg->solo->stream()));
      HN_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      HN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      const double per = ms / reps;
      const int idx = (mi * (tmax - mg->coarse + 1) + (T - mg->coarse)) * 5 + ci;
      if (times_ms && idx < cap) times_ms[idx] = per;
      if (per < best_ms) { best_ms = per; bt = t; }
    }
  HN_TRY(hn_mg_set_tuning(mg, &bt));
  if (best) *best = bt;
  if (const char* path = std::getenv("HN_TUNE_CACHE")) {
    char gpu[256];
    if (path[0] && gpu_name(gpu, sizeof gpu) == HN_OK) {
      const hn_mg_opts& o = mg->opts;
      const hn_status st = hn_tune_cache_store(path, gpu, mg->L, (int)o.prec, (int)o.solver,
                                               (int)o.coarse_solver, o.coarse_L, &bt);
      if (st != HN_OK) return set_error(st, "cannot write the launch-shape cache %s", path);
    }
  }
  return HN_OK;
}

hn_status hn_mg_autotune_batch(hn_mg* const* mgs, int count, const double* const* b, int reps,
                               hn_tuning* best) {
  clear_error();
  if (!mgs || !b || count < 1 || reps < 1) return set_error(HN_ERR_ARG, "bad arguments");
  std::vector<double*> xs(count, nullptr);
  struct FreeAll { std::vector<double*>& v; ~FreeAll() { for (double* p : v) if (p) cudaFreeHost(p); } } fa{xs};
  for (int j = 0; j < count; ++j)
    HN_CUDA(cudaMallocHost(reinterpret_cast<void**>(&xs[j]), (size_t)N_of(mgs[j]->L) * 8));
  const int clusters[3] = {1, 2, 4};
  int Lmax = 0;
  for (int j = 0; j < count; ++j) Lmax = std::max(Lmax, mgs[j]->L);
  double best_ms = 1e300;
  const int mids[2] = {0, kMidCandidate};
  hn_tuning bt{5, 1, 2, 0, 1, 0, mids[1], 0};
  for (int mi = 0; mi < 2; ++mi)
  for (int T = mgs[0]->coarse; T <= std::min(Lmax, 8); ++T)
    for (int ci = 0; ci < 3; ++ci) {
      hn_tuning t{T, clusters[ci], 2, 0, 1, 0, mids[mi], 0};
      for (int j = 0; j < count; ++j) {
        Tuning tu; tu.tail_level = T; tu.cluster = clusters[ci]; tu.pdl = 2; tu.mid = mids[mi];
        mgs[j]->tuning = tu;
        mgs[j]->tuned = true;
      }
      HN_TRY(hn_mg_solve_batch(mgs, count, b, xs.data(), 0, nullptr));   // capture + warm-up
      const long long t0 = now_ns();
      for (int r = 0; r < reps; ++r) {
        hn_status st = hn_mg_solve_batch(mgs, count, b, xs.data(), 0, nullptr);
        if (st != HN_OK && st != HN_ERR_NOT_CONVERGED) return st;
      }
      const double ms = (now_ns() - t0) * 1e-6 / reps;
      if (ms < best_ms) { best_ms = ms; bt = t; }
    }
  for (int j = 0; j < count; ++j) {
    Tuning tu; tu.tail_level = bt.tail_level; tu.cluster = bt.cluster; tu.pdl = bt.pdl; tu.mid = bt.mid;
    mgs[j]->tuning = tu;
    mgs[j]->tuned = true;
  }
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_batch_engine.reset();
    g_batch_key.clear();
  }
  if (best) *best = bt;
  return HN_OK;
}

hn_status hn_mg_time_kernel(hn_mg* mg, int op, int level, int reps, double* avg_ms, double* bytes) {
  clear_error();
  if (!mg || !avg_ms || reps < 1) return set_error(HN_ERR_ARG, "bad arguments");
  if (op != HN_OP_SPMV && op != HN_OP_DEFECT && op != HN_OP_JACOBI && op != HN_OP_RESTRICT &&
      op != HN_OP_PROLONG_ADD && op != HN_OP_PROLONG_JACOBI)
    return set_error(HN_ERR_ARG, "op must be SPMV, DEFECT, JACOBI, RESTRICT, PROLONG_ADD or PROLONG_JACOBI");
  if (level <= mg->coarse && (op == HN_OP_RESTRICT || op == HN_OP_PROLONG_ADD || op == HN_OP_PROLONG_JACOBI))
    return set_error(HN_ERR_ARG, "transfers need a coarser level");
  if (level < mg->coarse || level > mg->L) return set_error(HN_ERR_ARG, "level out of range");
  HN_TRY(ensure_solo(mg));
  Engine& e = *mg->solo;
  cudaStream_t s = e.stream();
  HN_TRY(e.set_phase(0, PH_CYCLE, 0));
  HN_TRY(e.apply(op, level, PH_CYCLE, s));                   // warm-up
  cudaEvent_t e0, e1;
  HN_CUDA(cudaEventCreate(&e0));
  HN_CUDA(cudaEventCreate(&e1));
  struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
  HN_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) HN_TRY(e.apply(op, level, PH_CYCLE, s));
  HN_CUDA(cudaEventRecord(e1, s));
  HN_CUDA(cudaEventSynchronize(e1));
  float ms = 0.0f;
  HN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *avg_ms = ms / reps;
  if (bytes) {
    const int prec = mg->prm.prec;
    const double vb = prec == P64 ? 8 : 4, bb = prec == P64 ? 8 : (prec == P32 ? 4 : 2);
    // restriction / prolongation per fine node: read r (1) + write coarse (1/4); read coarse
    // (1/4) + read and write x (2)
    const double per = op == HN_OP_SPMV ? 9 * bb + 2 * vb
                     : op == HN_OP_DEFECT ? 9 * bb + 3 * vb
                     : op == HN_OP_RESTRICT ? 1.25 * vb
                     : op == HN_OP_PROLONG_ADD ? 2.25 * vb
                     : op == HN_OP_PROLONG_JACOBI ? 9 * bb + 3.25 * vb + (prec == P64 ? 8 : 0)
                     : 9 * bb + 3 * vb + (prec == P64 ? 8 : 0);
    *bytes = per * (double)N_of(level);
  }
  return HN_OK;
}

long long hn_mg_last_launches(const hn_mg* mg) {
  return (mg && mg->solo) ? mg->solo->last_launches() : 0;
}

int hn_mg_kernel_times(const hn_mg* mg, hn_kernel_time* out, int max) {
  if (!mg || !mg->solo) return 0;
  return mg->solo->kernel_times(out, max);
}

}  // extern "C"
