// Host-side engine: hierarchy construction (Sec. 2.1 assembly per level, Sec. 6.2 multigrid
// hierarchy) and the batch engine that runs the V-cycle schedule of Sec. 6.2 over any set of
// hierarchies as CUDA graphs.
//
// Schedule.  Problems of different finest levels are aligned by absolute level: the launch for
// "level l" covers every problem that has a level l, problems whose finest level is l start their
// cycle there.  One iteration of the schedule is: [FP64 outer defect -> control] -> V cycle over
// levels Lmax..coarse..Lmax -> fine-level residual norm -> control [-> update -> control].  A
// per-problem state machine on the device decides, from the deterministic per-problem norms, what
// each problem does next, so the host never waits inside a solve: a closed-world solve is one
// graph launch whose body is a device-side while loop (graph conditional node) that ends when
// every problem is done.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>

#include "engine.h"

namespace hn {

// ---------------------------------------------------------------------------- error messages
namespace {
thread_local std::string t_err;
}

hn_status set_error(hn_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return st;
}
void clear_error() { t_err.clear(); }
const char* last_error() { return t_err.c_str(); }

hn_status guarded_alloc(size_t bytes, void** base, void** mem) {
  *base = *mem = nullptr;
  char* p = nullptr;
  HN_CUDA(cudaMalloc(reinterpret_cast<void**>(&p), bytes + 2 * kGuardBytes));
  if (kGuardBytes) {
    const cudaError_t e1 = cudaMemset(p, kGuardByte, kGuardBytes);
    const cudaError_t e2 = cudaMemset(p + kGuardBytes + bytes, kGuardByte, kGuardBytes);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      cudaFree(p);
      return set_error(HN_ERR_CUDA, "guard initialisation failed");
    }
  }
  *base = p;
  *mem = p + kGuardBytes;
  return HN_OK;
}

hn_status guards_intact(const void* base, size_t bytes, const char* what) {
  if (!kGuardBytes || !base) return HN_OK;
  std::vector<unsigned char> g(2 * kGuardBytes);
  const char* p = static_cast<const char*>(base);
  HN_CUDA(cudaMemcpy(g.data(), p, kGuardBytes, cudaMemcpyDeviceToHost));
  HN_CUDA(cudaMemcpy(g.data() + kGuardBytes, p + kGuardBytes + bytes, kGuardBytes, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < g.size(); ++i)
    if (g[i] != kGuardByte)
      return set_error(HN_ERR_STATE, "%s: guard byte %s the block overwritten (offset %lld)", what,
                       i < kGuardBytes ? "before" : "after",
                       i < kGuardBytes ? (long long)i - (long long)kGuardBytes : (long long)(i - kGuardBytes));
  return HN_OK;
}

int sm_count() {
  static int cached = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      cached = v;
    if (cached <= 0) cached = 1;
  });
  return cached;
}

// ----------------------------------------------------------------------------- hierarchy
namespace {

struct LevelLayout {
  long long pitch, halo;
};

size_t vec_elems(int l) { return (size_t)(pitch_of(l) + 2 * halo_of(l)); }

template <class F>
void walk_layout(int L, int coarse, int prec, int solver, F&& take) {
  // take(bytes) is called for every piece in construction order
  const size_t vs = prec == P64 ? 8 : 4;
  const size_t bs = prec == P64 ? 8 : (prec == P32 ? 4 : 2);
  for (int l = L; l >= coarse; --l) {
    for (int v = 0; v < 4; ++v) take(vec_elems(l) * vs);
    for (int k = 0; k < 9; ++k) take(vec_elems(l) * bs);
    take(vec_elems(l) * (prec == P64 ? 8 : 4));    // omega / diag
  }
  if (prec != P64) {
    for (int k = 0; k < 9; ++k) take(vec_elems(L) * 8);
    take(vec_elems(L) * 8);
    take(vec_elems(L) * 8);
  } else if (solver == SOLVER_PCG) {               // x, b apart from the cycle's vectors
    take(vec_elems(L) * 8);
    take(vec_elems(L) * 8);
  }
  if (solver == SOLVER_PCG)
    for (int v = 0; v < 3; ++v) take(vec_elems(L) * 8);   // r, p, q
  const long long m = n_of(coarse) * n_of(coarse);   // unknowns of the coarsest level, at most
  take((size_t)(m * m) * 8);
}

// dense inverse of an SPD matrix by Gauss-Jordan elimination with partial pivoting (FP64)
bool invert(std::vector<double>& a, int m) {
  std::vector<double> inv((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) inv[(size_t)i * m + i] = 1.0;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(a[(size_t)r * m + c]) > std::fabs(a[(size_t)piv * m + c])) piv = r;
    if (!(std::fabs(a[(size_t)piv * m + c]) > 0.0)) return false;
    if (piv != c)
      for (int k = 0; k < m; ++k) {
        std::swap(a[(size_t)c * m + k], a[(size_t)piv * m + k]);
        std::swap(inv[(size_t)c * m + k], inv[(size_t)piv * m + k]);
      }
    const double d = a[(size_t)c * m + c];
    for (int k = 0; k < m; ++k) { a[(size_t)c * m + k] /= d; inv[(size_t)c * m + k] /= d; }
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * m + c];
      if (f == 0.0) continue;
      for (int k = 0; k < m; ++k) {
        a[(size_t)r * m + k] -= f * a[(size_t)c * m + k];
        inv[(size_t)r * m + k] -= f * inv[(size_t)c * m + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

struct TempDev {
  void* p = nullptr;
  ~TempDev() { if (p) cudaFree(p); }
};

}  // namespace

size_t hierarchy_bytes(int L, int coarse, int prec, int solver) {
  size_t off = 0;
  walk_layout(L, coarse, prec, solver, [&](size_t b) { off = ((off + 255) & ~size_t(255)) + b; });
  return off + 256;
}

Params params_from(const hn_mg_opts& o) {
  Params p{};
  p.prec = o.prec == HN_PREC_FP64 ? P64 : (o.prec == HN_PREC_FP32_DC ? P32 : P16);
  p.pre = o.pre;
  p.post = o.post;
  p.coarse = o.coarse_L;
  p.max_cycles = o.max_cycles;
  p.max_outer = o.max_outer;
  p.inner_max = o.inner_max;
  p.omega = o.omega;
  p.tol = o.tol;
  p.inner_tol = o.inner_tol;
  p.solver = o.solver == HN_SOLVER_PCG ? SOLVER_PCG : SOLVER_MG;
  p.coarse_cg = o.coarse_solver == HN_COARSE_CG ? 1 : 0;
  return p;
}

hn_status validate_opts(const hn_mg_opts& o, int L) {
  if (o.prec != HN_PREC_FP64 && o.prec != HN_PREC_FP32_DC && o.prec != HN_PREC_FP16BAND_DC)
    return set_error(HN_ERR_ARG, "unknown precision %d", (int)o.prec);
  if (o.coarse_L < HN_MIN_LEVEL || o.coarse_L > kMaxCoarse)
    return set_error(HN_ERR_ARG, "coarse_L must be in [%d, %d]", HN_MIN_LEVEL, kMaxCoarse);
  if (L >= 0 && o.coarse_L > L) return set_error(HN_ERR_ARG, "coarse_L %d > level %d", o.coarse_L, L);
  if (o.pre < 1 || o.post < 0 || ((o.pre + o.post) & 1) || o.pre + o.post > 64)
    return set_error(HN_ERR_ARG, "need pre >= 1, post >= 0, pre + post even and <= 64");
  if (!(o.omega > 0.0 && o.omega < 2.0)) return set_error(HN_ERR_ARG, "omega must be in (0, 2)");
  if (o.dirichlet_sides < 1u || o.dirichlet_sides > 15u)
    return set_error(HN_ERR_ARG, "dirichlet_sides must be a nonzero mask of the 4 sides");
  if (o.solver != HN_SOLVER_MG && o.solver != HN_SOLVER_PCG)
    return set_error(HN_ERR_ARG, "unknown solver %d", (int)o.solver);
  if (o.coarse_solver != HN_COARSE_EXACT && o.coarse_solver != HN_COARSE_CG)
    return set_error(HN_ERR_ARG, "unknown coarse solver %d", (int)o.coarse_solver);
  if (o.solver == HN_SOLVER_PCG && o.pre != o.post)
    return set_error(HN_ERR_ARG, "PCG needs a symmetric cycle (pre == post)");
  if (!(o.tol >= 0.0) || !(o.inner_tol > 0.0 && o.inner_tol < 1.0))
    return set_error(HN_ERR_ARG, "need tol >= 0 and 0 < inner_tol < 1");
  if (o.max_cycles < 1 || o.max_outer < 1 || o.inner_max < 1 || o.max_cycles > 100000 ||
      o.max_outer > 100000 || o.inner_max > 100000)
    return set_error(HN_ERR_ARG, "iteration caps must be in [1, 100000]");
  return HN_OK;
}

namespace {

// the work lists of Engine::set_members: block row y = level (items and chunks), y = kMaxLevel + 1
// the fine list
__global__ void __launch_bounds__(256) k_work_lists(WorkListOut o, const int* slots, const int* fslots,
                                                    const int* foff, int cap) {
  const int l = blockIdx.y;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l <= kMaxLevel) {
    const int n = o.n[l], nt = o.nt[l];
    if (n == 0) return;
    const int cpl = (nt + kChunkTiles - 1) / kChunkTiles;
    for (long long i = i0; i < (long long)n * nt; i += stride) {
      const int k = (int)(i / nt);
      o.items[l][i] = make_int2(slots[(size_t)l * cap + k], (int)(i - (long long)k * nt));
    }
    for (long long j = i0; j < (long long)n * cpl; j += stride) {
      const int k = (int)(j / cpl);
      const int t = (int)(j - (long long)k * cpl) * kChunkTiles;
      o.chunks[l][j] = make_int4(slots[(size_t)l * cap + k], t, min(kChunkTiles, nt - t), 0);
    }
  } else {
    const int nf = o.nfine;
    for (long long i = i0; i < foff[nf]; i += stride) {
      int lo = 0, hi = nf - 1;                      // the member k with foff[k] <= i < foff[k + 1]
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (foff[mid] <= i) lo = mid; else hi = mid - 1;
      }
      o.fine[i] = make_int2(fslots[lo], (int)(i - foff[lo]));
    }
  }
}

}  // namespace

hn_status check_band_inputs(int L, const double* cell_coef, unsigned dirichlet_sides) {
  if (dirichlet_sides < 1u || dirichlet_sides > 15u)
    return set_error(HN_ERR_ARG, "dirichlet_sides %u: need a nonzero mask of the 4 sides", dirichlet_sides);
  if (L < HN_MIN_LEVEL || L > HN_MAX_LEVEL)
    return set_error(HN_ERR_ARG, "level %d outside [%d, %d]", L, HN_MIN_LEVEL, HN_MAX_LEVEL);
  const long long cells = (1LL << L) * (1LL << L);
  if (cell_coef)
    for (long long i = 0; i < cells; ++i)
      if (!(std::isfinite(cell_coef[i]) && cell_coef[i] > 0.0))
        return set_error(HN_ERR_ARG, "cell coefficient %lld is not a positive finite number", i);
  return HN_OK;
}

size_t band_bytes(int L, bool has_coef) {
  size_t bytes = 0;
  auto take = [&](size_t b) { bytes = ((bytes + 255) & ~size_t(255)) + b; };
  for (int k = 0; k < 9; ++k) take((size_t)pitch_of(L) * 8);
  if (has_coef) take((size_t)(1LL << L) * (1LL << L) * 8);
  return bytes + 256;
}

hn_status build_band(int L, const double* cell_coef, unsigned bc, cudaStream_t s, void* mem,
                     hn_band** out) {
  std::unique_ptr<hn_band> A(new hn_band());
  A->L = L;
  HN_CUDA(cudaGetDevice(&A->device));
  A->bc = bc;
  A->n = n_of(L);
  A->N = N_of(L);
  A->pitch = pitch_of(L);
  const long long cells = (1LL << L) * (1LL << L);
  if (mem) A->mem = mem;
  else {
    A->mem_bytes = band_bytes(L, cell_coef != nullptr);
    HN_TRY(guarded_alloc(A->mem_bytes, &A->mem_base, &A->mem));
  }
  Bump b{static_cast<char*>(A->mem), 0};
  BandPtrs64 bp{};
  for (int k = 0; k < 9; ++k) bp.p[k] = A->band[k] = b.take<double>(A->pitch);
  if (cell_coef) {
    A->coef = b.take<double>((size_t)cells);
    HN_CUDA(cudaMemcpyAsync(A->coef, cell_coef, (size_t)cells * 8, cudaMemcpyHostToDevice, s));
  }
  HN_CUDA(launch_assemble(L, A->coef, bp, nullptr, 1.0, (int)A->bc, s));
  HN_CUDA(cudaStreamSynchronize(s));
  *out = A.release();
  return HN_OK;
}

size_t hierarchy_tmp_bytes(int L, int c, int prec, bool has_coef) {
  const long long cells_L = (1LL << L) * (1LL << L);
  const size_t coef_bytes = has_coef ? (size_t)(cells_L + cells_L / 4 + 64) * 8 : 0;
  const size_t tmpband_bytes = (prec != P64 && L > c) ? (size_t)9 * pitch_of(L - 1) * 8 + 9 * 256 : 0;
  return coef_bytes + tmpband_bytes + 1024;
}

hn_status build_hierarchy(const hn_band* A, const hn_mg_opts& o, cudaStream_t s, hn_mg* mg,
                          void* mem, void* scratch, size_t scratch_bytes) {
  const int L = A->L, c = o.coarse_L;
  const Params prm = params_from(o);
  const int prec = prm.prec;
  mg->L = L;
  mg->coarse = c;
  mg->opts = o;
  mg->prm = prm;
  const UnknownRect ur = unknown_rect((int)n_of(c), (int)A->bc);
  mg->m = ur.nx * ur.ny;
  mg->bytes = hierarchy_bytes(L, c, prec, prm.solver);
  if (mem) mg->mem = mem;                       // a block of exactly mg->bytes from the caller
  else HN_TRY(guarded_alloc(mg->bytes, &mg->mem_base, &mg->mem));
  HN_CUDA(cudaMemsetAsync(mg->mem, 0, mg->bytes, s));

  ProblemDev& P = mg->host;
  std::memset(&P, 0, sizeof P);
  P.L = L;
  P.coarse = c;
  P.m = mg->m;
  Bump b{static_cast<char*>(mg->mem), 0};
  const size_t vsz = prec == P64 ? 8 : 4;
  for (int l = L; l >= c; --l) {
    LevelDev& d = P.lev[l];
    d.L = l;
    d.n = (int)n_of(l);
    d.pitch = (int)pitch_of(l);
    d.bc = (int)A->bc;
    const long long H = halo_of(l);
    void* vecs[4];
    for (int v = 0; v < 4; ++v) {
      char* base = b.take<char>(vec_elems(l) * vsz);
      vecs[v] = base + H * vsz;
    }
    d.x[0] = vecs[0];
    d.x[1] = vecs[1];
    d.rhs = vecs[2];
    d.r = vecs[3];
    for (int k = 0; k < 9; ++k) {
      if (prec == P64) d.band[k] = b.take<double>(vec_elems(l)) + H;
      else if (prec == P32) d.band[k] = b.take<float>(vec_elems(l)) + H;
      else d.band[k] = b.take<__half>(vec_elems(l)) + H;
    }
    for (int k = 0; k < 9; ++k) d.scale[k] = 1.0f;
    if (prec == P64) d.wdinv = b.take<double>(vec_elems(l)) + H;
    else d.wdf = b.take<float>(vec_elems(l)) + H;
  }
  if (prec != P64) {
    for (int k = 0; k < 9; ++k) P.band64[k] = b.take<double>(vec_elems(L)) + halo_of(L);
    P.x64 = b.take<double>(vec_elems(L)) + halo_of(L);
    P.b64 = b.take<double>(vec_elems(L)) + halo_of(L);
  } else {
    for (int k = 0; k < 9; ++k) P.band64[k] = static_cast<const double*>(P.lev[L].band[k]);
    if (prm.solver == SOLVER_PCG) {   // the cycle's top vectors are the preconditioner's
      P.x64 = b.take<double>(vec_elems(L)) + halo_of(L);
      P.b64 = b.take<double>(vec_elems(L)) + halo_of(L);
    } else {
      P.x64 = static_cast<double*>(P.lev[L].x[0]);
      P.b64 = static_cast<double*>(P.lev[L].rhs);
    }
  }
  if (prm.solver == SOLVER_PCG) {
    P.r64 = b.take<double>(vec_elems(L)) + halo_of(L);
    P.p64 = b.take<double>(vec_elems(L)) + halo_of(L);
    P.q64 = b.take<double>(vec_elems(L)) + halo_of(L);
  }
  // the coarse inverse (m x m), or for the CG coarse solver the 9 coarse bands (9 N_c); the
  // layout reserves (N_c)^2 >= both
  const size_t cwords = prm.coarse_cg ? (size_t)(9 * N_of(c)) : (size_t)mg->m * mg->m;
  double* cinv = b.take<double>(cwords);
  P.cinv = cinv;
  if (b.off > mg->bytes) return set_error(HN_ERR_STATE, "hierarchy layout overflow");

  // temporaries: coefficients of two consecutive levels, FP64 bands of one coarse level,
  // FP16 scale reduction words (in the caller's scratch when it is large enough)
  const long long cells_L = (1LL << L) * (1LL << L);
  const size_t tmpband_bytes = (prec != P64 && L > c) ? (size_t)9 * pitch_of(L - 1) * 8 + 9 * 256 : 0;
  TempDev tmp;
  const size_t tmp_bytes = hierarchy_tmp_bytes(L, c, prec, A->coef != nullptr);
  char* tmp_base = static_cast<char*>(scratch);
  if (!scratch || scratch_bytes < tmp_bytes) {
    HN_CUDA(cudaMalloc(&tmp.p, tmp_bytes));
    tmp_base = static_cast<char*>(tmp.p);
  }
  Bump tb{tmp_base, 0};
  double* coef_a = A->coef ? tb.take<double>((size_t)cells_L) : nullptr;
  double* coef_b = A->coef ? tb.take<double>((size_t)(cells_L / 4 + 1)) : nullptr;
  double* tband[9] = {};
  if (tmpband_bytes)
    for (int k = 0; k < 9; ++k) tband[k] = tb.take<double>(pitch_of(L - 1));
  unsigned long long* absmax = tb.take<unsigned long long>(9);
  float* dscales = tb.take<float>(9);

  if (A->coef) HN_CUDA(cudaMemcpyAsync(coef_a, A->coef, (size_t)cells_L * 8, cudaMemcpyDeviceToDevice, s));
  const double* coef_cur = A->coef ? coef_a : nullptr;
  std::vector<double> coarse64((size_t)9 * pitch_of(c));
  for (int l = L; l >= c; --l) {
    LevelDev& d = P.lev[l];
    // FP64 bands of level l
    BandPtrs64 b64{};
    if (l == L) {
      double* dst[9];
      for (int k = 0; k < 9; ++k) dst[k] = const_cast<double*>(P.band64[k]);
      for (int k = 0; k < 9; ++k)
        HN_CUDA(cudaMemcpyAsync(dst[k], A->band[k], (size_t)pitch_of(L) * 8, cudaMemcpyDeviceToDevice, s));
      for (int k = 0; k < 9; ++k) b64.p[k] = dst[k];
      if (prec == P64) {
        // the fine level also needs omega / diag: reassemble writes identical bands plus it
        HN_CUDA(launch_assemble(l, coef_cur, b64, const_cast<double*>(d.wdinv), o.omega, (int)A->bc, s));
      }
    } else if (prec == P64) {
      for (int k = 0; k < 9; ++k) b64.p[k] = static_cast<double*>(const_cast<void*>(d.band[k]));
      HN_CUDA(launch_assemble(l, coef_cur, b64, const_cast<double*>(d.wdinv), o.omega, (int)A->bc, s));
    } else {
      for (int k = 0; k < 9; ++k) b64.p[k] = tband[k];
      HN_CUDA(launch_assemble(l, coef_cur, b64, nullptr, o.omega, (int)A->bc, s));
    }
    BandPtrs64c src{};
    for (int k = 0; k < 9; ++k) src.p[k] = b64.p[k];
    if (prec == P32) {
      BandPtrs32 dst{};
      for (int k = 0; k < 9; ++k) dst.p[k] = static_cast<float*>(const_cast<void*>(d.band[k]));
      HN_CUDA(launch_band_to_f32(l, src, dst, s));
    } else if (prec == P16) {
      BandPtrs16 dst{};
      for (int k = 0; k < 9; ++k) dst.p[k] = static_cast<__half*>(const_cast<void*>(d.band[k]));
      HN_CUDA(launch_band_to_f16(l, src, absmax, dst, dscales, s));
      float hs[9];
      HN_CUDA(cudaMemcpyAsync(hs, dscales, sizeof hs, cudaMemcpyDeviceToHost, s));
      HN_CUDA(cudaStreamSynchronize(s));
      for (int k = 0; k < 9; ++k) d.scale[k] = hs[k];
    }
    if (prec != P64) HN_CUDA(launch_wdf(l, prec, d.band, d.scale, o.omega, const_cast<float*>(d.wdf), s));
    if (l == c) {
      for (int k = 0; k < 9; ++k)
        HN_CUDA(cudaMemcpyAsync(coarse64.data() + (size_t)k * pitch_of(c), src.p[k],
                                (size_t)pitch_of(c) * 8, cudaMemcpyDeviceToHost, s));
    }
    if (l > c && coef_cur) {
      double* next = (coef_cur == coef_a) ? coef_b : coef_a;
      HN_CUDA(launch_coarsen_coef(l, coef_cur, next, s));
      coef_cur = next;
    }
  }
  HN_CUDA(cudaStreamSynchronize(s));
  // exact coarse solver: inverse of the coarsest operator restricted to its unknowns (the
  // rectangle of nodes that are not Dirichlet), row-major
  {
    const long long n = n_of(c), pc = pitch_of(c);
    const int m = mg->m;
    std::vector<double> a((size_t)m * m, 0.0);
    for (long long iy = ur.y0; iy < ur.y0 + ur.ny; ++iy)
      for (long long ix = ur.x0; ix < ur.x0 + ur.nx; ++ix) {
        const long long I = (iy - ur.y0) * ur.nx + (ix - ur.x0);
        for (int k = 0; k < 9; ++k) {
          const long long jx = ix + (k % 3 - 1), jy = iy + (k / 3 - 1);
          if (jx < ur.x0 || jy < ur.y0 || jx >= ur.x0 + ur.nx || jy >= ur.y0 + ur.ny) continue;
          const long long J = (jy - ur.y0) * ur.nx + (jx - ur.x0);
          a[(size_t)(I * m + J)] = coarse64[(size_t)k * pc + iy * n + ix];
        }
      }
    if (!invert(a, m)) return set_error(HN_ERR_STATE, "coarse matrix is singular");
    if (prm.coarse_cg) {
      // CG works on the 9 FP64 bands of the level, band k at k * N_c
      const long long Nc = n * n;
      std::vector<double> cb((size_t)(9 * Nc));
      for (int k = 0; k < 9; ++k)
        for (long long i = 0; i < Nc; ++i) cb[(size_t)(k * Nc + i)] = coarse64[(size_t)k * pc + i];
      a.swap(cb);
    }
    HN_CUDA(cudaMemcpyAsync(cinv, a.data(), a.size() * 8, cudaMemcpyHostToDevice, s));
    HN_CUDA(cudaStreamSynchronize(s));
  }
  return HN_OK;
}

// ------------------------------------------------------------------------------- engine
Engine::~Engine() {
  destroy_graphs();
  for (auto& m : marks_) { cudaEventDestroy(m.b); cudaEventDestroy(m.e); }
  if (upEv_) cudaEventSynchronize(upEv_);
  if (memBase_) cudaFree(memBase_);
  if (hActive_) cudaFreeHost(hActive_);
  if (hStage_) cudaFreeHost(hStage_);
  if (hLists_) cudaFreeHost(hLists_);
  if (upEv_) cudaEventDestroy(upEv_);
}

void Engine::destroy_graphs() {
  if (gSolve_) cudaGraphExecDestroy(gSolve_);
  if (gInit_) cudaGraphExecDestroy(gInit_);
  if (gIter_) cudaGraphExecDestroy(gIter_);
  gSolve_ = gInit_ = gIter_ = nullptr;
  graphsValid_ = false;
}

int Engine::grid_for(long long tiles) const {
  const long long warps_per_cta = 8;
  long long g = (tiles + warps_per_cta - 1) / warps_per_cta;
  if (g < 1) g = 1;
  if (g > maxGrid_) g = maxGrid_;
  return (int)g;
}

hn_status Engine::create(const Params& prm, int cap, int Lmax, const std::vector<long long>& tiles_cap,
                         long long fine_cap, cudaStream_t s) {
  prm_ = prm;
  cap_ = cap;
  Lmax_ = Lmax;
  s_ = s;
  {
    static std::once_flag once;
    static cudaError_t prep = cudaSuccess;
    std::call_once(once, [] { prep = prepare_kernels(); });
    HN_CUDA(prep);
  }
  maxGrid_ = sm_count() * 8;     // each launch is clamped to its kernel's resident blocks
  size_t bytes = 0;
  auto take = [&](size_t b) { bytes = ((bytes + 255) & ~size_t(255)) + b; };
  take(sizeof(ProblemDev) * cap);
  take(sizeof(ProbState) * cap);
  take(sizeof(int) * cap);
  take(sizeof(int) * (kMaxLevel + 2));
  for (int l = 0; l <= kMaxLevel; ++l) {
    itemCap_[l] = l < (int)tiles_cap.size() ? tiles_cap[l] : 0;
    take(sizeof(int2) * (size_t)std::max<long long>(itemCap_[l], 1));
    chunkCap_[l] = itemCap_[l] > 0 ? itemCap_[l] / kChunkTiles + cap + 1 : 0;
    take(sizeof(int4) * (size_t)std::max<long long>(chunkCap_[l], 1));
  }
  take(sizeof(int) * (kMaxLevel + 1));
  take(sizeof(int) * 4);
  fineCap_ = fine_cap;
  take(sizeof(int2) * (size_t)std::max<long long>(fine_cap, 1));
  take(sizeof(double) * (size_t)std::max<long long>(fine_cap, 1));
  take(sizeof(double) * (size_t)std::max<long long>(fine_cap, 1));
  take(sizeof(unsigned));
  take(sizeof(unsigned) * 4);
  take(sizeof(unsigned long long));
  // the control kernel's groups: as many as the largest problem's norm sum has
  const int ctl_groups = (int)((pitch_of(Lmax) / kTile + kSumGroup - 1) / kSumGroup);
  take(sizeof(double) * (size_t)cap * ctl_groups);
  take(sizeof(unsigned) * (size_t)cap);
  take(sizeof(int) * plan_ints());
  take(sizeof(TileList) * (kMaxLevel + 1));
  take(sizeof(unsigned long long) * 3);
  take(sizeof(unsigned));
  bytes += 256;
  memBytes_ = bytes;
  HN_TRY(guarded_alloc(bytes, &memBase_, &mem_));
  HN_CUDA(cudaMemsetAsync(mem_, 0, bytes, s_));
  Bump b{static_cast<char*>(mem_), 0};
  dP_ = b.take<ProblemDev>(cap);
  dS_ = b.take<ProbState>(cap);
  dFineOff_ = b.take<int>(cap);
  dCounts_ = b.take<int>(kMaxLevel + 2);
  for (int l = 0; l <= kMaxLevel; ++l) {
    dItems_[l] = b.take<int2>((size_t)std::max<long long>(itemCap_[l], 1));
    dChunks_[l] = b.take<int4>((size_t)std::max<long long>(chunkCap_[l], 1));
  }
  dChunkCounts_ = b.take<int>(kMaxLevel + 1);
  dErr_ = b.take<int>(4);
  dFine_ = b.take<int2>((size_t)std::max<long long>(fine_cap, 1));
  double* part = b.take<double>((size_t)std::max<long long>(fine_cap, 1));
  double* part2 = b.take<double>((size_t)std::max<long long>(fine_cap, 1));
  unsigned* iter = b.take<unsigned>(1);
  dTaken_ = b.take<unsigned>(4);
  dLaunches_ = b.take<unsigned long long>(1);
  double* gsum = b.take<double>((size_t)cap * ctl_groups);
  unsigned* gticket = b.take<unsigned>((size_t)cap);
  dPlan_ = b.take<int>(plan_ints());
  dLists_ = b.take<TileList>(kMaxLevel + 1);
  dBar_ = b.take<unsigned long long>(3);
  unsigned* ticket = b.take<unsigned>(1);
  HN_CUDA(cudaHostAlloc(&hStage_, stage_bytes(), cudaHostAllocDefault));
  HN_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&hLists_), sizeof(TileList) * (kMaxLevel + 1),
                        cudaHostAllocDefault));
  HN_CUDA(cudaEventCreateWithFlags(&upEv_, cudaEventDisableTiming));
  HN_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&hActive_), sizeof(unsigned), cudaHostAllocMapped));
  *hActive_ = 0;
  unsigned* dActive = nullptr;
  HN_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&dActive), hActive_, 0));
  E_.P = dP_;
  E_.S = dS_;
  E_.fine_off = dFineOff_;
  E_.partial = part;
  E_.partial2 = part2;
  E_.nprob = cap;
  E_.prm = prm;
  E_.active_host = dActive;
  E_.iter = iter;
  E_.pdl = tune_.pdl;
  E_.err = dErr_;
  E_.staged = tune_.staged;
  E_.dsm = tune_.dsm;
  E_.ctl_groups = ctl_groups;
  E_.gsum = gsum;
  E_.gticket = gticket;
  E_.gbar = dBar_;
  E_.ticket = ticket;
  E_.iter_limit = (unsigned)(prm.max_cycles + prm.max_outer + 8);
  for (int l = 0; l <= kMaxLevel; ++l) {
    lists_[l] = TileList{dItems_[l], dCounts_ + l, dChunks_[l], dChunkCounts_ + l, (int)chunkCap_[l]};
    grid_[l] = grid_for(itemCap_[l]);
  }
  fine_ = TileList{dFine_, dCounts_ + kMaxLevel + 1};
  fineGrid_ = grid_for(fine_cap);
  hCounts_.assign(kMaxLevel + 2, 0);
  members_.assign(cap, nullptr);
  return HN_OK;
}

hn_status Engine::set_members(const std::vector<hn_mg*>& slots) {
  if ((int)slots.size() > cap_) return set_error(HN_ERR_ARG, "too many problems for the engine");
  // The work lists hold, per level, the (problem, tile) pairs of every member having that level,
  // members in slot order; the chunk lists the same in chunks of kChunkTiles tiles; the fine list
  // each member's tiles of its finest level.  Every member contributes the same tiles to a level,
  // so the host only ranks the members (O(slots)) and k_work_lists writes the pairs.
  HN_CUDA(cudaEventSynchronize(upEv_));        // the previous upload has left the staging area
  char* stage = static_cast<char*>(hStage_);
  int* h_counts = reinterpret_cast<int*>(stage);                 // kMaxLevel + 2
  int* h_ccounts = h_counts + (kMaxLevel + 2);                   // kMaxLevel + 1
  int* h_fine_off = h_ccounts + (kMaxLevel + 1);                 // cap
  int* h_plan = h_fine_off + cap_;                               // plan_ints()
  int* h_slots = h_plan;                                         // (kMaxLevel + 1) x cap
  int* h_fslots = h_slots + (size_t)(kMaxLevel + 1) * cap_;      // cap
  int* h_foff = h_fslots + cap_;                                 // cap + 1
  ProblemDev* h_probs = reinterpret_cast<ProblemDev*>(stage + stage_probs_off());
  std::memset(h_probs, 0, sizeof(ProblemDev) * cap_);
  std::memset(h_fine_off, 0, sizeof(int) * cap_);
  WorkListOut o{};
  int nfine = 0;
  long long fine_total = 0;
  for (int p = 0; p < (int)slots.size(); ++p) {
    hn_mg* mg = slots[p];
    if (!mg) continue;
    if (mg->L > Lmax_) return set_error(HN_ERR_ARG, "level %d above the engine's %d", mg->L, Lmax_);
    h_probs[p] = mg->host;
    for (int l = mg->coarse; l <= mg->L; ++l) h_slots[(size_t)l * cap_ + o.n[l]++] = p;
    h_fine_off[p] = (int)fine_total;
    h_fslots[nfine] = p;
    h_foff[nfine++] = (int)fine_total;
    fine_total += pitch_of(mg->L) / kTile;
  }
  h_foff[nfine] = (int)fine_total;
  o.nfine = nfine;
  long long most = fine_total;
  for (int l = 0; l <= kMaxLevel; ++l) {
    o.nt[l] = (int)(pitch_of(l) / kTile);
    const long long items = (long long)o.n[l] * o.nt[l];
    const long long chunks = (long long)o.n[l] * ((o.nt[l] + kChunkTiles - 1) / kChunkTiles);
    if (items > itemCap_[l] || chunks > chunkCap_[l])
      return set_error(HN_ERR_ARG, "work list of level %d exceeds the engine capacity", l);
    hCounts_[l] = h_counts[l] = (int)items;
    h_ccounts[l] = (int)chunks;
    o.items[l] = dItems_[l];
    o.chunks[l] = dChunks_[l];
    most = std::max(most, items);
  }
  if (fine_total > fineCap_) return set_error(HN_ERR_ARG, "fine work list exceeds capacity");
  hCounts_[kMaxLevel + 1] = h_counts[kMaxLevel + 1] = (int)fine_total;
  o.fine = dFine_;
  HN_CUDA(cudaMemcpyAsync(dCounts_, h_counts, sizeof(int) * (kMaxLevel + 2), cudaMemcpyHostToDevice, s_));
  HN_CUDA(cudaMemcpyAsync(dChunkCounts_, h_ccounts, sizeof(int) * (kMaxLevel + 1), cudaMemcpyHostToDevice, s_));
  HN_CUDA(cudaMemcpyAsync(dFineOff_, h_fine_off, sizeof(int) * cap_, cudaMemcpyHostToDevice, s_));
  HN_CUDA(cudaMemcpyAsync(dPlan_, h_plan, sizeof(int) * plan_ints(), cudaMemcpyHostToDevice, s_));
  HN_CUDA(cudaMemcpyAsync(dP_, h_probs, sizeof(ProblemDev) * cap_, cudaMemcpyHostToDevice, s_));
  if (most > 0) {
    const int gx = (int)std::min<long long>((most + 255) / 256, 1024);
    k_work_lists<<<dim3((unsigned)gx, kMaxLevel + 2), 256, 0, s_>>>(
        o, dPlan_, dPlan_ + (size_t)(kMaxLevel + 1) * cap_, dPlan_ + (size_t)(kMaxLevel + 2) * cap_, cap_);
    HN_CUDA(cudaGetLastError());
  }
  HN_CUDA(cudaEventRecord(upEv_, s_));
  // an engine of one problem passes its descriptors to the kernels by value (captured into its
  // graphs, which therefore must be captured again when its member changes)
  if (cap_ == 1) graphsValid_ = false;
  for (int l = 0; l <= kMaxLevel; ++l) {
    TileList& t = lists_[l];
    t.solo_tiles = 0;
    t.solo_L = 0;
    t.solo_d = t.solo_c = t.solo_f = LevelDev{};
    if (cap_ != 1 || slots.empty() || !slots[0]) continue;
    const ProblemDev& P = slots[0]->host;
    if (l < P.coarse || l > P.L) continue;
    t.solo_tiles = (int)(pitch_of(l) / kTile);
    t.solo_L = P.L;
    t.solo_d = P.lev[l];
    if (l > P.coarse) t.solo_c = P.lev[l - 1];
    if (l < P.L) t.solo_f = P.lev[l + 1];
  }
  // the persistent kernels read the tile lists (with the one-problem descriptors) from device
  // memory; the staging copy is free again once the previous upload finished (event above)
  std::memcpy(hLists_, lists_, sizeof(TileList) * (kMaxLevel + 1));
  HN_CUDA(cudaMemcpyAsync(dLists_, hLists_, sizeof(TileList) * (kMaxLevel + 1), cudaMemcpyHostToDevice, s_));
  HN_CUDA(cudaEventRecord(upEv_, s_));
  members_ = slots;
  members_.resize(cap_, nullptr);
  unsigned mask = 0;
  for (hn_mg* mg : members_)
    if (mg) mask |= 1u << mg->L;
  if (mask != topMask_ && !topMaskAll_) graphsValid_ = false;
  topMask_ = mask;
  return HN_OK;
}

hn_status Engine::start(const std::vector<int>& slots, const std::vector<int>& have_guess) {
  for (size_t q = 0; q < slots.size(); ++q) {
    ProbState st;
    std::memset(&st, 0, sizeof st);
    st.phase = PH_INIT;
    st.status = HN_PENDING;
    const int g = q < have_guess.size() ? have_guess[q] : 0;
    st.zero_top = g ? 0 : 1;
    st.x_zero = g ? 0 : 1;
    st.s = 1.0;
    st.inv_s = 1.0;
    HN_CUDA(cudaMemcpyAsync(dS_ + slots[q], &st, sizeof st, cudaMemcpyHostToDevice, s_));
  }
  // the iteration counter restarts with every closed-world solve (serving keeps counting and
  // relies on per-problem caps; its limit is set out of reach)
  HN_CUDA(cudaMemsetAsync(E_.iter, 0, sizeof(unsigned), s_));
  HN_CUDA(cudaMemsetAsync(dErr_, 0, sizeof(int) * 4, s_));
  HN_CUDA(cudaMemsetAsync(dBar_, 0, sizeof(unsigned long long) * 3, s_));
  HN_CUDA(cudaMemsetAsync(E_.ticket, 0, sizeof(unsigned), s_));
  // mirrors of the IF values as the closed-world graph sets them at its launch
  static const unsigned taken0[4] = {0u, 1u, 0u, 0u};
  HN_CUDA(cudaMemcpyAsync(dTaken_, taken0, sizeof taken0, cudaMemcpyHostToDevice, s_));
  HN_CUDA(cudaMemsetAsync(dLaunches_, 0, sizeof(unsigned long long), s_));
  return HN_OK;
}

hn_status Engine::set_phase(int slot, int phase, int zero_top) {
  ProbState st;
  std::memset(&st, 0, sizeof st);
  st.phase = phase;
  st.status = HN_PENDING;
  st.zero_top = zero_top;
  st.x_zero = zero_top;
  st.s = 1.0;
  st.inv_s = 1.0;
  HN_CUDA(cudaMemcpyAsync(dS_ + slot, &st, sizeof st, cudaMemcpyHostToDevice, s_));
  return HN_OK;
}

long long Engine::launch_bytes(int cls, int level) const {
  // algorithmic DRAM bytes of one launch: nodes of the level summed over members x bytes per node
  long long nodes = 0;
  for (hn_mg* mg : members_) {
    if (!mg) continue;
    const int lv = level < 0 ? mg->L : level;
    if (lv < mg->coarse || lv > mg->L) continue;
    nodes += N_of(lv);
  }
  const int prec = prm_.prec;
  const double vb = prec == P64 ? 8 : 4;
  const double bb = prec == P64 ? 8 : (prec == P32 ? 4 : 2);
  const double wd = prec == P64 ? 8 : 0;   // stored omega/diag read by Jacobi (FP64 hierarchy only)
  double per = 0;
  switch (cls) {
    case KC_JACOBI: per = 9 * bb + 3 * vb + wd; break;
    case KC_JACOBI_FIRST: per = 9 * bb + 2 * vb + (prec == P64 ? 8 : 4); break;   // fused from x = 0
    case KC_DEFECT: per = 9 * bb + 3 * vb; break;
    case KC_CHECK: per = 9 * bb + 2 * vb; break;
    case KC_RESTRICT: per = 1.25 * vb; break;                   // per fine node
    case KC_PROLONG: per = 2.25 * vb; break;                    // per fine node
    case KC_PROLONG_JACOBI: per = 9 * bb + 3.25 * vb + wd; break; // Jacobi + coarse reads
    case KC_OUTER_DEFECT: per = 72 + 8 + 8 + vb; break;
    case KC_UPDATE: per = 4 + 8 + 8; break;
    case KC_PCG_Q: per = 72 + 8 + 8; break;                    // bands, p; write q
    case KC_PCG_X: per = 4 * 8 + 2 * 8 + vb; break;            // x, r, p, q; write x, r, rhs
    case KC_PCG_DOT: per = 8 + vb; break;                       // r, z
    case KC_PCG_P: per = vb + 8 + 8; break;                     // z, p; write p
    case KC_SWEEP_DOWN: {
      // the fused down sweep: bands, rhs and either omega / D (from a zero iterate) or the first
      // iterate (the problem's own finest level), the second iterate written, the coarse rhs
      long long sum = 0;
      for (hn_mg* mg : members_) {
        if (!mg || level > mg->L || level <= mg->coarse) continue;
        const bool own = level == mg->L && prm_.solver != SOLVER_PCG;
        const double pn = 9 * bb + vb + (own ? vb + wd : (prec == P64 ? 8 : 4)) + vb + 0.25 * vb;
        sum += (long long)(pn * (double)N_of(level));
      }
      return sum;
    }
    case KC_SWEEP_UP: per = 9 * bb + vb + 0.25 * vb + vb + wd + vb; break;   // bands, x, e_c, rhs; write
    case KC_MID_DOWN:
    case KC_MID_UP: {
      // the persistent kernels: the sum of their steps' bytes over levels T+1..level (the top
      // level of a problem counted with two full smoothing steps, the levels below it with the
      // two steps fused from a zero iterate)
      const int T = std::max(tune_.tail_level, prm_.coarse);
      long long sum = 0;
      for (int l = T + 1; l <= level; ++l)
        sum += cls == KC_MID_DOWN
                   ? launch_bytes(KC_JACOBI_FIRST, l) + launch_bytes(KC_DEFECT, l) + launch_bytes(KC_RESTRICT, l)
                   : launch_bytes(KC_PROLONG, l) + prm_.post * launch_bytes(KC_JACOBI, l);
      if (cls == KC_MID_DOWN)
        for (hn_mg* mg : members_)
          if (mg && mg->L > T && mg->L <= level)
            sum += (long long)((2 * (9 * bb + 3 * vb + wd) - (9 * bb + 2 * vb + (prec == P64 ? 8 : 4))) *
                               (double)N_of(mg->L));
      return sum;
    }
    default: per = 0; break;
  }
  return (long long)(per * (double)nodes);
}

// events around one launch of a profiled (directly issued) iteration
hn_status Engine::mark(cudaStream_t s, int cls, int level, bool begin) {
  if (!profiling_) return HN_OK;
  if (begin) {
    cudaEvent_t e;
    HN_CUDA(cudaEventCreate(&e));
    HN_CUDA(cudaEventRecord(e, s));
    openBegin_.push_back(e);
  } else {
    cudaEvent_t e;
    HN_CUDA(cudaEventCreate(&e));
    HN_CUDA(cudaEventRecord(e, s));
    Mark m{openBegin_.back(), e, cls, level, launch_bytes(cls, level)};
    openBegin_.pop_back();
    marks_.push_back(m);
  }
  return HN_OK;
}

// A launch right after an IF node, or first in an IF body, has no kernel before it to overlap
// with: it goes without programmatic dependent launch.
#define HN_LAUNCH(cls, level, call)                 \
  do {                                              \
    HN_TRY(mark(s, cls, level, true));              \
    const int pdl_saved = E_.pdl;                   \
    if (pdlBarrier_) E_.pdl = 0;                    \
    const cudaError_t launch_err = (call);          \
    E_.pdl = pdl_saved;                             \
    pdlBarrier_ = false;                            \
    HN_CUDA(launch_err);                            \
    ++counting_;                                    \
    HN_TRY(mark(s, cls, level, false));             \
  } while (0)
#define HN_LAUNCH0(call)                            \
  do {                                              \
    const int pdl_saved = E_.pdl;                   \
    if (pdlBarrier_) E_.pdl = 0;                    \
    const cudaError_t launch_err = (call);          \
    E_.pdl = pdl_saved;                             \
    pdlBarrier_ = false;                            \
    HN_CUDA(launch_err);                            \
    ++counting_;                                    \
  } while (0)

hn_status Engine::open_if(cudaStream_t& s, int which) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  HN_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &ed, &nd));
  if (cst != cudaStreamCaptureStatusActive) return set_error(HN_ERR_STATE, "IF node outside a capture");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  const CondDev& cdv = E_.prm.cond;               // the handles of the half being captured
  cp.conditional.handle = which == 0 ? cdv.h_cycle : (which == 1 ? cdv.h_outer : cdv.h_update);
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  HN_CUDA(cudaGraphAddNode(&node, g, deps, ed, nd, &cp));
  HN_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  HN_CUDA(cudaStreamBeginCaptureToGraph(aux_, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  s = aux_;
  pdlBarrier_ = true;
  return HN_OK;
}

hn_status Engine::close_if(cudaStream_t& s, cudaStream_t outer) {
  cudaGraph_t body = nullptr;
  HN_CUDA(cudaStreamEndCapture(aux_, &body));
  s = outer;
  pdlBarrier_ = true;
  return HN_OK;
}

int Engine::mid_top() const {
  const int T = std::max(tune_.tail_level, prm_.coarse);
  if (tune_.mid <= T || tune_.staged || tune_.fuse_up) return T;
  return std::min(Lmax_, tune_.mid);
}

bool Engine::sweep_on() const {
  const int T = std::max(tune_.tail_level, prm_.coarse);
  return tune_.sweep && cap_ == 1 && prm_.pre == 2 && prm_.post == 2 && !tune_.staged && mid_top() <= T;
}

// Levels in fused sweeps.  sweep 1: the levels below the finest up to kSweepMaxLevel, where a step
// is bound by latency (a sweep's tile takes several dependent phases, each about one memory
// latency; larger levels stream enough data that the halo re-reads cost more than the launches
// saved: measured at L = 10..12).  sweep 2: every level above the tail, the finest one's down part
// included.
bool Engine::sweep_level(int l) const {
  if (!sweep_on()) return false;
  return tune_.sweep == 2 || (!is_top(l) && l <= kSweepMaxLevel);
}

hn_status Engine::issue_vcycle(cudaStream_t s0, int want) {
  const int c = prm_.coarse, pre = prm_.pre, post = prm_.post;
  const int T = std::max(tune_.tail_level, c);
  cudaStream_t s = s0;
  bool opened = false;
  int c0 = 0;
  // inside the closed-world loop the rest of the cycle after the first lagged check is an IF body
  auto after_check = [&]() -> hn_status {
    if (!cond_on(0) || opened) return HN_OK;
    HN_TRY(open_if(s, 0));
    opened = true;
    c0 = counting_;
    return HN_OK;
  };
  const int M = mid_top();                 // levels T+1..M: the persistent kernels
  for (int l = Lmax_; l > std::max(T, M); --l) {
    // a finest level: lagged check (the PCG preconditioner's cycle has none)
    const bool top = prm_.solver != SOLVER_PCG && is_top(l);
    if (sweep_level(l) && !top) {
      // a zero iterate: both smoothing steps, the defect and the restriction in one launch
      HN_LAUNCH(KC_SWEEP_DOWN, l, launch_sweep_down(E_, lists_[l], l, want, 0, s));
      continue;
    }
    // an engine of one problem takes the check inside the first smoothing step when the norm is
    // one group of partials (the register-path kernel; saves the control launch)
    const bool fuse = top && cap_ == 1 && !tune_.staged && pitch_of(l) / kTile <= kSumGroup;
    if (pre >= 2) {
      HN_LAUNCH(KC_JACOBI_FIRST, l, launch_pre12(E_, lists_[l], l, want, grid_[l], s, fuse ? 1 : 0));
      if (top) {
        if (!fuse) HN_LAUNCH(KC_CONTROL, l, launch_control(E_, CTRL_PRE, s, l));
        HN_TRY(after_check());
      }
      if (sweep_level(l)) {
        // the second step, the defect and the restriction in one launch
        HN_LAUNCH(KC_SWEEP_DOWN, l, launch_sweep_down(E_, lists_[l], l, want, 1, s));
        continue;
      }
      if (!pre_fuses(prm_.prec) || top)
        HN_LAUNCH(KC_JACOBI, l, launch_pre2b(E_, lists_[l], l, want, grid_[l], s));
      for (int sw = 3; sw <= pre; ++sw)
        HN_LAUNCH(KC_JACOBI, l, launch_jacobi(E_, lists_[l], l, want, (sw - 1) & 1, 0, grid_[l], s));
    } else {
      HN_LAUNCH(KC_JACOBI_FIRST, l, launch_jacobi(E_, lists_[l], l, want, 0, 1, grid_[l], s, fuse ? 1 : 0));
      if (top) {
        if (!fuse) HN_LAUNCH(KC_CONTROL, l, launch_control(E_, CTRL_PRE, s, l));
        HN_TRY(after_check());
      }
    }
    HN_LAUNCH(KC_DEFECT, l, launch_defect(E_, lists_[l], l, want, pre & 1, grid_[l], s));
    HN_LAUNCH(KC_RESTRICT, l, launch_restrict(E_, lists_[l - 1], l, want, grid_[l - 1], s));
  }
  if (M > T) HN_LAUNCH(KC_MID_DOWN, M, launch_mid(E_, dLists_, M, T, want, 0, s));
  HN_LAUNCH(KC_TAIL, T, launch_tail(E_, T, want, tune_.cluster, s));
  if (M > T) HN_LAUNCH(KC_MID_UP, M, launch_mid(E_, dLists_, M, T, want, 1, s));
  int e_sel = 0;                           // buffer of the coarse iterate (the tail's: 0)
  for (int l = std::max(T, M) + 1; l <= Lmax_; ++l) {
    if (sweep_level(l) && !is_top(l)) {
      // prolongation and both post-smoothing steps in one launch; the result in buffer 1 (a
      // problem's own finest level keeps its iterate in buffer 0)
      HN_LAUNCH(KC_SWEEP_UP, l, launch_sweep_up(E_, lists_[l], l, want, e_sel, s));
      e_sel = 1;
      continue;
    }
    int sw = 1;
    if (tune_.fuse_up && post >= 1) {
      // prolongation and the first post-smoothing step in one pass
      HN_LAUNCH(KC_PROLONG_JACOBI, l, launch_prolong_jacobi(E_, lists_[l], l, want, (pre & 1) | (e_sel << 1), grid_[l], s));
      sw = 2;
    } else {
      HN_LAUNCH(KC_PROLONG, l, launch_prolong(E_, lists_[l], l, want, (pre & 1) | (e_sel << 1), grid_[l], s));
    }
    e_sel = 0;
    for (; sw <= post; ++sw)
      HN_LAUNCH(KC_JACOBI, l, launch_jacobi(E_, lists_[l], l, want, (pre + sw - 1) & 1, 0, grid_[l], s));
  }
  if (opened) {
    E_.prm.cond.n_cycle = (unsigned)(counting_ - c0);
    HN_TRY(close_if(s, s0));
  }
  return HN_OK;
}

hn_status Engine::issue_init(cudaStream_t s, cudaGraphConditionalHandle h, int use_h) {
  HN_LAUNCH0(launch_boundary_check(E_, s));
  HN_LAUNCH0(launch_norm_b(E_, fine_, fineGrid_, s));
  HN_LAUNCH0(launch_control(E_, CTRL_INIT, s));
  if (prm_.solver == SOLVER_PCG) {
    // the initial residual r = b - A x and its check (then the first cycle preconditions it)
    HN_LAUNCH0(launch_outer_defect(E_, fine_, fineGrid_, s));
    HN_LAUNCH0(launch_control(E_, CTRL_OUTER, s));
  }
  HN_LAUNCH0(launch_summary(E_, h, use_h, 0, s));
  return HN_OK;
}

hn_status Engine::issue_iteration(cudaStream_t s0, cudaGraphConditionalHandle h, int use_h) {
  cudaStream_t s = s0;
  const int start = counting_;
  if (prm_.solver == SOLVER_PCG && fuse_control()) {
    // the same steps with each control step in the last block of the kernel before it, and the
    // summary in the last one's
    HN_TRY(issue_vcycle(s, PH_PRECOND));
    HN_LAUNCH(KC_PCG_DOT, -1, launch_pcg_dot(E_, fine_, fineGrid_, s, 1));
    HN_LAUNCH(KC_PCG_P, -1, launch_pcg_p(E_, fine_, fineGrid_, s, 1));
    HN_LAUNCH(KC_PCG_Q, -1, launch_pcg_q(E_, fine_, fineGrid_, s, 1));
    if (condCapture_) {
      const CondDev& cd = E_.prm.cond;
      E_.prm.cond.n_base = (unsigned)(counting_ + 1 - start) - cd.n_cycle - cd.n_outer - cd.n_update;
    }
    HN_LAUNCH(KC_PCG_X, -1, launch_pcg_x(E_, fine_, fineGrid_, s, 1, h, use_h));
    return HN_OK;
  } else if (prm_.solver == SOLVER_PCG) {
    // z = M r (one cycle from zero), rho' = (r, z), beta, p = z + beta p, then the CG step
    // q = A p, alpha, x += alpha p, r -= alpha q, and its check
    HN_TRY(issue_vcycle(s, PH_PRECOND));
    HN_LAUNCH(KC_PCG_DOT, -1, launch_pcg_dot(E_, fine_, fineGrid_, s));
    HN_LAUNCH(KC_CONTROL, -1, launch_control(E_, CTRL_PCG_BETA, s));
    HN_LAUNCH(KC_PCG_P, -1, launch_pcg_p(E_, fine_, fineGrid_, s));
    HN_LAUNCH(KC_CONTROL, -1, launch_control(E_, CTRL_POST, s));
    HN_LAUNCH(KC_PCG_Q, -1, launch_pcg_q(E_, fine_, fineGrid_, s));
    HN_LAUNCH(KC_CONTROL, -1, launch_control(E_, CTRL_PCG_ALPHA, s));
    HN_LAUNCH(KC_PCG_X, -1, launch_pcg_x(E_, fine_, fineGrid_, s));
    HN_LAUNCH(KC_CONTROL, -1, launch_control(E_, CTRL_OUTER, s));
  } else if (prm_.prec == P64) {
    HN_TRY(issue_vcycle(s, PH_CYCLE));
  } else if (fuse_control()) {
    // an engine of one problem: the outer control step inside the outer defect, the control step
    // after the update and the iteration's summary inside the update (their last blocks)
    HN_LAUNCH(KC_OUTER_DEFECT, -1, launch_outer_defect(E_, fine_, fineGrid_, s, 1));
    HN_TRY(issue_vcycle(s, PH_INNER));
    if (condCapture_) {                            // the launches outside IF nodes, the update's too
      const CondDev& cd = E_.prm.cond;
      E_.prm.cond.n_base = (unsigned)(counting_ + 1 - start) - cd.n_cycle - cd.n_outer - cd.n_update;
    }
    HN_LAUNCH(KC_UPDATE, -1, launch_update(E_, fine_, fineGrid_, s, 1, h, use_h));
    return HN_OK;
  } else {
    if (cond_on(1)) HN_TRY(open_if(s, 1));
    int c0 = counting_;
    HN_LAUNCH(KC_OUTER_DEFECT, -1, launch_outer_defect(E_, fine_, fineGrid_, s));
    HN_LAUNCH(KC_CONTROL, -1, launch_control(E_, CTRL_OUTER, s));
    if (cond_on(1)) {
      E_.prm.cond.n_outer = (unsigned)(counting_ - c0);
      HN_TRY(close_if(s, s0));
    }
    HN_TRY(issue_vcycle(s, PH_INNER));
    if (cond_on(2)) HN_TRY(open_if(s, 2));
    c0 = counting_;
    HN_LAUNCH(KC_UPDATE, -1, launch_update(E_, fine_, fineGrid_, s));
    HN_LAUNCH(KC_CONTROL, -1, launch_control(E_, CTRL_POST, s));
    if (cond_on(2)) {
      E_.prm.cond.n_update = (unsigned)(counting_ - c0);
      HN_TRY(close_if(s, s0));
    }
  }
  if (condCapture_) {
    const CondDev& cd = E_.prm.cond;
    E_.prm.cond.n_base = (unsigned)(counting_ + 1 - start) - cd.n_cycle - cd.n_outer - cd.n_update;
  }
  HN_LAUNCH0(launch_summary(E_, h, use_h, 1, s));
  return HN_OK;
}

// The defect correction and CG of an engine of one problem fold their control steps and the
// iteration summary into the kernels before them when the fine norm is one group of partials (one
// block sums it) and no step has an IF node of its own.
bool Engine::fuse_control() const {
  const bool dc = prm_.solver != SOLVER_PCG && prm_.prec != P64;
  return cap_ == 1 && (dc || prm_.solver == SOLVER_PCG) && !cond_on(1) && !cond_on(2) &&
         pitch_of(Lmax_) / kTile <= kSumGroup;
}

hn_status Engine::capture_graphs() {
  destroy_graphs();
  clear_marks();
  cudaStream_t cs;
  HN_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  // graphs carry no profiling events (profiled iterations are issued directly)
  struct Guard {
    cudaStream_t s; bool& prof; bool saved;
    ~Guard() { cudaStreamDestroy(s); prof = saved; }
  } guard{cs, profiling_, profiling_};
  profiling_ = false;
  const cudaGraphConditionalHandle none = 0;
  // host-driven pieces: init and one iteration
  {
    cudaGraph_t g;
    HN_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    counting_ = 0;
    hn_status st = issue_init(cs, none, 0);
    initLaunches_ = counting_;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    HN_TRY(st);
    HN_CUDA(e);
    e = cudaGraphInstantiate(&gInit_, g, 0);
    cudaGraphDestroy(g);
    HN_CUDA(e);
  }
  {
    cudaGraph_t g;
    HN_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    counting_ = 0;
    hn_status st = issue_iteration(cs, none, 0);
    iterLaunches_ = counting_;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    HN_TRY(st);
    HN_CUDA(e);
    e = cudaGraphInstantiate(&gIter_, g, 0);
    cudaGraphDestroy(g);
    HN_CUDA(e);
  }
  // closed-world solve: init, then while (any problem running) { iteration }, with the IF node
  // that skips the rest of a cycle no problem is in; the flat loop if that does not build
  {
    hn_status st = capture_solve(true);
    if (st != HN_OK) {
      cudaGetLastError();
      HN_TRY(capture_solve(false));
    }
  }
  graphsValid_ = true;
  return HN_OK;
}

hn_status Engine::capture_solve(bool cond) {
  cudaStream_t cs;
  HN_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  HN_CUDA(cudaStreamCreateWithFlags(&aux_, cudaStreamNonBlocking));
  struct Guard {
    Engine* e;
    cudaStream_t cs;
    cudaGraph_t main = nullptr;
    ~Guard() {
      for (cudaStream_t q : {cs, e->aux_}) {
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(q, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
          cudaGraph_t g = nullptr;
          if (cudaStreamEndCapture(q, &g) == cudaSuccess && g) cudaGraphDestroy(g);
        }
        cudaStreamDestroy(q);
      }
      e->aux_ = nullptr;
      e->condCapture_ = false;
      e->pdlBarrier_ = false;
      e->E_.prm.cond = CondDev{};
      if (main) cudaGraphDestroy(main);
    }
  } guard{this, cs};
  HN_CUDA(cudaGraphCreate(&guard.main, 0));
  cudaGraph_t main = guard.main;
  const cudaGraphConditionalHandle none = 0;
  cudaGraphConditionalHandle h;
  HN_CUDA(cudaGraphConditionalHandleCreate(&h, main, 1, cudaGraphCondAssignDefault));
  CondDev cd{};
  if (cond) {
    // An IF node costs about as much as several launches (measured: ~2 us skipped, ~5 us
    // taken), so only the rest of a V cycle after the lagged check gets one, and only in the
    // defect correction, where every outer step ends with one cycle that its check stops.  (The
    // outer defect and the update would each skip two small launches: not worth an IF node.)
    const int T = std::max(std::max(tune_.tail_level, prm_.coarse), mid_top());
    if (Lmax_ > T && prm_.prec != P64 && prm_.solver != SOLVER_PCG) cd.mask |= 1u;
    const unsigned defaults[3] = {0u, 1u, 0u};
    // two sets: the loop body holds two iterations, each with IF nodes of its own handles
    for (int w = 0; w < 3; ++w)
      if ((cd.mask >> w) & 1u)
        for (int half = 0; half < 2; ++half)
          HN_CUDA(cudaGraphConditionalHandleCreate(&hCond_[half][w], main, defaults[w], cudaGraphCondAssignDefault));
    cd.h_cycle = hCond_[0][0];
    cd.h_outer = hCond_[0][1];
    cd.h_update = hCond_[0][2];
    cd.taken = dTaken_;
    cd.launches = dLaunches_;
  }
  cudaGraph_t init;
  HN_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  hn_status st = issue_init(cs, none, 0);
  cudaError_t e = cudaStreamEndCapture(cs, &init);
  HN_TRY(st);
  HN_CUDA(e);
  cudaGraphNode_t nInit;
  e = cudaGraphAddChildGraphNode(&nInit, main, nullptr, 0, init);
  cudaGraphDestroy(init);
  HN_CUDA(e);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t nCond;
  HN_CUDA(cudaGraphAddNode(&nCond, main, &nInit, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  HN_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  // The loop body is two iterations: the first one's summary leaves the loop condition alone, the
  // second one's sets it (a problem that finishes in the first runs the second as no-ops).  Each
  // turn of a device-side loop costs several microseconds; this halves their number.
  E_.prm.cond = cd;
  condCapture_ = cd.mask != 0;
  counting_ = 0;
  st = issue_iteration(cs, h, 0);
  if (st == HN_OK) {
    CondDev cd2 = cd;
    cd2.h_cycle = hCond_[1][0];
    cd2.h_outer = hCond_[1][1];
    cd2.h_update = hCond_[1][2];
    cd2.n_base = E_.prm.cond.n_base;               // the counts of the first half (same shape)
    cd2.n_cycle = E_.prm.cond.n_cycle;
    cd2.n_outer = E_.prm.cond.n_outer;
    cd2.n_update = E_.prm.cond.n_update;
    E_.prm.cond = cd2;
    st = issue_iteration(cs, h, 1);
  }
  condCapture_ = false;
  e = cudaStreamEndCapture(cs, &body);
  HN_TRY(st);
  HN_CUDA(e);
  cudaGraphExec_t exec = nullptr;
  HN_CUDA(cudaGraphInstantiate(&exec, main, 0));
  if (gSolve_) cudaGraphExecDestroy(gSolve_);
  gSolve_ = exec;
  condUsed_ = cd.mask != 0;
  return HN_OK;
}

hn_status Engine::run_to_completion() {
  if (profiling_) {
    HN_TRY(run_init());
    lastLaunches_ = initLaunches_;
    const int limit = prm_.max_cycles + prm_.max_outer + 8;
    for (int it = 0; it < limit; ++it) {
      unsigned active = 0;
      HN_TRY(run_iteration(&active));
      lastLaunches_ += iterLaunches_;
      if (active == 0) break;
    }
    return HN_OK;
  }
  if (!graphsValid_) HN_TRY(capture_graphs());
  HN_CUDA(cudaGraphLaunch(gSolve_, s_));
  unsigned iters = 0;
  unsigned long long body = 0;
  HN_CUDA(cudaMemcpyAsync(&iters, E_.iter, sizeof iters, cudaMemcpyDeviceToHost, s_));
  HN_CUDA(cudaMemcpyAsync(&body, dLaunches_, sizeof body, cudaMemcpyDeviceToHost, s_));
  HN_CUDA(cudaStreamSynchronize(s_));
  // the init graph's summary also counts one iteration; with IF nodes the loop counts the
  // kernels it ran, otherwise each body iteration runs iterLaunches_ kernels
  lastLaunches_ = initLaunches_ + (condUsed_ ? (long long)body
                                             : (long long)(iters > 0 ? iters - 1 : 0) * iterLaunches_);
  return HN_OK;
}

// With profiling on, iterations are issued directly to the stream (every kernel between its
// own events, and visible to a profiler, which does not profile graph kernels that may set a
// conditional value); otherwise the captured init / iteration graphs run.
hn_status Engine::run_init() {
  if (profiling_) {
    counting_ = 0;
    HN_TRY(issue_init(s_, 0, 0));
    initLaunches_ = counting_;
    return HN_OK;
  }
  if (!graphsValid_) HN_TRY(capture_graphs());
  HN_CUDA(cudaGraphLaunch(gInit_, s_));
  return HN_OK;
}

hn_status Engine::run_iteration(unsigned* active_out) {
  HN_TRY(launch_iteration());
  return finish_iteration(active_out);
}

hn_status Engine::launch_iteration() {
  if (profiling_) {
    clear_marks();
    counting_ = 0;
    HN_TRY(issue_iteration(s_, 0, 0));
    iterLaunches_ = counting_;
    HN_CUDA(cudaStreamSynchronize(s_));
    HN_TRY(accumulate_marks());
    clear_marks();
  } else {
    if (!graphsValid_) HN_TRY(capture_graphs());
    HN_CUDA(cudaGraphLaunch(gIter_, s_));
  }
  return HN_OK;
}

hn_status Engine::finish_iteration(unsigned* active_out) {
  HN_CUDA(cudaStreamSynchronize(s_));
  if (active_out) *active_out = *reinterpret_cast<volatile unsigned*>(hActive_);
  return HN_OK;
}

void Engine::clear_marks() {
  for (auto& m : marks_) { cudaEventDestroy(m.b); cudaEventDestroy(m.e); }
  marks_.clear();
  for (auto& e : openBegin_) cudaEventDestroy(e);
  openBegin_.clear();
}

hn_status Engine::accumulate_marks() {
  for (const Mark& m : marks_) {
    float ms = 0.0f;
    HN_CUDA(cudaEventElapsedTime(&ms, m.b, m.e));
    const int lv = m.level < 0 ? 0 : m.level;
    Acc& a = acc_[m.cls][lv];
    a.ms += ms;
    a.launches += 1;
    a.bytes = m.bytes;
  }
  return HN_OK;
}

void Engine::set_profiling(bool on) {
  profiling_ = on;
  graphsValid_ = false;
  for (auto& row : acc_)
    for (auto& a : row) a = Acc{};
}

int Engine::kernel_times(hn_kernel_time* out, int max) const {
  static const char* names[KC_COUNT] = {"jacobi", "jacobi_first", "defect", "restrict", "prolong",
                                        "coarse", "check", "outer_defect", "update", "control",
                                        "tail", "pcg_q", "pcg_x", "pcg_dot", "pcg_p",
                                        "prolong_jacobi", "mid_down", "mid_up", "sweep_down",
                                        "sweep_up"};
  int n = 0;
  for (int c = 0; c < KC_COUNT; ++c)
    for (int l = 0; l <= kMaxLevel; ++l) {
      const Acc& a = acc_[c][l];
      if (a.launches == 0) continue;
      if (n < max && out) {
        hn_kernel_time& t = out[n];
        std::memset(&t, 0, sizeof t);
        std::snprintf(t.name, sizeof t.name, "%s", names[c]);
        t.level = (c == KC_CHECK || c == KC_OUTER_DEFECT || c == KC_UPDATE || c == KC_CONTROL ||
                   (c >= KC_PCG_Q && c <= KC_PCG_P)) ? -1 : l;
        t.launches = a.launches;
        t.total_ms = a.ms;
        t.bytes_per_launch = (double)a.bytes;
      }
      ++n;
    }
  return n < max ? n : max;
}

hn_status Engine::read_states(std::vector<ProbState>& out) {
  out.resize(cap_);
  HN_CUDA(cudaMemcpyAsync(out.data(), dS_, sizeof(ProbState) * cap_, cudaMemcpyDeviceToHost, s_));
  HN_CUDA(cudaStreamSynchronize(s_));
  return HN_OK;
}

hn_status Engine::read_error_detail(int (&err)[4]) {
  HN_CUDA(cudaMemcpyAsync(err, dErr_, sizeof(int) * 4, cudaMemcpyDeviceToHost, s_));
  HN_CUDA(cudaStreamSynchronize(s_));
  return HN_OK;
}

hn_status Engine::check_guards() const { return guards_intact(memBase_, memBytes_, "engine block"); }

hn_status Engine::read_error(int* err) {
  HN_CUDA(cudaMemcpyAsync(err, dErr_, sizeof(int), cudaMemcpyDeviceToHost, s_));
  HN_CUDA(cudaStreamSynchronize(s_));
  return HN_OK;
}

hn_status Engine::apply_check_norm(cudaStream_t s) {
  HN_CUDA(launch_check(E_, fine_, PH_CHECK, 0, fineGrid_, s));
  HN_CUDA(launch_control(E_, CTRL_CHECK0, s));
  return HN_OK;
}

hn_status Engine::apply(int op, int level, int want, cudaStream_t s) {
  switch (op) {
    case HN_OP_SPMV: HN_CUDA(launch_spmv(E_, lists_[level], level, want, 0, grid_[level], s)); break;
    case HN_OP_DEFECT: HN_CUDA(launch_defect(E_, lists_[level], level, want, 0, grid_[level], s)); break;
    case HN_OP_JACOBI: HN_CUDA(launch_jacobi(E_, lists_[level], level, want, 0, 0, grid_[level], s)); break;
    case HN_OP_JACOBI_ZERO: HN_CUDA(launch_jacobi(E_, lists_[level], level, want, 0, 1, grid_[level], s)); break;
    case HN_OP_RESTRICT:
      HN_CUDA(launch_restrict(E_, lists_[level - 1], level, want, grid_[level - 1], s));
      break;
    case HN_OP_PROLONG_ADD: HN_CUDA(launch_prolong(E_, lists_[level], level, want, 0, grid_[level], s)); break;
    case HN_OP_PROLONG_JACOBI:
      HN_CUDA(launch_prolong_jacobi(E_, lists_[level], level, want, 0, grid_[level], s));
      break;
    case HN_OP_COARSE: HN_CUDA(launch_coarse(E_, lists_[level], want, grid_[level], s)); break;
    default: return set_error(HN_ERR_ARG, "unknown op %d", op);
  }
  return HN_OK;
}

}  // namespace hn

hn_band::~hn_band() {
  if (mem_base) cudaFree(mem_base);
  else if (mem) cudaFree(mem);
}

hn_mg::~hn_mg() {
  delete solo;
  if (mem_base) cudaFree(mem_base);
  else if (mem) cudaFree(mem);
  if (own_stream && stream) cudaStreamDestroy(stream);
}
