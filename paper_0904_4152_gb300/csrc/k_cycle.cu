// Hot-path kernels of the multigrid V cycle (Sec. 6.2 of the HONEI paper): the 9-band product,
// defect (with deterministic norm), damped Jacobi, full-weighting restriction, bilinear
// prolongation with correction, the exact coarse solve, the FP64 outer defect of the
// mixed-precision defect correction, and the per-problem control kernels of the solver state
// machine.
//
// Work decomposition: a level's padded flat node range is cut into warp-tiles of 128 nodes; lane l
// owns nodes 4l..4l+3 of its tile.  A launch walks a device work list of (problem, tile) pairs
// with a grid-stride loop over warps, so one launch serves any mix of problems and levels, and a
// captured CUDA graph stays valid when the work list changes.  Bands are loaded as aligned
// vectors (double2 pairs, float4, or 4 packed halves); the three x rows of the stencil are loaded
// as aligned 4-vectors because the row offset n = 2^L + 1 equals 2^L plus one column, and the
// one- or two-column overhang at each side comes from the neighbouring lanes by warp shuffles.
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <cooperative_groups.h>

#include "hn_internal.h"

namespace cg = cooperative_groups;

namespace hn {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Programmatic dependent launch: a kernel lets its successor in the stream launch as soon as all
// of its blocks are running (launch_dependents), and waits for its predecessor's completion and
// memory before touching any data (wait).  Both are no-ops for a normal launch.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_start() {
  pdl_trigger();
  pdl_wait();
}

// ------------------------------------------------------------ debug-build index checks
// With HN_DEBUG_CHECKS the kernels check every work-list item (problem slot, level, tile) and
// every one-problem level descriptor against the hierarchy's layout before touching memory; a
// failed check records the source line and the indices in the engine's error words (the first
// failure wins), skips the access and lets the launch finish.  Release builds compile the checks
// to nothing.
#ifndef HN_DEBUG_CHECKS
#define HN_DEBUG_CHECKS 0
#endif
__device__ __forceinline__ void dbg_fail(const EngineDev& E, int line, int a, int b) {
  if (atomicCAS(E.err, 0, 5) == 0) {
    E.err[1] = line;
    E.err[2] = a;
    E.err[3] = b;
  }
}
// problem p's tile `tile` of level lv (lv < 0: its finest level)
__device__ __forceinline__ bool dbg_item(const EngineDev& E, int p, int tile, int lv, int line) {
#if HN_DEBUG_CHECKS
  bool ok = p >= 0 && p < E.nprob;
  if (ok) {
    const ProblemDev& P = E.P[p];
    const int l = lv < 0 ? P.L : lv;
    ok = l >= P.coarse && l <= P.L && P.lev[l].n == (1 << l) + 1 && tile >= 0 &&
         (long long)(tile + 1) * kTile <= (long long)P.lev[l].pitch;
  }
  if (!ok) dbg_fail(E, line, p, tile);
  return ok;
#else
  (void)E; (void)p; (void)tile; (void)lv; (void)line;
  return true;
#endif
}
// a one-problem descriptor of level l serving `tiles` tiles
__device__ __forceinline__ bool dbg_level(const EngineDev& E, const LevelDev& d, int l, int tiles, int line) {
#if HN_DEBUG_CHECKS
  const bool ok = l >= HN_MIN_LEVEL && l <= kMaxLevel && d.n == (1 << l) + 1 && tiles >= 0 &&
                  (long long)tiles * kTile <= (long long)d.pitch;
  if (!ok) dbg_fail(E, line, l, tiles);
  return ok;
#else
  (void)E; (void)d; (void)l; (void)tiles; (void)line;
  return true;
#endif
}

// Ask L2 for a tile's 9 band slices ahead of their loads (one prefetch per lane and band).  The
// FP16-band kernels move 8 bytes per lane and band, half of what an FP32 lane moves, so with the
// same warps in flight they keep fewer bytes outstanding; prefetching the bands of the warp's next
// tile while it works on the current one lifts them from 0.81-0.86 to 0.87-0.89 of HBM at L = 12.
// (Further ahead, with the x rows as well, or in the FP32 / FP64 kernels, it measured slower.)
template <class Pol>
__device__ __forceinline__ void prefetch_bands(const LevelDev& d, long long i0) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const char* p = static_cast<const char*>(d.band[k]) + i0 * (long long)sizeof(typename Pol::B);
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
  }
}

// An engine of one problem skips a whole fine-level launch when its problem is not in the phase
// the kernel serves (otherwise every warp would walk its share of the work list to find that out:
// ~20 us per empty launch at L = 12)
__device__ __forceinline__ bool solo_idle(const EngineDev& E, int phase);

// -------------------------------------------------------------------- precision policies
struct F64 { using B = double; using V = double; using A = double; static constexpr int prec = P64; };
struct F32 { using B = float; using V = float; using A = float; static constexpr int prec = P32; };
struct F16 { using B = __half; using V = float; using A = float; static constexpr int prec = P16; };

// Load kinds: LD_NC reads global memory through the non-coherent path (data written by an
// earlier launch); LD_CG reads global memory from L2 (data written earlier in the same launch by
// other SMs of the cluster); LD_GEN is a plain generic load (data in shared memory).  Bands are
// never written by the solver: NC from global memory, GEN from shared memory.
// LD_EF: non-coherent, marked first to be evicted from L2 (data read once per outer step, such as
// the FP64 operator of the outer defect, which would otherwise push the inner cycles' working set
// out of L2).
enum { LD_NC = 0, LD_CG = 1, LD_GEN = 2, LD_EF = 3 };
template <int LK> __device__ __forceinline__ constexpr int band_kind() { return LK == LD_GEN ? LD_GEN : LD_NC; }

__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double2 ld_ef(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(l2_evict_first_policy()));
  return v;
}
__device__ __forceinline__ double ld_ef(const double* p) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(l2_evict_first_policy()));
  return v;
}

template <int LK, class T> __device__ __forceinline__ T ldk(const T* p) {
  if constexpr (LK == LD_NC) return __ldg(p);
  else if constexpr (LK == LD_CG) return __ldcg(p);
  else if constexpr (LK == LD_EF) return ld_ef(p);
  else return *p;
}
template <int LK> __device__ __forceinline__ double ld1(const double* p) { return ldk<LK>(p); }
template <int LK> __device__ __forceinline__ float ld1(const float* p) { return ldk<LK>(p); }

template <int LK>
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = ldk<LK>(q);
  const double2 b = ldk<LK>(q + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <int LK>
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 a = ldk<LK>(reinterpret_cast<const float4*>(p));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
// plain (coherent) loads for data the same thread also writes
__device__ __forceinline__ void ld4c(const double* p, double (&o)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4c(const float* p, float (&o)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}

// products rounded on their own (never contracted into a following add or subtract)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// 4 consecutive band values of band k at node i0, in the arithmetic type
template <class Pol, int LKB = LD_NC>
__device__ __forceinline__ void load_band(const void* band, float scale, long long i0,
                                          typename Pol::A (&o)[4]) {
  if constexpr (Pol::prec == P16) {
    const uint2 u = ldk<LKB>(reinterpret_cast<const uint2*>(static_cast<const __half*>(band) + i0));
    const __half2 h0 = *reinterpret_cast<const __half2*>(&u.x);
    const __half2 h1 = *reinterpret_cast<const __half2*>(&u.y);
    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    // each value rounded on its own (never contracted into a following add)
    o[0] = __fmul_rn(scale, f0.x); o[1] = __fmul_rn(scale, f0.y);
    o[2] = __fmul_rn(scale, f1.x); o[3] = __fmul_rn(scale, f1.y);
  } else {
    ld4<LKB>(static_cast<const typename Pol::B*>(band) + i0, o);
  }
}

// Row window around the lane's 4 nodes: w[o + 2] = v[a + o], o = -2..5, a aligned to 4.
template <class V, int LK>
__device__ __forceinline__ void load_row(const V* __restrict__ v, long long a, int lane, V (&w)[8]) {
  V c[4];
  ld4<LK>(v + a, c);
  V l2 = __shfl_up_sync(kFull, c[2], 1), l1 = __shfl_up_sync(kFull, c[3], 1);
  V r0 = __shfl_down_sync(kFull, c[0], 1), r1 = __shfl_down_sync(kFull, c[1], 1);
  if (lane == 0) { l2 = ld1<LK>(v + a - 2); l1 = ld1<LK>(v + a - 1); }
  if (lane == 31) { r0 = ld1<LK>(v + a + 4); r1 = ld1<LK>(v + a + 5); }
  w[0] = l2; w[1] = l1; w[2] = c[0]; w[3] = c[1]; w[4] = c[2]; w[5] = c[3]; w[6] = r0; w[7] = r1;
}

// The FP64 kernels form a defect b - A x as one FMA chain from b (b - a_0 x_0 - a_1 x_1 ...), one
// FP64 operation per node fewer than b - (A x): they are bound by the FP64 pipe on this part.  The
// FP32 and FP16-band kernels, bound by HBM, subtract the finished product.
template <class Pol> __device__ __forceinline__ constexpr bool def_chain() { return Pol::prec == P64; }

// acc[j] = sum_k band_k[i0+j] * x[i0+j+off_k] over the windows w (rows dy = -1, 0, 1), in band
// order k = 0..8; also the diagonal.  off_k = dy*n + dx = dy*shift + (dy + dx), shift = n - 1.
// DEF: acc enters holding b and leaves holding b - sum_k (same order).
template <class Pol, int LKB, bool DEF = false>
__device__ __forceinline__ void stencil_windows(const void* const* band, const float* scale,
                                                const typename Pol::V (&w)[3][8], long long i0,
                                                typename Pol::A (&acc)[4],
                                                typename Pol::A (&dg)[4]) {
  using A = typename Pol::A;
  if constexpr (!DEF) {
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = A(0);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int dy = k / 3 - 1, dx = k % 3 - 1;
    A b[4];
    load_band<Pol, LKB>(band[k], scale ? scale[k] : 1.0f, i0, b);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      acc[j] = DEF ? fma(-b[j], A(w[dy + 1][j + dy + dx + 2]), acc[j])
                   : fma(b[j], A(w[dy + 1][j + dy + dx + 2]), acc[j]);
    if (k == 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) dg[j] = b[j];
    }
  }
}

// FP16-band operator in row-sum form (array 4 holds the row sum rho):
// acc[j] = rho x_i + sum_{k != 4} a_k (x_{i+off_k} - x_i) in band order; dg[j] = rho - sum a_k.
// The nine 8-byte band loads of the lane are issued before any arithmetic (the FP16 kernels move
// half an FP32 lane's bytes per load, so more of them must be in flight: L = 12 Jacobi 0.88 ->
// 0.90 of HBM); each value is then scaled and used in band order as before.
template <int LKB>
__device__ __forceinline__ void stencil_windows_rowsum(const void* const* band, const float* scale,
                                                       const float (&w)[3][8], long long i0,
                                                       float (&acc)[4], float (&dg)[4]) {
  uint2 raw[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) raw[k] = ldk<LKB>(reinterpret_cast<const uint2*>(static_cast<const __half*>(band[k]) + i0));
  // 4 consecutive values of band k, each rounded on its own (never contracted into a following add)
  auto unpack = [&](int k, float (&o)[4]) {
    const __half2 h0 = *reinterpret_cast<const __half2*>(&raw[k].x);
    const __half2 h1 = *reinterpret_cast<const __half2*>(&raw[k].y);
    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    o[0] = __fmul_rn(scale[k], f0.x); o[1] = __fmul_rn(scale[k], f0.y);
    o[2] = __fmul_rn(scale[k], f1.x); o[3] = __fmul_rn(scale[k], f1.y);
  };
  float rho[4];
  unpack(4, rho);
#pragma unroll
  for (int j = 0; j < 4; ++j) { acc[j] = rho[j] * w[1][j + 2]; dg[j] = rho[j]; }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (k == 4) continue;
    const int dy = k / 3 - 1, dx = k % 3 - 1;
    float b[4];
    unpack(k, b);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[j] = fmaf(b[j], w[dy + 1][j + dy + dx + 2] - w[1][j + 2], acc[j]);
      dg[j] -= b[j];
    }
  }
}

// diagonal of the row-sum form without x (for the zero-guess Jacobi step)
template <int LKB>
__device__ __forceinline__ void diag_rowsum(const void* const* band, const float* scale,
                                            long long i0, float (&dg)[4]) {
  load_band<F16, LKB>(band[4], scale[4], i0, dg);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (k == 4) continue;
    float b[4];
    load_band<F16, LKB>(band[k], scale[k], i0, b);
#pragma unroll
    for (int j = 0; j < 4; ++j) dg[j] -= b[j];
  }
}

// y = A x at the lane's 4 nodes (x read with load kind LK); xc = x at the nodes, dg = diagonal.
// DEF (plain band form, not the FP16 row sums): acc enters holding b and leaves holding b - A x.
template <class Pol, int LK, bool DEF = false>
__device__ __forceinline__ void apply_op4(const LevelDev& d, const typename Pol::V* __restrict__ x,
                                          long long i0, long long ib, long long shift, int lane,
                                          typename Pol::A (&acc)[4], typename Pol::V (&xc)[4],
                                          typename Pol::A (&dg)[4]) {
  typename Pol::V w[3][8];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) load_row<typename Pol::V, LK>(x, i0 + dy * shift, lane, w[dy + 1]);
#pragma unroll
  for (int j = 0; j < 4; ++j) xc[j] = w[1][j + 2];
  if constexpr (Pol::prec == P16) stencil_windows_rowsum<band_kind<LK>()>(d.band, d.scale, w, ib, acc, dg);
  else stencil_windows<Pol, band_kind<LK>(), DEF>(d.band, nullptr, w, ib, acc, dg);
}

// deterministic warp sum (butterfly; every lane ends with the same value)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Tile partial of a residual norm: the sum over the warp of the squares of each lane's 4 values.
// FP64 values: squares and sums in FP64.  FP32 values: on the FP32 pipe in double-float
// arithmetic (each square exactly as p + e by an FMA, sums by TwoSum), within ~2^-46 of the exact
// sum of the non-negative terms; FP64 operations run at 1/74 of the FP32 rate on this part, and
// per node four of them (two conversions, a product, a sum) cost as much as the band kernel's
// memory traffic at L = 10.  Every lane gets the same value (each butterfly step is symmetric in
// its two operands).
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (bh - bb);  // TwoSum: hi + bh = s + err exactly
  const float t = err + (lo + bl);
  hi = s + t;                                      // FastTwoSum (|s| >= |t|)
  lo = t - (hi - s);
}
__device__ __forceinline__ double tile_sumsq(const double (&r)[4]) {
  double q = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) q += r[j] * r[j];
  return warp_sum(q);
}
// FP32: the pair (hi, lo) itself, stored in the partial's 8 bytes; every consumer of the partials
// of an FP32 / FP16 cycle sums them as pairs (problem_partial_sum with df)
__device__ __forceinline__ float2 tile_sumsq(const float (&r)[4]) {
  float hi = __fmul_rn(r[0], r[0]), lo = fmaf(r[0], r[0], -hi);
#pragma unroll
  for (int j = 1; j < 4; ++j) {
    const float p = __fmul_rn(r[j], r[j]);
    df_add(hi, lo, p, fmaf(r[j], r[j], -p));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(kFull, hi, o), bl = __shfl_xor_sync(kFull, lo, o);
    df_add(hi, lo, bh, bl);
  }
  return make_float2(hi, lo);
}
__device__ __forceinline__ void store_partial(double* slot, double q) { *slot = q; }
__device__ __forceinline__ void store_partial(double* slot, float2 q) { *reinterpret_cast<float2*>(slot) = q; }

// the same butterfly over the block (any multiple of 32 threads up to 1024); valid in warp 0.
// sh: 32 doubles of shared memory, used as 64 floats
__device__ double block_sum_df(float hi, float lo, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_xor_sync(kFull, hi, o), bl = __shfl_xor_sync(kFull, lo, o);
    df_add(hi, lo, bh, bl);
  }
  float* sf = reinterpret_cast<float*>(sh);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sf[2 * w] = hi; sf[2 * w + 1] = lo; }
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    const bool in = lane < (int)(blockDim.x >> 5);
    float h = in ? sf[2 * lane] : 0.0f, l = in ? sf[2 * lane + 1] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float bh = __shfl_xor_sync(kFull, h, o), bl = __shfl_xor_sync(kFull, l, o);
      df_add(h, l, bh, bl);
    }
    t = double(h) + double(l);                    // exact (l is below half an ulp of h)
  }
  __syncthreads();
  return t;
}

// deterministic block sum of a per-thread value (256 threads)
__device__ double block_sum256(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;   // valid in warp 0
}

// Fixed-order sum of one problem's per-tile partials by one block of 256 threads: thread t adds
// slots t + 256 (4j + c) into chain c = 0..3 (in order of j), then (c0 + c1) + (c2 + c3), then
// the block tree.  Every caller uses this order, so a problem's norm does not depend on which
// kernel or batch computed it.  (Four chains: a dependent FP64 add costs ~64 cycles here.)
// Valid in thread 0.
// df: the partials are double-float pairs (an FP32 / FP16 cycle's), summed in the same order in
// double-float arithmetic on the FP32 pipe: one SM's FP64 rate (~1.7 operations per cycle) made
// the 8,209 FP64 additions of an L = 10 norm the longest part of its lagged check (~10 us).
__device__ double problem_partial_sum_df(const double* part, int ntiles, double* sh) {
  const float2* pp = reinterpret_cast<const float2*>(part);
  float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, l[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (threadIdx.x < 256) {
    int q = threadIdx.x;
    for (; q + 31 * 256 < ntiles; q += 32 * 256) {
      float2 v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = __ldcg(pp + q + k * 256);
#pragma unroll
      for (int k = 0; k < 32; k += 4)
#pragma unroll
        for (int c = 0; c < 4; ++c) df_add(h[c], l[c], v[k + c].x, v[k + c].y);
    }
    for (; q + 3 * 256 < ntiles; q += 4 * 256)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 v = __ldcg(pp + q + c * 256);
        df_add(h[c], l[c], v.x, v.y);
      }
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (q + c * 256 < ntiles) {
        const float2 v = __ldcg(pp + q + c * 256);
        df_add(h[c], l[c], v.x, v.y);
      }
  }
  df_add(h[0], l[0], h[1], l[1]);
  df_add(h[2], l[2], h[3], l[3]);
  df_add(h[0], l[0], h[2], l[2]);
  return block_sum_df(h[0], l[0], sh);
}

__device__ double problem_partial_sum(const double* part, int ntiles, double* sh, bool df = false) {
  if (df) return problem_partial_sum_df(part, ntiles, sh);
  double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
  if (threadIdx.x < 256) {                    // larger blocks: the other threads add +0.0
    int q = threadIdx.x;
    // batches of 8 rounds: the 32 loads of a batch are issued before its adds (the adds keep
    // the order above), so L2 latency is paid once per batch rather than once per round
    for (; q + 31 * 256 < ntiles; q += 32 * 256) {
      double v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = __ldcg(part + q + k * 256);
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        c0 += v[k];
        c1 += v[k + 1];
        c2 += v[k + 2];
        c3 += v[k + 3];
      }
    }
    for (; q + 3 * 256 < ntiles; q += 4 * 256) {
      c0 += __ldcg(part + q);
      c1 += __ldcg(part + q + 256);
      c2 += __ldcg(part + q + 512);
      c3 += __ldcg(part + q + 768);
    }
    if (q < ntiles) c0 += __ldcg(part + q);
    if (q + 256 < ntiles) c1 += __ldcg(part + q + 256);
    if (q + 512 < ntiles) c2 += __ldcg(part + q + 512);
  }
  return block_sum256((c0 + c1) + (c2 + c3), sh);
}

// A problem's tiles are summed in groups of kSumGroup consecutive tiles when it has more than one
// group: each group by problem_partial_sum, then the group sums in group order.  (One block adding
// 131,072 FP64 partials at L = 12 is bound by one SM's FP64 rate, ~30 us; the control kernel
// gives each group its own block.)  Every path that forms a problem's norm uses this order.
__device__ __forceinline__ int sum_groups(int ntiles) { return (ntiles + kSumGroup - 1) / kSumGroup; }

__device__ double group_partial_sum(const double* part, int ntiles, int j, double* sh, bool df = false) {
  const int lo = j * kSumGroup;
  return problem_partial_sum(part + lo, min(kSumGroup, ntiles - lo), sh, df);
}

// the same order in one block (valid in thread 0)
__device__ double problem_norm_sum(const double* part, int ntiles, double* sh, bool df = false) {
  const int ng = sum_groups(ntiles);
  if (ng == 1) return problem_partial_sum(part, ntiles, sh, df);
  double t = 0.0;
  for (int j = 0; j < ng; ++j) {
    const double g = group_partial_sum(part, ntiles, j, sh, df);
    if (threadIdx.x == 0) t += g;
  }
  return t;
}

__host__ __device__ inline int fine_tiles(int L) {
  const long long n = (1LL << L) + 1;
  return (int)((n * n + kTile - 1) / kTile);
}

// Lagged convergence test: the first smoothing step of a cycle from a nonzero iterate computes
// the residual of that iterate; nrm is its norm.  FP64 multigrid stops when relres <= tol (the
// iterate in buffer 0 is the result) or at the cycle cap; inner cycles of the defect correction
// stop at the inner tolerance or the inner caps (the correction goes to the update).  Otherwise
// the cycle proceeds and is counted.
__device__ __forceinline__ void cond_set(const CondDev& c, int which, unsigned v) {
  if (!((c.mask >> which) & 1u)) return;
  cudaGraphSetConditional(which == 0 ? c.h_cycle : (which == 1 ? c.h_outer : c.h_update), v);
  c.taken[which] = v;
}

__device__ void pre_check(ProbState& st, const Params& prm, double nrm) {
  if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; return; }
  if (st.phase == PH_CYCLE) {
    st.dnorm = nrm;
    st.relres = nrm / st.bnorm;
    if (st.relres <= prm.tol) { st.status = HN_OK; st.phase = PH_DONE; }
    else if (st.cycles >= prm.max_cycles) { st.status = HN_ERR_NOT_CONVERGED; st.phase = PH_DONE; }
    else st.cycles += 1;
  } else {
    st.inner_res = nrm;
    if (nrm <= prm.inner_tol * st.inner_ref || st.inner_k >= prm.inner_max ||
        st.inner_cycles >= prm.max_cycles) {
      st.phase = PH_UPDATE;
      cond_set(prm.cond, 2, 1u);
    } else { st.inner_k += 1; st.inner_cycles += 1; st.cycles += 1; }
  }
}

__device__ __forceinline__ bool solo_idle(const EngineDev& E, int phase) {
  return E.nprob == 1 && E.S[0].phase != phase;
}

// Modes of the band kernel.  PRE12 / PRE2B split the first two smoothing steps: from a zero
// iterate both steps fuse into one pass (x1 = omega D^-1 b is formed on the fly from windows of b
// and of the stored omega / D, then x2 = x1 + omega D^-1 (b - A x1) goes to buffer 0) and PRE2B
// skips the tile; otherwise PRE12 does step 1 (buffer 0 -> 1) and PRE2B step 2 (1 -> 0).
enum BandMode {
  M_SPMV = 0, M_DEFECT = 1, M_JACOBI = 2, M_JACOBI_FIRST = 3, M_CHECK = 4, M_PRE12 = 5,
  M_PRE2B = 6,
  M_PJ = 7        // prolongation x += P e_c fused into the first post-smoothing step
};

template <class Pol> __device__ __forceinline__ constexpr bool fuses_pre() { return true; }

// omega / diag at the lane's 4 nodes.  FP64: the stored wdinv (LKB: load kind of the bands, with
// which it is staged).  FP32 / FP16: omega / dg from the diagonal the stencil formed anyway;
// reading the stored wdf instead (4 more bytes per node) measured slower for both.
template <class Pol, int LKB>
__device__ __forceinline__ void wd4_of(const LevelDev& d, long long i0, typename Pol::A omega,
                                       const typename Pol::A (&dg)[4], typename Pol::A (&wd)[4]) {
  if constexpr (Pol::prec == P64) {
    ld4<LKB>(d.wdinv + i0, wd);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) wd[j] = omega / dg[j];
  }
}

// One warp-tile of the band kernel on level d.  zg: the iterate of this level is zero.
// boff: bands are indexed at i0 - boff (a chunk of bands staged in shared memory); LKB_ is the
// load kind of the bands (shared memory: LD_GEN).
template <class Pol, int MODE, int LK, int LKB_ = band_kind<LK>()>
__device__ __forceinline__ void band_tile(const LevelDev& d, long long shift, bool zg, long long i0,
                                          int lane, int in_sel, typename Pol::A omega,
                                          double* partial_slot, long long boff = 0) {
  using A = typename Pol::A;
  using V = typename Pol::V;
  constexpr int LKB = LKB_;
  const long long ib = i0 - boff;
  const V* rhs = static_cast<const V*>(d.rhs);
  if constexpr (MODE == M_PRE2B) {
    if (zg && fuses_pre<Pol>()) return;
  }
  if constexpr (MODE == M_JACOBI_FIRST || MODE == M_PRE12) {
    if (zg && (MODE == M_JACOBI_FIRST || !fuses_pre<Pol>())) {   // x = 0: x' = omega D^-1 rhs
      V b[4], out[4];
      ld4<LK>(rhs + i0, b);
      if constexpr (Pol::prec == P64) {
        double wd[4];
        ld4<LKB>(d.wdinv + i0, wd);
#pragma unroll
        for (int j = 0; j < 4; ++j) out[j] = wd[j] * b[j];
      } else {
        float wd[4];                              // omega / D, stored (never staged)
        ld4<band_kind<LK>()>(d.wdf + i0, wd);
#pragma unroll
        for (int j = 0; j < 4; ++j) out[j] = wd[j] * A(b[j]);
      }
      st4(static_cast<V*>(d.x[1]) + i0, out);
      return;
    }
    if constexpr (MODE == M_PRE12 && fuses_pre<Pol>()) {
      if (zg) {                                   // two steps from zero in one pass
        // windows of b and of omega / D (zero in the halos, so x1 is zero there)
        V bw[3][8], dw[3][8], x1[3][8];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          load_row<V, LK>(rhs, i0 + dy * shift, lane, bw[dy + 1]);
          if constexpr (Pol::prec == P64) load_row<V, LKB>(d.wdinv, i0 + dy * shift, lane, dw[dy + 1]);
          else load_row<V, band_kind<LK>()>(d.wdf, i0 + dy * shift, lane, dw[dy + 1]);
        }
        // x1 rounded on its own: the FP16 form subtracts x1 values, where a contracted product
        // would round differently from one path to another
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int o = 0; o < 8; ++o) x1[r][o] = mul_rn(dw[r][o], bw[r][o]);
        constexpr bool DEF = def_chain<Pol>();
        A acc[4], dg[4];
        if constexpr (DEF) {
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = A(bw[1][j + 2]);
        }
        if constexpr (Pol::prec == P16) stencil_windows_rowsum<LKB>(d.band, d.scale, x1, ib, acc, dg);
        else stencil_windows<Pol, LKB, DEF>(d.band, nullptr, x1, ib, acc, dg);
        V out[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const A r = DEF ? acc[j] : A(bw[1][j + 2]) - acc[j];
          out[j] = fma(A(dw[1][j + 2]), r, A(x1[1][j + 2]));
        }
        st4(static_cast<V*>(d.x[0]) + i0, out);
        return;
      }
    }
  }
  int src = in_sel, dst = 1 - in_sel;
  if constexpr (MODE == M_JACOBI_FIRST || MODE == M_PRE12) { src = 0; dst = 1; }
  if constexpr (MODE == M_PRE2B) { src = 1; dst = 0; }
  const V* xin = static_cast<const V*>(d.x[src]);
  constexpr bool DEF = MODE != M_SPMV && def_chain<Pol>();
  A acc[4], dg[4];
  V xc[4], b[4];
  if constexpr (DEF) {                            // the chain starts from b
    ld4<LK>(rhs + i0, b);
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = A(b[j]);
  }
  if constexpr (LKB == band_kind<LK>()) apply_op4<Pol, LK, DEF>(d, xin, i0, ib, shift, lane, acc, xc, dg);
  else {                                          // bands from a shared-memory stage
    V w[3][8];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) load_row<V, LK>(xin, i0 + dy * shift, lane, w[dy + 1]);
#pragma unroll
    for (int j = 0; j < 4; ++j) xc[j] = w[1][j + 2];
    if constexpr (Pol::prec == P16) stencil_windows_rowsum<LKB>(d.band, d.scale, w, ib, acc, dg);
    else stencil_windows<Pol, LKB, DEF>(d.band, nullptr, w, ib, acc, dg);
  }
  if constexpr (MODE == M_SPMV) {
    V out[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = V(acc[j]);
    st4(static_cast<V*>(d.r) + i0, out);
  } else {
    if constexpr (!DEF) ld4<LK>(rhs + i0, b);
    A r[4];                                       // the defect b - A x
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = DEF ? acc[j] : A(b[j]) - acc[j];
    if constexpr (MODE == M_DEFECT) {
      V out[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = V(r[j]);
      st4(static_cast<V*>(d.r) + i0, out);
    } else if constexpr (MODE == M_CHECK) {
      const auto q = tile_sumsq(r);
      if (lane == 0) store_partial(partial_slot, q);
    } else {                                      // a Jacobi step src -> dst
      A wd[4];
      wd4_of<Pol, LKB>(d, i0, omega, dg, wd);
      V out[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = fma(wd[j], r[j], A(xc[j]));
      st4(static_cast<V*>(d.x[dst]) + i0, out);
      if constexpr (MODE == M_PRE12 || MODE == M_JACOBI_FIRST) {
        if (partial_slot) {                       // residual norm of the iterate (lagged check)
          const auto q = tile_sumsq(r);
          if (lane == 0) store_partial(partial_slot, q);
        }
      }
    }
  }
}

// Full-weighting restriction of the fine defect onto coarse node (I, J) (Dirichlet and padding
// nodes get 0).  Summation order: fine rows 2J-1, 2J, 2J+1, columns 2I-1, 2I, 2I+1, weights 1/4,
// 1/2, 1/4 x 1/4, 1/2, 1/4 (products by powers of two are exact); a fine node off the grid (next
// to a free Neumann side) contributes 0.  rd(y, x) reads fine node (x, y).
template <class V, class F>
__device__ __forceinline__ V restrict_value_xy(int I, int J, int nc, int nf, int bc, F rd) {
  if (I < 0 || J >= nc || is_dirichlet(I, J, nc, bc)) return V(0);
  const int fx = 2 * I, fy = 2 * J;
  auto R = [&](int dy, int dx) -> V {
    const int x = fx + dx, y = fy + dy;
    return (x >= 0 && y >= 0 && x < nf && y < nf) ? rd(y, x) : V(0);
  };
  const V q = V(0.25), h = V(0.5);
  V v = q * R(-1, -1);
  v = fma(h, R(-1, 0), v);
  v = fma(q, R(-1, 1), v);
  v = fma(h, R(0, -1), v);
  v = v + R(0, 0);
  v = fma(h, R(0, 1), v);
  v = fma(q, R(1, -1), v);
  v = fma(h, R(1, 0), v);
  v = fma(q, R(1, 1), v);
  return v;
}
// the same with rd(i) reading fine node i = y nf + x
template <class V, class F>
__device__ __forceinline__ V restrict_value(int I, int J, int nc, int nf, int bc, F rd) {
  return restrict_value_xy<V>(I, J, nc, nf, bc, [&](int y, int x) { return rd((long long)y * nf + x); });
}

// Restriction of the coarse warp-tile starting at t0 (128 nodes): lane l takes the coarse nodes
// t0 + l + 32 j, j = 0..3, so that the lanes of one load read consecutive pairs of fine nodes (a
// coalesced span of the fine row) and the stores are coalesced too; padding nodes get 0.
template <class V, int LK>
__device__ __forceinline__ void restrict_tile(const LevelDev& f, const LevelDev& c, long long t0,
                                              int lane) {
  const int nc = c.n, nf = f.n, Nc = nc * nc;
  const V* r = static_cast<const V*>(f.r);
  V* out = static_cast<V*>(c.rhs);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = (int)t0 + lane + 32 * j;
    V v = V(0);
    if (q < Nc) {
      const int J = (int)((unsigned)q / (unsigned)nc), I = q - J * nc;
      if (I > 0 && J > 0 && I < nc - 1 && J < nc - 1) {
        // an interior coarse node: its 3 x 3 fine neighbourhood lies on the grid and it is no
        // Dirichlet node; restrict_value's sum without its per-tap bounds checks
        const V* f = r + (long long)(2 * J) * nf + 2 * I;
        const V qw = V(0.25), h = V(0.5);
        v = qw * ld1<LK>(f - nf - 1);
        v = fma(h, ld1<LK>(f - nf), v);
        v = fma(qw, ld1<LK>(f - nf + 1), v);
        v = fma(h, ld1<LK>(f - 1), v);
        v = v + ld1<LK>(f);
        v = fma(h, ld1<LK>(f + 1), v);
        v = fma(qw, ld1<LK>(f + nf - 1), v);
        v = fma(h, ld1<LK>(f + nf), v);
        v = fma(qw, ld1<LK>(f + nf + 1), v);
      } else {
        v = restrict_value<V>(I, J, nc, nf, c.bc, [&](long long k) { return ld1<LK>(r + k); });
      }
    }
    out[q] = v;
  }
}

// x_f[x_sel] += P e_c at fine node (ix, iy): bilinear interpolation of the coarse iterate, ec(cy, cx)
// reading coarse node (cx, cy); Dirichlet fine nodes are left unchanged (their coarse neighbours on
// the same side are Dirichlet too and hold 0).  Returns false for them, else the value added.
template <class V, class F>
__device__ __forceinline__ bool prolong_value_xy(int ix, int iy, int nf, int bc, F ec, V* add) {
  if (is_dirichlet(ix, iy, nf, bc)) return false;
  const int cx0 = ix >> 1, cx1 = (ix + 1) >> 1, cy0 = iy >> 1, cy1 = (iy + 1) >> 1;
  const bool ox = ix & 1, oy = iy & 1;
  if (!ox && !oy) *add = ec(cy0, cx0);
  else if (ox && !oy) *add = V(0.5) * (ec(cy0, cx0) + ec(cy0, cx1));
  else if (!ox && oy) *add = V(0.5) * (ec(cy0, cx0) + ec(cy1, cx0));
  else *add = V(0.25) * (((ec(cy0, cx0) + ec(cy0, cx1)) + ec(cy1, cx0)) + ec(cy1, cx1));
  return true;
}
// the same with ec(k) reading coarse node k = cy nc + cx
template <class V, class F>
__device__ __forceinline__ bool prolong_value(int ix, int iy, int nf, int nc, int bc, F ec, V* add) {
  return prolong_value_xy<V>(ix, iy, nf, bc, [&](int cy, int cx) { return ec(cy * nc + cx); }, add);
}

// x_f[x_sel & 1] += P e_c on fine tile i0; e_c is the coarse iterate in buffer (x_sel >> 1) & 1
// (buffer 1 after a fused up sweep of the coarse level, else buffer 0)
template <class V, int LK>
__device__ __forceinline__ void prolong_tile(const LevelDev& f, const LevelDev& c, int x_sel,
                                             long long i0) {
  const int nf = f.n, nc = c.n, Nf = nf * nf;
  const V* e = static_cast<const V*>(c.x[(x_sel >> 1) & 1]);
  V* x = static_cast<V*>(f.x[x_sel & 1]);
  V v[4];
  if constexpr (LK == LD_NC) ld4c(x + i0, v);   // read and rewritten by this thread only
  else ld4<LK>(x + i0, v);                      // written earlier in this launch
  // fine coordinates of the lane's first node
  int iy = (int)((unsigned)i0 / (unsigned)nf), ix = (int)i0 - iy * nf;
  if (ix + 3 < nf && (int)i0 + 3 < Nf) {
    // the 4 nodes lie in one fine row: they interpolate from coarse columns cxa .. cxa + 2 (all on
    // the grid, as ix + 3 <= nf - 1) of coarse row iy / 2 and, for an odd row, of the next one;
    // each coarse value is loaded once and the arithmetic is prolong_value's, term for term
    const int cxa = ix >> 1, cy0 = iy >> 1, odd = ix & 1;
    const bool oy = iy & 1;
    V e0[3], e1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e0[k] = ld1<LK>(e + cy0 * nc + cxa + k);
      e1[k] = oy ? ld1<LK>(e + (cy0 + 1) * nc + cxa + k) : V(0);
    }
    // Node j sits at fine column 2 cxa + odd + j.  The row parity (oy) and the column parity
    // (odd) are the same for all lanes of a warp that lie in one fine row, so the four cases
    // below are separate code paths: each node does its own formula's operations only (a
    // per-node choice between the formulas had the FP64 pipe evaluate several of them).
    // A node adds a coarse value (x + e), an edge midpoint (x + 0.5 (a + b)) or a cell centre
    // (x + 0.25 (((a + b) + c) + d)).  The products by 0.5 and 0.25 are exact, so one FMA of the
    // scale, the sum and x rounds exactly as prolong_value's product followed by the addition, with
    // one FP64 operation fewer per midpoint and centre (the FP64 transfers are bound by the pipe).
    auto pt = [](V x, V a) { return x + a; };
    auto mid = [](V x, V a, V b) { return fma(V(0.5), a + b, x); };
    auto ctr = [](V x, V a, V b, V c, V d) { return fma(V(0.25), ((a + b) + c) + d, x); };
    V out[4];
    if (!oy) {
      if (!odd) {
        out[0] = pt(v[0], e0[0]); out[1] = mid(v[1], e0[0], e0[1]);
        out[2] = pt(v[2], e0[1]); out[3] = mid(v[3], e0[1], e0[2]);
      } else {
        out[0] = mid(v[0], e0[0], e0[1]); out[1] = pt(v[1], e0[1]);
        out[2] = mid(v[2], e0[1], e0[2]); out[3] = pt(v[3], e0[2]);
      }
    } else {
      if (!odd) {
        out[0] = mid(v[0], e0[0], e1[0]);
        out[1] = ctr(v[1], e0[0], e0[1], e1[0], e1[1]);
        out[2] = mid(v[2], e0[1], e1[1]);
        out[3] = ctr(v[3], e0[1], e0[2], e1[1], e1[2]);
      } else {
        out[0] = ctr(v[0], e0[0], e0[1], e1[0], e1[1]);
        out[1] = mid(v[1], e0[1], e1[1]);
        out[2] = ctr(v[2], e0[1], e0[2], e1[1], e1[2]);
        out[3] = mid(v[3], e0[2], e1[2]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (!is_dirichlet(ix + j, iy, nf, f.bc)) v[j] = out[j];
  } else {
    // the nodes wrap into the next row (or reach the padding): node by node
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      V add;
      if ((int)i0 + j < Nf && prolong_value<V>(ix, iy, nf, nc, f.bc, [&](int k) { return ld1<LK>(e + k); }, &add))
        v[j] = v[j] + add;
      if (++ix == nf) { ix = 0; ++iy; }
    }
  }
  st4(x + i0, v);
}

// P e_c at fine node q = (qx, qy) if q is a grid node (0 <= q < Nf), else 0 (halo, padding, or a
// Dirichlet node); the same value prolong_value adds
template <class V, int LK>
__device__ __forceinline__ V prolong_at(const V* e, long long q, int qx, int qy, int nf, int nc,
                                        int bc, long long Nf) {
  V add = V(0);
  if (q >= 0 && q < Nf && !prolong_value<V>(qx, qy, nf, nc, bc, [&](int k) { return ld1<LK>(e + k); }, &add))
    add = V(0);
  return add;
}

// (qx, qy) of flat index a + o from (ax, ay) of a, |o| < nf: one wrap at most
__device__ __forceinline__ void step_xy(int ax, int ay, int o, int nf, int& qx, int& qy) {
  qx = ax + o;
  qy = ay;
  if (qx < 0) { qx += nf; --qy; }
  else if (qx >= nf) { qx -= nf; ++qy; }
}

// Row window of y = x + P e_c around the lane's 4 nodes: w[o + 2] = y at a + o, o = -2..5 (a =
// the flat index of the lane's first node in this row, (ax, ay) its coordinates, possibly off the
// grid).  Each y is formed exactly as the prolongation kernel forms it (x + add), so the step that
// follows sees the same values it would read after a separate prolongation.
template <class V, int LK>
__device__ __forceinline__ void load_row_prolonged(const V* x, const V* e, long long a, int ax, int ay,
                                                   int nf, int nc, int bc, long long Nf, int lane,
                                                   V (&w)[8]) {
  V c[4];
  ld4<LK>(x + a, c);
  if (a >= 0 && a + 3 < Nf && ax + 3 < nf && ay >= 0) {
    // one fine row: coarse columns cxa .. cxa + 2 of coarse row ay / 2 (and the next one)
    const int cxa = ax >> 1, cy0 = ay >> 1, odd = ax & 1;
    const bool oy = ay & 1;
    V e0[3], e1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      e0[k] = ld1<LK>(e + cy0 * nc + cxa + k);
      e1[k] = oy ? ld1<LK>(e + (cy0 + 1) * nc + cxa + k) : V(0);
    }
    auto pick = [](const V (&q)[3], int i) { return i == 0 ? q[0] : (i == 1 ? q[1] : q[2]); };
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (is_dirichlet(ax + j, ay, nf, bc)) continue;
      const int c0 = (j + odd) >> 1, c1 = (j + 1 + odd) >> 1;
      const bool ox = (j + odd) & 1;
      V add;
      if (!ox && !oy) add = pick(e0, c0);
      else if (ox && !oy) add = V(0.5) * (pick(e0, c0) + pick(e0, c1));
      else if (!ox && oy) add = V(0.5) * (pick(e0, c0) + pick(e1, c0));
      else add = V(0.25) * (((pick(e0, c0) + pick(e0, c1)) + pick(e1, c0)) + pick(e1, c1));
      c[j] = c[j] + add;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int qx, qy;
      step_xy(ax, ay, j, nf, qx, qy);
      if (a + j >= 0 && a + j < Nf) {
        V add;
        if (prolong_value<V>(qx, qy, nf, nc, bc, [&](int k) { return ld1<LK>(e + k); }, &add)) c[j] = c[j] + add;
      }
    }
  }
  V l2 = __shfl_up_sync(kFull, c[2], 1), l1 = __shfl_up_sync(kFull, c[3], 1);
  V r0 = __shfl_down_sync(kFull, c[0], 1), r1 = __shfl_down_sync(kFull, c[1], 1);
  if (lane == 0) {
    int qx, qy;
    step_xy(ax, ay, -2, nf, qx, qy);
    l2 = ld1<LK>(x + a - 2) + prolong_at<V, LK>(e, a - 2, qx, qy, nf, nc, bc, Nf);
    step_xy(ax, ay, -1, nf, qx, qy);
    l1 = ld1<LK>(x + a - 1) + prolong_at<V, LK>(e, a - 1, qx, qy, nf, nc, bc, Nf);
  }
  if (lane == 31) {
    int qx, qy;
    step_xy(ax, ay, 4, nf, qx, qy);
    r0 = ld1<LK>(x + a + 4) + prolong_at<V, LK>(e, a + 4, qx, qy, nf, nc, bc, Nf);
    step_xy(ax, ay, 5, nf, qx, qy);
    r1 = ld1<LK>(x + a + 5) + prolong_at<V, LK>(e, a + 5, qx, qy, nf, nc, bc, Nf);
  }
  w[0] = l2; w[1] = l1; w[2] = c[0]; w[3] = c[1]; w[4] = c[2]; w[5] = c[3]; w[6] = r0; w[7] = r1;
}

// The prolongation x_f[s] += P e_c and the first post-smoothing Jacobi step in one pass (s =
// in_sel & 1; e_c in coarse buffer (in_sel >> 1) & 1, as for prolong_tile): the step's windows are
// formed from x and e_c on the fly, the corrected iterate is not stored (the second step
// overwrites it), the step's result goes to buffer 1 - s.  Identical values to the separate
// prolongation and Jacobi kernels.
template <class Pol, int LK>
__device__ __forceinline__ void prolong_jacobi_tile(const LevelDev& d, const LevelDev& c, long long shift,
                                                    long long i0, int lane, int in_sel,
                                                    typename Pol::A omega) {
  using A = typename Pol::A;
  using V = typename Pol::V;
  const int nf = d.n, nc = c.n;
  const long long Nf = (long long)nf * nf;
  const V* e = static_cast<const V*>(c.x[(in_sel >> 1) & 1]);
  in_sel &= 1;
  const V* x = static_cast<const V*>(d.x[in_sel]);
  const int iy0 = (int)((unsigned long long)i0 / (unsigned)nf), ix0 = (int)(i0 - (long long)iy0 * nf);
  V w[3][8];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    int ax = ix0 - dy, ay = iy0 + dy;                 // i0 + dy * shift, shift = nf - 1
    if (ax < 0) { ax += nf; --ay; } else if (ax >= nf) { ax -= nf; ++ay; }
    load_row_prolonged<V, LK>(x, e, i0 + dy * shift, ax, ay, nf, nc, d.bc, Nf, lane, w[dy + 1]);
  }
  constexpr bool DEF = def_chain<Pol>();
  A acc[4], dg[4];
  V b[4];
  if constexpr (DEF) {
    ld4<LK>(static_cast<const V*>(d.rhs) + i0, b);
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = A(b[j]);
  }
  if constexpr (Pol::prec == P16) stencil_windows_rowsum<band_kind<LK>()>(d.band, d.scale, w, i0, acc, dg);
  else stencil_windows<Pol, band_kind<LK>(), DEF>(d.band, nullptr, w, i0, acc, dg);
  if constexpr (!DEF) ld4<LK>(static_cast<const V*>(d.rhs) + i0, b);
  A wd[4];
  wd4_of<Pol, band_kind<LK>()>(d, i0, omega, dg, wd);
  V out[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) out[j] = fma(wd[j], DEF ? acc[j] : A(b[j]) - acc[j], A(w[1][j + 2]));
  st4(static_cast<V*>(d.x[1 - in_sel]) + i0, out);
}

// One row of the coarse inverse times the coarse right-hand side: four interleaved FP64 chains
// (v mod 4), then (a0 + a1) + (a2 + a3); a dependent FP64 operation costs ~64 cycles on this part,
// so one chain of m would dominate the coarse solve.  rd(v) gives the v-th interior rhs in FP64.
template <class F>
__device__ __forceinline__ double coarse_dot(const double* row, int m, F rd) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int v = 0;
  for (; v + 3 < m; v += 4) {
    a0 = fma(row[v], rd(v), a0);
    a1 = fma(row[v + 1], rd(v + 1), a1);
    a2 = fma(row[v + 2], rd(v + 2), a2);
    a3 = fma(row[v + 3], rd(v + 3), a3);
  }
  if (v < m) a0 = fma(row[v], rd(v), a0);
  if (v + 1 < m) a1 = fma(row[v + 1], rd(v + 1), a1);
  if (v + 2 < m) a2 = fma(row[v + 2], rd(v + 2), a2);
  return (a0 + a1) + (a2 + a3);
}

// Exact coarsest-level solve x_c = A_c^-1 rhs_c (precomputed FP64 inverse of the interior block)
// by one warp; result into buffer 0.  sol: m doubles of shared memory.
template <class V, int LK>
__device__ __forceinline__ void coarse_warp(const ProblemDev& P, int lane, double* sol) {
  const LevelDev& d = P.lev[P.coarse];
  const int n = d.n, m = P.m;
  const UnknownRect ur = unknown_rect(n, d.bc);
  const V* rhs = static_cast<const V*>(d.rhs);
  for (int u = lane; u < m; u += 32) {
    const double* row = P.cinv + (long long)u * m;
    sol[u] = coarse_dot(row, m, [&](int v) {
      return double(ld1<LK>(rhs + (v / ur.nx + ur.y0) * n + (v % ur.nx + ur.x0)));
    });
  }
  __syncwarp();
  V* x = static_cast<V*>(d.x[0]);
  for (int q = lane; q < d.pitch; q += 32) {
    const int iy = q / n - ur.y0, ix = q - (q / n) * n - ur.x0;
    V val = V(0);
    if (q < n * n && ix >= 0 && iy >= 0 && ix < ur.nx && iy < ur.ny) val = V(sol[iy * ur.nx + ix]);
    x[q] = val;
  }
  __syncwarp();
}

// Unpreconditioned conjugate gradients on the coarsest level (Sec. 6.2 configures the coarse
// solver so), in FP64 by the whole block over all N_c = n^2 nodes of the level: ab holds its 9
// FP64 bands (band k at ab + k N_c; Dirichlet rows are identity rows and no row couples to a
// Dirichlet node, so with a zero right-hand side there these nodes stay 0 and the iteration is CG
// on the unknowns).  r holds the right-hand side on entry and the residual on exit, x receives the
// solution, p, q and sc (4 doubles) are scratch.  Textbook CG from x = 0 (Hestenes and Stiefel):
// q = A p, alpha = (r, r) / (p, q), x += alpha p, r -= alpha q; stop once (r, r) <=
// kCoarseCgTol^2 (b, b) or after coarse_cg_steps(m) steps (m unknowns); else p = r + ((r, r)_new /
// (r, r)) p.  Inner products: warp 0, lane l adds nodes l, l + 32, ... in order, then the
// butterfly, so the result does not depend on the block size; the scalar divisions run in one
// thread (FP64 is slow on this part: redundant divisions across the block cost microseconds).
__device__ __forceinline__ double coarse_warp0_dot(const double* u, const double* v, int N) {
  double t = 0.0;
  for (int i = threadIdx.x; i < N; i += 32) t = fma(u[i], v[i], t);
  return warp_sum(t);
}

__device__ void coarse_cg(const double* ab, int n, int m, double* x, double* r, double* p,
                          double* q, double* sc) {
  const int N = n * n, nt = blockDim.x;
  for (int i = threadIdx.x; i < N; i += nt) { x[i] = 0.0; p[i] = r[i]; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const double rr = coarse_warp0_dot(r, r, N);
    if (threadIdx.x == 0) { sc[0] = rr; sc[1] = kCoarseCgTol * kCoarseCgTol * rr; }
  }
  __syncthreads();
  const int kmax = coarse_cg_steps(m);
  for (int k = 0; k < kmax; ++k) {
    if (!(sc[0] > 0.0)) break;                  // uniform: read by all after a barrier
    for (int i = threadIdx.x; i < N; i += nt) {
      // one chain per stencil row (FP64 latency), then (row -1 + row 0) + row +1
      const int iy = i / n, ix = i - iy * n;
      double t[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int b = 0; b < 9; ++b) {
        const int jx = ix + b % 3 - 1, jy = iy + b / 3 - 1;
        if (jx >= 0 && jy >= 0 && jx < n && jy < n) t[b / 3] = fma(ab[b * N + i], p[jy * n + jx], t[b / 3]);
      }
      q[i] = (t[0] + t[1]) + t[2];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const double pq = coarse_warp0_dot(p, q, N);
      if (threadIdx.x == 0) sc[2] = sc[0] / pq;             // alpha
    }
    __syncthreads();
    const double alpha = sc[2];
    for (int i = threadIdx.x; i < N; i += nt) {
      x[i] = fma(alpha, p[i], x[i]);
      r[i] = fma(-alpha, q[i], r[i]);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const double rr1 = coarse_warp0_dot(r, r, N);
      if (threadIdx.x == 0) {
        sc[3] = rr1 > sc[1] ? rr1 / sc[0] : -1.0;            // beta, or stop (also on a NaN)
        sc[0] = rr1;
      }
    }
    __syncthreads();
    const double beta = sc[3];
    if (beta < 0.0) break;
    for (int i = threadIdx.x; i < N; i += nt) p[i] = fma(beta, p[i], r[i]);
    __syncthreads();
  }
  __syncthreads();
}

// mbarrier and bulk-copy (TMA engine, 1D) helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// one bulk copy global -> this block's shared memory, accounted on bar (16-byte aligned, size a
// multiple of 16); issued by one thread, which arrives on bar once all its copies are issued
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  if (bytes == 0) return;
  mbar_expect(bar, bytes);
  bulk_g2s(dst, src, bytes, bar);
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for phase `parity` of an mbarrier; false if it did not complete in time
constexpr int kWaitTries = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < kWaitTries; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------------ per-level kernels
// One warp-tile per loop trip over the work list.  level < 0: each problem's own finest level.
// Resident blocks per SM asked of the register allocator.  The streaming modes keep 5 blocks
// (40 warps) of FP32 / FP16 loads in flight, enough to saturate HBM (the FP16 Jacobi step spills
// a few bytes at 5 blocks and is still faster than at 4: 89.8 vs 96.3 us at L = 12), except the
// FP16 defect, faster at 4 with its band loads hoisted; the fused pre-smoothing (4 blocks) and
// check modes run once per cycle and get more registers per thread.
// The lagged check of an engine of one problem taken inside its first smoothing step (in place of
// a separate control launch, for problems whose norm is one group of partials): the last block to
// finish sums the tile partials in the fixed order and updates the state, and the cycle's IF value
// is set as the control kernel sets it (the problem is still in the cycle).  A uniform early
// return of every block (problem not in the phase) leaves the ticket at zero.
__device__ void control_apply(const EngineDev& E, ProbState& st, int kind, double sum);
__device__ void summary_apply(const EngineDev& E, cudaGraphConditionalHandle h, int use_handle,
                              int end_of_iteration, double* sh);

// true in the last block of the launch to get here (every block calls it once, after its work;
// the block's writes are visible to that block); the last block resets the ticket when done
__device__ bool solo_last_block(const EngineDev& E) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(E.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// The last block of a launch of an engine of one problem takes control step `kind` in place of a
// control launch: with the launch's FP64 partials summed in the fixed order (sum_partials), if
// the problem was in the phase the step serves (mine: block-uniform, read at the launch's start)
__device__ void solo_fused_control(const EngineDev& E, int kind, bool mine, bool sum_partials) {
  if (!solo_last_block(E)) return;
  __shared__ double sh[32];
  double sum = 0.0;
  if (mine && sum_partials) sum = problem_norm_sum(E.partial, fine_tiles(E.P[0].L), sh);
  if (threadIdx.x == 0) {
    if (mine) control_apply(E, E.S[0], kind, sum);
    *E.ticket = 0u;
  }
}

__device__ void solo_fused_check(const EngineDev& E, int level, bool checked, int want) {
  __shared__ double sh[32];
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();                              // this block's partials before its ticket
    s_last = atomicAdd(E.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  ProbState& st = E.S[0];
  double sum = 0.0;
  if (checked) sum = problem_norm_sum(E.partial, fine_tiles(level), sh, E.prm.prec != P64);
  if (threadIdx.x == 0) {
    if (checked) pre_check(st, E.prm, sqrt(sum));
    if (st.phase == want && (st.phase == PH_INNER || st.phase == PH_CYCLE)) cond_set(E.prm.cond, 0, 1u);
    *E.ticket = 0u;                                 // ready for the next launch
  }
}

template <class Pol, int MODE> constexpr int band_min_blocks() {
  if (MODE == M_CHECK) return Pol::prec == P64 ? 2 : 3;
  if (MODE == M_PRE12) return Pol::prec == P64 ? 2 : 4;
  if (MODE == M_PJ) return Pol::prec == P64 ? 2 : (Pol::prec == P32 ? 4 : 3);
  if (Pol::prec == P32) return 5;
  if (Pol::prec == P16) return (MODE == M_SPMV || MODE == M_JACOBI) ? 5 : 4;   // defect: 0.90 -> 0.92 at 4
  return MODE == M_SPMV ? 4 : 3;
}

template <class Pol, int MODE>
__global__ void __launch_bounds__(256, band_min_blocks<Pol, MODE>()) k_band(EngineDev E, TileList tl,
                                                                     int level, int want,
                                                                     int in_sel) {
  pdl_start();
  using A = typename Pol::A;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const A omega = A(E.prm.omega);
  if (tl.solo_tiles > 0 && level >= 0) {          // one problem: descriptors by value
    const ProbState& st = E.S[0];
    if (st.phase != want) return;
    if (!dbg_level(E, tl.solo_d, level, tl.solo_tiles, __LINE__)) return;
    if constexpr (MODE == M_PJ) {
      if (tl.solo_c.n == 0) return;               // (no coarser level: nothing to prolong)
      for (int t = gw; t < tl.solo_tiles; t += nw)
        prolong_jacobi_tile<Pol, LD_NC>(tl.solo_d, tl.solo_c, 1LL << level, (long long)t * kTile + lane * kLaneNodes,
                                        lane, in_sel, omega);
      return;
    }
    const bool zg = (tl.solo_L > level) || st.zero_top;
    for (int t = gw; t < tl.solo_tiles; t += nw) {
      if constexpr (Pol::prec == P16)
        if (t + nw < tl.solo_tiles) prefetch_bands<Pol>(tl.solo_d, (long long)(t + nw) * kTile + lane * kLaneNodes);
      double* slot = nullptr;
      if constexpr (MODE == M_CHECK) slot = E.partial + t;
      if constexpr (MODE == M_PRE12 || MODE == M_JACOBI_FIRST)
        if (level == tl.solo_L && !zg) slot = E.partial + t;
      band_tile<Pol, MODE, LD_NC>(tl.solo_d, 1LL << level, zg, (long long)t * kTile + lane * kLaneNodes,
                                  lane, in_sel & 1, omega, slot);
    }
    if constexpr (MODE == M_PRE12 || MODE == M_JACOBI_FIRST)
      if (in_sel & 2) solo_fused_check(E, level, level == tl.solo_L && !zg, want);
    return;
  }
  if (solo_idle(E, want)) return;
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (!dbg_item(E, p, it.y, level, __LINE__)) continue;
    const ProbState& st = E.S[p];
    if (st.phase != want) continue;
    const ProblemDev& P = E.P[p];
    const int lv = level < 0 ? P.L : level;
    if constexpr (MODE == M_PJ) {
      prolong_jacobi_tile<Pol, LD_NC>(P.lev[lv], P.lev[lv - 1], 1LL << lv, (long long)it.y * kTile + lane * kLaneNodes,
                                      lane, in_sel, omega);
      continue;
    }
    const bool zg = (P.L > lv) || st.zero_top;
    double* slot = nullptr;
    if constexpr (MODE == M_CHECK) slot = E.partial + E.fine_off[p] + it.y;
    if constexpr (MODE == M_PRE12 || MODE == M_JACOBI_FIRST)
      if (lv == P.L && !zg) slot = E.partial + E.fine_off[p] + it.y;
    band_tile<Pol, MODE, LD_NC>(P.lev[lv], 1LL << lv, zg, (long long)it.y * kTile + lane * kLaneNodes,
                                lane, in_sel & 1, omega, slot);
  }
}

// Band kernel with the bands streamed through shared memory by the bulk-copy engine.  A block
// walks chunks of up to 8 consecutive warp-tiles of one problem-level (one warp per tile); for
// each chunk one thread issues 9 bulk copies (one per band) into one of two stages, signalled on
// that stage's mbarrier, two chunks ahead of the warps, which compute from shared memory with the
// vectors read as in k_band.  Chunks of problems not in phase `want` are skipped; chunks whose
// first two smoothing steps fuse from a zero iterate run the register path (their stencil reads
// diagonal windows beyond the chunk).  A wait that does not complete in time sets E.err, stops
// further copies and the block drains its outstanding copies (bounded) before returning.
template <class Pol, int MODE>
__global__ void __launch_bounds__(256) k_band_staged(EngineDev E, TileList tl, int level, int want,
                                                     int in_sel) {
  using A = typename Pol::A;
  using B = typename Pol::B;
  extern __shared__ __align__(128) unsigned char sbuf[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ LevelDev sdesc[2];
  __shared__ int sinfo[2][4];        // problem, first tile, tiles, kind (-1 end, 0 skip, 1 staged, 2 register path)
  __shared__ int s_abort;
  pdl_start();
  constexpr size_t kBandBytes = (size_t)kChunkTiles * kTile * sizeof(B);
  constexpr size_t kStage = 9 * kBandBytes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int count = *tl.chunk_count;
  const int G = gridDim.x;
  const A omega = A(E.prm.omega);
  const long long shift = 1LL << level;
  bool pending[2] = {false, false};   // thread 0: a fill of the stage is outstanding
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  auto prepare = [&](int k) {         // thread 0: chunk k of this block into stage k & 1
    const int st = k & 1;
    const int c = blockIdx.x + k * G;
    if (c >= count || s_abort) { sinfo[st][3] = -1; return; }
    const int4 ch = tl.chunks[c];
    const ProblemDev& P = E.P[ch.x];
    const ProbState& S = E.S[ch.x];
    int kind = 1;
    if (S.phase != want) kind = 0;
    else if ((MODE == M_PRE12 || MODE == M_PRE2B) && fuses_pre<Pol>() && ((P.L > level) || S.zero_top))
      kind = MODE == M_PRE12 ? 2 : 0;
    sinfo[st][0] = ch.x; sinfo[st][1] = ch.y; sinfo[st][2] = ch.z; sinfo[st][3] = kind;
    if (kind != 1) return;
    const LevelDev& g = P.lev[level];
    LevelDev& sd = sdesc[st];
    sd = g;
    unsigned char* base = sbuf + st * kStage;
    const long long start = (long long)ch.y * kTile;
    const unsigned bytes = (unsigned)(ch.z * kTile * sizeof(B));
    fence_proxy_async();
    mbar_expect_tx(&bar[st], 9 * bytes);
    for (int q = 0; q < 9; ++q) {
      B* dst = reinterpret_cast<B*>(base + q * kBandBytes);
      bulk_g2s(dst, static_cast<const B*>(g.band[q]) + start, bytes, &bar[st]);
      sd.band[q] = dst;
    }
    pending[st] = true;
  };
  if (threadIdx.x == 0) { prepare(0); prepare(1); }
  __syncthreads();
  unsigned phase[2] = {0u, 0u};
  for (int k = 0;; ++k) {
    const int st = k & 1;
    const int kind = sinfo[st][3];
    if (kind < 0) break;
    bool ok = true;
    if (kind == 1) {
      ok = mbar_wait(&bar[st], phase[st]);
      phase[st] ^= 1u;
      if (threadIdx.x == 0) pending[st] = false;
      if (!ok) { s_abort = 1; if (lane == 0) atomicExch(E.err, 1); }
    }
    if (ok && kind != 0 && warp < sinfo[st][2]) {
      const int p = sinfo[st][0], t = sinfo[st][1] + warp;
      const ProblemDev& P = E.P[p];
      const ProbState& S = E.S[p];
      const bool zg = (P.L > level) || S.zero_top;
      double* slot = nullptr;
      if constexpr (MODE == M_PRE12 || MODE == M_JACOBI_FIRST)
        if (level == P.L && !zg) slot = E.partial + E.fine_off[p] + t;
      const long long i0 = (long long)t * kTile + lane * kLaneNodes;
      if (kind == 1)
        band_tile<Pol, MODE, LD_NC, LD_GEN>(sdesc[st], shift, zg, i0, lane, in_sel, omega, slot,
                                            (long long)sinfo[st][1] * kTile);
      else
        band_tile<Pol, MODE, LD_NC>(P.lev[level], shift, zg, i0, lane, in_sel, omega, slot);
    }
    __syncthreads();
    if (threadIdx.x == 0) prepare(k + 2);
    __syncthreads();
  }
  if (threadIdx.x == 0) {            // after an abort: let outstanding copies land (bounded)
    for (int st = 0; st < 2; ++st)
      if (pending[st]) (void)mbar_wait(&bar[st], phase[st]);
  }
}

template <class V>
__global__ void __launch_bounds__(256) k_restrict(EngineDev E, TileList tl, int fine_level,
                                                  int want) {
  pdl_start();
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  if (tl.solo_tiles > 0) {                        // one problem: tl is the coarse level's list
    if (tl.solo_L < fine_level || E.S[0].phase != want) return;   // (no finer level: no descriptor)
    if (!dbg_level(E, tl.solo_d, fine_level - 1, tl.solo_tiles, __LINE__) ||
        !dbg_level(E, tl.solo_f, fine_level, 0, __LINE__)) return;
    for (int t = gw; t < tl.solo_tiles; t += nw)
      restrict_tile<V, LD_NC>(tl.solo_f, tl.solo_d, (long long)t * kTile, lane);
    return;
  }
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (!dbg_item(E, p, it.y, fine_level - 1, __LINE__)) continue;
    const ProblemDev& P = E.P[p];
    if (P.L < fine_level || E.S[p].phase != want) continue;
    restrict_tile<V, LD_NC>(P.lev[fine_level], P.lev[fine_level - 1], (long long)it.y * kTile, lane);
  }
}

template <class V>
__global__ void __launch_bounds__(256) k_prolong(EngineDev E, TileList tl, int level, int want,
                                                 int x_sel) {
  pdl_start();
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  if (tl.solo_tiles > 0) {                        // one problem: descriptors by value
    if (tl.solo_c.n == 0 || E.S[0].phase != want) return;   // (no coarser level: nothing to add)
    if (!dbg_level(E, tl.solo_d, level, tl.solo_tiles, __LINE__) ||
        !dbg_level(E, tl.solo_c, level - 1, 0, __LINE__)) return;
    for (int t = gw; t < tl.solo_tiles; t += nw)
      prolong_tile<V, LD_NC>(tl.solo_d, tl.solo_c, x_sel, (long long)t * kTile + lane * kLaneNodes);
    return;
  }
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (!dbg_item(E, p, it.y, level, __LINE__) || !dbg_item(E, p, 0, level - 1, __LINE__)) continue;
    if (E.S[p].phase != want) continue;
    const ProblemDev& P = E.P[p];
    prolong_tile<V, LD_NC>(P.lev[level], P.lev[level - 1], x_sel,
                           (long long)it.y * kTile + lane * kLaneNodes);
  }
}

template <class V>
__global__ void __launch_bounds__(256) k_coarse(EngineDev E, TileList tl, int want) {
  pdl_start();
  __shared__ double sol[8][kMaxCoarseM];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (it.y != 0) continue;
    const int p = it.x;
    if (E.S[p].phase != want) continue;
    coarse_warp<V, LD_NC>(E.P[p], lane, sol[wib]);
  }
}

// the coarsest-level solve by CG, one block per problem slot; result into buffer 0
template <class V>
__global__ void __launch_bounds__(256) k_coarse_cg(EngineDev E, int want) {
  pdl_start();
  __shared__ double x[kMaxCoarseM], r[kMaxCoarseM], pv[kMaxCoarseM], qv[kMaxCoarseM];
  __shared__ double sc[4];
  const int p = blockIdx.x;
  if (p >= E.nprob || E.S[p].phase != want) return;
  const ProblemDev& P = E.P[p];
  if (P.L < HN_MIN_LEVEL) return;
  const LevelDev& d = P.lev[P.coarse];
  const int n = d.n, N = n * n;
  const V* rhs = static_cast<const V*>(d.rhs);
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    r[i] = is_dirichlet(i % n, i / n, n, d.bc) ? 0.0 : double(rhs[i]);
  __syncthreads();
  coarse_cg(P.cinv, n, P.m, x, r, pv, qv, sc);
  V* xo = static_cast<V*>(d.x[0]);
  for (int i = threadIdx.x; i < d.pitch; i += blockDim.x) xo[i] = i < N ? V(x[i]) : V(0);
}

// ----------------------------------------------------------- fused coarse-level V cycle
// One thread-block cluster per problem runs the part of the V cycle on levels coarse..min(T, L):
// pre-smoothing, defect and restriction down to the coarsest level, the exact solve, then
// prolongation and post-smoothing back up.
//  * Levels above S run on the whole cluster over global memory: phases are separated by cluster
//    barriers (release / acquire at cluster scope) and data produced inside the launch are read
//    from L2 (LD_CG).
//  * Levels coarse..S run inside block 0 alone, entirely in its shared memory (all bands and
//    vectors of those levels, with zero halos), phases separated by block barriers; on the way in
//    the restricted right-hand side of level S (and its iterate, if nonzero) is copied in, on
//    the way out the iterate of level S is copied back.
// The problem's level descriptors are copied to shared memory once.  The barrier sequence depends
// only on the problem's levels and the engine parameters, so every block of a cluster passes the
// same barriers.

constexpr long long kCinvSmemMax = 32 * 1024;

// 16-byte asynchronous global -> shared copy (cp.async, L2 only); completion by cp_async_wait()
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// Copy of `bytes` (a multiple of 16; both ends 16-byte aligned) from global to this block's
// shared memory as one bulk copy (the TMA engine) issued by thread 0 and accounted on the mbarrier
// `bar`, whose phase completes once thread 0 has arrived and every byte has landed.  The copies ask
// L2 to keep the lines (evict-last): the tail reads the same constant data (~2 MB) once per cycle,
// between which the finer levels stream tens of MB through L2.  (Staging block 0's levels 2..5,
// ~40 arrays and ~70 KB, measured 5.7 us issued as 16-byte cp.async by every thread and 6.1 us as
// bulk copies, with or without the hint: the time is not in the copies.)
__device__ __forceinline__ void block_copy16(void* dst, const void* src, long long bytes,
                                             unsigned long long* bar) {
  if (threadIdx.x != 0 || bytes <= 0) return;
  unsigned long long pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(bar)), "r"((unsigned)bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          (unsigned)__cvta_generic_to_shared(dst)),
      "l"(src), "r"((unsigned)bytes), "r"((unsigned)__cvta_generic_to_shared(bar)), "l"(pol)
      : "memory");
}

// shared-memory bytes of levels coarse..S for a precision (16-byte aligned pieces)
__host__ __device__ inline long long smem_level_bytes(int l, int prec) {
  const long long ve = ((1LL << l) + 1) * ((1LL << l) + 1);
  const long long pitch = (ve + kTile - 1) / kTile * kTile;
  const long long halo = (((1LL << l) + 1 + 8) + 31) / 32 * 32;
  const long long e = pitch + 2 * halo;
  const long long bs = prec == P64 ? 8 : (prec == P32 ? 4 : 2);
  const long long vs = prec == P64 ? 8 : 4;
  auto al = [](long long b) { return (b + 15) / 16 * 16; };
  return 9 * al(e * bs) + 4 * al(e * vs) + al(e * (prec == P64 ? 8 : 4));
}

// carve level l of the shared-memory hierarchy starting at *off; with `fill`, start the copies of
// its bands and omega/D (block_copy16, on the mbarrier bar) and zero its vectors.  The caller
// waits for the copies (the mbarrier phase) and synchronizes the block before use.  Every block of a cluster carves
// the same layout, so a block can address block 0's copy through distributed shared memory.
template <class Pol>
__device__ void smem_level_setup(const LevelDev& g, LevelDev& s, unsigned char* base, long long* off,
                                 int l, bool fill, unsigned long long* bar) {
  using V = typename Pol::V;
  using B = typename Pol::B;
  const long long halo = (((1LL << l) + 1 + 8) + 31) / 32 * 32;
  const long long e = (long long)g.pitch + 2 * halo;    // a multiple of 32 elements
  auto take = [&](long long bytes) { unsigned char* r = base + *off; *off += (bytes + 15) / 16 * 16; return r; };
  // every thread computes the same carve-up; thread 0 publishes the pointers
  LevelDev t = g;
  for (int k = 0; k < 9; ++k) {
    B* dst = reinterpret_cast<B*>(take(e * sizeof(B)));
    const B* src = static_cast<const B*>(g.band[k]) - halo;
    if (fill) block_copy16(dst, src, e * (long long)sizeof(B), bar);
    t.band[k] = dst + halo;
  }
  if constexpr (Pol::prec == P64) {
    double* dst = reinterpret_cast<double*>(take(e * 8));
    if (fill) block_copy16(dst, g.wdinv - halo, e * 8, bar);
    t.wdinv = dst + halo;
  } else {
    float* dst = reinterpret_cast<float*>(take(e * 4));
    if (fill) block_copy16(dst, g.wdf - halo, e * 4, bar);
    t.wdf = dst + halo;
  }
  V* vec[4];
  for (int v = 0; v < 4; ++v) {
    vec[v] = reinterpret_cast<V*>(take(e * sizeof(V)));
    for (int q = threadIdx.x; fill && q < (int)(e * sizeof(V) / 16); q += blockDim.x)
      reinterpret_cast<uint4*>(vec[v])[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  t.x[0] = vec[0] + halo; t.x[1] = vec[1] + halo; t.rhs = vec[2] + halo; t.r = vec[3] + halo;
  if (threadIdx.x == 0) s = t;
}

// ---------------------------------------------- node-wise steps on shared-memory levels
// One thread per node on the small levels that the fused tail holds in shared memory: at most a
// few thousand nodes, where one warp per 128-node tile would leave most of the block idle.  Each
// function computes exactly the arithmetic of the corresponding tile step for that node (same
// operands, same order of operations), so the results do not depend on which path ran.

// acc = sum_k a_k[i] x[i + off_k] in band order (FP16: the row-sum form), dg = the diagonal
// DEF (plain band form): acc enters holding b and leaves holding b - A x (the tile step's chain)
template <class Pol, bool DEF = false>
__device__ __forceinline__ void stencil_node(const LevelDev& d, const typename Pol::V* x, int i,
                                             typename Pol::A& acc, typename Pol::A& dg) {
  using A = typename Pol::A;
  using B = typename Pol::B;
  const int n = d.n;
  if constexpr (Pol::prec == P16) {
    const float xi = x[i];
    const float rho = __fmul_rn(d.scale[4], __half2float(static_cast<const B*>(d.band[4])[i]));
    acc = rho * xi;
    dg = rho;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (k == 4) continue;
      const int off = (k / 3 - 1) * n + (k % 3 - 1);
      const float b = __fmul_rn(d.scale[k], __half2float(static_cast<const B*>(d.band[k])[i]));
      acc = fmaf(b, x[i + off] - xi, acc);
      dg -= b;
    }
  } else {
    if constexpr (!DEF) acc = A(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int off = (k / 3 - 1) * n + (k % 3 - 1);
      const A b = static_cast<const B*>(d.band[k])[i];
      acc = DEF ? fma(-b, A(x[i + off]), acc) : fma(b, A(x[i + off]), acc);
      if (k == 4) dg = b;
    }
  }
}

// omega / diag at node i (FP64: the stored array)
template <class Pol>
__device__ __forceinline__ typename Pol::A wd_node(const LevelDev& d, int i, typename Pol::A omega,
                                                   typename Pol::A dg) {
  if constexpr (Pol::prec == P64) return d.wdinv[i];
  else return omega / dg;
}

template <class Pol, int MODE>
__device__ __forceinline__ void band_node(const LevelDev& d, int i, bool zg, int in_sel,
                                          typename Pol::A omega) {
  using A = typename Pol::A;
  using V = typename Pol::V;
  const V* rhs = static_cast<const V*>(d.rhs);
  if constexpr (MODE == M_PRE2B) {
    if (zg && fuses_pre<Pol>()) return;
  }
  if constexpr (MODE == M_JACOBI_FIRST || MODE == M_PRE12) {
    if (zg && (MODE == M_JACOBI_FIRST || !fuses_pre<Pol>())) {   // x = 0: x' = omega D^-1 rhs
      V out;
      if constexpr (Pol::prec == P64) out = d.wdinv[i] * rhs[i];
      else out = d.wdf[i] * A(rhs[i]);
      static_cast<V*>(d.x[1])[i] = out;
      return;
    }
    if constexpr (MODE == M_PRE12 && fuses_pre<Pol>()) {
      if (zg) {                                   // two steps from zero in one pass
        const int n = d.n;
        V x1[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const int j = i + (k / 3 - 1) * n + (k % 3 - 1);
          if constexpr (Pol::prec == P64) x1[k] = mul_rn(d.wdinv[j], rhs[j]);
          else x1[k] = mul_rn(d.wdf[j], rhs[j]);
        }
        A acc;
        if constexpr (Pol::prec == P16) {
          const float rho = __fmul_rn(d.scale[4], __half2float(static_cast<const __half*>(d.band[4])[i]));
          acc = rho * x1[4];
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            if (k == 4) continue;
            const float b = __fmul_rn(d.scale[k], __half2float(static_cast<const __half*>(d.band[k])[i]));
            acc = fmaf(b, x1[k] - x1[4], acc);
          }
        } else if constexpr (def_chain<Pol>()) {
          acc = A(rhs[i]);
#pragma unroll
          for (int k = 0; k < 9; ++k)
            acc = fma(-A(static_cast<const typename Pol::B*>(d.band[k])[i]), A(x1[k]), acc);
        } else {
          acc = A(0);
#pragma unroll
          for (int k = 0; k < 9; ++k)
            acc = fma(A(static_cast<const typename Pol::B*>(d.band[k])[i]), A(x1[k]), acc);
        }
        A wd;
        if constexpr (Pol::prec == P64) wd = d.wdinv[i];
        else wd = d.wdf[i];
        const A r = def_chain<Pol>() ? acc : A(rhs[i]) - acc;
        static_cast<V*>(d.x[0])[i] = fma(wd, r, A(x1[4]));
        return;
      }
    }
  }
  int src = in_sel, dst = 1 - in_sel;
  if constexpr (MODE == M_JACOBI_FIRST || MODE == M_PRE12) { src = 0; dst = 1; }
  if constexpr (MODE == M_PRE2B) { src = 1; dst = 0; }
  const V* xin = static_cast<const V*>(d.x[src]);
  constexpr bool DEF = def_chain<Pol>();
  A acc, dg;
  if constexpr (DEF) acc = A(rhs[i]);
  stencil_node<Pol, DEF>(d, xin, i, acc, dg);
  const A r = DEF ? acc : A(rhs[i]) - acc;
  if constexpr (MODE == M_DEFECT) {
    static_cast<V*>(d.r)[i] = V(r);
  } else {                                        // a Jacobi step src -> dst
    const A wd = wd_node<Pol>(d, i, omega, dg);
    static_cast<V*>(d.x[dst])[i] = fma(wd, r, A(xin[i]));
  }
}

// full-weighting restriction onto coarse node i (the tile step's formula)
template <class V>
__device__ __forceinline__ void restrict_node(const LevelDev& f, const LevelDev& c, int i) {
  const int nc = c.n, J = i / nc, I = i - J * nc;
  const V* r = static_cast<const V*>(f.r);
  static_cast<V*>(c.rhs)[i] = i < nc * nc ? restrict_value<V>(I, J, nc, f.n, c.bc, [&](long long k) { return r[k]; })
                                          : V(0);
}

// x_f[x_sel] += P e_c at fine node i (the tile step's formula)
template <class V>
__device__ __forceinline__ void prolong_node(const LevelDev& f, const LevelDev& c, int x_sel, int i) {
  const int nf = f.n, iy = i / nf, ix = i - iy * nf;
  if (i >= nf * nf) return;
  const V* e = static_cast<const V*>(c.x[0]);
  V add;
  if (!prolong_value<V>(ix, iy, nf, c.n, f.bc, [&](int k) { return e[k]; }, &add)) return;
  V* x = static_cast<V*>(f.x[x_sel]);
  x[i] = x[i] + add;
}

// Down part of the cycle on shared-memory level l (block-wide, node-wise).  The first smoothing
// step of a problem's own finest level from a nonzero iterate takes the tile path, which also
// writes the residual partials of the lagged check; returns false if the problem leaves.
template <class Pol>
__device__ bool vcycle_down_smem(const LevelDev& d, const LevelDev& dc, int l, bool zg, int pre,
                                 typename Pol::A omega, int lane, double* check_part,
                                 ProbState* st, const Params& prm, int want, double* sh) {
  const int tid = threadIdx.x, nt = blockDim.x, np = d.pitch;
  if (check_part) {
    const int tiles = np / kTile, warp = tid >> 5, nwarp = nt >> 5;
    for (int t = warp; t < tiles; t += nwarp) {
      if (pre >= 2)
        band_tile<Pol, M_PRE12, LD_GEN>(d, 1LL << l, zg, (long long)t * kTile + lane * kLaneNodes,
                                        lane, 0, omega, check_part + t);
      else
        band_tile<Pol, M_JACOBI_FIRST, LD_GEN>(d, 1LL << l, zg, (long long)t * kTile + lane * kLaneNodes,
                                               lane, 0, omega, check_part + t);
    }
    __syncthreads();
    const double sum = problem_norm_sum(check_part, fine_tiles(l), sh, Pol::prec != P64);
    if (tid == 0) pre_check(*st, prm, sqrt(sum));
    __syncthreads();
    if (__ldcg(&st->phase) != want) return false;
  } else {
    for (int i = tid; i < np; i += nt) {
      if (pre >= 2) band_node<Pol, M_PRE12>(d, i, zg, 0, omega);
      else band_node<Pol, M_JACOBI_FIRST>(d, i, zg, 0, omega);
    }
    __syncthreads();
  }
  if (pre >= 2) {
    if (!(zg && fuses_pre<Pol>())) {
      for (int i = tid; i < np; i += nt) band_node<Pol, M_PRE2B>(d, i, zg, 0, omega);
      __syncthreads();
    }
    for (int s = 3; s <= pre; ++s) {
      for (int i = tid; i < np; i += nt) band_node<Pol, M_JACOBI>(d, i, zg, (s - 1) & 1, omega);
      __syncthreads();
    }
  }
  for (int i = tid; i < np; i += nt) band_node<Pol, M_DEFECT>(d, i, zg, pre & 1, omega);
  __syncthreads();
  for (int i = tid; i < dc.pitch; i += nt) restrict_node<typename Pol::V>(d, dc, i);
  __syncthreads();
  return true;
}

template <class Pol>
__device__ void vcycle_up_smem(const LevelDev& d, const LevelDev& dc, int pre, int post,
                               typename Pol::A omega) {
  const int tid = threadIdx.x, nt = blockDim.x, np = d.pitch;
  for (int i = tid; i < np; i += nt) prolong_node<typename Pol::V>(d, dc, pre & 1, i);
  __syncthreads();
  for (int s = 1; s <= post; ++s) {
    for (int i = tid; i < np; i += nt) band_node<Pol, M_JACOBI>(d, i, false, (pre + s - 1) & 1, omega);
    __syncthreads();
  }
}

// ------------------------------------------ cluster levels in distributed shared memory
// The levels between the shared-memory levels of block 0 (coarse..S) and the top of the fused
// tail live in the shared memory of the whole cluster: block r holds rows
// [part_row(l, r), part_row(l, r + 1)) of level l (its bands, and its vectors with one ghost row
// on each side).  The partition of level l + 1 is that of level l with every row doubled, so a
// block restricts to, and prolongs from, its own rows of the next coarser level (plus a ghost row).
// After each step a block stores its first and last own rows of the vector it wrote into the ghost
// rows of its neighbours (distributed shared memory), then the cluster synchronizes.

// C is a power of two no larger than 2^(S+1), so block r's first row r * 2^l / C is exact and
// doubles from one level to the next; the last block also takes the last row
__host__ __device__ inline int log2_pow2(int C) { int k = 0; while ((1 << k) < C) ++k; return k; }
__host__ __device__ inline int part_row(int l, int r, int C, int S) {
  (void)S;
  if (r >= C) return (1 << l) + 1;
  return (r << l) >> log2_pow2(C);
}
__host__ __device__ inline int part_maxrows(int l, int C, int S) {
  (void)S;
  return ((1 << l) >> log2_pow2(C)) + 1;
}
__host__ __device__ inline long long align_down(long long x, int a) {   // a: a power of two
  return x & ~(long long)(a - 1);
}
// elements of one block's vector array (own rows, a ghost row and a node on each side, 16-byte
// aligned start) and band array (own rows) of cluster level l
__host__ __device__ inline long long dsm_vec_elems(int l, int C, int S, int esize) {
  const long long n = (1LL << l) + 1;
  const int a = 16 / esize;
  return ((long long)(part_maxrows(l, C, S) + 2) * n + 2 + 3 * a) / a * a;
}
__host__ __device__ inline long long dsm_band_elems(int l, int C, int S, int esize) {
  const long long n = (1LL << l) + 1;
  const int a = 16 / esize;
  return ((long long)part_maxrows(l, C, S) * n + 3 * a) / a * a;
}
__host__ __device__ inline long long dsm_level_bytes(int l, int C, int S, int prec) {
  const int vs = prec == P64 ? 8 : 4, bs = prec == P64 ? 8 : (prec == P32 ? 4 : 2);
  return 9 * dsm_band_elems(l, C, S, bs) * bs + 5 * dsm_vec_elems(l, C, S, vs) * vs;
}

// first global node index of block r's vector arrays of level l
template <class V>
__device__ __forceinline__ long long dsm_vec_start(int l, int r, int C, int S) {
  const long long n = (1LL << l) + 1;
  return align_down((long long)part_row(l, r, C, S) * n - n - 1, 16 / (int)sizeof(V));
}

// carve block r's arrays of cluster level l at *off, bulk-copy its bands (own rows) and omega/D
// (own and ghost rows; thread 0, accounted on bar), zero its vectors; v gets views indexed by
// global node index
template <class Pol>
__device__ void dsm_level_setup(const LevelDev& g, LevelDev& v, unsigned char* base, long long* off,
                                int l, int r, int C, int S, unsigned long long* bar) {
  using V = typename Pol::V;
  using B = typename Pol::B;
  const long long n = (1LL << l) + 1;
  const long long R0n = (long long)part_row(l, r, C, S) * n, R1n = (long long)part_row(l, r + 1, C, S) * n;
  constexpr int av = 16 / (int)sizeof(V), ab = 16 / (int)sizeof(B);
  const long long g0v = dsm_vec_start<V>(l, r, C, S), g0b = align_down(R0n, ab);
  const long long nv = dsm_vec_elems(l, C, S, sizeof(V)), nb = dsm_band_elems(l, C, S, sizeof(B));
  auto take = [&](long long bytes) { unsigned char* p = base + *off; *off += (bytes + 15) / 16 * 16; return p; };
  LevelDev t = g;
  const int bchunks = (int)((R1n - g0b + ab - 1) / ab);
  for (int k = 0; k < 9; ++k) {
    B* dst = reinterpret_cast<B*>(take(nb * sizeof(B)));
    const B* src = static_cast<const B*>(g.band[k]) + g0b;
    block_copy16(dst, src, (long long)bchunks * 16, bar);
    t.band[k] = dst - g0b;
  }
  const int vchunks = (int)((R1n + n + 1 - g0v + av - 1) / av);
  {
    V* dst = reinterpret_cast<V*>(take(nv * sizeof(V)));
    const V* src;
    if constexpr (Pol::prec == P64) src = g.wdinv + g0v;
    else src = g.wdf + g0v;
    block_copy16(dst, src, (long long)vchunks * 16, bar);
    if constexpr (Pol::prec == P64) t.wdinv = dst - g0v;
    else t.wdf = dst - g0v;
  }
  V* vec[4];
  for (int k = 0; k < 4; ++k) {
    vec[k] = reinterpret_cast<V*>(take(nv * sizeof(V)));
    for (int q = threadIdx.x; q < (int)(nv / av); q += blockDim.x)
      reinterpret_cast<uint4*>(vec[k])[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  t.x[0] = vec[0] - g0v; t.x[1] = vec[1] - g0v; t.rhs = vec[2] - g0v; t.r = vec[3] - g0v;
  if (threadIdx.x == 0) v = t;
}

// copy block r's first and last own rows of `view` (level l, indexed by global node index) into
// the ghost rows of blocks r - 1 and r + 1
template <class V>
__device__ void dsm_push(V* view, int l, int r, int C, int S) {
  cg::cluster_group cl = cg::this_cluster();
  const long long n = (1LL << l) + 1;
  V* start = view + dsm_vec_start<V>(l, r, C, S);
  if (r > 0) {
    const long long R0n = (long long)part_row(l, r, C, S) * n;
    V* rv = cl.map_shared_rank(start, r - 1) - dsm_vec_start<V>(l, r - 1, C, S);
    for (int q = threadIdx.x; q < (int)n; q += blockDim.x) rv[R0n + q] = view[R0n + q];
  }
  if (r < C - 1) {
    const long long L1n = (long long)(part_row(l, r + 1, C, S) - 1) * n;
    V* rv = cl.map_shared_rank(start, r + 1) - dsm_vec_start<V>(l, r + 1, C, S);
    for (int q = threadIdx.x; q < (int)n; q += blockDim.x) rv[L1n + q] = view[L1n + q];
  }
}

// one node-wise step on block r's own rows of cluster level l, then the ghost exchange of the
// vector it wrote (dst: 0, 1 = x[0], x[1]; 2 = r; -1 = nothing written)
template <class Pol, int MODE>
__device__ __forceinline__ void dsm_step(const LevelDev& d, int l, int r, int C, int S, bool zg, int in_sel,
                                         typename Pol::A omega, int dst) {
  using V = typename Pol::V;
  const long long n = (1LL << l) + 1;
  const long long R0n = (long long)part_row(l, r, C, S) * n, R1n = (long long)part_row(l, r + 1, C, S) * n;
  for (long long i = R0n + threadIdx.x; i < R1n; i += blockDim.x) band_node<Pol, MODE>(d, (int)i, zg, in_sel, omega);
  __syncthreads();
  if (dst >= 0) dsm_push<V>(static_cast<V*>(dst == 2 ? d.r : d.x[dst]), l, r, C, S);
  cg::this_cluster().sync();
}

// down part of the cycle on cluster level l; the next coarser level is cluster level l - 1, or
// block 0's shared-memory level S (c0: block 0's view of it, addressed through the cluster)
template <class Pol>
__device__ void dsm_down(const LevelDev* cv, const LevelDev& c0, int l, int r, int C, int S, bool zg,
                         int pre, typename Pol::A omega) {
  using V = typename Pol::V;
  const LevelDev& d = cv[l];
  if (pre >= 2) {
    const bool fused = zg && fuses_pre<Pol>();
    dsm_step<Pol, M_PRE12>(d, l, r, C, S, zg, 0, omega, fused ? 0 : 1);
    if (!fused) dsm_step<Pol, M_PRE2B>(d, l, r, C, S, zg, 0, omega, 0);
    for (int s = 3; s <= pre; ++s)
      dsm_step<Pol, M_JACOBI>(d, l, r, C, S, zg, (s - 1) & 1, omega, 1 - ((s - 1) & 1));
  } else {
    dsm_step<Pol, M_JACOBI_FIRST>(d, l, r, C, S, zg, 0, omega, 1);
  }
  dsm_step<Pol, M_DEFECT>(d, l, r, C, S, zg, pre & 1, omega, 2);
  const long long nc = (1LL << (l - 1)) + 1;
  if (l - 1 > S) {
    const LevelDev& dc = cv[l - 1];
    const long long c0n = (long long)part_row(l - 1, r, C, S) * nc, c1n = (long long)part_row(l - 1, r + 1, C, S) * nc;
    for (long long i = c0n + threadIdx.x; i < c1n; i += blockDim.x) restrict_node<V>(d, dc, (int)i);
    __syncthreads();
    dsm_push<V>(static_cast<V*>(dc.rhs), l - 1, r, C, S);
  } else {
    // coarse rows whose centre fine row is one of this block's rows, into block 0
    const int J0 = (part_row(l, r, C, S) + 1) / 2, J1 = (part_row(l, r + 1, C, S) + 1) / 2;
    for (long long i = (long long)J0 * nc + threadIdx.x; i < (long long)J1 * nc; i += blockDim.x)
      restrict_node<V>(d, c0, (int)i);
  }
  cg::this_cluster().sync();
}

// up part on cluster level l.  From block 0's level S, the coarse rows this block interpolates
// from are first copied (one read each through the cluster) into this block's own, otherwise
// unused, copy of level S (buffer x[1], which block 0 no longer needs either).
template <class Pol>
__device__ void dsm_up(const LevelDev* cv, const LevelDev& c0, const LevelDev& s_own, int l, int r,
                       int C, int S, int pre, int post, typename Pol::A omega) {
  using V = typename Pol::V;
  const LevelDev& d = cv[l];
  const long long n = (1LL << l) + 1;
  const long long R0n = (long long)part_row(l, r, C, S) * n, R1n = (long long)part_row(l, r + 1, C, S) * n;
  LevelDev local = s_own;
  if (l - 1 == S) {
    const int nc = (1 << S) + 1;
    const int J0 = part_row(l, r, C, S) >> 1;
    const int J1 = min(part_row(l, r + 1, C, S) >> 1, nc - 1);
    const V* src = static_cast<const V*>(c0.x[0]);
    V* dst = static_cast<V*>(s_own.x[1]);
    for (int i = J0 * nc + threadIdx.x; i < (J1 + 1) * nc; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    local.x[0] = s_own.x[1];
  }
  const LevelDev& dc = l - 1 > S ? cv[l - 1] : local;
  for (long long i = R0n + threadIdx.x; i < R1n; i += blockDim.x) prolong_node<V>(d, dc, pre & 1, (int)i);
  __syncthreads();
  dsm_push<V>(static_cast<V*>(d.x[pre & 1]), l, r, C, S);
  cg::this_cluster().sync();
  for (int s = 1; s <= post; ++s) {
    const int in_sel = (pre + s - 1) & 1;
    dsm_step<Pol, M_JACOBI>(d, l, r, C, S, false, in_sel, omega, 1 - in_sel);
  }
}

// Pre-smoothing, defect and restriction of level l.  check_part (top level with a nonzero
// iterate): the first smoothing step also writes the residual partials, block 0 reduces them and
// takes the lagged convergence decision; returns false if the problem leaves the cycle.
template <class Pol, int LK>
__device__ __forceinline__ bool vcycle_down_level(const LevelDev& d, const LevelDev& dc, int l,
                                                  bool zg, int pre, typename Pol::A omega, int w0,
                                                  int nw, int lane, bool cluster_sync,
                                                  double* check_part, ProbState* st,
                                                  const Params& prm, int want, int rank,
                                                  double* sh) {
  const long long shift = 1LL << l;
  const int tiles = d.pitch / kTile;
  auto sync = [&] { if (cluster_sync) cg::this_cluster().sync(); else __syncthreads(); };
  if (pre >= 2) {
    for (int t = w0; t < tiles; t += nw)
      band_tile<Pol, M_PRE12, LK>(d, shift, zg, (long long)t * kTile + lane * kLaneNodes, lane, 0, omega,
                                  check_part ? check_part + t : nullptr);
  } else {
    for (int t = w0; t < tiles; t += nw)
      band_tile<Pol, M_JACOBI_FIRST, LK>(d, shift, zg, (long long)t * kTile + lane * kLaneNodes, lane, 0, omega,
                                         check_part ? check_part + t : nullptr);
  }
  sync();
  if (check_part) {
    if (rank == 0) {
      const double sum = problem_norm_sum(check_part, fine_tiles(l), sh, Pol::prec != P64);
      if (threadIdx.x == 0) pre_check(*st, prm, sqrt(sum));
    }
    sync();
    if (__ldcg(&st->phase) != want) return false;
  }
  if (pre >= 2) {
    if (!(zg && fuses_pre<Pol>())) {
      for (int t = w0; t < tiles; t += nw)
        band_tile<Pol, M_PRE2B, LK>(d, shift, zg, (long long)t * kTile + lane * kLaneNodes, lane, 0, omega, nullptr);
      sync();
    }
    for (int s = 3; s <= pre; ++s) {
      for (int t = w0; t < tiles; t += nw)
        band_tile<Pol, M_JACOBI, LK>(d, shift, zg, (long long)t * kTile + lane * kLaneNodes, lane, (s - 1) & 1, omega, nullptr);
      sync();
    }
  }
  for (int t = w0; t < tiles; t += nw)
    band_tile<Pol, M_DEFECT, LK>(d, shift, zg, (long long)t * kTile + lane * kLaneNodes, lane, pre & 1, omega, nullptr);
  sync();
  const int ctiles = dc.pitch / kTile;
  for (int t = w0; t < ctiles; t += nw)
    restrict_tile<typename Pol::V, LK>(d, dc, (long long)t * kTile, lane);
  sync();
  return true;
}

template <class Pol, int LK>
__device__ __forceinline__ void vcycle_up_level(const LevelDev& d, const LevelDev& dc, int l, int pre,
                                                int post, typename Pol::A omega, int w0, int nw,
                                                int lane, bool cluster_sync) {
  const long long shift = 1LL << l;
  const int tiles = d.pitch / kTile;
  auto sync = [&] { if (cluster_sync) cg::this_cluster().sync(); else __syncthreads(); };
  for (int t = w0; t < tiles; t += nw)
    prolong_tile<typename Pol::V, LK>(d, dc, pre & 1, (long long)t * kTile + lane * kLaneNodes);
  sync();
  for (int s = 1; s <= post; ++s) {
    for (int t = w0; t < tiles; t += nw)
      band_tile<Pol, M_JACOBI, LK>(d, shift, false, (long long)t * kTile + lane * kLaneNodes, lane, (pre + s - 1) & 1, omega, nullptr);
    sync();
  }
}

constexpr int kTailThreads = 512;

// dsm: the cluster levels (S, T] live in distributed shared memory (the launch reserved room for
// them); otherwise they run over global memory through L2
template <class Pol>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(EngineDev E, int T, int S, int want, int dsm) {
  using A = typename Pol::A;
  using V = typename Pol::V;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ LevelDev gd[kMaxLevel + 1];       // global-memory descriptors of this problem
  __shared__ LevelDev sd[kMaxLevel + 1];       // shared-memory levels coarse..S (block 0's data)
  __shared__ LevelDev cv[kMaxLevel + 1];       // this block's rows of the cluster levels
  __shared__ double sol[kMaxCoarseM];
  __shared__ double rd[kMaxCoarseM];          // coarse right-hand side in FP64
  __shared__ double sh[32];
  __shared__ const double* s_cinv;
  __shared__ __align__(8) unsigned long long s_bar;   // bulk copies: phase 0 constant data, 1 inputs
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int p = blockIdx.x / csize;
  pdl_trigger();
  if (p >= E.nprob) return;
  // constant data before the wait for the preceding launch: the level descriptors, the bands of
  // block 0's shared-memory levels and of this block's rows of the cluster levels (asynchronous
  // copies, completed before first use).  Descriptors change only between launches (host
  // copies); an empty slot's is all zero.
  const ProblemDev& P = E.P[p];
  if (P.L < HN_MIN_LEVEL) return;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int top = P.L < T ? P.L : T, c = P.coarse;
  const int Ss = S < top ? S : top;
  const int m = P.m;
  const bool use_dsm = dsm && top > Ss;
  {
    const int words = (int)(sizeof(LevelDev) / 4) * (top - c + 1);
    const unsigned* src = reinterpret_cast<const unsigned*>(&P.lev[c]);
    unsigned* dst = reinterpret_cast<unsigned*>(&gd[c]);
    for (int q = threadIdx.x; q < words; q += blockDim.x) dst[q] = src[q];
    if (threadIdx.x == 0) {
      mbar_init(&s_bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
  }
  long long off = 0;
  for (int l = c; l <= Ss; ++l) smem_level_setup<Pol>(gd[l], sd[l], smem, &off, l, rank == 0, &s_bar);
  double* cg_pq = nullptr;                      // CG coarse solver: p and q (N_c doubles each)
  {   // the coarse inverse (m*m doubles; CG: the 9 FP64 coarse bands, 9 N_c doubles) is staged in
      // shared memory when it is small
    const int Nc = (int)(n_of_dev(c) * n_of_dev(c));
    const long long words = E.prm.coarse_cg ? 9LL * Nc : (long long)m * m;
    const bool staged = words * 8 <= kCinvSmemMax;
    double* dst = reinterpret_cast<double*>(smem + off);
    if (staged) off += (words * 8 + 15) / 16 * 16;
    if (E.prm.coarse_cg) {
      cg_pq = reinterpret_cast<double*>(smem + off);
      off += ((long long)2 * Nc * 8 + 15) / 16 * 16;
    }
    if (rank == 0) {
      if (staged) block_copy16(dst, P.cinv, (words / 2) * 16, &s_bar);
      if (threadIdx.x == 0) {
        if (staged && (words & 1)) dst[words - 1] = __ldg(P.cinv + words - 1);
        s_cinv = staged ? dst : P.cinv;
      }
    }
  }
  if (use_dsm)
    for (int l = Ss + 1; l <= top; ++l) dsm_level_setup<Pol>(gd[l], cv[l], smem, &off, l, rank, csize, Ss, &s_bar);
  if (threadIdx.x == 0) mbar_arrive(&s_bar);   // all constant-data copies issued
  fence_proxy_async();                          // the zeroed vectors before later bulk copies into them
  __syncthreads();                              // shared-memory descriptors published
  pdl_wait();
  // a copy that does not land in time (it always does) sets the error word; the block still
  // waits, bounded, before it reads the data or exits
  auto wait_copies = [&](unsigned parity) {
    if (!mbar_wait(&s_bar, parity)) {
      if (threadIdx.x == 0) atomicExch(E.err, 1);
      (void)mbar_wait(&s_bar, parity);
    }
  };
  const ProbState& st = E.S[p];
  if (st.phase != want) {
    wait_copies(0);                             // no copy outlives the block
    cp_async_wait();
    return;
  }
  const int pre = E.prm.pre, post = E.prm.post;
  const A omega = A(E.prm.omega);
  const bool zero_top = st.zero_top;
  ProbState* stw = E.S + p;
  double* check_part = E.partial + E.fine_off[p];   // used on the problem's own finest level
  // the distributed path needs no residual check on a cluster level (only the top one can be the
  // problem's own finest level); otherwise the cluster levels run over L2
  const bool dsm_ok = use_dsm && !(top == P.L && !zero_top);
  // block 0's level Ss as seen from any block of the cluster
  LevelDev c0 = sd[Ss];
  c0.rhs = cl.map_shared_rank(static_cast<V*>(sd[Ss].rhs), 0);
  c0.x[0] = cl.map_shared_rank(static_cast<V*>(sd[Ss].x[0]), 0);
  const int w0 = rank * wpb + (threadIdx.x >> 5), nw = csize * wpb;
  if (dsm_ok) {
    wait_copies(0);                             // the next phase of bar may start only now
    cp_async_wait();                            // the constant data of this block's levels
    __syncthreads();
    {   // right-hand side of the top level: own and ghost rows
      const LevelDev& g = gd[top];
      const long long n = (1LL << top) + 1;
      const long long g0 = dsm_vec_start<V>(top, rank, csize, Ss);
      const long long R1n = (long long)part_row(top, rank + 1, csize, Ss) * n;
      constexpr int av = 16 / (int)sizeof(V);
      const int chunks = (int)((R1n + n + 1 - g0 + av - 1) / av);
      V* dst = static_cast<V*>(cv[top].rhs) + g0;
      const V* src = static_cast<const V*>(g.rhs) + g0;
      if (threadIdx.x == 0) {
        bulk_copy(dst, src, (unsigned)chunks * 16u, &s_bar);
        mbar_arrive(&s_bar);
      }
    }
    wait_copies(1);
    __syncthreads();
    cl.sync();                                  // every block's arrays are ready for its neighbours
    for (int l = top; l > Ss; --l) dsm_down<Pol>(cv, c0, l, rank, csize, Ss, true, pre, omega);
  } else {
    wait_copies(0);
    cp_async_wait();                            // the constant data of this block's levels
    __syncthreads();
    // cluster part over L2, down
    for (int l = top; l > Ss; --l) {
      const bool chk = (l == P.L) && !zero_top;
      if (!vcycle_down_level<Pol, LD_CG>(gd[l], gd[l - 1], l, (P.L > l) || zero_top, pre, omega, w0, nw,
                                         lane, true, chk ? check_part : nullptr, stw, E.prm, want, rank, sh))
        return;                                 // converged at the lagged check: cluster-uniform
    }
  }
  // block 0: levels coarse..Ss in shared memory, one thread per node
  if (rank == 0) {
    if (!(dsm_ok && top > Ss)) {
      // inputs of level Ss: restricted rhs (or the top rhs), and the iterate if it is nonzero
      const LevelDev& g = gd[Ss];
      const LevelDev& s = sd[Ss];
      const bool nonzero = (Ss == P.L) && !zero_top;
      const int chunks = (int)(g.pitch * sizeof(V) / 16);
      for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
        cp_async16(static_cast<uint4*>(s.rhs) + q, static_cast<const uint4*>(g.rhs) + q);
        if (nonzero) cp_async16(static_cast<uint4*>(s.x[0]) + q, static_cast<const uint4*>(g.x[0]) + q);
      }
      cp_async_wait();
    }
    __syncthreads();
    bool go = true;
    for (int l = Ss; l > c && go; --l) {
      const bool chk = (l == P.L) && !zero_top;
      go = vcycle_down_smem<Pol>(sd[l], sd[l - 1], l, (P.L > l) || zero_top, pre, omega, lane,
                                 chk ? check_part : nullptr, stw, E.prm, want, sh);
    }
    if (go && c == P.L && !zero_top) {
      // the problem is the coarsest level alone: its residual check before the exact solve
      const LevelDev& d = sd[c];
      const int sw0 = threadIdx.x >> 5;
      for (int t = sw0; t < d.pitch / kTile; t += wpb)
        band_tile<Pol, M_CHECK, LD_GEN>(d, 1LL << c, false, (long long)t * kTile + lane * kLaneNodes, lane, 0,
                                        omega, check_part + t);
      __syncthreads();
      const double sum = problem_norm_sum(check_part, fine_tiles(c), sh, Pol::prec != P64);
      if (threadIdx.x == 0) pre_check(*stw, E.prm, sqrt(sum));
      __syncthreads();
      go = __ldcg(&stw->phase) == want;
    }
    if (go) {
      // the coarsest level: the exact solve with the FP64 inverse, one thread per unknown
      const LevelDev& d = sd[c];
      const int n = d.n;
      const UnknownRect ur = unknown_rect(n, d.bc);
      const V* rhs = static_cast<const V*>(d.rhs);
      const double* cinv = s_cinv;
      V* x = static_cast<V*>(d.x[0]);
      if (E.prm.coarse_cg) {
        // CG over all nodes of the level (sol, rd: N_c <= kMaxCoarseM doubles)
        const int Nc = n * n;
        for (int i = threadIdx.x; i < Nc; i += blockDim.x)
          rd[i] = is_dirichlet(i % n, i / n, n, d.bc) ? 0.0 : double(rhs[i]);
        __syncthreads();
        coarse_cg(cinv, n, m, sol, rd, cg_pq, cg_pq + Nc, sh);
        for (int q = threadIdx.x; q < d.pitch; q += blockDim.x) x[q] = q < Nc ? V(sol[q]) : V(0);
      } else {
        for (int v = threadIdx.x; v < m; v += blockDim.x)
          rd[v] = double(rhs[(v / ur.nx + ur.y0) * n + (v % ur.nx + ur.x0)]);
        __syncthreads();
        for (int u = threadIdx.x; u < m; u += blockDim.x)
          sol[u] = coarse_dot(cinv + u * m, m, [&](int v) { return rd[v]; });
        __syncthreads();
        for (int q = threadIdx.x; q < d.pitch; q += blockDim.x) {
          const int iy = q / n - ur.y0, ix = q - (q / n) * n - ur.x0;
          V val = V(0);
          if (q < n * n && ix >= 0 && iy >= 0 && ix < ur.nx && iy < ur.ny) val = V(sol[iy * ur.nx + ix]);
          x[q] = val;
        }
      }
      __syncthreads();
      for (int l = c + 1; l <= Ss; ++l) vcycle_up_smem<Pol>(sd[l], sd[l - 1], pre, post, omega);
      if (!dsm_ok) {   // the iterate of level Ss back to global memory
        const LevelDev& g = gd[Ss];
        const LevelDev& s = sd[Ss];
        const int chunks = (int)(g.pitch * sizeof(V) / 16);
        for (int q = threadIdx.x; q < chunks; q += blockDim.x)
          static_cast<uint4*>(g.x[0])[q] = static_cast<const uint4*>(s.x[0])[q];
      }
    }
  }
  cl.sync();
  if (dsm_ok) {
    for (int l = Ss + 1; l <= top; ++l) dsm_up<Pol>(cv, c0, sd[Ss], l, rank, csize, Ss, pre, post, omega);
    // the top level's iterate (own rows) back to global memory
    const long long n = (1LL << top) + 1;
    const long long R0n = (long long)part_row(top, rank, csize, Ss) * n;
    const long long R1n = (long long)part_row(top, rank + 1, csize, Ss) * n;
    const V* xs = static_cast<const V*>(cv[top].x[0]);
    V* xg = static_cast<V*>(gd[top].x[0]);
    for (long long i = R0n + threadIdx.x; i < R1n; i += blockDim.x) xg[i] = xs[i];
  } else {
    // cluster part over L2, up
    for (int l = Ss + 1; l <= top; ++l)
      vcycle_up_level<Pol, LD_CG>(gd[l], gd[l - 1], l, pre, post, omega, w0, nw, lane, true);
  }
}

// ------------------------------------------------------ fused level sweeps over 2-D tiles
// An engine of one problem running V(2,2) cycles may take the down part of a level above the fused
// tail (the two pre-smoothing steps, the defect and the restriction) and the up part (the
// prolongation and the two post-smoothing steps) as one launch each, in place of three.  A block
// takes a tile of the coarse grid, coarse columns I0..I1-1 and rows J0..J1-1 (cx x cy coarse
// nodes; the last tile of a row or column also takes the leftover boundary node), and owns the
// fine nodes 2 I0 .. 2 I1 - 1 (clipped to the grid) in each direction.  Each step is recomputed on
// a halo as wide as the steps after it read, so blocks exchange nothing: the restriction reads
// the defect on fine columns 2 I0 - 1 .. 2 I1 - 1, the defect reads the second iterate one node
// further out, the second iterate reads the first one a node further still.  The tile-local copy
// of the level (bands, right-hand side, omega / D, both iterates, the defect) sits in shared
// memory with row pitch P = 2 cx + 7 and origin at fine node (2 I0 - 3, 2 J0 - 3), zero off the
// grid (where every coupling of a grid node is zero), and every value is computed by the node-wise
// steps of the fused tail's shared-memory levels (band_node: the tile steps' operands and order),
// so a fused sweep stores the bits the separate launches store.  A tile's inputs arrive by
// asynchronous copies (cp.async, zero-filled off the grid) that all its threads issue before one
// wait: one memory latency per tile.  The up sweep writes its result to buffer 1 (the halos of
// other blocks still read buffer 0); the next finer level's prolongation reads it there.
constexpr int kSweepCX = 16, kSweepCY = 16;      // coarse nodes per tile (largest)
// threads per tile: about one node of the widest region each, so that a tile's chain of dependent
// steps is short (a tile is latency-bound: 256 threads took ~10 us per tile at L = 8)
constexpr int kSweepThreads = 1024;
struct SweepTile { int I0, I1, J0, J1, ox, oy; };

__device__ __forceinline__ SweepTile sweep_tile(const SweepGeom& g, int nc, int tile) {
  SweepTile t;
  const int by = tile / g.tx, bx = tile - by * g.tx;
  t.I0 = bx * g.cx;
  t.I1 = bx == g.tx - 1 ? nc : t.I0 + g.cx;
  t.J0 = by * g.cy;
  t.J1 = by == g.ty - 1 ? nc : t.J0 + g.cy;
  t.ox = 2 * t.I0 - 3;
  t.oy = 2 * t.J0 - 3;
  return t;
}

// f(tile-local index, x, y, on the grid) for every fine node (x, y) of [x0, x1) x [y0, y1),
// strided over the block
template <class F>
__device__ __forceinline__ void sweep_region(const SweepTile& t, int P, int n, int x0, int x1, int y0,
                                             int y1, F&& f) {
  const int w = x1 - x0, cnt = w * (y1 - y0);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int v = q / w, u = q - v * w;
    const int gx = x0 + u, gy = y0 + v;
    f((gx - t.ox) + (gy - t.oy) * P, gx, gy, gx >= 0 && gy >= 0 && gx < n && gy < n);
  }
}

// an asynchronous copy of one 4- or 8-byte element to shared memory; with on == false nothing is
// read and the element is zero-filled (a source size of 0)
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem_dst, const void* gmem_src, bool on) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const unsigned sz = on ? (unsigned)BYTES : 0u;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(gmem_src), "n"(BYTES), "r"(sz)
               : "memory");
}
// element li of a tile-local array from element gi of a level array (zero if !on)
template <class T>
__device__ __forceinline__ void cp_elem(const void* dst, int li, const void* src, long long gi, bool on) {
  cp_async_elem<(int)sizeof(T)>(const_cast<T*>(static_cast<const T*>(dst)) + li,
                                static_cast<const T*>(src) + (on ? gi : 0), on);
}
// the 9 bands of grid node gi into tile-local element li.  Halves go in 4-byte pairs: the tile-local
// and global indices of a node have the same parity (P and n are odd, the origin's coordinates
// odd), so a node of even index copies itself and its right neighbour, a node of odd index whose
// left neighbour is not copied (left_in false) copies the pair ending at itself.
template <class Pol>
__device__ __forceinline__ void cp_bands(const LevelDev& t, const LevelDev& g, int li, long long gi,
                                         bool left_in) {
  using B = typename Pol::B;
  if constexpr (Pol::prec == P16) {
    int l2;
    long long g2;
    if ((gi & 1) == 0) { l2 = li; g2 = gi; }
    else if (!left_in) { l2 = li - 1; g2 = gi - 1; }
    else return;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      cp_async_elem<4>(const_cast<B*>(static_cast<const B*>(t.band[k])) + l2, static_cast<const B*>(g.band[k]) + g2,
                       true);
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) cp_elem<B>(t.band[k], li, g.band[k], gi, true);
  }
}

// the tile-local level in dynamic shared memory (the host sizes it by sweep_smem_bytes); e: the
// coarse iterate around the tile (up sweep), pitch cx + 4.  Every thread forms the descriptor in its
// own registers (the node-wise steps read its pointers for every node).
template <class Pol>
__device__ __forceinline__ void sweep_carve(LevelDev& t, const LevelDev& g, unsigned char* base,
                                            const SweepGeom& sg, typename Pol::V** e) {
  using B = typename Pol::B;
  using V = typename Pol::V;
  const long long cnt = (long long)sg.P * sg.R;
  long long off = 0;
  auto take = [&](long long bytes) { unsigned char* r = base + off; off += (bytes + 15) / 16 * 16; return r; };
  t = g;                                          // scales, boundary mask
  for (int k = 0; k < 9; ++k) t.band[k] = take(cnt * (long long)sizeof(B));
  if constexpr (Pol::prec == P64) t.wdinv = reinterpret_cast<const double*>(take(cnt * 8));
  else t.wdf = reinterpret_cast<const float*>(take(cnt * 4));
  t.x[0] = take(cnt * (long long)sizeof(V));
  t.x[1] = take(cnt * (long long)sizeof(V));
  t.rhs = take(cnt * (long long)sizeof(V));
  t.r = take(cnt * (long long)sizeof(V));
  *e = reinterpret_cast<V*>(take((long long)(sg.cx + 4) * (sg.cy + 4) * (long long)sizeof(V)));
  t.n = sg.P;
  t.pitch = (int)cnt;
}

__device__ __forceinline__ bool sweep_geom_ok(const EngineDev& E, const SweepGeom& sg, int nc, int line) {
#if HN_DEBUG_CHECKS
  const bool ok = sg.cx >= 1 && sg.cy >= 1 && sg.tx * sg.cx == nc - 1 && sg.ty * sg.cy == nc - 1 &&
                  sg.P == 2 * sg.cx + 7 && sg.R == 2 * sg.cy + 7;
  if (!ok) dbg_fail(E, line, sg.cx, sg.cy);
  return ok;
#else
  (void)E; (void)sg; (void)nc; (void)line;
  return true;
#endif
}

// Down sweep of level `level`.  top = 0: the iterate of the level is zero (a level below the
// problem's own finest, or the preconditioner's cycle of CG): both smoothing steps from b, as
// M_PRE12 forms them.  top = 1: the problem's own finest level, whose first smoothing step (with
// the lagged check) ran before: the second step from buffer 1 (M_PRE2B), or, in the first cycle
// from a zero iterate, where the first launch took both steps, the defect of buffer 0 alone.
template <class Pol>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_down(EngineDev E, TileList tl, int level, int want,
                                                              int top, SweepGeom sg) {
  using A = typename Pol::A;
  using V = typename Pol::V;
  using W = typename std::conditional<Pol::prec == P64, double, float>::type;   // omega / D
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_start();
  const ProbState& st = E.S[0];
  if (st.phase != want) return;
  const LevelDev& g = tl.solo_d;
  const LevelDev& gc = tl.solo_c;
  if (tl.solo_tiles == 0 || gc.n == 0) return;    // (a level the problem does not have, or no coarser)
  if (!dbg_level(E, g, level, tl.solo_tiles, __LINE__) || !dbg_level(E, gc, level - 1, 0, __LINE__) ||
      !sweep_geom_ok(E, sg, gc.n, __LINE__))
    return;
  // below the problem's own finest level the iterate starts at zero whatever the launch says (an
  // engine whose graphs serve any member level launches every level as a possible top)
  const int mode = (!top || tl.solo_L > level) ? 0 : (st.zero_top ? 2 : 1);
  LevelDev t;
  V* es;
  sweep_carve<Pol>(t, g, smem, sg, &es);
  (void)es;
  const int n = g.n, nc = gc.n, P = sg.P;
  const A omega = A(E.prm.omega);
  V* x0s = static_cast<V*>(t.x[0]);
  const V* rs = static_cast<const V*>(t.r);
  V* xg = static_cast<V*>(g.x[0]);
  V* rc = static_cast<V*>(gc.rhs);
  const void* wds = Pol::prec == P64 ? static_cast<const void*>(t.wdinv) : static_cast<const void*>(t.wdf);
  const void* wdg = Pol::prec == P64 ? static_cast<const void*>(g.wdinv) : static_cast<const void*>(g.wdf);
  for (int tile = blockIdx.x; tile < sg.tx * sg.ty; tile += gridDim.x) {
    const SweepTile w = sweep_tile(sg, nc, tile);
    // the defect's region; the second iterate's is one node wider, the first iterate's two
    const int ax = 2 * w.I0 - 1, bx = 2 * w.I1, ay = 2 * w.J0 - 1, by = 2 * w.J1;
    // the bands on the region of the first step computed here (mode 2: the defect's)
    const int bx0 = mode == 2 ? ax : ax - 1;
    sweep_region(w, P, n, ax - 2, bx + 2, ay - 2, by + 2, [&](int li, int gx, int gy, bool on) {
      const long long gi = (long long)gy * n + gx;
      const bool in2 = gx >= ax - 1 && gx < bx + 1 && gy >= ay - 1 && gy < by + 1;
      const bool inr = gx >= ax && gx < bx && gy >= ay && gy < by;
      const bool inb = mode == 2 ? inr : in2;
      if (mode == 0) {
        cp_elem<V>(t.rhs, li, g.rhs, gi, on);
        cp_elem<W>(wds, li, wdg, gi, on);
      } else if (mode == 1) {
        cp_elem<V>(t.x[1], li, g.x[1], gi, on);
        if (in2) {
          cp_elem<V>(t.rhs, li, g.rhs, gi, on);
          if constexpr (Pol::prec == P64) cp_elem<W>(wds, li, wdg, gi, on);
        }
      } else {
        if (in2) cp_elem<V>(t.x[0], li, g.x[0], gi, on);
        if (inr) cp_elem<V>(t.rhs, li, g.rhs, gi, on);
      }
      if (inb && on) cp_bands<Pol>(t, g, li, gi, gx - 1 >= bx0 && gx >= 1);
    });
    cp_async_wait();
    __syncthreads();
    if (mode != 2) {
      // the second iterate; the block's own nodes also go to buffer 0 of the level
      sweep_region(w, P, n, ax - 1, bx + 1, ay - 1, by + 1, [&](int li, int gx, int gy, bool on) {
        if (!on) { x0s[li] = V(0); return; }
        if (mode == 0) band_node<Pol, M_PRE12>(t, li, true, 0, omega);
        else band_node<Pol, M_PRE2B>(t, li, false, 0, omega);
        if (gx >= 2 * w.I0 && gx < 2 * w.I1 && gy >= 2 * w.J0 && gy < 2 * w.J1)
          xg[(long long)gy * n + gx] = x0s[li];
      });
      __syncthreads();
    }
    sweep_region(w, P, n, ax, bx, ay, by, [&](int li, int, int, bool on) {
      if (on) band_node<Pol, M_DEFECT>(t, li, false, 0, omega);
    });
    __syncthreads();
    // the restriction onto the block's own coarse nodes
    const int cw = w.I1 - w.I0, cnt = cw * (w.J1 - w.J0);
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const int jj = q / cw, J = w.J0 + jj, I = w.I0 + (q - jj * cw);
      rc[(long long)J * nc + I] = restrict_value_xy<V>(I, J, nc, n, gc.bc, [&](int y, int x) {
        return rs[(x - w.ox) + (y - w.oy) * P];
      });
    }
    __syncthreads();
  }
  if (blockIdx.x == 0)                            // the coarse padding nodes, as the restriction kernel
    for (int q = nc * nc + threadIdx.x; q < gc.pitch; q += blockDim.x) rc[q] = V(0);
}

// Up sweep of level `level` (below the problem's own finest level): x + P e_c from buffer 0 and
// the coarse iterate in buffer e_sel, then the two post-smoothing steps; the result to buffer 1.
template <class Pol>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_up(EngineDev E, TileList tl, int level, int want,
                                                            int e_sel, SweepGeom sg) {
  using A = typename Pol::A;
  using V = typename Pol::V;
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_start();
  const ProbState& st = E.S[0];
  if (st.phase != want) return;
  const LevelDev& g = tl.solo_d;
  const LevelDev& gc = tl.solo_c;
  if (tl.solo_tiles == 0 || gc.n == 0) return;
  if (!dbg_level(E, g, level, tl.solo_tiles, __LINE__) || !dbg_level(E, gc, level - 1, 0, __LINE__) ||
      !sweep_geom_ok(E, sg, gc.n, __LINE__))
    return;
  LevelDev t;
  V* es;
  sweep_carve<Pol>(t, g, smem, sg, &es);
  const int n = g.n, nc = gc.n, P = sg.P, Pe = sg.cx + 4;
  const A omega = A(E.prm.omega);
  V* x0s = static_cast<V*>(t.x[0]);
  V* x1s = static_cast<V*>(t.x[1]);
  const V* e = static_cast<const V*>(gc.x[e_sel & 1]);
  V* out = static_cast<V*>(g.x[1]);
  for (int tile = blockIdx.x; tile < sg.tx * sg.ty; tile += gridDim.x) {
    const SweepTile w = sweep_tile(sg, nc, tile);
    const int ax = 2 * w.I0, bx = min(2 * w.I1, n), ay = 2 * w.J0, by = min(2 * w.J1, n);   // own
    // the iterate two nodes around the own ones; bands, rhs (and omega / D) one node around
    sweep_region(w, P, n, ax - 2, bx + 2, ay - 2, by + 2, [&](int li, int gx, int gy, bool on) {
      const long long gi = (long long)gy * n + gx;
      cp_elem<V>(t.x[0], li, g.x[0], gi, on);
      if (gx >= ax - 1 && gx < bx + 1 && gy >= ay - 1 && gy < by + 1) {
        cp_elem<V>(t.rhs, li, g.rhs, gi, on);
        if constexpr (Pol::prec == P64) cp_elem<double>(t.wdinv, li, g.wdinv, gi, on);
        if (on) cp_bands<Pol>(t, g, li, gi, gx - 1 >= ax - 1 && gx >= 1);
      }
    });
    // the coarse iterate on coarse columns I0-1 .. I1+1 and rows J0-1 .. J1+1
    const int ew = w.I1 - w.I0 + 3, ecnt = ew * (w.J1 - w.J0 + 3);
    for (int q = threadIdx.x; q < ecnt; q += blockDim.x) {
      const int v = q / ew, u = q - v * ew;
      const int cxg = w.I0 - 1 + u, cyg = w.J0 - 1 + v;
      cp_elem<V>(es, u + v * Pe, e, (long long)cyg * nc + cxg, cxg >= 0 && cyg >= 0 && cxg < nc && cyg < nc);
    }
    cp_async_wait();
    __syncthreads();
    // y = x + P e_c (prolong_node's values; off the grid and at Dirichlet nodes x itself)
    sweep_region(w, P, n, ax - 2, bx + 2, ay - 2, by + 2, [&](int li, int gx, int gy, bool on) {
      if (!on) return;
      V add;
      if (prolong_value_xy<V>(gx, gy, n, g.bc, [&](int cy, int cx) {
            return es[(cx - (w.I0 - 1)) + (cy - (w.J0 - 1)) * Pe];
          }, &add))
        x0s[li] = x0s[li] + add;
    });
    __syncthreads();
    sweep_region(w, P, n, ax - 1, bx + 1, ay - 1, by + 1, [&](int li, int, int, bool on) {
      if (on) band_node<Pol, M_JACOBI>(t, li, false, 0, omega);
      else x1s[li] = V(0);
    });
    __syncthreads();
    sweep_region(w, P, n, ax, bx, ay, by, [&](int li, int gx, int gy, bool) {
      band_node<Pol, M_JACOBI>(t, li, false, 1, omega);
      out[(long long)gy * n + gx] = x0s[li];
    });
    __syncthreads();
  }
}

// ------------------------------------------------- persistent kernels of the middle levels
// The levels between the fused coarse-level kernel (k_tail, levels coarse..T) and a top level M
// run in two cooperative launches per V cycle: k_mid_down does pre-smoothing, defect and
// restriction on levels M..T+1, k_mid_up prolongation and post-smoothing on levels T+1..M.  All
// blocks of a cooperative launch are resident at once, so the steps are separated by grid-wide
// barriers instead of kernel boundaries.  The lagged convergence test of a problem whose finest
// level lies in this range is taken by the last block to reach the barrier after that level's
// first smoothing step, in the fixed summation order every other path uses.  Each step calls the
// same tile functions as the per-level kernels (vectors written inside the launch are read from
// L2), so the results do not depend on which path ran.  An engine of one problem copies its level
// descriptors to shared memory once per launch, so that no step waits on descriptor loads.

// wait limit of a grid barrier (globaltimer ns): a barrier that does not complete by then sets
// the error word, and every block leaves the kernel at its next barrier
constexpr unsigned long long kGridWaitNs = 500ull * 1000ull * 1000ull;

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;\n" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;\n" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// bounded wait (one thread) until *p >= target; false if it gave up or found the error word set
__device__ bool wait_at_least(const unsigned long long* p, unsigned long long target, int* err) {
  if (ld_acquire64(p) >= target) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (ld_acquire64(p) >= target) return true;
    if (*reinterpret_cast<volatile int*>(err) != 0) return false;
    if (global_ns() - t0 > kGridWaitNs) {
      atomicExch(err, 3);
      return false;
    }
  }
}

// Grid barrier state (used by thread 0 of each block).  cnt counts the arrivals of every launch
// of one kernel (monotonic; each launch has the same grid, so a launch starts at a multiple of
// it), done the barrier actions completed.  Both are read at the start of a launch, before any
// block of the launch can have completed a barrier.
struct GridBar {
  unsigned long long* cnt;
  unsigned long long* done;
  unsigned long long target, dtarget;
};

__device__ __forceinline__ void grid_bar_init(GridBar& g, unsigned long long* cnt, unsigned long long* done) {
  g.cnt = cnt;
  g.done = done;
  g.target = 0;
  g.dtarget = 0;
  if (threadIdx.x == 0) {
    g.target = ld_acquire64(cnt) / gridDim.x * gridDim.x;
    g.dtarget = ld_acquire64(done);
  }
}

// Grid-wide barrier of a cooperative launch.  With ACTION, the last block to arrive runs last()
// (block-wide) before any block goes on.  Returns false in every thread of a block whose wait gave
// up or that found the error word set (another block gave up): the block then leaves the kernel.
template <bool ACTION, class F>
__device__ bool grid_sync(const EngineDev& E, GridBar& g, F&& last) {
  __shared__ int s_state;                       // 1: runs the action; 0: go on; -1: failed
  __syncthreads();
  if (threadIdx.x == 0) {
    g.target += gridDim.x;
    const unsigned long long old = atom_add_acq_rel64(g.cnt, 1ull);   // releases this block's writes
    if (ACTION) {
      g.dtarget += 1;
      s_state = old + 1 == g.target ? 1 : (wait_at_least(g.done, g.dtarget, E.err) ? 0 : -1);
    } else {
      s_state = wait_at_least(g.cnt, g.target, E.err) ? 0 : -1;
    }
  }
  __syncthreads();
  if (ACTION && s_state == 1) {
    last();
    __syncthreads();
    if (threadIdx.x == 0) st_release64(g.done, g.dtarget);
    return true;
  }
  return s_state == 0;
}

template <class Pol> constexpr int mid_threads() { return Pol::prec == P64 ? 512 : 1024; }

// Per-block view of an engine of one problem: its descriptors of levels T..M (shared memory),
// its finest level, and whether it is in the phase the launch serves.
struct MidSolo {
  LevelDev lev[kMaxLevel + 1];
  int on, L, in_phase, zero_top;
};

__device__ void mid_solo_load(const EngineDev& E, const TileList* lists, int M, int T, int want,
                              MidSolo& ms) {
  if (threadIdx.x == 0) {
    ms.on = lists[M].solo_tiles > 0;
    ms.L = lists[M].solo_L;
    ms.in_phase = __ldcg(&E.S[0].phase) == want;
    ms.zero_top = __ldcg(&E.S[0].zero_top);
  }
  constexpr int words = (int)(sizeof(LevelDev) / 4);
  for (int q = threadIdx.x; q < words * (M - T + 1); q += blockDim.x) {
    const int l = T + q / words, w = q - (q / words) * words;
    reinterpret_cast<unsigned*>(&ms.lev[l])[w] = reinterpret_cast<const unsigned*>(&lists[l].solo_d)[w];
  }
  __syncthreads();
  if (threadIdx.x == 0 && ms.on)
    for (int l = T; l <= M; ++l)
      if (!dbg_level(E, ms.lev[l], l, (int)(ms.lev[l].pitch / kTile), __LINE__)) ms.in_phase = 0;
  __syncthreads();
}

// One pass of band-kernel mode MODE over level l of every problem in phase `want`, spread over all
// warps of the grid.
template <class Pol, int MODE>
__device__ __forceinline__ void mid_band_pass(const EngineDev& E, const MidSolo& ms, const TileList& tl,
                                              int l, int want, int in_sel, int gw, int nw, int lane) {
  using A = typename Pol::A;
  const A omega = A(E.prm.omega);
  const long long shift = 1LL << l;
  if (ms.on) {
    if (!ms.in_phase) return;
    const bool zg = (ms.L > l) || ms.zero_top;
    const bool slot = (MODE == M_PRE12 || MODE == M_JACOBI_FIRST) && l == ms.L && !zg;
    const int tiles = ms.lev[l].pitch / kTile;
    for (int t = gw; t < tiles; t += nw)
      band_tile<Pol, MODE, LD_CG>(ms.lev[l], shift, zg, (long long)t * kTile + lane * kLaneNodes, lane,
                                  in_sel, omega, slot ? E.partial + t : nullptr);
    return;
  }
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (!dbg_item(E, p, it.y, l, __LINE__)) continue;
    const ProbState& st = E.S[p];
    if (__ldcg(&st.phase) != want) continue;
    const ProblemDev& P = E.P[p];
    const bool zg = (P.L > l) || __ldcg(&st.zero_top);
    double* slot = nullptr;
    if constexpr (MODE == M_PRE12 || MODE == M_JACOBI_FIRST)
      if (l == P.L && !zg) slot = E.partial + E.fine_off[p] + it.y;
    band_tile<Pol, MODE, LD_CG>(P.lev[l], shift, zg, (long long)it.y * kTile + lane * kLaneNodes, lane,
                                in_sel, omega, slot);
  }
}

// restriction of level l's defect onto level l - 1 (tl: the coarse level's tile list)
template <class V>
__device__ __forceinline__ void mid_restrict_pass(const EngineDev& E, const MidSolo& ms, const TileList& tl,
                                                  int l, int want, int gw, int nw, int lane) {
  if (ms.on) {
    if (!ms.in_phase) return;
    const int tiles = ms.lev[l - 1].pitch / kTile;
    for (int t = gw; t < tiles; t += nw)
      restrict_tile<V, LD_CG>(ms.lev[l], ms.lev[l - 1], (long long)t * kTile, lane);
    return;
  }
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (!dbg_item(E, p, it.y, l - 1, __LINE__)) continue;
    const ProblemDev& P = E.P[p];
    if (P.L < l || __ldcg(&E.S[p].phase) != want) continue;
    restrict_tile<V, LD_CG>(P.lev[l], P.lev[l - 1], (long long)it.y * kTile, lane);
  }
}

// x_l[x_sel] += P e_{l-1} on level l
template <class V>
__device__ __forceinline__ void mid_prolong_pass(const EngineDev& E, const MidSolo& ms, const TileList& tl,
                                                 int l, int want, int x_sel, int gw, int nw, int lane) {
  if (ms.on) {
    if (!ms.in_phase) return;
    const int tiles = ms.lev[l].pitch / kTile;
    for (int t = gw; t < tiles; t += nw)
      prolong_tile<V, LD_CG>(ms.lev[l], ms.lev[l - 1], x_sel, (long long)t * kTile + lane * kLaneNodes);
    return;
  }
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (!dbg_item(E, p, it.y, l, __LINE__) || !dbg_item(E, p, 0, l - 1, __LINE__)) continue;
    if (__ldcg(&E.S[p].phase) != want) continue;
    const ProblemDev& P = E.P[p];
    prolong_tile<V, LD_CG>(P.lev[l], P.lev[l - 1], x_sel, (long long)it.y * kTile + lane * kLaneNodes);
  }
}

// The lagged convergence test of the problems whose finest level is l and whose iterate is not
// zero: problems p = first, first + stride, ... (one block: all of them, run by the last block to
// reach the barrier after the level's first smoothing step; many problems: spread over the blocks,
// followed by one more barrier).
__device__ void mid_check(const EngineDev& E, int l, int want, int first, int stride, double* sh) {
  for (int p = first; p < E.nprob; p += stride) {
    ProbState& st = E.S[p];
    if (E.P[p].L != l || __ldcg(&st.phase) != want || __ldcg(&st.zero_top)) continue;
    const double sum = problem_norm_sum(E.partial + E.fine_off[p], fine_tiles(l), sh, E.prm.prec != P64);
    if (threadIdx.x == 0) pre_check(st, E.prm, sqrt(sum));
    __syncthreads();
  }
}

// problems in phase `want` whose first smoothing step at their finest level l carries the lagged
// check, counted per level into cnt[0..kMaxLevel]; the same in every block (read before any block
// can change a state)
__device__ void mid_check_levels(const EngineDev& E, const MidSolo& ms, int want, int T, int M, int* cnt) {
  for (int l = threadIdx.x; l <= kMaxLevel; l += blockDim.x) cnt[l] = 0;
  __syncthreads();
  if (ms.on) {
    if (threadIdx.x == 0 && ms.in_phase && !ms.zero_top && ms.L > T && ms.L <= M) cnt[ms.L] = 1;
  } else {
    for (int p = threadIdx.x; p < E.nprob; p += blockDim.x) {
      const int L = E.P[p].L;
      if (L > T && L <= M && __ldcg(&E.S[p].phase) == want && !__ldcg(&E.S[p].zero_top))
        atomicAdd(&cnt[L], 1);
    }
  }
  __syncthreads();
}

// up to this many checks at one level run in the last block to arrive; more are spread
constexpr int kMidCheckSerial = 2;

// Down part of the V cycle on levels M..T+1 (mirrors vcycle_down_level step for step).
template <class Pol>
__global__ void __launch_bounds__(mid_threads<Pol>(), 1) k_mid_down(EngineDev E, const TileList* lists,
                                                                    int M, int T, int want) {
  __shared__ double sh[32];
  __shared__ int cnt[kMaxLevel + 1];
  __shared__ MidSolo ms;
  pdl_wait();
  GridBar gb;
  grid_bar_init(gb, E.gbar, E.gbar + 2);
  mid_solo_load(E, lists, M, T, want, ms);
  if (ms.on && !ms.in_phase) return;                             // (every block alike)
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int pre = E.prm.pre;
  mid_check_levels(E, ms, want, T, M, cnt);
  auto nothing = [] {};
  for (int l = M; l > T; --l) {
    const TileList& tl = lists[l];
    const int nc = cnt[l];
    // after the first smoothing step: the checks (in the last block to arrive, or spread over
    // the blocks followed by one more barrier); an engine of one problem leaves once its problem
    // has left the cycle
    auto first_done = [&]() -> bool {
      bool ok;
      if (nc == 0) {
        ok = grid_sync<false>(E, gb, nothing);
      } else if (nc <= kMidCheckSerial) {
        ok = grid_sync<true>(E, gb, [&] { mid_check(E, l, want, 0, 1, sh); });
      } else {
        ok = grid_sync<false>(E, gb, nothing);
        if (ok) {
          mid_check(E, l, want, blockIdx.x, gridDim.x, sh);
          ok = grid_sync<false>(E, gb, nothing);
        }
      }
      if (!ok) return false;
      if (nc > 0 && ms.on) {
        if (threadIdx.x == 0) ms.in_phase = __ldcg(&E.S[0].phase) == want;
        __syncthreads();
        if (!ms.in_phase) return false;
      }
      return true;
    };
    if (pre >= 2) {
      mid_band_pass<Pol, M_PRE12>(E, ms, tl, l, want, 0, gw, nw, lane);
      if (!first_done()) return;
      if (nc > 0) {
        mid_band_pass<Pol, M_PRE2B>(E, ms, tl, l, want, 0, gw, nw, lane);
        if (!grid_sync<false>(E, gb, nothing)) return;
      }
      for (int s = 3; s <= pre; ++s) {
        mid_band_pass<Pol, M_JACOBI>(E, ms, tl, l, want, (s - 1) & 1, gw, nw, lane);
        if (!grid_sync<false>(E, gb, nothing)) return;
      }
    } else {
      mid_band_pass<Pol, M_JACOBI_FIRST>(E, ms, tl, l, want, 0, gw, nw, lane);
      if (!first_done()) return;
    }
    mid_band_pass<Pol, M_DEFECT>(E, ms, tl, l, want, pre & 1, gw, nw, lane);
    if (!grid_sync<false>(E, gb, nothing)) return;
    if (l - 1 == T) pdl_trigger();            // the fused tail may start its constant-data staging
    mid_restrict_pass<typename Pol::V>(E, ms, lists[l - 1], l, want, gw, nw, lane);
    if (l - 1 > T && !grid_sync<false>(E, gb, nothing)) return;
  }
}

// Up part of the V cycle on levels T+1..M (mirrors vcycle_up_level).
template <class Pol>
__global__ void __launch_bounds__(mid_threads<Pol>(), 1) k_mid_up(EngineDev E, const TileList* lists,
                                                                  int M, int T, int want) {
  __shared__ MidSolo ms;
  pdl_wait();
  GridBar gb;
  grid_bar_init(gb, E.gbar + 1, E.gbar + 2);
  mid_solo_load(E, lists, M, T, want, ms);
  if (ms.on && !ms.in_phase) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int pre = E.prm.pre, post = E.prm.post;
  auto nothing = [] {};
  for (int l = T + 1; l <= M; ++l) {
    const TileList& tl = lists[l];
    mid_prolong_pass<typename Pol::V>(E, ms, tl, l, want, pre & 1, gw, nw, lane);
    if ((post > 0 || l < M) && !grid_sync<false>(E, gb, nothing)) return;
    for (int s = 1; s <= post; ++s) {
      mid_band_pass<Pol, M_JACOBI>(E, ms, tl, l, want, (pre + s - 1) & 1, gw, nw, lane);
      if ((s < post || l < M) && !grid_sync<false>(E, gb, nothing)) return;
    }
  }
}

// FP64 outer defect of the defect correction: d = b - A x (FP64 bands, FP64 x), written to the
// inner top-level right-hand side as V(d * s); partial[g] = sum d^2.  x = 0 gives d = b.  PCG:
// the initial residual (before the first cycle), also kept in FP64 (r64).
template <class V>
// fuse (an engine of one problem whose norm is one group of partials): the last block to finish
// sums the partials in the fixed order and takes the outer control step (in place of a control
// launch)
__global__ void __launch_bounds__(256) k_outer_defect(EngineDev E, TileList tl, int fuse) {
  pdl_start();
  if (solo_idle(E, PH_OUTER)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (!dbg_item(E, it.x, it.y, -1, __LINE__)) continue;   // a tile of the finest level
    const int p = it.x;
    const ProbState& st = E.S[p];
    if (st.phase != PH_OUTER) continue;
    const bool pcg = E.prm.solver == SOLVER_PCG;
    if (pcg && st.cycles > 0) continue;
    const ProblemDev& P = E.P[p];
    const LevelDev& top = P.lev[P.L];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    double b[4], r[4];
    ld4<LD_EF>(P.b64 + i0, b);
    if (st.x_zero) {
#pragma unroll
      for (int j = 0; j < 4; ++j) r[j] = b[j];
    } else {
      double w[3][8], dg[4];
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) load_row<double, LD_NC>(P.x64, i0 + dy * (1LL << P.L), lane, w[dy + 1]);
#pragma unroll
      for (int j = 0; j < 4; ++j) r[j] = b[j];       // r = b - A x as one chain from b
      stencil_windows<F64, LD_EF, true>(reinterpret_cast<const void* const*>(P.band64), nullptr, w, i0, r, dg);
    }
    const double s = st.s;
    V out[4];
    double q = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      out[j] = V(r[j] * s);
      q += r[j] * r[j];
    }
    st4(static_cast<V*>(top.rhs) + i0, out);
    if (pcg) st4(P.r64 + i0, r);
    q = warp_sum(q);
    if (lane == 0) E.partial[g] = q;
  }
  if (fuse && solo_last_block(E)) {               // (every block was in the outer phase)
    __shared__ double sh[32];
    const double sum = problem_norm_sum(E.partial, fine_tiles(E.P[0].L), sh);
    if (threadIdx.x == 0) {
      control_apply(E, E.S[0], CTRL_OUTER, sum);
      *E.ticket = 0u;
    }
  }
}

// ----------------------------------------------------------------- PCG vector steps (FP64)
// Conjugate gradients on each problem's finest level with the V cycle as preconditioner (a
// solver plugged into another, Sec. 4.1): every step below is one pass over the fine work list.

// q = A p (FP64 bands, p with zero halos), partial[g] = sum p q, for problems in their CG step
__global__ void __launch_bounds__(256) k_pcg_q(EngineDev E, TileList tl, int fuse) {
  pdl_start();
  if (solo_idle(E, PH_OUTER)) return;
  const bool mine = E.S[0].cycles > 0;            // (fuse: one problem, in the outer phase)
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (!dbg_item(E, it.x, it.y, -1, __LINE__)) continue;   // a tile of the finest level
    const ProbState& st = E.S[it.x];
    if (st.phase != PH_OUTER || st.cycles == 0) continue;
    const ProblemDev& P = E.P[it.x];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    double w[3][8], acc[4], dg[4];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) load_row<double, LD_NC>(P.p64, i0 + dy * (1LL << P.L), lane, w[dy + 1]);
    stencil_windows<F64, LD_NC>(reinterpret_cast<const void* const*>(P.band64), nullptr, w, i0, acc, dg);
    st4(P.q64 + i0, acc);
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) t = fma(w[1][j + 2], acc[j], t);
    t = warp_sum(t);
    if (lane == 0) E.partial[g] = t;
  }
  if (fuse) solo_fused_control(E, CTRL_PCG_ALPHA, mine, true);
}

// x += alpha p, r -= alpha q; partial[g] = sum r^2; the cycle's right-hand side V(s r)
// fuse (one problem): the last block takes the check after the step and the iteration's summary;
// every block then runs to the end whatever the phase
template <class V>
__global__ void __launch_bounds__(256) k_pcg_x(EngineDev E, TileList tl, int fuse,
                                               cudaGraphConditionalHandle h, int use_handle) {
  pdl_start();
  const bool outer = E.nprob != 1 || E.S[0].phase == PH_OUTER;
  if (!fuse && !outer) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (!dbg_item(E, it.x, it.y, -1, __LINE__)) continue;   // a tile of the finest level
    const ProbState& st = E.S[it.x];
    if (st.phase != PH_OUTER || st.cycles == 0) continue;
    const ProblemDev& P = E.P[it.x];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    double x[4], r[4], pv[4], qv[4];
    ld4c(P.x64 + i0, x);
    ld4c(P.r64 + i0, r);
    ld4<LD_NC>(P.p64 + i0, pv);
    ld4<LD_NC>(P.q64 + i0, qv);
    const double alpha = st.alpha, sc = st.s;
    V out[4];
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = fma(alpha, pv[j], x[j]);
      r[j] = fma(-alpha, qv[j], r[j]);
      t = fma(r[j], r[j], t);
      out[j] = V(r[j] * sc);
    }
    st4(P.x64 + i0, x);
    st4(P.r64 + i0, r);
    st4(static_cast<V*>(P.lev[P.L].rhs) + i0, out);
    t = warp_sum(t);
    if (lane == 0) E.partial[g] = t;
  }
  if (fuse && solo_last_block(E)) {
    __shared__ double sh[32];
    double sum = 0.0;
    if (outer) sum = problem_norm_sum(E.partial, fine_tiles(E.P[0].L), sh);
    if (threadIdx.x == 0) {
      if (outer) control_apply(E, E.S[0], CTRL_OUTER, sum);
      *E.ticket = 0u;
    }
    __syncthreads();
    summary_apply(E, h, use_handle, 1, sh);
  }
}

// partial[g] = sum r c, c = the cycle's result (top-level buffer 0, z = c / s)
template <class V>
__global__ void __launch_bounds__(256) k_pcg_dot(EngineDev E, TileList tl, int fuse) {
  pdl_start();
  if (solo_idle(E, PH_PRECOND)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (!dbg_item(E, it.x, it.y, -1, __LINE__)) continue;   // a tile of the finest level
    if (E.S[it.x].phase != PH_PRECOND) continue;
    const ProblemDev& P = E.P[it.x];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    double r[4];
    V c[4];
    ld4<LD_NC>(P.r64 + i0, r);
    ld4<LD_NC>(static_cast<const V*>(P.lev[P.L].x[0]) + i0, c);
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) t = fma(r[j], double(c[j]), t);
    t = warp_sum(t);
    if (lane == 0) E.partial[g] = t;
  }
  if (fuse) solo_fused_control(E, CTRL_PCG_BETA, true, true);
}

// p = c / s + beta p (the new search direction), for problems in PH_UPDATE
template <class V>
__global__ void __launch_bounds__(256) k_pcg_p(EngineDev E, TileList tl, int fuse) {
  pdl_start();
  if (solo_idle(E, PH_UPDATE)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (!dbg_item(E, it.x, it.y, -1, __LINE__)) continue;   // a tile of the finest level
    const ProbState& st = E.S[it.x];
    if (st.phase != PH_UPDATE) continue;
    const ProblemDev& P = E.P[it.x];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    V c[4];
    double pv[4];
    ld4<LD_NC>(static_cast<const V*>(P.lev[P.L].x[0]) + i0, c);
    ld4c(P.p64 + i0, pv);
    const double beta = st.beta, inv_s = st.inv_s;
#pragma unroll
    for (int j = 0; j < 4; ++j) pv[j] = fma(beta, pv[j], double(c[j]) * inv_s);
    st4(P.p64 + i0, pv);
  }
  if (fuse) solo_fused_control(E, CTRL_POST, true, false);
}

// x64 += c / s (c = inner top-level iterate, buffer 0), for problems in PH_UPDATE
// fuse (an engine of one problem, defect correction): the last block to finish takes the control
// step after the update and the end-of-iteration summary (in place of two launches); then every
// block runs to the end whatever the phase
__global__ void __launch_bounds__(256) k_update(EngineDev E, TileList tl, int fuse,
                                                cudaGraphConditionalHandle h, int use_handle) {
  pdl_start();
  const bool updating = E.nprob != 1 || E.S[0].phase == PH_UPDATE;
  if (!fuse && !updating) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (!dbg_item(E, it.x, it.y, -1, __LINE__)) continue;   // a tile of the finest level
    const int p = it.x;
    const ProbState& st = E.S[p];
    if (st.phase != PH_UPDATE) continue;
    const ProblemDev& P = E.P[p];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    float c[4];
    ld4<LD_NC>(static_cast<const float*>(P.lev[P.L].x[0]) + i0, c);
    double x[4];
    ld4c(P.x64 + i0, x);
    const double inv_s = st.inv_s;
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = fma(double(c[j]), inv_s, x[j]);
    st4(P.x64 + i0, x);
  }
  if (fuse && solo_last_block(E)) {
    __shared__ double sh[32];
    if (threadIdx.x == 0) {
      if (updating) control_apply(E, E.S[0], CTRL_POST, 0.0);
      *E.ticket = 0u;
    }
    __syncthreads();
    summary_apply(E, h, use_handle, 1, sh);
  }
}

// ||b||^2 partials for problems starting a solve
__global__ void __launch_bounds__(256) k_norm_b(EngineDev E, TileList tl) {
  pdl_start();
  if (solo_idle(E, PH_INIT)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    if (!dbg_item(E, it.x, it.y, -1, __LINE__)) continue;   // a tile of the finest level
    const int p = it.x;
    if (E.S[p].phase != PH_INIT) continue;
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    double b[4];
    ld4<LD_NC>(E.P[p].b64 + i0, b);
    double q = b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3];
    q = warp_sum(q);
    if (lane == 0) E.partial2[g] = q;
  }
}

// Reject right-hand sides with non-zero entries on Dirichlet nodes (one block per problem).
__global__ void __launch_bounds__(256) k_boundary_check(EngineDev E) {
  pdl_start();
  const int p = blockIdx.x;
  if (p >= E.nprob) return;
  ProbState& st = E.S[p];
  if (st.phase != PH_INIT) return;
  const ProblemDev& P = E.P[p];
  const long long n = n_of_dev(P.L);
  const int bc = P.lev[P.L].bc;
  int bad = 0;
  for (long long t = threadIdx.x; t < 4 * (n - 1); t += blockDim.x) {
    const long long side = t / (n - 1), k = t - side * (n - 1);
    long long ix, iy;
    if (side == 0) { ix = k; iy = 0; }                     // bottom row, ix = 0..n-2
    else if (side == 1) { ix = n - 1; iy = k; }            // right column
    else if (side == 2) { ix = n - 1 - k; iy = n - 1; }    // top row
    else { ix = 0; iy = n - 1 - k; }                       // left column
    if (is_dirichlet(ix, iy, n, bc) && P.b64[iy * n + ix] != 0.0) bad = 1;
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) { st.status = HN_ERR_ARG; st.phase = PH_DONE; }
}

// Per-problem control of the solver state machine: reduce the problem's norm partials in a fixed
// order (bit-reproducible, independent of the batch), then update its state.
// The norm of problem p from its tile partials, by the ctl_groups blocks of p in this launch
// (block j adds group j; the block that finishes last adds the group sums in order).  Returns
// true in the one block that holds the result (in thread 0); the others return false.
// df: double-float partials (the checks of an FP32 / FP16 cycle)
__device__ bool control_sum(const EngineDev& E, int p, int j, const double* part, int ntiles,
                            double* sh, double* sum, bool df) {
  const int ng = sum_groups(ntiles);
  if (ng == 1) {
    if (j != 0) return false;
    *sum = problem_partial_sum(part, ntiles, sh, df);
    return true;
  }
  if (j >= ng) return false;
  __shared__ int last;
  const double g = group_partial_sum(part, ntiles, j, sh, df);
  if (threadIdx.x == 0) {
    E.gsum[(long long)p * E.ctl_groups + j] = g;
    __threadfence();
    last = atomicAdd(E.gticket + p, 1u) == (unsigned)(ng - 1);
  }
  __syncthreads();
  if (!last) return false;
  if (threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (int q = 0; q < ng; ++q) t += __ldcg(E.gsum + (long long)p * E.ctl_groups + q);
    *sum = t;
    E.gticket[p] = 0u;                          // ready for the next launch
  }
  return true;
}

// The state transition of control step `kind` for problem state st, given the summed partials
// (thread 0 of one block; the control kernel, or the last block of a kernel that folds the step in)
__device__ void control_apply(const EngineDev& E, ProbState& st, int kind, double sum) {
  const int ph = st.phase;
  const Params& prm = E.prm;
  const double nrm = sqrt(sum);
  switch (kind) {
    case CTRL_INIT:
      if (st.status == HN_ERR_ARG) { st.phase = PH_DONE; break; }
      if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; break; }
      if (nrm == 0.0) { st.bnorm = 0.0; st.relres = 0.0; st.status = HN_OK; st.phase = PH_DONE; break; }
      st.bnorm = nrm;
      st.s = 1.0 / nrm;
      st.inv_s = 1.0 / st.s;
      st.relres = 1.0;
      if (prm.prec == P64 && prm.solver != SOLVER_PCG) {
        // a zero initial guess starts its first cycle unchecked (relres 1); a given guess is
        // checked by the first smoothing step of its first cycle
        st.phase = PH_CYCLE;
        st.cycles = st.x_zero ? 1 : 0;
      } else {
        st.phase = PH_OUTER;
      }
      break;
    case CTRL_CHECK0:
    case CTRL_CHECK:
      if (ph == PH_CYCLE) { st.cycles += 1; st.zero_top = 0; st.x_zero = 0; }
      st.dnorm = nrm;
      st.relres = nrm / st.bnorm;
      if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; }
      else if (st.relres <= prm.tol) { st.status = HN_OK; st.phase = PH_DONE; }
      else if (st.cycles >= prm.max_cycles) { st.status = HN_ERR_NOT_CONVERGED; st.phase = PH_DONE; }
      else st.phase = PH_CYCLE;
      break;
    case CTRL_OUTER:
      if (prm.solver == SOLVER_PCG) {
        // after the initial residual or a CG step: check, then precondition the new residual
        if (st.cycles > 0) st.outer_iters += 1;
        st.dnorm = nrm;
        st.relres = nrm / st.bnorm;
        if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; }
        else if (st.relres <= prm.tol) { st.status = HN_OK; st.phase = PH_DONE; }
        else if (st.outer_iters >= prm.max_outer || st.cycles >= prm.max_cycles) {
          st.status = HN_ERR_NOT_CONVERGED; st.phase = PH_DONE;
        } else {
          st.phase = PH_PRECOND; st.zero_top = 1; st.cycles += 1;
          if (prm.prec != P64) st.inner_cycles += 1;
        }
        break;
      }
      st.dnorm = nrm;
      st.relres = nrm / st.bnorm;
      if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; }
      else if (st.relres <= prm.tol) { st.status = HN_OK; st.phase = PH_DONE; }
      else if (st.outer_iters >= prm.max_outer || st.inner_cycles >= prm.max_cycles) {
        st.status = HN_ERR_NOT_CONVERGED; st.phase = PH_DONE;
      } else {
        // the first inner cycle starts from zero: it runs unchecked and is counted here
        st.phase = PH_INNER; st.zero_top = 1; st.inner_ref = st.s * nrm;
        st.inner_k = 1; st.inner_cycles += 1; st.cycles += 1;
      }
      break;
    case CTRL_PCG_ALPHA:
      // sum = (p, q); a breakdown (not positive: the preconditioned operator is not definite in
      // this arithmetic) stops the solve
      if (!isfinite(sum) || !(sum > 0.0)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; }
      else st.alpha = st.rho / sum;
      break;
    case CTRL_PCG_BETA: {
      // sum = (r, c) with z = c / s: rho' = (r, z); the first direction is z itself
      const double rho = sum / st.s;
      if (!isfinite(rho) || !(rho > 0.0)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; break; }
      st.beta = st.cycles > 1 ? rho / st.rho : 0.0;
      st.rho = rho;
      st.phase = PH_UPDATE;
      break;
    }
    case CTRL_POST: {
      if (prm.solver == SOLVER_PCG) {
        // the next cycle's right-hand side is scaled by 1 / ||r|| of this step
        if (st.dnorm > 0.0 && isfinite(st.dnorm)) { st.s = 1.0 / st.dnorm; st.inv_s = 1.0 / st.s; }
        st.phase = PH_OUTER;
        break;
      }
      st.outer_iters += 1;
      st.x_zero = 0;
      // scale for the next defect: the inner solve reduced the defect by about inner_res/inner_ref
      const double red = st.inner_ref > 0.0 ? st.inner_res / st.inner_ref : 1.0;
      const double pred = st.dnorm * fmax(red, 1e-7);
      if (pred > 0.0 && isfinite(pred)) { st.s = 1.0 / pred; st.inv_s = 1.0 / st.s; }
      st.phase = PH_OUTER;
      break;
    }
    default: break;
  }
}

__global__ void __launch_bounds__(256) k_control(EngineDev E, int kind, int level) {
  pdl_start();
  __shared__ double sh[32];
  const int p = blockIdx.x / E.ctl_groups, j = blockIdx.x - p * E.ctl_groups;
  if (p >= E.nprob) return;
  ProbState& st = E.S[p];
  const int ph = st.phase;
  if (kind == CTRL_PRE) {
    bool owner = j == 0;                        // the block that sets the cycle's IF value
    if ((ph == PH_INNER || ph == PH_CYCLE) && E.P[p].L == level && !st.zero_top) {
      double sum = 0.0;
      owner = control_sum(E, p, j, E.partial + E.fine_off[p], fine_tiles(level), sh, &sum, E.prm.prec != P64);
      if (owner && threadIdx.x == 0) pre_check(st, E.prm, sqrt(sum));
    }
    // the rest of the V cycle runs if any problem is still in it
    if (owner && threadIdx.x == 0 && (st.phase == PH_INNER || st.phase == PH_CYCLE))
      cond_set(E.prm.cond, 0, 1u);
    return;
  }
  const bool mine = (kind == CTRL_INIT && ph == PH_INIT) ||
                    (kind == CTRL_CHECK0 && ph == PH_CHECK) ||
                    (kind == CTRL_CHECK && ph == PH_CYCLE) ||
                    (kind == CTRL_OUTER && ph == PH_OUTER) ||
                    (kind == CTRL_POST && ph == PH_UPDATE) ||
                    (kind == CTRL_PCG_ALPHA && ph == PH_OUTER && st.cycles > 0) ||
                    (kind == CTRL_PCG_BETA && ph == PH_PRECOND);
  if (!mine) return;
  double sum = 0.0;
  if (kind != CTRL_POST) {
    const double* part = kind == CTRL_INIT ? E.partial2 : E.partial;
    // the checks of the cycle's own precision: double-float partials in FP32 / FP16 cycles
    const bool df = (kind == CTRL_CHECK || kind == CTRL_CHECK0) && E.prm.prec != P64;
    if (!control_sum(E, p, j, part + E.fine_off[p], fine_tiles(E.P[p].L), sh, &sum, df)) return;
  } else if (j != 0) {
    return;
  }
  if (threadIdx.x != 0) return;
  control_apply(E, st, kind, sum);
}

// Count problems still running; publish to the host word and, inside a device-side loop, to the
// graph's while-condition.  Past the iteration limit every running problem is stopped as not
// converged, so a device-side loop always ends.
__device__ void summary_apply(const EngineDev& E, cudaGraphConditionalHandle h, int use_handle,
                              int end_of_iteration, double* sh) {
  __shared__ unsigned over;
  if (threadIdx.x == 0) {
    const unsigned it = E.iter ? (*E.iter += 1) : 0u;
    over = (E.iter && it > E.iter_limit) ? 1u : 0u;
  }
  __syncthreads();
  double c = 0.0, o = 0.0;
  for (int p = threadIdx.x; p < E.nprob; p += blockDim.x) {
    ProbState& st = E.S[p];
    if (st.phase != PH_DONE && over) { st.status = HN_ERR_NOT_CONVERGED; st.phase = PH_DONE; }
    // after an iteration the finest-level iterate of a running cycle is no longer zero
    if (end_of_iteration && (st.phase == PH_INNER || st.phase == PH_CYCLE)) st.zero_top = 0;
    c += st.phase != PH_DONE ? 1.0 : 0.0;
    o += st.phase == PH_OUTER ? 1.0 : 0.0;
  }
  c = block_sum256(c, sh);
  o = block_sum256(o, sh);
  if (threadIdx.x == 0) {
    const unsigned active = (unsigned)c;
    if (E.active_host) *E.active_host = active;
    if (use_handle) cudaGraphSetConditional(h, active > 0 ? 1u : 0u);
    const CondDev& cd = E.prm.cond;
    if (cd.mask) {
      *cd.launches += cd.n_base + (cd.taken[0] ? cd.n_cycle : 0u) + (cd.taken[1] ? cd.n_outer : 0u) +
                      (cd.taken[2] ? cd.n_update : 0u);
      cond_set(cd, 0, 0u);
      cond_set(cd, 2, 0u);
      cond_set(cd, 1, o > 0.0 ? 1u : 0u);
    }
  }
}

__global__ void __launch_bounds__(256) k_summary(EngineDev E, cudaGraphConditionalHandle h,
                                                 int use_handle, int end_of_iteration) {
  pdl_start();
  __shared__ double sh[32];
  summary_apply(E, h, use_handle, end_of_iteration, sh);
}

inline int grid_or_one(int g) { return g < 1 ? 1 : g; }

// resident blocks per SM of a kernel at a block size (cached per kernel)
int resident_blocks(const void* f, int threads, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(f);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, threads, smem) != cudaSuccess || b < 1) b = 1;
  cache[f] = b;
  return b;
}

// launch with optional programmatic dependent launch and thread-block clusters.  Grid-stride
// kernels (cluster == 0) get at most one wave of resident blocks.
template <typename... KArgs, typename... Args>
cudaError_t launch_kt(void (*kern)(KArgs...), int grid, int threads, size_t smem, cudaStream_t s,
                      int pdl, int cluster, Args... args) {
  if (cluster == 0) grid = std::min(grid, resident_blocks(reinterpret_cast<const void*>(kern), threads, smem) * sm_count());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid_or_one(grid), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  // pdl: 1 = every launch; 2 = launches of fewer blocks than SMs (their waiting blocks do not
  // take occupancy from a bandwidth-bound predecessor); 3 = fewer blocks than twice the SMs
  if (pdl == 1 || (pdl == 2 && grid_or_one(grid) < sm_count()) ||
      (pdl == 3 && grid_or_one(grid) < 2 * sm_count())) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cluster > 0) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = (unsigned)cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// cooperative launch of one wave of resident blocks (all blocks run at once: grid barriers)
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kern)(KArgs...), int threads, cudaStream_t s, Args... args) {
  const int grid = resident_blocks(reinterpret_cast<const void*>(kern), threads, 0) * sm_count();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), int grid, size_t smem, cudaStream_t s, int pdl,
                     int cluster, Args... args) {
  return launch_kt(kern, grid, 256, smem, s, pdl, cluster, args...);
}

// shared memory of the staged band kernels: two stages of 9 band slices of 8 tiles
template <class Pol>
constexpr size_t staged_smem() { return 2 * 9 * (size_t)kChunkTiles * kTile * sizeof(typename Pol::B); }

template <class Pol>
cudaError_t launch_band_t(int mode, const EngineDev& E, TileList tl, int level, int want,
                          int in_sel, int grid, cudaStream_t s) {
  grid = grid_or_one(grid);
  // large levels of the FP32 / FP16 hierarchies may stream their bands through shared memory
  if (E.staged && Pol::prec != P64 && level >= 0 && tl.chunks && tl.chunk_cap >= sm_count() &&
      (mode == M_SPMV || mode == M_DEFECT || mode == M_JACOBI || mode == M_JACOBI_FIRST ||
       mode == M_PRE12 || mode == M_PRE2B)) {
    const size_t sm = staged_smem<Pol>();
    const int g = tl.chunk_cap;
    switch (mode) {
      case M_SPMV: return launch_k(k_band_staged<Pol, M_SPMV>, g, sm, s, E.pdl, 0, E, tl, level, want, in_sel);
      case M_DEFECT: return launch_k(k_band_staged<Pol, M_DEFECT>, g, sm, s, E.pdl, 0, E, tl, level, want, in_sel);
      case M_JACOBI: return launch_k(k_band_staged<Pol, M_JACOBI>, g, sm, s, E.pdl, 0, E, tl, level, want, in_sel);
      case M_JACOBI_FIRST: return launch_k(k_band_staged<Pol, M_JACOBI_FIRST>, g, sm, s, E.pdl, 0, E, tl, level, want, in_sel);
      case M_PRE12: return launch_k(k_band_staged<Pol, M_PRE12>, g, sm, s, E.pdl, 0, E, tl, level, want, in_sel);
      default: return launch_k(k_band_staged<Pol, M_PRE2B>, g, sm, s, E.pdl, 0, E, tl, level, want, in_sel);
    }
  }
  switch (mode) {
    case M_SPMV: return launch_k(k_band<Pol, M_SPMV>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    case M_DEFECT: return launch_k(k_band<Pol, M_DEFECT>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    case M_JACOBI: return launch_k(k_band<Pol, M_JACOBI>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    case M_JACOBI_FIRST:
      return launch_k(k_band<Pol, M_JACOBI_FIRST>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    case M_CHECK: return launch_k(k_band<Pol, M_CHECK>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    case M_PRE12: return launch_k(k_band<Pol, M_PRE12>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    case M_PRE2B: return launch_k(k_band<Pol, M_PRE2B>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    case M_PJ: return launch_k(k_band<Pol, M_PJ>, grid, 0, s, E.pdl, 0, E, tl, level, want, in_sel);
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_band(int mode, const EngineDev& E, TileList tl, int level, int want, int in_sel,
                        int grid, cudaStream_t s) {
  switch (E.prm.prec) {
    case P64: return launch_band_t<F64>(mode, E, tl, level, want, in_sel, grid, s);
    case P32: return launch_band_t<F32>(mode, E, tl, level, want, in_sel, grid, s);
    case P16: return launch_band_t<F16>(mode, E, tl, level, want, in_sel, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_jacobi(const EngineDev& E, TileList tl, int level, int want, int in_sel,
                          int first, int grid, cudaStream_t s, int fuse_check) {
  return launch_band(first ? M_JACOBI_FIRST : M_JACOBI, E, tl, level, want,
                     in_sel | (first && fuse_check ? 2 : 0), grid, s);
}
cudaError_t launch_pre12(const EngineDev& E, TileList tl, int level, int want, int grid,
                         cudaStream_t s, int fuse_check) {
  return launch_band(M_PRE12, E, tl, level, want, fuse_check ? 2 : 0, grid, s);
}
cudaError_t launch_pre2b(const EngineDev& E, TileList tl, int level, int want, int grid,
                         cudaStream_t s) {
  return launch_band(M_PRE2B, E, tl, level, want, 0, grid, s);
}
cudaError_t launch_prolong_jacobi(const EngineDev& E, TileList tl, int level, int want, int x_sel,
                                  int grid, cudaStream_t s) {
  return launch_band(M_PJ, E, tl, level, want, x_sel, grid, s);
}
bool pre_fuses(int) { return true; }

// shared memory the fused coarse-level kernel may use for levels coarse..S
constexpr long long kTailSmemBudget = 160 * 1024;   // block 0's shared-memory levels
constexpr long long kTailSmemMax = 212 * 1024;      // with the cluster levels (dynamic part)

// shared memory reserved for a staged coarse inverse: the unknowns of the coarsest level number at
// most n^2 (free Neumann sides), and an inverse is staged only if it takes <= kCinvSmemMax bytes
long long tail_cinv_bytes(int coarse, int cg) {
  const long long m = ((1LL << coarse) + 1) * ((1LL << coarse) + 1);   // nodes >= unknowns
  if (cg) return (std::min(9 * m * 8, kCinvSmemMax) + 15) / 16 * 16 + (2 * m * 8 + 15) / 16 * 16;
  return (std::min(m * m * 8, kCinvSmemMax) + 15) / 16 * 16;
}

int tail_smem_level(int prec, int coarse, int cg, int T) {
  long long bytes = tail_cinv_bytes(coarse, cg);
  int S = coarse;
  for (int l = coarse; l <= T; ++l) {
    bytes += smem_level_bytes(l, prec);
    if (bytes > kTailSmemBudget) break;
    S = l;
  }
  return S;
}

long long tail_smem_bytes(int prec, int coarse, int cg, int S) {
  long long bytes = 0;
  for (int l = coarse; l <= S; ++l) bytes += smem_level_bytes(l, prec);
  return bytes + tail_cinv_bytes(coarse, cg);
}

// shared memory of the cluster levels (S, T] in distributed shared memory, or -1 if they do not
// fit (or the partition would leave a block without rows; C must be a power of two)
long long tail_dsm_bytes(int prec, int coarse, int cg, int S, int T, int C) {
  if (T <= S || (1 << (S + 1)) < C || (C & (C - 1)) != 0) return -1;
  long long bytes = tail_smem_bytes(prec, coarse, cg, S);
  for (int l = S + 1; l <= T; ++l) bytes += dsm_level_bytes(l, C, S, prec);
  return bytes <= kTailSmemMax ? bytes : -1;
}

// clusters of up to 16 blocks need the non-portable opt-in, the shared-memory levels a larger
// dynamic shared-memory size; set once, outside any stream capture
cudaError_t prepare_kernels() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
  };
  set(reinterpret_cast<const void*>(k_tail<F64>));
  set(reinterpret_cast<const void*>(k_tail<F32>));
  set(reinterpret_cast<const void*>(k_tail<F16>));
  auto staged = [&](const void* f, size_t bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  staged((const void*)k_band_staged<F32, M_SPMV>, staged_smem<F32>());
  staged((const void*)k_band_staged<F32, M_DEFECT>, staged_smem<F32>());
  staged((const void*)k_band_staged<F32, M_JACOBI>, staged_smem<F32>());
  staged((const void*)k_band_staged<F32, M_JACOBI_FIRST>, staged_smem<F32>());
  staged((const void*)k_band_staged<F32, M_PRE12>, staged_smem<F32>());
  staged((const void*)k_band_staged<F32, M_PRE2B>, staged_smem<F32>());
  staged((const void*)k_band_staged<F16, M_SPMV>, staged_smem<F16>());
  staged((const void*)k_band_staged<F16, M_DEFECT>, staged_smem<F16>());
  staged((const void*)k_band_staged<F16, M_JACOBI>, staged_smem<F16>());
  staged((const void*)k_band_staged<F16, M_JACOBI_FIRST>, staged_smem<F16>());
  staged((const void*)k_band_staged<F16, M_PRE12>, staged_smem<F16>());
  staged((const void*)k_band_staged<F16, M_PRE2B>, staged_smem<F16>());
  // the fused sweeps: their largest tiles
  SweepGeom g;
  g.cx = kSweepCX; g.cy = kSweepCY; g.P = 2 * g.cx + 7; g.R = 2 * g.cy + 7; g.tx = g.ty = 1;
  staged((const void*)k_sweep_down<F64>, sweep_smem_bytes(P64, g));
  staged((const void*)k_sweep_down<F32>, sweep_smem_bytes(P32, g));
  staged((const void*)k_sweep_down<F16>, sweep_smem_bytes(P16, g));
  staged((const void*)k_sweep_up<F64>, sweep_smem_bytes(P64, g));
  staged((const void*)k_sweep_up<F32>, sweep_smem_bytes(P32, g));
  staged((const void*)k_sweep_up<F16>, sweep_smem_bytes(P16, g));
  return e;
}

template <class Pol>
cudaError_t launch_tail_t(const EngineDev& E, int T, int want, int cluster, cudaStream_t s) {
  const int cg = E.prm.coarse_cg;
  const int S = tail_smem_level(Pol::prec, E.prm.coarse, cg, T);
  const long long dsm = E.dsm ? tail_dsm_bytes(Pol::prec, E.prm.coarse, cg, S, T, cluster) : -1;
  const size_t smem = (size_t)(dsm > 0 ? dsm : tail_smem_bytes(Pol::prec, E.prm.coarse, cg, S));
  return launch_kt(k_tail<Pol>, E.nprob * cluster, kTailThreads, smem, s, E.pdl, cluster, E, T, S, want,
                   dsm > 0 ? 1 : 0);
}

cudaError_t launch_tail(const EngineDev& E, int T, int want, int cluster, cudaStream_t s) {
  switch (E.prm.prec) {
    case P64: return launch_tail_t<F64>(E, T, want, cluster, s);
    case P32: return launch_tail_t<F32>(E, T, want, cluster, s);
    case P16: return launch_tail_t<F16>(E, T, want, cluster, s);
  }
  return cudaErrorInvalidValue;
}
template <class Pol>
cudaError_t launch_mid_t(const EngineDev& E, const TileList* lists, int M, int T, int want, int up,
                         cudaStream_t s) {
  if (up) return launch_coop(k_mid_up<Pol>, mid_threads<Pol>(), s, E, lists, M, T, want);
  return launch_coop(k_mid_down<Pol>, mid_threads<Pol>(), s, E, lists, M, T, want);
}

cudaError_t launch_mid(const EngineDev& E, const TileList* lists, int M, int T, int want, int up,
                       cudaStream_t s) {
  switch (E.prm.prec) {
    case P64: return launch_mid_t<F64>(E, lists, M, T, want, up, s);
    case P32: return launch_mid_t<F32>(E, lists, M, T, want, up, s);
    case P16: return launch_mid_t<F16>(E, lists, M, T, want, up, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_defect(const EngineDev& E, TileList tl, int level, int want, int in_sel,
                          int grid, cudaStream_t s) {
  return launch_band(M_DEFECT, E, tl, level, want, in_sel, grid, s);
}
cudaError_t launch_spmv(const EngineDev& E, TileList tl, int level, int want, int in_sel, int grid,
                        cudaStream_t s) {
  return launch_band(M_SPMV, E, tl, level, want, in_sel, grid, s);
}

cudaError_t launch_restrict(const EngineDev& E, TileList tl_coarse, int fine_level, int want,
                            int grid, cudaStream_t s) {
  grid = grid_or_one(grid);
  if (E.prm.prec == P64) return launch_k(k_restrict<double>, grid, 0, s, E.pdl, 0, E, tl_coarse, fine_level, want);
  return launch_k(k_restrict<float>, grid, 0, s, E.pdl, 0, E, tl_coarse, fine_level, want);
}

cudaError_t launch_prolong(const EngineDev& E, TileList tl, int level, int want, int x_sel,
                           int grid, cudaStream_t s) {
  grid = grid_or_one(grid);
  if (E.prm.prec == P64) return launch_k(k_prolong<double>, grid, 0, s, E.pdl, 0, E, tl, level, want, x_sel);
  return launch_k(k_prolong<float>, grid, 0, s, E.pdl, 0, E, tl, level, want, x_sel);
}

SweepGeom sweep_geom(int level) {
  const int h = 1 << (level - 1);                 // coarse intervals per side
  SweepGeom g;
  // 16 x 16 coarse nodes from 256 coarse intervals per side up (L = 9: 256 tiles, one wave of two
  // blocks per SM), 16 x 8 below (L = 8: 128 tiles)
  g.cx = std::min(kSweepCX, h);
  g.cy = std::min(h >= 256 ? kSweepCY : kSweepCY / 2, h);
  g.tx = h / g.cx;
  g.ty = h / g.cy;
  g.P = 2 * g.cx + 7;
  g.R = 2 * g.cy + 7;
  return g;
}

size_t sweep_smem_bytes(int prec, const SweepGeom& g) {
  const size_t cnt = (size_t)g.P * g.R;
  const size_t bb = prec == P64 ? 8 : (prec == P32 ? 4 : 2), vb = prec == P64 ? 8 : 4;
  auto al = [](size_t b) { return (b + 15) / 16 * 16; };
  // bands, omega / D, x0, x1, rhs, r; the coarse iterate around the tile
  return 9 * al(cnt * bb) + al(cnt * vb) + 4 * al(cnt * vb) + al((size_t)(g.cx + 4) * (g.cy + 4) * vb);
}

template <class Pol>
cudaError_t launch_sweep_t(const EngineDev& E, TileList tl, int level, int want, int arg, int up,
                           cudaStream_t s) {
  const SweepGeom g = sweep_geom(level);
  const size_t smem = sweep_smem_bytes(Pol::prec, g);
  if (up) return launch_kt(k_sweep_up<Pol>, g.tx * g.ty, kSweepThreads, smem, s, E.pdl, 0, E, tl, level, want, arg, g);
  return launch_kt(k_sweep_down<Pol>, g.tx * g.ty, kSweepThreads, smem, s, E.pdl, 0, E, tl, level, want, arg, g);
}

cudaError_t launch_sweep_down(const EngineDev& E, TileList tl, int level, int want, int top, cudaStream_t s) {
  switch (E.prm.prec) {
    case P64: return launch_sweep_t<F64>(E, tl, level, want, top, 0, s);
    case P32: return launch_sweep_t<F32>(E, tl, level, want, top, 0, s);
    case P16: return launch_sweep_t<F16>(E, tl, level, want, top, 0, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_up(const EngineDev& E, TileList tl, int level, int want, int e_sel, cudaStream_t s) {
  switch (E.prm.prec) {
    case P64: return launch_sweep_t<F64>(E, tl, level, want, e_sel, 1, s);
    case P32: return launch_sweep_t<F32>(E, tl, level, want, e_sel, 1, s);
    case P16: return launch_sweep_t<F16>(E, tl, level, want, e_sel, 1, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_coarse(const EngineDev& E, TileList tl, int want, int grid, cudaStream_t s) {
  if (E.prm.coarse_cg) {
    if (E.prm.prec == P64) return launch_k(k_coarse_cg<double>, E.nprob, 0, s, E.pdl, 0, E, want);
    return launch_k(k_coarse_cg<float>, E.nprob, 0, s, E.pdl, 0, E, want);
  }
  grid = grid_or_one(grid);
  if (E.prm.prec == P64) return launch_k(k_coarse<double>, grid, 0, s, E.pdl, 0, E, tl, want);
  return launch_k(k_coarse<float>, grid, 0, s, E.pdl, 0, E, tl, want);
}

cudaError_t launch_outer_defect(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse) {
  if (E.prm.prec == P64) return launch_k(k_outer_defect<double>, grid, 0, s, E.pdl, 0, E, fine, fuse);
  return launch_k(k_outer_defect<float>, grid, 0, s, E.pdl, 0, E, fine, fuse);
}

cudaError_t launch_pcg_q(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse) {
  return launch_k(k_pcg_q, grid, 0, s, E.pdl, 0, E, fine, fuse);
}
cudaError_t launch_pcg_x(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse,
                         cudaGraphConditionalHandle h, int use_handle) {
  if (E.prm.prec == P64) return launch_k(k_pcg_x<double>, grid, 0, s, E.pdl, 0, E, fine, fuse, h, use_handle);
  return launch_k(k_pcg_x<float>, grid, 0, s, E.pdl, 0, E, fine, fuse, h, use_handle);
}
cudaError_t launch_pcg_dot(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse) {
  if (E.prm.prec == P64) return launch_k(k_pcg_dot<double>, grid, 0, s, E.pdl, 0, E, fine, fuse);
  return launch_k(k_pcg_dot<float>, grid, 0, s, E.pdl, 0, E, fine, fuse);
}
cudaError_t launch_pcg_p(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse) {
  if (E.prm.prec == P64) return launch_k(k_pcg_p<double>, grid, 0, s, E.pdl, 0, E, fine, fuse);
  return launch_k(k_pcg_p<float>, grid, 0, s, E.pdl, 0, E, fine, fuse);
}

cudaError_t launch_update(const EngineDev& E, TileList fine, int grid, cudaStream_t s, int fuse,
                          cudaGraphConditionalHandle h, int use_handle) {
  return launch_k(k_update, grid, 0, s, E.pdl, 0, E, fine, fuse, h, use_handle);
}

cudaError_t launch_norm_b(const EngineDev& E, TileList fine, int grid, cudaStream_t s) {
  return launch_k(k_norm_b, grid, 0, s, E.pdl, 0, E, fine);
}

cudaError_t launch_control(const EngineDev& E, int kind, cudaStream_t s, int level) {
  return launch_k(k_control, E.nprob * E.ctl_groups, 0, s, E.pdl, 0, E, kind, level);
}

cudaError_t launch_summary(const EngineDev& E, cudaGraphConditionalHandle h, int use_handle,
                           int end_of_iteration, cudaStream_t s) {
  return launch_k(k_summary, 1, 0, s, E.pdl, 0, E, h, use_handle, end_of_iteration);
}

cudaError_t launch_boundary_check(const EngineDev& E, cudaStream_t s) {
  return launch_k(k_boundary_check, E.nprob, 0, s, 0, 0, E);
}

// the fine-level defect norm of the V-cycle's own precision (convergence check)
cudaError_t launch_check(const EngineDev& E, TileList fine_by_problem_top, int want, int x_sel,
                         int grid, cudaStream_t s) {
  // the fine work list enumerates every problem's top level; the level is taken per problem
  return launch_band(M_CHECK, E, fine_by_problem_top, -1, want, x_sel, grid, s);
}

}  // namespace hn
