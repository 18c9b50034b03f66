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
#include "hn_internal.h"

namespace hn {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// -------------------------------------------------------------------- precision policies
struct F64 { using B = double; using V = double; using A = double; static constexpr int prec = P64; };
struct F32 { using B = float; using V = float; using A = float; static constexpr int prec = P32; };
struct F16 { using B = __half; using V = float; using A = float; static constexpr int prec = P16; };

__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
// plain (coherent) loads for data the same kernel also writes
__device__ __forceinline__ void ld4c(const double* p, double (&o)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void ld4c(const float* p, float (&o)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
}

// 4 consecutive band values of band k at node i0, in the arithmetic type
template <class Pol>
__device__ __forceinline__ void load_band(const void* band, float scale, long long i0,
                                          typename Pol::A (&o)[4]) {
  if constexpr (Pol::prec == P16) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(static_cast<const __half*>(band) + i0));
    const __half2 h0 = *reinterpret_cast<const __half2*>(&u.x);
    const __half2 h1 = *reinterpret_cast<const __half2*>(&u.y);
    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    o[0] = scale * f0.x; o[1] = scale * f0.y; o[2] = scale * f1.x; o[3] = scale * f1.y;
  } else {
    ld4(static_cast<const typename Pol::B*>(band) + i0, o);
  }
}

// Row window of x around the lane's 4 nodes: w[o + 2] = x[a + o], o = -2..5, a aligned to 4.
template <class V>
__device__ __forceinline__ void load_row(const V* __restrict__ x, long long a, int lane, V (&w)[8]) {
  V c[4];
  ld4(x + a, c);
  V l2 = __shfl_up_sync(kFull, c[2], 1), l1 = __shfl_up_sync(kFull, c[3], 1);
  V r0 = __shfl_down_sync(kFull, c[0], 1), r1 = __shfl_down_sync(kFull, c[1], 1);
  if (lane == 0) { l2 = __ldg(x + a - 2); l1 = __ldg(x + a - 1); }
  if (lane == 31) { r0 = __ldg(x + a + 4); r1 = __ldg(x + a + 5); }
  w[0] = l2; w[1] = l1; w[2] = c[0]; w[3] = c[1]; w[4] = c[2]; w[5] = c[3]; w[6] = r0; w[7] = r1;
}

// acc[j] = sum_k band_k[i0+j] * x[i0+j+off_k] in band order k = 0..8; also returns x[i0+j] and
// the diagonal.  shift = 2^L = n - 1, so off_k = dy*n + dx = dy*shift + (dy + dx).
template <class Pol>
__device__ __forceinline__ void stencil4(const void* const* band, const float* scale,
                                         const typename Pol::V* __restrict__ x, long long i0,
                                         long long shift, int lane, typename Pol::A (&acc)[4],
                                         typename Pol::V (&xc)[4], typename Pol::A (&dg)[4]) {
  using A = typename Pol::A;
  using V = typename Pol::V;
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = A(0);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    V w[8];
    load_row<V>(x, i0 + dy * shift, lane, w);
    if (dy == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) xc[j] = w[j + 2];
    }
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int k = (dy + 1) * 3 + (dx + 1);
      A b[4];
      load_band<Pol>(band[k], scale ? scale[k] : 1.0f, i0, b);
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fma(b[j], A(w[j + dy + dx + 2]), acc[j]);
      if (k == 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) dg[j] = b[j];
      }
    }
  }
}

// FP16-band operator in row-sum form (array 4 holds the row sum rho):
// acc[j] = rho x_i + sum_{k != 4} a_k (x_{i+off_k} - x_i) in band order; dg[j] = rho - sum a_k.
__device__ __forceinline__ void stencil4_rowsum(const void* const* band, const float* scale,
                                                const float* __restrict__ x, long long i0,
                                                long long shift, int lane, float (&acc)[4],
                                                float (&xc)[4], float (&dg)[4]) {
  float w[3][8];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) load_row<float>(x, i0 + dy * shift, lane, w[dy + 1]);
#pragma unroll
  for (int j = 0; j < 4; ++j) xc[j] = w[1][j + 2];
  float rho[4];
  load_band<F16>(band[4], scale[4], i0, rho);
#pragma unroll
  for (int j = 0; j < 4; ++j) { acc[j] = rho[j] * xc[j]; dg[j] = rho[j]; }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (k == 4) continue;
    const int dy = k / 3 - 1, dx = k % 3 - 1;
    float b[4];
    load_band<F16>(band[k], scale[k], i0, b);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[j] = fmaf(b[j], w[dy + 1][j + dy + dx + 2] - xc[j], acc[j]);
      dg[j] -= b[j];
    }
  }
}

// diagonal of the row-sum form without x (for the zero-guess Jacobi step)
__device__ __forceinline__ void diag_rowsum(const void* const* band, const float* scale,
                                            long long i0, float (&dg)[4]) {
  load_band<F16>(band[4], scale[4], i0, dg);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (k == 4) continue;
    float b[4];
    load_band<F16>(band[k], scale[k], i0, b);
#pragma unroll
    for (int j = 0; j < 4; ++j) dg[j] -= b[j];
  }
}

template <class Pol>
__device__ __forceinline__ void apply_op4(const void* const* band, const float* scale,
                                          const typename Pol::V* __restrict__ x, long long i0,
                                          long long shift, int lane, typename Pol::A (&acc)[4],
                                          typename Pol::V (&xc)[4], typename Pol::A (&dg)[4]) {
  if constexpr (Pol::prec == P16) stencil4_rowsum(band, scale, x, i0, shift, lane, acc, xc, dg);
  else stencil4<Pol>(band, scale, x, i0, shift, lane, acc, xc, dg);
}

// deterministic warp sum (butterfly; every lane ends with the same value)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
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

enum BandMode { M_SPMV = 0, M_DEFECT = 1, M_JACOBI = 2, M_JACOBI_FIRST = 3, M_CHECK = 4 };

// One warp-tile per loop trip.  in_sel selects the iterate buffer read; Jacobi writes the other.
template <class Pol, int MODE>
__global__ void __launch_bounds__(256) k_band(EngineDev E, TileList tl, int level, int want,
                                              int in_sel) {
  using A = typename Pol::A;
  using V = typename Pol::V;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  const A omega = A(E.prm.omega);
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (E.S[p].phase != want) continue;
    const ProblemDev& P = E.P[p];
    const int lv = level < 0 ? P.L : level;
    const LevelDev& d = P.lev[lv];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    const long long shift = 1LL << lv;
    const V* rhs = static_cast<const V*>(d.rhs);
    const float* scale = Pol::prec == P16 ? d.scale : nullptr;

    if constexpr (MODE == M_JACOBI_FIRST) {
      const bool zg = (P.L > lv) || E.S[p].zero_top;
      if (zg) {                                   // x = 0: x' = omega D^-1 rhs
        V b[4], out[4];
        ld4(rhs + i0, b);
        if constexpr (Pol::prec == P64) {
          double wd[4];
          ld4(d.wdinv + i0, wd);
#pragma unroll
          for (int j = 0; j < 4; ++j) out[j] = wd[j] * b[j];
        } else {
          A dgv[4];
          if constexpr (Pol::prec == P16) diag_rowsum(d.band, scale, i0, dgv);
          else load_band<Pol>(d.band[4], 1.0f, i0, dgv);
#pragma unroll
          for (int j = 0; j < 4; ++j) out[j] = (omega / dgv[j]) * A(b[j]);
        }
        st4(static_cast<V*>(d.x[1]) + i0, out);
        continue;
      }
    }
    const V* xin = static_cast<const V*>(d.x[MODE == M_JACOBI_FIRST ? 0 : in_sel]);
    A acc[4], dg[4];
    V xc[4];
    apply_op4<Pol>(d.band, scale, xin, i0, shift, lane, acc, xc, dg);
    if constexpr (MODE == M_SPMV) {
      V out[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) out[j] = V(acc[j]);
      st4(static_cast<V*>(d.r) + i0, out);
    } else {
      V b[4];
      ld4(rhs + i0, b);
      if constexpr (MODE == M_DEFECT) {
        V out[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) out[j] = V(A(b[j]) - acc[j]);
        st4(static_cast<V*>(d.r) + i0, out);
      } else if constexpr (MODE == M_CHECK) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double r = double(A(b[j]) - acc[j]);
          s += r * r;
        }
        s = warp_sum(s);
        if (lane == 0) E.partial[g] = s;
      } else {                                    // Jacobi
        V out[4];
        if constexpr (Pol::prec == P64) {
          double wd[4];
          ld4(d.wdinv + i0, wd);
#pragma unroll
          for (int j = 0; j < 4; ++j) out[j] = fma(wd[j], b[j] - acc[j], xc[j]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) out[j] = fma(omega / dg[j], A(b[j]) - acc[j], A(xc[j]));
        }
        const int out_sel = MODE == M_JACOBI_FIRST ? 1 : 1 - in_sel;
        st4(static_cast<V*>(d.x[out_sel]) + i0, out);
      }
    }
  }
}

// Full-weighting restriction r_c = P^T r_f onto the coarse level (work list of the coarse level).
// Coarse boundary and padding nodes are set to 0.  Summation order: fine rows 2J-1, 2J, 2J+1,
// columns 2I-1, 2I, 2I+1, weights 1/4, 1/2, 1/4 x 1/4, 1/2, 1/4 (products by powers of two exact).
template <class V>
__global__ void __launch_bounds__(256) k_restrict(EngineDev E, TileList tl, int fine_level,
                                                  int want) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    const ProblemDev& P = E.P[p];
    if (P.L < fine_level || E.S[p].phase != want) continue;
    const LevelDev& f = P.lev[fine_level];
    const LevelDev& c = P.lev[fine_level - 1];
    const long long nc = c.n, nf = f.n, Nc = nc * nc;
    const V* r = static_cast<const V*>(f.r);
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    V out[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long ci = i0 + j;
      V v = V(0);
      if (ci < Nc) {
        const long long J = ci / nc, I = ci - J * nc;
        if (I > 0 && J > 0 && I < nc - 1 && J < nc - 1) {
          const long long fc = 2 * J * nf + 2 * I;
          const V q = V(0.25), h = V(0.5);
          v = q * __ldg(r + fc - nf - 1);
          v = fma(h, __ldg(r + fc - nf), v);
          v = fma(q, __ldg(r + fc - nf + 1), v);
          v = fma(h, __ldg(r + fc - 1), v);
          v = v + __ldg(r + fc);
          v = fma(h, __ldg(r + fc + 1), v);
          v = fma(q, __ldg(r + fc + nf - 1), v);
          v = fma(h, __ldg(r + fc + nf), v);
          v = fma(q, __ldg(r + fc + nf + 1), v);
        }
      }
      out[j] = v;
    }
    st4(static_cast<V*>(c.rhs) + i0, out);
  }
}

// x_f[x_sel] += P e_c (bilinear interpolation of the coarse iterate, buffer 0 of level-1);
// boundary fine nodes are left unchanged.
template <class V>
__global__ void __launch_bounds__(256) k_prolong(EngineDev E, TileList tl, int level, int want,
                                                 int x_sel) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (E.S[p].phase != want) continue;
    const ProblemDev& P = E.P[p];
    const LevelDev& f = P.lev[level];
    const LevelDev& c = P.lev[level - 1];
    const long long nf = f.n, nc = c.n, Nf = nf * nf;
    const V* e = static_cast<const V*>(c.x[0]);
    V* x = static_cast<V*>(f.x[x_sel]);
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    V v[4];
    ld4c(x + i0, v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long fi = i0 + j;
      if (fi >= Nf) continue;
      const long long iy = fi / nf, ix = fi - iy * nf;
      if (ix == 0 || iy == 0 || ix == nf - 1 || iy == nf - 1) continue;
      const long long cx0 = ix >> 1, cx1 = (ix + 1) >> 1, cy0 = iy >> 1, cy1 = (iy + 1) >> 1;
      V add;
      const bool ox = ix & 1, oy = iy & 1;
      if (!ox && !oy) {
        add = __ldg(e + cy0 * nc + cx0);
      } else if (ox && !oy) {
        add = V(0.5) * (__ldg(e + cy0 * nc + cx0) + __ldg(e + cy0 * nc + cx1));
      } else if (!ox && oy) {
        add = V(0.5) * (__ldg(e + cy0 * nc + cx0) + __ldg(e + cy1 * nc + cx0));
      } else {
        add = V(0.25) * (((__ldg(e + cy0 * nc + cx0) + __ldg(e + cy0 * nc + cx1)) +
                          __ldg(e + cy1 * nc + cx0)) + __ldg(e + cy1 * nc + cx1));
      }
      v[j] = v[j] + add;
    }
    st4(x + i0, v);
  }
}

// Exact coarsest-level solve x_c = A_c^-1 rhs_c with the precomputed FP64 inverse of the interior
// block; one warp per problem (tile 0 of its coarsest level), result into buffer 0.
template <class V>
__global__ void __launch_bounds__(256) k_coarse(EngineDev E, TileList tl, int want) {
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
    const ProblemDev& P = E.P[p];
    const LevelDev& d = P.lev[P.coarse];
    const int n = d.n, ni = n - 2, m = P.m;
    const V* rhs = static_cast<const V*>(d.rhs);
    for (int u = lane; u < m; u += 32) {
      const double* row = P.cinv + (long long)u * m;
      double s = 0.0;
      for (int v = 0; v < m; ++v) s = fma(row[v], double(rhs[(v / ni + 1) * n + (v % ni + 1)]), s);
      sol[wib][u] = s;
    }
    __syncwarp();
    V* x = static_cast<V*>(d.x[0]);
    for (int q = lane; q < d.pitch; q += 32) {
      const int iy = q / n, ix = q - iy * n;
      V val = V(0);
      if (q < n * n && ix > 0 && iy > 0 && ix < n - 1 && iy < n - 1)
        val = V(sol[wib][(iy - 1) * ni + (ix - 1)]);
      x[q] = val;
    }
    __syncwarp();
  }
}

// FP64 outer defect of the defect correction: d = b - A x (FP64 bands, FP64 x), written to the
// inner top-level right-hand side as float(d * s); partial[g] = sum d^2.  x = 0 gives d = b.
__global__ void __launch_bounds__(256) k_outer_defect(EngineDev E, TileList tl) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    const ProbState& st = E.S[p];
    if (st.phase != PH_OUTER) continue;
    const ProblemDev& P = E.P[p];
    const LevelDev& top = P.lev[P.L];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    double b[4], r[4];
    ld4(P.b64 + i0, b);
    if (st.x_zero) {
#pragma unroll
      for (int j = 0; j < 4; ++j) r[j] = b[j];
    } else {
      double acc[4], xc[4], dg[4];
      stencil4<F64>(reinterpret_cast<const void* const*>(P.band64), nullptr, P.x64, i0,
                    1LL << P.L, lane, acc, xc, dg);
#pragma unroll
      for (int j = 0; j < 4; ++j) r[j] = b[j] - acc[j];
    }
    const double s = st.s;
    float out[4];
    double q = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      out[j] = __double2float_rn(r[j] * s);
      q += r[j] * r[j];
    }
    st4(static_cast<float*>(top.rhs) + i0, out);
    q = warp_sum(q);
    if (lane == 0) E.partial[g] = q;
  }
}

// x64 += c / s (c = inner top-level iterate, buffer 0), for problems in PH_UPDATE
__global__ void __launch_bounds__(256) k_update(EngineDev E, TileList tl) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    const ProbState& st = E.S[p];
    if (st.phase != PH_UPDATE) continue;
    const ProblemDev& P = E.P[p];
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    float c[4];
    ld4(static_cast<const float*>(P.lev[P.L].x[0]) + i0, c);
    double x[4];
    ld4c(P.x64 + i0, x);
    const double inv_s = 1.0 / st.s;
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = fma(double(c[j]), inv_s, x[j]);
    st4(P.x64 + i0, x);
  }
}

// ||b||^2 partials for problems starting a solve
__global__ void __launch_bounds__(256) k_norm_b(EngineDev E, TileList tl) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int count = *tl.count;
  for (int g = gw; g < count; g += nw) {
    const int2 it = tl.items[g];
    const int p = it.x;
    if (E.S[p].phase != PH_INIT) continue;
    const long long i0 = (long long)it.y * kTile + lane * kLaneNodes;
    double b[4];
    ld4(E.P[p].b64 + i0, b);
    double q = b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3];
    q = warp_sum(q);
    if (lane == 0) E.partial2[g] = q;
  }
}

// Reject right-hand sides with non-zero boundary entries (one block per problem).
__global__ void __launch_bounds__(256) k_boundary_check(EngineDev E) {
  const int p = blockIdx.x;
  if (p >= E.nprob) return;
  ProbState& st = E.S[p];
  if (st.phase != PH_INIT) return;
  const ProblemDev& P = E.P[p];
  const long long n = n_of_dev(P.L);
  int bad = 0;
  for (long long t = threadIdx.x; t < 4 * (n - 1); t += blockDim.x) {
    const long long side = t / (n - 1), k = t - side * (n - 1);
    long long i;
    if (side == 0) i = k;                          // bottom row, ix = 0..n-2
    else if (side == 1) i = k * n + (n - 1);       // right column
    else if (side == 2) i = (n - 1) * n + (n - 1 - k);   // top row
    else i = (n - 1 - k) * n;                      // left column
    if (P.b64[i] != 0.0) bad = 1;
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) { st.status = HN_ERR_ARG; st.phase = PH_DONE; }
}

// Per-problem control of the solver state machine: reduce the problem's norm partials in a fixed
// order (bit-reproducible, independent of the batch), then update its state.
__global__ void __launch_bounds__(256) k_control(EngineDev E, int kind) {
  __shared__ double sh[32];
  const int p = blockIdx.x;
  if (p >= E.nprob) return;
  ProbState& st = E.S[p];
  const int ph = st.phase;
  const bool mine = (kind == CTRL_INIT && ph == PH_INIT) ||
                    (kind == CTRL_CHECK0 && ph == PH_CHECK) ||
                    (kind == CTRL_CHECK && ph == PH_CYCLE) ||
                    (kind == CTRL_OUTER && ph == PH_OUTER) ||
                    (kind == CTRL_INNER && ph == PH_INNER) ||
                    (kind == CTRL_POST && ph == PH_UPDATE);
  if (!mine) return;
  double sum = 0.0;
  if (kind != CTRL_POST) {
    const double* part = kind == CTRL_INIT ? E.partial2 : E.partial;
    const int L = E.P[p].L;
    const int ntiles = (int)(((n_of_dev(L) * n_of_dev(L)) + kTile - 1) / kTile);
    const int off = E.fine_off[p];
    double t = 0.0;
    for (int q = threadIdx.x; q < ntiles; q += blockDim.x) t += part[off + q];
    sum = block_sum256(t, sh);
  }
  if (threadIdx.x != 0) return;
  const Params& prm = E.prm;
  const double nrm = sqrt(sum);
  switch (kind) {
    case CTRL_INIT:
      if (st.status == HN_ERR_ARG) { st.phase = PH_DONE; break; }
      if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; break; }
      if (nrm == 0.0) { st.bnorm = 0.0; st.relres = 0.0; st.status = HN_OK; st.phase = PH_DONE; break; }
      st.bnorm = nrm;
      st.s = 1.0 / nrm;
      st.relres = 1.0;
      if (prm.prec == P64) st.phase = st.x_zero ? PH_CYCLE : PH_CHECK;
      else st.phase = PH_OUTER;
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
      st.dnorm = nrm;
      st.relres = nrm / st.bnorm;
      if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; }
      else if (st.relres <= prm.tol) { st.status = HN_OK; st.phase = PH_DONE; }
      else if (st.outer_iters >= prm.max_outer || st.inner_cycles >= prm.max_cycles) {
        st.status = HN_ERR_NOT_CONVERGED; st.phase = PH_DONE;
      } else {
        st.phase = PH_INNER; st.inner_k = 0; st.zero_top = 1; st.inner_ref = st.s * nrm;
      }
      break;
    case CTRL_INNER:
      st.inner_res = nrm;
      st.inner_k += 1; st.inner_cycles += 1; st.cycles += 1; st.zero_top = 0;
      if (!isfinite(nrm)) { st.status = HN_ERR_NONFINITE; st.phase = PH_DONE; }
      else if (nrm <= prm.inner_tol * st.inner_ref || st.inner_k >= prm.inner_max ||
               st.inner_cycles >= prm.max_cycles)
        st.phase = PH_UPDATE;
      break;
    case CTRL_POST: {
      st.outer_iters += 1;
      st.x_zero = 0;
      // scale for the next defect: the inner solve reduced the defect by about inner_res/inner_ref
      const double red = st.inner_ref > 0.0 ? st.inner_res / st.inner_ref : 1.0;
      const double pred = st.dnorm * fmax(red, 1e-7);
      if (pred > 0.0 && isfinite(pred)) st.s = 1.0 / pred;
      st.phase = PH_OUTER;
      break;
    }
    default: break;
  }
}

// Count problems still running; publish to the host word and, inside a device-side loop, to the
// graph's while-condition.  Past the iteration limit every running problem is stopped as not
// converged, so a device-side loop always ends.
__global__ void __launch_bounds__(256) k_summary(EngineDev E, cudaGraphConditionalHandle h,
                                                 int use_handle) {
  __shared__ double sh[32];
  __shared__ unsigned over;
  if (threadIdx.x == 0) {
    const unsigned it = E.iter ? (*E.iter += 1) : 0u;
    over = (E.iter && it > E.iter_limit) ? 1u : 0u;
  }
  __syncthreads();
  double c = 0.0;
  for (int p = threadIdx.x; p < E.nprob; p += blockDim.x) {
    ProbState& st = E.S[p];
    if (st.phase != PH_DONE && over) { st.status = HN_ERR_NOT_CONVERGED; st.phase = PH_DONE; }
    c += st.phase != PH_DONE ? 1.0 : 0.0;
  }
  c = block_sum256(c, sh);
  if (threadIdx.x == 0) {
    const unsigned active = (unsigned)c;
    if (E.active_host) *E.active_host = active;
    if (use_handle) cudaGraphSetConditional(h, active > 0 ? 1u : 0u);
  }
}

inline int grid_or_one(int g) { return g < 1 ? 1 : g; }

template <class Pol>
cudaError_t launch_band_t(int mode, const EngineDev& E, TileList tl, int level, int want,
                          int in_sel, int grid, cudaStream_t s) {
  grid = grid_or_one(grid);
  switch (mode) {
    case M_SPMV: k_band<Pol, M_SPMV><<<grid, 256, 0, s>>>(E, tl, level, want, in_sel); break;
    case M_DEFECT: k_band<Pol, M_DEFECT><<<grid, 256, 0, s>>>(E, tl, level, want, in_sel); break;
    case M_JACOBI: k_band<Pol, M_JACOBI><<<grid, 256, 0, s>>>(E, tl, level, want, in_sel); break;
    case M_JACOBI_FIRST:
      k_band<Pol, M_JACOBI_FIRST><<<grid, 256, 0, s>>>(E, tl, level, want, in_sel); break;
    case M_CHECK: k_band<Pol, M_CHECK><<<grid, 256, 0, s>>>(E, tl, level, want, in_sel); break;
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
                          int first, int grid, cudaStream_t s) {
  return launch_band(first ? M_JACOBI_FIRST : M_JACOBI, E, tl, level, want, in_sel, grid, s);
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
  if (E.prm.prec == P64) k_restrict<double><<<grid, 256, 0, s>>>(E, tl_coarse, fine_level, want);
  else k_restrict<float><<<grid, 256, 0, s>>>(E, tl_coarse, fine_level, want);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const EngineDev& E, TileList tl, int level, int want, int x_sel,
                           int grid, cudaStream_t s) {
  grid = grid_or_one(grid);
  if (E.prm.prec == P64) k_prolong<double><<<grid, 256, 0, s>>>(E, tl, level, want, x_sel);
  else k_prolong<float><<<grid, 256, 0, s>>>(E, tl, level, want, x_sel);
  return cudaGetLastError();
}

cudaError_t launch_coarse(const EngineDev& E, TileList tl, int want, int grid, cudaStream_t s) {
  grid = grid_or_one(grid);
  if (E.prm.prec == P64) k_coarse<double><<<grid, 256, 0, s>>>(E, tl, want);
  else k_coarse<float><<<grid, 256, 0, s>>>(E, tl, want);
  return cudaGetLastError();
}

cudaError_t launch_outer_defect(const EngineDev& E, TileList fine, int grid, cudaStream_t s) {
  k_outer_defect<<<grid_or_one(grid), 256, 0, s>>>(E, fine);
  return cudaGetLastError();
}

cudaError_t launch_update(const EngineDev& E, TileList fine, int grid, cudaStream_t s) {
  k_update<<<grid_or_one(grid), 256, 0, s>>>(E, fine);
  return cudaGetLastError();
}

cudaError_t launch_norm_b(const EngineDev& E, TileList fine, int grid, cudaStream_t s) {
  k_norm_b<<<grid_or_one(grid), 256, 0, s>>>(E, fine);
  return cudaGetLastError();
}

cudaError_t launch_control(const EngineDev& E, int kind, cudaStream_t s) {
  k_control<<<grid_or_one(E.nprob), 256, 0, s>>>(E, kind);
  return cudaGetLastError();
}

cudaError_t launch_summary(const EngineDev& E, cudaGraphConditionalHandle h, int use_handle,
                           cudaStream_t s) {
  k_summary<<<1, 256, 0, s>>>(E, h, use_handle);
  return cudaGetLastError();
}

cudaError_t launch_boundary_check(const EngineDev& E, cudaStream_t s) {
  k_boundary_check<<<grid_or_one(E.nprob), 256, 0, s>>>(E);
  return cudaGetLastError();
}

// the fine-level defect norm of the V-cycle's own precision (convergence check)
cudaError_t launch_check(const EngineDev& E, TileList fine_by_problem_top, int want, int x_sel,
                         int grid, cudaStream_t s) {
  // the fine work list enumerates every problem's top level; the level is taken per problem
  return launch_band(M_CHECK, E, fine_by_problem_top, -1, want, x_sel, grid, s);
}

}  // namespace hn
