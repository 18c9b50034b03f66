// Setup kernels: GPU assembly of the Q1 stiffness matrix into 9 bands (Sec. 2.1, full assembly
// with fixed band positions), coefficient coarsening for re-discretised coarse levels, and the
// conversions of the FP64 bands to the inner storage precisions (FP32 cast; FP16 codes with one
// FP32 scale per band).
#include "hn_internal.h"

namespace hn {

namespace {

// Q1 element stiffness on a square cell (h-independent in 2D), local nodes (0,0), (1,0), (1,1),
// (0,1): diagonal 4/6, edge neighbours -1/6, opposite corner -2/6.
__device__ __forceinline__ double kdiag() { return 4.0 / 6.0; }
__device__ __forceinline__ double kedge() { return -1.0 / 6.0; }
__device__ __forceinline__ double kcorner() { return -2.0 / 6.0; }

// One thread per node of the padded range.  For node (ix, iy) the 4 surrounding cells are taken
// in the order sw (ix-1, iy-1), se (ix, iy-1), nw (ix-1, iy), ne (ix, iy); a cell off the grid
// (at a free Neumann side) contributes nothing.  Every band entry is the sum of its cells'
// element-matrix contributions a_c * K in that order, with explicit round-to-nearest operations
// (no contraction).  Entries towards off-grid or Dirichlet neighbours are exactly 0; Dirichlet
// nodes are eliminated symmetrically and become identity rows, as do padding rows.
__global__ void k_assemble(int L, const double* __restrict__ coef, BandPtrs64 band,
                           double* __restrict__ wdinv, double omega, int bc) {
  const long long n = n_of_dev(L), N = n * n, nc = n - 1;
  const long long pitch = ((N + kTile - 1) / kTile) * kTile;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pitch) return;
  double v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = 0.0;
  bool inner = false;
  long long ix = 0, iy = 0;
  if (i < N) {
    iy = i / n;
    ix = i - iy * n;
    inner = !is_dirichlet(ix, iy, n, bc);
  }
  if (!inner) {
    v[4] = 1.0;
  } else {
    auto A = [&](long long ex, long long ey) {
      if (ex < 0 || ey < 0 || ex >= nc || ey >= nc) return 0.0;   // no cell there
      return coef ? coef[ey * nc + ex] : 1.0;
    };
    const double sw = A(ix - 1, iy - 1), se = A(ix, iy - 1), nw = A(ix - 1, iy), ne = A(ix, iy);
    // k = 0: (-1,-1) via sw; 1: (-1,0) via sw, se; 2: (-1,+1) via se; 3: (0,-1) via sw, nw;
    // 4: diagonal via sw, se, nw, ne; 5: (0,+1) via se, ne; 6: (+1,-1) via nw; 7: (+1,0) via
    // nw, ne; 8: (+1,+1) via ne
    v[0] = __dmul_rn(sw, kcorner());
    v[1] = __dadd_rn(__dmul_rn(sw, kedge()), __dmul_rn(se, kedge()));
    v[2] = __dmul_rn(se, kcorner());
    v[3] = __dadd_rn(__dmul_rn(sw, kedge()), __dmul_rn(nw, kedge()));
    v[4] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(sw, kdiag()), __dmul_rn(se, kdiag())),
                               __dmul_rn(nw, kdiag())), __dmul_rn(ne, kdiag()));
    v[5] = __dadd_rn(__dmul_rn(se, kedge()), __dmul_rn(ne, kedge()));
    v[6] = __dmul_rn(nw, kcorner());
    v[7] = __dadd_rn(__dmul_rn(nw, kedge()), __dmul_rn(ne, kedge()));
    v[8] = __dmul_rn(ne, kcorner());
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const long long jx = ix + (k % 3 - 1), jy = iy + (k / 3 - 1);
      if (jx < 0 || jy < 0 || jx >= n || jy >= n || is_dirichlet(jx, jy, n, bc)) v[k] = 0.0;
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) band.p[k][i] = v[k];
  if (wdinv) wdinv[i] = omega / v[4];
}

// coarse cell coefficient = mean of the 4 child cells, summed row by row, left to right
__global__ void k_coarsen_coef(int Lf, const double* __restrict__ af, double* __restrict__ ac) {
  const long long ncf = 1LL << Lf, ncc = ncf >> 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncc * ncc) return;
  const long long Ey = t / ncc, Ex = t - Ey * ncc, y = 2 * Ey, x = 2 * Ex;
  const double s = __dadd_rn(__dadd_rn(__dadd_rn(af[y * ncf + x], af[y * ncf + x + 1]),
                                       af[(y + 1) * ncf + x]), af[(y + 1) * ncf + x + 1]);
  ac[t] = __dmul_rn(s, 0.25);
}

__global__ void k_to_f32(long long pitch, BandPtrs64c src, BandPtrs32 dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pitch) return;
#pragma unroll
  for (int k = 0; k < 9; ++k) dst.p[k][i] = __double2float_rn(src.p[k][i]);
}

// FP16 storage in row-sum form: arrays k != 4 are the couplings, array 4 the row sum
// rho_i = sum_k band_k[i] (k = 0..8 in order, FP64).  Applied as rho_i x_i + sum a_k (x_j - x_i),
// the quantized operator keeps the zero row sums of the Laplacian exactly.
__device__ __forceinline__ double rowsum_value(const BandPtrs64c& src, int k, long long i) {
  if (k != 4) return src.p[k][i];
  double r = src.p[0][i];
#pragma unroll
  for (int q = 1; q < 9; ++q) r = __dadd_rn(r, src.p[q][i]);
  return r;
}

// max_i |v_k[i]| per array: non-negative doubles order like their bit patterns
__global__ void k_absmax(long long pitch, BandPtrs64c src, unsigned long long* absmax9) {
  __shared__ unsigned long long sh[9];
  if (threadIdx.x < 9) sh[threadIdx.x] = 0ull;
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < pitch) {
#pragma unroll
    for (int k = 0; k < 9; ++k)
      atomicMax(&sh[k], (unsigned long long)__double_as_longlong(fabs(rowsum_value(src, k, i))));
  }
  __syncthreads();
  if (threadIdx.x < 9) atomicMax(&absmax9[threadIdx.x], sh[threadIdx.x]);
}

// FP16 code = round-to-nearest-even(v_k / s_k), quotient in FP64, s_k = float(max |v_k|)
__global__ void k_to_f16(long long pitch, BandPtrs64c src, const unsigned long long* absmax9,
                         BandPtrs16 dst, float* scales) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float sk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float s = __double2float_rn(__longlong_as_double((long long)absmax9[k]));
    sk[k] = s == 0.0f ? 1.0f : s;
  }
  if (i == 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) scales[k] = sk[k];
  }
  if (i >= pitch) return;
#pragma unroll
  for (int k = 0; k < 9; ++k) dst.p[k][i] = __double2half(rowsum_value(src, k, i) / (double)sk[k]);
}

// omega / diag in FP32: FP32 bands divide by array 4; FP16 bands by the row-sum diagonal
// rho - sum_{k != 4} a_k with every a_k = scale_k * code rounded on its own (band order)
struct BandPtrsAny { const void* p[9]; };
struct Scales9 { float s[9]; };
__global__ void k_wdf(long long pitch, int prec, BandPtrsAny band, Scales9 sc, float omega,
                      float* __restrict__ wdf) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pitch) return;
  float dg;
  if (prec == P32) {
    dg = static_cast<const float*>(band.p[4])[i];
  } else {
    dg = __fmul_rn(sc.s[4], __half2float(static_cast<const __half*>(band.p[4])[i]));
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (k == 4) continue;
      dg -= __fmul_rn(sc.s[k], __half2float(static_cast<const __half*>(band.p[k])[i]));
    }
  }
  wdf[i] = omega / dg;
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_assemble(int L, const double* coef, const BandPtrs64& band, double* wdinv,
                            double omega, int bc, cudaStream_t s) {
  const long long pitch = pitch_of(L);
  k_assemble<<<blocks_for(pitch, 256), 256, 0, s>>>(L, coef, band, wdinv, omega, bc);
  return cudaGetLastError();
}

cudaError_t launch_coarsen_coef(int Lf, const double* af, double* ac, cudaStream_t s) {
  const long long ncc = 1LL << (Lf - 1);
  k_coarsen_coef<<<blocks_for(ncc * ncc, 256), 256, 0, s>>>(Lf, af, ac);
  return cudaGetLastError();
}

cudaError_t launch_band_to_f32(int L, const BandPtrs64c& src, const BandPtrs32& dst,
                               cudaStream_t s) {
  const long long pitch = pitch_of(L);
  k_to_f32<<<blocks_for(pitch, 256), 256, 0, s>>>(pitch, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_band_to_f16(int L, const BandPtrs64c& src, unsigned long long* absmax9,
                               const BandPtrs16& dst, float* scales_dev, cudaStream_t s) {
  const long long pitch = pitch_of(L);
  cudaError_t e = cudaMemsetAsync(absmax9, 0, 9 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_absmax<<<blocks_for(pitch, 256), 256, 0, s>>>(pitch, src, absmax9);
  k_to_f16<<<blocks_for(pitch, 256), 256, 0, s>>>(pitch, src, absmax9, dst, scales_dev);
  return cudaGetLastError();
}

cudaError_t launch_wdf(int L, int prec, const void* const* band, const float* scale, double omega,
                       float* wdf, cudaStream_t s) {
  const long long pitch = pitch_of(L);
  BandPtrsAny b{};
  Scales9 sc{};
  for (int k = 0; k < 9; ++k) { b.p[k] = band[k]; sc.s[k] = scale[k]; }
  k_wdf<<<blocks_for(pitch, 256), 256, 0, s>>>(pitch, prec, b, sc, (float)omega, wdf);
  return cudaGetLastError();
}

}  // namespace hn
