// BLAS level-1 kernels (axpy, dot, nrm2) on device vectors: the memory-bound operations the paper
// measures on every backend (Sec. 6.1, Fig. 2).  The declarations and their contract are in
// include/hn_blas1.h.
#include "engine.h"
#include "../../include/hn_blas1.h"

namespace hn {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 16384;          // elements reduced by one block (64 per thread)
constexpr unsigned kFull = 0xffffffffu;

inline int stream_grid(long long work_items) {
  // a grid-stride launch of at most 8 resident 256-thread blocks per SM
  const long long cap = (long long)sm_count() * 8;
  const long long g = (work_items + kThreads - 1) / kThreads;
  return (int)std::max<long long>(1, std::min(g, cap));
}

// ------------------------------------------------------------------------------------ axpy
__global__ void __launch_bounds__(kThreads) k_axpy_f32(long long n, float a, const float* __restrict__ x,
                                                       float* __restrict__ y, int vec) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  long long done = 0;
  if (vec) {
    const long long n4 = n / 4;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4* y4 = reinterpret_cast<float4*>(y);
    long long i = tid;
    for (; i + nt < n4; i += 2 * nt) {           // two independent 16-byte loads per operand
      const float4 xa = __ldg(x4 + i), xb = __ldg(x4 + i + nt);
      float4 ya = y4[i], yb = y4[i + nt];
      ya.x = fmaf(a, xa.x, ya.x); ya.y = fmaf(a, xa.y, ya.y); ya.z = fmaf(a, xa.z, ya.z); ya.w = fmaf(a, xa.w, ya.w);
      yb.x = fmaf(a, xb.x, yb.x); yb.y = fmaf(a, xb.y, yb.y); yb.z = fmaf(a, xb.z, yb.z); yb.w = fmaf(a, xb.w, yb.w);
      y4[i] = ya;
      y4[i + nt] = yb;
    }
    for (; i < n4; i += nt) {
      const float4 xa = __ldg(x4 + i);
      float4 ya = y4[i];
      ya.x = fmaf(a, xa.x, ya.x); ya.y = fmaf(a, xa.y, ya.y); ya.z = fmaf(a, xa.z, ya.z); ya.w = fmaf(a, xa.w, ya.w);
      y4[i] = ya;
    }
    done = n4 * 4;
  }
  for (long long i = done + tid; i < n; i += nt) y[i] = fmaf(a, __ldg(x + i), y[i]);
}

__global__ void __launch_bounds__(kThreads) k_axpy_f64(long long n, double a, const double* __restrict__ x,
                                                       double* __restrict__ y, int vec) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  long long done = 0;
  if (vec) {
    const long long n2 = n / 2;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    double2* y2 = reinterpret_cast<double2*>(y);
    long long i = tid;
    for (; i + nt < n2; i += 2 * nt) {
      const double2 xa = __ldg(x2 + i), xb = __ldg(x2 + i + nt);
      double2 ya = y2[i], yb = y2[i + nt];
      ya.x = fma(a, xa.x, ya.x); ya.y = fma(a, xa.y, ya.y);
      yb.x = fma(a, xb.x, yb.x); yb.y = fma(a, xb.y, yb.y);
      y2[i] = ya;
      y2[i + nt] = yb;
    }
    for (; i < n2; i += nt) {
      const double2 xa = __ldg(x2 + i);
      double2 ya = y2[i];
      ya.x = fma(a, xa.x, ya.x); ya.y = fma(a, xa.y, ya.y);
      y2[i] = ya;
    }
    done = n2 * 2;
  }
  for (long long i = done + tid; i < n; i += nt) y[i] = fma(a, __ldg(x + i), y[i]);
}

// --------------------------------------------------------------------------- dot and nrm2
// Chunk b holds elements [b*kChunk, min(n, (b+1)*kChunk)).  In a chunk, thread t takes the
// element groups {4t + 1024 j .. 4t + 1024 j + 3}, j = 0..15 (FP32; FP64: {2t + 512 j, +1},
// j = 0..31), and group j goes to chain j mod 4, its products added in element order.  FP32
// vectors form each chain in FP32 (fused multiply-add; the FP64 pipe of this part would bound
// the kernel below the memory bandwidth), FP64 vectors in FP64.  The chains combine as
// (c0 + c1) + (c2 + c3) in FP64, then the block adds its threads in a fixed tree.  Blocks walk
// the chunks with a stride of the grid; the last block to finish adds the chunk sums in order.
// 16-byte aligned vectors use 16-byte loads; others take the same order element by element.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();                                 // sh may still be read by an earlier call
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    t = warp_sum_d(t);
  }
  return t;   // valid in thread 0
}

template <class T> struct Lanes;                   // elements per 16-byte group
template <> struct Lanes<float> { static constexpr int k = 4; using V = float4; };
template <> struct Lanes<double> { static constexpr int k = 2; using V = double2; };

template <class T>
__device__ __forceinline__ T dot_group(const T* x, const T* y, long long i, long long end, bool vec,
                                       T c) {
  constexpr int K = Lanes<T>::k;
  if (vec && i + K <= end) {
    const typename Lanes<T>::V a = __ldg(reinterpret_cast<const typename Lanes<T>::V*>(x + i));
    const typename Lanes<T>::V b = __ldg(reinterpret_cast<const typename Lanes<T>::V*>(y + i));
    if constexpr (K == 4) {
      c = fma(a.x, b.x, c); c = fma(a.y, b.y, c); c = fma(a.z, b.z, c); c = fma(a.w, b.w, c);
    } else {
      c = fma(a.x, b.x, c); c = fma(a.y, b.y, c);
    }
    return c;
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (i + k < end) c = fma(__ldg(x + i + k), __ldg(y + i + k), c);
  return c;
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_dot(long long n, long long m, const T* __restrict__ x,
                                                  const T* __restrict__ y, double* __restrict__ part,
                                                  unsigned* __restrict__ ticket, double* __restrict__ result,
                                                  int root, int vec) {
  constexpr int K = Lanes<T>::k;
  constexpr int G = kChunk / (kThreads * K);       // groups per thread per chunk (16 or 32)
  __shared__ double sh[32];
  __shared__ bool last;
  for (long long b = blockIdx.x; b < m; b += gridDim.x) {
    const long long base = b * kChunk;
    const long long end = min(n, base + kChunk);
    T c[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const long long i = base + (long long)K * threadIdx.x + (long long)j * K * kThreads;
      c[j & 3] = dot_group<T>(x, y, i, end, vec != 0, c[j & 3]);
    }
    const double s = block_sum_d((double(c[0]) + double(c[1])) + (double(c[2]) + double(c[3])), sh);
    if (threadIdx.x == 0) part[b] = s;
  }
  // the last block to finish adds the chunk sums in order: thread t takes chunks t + 256 j into
  // chain j mod 4
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double c[4] = {0.0, 0.0, 0.0, 0.0};
  long long j = 0;
  for (long long q = threadIdx.x; q < m; q += kThreads, ++j) c[j & 3] += __ldcg(part + q);
  const double s = block_sum_d((c[0] + c[1]) + (c[2] + c[3]), sh);
  if (threadIdx.x == 0) {
    *result = root ? sqrt(s) : s;
    *ticket = 0u;                                  // ready for the next call
  }
}

__global__ void k_zero(double* result) { *result = 0.0; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

hn_status check_common(hn_dtype t, long long n) {
  if (t != HN_F32 && t != HN_F64) return set_error(HN_ERR_ARG, "unknown element type %d", (int)t);
  if (n < 0) return set_error(HN_ERR_ARG, "negative length");
  return HN_OK;
}

hn_status reduce(hn_dtype t, long long n, const void* x, const void* y, double* result, int root,
                 cudaStream_t s) {
  if (n == 0) {
    k_zero<<<1, 1, 0, s>>>(result);
    HN_CUDA(cudaGetLastError());
    return HN_OK;
  }
  const long long m = (n + kChunk - 1) / kChunk;
  // chunk sums and the finishing ticket, stream-ordered
  void* scratch = nullptr;
  HN_CUDA(cudaMallocAsync(&scratch, (size_t)m * sizeof(double) + 16, s));
  double* part = static_cast<double*>(scratch);
  unsigned* ticket = reinterpret_cast<unsigned*>(part + m);
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
  const int vec = aligned16(x) && aligned16(y);
  const int grid = (int)std::min<long long>(m, (long long)sm_count() * 8);
  if (e == cudaSuccess) {
    if (t == HN_F32)
      k_dot<float><<<grid, kThreads, 0, s>>>(n, m, static_cast<const float*>(x), static_cast<const float*>(y),
                                             part, ticket, result, root, vec);
    else
      k_dot<double><<<grid, kThreads, 0, s>>>(n, m, static_cast<const double*>(x), static_cast<const double*>(y),
                                              part, ticket, result, root, vec);
    e = cudaGetLastError();
  }
  const cudaError_t f = cudaFreeAsync(scratch, s);
  HN_CUDA(e);
  HN_CUDA(f);
  return HN_OK;
}

}  // namespace
}  // namespace hn

using namespace hn;

extern "C" hn_status hn_axpy(hn_dtype type, long long n, double alpha, const void* x, void* y, void* stream) {
  clear_error();
  HN_TRY(check_common(type, n));
  if (n == 0) return HN_OK;
  if (!x || !y) return set_error(HN_ERR_ARG, "null vector");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int vec = aligned16(x) && aligned16(y);
  if (type == HN_F32) {
    k_axpy_f32<<<stream_grid(vec ? n / 8 + 1 : n), kThreads, 0, s>>>(
        n, (float)alpha, static_cast<const float*>(x), static_cast<float*>(y), vec);
  } else {
    k_axpy_f64<<<stream_grid(vec ? n / 4 + 1 : n), kThreads, 0, s>>>(
        n, alpha, static_cast<const double*>(x), static_cast<double*>(y), vec);
  }
  HN_CUDA(cudaGetLastError());
  return HN_OK;
}

extern "C" hn_status hn_dot(hn_dtype type, long long n, const void* x, const void* y, double* result,
                            void* stream) {
  clear_error();
  HN_TRY(check_common(type, n));
  if (!result || (n > 0 && (!x || !y))) return set_error(HN_ERR_ARG, "null pointer");
  return reduce(type, n, x, y, result, 0, static_cast<cudaStream_t>(stream));
}

extern "C" hn_status hn_nrm2(hn_dtype type, long long n, const void* x, double* result, void* stream) {
  clear_error();
  HN_TRY(check_common(type, n));
  if (!result || (n > 0 && !x)) return set_error(HN_ERR_ARG, "null pointer");
  return reduce(type, n, x, x, result, 1, static_cast<cudaStream_t>(stream));
}
