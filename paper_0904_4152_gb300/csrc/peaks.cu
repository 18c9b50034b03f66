// Arithmetic-rate measurement (measurement support, not part of the method).  The FP64 band and
// transfer kernels on this part do more FP64 work per byte than the pipe sustains at the HBM
// rate, so their roofline is min(HBM bandwidth, FP64 rate / FP64 operations per node); these
// kernels measure the FP64 rate (and the FP32 rate for comparison) on the device they run on.
//
// Each thread keeps 8 independent chains of one operation in registers (so that the pipe, not the
// latency of a chain, is the limit), `iters` steps each; one wave of 4 blocks of 256 threads per
// SM.  The chains' final values are written out so that the work is not removed.
#include <algorithm>

#include "engine.h"
#include "../../include/hn_profile.h"

namespace hn {
namespace {

constexpr int kChains = 8;

// op 0: fma(a, x, y), 1: a + x, 2: a * x; chains start from distinct values near 1 so that
// nothing overflows or becomes subnormal over the loop
template <class T, int OP>
__global__ void __launch_bounds__(256) k_rate(int iters, T x, T y, T* out) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = T(1) + T(c + threadIdx.x) * T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (OP == 0) a[c] = fma(a[c], x, y);
      else if constexpr (OP == 1) a[c] = a[c] + x;
      else a[c] = a[c] * x;
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T, int OP>
hn_status time_rate(int iters, int grid, T* out, cudaStream_t s, double* ops_per_s) {
  // x, y keep every chain bounded: a -> a * x + y with |x| < 1 converges; additions of a tiny
  // x and multiplications by x near 1 drift slowly
  const T x = OP == 1 ? T(1e-12) : T(0.999999);
  const T y = T(1e-6);
  k_rate<T, OP><<<grid, 256, 0, s>>>(iters / 8, x, y, out);   // warm-up
  HN_CUDA(cudaGetLastError());
  cudaEvent_t e0, e1;
  HN_CUDA(cudaEventCreate(&e0));
  HN_CUDA(cudaEventCreate(&e1));
  struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
  HN_CUDA(cudaEventRecord(e0, s));
  k_rate<T, OP><<<grid, 256, 0, s>>>(iters, x, y, out);
  HN_CUDA(cudaGetLastError());
  HN_CUDA(cudaEventRecord(e1, s));
  HN_CUDA(cudaEventSynchronize(e1));
  float ms = 0.0f;
  HN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *ops_per_s = (double)grid * 256.0 * kChains * iters / (ms * 1e-3);
  return HN_OK;
}

}  // namespace
}  // namespace hn

using namespace hn;

extern "C" hn_status hn_measure_fp_rates(hn_fp_rates* out) {
  clear_error();
  if (!out) return set_error(HN_ERR_ARG, "null argument");
  int dev = 0, sms = 0;
  HN_CUDA(cudaGetDevice(&dev));
  HN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(sms, 1) * 4;
  cudaStream_t s = nullptr;
  HN_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct St { cudaStream_t s; ~St() { cudaStreamDestroy(s); } } st{s};
  void* buf = nullptr;
  HN_CUDA(cudaMalloc(&buf, (size_t)grid * 256 * sizeof(double)));
  struct Buf { void* p; ~Buf() { cudaFree(p); } } bf{buf};
  double* d = static_cast<double*>(buf);
  float* f = static_cast<float*>(buf);
  // FP64 steps: ~2 ms each at the expected rate (4 blocks x 256 threads x 8 chains per SM)
  hn_status st0 = time_rate<double, 0>(2048, grid, d, s, &out->fp64_fma_per_s);
  if (st0 == HN_OK) st0 = time_rate<double, 1>(2048, grid, d, s, &out->fp64_add_per_s);
  if (st0 == HN_OK) st0 = time_rate<double, 2>(2048, grid, d, s, &out->fp64_mul_per_s);
  if (st0 == HN_OK) st0 = time_rate<float, 0>(65536, grid, f, s, &out->fp32_fma_per_s);
  return st0;
}
