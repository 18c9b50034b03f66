// Defect and norm of an assembled operator without any device allocation.
//
// hn_band_defect_norm_static computes r = b - A x and ||r||_2 for an operator built by
// hn_band_create, on caller-owned device vectors.  It exists for callers that cannot call
// cudaMalloc at that point: code that runs while another thread captures a CUDA graph in global
// mode (allocation is not permitted then), processes that hand out their whole device-memory plan
// up front, and latency-critical paths where cudaMalloc / cudaFree would synchronize the device.
// The only temporary, one partial sum of squares per 128-node tile, lives in the file-scope array
// below, so the call allocates nothing: every GPU that loads the library holds the array (512 KiB)
// until the process exits.
#include <algorithm>
#include <mutex>

#include "engine.h"

namespace hn {
namespace {

constexpr int kStaticTiles = 65536;                      // partial sums the array holds
constexpr long long kStaticMaxNodes = (long long)kStaticTiles * kTile;   // 8,388,608 nodes
constexpr unsigned kFullMask = 0xffffffffu;

// Scratch shared by every call on a device.  Each call writes slots [0, tiles) before reading
// them, so nothing has to start at zero; calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_partials[kStaticTiles];

// device address of g_partials, looked up once per device with that device current
constexpr int kMaxDevices = 64;
double* g_addr[kMaxDevices] = {};
std::mutex g_addr_mu;

hn_status scratch_for_current_device(double** out) {
  int dev = 0;
  HN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(HN_ERR_ARG, "device ordinal %d unsupported", dev);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    HN_CUDA(cudaGetSymbolAddress(&p, g_partials));
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return HN_OK;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
  return v;
}

// Row window w[o + 2] = x[a + o], o = -2..5, of plain (unpadded) vectors: entries outside [0, N)
// read as 0 (their band entries are 0).  Warps whose windows lie inside use aligned vector loads
// and shuffles for the overhang, as the solver's kernel does; the first and last rows fall back
// to guarded scalar loads.
__device__ __forceinline__ void row_window(const double* __restrict__ x, long long a, long long N,
                                           int lane, double (&w)[8]) {
  const bool inside = __all_sync(kFullMask, a - 2 >= 0 && a + 5 < N);
  if (inside) {
    const double2 p = __ldg(reinterpret_cast<const double2*>(x + a));
    const double2 q = __ldg(reinterpret_cast<const double2*>(x + a) + 1);
    double l2 = __shfl_up_sync(kFullMask, q.x, 1), l1 = __shfl_up_sync(kFullMask, q.y, 1);
    double r0 = __shfl_down_sync(kFullMask, p.x, 1), r1 = __shfl_down_sync(kFullMask, p.y, 1);
    if (lane == 0) { l2 = __ldg(x + a - 2); l1 = __ldg(x + a - 1); }
    if (lane == 31) { r0 = __ldg(x + a + 4); r1 = __ldg(x + a + 5); }
    w[0] = l2; w[1] = l1; w[2] = p.x; w[3] = p.y; w[4] = q.x; w[5] = q.y; w[6] = r0; w[7] = r1;
  } else {
#pragma unroll
    for (int o = -2; o <= 5; ++o) {
      const long long j = a + o;
      w[o + 2] = (j >= 0 && j < N) ? __ldg(x + j) : 0.0;
    }
  }
}

// r = b - A x on 128-node warp-tiles of [0, N) (the last one ragged); slot t of the scratch gets
// the tile's sum of r^2.  Bands are the operator's pitch-padded FP64 arrays.
__global__ void __launch_bounds__(256) k_defect_static(BandPtrs64c band, int L, long long N,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ b,
                                                       double* __restrict__ r, double* partials,
                                                       int tiles) {
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const long long shift = 1LL << L;
  for (int t = gw; t < tiles; t += nw) {
    const long long i0 = (long long)t * kTile + lane * kLaneNodes;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      double w[8];
      row_window(x, i0 + dy * shift, N, lane, w);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int k = (dy + 1) * 3 + (dx + 1);
        const double2 p = __ldg(reinterpret_cast<const double2*>(band.p[k] + i0));
        const double2 q = __ldg(reinterpret_cast<const double2*>(band.p[k] + i0) + 1);
        const double bk[4] = {p.x, p.y, q.x, q.y};
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fma(bk[j], w[j + dy + dx + 2], acc[j]);
      }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long i = i0 + j;
      if (i < N) {
        const double ri = __ldg(b + i) - acc[j];
        r[i] = ri;
        s += ri * ri;
      }
    }
    s = warp_sum_d(s);
    if (lane == 0) partials[t] = s;
  }
}

// ||r|| = sqrt of the tile sums added in a fixed order (one block): the result does not depend
// on the grid of the first kernel
__global__ void __launch_bounds__(256) k_sum_partials(const double* partials, int tiles,
                                                      double* norm) {
  __shared__ double sh[8];
  double t = 0.0;
  for (int q = threadIdx.x; q < tiles; q += blockDim.x) t += partials[q];
  t = warp_sum_d(t);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
    v = warp_sum_d(v);
    if (threadIdx.x == 0) *norm = sqrt(v);
  }
}

}  // namespace
}  // namespace hn

using namespace hn;

extern "C" hn_status hn_band_defect_norm_static(const hn_band* A, const double* x, const double* b,
                                                double* r, double* norm, void* stream) {
  clear_error();
  if (!A || !x || !b || !r || !norm) return set_error(HN_ERR_ARG, "null argument");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(b) |
       reinterpret_cast<uintptr_t>(r)) & 15)
    return set_error(HN_ERR_ARG, "x, b and r must be 16-byte aligned device pointers");
  if ((reinterpret_cast<uintptr_t>(norm) & 7))
    return set_error(HN_ERR_ARG, "norm must be an 8-byte aligned device pointer");
  {   // r is written while neighbouring warps still read x and b over the stencil's reach
    const uintptr_t r0 = reinterpret_cast<uintptr_t>(r), r1 = r0 + (uintptr_t)A->N * 8;
    for (const double* v : {x, b}) {
      const uintptr_t v0 = reinterpret_cast<uintptr_t>(v), v1 = v0 + (uintptr_t)A->N * 8;
      if (r0 < v1 && v0 < r1) return set_error(HN_ERR_ARG, "r must not overlap x or b");
    }
  }
  {
    int dev = 0;
    HN_CUDA(cudaGetDevice(&dev));
    if (dev != A->device)
      return set_error(HN_ERR_ARG, "the operator lives on device %d, the current device is %d",
                       A->device, dev);
  }
  if (A->N > kStaticMaxNodes)
    return set_error(HN_ERR_ARG,
                     "%lld nodes exceed the static scratch of this entry point (at most %lld nodes, "
                     "level 11); use hn_mg_apply",
                     A->N, kStaticMaxNodes);
  double* scratch = nullptr;
  HN_TRY(scratch_for_current_device(&scratch));
  const int tiles = (int)((A->N + kTile - 1) / kTile);
  BandPtrs64c bp{};
  for (int k = 0; k < 9; ++k) bp.p[k] = A->band[k];
  int sms = 0;
  HN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, A->device));
  const int grid = std::max(1, std::min((tiles + 7) / 8, std::max(sms, 1) * 4));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_defect_static<<<grid, 256, 0, s>>>(bp, A->L, A->N, x, b, r, scratch, tiles);
  HN_CUDA(cudaGetLastError());
  k_sum_partials<<<1, 256, 0, s>>>(scratch, tiles, norm);
  HN_CUDA(cudaGetLastError());
  return HN_OK;
}
