// Banded matrices with four bands at arbitrary positions and the fused shallow-water prediction
// step (Sec. 2.2, Sec. 4.1).  The contract (operands, rounding order, errors) is in
// include/hn_swe.h.  Both kernels are memory bound: a thread owns 4 consecutive rows, reads the
// band values and the centre vectors with 16-byte loads, and gathers the shifted operand windows
// x[i + offset .. i + offset + 3] with two aligned 16-byte loads (the misalignment offset mod 4 is
// the same for every thread of a launch, so the selection does not diverge); neighbouring
// threads share those lines through L1.  Rows whose window leaves 0..n-1 take a checked path.
#include <climits>

#include "engine.h"
#include "../../include/hn_swe.h"

namespace hn {
namespace {

constexpr int kThreads = 256;

struct Band4Arg {
  long long off[4];
  const void* band[4];
};
struct SweArg {
  Band4Arg M[4];
  const void* x[4];      // operand of each matrix (v, w, u, u; one matrix for the SpMV)
  const void* u;         // start of the running sum (nullptr: 0)
  const void* s;         // added last (nullptr: nothing)
  void* out;
  long long n;
  long long lo, hi;      // rows i0 with i0 + lo >= 0 and i0 + hi <= n read every window in range
  int nmat;
};

template <class T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void ld(const float* p, float (&o)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  }
  static __device__ __forceinline__ void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void ld(const double* p, double (&o)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  static __device__ __forceinline__ void st(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// x[j0 .. j0+3], j0 = i0 + off with i0 a multiple of 4: from the aligned 8-element span starting
// at j0 - mis, mis = off mod 4 (the same for every thread of a launch); selects, not branches, so
// the loads of all bands can be issued together
template <class T>
__device__ __forceinline__ void window4(const T* x, long long base, int mis, T (&o)[4]) {
  T v[8];
  Vec4<T>::ld(x + base, *reinterpret_cast<T(*)[4]>(&v[0]));
  // FP32: an aligned window needs one 16-byte load (247 vs 274 us at 4096^2); FP64 loads both
  // (measured faster with the two loads: 554 vs 643 us)
  if (sizeof(T) == 8 || mis != 0) {
    Vec4<T>::ld(x + base + 4, *reinterpret_cast<T(*)[4]>(&v[4]));
  } else {
#pragma unroll
    for (int e = 4; e < 8; ++e) v[e] = v[e - 4];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) o[e] = mis == 0 ? v[e] : mis == 1 ? v[e + 1] : mis == 2 ? v[e + 2] : v[e + 3];
}

// rows i0..i0+3, every window inside the vector (the caller checked the extreme offsets)
template <class T, int NMAT>
__device__ __forceinline__ void rows4_fast(const SweArg& a, long long i0, T (&t)[4]) {
#pragma unroll
  for (int m = 0; m < NMAT; ++m) {
    const T* x = static_cast<const T*>(a.x[m]);
    T b[4][4], xv[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long off = a.M[m].off[k];
      Vec4<T>::ld(static_cast<const T*>(a.M[m].band[k]) + i0, b[k]);
      window4<T>(x, i0 + (off & ~3LL), (int)(off & 3), xv[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) t[e] = fma(b[k][e], xv[k][e], t[e]);
  }
}

template <class T, int NMAT>
__global__ void __launch_bounds__(kThreads) k_band4(SweArg a) {
  const long long n = a.n;
  const long long stride = 4LL * gridDim.x * blockDim.x;
  for (long long i0 = 4LL * (blockIdx.x * (long long)blockDim.x + threadIdx.x); i0 < n; i0 += stride) {
    T t[4];
    if (i0 + 4 <= n) {
      if (a.u) Vec4<T>::ld(static_cast<const T*>(a.u) + i0, t);
      else t[0] = t[1] = t[2] = t[3] = T(0);
      if (i0 + a.lo >= 0 && i0 + a.hi <= n) {
        rows4_fast<T, NMAT>(a, i0, t);
      } else {
#pragma unroll
        for (int m = 0; m < NMAT; ++m) {
          const T* x = static_cast<const T*>(a.x[m]);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            T b[4];
            Vec4<T>::ld(static_cast<const T*>(a.M[m].band[k]) + i0, b);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const long long j = i0 + a.M[m].off[k] + e;
              if (j >= 0 && j < n) t[e] = fma(b[e], __ldg(x + j), t[e]);
            }
          }
        }
      }
      if (a.s) {
        T sv[4];
        Vec4<T>::ld(static_cast<const T*>(a.s) + i0, sv);
#pragma unroll
        for (int e = 0; e < 4; ++e) t[e] = t[e] + sv[e];
      }
      Vec4<T>::st(static_cast<T*>(a.out) + i0, t);
    } else {
      for (long long i = i0; i < n; ++i) {          // the last, partial group of rows
        T r = a.u ? __ldg(static_cast<const T*>(a.u) + i) : T(0);
        for (int m = 0; m < NMAT; ++m) {
          const T* x = static_cast<const T*>(a.x[m]);
          for (int k = 0; k < 4; ++k) {
            const long long j = i + a.M[m].off[k];
            if (j >= 0 && j < n) r = fma(__ldg(static_cast<const T*>(a.M[m].band[k]) + i), __ldg(x + j), r);
          }
        }
        if (a.s) r = r + __ldg(static_cast<const T*>(a.s) + i);
        static_cast<T*>(a.out)[i] = r;
      }
    }
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

hn_status launch(hn_dtype type, SweArg a, cudaStream_t s) {
  if (a.n == 0) return HN_OK;
  // the aligned 8-element span of a window starts at i0 + (off & ~3)
  a.lo = LLONG_MAX;
  a.hi = LLONG_MIN;
  for (int m = 0; m < a.nmat; ++m)
    for (int k = 0; k < 4; ++k) {
      const long long base = a.M[m].off[k] & ~3LL;
      a.lo = std::min(a.lo, base);
      a.hi = std::max(a.hi, base + 8);
    }
  void (*kern)(SweArg) = type == HN_F32 ? (a.nmat == 1 ? k_band4<float, 1> : k_band4<float, 4>)
                                         : (a.nmat == 1 ? k_band4<double, 1> : k_band4<double, 4>);
  // one wave of resident blocks (grid-stride loop); the occupancy of each kernel is asked once
  static int occ[2][2] = {{0, 0}, {0, 0}};
  int& per_sm = occ[type == HN_F32 ? 0 : 1][a.nmat == 1 ? 0 : 1];
  if (per_sm == 0) HN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
  const long long groups = (a.n + 3) / 4;
  const long long cap = (long long)sm_count() * std::max(per_sm, 1);
  const int grid = (int)std::max<long long>(1, std::min((groups + kThreads - 1) / kThreads, cap));
  kern<<<grid, kThreads, 0, s>>>(a);
  HN_CUDA(cudaGetLastError());
  return HN_OK;
}

hn_status take_matrix(const hn_band4* M, Band4Arg* out) {
  if (!M) return set_error(HN_ERR_ARG, "null matrix");
  for (int k = 0; k < 4; ++k) {
    if (!M->band[k] || !aligned16(M->band[k])) return set_error(HN_ERR_ARG, "band %d null or not 16-byte aligned", k);
    out->off[k] = M->offset[k];
    out->band[k] = M->band[k];
  }
  return HN_OK;
}

hn_status check_vec(const void* p, const char* what) {
  if (!p || !aligned16(p)) return set_error(HN_ERR_ARG, "%s null or not 16-byte aligned", what);
  return HN_OK;
}

}  // namespace
}  // namespace hn

using namespace hn;

extern "C" hn_status hn_band4_spmv(hn_dtype type, long long n, const hn_band4* M, const void* x,
                                   void* y, void* stream) {
  clear_error();
  if (type != HN_F32 && type != HN_F64) return set_error(HN_ERR_ARG, "unknown type %d", (int)type);
  if (n < 0) return set_error(HN_ERR_ARG, "negative length");
  if (n == 0) return HN_OK;
  SweArg a{};
  HN_TRY(take_matrix(M, &a.M[0]));
  HN_TRY(check_vec(x, "x"));
  HN_TRY(check_vec(y, "y"));
  a.x[0] = x;
  a.out = y;
  a.n = n;
  a.nmat = 1;
  return launch(type, a, static_cast<cudaStream_t>(stream));
}

extern "C" hn_status hn_swe_predict(hn_dtype type, long long n, const hn_band4* M, const void* u,
                                    const void* v, const void* w, const void* s, void* u_new,
                                    void* stream) {
  clear_error();
  if (type != HN_F32 && type != HN_F64) return set_error(HN_ERR_ARG, "unknown type %d", (int)type);
  if (n < 0) return set_error(HN_ERR_ARG, "negative length");
  if (n == 0) return HN_OK;
  if (!M) return set_error(HN_ERR_ARG, "null matrices");
  SweArg a{};
  for (int m = 0; m < 4; ++m) HN_TRY(take_matrix(M + m, &a.M[m]));
  HN_TRY(check_vec(u, "u"));
  HN_TRY(check_vec(v, "v"));
  HN_TRY(check_vec(w, "w"));
  HN_TRY(check_vec(u_new, "u_new"));
  if (s) HN_TRY(check_vec(s, "s"));
  a.x[0] = v;
  a.x[1] = w;
  a.x[2] = u;
  a.x[3] = u;
  a.u = u;
  a.s = s;
  a.out = u_new;
  a.n = n;
  a.nmat = 4;
  return launch(type, a, static_cast<cudaStream_t>(stream));
}
