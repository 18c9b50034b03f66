/* hn_blas1.h -- BLAS level-1 kernels on device vectors.
 *
 * The paper measures the axpy kernel y = a x + y on every backend it supports and notes that the
 * other level-1 operations behave alike (Sec. 6.1, Fig. 2): they are purely memory bound, so
 * their rate is set by the off-chip bandwidth once the vectors are long, and by the launch
 * overhead below that.  These entry points are those operations on one GB300.
 *
 * Conventions:
 *  - x, y, result are DEVICE pointers (cudaMalloc or equivalent).  Vectors of n elements of the
 *    given type; n = 0 is valid (axpy does nothing, dot and nrm2 write 0).  Any alignment of the
 *    element type works; 16-byte aligned vectors use 16-byte loads.
 *  - stream: a cudaStream_t, or NULL for the legacy default stream.  The calls are asynchronous:
 *    the result is complete when the stream reaches that point.
 *  - dot and nrm2 sum in a fixed order that depends only on n, so repeated calls give identical
 *    bits: each 16,384-element chunk is split over 256 threads; thread t takes the element groups
 *    4t + 1024 j .. +3 (FP32; FP64: 2t + 512 j, +1) and group j goes to chain j mod 4 (at most 16
 *    products per chain), the chains are added in FP64, then the threads in a fixed tree, then
 *    the chunks in order.  Chains of FP64 vectors are FP64; chains of FP32 vectors are FP32 fused
 *    multiply-adds (relative error of a chain <= 16 units of 2^-24), because FP64 arithmetic on
 *    this part is too slow to keep up with the memory.
 *    nrm2 does not rescale: squares must stay finite in the element type.
 *  - Errors: HN_ERR_ARG for a negative n, a null pointer with n > 0 or an unknown type;
 *    HN_ERR_CUDA / HN_ERR_OOM if a launch or the stream-ordered scratch allocation fails.
 */
#ifndef HN_BLAS1_H
#define HN_BLAS1_H

#include "hn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { HN_F32 = 0, HN_F64 = 1 } hn_dtype;

/* y[i] = alpha * x[i] + y[i], one rounding per element (fused multiply-add in the element type;
 * for HN_F32 alpha is first rounded to float). */
hn_status hn_axpy(hn_dtype type, long long n, double alpha, const void* x, void* y, void* stream);

/* *result = sum_i x[i] * y[i] in the order above (result: one double on the device). */
hn_status hn_dot(hn_dtype type, long long n, const void* x, const void* y, double* result, void* stream);

/* *result = sqrt(sum_i x[i]^2), the sum as for dot, the root in FP64 (one double on the device). */
hn_status hn_nrm2(hn_dtype type, long long n, const void* x, double* result, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HN_BLAS1_H */
