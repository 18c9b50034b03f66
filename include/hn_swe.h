/* hn_swe.h -- banded matrices with four bands at arbitrary positions, and the fused prediction
 * step of the explicit shallow-water solver.
 *
 * HONEI's banded matrices keep their bands at fixed or at arbitrary positions (Sec. 4.1).  Its
 * shallow-water client writes the prediction step of its relaxation scheme as a linear combination
 * of products with four-band matrices (Sec. 2.2):
 *     u_new = u + M1 v + M2 w + M3 u + M4 u + S(u)
 * The scheme that defines the matrices, the temporaries v, w and the source term S is external to
 * the paper (Sec. 2.2 cites it and leaves it out), so these calls take them as inputs: they are the
 * linear-algebra kernel of the step, as one fused pass over memory (the paper's Sec. 7 notes that
 * composing such a step from generic library calls loses performance).
 *
 * Conventions:
 *  - An hn_band4 describes an n x n matrix: band k (k = 0..3) is a device array of n elements with
 *    M[i, i + offset[k]] = band[k][i]; an entry whose column i + offset[k] is outside 0..n-1 does
 *    not exist (its band value is ignored).  Offsets may repeat and may be 0 or beyond +-n.
 *  - Vectors and bands are DEVICE pointers of the call's element type, 16-byte aligned (as
 *    cudaMalloc returns them); n >= 0 (n = 0 does nothing).  u_new / y must not overlap any input.
 *  - Rounding order (part of the definition, so results are bit-reproducible): a running sum per
 *    row, updated by one fused multiply-add per existing entry, bands k = 0..3 in order; for the
 *    prediction step the sum starts at u_i and takes M1 (with v), M2 (w), M3 (u), M4 (u) in order,
 *    then adds s_i once (s may be NULL: no source term).
 *  - stream: a cudaStream_t or NULL; the calls return without waiting.
 *  - Errors: HN_ERR_ARG for n < 0, an unknown type, a null or misaligned pointer; HN_ERR_CUDA if
 *    the launch fails.
 */
#ifndef HN_SWE_H
#define HN_SWE_H

#include "hn_blas1.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  long long offset[4];
  const void* band[4];
} hn_band4;

/* y = M x for one four-band matrix (Sec. 4.1 banded matrix-vector product, arbitrary positions). */
hn_status hn_band4_spmv(hn_dtype type, long long n, const hn_band4* M, const void* x, void* y,
                        void* stream);

/* u_new = u + M[0] v + M[1] w + M[2] u + M[3] u + s in one pass (Sec. 2.2 prediction step).
 * M: 4 matrices. */
hn_status hn_swe_predict(hn_dtype type, long long n, const hn_band4* M, const void* u,
                         const void* v, const void* w, const void* s, void* u_new, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HN_SWE_H */
