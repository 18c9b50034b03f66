/* hn_profile.h -- per-kernel timing of the hn solver (measurement support, not part of the
 * method).  With profiling on, a hierarchy's solves run the V-cycle schedule one iteration per
 * graph launch with a CUDA event recorded on the solve stream before and after every kernel
 * launch; elapsed times accumulate per kernel class and level.  Profiling adds a host
 * synchronisation per iteration and the event nodes, so headline timings are taken with it off.
 */
#ifndef HN_PROFILE_H
#define HN_PROFILE_H

#include "hn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  char name[24];          /* kernel class: jacobi, jacobi_first, defect, restrict, prolong,
                             prolong_jacobi, coarse, check, outer_defect, update, control, tail,
                             pcg_q, pcg_x, pcg_dot, pcg_p */
  int level;              /* refinement level the launches worked on (-1: per-problem finest) */
  long long launches;     /* launches timed */
  double total_ms;        /* summed event-to-event time */
  double bytes_per_launch;/* algorithmic DRAM bytes of one launch (unit counts x bytes per node of
                             the kernel and precision; 0 for control kernels) */
} hn_kernel_time;

/* Turn per-kernel event timing on (1) or off (0) for later solves of mg; clears the totals. */
hn_status hn_mg_set_profiling(hn_mg* mg, int enable);

/* Copy up to max accumulated entries (classes x levels with launches > 0); returns the count. */
int hn_mg_kernel_times(const hn_mg* mg, hn_kernel_time* out, int max);

/* Time one kernel of the solver on its own: `reps` back-to-back launches of op (HN_OP_SPMV,
 * HN_OP_DEFECT, HN_OP_JACOBI, HN_OP_RESTRICT, HN_OP_PROLONG_ADD or HN_OP_PROLONG_JACOBI) on
 * `level` of mg's hierarchy (the inner hierarchy of a DC hierarchy), on whatever the level's
 * vectors hold, timed with CUDA events on mg's stream after one warm-up launch.  *avg_ms receives the mean launch time, *bytes the algorithmic DRAM bytes of
 * one launch (N_l x bytes per node of the kernel and precision). */
hn_status hn_mg_time_kernel(hn_mg* mg, int op, int level, int reps, double* avg_ms, double* bytes);

/* Arithmetic rates of the current device, measured by kernels that keep the pipe busy with
 * independent chains of one operation (operations per second; an FMA counts as one operation).
 * The FP64 band and transfer kernels are bounded by min(HBM bandwidth / bytes per node, FP64
 * rate / FP64 operations per node) on a part whose FP64 rate is low.  Allocates a small device
 * buffer and a stream for the duration of the call; takes a few milliseconds. */
typedef struct {
  double fp64_fma_per_s, fp64_add_per_s, fp64_mul_per_s, fp32_fma_per_s;
} hn_fp_rates;
hn_status hn_measure_fp_rates(hn_fp_rates* out);

/* Kernel launches of mg's last single solve (hn_mg_solve): the graph's init kernels plus the
 * kernels of every loop iteration that ran.  0 before the first solve. */
long long hn_mg_last_launches(const hn_mg* mg);

#ifdef __cplusplus
}
#endif
#endif /* HN_PROFILE_H */
