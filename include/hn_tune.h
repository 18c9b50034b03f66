/* hn_tune.h -- launch-shape tuning of the hn solver (performance only; results do not change).
 *
 * The V-cycle schedule runs levels coarse_L..tail_level of every problem inside one fused launch
 * of one thread-block cluster (`cluster` blocks of 512 threads) per problem, levels
 * tail_level+1..mid in two persistent cooperative launches per cycle (one down, one up; their
 * steps separated by grid-wide barriers), and levels above mid as one launch per step over the
 * device work list, or (sweep) as one launch per level and direction over 2-D tiles.  Inside that launch the
 * smallest levels live in the shared memory of the cluster's first block; the levels between
 * them and tail_level either live in the distributed shared memory of the whole cluster (`dsm`,
 * when they fit) or are read through L2.  The best split depends on the levels and the batch;
 * hn_mg_autotune measures candidates on the hierarchy itself.
 */
#ifndef HN_TUNE_H
#define HN_TUNE_H

#include "hn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int tail_level;   /* levels <= tail_level run fused (coarse_L .. HN_MAX_LEVEL) */
  int cluster;      /* blocks per cluster of the fused launch: 1, 2, 4, 8 or 16 */
  int pdl;          /* programmatic dependent launch (a kernel launches while its predecessor
                       runs and waits for its results): 0 off, 1 every kernel, 2 kernels of
                       fewer blocks than SMs only, 3 fewer blocks than twice the SMs */
  int staged;       /* 1: the band kernels of large FP32 / FP16 levels stream the bands through
                       shared memory with bulk copies (TMA engine) on mbarriers; 0: register path */
  int dsm;          /* 1: the fused launch keeps its cluster levels in distributed shared memory
                       when they fit (else, and with 0, they run through L2) */
  int fuse_up;      /* 1: on the levels above tail_level the prolongation runs inside the first
                       post-smoothing step (one pass instead of two, each lane forming the
                       prolonged values of its three stencil rows); 0: separate kernels (default:
                       the fused pass measured slower, its extra work outweighing the pass saved) */
  int mid;          /* levels tail_level+1 .. mid run in the persistent kernels (0, or any value
                       <= tail_level: none); not combined with staged or fuse_up, which are forms
                       of the per-step launches (default 0: on this part a grid barrier plus the
                       memory latency of a step costs as much as a kernel boundary) */
  int sweep;        /* 1 (default): a hierarchy solved alone with V(2,2) cycles runs the down
                       part of each level between tail_level and the finest, up to level 9 (both
                       pre-smoothing steps, the defect and the restriction), and the up part (the
                       prolongation and both post-smoothing steps) as one launch each, over 2-D
                       tiles whose blocks recompute the halos they need instead of waiting for one
                       another; 2: every level above tail_level and, on the finest level, the steps
                       after the first smoothing step (the second step, the defect, the
                       restriction) in one launch; 0: one launch per step.  Not combined with
                       staged or mid; without effect in batches and in the server */
} hn_tuning;

/* Set / read the launch shape used by mg's later solves.  HN_ERR_ARG on values out of range. */
hn_status hn_mg_set_tuning(hn_mg* mg, const hn_tuning* t);
hn_status hn_mg_get_tuning(const hn_mg* mg, hn_tuning* t);

/* Time `reps` solves of b (host vector, N doubles) for every candidate shape (three forms of the
 * levels above the tail: one launch per step (mid 0, sweep 0), persistent kernels (mid 10), fused
 * sweeps (sweep 1); tail_level from coarse_L to min(L, 9); cluster 1..16) and keep the fastest; the
 * candidate timings are returned in `times_ms` (may be NULL, capacity `cap` entries, row-major
 * 3 forms x tail_level x 5 cluster sizes) and the chosen shape in *best.  The solution is unchanged
 * by the shape. */
hn_status hn_mg_autotune(hn_mg* mg, const double* b, int reps, hn_tuning* best, double* times_ms,
                         int cap);

/* The same for a batch (hn_mg_solve_batch over mgs[0..count)): candidates mid 0 and 10,
 * tail_level coarse_L..8, cluster 1, 2, 4; the fastest shape is stored in every member and used by
 * later batch solves of the same members (a batch whose members carry no common tuned shape picks
 * one by its size). */
hn_status hn_mg_autotune_batch(hn_mg* const* mgs, int count, const double* const* b, int reps,
                               hn_tuning* best);

/* Persisted launch shapes (the runtime configuration file of Sec. 3: choices measured on this
 * machine, kept in a file that later runs read).  When the environment variable HN_TUNE_CACHE
 * names a file, hn_mg_autotune stores its result there under the key (GPU name, level, precision,
 * solver, coarse solver, coarse level), and hn_mg_setup applies the stored shape of its key to the
 * new hierarchy (as hn_mg_set_tuning would).  The file is text, one entry per line:
 *     <gpu name>|<L>|<prec>|<solver>|<coarse solver>|<coarse L> <tail_level> <cluster> <pdl> <staged> <dsm> <fuse_up> <mid> <sweep>
 * (an entry without the last field has sweep 0).  A store replaces the entry of its key (the file is rewritten through a temporary file and a
 * rename); lines that do not parse, or hold values out of range, are ignored by lookups.
 *
 * The two calls below are the file operations themselves (host only, no device call):
 * hn_tune_cache_lookup fills *out with the entry of the key and returns HN_OK, or returns
 * HN_ERR_STATE when the file is missing or has no valid entry for the key; hn_tune_cache_store
 * returns HN_ERR_ARG for a shape out of range and HN_ERR_STATE when the file cannot be written.
 * prec, solver, coarse_solver take the values of hn_precision, hn_solver, hn_coarse_solver. */
hn_status hn_tune_cache_lookup(const char* path, const char* gpu, int L, int prec, int solver,
                               int coarse_solver, int coarse_L, hn_tuning* out);
hn_status hn_tune_cache_store(const char* path, const char* gpu, int L, int prec, int solver,
                              int coarse_solver, int coarse_L, const hn_tuning* t);

#ifdef __cplusplus
}
#endif
#endif /* HN_TUNE_H */
