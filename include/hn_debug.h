/* hn_debug.h -- the checked build of the hn library (development support, not part of the method).
 *
 * build.py builds the library twice: libhn.so and libhn_debug.so, the same sources compiled with
 * HN_DEBUG_CHECKS=1.  In the checked build
 *  - every kernel checks each work-list item (problem slot, level, tile) and each one-problem level
 *    descriptor against the hierarchy's layout before it touches memory; a failed check records the
 *    source line and the indices in the engine's error words, skips the access (it never traps) and
 *    the solve returns HN_ERR_STATE with the line in hn_last_error();
 *  - every device block the library allocates for an operator, a hierarchy or an engine carries
 *    4 KiB of a fixed byte pattern before and after it, which the calls below verify.
 * The checked build stands in for a memory checker: it runs the small-level tests and verifies the
 * guards when their hierarchies are destroyed.  In the release library these calls return
 * HN_ERR_STATE (hn_debug_build returns 0).
 */
#ifndef HN_DEBUG_H
#define HN_DEBUG_H

#include "hn.h"

#ifdef __cplusplus
extern "C" {
#endif

/* 1 in the checked build, 0 in the release build. */
int hn_debug_build(void);

/* Verify the guard bytes around the hierarchy's device block (if the library allocated it) and
 * around its one-problem engine's block; waits for the hierarchy's stream.  HN_OK if intact,
 * HN_ERR_STATE naming the block and the offset of the first overwritten byte otherwise. */
hn_status hn_debug_check_mg(const hn_mg* mg);

/* The same for an operator's device block. */
hn_status hn_debug_check_band(const hn_band* A);

/* Overwrite one guard byte after the hierarchy's block (a host-side cudaMemset inside the guard
 * allocation): lets a test see hn_debug_check_mg report a damaged guard.  HN_ERR_STATE in the
 * release build or for a block the caller supplied. */
hn_status hn_debug_overwrite_guard(hn_mg* mg);

#ifdef __cplusplus
}
#endif
#endif /* HN_DEBUG_H */
