/*
 * afr_debug.h -- test hooks of the debug build of the reconstruction library
 * (libafr_debug.so, compiled with AFR_DEBUG). That build also bounds-checks
 * record, slot and bucket indices on the device: a failed check records
 * AFR_ERR_DEVICE_CHECK in the context's status word (afr_get_status) and the
 * guarded access is skipped, never performed. The release library
 * (libafr.so) has neither the checks nor these calls. The paper has no
 * counterpart.
 */
#ifndef AFR_DEBUG_H
#define AFR_DEBUG_H

#include "afr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Allocation-failure injection: device allocation number `after` (counted
 * from this call, 0-based) and every later one fail as if the device were
 * out of memory, so callers see AFR_ERR_OOM; a negative value switches the
 * injection off. Process-wide, not thread-safe. */
AFR_API void afr_debug_fail_alloc(int32_t after);

/* Overwrites the frame view's bin offsets with off_host (width*height+1
 * uint32, host memory), to feed the filter an inconsistent frame view in
 * tests of the device checks. Offsets must not decrease. Synchronises. */
AFR_API AfrStatus afr_debug_set_frame_offsets(AfrContext *ctx, const uint32_t *off_host);

#ifdef __cplusplus
}
#endif
#endif
