/*
 * fdk_testing.h -- testing hooks of libfdk.  The paper has no counterpart:
 * these exist so that tests can drive the library's failure paths without
 * faulting a GPU or exhausting its memory.  Not for production use; both
 * settings are process-wide and apply to every thread and device.
 */
#ifndef FDK_TESTING_H
#define FDK_TESTING_H

#include "fdk.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * fdk_testing_set_wait_limit -- how many times the consumer waits of later
 * launches poll their mbarrier before they give up: the wait for a staged
 * view in the FDK_FETCH_STAGE back-projection and the wait for a staged row
 * pair in fdk_preweight_filter.  polls = 0 makes every such wait give up
 * without polling, so the CTA takes its error path on its first staged view
 * or row pair: it records the timeout for fdk_device_status(), waits (with
 * the full built-in limit) for the copies it has in flight, and returns with
 * its tile or rows unwritten.  polls < 0 restores the built-in limit (2^22
 * polls).  The value is read when a call enqueues its kernels, so it does
 * not affect work already enqueued.  Always FDK_OK.
 */
FDK_API fdk_status fdk_testing_set_wait_limit(int64_t polls);

/*
 * fdk_testing_fail_allocations -- make the library's next n device
 * allocations fail as they would on a device out of memory (each failing
 * allocation is counted once; 0 cancels what is left).  The entry points
 * then return their out-of-memory status (FDK_ERR_OOM, or FDK_ERR_CUDA where
 * the failing call is documented as a CUDA error) and leave their caches
 * empty, so a later call allocates again.  n < 0: FDK_ERR_INVALID_ARG.
 */
FDK_API fdk_status fdk_testing_fail_allocations(int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* FDK_TESTING_H */
