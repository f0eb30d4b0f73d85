/*
 * sense_testing.h -- test hooks of libsense.so's request queue.  Not for
 * production use: these exist so that the queue's scheduler (admission,
 * ordering, refusal, cancellation, failure handling) can be tested on a host
 * without a GPU, and so that a device allocation failure can be injected
 * without exhausting device memory.  The paper has no counterpart.
 */
#ifndef SENSE_TESTING_H
#define SENSE_TESTING_H

#include "sense.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int fake_device;      /* 1: no GPU work at all -- each tick sleeps fake_tick_us and every frame
                           "converges" after min(max_iter, fake_iters) ticks */
  int fake_tick_us;
  int fake_iters;
  int fail_admit_every; /* 0 = off: every k-th admission fails as if a device allocation had failed
                           (after the others succeeded); the request ends FAILED and sense_queue_wait
                           returns SENSE_ENOMEM.  Negative values are rejected with SENSE_EINVAL. */
} sense_queue_test_hooks;

/* sense_queue_create with test hooks (hooks may be NULL: none). */
sense_status sense_queue_create_with_hooks(int device, const sense_queue_cfg* cfg, const sense_queue_test_hooks* hooks,
                                           sense_queue** out);

#ifdef __cplusplus
}
#endif

#endif /* SENSE_TESTING_H */
