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

/* The frame-staggered item order that the persistent CG kernel (units =
   frame-iterations k*frames + f; first phase = normal-product tiles, second =
   update chunks) and the single-launch operators (units = frames) hand out:
   ticket t -> out[0] = 1 for a second-phase item, out[1] = unit, out[2] =
   piece.  Stage s holds the first-phase items of unit s, then the
   second-phase items of unit s - lag.  Host only; needs no GPU. */
void sense_testing_staggered_item(long long t, int units, int first_items, int second_items, int lag, int out[3]);
/* The stagger the persistent CG kernel uses for a table of independent
   frames: frames, tiles per frame, grid blocks -> lag (0 .. frames - 1). */
int sense_testing_persistent_lag(int frames, int tiles, int grid);
/* Pins the item order of a plan's persistent CG launches: -1 iteration-major,
   -2 automatic (the default), D >= 0 the frame-staggered order with lag D
   (D < frames, else the solve fails with SENSE_ECUDA).  Frames coupled in
   time always run iteration-major.  The order changes no arithmetic, so
   every order gives the same bits; tests use this to check that. */
sense_status sense_testing_plan_set_order(sense_plan* plan, int order);

#ifdef __cplusplus
}
#endif

#endif /* SENSE_TESTING_H */
