/*
 * libtp failure-injection hook: for tests of the bounded device waits only.
 *
 * The tcgen05 apply (k = 3 with FP16/BF16 vectors on the tensor kernel) bounds
 * every wait on its pipeline barriers; a wait that runs out records a code in
 * the operator's device status word, the other roles stop at their next wait,
 * copies and products already issued are drained, TMEM is released, and the
 * launch returns normally, leaving the context usable (tp_op_check then
 * returns TP_ERR_TIMEOUT). This hook lets a test make such a wait run out
 * without any fault: it shortens the limit and has CTA 0 skip the copy of its
 * first input tile, so the barrier of that slot never completes. Not for
 * production use; the paper has no counterpart.
 */
#ifndef TP_TEST_H
#define TP_TEST_H

#include "tp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* For the tcgen05 apply of `op`, from the next launch on: wait_limit_s > 0
 * replaces the one-second limit of every bounded barrier wait (0 restores it);
 * withhold_first_copy = 1 makes CTA 0 skip the TMA copy of its first input
 * tile (0 restores normal operation). Host-side only: changes the parameters
 * of later launches, touches no device memory. Errors: TP_ERR_INVALID_ARG
 * (NULL op, negative or non-finite limit), TP_ERR_UNSUPPORTED (the operator
 * does not run the tcgen05 apply). */
tp_status tp_test_set_wait_fault(tp_op op, int withhold_first_copy, double wait_limit_s);

#ifdef __cplusplus
}
#endif

#endif /* TP_TEST_H */
