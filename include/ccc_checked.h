/* Test hook of the bounds-checking build of the library.
 *
 * The library built with -DCCC_BOUNDS_CHECK (paper_1705_08213_gb300/build.py
 * checked=True: _build_checked/libccc_checked.so) tests on the device every
 * output index of the tally kernels (pair and triple indices, phase offsets,
 * K-split partial reductions, s-state rows), the 2-way table reads of the
 * 3-way genotype-class route and the shared-memory stores of the code
 * expansion (ccc_opts.tile = 3).  An index outside its buffer records
 * CCC_EBOUNDS in the status word (ccc_status) and the access is skipped.  The
 * normal build has no checks; there this header's call returns
 * CCC_EUNSUPPORTED.
 */
#ifndef CCC_CHECKED_H
#define CCC_CHECKED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* From the next call on, every tally launch is told that its output arrays
 * hold n fewer entries (pairs or triples) than they do, so the stores of the
 * last n entries must be caught: the call records CCC_EBOUNDS and leaves
 * those entries untouched, while every real access stays inside the arrays.
 * n = 0 restores the true lengths.  Returns CCC_OK, CCC_EINVAL for n < 0, or
 * CCC_EUNSUPPORTED from the normal build.
 * Host state of the process, not thread-safe against concurrent calls. */
int ccc_checked_shrink_outputs(int64_t n);

#ifdef __cplusplus
}
#endif

#endif /* CCC_CHECKED_H */
