/* qmc_debug.h — test hook of the bounds-checked build of libqmcfft.
 *
 * Exported only by libraries compiled with -DQMC_CHECK_BOUNDS
 * (libqmcfft_checked.so, paper_1501_06286_gb300/build.py with checked=True);
 * the default library does not export it.  It lets a test plant an
 * out-of-range index in a plan's device tables and confirm that the
 * kernels' checks latch QMC_ERR_BOUNDS (qmc_plan_sync_status) instead of
 * reading or writing outside a buffer.  Nothing on the product path calls
 * it.
 */
#ifndef QMC_DEBUG_H
#define QMC_DEBUG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Overwrites entry `index` of one of the plan's int32 device tables with
 * `value` and returns the previous entry in *old (host).  Synchronous.
 *   which   QMC_TABLE_OUT_ROW (L entries: output row of each circulant row,
 *           read by the un-permute stores and the adjoint's loads of G) or
 *           QMC_TABLE_JLIST (s entries: rows of A by position, read by the
 *           generic and dense first passes and by the adjoint's stores of
 *           dA), as in qmc.h.
 * QMC_ERR_INVALID: null plan or old, another table; QMC_ERR_SHAPE: index
 * outside the table; QMC_ERR_CUDA: a failed copy. */
int qmc_debug_poke_table(void* plan, int32_t which, int64_t index, int32_t value, int32_t* old);

#ifdef __cplusplus
}
#endif

#endif /* QMC_DEBUG_H */
