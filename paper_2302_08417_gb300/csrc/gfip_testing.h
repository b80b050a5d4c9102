// gfip_testing.h -- test-only entry points of libgemmfip.so.  Not part of the public ABI
// (include/gemmfip.h): nothing in the library's normal use calls them, and the only caller is
// the failure-path test of the tensor-core FP64 emulation.
#pragma once

#include <stdint.h>

#include "../../include/gemmfip.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Test hook for the failure path of gfip_dgemm_ozaki (no counterpart in the paper; the
 * paper's CPU kernels have no waits).  Sets, for this handle's later gfip_dgemm_ozaki calls,
 * the budget of every pipeline wait in nanoseconds (0 restores the default, 2 s), and with
 * enable != 0 makes the first CTA withhold its first operand copy, so that its wait runs out:
 * the call then raises GFIP_STATUS_MMA_TIMEOUT, leaves that CTA's 128 x 128 tile of C
 * unwritten (every other tile is computed), waits for its own copies in flight, releases its
 * tensor memory and returns; the context stays usable.  Nothing else is affected.
 * Returns GFIP_ERR_HANDLE for an invalid handle. */
int gfip_debug_ozaki_timeout(gfip_handle_t handle, int enable, uint64_t wait_ns);

#ifdef __cplusplus
}
#endif
