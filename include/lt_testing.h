/* Fault injection for tests (no counterpart in the paper).
 *
 * These entry points exist only in the test build of the library
 * (_lib/liblt_testhooks.so, compiled with -DLT_TEST_HOOKS); the product
 * library _lib/liblt.so exports neither and carries none of their checks.
 * Faults are made on the host or by withholding work: nothing here faults,
 * traps or hangs a GPU.
 *
 *   lt_test_fail_allocation_after  the n-th device allocation the library
 *       makes from now on fails as if the device were out of memory (n >= 1);
 *       n <= 0 turns the injection off.  The failing call returns LT_ENOMEM
 *       through its normal error path and frees what it had allocated.
 *   lt_nn_test_stall_tensor_core   with on != 0 the tcgen05 convolution
 *       kernels issue no tensor-core work, so their bounded mbarrier waits
 *       (shortened to 4096 polls) run out; each CTA then records LT_ETIMEOUT
 *       for lt_nn_device_status and writes no output.  Nothing is left in
 *       flight.  on == 0 restores normal operation.  Synchronises the stream.
 */
#ifndef LT_TESTING_H
#define LT_TESTING_H

#include "lt.h"

#ifdef __cplusplus
extern "C" {
#endif

LT_API void lt_test_fail_allocation_after(int32_t n);
LT_API lt_status lt_nn_test_stall_tensor_core(int32_t on, void* stream);

#ifdef __cplusplus
}
#endif

#endif
