// xy_alloc.cu -- the one device-allocation wrapper of the library, with a
// host-side failure hook for tests.
//
// Every cudaMalloc of the library's engines (contexts, batches, HMC, four
// replicas, record growth) goes through xyk::dev_malloc.  xy_debug_fail_alloc
// arms a countdown: the k-th allocation after the call fails with
// cudaErrorMemoryAllocation without reaching the driver, so the engines'
// out-of-memory paths (XY_ENOMEM, nothing leaked, the device still usable) can
// be exercised on a GPU without exhausting its memory.
#include <cuda_runtime.h>

#include <atomic>

#include "xy.h"
#include "xy_internal.h"

namespace {

// Allocations left before the armed failure (0: disarmed).
std::atomic<int> g_fail_countdown{0};

}  // namespace

namespace xyk {

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  int left = g_fail_countdown.load();
  while (left > 0) {
    if (g_fail_countdown.compare_exchange_weak(left, left - 1)) {
      if (left == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

}  // namespace xyk

extern "C" {

xy_status xy_debug_fail_alloc(int32_t k) {
  if (k < 0) return XY_EINVAL;
  g_fail_countdown.store(k);
  return XY_OK;
}

}  // extern "C"
