// xy_debug.h -- device-side index checks of the library's debug build.
//
// Built with -DXY_DEBUG (paper_0811_2111_gb300/build.py: build(debug=True),
// libxy_debug.so), a kernel guards its index arithmetic with
//     if (XY_DCHECK(index_in_range, bit)) access;
// A failed check sets `bit` of this translation unit's debug word and skips
// the access: it never traps, so a faulty index shows up as a word the host
// reads (xy_debug_checks) instead of as a fault of the GPU.  In the release
// build XY_DCHECK is the constant true and the checks compile away.
#pragma once

#include <cuda_runtime.h>

#ifdef XY_DEBUG
namespace {
__device__ unsigned int g_xy_debug_word;   // one per translation unit
}  // namespace
#define XY_DCHECK(cond, bit) ((cond) ? true : (atomicOr(&g_xy_debug_word, 1u << (bit)), false))

namespace {
// This translation unit's word, read and cleared (synchronizes the device).
inline unsigned int xy_debug_take_word() {
  unsigned int v = 0, zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return 0xffffffffu;
  if (cudaMemcpyFromSymbol(&v, g_xy_debug_word, sizeof(v)) != cudaSuccess) return 0xffffffffu;
  if (cudaMemcpyToSymbol(g_xy_debug_word, &zero, sizeof(zero)) != cudaSuccess) return 0xffffffffu;
  return v;
}
}  // namespace
#else
#define XY_DCHECK(cond, bit) true
namespace {
inline unsigned int xy_debug_take_word() { return 0u; }
}  // namespace
#endif
