// xy_device.cuh -- device-side building blocks of the XY Metropolis kernels:
// the Philox4x32-10 counter generator, the 24-bit uniforms, the precision
// switch between CUDA's accurate and fast intrinsics, and warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace xyd {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): two 32x32->64 products per round, the high halves
// xored into the other lanes with the round key, the key advanced by a Weyl
// sequence.  Counter x = (site, sweep, lattice_id, domain); key = seed words.
constexpr uint32_t kMulA = 0xD2511F53u;
constexpr uint32_t kMulB = 0xCD9E8D57u;
constexpr uint32_t kWeylA = 0x9E3779B9u;
constexpr uint32_t kWeylB = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi_a = __umulhi(kMulA, x.x);
    const uint32_t lo_a = kMulA * x.x;
    const uint32_t hi_b = __umulhi(kMulB, x.z);
    const uint32_t lo_b = kMulB * x.z;
    x = make_uint4(hi_b ^ x.y ^ k0, lo_b, hi_a ^ x.w ^ k1, lo_a);
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return x;
}

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kU24 = 1.0f / 16777216.0f;   // 2^-24
constexpr float kR23 = 1.0f / 8388608.0f;    // 2^-23
// 2 pi / 2^24, rounded once: hot-start angle = (w0 >> 8) * kHotScale.
constexpr float kHotScale = (float)(6.283185307179586476925 / 16777216.0);

// Exact 24-bit uniform in [0, 1).
__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * kU24; }

// 2 u24(w) - 1 = ((w >> 8) - 2^23) / 2^23, exact in FP32, in [-1, 1).
__device__ __forceinline__ float sym24(uint32_t w) {
  return (float)((int32_t)(w >> 8) - 8388608) * kR23;
}

// Precision switch: MODE 0 = CUDA's accurate sincosf/expf, MODE 1 = the
// SFU intrinsics __sincosf/__expf.
template <int MODE>
__device__ __forceinline__ void sincos_m(float t, float* s, float* c) {
  if (MODE == 0) {
    sincosf(t, s, c);
  } else {
    __sincosf(t, s, c);
  }
}

template <int MODE>
__device__ __forceinline__ float exp_m(float x) {
  if (MODE == 0) return expf(x);
  return __expf(x);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Neumaier-compensated accumulation (sum, correction) in FP32.
__device__ __forceinline__ void neumaier_add(float& sum, float& comp, float v) {
  const float t = sum + v;
  if (fabsf(sum) >= fabsf(v)) {
    comp += (sum - t) + v;
  } else {
    comp += (v - t) + sum;
  }
  sum = t;
}

// Wrap an index into [0, n) when it is at most a few periods away.
__device__ __forceinline__ int wrap_index(int v, int n) {
  while (v < 0) v += n;
  while (v >= n) v -= n;
  return v;
}

}  // namespace xyd
