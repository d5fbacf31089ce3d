// xy_hmc_device.cuh -- per-site arithmetic of the Hybrid Monte Carlo kernels
// (Sec. 1.2): the drift wrap, the Gaussian momenta, the force, the exact
// fixed-point sums and the global accept test.  Every HMC kernel calls these
// and only these, with pinned rounding, so all of them agree bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "xy_internal.h"

namespace xyh {

using xyd::RoundKeys;
using xyk::HmcArgs;
using xyk::HmcCtl;
using xyk::kHmcSums;


// 2 pi split for the drift wrap: kTwoPiHi has 21 significant bits, so k * kTwoPiHi
// is exact for |k| < 8.
constexpr float kTwoPiHi = 4.0f * xyd::kPio2Hi;
constexpr float kTwoPiLo = 4.0f * xyd::kPio2Lo;
constexpr float kInvTwoPi = 0.159154943091895335769f;
constexpr float kKinFx = 8388608.0f;          // 2^23: (p^2 / 2) * 2^24 = p^2 * 2^23
constexpr float kFx30 = 1073741824.0f;        // 2^30

// Rounding is pinned with explicit intrinsics.

// theta + eps p wrapped into [0, 2 pi).
__device__ __forceinline__ float hmc_wrap(float t) {
  const float k = floorf(__fmul_rn(t, kInvTwoPi));
  float r = __fmaf_rn(-k, kTwoPiHi, t);
  r = __fmaf_rn(-k, kTwoPiLo, r);
  r = r < 0.f ? __fadd_rn(r, xyd::kTwoPi) : r;
  r = r >= xyd::kTwoPi ? __fsub_rn(r, xyd::kTwoPi) : r;
  return r;
}

// Box-Muller: u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1], u2 = (w1 >> 8) 2^-24,
// p = sqrt(-2 ln u1) cos(2 pi u2); CUDA's accurate logf, sqrtf and cospif.
__device__ __forceinline__ float hmc_gauss(uint32_t w0, uint32_t w1) {
  const float u1 = (float)((w0 >> 8) + 1u) * xyd::kU24;
  const float u2 = xyd::u24(w1);
  return __fmul_rn(sqrtf(__fmul_rn(-2.0f, logf(u1))), cospif(__fmul_rn(2.0f, u2)));
}

__device__ __forceinline__ float hmc_momentum(uint32_t site, uint32_t traj, uint32_t lattice_id,
                                              const RoundKeys& rk) {
  const uint4 w = xyd::philox4x32_10(make_uint4(site, traj, lattice_id, 3u), rk);
  return hmc_gauss(w.x, w.y);
}

// F = K (c Ss - s Sc) = -K sum_nn sin(t - t_j), (Sc, Ss) the neighbour unit-vector sum.
__device__ __forceinline__ float hmc_force(float c, float s, float Sc, float Ss, float K) {
  return __fmul_rn(K, __fmaf_rn(c, Ss, -__fmul_rn(s, Sc)));
}

// Fixed-point rounding with FP32 operations only (GB300 runs float -> int64
// conversions on its narrow FP64 pipe).  Adding 1.5 * 2^23 rounds any |x| <
// 2^22 to the nearest integer (ties to even), which the low bits of the sum
// then hold.  Larger values are split: x = h 2^21 + r with h the rounded
// quotient, r exact in FP32 (|r| <= 2^20), then r is rounded the same way, so
// h 2^21 + round(r) = round(x) exactly for |x| < 2^43.
constexpr float kRoundMagic = 12582912.0f;            // 1.5 * 2^23
constexpr int kRoundMagicBits = 0x4B400000;           // its bit pattern
constexpr float kTwo21 = 2097152.0f;

// round(v 2^21) for |v 2^21| < 2^22.
__device__ __forceinline__ int fx21(float v) {
  return __float_as_int(__fmaf_rn(v, kTwo21, kRoundMagic)) - kRoundMagicBits;
}

// round(v 2^S) = h 2^21 + l for |v 2^S| < 2^43; h and l are added to hs, ls.
template <int S>
__device__ __forceinline__ void fx_split(float v, int& hs, int& ls) {
  const float up = (float)(1ll << S);
  const float t = __fmaf_rn(v, up / kTwo21, kRoundMagic);
  const float hf = __fsub_rn(t, kRoundMagic);                          // exact
  const float r = __fmaf_rn(v, up, -__fmul_rn(hf, kTwo21));            // exact
  hs += __float_as_int(t) - kRoundMagicBits;
  ls += __float_as_int(__fadd_rn(r, kRoundMagic)) - kRoundMagicBits;
}

// Per-thread fixed-point accumulators (int32 partial sums of at most 16 sites).
struct HmcAcc {
  int kh, kl;           // K = p^2/2 at 2^-24: h 2^21 + l
  int ch, cl;           // C at 2^-30
  int ix, iy, mx, my;   // at 2^-21
};

__device__ __forceinline__ void acc_zero(HmcAcc& a) {
  a.kh = a.kl = a.ch = a.cl = a.ix = a.iy = a.mx = a.my = 0;
}

// Per-site terms of the sums, each rounded to fixed point before it is added:
// K: p^2/2; C: cos(t - t_r) + cos(t - t_u); Ix: sin(t - t_r); Iy: sin(t - t_u);
// Mx, My: c, s  (r = +x neighbour, u = +y neighbour).  The kinetic term is
// capped at 2^18 (|p| < 724), far beyond any momentum of a working chain.
__device__ __forceinline__ void hmc_terms(float p, float c, float s, float cr, float sr, float cu,
                                          float su, HmcAcc& acc) {
  const float cx = __fmaf_rn(c, cr, __fmul_rn(s, sr));
  const float cy = __fmaf_rn(c, cu, __fmul_rn(s, su));
  const float ix = __fmaf_rn(s, cr, -__fmul_rn(c, sr));
  const float iy = __fmaf_rn(s, cu, -__fmul_rn(c, su));
  const float kin = fminf(__fmul_rn(0.5f, __fmul_rn(p, p)), 262144.0f);
  fx_split<24>(kin, acc.kh, acc.kl);
  fx_split<30>(__fadd_rn(cx, cy), acc.ch, acc.cl);
  acc.ix += fx21(ix);
  acc.iy += fx21(iy);
  acc.mx += fx21(c);
  acc.my += fx21(s);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of the accumulators into dst[0..5] (K at 2^-24, the others at
// 2^-30; one 64-bit atomic each per CTA).  Called by every thread.
template <int NWARPS>
__device__ __forceinline__ void hmc_commit(const HmcAcc& a, unsigned long long* dst,
                                           long long (*sh)[kHmcSums]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long v[kHmcSums];
  v[0] = ((long long)a.kh << 21) + (long long)a.kl;
  v[1] = ((long long)a.ch << 21) + (long long)a.cl;
  v[2] = (long long)a.ix << 9;
  v[3] = (long long)a.iy << 9;
  v[4] = (long long)a.mx << 9;
  v[5] = (long long)a.my << 9;
#pragma unroll
  for (int j = 0; j < kHmcSums; ++j) v[j] = warp_sum_ll(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < kHmcSums; ++j) sh[warp][j] = v[j];
  }
  __syncthreads();
  if (threadIdx.x < kHmcSums) {
    long long t = 0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) t += sh[w][threadIdx.x];
    atomicAdd(dst + threadIdx.x, (unsigned long long)t);
  }
}

// Angle buffer i of the three (a select, not an indexed parameter load).
__device__ __forceinline__ float* hmc_buf(const HmcArgs& a, int i) {
  return i == 0 ? a.th[0] : (i == 1 ? a.th[1] : a.th[2]);
}

// Source and destination angle buffers of a launch, relative to the state
// buffer `cur`.
__device__ __forceinline__ void hmc_buffers(const HmcArgs& a, uint32_t cur, int* src, int* dst) {
  *src = (int)((cur + (uint32_t)a.src_off) % 3u);
  *dst = (int)((cur + (uint32_t)a.dst_off) % 3u);
}

// The test (mode 0: u < exp(-dH) with u = u24 of Philox counter (0, traj,
// lattice id, 4), writes a record and advances the counters) or the commit of
// a plain integration (mode 1).  dH is formed in FP64 from the exact integer
// sums.  Returns whether the end state is taken; also moves acc to last and
// clears acc.  One thread.
__device__ __forceinline__ bool hmc_decide(HmcCtl* c, uint32_t lattice_id, const RoundKeys& rk,
                                           int mode, double beta, double J) {
  const long long dK = (long long)(c->acc[1][0] - c->acc[0][0]);
  const long long dC = (long long)(c->acc[1][1] - c->acc[0][1]);
  const double dH = (double)dK * 0x1p-24 - beta * J * ((double)dC * 0x1p-30);
  bool take = true;
  if (mode == 0) {
    const uint4 w = xyd::philox4x32_10(make_uint4(0u, (uint32_t)c->traj, lattice_id, 4u), rk);
    take = (double)(w.x >> 8) * 0x1p-24 < exp(-dH);
    xy_hmc_record* r = c->records + c->rec;
    const int ph = take ? 1 : 0;
    for (int j = 0; j < 5; ++j) r->sum[j] = (int64_t)c->acc[ph][j + 1];
    r->kinetic[0] = (int64_t)c->acc[0][0];
    r->kinetic[1] = (int64_t)c->acc[1][0];
    r->bonds[0] = (int64_t)c->acc[0][1];
    r->bonds[1] = (int64_t)c->acc[1][1];
    r->dH = dH;
    r->beta = beta;
    r->accepted = take ? 1ull : 0ull;
    c->rec += 1ull;
    c->traj += 1ull;
    c->accepted += take ? 1ull : 0ull;
  }
  for (int ph = 0; ph < 2; ++ph)
    for (int j = 0; j < kHmcSums; ++j) {
      c->last[ph][j] = c->acc[ph][j];
      c->acc[ph][j] = 0ull;
    }
  return take;
}

}  // namespace xyh
