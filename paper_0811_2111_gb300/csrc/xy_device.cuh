// xy_device.cuh -- device-side building blocks of the XY Metropolis kernels:
// the Philox4x32-10 counter generator, the 24-bit uniforms, the precision
// switch between CUDA's accurate and fast intrinsics, and warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xy.h"

namespace xyd {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): two 32x32->64 products per round, the high halves
// xored into the other lanes with the round key, the key advanced by a Weyl
// sequence.  Counter x = (site, sweep, lattice_id, domain); key = seed words
// (the Metropolis draws pair two sites per counter: metropolis_counter).
constexpr uint32_t kMulA = 0xD2511F53u;
constexpr uint32_t kMulB = 0xCD9E8D57u;
constexpr uint32_t kWeylA = 0x9E3779B9u;
constexpr uint32_t kWeylB = 0xBB67AE85u;

// 32x32 -> 64-bit product as one wide multiply.
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

// The ten round keys of one seed, (k0 + r * kWeylA, k1 + r * kWeylB), computed
// on the host and passed as kernel arguments so the xors read them directly.
struct RoundKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

__host__ __device__ inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0;
    rk.k1[r] = k1;
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, const RoundKeys& rk) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint32_t hi_a, lo_a, hi_b, lo_b;
    mul_wide(kMulA, x.x, &hi_a, &lo_a);
    mul_wide(kMulB, x.z, &hi_b, &lo_b);
    x = make_uint4(hi_b ^ x.y ^ rk.k0[round], lo_b, hi_a ^ x.w ^ rk.k1[round], lo_a);
  }
  return x;
}

// The Metropolis draws (domain 1) use all four words of a block: the sites x
// and x + 2 of a row with x & 2 == 0 (plane columns 2m and 2m + 1 of one
// colour) share the block with counter (y*L + x, sweep, lattice_id, 1), the
// first taking words (w.x, w.y), the second (w.z, w.w).  Site s = y*L + x thus
// has counter s - (x & 2) and the upper pair iff x & 2: one generator call per
// two updates where a thread updates both sites of a pair.
__device__ __forceinline__ uint32_t metropolis_counter(uint32_t site, uint32_t x) {
  return site - (x & 2u);
}

__device__ __forceinline__ uint2 metropolis_words(const uint4& w, uint32_t x) {
  return (x & 2u) ? make_uint2(w.z, w.w) : make_uint2(w.x, w.y);
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

namespace xyd {

// Unit vector of an angle in [0, 2 pi] (or up to pi/4 outside), written from the
// mathematics: Cody-Waite reduction by pi/2 (W. J. Cody, W. Waite, "Software
// Manual for the Elementary Functions", 1980) with a two-part constant whose
// high part has three trailing zero bits (so q * hi is exact for |q| <= 7),
// then minimax polynomials for sin (to r^7) and cos (to r^8) on |r| <= pi/4,
// fitted for absolute error by Remez exchange (csrc/fit_sincos.py; truncation
// errors 1.8e-9 and 5.4e-11, far below FP32 rounding), and the quadrant
// identities sin(r + q pi/2), cos(r + q pi/2).
constexpr float kTwoOverPi = 0.636619772367581343f;
constexpr float kPio2Hi = 1.57079601287841796875f;       // pi/2 with 21 significant bits
constexpr float kPio2Lo = 3.13916473532088954e-07f;      // pi/2 - kPio2Hi
constexpr float kRoundMagic = 12582912.0f;               // 1.5 * 2^23: x + M - M = rint(x)

__device__ __forceinline__ void sincos_poly(float t, float* s_out, float* c_out) {
  const float qt = __fmaf_rn(t, kTwoOverPi, kRoundMagic);
  const float qf = __fsub_rn(qt, kRoundMagic);            // q = rint(t * 2/pi)
  float r = __fmaf_rn(-qf, kPio2Hi, t);                   // exact
  r = __fmaf_rn(-qf, kPio2Lo, r);
  const float r2 = __fmul_rn(r, r);
  // sin r = r + r^3 (c3 + r^2 (c5 + r^2 c7))
  float ps = __fmaf_rn(r2, -0.000194956359337084f, 0.00833197869360447f);
  ps = __fmaf_rn(r2, ps, -0.16666650772094727f);
  const float sr = __fmaf_rn(__fmul_rn(r, r2), ps, r);
  // cos r = 1 + r^2 (c2 + r^2 (c4 + r^2 (c6 + r^2 c8)))
  float pc = __fmaf_rn(r2, 2.4390450562350452e-05f, -0.0013886763481423259f);
  pc = __fmaf_rn(r2, pc, 0.04166662320494652f);
  pc = __fmaf_rn(r2, pc, -0.5f);
  const float cr = __fmaf_rn(r2, pc, 1.0f);
  // quadrant, on the FMA pipes (the ALU pipe is the sweep kernels' busiest):
  // with p = q - 2 in {-2, ..., 2} (t in [-pi/4, 2 pi + pi/4]),
  // t = r + p pi/2 + pi, so (sin t, cos t) = -(a sr + b cr, a cr - b sr) with
  // a = cos(p pi/2) = 1 - |p| and b = sin(p pi/2) = p (2 - |p|), both in
  // {-1, 0, 1} and never both nonzero: every product and sum is exact, the
  // same bits as swapping and negating sr and cr by the bits of q.
  const float pq = __fsub_rn(qf, 2.0f);
  const float a = __fsub_rn(1.0f, fabsf(pq));
  const float b = __fmul_rn(pq, __fsub_rn(2.0f, fabsf(pq)));
  *s_out = __fmaf_rn(-a, sr, __fmul_rn(-b, cr));
  *c_out = __fmaf_rn(b, sr, __fmul_rn(-a, cr));
}

// Precision switch of the kernels: 0 = the polynomial above with CUDA's
// expf, 1 = the SFU intrinsics __sincosf/__expf, 2 = CUDA's sincosf/expf.
template <int MODE>
__device__ __forceinline__ void unit_vector(float t, float* s, float* c) {
  if (MODE == 0) {
    sincos_poly(t, s, c);
  } else if (MODE == 1) {
    __sincosf(t, s, c);
  } else {
    sincosf(t, s, c);
  }
}

template <int MODE>
__device__ __forceinline__ float boltzmann(float x) {
  if (MODE == 1) return __expf(x);
  return expf(x);
}

// Sum of the four neighbour components in one fixed order.
__device__ __forceinline__ float nb_sum(float l, float r, float d, float u) {
  return __fadd_rn(__fadd_rn(l, r), __fadd_rn(d, u));
}

// Per-site contributions of a black site b (unit vector (cb, sb)) to the
// sweep sums, from its four red neighbours (left l, right r, down d, up u)
// and the red site (cm, sm) that shares its (y, k) index:
//   v0 = sum_4 cos(t_b - t_j)                 (its four bonds of C)
//   v1 = sin(t_b - t_r) - sin(t_b - t_l)      (its two x bonds of Ix)
//   v2 = sin(t_b - t_u) - sin(t_b - t_d)      (its two y bonds of Iy)
//   v3, v4 = cb + cm, sb + sm                 (M of both sites)
__device__ __forceinline__ void measure_terms(float cb, float sb, float cl, float sl, float cr,
                                              float sr, float cd, float sd, float cu, float su,
                                              float Sc, float Ss, float cm, float sm,
                                              float v[5]) {
  v[0] = __fmaf_rn(cb, Sc, __fmul_rn(sb, Ss));
  v[1] = __fmaf_rn(sb, __fsub_rn(cr, cl), -__fmul_rn(cb, __fsub_rn(sr, sl)));
  v[2] = __fmaf_rn(sb, __fsub_rn(cu, cd), -__fmul_rn(cb, __fsub_rn(su, sd)));
  v[3] = __fadd_rn(cb, cm);
  v[4] = __fadd_rn(sb, sm);
}

struct SiteResult {
  float th, c, s;
  bool accept;
};

// One Metropolis step of a site with angle t, unit vector (c0, s0) and
// neighbour sum (Sc, Ss), from its Philox words w0 (proposal) and w1
// (accept).  Rounding is pinned with explicit intrinsics so every kernel that
// calls this gets bit-identical decisions.  The select is the per-site vector
// accept of Sec. 3.2: new = z * proposal + (1 - z) * old.
template <int MODE>
__device__ __forceinline__ SiteResult metropolis_step(float t, float c0, float s0, float Sc,
                                                      float Ss, uint32_t w0, uint32_t w1,
                                                      float K, float delta) {
  // wrap once into [0, 2 pi): both candidates are formed and selected on the
  // unwrapped value (no branches).  delta * sym24(w0) is formed as
  // (delta 2^-23) * ((w0 >> 8) - 2^23): both products are exact, so the FMA
  // rounds the same real number, and delta 2^-23 is common to every site of a
  // kernel (one multiply per thread instead of one per site).
  const float raw = __fmaf_rn(delta * kR23, (float)((int32_t)(w0 >> 8) - 8388608), t);
  const float up = __fadd_rn(raw, kTwoPi), down = __fsub_rn(raw, kTwoPi);
  const float tp = raw < 0.f ? up : (raw >= kTwoPi ? down : raw);
  float s1, c1;
  unit_vector<MODE>(tp, &s1, &c1);
  // X = -dE / J = (cos t' - cos t) Sc + (sin t' - sin t) Ss
  const float X = __fmaf_rn(__fsub_rn(c1, c0), Sc, __fmul_rn(__fsub_rn(s1, s0), Ss));
  const bool acc = u24(w1) < boltzmann<MODE>(__fmul_rn(K, X));
  SiteResult r;
  r.th = acc ? tp : t;
  r.c = acc ? c1 : c0;
  r.s = acc ? s1 : s0;
  r.accept = acc;
  return r;
}

}  // namespace xyd

namespace xyd {

// ---- exact per-sweep sums (reduce mode 0) ----
// Each per-site term of the sweep sums is rounded to a signed integer before
// any addition: one FMA adds v * 2^shift to 1.5 * 2^23, whose unit in the
// last place is 1, so the result's mantissa holds v * 2^shift rounded half
// to even (exact for |v| 2^shift < 2^22), and the integers are added exactly.
// The sums are then independent of the order of addition: every kernel, tile
// shape and launch plan produces the same record bits for the same state.
// Shifts: 19 for v0 (four bond cosines, |v0| <= 4) and 20 for v1..v4
// (|v| <= 2), so |v| 2^shift <= 2^21; the record keeps 2^-XY_FX_SHIFT units.
__host__ __device__ constexpr int fx_term_shift(int i) { return i == 0 ? 19 : 20; }
constexpr float kFxScaleC = 524288.0f;        // 2^19
constexpr float kFxScale = 1048576.0f;        // 2^20
constexpr uint32_t kRoundMagicBits = 0x4B400000u;   // bit pattern of 1.5 * 2^23

// Per-thread sums of the terms' bit patterns (modulo 2^32) and their count.
struct FxSums {
  uint32_t s[5];
  uint32_t n;
};

__device__ __forceinline__ void fx_init(FxSums& f) {
#pragma unroll
  for (int i = 0; i < 5; ++i) f.s[i] = 0u;
  f.n = 0u;
}

__device__ __forceinline__ uint32_t fx_bits(float v, float scale) {
  return __float_as_uint(__fmaf_rn(v, scale, kRoundMagic));
}

// One black site's five terms.
__device__ __forceinline__ void fx_add(FxSums& f, const float v[5]) {
  f.s[0] += fx_bits(v[0], kFxScaleC);
#pragma unroll
  for (int i = 1; i < 5; ++i) f.s[i] += fx_bits(v[i], kFxScale);
  f.n += 1u;
}

// Two black sites' terms (three-input integer adds).
__device__ __forceinline__ void fx_add2(FxSums& f, const float a[5], const float b[5]) {
  f.s[0] += fx_bits(a[0], kFxScaleC) + fx_bits(b[0], kFxScaleC);
#pragma unroll
  for (int i = 1; i < 5; ++i) f.s[i] += fx_bits(a[i], kFxScale) + fx_bits(b[i], kFxScale);
  f.n += 2u;
}

// The thread's sum of term i in units of 2^-fx_term_shift(i).  Exact while
// the thread holds at most 1023 terms.
__device__ __forceinline__ int32_t fx_value(const FxSums& f, int i) {
  return (int32_t)(f.s[i] - f.n * kRoundMagicBits);
}

// Whether a non-finite value entered the thread's terms.  Every site of the
// lattice enters some black site's v0 (its own, or a neighbour's), and a NaN
// or infinite term moves the bit-pattern sum by a nonzero multiple of 2^22
// (modulo 2^32, for fewer than 512 such terms), far outside the finite range
// |sum| <= n 2^21.
__device__ __forceinline__ bool fx_nonfinite(const FxSums& f) {
  const int32_t v = fx_value(f, 0);
  const uint32_t mag = v < 0 ? (uint32_t)(-(int64_t)v) : (uint32_t)v;
  return mag > (f.n << 21);
}

// End-of-CTA commit of exact sums: warp reduction of the integers
// (redux.sync; WIDE splits each 32-bit value into 16-bit halves first, for
// threads that may hold more than 31 terms), int64 over the CTA's warps, and
// one 64-bit atomic per sum into the record, rescaled to 2^-XY_FX_SHIFT.
// `part` holds [warps][5][2] 32-bit words and `cnt` [warps] counters in shared
// memory.  Must be reached by every thread of the CTA.
template <int NWARPS, bool WIDE>
__device__ __forceinline__ void commit_block_fx(const FxSums& f, unsigned int n_acc,
                                                float (*part)[5][2], unsigned int* cnt,
                                                xy_record* rec, double beta, bool first_block,
                                                bool measure) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned int warp_acc = __reduce_add_sync(0xffffffffu, n_acc);
  long long ws[5] = {0, 0, 0, 0, 0};
  bool bad = false;
  if (measure) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const int32_t v = fx_value(f, i);
      if (!WIDE) {
        ws[i] = (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)v);
      } else {
        const uint32_t lo = __reduce_add_sync(0xffffffffu, (uint32_t)v & 0xffffu);
        const int32_t hi = (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)(v >> 16));
        ws[i] = (long long)hi * 65536ll + (long long)lo;
      }
    }
    bad = __any_sync(0xffffffffu, fx_nonfinite(f));
  }
  if (lane == 0) {
    cnt[warp] = warp_acc | (bad ? 0x80000000u : 0u);
    if (measure) {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        reinterpret_cast<uint32_t*>(part[warp][i])[0] = (uint32_t)(unsigned long long)ws[i];
        reinterpret_cast<uint32_t*>(part[warp][i])[1] = (uint32_t)((unsigned long long)ws[i] >> 32);
      }
    }
  }
  __syncthreads();
  if (warp != 0) return;
  if (lane == 0) {
    unsigned long long total = 0;
    bool any_bad = false;
    for (int w = 0; w < NWARPS; ++w) {
      total += cnt[w] & 0x7fffffffu;
      any_bad |= (cnt[w] & 0x80000000u) != 0u;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&rec->accepted), total);
    if (any_bad) atomicOr(reinterpret_cast<unsigned long long*>(&rec->flags), 1ull);
    if (measure && first_block) rec->beta = beta;
  }
  if (!measure || lane >= 5) return;
  // lanes 0..4 each own one of the five sums
  unsigned long long t = 0;
  for (int w = 0; w < NWARPS; ++w) {
    const uint32_t* pw = reinterpret_cast<const uint32_t*>(part[w][lane]);
    t += (unsigned long long)pw[0] | ((unsigned long long)pw[1] << 32);
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(&rec->sum[lane]),
            t << (XY_FX_SHIFT - fx_term_shift(lane)));
}

// Per-thread sums of a sweep kernel: exact fixed point (RED == 0) or
// Neumaier-compensated FP32 pairs (RED == 1), with one commit for both.
template <int RED>
struct SweepSums {
  FxSums fx;
  float acc[5], cmp[5];
  __device__ __forceinline__ void init() {
    if (RED == 0) {
      fx_init(fx);
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) acc[i] = cmp[i] = 0.f;
    }
  }
  __device__ __forceinline__ void add(const float v[5]) {
    if (RED == 0) {
      fx_add(fx, v);
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) neumaier_add(acc[i], cmp[i], v[i]);
    }
  }
  __device__ __forceinline__ void add2(const float a[5], const float b[5]) {
    if (RED == 0) {
      fx_add2(fx, a, b);
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        neumaier_add(acc[i], cmp[i], a[i]);
        neumaier_add(acc[i], cmp[i], b[i]);
      }
    }
  }
};

template <int NWARPS, int RED, bool MEASURE, bool WIDE = false>
__device__ __forceinline__ void commit_block(float acc[5], float cmp[5], unsigned int n_acc,
                                             float (*part)[5][2], unsigned int* cnt,
                                             xy_record* rec, double beta, bool first_block);

template <int NWARPS, int RED, bool MEASURE, bool WIDE = false>
__device__ __forceinline__ void commit_sums(SweepSums<RED>& s, unsigned int n_acc,
                                            float (*part)[5][2], unsigned int* cnt,
                                            xy_record* rec, double beta, bool first_block) {
  if (RED == 0) {
    commit_block_fx<NWARPS, WIDE>(s.fx, n_acc, part, cnt, rec, beta, first_block, MEASURE);
  } else {
    commit_block<NWARPS, 1, MEASURE>(s.acc, s.cmp, n_acc, part, cnt, rec, beta, first_block);
  }
}

}  // namespace xyd

namespace xyd {

// End-of-CTA reduction of the compensated sums (reduce mode 1): per-thread
// Neumaier pairs -> warp shuffle -> compensated FP32 over the CTA's warps ->
// FP64 -> fixed-point atomics into the record.  `part` holds [warps][5][2]
// floats and `cnt` [warps] counters in shared memory.  Must be reached by
// every thread of the CTA.  (Reduce mode 0 commits through commit_block_fx.)
template <int NWARPS, int RED, bool MEASURE, bool WIDE>
__device__ __forceinline__ void commit_block(float acc[5], float cmp[5], unsigned int n_acc,
                                             float (*part)[5][2], unsigned int* cnt,
                                             xy_record* rec, double beta, bool first_block) {
  static_assert(RED == 1, "reduce mode 0 commits through commit_block_fx");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned int warp_acc = __reduce_add_sync(0xffffffffu, n_acc);
  if (MEASURE) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      acc[i] = warp_sum(acc[i]);
      cmp[i] = warp_sum(cmp[i]);
    }
  }
  if (lane == 0) {
    cnt[warp] = warp_acc;
    if (MEASURE) {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        part[warp][i][0] = acc[i];
        part[warp][i][1] = cmp[i];
      }
    }
  }
  __syncthreads();
  if (warp != 0) return;
  if (lane == 0) {
    unsigned long long total = 0;
    for (int w = 0; w < NWARPS; ++w) total += cnt[w];
    atomicAdd(reinterpret_cast<unsigned long long*>(&rec->accepted), total);
    if (MEASURE && first_block) rec->beta = beta;
  }
  if (!MEASURE || lane >= 5) return;
  // lanes 0..4 each own one of the five sums
  float hi = 0.f, lo = 0.f;
  for (int w = 0; w < NWARPS; ++w) {
    neumaier_add(hi, lo, part[w][lane][0]);
    lo += part[w][lane][1];
  }
  const double d = (double)hi + (double)lo;
  const double scaled = d * (double)(1ll << XY_FX_SHIFT);
  if (!(fabs(scaled) < 9.0e18)) {
    atomicOr(reinterpret_cast<unsigned long long*>(&rec->flags), 1ull);
    return;
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(&rec->sum[lane]),
            (unsigned long long)__double2ll_rn(scaled));
}

}  // namespace xyd
