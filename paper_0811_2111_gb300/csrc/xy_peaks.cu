// xy_peaks.cu -- instruction-rate microbenchmarks (xy_peaks.h): the measured
// peaks that the sweep kernels' compute roofline divides by.
//
// Every kind is one kernel: each thread keeps CHAINS independent dependency
// chains of one instruction form and advances each of them 16 times per loop
// trip (the trip's own counter and branch are 3 instructions per 16 * CHAINS
// operations).  The forms are inline PTX with asm volatile, so neither the
// instruction nor its count is the compiler's choice; the library's own
// device functions (Philox block, unit vectors, expf) are called as the sweep
// kernels call them.  A thread stores its chains' combination only if it
// equals a value it cannot take, so nothing is eliminated and nothing is
// written.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>

#include "xy_device.cuh"
#include "xy_peaks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 16;

static __device__ uint32_t g_peak_sink[256];

thread_local char g_peak_msg[256] = "no error";

void peak_msg(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_peak_msg, sizeof(g_peak_msg), fmt, ap);
  va_end(ap);
}

__device__ __forceinline__ void sink(uint32_t v, uint32_t impossible) {
  if (v == impossible) g_peak_sink[threadIdx.x & 255] = v;
}

// Operations per chain advance, and chains per thread, of each kind.
__host__ __device__ constexpr int chains_of(int kind) {
  return (kind == XY_PEAK_ISSUE || kind == XY_PEAK_PHILOX) ? 4 : 8;
}
__host__ __device__ constexpr int ops_per_advance(int kind) {
  return kind == XY_PEAK_ISSUE ? 4 : 1;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_peak(uint32_t seed, int trips, xyd::RoundKeys rk) {
  constexpr int CH = chains_of(KIND);
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t b = seed | 1u, c = seed ^ 0x9e3779b9u;
  const float fb = 1.0f + (float)(seed & 7u) * 1e-7f, fc = 1e-7f * (float)(seed >> 29);
  uint32_t acc = 0;
  if (KIND == XY_PEAK_FFMA || KIND == XY_PEAK_MUFU_SIN || KIND == XY_PEAK_MUFU_EX2 ||
      KIND == XY_PEAK_UNIT_VECTOR || KIND == XY_PEAK_UNIT_VECTOR_SFU || KIND == XY_PEAK_EXPF) {
    float f[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) f[j] = (float)((t + 97u * j) & 1023u) * (1.0f / 1024.0f);
    for (int it = 0; it < trips; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          if (KIND == XY_PEAK_FFMA) {
            asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[j]) : "f"(fb), "f"(fc));
          } else if (KIND == XY_PEAK_MUFU_SIN) {
            asm volatile("sin.approx.f32 %0, %0;" : "+f"(f[j]));
          } else if (KIND == XY_PEAK_MUFU_EX2) {
            asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
          } else if (KIND == XY_PEAK_UNIT_VECTOR) {
            float s, co;
            xyd::sincos_poly(f[j], &s, &co);
            f[j] = s + co;
          } else if (KIND == XY_PEAK_UNIT_VECTOR_SFU) {
            float s, co;
            __sincosf(f[j], &s, &co);
            f[j] = s + co;
          } else {
            f[j] = __fmaf_rn(expf(f[j]), 0.25f, -0.5f);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) acc ^= __float_as_uint(f[j]);
  } else if (KIND == XY_PEAK_DFMA) {
    double d[CH];
    const double db = 1.0 + 1e-12 * (double)(seed & 7u), dc = 1e-12;
#pragma unroll
    for (int j = 0; j < CH; ++j) d[j] = (double)(t + j);
    for (int it = 0; it < trips; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int j = 0; j < CH; ++j)
          asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[j]) : "d"(db), "d"(dc));
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) acc ^= (uint32_t)__double_as_longlong(d[j]);
  } else if (KIND == XY_PEAK_IMAD_WIDE) {
    uint64_t w[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) w[j] = ((uint64_t)(t * 2654435761u + j) << 32) | (t + j);
    for (int it = 0; it < trips; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int j = 0; j < CH; ++j)
          // the multiplicand is the low word of the chain, so the product
          // cannot be hoisted out of the loop
          asm volatile("{\n\t.reg .u32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\t"
                       "mad.wide.u32 %0, lo, %1, %0;\n\t}" : "+l"(w[j]) : "r"(b));
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) acc ^= (uint32_t)w[j] ^ (uint32_t)(w[j] >> 32);
  } else if (KIND == XY_PEAK_ISSUE) {
    // per advance: three FP32 FMAs of separate chains and one three-input xor,
    // all independent of each other: no pipe above 3/4 of its rate
    float f[CH], g[CH], h[CH];
    uint32_t a[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      f[j] = (float)(t & 255u);
      g[j] = f[j] + 1.0f;
      h[j] = f[j] + 2.0f;
      a[j] = t + j;
    }
    for (int it = 0; it < trips; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[j]) : "f"(fb), "f"(fc));
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(g[j]) : "f"(fb), "f"(fc));
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(h[j]) : "f"(fb), "f"(fc));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j)
      acc ^= a[j] ^ __float_as_uint(f[j]) ^ __float_as_uint(g[j]) ^ __float_as_uint(h[j]);
  } else if (KIND == XY_PEAK_PHILOX) {
    uint4 x[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) x[j] = make_uint4(t, j, seed, 1u);
    for (int it = 0; it < trips; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int j = 0; j < CH; ++j) x[j] = xyd::philox4x32_10(x[j], rk);
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) acc ^= x[j].x ^ x[j].y ^ x[j].z ^ x[j].w;
  } else {
    uint32_t a[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) a[j] = t * 2654435761u + j;
    for (int it = 0; it < trips; ++it) {
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          if (KIND == XY_PEAK_IMAD) {
            asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
          } else if (KIND == XY_PEAK_IMAD_HI) {
            asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
          } else if (KIND == XY_PEAK_LOP3) {
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
          } else if (KIND == XY_PEAK_IADD) {
            // two dependent adds, which the assembler fuses into one
            // three-input add (one instruction per operation)
            asm volatile("add.u32 %0, %0, %1;\n\tadd.u32 %0, %0, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
          } else {   // XY_PEAK_F2I: the result's bits are the next input
            asm volatile("{\n\t.reg .f32 tf;\n\tmov.b32 tf, %0;\n\tcvt.rni.s32.f32 %0, tf;\n\t}"
                         : "+r"(a[j]));
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) acc ^= a[j];
  }
  sink(acc, seed ^ 0xdeadbeefu);
}

typedef void (*PeakKernel)(uint32_t, int, xyd::RoundKeys);

PeakKernel kernel_of(int kind) {
  switch (kind) {
    case XY_PEAK_FFMA: return k_peak<XY_PEAK_FFMA>;
    case XY_PEAK_IMAD: return k_peak<XY_PEAK_IMAD>;
    case XY_PEAK_IMAD_WIDE: return k_peak<XY_PEAK_IMAD_WIDE>;
    case XY_PEAK_IMAD_HI: return k_peak<XY_PEAK_IMAD_HI>;
    case XY_PEAK_LOP3: return k_peak<XY_PEAK_LOP3>;
    case XY_PEAK_IADD: return k_peak<XY_PEAK_IADD>;
    case XY_PEAK_MUFU_SIN: return k_peak<XY_PEAK_MUFU_SIN>;
    case XY_PEAK_MUFU_EX2: return k_peak<XY_PEAK_MUFU_EX2>;
    case XY_PEAK_F2I: return k_peak<XY_PEAK_F2I>;
    case XY_PEAK_DFMA: return k_peak<XY_PEAK_DFMA>;
    case XY_PEAK_ISSUE: return k_peak<XY_PEAK_ISSUE>;
    case XY_PEAK_PHILOX: return k_peak<XY_PEAK_PHILOX>;
    case XY_PEAK_UNIT_VECTOR: return k_peak<XY_PEAK_UNIT_VECTOR>;
    case XY_PEAK_UNIT_VECTOR_SFU: return k_peak<XY_PEAK_UNIT_VECTOR_SFU>;
    case XY_PEAK_EXPF: return k_peak<XY_PEAK_EXPF>;
    default: return nullptr;
  }
}

}  // namespace

extern "C" {

xy_status xy_peak_measure(int32_t kind, int32_t iters, int32_t reps, void* cuda_stream,
                          double* ops_per_s, double* ms_best, double* ops_per_launch) {
  PeakKernel k = kernel_of(kind);
  if (!k || iters < 1 || iters > (1 << 20) || reps < 1 || reps > 100 || !ops_per_s) {
    peak_msg("xy_peak_measure: bad kind, iters, reps or NULL ops_per_s");
    return XY_EINVAL;
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int trips = (iters + kUnroll - 1) / kUnroll;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(k),
                                                      kThreads, 0);
  if (e != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    peak_msg("xy_peak_measure: %s", e != cudaSuccess ? cudaGetErrorString(e) : "no residency");
    return XY_ECUDA;
  }
  const int grid = sms * per_sm;
  const xyd::RoundKeys rk = xyd::make_round_keys(0x243f6a8885a308d3ull);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float best = 0.f;
  for (int r = 0; e == cudaSuccess && r <= reps; ++r) {     // launch 0 warms up
    e = cudaEventRecord(ev[0], stream);
    if (e != cudaSuccess) break;
    k<<<grid, kThreads, 0, stream>>>(0x51ed27u + (uint32_t)r, trips, rk);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess && r > 0 && (best == 0.f || ms < best)) best = ms;
  }
  for (int i = 0; i < 2; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess || best <= 0.f) {
    (void)cudaGetLastError();
    peak_msg("xy_peak_measure: %s", e != cudaSuccess ? cudaGetErrorString(e) : "zero duration");
    return XY_ECUDA;
  }
  const double ops = (double)grid * kThreads * (double)trips * kUnroll * chains_of(kind) *
                     ops_per_advance(kind);
  *ops_per_s = ops / (best * 1e-3);
  if (ms_best) *ms_best = best;
  if (ops_per_launch) *ops_per_launch = ops;
  return XY_OK;
}

const char* xy_peak_last_error(void) { return g_peak_msg; }

}  // extern "C"
