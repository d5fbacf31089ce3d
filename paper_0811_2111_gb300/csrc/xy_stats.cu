// xy_stats.cu -- per-chain series statistics and the beta derivatives that a
// torch.autograd backward needs, from the device-resident per-sweep records.
//
// For a chain at fixed beta with per-sweep energy E_s = -J C_s and an
// observable O_s that may depend on beta explicitly,
//     d<O>/dbeta = <dO_s/dbeta> - (<O_s E_s> - <O_s><E_s>)
// (differentiate <O> = sum O e^{-beta E} / Z).  For e_s = E_s / N the explicit
// term is zero, so d<e>/dbeta = -cov(e, E) = -var(E)/N (the specific heat is
// c_v = beta^2 var(E) / N).  For the helicity modulus
//     Upsilon_s = (J C_s - beta J^2 (Ix_s^2 + Iy_s^2)) / (2N)
// the explicit term is -J^2 <Ix^2 + Iy^2> / (2N).
//
// The series of each chain is cut into up to kMaxSegments segments, one CTA
// each (so all SMs share GB300's narrow FP64 pipes); every sum is FP64 in a
// fixed order (per thread in series order, a fixed shared-memory tree, the
// segments in order), so results are deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_internal.h"

namespace xyk {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Per record: E = -J C and jj = Ix^2 + Iy^2 in FP64 (the only FP64 work per
// record: three conversions and a handful of adds and fused multiply-adds; the
// FP64 pipe is narrow on this GPU), |m| in FP32.  Every other moment follows
// from these because e = E/N, C = -E/J and Upsilon is linear in C and jj:
//   cov(e, E)       = var(E) / N
//   cov(Upsilon, E) = (-var(E) - beta J^2 cov(jj, E)) / (2N)
struct Sample {
  double E, jj;
  float m;
};

__device__ __forceinline__ Sample sample(const xy_record& r, double J, float invNf) {
  const double unit = 1.0 / (double)(1ll << XY_FX_SHIFT);
  const double C = (double)r.sum[0] * unit;
  const double Ix = (double)r.sum[1] * unit, Iy = (double)r.sum[2] * unit;
  const float unitf = 1.0f / (float)(1ll << XY_FX_SHIFT);
  const float Mx = __ll2float_rn(r.sum[3]) * unitf, My = __ll2float_rn(r.sum[4]) * unitf;
  Sample s;
  s.E = -J * C;
  s.jj = fma(Ix, Ix, Iy * Iy);
  s.m = sqrtf(fmaf(Mx, Mx, My * My)) * invNf;
  return s;
}

// Pass 1: segment `blockIdx.y` of chain `blockIdx.x` accumulates moments of
// the samples shifted by the window's first sample K (one-pass covariances
// without cancellation): sums of dE, dE^2, djj, djj dE and |m|.
__global__ void __launch_bounds__(kThreads) k_series_partials(StatsArgs a) {
  __shared__ double sh[kThreads];
  const int chain = blockIdx.x, seg = blockIdx.y, nseg = gridDim.y;
  const xy_record* rec = a.records + (size_t)chain * a.stride + a.first;
  const float invNf = 1.0f / ((float)a.L[chain] * (float)a.L[chain]);
  const Sample k = sample(rec[0], a.J, invNf);
  const int64_t n = a.count;
  const int64_t lo = n * seg / nseg, hi = n * (seg + 1) / nseg;
  double m[kPartials] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
    const Sample s = sample(rec[i], a.J, invNf);
    const double dE = s.E - k.E, dj = s.jj - k.jj;
    m[0] += dE;
    m[1] = fma(dE, dE, m[1]);
    m[2] += dj;
    m[3] = fma(dj, dE, m[3]);
    m[4] += (double)s.m;
  }
  double* out = a.partials + ((size_t)chain * nseg + seg) * kPartials;
  for (int j = 0; j < 5; ++j) {
    const double t = block_sum(m[j], sh);
    if (threadIdx.x == 0) out[j] = t;
  }
}

// Pass 2: one thread per chain adds the segments in order and forms the
// means, covariances and derivatives.
__global__ void k_series_combine(StatsArgs a, int n_chains, int nseg) {
  const int chain = blockIdx.x * blockDim.x + threadIdx.x;
  if (chain >= n_chains) return;
  const xy_record* rec = a.records + (size_t)chain * a.stride + a.first;
  const double N = (double)a.L[chain] * (double)a.L[chain];
  const double J = a.J;
  const double beta = rec[0].beta;
  const Sample k = sample(rec[0], J, (float)(1.0 / N));
  double m[kPartials] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int sg = 0; sg < nseg; ++sg)
    for (int j = 0; j < 5; ++j) m[j] += a.partials[((size_t)chain * nseg + sg) * kPartials + j];
  const double inv = 1.0 / (double)a.count;
  const double mdE = m[0] * inv, mdj = m[2] * inv;
  const double varE = m[1] * inv - mdE * mdE;
  const double cov_jE = m[3] * inv - mdj * mdE;
  const double meanE = k.E + mdE, meanjj = k.jj + mdj;
  const double mean_e = meanE / N;
  const double mean_u = (-meanE - beta * J * J * meanjj) / (2.0 * N);    // J C = -E
  const double cov_uE = (-varE - beta * J * J * cov_jE) / (2.0 * N);
  double* o = a.out + (size_t)chain * kStatsFields;
  o[0] = mean_e;                                  // <e>
  o[1] = mean_u;                                  // <Upsilon>
  o[2] = m[4] * inv;                              // <|m|>
  o[3] = -varE / N;                               // d<e>/dbeta = -cov(e, E)
  o[4] = -cov_uE - J * J * meanjj / (2.0 * N);    // d<Upsilon>/dbeta
  o[5] = -cov_uE;                                 // covariance part alone
  o[6] = varE / N;                                // var(E)/N = c_v / beta^2
  o[7] = (double)a.count;
}

}  // namespace

cudaError_t launch_series_stats(const StatsArgs& a, int n_chains, cudaStream_t stream) {
  if (n_chains <= 0 || a.count <= 0 || !a.partials) return cudaErrorInvalidValue;
  // enough segments to fill the GPU, at least a few hundred samples each
  int nseg = (int)((a.count + 511) / 512);
  if (nseg > kMaxSegments) nseg = kMaxSegments;
  if (nseg < 1) nseg = 1;
  k_series_partials<<<dim3(n_chains, nseg), kThreads, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_series_combine<<<(n_chains + 63) / 64, 64, 0, stream>>>(a, n_chains, nseg);
  return cudaGetLastError();
}

}  // namespace xyk
