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
// One CTA per chain; two passes over the series (means, then centred
// products), all sums in FP64 (per thread in series order, then a fixed
// shared-memory tree), so results are deterministic.
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

struct Sample {
  double E, e, ups, jj, m;
};

__device__ __forceinline__ Sample sample(const xy_record& r, double N, double J) {
  const double unit = 1.0 / (double)(1ll << XY_FX_SHIFT);
  const double C = (double)r.sum[0] * unit, Ix = (double)r.sum[1] * unit;
  const double Iy = (double)r.sum[2] * unit, Mx = (double)r.sum[3] * unit;
  const double My = (double)r.sum[4] * unit;
  Sample s;
  s.E = -J * C;
  s.e = s.E / N;
  s.jj = Ix * Ix + Iy * Iy;
  s.ups = (J * C - r.beta * J * J * s.jj) / (2.0 * N);
  s.m = sqrt(Mx * Mx + My * My) / N;
  return s;
}

__global__ void __launch_bounds__(kThreads) k_series_stats(StatsArgs a) {
  __shared__ double sh[kThreads];
  const int chain = blockIdx.x;
  const xy_record* rec = a.records + (size_t)chain * a.stride + a.first;
  const double N = (double)a.L[chain] * (double)a.L[chain];
  const double J = a.J;
  const int64_t n = a.count;
  double sE = 0, se = 0, su = 0, sj = 0, sm = 0;
  for (int64_t i = threadIdx.x; i < n; i += kThreads) {
    const Sample s = sample(rec[i], N, J);
    sE += s.E;
    se += s.e;
    su += s.ups;
    sj += s.jj;
    sm += s.m;
  }
  const double inv = 1.0 / (double)n;
  const double mE = block_sum(sE, sh) * inv, me = block_sum(se, sh) * inv;
  const double mu = block_sum(su, sh) * inv, mj = block_sum(sj, sh) * inv;
  const double mm = block_sum(sm, sh) * inv;
  double cEE = 0, ceE = 0, cuE = 0;
  for (int64_t i = threadIdx.x; i < n; i += kThreads) {
    const Sample s = sample(rec[i], N, J);
    const double dE = s.E - mE;
    cEE += dE * dE;
    ceE += (s.e - me) * dE;
    cuE += (s.ups - mu) * dE;
  }
  const double varE = block_sum(cEE, sh) * inv;
  const double cov_eE = block_sum(ceE, sh) * inv;
  const double cov_uE = block_sum(cuE, sh) * inv;
  if (threadIdx.x == 0) {
    double* o = a.out + (size_t)chain * kStatsFields;
    o[0] = me;                                  // <e>
    o[1] = mu;                                  // <Upsilon>
    o[2] = mm;                                  // <|m|>
    o[3] = -cov_eE;                             // d<e>/dbeta
    o[4] = -cov_uE - J * J * mj / (2.0 * N);    // d<Upsilon>/dbeta
    o[5] = -cov_uE;                             // covariance part alone
    o[6] = varE / N;                            // var(E)/N = c_v / beta^2
    o[7] = (double)n;
  }
}

}  // namespace

cudaError_t launch_series_stats(const StatsArgs& a, int n_chains, cudaStream_t stream) {
  if (n_chains <= 0 || a.count <= 0) return cudaErrorInvalidValue;
  k_series_stats<<<n_chains, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace xyk
