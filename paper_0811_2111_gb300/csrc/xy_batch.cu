// xy_batch.cu -- many independent lattices of uneven sides and temperatures in
// one launch per round of sweeps, and replica exchange between neighbouring
// temperatures of a ladder.
//
// Work decomposition.  Every lattice is cut into bands of whole rows; each band
// is one CTA of 256 threads, and all bands of a lattice belong to one cluster
// of kClusterSize CTAs (a cluster may hold several small lattices, and padding
// CTAs with no band).  A launch runs `sweeps` sweeps: for each colour a CTA
//   1. stages the unit vectors of the other colour on its band's rows and one
//      row above and below (periodic within the lattice) in shared memory,
//   2. updates its band's sites of this colour in global memory (the 12.7 MB of
//      the replica-exchange workload stays in the 129 MB L2),
//   3. after the black half adds its sums to the lattice's record of the sweep,
//   4. meets the other CTAs of its cluster at a hardware cluster barrier
//      (release/acquire at cluster scope) so that the next half-sweep sees the
//      neighbouring bands' new angles.
// No CTA ever waits for a CTA outside its cluster, so clusters run in any
// order and need no co-residency beyond what the cluster launch guarantees.
// Every CTA of a cluster reaches every barrier (padding CTAs included).
//
// The site update is the same pinned-rounding device function the single
// lattice kernels use, with the same Philox counters (the site's Metropolis
// counter, sweep, lattice id, 1) and words: a lattice evolves bit-identically
// whether it runs alone or in a batch.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_device.cuh"
#include "xy_internal.h"

namespace cg = cooperative_groups;

namespace xyk {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ int wrap_row(int y, int L) {
  y += (y < 0) ? L : 0;
  y -= (y >= L) ? L : 0;
  return y;
}

template <int MODE, int RED>
__global__ void __launch_bounds__(kThreads) k_batch_round(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* cs = reinterpret_cast<float2*>(smem);                       // [(rows+2) * W]
  float(*part)[5][2] = reinterpret_cast<float(*)[5][2]>(smem + a.cs_bytes);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(smem + a.cs_bytes + sizeof(float) * kWarps * 10);

  cg::cluster_group cluster = cg::this_cluster();
  const BatchBand band = a.bands[blockIdx.x];
  const bool active = band.lattice >= 0;
  const int L = active ? a.L[band.lattice] : 2;
  const int W = L / 2;
  const int rows = band.y_end - band.y_begin;
  const size_t plane = (size_t)L * (size_t)W;
  float* theta = active ? a.theta + a.offset[band.lattice] : nullptr;
  const uint32_t lid = active ? a.lattice_id0 + (uint32_t)band.lattice : 0u;
  const double beta = active ? a.beta[band.lattice] : 0.0;
  const float K = (float)(beta * a.J);
  xy_record* rec = active ? a.records + (size_t)band.lattice * a.rec_stride : nullptr;

  // 2-d thread layout over a band of width W: tx along k, ty along rows
  const int tx_w = W < kThreads ? W : kThreads;
  const int ty_n = kThreads / tx_w;
  const int tx = threadIdx.x % tx_w;
  const int ty = threadIdx.x / tx_w;
  const bool lane_on = ty < ty_n;

  const uint32_t sweep0 = a.counters[0];
  for (int sw = 0; sw < a.sweeps; ++sw) {
    const uint32_t sweep = sweep0 + (uint32_t)sw;
    for (int colour = 0; colour < 2; ++colour) {
      if (active) {
        const float* other = theta + (size_t)(1 - colour) * plane;
        float* own = theta + (size_t)colour * plane;
        // 1. stage the other colour on rows y_begin-1 .. y_end (stage row = row - y_begin + 1)
        for (int idx = threadIdx.x; idx < (rows + 2) * W; idx += kThreads) {
          const int sr = idx / W;
          const int k = idx - sr * W;
          const int y = wrap_row(band.y_begin - 1 + sr, L);
          float s, c;
          xyd::unit_vector<MODE>(__ldcg(other + (size_t)y * W + k), &s, &c);
          cs[idx] = make_float2(c, s);
        }
        __syncthreads();
        // 2. update this colour's sites of the band
        unsigned int n_acc = 0;
        xyd::SweepSums<RED> sums;
        sums.init();
        if (lane_on) {
          for (int r = ty; r < rows; r += ty_n) {
            const int y = band.y_begin + r;
            const int q = (y + colour) & 1;                 // x = 2k + q
            const float2* row = cs + (size_t)(r + 1) * W;
            const float2* down = cs + (size_t)r * W;
            const float2* up = cs + (size_t)(r + 2) * W;
            for (int k = tx; k < W; k += tx_w) {
              int kl = k + q - 1, kr = k + q;
              kl += (kl < 0) ? W : 0;
              kr -= (kr >= W) ? W : 0;
              const float2 l = row[kl], rt = row[kr], d = down[k], u = up[k];
              const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
              const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
              const uint32_t x = 2u * (uint32_t)k + (uint32_t)q;
              const uint32_t ctr = xyd::metropolis_counter((uint32_t)y * (uint32_t)L + x, x);
              const uint4 w = xyd::philox4x32_10(make_uint4(ctr, sweep, lid, 1u), a.rk);
              const uint2 uw = xyd::metropolis_words(w, x);
              float* tp = own + (size_t)y * W + k;
              const float t = __ldcg(tp);
              float s0, c0;
              xyd::unit_vector<MODE>(t, &s0, &c0);
              const xyd::SiteResult res =
                  xyd::metropolis_step<MODE>(t, c0, s0, Sc, Ss, uw.x, uw.y, K, a.delta);
              *tp = res.th;
              n_acc += res.accept ? 1u : 0u;
              if (colour == 1) {
                const float2 m = row[k];
                float v[5];
                xyd::measure_terms(res.c, res.s, l.x, l.y, rt.x, rt.y, d.x, d.y, u.x, u.y, Sc,
                                   Ss, m.x, m.y, v);
                sums.add(v);
              }
            }
          }
        }
        // 3. the sweep's record (the red half adds only its accept count)
        // a thread may hold more than 31 terms here: the wide warp reduction
        if (colour == 0) {
          xyd::commit_sums<kWarps, RED, false, true>(sums, n_acc, part, cnt,
                                                     rec + sweep - a.rec_sweep0, beta, false);
        } else {
          xyd::commit_sums<kWarps, RED, true, true>(sums, n_acc, part, cnt,
                                                    rec + sweep - a.rec_sweep0, beta,
                                                    band.y_begin == 0);
        }
        __threadfence();
      }
      // 4. all bands of the lattice finish this half before any starts the next
      cluster.sync();
    }
  }
}

// ---------------------------------------------------------------------------
// Fused variant: one staging and one cluster barrier per sweep.
//
// The state ping-pongs between two buffers by sweep parity (sweep t reads
// buffer t mod 2 and writes the other).  Per sweep a CTA stages both colours of
// its band's rows and two halo rows above and below (angle and unit vector),
// updates the red sites of its rows and of the ring rows just outside them
// (those belong to the neighbouring bands, which compute them identically from
// the same old state and counter-based words), then its black sites against
// the new red values, writes its rows to the other buffer and meets its
// cluster once.  The same site function, counters and measure terms as every
// other kernel: results are bit-identical to the two-pass variant.
// ---------------------------------------------------------------------------
constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;

template <int MODE, int RED>
__global__ void __launch_bounds__(kFusedThreads, 2) k_batch_fused(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const BatchBand band = a.bands[blockIdx.x];
  const bool active = band.lattice >= 0;
  const int L = active ? a.L[band.lattice] : 2;
  const int W = L / 2;
  const int R = band.y_end - band.y_begin;
  const int SR = R + 4;                                   // stage rows y_begin-2 .. y_end+1
  const size_t nst = (size_t)SR * (size_t)W;
  float2* cs_r = reinterpret_cast<float2*>(smem);         // red plane unit vectors
  float2* cs_b = cs_r + nst;                              // black plane unit vectors
  float* th_r = reinterpret_cast<float*>(cs_b + nst);     // red plane angles
  float* th_b = th_r + nst;                               // black plane angles
  float(*part)[5][2] = reinterpret_cast<float(*)[5][2]>(smem + a.cs_bytes);
  unsigned int* cnt =
      reinterpret_cast<unsigned int*>(smem + a.cs_bytes + sizeof(float) * kFusedWarps * 10);

  const size_t plane = (size_t)L * (size_t)W;
  const int64_t off = active ? a.offset[band.lattice] : 0;
  const uint32_t lid = active ? a.lattice_id0 + (uint32_t)band.lattice : 0u;
  const double beta = active ? a.beta[band.lattice] : 0.0;
  const float K = (float)(beta * a.J);
  xy_record* rec = active ? a.records + (size_t)band.lattice * a.rec_stride : nullptr;
  const uint32_t uL = (uint32_t)L;

  const int tx_w = W < kFusedThreads ? W : kFusedThreads;
  const int ty_n = kFusedThreads / tx_w;
  const int tx = threadIdx.x % tx_w;
  const int ty = threadIdx.x / tx_w;
  const bool lane_on = ty < ty_n;

  const uint32_t sweep0 = a.counters[0];
  for (int sw = 0; sw < a.sweeps; ++sw) {
    const uint32_t sweep = sweep0 + (uint32_t)sw;
    if (active) {
      const float* src = ((sweep & 1u) ? a.theta2 : a.theta) + off;
      float* dst = ((sweep & 1u) ? a.theta : a.theta2) + off;
      // 1. stage both planes (red is not needed on the outermost rows).  A
      // band spans its lattice's full width W <= 128, so a thread owns column
      // k = tx and rows ty, ty + ty_n, ...; all of a pass's loads are issued
      // before any sincos so that their latencies overlap.
      if (lane_on) {
        constexpr int kPF = 10;
        for (int base = ty; base < SR; base += kPF * ty_n) {
          float vb[kPF], vr[kPF];
#pragma unroll
          for (int i = 0; i < kPF; ++i) {
            const int sr = base + i * ty_n;
            vb[i] = 0.f;
            vr[i] = 0.f;
            if (sr < SR) {
              const size_t g = (size_t)wrap_row(band.y_begin - 2 + sr, L) * W + tx;
              vb[i] = __ldcg(src + plane + g);
              if (sr > 0 && sr < SR - 1) vr[i] = __ldcg(src + g);
            }
          }
#pragma unroll
          for (int i = 0; i < kPF; ++i) {
            const int sr = base + i * ty_n;
            if (sr < SR) {
              const size_t idx = (size_t)sr * W + tx;
              float s, c;
              xyd::unit_vector<MODE>(vb[i], &s, &c);
              th_b[idx] = vb[i];
              cs_b[idx] = make_float2(c, s);
              if (sr > 0 && sr < SR - 1) {
                xyd::unit_vector<MODE>(vr[i], &s, &c);
                th_r[idx] = vr[i];
                cs_r[idx] = make_float2(c, s);
              }
            }
          }
        }
      }
      __syncthreads();
      // 2. red: stage rows 1 .. SR-2 (the band and its two ring rows)
      unsigned int n_acc = 0;
      if (lane_on) {
        for (int sr = 1 + ty; sr <= SR - 2; sr += ty_n) {
          const int y = wrap_row(band.y_begin - 2 + sr, L);
          const int q = y & 1;                              // red: x = 2k + (y & 1)
          const bool own = sr >= 2 && sr <= R + 1;
          const float2* row = cs_b + (size_t)sr * W;
          for (int k = tx; k < W; k += tx_w) {
            int kl = k + q - 1, kr = k + q;
            kl += (kl < 0) ? W : 0;
            kr -= (kr >= W) ? W : 0;
            const float2 l = row[kl], rt = row[kr], d = row[k - W], u = row[k + W];
            const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
            const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
            const uint32_t x = 2u * (uint32_t)k + (uint32_t)q;
            const uint4 w = xyd::philox4x32_10(
                make_uint4(xyd::metropolis_counter((uint32_t)y * uL + x, x), sweep, lid, 1u), a.rk);
            const uint2 uw = xyd::metropolis_words(w, x);
            const size_t idx = (size_t)sr * W + k;
            const float2 o = cs_r[idx];
            const xyd::SiteResult res =
                xyd::metropolis_step<MODE>(th_r[idx], o.x, o.y, Sc, Ss, uw.x, uw.y, K, a.delta);
            th_r[idx] = res.th;
            cs_r[idx] = make_float2(res.c, res.s);
            if (own) {
              n_acc += res.accept ? 1u : 0u;
              dst[(size_t)y * W + k] = res.th;
            }
          }
        }
      }
      __syncthreads();
      // 3. black: the band rows (stage rows 2 .. R+1), with the sweep sums
      xyd::SweepSums<RED> sums;
      sums.init();
      if (lane_on) {
        for (int sr = 2 + ty; sr <= R + 1; sr += ty_n) {
          const int y = band.y_begin - 2 + sr;
          const int q = (y + 1) & 1;                        // black: x = 2k + ((y + 1) & 1)
          const float2* row = cs_r + (size_t)sr * W;
          for (int k = tx; k < W; k += tx_w) {
            int kl = k + q - 1, kr = k + q;
            kl += (kl < 0) ? W : 0;
            kr -= (kr >= W) ? W : 0;
            const float2 l = row[kl], rt = row[kr], d = row[k - W], u = row[k + W];
            const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
            const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
            const uint32_t x = 2u * (uint32_t)k + (uint32_t)q;
            const uint4 w = xyd::philox4x32_10(
                make_uint4(xyd::metropolis_counter((uint32_t)y * uL + x, x), sweep, lid, 1u), a.rk);
            const uint2 uw = xyd::metropolis_words(w, x);
            const size_t idx = (size_t)sr * W + k;
            const float2 o = cs_b[idx];
            const xyd::SiteResult res =
                xyd::metropolis_step<MODE>(th_b[idx], o.x, o.y, Sc, Ss, uw.x, uw.y, K, a.delta);
            n_acc += res.accept ? 1u : 0u;
            dst[plane + (size_t)y * W + k] = res.th;
            const float2 m = row[k];
            float v[5];
            xyd::measure_terms(res.c, res.s, l.x, l.y, rt.x, rt.y, d.x, d.y, u.x, u.y, Sc, Ss,
                               m.x, m.y, v);
            sums.add(v);
          }
        }
      }
      // a thread may hold more than 31 terms here: the wide warp reduction
      xyd::commit_sums<kFusedWarps, RED, true, true>(sums, n_acc, part, cnt,
                                                     rec + sweep - a.rec_sweep0, beta,
                                                     band.y_begin == 0);
    }
    // every band of the lattice has written this sweep before any reads it:
    // the cluster barrier's arrive has release and its wait acquire semantics
    // at cluster scope, which order the global stores before the next loads
    cluster.sync();
  }
}

// Replica exchange after a round (one CTA).  For every candidate pair of the
// round's parity -- ladder l, positions p and p+1 of the ladder ordered by
// beta, p = round mod 2, round mod 2 + 2, ... -- the pair swaps its two
// lattices' temperatures iff
//   u24(w0) < exp((beta_p - beta_{p+1}) (E_p - E_{p+1})),
// E = -J C of each lattice's last sweep of the round, Philox counter
// (l * 65536 + p, round, lattice_id0, 2).  Pairs of one parity never share a
// position, so they are independent.  Thread 0 then advances the round
// counters for the next launch.
__global__ void k_exchange(ExchangeArgs a) {
  const uint32_t round = a.counters[1];
  const uint32_t last_sweep = a.counters[0] + (uint32_t)a.sweeps - 1u;
  for (int i = threadIdx.x; i < a.n_pairs; i += blockDim.x) {
    const int l = a.pair_ladder[i];
    const int p = a.pair_pos[i];
    if ((p & 1) != (int)(round & 1u)) continue;
    const int base = a.ladder_start[l];
    const int la = a.pos_lattice[base + p];
    const int lb = a.pos_lattice[base + p + 1];
    const xy_record& ra = a.records[(size_t)la * a.rec_stride + (last_sweep - a.rec_sweep0)];
    const xy_record& rb = a.records[(size_t)lb * a.rec_stride + (last_sweep - a.rec_sweep0)];
    const double unit = 1.0 / (double)(1ll << XY_FX_SHIFT);
    const double Ea = -a.J * (double)ra.sum[0] * unit;
    const double Eb = -a.J * (double)rb.sum[0] * unit;
    const double ba = a.pos_beta[base + p], bb = a.pos_beta[base + p + 1];
    const uint4 w = xyd::philox4x32_10(
        make_uint4((uint32_t)l * 65536u + (uint32_t)p, round, a.lattice_id0, 2u), a.rk);
    const double u = (double)(w.x >> 8) * (1.0 / 16777216.0);
    if (u < exp((ba - bb) * (Ea - Eb))) {
      a.pos_lattice[base + p] = lb;
      a.pos_lattice[base + p + 1] = la;
      a.beta[lb] = ba;
      a.beta[la] = bb;
      a.accepted[base + p] += 1ull;
    }
    a.attempted[base + p] += 1ull;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.counters[0] += (uint32_t)a.sweeps;
    a.counters[1] += 1u;
  }
}

template <int MODE, int RED>
cudaError_t launch_round_t(const BatchArgs& a, int n_ctas, size_t smem, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_ctas, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterSize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_round<MODE, RED>, a);
}

template <int MODE, int RED>
cudaError_t launch_fused_round_t(const BatchArgs& a, int n_ctas, size_t smem, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_ctas, 1, 1);
  cfg.blockDim = dim3(kFusedThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterSize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_fused<MODE, RED>, a);
}

const void* fused_kernel_ptr(int sincos_mode, int reduce_mode) {
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? (const void*)k_batch_fused<0, 1> : (const void*)k_batch_fused<0, 0>;
    case 1: return comp ? (const void*)k_batch_fused<1, 1> : (const void*)k_batch_fused<1, 0>;
    default: return comp ? (const void*)k_batch_fused<2, 1> : (const void*)k_batch_fused<2, 0>;
  }
}

}  // namespace

size_t batch_fused_tail_bytes() {
  return sizeof(float) * kFusedWarps * 10 + sizeof(unsigned int) * kFusedWarps;
}

cudaError_t prepare_batch_fused(int sincos_mode, int reduce_mode, size_t smem) {
  return cudaFuncSetAttribute(fused_kernel_ptr(sincos_mode, reduce_mode),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_batch_fused(int sincos_mode, int reduce_mode, const BatchArgs& a, int n_ctas,
                               cudaStream_t stream) {
  if (n_ctas <= 0 || n_ctas % kClusterSize != 0 || !a.theta2) return cudaErrorInvalidValue;
  const size_t smem = a.cs_bytes + batch_fused_tail_bytes();
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_fused_round_t<0, 1>(a, n_ctas, smem, stream)
                        : launch_fused_round_t<0, 0>(a, n_ctas, smem, stream);
    case 1: return comp ? launch_fused_round_t<1, 1>(a, n_ctas, smem, stream)
                        : launch_fused_round_t<1, 0>(a, n_ctas, smem, stream);
    default: return comp ? launch_fused_round_t<2, 1>(a, n_ctas, smem, stream)
                         : launch_fused_round_t<2, 0>(a, n_ctas, smem, stream);
  }
}

size_t batch_smem_bytes(int max_stage_floats2) {
  return sizeof(float2) * (size_t)max_stage_floats2 + sizeof(float) * kWarps * 10 +
         sizeof(unsigned int) * kWarps;
}

cudaError_t prepare_batch_round(int sincos_mode, int reduce_mode, size_t smem) {
  const bool comp = reduce_mode != 0;
  const void* f;
  switch (sincos_mode) {
    case 0: f = comp ? (const void*)k_batch_round<0, 1> : (const void*)k_batch_round<0, 0>; break;
    case 1: f = comp ? (const void*)k_batch_round<1, 1> : (const void*)k_batch_round<1, 0>; break;
    default: f = comp ? (const void*)k_batch_round<2, 1> : (const void*)k_batch_round<2, 0>; break;
  }
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_batch_round(int sincos_mode, int reduce_mode, const BatchArgs& a, int n_ctas,
                               cudaStream_t stream) {
  if (n_ctas <= 0 || n_ctas % kClusterSize != 0) return cudaErrorInvalidValue;
  const size_t smem = a.cs_bytes + sizeof(float) * kWarps * 10 + sizeof(unsigned int) * kWarps;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_round_t<0, 1>(a, n_ctas, smem, stream)
                        : launch_round_t<0, 0>(a, n_ctas, smem, stream);
    case 1: return comp ? launch_round_t<1, 1>(a, n_ctas, smem, stream)
                        : launch_round_t<1, 0>(a, n_ctas, smem, stream);
    default: return comp ? launch_round_t<2, 1>(a, n_ctas, smem, stream)
                         : launch_round_t<2, 0>(a, n_ctas, smem, stream);
  }
}

cudaError_t launch_exchange(const ExchangeArgs& a, cudaStream_t stream) {
  k_exchange<<<1, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace xyk
