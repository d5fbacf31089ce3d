// xy_hmc_cluster.cu -- a whole HMC trajectory in one launch for small lattices:
// one thread-block cluster holds the lattice in shared memory.
//
// For L <= 256 every leap-frog launch of the tiled kernels costs a few
// microseconds of launch and grid latency for very little work.  Here the
// lattice (a power of two, 16 <= L <= 256) is cut into strips of 16 full
// rows, one CTA per strip and one cluster of C = L / 16 CTAs (up to 16, a
// non-portable cluster size) for the lattice.  Each CTA keeps its strip's angles and momenta in shared memory for
// the whole trajectory.  Per leap-frog step it writes its strip's unit vectors
// into one of two shared buffers (by step parity), the cluster meets at one
// barrier (release/acquire at cluster scope), and the strip's first and last
// rows read the neighbouring strips' unit vectors straight from those CTAs'
// shared memory (distributed shared memory).  Two buffers mean a CTA never
// overwrites unit vectors a neighbour may still be reading: to write a buffer
// again it must pass the next step's barrier, which the neighbour reaches only
// after its reads.  The sums go to the control block with the same exact
// fixed-point atomics as the other kernels; after a last barrier one thread
// takes the accept decision (the same device function as k_hmc_accept), and
// every CTA writes its strip back to the state buffer if it was accepted and
// its momenta in any case.  The per-site arithmetic is the shared HMC device
// code, so results are bit-identical to the tiled and per-site kernels.  The
// state stays in the buffer `cur`; only that buffer and the momenta change.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_hmc_device.cuh"
#include "xy_internal.h"

namespace cg = cooperative_groups;

namespace xyk {

namespace {

using namespace xyh;

constexpr int kStripRows = 16;
constexpr int kCThreads = 512;
constexpr int kCWarps = kCThreads / 32;

size_t cluster_smem(int L) {
  return (size_t)L * (2 * kStripRows * sizeof(float) + 2 * (kStripRows + 2) * sizeof(float2));
}

constexpr int kMaxIter = kStripRows * 256 / kCThreads;   // sites per thread at L = 256

template <int MODE>
__global__ void __launch_bounds__(kCThreads) k_hmc_traj_cluster(HmcArgs a, int n_md, int draw,
                                                                int mode, double beta, double J) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long red[kCWarps][kHmcSums];
  __shared__ int decision;
  cg::cluster_group cluster = cg::this_cluster();
  const int L = a.L;
  const int rank = (int)cluster.block_rank(), C = (int)cluster.num_blocks();
  const int up_rank = rank + 1 == C ? 0 : rank + 1;      // strip holding rows y0 + 16 ...
  const int dn_rank = rank == 0 ? C - 1 : rank - 1;      // strip holding rows ... y0 - 1
  const int y0 = rank * kStripRows;
  const int nloc = kStripRows * L;
  const int tid = threadIdx.x;
  // L is a power of two: a thread owns column x of strip rows r0, r0 + rstep, ...
  const int lgL = __ffs(L) - 1;
  const int x = tid & (L - 1);
  const int r0 = tid >> lgL, rstep = kCThreads >> lgL;
  const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
  float* th = reinterpret_cast<float*>(smem);            // [16][L]
  float* pm = th + nloc;                                 // [16][L]
  float2* cs0 = reinterpret_cast<float2*>(pm + nloc);    // [2][18][L]: row r + 1 = strip row r
  const size_t buf_len = (size_t)(kStripRows + 2) * L;

  HmcCtl* ctl = a.ctl;
  const uint32_t cur = ctl->cur;
  const uint32_t traj = (uint32_t)ctl->traj;
  float* state = hmc_buf(a, (int)cur);
#pragma unroll
  for (int k = 0; k < kMaxIter; ++k) {
    const int r = r0 + k * rstep;
    if (r < kStripRows) {
      const uint32_t site = (uint32_t)(y0 + r) * (uint32_t)L + (uint32_t)x;
      th[r * L + x] = state[site];
      pm[r * L + x] = draw ? hmc_momentum(site, traj, a.lattice_id, a.rk) : a.p_in[site];
    }
  }

  const float half = 0.5f * a.eps;
  for (int s = 0; s <= n_md; ++s) {
    float2* buf = cs0 + (size_t)(s & 1) * buf_len;
#pragma unroll
    for (int k = 0; k < kMaxIter; ++k) {
      const int r = r0 + k * rstep;
      if (r < kStripRows) {
        float sn, cn;
        xyd::unit_vector<MODE>(th[r * L + x], &sn, &cn);
        buf[(r + 1) * L + x] = make_float2(cn, sn);
      }
    }
    cluster.sync();
    const float2* up_buf = cluster.map_shared_rank(buf, up_rank);
    const float2* dn_buf = cluster.map_shared_rank(buf, dn_rank);
    const float coef = (s == 0 || s == n_md) ? half : a.eps;
    HmcAcc acc;
    acc_zero(acc);
#pragma unroll
    for (int k = 0; k < kMaxIter; ++k) {
      const int r = r0 + k * rstep;
      if (r < kStripRows) {
        const float2* row = buf + (size_t)(r + 1) * L;
        const float2 o = row[x], l = row[xl], rt = row[xr];
        const float2 dn = r > 0 ? buf[(size_t)r * L + x] : dn_buf[(size_t)kStripRows * L + x];
        const float2 up = r < kStripRows - 1 ? buf[(size_t)(r + 2) * L + x] : up_buf[(size_t)L + x];
        const float Sc = xyd::nb_sum(l.x, rt.x, dn.x, up.x);
        const float Ss = xyd::nb_sum(l.y, rt.y, dn.y, up.y);
        const float F = hmc_force(o.x, o.y, Sc, Ss, a.K);
        const int i = r * L + x;
        if (s == 0) hmc_terms(pm[i], o.x, o.y, rt.x, rt.y, up.x, up.y, acc);
        const float p = __fmaf_rn(coef, F, pm[i]);
        pm[i] = p;
        if (s == n_md) {
          hmc_terms(p, o.x, o.y, rt.x, rt.y, up.x, up.y, acc);
        } else {
          th[i] = hmc_wrap(__fmaf_rn(a.eps, p, th[i]));
        }
      }
    }
    if (s == 0) hmc_commit<kCWarps>(acc, ctl->acc[0], red);
    if (s == n_md) hmc_commit<kCWarps>(acc, ctl->acc[1], red);
  }
  // every CTA's sums are in: one thread decides
  cluster.sync();
  if (rank == 0 && tid == 0) decision = hmc_decide(ctl, a.lattice_id, a.rk, mode, beta, J) ? 1 : 0;
  cluster.sync();
  const int take = *cluster.map_shared_rank(&decision, 0);
#pragma unroll
  for (int k = 0; k < kMaxIter; ++k) {
    const int r = r0 + k * rstep;
    if (r < kStripRows) {
      const size_t site = (size_t)(y0 + r) * L + x;
      if (take) state[site] = th[r * L + x];
      a.p_out[site] = pm[r * L + x];
    }
  }
  // rank 0's decision word is read remotely: it must outlive those reads
  cluster.sync();
}

template <int MODE>
cudaError_t launch_cluster_t(const HmcArgs& a, int n_md, int draw, int mode, double beta, double J,
                             cudaStream_t stream) {
  const int C = a.L / kStripRows;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kCThreads, 1, 1);
  cfg.dynamicSmemBytes = cluster_smem(a.L);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_hmc_traj_cluster<MODE>, a, n_md, draw, mode, beta, J);
}

}  // namespace

bool hmc_cluster_ok(int L) { return L >= kStripRows && L <= 256 && (L & (L - 1)) == 0; }

cudaError_t hmc_cluster_prepare(int sincos_mode) {
  const void* f = sincos_mode == 0 ? (const void*)k_hmc_traj_cluster<0>
                                   : (sincos_mode == 1 ? (const void*)k_hmc_traj_cluster<1>
                                                       : (const void*)k_hmc_traj_cluster<2>);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cluster_smem(256));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t launch_hmc_cluster(int sincos_mode, const HmcArgs& a, int n_md, int draw, int mode,
                               double beta, double J, cudaStream_t stream) {
  if (!hmc_cluster_ok(a.L) || n_md < 1) return cudaErrorInvalidValue;
  switch (sincos_mode) {
    case 0: return launch_cluster_t<0>(a, n_md, draw, mode, beta, J, stream);
    case 1: return launch_cluster_t<1>(a, n_md, draw, mode, beta, J, stream);
    default: return launch_cluster_t<2>(a, n_md, draw, mode, beta, J, stream);
  }
}

}  // namespace xyk
