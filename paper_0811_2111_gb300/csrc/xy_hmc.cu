// xy_hmc.cu -- Hybrid Monte Carlo for the 2-d XY model (Sec. 1.2 of the
// paper): Gaussian momenta, the leap-frog integration of the equations of
// motion (the parallel core of the method) and the global Metropolis test.
//
//   H_hmc = sum_s p_s^2 / 2 + beta H(theta),  F_s = -beta J sum_nn sin(t_s - t_j)
//
// A trajectory of n_md steps is a chain of launches plus the test:
//   begin   draw p (Philox domain 3, Box-Muller), sums of (theta_0, p_0),
//           p += eps/2 F(theta_0), theta_1 = theta_0 + eps p
//   step    p += eps F(theta_k), theta_{k+1} = theta_k + eps p; on the tiled
//           path two such steps per launch (halo of two recomputed), one
//           single step for an odd remainder
//   final   p += eps/2 F(theta_n), sums of (theta_n, p_n)
//   accept  one thread: dH from the exact fixed-point sums, u < exp(-dH)
// Three angle buffers: the state stays untouched in buffer `cur` (restored on
// rejection for free), the integration ping-pongs between the other two, and
// the accept kernel moves `cur` on the device, so trajectories replay as one
// captured graph with no host round trip.  Sums are formed per site in FP32
// and converted to 64-bit fixed point before any addition: exact, and the
// same for every launch shape (the tiled and per-site kernels agree bit for
// bit in angles, momenta and sums).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "xy_hmc_device.cuh"
#include "xy_internal.h"
#include "xy_tma.cuh"

namespace xyk {

namespace {

using namespace xyh;

// ---------------------------------------------------------------------------
// Tiled kernel: a CTA of 256 threads owns 32 rows x 128 columns; a thread owns
// 4 rows x 4 columns (one float4 per row).  Horizontal neighbours come from
// the neighbouring lanes by shuffle (the warp's edge lanes read the tile's
// halo columns from shared memory); vertical neighbours from the thread's own
// rows, or from the edge rows that every warp leaves in shared memory (the
// tile's halo rows included).  Halo unit vectors are recomputed, not exchanged.
// ---------------------------------------------------------------------------
constexpr int kTileRows = 32;
constexpr int kTileCols = 128;
constexpr int kTileThreads = 256;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kRowsPerThread = kTileRows / kTileWarps;   // 4

template <int MODE, int KIND>
__global__ void __launch_bounds__(kTileThreads, KIND == kHmcStep ? 3 : 2) k_hmc_tile(HmcArgs a) {
  // cos / sin of tile rows -1 .. 32 (index row + 1); only each warp's first and
  // last row and the two halo rows are written and read
  __shared__ __align__(16) float sh_c[kTileRows + 2][kTileCols];
  __shared__ __align__(16) float sh_s[kTileRows + 2][kTileCols];
  __shared__ float side_c[2][kTileRows];   // [0] column -1, [1] column 128
  __shared__ float side_s[2][kTileRows];
  __shared__ long long red[kTileWarps][kHmcSums];

  const int L = a.L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kTileCols, y0 = blockIdx.y * kTileRows;
  const uint32_t cur = a.ctl->cur;
  int src, dst;
  hmc_buffers(a, cur, &src, &dst);
  const float* __restrict__ th_src = hmc_buf(a, src);

  // ---- loads: own 4 x 4 block, then halo sites ---------------------------
  const int xb = x0 + 4 * lane;
  const int yb = y0 + kRowsPerThread * warp;
  float4 t4[kRowsPerThread], p4[kRowsPerThread];
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r)
    t4[r] = *reinterpret_cast<const float4*>(th_src + (size_t)(yb + r) * L + xb);
  if (KIND != kHmcBeginDraw) {
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r)
      p4[r] = *reinterpret_cast<const float4*>(a.p_in + (size_t)(yb + r) * L + xb);
  }
  // halo: threads 0..127 row y0-1, 128..255 row y0+32; threads 0..31 column
  // x0-1 and 32..63 column x0+128 (rows y0..y0+31)
  const int tid = threadIdx.x;
  const int hy = tid < kTileCols ? (y0 == 0 ? L - 1 : y0 - 1)
                                 : (y0 + kTileRows == L ? 0 : y0 + kTileRows);
  const int hx = x0 + (tid & (kTileCols - 1));
  const float th_row = th_src[(size_t)hy * L + hx];
  float th_side = 0.f;
  const bool side = tid < 64;
  if (side) {
    const int sx = tid < 32 ? (x0 == 0 ? L - 1 : x0 - 1) : (x0 + kTileCols == L ? 0 : x0 + kTileCols);
    th_side = th_src[(size_t)(y0 + (tid & 31)) * L + sx];
  }

  // ---- momenta of the trajectory (begin with draw) -------------------------
  if (KIND == kHmcBeginDraw) {
    const uint32_t traj = (uint32_t)a.ctl->traj;
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r) {
      const uint32_t s0 = (uint32_t)(yb + r) * (uint32_t)L + (uint32_t)xb;
      p4[r].x = hmc_momentum(s0 + 0u, traj, a.lattice_id, a.rk);
      p4[r].y = hmc_momentum(s0 + 1u, traj, a.lattice_id, a.rk);
      p4[r].z = hmc_momentum(s0 + 2u, traj, a.lattice_id, a.rk);
      p4[r].w = hmc_momentum(s0 + 3u, traj, a.lattice_id, a.rk);
    }
  }

  // ---- unit vectors -------------------------------------------------------
  float c[kRowsPerThread][4], s[kRowsPerThread][4];
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r) {
    xyd::unit_vector<MODE>(t4[r].x, &s[r][0], &c[r][0]);
    xyd::unit_vector<MODE>(t4[r].y, &s[r][1], &c[r][1]);
    xyd::unit_vector<MODE>(t4[r].z, &s[r][2], &c[r][2]);
    xyd::unit_vector<MODE>(t4[r].w, &s[r][3], &c[r][3]);
  }
  {
    float hs, hc;
    xyd::unit_vector<MODE>(th_row, &hs, &hc);
    const int row = tid < kTileCols ? 0 : kTileRows + 1;
    sh_c[row][tid & (kTileCols - 1)] = hc;
    sh_s[row][tid & (kTileCols - 1)] = hs;
    if (side) {
      xyd::unit_vector<MODE>(th_side, &hs, &hc);
      side_c[tid >> 5][tid & 31] = hc;
      side_s[tid >> 5][tid & 31] = hs;
    }
  }
  // first and last row of this warp's band
  {
    const int rf = kRowsPerThread * warp + 1, rl = kRowsPerThread * warp + kRowsPerThread;
    *reinterpret_cast<float4*>(&sh_c[rf][4 * lane]) = make_float4(c[0][0], c[0][1], c[0][2], c[0][3]);
    *reinterpret_cast<float4*>(&sh_s[rf][4 * lane]) = make_float4(s[0][0], s[0][1], s[0][2], s[0][3]);
    *reinterpret_cast<float4*>(&sh_c[rl][4 * lane]) = make_float4(c[3][0], c[3][1], c[3][2], c[3][3]);
    *reinterpret_cast<float4*>(&sh_s[rl][4 * lane]) = make_float4(s[3][0], s[3][1], s[3][2], s[3][3]);
  }
  __syncthreads();

  // rows below (y - 1) and above (y + 4) the band
  const int rb = kRowsPerThread * warp;                  // index of row yb - 1
  const int ra = kRowsPerThread * warp + kRowsPerThread + 1;   // index of row yb + 4
  const float4 cdn = *reinterpret_cast<const float4*>(&sh_c[rb][4 * lane]);
  const float4 sdn = *reinterpret_cast<const float4*>(&sh_s[rb][4 * lane]);
  const float4 cup = *reinterpret_cast<const float4*>(&sh_c[ra][4 * lane]);
  const float4 sup = *reinterpret_cast<const float4*>(&sh_s[ra][4 * lane]);
  const float cdn_a[4] = {cdn.x, cdn.y, cdn.z, cdn.w}, sdn_a[4] = {sdn.x, sdn.y, sdn.z, sdn.w};
  const float cup_a[4] = {cup.x, cup.y, cup.z, cup.w}, sup_a[4] = {sup.x, sup.y, sup.z, sup.w};

  HmcAcc acc;
  acc_zero(acc);
  float4 tn[kRowsPerThread];
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r) {
    // horizontal neighbours of the row's first and last column
    float cl = __shfl_up_sync(0xffffffffu, c[r][3], 1);
    float sl = __shfl_up_sync(0xffffffffu, s[r][3], 1);
    float cr = __shfl_down_sync(0xffffffffu, c[r][0], 1);
    float sr = __shfl_down_sync(0xffffffffu, s[r][0], 1);
    const int row = kRowsPerThread * warp + r;
    if (lane == 0) {
      cl = side_c[0][row];
      sl = side_s[0][row];
    }
    if (lane == 31) {
      cr = side_c[1][row];
      sr = side_s[1][row];
    }
    float pr[4] = {p4[r].x, p4[r].y, p4[r].z, p4[r].w};
    const float tr[4] = {t4[r].x, t4[r].y, t4[r].z, t4[r].w};
    float out[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float nlc = j == 0 ? cl : c[r][j - 1], nls = j == 0 ? sl : s[r][j - 1];
      const float nrc = j == 3 ? cr : c[r][j + 1], nrs = j == 3 ? sr : s[r][j + 1];
      const float ndc = r == 0 ? cdn_a[j] : c[r - 1][j], nds = r == 0 ? sdn_a[j] : s[r - 1][j];
      const float nuc = r == kRowsPerThread - 1 ? cup_a[j] : c[r + 1][j];
      const float nus = r == kRowsPerThread - 1 ? sup_a[j] : s[r + 1][j];
      const float Sc = xyd::nb_sum(nlc, nrc, ndc, nuc);
      const float Ss = xyd::nb_sum(nls, nrs, nds, nus);
      const float F = hmc_force(c[r][j], s[r][j], Sc, Ss, a.K);
      if (KIND == kHmcBeginDraw || KIND == kHmcBeginRead)
        hmc_terms(pr[j], c[r][j], s[r][j], nrc, nrs, nuc, nus, acc);
      pr[j] = __fmaf_rn(a.a, F, pr[j]);
      if (KIND == kHmcFinal) {
        hmc_terms(pr[j], c[r][j], s[r][j], nrc, nrs, nuc, nus, acc);
        out[j] = tr[j];
      } else {
        out[j] = hmc_wrap(__fmaf_rn(a.eps, pr[j], tr[j]));
      }
    }
    p4[r] = make_float4(pr[0], pr[1], pr[2], pr[3]);
    tn[r] = make_float4(out[0], out[1], out[2], out[3]);
  }

  // ---- stores -------------------------------------------------------------
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r)
    *reinterpret_cast<float4*>(a.p_out + (size_t)(yb + r) * L + xb) = p4[r];
  if (KIND != kHmcFinal) {
    float* __restrict__ th_dst = hmc_buf(a, dst);
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r)
      *reinterpret_cast<float4*>(th_dst + (size_t)(yb + r) * L + xb) = tn[r];
  }
  if (KIND == kHmcBeginDraw || KIND == kHmcBeginRead)
    hmc_commit<kTileWarps>(acc, a.ctl->acc[0], red);
  if (KIND == kHmcFinal) hmc_commit<kTileWarps>(acc, a.ctl->acc[1], red);
}

// ---------------------------------------------------------------------------
// Persistent TMA step kernel: the same step as k_hmc_tile<MODE, kHmcStep>, but
// a grid of about two CTAs per SM walks the tiles, and each CTA streams its
// next tiles' angles and momenta (two 32 x 128 boxes, 32 KB) into a
// double-buffered shared-memory stage with cp.async.bulk.tensor, completing on
// an mbarrier, while it computes the current tile.  The one-site halo (320
// floats) is read with plain loads issued before the wait.  Every wait is
// bounded: each thread polls the stage's barrier a fixed number of times; a
// thread that runs out flags HmcCtl::error and stops computing but keeps
// meeting the CTA's barriers, and thread 0 then issues no more loads and
// drains the ones in flight before the CTA exits.
// ---------------------------------------------------------------------------
// ROWS rows per thread: tiles of 8 ROWS x 128 sites.  ROWS = 4 (the tile of
// k_hmc_tile, two CTAs per SM) is the one launched: 16 x 128 tiles at four
// CTAs per SM measured slower (57.4 against 54.1 us per step at L = 4096; the
// halo grows from 8 % to 14 % of the sincos work and occupancy was not the
// limit).
template <int ROWS>
struct TmaGeom {
  static constexpr int kRows = 8 * ROWS;                               // tile rows
  static constexpr int kBox = kRows * kTileCols;                       // floats per box
  static constexpr uint32_t kStageBytes = 2u * kBox * sizeof(float);  // angles + momenta
  static constexpr size_t kSmem = 2 * (size_t)kStageBytes;             // two stages
  static constexpr int kMinBlocks = ROWS == 4 ? 2 : 4;
};
constexpr long long kSpinLimit = 1ll << 22;

template <int MODE, int ROWS>
__global__ void __launch_bounds__(kTileThreads, TmaGeom<ROWS>::kMinBlocks)
    k_hmc_step_tma(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                   const __grid_constant__ CUtensorMap map2, const __grid_constant__ CUtensorMap mapp,
                   HmcArgs a, int tiles_x, int n_tiles) {
  using G = TmaGeom<ROWS>;
  constexpr int TR = G::kRows;
  constexpr uint32_t kTmaStageBytes = G::kStageBytes;
  constexpr int kTmaBox = G::kBox;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  // unit vectors (cos and sin planes) of the rows other warps read,
  // double-buffered by tile parity: lastrow[b][w + 1] = last row of warp w
  // (lastrow[b][0]: the halo row above the tile), firstrow[b][w] = first row of
  // warp w (firstrow[b][kTileWarps]: the halo row below); plus the halo columns
  __shared__ __align__(16) float lastrow_c[2][kTileWarps + 1][kTileCols];
  __shared__ __align__(16) float lastrow_s[2][kTileWarps + 1][kTileCols];
  __shared__ __align__(16) float firstrow_c[2][kTileWarps + 1][kTileCols];
  __shared__ __align__(16) float firstrow_s[2][kTileWarps + 1][kTileCols];
  __shared__ float2 side[2][2][TR];
  __shared__ __align__(8) uint64_t bar[2];

  const int L = a.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int src, dst;
  hmc_buffers(a, a.ctl->cur, &src, &dst);
  const CUtensorMap* mth = src == 0 ? &map0 : (src == 1 ? &map1 : &map2);
  const float* __restrict__ th_src = hmc_buf(a, src);
  float* __restrict__ th_dst = hmc_buf(a, dst);
  // stage s: angles [TR][128] then momenta [TR][128]
  auto stage_th = [&](int s) {
    return reinterpret_cast<float (*)[kTileCols]>(tma_smem + s * kTmaStageBytes);
  };
  auto stage_p = [&](int s) {
    return reinterpret_cast<float (*)[kTileCols]>(tma_smem + s * kTmaStageBytes +
                                                 kTmaBox * sizeof(float));
  };
  // Consecutive steps (buffer offsets 1, 2, 1, ...) walk the tiles in
  // opposite orders, so a step starts with the tiles the launch before it
  // wrote last, which are still in L2.  Every tile reads only the source
  // buffer and its own momenta, so the order changes no result.
  const bool rev = (a.src_off & 1) != 0;
  auto tile_at = [&](int t) { return rev ? n_tiles - 1 - t : t; };
  // thread 0's count of loads issued per stage (for the drain on a timeout)
  int issued[2] = {0, 0};
  auto issue = [&](int t, int s) {
    const int tt = tile_at(t);
    const int x0 = (tt % tiles_x) * kTileCols, y0 = (tt / tiles_x) * TR;
    xyt::mbar_arrive_expect_tx(&bar[s], kTmaStageBytes);
    xyt::tma_load_2d(stage_th(s), mth, x0, y0, &bar[s]);
    xyt::tma_load_2d(stage_p(s), &mapp, x0, y0, &bar[s]);
    ++issued[s];
  };
  auto bounded_wait = [&](int s, uint32_t parity) {
    return xyt::mbar_wait_bounded(&bar[s], parity, kSpinLimit);
  };

  if (tid == 0) {
    xyt::mbar_init(&bar[0], 1);
    xyt::mbar_init(&bar[1], 1);
    xyt::fence_mbarrier_init();
    xyt::fence_async_shared();
    for (int s = 0; s < 2; ++s) {
      const int t = blockIdx.x + s * gridDim.x;
      if (t < n_tiles) issue(t, s);
    }
  }
  __syncthreads();

  // A thread whose wait runs out flags the error and stops computing, but
  // keeps meeting the CTA's barriers (so no thread waits on one that left);
  // thread 0 then issues no more loads and drains the ones in flight.
  bool ok = true;
  int it = 0;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
    const int s = it & 1, b = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const int tt = tile_at(t);
    const int x0 = (tt % tiles_x) * kTileCols, y0 = (tt / tiles_x) * TR;
    // halo loads first: rows y0-1, y0+TR (threads 0..127 / 128..255), columns
    // x0-1 and x0+128 (threads 0..TR-1 / TR..2TR-1)
    const int hy = tid < kTileCols ? (y0 == 0 ? L - 1 : y0 - 1) : (y0 + TR == L ? 0 : y0 + TR);
    const float th_row = th_src[(size_t)hy * L + x0 + (tid & (kTileCols - 1))];
    float th_side = 0.f;
    const bool is_side = tid < 2 * TR;
    if (is_side) {
      const int sx = tid < TR ? (x0 == 0 ? L - 1 : x0 - 1) : (x0 + kTileCols == L ? 0 : x0 + kTileCols);
      th_side = th_src[(size_t)(y0 + (tid % TR)) * L + sx];
    }
    if (ok && !bounded_wait(s, parity)) {
      ok = false;
      atomicOr(&a.ctl->error, 1u);
    }

    const int xb = 4 * lane, rb0 = ROWS * warp;
    float4 t4[ROWS], p4[ROWS];
    float c[ROWS][4], sn[ROWS][4];
    if (ok) {
      float (*sth)[kTileCols] = stage_th(s);
      float (*sp)[kTileCols] = stage_p(s);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        t4[r] = *reinterpret_cast<const float4*>(&sth[rb0 + r][xb]);
        p4[r] = *reinterpret_cast<const float4*>(&sp[rb0 + r][xb]);
      }
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        xyd::unit_vector<MODE>(t4[r].x, &sn[r][0], &c[r][0]);
        xyd::unit_vector<MODE>(t4[r].y, &sn[r][1], &c[r][1]);
        xyd::unit_vector<MODE>(t4[r].z, &sn[r][2], &c[r][2]);
        xyd::unit_vector<MODE>(t4[r].w, &sn[r][3], &c[r][3]);
      }
      float hs, hc;
      xyd::unit_vector<MODE>(th_row, &hs, &hc);
      if (tid < kTileCols) {
        lastrow_c[b][0][tid] = hc;
        lastrow_s[b][0][tid] = hs;
      } else {
        firstrow_c[b][kTileWarps][tid - kTileCols] = hc;
        firstrow_s[b][kTileWarps][tid - kTileCols] = hs;
      }
      if (is_side) {
        xyd::unit_vector<MODE>(th_side, &hs, &hc);
        side[b][tid / TR][tid % TR] = make_float2(hc, hs);
      }
      *reinterpret_cast<float4*>(&firstrow_c[b][warp][xb]) = make_float4(c[0][0], c[0][1], c[0][2], c[0][3]);
      *reinterpret_cast<float4*>(&firstrow_s[b][warp][xb]) =
          make_float4(sn[0][0], sn[0][1], sn[0][2], sn[0][3]);
      *reinterpret_cast<float4*>(&lastrow_c[b][warp + 1][xb]) =
          make_float4(c[ROWS - 1][0], c[ROWS - 1][1], c[ROWS - 1][2], c[ROWS - 1][3]);
      *reinterpret_cast<float4*>(&lastrow_s[b][warp + 1][xb]) =
          make_float4(sn[ROWS - 1][0], sn[ROWS - 1][1], sn[ROWS - 1][2], sn[ROWS - 1][3]);
    }
    __syncthreads();   // stage s fully read; edges visible
    if (tid == 0 && ok) {
      const int tn = t + 2 * gridDim.x;
      if (tn < n_tiles) {
        xyt::fence_async_shared();
        issue(tn, s);
      }
    }
    if (!ok) continue;

    const float4 cdn = *reinterpret_cast<const float4*>(&lastrow_c[b][warp][xb]);
    const float4 sdn = *reinterpret_cast<const float4*>(&lastrow_s[b][warp][xb]);
    const float4 cup = *reinterpret_cast<const float4*>(&firstrow_c[b][warp + 1][xb]);
    const float4 sup = *reinterpret_cast<const float4*>(&firstrow_s[b][warp + 1][xb]);
    const float cdn_a[4] = {cdn.x, cdn.y, cdn.z, cdn.w}, sdn_a[4] = {sdn.x, sdn.y, sdn.z, sdn.w};
    const float cup_a[4] = {cup.x, cup.y, cup.z, cup.w}, sup_a[4] = {sup.x, sup.y, sup.z, sup.w};
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      float cl = __shfl_up_sync(0xffffffffu, c[r][3], 1);
      float sl = __shfl_up_sync(0xffffffffu, sn[r][3], 1);
      float cr = __shfl_down_sync(0xffffffffu, c[r][0], 1);
      float sr = __shfl_down_sync(0xffffffffu, sn[r][0], 1);
      const int row = rb0 + r;
      if (lane == 0) {
        const float2 v = side[b][0][row];
        cl = v.x;
        sl = v.y;
      }
      if (lane == 31) {
        const float2 v = side[b][1][row];
        cr = v.x;
        sr = v.y;
      }
      float pr[4] = {p4[r].x, p4[r].y, p4[r].z, p4[r].w};
      const float tr[4] = {t4[r].x, t4[r].y, t4[r].z, t4[r].w};
      float out[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float nlc = j == 0 ? cl : c[r][j - 1], nls = j == 0 ? sl : sn[r][j - 1];
        const float nrc = j == 3 ? cr : c[r][j + 1], nrs = j == 3 ? sr : sn[r][j + 1];
        const float ndc = r == 0 ? cdn_a[j] : c[r - 1][j], nds = r == 0 ? sdn_a[j] : sn[r - 1][j];
        const float nuc = r == ROWS - 1 ? cup_a[j] : c[r + 1][j];
        const float nus = r == ROWS - 1 ? sup_a[j] : sn[r + 1][j];
        const float Sc = xyd::nb_sum(nlc, nrc, ndc, nuc);
        const float Ss = xyd::nb_sum(nls, nrs, nds, nus);
        pr[j] = __fmaf_rn(a.a, hmc_force(c[r][j], sn[r][j], Sc, Ss, a.K), pr[j]);
        out[j] = hmc_wrap(__fmaf_rn(a.eps, pr[j], tr[j]));
      }
      const size_t g = (size_t)(y0 + row) * L + x0 + xb;
      *reinterpret_cast<float4*>(a.p_out + g) = make_float4(pr[0], pr[1], pr[2], pr[3]);
      *reinterpret_cast<float4*>(th_dst + g) = make_float4(out[0], out[1], out[2], out[3]);
    }
  }
  // loads still in flight after a timeout land in this CTA's shared memory:
  // wait for them (bounded) before the CTA exits
  if (tid == 0 && !ok) {
    for (int q = 0; q < 2; ++q)
      if (issued[q] > 0) (void)bounded_wait(q, (uint32_t)((issued[q] - 1) & 1));
  }
}

// ---------------------------------------------------------------------------
// All kick-drift steps of a trajectory in one cooperative launch (every CTA
// resident).  The work items (step j, tile) are ordered step-major, with the
// tile rows of a step visited folded (0, T-1, 1, T-2, ...) so that a tile's
// periodic neighbours are never more than two tile rows apart in that order;
// iteration i of CTA b takes item b + i * gridDim.x, so every CTA gets the
// same number of tiles to within one over the whole trajectory.  Step j of a
// tile reads the angles of the tile and of its one-site halo after step j - 1
// (its eight neighbours), its own momenta (updated in place by its step j - 1,
// which may have run on another CTA) and overwrites the angle buffer those
// nine tiles read during step j - 1, so it starts once the nine have published
// flags >= j.  A tile is published (j + 1) after the next tile's first CTA
// barrier, when its stores have long landed and the fence is cheap, or before
// that tile waits; either way without waiting on anything else.  Thread 0
// streams the next-but-one tile's angle and momentum boxes into the free TMA
// stage once that item's nine counters are found set (relaxed loads issued
// when the stage frees, looked at once the current tile is computed, then an
// acquire fence; at large L they are always set); otherwise the load is
// issued at the item's own turn, after a bounded wait.  Every wait is bounded
// (counters and stage barriers); a wait that runs out sets HmcCtl::error, the
// CTA drains its loads in flight (bounded) and ends, and CTAs waiting on it see
// the error word and end too.  Items wait only on items of the step before,
// and a finished item is published without waiting, so with every CTA
// resident every wait ends.  Per tile the arithmetic is k_hmc_step_tma's, so
// the trajectory is bit for bit that of one step launch per step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int hmc_load_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int hmc_load_relaxed(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void hmc_store_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}


__device__ __forceinline__ int hmc_wrap_tile(int v, int n) {
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}

template <int MODE>
__global__ void __launch_bounds__(kTileThreads, TmaGeom<4>::kMinBlocks)
    k_hmc_steps_persist(const __grid_constant__ CUtensorMap map0,
                        const __grid_constant__ CUtensorMap map1,
                        const __grid_constant__ CUtensorMap map2,
                        const __grid_constant__ CUtensorMap mapp, HmcStepsArgs q, int tiles_x,
                        int n_tiles) {
  using G = TmaGeom<4>;
  constexpr int ROWS = 4;
  constexpr int TR = G::kRows;
  constexpr uint32_t kTmaStageBytes = G::kStageBytes;
  constexpr int kTmaBox = G::kBox;
  constexpr int kPublisher = kTileThreads - 32;   // lane 0 of the last warp
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(16) float lastrow_c[2][kTileWarps + 1][kTileCols];
  __shared__ __align__(16) float lastrow_s[2][kTileWarps + 1][kTileCols];
  __shared__ __align__(16) float firstrow_c[2][kTileWarps + 1][kTileCols];
  __shared__ __align__(16) float firstrow_s[2][kTileWarps + 1][kTileCols];
  __shared__ float2 side[2][2][TR];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_issued[2];        // the stage's load for its next item is in flight
  __shared__ int s_abort;

  const HmcArgs& a = q.a;
  const int L = a.L;
  const int tiles_y = L / TR;
  const int total = q.n_steps * n_tiles;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t cur = a.ctl->cur;
  auto stage_th = [&](int s) {
    return reinterpret_cast<float (*)[kTileCols]>(tma_smem + s * kTmaStageBytes);
  };
  auto stage_p = [&](int s) {
    return reinterpret_cast<float (*)[kTileCols]>(tma_smem + s * kTmaStageBytes +
                                                 kTmaBox * sizeof(float));
  };
  // item -> (step, tile x, tile y); iteration it of this CTA takes item
  // blockIdx.x + it * gridDim.x
  auto decode = [&](int item, int* j, int* tx, int* ty) {
    *j = item / n_tiles;
    const int k = item - *j * n_tiles;
    const int prow = k / tiles_x;
    *tx = k - prow * tiles_x;
    *ty = (prow & 1) ? tiles_y - 1 - (prow >> 1) : (prow >> 1);
  };
  // angle buffers of step j: read (cur + 1 or 2), written (cur + 2 or 1)
  auto src_of = [&](int j) { return (int)((cur + (j & 1 ? 2u : 1u)) % 3u); };
  auto dst_of = [&](int j) { return (int)((cur + (j & 1 ? 1u : 2u)) % 3u); };
  int issued[2] = {0, 0};            // thread 0: loads issued per stage (for the drain)
  auto issue = [&](int item, int s) {
    int j, tx, ty;
    decode(item, &j, &tx, &ty);
    const int sb = src_of(j);
    const CUtensorMap* mth = sb == 0 ? &map0 : (sb == 1 ? &map1 : &map2);
    xyt::fence_proxy_async_global();
    xyt::mbar_arrive_expect_tx(&bar[s], kTmaStageBytes);
    xyt::tma_load_2d(stage_th(s), mth, tx * kTileCols, ty * TR, &bar[s]);
    xyt::tma_load_2d(stage_p(s), &mapp, tx * kTileCols, ty * TR, &bar[s]);
    ++issued[s];
  };
  auto drain = [&]() {
    if (tid == 0)
      for (int s = 0; s < 2; ++s)
        if (issued[s] > 0) (void)xyt::mbar_wait_bounded(&bar[s], (uint32_t)((issued[s] - 1) & 1),
                                                   q.spin_limit);
  };
  // the previous tile, stored but not yet published (its counter slot and value)
  int pend_slot = -1;
  unsigned int pend_val = 0;
  // publish it: the caller has passed a CTA barrier after every thread's stores
  // of that tile; the GPU-scope release is cumulative over them
  auto publish = [&]() {
    if (tid == kPublisher && pend_slot >= 0) hmc_store_release(q.flags + pend_slot, pend_val);
    pend_slot = -1;
  };

  if (tid == 0) {
    s_abort = 0;
    xyt::mbar_init(&bar[0], 1);
    xyt::mbar_init(&bar[1], 1);
    xyt::fence_mbarrier_init();
    xyt::fence_async_shared();
    for (int s = 0; s < 2; ++s) {
      const int item = blockIdx.x + s * gridDim.x;
      s_issued[s] = 0;
      int j, tx, ty;
      if (item < total) {
        decode(item, &j, &tx, &ty);
        if (j == 0) {            // the first step reads the begin launch's output
          issue(item, s);
          s_issued[s] = 1;
        }
      }
    }
  }
  __syncthreads();

  for (int it = 0;; ++it) {
    const int item = blockIdx.x + it * gridDim.x;
    if (item >= total) break;
    const int s = it & 1, b = it & 1;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    int j, tx, ty;
    decode(item, &j, &tx, &ty);
    const int x0 = tx * kTileCols, y0 = ty * TR;

    if (!s_issued[s]) {
      // its load was not issued ahead: publish the previous tile (this wait may
      // be for it), wait for the nine counters, then load
      __syncthreads();
      publish();
      if (j > 0 && tid < 9) {
        const int nx = hmc_wrap_tile(tx + tid % 3 - 1, tiles_x);
        const int ny = hmc_wrap_tile(ty + tid / 3 - 1, tiles_y);
        const unsigned int* f = q.flags + (ny * tiles_x + nx);
        long long n = 0;
        while (hmc_load_acquire(f) < (unsigned int)j) {
          if (++n > q.spin_limit ||
              ((n & 255) == 0 && *reinterpret_cast<volatile unsigned int*>(&a.ctl->error) != 0u)) {
            atomicOr(&a.ctl->error, 1u);
            s_abort = 1;
            break;
          }
          __nanosleep(128);
        }
      }
      __syncthreads();
      if (s_abort) {
        drain();
        return;
      }
      if (tid == 0) issue(item, s);
    }

    const float* __restrict__ th_src = hmc_buf(a, src_of(j));
    float* __restrict__ th_dst = hmc_buf(a, dst_of(j));
    // halo: rows y0-1, y0+TR (threads 0..127 / 128..255), columns x0-1 and
    // x0+128 (threads 0..TR-1 / TR..2TR-1), through L2 (written in this launch)
    const int hy = tid < kTileCols ? (y0 == 0 ? L - 1 : y0 - 1) : (y0 + TR == L ? 0 : y0 + TR);
    const float th_row = __ldcg(th_src + (size_t)hy * L + x0 + (tid & (kTileCols - 1)));
    float th_side = 0.f;
    const bool is_side = tid < 2 * TR;
    if (is_side) {
      const int sx = tid < TR ? (x0 == 0 ? L - 1 : x0 - 1) : (x0 + kTileCols == L ? 0 : x0 + kTileCols);
      th_side = __ldcg(th_src + (size_t)(y0 + (tid % TR)) * L + sx);
    }
    if (!xyt::mbar_wait_bounded(&bar[s], parity, q.spin_limit)) {
      atomicOr(&a.ctl->error, 1u);
      s_abort = 1;
    }

    const int xb = 4 * lane, rb0 = ROWS * warp;
    float4 t4[ROWS], p4[ROWS];
    float c[ROWS][4], sn[ROWS][4];
    {
      float (*sth)[kTileCols] = stage_th(s);
      float (*sp)[kTileCols] = stage_p(s);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        t4[r] = *reinterpret_cast<const float4*>(&sth[rb0 + r][xb]);
        p4[r] = *reinterpret_cast<const float4*>(&sp[rb0 + r][xb]);
      }
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        xyd::unit_vector<MODE>(t4[r].x, &sn[r][0], &c[r][0]);
        xyd::unit_vector<MODE>(t4[r].y, &sn[r][1], &c[r][1]);
        xyd::unit_vector<MODE>(t4[r].z, &sn[r][2], &c[r][2]);
        xyd::unit_vector<MODE>(t4[r].w, &sn[r][3], &c[r][3]);
      }
      float hs, hc;
      xyd::unit_vector<MODE>(th_row, &hs, &hc);
      if (tid < kTileCols) {
        lastrow_c[b][0][tid] = hc;
        lastrow_s[b][0][tid] = hs;
      } else {
        firstrow_c[b][kTileWarps][tid - kTileCols] = hc;
        firstrow_s[b][kTileWarps][tid - kTileCols] = hs;
      }
      if (is_side) {
        xyd::unit_vector<MODE>(th_side, &hs, &hc);
        side[b][tid / TR][tid % TR] = make_float2(hc, hs);
      }
      *reinterpret_cast<float4*>(&firstrow_c[b][warp][xb]) = make_float4(c[0][0], c[0][1], c[0][2], c[0][3]);
      *reinterpret_cast<float4*>(&firstrow_s[b][warp][xb]) =
          make_float4(sn[0][0], sn[0][1], sn[0][2], sn[0][3]);
      *reinterpret_cast<float4*>(&lastrow_c[b][warp + 1][xb]) =
          make_float4(c[ROWS - 1][0], c[ROWS - 1][1], c[ROWS - 1][2], c[ROWS - 1][3]);
      *reinterpret_cast<float4*>(&lastrow_s[b][warp + 1][xb]) =
          make_float4(sn[ROWS - 1][0], sn[ROWS - 1][1], sn[ROWS - 1][2], sn[ROWS - 1][3]);
    }
    __syncthreads();   // stage s fully read; edges visible; the previous tile's stores done
    if (s_abort) {
      drain();
      return;
    }
    publish();
    // the item after next: its nine counters are loaded now (relaxed, all in
    // flight together) and looked at once this tile is computed
    const int next = item + 2 * gridDim.x;
    unsigned int fl[9];
    int nj = 0;
    if (tid == 0) {
      s_issued[s] = 0;
      if (next < total) {
        int ntx, nty;
        decode(next, &nj, &ntx, &nty);
        if (nj > 0) {
#pragma unroll
          for (int d = 0; d < 9; ++d) {
            const int nx = hmc_wrap_tile(ntx + d % 3 - 1, tiles_x);
            const int ny = hmc_wrap_tile(nty + d / 3 - 1, tiles_y);
            fl[d] = hmc_load_relaxed(q.flags + (ny * tiles_x + nx));
          }
        }
      }
    }

    const float4 cdn = *reinterpret_cast<const float4*>(&lastrow_c[b][warp][xb]);
    const float4 sdn = *reinterpret_cast<const float4*>(&lastrow_s[b][warp][xb]);
    const float4 cup = *reinterpret_cast<const float4*>(&firstrow_c[b][warp + 1][xb]);
    const float4 sup = *reinterpret_cast<const float4*>(&firstrow_s[b][warp + 1][xb]);
    const float cdn_a[4] = {cdn.x, cdn.y, cdn.z, cdn.w}, sdn_a[4] = {sdn.x, sdn.y, sdn.z, sdn.w};
    const float cup_a[4] = {cup.x, cup.y, cup.z, cup.w}, sup_a[4] = {sup.x, sup.y, sup.z, sup.w};
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      float cl = __shfl_up_sync(0xffffffffu, c[r][3], 1);
      float sl = __shfl_up_sync(0xffffffffu, sn[r][3], 1);
      float cr = __shfl_down_sync(0xffffffffu, c[r][0], 1);
      float sr = __shfl_down_sync(0xffffffffu, sn[r][0], 1);
      const int row = rb0 + r;
      if (lane == 0) {
        const float2 v = side[b][0][row];
        cl = v.x;
        sl = v.y;
      }
      if (lane == 31) {
        const float2 v = side[b][1][row];
        cr = v.x;
        sr = v.y;
      }
      float pr[4] = {p4[r].x, p4[r].y, p4[r].z, p4[r].w};
      const float tr[4] = {t4[r].x, t4[r].y, t4[r].z, t4[r].w};
      float out[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const float nlc = jj == 0 ? cl : c[r][jj - 1], nls = jj == 0 ? sl : sn[r][jj - 1];
        const float nrc = jj == 3 ? cr : c[r][jj + 1], nrs = jj == 3 ? sr : sn[r][jj + 1];
        const float ndc = r == 0 ? cdn_a[jj] : c[r - 1][jj], nds = r == 0 ? sdn_a[jj] : sn[r - 1][jj];
        const float nuc = r == ROWS - 1 ? cup_a[jj] : c[r + 1][jj];
        const float nus = r == ROWS - 1 ? sup_a[jj] : sn[r + 1][jj];
        const float Sc = xyd::nb_sum(nlc, nrc, ndc, nuc);
        const float Ss = xyd::nb_sum(nls, nrs, nds, nus);
        pr[jj] = __fmaf_rn(a.a, hmc_force(c[r][jj], sn[r][jj], Sc, Ss, a.K), pr[jj]);
        out[jj] = hmc_wrap(__fmaf_rn(a.eps, pr[jj], tr[jj]));
      }
      p4[r] = make_float4(pr[0], pr[1], pr[2], pr[3]);
      t4[r] = make_float4(out[0], out[1], out[2], out[3]);
    }
    if (tid == 0 && next < total) {
      bool ready = true;
      if (nj > 0) {
#pragma unroll
        for (int d = 0; d < 9; ++d) ready = ready && fl[d] >= (unsigned int)nj;
      }
      if (ready) {
        // the relaxed loads saw every counter set: this acquire fence makes
        // the stores they publish visible to thread 0, and issue()'s proxy
        // fence to its TMA reads
        fence_acq_rel_gpu();
        xyt::fence_async_shared();
        issue(next, s);
        s_issued[s] = 1;
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const size_t g = (size_t)(y0 + rb0 + r) * L + x0 + xb;
      *reinterpret_cast<float4*>(a.p_out + g) = p4[r];
      *reinterpret_cast<float4*>(th_dst + g) = t4[r];
    }
    // published after the next tile's first barrier (its stores have landed
    // by then), or before that tile waits
    pend_slot = ty * tiles_x + tx;
    pend_val = (unsigned int)(j + 1);
  }
  __syncthreads();
  publish();
}

// ---------------------------------------------------------------------------
// Two full kick-drift steps per launch (temporal blocking).  A CTA of 256
// threads owns 32 rows x 128 columns, a thread 4 rows x 4 columns in
// registers as in k_hmc_tile.  The first step also updates the ring around
// the tile (rows -1 and 32, columns -1 and 128: 320 sites that belong to the
// neighbouring tiles, recomputed from the same inputs with the same
// arithmetic, so every copy agrees bit for bit); the second updates the tile
// and writes angles and momenta once: 8 bytes read and 8 written per site for
// two steps.  Shared memory holds one frame of unit vectors, rows -2 .. 33 and
// columns -4 .. 131 of the tile (cos and sin planes), of which only what
// crosses a warp is written: the halo of two (rows -2 and 33, columns -2 and
// 129, the four ring corners), the ring, each warp's first and last row and
// the tile's first and last column; after the first step the ring and the
// warps' edge rows are overwritten with their new values.  Horizontal
// neighbours inside a warp's rows come by shuffle.  Momenta are read from one
// buffer and written to another (the ring reads the neighbours' old momenta).
// ---------------------------------------------------------------------------
constexpr int kP2Rows = 32;
constexpr int kP2Cols = 128;
constexpr int kP2Threads = 256;
constexpr int kP2Warps = kP2Threads / 32;
constexpr int kP2Band = kP2Rows / kP2Warps;                  // 4 rows per warp
constexpr int kFrRows = kP2Rows + 4;                         // tile rows -2 .. 33
constexpr int kFrCols = kP2Cols + 8;                         // tile columns -4 .. 131
constexpr size_t kP2Smem = sizeof(float) * 2 * kFrRows * kFrCols;
// The tile-walking form (PREF) adds the next tile's loads, brought in while the
// current tile runs: its angle and momentum rows as two TMA boxes of 32 x 128
// floats, then each thread's six scalars by cp.async (ring site A's angle and
// momentum, ring site B's, the halo-two sites H and G).
constexpr size_t kP2PreRowsAt = kP2Smem;
constexpr size_t kP2PreScalarsAt = kP2PreRowsAt + sizeof(float4) * 2 * kP2Band * kP2Threads;
constexpr size_t kP2SmemPref = kP2PreScalarsAt + sizeof(float) * 6 * kP2Threads;
static_assert(2 * (kP2SmemPref + 1024) <= 228 * 1024, "two tile-walking CTAs must fit one SM");
static_assert(kP2PreRowsAt % 128 == 0 && 2 * kP2Band * kP2Threads * 4 == 2 * kP2Rows * kP2Cols,
              "the TMA boxes (two of 32 x 128 floats) fill the 128-byte aligned row slots");
// The tile-walking form runs when every resident CTA gets at least this many
// tiles of a launch (measured per unit trajectory with the rows by per-thread
// cp.async: 3.44 against 3.56 ms at L = 4096, 17.8 against 18.9 at 8192; a tie
// at 2048, about 3.4 tiles per CTA; with a tile per CTA only the extra
// shared-memory round trip is left).
constexpr int kP2PrefMinTilesPerCta = 4;

__device__ __forceinline__ void hmc_cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

__device__ __forceinline__ int wrap_near(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// One leap-frog step of a site: kick by a F(unit vector, neighbour sums),
// drift by eps p, wrap (the per-site arithmetic of every HMC kernel).
__device__ __forceinline__ void hmc_site_step(float c, float s, float Sc, float Ss, float K,
                                              float a, float eps, float& p, float& t) {
  p = __fmaf_rn(a, hmc_force(c, s, Sc, Ss, K), p);
  t = hmc_wrap(__fmaf_rn(eps, p, t));
}

// PREF = false: one tile per CTA (grid = the tile columns x rows), its loads straight into
// registers.  PREF = true: a grid of resident CTAs walks the tiles blockIdx.x,
// + gridDim.x, ... (the tiles of a launch are independent: it reads one angle
// and one momentum buffer and writes two others); right after the current
// tile's staging barrier thread 0 has TMA copy the next tile's rows and every
// thread copies its ring and halo sites into its own shared-memory slots by
// cp.async, so they arrive while the two steps run.  Both forms run the same
// arithmetic on the same values: bit-identical.
// The tile-walking form's tensor maps (boxes of 32 rows x 128 columns): the
// three angle buffers (the launch reads the one the control block names) and
// the momenta it reads; a kernel parameter.
struct Tile2Maps {
  CUtensorMap th[3];
  CUtensorMap p;
};

template <int MODE, bool PREF>
__global__ void __launch_bounds__(kP2Threads, 2)
    k_hmc_tile2(HmcArgs a, const __grid_constant__ Tile2Maps maps) {
  extern __shared__ __align__(128) unsigned char smem[];
  float (*fc)[kFrCols] = reinterpret_cast<float (*)[kFrCols]>(smem);
  float (*fs)[kFrCols] = reinterpret_cast<float (*)[kFrCols]>(smem + sizeof(float) * kFrRows * kFrCols);
  float4* pre_rows = reinterpret_cast<float4*>(smem + kP2PreRowsAt);   // [2 * kP2Band][threads]
  float* pre_sc = reinterpret_cast<float*>(smem + kP2PreScalarsAt);     // [6][threads]

  const int L = a.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_x = L / kP2Cols, n_tiles = tiles_x * (L / kP2Rows);
  int src, dst;
  hmc_buffers(a, a.ctl->cur, &src, &dst);
  const float* __restrict__ th_src = hmc_buf(a, src);

  const int rb = kP2Band * warp;                             // first tile row of the band
  // the loads of tile t (PREF): the tile's angle and momentum rows as two
  // TMA boxes of 32 x 128 (thread 0, completing on s_bar), and this thread's
  // ring and halo sites by cp.async into its own slots: the same sites as the
  // loads in the tile loop below
  __shared__ __align__(8) uint64_t s_bar;
  uint32_t phase = 0;
  if (PREF) {
    if (tid == 0) {
      xyt::mbar_init(&s_bar, 1);
      xyt::fence_mbarrier_init();
    }
    __syncthreads();
  }
  auto prefetch = [&](int t) {
    const int px0 = (t % tiles_x) * kP2Cols, py0 = (t / tiles_x) * kP2Rows;
    if (tid == 0) {
      xyt::mbar_arrive_expect_tx(&s_bar, (uint32_t)(2 * sizeof(float) * kP2Rows * kP2Cols));
      xyt::tma_load_2d(pre_rows, &maps.th[src], px0, py0, &s_bar);
      xyt::tma_load_2d(pre_rows + kP2Rows * kP2Cols / 4, &maps.p, px0, py0, &s_bar);
    }
    const int ay = tid < kP2Cols ? -1 : kP2Rows, ax = tid & (kP2Cols - 1);
    const size_t ga = (size_t)wrap_near(py0 + ay, L) * L + (px0 + ax);
    hmc_cp4(&pre_sc[0 * kP2Threads + tid], th_src + ga);
    hmc_cp4(&pre_sc[1 * kP2Threads + tid], a.p_in + ga);
    if (tid < 2 * kP2Rows) {
      const int bx = tid < kP2Rows ? -1 : kP2Cols, by = tid & (kP2Rows - 1);
      const size_t gb = (size_t)(py0 + by) * L + wrap_near(px0 + bx, L);
      hmc_cp4(&pre_sc[2 * kP2Threads + tid], th_src + gb);
      hmc_cp4(&pre_sc[3 * kP2Threads + tid], a.p_in + gb);
    }
    const int hy = tid < kP2Cols ? -2 : kP2Rows + 1;
    hmc_cp4(&pre_sc[4 * kP2Threads + tid], th_src + (size_t)wrap_near(py0 + hy, L) * L + (px0 + ax));
    if (tid >= 64 && tid < 132) {
      int gy, gx;
      if (tid < 128) {
        gx = (tid - 64) < kP2Rows ? -2 : kP2Cols + 1;
        gy = (tid - 64) & (kP2Rows - 1);
      } else {
        gy = (tid & 2) ? kP2Rows : -1;
        gx = (tid & 1) ? kP2Cols : -1;
      }
      hmc_cp4(&pre_sc[5 * kP2Threads + tid],
              th_src + (size_t)wrap_near(py0 + gy, L) * L + wrap_near(px0 + gx, L));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (PREF && (int)blockIdx.x < n_tiles) prefetch(blockIdx.x);
  for (int tile = PREF ? (int)blockIdx.x : 0; tile < (PREF ? n_tiles : 1);
       tile += PREF ? (int)gridDim.x : 1) {
  const int x0 = PREF ? (tile % tiles_x) * kP2Cols : (int)blockIdx.x * kP2Cols;
  const int y0 = PREF ? (tile / tiles_x) * kP2Rows : (int)blockIdx.y * kP2Rows;

  // ---- loads: own 4 x 4 block (angles and momenta), one site of the ring's
  // top or bottom row (threads 0..255), one of its side columns (0..63), one
  // halo-two site of rows -2 / 33 (0..255), of columns -2 / 129 (64..127) or a
  // ring corner (128..131); from this thread's slots (PREF) or from global
  // memory
  const int xb = x0 + 4 * lane;
  float4 t4[kP2Band], p4[kP2Band];
  if (PREF) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (!xyt::mbar_wait_bounded(&s_bar, phase, kSpinLimit)) atomicOr(&a.ctl->error, 1u);
    phase ^= 1u;
  }
#pragma unroll
  for (int r = 0; r < kP2Band; ++r) {
    const size_t g = (size_t)(y0 + rb + r) * L + xb;
    // the boxes: rows of 128 floats, the thread's 4 x 4 block at row rb + r,
    // columns 4 lane .. 4 lane + 3
    t4[r] = PREF ? pre_rows[(rb + r) * (kP2Cols / 4) + lane]
                 : *reinterpret_cast<const float4*>(th_src + g);
    p4[r] = PREF ? pre_rows[(kP2Rows + rb + r) * (kP2Cols / 4) + lane]
                 : *reinterpret_cast<const float4*>(a.p_in + g);
  }
  // ring site A: row -1 (tid < 128) or 32, column tid & 127
  const int ay = tid < kP2Cols ? -1 : kP2Rows, ax = tid & (kP2Cols - 1);
  const size_t ga = (size_t)wrap_near(y0 + ay, L) * L + (x0 + ax);
  float ta = PREF ? pre_sc[0 * kP2Threads + tid] : th_src[ga];
  float pa = PREF ? pre_sc[1 * kP2Threads + tid] : a.p_in[ga];
  // ring site B: column -1 (tid < 32) or 128, row tid & 31
  const bool hasb = tid < 2 * kP2Rows;
  const int bx = tid < kP2Rows ? -1 : kP2Cols, by = tid & (kP2Rows - 1);
  float tb = 0.f, pb = 0.f;
  if (hasb) {
    const size_t gb = (size_t)(y0 + by) * L + wrap_near(x0 + bx, L);
    tb = PREF ? pre_sc[2 * kP2Threads + tid] : th_src[gb];
    pb = PREF ? pre_sc[3 * kP2Threads + tid] : a.p_in[gb];
  }
  // halo-two site H: rows -2 / 33; G: columns -2 / 129 or a corner
  const int hy = tid < kP2Cols ? -2 : kP2Rows + 1;
  const float th_h =
      PREF ? pre_sc[4 * kP2Threads + tid] : th_src[(size_t)wrap_near(y0 + hy, L) * L + (x0 + ax)];
  const bool hasg = tid >= 64 && tid < 132;
  int gy = 0, gx = 0;
  float th_g = 0.f;
  if (hasg) {
    if (tid < 128) {
      gx = (tid - 64) < kP2Rows ? -2 : kP2Cols + 1;
      gy = (tid - 64) & (kP2Rows - 1);
    } else {
      gy = (tid & 2) ? kP2Rows : -1;
      gx = (tid & 1) ? kP2Cols : -1;
    }
    th_g = PREF ? pre_sc[5 * kP2Threads + tid]
                : th_src[(size_t)wrap_near(y0 + gy, L) * L + wrap_near(x0 + gx, L)];
  }

  // ---- unit vectors of the old state; what crosses a warp goes to the frame
  float c[kP2Band][4], s[kP2Band][4];
#pragma unroll
  for (int r = 0; r < kP2Band; ++r) {
    xyd::unit_vector<MODE>(t4[r].x, &s[r][0], &c[r][0]);
    xyd::unit_vector<MODE>(t4[r].y, &s[r][1], &c[r][1]);
    xyd::unit_vector<MODE>(t4[r].z, &s[r][2], &c[r][2]);
    xyd::unit_vector<MODE>(t4[r].w, &s[r][3], &c[r][3]);
  }
  float ca, sa, cb = 0.f, sb = 0.f;
  xyd::unit_vector<MODE>(ta, &sa, &ca);
  if (hasb) xyd::unit_vector<MODE>(tb, &sb, &cb);
  {
    float hs, hc;
    xyd::unit_vector<MODE>(th_h, &hs, &hc);
    fc[hy + 2][ax + 4] = hc;
    fs[hy + 2][ax + 4] = hs;
    if (hasg) {
      xyd::unit_vector<MODE>(th_g, &hs, &hc);
      fc[gy + 2][gx + 4] = hc;
      fs[gy + 2][gx + 4] = hs;
    }
  }
  fc[ay + 2][ax + 4] = ca;
  fs[ay + 2][ax + 4] = sa;
  if (hasb) {
    fc[by + 2][bx + 4] = cb;
    fs[by + 2][bx + 4] = sb;
  }
  // the band's first and last row, and the tile's first and last column
  *reinterpret_cast<float4*>(&fc[rb + 2][4 * lane + 4]) = make_float4(c[0][0], c[0][1], c[0][2], c[0][3]);
  *reinterpret_cast<float4*>(&fs[rb + 2][4 * lane + 4]) = make_float4(s[0][0], s[0][1], s[0][2], s[0][3]);
  *reinterpret_cast<float4*>(&fc[rb + kP2Band + 1][4 * lane + 4]) =
      make_float4(c[kP2Band - 1][0], c[kP2Band - 1][1], c[kP2Band - 1][2], c[kP2Band - 1][3]);
  *reinterpret_cast<float4*>(&fs[rb + kP2Band + 1][4 * lane + 4]) =
      make_float4(s[kP2Band - 1][0], s[kP2Band - 1][1], s[kP2Band - 1][2], s[kP2Band - 1][3]);
  if (lane == 0 || lane == 31) {
    const int q = lane == 0 ? 4 : kP2Cols + 3;             // tile column 0 or 127
#pragma unroll
    for (int r = 1; r < kP2Band - 1; ++r) {
      fc[rb + r + 2][q] = lane == 0 ? c[r][0] : c[r][3];
      fs[rb + r + 2][q] = lane == 0 ? s[r][0] : s[r][3];
    }
  }
  __syncthreads();

  // every thread has read its slots before the barrier above: the next tile's
  // copies land there while this one runs
  if (PREF && tile + (int)gridDim.x < n_tiles) prefetch(tile + (int)gridDim.x);

  // ---- first step: the ring sites (from the frame), then the tile --------
  const float K = a.K, ka = a.a, eps = a.eps;
  {
    const int r = ay + 2, q = ax + 4;
    const float Sc = xyd::nb_sum(fc[r][q - 1], fc[r][q + 1], fc[r - 1][q], fc[r + 1][q]);
    const float Ss = xyd::nb_sum(fs[r][q - 1], fs[r][q + 1], fs[r - 1][q], fs[r + 1][q]);
    hmc_site_step(ca, sa, Sc, Ss, K, ka, eps, pa, ta);
  }
  if (hasb) {
    const int r = by + 2, q = bx + 4;
    const float Sc = xyd::nb_sum(fc[r][q - 1], fc[r][q + 1], fc[r - 1][q], fc[r + 1][q]);
    const float Ss = xyd::nb_sum(fs[r][q - 1], fs[r][q + 1], fs[r - 1][q], fs[r + 1][q]);
    hmc_site_step(cb, sb, Sc, Ss, K, ka, eps, pb, tb);
  }
  // the ring's new unit vectors (its momenta and angles are not needed again)
  xyd::unit_vector<MODE>(ta, &sa, &ca);
  if (hasb) xyd::unit_vector<MODE>(tb, &sb, &cb);
  // vertical neighbours of the band: the row below its first and above its last
  float4 cdn = *reinterpret_cast<const float4*>(&fc[rb + 1][4 * lane + 4]);
  float4 sdn = *reinterpret_cast<const float4*>(&fs[rb + 1][4 * lane + 4]);
  float4 cup = *reinterpret_cast<const float4*>(&fc[rb + kP2Band + 2][4 * lane + 4]);
  float4 sup = *reinterpret_cast<const float4*>(&fs[rb + kP2Band + 2][4 * lane + 4]);
#pragma unroll
  for (int r = 0; r < kP2Band; ++r) {
    float cl = __shfl_up_sync(0xffffffffu, c[r][3], 1);
    float sl = __shfl_up_sync(0xffffffffu, s[r][3], 1);
    float cr = __shfl_down_sync(0xffffffffu, c[r][0], 1);
    float sr = __shfl_down_sync(0xffffffffu, s[r][0], 1);
    if (lane == 0) {
      cl = fc[rb + r + 2][3];
      sl = fs[rb + r + 2][3];
    }
    if (lane == 31) {
      cr = fc[rb + r + 2][kP2Cols + 4];
      sr = fs[rb + r + 2][kP2Cols + 4];
    }
    const float pr[4] = {p4[r].x, p4[r].y, p4[r].z, p4[r].w};
    const float tr[4] = {t4[r].x, t4[r].y, t4[r].z, t4[r].w};
    const float cd[4] = {cdn.x, cdn.y, cdn.z, cdn.w}, sd[4] = {sdn.x, sdn.y, sdn.z, sdn.w};
    const float cu[4] = {cup.x, cup.y, cup.z, cup.w}, su[4] = {sup.x, sup.y, sup.z, sup.w};
    float po[4], to[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float nlc = j == 0 ? cl : c[r][j - 1], nls = j == 0 ? sl : s[r][j - 1];
      const float nrc = j == 3 ? cr : c[r][j + 1], nrs = j == 3 ? sr : s[r][j + 1];
      const float ndc = r == 0 ? cd[j] : c[r - 1][j], nds = r == 0 ? sd[j] : s[r - 1][j];
      const float nuc = r == kP2Band - 1 ? cu[j] : c[r + 1][j];
      const float nus = r == kP2Band - 1 ? su[j] : s[r + 1][j];
      float p = pr[j], t = tr[j];
      hmc_site_step(c[r][j], s[r][j], xyd::nb_sum(nlc, nrc, ndc, nuc),
                    xyd::nb_sum(nls, nrs, nds, nus), K, ka, eps, p, t);
      po[j] = p;
      to[j] = t;
    }
    p4[r] = make_float4(po[0], po[1], po[2], po[3]);
    t4[r] = make_float4(to[0], to[1], to[2], to[3]);
  }
  // new unit vectors (the old ones are no longer read by this thread)
#pragma unroll
  for (int r = 0; r < kP2Band; ++r) {
    xyd::unit_vector<MODE>(t4[r].x, &s[r][0], &c[r][0]);
    xyd::unit_vector<MODE>(t4[r].y, &s[r][1], &c[r][1]);
    xyd::unit_vector<MODE>(t4[r].z, &s[r][2], &c[r][2]);
    xyd::unit_vector<MODE>(t4[r].w, &s[r][3], &c[r][3]);
  }
  __syncthreads();   // every old frame value has been read
  fc[ay + 2][ax + 4] = ca;
  fs[ay + 2][ax + 4] = sa;
  if (hasb) {
    fc[by + 2][bx + 4] = cb;
    fs[by + 2][bx + 4] = sb;
  }
  *reinterpret_cast<float4*>(&fc[rb + 2][4 * lane + 4]) = make_float4(c[0][0], c[0][1], c[0][2], c[0][3]);
  *reinterpret_cast<float4*>(&fs[rb + 2][4 * lane + 4]) = make_float4(s[0][0], s[0][1], s[0][2], s[0][3]);
  *reinterpret_cast<float4*>(&fc[rb + kP2Band + 1][4 * lane + 4]) =
      make_float4(c[kP2Band - 1][0], c[kP2Band - 1][1], c[kP2Band - 1][2], c[kP2Band - 1][3]);
  *reinterpret_cast<float4*>(&fs[rb + kP2Band + 1][4 * lane + 4]) =
      make_float4(s[kP2Band - 1][0], s[kP2Band - 1][1], s[kP2Band - 1][2], s[kP2Band - 1][3]);
  __syncthreads();

  // ---- second step: the tile, written out ----------------------------------
  cdn = *reinterpret_cast<const float4*>(&fc[rb + 1][4 * lane + 4]);
  sdn = *reinterpret_cast<const float4*>(&fs[rb + 1][4 * lane + 4]);
  cup = *reinterpret_cast<const float4*>(&fc[rb + kP2Band + 2][4 * lane + 4]);
  sup = *reinterpret_cast<const float4*>(&fs[rb + kP2Band + 2][4 * lane + 4]);
  float* __restrict__ th_dst = hmc_buf(a, dst);
#pragma unroll
  for (int r = 0; r < kP2Band; ++r) {
    float cl = __shfl_up_sync(0xffffffffu, c[r][3], 1);
    float sl = __shfl_up_sync(0xffffffffu, s[r][3], 1);
    float cr = __shfl_down_sync(0xffffffffu, c[r][0], 1);
    float sr = __shfl_down_sync(0xffffffffu, s[r][0], 1);
    if (lane == 0) {
      cl = fc[rb + r + 2][3];
      sl = fs[rb + r + 2][3];
    }
    if (lane == 31) {
      cr = fc[rb + r + 2][kP2Cols + 4];
      sr = fs[rb + r + 2][kP2Cols + 4];
    }
    const float cd[4] = {cdn.x, cdn.y, cdn.z, cdn.w}, sd[4] = {sdn.x, sdn.y, sdn.z, sdn.w};
    const float cu[4] = {cup.x, cup.y, cup.z, cup.w}, su[4] = {sup.x, sup.y, sup.z, sup.w};
    float po[4], to[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float nlc = j == 0 ? cl : c[r][j - 1], nls = j == 0 ? sl : s[r][j - 1];
      const float nrc = j == 3 ? cr : c[r][j + 1], nrs = j == 3 ? sr : s[r][j + 1];
      const float ndc = r == 0 ? cd[j] : c[r - 1][j], nds = r == 0 ? sd[j] : s[r - 1][j];
      const float nuc = r == kP2Band - 1 ? cu[j] : c[r + 1][j];
      const float nus = r == kP2Band - 1 ? su[j] : s[r + 1][j];
      po[j] = (&p4[r].x)[j];
      to[j] = (&t4[r].x)[j];
      hmc_site_step(c[r][j], s[r][j], xyd::nb_sum(nlc, nrc, ndc, nuc),
                    xyd::nb_sum(nls, nrs, nds, nus), K, ka, eps, po[j], to[j]);
    }
    const size_t g = (size_t)(y0 + rb + r) * L + xb;
    *reinterpret_cast<float4*>(a.p_out + g) = make_float4(po[0], po[1], po[2], po[3]);
    *reinterpret_cast<float4*>(th_dst + g) = make_float4(to[0], to[1], to[2], to[3]);
  }
  if (PREF) __syncthreads();   // the next tile's staging rewrites the frame
  }
}

// ---------------------------------------------------------------------------
// Per-site kernel (any L >= 2): one thread per site, the four neighbours' unit
// vectors recomputed from global memory.  Same per-site arithmetic as above.
// ---------------------------------------------------------------------------
constexpr int kSiteThreads = 256;

template <int MODE, int KIND>
__global__ void __launch_bounds__(kSiteThreads) k_hmc_site(HmcArgs a) {
  __shared__ long long red[kSiteThreads / 32][kHmcSums];
  const int L = a.L;
  const uint32_t N = (uint32_t)L * (uint32_t)L;
  const uint32_t cur = a.ctl->cur;
  int src, dst;
  hmc_buffers(a, cur, &src, &dst);
  const float* __restrict__ th_src = hmc_buf(a, src);
  HmcAcc acc;
  acc_zero(acc);
  const uint32_t site = blockIdx.x * kSiteThreads + threadIdx.x;
  if (site < N) {
    const int y = (int)(site / (uint32_t)L), x = (int)(site - (uint32_t)y * (uint32_t)L);
    const int xl = x == 0 ? L - 1 : x - 1, xr = x == L - 1 ? 0 : x + 1;
    const int yd = y == 0 ? L - 1 : y - 1, yu = y == L - 1 ? 0 : y + 1;
    const size_t row = (size_t)y * L;
    const float t = th_src[row + x];
    float cs[5], sn[5];
    xyd::unit_vector<MODE>(t, &sn[0], &cs[0]);
    xyd::unit_vector<MODE>(th_src[row + xl], &sn[1], &cs[1]);
    xyd::unit_vector<MODE>(th_src[row + xr], &sn[2], &cs[2]);
    xyd::unit_vector<MODE>(th_src[(size_t)yd * L + x], &sn[3], &cs[3]);
    xyd::unit_vector<MODE>(th_src[(size_t)yu * L + x], &sn[4], &cs[4]);
    float p = KIND == kHmcBeginDraw ? hmc_momentum(site, (uint32_t)a.ctl->traj, a.lattice_id, a.rk)
                                    : a.p_in[site];
    const float Sc = xyd::nb_sum(cs[1], cs[2], cs[3], cs[4]);
    const float Ss = xyd::nb_sum(sn[1], sn[2], sn[3], sn[4]);
    const float F = hmc_force(cs[0], sn[0], Sc, Ss, a.K);
    if (KIND == kHmcBeginDraw || KIND == kHmcBeginRead)
      hmc_terms(p, cs[0], sn[0], cs[2], sn[2], cs[4], sn[4], acc);
    p = __fmaf_rn(a.a, F, p);
    if (KIND == kHmcFinal) {
      hmc_terms(p, cs[0], sn[0], cs[2], sn[2], cs[4], sn[4], acc);
    } else {
      hmc_buf(a, dst)[site] = hmc_wrap(__fmaf_rn(a.eps, p, t));
    }
    a.p_out[site] = p;
  }
  if (KIND == kHmcBeginDraw || KIND == kHmcBeginRead)
    hmc_commit<kSiteThreads / 32>(acc, a.ctl->acc[0], red);
  if (KIND == kHmcFinal) hmc_commit<kSiteThreads / 32>(acc, a.ctl->acc[1], red);
}

// ---------------------------------------------------------------------------
// The test (mode 0) or the commit of a plain integration (mode 1).
// ---------------------------------------------------------------------------
__global__ void k_hmc_accept(HmcArgs a, int mode, double beta, double J) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  HmcCtl* c = a.ctl;
  int fin, unused;
  hmc_buffers(a, c->cur, &fin, &unused);
  if (xyh::hmc_decide(c, a.lattice_id, a.rk, mode, beta, J)) c->cur = (uint32_t)fin;
}

__global__ void k_hmc_draw(HmcArgs a) {
  const uint32_t N = (uint32_t)a.L * (uint32_t)a.L;
  const uint32_t traj = (uint32_t)a.ctl->traj;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x)
    a.p_out[s] = hmc_momentum(s, traj, a.lattice_id, a.rk);
}

__global__ void k_hmc_start(HmcArgs a, int hot) {
  const uint32_t N = (uint32_t)a.L * (uint32_t)a.L;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
    float t = 0.f;
    if (hot) {
      const uint4 w = xyd::philox4x32_10(make_uint4(s, 0u, a.lattice_id, 0u), a.rk);
      t = (float)(w.x >> 8) * xyd::kHotScale;
    }
    a.th[0][s] = t;
    a.p_out[s] = 0.f;
  }
}

__global__ void k_hmc_canon_copy(HmcArgs a) {
  const uint32_t cur = a.ctl->cur;
  if (cur == 0u) return;
  const uint32_t N = (uint32_t)a.L * (uint32_t)a.L;
  const float* __restrict__ from = hmc_buf(a, (int)cur);
  float* __restrict__ to = a.th[0];
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x)
    to[s] = from[s];
}

__global__ void k_hmc_canon_reset(HmcCtl* ctl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctl->cur = 0u;
}

// Two full steps per launch: two CTAs per SM (the registers' limit); the
// tile-walking form when each would get at least kP2PrefMinTilesPerCta tiles
// and the tensor maps are given, else one tile per CTA.
template <int MODE>
cudaError_t launch_step2(const HmcArgs& a, const CUtensorMap* th_maps, const CUtensorMap* p_map,
                         cudaStream_t stream) {
  if (!a.tiled || !a.pairs || a.p_in == a.p_out) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int n_tiles = (a.L / kP2Cols) * (a.L / kP2Rows);
  Tile2Maps m;
  if (th_maps && p_map && n_tiles >= kP2PrefMinTilesPerCta * 2 * sms) {
    for (int i = 0; i < 3; ++i) m.th[i] = th_maps[i];
    m.p = *p_map;
    k_hmc_tile2<MODE, true><<<2 * sms, kP2Threads, kP2SmemPref, stream>>>(a, m);
  } else {
    memset(&m, 0, sizeof(m));
    k_hmc_tile2<MODE, false>
        <<<dim3(a.L / kP2Cols, a.L / kP2Rows), kP2Threads, kP2Smem, stream>>>(a, m);
  }
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(int kind, const HmcArgs& a, cudaStream_t stream) {
  if (kind == kHmcStep2) return launch_step2<MODE>(a, nullptr, nullptr, stream);
  if (a.tiled) {
    const dim3 grid(a.L / kTileCols, a.L / kTileRows);
    switch (kind) {
      case kHmcBeginDraw: k_hmc_tile<MODE, kHmcBeginDraw><<<grid, kTileThreads, 0, stream>>>(a); break;
      case kHmcBeginRead: k_hmc_tile<MODE, kHmcBeginRead><<<grid, kTileThreads, 0, stream>>>(a); break;
      case kHmcStep: k_hmc_tile<MODE, kHmcStep><<<grid, kTileThreads, 0, stream>>>(a); break;
      default: k_hmc_tile<MODE, kHmcFinal><<<grid, kTileThreads, 0, stream>>>(a); break;
    }
  } else {
    const int64_t N = (int64_t)a.L * a.L;
    const int grid = (int)((N + kSiteThreads - 1) / kSiteThreads);
    switch (kind) {
      case kHmcBeginDraw: k_hmc_site<MODE, kHmcBeginDraw><<<grid, kSiteThreads, 0, stream>>>(a); break;
      case kHmcBeginRead: k_hmc_site<MODE, kHmcBeginRead><<<grid, kSiteThreads, 0, stream>>>(a); break;
      case kHmcStep: k_hmc_site<MODE, kHmcStep><<<grid, kSiteThreads, 0, stream>>>(a); break;
      default: k_hmc_site<MODE, kHmcFinal><<<grid, kSiteThreads, 0, stream>>>(a); break;
    }
  }
  return cudaGetLastError();
}

}  // namespace

bool hmc_tiled_ok(int L) { return L >= kTileCols && L % kTileCols == 0; }

cudaError_t hmc_prepare(int sincos_mode) {
  static bool done[3][64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int m = sincos_mode < 0 || sincos_mode > 2 ? 0 : sincos_mode;
  if (dev >= 0 && dev < 64 && done[m][dev]) return cudaSuccess;
  const void* f = m == 0 ? (const void*)k_hmc_tile2<0, false>
                         : (m == 1 ? (const void*)k_hmc_tile2<1, false>
                                   : (const void*)k_hmc_tile2<2, false>);
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP2Smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  const void* fp = m == 0 ? (const void*)k_hmc_tile2<0, true>
                          : (m == 1 ? (const void*)k_hmc_tile2<1, true>
                                    : (const void*)k_hmc_tile2<2, true>);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP2SmemPref);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fp, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  const void* g4 = m == 0 ? (const void*)k_hmc_step_tma<0, 4>
                          : (m == 1 ? (const void*)k_hmc_step_tma<1, 4> : (const void*)k_hmc_step_tma<2, 4>);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(g4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TmaGeom<4>::kSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(g4, cudaFuncAttributePreferredSharedMemoryCarveout, 100);

  if (e == cudaSuccess && dev >= 0 && dev < 64) done[m][dev] = true;
  return e;
}

cudaError_t launch_hmc_step2(int sincos_mode, const HmcArgs& a, const void* th_maps3,
                             const void* p_map, cudaStream_t stream) {
  if (!hmc_tiled_ok(a.L)) return cudaErrorInvalidValue;
  const CUtensorMap* tm = static_cast<const CUtensorMap*>(th_maps3);
  const CUtensorMap* pm = static_cast<const CUtensorMap*>(p_map);
  switch (sincos_mode) {
    case 0: return launch_step2<0>(a, tm, pm, stream);
    case 1: return launch_step2<1>(a, tm, pm, stream);
    default: return launch_step2<2>(a, tm, pm, stream);
  }
}

cudaError_t launch_hmc(int kind, int sincos_mode, const HmcArgs& a, cudaStream_t stream) {
  if (kind < kHmcBeginDraw || kind > kHmcStep2) return cudaErrorInvalidValue;
  if (a.tiled && !hmc_tiled_ok(a.L)) return cudaErrorInvalidValue;
  switch (sincos_mode) {
    case 0: return launch_mode<0>(kind, a, stream);
    case 1: return launch_mode<1>(kind, a, stream);
    default: return launch_mode<2>(kind, a, stream);
  }
}

template <int ROWS>
cudaError_t launch_tma_rows(int sincos_mode, const HmcArgs& a, const CUtensorMap* m, int ctas,
                            cudaStream_t stream) {
  const int tiles_x = a.L / kTileCols;
  const int n_tiles = tiles_x * (a.L / TmaGeom<ROWS>::kRows);
  const int grid = ctas < n_tiles ? ctas : n_tiles;
  const size_t smem = TmaGeom<ROWS>::kSmem;
  switch (sincos_mode) {
    case 0:
      k_hmc_step_tma<0, ROWS><<<grid, kTileThreads, smem, stream>>>(m[0], m[1], m[2], m[3], a, tiles_x, n_tiles);
      break;
    case 1:
      k_hmc_step_tma<1, ROWS><<<grid, kTileThreads, smem, stream>>>(m[0], m[1], m[2], m[3], a, tiles_x, n_tiles);
      break;
    default:
      k_hmc_step_tma<2, ROWS><<<grid, kTileThreads, smem, stream>>>(m[0], m[1], m[2], m[3], a, tiles_x, n_tiles);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_hmc_step_tma(int sincos_mode, const HmcArgs& a, const void* maps4, int box_rows,
                                int ctas, cudaStream_t stream) {
  if (!a.tiled || a.p_in != a.p_out || !maps4 || ctas < 1) return cudaErrorInvalidValue;
  const CUtensorMap* m = static_cast<const CUtensorMap*>(maps4);
  if (box_rows == TmaGeom<4>::kRows) return launch_tma_rows<4>(sincos_mode, a, m, ctas, stream);
  return cudaErrorInvalidValue;
}

cudaError_t launch_hmc_steps_persist(int sincos_mode, const HmcStepsArgs& q, const void* maps4,
                                     cudaStream_t stream) {
  const HmcArgs& a = q.a;
  if (!a.tiled || a.p_in != a.p_out || !maps4 || q.n_steps < 1 || !q.flags ||
      q.spin_limit < 1 || (a.L % kTileCols) != 0 || (a.L % TmaGeom<4>::kRows) != 0)
    return cudaErrorInvalidValue;
  const int tiles_x = a.L / kTileCols;
  const int n_tiles = tiles_x * (a.L / TmaGeom<4>::kRows);
  if ((long long)q.n_steps * n_tiles > 0x7fffffffll - (1ll << 20)) return cudaErrorInvalidValue;
  const void* fn = sincos_mode == 0 ? (const void*)k_hmc_steps_persist<0>
                                    : (sincos_mode == 1 ? (const void*)k_hmc_steps_persist<1>
                                                        : (const void*)k_hmc_steps_persist<2>);
  const size_t smem = TmaGeom<4>::kSmem;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTileThreads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int grid = n_tiles < per_sm * sms ? n_tiles : per_sm * sms;
  e = cudaMemsetAsync(q.flags, 0, sizeof(unsigned int) * (size_t)n_tiles, stream);
  if (e != cudaSuccess) return e;
  const CUtensorMap* m = static_cast<const CUtensorMap*>(maps4);
  HmcStepsArgs qq = q;
  int tx = tiles_x, nt = n_tiles;
  void* args[] = {const_cast<CUtensorMap*>(&m[0]), const_cast<CUtensorMap*>(&m[1]),
                  const_cast<CUtensorMap*>(&m[2]), const_cast<CUtensorMap*>(&m[3]), &qq, &tx, &nt};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTileThreads), args, smem, stream);
}

int hmc_persist_tiles(int L) {
  return (L % kTileCols == 0 && L % TmaGeom<4>::kRows == 0) ? (L / kTileCols) * (L / TmaGeom<4>::kRows)
                                                             : 0;
}

long long hmc_persist_spin_limit() { return kSpinLimit; }

namespace {
// The failure path of the bounded waits, exercised without a fault: wait on a
// barrier that nothing ever completes, exactly as the TMA kernel waits on its
// stage barriers, and set the error word when the bound runs out.
__global__ void k_selftest_wait(unsigned int* error, long long polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    xyt::mbar_init(&bar, 1);
    xyt::fence_mbarrier_init();
  }
  __syncthreads();
  const bool done = xyt::mbar_wait_bounded(&bar, 0u, polls);   // no arrival: must run out
  if (!done && threadIdx.x == 0) atomicOr(error, 1u);
}
}  // namespace

cudaError_t launch_selftest_wait(unsigned int* d_error, long long polls, cudaStream_t stream) {
  k_selftest_wait<<<1, 32, 0, stream>>>(d_error, polls);
  return cudaGetLastError();
}

cudaError_t launch_hmc_accept(int mode, const HmcArgs& a, double beta, double J,
                              cudaStream_t stream) {
  k_hmc_accept<<<1, 32, 0, stream>>>(a, mode, beta, J);
  return cudaGetLastError();
}

cudaError_t launch_hmc_draw(const HmcArgs& a, cudaStream_t stream) {
  k_hmc_draw<<<grid_for((int64_t)a.L * a.L, 256), 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_hmc_start(const HmcArgs& a, int hot, cudaStream_t stream) {
  k_hmc_start<<<grid_for((int64_t)a.L * a.L, 256), 256, 0, stream>>>(a, hot);
  return cudaGetLastError();
}

cudaError_t launch_hmc_canonical(const HmcArgs& a, cudaStream_t stream) {
  k_hmc_canon_copy<<<grid_for((int64_t)a.L * a.L, 256), 256, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_hmc_canon_reset<<<1, 32, 0, stream>>>(a.ctl);
  return cudaGetLastError();
}

}  // namespace xyk
