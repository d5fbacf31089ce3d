// xy_hmc.cu -- Hybrid Monte Carlo for the 2-d XY model (Sec. 1.2 of the
// paper): Gaussian momenta, the leap-frog integration of the equations of
// motion (the parallel core of the method) and the global Metropolis test.
//
//   H_hmc = sum_s p_s^2 / 2 + beta H(theta),  F_s = -beta J sum_nn sin(t_s - t_j)
//
// A trajectory of n_md steps is n_md + 2 launches plus the test:
//   begin   draw p (Philox domain 3, Box-Muller), sums of (theta_0, p_0),
//           p += eps/2 F(theta_0), theta_1 = theta_0 + eps p
//   step k  p += eps F(theta_k), theta_{k+1} = theta_k + eps p   (k = 1..n-1)
//   final   p += eps/2 F(theta_n), sums of (theta_n, p_n)
//   accept  one thread: dH from the exact fixed-point sums, u < exp(-dH)
// Three angle buffers: the state stays untouched in buffer `cur` (restored on
// rejection for free), the integration ping-pongs between the other two, and
// the accept kernel moves `cur` on the device, so trajectories replay as one
// captured graph with no host round trip.  Sums are formed per site in FP32
// and converted to 64-bit fixed point before any addition: exact, and the
// same for every launch shape (the tiled and per-site kernels agree bit for
// bit in angles, momenta and sums).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "xy_internal.h"

namespace xyk {

namespace {

using xyd::RoundKeys;

// 2 pi split for the drift wrap: kTwoPiHi has 21 significant bits, so k * kTwoPiHi
// is exact for |k| < 8.
constexpr float kTwoPiHi = 4.0f * xyd::kPio2Hi;
constexpr float kTwoPiLo = 4.0f * xyd::kPio2Lo;
constexpr float kInvTwoPi = 0.159154943091895335769f;
constexpr float kKinFx = 8388608.0f;          // 2^23: (p^2 / 2) * 2^24 = p^2 * 2^23
constexpr float kFx30 = 1073741824.0f;        // 2^30

// ---------------------------------------------------------------------------
// Per-site arithmetic, shared by the tiled and the per-site kernels.  Rounding
// is pinned with explicit intrinsics so both kernels agree bit for bit.
// ---------------------------------------------------------------------------

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

// Per-site terms of the sums, each rounded to fixed point before it is added:
// K: p^2/2; C: cos(t - t_r) + cos(t - t_u); Ix: sin(t - t_r); Iy: sin(t - t_u);
// Mx, My: c, s  (r = +x neighbour, u = +y neighbour).
__device__ __forceinline__ void hmc_terms(float p, float c, float s, float cr, float sr, float cu,
                                          float su, long long v[kHmcSums]) {
  const float cx = __fmaf_rn(c, cr, __fmul_rn(s, sr));
  const float cy = __fmaf_rn(c, cu, __fmul_rn(s, su));
  const float ix = __fmaf_rn(s, cr, -__fmul_rn(c, sr));
  const float iy = __fmaf_rn(s, cu, -__fmul_rn(c, su));
  v[0] += __float2ll_rn(__fmul_rn(__fmul_rn(p, p), kKinFx));
  v[1] += __float2ll_rn(__fmul_rn(__fadd_rn(cx, cy), kFx30));
  v[2] += __float2ll_rn(__fmul_rn(ix, kFx30));
  v[3] += __float2ll_rn(__fmul_rn(iy, kFx30));
  v[4] += __float2ll_rn(__fmul_rn(c, kFx30));
  v[5] += __float2ll_rn(__fmul_rn(s, kFx30));
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of the six accumulators into dst (one 64-bit atomic each per CTA).
// Called by every thread of the block.
template <int NWARPS>
__device__ __forceinline__ void hmc_commit(long long v[kHmcSums], unsigned long long* dst,
                                           long long (*sh)[kHmcSums]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

// Source and destination angle buffers of a launch, from the state buffer `cur`.
__device__ __forceinline__ void hmc_buffers(int kind, int k, int n_md, uint32_t cur, int* src,
                                            int* dst) {
  if (kind == kHmcBeginDraw || kind == kHmcBeginRead) {
    *src = (int)cur;
    *dst = (int)((cur + 1u) % 3u);
  } else if (kind == kHmcStep) {
    *src = (int)((cur + 1u + (uint32_t)((k - 1) & 1)) % 3u);
    *dst = (int)((cur + 1u + (uint32_t)(k & 1)) % 3u);
  } else {
    *src = (int)((cur + 1u + (uint32_t)((n_md - 1) & 1)) % 3u);
    *dst = *src;
  }
}

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
__global__ void __launch_bounds__(kTileThreads) k_hmc_tile(HmcArgs a) {
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
  hmc_buffers(KIND, a.k, a.n_md, cur, &src, &dst);
  const float* __restrict__ th_src = hmc_buf(a, src);
  float* __restrict__ p_buf = a.p;

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
      p4[r] = *reinterpret_cast<const float4*>(p_buf + (size_t)(yb + r) * L + xb);
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

  long long acc[kHmcSums] = {0, 0, 0, 0, 0, 0};
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
    *reinterpret_cast<float4*>(p_buf + (size_t)(yb + r) * L + xb) = p4[r];
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
  hmc_buffers(KIND, a.k, a.n_md, cur, &src, &dst);
  const float* __restrict__ th_src = hmc_buf(a, src);
  long long acc[kHmcSums] = {0, 0, 0, 0, 0, 0};
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
                                    : a.p[site];
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
    a.p[site] = p;
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
  hmc_buffers(kHmcFinal, 0, a.n_md, c->cur, &fin, &unused);
  const long long dK = (long long)(c->acc[1][0] - c->acc[0][0]);
  const long long dC = (long long)(c->acc[1][1] - c->acc[0][1]);
  const double dH = (double)dK * 0x1p-24 - beta * J * ((double)dC * 0x1p-30);
  bool take = true;
  if (mode == 0) {
    const uint4 w = xyd::philox4x32_10(make_uint4(0u, (uint32_t)c->traj, a.lattice_id, 4u), a.rk);
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
  if (take) c->cur = (uint32_t)fin;
  for (int ph = 0; ph < 2; ++ph)
    for (int j = 0; j < kHmcSums; ++j) {
      c->last[ph][j] = c->acc[ph][j];
      c->acc[ph][j] = 0ull;
    }
}

__global__ void k_hmc_draw(HmcArgs a) {
  const uint32_t N = (uint32_t)a.L * (uint32_t)a.L;
  const uint32_t traj = (uint32_t)a.ctl->traj;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x)
    a.p[s] = hmc_momentum(s, traj, a.lattice_id, a.rk);
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
    a.p[s] = 0.f;
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

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

template <int MODE>
cudaError_t launch_mode(int kind, const HmcArgs& a, cudaStream_t stream) {
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

cudaError_t launch_hmc(int kind, int sincos_mode, const HmcArgs& a, cudaStream_t stream) {
  if (kind < kHmcBeginDraw || kind > kHmcFinal) return cudaErrorInvalidValue;
  if (a.tiled && !hmc_tiled_ok(a.L)) return cudaErrorInvalidValue;
  switch (sincos_mode) {
    case 0: return launch_mode<0>(kind, a, stream);
    case 1: return launch_mode<1>(kind, a, stream);
    default: return launch_mode<2>(kind, a, stream);
  }
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
