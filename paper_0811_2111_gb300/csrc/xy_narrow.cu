// xy_narrow.cu -- the one-launch checkerboard sweep on narrow tiles, for the
// batched engine's lattices whose side is a multiple of 32 but not of 128
// (L = 32, 64, 96, ...), which the 32 x 64 tiles of xy_fused.cu do not fit.
//
// The scheme is xy_fused.cu's (one launch per sweep, src -> dst ping-pong):
// a CTA owns a tile of 32 rows x 16 plane columns (32 natural columns) of both
// colours, stages both planes plus two halo rows and one halo plane column as
// (angle, cos, sin), updates the red sites of the tile and of the ring at
// distance one around it (recomputed from the same old state and the same
// counter-based Philox words as the neighbouring tiles' own updates, hence
// identical), then the black sites against the new red ones with the sweep
// sums, and writes the tile to dst.  Here each thread takes one pair of
// adjacent plane columns in two rows (ty and ty + 16) per colour (8 lanes per
// row, four warps of 4 rows each), the staging 4 lanes per row.  Every site
// runs the single-lattice arithmetic (xyd::metropolis_step etc.), so each
// lattice is bit for bit what the single-lattice kernels make of it.
//
// Requires W = L/2 to be a multiple of 16 and L a multiple of 32 (L % 32 == 0).
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_debug.h"
#include "xy_device.cuh"
#include "xy_internal.h"

namespace xyk {

namespace {

constexpr int kNTileRows = 32;
constexpr int kNTileK = 16;                   // plane columns
constexpr int kNThreads = 128;
constexpr int kNWarps = kNThreads / 32;
constexpr int kNSRows = kNTileRows + 4;       // rows y0-2 .. y0+33
constexpr int kNSCols = kNTileK + 8;          // plane cols k0-4 .. k0+19 (k0-1 .. k0+16 used)
constexpr int kNRing = 2 * kNTileK + kNTileRows;          // 64 red ring sites
constexpr int kNStageRowsTotal = kNSRows + (kNSRows - 2);  // black rows + red rows staged

constexpr size_t kNThBytes = sizeof(float) * 2 * kNSRows * kNSCols;
constexpr size_t kNCsBytes = sizeof(float2) * 2 * kNSRows * kNSCols;
constexpr size_t kNPartBytes = sizeof(float) * kNWarps * 5 * 2;
constexpr size_t kNCntBytes = sizeof(unsigned int) * kNWarps;
constexpr size_t kNSmemBytes = kNThBytes + kNCsBytes + kNPartBytes + kNCntBytes;

typedef float NThArr[kNSRows][kNSCols];
typedef float2 NCsArr[kNSRows][kNSCols];

__device__ __forceinline__ int nwrap(int v, int n) {
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}

// The four neighbour unit vectors of the two sites at stage columns c0, c0+1
// of row r in plane `nb` (the other colour): same-row neighbours of a site at
// column c are c+q-1 and c+q.
struct NPair {
  float Sc[2], Ss[2];
  float2 l[2], r[2], d[2], u[2];
};

__device__ __forceinline__ void npair_neighbours(const NCsArr& nb, int r, int c0, int q, NPair& n) {
  const float2 a = nb[r][c0 + q - 1], m = nb[r][c0 + q], b = nb[r][c0 + q + 1];
  const float4 D = *reinterpret_cast<const float4*>(&nb[r - 1][c0]);
  const float4 U = *reinterpret_cast<const float4*>(&nb[r + 1][c0]);
  n.l[0] = a;
  n.r[0] = m;
  n.l[1] = m;
  n.r[1] = b;
  n.d[0] = make_float2(D.x, D.y);
  n.d[1] = make_float2(D.z, D.w);
  n.u[0] = make_float2(U.x, U.y);
  n.u[1] = make_float2(U.z, U.w);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    n.Sc[j] = xyd::nb_sum(n.l[j].x, n.r[j].x, n.d[j].x, n.u[j].x);
    n.Ss[j] = xyd::nb_sum(n.l[j].y, n.r[j].y, n.d[j].y, n.u[j].y);
  }
}

// One lattice of a batch group (blockIdx.z), one sweep: the sweep index comes
// from the device counters and beta from the device (replica exchange moves
// it); the state ping-pongs between the batch's two buffers by sweep parity.
template <int MODE, int RED>
__global__ void __launch_bounds__(kNThreads, 6) k_sweep_narrow_batch(FusedBatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  NThArr* th = reinterpret_cast<NThArr*>(smem);
  NCsArr* cs = reinterpret_cast<NCsArr*>(smem + kNThBytes);
  float(*part)[5][2] = reinterpret_cast<float(*)[5][2]>(smem + kNThBytes + kNCsBytes);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(smem + kNThBytes + kNCsBytes + kNPartBytes);

  const int li = b.lattices[blockIdx.z];
  const uint32_t sweep = b.counters[0] + (uint32_t)b.s;
  const float* src = ((sweep & 1u) ? b.theta2 : b.theta) + b.offset[li];
  float* dst = ((sweep & 1u) ? b.theta : b.theta2) + b.offset[li];
  const double beta = b.beta[li];
  const float K = (float)(beta * b.J);
  const uint32_t lid = b.lattice_id0 + (uint32_t)li;
  xy_record* rec = b.records + (size_t)li * b.rec_stride + (sweep - b.rec_sweep0);

  const int L = b.L, W = b.L / 2;
  const int k0 = blockIdx.x * kNTileK;
  const int y0 = blockIdx.y * kNTileRows;
  const size_t plane = (size_t)L * (size_t)W;

  // ---- stage both planes (angle + unit vector) ----
  // Rows: the black plane's 36 (stage rows 0..35) then the red plane's 34
  // (stage rows 1..34); 4 lanes per row, one float4 per lane; the halo
  // columns k0-1 and k0+16 (rows 1..34) are a separate pass.
  {
    const int warp_s = threadIdx.x >> 5, lane_s = threadIdx.x & 31;
    const int sub = lane_s >> 2, g = lane_s & 3;
    constexpr int kRowsPerStep = 8 * kNWarps;
    constexpr int kSteps = (kNStageRowsTotal + kRowsPerStep - 1) / kRowsPerStep;
    float4 v[kSteps];
#pragma unroll
    for (int i = 0; i < kSteps; ++i) {
      const int rr = 8 * warp_s + sub + kRowsPerStep * i;
      v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rr < kNStageRowsTotal) {
        const int p = rr < kNSRows ? 1 : 0;
        const int r = rr < kNSRows ? rr : rr - kNSRows + 1;
        const size_t row = p * plane + (size_t)nwrap(y0 - 2 + r, L) * W + k0 + 4 * g;
        v[i] = __ldg(reinterpret_cast<const float4*>(src + row));
      }
    }
#pragma unroll
    for (int i = 0; i < kSteps; ++i) {
      const int rr = 8 * warp_s + sub + kRowsPerStep * i;
      if (rr < kNStageRowsTotal) {
        const int p = rr < kNSRows ? 1 : 0;
        const int r = rr < kNSRows ? rr : rr - kNSRows + 1;
        const int col = 4 + 4 * g;
        float s0, c0, s1, c1, s2, c2, s3, c3;
        xyd::unit_vector<MODE>(v[i].x, &s0, &c0);
        xyd::unit_vector<MODE>(v[i].y, &s1, &c1);
        xyd::unit_vector<MODE>(v[i].z, &s2, &c2);
        xyd::unit_vector<MODE>(v[i].w, &s3, &c3);
        *reinterpret_cast<float4*>(&th[p][r][col]) = v[i];
        *reinterpret_cast<float4*>(&cs[p][r][col]) = make_float4(c0, s0, c1, s1);
        *reinterpret_cast<float4*>(&cs[p][r][col + 2]) = make_float4(c2, s2, c3, s3);
      }
    }
    for (int h = kNThreads - 1 - threadIdx.x; h < 2 * (kNSRows - 2) * 2; h += kNThreads) {
      const int p = h / ((kNSRows - 2) * 2);
      const int rem = h - p * ((kNSRows - 2) * 2);
      const int r = 1 + (rem >> 1);
      const int side = rem & 1;
      const size_t row = p * plane + (size_t)nwrap(y0 - 2 + r, L) * W;
      const int kk = side ? nwrap(k0 + kNTileK, W) : nwrap(k0 - 1, W);
      const int col = side ? kNTileK + 4 : 3;
      const float v1 = __ldg(src + row + kk);
      float sv, cv;
      xyd::unit_vector<MODE>(v1, &sv, &cv);
      th[p][r][col] = v1;
      cs[p][r][col] = make_float2(cv, sv);
    }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t uL = (uint32_t)L;
  const int pr = lane & 7;                               // the thread's pair in its rows
  const int c0 = 2 * pr + 4;                             // stage column of the pair
  const int kp = k0 + 2 * pr;                            // plane column of the pair
  unsigned int n_acc = 0;

  // ---- red half: the tile (counted, written to dst) ----
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int ty = warp * 4 + (lane >> 3) + 16 * half;   // the tile row
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = y & 1;                                 // red: x = 2k + (y & 1)
    NPair n;
    npair_neighbours(cs[1], r, c0, q, n);
    const uint32_t site0 = (uint32_t)y * uL + 2u * (uint32_t)kp + (uint32_t)q;
    // sites x and x + 2 of the pair (kp even, so x & 2 == 0): one block
    const uint4 w = xyd::philox4x32_10(make_uint4(site0, sweep, lid, 1u), b.rk);
    const float2 t = *reinterpret_cast<const float2*>(&th[0][r][c0]);
    const float4 o = *reinterpret_cast<const float4*>(&cs[0][r][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w.x, w.y, K, b.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w.z, w.w, K, b.delta);
    n_acc += (r0.accept ? 1u : 0u) + (r1.accept ? 1u : 0u);
    *reinterpret_cast<float2*>(&th[0][r][c0]) = make_float2(r0.th, r1.th);
    *reinterpret_cast<float4*>(&cs[0][r][c0]) = make_float4(r0.c, r0.s, r1.c, r1.s);
    *reinterpret_cast<float2*>(dst + (size_t)y * W + kp) = make_float2(r0.th, r1.th);
  }
  // ---- red half: the ring at distance one (recomputed, not counted) ----
  // 64 sites on the first two warps, one per lane
  if (threadIdx.x < kNRing) {
    const int i = threadIdx.x;
    int gy, tk;
    if (i < kNTileK) {
      gy = -1;
      tk = i;
    } else if (i < 2 * kNTileK) {
      gy = kNTileRows;
      tk = i - kNTileK;
    } else {
      gy = i - 2 * kNTileK;
      tk = ((y0 + gy) & 1) ? -1 : kNTileK;               // left ring on odd rows, right on even
    }
    const int yy = nwrap(y0 + gy, L);
    const int kk = nwrap(k0 + tk, W);
    const int q = yy & 1;
    const int rr = gy + 2, c = tk + 4;
    const uint32_t x = 2u * (uint32_t)kk + (uint32_t)q;
    const uint32_t site = (uint32_t)yy * uL + x;
    const float2 l = cs[1][rr][c + q - 1], rt = cs[1][rr][c + q];
    const float2 d = cs[1][rr - 1][c], u = cs[1][rr + 1][c];
    const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
    const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
    const uint4 w =
        xyd::philox4x32_10(make_uint4(xyd::metropolis_counter(site, x), sweep, lid, 1u), b.rk);
    const uint2 uw = xyd::metropolis_words(w, x);
    const float2 own = cs[0][rr][c];
    const xyd::SiteResult res =
        xyd::metropolis_step<MODE>(th[0][rr][c], own.x, own.y, Sc, Ss, uw.x, uw.y, K, b.delta);
    th[0][rr][c] = res.th;
    cs[0][rr][c] = make_float2(res.c, res.s);
  }
  __syncthreads();

  // ---- black half of the tile, with the sweep sums ----
  xyd::SweepSums<RED> sums;                      // 4 black sites per thread
  sums.init();
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int ty = warp * 4 + (lane >> 3) + 16 * half;   // the tile row
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = (y + 1) & 1;                           // black: x = 2k + ((y + 1) & 1)
    NPair n;
    npair_neighbours(cs[0], r, c0, q, n);
    const uint32_t site0 = (uint32_t)y * uL + 2u * (uint32_t)kp + (uint32_t)q;
    // sites x and x + 2 of the pair (kp even, so x & 2 == 0): one block
    const uint4 w = xyd::philox4x32_10(make_uint4(site0, sweep, lid, 1u), b.rk);
    const float2 t = *reinterpret_cast<const float2*>(&th[1][r][c0]);
    const float4 o = *reinterpret_cast<const float4*>(&cs[1][r][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w.x, w.y, K, b.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w.z, w.w, K, b.delta);
    n_acc += (r0.accept ? 1u : 0u) + (r1.accept ? 1u : 0u);
    *reinterpret_cast<float2*>(dst + plane + (size_t)y * W + kp) = make_float2(r0.th, r1.th);

    // red sites with the same (y, k): their spins enter M once each
    const float4 m = *reinterpret_cast<const float4*>(&cs[0][r][c0]);
    float v0[5], v1[5];
    xyd::measure_terms(r0.c, r0.s, n.l[0].x, n.l[0].y, n.r[0].x, n.r[0].y, n.d[0].x, n.d[0].y,
                       n.u[0].x, n.u[0].y, n.Sc[0], n.Ss[0], m.x, m.y, v0);
    xyd::measure_terms(r1.c, r1.s, n.l[1].x, n.l[1].y, n.r[1].x, n.r[1].y, n.d[1].x, n.d[1].y,
                       n.u[1].x, n.u[1].y, n.Sc[1], n.Ss[1], m.z, m.w, v1);
    sums.add2(v0, v1);
  }
  xyd::commit_sums<kNWarps, RED, true>(sums, n_acc, part, cnt, rec, beta,
                                       blockIdx.x == 0 && blockIdx.y == 0);
}

template <int MODE, int RED>
cudaError_t prepare_narrow_one() {
  cudaError_t e = cudaFuncSetAttribute(k_sweep_narrow_batch<MODE, RED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sweep_narrow_batch<MODE, RED>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

template <int MODE, int RED>
cudaError_t launch_narrow_one(const FusedBatchArgs& b, int n_lattices, cudaStream_t stream) {
  const dim3 grid(b.L / 2 / kNTileK, b.L / kNTileRows, n_lattices);
  k_sweep_narrow_batch<MODE, RED><<<grid, kNThreads, kNSmemBytes, stream>>>(b);
  return cudaGetLastError();
}

}  // namespace

bool narrow_supported(int L) { return L >= 32 && (L % 32) == 0; }

int narrow_tiles(int L) { return narrow_supported(L) ? (L / 2 / kNTileK) * (L / kNTileRows) : 0; }

cudaError_t prepare_narrow_batch(int sincos_mode, int reduce_mode) {
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? prepare_narrow_one<0, 1>() : prepare_narrow_one<0, 0>();
    case 1: return comp ? prepare_narrow_one<1, 1>() : prepare_narrow_one<1, 0>();
    default: return comp ? prepare_narrow_one<2, 1>() : prepare_narrow_one<2, 0>();
  }
}

cudaError_t launch_narrow_batch_sweep(int sincos_mode, int reduce_mode, const FusedBatchArgs& b,
                                      int n_lattices, cudaStream_t stream) {
  if (!narrow_supported(b.L) || n_lattices < 1) return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0:
      return comp ? launch_narrow_one<0, 1>(b, n_lattices, stream)
                  : launch_narrow_one<0, 0>(b, n_lattices, stream);
    case 1:
      return comp ? launch_narrow_one<1, 1>(b, n_lattices, stream)
                  : launch_narrow_one<1, 0>(b, n_lattices, stream);
    default:
      return comp ? launch_narrow_one<2, 1>(b, n_lattices, stream)
                  : launch_narrow_one<2, 0>(b, n_lattices, stream);
  }
}

}  // namespace xyk

// ---------------------------------------------------------------------------
// Whole lattices in one CTA: the batch's lattices small enough for one CTA's
// shared memory (12 bytes per site: angle and unit vector) run all sweeps of a
// round in one launch, one CTA per lattice, the lattice never leaving shared
// memory between the round's first read and last write.  A half-sweep is a
// pass over the sites of one colour against the other colour's unit vectors
// (periodic neighbours straight from shared memory: no halo, no recomputed
// ring), with a barrier between the halves.  Each site's unit vector is
// computed once at the start and then carried: after an update it is the one
// xyd::metropolis_step returns (the proposal's if accepted, else the old
// one), which is exactly what recomputing it from the stored angle would give,
// so every site update -- and each lattice's state -- is bit for bit that of
// the single-lattice kernels, at one sincos per update instead of two.
// ---------------------------------------------------------------------------
namespace xyk {

namespace {

constexpr int kSThreads = 256;
constexpr int kSWarps = kSThreads / 32;
constexpr size_t kSTailBytes = sizeof(float) * kSWarps * 5 * 2 + sizeof(unsigned int) * kSWarps;

template <int MODE, int RED>
__global__ void __launch_bounds__(kSThreads, 2) k_batch_small(SmallBatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int li = a.lattices[blockIdx.x];
  const int L = a.L[li], W = L / 2;
  const int half = L * W;                                   // sites per colour
  float* th = reinterpret_cast<float*>(smem);               // [2][L][W]
  float2* cs = reinterpret_cast<float2*>(smem + (((size_t)2 * half * sizeof(float) + 15) & ~(size_t)15));
  unsigned char* tail = reinterpret_cast<unsigned char*>(cs + 2 * half);
  float(*part)[5][2] = reinterpret_cast<float(*)[5][2]>(tail);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(tail + sizeof(float) * kSWarps * 5 * 2);

  const uint32_t sweep0 = a.counters[0];
  const uint32_t last = sweep0 + (uint32_t)a.sweeps - 1u;
  const float* src = ((sweep0 & 1u) ? a.theta2 : a.theta) + a.offset[li];
  float* dst = ((last & 1u) ? a.theta : a.theta2) + a.offset[li];
  const double beta = a.beta[li];
  const float K = (float)(beta * a.J);
  const uint32_t lid = a.lattice_id0 + (uint32_t)li;
  const uint32_t uL = (uint32_t)L;
  // a half-sweep spreads one colour's L*W sites evenly over the threads (a
  // warp may straddle rows): thread t starts at flat index t = y0*W + k0 and
  // steps by kSThreads = dy*W + dk, the (y, k) carried without a division
  const int y0 = threadIdx.x / W, k0 = threadIdx.x % W;
  const int dy = kSThreads / W, dk = kSThreads % W;
  auto step_site = [&](int& y, int& k) {
    k += dk;
    y += dy;
    if (k >= W) {
      k -= W;
      ++y;
    }
  };
  // with W even a thread takes both sites of a pair, (y, 2m) and (y, 2m + 1)
  // -- the sites x and x + 2 that share one Philox block -- stepping over the
  // L*W/2 pairs the same way; with W odd (L % 4 == 2) a site at a time
  const bool paired = (W & 1) == 0;
  const int Wp = paired ? W / 2 : 1;
  const int npairs = half / 2;
  const int py0 = threadIdx.x / Wp, pm0 = threadIdx.x % Wp;
  const int pdy = kSThreads / Wp, pdm = kSThreads % Wp;
  auto step_pair = [&](int& y, int& m) {
    m += pdm;
    y += pdy;
    if (m >= Wp) {
      m -= Wp;
      ++y;
    }
  };

  for (int i = threadIdx.x; i < 2 * half; i += kSThreads) {
    const float t = __ldg(src + i);
    float s, c;
    xyd::unit_vector<MODE>(t, &s, &c);
    th[i] = t;
    cs[i] = make_float2(c, s);
  }
  __syncthreads();

  for (int sw = 0; sw < a.sweeps; ++sw) {
    const uint32_t sweep = sweep0 + (uint32_t)sw;
    unsigned int n_acc = 0;
    // at most L^2 / 2 / 256 = 18 black sites per thread (L <= 96)
    xyd::SweepSums<RED> sums;
    sums.init();
    auto add_terms = [&](const float* v) { sums.add(v); };
    if (paired) {
      // ---- red half, a pair per step: sites k = 2m and k + 1 of row y
      // (flat index o = 2P); left/right neighbours k+q-1, k+q for the first,
      // k+q, k+q+1 for the second ----
      for (int P = threadIdx.x, y = py0, m = pm0; P < npairs; P += kSThreads) {
        // debug build: the carried (y, m) is the pair's position, in range
        if (!XY_DCHECK(y >= 0 && y < L && m >= 0 && m < Wp && y * Wp + m == P, 0)) {
          step_pair(y, m);
          continue;
        }
        const int k = 2 * m, o = 2 * P;
        const int q = y & 1;
        const int yd = y == 0 ? L - 1 : y - 1, yu = y == L - 1 ? 0 : y + 1;
        int kl = k + q - 1, kr = k + q + 1;
        kl += kl < 0 ? W : 0;
        kr -= kr >= W ? W : 0;
        const float2* row = cs + half + y * W;
        const float2 lf = row[kl], md = row[k + q], rg = row[kr];
        const float4 dn = *reinterpret_cast<const float4*>(cs + half + yd * W + k);
        const float4 up = *reinterpret_cast<const float4*>(cs + half + yu * W + k);
        const float Sc0 = xyd::nb_sum(lf.x, md.x, dn.x, up.x);
        const float Ss0 = xyd::nb_sum(lf.y, md.y, dn.y, up.y);
        const float Sc1 = xyd::nb_sum(md.x, rg.x, dn.z, up.z);
        const float Ss1 = xyd::nb_sum(md.y, rg.y, dn.w, up.w);
        const uint32_t x0 = 2u * (uint32_t)k + (uint32_t)q;          // x0 & 2 == 0
        const uint4 w =
            xyd::philox4x32_10(make_uint4((uint32_t)y * uL + x0, sweep, lid, 1u), a.rk);
        const float2 t = *reinterpret_cast<const float2*>(th + o);
        const float4 own = *reinterpret_cast<const float4*>(cs + o);
        const xyd::SiteResult r0 =
            xyd::metropolis_step<MODE>(t.x, own.x, own.y, Sc0, Ss0, w.x, w.y, K, a.delta);
        const xyd::SiteResult r1 =
            xyd::metropolis_step<MODE>(t.y, own.z, own.w, Sc1, Ss1, w.z, w.w, K, a.delta);
        *reinterpret_cast<float2*>(th + o) = make_float2(r0.th, r1.th);
        *reinterpret_cast<float4*>(cs + o) = make_float4(r0.c, r0.s, r1.c, r1.s);
        n_acc += (r0.accept ? 1u : 0u) + (r1.accept ? 1u : 0u);
        step_pair(y, m);
      }
      __syncthreads();
      // ---- black half, a pair per step, with the sweep sums ----
      for (int P = threadIdx.x, y = py0, m = pm0; P < npairs; P += kSThreads) {
        // debug build: the carried (y, m) is the pair's position, in range
        if (!XY_DCHECK(y >= 0 && y < L && m >= 0 && m < Wp && y * Wp + m == P, 0)) {
          step_pair(y, m);
          continue;
        }
        const int k = 2 * m, o = half + 2 * P;
        const int q = (y + 1) & 1;
        const int yd = y == 0 ? L - 1 : y - 1, yu = y == L - 1 ? 0 : y + 1;
        int kl = k + q - 1, kr = k + q + 1;
        kl += kl < 0 ? W : 0;
        kr -= kr >= W ? W : 0;
        const float2* row = cs + y * W;
        const float2 lf = row[kl], md = row[k + q], rg = row[kr];
        const float4 dn = *reinterpret_cast<const float4*>(cs + yd * W + k);
        const float4 up = *reinterpret_cast<const float4*>(cs + yu * W + k);
        const float Sc0 = xyd::nb_sum(lf.x, md.x, dn.x, up.x);
        const float Ss0 = xyd::nb_sum(lf.y, md.y, dn.y, up.y);
        const float Sc1 = xyd::nb_sum(md.x, rg.x, dn.z, up.z);
        const float Ss1 = xyd::nb_sum(md.y, rg.y, dn.w, up.w);
        const uint32_t x0 = 2u * (uint32_t)k + (uint32_t)q;          // x0 & 2 == 0
        const uint4 w =
            xyd::philox4x32_10(make_uint4((uint32_t)y * uL + x0, sweep, lid, 1u), a.rk);
        const float2 t = *reinterpret_cast<const float2*>(th + o);
        const float4 own = *reinterpret_cast<const float4*>(cs + o);
        const xyd::SiteResult r0 =
            xyd::metropolis_step<MODE>(t.x, own.x, own.y, Sc0, Ss0, w.x, w.y, K, a.delta);
        const xyd::SiteResult r1 =
            xyd::metropolis_step<MODE>(t.y, own.z, own.w, Sc1, Ss1, w.z, w.w, K, a.delta);
        *reinterpret_cast<float2*>(th + o) = make_float2(r0.th, r1.th);
        *reinterpret_cast<float4*>(cs + o) = make_float4(r0.c, r0.s, r1.c, r1.s);
        n_acc += (r0.accept ? 1u : 0u) + (r1.accept ? 1u : 0u);
        // the red sites with the same (y, k) and (y, k + 1) enter M once each
        const float4 mr = *reinterpret_cast<const float4*>(cs + 2 * P);
        float v[5];
        xyd::measure_terms(r0.c, r0.s, lf.x, lf.y, md.x, md.y, dn.x, dn.y, up.x, up.y, Sc0, Ss0,
                           mr.x, mr.y, v);
        add_terms(v);
        xyd::measure_terms(r1.c, r1.s, md.x, md.y, rg.x, rg.y, dn.z, dn.w, up.z, up.w, Sc1, Ss1,
                           mr.z, mr.w, v);
        add_terms(v);
        step_pair(y, m);
      }
    } else {
      // ---- red half: red site (y, k) is x = 2k + (y & 1); its black
      // neighbours (y, k+q-1), (y, k+q), (y-1, k), (y+1, k) ----
      for (int o = threadIdx.x, y = y0, k = k0; o < half; o += kSThreads) {
        if (!XY_DCHECK(y >= 0 && y < L && k >= 0 && k < W && y * W + k == o, 1)) {
          step_site(y, k);
          continue;
        }
        const int q = y & 1;
        const int yd = y == 0 ? L - 1 : y - 1, yu = y == L - 1 ? 0 : y + 1;
        int kl = k + q - 1, kr = k + q;
        kl += kl < 0 ? W : 0;
        kr -= kr >= W ? W : 0;
        const float2 l = cs[half + y * W + kl], rt = cs[half + y * W + kr];
        const float2 d = cs[half + yd * W + k], u = cs[half + yu * W + k];
        const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
        const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
        const uint32_t x = 2u * (uint32_t)k + (uint32_t)q;
        const uint4 w = xyd::philox4x32_10(
            make_uint4(xyd::metropolis_counter((uint32_t)y * uL + x, x), sweep, lid, 1u), a.rk);
        const uint2 uw = xyd::metropolis_words(w, x);
        const float2 own = cs[o];
        const xyd::SiteResult res =
            xyd::metropolis_step<MODE>(th[o], own.x, own.y, Sc, Ss, uw.x, uw.y, K, a.delta);
        th[o] = res.th;
        cs[o] = make_float2(res.c, res.s);
        n_acc += res.accept ? 1u : 0u;
        step_site(y, k);
      }
      __syncthreads();
      // ---- black half, with the sweep sums: black site (y, k) is
      // x = 2k + ((y + 1) & 1); its red neighbours as above ----
      for (int i = threadIdx.x, y = y0, k = k0; i < half; i += kSThreads) {
        if (!XY_DCHECK(y >= 0 && y < L && k >= 0 && k < W && y * W + k == i, 1)) {
          step_site(y, k);
          continue;
        }
        const int q = (y + 1) & 1;
        const int yd = y == 0 ? L - 1 : y - 1, yu = y == L - 1 ? 0 : y + 1;
        int kl = k + q - 1, kr = k + q;
        kl += kl < 0 ? W : 0;
        kr -= kr >= W ? W : 0;
        const float2 l = cs[y * W + kl], rt = cs[y * W + kr];
        const float2 d = cs[yd * W + k], u = cs[yu * W + k];
        const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
        const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
        const uint32_t x = 2u * (uint32_t)k + (uint32_t)q;
        const uint4 w = xyd::philox4x32_10(
            make_uint4(xyd::metropolis_counter((uint32_t)y * uL + x, x), sweep, lid, 1u), a.rk);
        const uint2 uw = xyd::metropolis_words(w, x);
        const int o = half + i;
        const float2 own = cs[o];
        const xyd::SiteResult res =
            xyd::metropolis_step<MODE>(th[o], own.x, own.y, Sc, Ss, uw.x, uw.y, K, a.delta);
        th[o] = res.th;
        cs[o] = make_float2(res.c, res.s);
        n_acc += res.accept ? 1u : 0u;
        // the red site with the same (y, k): its spin enters M once
        const float2 m = cs[i];
        float v[5];
        xyd::measure_terms(res.c, res.s, l.x, l.y, rt.x, rt.y, d.x, d.y, u.x, u.y, Sc, Ss, m.x,
                           m.y, v);
        add_terms(v);
        step_site(y, k);
      }
    }
    // (its barrier also ends the black half before the next sweep's red half)
    xyd::commit_sums<kSWarps, RED, true>(
        sums, n_acc, part, cnt,
        a.records + (size_t)li * a.rec_stride + (sweep - a.rec_sweep0), beta, true);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * half; i += kSThreads) dst[i] = th[i];
}

template <int MODE, int RED>
cudaError_t launch_small_one(const SmallBatchArgs& a, int n_lattices, size_t smem,
                             cudaStream_t stream) {
  k_batch_small<MODE, RED><<<n_lattices, kSThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

template <int MODE, int RED>
cudaError_t prepare_small_one(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_small<MODE, RED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_batch_small<MODE, RED>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

}  // namespace

size_t small_smem_bytes(int L) {
  const size_t half = (size_t)L * (size_t)(L / 2);
  return ((2 * half * sizeof(float) + 15) & ~(size_t)15) + 2 * half * sizeof(float2) + kSTailBytes;
}

bool small_supported(int L) { return L >= 2 && (L % 2) == 0 && small_smem_bytes(L) <= kSmallBudget; }

cudaError_t prepare_small_batch(int sincos_mode, int reduce_mode, size_t smem) {
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? prepare_small_one<0, 1>(smem) : prepare_small_one<0, 0>(smem);
    case 1: return comp ? prepare_small_one<1, 1>(smem) : prepare_small_one<1, 0>(smem);
    default: return comp ? prepare_small_one<2, 1>(smem) : prepare_small_one<2, 0>(smem);
  }
}

cudaError_t launch_small_batch(int sincos_mode, int reduce_mode, const SmallBatchArgs& a,
                               int n_lattices, size_t smem, cudaStream_t stream) {
  if (n_lattices < 1 || a.sweeps < 1 || smem > kSmallBudget) return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_small_one<0, 1>(a, n_lattices, smem, stream)
                        : launch_small_one<0, 0>(a, n_lattices, smem, stream);
    case 1: return comp ? launch_small_one<1, 1>(a, n_lattices, smem, stream)
                        : launch_small_one<1, 0>(a, n_lattices, smem, stream);
    default: return comp ? launch_small_one<2, 1>(a, n_lattices, smem, stream)
                         : launch_small_one<2, 0>(a, n_lattices, smem, stream);
  }
}

}  // namespace xyk

namespace xyk {

// The debug word of this translation unit (whole-lattice and narrow batch
// kernels; bits 0-1), read and cleared.  0 in the release build.
unsigned int debug_take_narrow() { return xy_debug_take_word(); }

}  // namespace xyk
