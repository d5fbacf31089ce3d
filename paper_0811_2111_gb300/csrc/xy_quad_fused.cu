// xy_quad_fused.cu -- one-launch sweep of four replicas per site (the RGBA
// packing of Sec. 3.2): red half, black half and the four replicas' sweep sums
// in one kernel, reading the state from `src` and writing it to `dst`.
//
// A plane of float4 sites [y][k] is read as a plane of floats [y][4k + r]
// (r = replica): element f = 4k + r has its same-row neighbours, of the same
// replica, at f - 4 and f + 4 (the site's k + q - 1 and k + q in the other
// colour) and its up/down neighbours at f in the rows y -/+ 1.  Each CTA owns
// 32 rows x 64 elements (16 sites x 4 replicas) of both colours and stages
// both planes of that tile plus two halo rows and one halo site (4 elements)
// per side as (angle, cos, sin), then
//   1. updates the red elements of the tile and of the ring at distance one
//      (rows -1 and 32, and the halo site on the side the black tile needs;
//      recomputed from the same old state and the same Philox words as the
//      neighbouring tiles' own updates, hence identical),
//   2. updates the black elements against the new red ones,
//   3. accumulates each replica's sweep sums,
// and writes the tile's new angles to `dst`.  Every element runs the
// single-lattice arithmetic (xyd::metropolis_step with Philox counter
// (site, sweep, lattice_id0 + r, 1) and K_r = beta_r J), so replica r is bit
// for bit the single lattice with lattice id lattice_id0 + r.
//
// A lane updates two adjacent elements -- two replicas of one site -- so its
// same-row neighbours are two aligned float4 loads of (cos, sin) pairs.
// Requires L % 32 == 0 (then 4W = 2L is a multiple of 64).
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_device.cuh"
#include "xy_internal.h"

namespace xyk {

namespace {

constexpr int kR = 4;                        // replicas per site
constexpr int kTileRows = 32;
constexpr int kTileF = 64;                   // elements per tile row (16 sites x 4 replicas)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSRows = kTileRows + 4;        // rows y0-2 .. y0+33
constexpr int kSCols = kTileF + 8;           // elements f0-4 .. f0+67 (one halo site per side)
constexpr int kRing = 2 * kTileF + kTileRows * kR;   // 256 ring elements, one per thread
constexpr int kStageRowsTotal = kSRows + (kSRows - 2);

constexpr size_t kThBytes = sizeof(float) * 2 * kSRows * kSCols;
constexpr size_t kCsBytes = sizeof(float2) * 2 * kSRows * kSCols;
constexpr size_t kPartBytes = sizeof(float) * kWarps * kR * 5 * 2;
constexpr size_t kCntBytes = sizeof(unsigned int) * kWarps * kR;
constexpr size_t kSmemBytes = kThBytes + kCsBytes + kPartBytes + kCntBytes;

static_assert(kRing == kThreads, "one ring element per thread");

typedef float ThArr[kSRows][kSCols];
typedef float2 CsArr[kSRows][kSCols];

__device__ __forceinline__ int wrap_once(int v, int n) {
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}

// Sum over the 16 lanes of one parity (lane & 1): those lanes hold the same
// pair of replicas.
__device__ __forceinline__ float parity_sum(float v) {
#pragma unroll
  for (int o = 16; o > 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned int parity_sum(unsigned int v) {
#pragma unroll
  for (int o = 16; o > 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// K of replica j (j in 0..3, not known at compile time) without indexing the
// parameter array.
__device__ __forceinline__ float replica_k(const QuadFusedArgs& a, int j) {
  const float k01 = (j & 1) ? a.K[1] : a.K[0];
  const float k23 = (j & 1) ? a.K[3] : a.K[2];
  return (j & 2) ? k23 : k01;
}

// Two adjacent elements (replicas j0, j0 + 1 of one site) of row r at stage
// columns c0, c0 + 1 of colour `own`, against the other colour's plane `nb`:
// same-row neighbours of the site at k + q - 1 (columns c0 + 4q - 4, +1) and
// k + q (c0 + 4q, +1).
struct PairNb {
  float Sc[2], Ss[2];
  float2 l[2], r[2], d[2], u[2];
};

__device__ __forceinline__ void pair_nb(const CsArr& nb, int r, int c0, int q, PairNb& n) {
  const float4 Lf = *reinterpret_cast<const float4*>(&nb[r][c0 + 4 * q - 4]);
  const float4 Rt = *reinterpret_cast<const float4*>(&nb[r][c0 + 4 * q]);
  const float4 D = *reinterpret_cast<const float4*>(&nb[r - 1][c0]);
  const float4 U = *reinterpret_cast<const float4*>(&nb[r + 1][c0]);
  n.l[0] = make_float2(Lf.x, Lf.y);
  n.l[1] = make_float2(Lf.z, Lf.w);
  n.r[0] = make_float2(Rt.x, Rt.y);
  n.r[1] = make_float2(Rt.z, Rt.w);
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

template <int MODE, int RED>
__global__ void __launch_bounds__(kThreads, 3) k_quad_fused(QuadFusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  ThArr* th = reinterpret_cast<ThArr*>(smem);
  CsArr* cs = reinterpret_cast<CsArr*>(smem + kThBytes);
  float(*part)[kR][5][2] = reinterpret_cast<float(*)[kR][5][2]>(smem + kThBytes + kCsBytes);
  unsigned int(*cnt)[kR] =
      reinterpret_cast<unsigned int(*)[kR]>(smem + kThBytes + kCsBytes + kPartBytes);

  const int L = a.L, W = a.W;
  const int F = 4 * W;                                     // elements per plane row
  const int f0 = blockIdx.x * kTileF;                      // first element of the tile
  const int ks0 = f0 >> 2;                                 // its first site column
  const int y0 = blockIdx.y * kTileRows;
  const size_t plane = (size_t)L * (size_t)F;

  // ---- stage both planes (angle + unit vector) ----
  // Rows: the black plane's 36 (stage rows 0..35) then the red plane's 34
  // (stage rows 1..34); 16 lanes per row, one float4 (one site, four
  // replicas) per lane; the halo sites ks0 - 1 and ks0 + 16 (rows 1..34) are
  // a separate pass taken by the last warps.
  {
    const int warp_s = threadIdx.x >> 5, lane_s = threadIdx.x & 31;
    const int half = lane_s >> 4, g = lane_s & 15;
    constexpr int kSteps = (kStageRowsTotal + 2 * kWarps - 1) / (2 * kWarps);
    float4 v[kSteps];
#pragma unroll
    for (int i = 0; i < kSteps; ++i) {
      const int rr = 2 * warp_s + half + 2 * kWarps * i;
      v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rr < kStageRowsTotal) {
        const int p = rr < kSRows ? 1 : 0;
        const int r = rr < kSRows ? rr : rr - kSRows + 1;
        const size_t row = p * plane + (size_t)wrap_once(y0 - 2 + r, L) * F + f0 + 4 * g;
        v[i] = __ldg(reinterpret_cast<const float4*>(a.src + row));
      }
    }
#pragma unroll
    for (int i = 0; i < kSteps; ++i) {
      const int rr = 2 * warp_s + half + 2 * kWarps * i;
      if (rr < kStageRowsTotal) {
        const int p = rr < kSRows ? 1 : 0;
        const int r = rr < kSRows ? rr : rr - kSRows + 1;
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
    for (int h = kThreads - 1 - threadIdx.x; h < 2 * (kSRows - 2) * 2; h += kThreads) {
      const int p = h / ((kSRows - 2) * 2);
      const int rem = h - p * ((kSRows - 2) * 2);
      const int r = 1 + (rem >> 1);
      const int side = rem & 1;
      const int ks = side ? wrap_once(ks0 + kTileF / 4, W) : wrap_once(ks0 - 1, W);
      const size_t at = p * plane + (size_t)wrap_once(y0 - 2 + r, L) * F + 4 * (size_t)ks;
      const int col = side ? kTileF + 4 : 0;
      const float4 t = __ldg(reinterpret_cast<const float4*>(a.src + at));
      float s0, c0, s1, c1, s2, c2, s3, c3;
      xyd::unit_vector<MODE>(t.x, &s0, &c0);
      xyd::unit_vector<MODE>(t.y, &s1, &c1);
      xyd::unit_vector<MODE>(t.z, &s2, &c2);
      xyd::unit_vector<MODE>(t.w, &s3, &c3);
      *reinterpret_cast<float4*>(&th[p][r][col]) = t;
      *reinterpret_cast<float4*>(&cs[p][r][col]) = make_float4(c0, s0, c1, s1);
      *reinterpret_cast<float4*>(&cs[p][r][col + 2]) = make_float4(c2, s2, c3, s3);
    }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t uL = (uint32_t)L;
  const int c0 = 2 * lane + 4;                             // stage column of the lane's pair
  const int fp = f0 + 2 * lane;                            // element of the pair
  const int j0 = fp & 3;                                   // its replicas j0, j0 + 1
  const uint32_t kq = (uint32_t)(fp >> 2);                 // its site column
  const uint32_t id0 = a.lattice_id0 + (uint32_t)j0, id1 = id0 + 1u;
  const float K0 = (lane & 1) ? a.K[2] : a.K[0];
  const float K1 = (lane & 1) ? a.K[3] : a.K[1];
  unsigned int n_acc[2] = {0u, 0u};

  // ---- red half: the tile (counted, written to dst) ----
#pragma unroll 2
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = y & 1;                                   // red: x = 2k + (y & 1)
    PairNb n;
    pair_nb(cs[1], r, c0, q, n);
    const uint32_t site = (uint32_t)y * uL + 2u * kq + (uint32_t)q;
    const uint4 w0 = xyd::philox4x32_10(make_uint4(site, a.sweep, id0, 1u), a.rk);
    const uint4 w1 = xyd::philox4x32_10(make_uint4(site, a.sweep, id1, 1u), a.rk);
    const float2 t = *reinterpret_cast<const float2*>(&th[0][r][c0]);
    const float4 o = *reinterpret_cast<const float4*>(&cs[0][r][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w0.x, w0.y, K0, a.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w1.x, w1.y, K1, a.delta);
    n_acc[0] += r0.accept ? 1u : 0u;
    n_acc[1] += r1.accept ? 1u : 0u;
    *reinterpret_cast<float2*>(&th[0][r][c0]) = make_float2(r0.th, r1.th);
    *reinterpret_cast<float4*>(&cs[0][r][c0]) = make_float4(r0.c, r0.s, r1.c, r1.s);
    *reinterpret_cast<float2*>(a.dst + (size_t)y * F + fp) = make_float2(r0.th, r1.th);
  }
  // ---- red half: the ring at distance one (recomputed, not counted) ----
  // elements 0..63: row -1; 64..127: row 32; 128..255: the halo site of rows
  // 0..31 on the side the black tile reaches (left on odd rows, right on even)
  {
    const int i = threadIdx.x;
    int ty, sc;
    if (i < kTileF) {
      ty = -1;
      sc = 4 + i;
    } else if (i < 2 * kTileF) {
      ty = kTileRows;
      sc = 4 + i - kTileF;
    } else {
      const int e = i - 2 * kTileF;
      ty = e >> 2;
      sc = (((y0 + ty) & 1) ? 0 : kTileF + 4) + (e & 3);
    }
    const int r = ty + 2;
    const int y = wrap_once(y0 + ty, L);
    const int q = y & 1;
    const int ks = wrap_once(ks0 + ((sc - 4) >> 2), W);   // floor: stage columns 0..3 -> ks0 - 1
    const int j = sc & 3;
    const uint32_t site = (uint32_t)y * uL + 2u * (uint32_t)ks + (uint32_t)q;
    const float2 l = cs[1][r][sc + 4 * q - 4], rt = cs[1][r][sc + 4 * q];
    const float2 d = cs[1][r - 1][sc], u = cs[1][r + 1][sc];
    const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
    const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
    const uint4 w =
        xyd::philox4x32_10(make_uint4(site, a.sweep, a.lattice_id0 + (uint32_t)j, 1u), a.rk);
    const float2 own = cs[0][r][sc];
    const xyd::SiteResult res = xyd::metropolis_step<MODE>(th[0][r][sc], own.x, own.y, Sc, Ss,
                                                           w.x, w.y, replica_k(a, j), a.delta);
    th[0][r][sc] = res.th;
    cs[0][r][sc] = make_float2(res.c, res.s);
  }
  __syncthreads();

  // ---- black half of the tile, with the sweep sums ----
  float acc[2][5], cmp[2][5];
#pragma unroll
  for (int e = 0; e < 2; ++e)
#pragma unroll
    for (int i = 0; i < 5; ++i) acc[e][i] = cmp[e][i] = 0.f;
  float* dst_blk = a.dst + plane;
#pragma unroll 2
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = (y + 1) & 1;                             // black: x = 2k + ((y + 1) & 1)
    PairNb n;
    pair_nb(cs[0], r, c0, q, n);
    const uint32_t site = (uint32_t)y * uL + 2u * kq + (uint32_t)q;
    const uint4 w0 = xyd::philox4x32_10(make_uint4(site, a.sweep, id0, 1u), a.rk);
    const uint4 w1 = xyd::philox4x32_10(make_uint4(site, a.sweep, id1, 1u), a.rk);
    const float2 t = *reinterpret_cast<const float2*>(&th[1][r][c0]);
    const float4 o = *reinterpret_cast<const float4*>(&cs[1][r][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w0.x, w0.y, K0, a.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w1.x, w1.y, K1, a.delta);
    n_acc[0] += r0.accept ? 1u : 0u;
    n_acc[1] += r1.accept ? 1u : 0u;
    *reinterpret_cast<float2*>(dst_blk + (size_t)y * F + fp) = make_float2(r0.th, r1.th);

    // red elements with the same (y, k, replica): their spins enter M once each
    const float4 m = *reinterpret_cast<const float4*>(&cs[0][r][c0]);
    float v0[5], v1[5];
    xyd::measure_terms(r0.c, r0.s, n.l[0].x, n.l[0].y, n.r[0].x, n.r[0].y, n.d[0].x, n.d[0].y,
                       n.u[0].x, n.u[0].y, n.Sc[0], n.Ss[0], m.x, m.y, v0);
    xyd::measure_terms(r1.c, r1.s, n.l[1].x, n.l[1].y, n.r[1].x, n.r[1].y, n.d[1].x, n.d[1].y,
                       n.u[1].x, n.u[1].y, n.Sc[1], n.Ss[1], m.z, m.w, v1);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      if (RED == 0) {
        acc[0][i] += v0[i];
        acc[1][i] += v1[i];
      } else {
        xyd::neumaier_add(acc[0][i], cmp[0][i], v0[i]);
        xyd::neumaier_add(acc[1][i], cmp[1][i], v1[i]);
      }
    }
  }

  // ---- per-replica sums: lanes of one parity -> warps -> FP64 -> records ----
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    n_acc[e] = parity_sum(n_acc[e]);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      acc[e][i] = parity_sum(acc[e][i]);
      if (RED == 1) cmp[e][i] = parity_sum(cmp[e][i]);
    }
  }
  if (lane < 2) {                                          // lane 0: replicas 0, 1; lane 1: 2, 3
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      cnt[warp][j0 + e] = n_acc[e];
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        part[warp][j0 + e][i][0] = acc[e][i];
        part[warp][j0 + e][i][1] = (RED == 1) ? cmp[e][i] : 0.f;
      }
    }
  }
  __syncthreads();
  if (warp != 0) return;
  const bool first_block = blockIdx.x == 0 && blockIdx.y == 0;
  if (lane < kR) {
    unsigned long long total = 0;
    for (int w = 0; w < kWarps; ++w) total += cnt[w][lane];
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.rec[lane].accepted), total);
    if (first_block) a.rec[lane].beta = a.beta[lane];
  }
  if (lane >= kR * 5) return;
  // lanes 0..19 each own one (replica, sum)
  const int jr = lane / 5, si = lane - 5 * jr;
  double d;
  if (RED == 0) {
    d = 0.0;
    for (int w = 0; w < kWarps; ++w) d += (double)part[w][jr][si][0];
  } else {
    float hi = 0.f, lo = 0.f;
    for (int w = 0; w < kWarps; ++w) {
      xyd::neumaier_add(hi, lo, part[w][jr][si][0]);
      lo += part[w][jr][si][1];
    }
    d = (double)hi + (double)lo;
  }
  const double scaled = d * (double)(1ll << XY_FX_SHIFT);
  if (!(fabs(scaled) < 9.0e18)) {
    atomicOr(reinterpret_cast<unsigned long long*>(&a.rec[jr].flags), 1ull);
    return;
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(&a.rec[jr].sum[si]),
            (unsigned long long)__double2ll_rn(scaled));
}

template <int MODE, int RED>
cudaError_t launch_one(const QuadFusedArgs& a, cudaStream_t stream) {
  static bool configured[64] = {};   // attributes set once per instantiation and device
  int dev = 0;
  cudaError_t ge = cudaGetDevice(&dev);
  if (ge != cudaSuccess) return ge;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_quad_fused<MODE, RED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_quad_fused<MODE, RED>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const dim3 grid(4 * a.W / kTileF, a.L / kTileRows);
  k_quad_fused<MODE, RED><<<grid, kThreads, kSmemBytes, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool quad_fused_supported(int L) { return L >= 32 && (L % 32) == 0; }

cudaError_t launch_quad_fused(int sincos_mode, int reduce_mode, const QuadFusedArgs& a,
                              cudaStream_t stream) {
  if (!quad_fused_supported(a.L) || a.W * 2 != a.L || a.src == a.dst) return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_one<0, 1>(a, stream) : launch_one<0, 0>(a, stream);
    case 1: return comp ? launch_one<1, 1>(a, stream) : launch_one<1, 0>(a, stream);
    default: return comp ? launch_one<2, 1>(a, stream) : launch_one<2, 0>(a, stream);
  }
}

}  // namespace xyk
