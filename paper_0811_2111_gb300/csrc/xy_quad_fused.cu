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
// single-lattice arithmetic (xyd::metropolis_step with the site's Metropolis
// words under lattice id lattice_id0 + r, and K_r = beta_r J), so replica r is
// bit for bit the single lattice with lattice id lattice_id0 + r.
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

// Per-thread sums of the two replicas a lane holds: exact fixed point
// (RED == 0, see xyd::FxSums) or Neumaier-compensated FP32 pairs (RED == 1).
template <int RED>
struct QuadSums {
  xyd::FxSums fx[2];
  float acc[2][5], cmp[2][5];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (RED == 0) {
        xyd::fx_init(fx[e]);
      } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) acc[e][i] = cmp[e][i] = 0.f;
      }
    }
  }
  __device__ __forceinline__ void add(const float v0[5], const float v1[5]) {
    if (RED == 0) {
      xyd::fx_add(fx[0], v0);
      xyd::fx_add(fx[1], v1);
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        xyd::neumaier_add(acc[0][i], cmp[0][i], v0[i]);
        xyd::neumaier_add(acc[1][i], cmp[1][i], v1[i]);
      }
    }
  }
};

// One tile's per-replica sums into the sweep's kR records: the 16 lanes of
// one parity (they hold the same two replicas, j0 and j0 + 1) -> warps ->
// one atomic per (replica, sum).  Exact integers for RED == 0 (a lane holds
// at most 4 terms per replica, so the 16-lane sums fit 32 bits), FP64 of the
// compensated pairs for RED == 1.  Must be reached by every thread.
template <int RED>
__device__ __forceinline__ void quad_commit(QuadSums<RED>& sums, unsigned int n_acc[2],
                                            float (*part)[kR][5][2], unsigned int (*cnt)[kR],
                                            xy_record* rec, const double* beta,
                                            bool first_block, int j0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bool bad[2] = {false, false};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    n_acc[e] = parity_sum(n_acc[e]);
    if (RED == 0) {
      // lanes of one parity hold the same replicas: or of their flags
      const unsigned int b = __ballot_sync(0xffffffffu, xyd::fx_nonfinite(sums.fx[e]));
      bad[e] = (b & ((lane & 1) ? 0xaaaaaaaau : 0x55555555u)) != 0u;
#pragma unroll
      for (int i = 0; i < 5; ++i)
        sums.fx[e].s[i] = parity_sum((unsigned int)xyd::fx_value(sums.fx[e], i));
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        sums.acc[e][i] = parity_sum(sums.acc[e][i]);
        sums.cmp[e][i] = parity_sum(sums.cmp[e][i]);
      }
    }
  }
  if (lane < 2) {                                          // lane 0: replicas 0, 1; lane 1: 2, 3
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      cnt[warp][j0 + e] = n_acc[e] | (bad[e] ? 0x80000000u : 0u);
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        if (RED == 0) {
          part[warp][j0 + e][i][0] = __uint_as_float(sums.fx[e].s[i]);
        } else {
          part[warp][j0 + e][i][0] = sums.acc[e][i];
          part[warp][j0 + e][i][1] = sums.cmp[e][i];
        }
      }
    }
  }
  __syncthreads();
  if (warp != 0) return;
  if (lane < kR) {
    unsigned long long total = 0;
    bool any_bad = false;
    for (int w = 0; w < kWarps; ++w) {
      total += cnt[w][lane] & 0x7fffffffu;
      any_bad |= (cnt[w][lane] & 0x80000000u) != 0u;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&rec[lane].accepted), total);
    if (any_bad) atomicOr(reinterpret_cast<unsigned long long*>(&rec[lane].flags), 1ull);
    if (first_block) rec[lane].beta = beta[lane];
  }
  if (lane >= kR * 5) return;
  // lanes 0..19 each own one (replica, sum)
  const int jr = lane / 5, si = lane - 5 * jr;
  if (RED == 0) {
    long long t = 0;
    for (int w = 0; w < kWarps; ++w) t += (int32_t)__float_as_uint(part[w][jr][si][0]);
    atomicAdd(reinterpret_cast<unsigned long long*>(&rec[jr].sum[si]),
              (unsigned long long)t << (XY_FX_SHIFT - xyd::fx_term_shift(si)));
    return;
  }
  float hi = 0.f, lo = 0.f;
  for (int w = 0; w < kWarps; ++w) {
    xyd::neumaier_add(hi, lo, part[w][jr][si][0]);
    lo += part[w][jr][si][1];
  }
  const double scaled = ((double)hi + (double)lo) * (double)(1ll << XY_FX_SHIFT);
  if (!(fabs(scaled) < 9.0e18)) {
    atomicOr(reinterpret_cast<unsigned long long*>(&rec[jr].flags), 1ull);
    return;
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(&rec[jr].sum[si]),
            (unsigned long long)__double2ll_rn(scaled));
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

// Stage both planes of the tile (bx, by) as (angle, cos, sin): the black
// plane's 36 rows (stage rows 0..35), then the red plane's 34 (stage rows
// 1..34), 16 float4 (one site, four replicas) per row, plus the halo site on
// each side of stage rows 1..34 of both planes (136 float4).  Thread t takes
// the float4 column group t & 15 of staged rows (t >> 4) + 16 i, i = 0..3
// (rows 0..63), then threads 0..95 one float4 of rows 64..69 and threads
// 96..231 one halo site: at most 5 float4 (20 unit vectors) per thread
// against a mean of 19.6.  Every load is issued before the first unit vector.
// Angles are kept only where the tile reads them: the red rows (with their
// halo sites) and the black tile rows 2..33.
template <int MODE, bool COHERENT>
__device__ __forceinline__ void quad_stage(const float* src, ThArr* th, CsArr* cs, int y0, int f0,
                                           int ks0, int L, int W, int F, size_t plane) {
  const int t = threadIdx.x, g = t & 15;
  auto ld = [&](size_t at) {
    return COHERENT ? __ldcg(reinterpret_cast<const float4*>(src + at))
                    : __ldg(reinterpret_cast<const float4*>(src + at));
  };
  float4 v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = (t >> 4) + 16 * i;
    const int p = rr < kSRows ? 1 : 0;
    const int r = rr < kSRows ? rr : rr - kSRows + 1;
    v[i] = ld(p * plane + (size_t)wrap_once(y0 - 2 + r, L) * F + f0 + 4 * g);
  }
  const bool has_tail = t < 96;                            // rows 64..69: red stage rows 29..34
  const int tail_r = 29 + (t >> 4);
  float4 vt = make_float4(0.f, 0.f, 0.f, 0.f);
  if (has_tail) vt = ld((size_t)wrap_once(y0 - 2 + tail_r, L) * F + f0 + 4 * g);
  const bool has_halo = t >= 96 && t < 96 + 4 * (kSRows - 2);
  const int h = t - 96;                                    // plane h / 68, stage row 1 + (h % 68) / 2
  const int hp = h >= 2 * (kSRows - 2) ? 1 : 0;
  const int hrem = h - hp * 2 * (kSRows - 2);
  const int hr = 1 + (hrem >> 1), hside = hrem & 1;
  float4 vh = make_float4(0.f, 0.f, 0.f, 0.f);
  if (has_halo) {
    const int ks = hside ? wrap_once(ks0 + kTileF / 4, W) : wrap_once(ks0 - 1, W);
    vh = ld(hp * plane + (size_t)wrap_once(y0 - 2 + hr, L) * F + 4 * (size_t)ks);
  }
  auto put = [&](int p, int r, int col, float4 a, bool keep_angles) {
    float s0, c0, s1, c1, s2, c2, s3, c3;
    xyd::unit_vector<MODE>(a.x, &s0, &c0);
    xyd::unit_vector<MODE>(a.y, &s1, &c1);
    xyd::unit_vector<MODE>(a.z, &s2, &c2);
    xyd::unit_vector<MODE>(a.w, &s3, &c3);
    if (keep_angles) *reinterpret_cast<float4*>(&th[p][r][col]) = a;
    *reinterpret_cast<float4*>(&cs[p][r][col]) = make_float4(c0, s0, c1, s1);
    *reinterpret_cast<float4*>(&cs[p][r][col + 2]) = make_float4(c2, s2, c3, s3);
  };
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = (t >> 4) + 16 * i;
    const int p = rr < kSRows ? 1 : 0;
    const int r = rr < kSRows ? rr : rr - kSRows + 1;
    put(p, r, 4 + 4 * g, v[i], p == 0 || (r >= 2 && r < kSRows - 2));
  }
  if (has_tail) put(0, tail_r, 4 + 4 * g, vt, true);
  if (has_halo) put(hp, hr, hside ? kTileF + 4 : 0, vh, hp == 0);
}

// pair_nb with the other colour's rows r - 1 and r of the pair's columns in
// registers (D, P: the previous row's P and U, as a warp walks its rows
// downwards): loads the same-row edge element and row r + 1 (returned in U).
__device__ __forceinline__ void pair_nb_rolled(const CsArr& nb, int r, int c0, int q,
                                               const float4 D, const float4 P, float4& U,
                                               PairNb& n) {
  const float4 E = *reinterpret_cast<const float4*>(&nb[r][q ? c0 + 4 : c0 - 4]);
  U = *reinterpret_cast<const float4*>(&nb[r + 1][c0]);
  const float4 Lf = q ? P : E, Rt = q ? E : P;
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

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// A work item of the persistent kernel: its sweep's buffers, Philox sweep word
// and records, and the launch's constants (left in parameter space).
struct QuadItem {
  const QuadFusedArgs& base;
  const float* src;
  float* dst;
  uint32_t sweep;
  xy_record* rec;
};

// The constants of a sweep (L, W, K, delta, rk, lattice_id0, beta).
__device__ __forceinline__ const QuadFusedArgs& constants(const QuadFusedArgs& a) { return a; }
__device__ __forceinline__ const QuadFusedArgs& constants(const QuadItem& a) { return a.base; }

// One sweep of the tile (bx, by) of the sweep `a` describes (a QuadFusedArgs:
// the per-sweep kernel passes its parameter, so every field is read from
// parameter space where it is used; the persistent kernel a per-item copy).
// COHERENT: `src` was written earlier in the same launch by other CTAs
// (persistent kernel), so it is read through L2 (ld.global.cg).  `mid` runs in
// every thread before the barrier between the red and the black half, `end`
// after the tile's last store to dst and before the sums' barrier.
template <int MODE, int RED, bool COHERENT, class Args, class MidHook = NoHook,
          class EndHook = NoHook>
__device__ __forceinline__ void quad_sweep_body(const Args& item, int bx, int by,
                                                const MidHook& mid = MidHook(),
                                                const EndHook& end = EndHook()) {
  const QuadFusedArgs& a = constants(item);
  extern __shared__ __align__(16) unsigned char smem[];
  ThArr* th = reinterpret_cast<ThArr*>(smem);
  CsArr* cs = reinterpret_cast<CsArr*>(smem + kThBytes);
  float(*part)[kR][5][2] = reinterpret_cast<float(*)[kR][5][2]>(smem + kThBytes + kCsBytes);
  unsigned int(*cnt)[kR] =
      reinterpret_cast<unsigned int(*)[kR]>(smem + kThBytes + kCsBytes + kPartBytes);

  const int L = a.L, W = a.W;
  const int F = 4 * W;                                     // elements per plane row
  const int f0 = bx * kTileF;                      // first element of the tile
  const int ks0 = f0 >> 2;                                 // its first site column
  const int y0 = by * kTileRows;
  const size_t plane = (size_t)L * (size_t)F;

  // ---- stage both planes (angle + unit vector) ----
  quad_stage<MODE, COHERENT>(item.src, th, cs, y0, f0, ks0, L, W, F, plane);
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
  float4 nbD = *reinterpret_cast<const float4*>(&cs[1][warp * 4 + 1][c0]);
  float4 nbP = *reinterpret_cast<const float4*>(&cs[1][warp * 4 + 2][c0]);
#pragma unroll 2
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = y & 1;                                   // red: x = 2k + (y & 1)
    PairNb n;
    float4 nbU;
    pair_nb_rolled(cs[1], r, c0, q, nbD, nbP, nbU, n);
    nbD = nbP;
    nbP = nbU;
    const uint32_t x = 2u * kq + (uint32_t)q;
    const uint32_t ctr = xyd::metropolis_counter((uint32_t)y * uL + x, x);
    // lanes l and l ^ 2 hold replicas j0, j0 + 1 of the pair's two sites
    // (x & 2 == lane & 2): each draws one replica's block, keeps its own
    // half and passes the other half across
    const bool up = (x & 2u) != 0u;
    const uint4 wb = xyd::philox4x32_10(make_uint4(ctr, item.sweep, up ? id1 : id0, 1u), a.rk);
    const uint32_t g0 = __shfl_xor_sync(0xffffffffu, up ? wb.x : wb.z, 2);
    const uint32_t g1 = __shfl_xor_sync(0xffffffffu, up ? wb.y : wb.w, 2);
    const uint2 w0 = up ? make_uint2(g0, g1) : make_uint2(wb.x, wb.y);
    const uint2 w1 = up ? make_uint2(wb.z, wb.w) : make_uint2(g0, g1);
    const float2 t = *reinterpret_cast<const float2*>(&th[0][r][c0]);
    const float4 o = *reinterpret_cast<const float4*>(&cs[0][r][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w0.x, w0.y, K0, a.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w1.x, w1.y, K1, a.delta);
    n_acc[0] += r0.accept ? 1u : 0u;
    n_acc[1] += r1.accept ? 1u : 0u;
    *reinterpret_cast<float4*>(&cs[0][r][c0]) = make_float4(r0.c, r0.s, r1.c, r1.s);
    *reinterpret_cast<float2*>(item.dst + (size_t)y * F + fp) = make_float2(r0.th, r1.th);
  }
  // ---- red half: the ring at distance one (recomputed, not counted) ----
  // rows -1 and 32 (64 elements each): one lane per pair of sites (sites 2j
  // and 2j + 1 of the tile row share a Philox block, as in the tile) and
  // replica, warps 0 and 1; the halo site of rows 0..31 on the side the black
  // tile reaches (left on odd rows, right on even; 128 elements), one per lane
  // of warps 2..5.  Warps 6 and 7 wait at the barrier.
  if (threadIdx.x < 64) {
    const int ty = threadIdx.x < 32 ? -1 : kTileRows;
    const int j = threadIdx.x & 31;
    const int rep = j & 3;                                 // replica
    const int sc = 4 + 8 * (j >> 2) + rep;                 // element of site 2 (j >> 2)
    const int r = ty + 2;
    const int y = wrap_once(y0 + ty, L);
    const int q = y & 1;
    const uint32_t x = 2u * (uint32_t)(ks0 + 2 * (j >> 2)) + (uint32_t)q;   // x & 2 == 0
    const uint4 w = xyd::philox4x32_10(
        make_uint4((uint32_t)y * uL + x, item.sweep, a.lattice_id0 + (uint32_t)rep, 1u), a.rk);
    const float K = replica_k(a, rep);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = sc + 4 * e;
      const float2 l = cs[1][r][c + 4 * q - 4], rt = cs[1][r][c + 4 * q];
      const float2 d = cs[1][r - 1][c], u = cs[1][r + 1][c];
      const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
      const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
      const float2 own = cs[0][r][c];
      const xyd::SiteResult res = xyd::metropolis_step<MODE>(
          th[0][r][c], own.x, own.y, Sc, Ss, e ? w.z : w.x, e ? w.w : w.y, K, a.delta);
      cs[0][r][c] = make_float2(res.c, res.s);
    }
  } else if (threadIdx.x < 64 + kTileRows * kR) {
    const int e = threadIdx.x - 64;
    const int ty = e >> 2;
    const int sc = (((y0 + ty) & 1) ? 0 : kTileF + 4) + (e & 3);
    const int r = ty + 2;
    const int y = y0 + ty;
    const int q = y & 1;
    const int ks = wrap_once(ks0 + ((sc - 4) >> 2), W);   // floor: stage columns 0..3 -> ks0 - 1
    const int j = sc & 3;
    const uint32_t x = 2u * (uint32_t)ks + (uint32_t)q;
    const uint32_t site = (uint32_t)y * uL + x;
    const float2 l = cs[1][r][sc + 4 * q - 4], rt = cs[1][r][sc + 4 * q];
    const float2 d = cs[1][r - 1][sc], u = cs[1][r + 1][sc];
    const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
    const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
    const uint4 w = xyd::philox4x32_10(
        make_uint4(xyd::metropolis_counter(site, x), item.sweep, a.lattice_id0 + (uint32_t)j, 1u), a.rk);
    const uint2 uw = xyd::metropolis_words(w, x);
    const float2 own = cs[0][r][sc];
    const xyd::SiteResult res = xyd::metropolis_step<MODE>(th[0][r][sc], own.x, own.y, Sc, Ss,
                                                           uw.x, uw.y, replica_k(a, j), a.delta);
    cs[0][r][sc] = make_float2(res.c, res.s);
  }
  mid();
  __syncthreads();

  // ---- black half of the tile, with the sweep sums ----
  QuadSums<RED> sums;
  sums.init();
  float* dst_blk = item.dst + plane;
  nbD = *reinterpret_cast<const float4*>(&cs[0][warp * 4 + 1][c0]);
  nbP = *reinterpret_cast<const float4*>(&cs[0][warp * 4 + 2][c0]);
#pragma unroll 2
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = (y + 1) & 1;                             // black: x = 2k + ((y + 1) & 1)
    PairNb n;
    float4 nbU;
    pair_nb_rolled(cs[0], r, c0, q, nbD, nbP, nbU, n);
    const float4 m = nbP;                                  // the red pair of the same row
    nbD = nbP;
    nbP = nbU;
    const uint32_t x = 2u * kq + (uint32_t)q;
    const uint32_t ctr = xyd::metropolis_counter((uint32_t)y * uL + x, x);
    // lanes l and l ^ 2 hold replicas j0, j0 + 1 of the pair's two sites
    // (x & 2 == lane & 2): each draws one replica's block, keeps its own
    // half and passes the other half across
    const bool up = (x & 2u) != 0u;
    const uint4 wb = xyd::philox4x32_10(make_uint4(ctr, item.sweep, up ? id1 : id0, 1u), a.rk);
    const uint32_t g0 = __shfl_xor_sync(0xffffffffu, up ? wb.x : wb.z, 2);
    const uint32_t g1 = __shfl_xor_sync(0xffffffffu, up ? wb.y : wb.w, 2);
    const uint2 w0 = up ? make_uint2(g0, g1) : make_uint2(wb.x, wb.y);
    const uint2 w1 = up ? make_uint2(wb.z, wb.w) : make_uint2(g0, g1);
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
    float v0[5], v1[5];
    xyd::measure_terms(r0.c, r0.s, n.l[0].x, n.l[0].y, n.r[0].x, n.r[0].y, n.d[0].x, n.d[0].y,
                       n.u[0].x, n.u[0].y, n.Sc[0], n.Ss[0], m.x, m.y, v0);
    xyd::measure_terms(r1.c, r1.s, n.l[1].x, n.l[1].y, n.r[1].x, n.r[1].y, n.d[1].x, n.d[1].y,
                       n.u[1].x, n.u[1].y, n.Sc[1], n.Ss[1], m.z, m.w, v1);
    sums.add(v0, v1);
  }

  end();
  // ---- per-replica sums -> records ----
  quad_commit<RED>(sums, n_acc, part, cnt, item.rec, a.beta, bx == 0 && by == 0, j0);
}

// The per-sweep kernel keeps its own copy of the tile arithmetic of
// quad_sweep_body (identical statements; the two are tested bit for bit
// against each other): compiled through the shared template body it issued
// 2.5 % more instructions (363.7 M against 354.6 M warp instructions per
// L = 4096 launch) and took 4 % longer.
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
  quad_stage<MODE, false>(a.src, th, cs, y0, f0, ks0, L, W, F, plane);
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
  float4 nbD = *reinterpret_cast<const float4*>(&cs[1][warp * 4 + 1][c0]);
  float4 nbP = *reinterpret_cast<const float4*>(&cs[1][warp * 4 + 2][c0]);
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = y & 1;                                   // red: x = 2k + (y & 1)
    PairNb n;
    float4 nbU;
    pair_nb_rolled(cs[1], r, c0, q, nbD, nbP, nbU, n);
    nbD = nbP;
    nbP = nbU;
    const uint32_t x = 2u * kq + (uint32_t)q;
    const uint32_t ctr = xyd::metropolis_counter((uint32_t)y * uL + x, x);
    // lanes l and l ^ 2 hold replicas j0, j0 + 1 of the pair's two sites
    // (x & 2 == lane & 2): each draws one replica's block, keeps its own
    // half and passes the other half across
    const bool up = (x & 2u) != 0u;
    const uint4 wb = xyd::philox4x32_10(make_uint4(ctr, a.sweep, up ? id1 : id0, 1u), a.rk);
    const uint32_t g0 = __shfl_xor_sync(0xffffffffu, up ? wb.x : wb.z, 2);
    const uint32_t g1 = __shfl_xor_sync(0xffffffffu, up ? wb.y : wb.w, 2);
    const uint2 w0 = up ? make_uint2(g0, g1) : make_uint2(wb.x, wb.y);
    const uint2 w1 = up ? make_uint2(wb.z, wb.w) : make_uint2(g0, g1);
    const float2 t = *reinterpret_cast<const float2*>(&th[0][r][c0]);
    const float4 o = *reinterpret_cast<const float4*>(&cs[0][r][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w0.x, w0.y, K0, a.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w1.x, w1.y, K1, a.delta);
    n_acc[0] += r0.accept ? 1u : 0u;
    n_acc[1] += r1.accept ? 1u : 0u;
    *reinterpret_cast<float4*>(&cs[0][r][c0]) = make_float4(r0.c, r0.s, r1.c, r1.s);
    *reinterpret_cast<float2*>(a.dst + (size_t)y * F + fp) = make_float2(r0.th, r1.th);
  }
  // ---- red half: the ring at distance one (recomputed, not counted) ----
  // rows -1 and 32 (64 elements each): one lane per pair of sites (sites 2j
  // and 2j + 1 of the tile row share a Philox block, as in the tile) and
  // replica, warps 0 and 1; the halo site of rows 0..31 on the side the black
  // tile reaches (left on odd rows, right on even; 128 elements), one per lane
  // of warps 2..5.  Warps 6 and 7 wait at the barrier.
  if (threadIdx.x < 64) {
    const int ty = threadIdx.x < 32 ? -1 : kTileRows;
    const int j = threadIdx.x & 31;
    const int rep = j & 3;                                 // replica
    const int sc = 4 + 8 * (j >> 2) + rep;                 // element of site 2 (j >> 2)
    const int r = ty + 2;
    const int y = wrap_once(y0 + ty, L);
    const int q = y & 1;
    const uint32_t x = 2u * (uint32_t)(ks0 + 2 * (j >> 2)) + (uint32_t)q;   // x & 2 == 0
    const uint4 w = xyd::philox4x32_10(
        make_uint4((uint32_t)y * uL + x, a.sweep, a.lattice_id0 + (uint32_t)rep, 1u), a.rk);
    const float K = replica_k(a, rep);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = sc + 4 * e;
      const float2 l = cs[1][r][c + 4 * q - 4], rt = cs[1][r][c + 4 * q];
      const float2 d = cs[1][r - 1][c], u = cs[1][r + 1][c];
      const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
      const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
      const float2 own = cs[0][r][c];
      const xyd::SiteResult res = xyd::metropolis_step<MODE>(
          th[0][r][c], own.x, own.y, Sc, Ss, e ? w.z : w.x, e ? w.w : w.y, K, a.delta);
      cs[0][r][c] = make_float2(res.c, res.s);
    }
  } else if (threadIdx.x < 64 + kTileRows * kR) {
    const int e = threadIdx.x - 64;
    const int ty = e >> 2;
    const int sc = (((y0 + ty) & 1) ? 0 : kTileF + 4) + (e & 3);
    const int r = ty + 2;
    const int y = y0 + ty;
    const int q = y & 1;
    const int ks = wrap_once(ks0 + ((sc - 4) >> 2), W);   // floor: stage columns 0..3 -> ks0 - 1
    const int j = sc & 3;
    const uint32_t x = 2u * (uint32_t)ks + (uint32_t)q;
    const uint32_t site = (uint32_t)y * uL + x;
    const float2 l = cs[1][r][sc + 4 * q - 4], rt = cs[1][r][sc + 4 * q];
    const float2 d = cs[1][r - 1][sc], u = cs[1][r + 1][sc];
    const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
    const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
    const uint4 w = xyd::philox4x32_10(
        make_uint4(xyd::metropolis_counter(site, x), a.sweep, a.lattice_id0 + (uint32_t)j, 1u), a.rk);
    const uint2 uw = xyd::metropolis_words(w, x);
    const float2 own = cs[0][r][sc];
    const xyd::SiteResult res = xyd::metropolis_step<MODE>(th[0][r][sc], own.x, own.y, Sc, Ss,
                                                           uw.x, uw.y, replica_k(a, j), a.delta);
    cs[0][r][sc] = make_float2(res.c, res.s);
  }
  __syncthreads();

  // ---- black half of the tile, with the sweep sums ----
  QuadSums<RED> sums;
  sums.init();
  float* dst_blk = a.dst + plane;
  nbD = *reinterpret_cast<const float4*>(&cs[0][warp * 4 + 1][c0]);
  nbP = *reinterpret_cast<const float4*>(&cs[0][warp * 4 + 2][c0]);
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = (y + 1) & 1;                             // black: x = 2k + ((y + 1) & 1)
    PairNb n;
    float4 nbU;
    pair_nb_rolled(cs[0], r, c0, q, nbD, nbP, nbU, n);
    const float4 m = nbP;                                  // the red pair of the same row
    nbD = nbP;
    nbP = nbU;
    const uint32_t x = 2u * kq + (uint32_t)q;
    const uint32_t ctr = xyd::metropolis_counter((uint32_t)y * uL + x, x);
    // lanes l and l ^ 2 hold replicas j0, j0 + 1 of the pair's two sites
    // (x & 2 == lane & 2): each draws one replica's block, keeps its own
    // half and passes the other half across
    const bool up = (x & 2u) != 0u;
    const uint4 wb = xyd::philox4x32_10(make_uint4(ctr, a.sweep, up ? id1 : id0, 1u), a.rk);
    const uint32_t g0 = __shfl_xor_sync(0xffffffffu, up ? wb.x : wb.z, 2);
    const uint32_t g1 = __shfl_xor_sync(0xffffffffu, up ? wb.y : wb.w, 2);
    const uint2 w0 = up ? make_uint2(g0, g1) : make_uint2(wb.x, wb.y);
    const uint2 w1 = up ? make_uint2(wb.z, wb.w) : make_uint2(g0, g1);
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
    float v0[5], v1[5];
    xyd::measure_terms(r0.c, r0.s, n.l[0].x, n.l[0].y, n.r[0].x, n.r[0].y, n.d[0].x, n.d[0].y,
                       n.u[0].x, n.u[0].y, n.Sc[0], n.Ss[0], m.x, m.y, v0);
    xyd::measure_terms(r1.c, r1.s, n.l[1].x, n.l[1].y, n.r[1].x, n.r[1].y, n.d[1].x, n.d[1].y,
                       n.u[1].x, n.u[1].y, n.Sc[1], n.Ss[1], m.z, m.w, v1);
    sums.add(v0, v1);
  }

  // ---- per-replica sums -> records ----
  quad_commit<RED>(sums, n_acc, part, cnt, a.rec, a.beta,
                   blockIdx.x == 0 && blockIdx.y == 0, j0);
}

// Polls of a tile counter before a wait gives up (with a short sleep between
// polls: about a second in all).
constexpr long long kQuadSpinLimit = 1ll << 22;

__device__ __forceinline__ unsigned int q_load_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void q_store_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All sweeps of a call in one cooperative launch (every CTA resident), the
// scheme of the single-lattice persistent sweep: work items (sweep s, tile)
// handed out in increasing order by one atomic counter, sweep-major, tile rows
// folded (0, T-1, 1, T-2, ...); a tile's sweep s starts once its eight
// neighbours and itself have published counters >= s (its halo of two rows and
// one site reaches into all eight, and it overwrites the buffer they read
// during sweep s - 1); it is published (s + 1) by warp 7 with a GPU-scope
// release store after the closing barrier.  Warp 0 looks at the next item's nine
// counters once, after the black half, and when all are set the next tile
// neither waits nor takes the barrier in front of it.  Every wait is bounded;
// one that runs out sets *error and ends the CTA, and waiting CTAs that see
// *error end too.  The tile arithmetic is quad_sweep_body's, so the result is
// bit for bit that of one k_quad_fused launch per sweep.
template <int MODE, int RED>
__global__ void __launch_bounds__(kThreads, 3) k_quad_fused_persist(QuadPersistArgs p) {
  __shared__ int s_abort;
  __shared__ int s_item[2];
  __shared__ int s_ready[2];
  const int tiles_x = 4 * p.a.W / kTileF, tiles_y = p.a.L / kTileRows;
  const int ntiles = tiles_x * tiles_y;
  const int total = p.n_sweeps * ntiles;          // < 2^31 - 2^20 (the host splits longer runs)
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_item[0] = (int)atomicAdd(p.counter, 1u);
    s_ready[0] = 0;
  }
  __syncthreads();
  int par = 0;
  int item = s_item[0];
  while (item < total) {
    const int s = item / ntiles;
    const int k = item - s * ntiles;
    const int prow = k / tiles_x;
    const int bx = k - prow * tiles_x;
    const int by = (prow & 1) ? tiles_y - 1 - (prow >> 1) : (prow >> 1);
    const bool ready = s_ready[par] != 0;
    if (s > 0 && threadIdx.x < 9 && !ready) {
      const int d = threadIdx.x;
      const int nx = wrap_once(bx + d % 3 - 1, tiles_x);
      const int ny = wrap_once(by + d / 3 - 1, tiles_y);
      const unsigned int* f = p.flags + (ny * tiles_x + nx);
      long long it = 0;
      while (q_load_acquire(f) < (unsigned int)s) {
        if (++it > p.spin_limit ||
            ((it & 255) == 0 && *reinterpret_cast<volatile unsigned int*>(p.error) != 0u)) {
          atomicOr(p.error, 1u);
          s_abort = 1;
          break;
        }
        __nanosleep(128);
      }
    }
    if (!ready) {
      __syncthreads();
      if (s_abort) return;            // read by every thread between the same two barriers
    }
    int next = 0;
    if (threadIdx.x == 0) next = (int)atomicAdd(p.counter, 1u);
    int* slot = &s_item[par ^ 1];
    const QuadItem c{p.a, p.buf[s & 1], p.buf[(s + 1) & 1], p.sweep0 + (uint32_t)s,
                     p.rec + (size_t)s * kR};
    quad_sweep_body<MODE, RED, true>(
        c, bx, by,
        [&]() {
          if (threadIdx.x == 0) *slot = next;
        },
        [&]() {
          if (threadIdx.x >= kThreads - 32) {
            const int l = threadIdx.x - (kThreads - 32);
            bool ok = l >= 9;
            const int ni = *slot;
            if (l < 9 && ni < total) {
              const int ns = ni / ntiles;
              const int nk = ni - ns * ntiles;
              const int nrow = nk / tiles_x;
              const int nbx = nk - nrow * tiles_x;
              const int nby = (nrow & 1) ? tiles_y - 1 - (nrow >> 1) : (nrow >> 1);
              const int d = l;
              const int nx = wrap_once(nbx + d % 3 - 1, tiles_x);
              const int ny = wrap_once(nby + d / 3 - 1, tiles_y);
              ok = ns == 0 || q_load_acquire(p.flags + (ny * tiles_x + nx)) >= (unsigned int)ns;
            }
            const unsigned int all = __ballot_sync(0xffffffffu, ok);
            if (l == 0) s_ready[par ^ 1] = (all == 0xffffffffu) ? 1 : 0;
          }
        });
    if (threadIdx.x == kThreads - 64) {
      // a warp other than the early look's publishes the tile: the closing
      // barrier orders every thread's stores to dst before this
      // GPU-scope release, which is cumulative over the writes that happen
      // before it
      q_store_release(p.flags + (by * tiles_x + bx), (unsigned int)(s + 1));
    }
    par ^= 1;
    item = s_item[par];
  }
}

template <int MODE, int RED>
cudaError_t launch_persist_one(const QuadPersistArgs& p, cudaStream_t stream) {
  auto fn = k_quad_fused_persist<MODE, RED>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, kSmemBytes);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int tiles = quad_persistent_tiles(p.a.L);
  const int grid = tiles < per_sm * sms ? tiles : per_sm * sms;
  // the tile counters and, after them, the work counter
  e = cudaMemsetAsync(p.flags, 0, sizeof(unsigned int) * ((size_t)tiles + 1), stream);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<QuadPersistArgs*>(&p)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(fn), dim3(grid), dim3(kThreads),
                                     args, kSmemBytes, stream);
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

namespace xyk {

int quad_persistent_tiles(int L) { return quad_fused_supported(L) ? (L / 32) * (L / kTileRows) : 0; }

int quad_persistent_max_sweeps(int L) {
  const int t = quad_persistent_tiles(L);
  return t > 0 ? (int)((0x7fffffffu - (1u << 20)) / (unsigned)t) : 0;
}

long long quad_persistent_spin_limit() { return kQuadSpinLimit; }

cudaError_t launch_quad_persistent(int sincos_mode, int reduce_mode, const QuadPersistArgs& p,
                                   cudaStream_t stream) {
  const int tiles = quad_persistent_tiles(p.a.L);
  if (tiles == 0 || p.a.W * 2 != p.a.L || p.n_sweeps < 1 ||
      p.n_sweeps > quad_persistent_max_sweeps(p.a.L) || p.buf[0] == p.buf[1] || !p.flags ||
      p.counter != p.flags + tiles || !p.error || p.spin_limit < 1)
    return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_persist_one<0, 1>(p, stream) : launch_persist_one<0, 0>(p, stream);
    case 1: return comp ? launch_persist_one<1, 1>(p, stream) : launch_persist_one<1, 0>(p, stream);
    default: return comp ? launch_persist_one<2, 1>(p, stream) : launch_persist_one<2, 0>(p, stream);
  }
}

}  // namespace xyk
