// xy_fused.cu -- one-launch checkerboard sweep (red half, black half and the
// fused measure) reading the lattice from `src` and writing it to `dst`.
//
// Each CTA owns a tile of 32 rows x 64 plane columns (128 natural columns) of
// both colours.  It stages both planes of the tile plus a halo of two rows and
// one plane column into shared memory as (angle, cos, sin), then
//   1. updates the red sites of the tile and of the ring at distance one
//      around it (the ring sites belong to neighbouring tiles; they are
//      recomputed here from the same old state and the same counter-based
//      Philox words, so every copy makes the identical decision),
//   2. updates the black sites of the tile against the new red values,
//   3. accumulates the sweep sums over the tile's bonds and spins,
// and writes the tile's new angles to `dst`.  Reading the old state from a
// separate buffer is what lets one CTA use its neighbours' old angles while
// those neighbours write their new ones (the ping-pong of the paper's GL
// implementation, Sec. 3.1, applied to whole sweeps).
//
// Compared with the two-pass kernels each angle is read once and written once
// per sweep (8 B per update instead of 12 B) and each site's unit vector is
// computed once per sweep instead of once per half-sweep.
//
// Requires W = L/2 to be a multiple of 64 and L a multiple of 32 (L % 128 == 0).
// Decisions are bit-identical to the two-pass kernels: both call the same
// xyd::unit_vector / xyd::nb_sum / xyd::metropolis_step with pinned rounding.
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_device.cuh"
#include "xy_internal.h"
#include "xy_tma.cuh"

namespace xyk {

namespace {

constexpr int kTileRows = 32;
constexpr int kTileK = 64;                   // plane columns (2 per lane)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSRows = kTileRows + 4;        // stage rows: global rows y0-2 .. y0+33
constexpr int kRedRows = kSRows - 2;         // the red plane's stage rows 1 .. 34

// Shared memory of a tile, 55.3 KB (four CTAs fit an SM).  Stage row r is
// global row y0 - 2 + r.  Only what the tile reads is kept:
//   ang   raw angles of the 70 staged rows, 64 plane columns each: black
//         stage rows 0..35 as rows 0..35, red stage rows 1..34 as rows
//         36..69 (the layout TMA writes; 128-byte aligned)
//   angs  red angles of the halo columns k0-1 and k0+64, stage rows 1..34
//   csr   red unit vectors (cos, sin) of stage rows 1..34, plane cols k0-2 ..
//         k0+65 (column k - k0 + kCsOff: lane l's pair at 2l + 2 is 16-byte
//         aligned; k0-1 .. k0+64 used)
//   csb   black unit vectors of stage rows 0..35, same columns
// then the commit's per-warp partial sums and counters.  The persistent
// kernel keeps NANG = 2 ang buffers: the next tile's rows arrive in the other.
constexpr int kCsOff = 2;
constexpr int kCsCols = kTileK + 4;
constexpr int kRawRows = kSRows + kRedRows;
constexpr int kRedRaw0 = kSRows - 1;        // ang row of red stage row r: kRedRaw0 + r
typedef float2 CsRow[kCsCols];
typedef float AngRow[kTileK];
constexpr size_t kRawRowBytes = sizeof(AngRow);
constexpr size_t kAngBytes = kRawRowBytes * kRawRows;
constexpr size_t kAngsBytes = sizeof(float) * 2 * kRedRows;
constexpr size_t kCsrBytes = sizeof(CsRow) * kRedRows;
constexpr size_t kCsbBytes = sizeof(CsRow) * kSRows;
constexpr size_t kPartBytes = sizeof(float) * kWarps * 5 * 2;
constexpr size_t kCntBytes = sizeof(unsigned int) * kWarps;
template <int NANG>
struct Layout {
  static constexpr size_t kAngsAt = NANG * kAngBytes;
  static constexpr size_t kCsrAt = kAngsAt + kAngsBytes;
  static constexpr size_t kCsbAt = kCsrAt + kCsrBytes;
  static constexpr size_t kPartAt = kCsbAt + kCsbBytes;
  static constexpr size_t kCntAt = kPartAt + kPartBytes;
  static constexpr size_t kBytes = kCntAt + kCntBytes;
  static_assert(kAngBytes % 128 == 0 && kCsrAt % 16 == 0 && kCsbAt % 16 == 0 && kPartAt % 16 == 0,
                "shared-memory regions must stay aligned (ang: 128 bytes for TMA)");
};
constexpr size_t kSmemBytes = Layout<1>::kBytes;
constexpr size_t kPersistSmemBytes = Layout<2>::kBytes;
static_assert(4 * (kSmemBytes + 1024 + 128) <= 228 * 1024,
              "four tiles (and their static shared memory) must fit one SM");
static_assert(3 * (kPersistSmemBytes + 1024 + 512) <= 228 * 1024,
              "three persistent tiles (and their static shared memory) must fit one SM");

// Tiles of one sweep of side L (L % 128 == 0).
inline int fused_tiles_of(int L) { return (L / 2 / kTileK) * (L / kTileRows); }

__device__ __forceinline__ int wrap_once(int v, int n) {
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}

// The four neighbour unit vectors of the two sites at columns c0, c0+1 (c0
// even) of row i of the other colour's unit vectors `nb`, where a site at
// column c has its same-row neighbours at c+q-1 and c+q.  The three same-row
// columns c0+q-1 .. c0+q+1 are the aligned pair (c0, c0+1) and one edge
// column, c0-1 (q = 0) or c0+2 (q = 1); q is a compile-time constant where the
// row loops are unrolled (rows alternate q), so no selects are issued.  Rows
// i-1 and i of the pair's columns come in as D and P (a warp walks its rows
// downwards, so they are the previous row's P and U); row i+1 is loaded and
// returned in U.
struct PairNeighbours {
  float Sc[2], Ss[2];
  float2 l[2], r[2], d[2], u[2];
};

__device__ __forceinline__ void pair_neighbours(const CsRow* nb, int i, int c0, int q,
                                                const float4 D, const float4 P, float4& U,
                                                PairNeighbours& n) {
  const float2 e = nb[i][q ? c0 + 2 : c0 - 1];
  const float2 p0 = make_float2(P.x, P.y), p1 = make_float2(P.z, P.w);
  U = *reinterpret_cast<const float4*>(&nb[i + 1][c0]);
  if (q) {
    n.l[0] = p0;
    n.r[0] = p1;
    n.l[1] = p1;
    n.r[1] = e;
  } else {
    n.l[0] = e;
    n.r[0] = p0;
    n.l[1] = p0;
    n.r[1] = p1;
  }
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

__device__ __forceinline__ float4 ld4(const float2* p) {
  return *reinterpret_cast<const float4*>(p);
}

__device__ __forceinline__ void st4(float2* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// The scalars of one fused sweep; the Philox round keys are passed separately
// (by reference, so a kernel can leave them in its parameter space).
struct FusedCore {
  const float* src;
  float* dst;
  int L;
  int W;
  float K;
  float delta;
  uint32_t lattice_id;
  uint32_t sweep;
  xy_record* rec;
  double beta;
};

// One red ring site at stage row r, unit-vector column c: the tile sites'
// arithmetic, with the site's own Philox block.
template <int MODE, class Args>
__device__ __forceinline__ void red_ring_site(float th, CsRow* csr, const CsRow* csb, int r,
                                              int c, int q, uint32_t site, uint32_t x,
                                              const Args& a, const xyd::RoundKeys& rk) {
  const float2 l = csb[r][c + q - 1], rt = csb[r][c + q];
  const float2 d = csb[r - 1][c], u = csb[r + 1][c];
  const float Sc = xyd::nb_sum(l.x, rt.x, d.x, u.x);
  const float Ss = xyd::nb_sum(l.y, rt.y, d.y, u.y);
  const uint4 w = xyd::philox4x32_10(
      make_uint4(xyd::metropolis_counter(site, x), a.sweep, a.lattice_id, 1u), rk);
  const uint2 uw = xyd::metropolis_words(w, x);
  const float2 own = csr[r - 1][c];
  const xyd::SiteResult res =
      xyd::metropolis_step<MODE>(th, own.x, own.y, Sc, Ss, uw.x, uw.y, a.K, a.delta);
  csr[r - 1][c] = make_float2(res.c, res.s);   // the black half reads the unit vector only
}

// One sweep of the tile (bx, by) of one lattice.  Args is FusedArgs (the
// single-lattice kernel passes its parameter, so every field is read from
// parameter space where it is used) or FusedCore (built per CTA by the batched
// and persistent kernels); both have the fields used here.  COHERENT: the
// source was written earlier in the same launch by other CTAs (persistent
// kernel), so it is read through L2 (ld.global.cg) rather than the
// non-coherent path.  TMA: the 70 staged rows of raw angles are not loaded
// here but arrive in the ang buffer by TMA, issued by the caller (the per-sweep
// kernel at its start, the persistent kernel during the previous tile);
// `raw_wait` waits for them.  Otherwise each thread loads its rows and stores
// them there itself.  NANG: ang buffers in the layout (the persistent kernel's
// two alternate, `ang_sel` picks this tile's).  `pre` runs in every thread
// before the barrier that ends the staging, `mid` before the barrier between
// the red and the black half, `post` right after that barrier, `end` after the
// tile's last store to dst and before the CTA's closing barrier.
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

__device__ __forceinline__ unsigned char* smem_base() {
  extern __shared__ __align__(128) unsigned char smem[];
  return smem;
}

template <int MODE, int RED, bool COHERENT = false, bool TMA = false, int NANG = 1, class Args,
          class PreHook = NoHook, class MidHook = NoHook, class EndHook = NoHook,
          class PostHook = NoHook, class RawWait = NoHook>
__device__ __forceinline__ void fused_sweep_body(const Args& a, const xyd::RoundKeys& rk, int bx,
                                                 int by, int ang_sel = 0,
                                                 const PreHook& pre = PreHook(),
                                                 const MidHook& mid = MidHook(),
                                                 const EndHook& end = EndHook(),
                                                 const PostHook& post = PostHook(),
                                                 const RawWait& raw_wait = RawWait()) {
  using Lay = Layout<NANG>;
  extern __shared__ __align__(128) unsigned char smem[];
  AngRow* ang = reinterpret_cast<AngRow*>(smem + (size_t)ang_sel * kAngBytes);
  float* angs = reinterpret_cast<float*>(smem + Lay::kAngsAt);     // [34][2]
  CsRow* csr = reinterpret_cast<CsRow*>(smem + Lay::kCsrAt);
  CsRow* csb = reinterpret_cast<CsRow*>(smem + Lay::kCsbAt);
  float(*part)[5][2] = reinterpret_cast<float(*)[5][2]>(smem + Lay::kPartAt);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(smem + Lay::kCntAt);

  const int L = a.L, W = a.W;
  const int k0 = bx * kTileK;
  const int y0 = by * kTileRows;
  const size_t plane = (size_t)L * (size_t)W;

  // ---- stage both planes (angle + unit vector) ----
  // Staged rows: the black plane's 36 (stage rows 0..35) then the red plane's
  // 34 (stage rows 1..34; red is never needed two rows out), 70 rows of 64
  // plane columns, plus the halo columns k0-1 and k0+64 of stage rows 1..34 of
  // both planes (136 sites): 4616 unit vectors over 256 threads.  Thread t
  // takes the float4 column group t & 15 of staged rows (t >> 4) + 16 i,
  // i = 0..3 (rows 0..63; half a warp per row, so the addressing is a shift
  // and an add), then threads 0..191 one float2 of rows 64..69 and threads
  // 184..255 one or two halo sites: at most 19 unit vectors per thread against
  // a mean of 18.03.  Every load is issued before the first unit vector.
  {
    const int t = (int)threadIdx.x;
    const int cg = t & 15;
    float4 v[4];
    if (!TMA) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = (t >> 4) + 16 * i;
        const int p = rr < kSRows ? 1 : 0;
        const int r = rr < kSRows ? rr : rr - kSRows + 1;
        const size_t row = p * plane + (size_t)wrap_once(y0 - 2 + r, L) * W + k0 + 4 * cg;
        v[i] = COHERENT ? __ldcg(reinterpret_cast<const float4*>(a.src + row))
                        : __ldg(reinterpret_cast<const float4*>(a.src + row));
      }
    }
    // the tail rows 64..69 are red stage rows 29..34
    const bool has_tail = t < 192;
    const int tail_r = 29 + (t >> 5), tail_c = t & 31;
    float2 vt = make_float2(0.f, 0.f);
    if (has_tail && !TMA) {
      const size_t row = (size_t)wrap_once(y0 - 2 + tail_r, L) * W + k0 + 2 * tail_c;
      vt = COHERENT ? __ldcg(reinterpret_cast<const float2*>(a.src + row))
                    : __ldg(reinterpret_cast<const float2*>(a.src + row));
    }
    // halo sites h = 0..135: plane h / 68, stage row 1 + (h % 68) / 2, side h & 1
    const int nh = t >= 192 ? 2 : (t >= 184 ? 1 : 0);
    float vh[2] = {0.f, 0.f};
    int hp[2] = {0, 0}, hr[2] = {0, 0}, hside[2] = {0, 0};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (j < nh) {
        const int h = t >= 192 ? (j == 0 ? t - 192 : t - 128) : t - 56;
        const int p = h >= 2 * kRedRows ? 1 : 0;
        const int rem = h - p * 2 * kRedRows;
        const int r = 1 + (rem >> 1);
        const int side = rem & 1;
        const size_t row = p * plane + (size_t)wrap_once(y0 - 2 + r, L) * W;
        const int kk = side ? wrap_once(k0 + kTileK, W) : wrap_once(k0 - 1, W);
        hp[j] = p;
        hr[j] = r;
        hside[j] = side;
        vh[j] = COHERENT ? __ldcg(a.src + row + kk) : __ldg(a.src + row + kk);
      }
    }
    if (TMA) {
      // the staged rows, written by TMA: wait for them, then read this
      // thread's groups and tail
      raw_wait();
#pragma unroll
      for (int i = 0; i < 4; ++i)
        v[i] = *reinterpret_cast<const float4*>(&ang[(t >> 4) + 16 * i][4 * cg]);
      if (has_tail) vt = *reinterpret_cast<const float2*>(&ang[64 + (t >> 5)][2 * tail_c]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rr = (t >> 4) + 16 * i;
      const int p = rr < kSRows ? 1 : 0;
      const int r = rr < kSRows ? rr : rr - kSRows + 1;
      float s0, c0, s1, c1, s2, c2, s3, c3;
      xyd::unit_vector<MODE>(v[i].x, &s0, &c0);
      xyd::unit_vector<MODE>(v[i].y, &s1, &c1);
      xyd::unit_vector<MODE>(v[i].z, &s2, &c2);
      xyd::unit_vector<MODE>(v[i].w, &s3, &c3);
      // the group's angles go to its ang row (staged row rr) unless TMA put
      // them there; only the red rows and the black tile rows 2..33 are read
      // (uniform over each half warp)
      if (!TMA && (p == 0 || (r >= 2 && r < kSRows - 2)))
        *reinterpret_cast<float4*>(&ang[rr][4 * cg]) = v[i];
      float2* u = p ? &csb[r][kCsOff + 4 * cg] : &csr[r - 1][kCsOff + 4 * cg];
      st4(u, make_float4(c0, s0, c1, s1));
      st4(u + 2, make_float4(c2, s2, c3, s3));
    }
    if (has_tail) {
      float s0, c0, s1, c1;
      xyd::unit_vector<MODE>(vt.x, &s0, &c0);
      xyd::unit_vector<MODE>(vt.y, &s1, &c1);
      if (!TMA) *reinterpret_cast<float2*>(&ang[64 + (t >> 5)][2 * tail_c]) = vt;
      st4(&csr[tail_r - 1][kCsOff + 2 * tail_c], make_float4(c0, s0, c1, s1));
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (j < nh) {
        float sv, cv;
        xyd::unit_vector<MODE>(vh[j], &sv, &cv);
        const int hcol = hside[j] ? kCsOff + kTileK : kCsOff - 1;
        if (hp[j] == 0) {                                  // red side-ring angles
          angs[2 * (hr[j] - 1) + hside[j]] = vh[j];
          csr[hr[j] - 1][hcol] = make_float2(cv, sv);
        } else {
          csb[hr[j]][hcol] = make_float2(cv, sv);
        }
      }
    }
  }
  pre();
  __syncthreads();

  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const uint32_t uL = (uint32_t)L;
  const int c0 = 2 * lane + kCsOff;                        // unit-vector column of the lane's pair
  const int kp = k0 + 2 * lane;                            // plane column of the pair
  unsigned int n_acc = 0;

  // ---- red half: the tile (counted, written to dst) ----
  float4 nbD = ld4(&csb[warp * 4 + 1][c0]);
  float4 nbP = ld4(&csb[warp * 4 + 2][c0]);
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = y & 1;                                   // red: x = 2k + (y & 1)
    PairNeighbours n;
    float4 nbU;
    pair_neighbours(csb, r, c0, q, nbD, nbP, nbU, n);
    nbD = nbP;
    nbP = nbU;
    const uint32_t site0 = (uint32_t)y * uL + 2u * (uint32_t)kp + (uint32_t)q;
    // sites x and x + 2 of the pair (kp even, so x & 2 == 0): one block
    const uint4 w = xyd::philox4x32_10(make_uint4(site0, a.sweep, a.lattice_id, 1u), rk);
    const float2 t = *reinterpret_cast<const float2*>(&ang[kRedRaw0 + r][2 * lane]);
    const float4 o = ld4(&csr[r - 1][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w.x, w.y, a.K, a.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w.z, w.w, a.K, a.delta);
    n_acc += (r0.accept ? 1u : 0u) + (r1.accept ? 1u : 0u);
    st4(&csr[r - 1][c0], make_float4(r0.c, r0.s, r1.c, r1.s));
    *reinterpret_cast<float2*>(a.dst + (size_t)y * W + kp) = make_float2(r0.th, r1.th);
  }
  // ---- red half: the ring at distance one (recomputed, not counted) ----
  // The ring rows above and below the tile are 32 pairs each (sites x and
  // x + 2 share a Philox block, as in the tile): warp 0 takes the row above,
  // warp 1 the row below; warp 2 takes the 32 side sites (left ring on odd
  // rows, right on even), one per lane.  The other warps wait at the barrier
  // and leave their issue slots to the SM's other CTAs.
  if (warp < 2) {
    const int ty = warp == 0 ? -1 : kTileRows;
    const int y = wrap_once(y0 + ty, L);
    const int r = ty + 2;
    const int q = y & 1;
    PairNeighbours n;
    float4 U;
    pair_neighbours(csb, r, c0, q, ld4(&csb[r - 1][c0]), ld4(&csb[r][c0]), U, n);
    const uint32_t site0 = (uint32_t)y * uL + 2u * (uint32_t)kp + (uint32_t)q;
    const uint4 w = xyd::philox4x32_10(make_uint4(site0, a.sweep, a.lattice_id, 1u), rk);
    const float2 t = *reinterpret_cast<const float2*>(&ang[kRedRaw0 + r][2 * lane]);
    const float4 o = ld4(&csr[r - 1][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w.x, w.y, a.K, a.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w.z, w.w, a.K, a.delta);
    st4(&csr[r - 1][c0], make_float4(r0.c, r0.s, r1.c, r1.s));
  } else if (warp == 2) {
    const int ty = lane;
    const int tk = ((y0 + ty) & 1) ? -1 : kTileK;          // left ring on odd rows, right on even
    const int y = wrap_once(y0 + ty, L);
    const int k = wrap_once(k0 + tk, W);
    const int q = y & 1;
    const uint32_t x = 2u * (uint32_t)k + (uint32_t)q;
    red_ring_site<MODE>(angs[2 * (ty + 1) + (tk < 0 ? 0 : 1)], csr, csb, ty + 2, tk + kCsOff, q,
                        (uint32_t)y * uL + x, x, a, rk);
  }
  mid();
  __syncthreads();
  post();

  // ---- black half of the tile, with the sweep sums ----
  xyd::SweepSums<RED> sums;
  sums.init();
  float* dst_blk = a.dst + plane;
  nbD = ld4(&csr[warp * 4][c0]);                           // red stage rows r - 1, r
  nbP = ld4(&csr[warp * 4 + 1][c0]);
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    const int r = ty + 2;
    const int q = (y + 1) & 1;                             // black: x = 2k + ((y + 1) & 1)
    PairNeighbours n;
    float4 nbU;
    pair_neighbours(csr, r - 1, c0, q, nbD, nbP, nbU, n);
    const float4 m = nbP;                                  // the red pair of the same row
    nbD = nbP;
    nbP = nbU;
    const uint32_t site0 = (uint32_t)y * uL + 2u * (uint32_t)kp + (uint32_t)q;
    // sites x and x + 2 of the pair (kp even, so x & 2 == 0): one block
    const uint4 w = xyd::philox4x32_10(make_uint4(site0, a.sweep, a.lattice_id, 1u), rk);
    const float2 t = *reinterpret_cast<const float2*>(&ang[r][2 * lane]);
    const float4 o = ld4(&csb[r][c0]);
    const xyd::SiteResult r0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, n.Sc[0], n.Ss[0], w.x, w.y, a.K, a.delta);
    const xyd::SiteResult r1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, n.Sc[1], n.Ss[1], w.z, w.w, a.K, a.delta);
    n_acc += (r0.accept ? 1u : 0u) + (r1.accept ? 1u : 0u);
    *reinterpret_cast<float2*>(dst_blk + (size_t)y * W + kp) = make_float2(r0.th, r1.th);

    // red sites with the same (y, k): their spins enter M once each
    float v0[5], v1[5];
    xyd::measure_terms(r0.c, r0.s, n.l[0].x, n.l[0].y, n.r[0].x, n.r[0].y, n.d[0].x, n.d[0].y,
                       n.u[0].x, n.u[0].y, n.Sc[0], n.Ss[0], m.x, m.y, v0);
    xyd::measure_terms(r1.c, r1.s, n.l[1].x, n.l[1].y, n.r[1].x, n.r[1].y, n.d[1].x, n.d[1].y,
                       n.u[1].x, n.u[1].y, n.Sc[1], n.Ss[1], m.z, m.w, v1);
    sums.add2(v0, v1);
  }

  end();
  // 8 black sites per thread: the per-warp integer sums fit 32 bits
  xyd::commit_sums<kWarps, RED, true>(sums, n_acc, part, cnt, a.rec, a.beta,
                                      bx == 0 && by == 0);
}

// Polls of a neighbour's flag or of the staging's mbarrier before a wait gives
// up (about a second in all).
constexpr long long kPersistSpinLimit = 1ll << 22;

// The TMA tensor maps of one state buffer read as a [2 L][W] float array
// (row p L + y: colour p, lattice row y), boxes of 64 plane columns and 1, 2
// and 32 rows; kernel parameters (__grid_constant__).
struct SweepMaps {
  CUtensorMap m[3];
};
struct PersistMaps {
  CUtensorMap m[2][3];   // of buf[0] and buf[1]
};

// The 70 staged rows of the tile at plane column x, rows y0.. into the ang
// buffer `dst` by TMA, completing on `bar` (one thread): black stage rows
// 0..35 (rows L + y0 - 2 .. L + y0 + 33) to ang rows 0..35, red stage rows
// 1..34 (rows y0 - 1 .. y0 + 32) to ang rows 36..69; the 32 tile rows of each
// plane are one box, the rows above and below boxes of 2 (black) and 1 (red)
// at their wrapped positions, so the lattice's first and last tile rows need
// no special case.  x is a multiple of 64 floats (256 bytes).
__device__ __forceinline__ void issue_tile_rows(uint64_t* bar, unsigned char* dst,
                                                const CUtensorMap* m, int x, int y0, int L) {
  xyt::mbar_arrive_expect_tx(bar, (uint32_t)kAngBytes);
  xyt::tma_load_2d(dst, &m[1], x, L + wrap_once(y0 - 2, L), bar);
  xyt::tma_load_2d(dst + 2 * kRawRowBytes, &m[2], x, L + y0, bar);
  xyt::tma_load_2d(dst + 34 * kRawRowBytes, &m[1], x, L + wrap_once(y0 + kTileRows, L), bar);
  xyt::tma_load_2d(dst + 36 * kRawRowBytes, &m[0], x, wrap_once(y0 - 1, L), bar);
  xyt::tma_load_2d(dst + 37 * kRawRowBytes, &m[2], x, y0, bar);
  xyt::tma_load_2d(dst + 69 * kRawRowBytes, &m[0], x, wrap_once(y0 + kTileRows, L), bar);
}

// MINB: CTAs per SM the kernel is compiled for (4: at most 64 registers a
// thread, 32 warps per SM; 3: at most 80; 2: at most 128, more independent
// work in flight per warp, 16 warps).  The tile's 55.3 KB of shared memory
// let four CTAs share an SM.  Thread 0 has TMA copy the tile's staged rows
// while every thread loads its halo sites; a bounded wait for them that runs
// out sets *a.error.  With compensated sums (RED = 1) every thread loads its
// rows itself instead: that variant's larger body fed by TMA stalled on
// instruction fetch (ncu: 2.2 no-instruction stalls per issued instruction,
// 172 against 188 G updates/s at L = 16384).
template <int MODE, int RED, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    k_sweep_fused(FusedArgs a, const __grid_constant__ SweepMaps maps) {
  if (RED != 0) {
    fused_sweep_body<MODE, RED>(a, a.rk, blockIdx.x, blockIdx.y);
    return;
  }
  __shared__ __align__(8) uint64_t s_bar;
  if (threadIdx.x == 0) {
    xyt::mbar_init(&s_bar, 1);
    xyt::fence_mbarrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    issue_tile_rows(&s_bar, smem_base(), maps.m, blockIdx.x * kTileK, blockIdx.y * kTileRows, a.L);
  fused_sweep_body<MODE, RED, false, true>(
      a, a.rk, blockIdx.x, blockIdx.y, 0, NoHook(), NoHook(), NoHook(), NoHook(), [&]() {
        if (!xyt::mbar_wait_bounded(&s_bar, 0u, kPersistSpinLimit) && a.error)
          atomicOr(a.error, 1u);
      });
}

// Many lattices of one side in one launch (blockIdx.z = lattice of the group),
// for the batched engine: the sweep index comes from the device counters and
// beta from the device (replica exchange moves it), the state ping-pongs
// between the batch's two buffers by sweep parity.
template <int MODE, int RED, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_sweep_fused_batch(FusedBatchArgs b) {
  const int i = b.lattices[blockIdx.z];
  const uint32_t sweep = b.counters[0] + (uint32_t)b.s;
  const float* base = (sweep & 1u) ? b.theta2 : b.theta;
  float* out = (sweep & 1u) ? b.theta : b.theta2;
  const double beta = b.beta[i];
  const FusedCore c{base + b.offset[i], out + b.offset[i], b.L, b.L / 2, (float)(beta * b.J),
                    b.delta, b.lattice_id0 + (uint32_t)i, sweep,
                    b.records + (size_t)i * b.rec_stride + (sweep - b.rec_sweep0), beta};
  fused_sweep_body<MODE, RED>(c, b.rk, blockIdx.x, blockIdx.y);
}


__device__ __forceinline__ unsigned int load_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void store_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A work item decoded once by the thread that fetched it: the item, its
// sweep and its tile position (so no other thread divides).
struct PersistItem {
  int item, s, bx, by;
};

__device__ __forceinline__ PersistItem decode_item(int item, int ntiles, int tiles_x,
                                                   int tiles_y) {
  PersistItem it;
  it.item = item;
  it.s = item / ntiles;
  const int k = item - it.s * ntiles;
  const int prow = k / tiles_x;
  it.bx = k - prow * tiles_x;
  it.by = (prow & 1) ? tiles_y - 1 - (prow >> 1) : (prow >> 1);
  return it;
}

// All n sweeps of one lattice in one cooperative launch (every CTA resident).
// The work items (sweep s, tile position k) are handed out in increasing order
// by one atomic counter, s-major, with the tile rows of a sweep visited folded
// (0, T-1, 1, T-2, ...) so that a tile's periodic neighbours are never more
// than two tile rows away in that order.  A tile's sweep s reads its own and
// its eight neighbours' state after sweep s - 1 (the halo of two rows and one
// column reaches into all eight) and overwrites the buffer they read during
// sweep s - 1, so it starts once those nine tiles (its own sweep s - 1 may have
// run on another CTA) have published flags[t] >= s; it publishes s + 1 after
// its stores.  An item waits only on
// items handed out before it, and every CTA holds at most its current item
// and the next (fetched while the current one runs), so with every CTA
// resident the waits always end; each is bounded anyway, and a wait that runs
// out sets *error and ends the CTA (the CTAs that wait on it see *error and
// end too).  Dynamic hand-out keeps the SMs evenly loaded as a launch per
// sweep does, without the launch's fill and drain.  Thread 0 fetches the next
// item at the start of a tile and decodes it before the staging barrier; the
// last warp, idle while the first three update the red ring, looks at that
// item's nine counters before the red/black barrier, and when all were set
// its first lane has TMA copy the next tile's 70 staged rows (issue_tile_rows)
// into the other of the CTA's two ang buffers while the ring and the black
// half run, and the next tile starts without waiting or a barrier; otherwise the
// next tile waits and then issues the same copies itself.  The copies
// complete on one mbarrier, one phase per tile; each wait for it is bounded
// too.  The arithmetic of a tile is fused_sweep_body's, so the result is bit
// for bit that of n launches of k_sweep_fused.
template <int MODE, int RED, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    k_sweep_fused_persist(FusedPersistArgs p, const __grid_constant__ PersistMaps maps) {
  __shared__ int s_abort;
  __shared__ PersistItem s_item[2];  // this tile's item and the next (alternating)
  __shared__ int s_ready[2];         // the next item's nine counters were all seen set
  __shared__ __align__(8) uint64_t s_bar;   // the staged rows' TMA completion
  constexpr int kIssuer = kThreads - 32;    // lane 0 of the last warp
  const int tiles_x = p.W / kTileK, tiles_y = p.L / kTileRows;
  const int ntiles = tiles_x * tiles_y;
  const int total = p.n_sweeps * ntiles;          // < 2^31 - 2^20 (the host splits longer runs)
  FusedCore c;
  c.L = p.L;
  c.W = p.W;
  c.K = p.K;
  c.delta = p.delta;
  c.lattice_id = p.lattice_id;
  c.beta = p.beta;
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_item[0] = decode_item((int)atomicAdd(p.counter, 1u) + p.skip_items, ntiles, tiles_x,
                            tiles_y);
    s_ready[0] = 0;
    xyt::mbar_init(&s_bar, 1);
    xyt::fence_mbarrier_init();
  }
  __syncthreads();
  int par = 0;
  uint32_t phase = 0;                // parity of the staged rows' next completion
  PersistItem cur = s_item[0];
  // the 70 staged rows of item `it` into ang buffer `buf` (by kIssuer; the
  // tile with item slot par uses ang buffer par)
  auto issue_raw = [&](const PersistItem& it, int buf) {
    xyt::fence_proxy_async_global();
    issue_tile_rows(&s_bar, smem_base() + (size_t)buf * kAngBytes, maps.m[it.s & 1],
                    it.bx * kTileK, it.by * kTileRows, p.L);
  };
  while (cur.item < total) {
    const int s = cur.s, bx = cur.bx, by = cur.by;
    // when the previous tile's early look found all nine counters set, this
    // tile neither waits nor needs the barrier (the acquire loads came before
    // the previous tile's closing barrier)
    const bool ready = s_ready[par] != 0;
    if (s > 0 && threadIdx.x < 9 && !ready) {
      // the eight neighbours and the tile itself (its sweep s - 1 may have run
      // on another CTA)
      const int d = threadIdx.x;
      const int nx = wrap_once(bx + d % 3 - 1, tiles_x);
      const int ny = wrap_once(by + d / 3 - 1, tiles_y);
      const unsigned int* f = p.flags + (ny * tiles_x + nx);
      long long it = 0;
      while (load_acquire(f) < (unsigned int)s) {
        // give up when the limit runs out, or early once another CTA has
        // given up (so a failure does not cascade from wait to wait)
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
    if (threadIdx.x == 0) next = (int)atomicAdd(p.counter, 1u) + p.skip_items;
    c.src = p.buf[s & 1];
    c.dst = p.buf[(s + 1) & 1];
    c.sweep = p.sweep0 + (uint32_t)s;
    c.rec = p.rec + s;
    PersistItem* slot = &s_item[par ^ 1];
    if (!ready && threadIdx.x == kIssuer) issue_raw(cur, par);
    fused_sweep_body<MODE, RED, true, true, 2>(
        c, p.rk, bx, by, par,
        // before the staging barrier: the next item, decoded, to the other slot
        // (the atomic was issued before the staging loads, so it has returned)
        [&]() {
          if (threadIdx.x == 0) *slot = decode_item(next, ntiles, tiles_x, tiles_y);
        },
        // before the red/black barrier, in the last warp (idle while the first
        // three update the ring): one early look at the next item's nine
        // counters, so that its wait usually costs nothing.  The acquire loads'
        // latency overlaps the ring instead of holding the CTA at its closing
        // barrier.  When all were set, the warp's first lane issues the next
        // tile's TMA copies at once, into the ang buffer the previous tile
        // used (free since that tile's closing barrier; __syncwarp orders the
        // other lanes' acquire loads before its proxy fence)
        [&]() {
          if (threadIdx.x >= kThreads - 32) {
            const int l = threadIdx.x - (kThreads - 32);
            bool ok = l >= 9;
            const PersistItem ni = *slot;
            if (l < 9 && ni.item < total) {
              const int nx = wrap_once(ni.bx + l % 3 - 1, tiles_x);
              const int ny = wrap_once(ni.by + l / 3 - 1, tiles_y);
              ok = ni.s == 0 || load_acquire(p.flags + (ny * tiles_x + nx)) >= (unsigned int)ni.s;
            }
            const bool all = __ballot_sync(0xffffffffu, ok) == 0xffffffffu;
            __syncwarp();
            if (l == 0) {
              s_ready[par ^ 1] = all ? 1 : 0;
              if (all) issue_raw(ni, par ^ 1);
            }
          }
        },
        NoHook(), NoHook(),
        // the staging's wait for its rows (bounded: a wait that runs out
        // sets the error word, and the tile goes on with what is there)
        [&]() {
          if (!xyt::mbar_wait_bounded(&s_bar, phase, p.spin_limit)) atomicOr(p.error, 1u);
          phase ^= 1u;
        });
    if (threadIdx.x == kThreads - 64) {
      // a warp other than the pollers' publishes the tile: the closing barrier
      // orders every thread's stores to dst before this GPU-scope release,
      // which is cumulative over the writes that happen before it
      store_release(p.flags + (by * tiles_x + bx), (unsigned int)(s + 1));
    }
    par ^= 1;
    cur = s_item[par];
  }
}

template <int MODE, int RED, int MINB>
cudaError_t launch_fused_one(const FusedArgs& a, cudaStream_t stream) {
  const int b = a.maps ? fused_map_index(*a.maps, a.src) : -1;
  if (b < 0) return cudaErrorInvalidValue;
  SweepMaps sm;
  for (int k = 0; k < 3; ++k) sm.m[k] = a.maps->m[b][k];
  static bool configured[64] = {};   // attributes set once per instantiation and device
  int dev = 0;
  cudaError_t ge = cudaGetDevice(&dev);
  if (ge != cudaSuccess) return ge;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_fused<MODE, RED, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_sweep_fused<MODE, RED, MINB>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const dim3 grid(a.W / kTileK, a.L / kTileRows);
  k_sweep_fused<MODE, RED, MINB><<<grid, kThreads, kSmemBytes, stream>>>(a, sm);
  return cudaGetLastError();
}

template <int MODE, int RED>
cudaError_t launch_fused_plan(const FusedArgs& a, cudaStream_t stream) {
  return a.minb == 2   ? launch_fused_one<MODE, RED, 2>(a, stream)
         : a.minb == 4 ? launch_fused_one<MODE, RED, 4>(a, stream)
                       : launch_fused_one<MODE, RED, 3>(a, stream);
}

template <int MODE, int RED>
cudaError_t launch_fused_batch_one(const FusedBatchArgs& b, int n_lattices, cudaStream_t stream) {
  // the attributes are set per device before any capture (prepare_fused_batch)
  const dim3 grid(b.L / 2 / kTileK, b.L / kTileRows, n_lattices);
  if (b.minb == 2)
    k_sweep_fused_batch<MODE, RED, 2><<<grid, kThreads, kSmemBytes, stream>>>(b);
  else if (b.minb == 4)
    k_sweep_fused_batch<MODE, RED, 4><<<grid, kThreads, kSmemBytes, stream>>>(b);
  else
    k_sweep_fused_batch<MODE, RED, 3><<<grid, kThreads, kSmemBytes, stream>>>(b);
  return cudaGetLastError();
}

template <int MODE, int RED, int MINB>
cudaError_t prepare_plan() {
  cudaError_t e = cudaFuncSetAttribute(k_sweep_fused_batch<MODE, RED, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sweep_fused_batch<MODE, RED, MINB>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

template <int MODE, int RED>
cudaError_t prepare_one() {
  cudaError_t e = prepare_plan<MODE, RED, 3>();
  if (e == cudaSuccess) e = prepare_plan<MODE, RED, 2>();
  return e == cudaSuccess ? prepare_plan<MODE, RED, 4>() : e;
}

template <int MODE, int RED, int MINB>
cudaError_t launch_persist_one(const FusedPersistArgs& a, int grid, cudaStream_t stream) {
  // the maps in buf order (the caller may have swapped the two buffers)
  PersistMaps pm;
  for (int b = 0; b < 2; ++b) {
    const int i = fused_map_index(*a.maps, a.buf[b]);
    if (i < 0) return cudaErrorInvalidValue;
    for (int k = 0; k < 3; ++k) pm.m[b][k] = a.maps->m[i][k];
  }
  void* args[] = {const_cast<FusedPersistArgs*>(&a), &pm};
  return cudaLaunchCooperativeKernel(
      reinterpret_cast<const void*>(&k_sweep_fused_persist<MODE, RED, MINB>), dim3(grid),
      dim3(kThreads), args, kPersistSmemBytes, stream);
}

template <int MODE, int RED, int MINB>
cudaError_t persist_grid_one(int L, int* grid) {
  static int per_sm[64] = {};        // resident CTAs per SM, per device (0: not yet set)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || per_sm[dev] == 0) {
    auto fn = k_sweep_fused_persist<MODE, RED, MINB>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPersistSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int n = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, kPersistSmemBytes);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorCooperativeLaunchTooLarge;
    if (dev >= 0 && dev < 64) per_sm[dev] = n;
    else per_sm[0] = n;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tiles = (L / 2 / kTileK) * (L / kTileRows);
  const int resident = per_sm[(dev >= 0 && dev < 64) ? dev : 0] * sms;
  *grid = tiles < resident ? tiles : resident;
  return cudaSuccess;
}

// The persistent launch of one instantiation: grid, then the launch.
template <int MODE, int RED, int MINB>
cudaError_t persist_plan(const FusedPersistArgs& a, cudaStream_t stream) {
  int grid = 0;
  cudaError_t e = persist_grid_one<MODE, RED, MINB>(a.L, &grid);
  if (e != cudaSuccess) return e;
  // the tile counters and, after them, the work counter
  e = cudaMemsetAsync(a.flags, 0, sizeof(unsigned int) * ((size_t)fused_tiles_of(a.L) + 1), stream);
  if (e != cudaSuccess) return e;
  return launch_persist_one<MODE, RED, MINB>(a, grid, stream);
}

template <int MODE, int RED>
cudaError_t persist_dispatch(const FusedPersistArgs& a, cudaStream_t stream) {
  return a.minb == 2   ? persist_plan<MODE, RED, 2>(a, stream)
         : a.minb == 4 ? persist_plan<MODE, RED, 4>(a, stream)
                       : persist_plan<MODE, RED, 3>(a, stream);
}

}  // namespace

bool fused_supported(int L) { return L >= 128 && (L % 128) == 0; }

cudaError_t prepare_fused_batch(int sincos_mode, int reduce_mode) {
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? prepare_one<0, 1>() : prepare_one<0, 0>();
    case 1: return comp ? prepare_one<1, 1>() : prepare_one<1, 0>();
    default: return comp ? prepare_one<2, 1>() : prepare_one<2, 0>();
  }
}

cudaError_t launch_fused_batch_sweep(int sincos_mode, int reduce_mode, const FusedBatchArgs& b,
                                     int n_lattices, cudaStream_t stream) {
  if (!fused_supported(b.L) || n_lattices < 1 || (b.minb < 2 || b.minb > 4))
    return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0:
      return comp ? launch_fused_batch_one<0, 1>(b, n_lattices, stream)
                  : launch_fused_batch_one<0, 0>(b, n_lattices, stream);
    case 1:
      return comp ? launch_fused_batch_one<1, 1>(b, n_lattices, stream)
                  : launch_fused_batch_one<1, 0>(b, n_lattices, stream);
    default:
      return comp ? launch_fused_batch_one<2, 1>(b, n_lattices, stream)
                  : launch_fused_batch_one<2, 0>(b, n_lattices, stream);
  }
}

cudaError_t launch_fused_sweep(int sincos_mode, int reduce_mode, const FusedArgs& a,
                               cudaStream_t stream) {
  if (!fused_supported(a.L) || (a.minb < 2 || a.minb > 4)) return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_fused_plan<0, 1>(a, stream) : launch_fused_plan<0, 0>(a, stream);
    case 1: return comp ? launch_fused_plan<1, 1>(a, stream) : launch_fused_plan<1, 0>(a, stream);
    default: return comp ? launch_fused_plan<2, 1>(a, stream) : launch_fused_plan<2, 0>(a, stream);
  }
}

}  // namespace xyk

namespace xyk {

int fused_tiles(int L) { return fused_supported(L) ? (L / 2 / kTileK) * (L / kTileRows) : 0; }

long long fused_persistent_spin_limit() { return kPersistSpinLimit; }

bool encode_fused_maps(FusedMaps* out, const float* buf0, const float* buf1, int L) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !out || !fused_supported(L)) return false;
  const float* bufs[2] = {buf0, buf1};
  out->base[0] = buf0;
  out->base[1] = buf1;
  const cuuint32_t rows[3] = {1u, 2u, (cuuint32_t)kTileRows};
  const cuuint64_t dims[2] = {(cuuint64_t)(L / 2), (cuuint64_t)(2 * L)};   // [2 L][W]
  const cuuint64_t strides[1] = {(cuuint64_t)(L / 2) * sizeof(float)};
  const cuuint32_t elem[2] = {1u, 1u};
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 3; ++k) {
      const cuuint32_t box[2] = {(cuuint32_t)kTileK, rows[k]};
      if (enc(&out->m[b][k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(bufs[b]), dims,
              strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    }
  return true;
}

int fused_persistent_max_sweeps(int L) {
  const int t = fused_tiles(L);
  // n x tiles items, plus one fetch past the end per CTA, stay below 2^31
  return t > 0 ? (int)((0x7fffffffu - (1u << 20)) / (unsigned)t) : 0;
}

cudaError_t launch_fused_persistent(int sincos_mode, int reduce_mode, const FusedPersistArgs& a,
                                    cudaStream_t stream) {
  if (!fused_supported(a.L) || a.W * 2 != a.L || a.n_sweeps < 1 ||
      a.n_sweeps > fused_persistent_max_sweeps(a.L) || !a.flags || a.counter != a.flags + fused_tiles(a.L) ||
      !a.error || a.buf[0] == a.buf[1] || !a.maps || a.spin_limit < 1 || a.skip_items < 0 ||
      a.skip_items > a.n_sweeps * fused_tiles(a.L) || (a.minb < 2 || a.minb > 4))
    return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? persist_dispatch<0, 1>(a, stream) : persist_dispatch<0, 0>(a, stream);
    case 1: return comp ? persist_dispatch<1, 1>(a, stream) : persist_dispatch<1, 0>(a, stream);
    default: return comp ? persist_dispatch<2, 1>(a, stream) : persist_dispatch<2, 0>(a, stream);
  }
}

}  // namespace xyk
