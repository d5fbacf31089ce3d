// xy_fused2.cu -- two sweeps per launch (temporal blocking of the fused sweep).
//
// A CTA owns the same tile as the one-sweep kernel (32 rows x 64 plane
// columns of both colours) but stages it with a halo of 4 rows and 4 plane
// columns on every side: after two sweeps (four half-sweeps) a site depends on
// the old state up to four half-sweeps away, one row and one plane column per
// half-sweep.  From the staged state it runs the four half-sweeps in shared
// memory on shrinking regions (stage rows and columns 1..38 / 1..70 for the
// red half of sweep s, 2..37 / 2..69 for its black half, 3..36 / 3..68 for
// the red half of sweep s + 1, and the tile itself for its black half), each
// site updated by the same device functions and Philox words as in the
// one-sweep kernels, so the angles, accept counts and exact sums are bit for
// bit those of two one-sweep launches.  The halo sites of the first three
// half-sweeps are recomputed copies of neighbouring tiles' updates.
//
// Against two one-sweep launches: DRAM traffic halves (the tile is read and
// written once per two sweeps: 4 B per update), staging unit vectors drop
// from 1.13 to 0.70 per update, and the recomputed halo adds 15 % updates
// (9400 site updates per 8192).
//
// Requires L % 128 == 0 (as the one-sweep fused kernel).
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_device.cuh"
#include "xy_internal.h"

namespace xyk {

namespace {

constexpr int kTileRows = 32;
constexpr int kTileK = 64;
constexpr int kHalo = 4;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSRows = kTileRows + 2 * kHalo;     // 40 stage rows: y0-4 .. y0+35
constexpr int kSC = kTileK + 2 * kHalo;           // 72 stage columns: k0-4 .. k0+67
// stage column c lives at index c + kCsPad of a cs row (neighbour reads reach
// c - 1 .. c + 2 for c in -1..71) and at c + kThPad of a th row (16-byte stores)
constexpr int kCsPad = 2, kCsCols = kSC + 4;
constexpr int kThPad = 4, kThCols = kSC + 8;

typedef float2 CsRow[kCsCols];
typedef float ThRow[kThCols];

constexpr size_t kCsBytes = sizeof(float2) * 2 * kSRows * kCsCols;
constexpr size_t kThBytes = sizeof(float) * 2 * kSRows * kThCols;
constexpr size_t kPartBytes = sizeof(float) * kWarps * 5 * 2;
constexpr size_t kCntBytes = sizeof(unsigned int) * kWarps;
constexpr size_t kSmemBytes = kCsBytes + kThBytes + kPartBytes + kCntBytes;

__device__ __forceinline__ int wrap_once(int v, int n) {
  v += (v < 0) ? n : 0;
  v -= (v >= n) ? n : 0;
  return v;
}

// One half-sweep of plane PLANE over stage rows [r_lo, r_hi] and stage
// columns [c_lo, c_hi], by Philox pairs (stage columns 2m, 2m + 1, which are
// plane columns k, k + 1 with k even): task i of a flat list over (row, pair)
// goes to thread i mod 256.  Sites of the pair outside the region are not
// updated (their words are drawn and dropped).  Sites inside the tile (stage
// rows and columns 4 .. 4 + tile - 1) count towards n_acc; with WRITE they are
// written to dst, and with MEASURE (black planes) their sweep sums are added.
template <int MODE, int RED, int PLANE, bool WRITE, bool MEASURE>
__device__ __forceinline__ void half_sweep(CsRow* cs, ThRow* th, const FusedArgs& a, int r_lo,
                                           int r_hi, int c_lo, int c_hi, uint32_t sweep,
                                           int y0, int k0, unsigned int& n_acc,
                                           xyd::SweepSums<RED>& sums) {
  CsRow* own_cs = cs + PLANE * kSRows;
  CsRow* nb_cs = cs + (1 - PLANE) * kSRows;
  ThRow* own_th = th + PLANE * kSRows;
  const int L = a.L, W = a.W;
  const uint32_t uL = (uint32_t)L;
  const int m_lo = c_lo >> 1, m_hi = c_hi >> 1;
  const int npairs = m_hi - m_lo + 1;
  const int ntasks = npairs * (r_hi - r_lo + 1);
  float* dst_plane = a.dst + (size_t)PLANE * (size_t)L * (size_t)W;
  for (int i = threadIdx.x; i < ntasks; i += kThreads) {
    const int rr = i / npairs;
    const int r = r_lo + rr;
    const int m = m_lo + (i - rr * npairs);
    const int c0 = 2 * m;                                // stage column of the pair
    const int y = wrap_once(y0 - kHalo + r, L);
    const int k = wrap_once(k0 - kHalo + c0, W);         // even (k0 % 64 == 0, W even)
    // red: x = 2k + (y & 1); black: x = 2k + ((y + 1) & 1); y0 is even
    const int q = PLANE == 0 ? (r & 1) : ((r + 1) & 1);
    const int ci = c0 + kCsPad;
    const float2 a0 = nb_cs[r][ci + q - 1], a1 = nb_cs[r][ci + q], a2 = nb_cs[r][ci + q + 1];
    const float4 D = *reinterpret_cast<const float4*>(&nb_cs[r - 1][ci]);
    const float4 U = *reinterpret_cast<const float4*>(&nb_cs[r + 1][ci]);
    // site j of the pair: left a_j, right a_{j+1}
    const float2 l0 = a0, r0n = a1, l1 = a1, r1n = a2;
    const float Sc0 = xyd::nb_sum(l0.x, r0n.x, D.x, U.x), Ss0 = xyd::nb_sum(l0.y, r0n.y, D.y, U.y);
    const float Sc1 = xyd::nb_sum(l1.x, r1n.x, D.z, U.z), Ss1 = xyd::nb_sum(l1.y, r1n.y, D.w, U.w);
    const uint32_t site0 = (uint32_t)y * uL + 2u * (uint32_t)k + (uint32_t)q;
    const uint4 w = xyd::philox4x32_10(make_uint4(site0, sweep, a.lattice_id, 1u), a.rk);
    const float2 t = *reinterpret_cast<const float2*>(&own_th[r][c0 + kThPad]);
    const float4 o = *reinterpret_cast<const float4*>(&own_cs[r][ci]);
    const xyd::SiteResult s0 =
        xyd::metropolis_step<MODE>(t.x, o.x, o.y, Sc0, Ss0, w.x, w.y, a.K, a.delta);
    const xyd::SiteResult s1 =
        xyd::metropolis_step<MODE>(t.y, o.z, o.w, Sc1, Ss1, w.z, w.w, a.K, a.delta);
    const bool in0 = c0 >= c_lo, in1 = c0 + 1 <= c_hi;
    // write back the sites of the region (both, the usual case, as one store)
    if (in0 && in1) {
      *reinterpret_cast<float2*>(&own_th[r][c0 + kThPad]) = make_float2(s0.th, s1.th);
      *reinterpret_cast<float4*>(&own_cs[r][ci]) = make_float4(s0.c, s0.s, s1.c, s1.s);
    } else if (in0) {
      own_th[r][c0 + kThPad] = s0.th;
      own_cs[r][ci] = make_float2(s0.c, s0.s);
    } else if (in1) {
      own_th[r][c0 + 1 + kThPad] = s1.th;
      own_cs[r][ci + 1] = make_float2(s1.c, s1.s);
    }
    const bool tile = r >= kHalo && r < kHalo + kTileRows && c0 >= kHalo && c0 < kHalo + kTileK;
    if (tile) {       // the pair lies in the tile entirely (c0 even, tile columns 4..67)
      n_acc += (s0.accept ? 1u : 0u) + (s1.accept ? 1u : 0u);
      if (WRITE)
        *reinterpret_cast<float2*>(dst_plane + (size_t)y * W + k) = make_float2(s0.th, s1.th);
      if (MEASURE) {
        // red sites with the same (y, k): their spins enter M once each
        const float4 mr = *reinterpret_cast<const float4*>(&nb_cs[r][ci]);
        float v0[5], v1[5];
        xyd::measure_terms(s0.c, s0.s, l0.x, l0.y, r0n.x, r0n.y, D.x, D.y, U.x, U.y, Sc0, Ss0,
                           mr.x, mr.y, v0);
        xyd::measure_terms(s1.c, s1.s, l1.x, l1.y, r1n.x, r1n.y, D.z, D.w, U.z, U.w, Sc1, Ss1,
                           mr.z, mr.w, v1);
        sums.add2(v0, v1);
      }
    }
  }
}

template <int MODE, int RED>
__global__ void __launch_bounds__(kThreads, 3) k_sweep_fused2(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  CsRow* cs = reinterpret_cast<CsRow*>(smem);                       // [2][kSRows]
  ThRow* th = reinterpret_cast<ThRow*>(smem + kCsBytes);            // [2][kSRows]
  float(*part)[5][2] = reinterpret_cast<float(*)[5][2]>(smem + kCsBytes + kThBytes);
  unsigned int* cnt = reinterpret_cast<unsigned int*>(smem + kCsBytes + kThBytes + kPartBytes);
  const int L = a.L, W = a.W;
  const int k0 = blockIdx.x * kTileK, y0 = blockIdx.y * kTileRows;
  const size_t plane = (size_t)L * (size_t)W;

  // ---- stage both planes, rows y0-4 .. y0+35, plane columns k0-4 .. k0+67:
  // 2 x 40 rows x 18 aligned groups of four columns (a group is wholly inside
  // the lattice or wholly wrapped, as k0 % 64 == 0 and W % 64 == 0) ----
  constexpr int kGroups = kSC / 4;
  constexpr int kUnits = 2 * kSRows * kGroups;                      // 1440
  for (int u = threadIdx.x; u < kUnits; u += kThreads) {
    const int p = u / (kSRows * kGroups);
    const int rem = u - p * (kSRows * kGroups);
    const int r = rem / kGroups;
    const int g = rem - r * kGroups;
    const int y = wrap_once(y0 - kHalo + r, L);
    const int kg = wrap_once(k0 - kHalo + 4 * g, W);
    const float4 v = __ldg(reinterpret_cast<const float4*>(a.src + p * plane + (size_t)y * W + kg));
    float s0, c0, s1, c1, s2, c2, s3, c3;
    xyd::unit_vector<MODE>(v.x, &s0, &c0);
    xyd::unit_vector<MODE>(v.y, &s1, &c1);
    xyd::unit_vector<MODE>(v.z, &s2, &c2);
    xyd::unit_vector<MODE>(v.w, &s3, &c3);
    CsRow* csp = cs + p * kSRows;
    ThRow* thp = th + p * kSRows;
    *reinterpret_cast<float4*>(&thp[r][4 * g + kThPad]) = v;
    *reinterpret_cast<float4*>(&csp[r][4 * g + kCsPad]) = make_float4(c0, s0, c1, s1);
    *reinterpret_cast<float4*>(&csp[r][4 * g + 2 + kCsPad]) = make_float4(c2, s2, c3, s3);
  }
  __syncthreads();

  const bool first = blockIdx.x == 0 && blockIdx.y == 0;
  unsigned int n_acc = 0;
  xyd::SweepSums<RED> sums;
  sums.init();
  // sweep s: red on rows 1..38 / columns 1..70, black on 2..37 / 2..69
  half_sweep<MODE, RED, 0, false, false>(cs, th, a, 1, kSRows - 2, 1, kSC - 2, a.sweep, y0, k0,
                                         n_acc, sums);
  __syncthreads();
  half_sweep<MODE, RED, 1, false, true>(cs, th, a, 2, kSRows - 3, 2, kSC - 3, a.sweep, y0, k0,
                                        n_acc, sums);
  xyd::commit_sums<kWarps, RED, true>(sums, n_acc, part, cnt, a.rec, a.beta, first);
  __syncthreads();   // the commit's warp 0 reads `part` after its barrier: keep it apart
  n_acc = 0;
  sums.init();
  // sweep s + 1: red on rows 3..36 / columns 3..68 (the tile and a ring of
  // one), black on the tile; both write their tile sites to dst
  half_sweep<MODE, RED, 0, true, false>(cs, th, a, 3, kSRows - 4, 3, kSC - 4, a.sweep + 1u, y0,
                                        k0, n_acc, sums);
  __syncthreads();
  half_sweep<MODE, RED, 1, true, true>(cs, th, a, kHalo, kHalo + kTileRows - 1, kHalo,
                                       kHalo + kTileK - 1, a.sweep + 1u, y0, k0, n_acc, sums);
  xyd::commit_sums<kWarps, RED, true>(sums, n_acc, part, cnt, a.rec + 1, a.beta, first);
}

template <int MODE, int RED>
cudaError_t launch_one(const FusedArgs& a, cudaStream_t stream) {
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(k_sweep_fused2<MODE, RED>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_sweep_fused2<MODE, RED>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const dim3 grid(a.W / kTileK, a.L / kTileRows);
  k_sweep_fused2<MODE, RED><<<grid, kThreads, kSmemBytes, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused2_sweeps(int sincos_mode, int reduce_mode, const FusedArgs& a,
                                 cudaStream_t stream) {
  if (!fused_supported(a.L) || a.src == a.dst) return cudaErrorInvalidValue;
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_one<0, 1>(a, stream) : launch_one<0, 0>(a, stream);
    case 1: return comp ? launch_one<1, 1>(a, stream) : launch_one<1, 0>(a, stream);
    default: return comp ? launch_one<2, 1>(a, stream) : launch_one<2, 0>(a, stream);
  }
}

}  // namespace xyk
