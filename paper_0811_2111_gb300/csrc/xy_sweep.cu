// xy_sweep.cu -- checkerboard Metropolis half-sweep kernels for one lattice.
//
// One launch updates every site of one colour in place.  Sites of a colour
// only neighbour sites of the other colour, so a half-sweep reads the other
// plane (unchanged during the launch) and rewrites its own plane; no two
// threads touch the same angle.
//
// Tile: 32 rows x 128 plane columns of the updated colour per CTA of 256
// threads (warp w owns rows 4w..4w+3, lane l owns columns 4l..4l+3, one
// float4 per row).  The other colour's tile plus a one-site halo is staged
// into shared memory once as (cos, sin) pairs, so every neighbour angle is
// turned into its unit vector once per half-sweep and read four times from
// shared memory.
//
// Per site (Metropolis step, xyd::metropolis_step; the select is the
// per-site vector accept of Sec. 3.2):
//   S     = sum of the four neighbour unit vectors
//   theta'= wrap(theta + delta (2 u0 - 1))                (Philox word 0)
//   X     = (cos theta' - cos theta) S_c + (sin theta' - sin theta) S_s
//         = -dE / J for dE = -J sum_nn [cos(theta'-theta_j) - cos(theta-theta_j)]
//   accept iff u1 < exp(beta J X)                          (Philox word 1)
// The black half also accumulates the sweep's sums (Eq. (1) bonds): every
// bond joins a red and a black site, so the four bonds of each black site
// cover all 2N bonds exactly once:
//   C  += cos_b S_c + sin_b S_s
//   Ix += sin(t_b - t_right) - sin(t_b - t_left)
//   Iy += sin(t_b - t_up)    - sin(t_b - t_down)
//   M  += unit vector of the black site + of the red site with the same (y, k).
// Reduction (xyd::commit_sums): every term rounded to fixed point before any
// addition, exact integer sums per thread, warp and CTA, then one 64-bit
// atomic add per sum into the record: the record depends on neither the
// order of addition nor the kernel (compensated FP32 in reduce mode 1).
#include <cuda_runtime.h>
#include <stdint.h>

#include "xy_debug.h"
#include "xy_device.cuh"
#include "xy_internal.h"

namespace xyk {

namespace {

constexpr int kTileRows = 32;        // rows of the updated plane per CTA
constexpr int kTileCols = 128;       // plane columns per CTA (32 lanes x 4)
constexpr int kThreads = 256;
constexpr int kStageRows = kTileRows + 2;
constexpr int kStageCols = kTileCols + 8;   // 4 pad columns each side keep float4 alignment
constexpr int kStageGroups = kStageCols / 4;

template <int COLOUR, int MODE, int RED>
__global__ void __launch_bounds__(kThreads)
k_half_sweep(HalfSweepArgs a) {
  __shared__ __align__(16) float s_cos[kStageRows][kStageCols];
  __shared__ __align__(16) float s_sin[kStageRows][kStageCols];
  __shared__ float s_part[kThreads / 32][5][2];
  __shared__ unsigned int s_cnt[kThreads / 32];

  const int L = a.L, W = a.W;
  const int k0 = blockIdx.x * kTileCols;
  const int y0 = blockIdx.y * kTileRows;
  const size_t plane = (size_t)L * (size_t)W;
  const float* __restrict__ other = a.theta + (size_t)(1 - COLOUR) * plane;
  float* __restrict__ own = a.theta + (size_t)COLOUR * plane;
  const bool vec4 = (W & 3) == 0;

  // ---- stage the other colour: rows y0-1 .. y0+32, columns k0-4 .. k0+131 ----
  for (int g = threadIdx.x; g < kStageRows * kStageGroups; g += kThreads) {
    const int r = g / kStageGroups;
    const int cg = g - r * kStageGroups;
    const int gy = xyd::wrap_index(y0 - 1 + r, L);
    const int kk = k0 - 4 + 4 * cg;
    const float* row = other + (size_t)gy * W;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (vec4) {
      const int kw = xyd::wrap_index(kk, W);
      if (XY_DCHECK(gy >= 0 && gy < L && kw >= 0 && kw + 3 < W, 0)) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(row + kw));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int kw = xyd::wrap_index(kk + e, W);
        if (XY_DCHECK(gy >= 0 && gy < L && kw >= 0 && kw < W, 0)) v[e] = __ldg(row + kw);
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int col = 4 * cg + e;
      // only columns k0-1 .. k0+128 are ever read
      if (col >= 3 && col <= kTileCols + 4) {
        float s, c;
        xyd::unit_vector<MODE>(v[e], &s, &c);
        if (XY_DCHECK(r >= 0 && r < kStageRows, 1)) {
          s_cos[r][col] = c;
          s_sin[r][col] = s;
        }
      }
    }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned int n_acc = 0;
  xyd::SweepSums<RED> sums;                    // at most 16 black sites per thread
  sums.init();
  const bool measure = (COLOUR == 1);

  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    if (y >= L) break;                                   // warp-uniform
    const int q = (y + COLOUR) & 1;                      // x = 2k + q
    const int kq = k0 + lane * 4;
    float* rowp = own + (size_t)y * W;
    float th[4] = {0.f, 0.f, 0.f, 0.f};
    const bool full = vec4 && (kq + 3 < W);
    if (full) {
      if (XY_DCHECK(y >= 0 && y < L && kq >= 0, 2)) {
        const float4 t = *reinterpret_cast<const float4*>(rowp + kq);
        th[0] = t.x; th[1] = t.y; th[2] = t.z; th[3] = t.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (kq + j < W && XY_DCHECK(y >= 0 && y < L && kq + j >= 0, 2)) th[j] = rowp[kq + j];
    }
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (kq + j >= W) continue;
      const int sc = lane * 4 + j + 4;                   // stage column of (y, k)
      // the stage rows ty .. ty + 2 and columns sc + q - 1 .. sc + q are read
      if (!XY_DCHECK(ty >= 0 && ty + 2 < kStageRows && sc + q - 1 >= 0 && sc + q < kStageCols, 3))
        continue;
      // neighbours in the other plane: same row at k+q-1 (left) and k+q
      // (right), rows y-1 (down) and y+1 (up) at k
      const float cl = s_cos[ty + 1][sc + q - 1], sl = s_sin[ty + 1][sc + q - 1];
      const float cr = s_cos[ty + 1][sc + q], sr = s_sin[ty + 1][sc + q];
      const float cd = s_cos[ty][sc], sd = s_sin[ty][sc];
      const float cu = s_cos[ty + 2][sc], su = s_sin[ty + 2][sc];
      const float Sc = xyd::nb_sum(cl, cr, cd, cu);
      const float Ss = xyd::nb_sum(sl, sr, sd, su);

      // kq is a multiple of 4: columns kq + {0, 1} and kq + {2, 3} are pairs
      // (x and x + 2 with x & 2 == 0), one block drawn for each
      const uint32_t x = 2u * (uint32_t)(kq + j) + (uint32_t)q;
      const uint32_t site = (uint32_t)y * (uint32_t)L + x;
      if ((j & 1) == 0)
        w = xyd::philox4x32_10(make_uint4(site, a.sweep, a.lattice_id, 1u), a.rk);
      const uint2 uw = xyd::metropolis_words(w, x);
      const float t = th[j];
      float s0, c0;
      xyd::unit_vector<MODE>(t, &s0, &c0);
      const xyd::SiteResult res = xyd::metropolis_step<MODE>(t, c0, s0, Sc, Ss, uw.x, uw.y, a.K,
                                                             a.delta);
      th[j] = res.th;
      n_acc += res.accept ? 1u : 0u;
      if (measure) {
        float v[5];
        xyd::measure_terms(res.c, res.s, cl, sl, cr, sr, cd, sd, cu, su, Sc, Ss,
                           s_cos[ty + 1][sc], s_sin[ty + 1][sc], v);
        sums.add(v);
      }
    }
    if (full) {
      if (XY_DCHECK(y >= 0 && y < L && kq >= 0, 2))
        *reinterpret_cast<float4*>(rowp + kq) = make_float4(th[0], th[1], th[2], th[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (kq + j < W && XY_DCHECK(y >= 0 && y < L && kq + j >= 0, 2)) rowp[kq + j] = th[j];
    }
  }

  xyd::commit_sums<kThreads / 32, RED, COLOUR == 1>(sums, n_acc, s_part, s_cnt, a.rec, a.beta,
                                                   blockIdx.x == 0 && blockIdx.y == 0);
}

__global__ void k_start(float* __restrict__ theta, int L, const xyd::RoundKeys rk,
                        uint32_t lattice_id, int hot) {
  const uint32_t N = (uint32_t)L * (uint32_t)L;
  const uint32_t W = (uint32_t)L / 2u;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    // i indexes the split layout: [colour][y][k]
    const uint32_t c = i / (N / 2u);
    const uint32_t rem = i - c * (N / 2u);
    const uint32_t y = rem / W, k = rem - y * W;
    const uint32_t x = 2u * k + ((y + c) & 1u);
    float t = 0.f;
    if (hot) {
      const uint4 w = xyd::philox4x32_10(make_uint4(y * (uint32_t)L + x, 0u, lattice_id, 0u), rk);
      t = (float)(w.x >> 8) * xyd::kHotScale;
    }
    // the split layout's index of (c, y, k) is i itself
    if (XY_DCHECK(c < 2u && y < (uint32_t)L && k < W &&
                  (size_t)c * (N / 2u) + (size_t)y * W + k == (size_t)i, 4))
      theta[i] = t;
  }
}

__global__ void k_natural_to_split(const float* __restrict__ nat, float* __restrict__ split,
                                   int L) {
  const uint32_t N = (uint32_t)L * (uint32_t)L, W = (uint32_t)L / 2u;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
    const uint32_t y = s / (uint32_t)L, x = s - y * (uint32_t)L;
    const uint32_t c = (x + y) & 1u;
    // angles are taken modulo 2 pi (in double) so the kernels only see [0, 2 pi)
    const double two_pi = 6.283185307179586476925;
    double v = fmod((double)nat[s], two_pi);
    if (v < 0.0) v += two_pi;
    float f = (float)v;
    if (f >= xyd::kTwoPi) f = 0.f;
    const size_t d = (size_t)c * (N / 2u) + (size_t)y * W + (x >> 1);
    if (XY_DCHECK(d < (size_t)N, 4)) split[d] = f;
  }
}

__global__ void k_split_to_natural(const float* __restrict__ split, float* __restrict__ nat,
                                   int L) {
  const uint32_t N = (uint32_t)L * (uint32_t)L, W = (uint32_t)L / 2u;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
    const uint32_t y = s / (uint32_t)L, x = s - y * (uint32_t)L;
    const uint32_t c = (x + y) & 1u;
    const size_t d = (size_t)c * (N / 2u) + (size_t)y * W + (x >> 1);
    if (XY_DCHECK(d < (size_t)N, 4)) nat[s] = split[d];
  }
}

__global__ void k_philox_words(const xyd::RoundKeys rk, uint32_t sweep, uint32_t lattice_id,
                               uint32_t domain, uint32_t first, int64_t n, uint4* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = xyd::philox4x32_10(make_uint4(first + (uint32_t)i, sweep, lattice_id, domain), rk);
  }
}

template <int MODE>
__global__ void k_eval_unit_vector(const float* __restrict__ t, float* __restrict__ c,
                                   float* __restrict__ s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float sv, cv;
    xyd::unit_vector<MODE>(t[i], &sv, &cv);
    c[i] = cv;
    s[i] = sv;
  }
}

__global__ void k_check_finite(const float* __restrict__ v, int64_t n, unsigned int* flag) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bad |= !isfinite(v[i]);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

template <int COLOUR, int MODE, int RED>
cudaError_t launch_one(const HalfSweepArgs& a, cudaStream_t stream) {
  const dim3 grid((a.W + kTileCols - 1) / kTileCols, (a.L + kTileRows - 1) / kTileRows);
  k_half_sweep<COLOUR, MODE, RED><<<grid, kThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_half_sweep(int colour, int sincos_mode, int reduce_mode,
                              const HalfSweepArgs& a, cudaStream_t stream) {
  if (colour == 0) {
    switch (sincos_mode) {
      case 0: return launch_one<0, 0, 0>(a, stream);
      case 1: return launch_one<0, 1, 0>(a, stream);
      default: return launch_one<0, 2, 0>(a, stream);
    }
  }
  const bool comp = reduce_mode != 0;
  switch (sincos_mode) {
    case 0: return comp ? launch_one<1, 0, 1>(a, stream) : launch_one<1, 0, 0>(a, stream);
    case 1: return comp ? launch_one<1, 1, 1>(a, stream) : launch_one<1, 1, 0>(a, stream);
    default: return comp ? launch_one<1, 2, 1>(a, stream) : launch_one<1, 2, 0>(a, stream);
  }
}

cudaError_t launch_start(float* theta, int L, const xyd::RoundKeys& rk, uint32_t lattice_id,
                         int hot, cudaStream_t stream) {
  const int64_t N = (int64_t)L * L;
  k_start<<<grid_for(N, 256), 256, 0, stream>>>(theta, L, rk, lattice_id, hot);
  return cudaGetLastError();
}

cudaError_t launch_natural_to_split(const float* nat, float* split, int L, cudaStream_t stream) {
  k_natural_to_split<<<grid_for((int64_t)L * L, 256), 256, 0, stream>>>(nat, split, L);
  return cudaGetLastError();
}

cudaError_t launch_split_to_natural(const float* split, float* nat, int L, cudaStream_t stream) {
  k_split_to_natural<<<grid_for((int64_t)L * L, 256), 256, 0, stream>>>(split, nat, L);
  return cudaGetLastError();
}

cudaError_t launch_philox_words(const xyd::RoundKeys& rk, uint32_t sweep, uint32_t lattice_id,
                                uint32_t domain, uint32_t first, int64_t n, uint32_t* out,
                                cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_philox_words<<<grid_for(n, 256), 256, 0, stream>>>(rk, sweep, lattice_id, domain,
                                                       first, n, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

cudaError_t launch_eval_unit_vector(int mode, const float* theta, float* c, float* s, int64_t n,
                                    cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int g = grid_for(n, 256);
  if (mode == 0) {
    k_eval_unit_vector<0><<<g, 256, 0, stream>>>(theta, c, s, n);
  } else if (mode == 1) {
    k_eval_unit_vector<1><<<g, 256, 0, stream>>>(theta, c, s, n);
  } else {
    k_eval_unit_vector<2><<<g, 256, 0, stream>>>(theta, c, s, n);
  }
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* theta, int64_t n, unsigned int* flag,
                                cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_check_finite<<<grid_for(n, 256), 256, 0, stream>>>(theta, n, flag);
  return cudaGetLastError();
}

}  // namespace xyk

namespace xyk {

// The debug word of this translation unit (two-pass sweep and layout
// kernels; bits 0-4), read and cleared.  0 in the release build.
unsigned int debug_take_sweep() { return xy_debug_take_word(); }

}  // namespace xyk
