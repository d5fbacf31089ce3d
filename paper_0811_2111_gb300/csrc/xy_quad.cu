// xy_quad.cu -- four replicas per site (the RGBA packing of Sec. 3.2): the
// two-pass checkerboard half-sweep over float4 sites (any even L), and the C
// ABI of include/xy_quad.h around it and around the one-launch sweep of
// xy_quad_fused.cu (L % 32 == 0).
//
// Layout: [colour][y][k] of float4, component r = replica r.  A half-sweep of
// colour c stages the other colour's tile plus a one-site halo as unit vectors
// (float4 cos, float4 sin: the four replicas of a site in one 16-byte word),
// then every thread updates one site of colour c per row for all four
// replicas: the neighbour loads and addressing are shared, the four Metropolis
// steps are independent (four-way instruction-level parallelism), and the
// accept is the vector select of Sec. 3.2, one component per replica.  Replica
// r runs the single-lattice arithmetic (xyd::metropolis_step with its own
// Metropolis words under lattice id lattice_id + r and its own beta), so it is
// bit-identical to that lattice swept by the kernels of xy_sweep.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "xy_device.cuh"
#include "xy_internal.h"
#include "xy_trace.h"
#include "xy_quad.h"

namespace {

constexpr int kR = XY_QUAD_REPLICAS;
constexpr int kTileRows = 32;        // rows of the updated plane per CTA
constexpr int kTileCols = 32;        // plane columns per CTA (one per lane)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kStage = kTileRows + 2;   // staged rows y0-1 .. y0+32 and columns k0-1 .. k0+32

struct QuadArgs {
  float4* theta;          // [2][L][W] float4
  int L;
  int W;
  float K[kR];            // beta_r * J
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id0;
  uint32_t sweep;
  xy_record* rec;         // the four records of this sweep (replica-major within the sweep)
  double beta[kR];
};

__device__ __forceinline__ float comp(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

template <int COLOUR, int MODE, int RED>
__global__ void __launch_bounds__(kThreads) k_quad_half(QuadArgs a) {
  __shared__ float4 s_cos[kStage][kStage];
  __shared__ float4 s_sin[kStage][kStage];
  __shared__ float s_part[kR][kWarps][5][2];
  __shared__ unsigned int s_cnt[kR][kWarps];

  const int L = a.L, W = a.W;
  const int k0 = blockIdx.x * kTileCols, y0 = blockIdx.y * kTileRows;
  const size_t plane = (size_t)L * (size_t)W;
  const float4* __restrict__ other = a.theta + (size_t)(1 - COLOUR) * plane;
  float4* __restrict__ own = a.theta + (size_t)COLOUR * plane;

  // ---- stage the other colour's unit vectors (four replicas per site) ----
  for (int g = threadIdx.x; g < kStage * kStage; g += kThreads) {
    const int r = g / kStage, c = g - r * kStage;
    const int gy = xyd::wrap_index(y0 - 1 + r, L);
    const int gk = xyd::wrap_index(k0 - 1 + c, W);
    const float4 t = other[(size_t)gy * W + gk];
    float4 cs, sn;
    xyd::unit_vector<MODE>(t.x, &sn.x, &cs.x);
    xyd::unit_vector<MODE>(t.y, &sn.y, &cs.y);
    xyd::unit_vector<MODE>(t.z, &sn.z, &cs.z);
    xyd::unit_vector<MODE>(t.w, &sn.w, &cs.w);
    s_cos[r][c] = cs;
    s_sin[r][c] = sn;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool measure = (COLOUR == 1);
  unsigned int n_acc[kR] = {0u, 0u, 0u, 0u};
  xyd::SweepSums<RED> sums[kR];                  // at most 4 black sites per replica and thread
#pragma unroll
  for (int j = 0; j < kR; ++j) sums[j].init();

  const int k = k0 + lane;
  const int sc = lane + 1;                               // stage column of (y, k)
  for (int rr = 0; rr < 4; ++rr) {
    const int ty = warp * 4 + rr;
    const int y = y0 + ty;
    if (y >= L || k >= W) continue;
    const int q = (y + COLOUR) & 1;                      // x = 2k + q
    // neighbours in the other plane: (y, k+q-1) left, (y, k+q) right,
    // (y-1, k) down, (y+1, k) up
    const float4 cl = s_cos[ty + 1][sc + q - 1], sl = s_sin[ty + 1][sc + q - 1];
    const float4 cr = s_cos[ty + 1][sc + q], sr = s_sin[ty + 1][sc + q];
    const float4 cd = s_cos[ty][sc], sd = s_sin[ty][sc];
    const float4 cu = s_cos[ty + 2][sc], su = s_sin[ty + 2][sc];
    const float4 cm = s_cos[ty + 1][sc], sm = s_sin[ty + 1][sc];
    float4* p = own + (size_t)y * W + k;
    const float4 th = *p;
    const uint32_t x = 2u * (uint32_t)k + (uint32_t)q;
    const uint32_t ctr = xyd::metropolis_counter((uint32_t)y * (uint32_t)L + x, x);
    float out[kR];
#pragma unroll
    for (int j = 0; j < kR; ++j) {
      const float Sc = xyd::nb_sum(comp(cl, j), comp(cr, j), comp(cd, j), comp(cu, j));
      const float Ss = xyd::nb_sum(comp(sl, j), comp(sr, j), comp(sd, j), comp(su, j));
      const uint2 w = xyd::metropolis_words(
          xyd::philox4x32_10(make_uint4(ctr, a.sweep, a.lattice_id0 + (uint32_t)j, 1u), a.rk), x);
      const float t = comp(th, j);
      float s0, c0;
      xyd::unit_vector<MODE>(t, &s0, &c0);
      const xyd::SiteResult res =
          xyd::metropolis_step<MODE>(t, c0, s0, Sc, Ss, w.x, w.y, a.K[j], a.delta);
      out[j] = res.th;
      n_acc[j] += res.accept ? 1u : 0u;
      if (measure) {
        float v[5];
        xyd::measure_terms(res.c, res.s, comp(cl, j), comp(sl, j), comp(cr, j), comp(sr, j),
                           comp(cd, j), comp(sd, j), comp(cu, j), comp(su, j), Sc, Ss, comp(cm, j),
                           comp(sm, j), v);
        sums[j].add(v);
      }
    }
    *p = make_float4(out[0], out[1], out[2], out[3]);
  }

  const bool first = blockIdx.x == 0 && blockIdx.y == 0;
#pragma unroll
  for (int j = 0; j < kR; ++j)
    xyd::commit_sums<kWarps, RED, COLOUR == 1>(sums[j], n_acc[j], s_part[j], s_cnt[j], a.rec + j,
                                               a.beta[j], first);
}

__global__ void k_quad_start(float4* theta, int L, const xyd::RoundKeys rk, uint32_t lattice_id0,
                             int hot) {
  const uint32_t N = (uint32_t)L * (uint32_t)L, half = N / 2u, W = (uint32_t)L / 2u;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < half * 2u; i += gridDim.x * blockDim.x) {
    const uint32_t c = i / half, rem = i - c * half;
    const uint32_t y = rem / W, kk = rem - y * W;
    const uint32_t x = 2u * kk + ((y + c) & 1u);
    float v[kR] = {0.f, 0.f, 0.f, 0.f};
    if (hot) {
#pragma unroll
      for (int j = 0; j < kR; ++j) {
        const uint4 w = xyd::philox4x32_10(make_uint4(y * (uint32_t)L + x, 0u, lattice_id0 + j, 0u), rk);
        v[j] = (float)(w.x >> 8) * xyd::kHotScale;
      }
    }
    theta[i] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

__global__ void k_quad_extract(const float4* __restrict__ theta, float* __restrict__ out, int j,
                               int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = comp(theta[i], j);
}

template <int COLOUR, int MODE, int RED>
cudaError_t launch_one(const QuadArgs& a, cudaStream_t s) {
  const dim3 grid((a.W + kTileCols - 1) / kTileCols, (a.L + kTileRows - 1) / kTileRows);
  k_quad_half<COLOUR, MODE, RED><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_quad_half(int colour, int mode, int red, const QuadArgs& a, cudaStream_t s) {
  if (colour == 0) {
    switch (mode) {
      case 0: return launch_one<0, 0, 0>(a, s);
      case 1: return launch_one<0, 1, 0>(a, s);
      default: return launch_one<0, 2, 0>(a, s);
    }
  }
  switch (mode) {
    case 0: return red ? launch_one<1, 0, 1>(a, s) : launch_one<1, 0, 0>(a, s);
    case 1: return red ? launch_one<1, 1, 1>(a, s) : launch_one<1, 1, 0>(a, s);
    default: return red ? launch_one<1, 2, 1>(a, s) : launch_one<1, 2, 0>(a, s);
  }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// XY_ALGO_AUTO takes the persistent sweep up to this side (beyond it one
// launch per sweep has enough waves of tiles to hide its fill and drain:
// measured at L = 2048 152.7 against 155.9 G updates/s, at 1024 152.4 against
// 136.5)
constexpr int kAutoPersistentMaxL = 1024;

constexpr uint32_t kMagicLive = 0x51554144u;   // "QUAD"
constexpr uint32_t kMagicDead = 0xDEADF00Du;

thread_local char g_msg[512] = "no error";
std::mutex g_mu;
std::unordered_set<const void*>& live() {
  static std::unordered_set<const void*> s;
  return s;
}
bool is_live(const void* q) {
  std::lock_guard<std::mutex> g(g_mu);
  return live().count(q) != 0;
}
void mark(const void* q, bool on) {
  std::lock_guard<std::mutex> g(g_mu);
  if (on) {
    live().insert(q);
  } else {
    live().erase(q);
  }
}
void tmsg(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}

}  // namespace

struct xy_quad {
  uint32_t magic;
  xy_params p;
  double beta[kR];
  cudaStream_t stream;
  bool fused;              // one-launch sweeps, state ping-ponged between the two buffers
  bool persistent;         // ... all sweeps of a call in one cooperative launch
  bool auto_persistent;    // chosen by XY_ALGO_AUTO: per-sweep launches if it does not fit
  unsigned int* d_tiles;   // the persistent launch's tile counters, work counter, error word
  int cur;                 // which buffer holds the state (0: d_theta, 1: d_theta2)
  float4* d_theta;         // [2][L][L/2] float4
  float4* d_theta2;        // the fused sweep's second buffer (NULL for two-pass)
  float* d_scratch;        // L*L floats: one replica, split then natural order
  float* d_nat;
  xy_record* d_rec;        // [sweep][replica]
  int64_t rec_cap;         // sweeps
  int64_t rec_count;       // sweeps
  uint64_t next_sweep;
  xy_status sticky;
  char msg[512];
};

namespace {

xy_status fail(xy_quad* q, xy_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  snprintf(g_msg, sizeof(g_msg), "%s", buf);
  if (q && is_live(q) && q->magic == kMagicLive && q->sticky == XY_OK) {
    q->sticky = st;
    snprintf(q->msg, sizeof(q->msg), "%s", buf);
  }
  return st;
}

xy_status cuda_fail(xy_quad* q, cudaError_t e, const char* what) {
  (void)cudaGetLastError();
  return fail(q, e == cudaErrorMemoryAllocation ? XY_ENOMEM : XY_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorName(e), cudaGetErrorString(e));
}

#define Q_CUDA(q, call, what)                              \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(q, e_, what);  \
  } while (0)

xy_status check(const xy_quad* q) {
  if (!q) {
    tmsg("NULL quad context");
    return XY_EINVAL;
  }
  if (!is_live(q) || q->magic != kMagicLive) {
    tmsg("quad context is not live (destroyed or never created)");
    return XY_ESTATE;
  }
  if (q->sticky != XY_OK) {
    tmsg("quad context is in an earlier error: %s", q->msg);
    return q->sticky;
  }
  return XY_OK;
}

float4* current(const xy_quad* q) { return q->cur ? q->d_theta2 : q->d_theta; }

// After a synchronize: whether a persistent launch's bounded wait ran out.
xy_status check_waits(xy_quad* q, const char* where) {
  if (!q->persistent || !q->d_tiles) return XY_OK;
  unsigned int w = 0;
  const int tiles = xyk::quad_persistent_tiles(q->p.L);
  Q_CUDA(q, cudaMemcpyAsync(&w, q->d_tiles + tiles + 1, sizeof(w), cudaMemcpyDeviceToHost, q->stream),
         where);
  Q_CUDA(q, cudaStreamSynchronize(q->stream), where);
  if (w) return fail(q, XY_ETIMEOUT, "%s: a persistent sweep's wait for a neighbouring tile ran out",
                     where);
  return XY_OK;
}

void release(xy_quad* q) {
  if (q->d_theta) cudaFree(q->d_theta);
  if (q->d_theta2) cudaFree(q->d_theta2);
  if (q->d_tiles) cudaFree(q->d_tiles);
  if (q->d_scratch) cudaFree(q->d_scratch);
  if (q->d_nat) cudaFree(q->d_nat);
  if (q->d_rec) cudaFree(q->d_rec);
}

xy_status grow(xy_quad* q, int64_t sweeps) {
  if (sweeps <= q->rec_cap) return XY_OK;
  int64_t cap = q->rec_cap > 0 ? q->rec_cap : 1024;
  while (cap < sweeps) cap *= 2;
  xy_record* nr = nullptr;
  Q_CUDA(q, xyk::dev_malloc(&nr, (size_t)cap * kR * sizeof(xy_record)), "record buffer");
  if (q->rec_count > 0) {
    cudaError_t e = cudaMemcpyAsync(nr, q->d_rec, (size_t)q->rec_count * kR * sizeof(xy_record),
                                    cudaMemcpyDeviceToDevice, q->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    if (e != cudaSuccess) {
      cudaFree(nr);
      return cuda_fail(q, e, "record copy");
    }
  }
  if (q->d_rec) cudaFree(q->d_rec);
  q->d_rec = nr;
  q->rec_cap = cap;
  return XY_OK;
}

}  // namespace

extern "C" {

xy_status xy_quad_create(const xy_params* p, const double beta[4], void* cuda_stream,
                         xy_quad** out) {
  if (!out) {
    tmsg("NULL output pointer");
    return XY_EINVAL;
  }
  *out = nullptr;
  if (!p || !beta) {
    tmsg("NULL params or beta");
    return XY_EINVAL;
  }
  if (p->L < 2 || p->L > XY_MAX_L || (p->L & 1)) {
    tmsg("L must be even and in [2, %d]; got %d", XY_MAX_L, p->L);
    return XY_EINVAL;
  }
  for (int j = 0; j < kR; ++j) {
    if (!(beta[j] >= 0.0) || !isfinite(beta[j])) {
      tmsg("beta[%d] must be finite and >= 0", j);
      return XY_EINVAL;
    }
  }
  if (!isfinite(p->J) || !(p->delta > 0.0) || p->delta > M_PI + 1e-12 ||
      (p->start != XY_START_HOT && p->start != XY_START_COLD) || p->sincos_mode < 0 ||
      p->sincos_mode > 2 || p->reduce_mode < 0 || p->reduce_mode > 1) {
    tmsg("bad J, delta, start, sincos_mode or reduce_mode");
    return XY_EINVAL;
  }
  if (p->algorithm != XY_ALGO_AUTO && p->algorithm != XY_ALGO_FUSED &&
      p->algorithm != XY_ALGO_TWO_PASS && p->algorithm != XY_ALGO_PERSISTENT) {
    tmsg("algorithm must be XY_ALGO_AUTO, _FUSED, _TWO_PASS or _PERSISTENT; got %d", p->algorithm);
    return XY_EINVAL;
  }
  if ((p->algorithm == XY_ALGO_FUSED || p->algorithm == XY_ALGO_PERSISTENT) &&
      !xyk::quad_fused_supported(p->L)) {
    tmsg("XY_ALGO_FUSED and XY_ALGO_PERSISTENT need L %% 32 == 0; got L = %d", p->L);
    return XY_EINVAL;
  }
  xy_quad* q = new (std::nothrow) xy_quad();
  if (!q) {
    tmsg("host allocation");
    return XY_ENOMEM;
  }
  q->p = *p;
  for (int j = 0; j < kR; ++j) q->beta[j] = beta[j];
  q->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  q->fused = p->algorithm != XY_ALGO_TWO_PASS && xyk::quad_fused_supported(p->L);
  q->persistent = p->algorithm == XY_ALGO_PERSISTENT ||
                  (p->algorithm == XY_ALGO_AUTO && q->fused && p->L <= kAutoPersistentMaxL);
  q->auto_persistent = q->persistent && p->algorithm == XY_ALGO_AUTO;
  q->cur = 0;
  const size_t N = (size_t)p->L * (size_t)p->L;
  const char* step = "angle buffer";
  cudaError_t e = xyk::dev_malloc(&q->d_theta, N * sizeof(float4));
  if (e == cudaSuccess && q->fused) e = xyk::dev_malloc(&q->d_theta2, N * sizeof(float4));
  if (e == cudaSuccess && q->persistent) {
    const size_t words = (size_t)xyk::quad_persistent_tiles(p->L) + 2;
    e = xyk::dev_malloc(&q->d_tiles, words * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(q->d_tiles, 0, words * sizeof(unsigned int), q->stream);
  }
  if (e == cudaSuccess) {
    step = "scratch buffers";
    e = xyk::dev_malloc(&q->d_scratch, N * sizeof(float));
    if (e == cudaSuccess) e = xyk::dev_malloc(&q->d_nat, N * sizeof(float));
  }
  if (e == cudaSuccess) {
    step = "start kernel";
    k_quad_start<<<xyk::grid_for((int64_t)N, 256), 256, 0, q->stream>>>(
        q->d_theta, p->L, xyd::make_round_keys(p->seed), p->lattice_id,
        p->start == XY_START_HOT ? 1 : 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    step = "synchronize";
    e = cudaStreamSynchronize(q->stream);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    tmsg("xy_quad_create: %s: %s (%s)", step, cudaGetErrorName(e), cudaGetErrorString(e));
    release(q);
    delete q;
    return e == cudaErrorMemoryAllocation ? XY_ENOMEM : XY_ECUDA;
  }
  q->magic = kMagicLive;
  q->sticky = XY_OK;
  snprintf(q->msg, sizeof(q->msg), "no error");
  mark(q, true);
  *out = q;
  return XY_OK;
}

xy_status xy_quad_sweep(xy_quad* q, int64_t n) {
  const xyk::TraceRange trace("xy_quad_sweep");
  xyk::NvtxRange range("xy_quad_sweep");
  xy_status st = check(q);
  if (st != XY_OK) return st;
  if (n < 0) return fail(q, XY_EINVAL, "xy_quad_sweep: negative sweep count");
  if (n == 0) return XY_OK;
  if (q->next_sweep + (uint64_t)n > 0xffffffffull)
    return fail(q, XY_EINVAL, "xy_quad_sweep: sweep counter would pass 2^32 - 1");
  st = grow(q, q->rec_count + n);
  if (st != XY_OK) return st;
  Q_CUDA(q, cudaMemsetAsync(q->d_rec + q->rec_count * kR, 0, (size_t)n * kR * sizeof(xy_record),
                            q->stream),
         "xy_quad_sweep: record clear");
  if (q->persistent) {
    xyk::QuadPersistArgs pa;
    pa.a.src = nullptr;
    pa.a.dst = nullptr;
    pa.a.L = q->p.L;
    pa.a.W = q->p.L / 2;
    for (int j = 0; j < kR; ++j) {
      pa.a.K[j] = (float)(q->beta[j] * q->p.J);
      pa.a.beta[j] = q->beta[j];
    }
    pa.a.delta = (float)q->p.delta;
    pa.a.rk = xyd::make_round_keys(q->p.seed);
    pa.a.lattice_id0 = q->p.lattice_id;
    pa.a.sweep = 0;
    pa.a.rec = nullptr;
    const int tiles = xyk::quad_persistent_tiles(q->p.L);
    pa.flags = q->d_tiles;
    pa.counter = q->d_tiles + tiles;
    pa.error = q->d_tiles + tiles + 1;
    pa.spin_limit = xyk::quad_persistent_spin_limit();
    const int64_t chunk = xyk::quad_persistent_max_sweeps(q->p.L);
    for (int64_t done = 0; done < n;) {
      const int64_t m = std::min<int64_t>(n - done, chunk);
      pa.buf[0] = reinterpret_cast<float*>(current(q));
      pa.buf[1] = reinterpret_cast<float*>(q->cur ? q->d_theta : q->d_theta2);
      pa.sweep0 = (uint32_t)(q->next_sweep + (uint64_t)done);
      pa.n_sweeps = (int)m;
      pa.rec = q->d_rec + (q->rec_count + done) * kR;
      cudaError_t e = xyk::launch_quad_persistent(q->p.sincos_mode, q->p.reduce_mode, pa, q->stream);
      if (e == cudaErrorCooperativeLaunchTooLarge && q->auto_persistent) {
        // the grid does not fit beside other work: one fused launch per sweep
        (void)cudaGetLastError();
        xyk::QuadFusedArgs f = pa.a;
        e = cudaSuccess;
        for (int64_t i = 0; i < m && e == cudaSuccess; ++i) {
          f.src = pa.buf[i & 1];
          f.dst = pa.buf[(i + 1) & 1];
          f.sweep = pa.sweep0 + (uint32_t)i;
          f.rec = pa.rec + i * kR;
          e = xyk::launch_quad_fused(q->p.sincos_mode, q->p.reduce_mode, f, q->stream);
        }
      }
      Q_CUDA(q, e, "xy_quad_sweep: persistent sweep");
      if (m & 1) q->cur ^= 1;
      done += m;
    }
    q->next_sweep += (uint64_t)n;
    q->rec_count += n;
    return XY_OK;
  }
  if (q->fused) {
    xyk::QuadFusedArgs f;
    f.L = q->p.L;
    f.W = q->p.L / 2;
    for (int j = 0; j < kR; ++j) {
      f.K[j] = (float)(q->beta[j] * q->p.J);
      f.beta[j] = q->beta[j];
    }
    f.delta = (float)q->p.delta;
    f.rk = xyd::make_round_keys(q->p.seed);
    f.lattice_id0 = q->p.lattice_id;
    for (int64_t i = 0; i < n; ++i) {
      f.src = reinterpret_cast<const float*>(current(q));
      f.dst = reinterpret_cast<float*>(q->cur ? q->d_theta : q->d_theta2);
      f.sweep = (uint32_t)(q->next_sweep + (uint64_t)i);
      f.rec = q->d_rec + (q->rec_count + i) * kR;
      Q_CUDA(q, xyk::launch_quad_fused(q->p.sincos_mode, q->p.reduce_mode, f, q->stream),
             "xy_quad_sweep: fused sweep");
      q->cur ^= 1;
    }
    q->next_sweep += (uint64_t)n;
    q->rec_count += n;
    return XY_OK;
  }
  QuadArgs a;
  a.theta = current(q);
  a.L = q->p.L;
  a.W = q->p.L / 2;
  for (int j = 0; j < kR; ++j) {
    a.K[j] = (float)(q->beta[j] * q->p.J);
    a.beta[j] = q->beta[j];
  }
  a.delta = (float)q->p.delta;
  a.rk = xyd::make_round_keys(q->p.seed);
  a.lattice_id0 = q->p.lattice_id;
  for (int64_t i = 0; i < n; ++i) {
    a.sweep = (uint32_t)(q->next_sweep + (uint64_t)i);
    a.rec = q->d_rec + (q->rec_count + i) * kR;
    Q_CUDA(q, launch_quad_half(0, q->p.sincos_mode, q->p.reduce_mode, a, q->stream),
           "xy_quad_sweep: red half");
    Q_CUDA(q, launch_quad_half(1, q->p.sincos_mode, q->p.reduce_mode, a, q->stream),
           "xy_quad_sweep: black half");
  }
  q->next_sweep += (uint64_t)n;
  q->rec_count += n;
  return XY_OK;
}

xy_status xy_quad_measure(xy_quad* q, int32_t replica, int64_t first, int64_t count, xy_obs* out) {
  xy_status st = check(q);
  if (st != XY_OK) return st;
  if (replica < 0 || replica >= kR) return fail(q, XY_EINVAL, "xy_quad_measure: replica out of range");
  if (first < 0 || count < 0 || first + count > q->rec_count)
    return fail(q, XY_EINVAL, "xy_quad_measure: range [%lld, %lld) outside [0, %lld)",
                (long long)first, (long long)(first + count), (long long)q->rec_count);
  if (count > 0 && !out) return fail(q, XY_EINVAL, "xy_quad_measure: NULL output");
  if (count == 0) return XY_OK;
  std::vector<xy_record> r;
  try {
    r.resize((size_t)count * kR);
  } catch (...) {
    return fail(q, XY_ENOMEM, "xy_quad_measure: host allocation");
  }
  Q_CUDA(q, cudaMemcpyAsync(r.data(), q->d_rec + first * kR, (size_t)count * kR * sizeof(xy_record),
                            cudaMemcpyDeviceToHost, q->stream),
         "xy_quad_measure: copy");
  Q_CUDA(q, cudaStreamSynchronize(q->stream), "xy_quad_measure: stream");
  st = check_waits(q, "xy_quad_measure");
  if (st != XY_OK) return st;
  const double N = (double)q->p.L * (double)q->p.L, J = q->p.J;
  for (int64_t i = 0; i < count; ++i) {
    const xy_record& rec = r[(size_t)i * kR + replica];
    xy_obs& o = out[i];
    if (rec.flags) return fail(q, XY_ENUMERIC, "xy_quad_measure: non-finite sums in a record");
    o.C = ldexp((double)rec.sum[0], -XY_FX_SHIFT);
    o.Ix = ldexp((double)rec.sum[1], -XY_FX_SHIFT);
    o.Iy = ldexp((double)rec.sum[2], -XY_FX_SHIFT);
    o.Mx = ldexp((double)rec.sum[3], -XY_FX_SHIFT);
    o.My = ldexp((double)rec.sum[4], -XY_FX_SHIFT);
    o.e = -J * o.C / N;
    o.abs_m = sqrt(o.Mx * o.Mx + o.My * o.My) / N;
    o.upsilon = (J * o.C - rec.beta * J * J * (o.Ix * o.Ix + o.Iy * o.Iy)) / (2.0 * N);
    o.accepted = rec.accepted;
    o.beta = rec.beta;
  }
  return XY_OK;
}

xy_status xy_quad_get_state(xy_quad* q, int32_t replica, float* host, uint64_t* next_sweep) {
  xy_status st = check(q);
  if (st != XY_OK) return st;
  if (replica < 0 || replica >= kR) return fail(q, XY_EINVAL, "xy_quad_get_state: replica out of range");
  if (!host) return fail(q, XY_EINVAL, "xy_quad_get_state: NULL output");
  const int64_t N = (int64_t)q->p.L * q->p.L;
  k_quad_extract<<<xyk::grid_for(N, 256), 256, 0, q->stream>>>(current(q), q->d_scratch, replica, N);
  Q_CUDA(q, cudaGetLastError(), "xy_quad_get_state: extract");
  Q_CUDA(q, xyk::launch_split_to_natural(q->d_scratch, q->d_nat, q->p.L, q->stream),
         "xy_quad_get_state: layout");
  Q_CUDA(q, cudaMemcpyAsync(host, q->d_nat, (size_t)N * sizeof(float), cudaMemcpyDeviceToHost,
                            q->stream),
         "xy_quad_get_state: copy");
  Q_CUDA(q, cudaStreamSynchronize(q->stream), "xy_quad_get_state: stream");
  st = check_waits(q, "xy_quad_get_state");
  if (st != XY_OK) return st;
  if (next_sweep) *next_sweep = q->next_sweep;
  return XY_OK;
}

xy_status xy_quad_info(const xy_quad* q, int64_t* n_records, uint64_t* next_sweep) {
  xy_status st = check(q);
  if (st != XY_OK) return st;
  if (n_records) *n_records = q->rec_count;
  if (next_sweep) *next_sweep = q->next_sweep;
  return XY_OK;
}

xy_status xy_quad_algorithm(const xy_quad* q, int32_t* algorithm) {
  xy_status st = check(q);
  if (st != XY_OK) return st;
  if (!algorithm) {
    tmsg("xy_quad_algorithm: NULL output");
    return XY_EINVAL;
  }
  *algorithm = q->persistent ? XY_ALGO_PERSISTENT : (q->fused ? XY_ALGO_FUSED : XY_ALGO_TWO_PASS);
  return XY_OK;
}

xy_status xy_quad_synchronize(xy_quad* q) {
  xy_status st = check(q);
  if (st != XY_OK) return st;
  Q_CUDA(q, cudaStreamSynchronize(q->stream), "xy_quad_synchronize");
  st = check_waits(q, "xy_quad_synchronize");
  if (st != XY_OK) return st;
  return XY_OK;
}

xy_status xy_quad_destroy(xy_quad* q) {
  if (!q) return XY_OK;
  if (!is_live(q) || q->magic != kMagicLive) {
    tmsg("xy_quad_destroy: not a live quad context");
    return XY_ESTATE;
  }
  mark(q, false);
  (void)cudaStreamSynchronize(q->stream);
  release(q);
  q->magic = kMagicDead;
  delete q;
  return XY_OK;
}

const char* xy_quad_last_error(const xy_quad* q) {
  if (q && is_live(q) && q->magic == kMagicLive && q->sticky != XY_OK) return q->msg;
  return g_msg;
}

}  // extern "C"
