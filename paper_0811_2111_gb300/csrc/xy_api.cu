// xy_api.cu -- the C ABI declared in include/xy.h: validation, ownership,
// sticky errors and launch sequencing around the kernels of xy_sweep.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "xy.h"
#include "xy_internal.h"
#include "xy_trace.h"

namespace {

constexpr uint32_t kMagicLive = 0x58594C54u;   // "XYLT"
constexpr uint32_t kMagicDead = 0xDEADC0DEu;

thread_local char g_thread_msg[512] = "no error";

// Live contexts, so that a destroyed or foreign pointer is refused without
// reading freed memory.
std::mutex g_live_mu;
std::unordered_set<const void*>& live_set() {
  static std::unordered_set<const void*> s;
  return s;
}
bool is_live(const void* c) {
  std::lock_guard<std::mutex> g(g_live_mu);
  return live_set().count(c) != 0;
}
void mark_live(const void* c, bool live) {
  std::lock_guard<std::mutex> g(g_live_mu);
  if (live) {
    live_set().insert(c);
  } else {
    live_set().erase(c);
  }
}

void set_thread_msg(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_thread_msg, sizeof(g_thread_msg), fmt, ap);
  va_end(ap);
}

}  // namespace

// XY_ALGO_AUTO takes the persistent sweep up to this side: there a sweep is
// at most nine waves of tiles and one launch per sweep pays its fill and drain
// every sweep; beyond it (L = 8192: 36 waves) the per-sweep launch is faster.
constexpr int kAutoPersistentMaxL = 4096;

struct xy_ctx {
  uint32_t magic;
  xy_params p;
  cudaStream_t stream;
  int device;
  float* d_theta;          // [2][L][L/2]: the state between calls
  bool owns_theta;
  float* d_pong;           // second buffer of the fused kernel (library-owned)
  bool fused;              // sweeps use the fused kernel
  bool persistent;         // ... all sweeps of an xy_sweep call in one cooperative launch
  bool auto_persistent;    // chosen by XY_ALGO_AUTO: per-sweep launches if it does not fit
  unsigned int* d_tiles;   // the persistent launch's per-tile sweep counters
  xyk::FusedMaps maps;     // TMA tensor maps of d_theta and d_pong (fused kernels)
  unsigned int* d_wait;    // set by a fused launch whose bounded wait ran out
  xy_record* d_rec;        // records [0, rec_cap)
  int64_t rec_cap;
  int64_t rec_count;       // records enqueued so far
  uint64_t next_sweep;     // Philox sweep word of the next sweep
  float* d_scratch;        // natural-order staging for get/set state
  unsigned int* d_flag;    // device flag word (non-finite check)
  int timing_every;        // bracket every k-th sweep's launches with events (0: off)
  std::vector<cudaEvent_t> ev[2];   // per kernel: start/stop pairs, in order
  size_t ev_used[2];
  xy_status sticky;
  char msg[512];
};

namespace {

xy_status fail(xy_ctx* c, xy_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  snprintf(g_thread_msg, sizeof(g_thread_msg), "%s", buf);
  if (c && is_live(c) && c->magic == kMagicLive && c->sticky == XY_OK) {
    c->sticky = st;
    snprintf(c->msg, sizeof(c->msg), "%s", buf);
  }
  return st;
}

xy_status cuda_fail(xy_ctx* c, cudaError_t e, const char* what) {
  (void)cudaGetLastError();   // do not leave a non-sticky error for the next launch check
  return fail(c, e == cudaErrorMemoryAllocation ? XY_ENOMEM : XY_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorName(e), cudaGetErrorString(e));
}

#define XY_CUDA(ctx, call, what)                       \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

xy_status check_ctx(const xy_ctx* c) {
  if (!c) {
    set_thread_msg("NULL context");
    return XY_EINVAL;
  }
  if (!is_live(c) || c->magic != kMagicLive) {
    set_thread_msg("context is not live (destroyed or never created)");
    return XY_ESTATE;
  }
  if (c->sticky != XY_OK) {
    set_thread_msg("context is in an earlier error: %s", c->msg);
    return c->sticky;
  }
  return XY_OK;
}

xy_status validate(const xy_params* p) {
  if (!p) {
    set_thread_msg("NULL params");
    return XY_EINVAL;
  }
  if (p->L < 2 || p->L > XY_MAX_L || (p->L & 1)) {
    set_thread_msg("L must be even and in [2, %d] (checkerboard needs a bipartite torus); got %d",
                   XY_MAX_L, p->L);
    return XY_EINVAL;
  }
  if (!(p->beta >= 0.0) || !isfinite(p->beta)) {
    set_thread_msg("beta must be finite and >= 0");
    return XY_EINVAL;
  }
  if (!isfinite(p->J)) {
    set_thread_msg("J must be finite");
    return XY_EINVAL;
  }
  if (!(p->delta > 0.0) || p->delta > M_PI + 1e-12) {
    set_thread_msg("delta must be in (0, pi]");
    return XY_EINVAL;
  }
  if (p->start != XY_START_HOT && p->start != XY_START_COLD) {
    set_thread_msg("start must be XY_START_HOT or XY_START_COLD");
    return XY_EINVAL;
  }
  if (p->sincos_mode != XY_SINCOS_ACCURATE && p->sincos_mode != XY_SINCOS_FAST &&
      p->sincos_mode != XY_SINCOS_LIBM) {
    set_thread_msg("bad sincos_mode");
    return XY_EINVAL;
  }
  if (p->reduce_mode != XY_REDUCE_EXACT && p->reduce_mode != XY_REDUCE_COMPENSATED) {
    set_thread_msg("bad reduce_mode");
    return XY_EINVAL;
  }
  if (p->algorithm != XY_ALGO_AUTO && p->algorithm != XY_ALGO_FUSED &&
      p->algorithm != XY_ALGO_TWO_PASS && p->algorithm != XY_ALGO_PERSISTENT &&
      p->algorithm != XY_ALGO_FUSED2) {
    set_thread_msg("bad algorithm");
    return XY_EINVAL;
  }
  if (p->ctas_per_sm != 0 && (p->ctas_per_sm < 2 || p->ctas_per_sm > 4)) {
    set_thread_msg("ctas_per_sm must be 0 (default), 2, 3 or 4; got %d", p->ctas_per_sm);
    return XY_EINVAL;
  }
  if ((p->algorithm == XY_ALGO_FUSED || p->algorithm == XY_ALGO_PERSISTENT ||
       p->algorithm == XY_ALGO_FUSED2) &&
      !xyk::fused_supported(p->L)) {
    set_thread_msg("the fused kernel needs L to be a multiple of 128; got %d", p->L);
    return XY_EINVAL;
  }
  return XY_OK;
}

xy_status grow_records(xy_ctx* c, int64_t need) {
  if (need <= c->rec_cap) return XY_OK;
  int64_t cap = c->rec_cap > 0 ? c->rec_cap : 1024;
  while (cap < need) cap *= 2;
  xy_record* nr = nullptr;
  XY_CUDA(c, xyk::dev_malloc(&nr, (size_t)cap * sizeof(xy_record)), "allocating records");
  cudaError_t e = cudaMemsetAsync(nr, 0, (size_t)cap * sizeof(xy_record), c->stream);
  if (e == cudaSuccess && c->rec_count > 0)
    e = cudaMemcpyAsync(nr, c->d_rec, (size_t)c->rec_count * sizeof(xy_record),
                        cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFree(nr);
    return cuda_fail(c, e, "growing records");
  }
  if (c->d_rec) cudaFree(c->d_rec);
  c->d_rec = nr;
  c->rec_cap = cap;
  return XY_OK;
}

// Event pair for the next timed launch of kernel k (grows the pool).
cudaError_t next_events(xy_ctx* c, int k, cudaEvent_t* a, cudaEvent_t* b) {
  std::vector<cudaEvent_t>& v = c->ev[k];
  while (v.size() < c->ev_used[k] + 2) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    v.push_back(e);
  }
  *a = v[c->ev_used[k]];
  *b = v[c->ev_used[k] + 1];
  c->ev_used[k] += 2;
  return cudaSuccess;
}

cudaError_t timed_half_sweep(xy_ctx* c, int colour, const xyk::HalfSweepArgs& a) {
  if (c->timing_every <= 0 || (a.sweep % (uint32_t)c->timing_every) != 0)
    return xyk::launch_half_sweep(colour, c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  cudaEvent_t e0, e1;
  cudaError_t e = next_events(c, colour, &e0, &e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  if (e == cudaSuccess)
    e = xyk::launch_half_sweep(colour, c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  return e;
}

cudaError_t timed_fused(xy_ctx* c, const xyk::FusedArgs& a) {
  if (c->timing_every <= 0 || (a.sweep % (uint32_t)c->timing_every) != 0)
    return xyk::launch_fused_sweep(c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  cudaEvent_t e0, e1;
  cudaError_t e = next_events(c, 0, &e0, &e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  if (e == cudaSuccess) e = xyk::launch_fused_sweep(c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  return e;
}

cudaError_t timed_fused2(xy_ctx* c, const xyk::FusedArgs& a) {
  if (c->timing_every <= 0 || (a.sweep / 2u % (uint32_t)c->timing_every) != 0)
    return xyk::launch_fused2_sweeps(c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  cudaEvent_t e0, e1;
  cudaError_t e = next_events(c, 0, &e0, &e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  if (e == cudaSuccess)
    e = xyk::launch_fused2_sweeps(c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  return e;
}

// After a synchronize: whether a fused launch's bounded wait ran out.
xy_status check_waits(xy_ctx* c, const char* where) {
  if (!c->d_wait) return XY_OK;
  unsigned int w = 0;
  XY_CUDA(c, cudaMemcpyAsync(&w, c->d_wait, sizeof(w), cudaMemcpyDeviceToHost, c->stream), where);
  XY_CUDA(c, cudaStreamSynchronize(c->stream), where);
  if (w) return fail(c, XY_ETIMEOUT,
                     "%s: a fused sweep's bounded wait (a neighbouring tile, or its staged rows) ran out",
                     where);
  return XY_OK;
}

cudaError_t timed_persistent(xy_ctx* c, const xyk::FusedPersistArgs& a) {
  if (c->timing_every <= 0)
    return xyk::launch_fused_persistent(c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  cudaEvent_t e0, e1;
  cudaError_t e = next_events(c, 0, &e0, &e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
  if (e == cudaSuccess)
    e = xyk::launch_fused_persistent(c->p.sincos_mode, c->p.reduce_mode, a, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
  return e;
}

void release(xy_ctx* c) {
  for (int k = 0; k < 2; ++k) {
    for (cudaEvent_t e : c->ev[k]) cudaEventDestroy(e);
    c->ev[k].clear();
    c->ev_used[k] = 0;
  }
  if (c->owns_theta && c->d_theta) cudaFree(c->d_theta);
  if (c->d_rec) cudaFree(c->d_rec);
  if (c->d_pong) cudaFree(c->d_pong);
  if (c->d_scratch) cudaFree(c->d_scratch);
  if (c->d_flag) cudaFree(c->d_flag);
  if (c->d_tiles) cudaFree(c->d_tiles);
  if (c->d_wait) cudaFree(c->d_wait);
  c->d_tiles = nullptr;
  c->d_wait = nullptr;
  c->d_theta = nullptr;
  c->d_rec = nullptr;
  c->d_pong = nullptr;
  c->d_scratch = nullptr;
  c->d_flag = nullptr;
}

}  // namespace

extern "C" {

int32_t xy_version(void) { return 101; }

int32_t xy_debug_build(void) {
#ifdef XY_DEBUG
  return 1;
#else
  return 0;
#endif
}

xy_status xy_debug_checks(uint32_t* failed) {
  if (!failed) {
    set_thread_msg("xy_debug_checks: NULL output");
    return XY_EINVAL;
  }
  const unsigned int a = xyk::debug_take_sweep(), b = xyk::debug_take_narrow();
  if (a == 0xffffffffu || b == 0xffffffffu) {
    (void)cudaGetLastError();
    set_thread_msg("xy_debug_checks: reading the device words failed");
    return XY_ECUDA;
  }
  *failed = (a & 0xffu) | ((b & 0xffu) << 8);
  return XY_OK;
}

const char* xy_last_error(const xy_ctx* ctx) {
  if (ctx && is_live(ctx) && ctx->magic == kMagicLive && ctx->sticky != XY_OK) return ctx->msg;
  return g_thread_msg;
}

xy_status xy_create(const xy_params* p, void* cuda_stream, void* d_angles, xy_ctx** out) {
  if (!out) {
    set_thread_msg("NULL output pointer");
    return XY_EINVAL;
  }
  *out = nullptr;
  xy_status st = validate(p);
  if (st != XY_OK) return st;
  if (d_angles && (reinterpret_cast<uintptr_t>(d_angles) & 15u)) {
    set_thread_msg("d_angles must be 16-byte aligned");
    return XY_EINVAL;
  }
  xy_ctx* c = new (std::nothrow) xy_ctx();   // value-initialised: pointers null, counts 0
  if (!c) {
    set_thread_msg("host allocation failed");
    return XY_ENOMEM;
  }
  c->magic = kMagicLive;
  c->p = *p;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  c->sticky = XY_OK;
  snprintf(c->msg, sizeof(c->msg), "no error");
  const size_t N = (size_t)p->L * (size_t)p->L;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) {
    if (d_angles) {
      c->d_theta = static_cast<float*>(d_angles);
      c->owns_theta = false;
    } else {
      e = xyk::dev_malloc(&c->d_theta, N * sizeof(float));
      c->owns_theta = true;
    }
  }
  if (e == cudaSuccess) e = xyk::dev_malloc(&c->d_flag, sizeof(unsigned int));
  c->persistent = p->algorithm == XY_ALGO_PERSISTENT ||
                  (p->algorithm == XY_ALGO_AUTO && xyk::fused_supported(p->L) &&
                   p->L <= kAutoPersistentMaxL);
  c->auto_persistent = c->persistent && p->algorithm == XY_ALGO_AUTO;
  c->fused = p->algorithm == XY_ALGO_FUSED || p->algorithm == XY_ALGO_FUSED2 ||
             c->persistent || (p->algorithm == XY_ALGO_AUTO && xyk::fused_supported(p->L));
  if (e == cudaSuccess && c->fused) {
    e = xyk::dev_malloc(&c->d_pong, N * sizeof(float));
    if (e == cudaSuccess) e = xyk::dev_malloc(&c->d_wait, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_wait, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess && !xyk::encode_fused_maps(&c->maps, c->d_theta, c->d_pong, p->L))
      e = cudaErrorNotSupported;
  }
  if (e == cudaSuccess && c->persistent)
    e = xyk::dev_malloc(&c->d_tiles, sizeof(unsigned int) * ((size_t)xyk::fused_tiles(p->L) + 1));
  if (e != cudaSuccess) {
    st = (e == cudaErrorMemoryAllocation) ? XY_ENOMEM : XY_ECUDA;
    set_thread_msg("xy_create: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
    release(c);
    c->magic = kMagicDead;
    delete c;
    return st;
  }
  e = xyk::launch_start(c->d_theta, p->L, xyd::make_round_keys(p->seed), p->lattice_id,
                        p->start == XY_START_HOT, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    set_thread_msg("xy_create: start kernel: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
    release(c);
    c->magic = kMagicDead;
    delete c;
    return XY_ECUDA;
  }
  c->next_sweep = 0;
  mark_live(c, true);
  *out = c;
  return XY_OK;
}

xy_status xy_reset(xy_ctx* c, uint64_t seed) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  c->p.seed = seed;
  XY_CUDA(c, xyk::launch_start(c->d_theta, c->p.L, xyd::make_round_keys(seed), c->p.lattice_id,
                               c->p.start == XY_START_HOT, c->stream),
          "xy_reset: start kernel");
  if (c->d_rec && c->rec_count > 0)
    XY_CUDA(c, cudaMemsetAsync(c->d_rec, 0, (size_t)c->rec_count * sizeof(xy_record), c->stream),
            "xy_reset: clear records");
  c->rec_count = 0;
  c->next_sweep = 0;
  return XY_OK;
}

xy_status xy_timing(xy_ctx* c, int every) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (every < 0) return fail(c, XY_EINVAL, "xy_timing: negative period");
  c->timing_every = every;
  c->ev_used[0] = c->ev_used[1] = 0;
  return XY_OK;
}

xy_status xy_kernel_time(xy_ctx* c, int kernel, double* total_ms, int64_t* launches) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (kernel < 0 || kernel > 1 || !total_ms || !launches)
    return fail(c, XY_EINVAL, "xy_kernel_time: bad arguments");
  XY_CUDA(c, cudaStreamSynchronize(c->stream), "xy_kernel_time: stream");
  st = check_waits(c, "xy_kernel_time");
  if (st != XY_OK) return st;
  double sum = 0.0;
  for (size_t i = 0; i + 1 < c->ev_used[kernel]; i += 2) {
    float ms = 0.f;
    XY_CUDA(c, cudaEventElapsedTime(&ms, c->ev[kernel][i], c->ev[kernel][i + 1]),
            "xy_kernel_time: elapsed");
    sum += ms;
  }
  *total_ms = sum;
  *launches = (int64_t)(c->ev_used[kernel] / 2);
  return XY_OK;
}

xy_status xy_reserve(xy_ctx* c, int64_t n_more) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (n_more < 0) return fail(c, XY_EINVAL, "xy_reserve: negative count");
  return grow_records(c, c->rec_count + n_more);
}

xy_status xy_sweep(xy_ctx* c, int64_t n) {
  const xyk::TraceRange trace("xy_sweep");
  xyk::NvtxRange range("xy_sweep");
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (n < 0) return fail(c, XY_EINVAL, "xy_sweep: negative sweep count");
  if (n == 0) return XY_OK;
  if (c->next_sweep + (uint64_t)n > 0xffffffffull)
    return fail(c, XY_EINVAL, "xy_sweep: sweep counter would pass 2^32 - 1");
  st = grow_records(c, c->rec_count + n);
  if (st != XY_OK) return st;
  const xyd::RoundKeys rk = xyd::make_round_keys(c->p.seed);
  if (c->persistent) {
    xyk::FusedPersistArgs a;
    a.buf[0] = c->d_theta;
    a.buf[1] = c->d_pong;
    a.L = c->p.L;
    a.W = c->p.L / 2;
    a.K = (float)(c->p.beta * c->p.J);
    a.delta = (float)c->p.delta;
    a.rk = rk;
    a.lattice_id = c->p.lattice_id;
    a.beta = c->p.beta;
    a.flags = c->d_tiles;
    a.counter = c->d_tiles + xyk::fused_tiles(c->p.L);
    a.maps = &c->maps;
    a.error = c->d_wait;
    a.spin_limit = xyk::fused_persistent_spin_limit();
    a.skip_items = 0;
    a.minb = c->p.ctas_per_sm ? c->p.ctas_per_sm : 3;
    // one launch per at most fused_persistent_max_sweeps sweeps (the kernel's
    // work items are counted in 32 bits)
    const int64_t chunk = xyk::fused_persistent_max_sweeps(c->p.L);
    for (int64_t done = 0; done < n;) {
      const int64_t m = std::min<int64_t>(n - done, chunk);
      a.sweep0 = (uint32_t)(c->next_sweep + (uint64_t)done);
      a.n_sweeps = (int)m;
      a.rec = c->d_rec + c->rec_count + done;
      cudaError_t e = timed_persistent(c, a);
      if (e == cudaErrorCooperativeLaunchTooLarge && c->auto_persistent) {
        // the grid does not fit beside other work on the device: the same
        // sweeps as one fused launch each (bit-identical)
        (void)cudaGetLastError();
        xyk::FusedArgs f;
        f.L = a.L;
        f.W = a.W;
        f.K = a.K;
        f.delta = a.delta;
        f.rk = a.rk;
        f.lattice_id = a.lattice_id;
        f.beta = a.beta;
        f.minb = a.minb;
        f.maps = &c->maps;
        f.error = c->d_wait;
        for (int64_t i = 0; i < m; ++i) {
          f.src = a.buf[i & 1];
          f.dst = a.buf[(i + 1) & 1];
          f.sweep = a.sweep0 + (uint32_t)i;
          f.rec = a.rec + i;
          e = timed_fused(c, f);
          if (e != cudaSuccess) break;
        }
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "xy_sweep: persistent launch");
      if (m & 1) std::swap(a.buf[0], a.buf[1]);
      done += m;
    }
    if (a.buf[0] != c->d_theta) {
      const size_t N = (size_t)c->p.L * (size_t)c->p.L;
      XY_CUDA(c, cudaMemcpyAsync(c->d_theta, a.buf[0], N * sizeof(float),
                                 cudaMemcpyDeviceToDevice, c->stream),
              "xy_sweep: copy back");
    }
  } else if (c->fused) {
    xyk::FusedArgs a;
    a.L = c->p.L;
    a.W = c->p.L / 2;
    a.K = (float)(c->p.beta * c->p.J);
    a.delta = (float)c->p.delta;
    a.rk = rk;
    a.lattice_id = c->p.lattice_id;
    a.beta = c->p.beta;
    // default plan of one launch per sweep: 4 CTAs per SM, the faster plan at
    // L = 8192 and 16384 for every precision mode (at 16384, against 3:
    // accurate 217.8 / 213.3, SFU 295.0 / 283.4, libm 185.9 / 171.4,
    // compensated sums 187.6 / 186.9 G updates/s)
    a.minb = c->p.ctas_per_sm ? c->p.ctas_per_sm : 4;
    a.maps = &c->maps;
    a.error = c->d_wait;
    float* cur = c->d_theta;
    float* nxt = c->d_pong;
    const bool two = c->p.algorithm == XY_ALGO_FUSED2;
    for (int64_t i = 0; i < n;) {
      a.src = cur;
      a.dst = nxt;
      a.sweep = (uint32_t)(c->next_sweep + (uint64_t)i);
      a.rec = c->d_rec + c->rec_count + i;
      // two sweeps per launch where two are left (XY_ALGO_FUSED2)
      const int step = (two && i + 1 < n) ? 2 : 1;
      cudaError_t e = step == 2 ? timed_fused2(c, a) : timed_fused(c, a);
      if (e != cudaSuccess) return cuda_fail(c, e, "xy_sweep: fused launch");
      float* t = cur;
      cur = nxt;
      nxt = t;
      i += step;
    }
    if (cur != c->d_theta) {
      const size_t N = (size_t)c->p.L * (size_t)c->p.L;
      XY_CUDA(c, cudaMemcpyAsync(c->d_theta, cur, N * sizeof(float), cudaMemcpyDeviceToDevice,
                                 c->stream),
              "xy_sweep: copy back");
    }
  } else {
    xyk::HalfSweepArgs a;
    a.theta = c->d_theta;
    a.L = c->p.L;
    a.W = c->p.L / 2;
    a.K = (float)(c->p.beta * c->p.J);
    a.delta = (float)c->p.delta;
    a.rk = rk;
    a.lattice_id = c->p.lattice_id;
    a.beta = c->p.beta;
    for (int64_t i = 0; i < n; ++i) {
      a.sweep = (uint32_t)(c->next_sweep + (uint64_t)i);
      a.rec = c->d_rec + c->rec_count + i;
      cudaError_t e = timed_half_sweep(c, 0, a);
      if (e == cudaSuccess) e = timed_half_sweep(c, 1, a);
      if (e != cudaSuccess) return cuda_fail(c, e, "xy_sweep: launch");
    }
  }
  c->next_sweep += (uint64_t)n;
  c->rec_count += n;
  return XY_OK;
}

xy_status xy_measure(xy_ctx* c, int64_t first, int64_t count, xy_obs* out) {
  const xyk::TraceRange trace("xy_measure");
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (first < 0 || count < 0 || first + count > c->rec_count)
    return fail(c, XY_EINVAL, "xy_measure: range [%lld, %lld) outside [0, %lld)",
                (long long)first, (long long)(first + count), (long long)c->rec_count);
  if (count > 0 && !out) return fail(c, XY_EINVAL, "xy_measure: NULL output");
  XY_CUDA(c, cudaStreamSynchronize(c->stream), "xy_measure: stream");
  st = check_waits(c, "xy_measure");
  if (st != XY_OK) return st;
  if (count == 0) return XY_OK;
  xy_record* h = new (std::nothrow) xy_record[count];
  if (!h) return fail(c, XY_ENOMEM, "xy_measure: host allocation");
  cudaError_t e = cudaMemcpy(h, c->d_rec + first, (size_t)count * sizeof(xy_record),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete[] h;
    return cuda_fail(c, e, "xy_measure: copy");
  }
  const double N = (double)c->p.L * (double)c->p.L, J = c->p.J;
  const double unit = ldexp(1.0, -XY_FX_SHIFT);
  bool bad = false;
  for (int64_t i = 0; i < count; ++i) {
    const xy_record& r = h[i];
    xy_obs& o = out[i];
    o.C = (double)r.sum[0] * unit;
    o.Ix = (double)r.sum[1] * unit;
    o.Iy = (double)r.sum[2] * unit;
    o.Mx = (double)r.sum[3] * unit;
    o.My = (double)r.sum[4] * unit;
    o.accepted = r.accepted;
    o.beta = r.beta;
    o.e = -J * o.C / N;
    o.abs_m = sqrt(o.Mx * o.Mx + o.My * o.My) / N;
    o.upsilon = (J * o.C - r.beta * J * J * (o.Ix * o.Ix + o.Iy * o.Iy)) / (2.0 * N);
    if (r.flags & 1ull) bad = true;
  }
  delete[] h;
  if (bad) return fail(c, XY_ENUMERIC, "xy_measure: a record saw a non-finite sum");
  return XY_OK;
}

xy_status xy_records_device(xy_ctx* c, const xy_record** d_records, int64_t* count) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (!d_records || !count) return fail(c, XY_EINVAL, "xy_records_device: NULL output");
  *d_records = c->d_rec;
  *count = c->rec_count;
  return XY_OK;
}

xy_status xy_info(const xy_ctx* c, int64_t* n_records, uint64_t* next_sweep) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (n_records) *n_records = c->rec_count;
  if (next_sweep) *next_sweep = c->next_sweep;
  return XY_OK;
}

xy_status xy_algorithm(const xy_ctx* c, int32_t* algorithm) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (!algorithm) {
    set_thread_msg("xy_algorithm: NULL output");
    return XY_EINVAL;
  }
  *algorithm = c->persistent ? XY_ALGO_PERSISTENT
                : c->p.algorithm == XY_ALGO_FUSED2 ? XY_ALGO_FUSED2
                : (c->fused ? XY_ALGO_FUSED : XY_ALGO_TWO_PASS);
  return XY_OK;
}

xy_status xy_selftest_persistent_wait(void* cuda_stream, int64_t polls) {
  if (polls < 1 || polls > (1 << 24)) {
    set_thread_msg("xy_selftest_persistent_wait: polls must be in [1, 2^24]");
    return XY_EINVAL;
  }
  // L = 128 (four tiles), two sweeps of which the first is never handed out:
  // every tile of the second waits for counters that nothing sets
  const int L = 128;
  const size_t N = (size_t)L * L;
  const int tiles = xyk::fused_tiles(L);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  float* buf = nullptr;
  unsigned int* words = nullptr;      // tile counters, work counter, error word
  xy_record* rec = nullptr;
  unsigned int err = 0;
  cudaError_t e = xyk::dev_malloc(&buf, 2 * N * sizeof(float));
  if (e == cudaSuccess) e = xyk::dev_malloc(&words, sizeof(unsigned int) * (size_t)(tiles + 2));
  if (e == cudaSuccess) e = xyk::dev_malloc(&rec, 2 * sizeof(xy_record));
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 2 * N * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, sizeof(unsigned int) * (size_t)(tiles + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(rec, 0, 2 * sizeof(xy_record), s);
  if (e == cudaSuccess) {
    xyk::FusedPersistArgs a;
    a.buf[0] = buf;
    a.buf[1] = buf + N;
    a.L = L;
    a.W = L / 2;
    a.K = 1.f;
    a.delta = (float)M_PI;
    a.rk = xyd::make_round_keys(1);
    a.lattice_id = 0;
    a.sweep0 = 0;
    a.n_sweeps = 2;
    a.rec = rec;
    a.beta = 1.0;
    a.flags = words;
    a.counter = words + tiles;
    a.error = words + tiles + 1;
    a.spin_limit = (long long)polls;
    a.skip_items = tiles;
    xyk::FusedMaps maps;
    a.maps = &maps;
    if (!xyk::encode_fused_maps(&maps, a.buf[0], a.buf[1], L)) e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = xyk::launch_fused_persistent(XY_SINCOS_ACCURATE, XY_REDUCE_EXACT, a, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&err, a.error, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (buf) cudaFree(buf);
  if (words) cudaFree(words);
  if (rec) cudaFree(rec);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_thread_msg("xy_selftest_persistent_wait: %s", cudaGetErrorString(e));
    return XY_ECUDA;
  }
  if (err) {
    set_thread_msg("xy_selftest_persistent_wait: the waits ran out after %lld polls",
                   (long long)polls);
    return XY_ETIMEOUT;
  }
  set_thread_msg("xy_selftest_persistent_wait: the waits completed, which they cannot");
  return XY_OK;
}

xy_status xy_get_state(xy_ctx* c, float* host, uint64_t* next_sweep) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (!host) return fail(c, XY_EINVAL, "xy_get_state: NULL output");
  const size_t N = (size_t)c->p.L * (size_t)c->p.L;
  if (!c->d_scratch) XY_CUDA(c, xyk::dev_malloc(&c->d_scratch, N * sizeof(float)), "xy_get_state: scratch");
  XY_CUDA(c, xyk::launch_split_to_natural(c->d_theta, c->d_scratch, c->p.L, c->stream),
          "xy_get_state: layout kernel");
  XY_CUDA(c, cudaMemcpyAsync(host, c->d_scratch, N * sizeof(float), cudaMemcpyDeviceToHost,
                             c->stream),
          "xy_get_state: copy");
  XY_CUDA(c, cudaStreamSynchronize(c->stream), "xy_get_state: stream");
  st = check_waits(c, "xy_get_state");
  if (st != XY_OK) return st;
  if (next_sweep) *next_sweep = c->next_sweep;
  return XY_OK;
}

xy_status xy_set_state(xy_ctx* c, const float* host, uint64_t next_sweep) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (!host) return fail(c, XY_EINVAL, "xy_set_state: NULL input");
  if (next_sweep > 0xffffffffull) return fail(c, XY_EINVAL, "xy_set_state: sweep >= 2^32");
  const size_t N = (size_t)c->p.L * (size_t)c->p.L;
  if (!c->d_scratch) XY_CUDA(c, xyk::dev_malloc(&c->d_scratch, N * sizeof(float)), "xy_set_state: scratch");
  XY_CUDA(c, cudaMemcpyAsync(c->d_scratch, host, N * sizeof(float), cudaMemcpyHostToDevice,
                             c->stream),
          "xy_set_state: copy");
  XY_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned int), c->stream), "xy_set_state: flag");
  XY_CUDA(c, xyk::launch_check_finite(c->d_scratch, (int64_t)N, c->d_flag, c->stream),
          "xy_set_state: check kernel");
  unsigned int flag = 0;
  XY_CUDA(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, c->stream),
          "xy_set_state: flag copy");
  XY_CUDA(c, cudaStreamSynchronize(c->stream), "xy_set_state: stream");
  if (flag) {
    set_thread_msg("xy_set_state: non-finite angle rejected; state unchanged");
    return XY_EINVAL;   // not sticky: the context is untouched
  }
  XY_CUDA(c, xyk::launch_natural_to_split(c->d_scratch, c->d_theta, c->p.L, c->stream),
          "xy_set_state: layout kernel");
  XY_CUDA(c, cudaStreamSynchronize(c->stream), "xy_set_state: stream");
  c->next_sweep = next_sweep;
  c->rec_count = 0;
  if (c->d_rec && c->rec_cap > 0)
    XY_CUDA(c, cudaMemsetAsync(c->d_rec, 0, (size_t)c->rec_cap * sizeof(xy_record), c->stream),
            "xy_set_state: clear records");
  return XY_OK;
}

xy_status xy_set_beta(xy_ctx* c, double beta) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  if (!(beta >= 0.0) || !isfinite(beta)) {
    set_thread_msg("xy_set_beta: beta must be finite and >= 0");
    return XY_EINVAL;
  }
  c->p.beta = beta;
  return XY_OK;
}

xy_status xy_synchronize(xy_ctx* c) {
  xy_status st = check_ctx(c);
  if (st != XY_OK) return st;
  XY_CUDA(c, cudaStreamSynchronize(c->stream), "xy_synchronize");
  st = check_waits(c, "xy_synchronize");
  if (st != XY_OK) return st;
  return XY_OK;
}

xy_status xy_destroy(xy_ctx* c) {
  if (!c) return XY_OK;
  if (!is_live(c) || c->magic != kMagicLive) {
    set_thread_msg("xy_destroy: context is not live (double destroy?)");
    return XY_ESTATE;
  }
  mark_live(c, false);
  cudaStreamSynchronize(c->stream);
  release(c);
  c->magic = kMagicDead;
  delete c;
  return XY_OK;
}

xy_status xy_eval_unit_vector(int32_t sincos_mode, const float* d_theta, float* d_cos,
                              float* d_sin, int64_t n, void* cuda_stream) {
  if (n < 0 || (n > 0 && (!d_theta || !d_cos || !d_sin)) || sincos_mode < 0 || sincos_mode > 2) {
    set_thread_msg("xy_eval_unit_vector: bad arguments");
    return XY_EINVAL;
  }
  cudaError_t e = xyk::launch_eval_unit_vector(sincos_mode, d_theta, d_cos, d_sin, n,
                                               reinterpret_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    set_thread_msg("xy_eval_unit_vector: %s", cudaGetErrorString(e));
    return XY_ECUDA;
  }
  return XY_OK;
}

xy_status xy_philox_words(uint64_t seed, uint32_t sweep, uint32_t lattice_id, uint32_t domain,
                          uint32_t first, int64_t n, uint32_t* d_out, void* cuda_stream) {
  if (n < 0 || (n > 0 && !d_out)) {
    set_thread_msg("xy_philox_words: bad arguments");
    return XY_EINVAL;
  }
  cudaError_t e = xyk::launch_philox_words(xyd::make_round_keys(seed), sweep, lattice_id, domain,
                                           first, n, d_out,
                                           reinterpret_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    set_thread_msg("xy_philox_words: %s", cudaGetErrorString(e));
    return XY_ECUDA;
  }
  return XY_OK;
}

}  // extern "C"
