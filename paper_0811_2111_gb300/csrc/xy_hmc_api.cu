// xy_hmc_api.cu -- the C ABI declared in include/xy_hmc.h: validation,
// ownership, sticky errors, record growth and the per-trajectory CUDA graph
// around the kernels of xy_hmc.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "xy_hmc.h"
#include "xy_internal.h"
#include "xy_trace.h"

namespace {

constexpr uint32_t kMagicLive = 0x484D434Cu;   // "HMCL"
constexpr uint32_t kMagicDead = 0xDEADBEEFu;

thread_local char g_msg[512] = "no error";

std::mutex g_mu;
std::unordered_set<const void*>& live() {
  static std::unordered_set<const void*> s;
  return s;
}
bool is_live(const void* h) {
  std::lock_guard<std::mutex> g(g_mu);
  return live().count(h) != 0;
}
void mark(const void* h, bool on) {
  std::lock_guard<std::mutex> g(g_mu);
  if (on) {
    live().insert(h);
  } else {
    live().erase(h);
  }
}

void tmsg(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}

}  // namespace

struct xy_hmc {
  CUtensorMap maps[5];               // TMA maps (32 x 128 boxes): angle buffers 0..2, d_p, d_p2
  bool use_tma;
  bool use_persist;                  // a trajectory's steps in one cooperative TMA launch
  unsigned int* d_tiles;             // its per-tile step counters
  bool use_cluster;                  // whole trajectories in one cluster launch
  bool use_pairs;                    // full steps two per launch (k_hmc_tile2)
  int tma_rows;                      // tile (and box) rows of the TMA step kernel: 32 or 16
  int tma_ctas;                      // persistent grid of the TMA step kernel
  uint32_t magic;
  xy_hmc_params p;
  cudaStream_t stream;
  cudaStream_t capture_stream;   // private stream the trajectory graph is captured on
  int device;
  float* th[3];                  // angle buffers (th[0] may be caller-owned)
  bool owns_th0;
  float* d_p;                    // momenta (between calls)
  float* d_p2;                   // second momentum buffer of the two-step kernel
  xyk::HmcCtl* d_ctl;
  xy_hmc_record* d_rec;
  int64_t rec_cap;
  int64_t rec_count;
  uint64_t next_traj;
  cudaGraphExec_t graph;         // one trajectory; rebuilt when a parameter changes
  xy_status sticky;
  char msg[512];
};

namespace {

xy_status fail(xy_hmc* h, xy_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  snprintf(g_msg, sizeof(g_msg), "%s", buf);
  if (h && is_live(h) && h->magic == kMagicLive && h->sticky == XY_OK) {
    h->sticky = st;
    snprintf(h->msg, sizeof(h->msg), "%s", buf);
  }
  return st;
}

xy_status cuda_fail(xy_hmc* h, cudaError_t e, const char* what) {
  (void)cudaGetLastError();   // leave no non-sticky error for a later launch check
  return fail(h, e == cudaErrorMemoryAllocation ? XY_ENOMEM : XY_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorName(e), cudaGetErrorString(e));
}

#define H_CUDA(h, call, what)                               \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what);   \
  } while (0)

xy_status check(const xy_hmc* h) {
  if (!h) {
    tmsg("NULL HMC context");
    return XY_EINVAL;
  }
  if (!is_live(h) || h->magic != kMagicLive) {
    tmsg("HMC context is not live (destroyed or never created)");
    return XY_ESTATE;
  }
  if (h->sticky != XY_OK) {
    tmsg("HMC context is in an earlier error: %s", h->msg);
    return h->sticky;
  }
  return XY_OK;
}

}  // namespace

namespace xyk {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    (void)cudaGetLastError();
  });
  return fn;
}

}  // namespace xyk

namespace {

// Tensor map of one L x L float buffer, boxes of box_rows rows x 128 columns.
bool encode_map(CUtensorMap* m, float* base, int L, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = xyk::tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)L, (cuuint64_t)L};
  const cuuint64_t strides[1] = {(cuuint64_t)L * sizeof(float)};
  const cuuint32_t box[2] = {128u, (cuuint32_t)box_rows};
  const cuuint32_t elem[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, elem,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool step_ok(double eps, int32_t n_md) { return eps > 0.0 && isfinite(eps) && n_md >= 1 && n_md <= 1000000; }

xy_status validate(const xy_hmc_params* p) {
  if (!p) {
    tmsg("NULL params");
    return XY_EINVAL;
  }
  if (p->L < 2 || p->L > XY_MAX_L) {
    tmsg("L must be in [2, %d]; got %d", XY_MAX_L, p->L);
    return XY_EINVAL;
  }
  if (!(p->beta >= 0.0) || !isfinite(p->beta) || !isfinite(p->J)) {
    tmsg("beta must be finite and >= 0 and J finite");
    return XY_EINVAL;
  }
  if (!step_ok(p->eps, p->n_md)) {
    tmsg("eps must be finite and > 0 and n_md in [1, 1000000]");
    return XY_EINVAL;
  }
  if (p->start != XY_START_HOT && p->start != XY_START_COLD) {
    tmsg("start must be XY_START_HOT or XY_START_COLD");
    return XY_EINVAL;
  }
  if (p->sincos_mode < 0 || p->sincos_mode > 2) {
    tmsg("bad sincos_mode");
    return XY_EINVAL;
  }
  if (p->kernel != XY_HMC_KERNEL_AUTO && p->kernel != XY_HMC_KERNEL_TILED &&
      p->kernel != XY_HMC_KERNEL_SITE && p->kernel != XY_HMC_KERNEL_TILED2 &&
      p->kernel != XY_HMC_KERNEL_TILED_TMA && p->kernel != XY_HMC_KERNEL_CLUSTER &&
      p->kernel != XY_HMC_KERNEL_PERSISTENT) {
    tmsg("bad kernel choice");
    return XY_EINVAL;
  }
  if (p->kernel == XY_HMC_KERNEL_CLUSTER && !xyk::hmc_cluster_ok(p->L)) {
    tmsg("the cluster kernel needs L to be a power of two in [16, 256]; got %d", p->L);
    return XY_EINVAL;
  }
  if ((p->kernel == XY_HMC_KERNEL_TILED || p->kernel == XY_HMC_KERNEL_TILED2 ||
       p->kernel == XY_HMC_KERNEL_TILED_TMA || p->kernel == XY_HMC_KERNEL_PERSISTENT) &&
      !xyk::hmc_tiled_ok(p->L)) {
    tmsg("the tiled kernel needs L to be a multiple of 128; got %d", p->L);
    return XY_EINVAL;
  }
  return XY_OK;
}

xyk::HmcArgs args_of(const xy_hmc* h) {
  xyk::HmcArgs a;
  for (int i = 0; i < 3; ++i) a.th[i] = h->th[i];
  a.p_in = h->d_p;
  a.p_out = h->d_p;
  a.ctl = h->d_ctl;
  a.L = h->p.L;
  a.K = (float)(h->p.beta * h->p.J);
  a.eps = (float)h->p.eps;
  a.a = 0.5f * a.eps;
  a.src_off = 0;
  a.dst_off = 0;
  a.rk = xyd::make_round_keys(h->p.seed);
  a.lattice_id = h->p.lattice_id;
  a.tiled = h->p.kernel == XY_HMC_KERNEL_TILED || h->p.kernel == XY_HMC_KERNEL_TILED2 ||
            h->p.kernel == XY_HMC_KERNEL_TILED_TMA || h->p.kernel == XY_HMC_KERNEL_PERSISTENT ||
            (h->p.kernel == XY_HMC_KERNEL_AUTO && xyk::hmc_tiled_ok(h->p.L));
  a.pairs = h->use_pairs ? 1 : 0;
  return a;
}

// Leap-frog of n steps from the state buffer (begin kind `begin`), then the
// test (mode 0) or the commit of an integration (mode 1).  Angle buffers:
// offset 0 (the state) -> 1, then 1 <-> 2 per launch; with two steps per
// launch the momenta ping-pong between d_p and d_p2, and the final half kick
// always leaves them in d_p.
cudaError_t enqueue_trajectory(const xy_hmc* h, int begin, int n, int mode, cudaStream_t s) {
  xyk::HmcArgs a = args_of(h);
  const int m = h->p.sincos_mode;
  if (h->use_cluster)
    return xyk::launch_hmc_cluster(m, a, n, begin == xyk::kHmcBeginDraw ? 1 : 0, mode, h->p.beta,
                                   h->p.J, s);
  float* pcur = h->d_p;
  float* pother = h->d_p2;
  a.a = 0.5f * a.eps;
  a.src_off = 0;
  a.dst_off = 1;
  cudaError_t e = xyk::launch_hmc(begin, m, a, s);
  int off = 1;
  a.a = a.eps;
  int left = n - 1;
  while (e == cudaSuccess && left > 0) {
    a.src_off = off;
    a.dst_off = 3 - off;
    if (a.pairs && left >= 2) {
      a.p_in = pcur;
      a.p_out = pother;
      // the tile-walking form reads its rows by TMA: the angle buffers' maps
      // and that of the momenta it reads
      e = h->use_tma ? xyk::launch_hmc_step2(m, a, h->maps, pcur == h->d_p ? &h->maps[3] : &h->maps[4], s)
                     : xyk::launch_hmc(xyk::kHmcStep2, m, a, s);
      float* t = pcur;
      pcur = pother;
      pother = t;
      left -= 2;
    } else if (h->use_persist) {
      // every remaining step in one launch; step j reads offset 1 + (j & 1)
      a.p_in = pcur;
      a.p_out = pcur;
      xyk::HmcStepsArgs q;
      q.a = a;
      q.n_steps = left;
      q.flags = h->d_tiles;
      q.spin_limit = xyk::hmc_persist_spin_limit();
      e = xyk::launch_hmc_steps_persist(m, q, h->maps, s);
      if (left & 1) off = 3 - off;
      left = 0;
      continue;
    } else {
      a.p_in = pcur;
      a.p_out = pcur;
      // the TMA kernel's momentum tensor map is of d_p: after an odd number
      // of two-step launches the momenta live in d_p2, and the plain tiled
      // step takes the remaining single step
      e = h->use_tma && pcur == h->d_p
              ? xyk::launch_hmc_step_tma(m, a, h->maps, h->tma_rows, h->tma_ctas, s)
              : xyk::launch_hmc(xyk::kHmcStep, m, a, s);
      left -= 1;
    }
    off = 3 - off;
  }
  if (e != cudaSuccess) return e;
  a.a = 0.5f * a.eps;
  a.src_off = off;
  a.dst_off = off;
  a.p_in = pcur;
  a.p_out = h->d_p;
  e = xyk::launch_hmc(xyk::kHmcFinal, m, a, s);
  if (e != cudaSuccess) return e;
  return xyk::launch_hmc_accept(mode, a, h->p.beta, h->p.J, s);
}

cudaError_t capture(xy_hmc* h) {
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = xyk::hmc_prepare(h->p.sincos_mode);   // function attributes: not capturable
  if (e == cudaSuccess && h->use_cluster) e = xyk::hmc_cluster_prepare(h->p.sincos_mode);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = enqueue_trajectory(h, xyk::kHmcBeginDraw, h->p.n_md, 0, h->capture_stream);
  e = cudaStreamEndCapture(h->capture_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  return e;
}

xy_status grow_records(xy_hmc* h, int64_t need) {
  if (need <= h->rec_cap) return XY_OK;
  int64_t cap = h->rec_cap > 0 ? h->rec_cap : 256;
  while (cap < need) cap *= 2;
  xy_hmc_record* nr = nullptr;
  H_CUDA(h, xyk::dev_malloc(&nr, (size_t)cap * sizeof(xy_hmc_record)), "record buffer");
  if (h->rec_count > 0) {
    cudaError_t e = cudaMemcpyAsync(nr, h->d_rec, (size_t)h->rec_count * sizeof(xy_hmc_record),
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) {
      cudaFree(nr);
      return cuda_fail(h, e, "record copy");
    }
  }
  xy_hmc_record* ptr = nr;
  cudaError_t e = cudaMemcpyAsync(&h->d_ctl->records, &ptr, sizeof(ptr), cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaFree(nr);
    return cuda_fail(h, e, "record pointer update");
  }
  if (h->d_rec) cudaFree(h->d_rec);
  h->d_rec = nr;
  h->rec_cap = cap;
  return XY_OK;
}

void release(xy_hmc* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (int i = 0; i < 3; ++i)
    if (h->th[i] && (i > 0 || h->owns_th0)) cudaFree(h->th[i]);
  if (h->d_p) cudaFree(h->d_p);
  if (h->d_p2) cudaFree(h->d_p2);
  if (h->d_ctl) cudaFree(h->d_ctl);
  if (h->d_rec) cudaFree(h->d_rec);
  if (h->d_tiles) cudaFree(h->d_tiles);
}

xy_status sync(xy_hmc* h, const char* what) {
  H_CUDA(h, cudaStreamSynchronize(h->stream), what);
  if (h->use_tma) {
    uint32_t err = 0;
    H_CUDA(h, cudaMemcpy(&err, &h->d_ctl->error, sizeof(err), cudaMemcpyDeviceToHost), what);
    if (err) return fail(h, XY_ETIMEOUT, "%s: a kernel's bounded wait for its data ran out", what);
  }
  return XY_OK;
}

}  // namespace

extern "C" {

xy_status xy_hmc_create(const xy_hmc_params* p, void* cuda_stream, void* d_angles,
                        xy_hmc** out) {
  if (!out) {
    tmsg("NULL output pointer");
    return XY_EINVAL;
  }
  *out = nullptr;
  xy_status st = validate(p);
  if (st != XY_OK) return st;
  if (d_angles && (reinterpret_cast<uintptr_t>(d_angles) & 15u)) {
    tmsg("d_angles must be 16-byte aligned");
    return XY_EINVAL;
  }
  xy_hmc* h = new (std::nothrow) xy_hmc();
  if (!h) {
    tmsg("host allocation");
    return XY_ENOMEM;
  }
  h->p = *p;
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->owns_th0 = d_angles == nullptr;
  const size_t N = (size_t)p->L * (size_t)p->L;
  const char* step = "device";
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) {
    step = "capture stream";
    e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) {
    step = "angle buffers";
    h->th[0] = static_cast<float*>(d_angles);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
      if (!h->th[i]) e = xyk::dev_malloc(&h->th[i], N * sizeof(float));
  }
  if (e == cudaSuccess) {
    step = "momentum buffers";
    e = xyk::dev_malloc(&h->d_p, N * sizeof(float));
    if (e == cudaSuccess) e = xyk::dev_malloc(&h->d_p2, N * sizeof(float));
  }
  if (e == cudaSuccess) {
    step = "control block";
    e = xyk::dev_malloc(&h->d_ctl, sizeof(xyk::HmcCtl));
  }
  // AUTO: the cluster kernel where it measured faster than the others (L =
  // 128, 256); below that the per-launch cost of any kernel dominates
  h->use_cluster = p->kernel == XY_HMC_KERNEL_CLUSTER ||
                   (p->kernel == XY_HMC_KERNEL_AUTO && (p->L == 128 || p->L == 256));
  // AUTO: full steps two per launch wherever the tiled kernels run (measured
  // faster than one TMA-fed step per launch at L = 512 ... 4096); the odd
  // step of a trajectory runs on the TMA kernel
  h->use_pairs = p->kernel == XY_HMC_KERNEL_TILED2 ||
                 (p->kernel == XY_HMC_KERNEL_AUTO && !h->use_cluster && xyk::hmc_tiled_ok(p->L));
  const bool want_tma = p->kernel == XY_HMC_KERNEL_TILED_TMA || p->kernel == XY_HMC_KERNEL_PERSISTENT ||
                        p->kernel == XY_HMC_KERNEL_TILED2 ||
                        (p->kernel == XY_HMC_KERNEL_AUTO && !h->use_cluster &&
                         xyk::hmc_tiled_ok(p->L));
  if (e == cudaSuccess && want_tma) {
    step = "tensor maps";
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
    bool ok = e == cudaSuccess;
    h->tma_rows = 32;   // 32 x 128 tiles measured faster than 16 x 128 (54.1 vs 57.4 us per step)
    for (int i = 0; i < 3 && ok; ++i) ok = encode_map(&h->maps[i], h->th[i], p->L, h->tma_rows);
    if (ok) ok = encode_map(&h->maps[3], h->d_p, p->L, h->tma_rows);
    if (ok) ok = encode_map(&h->maps[4], h->d_p2, p->L, h->tma_rows);
    // AUTO falls back to the plain tiled kernel without the encoder
    if (e == cudaSuccess && !ok && p->kernel == XY_HMC_KERNEL_TILED_TMA) e = cudaErrorNotSupported;
    h->use_tma = ok;
    h->tma_ctas = 2 * (n_sm > 0 ? n_sm : 1);
  }
  // the trajectory-long persistent launch of the TMA step (needs the encoder)
  const bool want_persist = p->kernel == XY_HMC_KERNEL_PERSISTENT;
  if (e == cudaSuccess && want_persist) {
    step = "persistent step counters";
    if (!h->use_tma) {
      e = cudaErrorNotSupported;
    } else {
      e = xyk::dev_malloc(&h->d_tiles, sizeof(unsigned int) * (size_t)xyk::hmc_persist_tiles(p->L));
      h->use_persist = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_ctl, 0, sizeof(xyk::HmcCtl), h->stream);
  if (e == cudaSuccess) {
    step = "start kernel";
    e = xyk::launch_hmc_start(args_of(h), p->start == XY_START_HOT ? 1 : 0, h->stream);
  }
  if (e == cudaSuccess) {
    step = "synchronize";
    e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    tmsg("xy_hmc_create: %s: %s (%s)", step, cudaGetErrorName(e), cudaGetErrorString(e));
    release(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? XY_ENOMEM : XY_ECUDA;
  }
  h->magic = kMagicLive;
  h->sticky = XY_OK;
  snprintf(h->msg, sizeof(h->msg), "no error");
  mark(h, true);
  *out = h;
  return XY_OK;
}

xy_status xy_hmc_run(xy_hmc* h, int64_t n_traj) {
  const xyk::TraceRange trace("xy_hmc_run");
  xyk::NvtxRange range("xy_hmc_run");
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (n_traj < 0) return fail(h, XY_EINVAL, "xy_hmc_run: negative trajectory count");
  if (n_traj == 0) return XY_OK;
  if (h->next_traj + (uint64_t)n_traj > 0xffffffffull)
    return fail(h, XY_EINVAL, "xy_hmc_run: trajectory counter would pass 2^32 - 1");
  st = grow_records(h, h->rec_count + n_traj);
  if (st != XY_OK) return st;
  if (h->use_persist) {
    // a trajectory is five launches here (begin, the counters' memset, the
    // steps, final, accept): launched directly, no graph
    H_CUDA(h, xyk::hmc_prepare(h->p.sincos_mode), "xy_hmc_run: kernel attributes");
    for (int64_t i = 0; i < n_traj; ++i)
      H_CUDA(h, enqueue_trajectory(h, xyk::kHmcBeginDraw, h->p.n_md, 0, h->stream),
             "xy_hmc_run: launch");
  } else {
    if (!h->graph) H_CUDA(h, capture(h), "xy_hmc_run: graph capture");
    for (int64_t i = 0; i < n_traj; ++i)
      H_CUDA(h, cudaGraphLaunch(h->graph, h->stream), "xy_hmc_run: graph launch");
  }
  H_CUDA(h, xyk::launch_hmc_canonical(args_of(h), h->stream),
         "xy_hmc_run: state copy");
  h->rec_count += n_traj;
  h->next_traj += (uint64_t)n_traj;
  return XY_OK;
}

xy_status xy_hmc_integrate(xy_hmc* h, int32_t n_steps) {
  const xyk::TraceRange trace("xy_hmc_integrate");
  xyk::NvtxRange range("xy_hmc_integrate");
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (n_steps < 1 || n_steps > 1000000)
    return fail(h, XY_EINVAL, "xy_hmc_integrate: n_steps must be in [1, 1000000]");
  H_CUDA(h, xyk::hmc_prepare(h->p.sincos_mode), "xy_hmc_integrate: kernel attributes");
  if (h->use_cluster)
    H_CUDA(h, xyk::hmc_cluster_prepare(h->p.sincos_mode), "xy_hmc_integrate: kernel attributes");
  H_CUDA(h, enqueue_trajectory(h, xyk::kHmcBeginRead, n_steps, 1, h->stream),
         "xy_hmc_integrate: launch");
  H_CUDA(h, xyk::launch_hmc_canonical(args_of(h), h->stream),
         "xy_hmc_integrate: state copy");
  return XY_OK;
}

xy_status xy_hmc_refresh(xy_hmc* h) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  H_CUDA(h, xyk::launch_hmc_draw(args_of(h), h->stream), "xy_hmc_refresh");
  return XY_OK;
}

xy_status xy_hmc_last_sums(xy_hmc* h, double out[12]) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (!out) return fail(h, XY_EINVAL, "xy_hmc_last_sums: NULL output");
  unsigned long long last[2][xyk::kHmcSums];
  H_CUDA(h, cudaMemcpyAsync(last, h->d_ctl->last, sizeof(last), cudaMemcpyDeviceToHost, h->stream),
         "xy_hmc_last_sums: copy");
  st = sync(h, "xy_hmc_last_sums: stream");
  if (st != XY_OK) return st;
  for (int ph = 0; ph < 2; ++ph) {
    out[6 * ph] = ldexp((double)(long long)last[ph][0], -XY_HMC_K_SHIFT);
    for (int j = 1; j < xyk::kHmcSums; ++j)
      out[6 * ph + j] = ldexp((double)(long long)last[ph][j], -XY_FX_SHIFT);
  }
  return XY_OK;
}

xy_status xy_hmc_measure(xy_hmc* h, int64_t first, int64_t count, xy_obs* out, double* dH_out) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (first < 0 || count < 0 || first + count > h->rec_count)
    return fail(h, XY_EINVAL, "xy_hmc_measure: range [%lld, %lld) outside [0, %lld)",
                (long long)first, (long long)(first + count), (long long)h->rec_count);
  if (count > 0 && !out) return fail(h, XY_EINVAL, "xy_hmc_measure: NULL output");
  st = sync(h, "xy_hmc_measure: stream");
  if (st != XY_OK || count == 0) return st;
  std::vector<xy_hmc_record> r;
  try {
    r.resize((size_t)count);
  } catch (...) {
    return fail(h, XY_ENOMEM, "xy_hmc_measure: host allocation");
  }
  H_CUDA(h, cudaMemcpyAsync(r.data(), h->d_rec + first, (size_t)count * sizeof(xy_hmc_record),
                            cudaMemcpyDeviceToHost, h->stream),
         "xy_hmc_measure: copy");
  st = sync(h, "xy_hmc_measure: stream");
  if (st != XY_OK) return st;
  const double N = (double)h->p.L * (double)h->p.L;
  for (int64_t i = 0; i < count; ++i) {
    const xy_hmc_record& q = r[(size_t)i];
    xy_obs& o = out[i];
    o.C = ldexp((double)q.sum[0], -XY_FX_SHIFT);
    o.Ix = ldexp((double)q.sum[1], -XY_FX_SHIFT);
    o.Iy = ldexp((double)q.sum[2], -XY_FX_SHIFT);
    o.Mx = ldexp((double)q.sum[3], -XY_FX_SHIFT);
    o.My = ldexp((double)q.sum[4], -XY_FX_SHIFT);
    const double J = h->p.J, beta = q.beta;
    o.e = -J * o.C / N;
    o.abs_m = sqrt(o.Mx * o.Mx + o.My * o.My) / N;
    o.upsilon = (J * o.C - beta * J * J * (o.Ix * o.Ix + o.Iy * o.Iy)) / (2.0 * N);
    o.accepted = q.accepted;
    o.beta = beta;
    if (dH_out) dH_out[i] = q.dH;
  }
  return XY_OK;
}

xy_status xy_hmc_records_device(xy_hmc* h, const xy_hmc_record** d_records, int64_t* count) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (d_records) *d_records = h->d_rec;
  if (count) *count = h->rec_count;
  return XY_OK;
}

xy_status xy_hmc_info(const xy_hmc* h, int64_t* n_records, uint64_t* next_traj,
                      uint64_t* accepted) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (n_records) *n_records = h->rec_count;
  if (next_traj) *next_traj = h->next_traj;
  if (accepted) {
    unsigned long long a = 0;
    cudaError_t e = cudaMemcpyAsync(&a, &h->d_ctl->accepted, sizeof(a), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(const_cast<xy_hmc*>(h), e, "xy_hmc_info: copy");
    *accepted = a;
  }
  return XY_OK;
}

xy_status xy_hmc_get_state(xy_hmc* h, float* host_angles, float* host_momenta,
                           uint64_t* next_traj) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (!host_angles) return fail(h, XY_EINVAL, "xy_hmc_get_state: NULL angles");
  st = sync(h, "xy_hmc_get_state: stream");
  if (st != XY_OK) return st;
  uint32_t cur = 0;
  H_CUDA(h, cudaMemcpyAsync(&cur, &h->d_ctl->cur, sizeof(cur), cudaMemcpyDeviceToHost, h->stream),
         "xy_hmc_get_state: control block");
  st = sync(h, "xy_hmc_get_state: stream");
  if (st != XY_OK) return st;
  if (cur > 2) return fail(h, XY_ESTATE, "xy_hmc_get_state: corrupt state buffer index");
  const size_t N = (size_t)h->p.L * (size_t)h->p.L;
  H_CUDA(h, cudaMemcpyAsync(host_angles, h->th[cur], N * sizeof(float), cudaMemcpyDeviceToHost,
                            h->stream),
         "xy_hmc_get_state: angles");
  if (host_momenta)
    H_CUDA(h, cudaMemcpyAsync(host_momenta, h->d_p, N * sizeof(float), cudaMemcpyDeviceToHost,
                              h->stream),
           "xy_hmc_get_state: momenta");
  st = sync(h, "xy_hmc_get_state: stream");
  if (st != XY_OK) return st;
  if (next_traj) *next_traj = h->next_traj;
  return XY_OK;
}

xy_status xy_hmc_set_state(xy_hmc* h, const float* host_angles, const float* host_momenta,
                           uint64_t next_traj) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (!host_angles) return fail(h, XY_EINVAL, "xy_hmc_set_state: NULL angles");
  if (next_traj > 0xffffffffull)
    return fail(h, XY_EINVAL, "xy_hmc_set_state: trajectory number must be < 2^32");
  const size_t N = (size_t)h->p.L * (size_t)h->p.L;
  for (size_t i = 0; i < N; ++i) {
    if (!isfinite(host_angles[i])) {
      tmsg("xy_hmc_set_state: non-finite angle at %zu", i);
      return XY_ENUMERIC;
    }
    if (host_momenta && !isfinite(host_momenta[i])) {
      tmsg("xy_hmc_set_state: non-finite momentum at %zu", i);
      return XY_ENUMERIC;
    }
  }
  // all copies stream-ordered on the context's stream, then one synchronisation
  H_CUDA(h, cudaMemcpyAsync(h->th[0], host_angles, N * sizeof(float), cudaMemcpyHostToDevice,
                            h->stream),
         "xy_hmc_set_state: angles");
  if (host_momenta) {
    H_CUDA(h, cudaMemcpyAsync(h->d_p, host_momenta, N * sizeof(float), cudaMemcpyHostToDevice,
                              h->stream),
           "xy_hmc_set_state: momenta");
  } else {
    H_CUDA(h, cudaMemsetAsync(h->d_p, 0, N * sizeof(float), h->stream), "xy_hmc_set_state: momenta");
  }
  const uint32_t zero = 0;
  const unsigned long long t = next_traj;
  H_CUDA(h, cudaMemcpyAsync(&h->d_ctl->cur, &zero, sizeof(zero), cudaMemcpyHostToDevice, h->stream),
         "xy_hmc_set_state: control block");
  H_CUDA(h, cudaMemcpyAsync(&h->d_ctl->traj, &t, sizeof(t), cudaMemcpyHostToDevice, h->stream),
         "xy_hmc_set_state: control block");
  st = sync(h, "xy_hmc_set_state: stream");
  if (st != XY_OK) return st;
  h->next_traj = next_traj;
  return XY_OK;
}

xy_status xy_hmc_set_step(xy_hmc* h, double eps, int32_t n_md) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (!step_ok(eps, n_md))
    return fail(h, XY_EINVAL, "xy_hmc_set_step: eps must be finite and > 0, n_md in [1, 1000000]");
  h->p.eps = eps;
  h->p.n_md = n_md;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return XY_OK;
}

xy_status xy_hmc_set_beta(xy_hmc* h, double beta) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  if (!(beta >= 0.0) || !isfinite(beta))
    return fail(h, XY_EINVAL, "xy_hmc_set_beta: beta must be finite and >= 0");
  h->p.beta = beta;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return XY_OK;
}

xy_status xy_selftest_bounded_wait(void* cuda_stream, int64_t polls) {
  if (polls < 1 || polls > (1 << 24)) {
    tmsg("xy_selftest_bounded_wait: polls must be in [1, 2^24]");
    return XY_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned int* d_err = nullptr;
  unsigned int err = 0;
  cudaError_t e = xyk::dev_malloc(&d_err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) e = xyk::launch_selftest_wait(d_err, (long long)polls, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_err) cudaFree(d_err);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    tmsg("xy_selftest_bounded_wait: %s", cudaGetErrorString(e));
    return XY_ECUDA;
  }
  if (err) {
    tmsg("xy_selftest_bounded_wait: the bounded wait ran out after %lld polls", (long long)polls);
    return XY_ETIMEOUT;
  }
  tmsg("xy_selftest_bounded_wait: the wait completed, which it cannot");
  return XY_OK;
}

xy_status xy_hmc_synchronize(xy_hmc* h) {
  xy_status st = check(h);
  if (st != XY_OK) return st;
  return sync(h, "xy_hmc_synchronize");
}

xy_status xy_hmc_destroy(xy_hmc* h) {
  if (!h) return XY_OK;
  if (!is_live(h) || h->magic != kMagicLive) {
    tmsg("xy_hmc_destroy: not a live HMC context");
    return XY_ESTATE;
  }
  mark(h, false);
  (void)cudaStreamSynchronize(h->stream);
  release(h);
  h->magic = kMagicDead;
  delete h;
  return XY_OK;
}

const char* xy_hmc_last_error(const xy_hmc* h) {
  if (h && is_live(h) && h->magic == kMagicLive && h->sticky != XY_OK) return h->msg;
  return g_msg;
}

}  // extern "C"
