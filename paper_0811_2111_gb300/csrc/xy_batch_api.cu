// xy_batch_api.cu -- C ABI of the batched engine (include/xy.h, "batches"):
// the work plan (bands of rows packed into clusters), buffers, replica
// exchange ladders, and one captured CUDA graph per round (round kernel +
// exchange kernel) replayed for every round.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "xy.h"
#include "xy_internal.h"
#include "xy_trace.h"

namespace {

constexpr uint32_t kBatchMagic = 0x58594254u;   // "XYBT"
thread_local char g_bmsg[512] = "no error";

std::mutex g_bmu;
std::unordered_set<const void*>& blive() {
  static std::unordered_set<const void*> s;
  return s;
}
bool batch_is_live(const void* b) {
  std::lock_guard<std::mutex> g(g_bmu);
  return blive().count(b) != 0;
}
void batch_mark(const void* b, bool live) {
  std::lock_guard<std::mutex> g(g_bmu);
  if (live) {
    blive().insert(b);
  } else {
    blive().erase(b);
  }
}

void bmsg(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_bmsg, sizeof(g_bmsg), fmt, ap);
  va_end(ap);
}

}  // namespace

struct xy_batch {
  uint32_t magic;
  int n;
  std::vector<int32_t> L;
  std::vector<double> beta0;
  std::vector<int32_t> ladder;
  xy_batch_params p;
  cudaStream_t stream;            // caller's stream (work is enqueued here)
  cudaStream_t capture_stream;    // private stream used only to record the graph
  // device buffers
  float* d_theta = nullptr;
  float* d_theta2 = nullptr;      // second buffer of the fused variant
  bool fused = true;
  int64_t* d_offset = nullptr;
  int32_t* d_L = nullptr;
  double* d_beta = nullptr;
  xyk::BatchBand* d_bands = nullptr;
  xy_record* d_rec = nullptr;
  uint32_t* d_counters = nullptr;
  int32_t* d_pair_ladder = nullptr;
  int32_t* d_pair_pos = nullptr;
  int32_t* d_ladder_start = nullptr;
  int32_t* d_pos_lattice = nullptr;
  double* d_pos_beta = nullptr;
  unsigned long long* d_acc = nullptr;
  unsigned long long* d_att = nullptr;
  float* d_scratch = nullptr;
  double* d_partials = nullptr;   // series-statistics scratch
  // host shadows
  std::vector<int64_t> offset;
  std::vector<xyk::BatchBand> bands;
  int n_ctas = 0;
  size_t cs_bytes = 0;
  int n_pairs = 0;
  int n_slots = 0;
  int n_ladders = 0;
  int64_t rec_cap = 0;            // records per lattice
  int64_t rec_count = 0;          // sweeps recorded per lattice
  uint64_t next_sweep = 0;
  // lattices whose side the single-lattice fused kernel takes (L % 128 == 0),
  // in groups of one side and about kGroupCtas CTAs per launch: each group
  // sweeps (one launch per sweep) on its own branch of the round's graph, in
  // parallel with the other groups and with the cluster kernel of the other
  // lattices, so that the groups fill each other's partial waves
  std::vector<int> group_L, group_start, group_size;
  std::vector<int32_t> group_lattices;
  int32_t* d_groups = nullptr;
  // lattices small enough for one CTA's shared memory: a whole round per launch
  std::vector<int32_t> small_lattices;
  int32_t* d_small = nullptr;
  size_t small_smem = 0;
  std::vector<cudaStream_t> branch_streams;
  std::vector<cudaEvent_t> ev_joins;
  cudaEvent_t ev_fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_cap = -1;         // rec_cap the graph was captured with
  xy_status sticky = XY_OK;
  char msg[512] = "no error";
};

namespace {

xy_status bfail(xy_batch* b, xy_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  snprintf(g_bmsg, sizeof(g_bmsg), "%s", buf);
  if (b && batch_is_live(b) && b->sticky == XY_OK) {
    b->sticky = st;
    snprintf(b->msg, sizeof(b->msg), "%s", buf);
  }
  return st;
}

xy_status bcuda(xy_batch* b, cudaError_t e, const char* what) {
  (void)cudaGetLastError();   // do not leave a non-sticky error for the next launch check
  return bfail(b, e == cudaErrorMemoryAllocation ? XY_ENOMEM : XY_ECUDA, "%s: %s", what,
               cudaGetErrorString(e));
}

#define B_CUDA(b, call, what)                              \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return bcuda(b, e_, what);      \
  } while (0)

xy_status check_batch(const xy_batch* b) {
  if (!b) {
    bmsg("NULL batch");
    return XY_EINVAL;
  }
  if (!batch_is_live(b) || b->magic != kBatchMagic) {
    bmsg("batch is not live (destroyed or never created)");
    return XY_ESTATE;
  }
  if (b->sticky != XY_OK) {
    bmsg("batch is in an earlier error: %s", b->msg);
    return b->sticky;
  }
  return XY_OK;
}

void free_all(xy_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  void* ptrs[] = {b->d_theta, b->d_theta2, b->d_offset, b->d_L, b->d_beta, b->d_bands, b->d_rec,
                  b->d_counters, b->d_pair_ladder, b->d_pair_pos, b->d_ladder_start,
                  b->d_pos_lattice, b->d_pos_beta, b->d_acc, b->d_att, b->d_scratch,
                  b->d_partials, b->d_groups, b->d_small};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  b->capture_stream = nullptr;
  for (cudaStream_t st : b->branch_streams)
    if (st) cudaStreamDestroy(st);
  b->branch_streams.clear();
  for (cudaEvent_t ev : b->ev_joins)
    if (ev) cudaEventDestroy(ev);
  b->ev_joins.clear();
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  b->ev_fork = nullptr;
}

// Bands: each lattice is cut into nb bands of whole rows (nb <= cluster size),
// about target_sites sites per band; lattices are packed first-fit (largest
// first) into clusters of kClusterSize CTAs, padded with idle CTAs.
// Shared memory a CTA may use for its band: two CTAs must fit one SM (228 KB).
constexpr size_t kStageBudget = 96 * 1024;          // two-pass: (r + 2) * L/2 unit vectors
constexpr size_t kFusedStageBudget = 108 * 1024;    // fused: (r + 4) * L/2 * (2 angles + 2 vectors)
constexpr int kGroupCtas = 128;                     // default CTAs per grouped launch (one branch each)

size_t band_bytes(bool fused, int rows, int L) {
  const size_t W = (size_t)(L / 2);
  return fused ? (size_t)(rows + 4) * W * 2 * (sizeof(float) + sizeof(float2))
               : (size_t)(rows + 2) * W * sizeof(float2);
}

void make_plan(xy_batch* b, int target_sites) {
  const int CS = xyk::kClusterSize;
  // fused algorithm: sides the single-lattice fused kernel takes (L % 128 ==
  // 0) go to groups; lattices that fit one CTA's shared memory run whole
  // rounds in one launch; the other multiples of 32 go to groups on the narrow
  // tiles; the rest to the cluster-launched bands
  std::map<int, std::vector<int>> groups;
  std::vector<int> banded;
  b->small_lattices.clear();
  b->small_smem = 0;
  for (int i = 0; i < b->n; ++i) {
    const int Li = b->L[i];
    if (b->fused && xyk::fused_supported(Li)) {
      groups[Li].push_back(i);
    } else if (b->fused && xyk::small_supported(Li)) {
      b->small_lattices.push_back(i);
      b->small_smem = std::max(b->small_smem, xyk::small_smem_bytes(Li));
    } else if (b->fused && xyk::narrow_supported(Li)) {
      groups[Li].push_back(i);
    } else {
      banded.push_back(i);
    }
  }
  // the largest lattices first, so they start first
  std::stable_sort(b->small_lattices.begin(), b->small_lattices.end(),
                   [&](int x, int y) { return b->L[x] > b->L[y]; });
  b->group_L.clear();
  b->group_start.clear();
  b->group_size.clear();
  b->group_lattices.clear();
  for (auto& kv : groups) {
    const int L = kv.first;
    const int tiles = xyk::fused_supported(L) ? (L / 2 / 64) * (L / 32)   // CTAs of one
                                              : xyk::narrow_tiles(L);      // lattice's sweep
    const int group_ctas = b->p.group_ctas > 0 ? b->p.group_ctas : kGroupCtas;
    const int per = std::max(1, group_ctas / tiles);
    // as few groups as `per` allows, their sizes differing by at most one
    const int count = (int)kv.second.size();
    const int ngroups = (count + per - 1) / per;
    for (int g = 0, k = 0; g < ngroups; ++g) {
      const int n = count / ngroups + (g < count % ngroups ? 1 : 0);
      b->group_L.push_back(L);
      b->group_start.push_back((int)b->group_lattices.size());
      b->group_size.push_back(n);
      for (int j = 0; j < n; ++j) b->group_lattices.push_back(kv.second[k + j]);
      k += n;
    }
  }
  std::vector<int> order;
  std::vector<int> nbands(b->n, 0), rows(b->n, 0);
  for (int i : banded) {
    const int Li = b->L[i];
    int nb = (int)((int64_t)Li * Li / std::max(target_sites, 1));
    // the largest band that fits the per-CTA shared-memory budget
    const size_t budget = b->fused ? kFusedStageBudget : kStageBudget;
    int rows_max = 1;
    while (rows_max < Li && band_bytes(b->fused, rows_max + 1, Li) <= budget) ++rows_max;
    nb = std::max(nb, (Li + rows_max - 1) / rows_max);
    nb = std::max(1, std::min(nb, std::min(CS, Li / 2)));
    const int r = (Li + nb - 1) / nb;
    nb = (Li + r - 1) / r;
    nbands[i] = nb;
    rows[i] = r;
    order.push_back(i);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return nbands[a] > nbands[c]; });
  std::vector<std::vector<xyk::BatchBand>> clusters;
  std::vector<int> fill;
  for (int i : order) {
    int cl = -1;
    for (size_t c = 0; c < clusters.size(); ++c)
      if (fill[c] + nbands[i] <= CS) {
        cl = (int)c;
        break;
      }
    if (cl < 0) {
      clusters.emplace_back();
      fill.push_back(0);
      cl = (int)clusters.size() - 1;
    }
    for (int k = 0; k < nbands[i]; ++k) {
      xyk::BatchBand band;
      band.lattice = i;
      band.y_begin = k * rows[i];
      band.y_end = std::min(b->L[i], (k + 1) * rows[i]);
      band.pad = 0;
      clusters[cl].push_back(band);
    }
    fill[cl] += nbands[i];
  }
  b->bands.clear();
  b->cs_bytes = 16;
  for (auto& c : clusters) {
    while ((int)c.size() < CS) c.push_back(xyk::BatchBand{-1, 0, 0, 0});
    for (auto& band : c) {
      b->bands.push_back(band);
      if (band.lattice >= 0)
        b->cs_bytes = std::max(b->cs_bytes,
                               band_bytes(b->fused, band.y_end - band.y_begin, b->L[band.lattice]));
    }
  }
  b->cs_bytes = (b->cs_bytes + 15) & ~(size_t)15;
  b->n_ctas = (int)b->bands.size();
}

xy_status grow(xy_batch* b, int64_t need) {
  if (need <= b->rec_cap) return XY_OK;
  int64_t cap = std::max<int64_t>(b->rec_cap > 0 ? b->rec_cap : 256, 16);
  while (cap < need) cap *= 2;
  xy_record* nr = nullptr;
  B_CUDA(b, xyk::dev_malloc(&nr, sizeof(xy_record) * (size_t)cap * b->n), "batch records");
  cudaError_t e = cudaMemsetAsync(nr, 0, sizeof(xy_record) * (size_t)cap * b->n, b->stream);
  if (e == cudaSuccess && b->rec_count > 0)
    e = cudaMemcpy2DAsync(nr, sizeof(xy_record) * cap, b->d_rec, sizeof(xy_record) * b->rec_cap,
                          sizeof(xy_record) * b->rec_count, b->n, cudaMemcpyDeviceToDevice,
                          b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    cudaFree(nr);
    return bcuda(b, e, "growing batch records");
  }
  if (b->d_rec) cudaFree(b->d_rec);
  b->d_rec = nr;
  b->rec_cap = cap;
  return XY_OK;
}

xyk::BatchArgs round_args(const xy_batch* b) {
  xyk::BatchArgs a;
  a.theta = b->d_theta;
  a.theta2 = b->d_theta2;
  a.offset = b->d_offset;
  a.L = b->d_L;
  a.beta = b->d_beta;
  a.bands = b->d_bands;
  a.records = b->d_rec;
  a.rec_stride = b->rec_cap;
  a.rec_sweep0 = 0;
  a.counters = b->d_counters;
  a.sweeps = b->p.sweeps_per_round;
  a.J = b->p.J;
  a.delta = (float)b->p.delta;
  a.rk = xyd::make_round_keys(b->p.seed);
  a.lattice_id0 = b->p.lattice_id0;
  a.cs_bytes = b->cs_bytes;
  return a;
}

xyk::ExchangeArgs exchange_args(const xy_batch* b) {
  xyk::ExchangeArgs x;
  x.n_pairs = b->n_pairs;
  x.pair_ladder = b->d_pair_ladder;
  x.pair_pos = b->d_pair_pos;
  x.ladder_start = b->d_ladder_start;
  x.pos_lattice = b->d_pos_lattice;
  x.pos_beta = b->d_pos_beta;
  x.beta = b->d_beta;
  x.records = b->d_rec;
  x.rec_stride = b->rec_cap;
  x.rec_sweep0 = 0;
  x.counters = b->d_counters;
  x.sweeps = b->p.sweeps_per_round;
  x.J = b->p.J;
  x.rk = xyd::make_round_keys(b->p.seed);
  x.lattice_id0 = b->p.lattice_id0;
  x.accepted = b->d_acc;
  x.attempted = b->d_att;
  return x;
}

xyk::FusedBatchArgs group_args(const xy_batch* b, size_t g, int s) {
  xyk::FusedBatchArgs f;
  f.theta = b->d_theta;
  f.theta2 = b->d_theta2;
  f.offset = b->d_offset;
  f.beta = b->d_beta;
  f.lattices = b->d_groups + b->group_start[g];
  f.records = b->d_rec;
  f.rec_stride = b->rec_cap;
  f.rec_sweep0 = 0;
  f.counters = b->d_counters;
  f.s = s;
  f.L = b->group_L[g];
  f.J = b->p.J;
  f.delta = (float)b->p.delta;
  f.rk = xyd::make_round_keys(b->p.seed);
  f.lattice_id0 = b->p.lattice_id0;
  f.minb = b->p.ctas_per_sm ? b->p.ctas_per_sm : 3;
  return f;
}

// One round: the banded cluster kernel (all of its sweeps in one launch) on
// the main branch and, on one parallel branch per group, the grouped fused
// sweeps (one launch per sweep); then, after all branches, the exchange
// kernel, which also advances the counters.
cudaError_t enqueue_round(const xy_batch* b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const size_t ng = b->group_L.size();
  if (ng > 0) e = cudaEventRecord(b->ev_fork, s);
  for (size_t g = 0; g < ng && e == cudaSuccess; ++g) {
    cudaStream_t gs = b->branch_streams[g];
    e = cudaStreamWaitEvent(gs, b->ev_fork, 0);
    for (int sw = 0; sw < b->p.sweeps_per_round && e == cudaSuccess; ++sw)
      e = xyk::fused_supported(b->group_L[g])
              ? xyk::launch_fused_batch_sweep(b->p.sincos_mode, b->p.reduce_mode,
                                              group_args(b, g, sw), b->group_size[g], gs)
              : xyk::launch_narrow_batch_sweep(b->p.sincos_mode, b->p.reduce_mode,
                                               group_args(b, g, sw), b->group_size[g], gs);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_joins[g], gs);
  }
  if (e == cudaSuccess && !b->small_lattices.empty()) {
    xyk::SmallBatchArgs sa;
    sa.theta = b->d_theta;
    sa.theta2 = b->d_theta2;
    sa.offset = b->d_offset;
    sa.L = b->d_L;
    sa.beta = b->d_beta;
    sa.lattices = b->d_small;
    sa.records = b->d_rec;
    sa.rec_stride = b->rec_cap;
    sa.rec_sweep0 = 0;
    sa.counters = b->d_counters;
    sa.sweeps = b->p.sweeps_per_round;
    sa.J = b->p.J;
    sa.delta = (float)b->p.delta;
    sa.rk = xyd::make_round_keys(b->p.seed);
    sa.lattice_id0 = b->p.lattice_id0;
    e = xyk::launch_small_batch(b->p.sincos_mode, b->p.reduce_mode, sa,
                                (int)b->small_lattices.size(), b->small_smem, s);
  }
  if (e == cudaSuccess && b->n_ctas > 0)
    e = b->fused ? xyk::launch_batch_fused(b->p.sincos_mode, b->p.reduce_mode, round_args(b),
                                           b->n_ctas, s)
                 : xyk::launch_batch_round(b->p.sincos_mode, b->p.reduce_mode, round_args(b),
                                           b->n_ctas, s);
  for (size_t g = 0; g < ng && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(s, b->ev_joins[g], 0);
  if (e == cudaSuccess) e = xyk::launch_exchange(exchange_args(b), s);
  return e;
}

// (Re)capture the graph of one round; the record buffer is baked in, so a
// growth of the records invalidates it.
cudaError_t capture_round(xy_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = enqueue_round(b, b->capture_stream);
  e = cudaStreamEndCapture(b->capture_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) b->graph_cap = b->rec_cap;
  return e;
}

}  // namespace

extern "C" {

xy_status xy_batch_create(const xy_batch_params* p, void* cuda_stream, xy_batch** out) {
  if (!out) {
    bmsg("NULL output pointer");
    return XY_EINVAL;
  }
  *out = nullptr;
  if (!p || p->n < 1 || !p->L || !p->beta) {
    bmsg("need n >= 1 and the L and beta arrays");
    return XY_EINVAL;
  }
  if (!(p->delta > 0.0) || p->delta > M_PI + 1e-12 || !isfinite(p->J) ||
      (p->start != XY_START_HOT && p->start != XY_START_COLD) || p->sincos_mode < 0 ||
      p->sincos_mode > 2 || p->reduce_mode < 0 || p->reduce_mode > 1 ||
      p->sweeps_per_round < 1 || p->sweeps_per_round > 1000000 || p->target_band_sites < 0 ||
      (p->algorithm != XY_ALGO_AUTO && p->algorithm != XY_ALGO_FUSED &&
       p->algorithm != XY_ALGO_TWO_PASS) || p->group_ctas < 0 || p->group_ctas > 4096 ||
      (p->ctas_per_sm != 0 && (p->ctas_per_sm < 2 || p->ctas_per_sm > 4))) {
    bmsg("bad delta, J, start, sincos_mode, reduce_mode, sweeps_per_round, target_band_sites, "
         "algorithm, group_ctas or ctas_per_sm");
    return XY_EINVAL;
  }
  for (int i = 0; i < p->n; ++i) {
    if (p->L[i] < 2 || p->L[i] > XY_BATCH_MAX_L || (p->L[i] & 1)) {
      bmsg("lattice %d: L must be even and in [2, %d]; got %d", i, XY_BATCH_MAX_L, p->L[i]);
      return XY_EINVAL;
    }
    if (!(p->beta[i] >= 0.0) || !isfinite(p->beta[i])) {
      bmsg("lattice %d: beta must be finite and >= 0", i);
      return XY_EINVAL;
    }
  }
  // ladders: lattices sharing a ladder id exchange temperatures; same L required
  std::map<int, std::vector<int>> ladders;
  if (p->ladder) {
    for (int i = 0; i < p->n; ++i) {
      const int l = p->ladder[i];
      if (l < -1 || l >= p->n) {
        bmsg("lattice %d: ladder id must be -1 or in [0, n)", i);
        return XY_EINVAL;
      }
      if (l >= 0) ladders[l].push_back(i);
    }
    for (auto& kv : ladders)
      for (int i : kv.second)
        if (p->L[i] != p->L[kv.second[0]]) {
          bmsg("ladder %d mixes lattice sides (replica exchange needs equal L)", kv.first);
          return XY_EINVAL;
        }
    // the exchange's Philox counter is ladder * 65536 + pair position: more
    // ladders, or longer ones, would reuse another pair's words
    if (ladders.size() > 65536u) {
      bmsg("more than 65536 ladders");
      return XY_EINVAL;
    }
    for (auto& kv : ladders)
      if (kv.second.size() > 65537u) {
        bmsg("ladder %d has more than 65537 lattices", kv.first);
        return XY_EINVAL;
      }
  }
  xy_batch* b = new (std::nothrow) xy_batch();
  if (!b) {
    bmsg("host allocation failed");
    return XY_ENOMEM;
  }
  b->magic = kBatchMagic;
  b->n = p->n;
  b->p = *p;
  b->L.assign(p->L, p->L + p->n);
  b->beta0.assign(p->beta, p->beta + p->n);
  if (p->ladder) b->ladder.assign(p->ladder, p->ladder + p->n);
  b->p.L = nullptr;
  b->p.beta = nullptr;
  b->p.ladder = nullptr;
  b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  b->fused = p->algorithm != XY_ALGO_TWO_PASS;
  batch_mark(b, true);

  auto fail_create = [&](xy_status st) {
    (void)cudaGetLastError();
    free_all(b);
    batch_mark(b, false);
    b->magic = 0;
    delete b;
    return st;
  };

  // layout: each lattice's split planes at a 16-byte aligned offset
  int64_t total = 0;
  b->offset.resize(b->n);
  for (int i = 0; i < b->n; ++i) {
    b->offset[i] = total;
    total += ((int64_t)b->L[i] * b->L[i] + 3) & ~(int64_t)3;
  }
  make_plan(b, p->target_band_sites > 0 ? p->target_band_sites : 8192);

  // ladder tables: positions ordered by initial beta
  std::vector<int32_t> pair_ladder, pair_pos, ladder_start, pos_lattice;
  std::vector<double> pos_beta;
  int li = 0;
  for (auto& kv : ladders) {
    std::vector<int> m = kv.second;
    std::stable_sort(m.begin(), m.end(), [&](int a, int c) { return b->beta0[a] < b->beta0[c]; });
    ladder_start.push_back((int32_t)pos_lattice.size());
    for (size_t k = 0; k < m.size(); ++k) {
      pos_lattice.push_back(m[k]);
      pos_beta.push_back(b->beta0[m[k]]);
      if (k + 1 < m.size()) {
        pair_ladder.push_back(li);
        pair_pos.push_back((int32_t)k);
      }
    }
    ++li;
  }
  b->n_ladders = li;
  b->n_pairs = (int)pair_ladder.size();
  b->n_slots = (int)pos_lattice.size();

  int64_t maxN = 4;
  for (int Li : b->L) maxN = std::max<int64_t>(maxN, (int64_t)Li * Li);
  const char* step = "capture stream";
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) step = "allocations";
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = xyk::dev_malloc(ptr, std::max<size_t>(bytes, 16));
  };
  alloc((void**)&b->d_theta, sizeof(float) * (size_t)std::max<int64_t>(total, 4));
  if (b->fused) alloc((void**)&b->d_theta2, sizeof(float) * (size_t)std::max<int64_t>(total, 4));
  alloc((void**)&b->d_offset, sizeof(int64_t) * b->n);
  alloc((void**)&b->d_L, sizeof(int32_t) * b->n);
  alloc((void**)&b->d_beta, sizeof(double) * b->n);
  alloc((void**)&b->d_bands, sizeof(xyk::BatchBand) * b->n_ctas);
  alloc((void**)&b->d_counters, sizeof(uint32_t) * 2);
  alloc((void**)&b->d_pair_ladder, sizeof(int32_t) * b->n_pairs);
  alloc((void**)&b->d_pair_pos, sizeof(int32_t) * b->n_pairs);
  alloc((void**)&b->d_ladder_start, sizeof(int32_t) * b->n_ladders);
  alloc((void**)&b->d_pos_lattice, sizeof(int32_t) * b->n_slots);
  alloc((void**)&b->d_pos_beta, sizeof(double) * b->n_slots);
  alloc((void**)&b->d_acc, sizeof(unsigned long long) * b->n_slots);
  alloc((void**)&b->d_att, sizeof(unsigned long long) * b->n_slots);
  alloc((void**)&b->d_scratch, sizeof(float) * (size_t)maxN);
  alloc((void**)&b->d_partials, sizeof(double) * (size_t)b->n * xyk::kMaxSegments * xyk::kPartials);
  alloc((void**)&b->d_groups, sizeof(int32_t) * b->group_lattices.size());
  alloc((void**)&b->d_small, sizeof(int32_t) * b->small_lattices.size());
  if (e == cudaSuccess && !b->group_L.empty()) {
    step = "branch streams";
    e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    for (size_t g = 0; g < b->group_L.size() && e == cudaSuccess; ++g) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->branch_streams.push_back(st);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->ev_joins.push_back(ev);
    }
  }
  if (e != cudaSuccess) {
    bmsg("xy_batch_create: %s: %s", step, cudaGetErrorString(e));
    return fail_create(e == cudaErrorMemoryAllocation ? XY_ENOMEM : XY_ECUDA);
  }
  step = "uploads";
  auto h2d = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  h2d(b->d_offset, b->offset.data(), sizeof(int64_t) * b->n);
  h2d(b->d_L, b->L.data(), sizeof(int32_t) * b->n);
  h2d(b->d_beta, b->beta0.data(), sizeof(double) * b->n);
  h2d(b->d_bands, b->bands.data(), sizeof(xyk::BatchBand) * b->n_ctas);
  h2d(b->d_pair_ladder, pair_ladder.data(), sizeof(int32_t) * b->n_pairs);
  h2d(b->d_pair_pos, pair_pos.data(), sizeof(int32_t) * b->n_pairs);
  h2d(b->d_ladder_start, ladder_start.data(), sizeof(int32_t) * b->n_ladders);
  h2d(b->d_pos_lattice, pos_lattice.data(), sizeof(int32_t) * b->n_slots);
  h2d(b->d_pos_beta, pos_beta.data(), sizeof(double) * b->n_slots);
  h2d(b->d_groups, b->group_lattices.data(), sizeof(int32_t) * b->group_lattices.size());
  h2d(b->d_small, b->small_lattices.data(), sizeof(int32_t) * b->small_lattices.size());
  if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, sizeof(uint32_t) * 2);
  if (e == cudaSuccess) e = cudaMemset(b->d_acc, 0, sizeof(unsigned long long) * std::max(b->n_slots, 1));
  if (e == cudaSuccess) e = cudaMemset(b->d_att, 0, sizeof(unsigned long long) * std::max(b->n_slots, 1));
  const xyd::RoundKeys rk = xyd::make_round_keys(p->seed);
  if (e == cudaSuccess) step = "start kernels";
  for (int i = 0; i < b->n && e == cudaSuccess; ++i)
    e = xyk::launch_start(b->d_theta + b->offset[i], b->L[i], rk, p->lattice_id0 + (uint32_t)i,
                          p->start == XY_START_HOT, b->stream);
  if (e == cudaSuccess) {
    // A kernel's dynamic shared-memory limit is one value for the whole
    // process, so it is set to the budget every plan stays within, not to this
    // batch's need: a later batch of smaller lattices must not lower it under
    // the launches an earlier batch has captured.
    step = "kernel attributes";
    e = b->fused ? xyk::prepare_batch_fused(p->sincos_mode, p->reduce_mode,
                                            kFusedStageBudget + xyk::batch_fused_tail_bytes())
                 : xyk::prepare_batch_round(p->sincos_mode, p->reduce_mode,
                                            kStageBudget + xyk::batch_smem_bytes(0));
    if (e == cudaSuccess && !b->group_L.empty())
      e = xyk::prepare_fused_batch(p->sincos_mode, p->reduce_mode);
    if (e == cudaSuccess && !b->group_L.empty())
      e = xyk::prepare_narrow_batch(p->sincos_mode, p->reduce_mode);
    if (e == cudaSuccess && !b->small_lattices.empty())
      e = xyk::prepare_small_batch(p->sincos_mode, p->reduce_mode, xyk::kSmallBudget);
  }
  if (e == cudaSuccess) {
    step = "synchronize";
    e = cudaStreamSynchronize(b->stream);
  }
  if (e != cudaSuccess) {
    bmsg("xy_batch_create: %s: %s (%d CTAs, %zu B staging)", step, cudaGetErrorString(e),
         b->n_ctas, b->cs_bytes);
    return fail_create(XY_ECUDA);
  }
  *out = b;
  return XY_OK;
}

xy_status xy_batch_reserve(xy_batch* b, int64_t n_rounds) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (n_rounds < 0) return bfail(b, XY_EINVAL, "xy_batch_reserve: negative count");
  return grow(b, b->rec_count + n_rounds * b->p.sweeps_per_round);
}

xy_status xy_batch_run(xy_batch* b, int64_t rounds) {
  const xyk::TraceRange trace("xy_batch_run");
  xyk::NvtxRange range("xy_batch_run");
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (rounds < 0) return bfail(b, XY_EINVAL, "xy_batch_run: negative round count");
  if (rounds == 0) return XY_OK;
  const int64_t sweeps = rounds * b->p.sweeps_per_round;
  if (b->next_sweep + (uint64_t)sweeps > 0xffffffffull)
    return bfail(b, XY_EINVAL, "xy_batch_run: sweep counter would pass 2^32 - 1");
  st = grow(b, b->rec_count + sweeps);
  if (st != XY_OK) return st;
  if (!b->graph || b->graph_cap != b->rec_cap) B_CUDA(b, capture_round(b), "xy_batch_run: graph capture");
  for (int64_t r = 0; r < rounds; ++r)
    B_CUDA(b, cudaGraphLaunch(b->graph, b->stream), "xy_batch_run: graph launch");
  b->next_sweep += (uint64_t)sweeps;
  b->rec_count += sweeps;
  return XY_OK;
}

xy_status xy_batch_info(const xy_batch* b, int32_t* n_lattices, int64_t* n_records,
                        uint64_t* next_sweep, int32_t* n_ctas) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (n_lattices) *n_lattices = b->n;
  if (n_records) *n_records = b->rec_count;
  if (next_sweep) *next_sweep = b->next_sweep;
  if (n_ctas) *n_ctas = b->n_ctas;
  return XY_OK;
}

xy_status xy_batch_launches_per_round(const xy_batch* b, int32_t* launches) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (!launches) {
    bmsg("xy_batch_launches_per_round: NULL output");
    return XY_EINVAL;
  }
  *launches = (int32_t)b->group_L.size() * b->p.sweeps_per_round + (b->n_ctas > 0 ? 1 : 0) +
              (b->small_lattices.empty() ? 0 : 1) + 1;
  return XY_OK;
}

xy_status xy_batch_measure(xy_batch* b, int32_t lattice, int64_t first, int64_t count,
                           xy_obs* out) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (lattice < 0 || lattice >= b->n || first < 0 || count < 0 || first + count > b->rec_count)
    return bfail(b, XY_EINVAL, "xy_batch_measure: lattice or record range out of bounds");
  if (count > 0 && !out) return bfail(b, XY_EINVAL, "xy_batch_measure: NULL output");
  B_CUDA(b, cudaStreamSynchronize(b->stream), "xy_batch_measure: stream");
  if (count == 0) return XY_OK;
  std::vector<xy_record> h((size_t)count);
  B_CUDA(b, cudaMemcpy(h.data(), b->d_rec + (size_t)lattice * b->rec_cap + first,
                       sizeof(xy_record) * (size_t)count, cudaMemcpyDeviceToHost),
         "xy_batch_measure: copy");
  const double N = (double)b->L[lattice] * b->L[lattice], J = b->p.J;
  const double unit = ldexp(1.0, -XY_FX_SHIFT);
  bool bad = false;
  for (int64_t i = 0; i < count; ++i) {
    const xy_record& r = h[(size_t)i];
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
    bad |= (r.flags & 1ull) != 0;
  }
  if (bad) return bfail(b, XY_ENUMERIC, "xy_batch_measure: a record saw a non-finite sum");
  return XY_OK;
}

xy_status xy_batch_records_device(xy_batch* b, const xy_record** d_records, int64_t* stride,
                                  int64_t* count) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (!d_records || !stride || !count) return bfail(b, XY_EINVAL, "NULL output");
  *d_records = b->d_rec;
  *stride = b->rec_cap;
  *count = b->rec_count;
  return XY_OK;
}

xy_status xy_batch_betas(xy_batch* b, double* host_beta) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (!host_beta) return bfail(b, XY_EINVAL, "xy_batch_betas: NULL output");
  B_CUDA(b, cudaStreamSynchronize(b->stream), "xy_batch_betas: stream");
  B_CUDA(b, cudaMemcpy(host_beta, b->d_beta, sizeof(double) * b->n, cudaMemcpyDeviceToHost),
         "xy_batch_betas: copy");
  return XY_OK;
}

xy_status xy_batch_exchange_stats(xy_batch* b, int32_t* n_slots, int32_t* slot_lattice,
                                  uint64_t* accepted, uint64_t* attempted) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (n_slots) *n_slots = b->n_slots;
  B_CUDA(b, cudaStreamSynchronize(b->stream), "xy_batch_exchange_stats: stream");
  if (b->n_slots == 0) return XY_OK;
  if (slot_lattice)
    B_CUDA(b, cudaMemcpy(slot_lattice, b->d_pos_lattice, sizeof(int32_t) * b->n_slots,
                         cudaMemcpyDeviceToHost), "copy");
  if (accepted)
    B_CUDA(b, cudaMemcpy(accepted, b->d_acc, sizeof(uint64_t) * b->n_slots,
                         cudaMemcpyDeviceToHost), "copy");
  if (attempted)
    B_CUDA(b, cudaMemcpy(attempted, b->d_att, sizeof(uint64_t) * b->n_slots,
                         cudaMemcpyDeviceToHost), "copy");
  return XY_OK;
}

xy_status xy_batch_get_state(xy_batch* b, int32_t lattice, float* host_angles) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (lattice < 0 || lattice >= b->n || !host_angles)
    return bfail(b, XY_EINVAL, "xy_batch_get_state: bad lattice or NULL output");
  const int L = b->L[lattice];
  const float* cur = (b->fused && (b->next_sweep & 1u)) ? b->d_theta2 : b->d_theta;
  B_CUDA(b, xyk::launch_split_to_natural(cur + b->offset[lattice], b->d_scratch, L, b->stream),
         "xy_batch_get_state: layout");
  B_CUDA(b, cudaMemcpyAsync(host_angles, b->d_scratch, sizeof(float) * (size_t)L * L,
                            cudaMemcpyDeviceToHost, b->stream), "xy_batch_get_state: copy");
  B_CUDA(b, cudaStreamSynchronize(b->stream), "xy_batch_get_state: stream");
  return XY_OK;
}

xy_status xy_batch_series_stats(xy_batch* b, int64_t first, int64_t count, double* d_out) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  if (!d_out || first < 0 || count < 1 || first + count > b->rec_count)
    return bfail(b, XY_EINVAL, "xy_batch_series_stats: bad window or NULL output");
  xyk::StatsArgs a;
  a.records = b->d_rec;
  a.stride = b->rec_cap;
  a.first = first;
  a.count = count;
  a.L = b->d_L;
  a.J = b->p.J;
  a.out = d_out;
  a.partials = b->d_partials;
  B_CUDA(b, xyk::launch_series_stats(a, b->n, b->stream), "xy_batch_series_stats");
  return XY_OK;
}

xy_status xy_batch_synchronize(xy_batch* b) {
  xy_status st = check_batch(b);
  if (st != XY_OK) return st;
  B_CUDA(b, cudaStreamSynchronize(b->stream), "xy_batch_synchronize");
  return XY_OK;
}

xy_status xy_batch_destroy(xy_batch* b) {
  if (!b) return XY_OK;
  if (!batch_is_live(b) || b->magic != kBatchMagic) {
    bmsg("xy_batch_destroy: batch is not live (double destroy?)");
    return XY_ESTATE;
  }
  batch_mark(b, false);
  cudaStreamSynchronize(b->stream);
  free_all(b);
  b->magic = 0;
  delete b;
  return XY_OK;
}

const char* xy_batch_last_error(const xy_batch* b) {
  if (b && batch_is_live(b) && b->sticky != XY_OK) return b->msg;
  return g_bmsg;
}

}  // extern "C"
