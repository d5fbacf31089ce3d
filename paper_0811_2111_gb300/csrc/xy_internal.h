// xy_internal.h -- launchers shared between the ABI layer (xy_api.cu) and the
// kernel translation units.  Not part of the public C ABI.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "xy.h"
#include "xy_device.cuh"
#include "xy_hmc.h"

namespace xyk {

// Blocks for a grid-stride loop over n items: a few waves over a GB300's 152
// SMs at most (16 CTAs per SM), the loop covering the rest.
inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = 152 * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Named range on the profiler timeline (NVTX) for the lifetime of the object:
// the entry points that enqueue work open one, so nsys/ncu timelines show
// which call launched which kernels.  Costs nothing without a tool attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Every device allocation of the library (xy_alloc.cu): cudaMalloc, unless a
// test armed xy_debug_fail_alloc, in which case the chosen allocation fails
// with cudaErrorMemoryAllocation.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}

// The debug build's device-side check words (xy_debug.h) of the instrumented
// translation units, read and cleared (0 in the release build).
unsigned int debug_take_sweep();    // xy_sweep.cu: two-pass sweep, layout kernels
unsigned int debug_take_narrow();   // xy_narrow.cu: whole-lattice batch kernel

// Arguments of one half-sweep launch over a single lattice.
struct HalfSweepArgs {
  float* theta;          // [2][L][W] split layout, W = L / 2
  int L;
  int W;
  float K;               // beta * J, the factor in exp(K * X), X = -dE / J
  float delta;           // proposal half-window
  xyd::RoundKeys rk;     // Philox round keys of the seed
  uint32_t lattice_id;
  uint32_t sweep;        // Philox counter word 1
  xy_record* rec;        // record of this sweep (zeroed before the red half)
  double beta;           // stored in the record by the black half
};

struct FusedMaps;

// Arguments of one fused sweep (both colours and the measure) src -> dst.
struct FusedArgs {
  const float* src;      // [2][L][W] state before the sweep
  float* dst;            // [2][L][W] state after the sweep (distinct buffer)
  int L;
  int W;
  float K;
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id;
  uint32_t sweep;
  xy_record* rec;
  double beta;
  int minb = 3;          // tile kernel instances per SM (2, 3 or 4: the register budget)
  const FusedMaps* maps = nullptr;   // tensor maps of src (required; host memory)
  unsigned int* error = nullptr;     // set nonzero if the wait for the staged rows runs out
};

// Whether the fused kernel handles side L (L a positive multiple of 128).
bool fused_supported(int L);

// One fused sweep of four replicas per site (float4 sites, read as floats
// [colour][y][4k + r]); replica r has lattice id lattice_id0 + r and K[r].
struct QuadFusedArgs {
  const float* src;      // [2][L][W] float4: state before the sweep
  float* dst;            // [2][L][W] float4: state after the sweep (distinct buffer)
  int L;
  int W;
  float K[4];
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id0;
  uint32_t sweep;
  xy_record* rec;        // the sweep's four records, replica r at rec + r
  double beta[4];
};

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point
// query; nullptr if unavailable).  Host only.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// TMA tensor maps of the fused sweep's two state buffers, each read as one
// [2 L][W] float array (row p L + y: colour p, lattice row y), boxes of 64
// plane columns and 1, 2 or 32 rows ([buffer][box]); host memory.
struct FusedMaps {
  CUtensorMap m[2][3];
  const float* base[2];  // the buffers they describe
};

// Encodes them for buffers buf0, buf1 of side L (host only; false if the
// encoder is unavailable or refuses the buffers).
bool encode_fused_maps(FusedMaps* out, const float* buf0, const float* buf1, int L);

// Which of the two buffers p is (0 or 1), -1 if neither.
inline int fused_map_index(const FusedMaps& m, const float* p) {
  return p == m.base[0] ? 0 : (p == m.base[1] ? 1 : -1);
}

// All n sweeps of one lattice in one cooperative launch of the fused sweep
// (tiles wait on their eight neighbours' per-tile sweep counters).
struct FusedPersistArgs {
  float* buf[2];         // [2][L][W] each: buf[0] holds the state before the first
                         // sweep; sweep s reads buf[s & 1] and writes buf[(s + 1) & 1]
  int L;
  int W;
  float K;
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id;
  uint32_t sweep0;       // Philox sweep word of the first sweep
  int n_sweeps;
  xy_record* rec;        // records of the n sweeps, zeroed
  double beta;
  unsigned int* flags;   // fused_tiles(L) tile counters, then the work counter
                         // (zeroed by the launch)
  unsigned int* counter; // == flags + fused_tiles(L)
  unsigned int* error;   // set nonzero when a bounded wait runs out
  long long spin_limit;  // polls before a wait gives up (fused_persistent_spin_limit())
  int skip_items;        // work items not handed out (0; > 0 only to test the
                         // failure path: their counters are then never set)
  int minb = 3;          // resident CTAs per SM the kernel is compiled for (2, 3 or 4)
  const FusedMaps* maps = nullptr;   // tensor maps of buf[0], buf[1] (host memory, required)
};

// The default bound of the persistent kernel's waits, in polls (about a second).
long long fused_persistent_spin_limit();

// Tiles of one fused sweep of side L (0 if !fused_supported(L)).
int fused_tiles(int L);

// Most sweeps one persistent launch takes (n_sweeps x tiles < 2^31).
int fused_persistent_max_sweeps(int L);

// One cooperative launch of a.n_sweeps fused sweeps; zeroes the counters first.
// cudaErrorInvalidValue on bad arguments; the launch's own error (e.g.
// cudaErrorCooperativeLaunchTooLarge) otherwise.
cudaError_t launch_fused_persistent(int sincos_mode, int reduce_mode, const FusedPersistArgs& a,
                                    cudaStream_t stream);

// All sweeps of a call of the four-replica fused sweep in one cooperative
// launch (tiles ordered by per-tile sweep counters, bounded waits).
struct QuadPersistArgs {
  QuadFusedArgs a;       // L, W, K, delta, rk, lattice_id0, beta (src, dst, sweep, rec unused)
  float* buf[2];         // buf[0] holds the state before the first sweep; sweep s
                         // reads buf[s & 1] and writes buf[(s + 1) & 1]
  uint32_t sweep0;       // Philox sweep word of the first sweep
  int n_sweeps;
  xy_record* rec;        // records of the n sweeps, [sweep][replica], zeroed
  unsigned int* flags;   // quad_persistent_tiles(L) tile counters, then the work counter
  unsigned int* counter; // == flags + quad_persistent_tiles(L)
  unsigned int* error;   // set nonzero when a bounded wait runs out
  long long spin_limit;  // polls before a wait gives up (quad_persistent_spin_limit())
};
int quad_persistent_tiles(int L);
int quad_persistent_max_sweeps(int L);
long long quad_persistent_spin_limit();
cudaError_t launch_quad_persistent(int sincos_mode, int reduce_mode, const QuadPersistArgs& p,
                                   cudaStream_t stream);

// Whether the fused four-replica kernel handles side L (a positive multiple of 32).
bool quad_fused_supported(int L);

// One fused four-replica sweep; cudaErrorInvalidValue if !quad_fused_supported(a.L)
// or src == dst.
cudaError_t launch_quad_fused(int sincos_mode, int reduce_mode, const QuadFusedArgs& a,
                              cudaStream_t stream);

// Two sweeps (a.sweep, a.sweep + 1) of a.src into a.dst in one launch, their
// records at a.rec and a.rec + 1 (xy_fused2.cu); cudaErrorInvalidValue if
// !fused_supported(a.L) or src == dst.
cudaError_t launch_fused2_sweeps(int sincos_mode, int reduce_mode, const FusedArgs& a,
                                 cudaStream_t stream);

// One fused sweep; cudaErrorInvalidValue if !fused_supported(a.L).
cudaError_t launch_fused_sweep(int sincos_mode, int reduce_mode, const FusedArgs& a,
                               cudaStream_t stream);

// The fused sweep over many lattices of one side L (a multiple of 128) of a
// batch, one launch per sweep: lattice lattices[z] for blockIdx.z = z.
struct FusedBatchArgs {
  float* theta;                 // batch buffer read on even sweeps, written on odd ones
  float* theta2;                // the other buffer
  const int64_t* offset;        // [n] floats from a buffer's start to lattice i
  const double* beta;           // [n] current beta (device)
  const int32_t* lattices;      // [n_lattices] lattices of this launch
  xy_record* records;           // [n][rec_stride]
  int64_t rec_stride;
  uint32_t rec_sweep0;
  const uint32_t* counters;     // [0] first sweep of the round
  int s;                        // sweep of the round (sweep = counters[0] + s)
  int L;
  double J;
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id0;
  int minb = 3;                 // fused tiles: CTAs per SM the kernel is compiled for (2, 3 or 4)
};
cudaError_t prepare_fused_batch(int sincos_mode, int reduce_mode);
cudaError_t launch_fused_batch_sweep(int sincos_mode, int reduce_mode, const FusedBatchArgs& b,
                                     int n_lattices, cudaStream_t stream);

// The same sweep on narrow tiles (32 rows x 16 plane columns, xy_narrow.cu)
// for batch lattices of side L % 32 == 0 that the fused tiles do not fit.
bool narrow_supported(int L);
int narrow_tiles(int L);                       // CTAs of one lattice's sweep
cudaError_t prepare_narrow_batch(int sincos_mode, int reduce_mode);
cudaError_t launch_narrow_batch_sweep(int sincos_mode, int reduce_mode, const FusedBatchArgs& b,
                                      int n_lattices, cudaStream_t stream);

// Whole lattices in one CTA's shared memory, all sweeps of a round per launch
// (xy_narrow.cu), for batch lattices with small_supported(L).
struct SmallBatchArgs {
  float* theta;                 // batch buffer read on even sweeps, written on odd ones
  float* theta2;                // the other buffer
  const int64_t* offset;        // [n] floats from a buffer's start to lattice i
  const int32_t* L;             // [n]
  const double* beta;           // [n] current beta (device)
  const int32_t* lattices;      // [grid] the lattice of each CTA
  xy_record* records;           // [n][rec_stride]
  int64_t rec_stride;
  uint32_t rec_sweep0;
  const uint32_t* counters;     // [0] first sweep of the round
  int sweeps;                   // sweeps of the round
  double J;
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id0;
};
constexpr size_t kSmallBudget = 112 * 1024;    // shared memory of one lattice (L <= 96)
size_t small_smem_bytes(int L);
bool small_supported(int L);
cudaError_t prepare_small_batch(int sincos_mode, int reduce_mode, size_t smem);
cudaError_t launch_small_batch(int sincos_mode, int reduce_mode, const SmallBatchArgs& a,
                               int n_lattices, size_t smem, cudaStream_t stream);

// Unit vectors of n angles with the kernels' sincos of precision `mode`
// (diagnostics and accuracy tests).
cudaError_t launch_eval_unit_vector(int mode, const float* theta, float* c, float* s, int64_t n,
                                    cudaStream_t stream);

// ---- batched lattices (xy_batch.cu) ----
constexpr int kClusterSize = 8;      // CTAs per cluster of the batched round kernel

// One CTA's band of rows [y_begin, y_end) of one lattice (lattice < 0: padding).
struct BatchBand {
  int32_t lattice;
  int32_t y_begin;
  int32_t y_end;
  int32_t pad;
};

struct BatchArgs {
  float* theta;                 // all lattices, split layout each, at offset[i] floats
  float* theta2;                // second buffer of the fused variant (sweep parity), or null
  const int64_t* offset;        // [n]
  const int32_t* L;             // [n]
  const double* beta;           // [n] current beta of each lattice
  const BatchBand* bands;       // [grid]
  xy_record* records;           // [n][rec_stride]
  int64_t rec_stride;
  uint32_t rec_sweep0;          // sweep index of each lattice's record 0
  const uint32_t* counters;     // device: [0] first sweep of this launch, [1] round
  int sweeps;                   // sweeps per launch
  double J;
  float delta;
  xyd::RoundKeys rk;
  uint32_t lattice_id0;         // lattice i uses lattice id lattice_id0 + i
  size_t cs_bytes;              // shared memory for the staged unit vectors
};

struct ExchangeArgs {
  int n_pairs;                  // candidate pairs (all ladders)
  const int32_t* pair_ladder;   // [n_pairs]
  const int32_t* pair_pos;      // [n_pairs] lower position p of the pair
  const int32_t* ladder_start;  // [n_ladders] first slot of each ladder in pos_*
  int32_t* pos_lattice;         // [slots] lattice at each position (beta order)
  const double* pos_beta;       // [slots] beta of each position
  double* beta;                 // [n] beta of each lattice (updated)
  const xy_record* records;
  int64_t rec_stride;
  uint32_t rec_sweep0;
  uint32_t* counters;           // device: [0] first sweep of the round, [1] round; advanced
  int sweeps;                   // sweeps per round (the last one's energies are compared)
  double J;
  xyd::RoundKeys rk;
  uint32_t lattice_id0;
  unsigned long long* accepted; // [slots] per lower position
  unsigned long long* attempted;
};

size_t batch_smem_bytes(int max_stage_floats2);
// Set the kernel's shared-memory limit (once, outside any stream capture).
cudaError_t prepare_batch_round(int sincos_mode, int reduce_mode, size_t smem);
cudaError_t launch_batch_round(int sincos_mode, int reduce_mode, const BatchArgs& a, int n_ctas,
                               cudaStream_t stream);
cudaError_t launch_exchange(const ExchangeArgs& a, cudaStream_t stream);
// Fused variant (512-thread CTAs, one stage and one cluster barrier per sweep).
size_t batch_fused_tail_bytes();
cudaError_t prepare_batch_fused(int sincos_mode, int reduce_mode, size_t smem);
cudaError_t launch_batch_fused(int sincos_mode, int reduce_mode, const BatchArgs& a, int n_ctas,
                               cudaStream_t stream);

// ---- series statistics / beta derivatives (xy_stats.cu) ----
constexpr int kStatsFields = 8;
constexpr int kPartials = 8;          // moment sums per segment
constexpr int kMaxSegments = 64;      // segments per chain
struct StatsArgs {
  const xy_record* records;   // [chains][stride]
  int64_t stride;
  int64_t first;              // first record of the window
  int64_t count;              // records in the window (> 0)
  const int32_t* L;           // [chains] device
  double J;
  double* out;                // [chains][kStatsFields] device
  double* partials;           // scratch [chains][kMaxSegments][kPartials] device
};
cudaError_t launch_series_stats(const StatsArgs& a, int n_chains, cudaStream_t stream);

// Red (colour 0) then black (colour 1) half-sweep; the black one also adds
// the sweep's bond/spin sums to *rec.  sincos_mode / reduce_mode as in xy.h.
cudaError_t launch_half_sweep(int colour, int sincos_mode, int reduce_mode,
                              const HalfSweepArgs& a, cudaStream_t stream);

// Hot (Philox domain 0) or cold start into the split layout.
cudaError_t launch_start(float* theta, int L, const xyd::RoundKeys& rk, uint32_t lattice_id,
                         int hot, cudaStream_t stream);

// Layout conversions between natural [y][x] order and the split layout.
cudaError_t launch_natural_to_split(const float* nat, float* split, int L, cudaStream_t stream);
cudaError_t launch_split_to_natural(const float* split, float* nat, int L, cudaStream_t stream);

// Philox words for counters (first + i, sweep, lattice_id, domain).
cudaError_t launch_philox_words(const xyd::RoundKeys& rk, uint32_t sweep, uint32_t lattice_id,
                                uint32_t domain, uint32_t first, int64_t n, uint32_t* out,
                                cudaStream_t stream);

// Non-finite check of the split-layout angles: sets *flag to 1 if any is.
cudaError_t launch_check_finite(const float* theta, int64_t n, unsigned int* flag,
                                cudaStream_t stream);

// ---- Hybrid Monte Carlo (xy_hmc.cu) ----
// Fixed-point accumulators of one phase of a trajectory (start or end):
// [0] K = sum p^2/2 (2^-24 units), [1..5] C, Ix, Iy, Mx, My (2^-30 units).
constexpr int kHmcSums = 6;

// Device-side control block of an HMC chain.  The accept kernel owns it
// between graph launches; every other kernel only reads `cur` and `traj`.
struct HmcCtl {
  unsigned long long acc[2][kHmcSums];   // sums of the running trajectory
  unsigned long long last[2][kHmcSums];  // sums of the last finished one
  xy_hmc_record* records;                // record array (host updates it on growth)
  unsigned long long rec;                // index of the next record
  unsigned long long traj;               // next trajectory number
  unsigned long long accepted;           // accepted trajectories so far
  uint32_t cur;                          // angle buffer (0..2) holding the state
  uint32_t error;                        // set by a kernel whose bounded wait ran out
};

// Kinds of leap-frog launch.
enum HmcKind {
  kHmcBeginDraw = 0,   // draw p, sums of (theta, p) -> acc[0], half kick, drift
  kHmcBeginRead = 1,   // p from the buffer, otherwise as kHmcBeginDraw
  kHmcStep = 2,        // full kick, drift
  kHmcFinal = 3,       // half kick, sums of (theta, p) -> acc[1], p written
  kHmcStep2 = 4        // two full kick-drift steps in one launch (tiled only)
};

// Angle buffers are addressed relative to the state buffer `cur` (read on the
// device): buffer (cur + off) % 3.  A trajectory reads offset 0 and writes 1
// in its first launch, then alternates 1 <-> 2, so offset 0 (the state before
// the trajectory) is never overwritten.
struct HmcArgs {
  float* th[3];          // the three angle buffers, natural order
  const float* p_in;     // momenta read by this launch (natural order)
  float* p_out;          // momenta written (may equal p_in, except for kHmcStep2)
  HmcCtl* ctl;           // device control block
  int L;
  float K;               // beta * J
  float eps;             // step
  float a;               // kick coefficient of this launch (eps or eps / 2)
  int src_off;           // buffer offset read (the accept step: offset of theta_n)
  int dst_off;           // buffer offset written
  xyd::RoundKeys rk;
  uint32_t lattice_id;
  int tiled;             // 1: tiled kernels (needs hmc_tiled_ok(L)), 0: one thread per site
  int pairs;             // 1: full steps two per launch (kHmcStep2; tiled only)
};

// One leap-frog launch of `kind` with the tiled or the per-site kernel (both
// give bit-identical results).
cudaError_t launch_hmc(int kind, int sincos_mode, const HmcArgs& a, cudaStream_t stream);
bool hmc_tiled_ok(int L);
// The test (mode 0: Metropolis on dH, writes a record) or, mode 1, the plain
// commit of an integration; both move acc to last and clear acc.
cudaError_t launch_hmc_accept(int mode, const HmcArgs& a, double beta, double J,
                              cudaStream_t stream);
// Momenta of the current trajectory into a.p_out.
cudaError_t launch_hmc_draw(const HmcArgs& a, cudaStream_t stream);
// Hot or cold start into th[0] (natural order), zero momenta into a.p_out.
cudaError_t launch_hmc_start(const HmcArgs& a, int hot, cudaStream_t stream);
// Move the state into th[0] if it lives elsewhere, and set cur = 0.
cudaError_t launch_hmc_canonical(const HmcArgs& a, cudaStream_t stream);
// Shared memory of the two-step and TMA kernels; set once per device before capture.
cudaError_t hmc_prepare(int sincos_mode);
// One leap-frog step (kick, drift) with the persistent TMA kernel: tensor maps
// (CUtensorMap, 128 bytes each) of the three angle buffers and of the momentum
// buffer a.p_in (== a.p_out), boxes of box_rows (32) rows x 128 columns,
// which is also the kernel's tile; grid = ctas.
// All kick-drift steps of a trajectory in one cooperative launch of the TMA
// step (per-tile step counters, bounded waits; see xy_hmc.cu).
struct HmcStepsArgs {
  HmcArgs a;             // a.a = eps, p_in == p_out (momenta in place), tiled
  int n_steps;           // kick-drift steps (step j reads buffer cur + 1 + (j & 1))
  unsigned int* flags;   // hmc_persist_tiles(L) tile counters (zeroed by the launch)
  long long spin_limit;  // polls before a wait gives up
};
cudaError_t launch_hmc_steps_persist(int sincos_mode, const HmcStepsArgs& q, const void* maps4,
                                     cudaStream_t stream);
int hmc_persist_tiles(int L);
long long hmc_persist_spin_limit();

// Two full steps in one launch (kHmcStep2) with the tensor maps (32 x 128
// boxes) of the three angle buffers and of a.p_in, which the tile-walking form
// reads by TMA; launch_hmc(kHmcStep2, ...) runs without them.
cudaError_t launch_hmc_step2(int sincos_mode, const HmcArgs& a, const void* th_maps3,
                             const void* p_map, cudaStream_t stream);

cudaError_t launch_hmc_step_tma(int sincos_mode, const HmcArgs& a, const void* maps4, int box_rows,
                                int ctas, cudaStream_t stream);

// One CTA waits, at most `polls` times, on an mbarrier nothing completes and
// sets *d_error (the bounded-wait failure path, without a fault).
cudaError_t launch_selftest_wait(unsigned int* d_error, long long polls, cudaStream_t stream);

// Whole trajectories in one cluster launch (xy_hmc_cluster.cu), for
// hmc_cluster_ok(L): L a power of two in [16, 256].  draw: momenta from Philox
// (else from a.p_in); mode as launch_hmc_accept.  The state stays in buffer cur.
bool hmc_cluster_ok(int L);
cudaError_t hmc_cluster_prepare(int sincos_mode);
cudaError_t launch_hmc_cluster(int sincos_mode, const HmcArgs& a, int n_md, int draw, int mode,
                               double beta, double J, cudaStream_t stream);

}  // namespace xyk
