/*
 * xy.h -- C ABI of the GB300 (sm_103a) checkerboard Metropolis engine for the
 * 2-d XY model.
 *
 * Model (Eq. (1) of "GPU computing for 2-d spin systems: CUDA vs OpenGL"):
 *     H = -J sum_<ij> cos(theta_i - theta_j)
 * on a periodic L x L square lattice; each site is bonded to its +x and +y
 * neighbour (2N bonds, N = L^2).  Sites are updated by single-site
 * Metropolis in red/black (checkerboard) order: all sites with (x + y) even,
 * then all with (x + y) odd.  A site proposes
 *     theta' = theta + delta * (2 u0 - 1), wrapped once into [0, 2 pi),
 * and takes it iff u1 < exp(-beta dE), dE = -J sum_{4 nn j}
 * [cos(theta' - theta_j) - cos(theta - theta_j)]; the accept is the per-site
 * select new = z * proposal + (1 - z) * old of Sec. 3.2.  The global sums
 * that the paper moved to the CPU (Sec. 1.2) are computed on the device,
 * fused into every sweep.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 * (seed_lo, seed_hi) and counter (c, sweep, lattice_id, domain), where
 * site = y * L + x (natural order); domain 0 draws the hot start
 * (c = site, theta = 2 pi u24(w0) at sweep 0), domain 1 the Metropolis words
 * of sweep t, domain 2 the replica-exchange words.  The Metropolis draws use
 * all four words of a block for two sites: the sites x and x + 2 of a row
 * with x & 2 == 0 share c = y * L + x, the first taking (w0 -> proposal,
 * w1 -> accept), the second (w2 -> proposal, w3 -> accept); so a site's
 * counter is c = site - (x & 2), and its words are w2, w3 iff x & 2.
 * u24(w) = (w >> 8) * 2^-24, exact in FP32.
 *
 * Conventions
 *   - Every call returns an xy_status; nothing aborts, nothing throws.  The
 *     first error is sticky in its context: later calls on that context
 *     return it until the context is destroyed.
 *   - Work is ordered on the context's CUDA stream.  xy_sweep only enqueues;
 *     asynchronous device errors surface at the next call that synchronizes
 *     (xy_measure, xy_get_state, xy_set_state, xy_synchronize).
 *   - Angles cross the ABI in natural order [y][x] as FP32 radians.  On the
 *     device they live in a checkerboard-split layout: two planes
 *     [colour][y][k], colour = (x + y) & 1, k = x >> 1, i.e. L*L floats.
 *   - Buffers passed in by the caller stay owned by the caller and are never
 *     freed by the library.
 *   - A context is thread-compatible, not thread-safe.
 */
#ifndef XY_H
#define XY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xy_ctx xy_ctx;

typedef enum {
    XY_OK = 0,
    XY_EINVAL = 1,     /* bad argument (odd L, NULL pointer, out of range)     */
    XY_ENOMEM = 2,     /* device or host allocation failed                     */
    XY_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed          */
    XY_ETIMEOUT = 4,   /* a bounded device-side wait ran out                   */
    XY_ESTATE = 5,     /* context destroyed, invalid, or in an earlier error   */
    XY_ENUMERIC = 6    /* a non-finite angle or sum was detected               */
} xy_status;

enum { XY_START_HOT = 0, XY_START_COLD = 1 };
/* Precision of the per-site unit vectors and Boltzmann factors (all FP32):
 *   XY_SINCOS_ACCURATE  own Cody-Waite + minimax sincos (max error 6.8e-8) and expf;
 *   XY_SINCOS_FAST      the SFU intrinsics __sincosf / __expf;
 *   XY_SINCOS_LIBM      CUDA's sincosf / expf. */
enum { XY_SINCOS_ACCURATE = 0, XY_SINCOS_FAST = 1, XY_SINCOS_LIBM = 2 };
/* Sweep kernel: AUTO picks PERSISTENT when L is a multiple of 128 up to 4096
 * (falling back to one fused launch per sweep when the cooperative grid does
 * not fit on the device), FUSED for larger multiples of 128, else TWO_PASS.
 *   XY_ALGO_FUSED      one launch per sweep (both colours + measure), the state
 *                      ping-pongs between the caller's buffer and a library
 *                      buffer of the same size (8 B moved per update);
 *   XY_ALGO_TWO_PASS   one launch per colour, in place (12 B per update);
 *   XY_ALGO_PERSISTENT the fused sweep, all sweeps of one xy_sweep call in one
 *                      cooperative launch: each tile of 32 x 128 sites starts
 *                      sweep s once its eight neighbouring tiles have finished
 *                      sweep s - 1 (per-tile counters in device memory, bounded
 *                      waits; a wait that runs out is reported as XY_ETIMEOUT
 *                      at the next synchronizing call); a tile's staged rows
 *                      are copied by TMA (tensor maps of the two buffers,
 *                      encoded at xy_create: XY_ECUDA there if the driver's
 *                      encoder is unavailable).  Needs L % 128 == 0 and every
 *                      CTA of the grid resident (the launch fails with XY_ECUDA
 *                      otherwise);
 *   XY_ALGO_FUSED2     two sweeps per launch (temporal blocking): each tile is
 *                      staged with a halo of four rows and columns and runs
 *                      both sweeps' half-sweeps in shared memory on shrinking
 *                      regions (half the DRAM traffic, 15 % recomputed halo
 *                      updates); an odd last sweep of a call runs as FUSED.
 *                      Needs L % 128 == 0; never chosen by AUTO.
 * All make bit-identical decisions. */
enum { XY_ALGO_AUTO = 0, XY_ALGO_FUSED = 1, XY_ALGO_TWO_PASS = 2, XY_ALGO_PERSISTENT = 3,
       XY_ALGO_FUSED2 = 4 };
/* Per-sweep sums (records below):
 *   XY_REDUCE_EXACT        every per-site term is rounded to fixed point
 *                          (2^-19 for the four bond cosines of a site, 2^-20
 *                          for the other terms: one FMA each) before any
 *                          addition, and the integers are added exactly, so
 *                          a record is independent of the order of addition:
 *                          every algorithm and batch plan gives the same bits;
 *   XY_REDUCE_COMPENSATED  Neumaier-compensated FP32 sums per CTA, FP64 over
 *                          the CTA's partials, then fixed point (results may
 *                          differ in the last bits between algorithms). */
enum { XY_REDUCE_EXACT = 0, XY_REDUCE_COMPENSATED = 1 };

/* Largest supported side (N = L^2 must fit the 32-bit site counter and the
 * fixed-point record sums). */
#define XY_MAX_L 32768

typedef struct {
    int32_t L;            /* side, even, 2 <= L <= XY_MAX_L                    */
    int32_t start;        /* XY_START_HOT (Philox domain 0) or XY_START_COLD   */
    double beta;          /* inverse temperature, >= 0                          */
    double J;             /* coupling (1 in the paper's model)                  */
    double delta;         /* proposal half-window, 0 < delta <= pi              */
    uint64_t seed;        /* Philox key                                         */
    int32_t sincos_mode;  /* XY_SINCOS_ACCURATE, _FAST or _LIBM                 */
    int32_t reduce_mode;  /* XY_REDUCE_EXACT or XY_REDUCE_COMPENSATED           */
    uint32_t lattice_id;  /* third Philox counter word                          */
    int32_t algorithm;    /* XY_ALGO_AUTO, _FUSED or _PERSISTENT (need L % 128 == 0), _TWO_PASS */
    int32_t ctas_per_sm;  /* work plan of the fused and persistent sweeps: 3 CTAs of the
                             tile kernel per SM (at most 80 registers a thread), 4 (at
                             most 64: more warps per SM), 2 (at most 128: more
                             independent work in flight per warp, fewer warps), or 0
                             for the library's default: 3 for the persistent sweep,
                             4 for one fused launch per sweep (the faster plans at
                             L = 4096 and at L = 8192, 16384).  Results do not
                             depend on it; tuning callers time the plans
                             (autotune.py). */
} xy_params;

/* Per-sweep record as stored on the device (64 bytes).  The five sums are
 * signed fixed point in units of 2^-XY_FX_SHIFT, accumulated with integer
 * atomics (order-independent; with XY_REDUCE_EXACT exact sums of the
 * per-site terms rounded to 2^-19 / 2^-20):
 *   sum[0] = C  = sum_s cos(t_s - t_{s+x}) + cos(t_s - t_{s+y})
 *   sum[1] = Ix = sum_s sin(t_s - t_{s+x})
 *   sum[2] = Iy = sum_s sin(t_s - t_{s+y})
 *   sum[3] = Mx = sum_s cos t_s,   sum[4] = My = sum_s sin t_s
 * accepted = accepted moves in the sweep (both colours); beta = the beta the
 * sweep ran at; flags bit 0 = a non-finite value was seen. */
#define XY_FX_SHIFT 30
typedef struct {
    int64_t sum[5];
    uint64_t accepted;
    double beta;
    uint64_t flags;
} xy_record;

/* Observables of one sweep, derived from its record:
 *   e = -J C / N,  abs_m = |M| / N,
 *   upsilon = (J C - beta J^2 (Ix^2 + Iy^2)) / (2N)  (helicity modulus,
 *   x/y averaged; <I> = 0 by symmetry). */
typedef struct {
    double e, abs_m, upsilon;
    double C, Ix, Iy, Mx, My;
    uint64_t accepted;
    double beta;
} xy_obs;

/* Create a lattice context and initialise it (hot or cold start, sweep 0).
 *   p          parameters, copied; validated as documented above.
 *   cuda_stream a cudaStream_t, or NULL for the legacy default stream.
 *   d_angles   NULL: the library allocates the L*L float working buffer;
 *              else a caller-owned device buffer of >= L*L floats, 16-byte
 *              aligned, used in the split layout (never freed here).  The
 *              fused kernel also allocates a second L*L float buffer.
 *   out        receives the context (NULL on failure).
 * Errors: XY_EINVAL, XY_ENOMEM, XY_ECUDA (see xy_last_error(NULL)). */
xy_status xy_create(const xy_params *p, void *cuda_stream, void *d_angles, xy_ctx **out);

/* Re-run the start (hot or cold, as created) with `seed`, set the next sweep
 * to 0 and clear the records.  Asynchronous, allocates nothing: one
 * independent chain after another can reuse a context. */
xy_status xy_reset(xy_ctx *ctx, uint64_t seed);

/* Make room for n more records so that xy_sweep allocates nothing. */
xy_status xy_reserve(xy_ctx *ctx, int64_t n_more);

/* Enqueue n >= 0 sweeps (red half then black half with the fused measure);
 * appends n records.  Asynchronous.  Fails with XY_EINVAL if the sweep
 * counter would pass 2^32.  With the fused kernel the state is back in the
 * caller's buffer when the call returns (an odd n costs one device copy). */
xy_status xy_sweep(xy_ctx *ctx, int64_t n_sweeps);

/* Copy records [first, first + count) to host_out (count >= 0 entries) and
 * derive the observables.  Synchronizes the stream.  XY_ENUMERIC if a record
 * carries the non-finite flag. */
xy_status xy_measure(xy_ctx *ctx, int64_t first, int64_t count, xy_obs *host_out);

/* Raw device records, for device-side consumers (e.g. a backward kernel):
 * *d_records points at the first record (xy_record[count]); stream-ordered. */
xy_status xy_records_device(xy_ctx *ctx, const xy_record **d_records, int64_t *count);

/* Number of records so far and the next sweep index. */
xy_status xy_info(const xy_ctx *ctx, int64_t *n_records, uint64_t *next_sweep);

/* The sweep algorithm the context runs (what XY_ALGO_AUTO resolved to):
 * XY_ALGO_FUSED, XY_ALGO_TWO_PASS or XY_ALGO_PERSISTENT. */
xy_status xy_algorithm(const xy_ctx *ctx, int32_t *algorithm);

/* Self-test of the persistent sweep's failure path (no context involved):
 * one persistent launch at L = 128 whose first sweep is never handed out, so
 * every wait of the second sweep runs out after `polls` polls (1 <= polls <=
 * 2^24; each poll sleeps ~128 ns) and the kernel ends with its error word set.
 * Returns XY_ETIMEOUT when that happened (the expected result), XY_OK if the
 * waits completed (a bug), XY_EINVAL / XY_ECUDA otherwise.  Stream-ordered on
 * cuda_stream, synchronizes it; allocates and frees ~130 KB of device memory.
 * Exists to test the failure path; the paper has no counterpart. */
xy_status xy_selftest_persistent_wait(void *cuda_stream, int64_t polls);

/* The library's debug build (libxy_debug.so, compiled with -DXY_DEBUG) guards
 * the index arithmetic of its two-pass sweep, layout and whole-lattice batch
 * kernels: a check that fails sets a bit of a device word and skips the
 * access instead of trapping.  xy_debug_build returns 1 in that build, 0 in
 * the release build.  xy_debug_checks synchronizes the device and returns the
 * failed checks since the last call (bits 0-4: two-pass staging loads, stage
 * stores, row loads and stores, stage reads, layout indices; bits 8-9:
 * whole-lattice pair and site positions) and clears them; always 0 in the
 * release build.  XY_EINVAL for a NULL output, XY_ECUDA if the words cannot
 * be read.  Test aids; the paper has no counterpart. */
int32_t xy_debug_build(void);
xy_status xy_debug_checks(uint32_t *failed);

/* Test hook of the out-of-memory paths: the k-th device allocation made by
 * the library after this call (k >= 1; counted across every engine and thread
 * of the process) fails as if the device were out of memory, without reaching
 * the driver; k = 0 disarms the hook.  The failing call returns XY_ENOMEM,
 * frees what it had allocated and leaves the device usable.  Returns XY_EINVAL
 * for k < 0.  Exists to test the failure path; the paper has no counterpart. */
xy_status xy_debug_fail_alloc(int32_t k);

/* Copy the angles (natural order, L*L floats) to host memory and report the
 * next sweep index.  Synchronizes. */
xy_status xy_get_state(xy_ctx *ctx, float *host_angles, uint64_t *next_sweep);

/* Replace the angles (natural order, finite) and the next sweep index; clears
 * the records.  Synchronizes.  With the counter-based RNG a restored state
 * continues bit-identically (checkpoint/resume). */
xy_status xy_set_state(xy_ctx *ctx, const float *host_angles, uint64_t next_sweep);

/* Change beta for later sweeps (records keep the beta they ran at). */
xy_status xy_set_beta(xy_ctx *ctx, double beta);

/* Kernel timing.  With every = k > 0, xy_sweep brackets the kernel launches
 * of every k-th sweep (sweep index % k == 0) with CUDA events on the context
 * stream, so that the timed sample costs almost nothing; every = 0 turns it
 * off.  xy_kernel_time synchronizes and returns the summed device time (ms)
 * and the number of timed launches of kernel k since timing was (re)enabled
 * (k = 0: red half-sweep, k = 1: black half-sweep with the fused measure). */
xy_status xy_timing(xy_ctx *ctx, int every);
xy_status xy_kernel_time(xy_ctx *ctx, int kernel, double *total_ms, int64_t *launches);

/* Wait for the stream and report any asynchronous error. */
xy_status xy_synchronize(xy_ctx *ctx);

/* Destroy; NULL-safe.  A destroyed context must not be used again. */
xy_status xy_destroy(xy_ctx *ctx);

/* Message of the context's sticky error, or of the calling thread's last
 * failure when ctx is NULL.  Never NULL. */
const char *xy_last_error(const xy_ctx *ctx);

/* Philox4x32-10 words for counters (first + i, sweep, lattice_id, domain),
 * i < n, written as uint32[n][4] to device memory d_out, on cuda_stream --
 * the same device generator the sweeps use (for bit-exact checks). */
xy_status xy_philox_words(uint64_t seed, uint32_t sweep, uint32_t lattice_id, uint32_t domain,
                          uint32_t first, int64_t n, uint32_t *d_out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices of uneven sides and temperatures swept
 * together, one launch per round of sweeps, with optional replica exchange.
 * The Sec. 3.2 remark that one RGBA texel holds four replicas "maybe at
 * different temperatures" is the precedent; here each lattice keeps its own
 * split-layout planes and the plan gives every lattice one of four kernels
 * (see `algorithm`).  Every lattice i evolves exactly as a single-lattice
 * context with the same L, beta, seed and lattice_id = lattice_id0 + i would
 * (same Philox counters and words, same site update).
 * Replica exchange: lattices sharing a ladder id (equal L required) are
 * ordered by initial beta; after every round the pairs of positions
 * (p, p+1), p = round mod 2, round mod 2 + 2, ..., swap temperatures iff
 * u24(w0) < exp((beta_p - beta_{p+1})(E_p - E_{p+1})), E = -J C of the round's
 * last sweep, Philox domain 2 with counter (ladder * 65536 + p, round,
 * lattice_id0, 2), ladder counted from 0 in increasing ladder id, so at most
 * 65536 ladders of at most 65537 lattices each (else XY_EINVAL).  Each round (round kernel + exchange kernel) is one
 * captured CUDA graph replayed round after round.
 * ------------------------------------------------------------------------ */
#define XY_BATCH_MAX_L 256

typedef struct xy_batch xy_batch;

typedef struct {
    int32_t n;                  /* number of lattices, >= 1                         */
    const int32_t *L;           /* [n] even sides in [2, XY_BATCH_MAX_L] (copied)    */
    const double *beta;         /* [n] initial inverse temperatures (copied)         */
    const int32_t *ladder;      /* [n] ladder id per lattice (-1: none), or NULL     */
    double J;                   /* coupling                                          */
    double delta;               /* proposal half-window, (0, pi]                     */
    uint64_t seed;              /* Philox key of every lattice                       */
    int32_t start;              /* XY_START_HOT or XY_START_COLD                     */
    int32_t sincos_mode;        /* as in xy_params                                   */
    int32_t reduce_mode;        /* as in xy_params                                   */
    uint32_t lattice_id0;       /* lattice i uses lattice id lattice_id0 + i         */
    int32_t sweeps_per_round;   /* sweeps per launch (and between exchanges), >= 1   */
    int32_t target_band_sites;  /* sites per CTA band of the work plan (0: 8192)     */
    int32_t algorithm;          /* XY_ALGO_AUTO / _FUSED: state ping-ponged between two
                                   buffers; lattices with L % 128 == 0 run the fused
                                   sweep kernel's tiles and other multiples of 32 its
                                   narrow tiles, in groups of about 128 CTAs (one launch
                                   per group and sweep, groups on parallel graph
                                   branches); lattices small enough for one CTA's shared
                                   memory (L <= 96) run whole, one CTA each, all sweeps
                                   of the round in one launch; the rest are cut into
                                   bands of rows, the bands of a lattice one thread-
                                   block cluster, one staging and one cluster barrier
                                   per sweep; XY_ALGO_TWO_PASS: every lattice in place
                                   in the cluster kernel, two barriers per sweep */
    int32_t group_ctas;         /* work plan: CTAs per grouped tile launch (each group one
                                   graph branch; 0: 128, at most 4096)               */
    int32_t ctas_per_sm;        /* work plan: the grouped tile kernel compiled for 2, 3
                                   or 4 CTAs per SM, as xy_params.ctas_per_sm (0: 3) */
} xy_batch_params;

/* Create and hot/cold-start all lattices; the plan, ladders and buffers are
 * built here.  Errors: XY_EINVAL (bad sizes, a ladder mixing sides), XY_ENOMEM,
 * XY_ECUDA; xy_batch_last_error(NULL) describes them. */
xy_status xy_batch_create(const xy_batch_params *p, void *cuda_stream, xy_batch **out);
/* Make room for n_rounds more rounds of records (so xy_batch_run allocates nothing). */
xy_status xy_batch_reserve(xy_batch *b, int64_t n_rounds);
/* Enqueue `rounds` rounds: sweeps_per_round sweeps of every lattice, then one
 * replica-exchange step.  Asynchronous; appends sweeps_per_round records per
 * lattice per round. */
xy_status xy_batch_run(xy_batch *b, int64_t rounds);
/* Lattice count, records per lattice, next sweep index, CTAs per launch. */
xy_status xy_batch_info(const xy_batch *b, int32_t *n_lattices, int64_t *n_records,
                        uint64_t *next_sweep, int32_t *n_ctas);
/* Observables of records [first, first + count) of one lattice (synchronizes). */
xy_status xy_batch_measure(xy_batch *b, int32_t lattice, int64_t first, int64_t count,
                           xy_obs *host_out);
/* Device records, laid out [lattice][stride]; `count` valid per lattice. */
xy_status xy_batch_records_device(xy_batch *b, const xy_record **d_records, int64_t *stride,
                                  int64_t *count);
/* Current beta of every lattice (host array of n; synchronizes). */
xy_status xy_batch_betas(xy_batch *b, double *host_beta);
/* Exchange bookkeeping per ladder slot (ladders in ascending id, positions in
 * beta order): lattice at each slot, accepted and attempted swaps of the pair
 * (slot, slot + 1).  Any output may be NULL; *n_slots receives the slot count. */
xy_status xy_batch_exchange_stats(xy_batch *b, int32_t *n_slots, int32_t *slot_lattice,
                                  uint64_t *accepted, uint64_t *attempted);
/* Angles of one lattice in natural order (L*L floats; synchronizes). */
xy_status xy_batch_get_state(xy_batch *b, int32_t lattice, float *host_angles);
/* Kernel launches one round replays: the grouped tile sweeps (groups x
 * sweeps_per_round), the whole-lattice launch if any lattice runs whole, the
 * cluster kernel if any lattice is banded, and the exchange kernel. */
xy_status xy_batch_launches_per_round(const xy_batch *b, int32_t *launches);
xy_status xy_batch_synchronize(xy_batch *b);

/* Series statistics and beta derivatives of every lattice of a batch over
 * records [first, first + count), written to device memory d_out as
 * double[n][XY_STATS_FIELDS] on the batch stream (asynchronous):
 *   [0] <e>   [1] <Upsilon>   [2] <|m|>
 *   [3] d<e>/dbeta       = -cov(e_s, E_s)
 *   [4] d<Upsilon>/dbeta = -cov(Upsilon_s, E_s) - J^2 <Ix^2 + Iy^2> / (2N)
 *   [5] -cov(Upsilon_s, E_s) alone   [6] var(E_s)/N (= c_v / beta^2)   [7] count
 * with E_s = -J C_s; beta must not change inside the window (no exchange).
 * FP64 throughout (moments shifted by the window's first sample), the series
 * cut into segments across CTAs, sums in a fixed order (deterministic). */
#define XY_STATS_FIELDS 8
xy_status xy_batch_series_stats(xy_batch *b, int64_t first, int64_t count, double *d_out);
xy_status xy_batch_destroy(xy_batch *b);          /* NULL-safe */
const char *xy_batch_last_error(const xy_batch *b);

/* Unit vectors (cos, sin) of n device angles with the sweep kernels' own
 * sincos of precision `sincos_mode` (accuracy checks against CUDA and FP64):
 * d_theta, d_cos, d_sin are device arrays of n floats; runs on cuda_stream.
 * XY_SINCOS_ACCURATE takes angles in [-pi/4, 2 pi + pi/4] (the sweeps keep
 * theirs in [0, 2 pi)); the other modes any finite angle. */
xy_status xy_eval_unit_vector(int32_t sincos_mode, const float *d_theta, float *d_cos,
                              float *d_sin, int64_t n, void *cuda_stream);

/* Sweeps without any allocation, for callers that cannot allocate device
 * memory when they run (their device memory belongs to their own caching
 * allocator, they cannot afford the device-wide synchronisation of cudaFree,
 * or a run must not fail half way with out-of-memory).  The paper has no
 * counterpart; this is a deployment convenience around the fused kernel.
 *   p           parameters (start, algorithm and lattice state are not used:
 *               the sweep starts from d_angles); L must be a multiple of 128
 *               and at most 1024, else XY_EINVAL.
 *   d_angles    caller-owned device buffer of L*L floats in the split layout
 *               (as xy_create uses it), 16-byte aligned; read and rewritten:
 *               it holds the state after the last sweep on return (stream order).
 *   first_sweep Philox sweep word of the first sweep; sweeps first_sweep ..
 *               first_sweep + n_sweeps - 1 are run.
 *   d_records   caller-owned device array of n_sweeps records, cleared and filled.
 *   cuda_stream stream to enqueue on (NULL: legacy default stream).
 * The kernel's second lattice buffer is a fixed 4 MiB array inside the
 * library, held by every GPU that loads it until the process exits.  Its
 * device address is looked up on the first call on each device, so make the
 * first call on a device before any stream capture.  All calls on a device
 * share that array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Nothing here calls
 * cudaMalloc, cudaFree or an allocating library routine.  Errors are returned
 * before any work is enqueued; xy_noalloc_last_error() describes them. */
xy_status xy_sweep_noalloc(const xy_params *p, float *d_angles, uint32_t first_sweep,
                           int64_t n_sweeps, xy_record *d_records, void *cuda_stream);
const char *xy_noalloc_last_error(void);

/* ABI version (major * 100 + minor). */
int32_t xy_version(void);

#ifdef __cplusplus
}
#endif

#endif /* XY_H */
