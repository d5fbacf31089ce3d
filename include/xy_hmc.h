/*
 * xy_hmc.h -- C ABI of the Hybrid Monte Carlo engine for the 2-d XY model,
 * the algorithm the paper benchmarks (Sec. 1.2 of "GPU computing for 2-d
 * spin systems: CUDA vs OpenGL"): Gaussian momenta, leap-frog integration of
 * the equations of motion as the parallel core, and a global Metropolis test
 * on the change of the fictitious Hamiltonian.
 *
 *   H_hmc(theta, p) = sum_s p_s^2 / 2 + beta H(theta),
 *   H = -J sum_<ij> cos(theta_i - theta_j)                  (Eq. (1))
 *   F_s = -beta J sum_{4 nn j} sin(theta_s - theta_j)
 *
 * One trajectory with step eps and n_md steps:
 *   p = Gaussian momenta of the trajectory (see below);
 *   p += eps/2 F(theta);
 *   n_md times: theta += eps p (wrapped into [0, 2 pi)); p += eps F(theta),
 *               eps/2 instead of eps in the last kick;
 *   accept iff u < exp(-dH), dH = H_hmc(end) - H_hmc(start), else restore theta.
 *
 * Random numbers: Philox4x32-10 as in xy.h, key (seed_lo, seed_hi).  The
 * momenta of trajectory t come from counter (site, t, lattice_id, 3) by
 * Box-Muller: u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1], u2 = (w1 >> 8) 2^-24,
 * p = sqrt(-2 ln u1) cos(2 pi u2).  The test draws u = u24(w0) from counter
 * (0, t, lattice_id, 4).  The hot start is xy.h's (domain 0).
 *
 * Precision: angles and momenta FP32; the per-site terms of H_hmc and of the
 * bond/spin sums are formed in FP32 and each one is rounded to fixed point
 * before it is added (the kinetic term p^2/2 to 2^-24, the bond term of C to
 * 2^-30, the terms of Ix, Iy, Mx, My to 2^-21; sums are reported in 2^-24 and
 * 2^-30 units), so every sum is exact, deterministic and independent of the
 * launch shape; dH and the test are FP64 on the device.
 *
 * Layout: angles and momenta on the device in natural order [y][x] (L*L
 * floats each).  During a run the chain's state lives in one of three angle
 * buffers and the accept step selects which, on the device, so trajectories
 * run as one captured CUDA graph each without any host synchronisation.
 *
 * Conventions as in xy.h: every call returns an xy_status; the first error is
 * sticky in its context; work is ordered on the context's stream and
 * asynchronous device errors surface at the next synchronizing call; a
 * context is thread-compatible, not thread-safe.
 */
#ifndef XY_HMC_H
#define XY_HMC_H

#include <stdint.h>

#include "xy.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xy_hmc xy_hmc;

/* Fixed-point scale of the kinetic sums in xy_hmc_record (2^-24 units). */
#define XY_HMC_K_SHIFT 24

typedef struct {
    int32_t L;            /* side, 2 <= L <= XY_MAX_L (any L: no checkerboard)   */
    int32_t start;        /* XY_START_HOT (Philox domain 0) or XY_START_COLD     */
    double beta;          /* inverse temperature, >= 0                            */
    double J;             /* coupling (1 in the paper's model)                    */
    double eps;           /* leap-frog step, > 0                                  */
    int32_t n_md;         /* leap-frog steps per trajectory, >= 1                 */
    int32_t sincos_mode;  /* XY_SINCOS_ACCURATE, _FAST or _LIBM (force and sums) */
    uint64_t seed;        /* Philox key                                           */
    uint32_t lattice_id;  /* third Philox counter word                            */
    int32_t kernel;       /* XY_HMC_KERNEL_* (see below)                        */
} xy_hmc_params;

/* Leap-frog kernels: TILED runs one step per launch on tiles of 32 x 128 sites
 * (needs L % 128 == 0); TILED_TMA runs the full steps with a persistent grid
 * that streams each tile into double-buffered shared memory with the tensor
 * memory accelerator (needs L % 128 == 0 and the driver's tensor-map encoder;
 * begin and final launches as TILED); TILED2 runs the full steps two per
 * launch (temporal blocking: half the DRAM traffic, a recomputed halo of two;
 * where every resident CTA gets at least four tiles, L >= 4096, two CTAs per
 * SM walk the tiles and bring the next tile's rows in ahead by TMA, which
 * needs the driver's tensor-map encoder: without it one tile per CTA runs);
 * SITE is one thread per site (any L); CLUSTER runs a whole trajectory in one
 * launch of one thread-block cluster that keeps the lattice in shared memory
 * (L a power of two in [16, 256]; strips of 16 rows per CTA, neighbouring strips
 * read through distributed shared memory); PERSISTENT runs all kick-drift
 * steps of a trajectory in one cooperative launch of the TILED_TMA step, tiles
 * handed out in order and each starting once its eight neighbours and itself
 * have finished the previous step (per-tile counters in device memory, bounded
 * waits reported as XY_ETIMEOUT; needs what TILED_TMA needs and every CTA of
 * the grid resident; bit-identical, but measured slower than TILED_TMA on
 * GB300: 256 against 331 G site-steps/s at L = 4096).  AUTO takes CLUSTER for L = 128
 * and 256, else TILED_TMA when L % 128 == 0 and the encoder is available
 * (TILED if not), else SITE (the choices measured fastest on GB300: e.g.
 * TILED_TMA 51.4 us per step at L = 4096 against 57.0 for TILED and 58.3 for
 * TILED2; CLUSTER 2.8 us per step at L = 128 against 4.0 for TILED_TMA).  All
 * give bit-identical angles, momenta and sums. */
enum { XY_HMC_KERNEL_AUTO = 0, XY_HMC_KERNEL_TILED = 1, XY_HMC_KERNEL_SITE = 2,
       XY_HMC_KERNEL_TILED2 = 3, XY_HMC_KERNEL_TILED_TMA = 4, XY_HMC_KERNEL_CLUSTER = 5,
       XY_HMC_KERNEL_PERSISTENT = 6 };

/* One record per trajectory (96 bytes).
 *   sum       C, Ix, Iy, Mx, My of the state after the test (2^-30 units,
 *             definitions as in xy.h's xy_record)
 *   kinetic   sum p^2/2 at the start [0] and at the end [1] (2^-24 units)
 *   bonds     C at the start [0] and at the end [1] of the integration
 *   dH        kinetic[1]-kinetic[0] (scaled) - beta J (bonds[1]-bonds[0]) (scaled),
 *             in FP64: the value the test used
 *   beta      inverse temperature of the trajectory
 *   accepted  1 if the trajectory was accepted, else 0 */
typedef struct {
    int64_t sum[5];
    int64_t kinetic[2];
    int64_t bonds[2];
    double dH;
    double beta;
    uint64_t accepted;
} xy_hmc_record;

/* Create a context and initialise the angles (hot or cold start, trajectory 0,
 * momenta zero).
 *   p           parameters, copied and validated: L in [2, XY_MAX_L], beta >= 0
 *               and finite, J finite, eps > 0 and finite, n_md >= 1, sincos_mode
 *               and kernel valid (TILED, TILED2, TILED_TMA need L % 128 == 0,
 *               CLUSTER a power of two in [16, 256]); else XY_EINVAL.
 *   cuda_stream a cudaStream_t, or NULL for the legacy default stream.
 *   d_angles    NULL: the library allocates all three angle buffers; else a
 *               caller-owned device buffer of >= L*L floats (16-byte aligned)
 *               used as the first one.  Within a call the state moves between
 *               the three buffers; every xy_hmc_run and xy_hmc_integrate ends by
 *               moving it back into the first one (stream order), so d_angles
 *               holds the chain's state between calls.  Never freed here.
 *   out         receives the context (NULL on failure).
 * Errors: XY_EINVAL, XY_ENOMEM, XY_ECUDA (message: xy_hmc_last_error(NULL)). */
xy_status xy_hmc_create(const xy_hmc_params *p, void *cuda_stream, void *d_angles,
                        xy_hmc **out);

/* Enqueue n_traj >= 0 trajectories (one graph launch each); appends n_traj
 * records.  The trajectory counter must stay below 2^32. */
xy_status xy_hmc_run(xy_hmc *h, int64_t n_traj);

/* Integrate the current (angles, momenta) for n_steps >= 1 leap-frog steps of
 * the context's eps, with no momentum refresh, no test and no record; the
 * result becomes the current state.  For checks of the integrator (e.g.
 * against an FP64 leap-frog, or reversibility with the momenta negated). */
xy_status xy_hmc_integrate(xy_hmc *h, int32_t n_steps);

/* Draw the momenta of the current trajectory number into the momentum buffer
 * (the draw xy_hmc_run makes at the start of that trajectory). */
xy_status xy_hmc_refresh(xy_hmc *h);

/* The sums of the last trajectory or integration as doubles (synchronizes):
 * out[0..5] = K, C, Ix, Iy, Mx, My at its start, out[6..11] the same at its
 * end (K = sum p^2/2; H_hmc = K - beta J C). */
xy_status xy_hmc_last_sums(xy_hmc *h, double out[12]);

/* Calls that synchronize also check the device error word: a kernel whose
 * bounded wait for its data ran out (TILED_TMA) makes them return XY_ETIMEOUT. */

/* Observables of records [first, first + count) (synchronizes), as in
 * xy_measure: e, abs_m, upsilon, the five sums, accepted (0/1) and beta;
 * dH_out (may be NULL) receives each trajectory's dH. */
xy_status xy_hmc_measure(xy_hmc *h, int64_t first, int64_t count, xy_obs *host_out,
                         double *dH_out);

/* Raw device records (xy_hmc_record[count]); stream-ordered. */
xy_status xy_hmc_records_device(xy_hmc *h, const xy_hmc_record **d_records, int64_t *count);

/* Number of records, next trajectory number, trajectories accepted so far. */
xy_status xy_hmc_info(const xy_hmc *h, int64_t *n_records, uint64_t *next_traj,
                      uint64_t *accepted);

/* Angles (natural order, L*L floats) and momenta (may be NULL) to host memory,
 * and the next trajectory number (may be NULL).  Synchronizes. */
xy_status xy_hmc_get_state(xy_hmc *h, float *host_angles, float *host_momenta,
                           uint64_t *next_traj);

/* Replace angles (natural order; finite, else XY_ENUMERIC) and momenta (NULL:
 * zero) and set the next trajectory number (< 2^32).  Records are kept.
 * Synchronizes. */
xy_status xy_hmc_set_state(xy_hmc *h, const float *host_angles, const float *host_momenta,
                           uint64_t next_traj);

/* Change the step (eps > 0, n_md >= 1) or beta (>= 0) for later trajectories. */
xy_status xy_hmc_set_step(xy_hmc *h, double eps, int32_t n_md);
xy_status xy_hmc_set_beta(xy_hmc *h, double beta);

/* Self-test of the bounded device waits, with no GPU fault: a one-CTA kernel
 * polls (at most `polls` times, 1 <= polls <= 2^24) an mbarrier that nothing
 * ever completes, the same bounded poll the TILED_TMA kernel uses, sets an
 * error word when the bound runs out, and the host reads it back.  Returns
 * XY_ETIMEOUT when the wait ran out as it must (XY_OK would mean it did not),
 * XY_EINVAL for a bad `polls`, XY_ECUDA on a CUDA error.  Synchronizes
 * cuda_stream.  The paper has no counterpart; this exists to test the failure
 * path. */
xy_status xy_selftest_bounded_wait(void *cuda_stream, int64_t polls);

xy_status xy_hmc_synchronize(xy_hmc *h);
xy_status xy_hmc_destroy(xy_hmc *h);             /* NULL-safe */
const char *xy_hmc_last_error(const xy_hmc *h);  /* thread-local message if h == NULL */

#ifdef __cplusplus
}
#endif

#endif /* XY_HMC_H */
