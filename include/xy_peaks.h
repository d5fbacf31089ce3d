/*
 * xy_peaks.h -- instruction-rate microbenchmarks of the GPU the library runs
 * on: the measured denominators of the sweep kernels' compute roofline.
 *
 * The Metropolis sweep of the XY model (Eq. (1), red/black order) is not a
 * contraction and, on GB300, not bound by HBM either: it is bound by how fast
 * the SMs issue its integer (Philox4x32-10), FP32 (unit vectors, Delta E) and
 * special-function (exp, fast sincos) instructions.  The paper states its
 * speed-ups as gain factors over a serial CPU code (Sec. 4, Table 1) and gives
 * no device peak; these entry points measure the device's own rates so that a
 * kernel's throughput can be quoted as a fraction of a measured peak rather
 * than of a nominal one.
 *
 * Each kind runs one kernel in which every thread keeps eight independent
 * dependency chains of one instruction form (inline PTX, so the form is
 * fixed), on every SM at full occupancy, timed with CUDA events on the given
 * stream (best of `reps` launches after one warm-up launch).  The result is
 * per-thread operations per second summed over the GPU; divide by
 * (SM count x SM clock) for operations per clock per SM.
 */
#ifndef XY_PEAKS_H
#define XY_PEAKS_H

#include <stdint.h>

#include "xy.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XY_PEAK_FFMA = 0,        /* fma.rn.f32                                        */
    XY_PEAK_IMAD = 1,        /* mad.lo.u32                                        */
    XY_PEAK_IMAD_WIDE = 2,   /* mad.wide.u32, chained through the low word (the Philox
                                round's 32x32->64 product)                           */
    XY_PEAK_IMAD_HI = 3,     /* mad.hi.u32                                        */
    XY_PEAK_LOP3 = 4,        /* lop3.b32, three-input xor (the Philox round's xor)  */
    XY_PEAK_IADD = 5,        /* a + b + c: two add.u32 fused into one three-input add */
    XY_PEAK_MUFU_SIN = 6,    /* sin.approx.f32 (range scaling + MUFU.SIN)         */
    XY_PEAK_MUFU_EX2 = 7,    /* ex2.approx.ftz.f32                                */
    XY_PEAK_F2I = 8,         /* cvt.rni.s32.f32                                   */
    XY_PEAK_DFMA = 9,        /* fma.rn.f64                                        */
    XY_PEAK_ISSUE = 10,      /* 3 fma.rn.f32 : 1 lop3.b32, independent: the dispatch
                                limit of one warp instruction per scheduler and clock */
    XY_PEAK_PHILOX = 11,     /* one Philox4x32-10 block of the sweep kernels (ops = blocks) */
    XY_PEAK_UNIT_VECTOR = 12,     /* the accurate unit vector of the sweep kernels */
    XY_PEAK_UNIT_VECTOR_SFU = 13, /* __sincosf                                     */
    XY_PEAK_EXPF = 14,       /* CUDA expf, the accurate path's Boltzmann factor   */
    XY_PEAK_KINDS = 15
} xy_peak_kind;

/* Runs microbenchmark `kind` (an xy_peak_kind) with `iters` loop iterations
 * per thread (1 <= iters <= 2^20; each iteration is 8 operations per thread)
 * and `reps` timed launches (1 <= reps <= 100) on `cuda_stream` (NULL: the
 * legacy default stream), synchronizing it.  On success *ops_per_s (required)
 * receives the best launch's operations per second over the whole GPU,
 * *ms_best (optional) that launch's duration, *ops_per_launch (optional) the
 * operations one launch performs.  The sink buffer the kernels write to (so
 * that nothing is optimised away) is a small internal device array.
 * Errors: XY_EINVAL for a bad kind, iters or reps or a NULL ops_per_s;
 * XY_ECUDA when a launch or event call fails (message: xy_peak_last_error). */
xy_status xy_peak_measure(int32_t kind, int32_t iters, int32_t reps, void *cuda_stream,
                          double *ops_per_s, double *ms_best, double *ops_per_launch);

/* Thread-local message of the calling thread's last failed xy_peak_measure. */
const char *xy_peak_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* XY_PEAKS_H */
