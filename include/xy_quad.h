/*
 * xy_quad.h -- four replicas per site: the RGBA packing of Sec. 3.2 of "GPU
 * computing for 2-d spin systems: CUDA vs OpenGL", where one RGBA texel holds
 * the spins of four independent replicas of the lattice (possibly at four
 * temperatures) and the Metropolis accept is the vector select
 *     Y = z Y_new + (1 - z) Y_old,   z in {0, 1}^4.
 *
 * Here the four replicas share one float4 per site in a checkerboard-split
 * layout [colour][y][k] of float4 (k = x >> 1), so every load and store moves
 * the four replicas of a site at once, the neighbour addressing and the shared
 * staging of a half-sweep serve all four, and each thread carries four
 * independent site updates.  Replica r is exactly the single lattice of xy.h
 * with lattice id p->lattice_id + r and inverse temperature beta[r]: the same
 * Philox counters, the same per-site arithmetic and the same decisions, bit
 * for bit (its records' sums agree to the reduction's rounding).
 *
 * Conventions as in xy.h (status codes, sticky errors, stream order, natural
 * order [y][x] across the ABI, thread-compatible contexts).
 */
#ifndef XY_QUAD_H
#define XY_QUAD_H

#include <stdint.h>

#include "xy.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct xy_quad xy_quad;

#define XY_QUAD_REPLICAS 4

/* Create four replicas of side p->L (even, 2 <= L <= XY_MAX_L) and start
 * them (hot: Philox domain 0 with each replica's lattice id; cold: zero).
 *   p           L, start, J, delta, seed, sincos_mode, reduce_mode and
 *               lattice_id are used as in xy.h; p->beta is ignored.
 *               p->algorithm: XY_ALGO_FUSED -- one launch per sweep (both
 *               colours and the sums; needs L % 32 == 0; a second float4
 *               buffer, the state ping-ponging between the two);
 *               XY_ALGO_TWO_PASS -- one launch per colour, in place;
 *               XY_ALGO_PERSISTENT -- the fused sweep, all sweeps of one
 *               xy_quad_sweep call in one cooperative launch, each tile of
 *               32 rows x 16 sites starting once its eight neighbours and
 *               itself have finished the previous sweep (per-tile counters in
 *               device memory, bounded waits reported as XY_ETIMEOUT at the
 *               next synchronizing call; needs L % 32 == 0 and every CTA of
 *               the grid resident, XY_ECUDA otherwise);
 *               XY_ALGO_AUTO -- persistent where L % 32 == 0 and L <= 1024
 *               (falling back to one fused launch per sweep when the
 *               cooperative grid does not fit), fused for larger multiples of
 *               32, else two-pass.
 *               All give the same angles, accept counts and (fused and
 *               persistent) records bit for bit.
 *   beta        four inverse temperatures (>= 0, finite), one per replica.
 *   cuda_stream cudaStream_t or NULL (legacy default stream).
 * Device memory: 16 L^2 bytes per buffer (two for the fused sweep) plus
 * 8 L^2 bytes of scratch and the records.
 * Errors: XY_EINVAL (bad parameter; XY_ALGO_FUSED or _PERSISTENT with
 * L % 32 != 0),
 * XY_ENOMEM, XY_ECUDA (xy_quad_last_error(NULL)). */
xy_status xy_quad_create(const xy_params *p, const double beta[4], void *cuda_stream,
                         xy_quad **out);

/* Enqueue n_sweeps >= 0 sweeps of all four replicas (one launch per call
 * persistent, one per sweep fused, two per sweep otherwise); appends n_sweeps
 * records per replica. */
xy_status xy_quad_sweep(xy_quad *q, int64_t n_sweeps);

/* Observables of replica r's records [first, first + count), as xy_measure
 * (synchronizes). */
xy_status xy_quad_measure(xy_quad *q, int32_t replica, int64_t first, int64_t count,
                          xy_obs *host_out);

/* Replica r's angles in natural order (L*L floats) and the next sweep index.
 * Synchronizes. */
xy_status xy_quad_get_state(xy_quad *q, int32_t replica, float *host_angles,
                            uint64_t *next_sweep);

/* Records per replica so far and the next sweep index. */
xy_status xy_quad_info(const xy_quad *q, int64_t *n_records, uint64_t *next_sweep);

/* The sweep algorithm the context runs: XY_ALGO_FUSED, XY_ALGO_TWO_PASS or
 * XY_ALGO_PERSISTENT. */
xy_status xy_quad_algorithm(const xy_quad *q, int32_t *algorithm);

xy_status xy_quad_synchronize(xy_quad *q);
xy_status xy_quad_destroy(xy_quad *q);            /* NULL-safe */
const char *xy_quad_last_error(const xy_quad *q); /* thread-local message if q == NULL */

#ifdef __cplusplus
}
#endif

#endif /* XY_QUAD_H */
