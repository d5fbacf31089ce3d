/*
 * xy_oracle.c -- plain FP64 CPU reference ("oracle") for the checkerboard
 * Metropolis simulation of the 2-d XY model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and bench.py's CPU
 * baseline may load this code.  It shares nothing with the CUDA library: it
 * has its own Philox, its own indexing and its own observables, written
 * straight from their definitions, slow and in double precision.
 *
 * What it computes (all citations are to the paper "GPU computing for 2-d
 * spin systems: CUDA vs OpenGL"):
 *   - the model, Eq. (1): H = -J sum_<ij> cos(theta_i - theta_j) on a
 *     periodic Lx x Ly square lattice, each site bonded to its +x and +y
 *     neighbour (2N bonds; on a side of length 2 the same pair is bonded
 *     twice, exactly as the four-neighbour stencil sees it);
 *   - single-site Metropolis: propose theta' = theta + delta*(2 u0 - 1),
 *     wrapped once into [0, 2pi); accept iff u1 < exp(-beta dE) with
 *     dE = -J sum_{4 nn j} [cos(theta' - theta_j) - cos(theta - theta_j)];
 *     the accept/select of Sec. 3.2 (new = z*proposal + (1-z)*old);
 *   - the per-sweep bond and spin sums used for the cross-checks of
 *     Sec. 1.2 (energy and acceptance);
 *   - Hybrid Monte Carlo (Sec. 1.2): Gaussian momenta, leap-frog
 *     integration, global Metropolis test (last section of this file).
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.3 and Table 2), keyed
 * by the 64-bit seed (low word first) with counter (site, sweep, lattice id,
 * domain); domain 0 draws the hot start, domain 1 the Metropolis words,
 * domain 2 the replica-exchange words, domain 3 the HMC momenta and
 * domain 4 the HMC accept words.  A Metropolis block serves two sites of a
 * row, x and x + 2 with x & 2 == 0, under the counter of the first: the
 * first site takes words 0 and 1, the second words 2 and 3.  The paper fixes
 * no generator (its flat random numbers came from the host, Sec. 1.2), so
 * this layout is a reading: every word is used once per sweep, and a thread
 * that updates both sites of a pair needs one block for two updates.
 * Uniforms use the top 24 bits of a word: u = (w >> 8) * 2^-24.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the published definition.                       */
/* ------------------------------------------------------------------ */

/* Round multipliers and Weyl key increments of Philox4x32 (SC'11, Table 2
 * and Sec. 3.3). */
static const uint32_t PHILOX_MULT_A = 0xD2511F53u;
static const uint32_t PHILOX_MULT_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {           /* key schedule: bump before rounds 2..10 */
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        /* the S-box: two 32x32 -> 64 products, halves swapped and xored */
        uint64_t prod_a = (uint64_t)PHILOX_MULT_A * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)PHILOX_MULT_B * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The four words drawn for one (site, sweep, lattice, domain). */
static void site_words(uint64_t seed, uint32_t site, uint32_t sweep,
                       uint32_t lattice_id, uint32_t domain, uint32_t w[4])
{
    uint32_t ctr[4] = { site, sweep, lattice_id, domain };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, w);
}

/* Exact 24-bit uniform in [0, 1). */
static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* Fill n x 4 words for counters (first + i, sweep, lattice_id, domain). */
void orc_philox_words(uint64_t seed, uint32_t sweep, uint32_t lattice_id,
                      uint32_t domain, uint32_t first, int64_t n, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        site_words(seed, first + (uint32_t)i, sweep, lattice_id, domain, out + 4 * i);
}

/* ------------------------------------------------------------------ */
/* Lattice geometry (natural order s = y*Lx + x, periodic).            */
/* ------------------------------------------------------------------ */

static int64_t site_right(int Lx, int64_t s) { int64_t x = s % Lx; return s - x + (x + 1) % Lx; }
static int64_t site_left (int Lx, int64_t s) { int64_t x = s % Lx; return s - x + (x + Lx - 1) % Lx; }
static int64_t site_up   (int Lx, int Ly, int64_t s)
{
    int64_t y = s / Lx, x = s % Lx;
    return ((y + 1) % Ly) * Lx + x;
}
static int64_t site_down (int Lx, int Ly, int64_t s)
{
    int64_t y = s / Lx, x = s % Lx;
    return ((y + Ly - 1) % Ly) * Lx + x;
}

/* ------------------------------------------------------------------ */
/* Observables: bond and spin sums of one configuration (FP64).        */
/* out = { C, Ix, Iy, Mx, My } with                                    */
/*   C  = sum_s cos(t_s - t_{s+x}) + cos(t_s - t_{s+y})   (2N bonds)   */
/*   Ix = sum_s sin(t_s - t_{s+x}),  Iy = sum_s sin(t_s - t_{s+y})     */
/*   Mx = sum_s cos t_s,             My = sum_s sin t_s                */
/* e = -J C / N, |m| = |M| / N, Upsilon = (J C - beta J^2 (Ix^2+Iy^2))/(2N) */
/* ------------------------------------------------------------------ */
void orc_measure(int Lx, int Ly, const double *theta, double out[5])
{
    int64_t N = (int64_t)Lx * Ly;
    double C = 0, Ix = 0, Iy = 0, Mx = 0, My = 0;
    for (int64_t s = 0; s < N; ++s) {
        double t = theta[s];
        double tx = theta[site_right(Lx, s)];
        double ty = theta[site_up(Lx, Ly, s)];
        C  += cos(t - tx) + cos(t - ty);
        Ix += sin(t - tx);
        Iy += sin(t - ty);
        Mx += cos(t);
        My += sin(t);
    }
    out[0] = C; out[1] = Ix; out[2] = Iy; out[3] = Mx; out[4] = My;
}

/* Energy change of moving site s from theta[s] to theta_new, from the
 * four-neighbour stencil (the quantity the Metropolis test uses). */
double orc_delta_energy(int Lx, int Ly, const double *theta, int64_t s,
                        double theta_new, double J)
{
    int64_t nb[4] = { site_right(Lx, s), site_left(Lx, s),
                      site_up(Lx, Ly, s), site_down(Lx, Ly, s) };
    double old = theta[s], dE = 0.0;
    for (int k = 0; k < 4; ++k) {
        double tj = theta[nb[k]];
        dE -= J * (cos(theta_new - tj) - cos(old - tj));
    }
    return dE;
}

/* ------------------------------------------------------------------ */
/* Start configurations.                                               */
/* ------------------------------------------------------------------ */

/* Hot start: theta_s = 2 pi u24(w0), words of domain 0, sweep 0.
 * Cold start (hot == 0): all angles zero. */
void orc_start(int Lx, int Ly, uint64_t seed, uint32_t lattice_id, int hot,
               double *theta)
{
    int64_t N = (int64_t)Lx * Ly;
    for (int64_t s = 0; s < N; ++s) {
        if (!hot) { theta[s] = 0.0; continue; }
        uint32_t w[4];
        site_words(seed, (uint32_t)s, 0u, lattice_id, 0u, w);
        theta[s] = ORC_TWO_PI * u24(w[0]);
    }
}

/* ------------------------------------------------------------------ */
/* One Metropolis attempt at site s against `theta` (not modified).    */
/* ------------------------------------------------------------------ */
typedef struct {
    double theta_prop;   /* proposed angle, wrapped into [0, 2pi)        */
    double u1;           /* accept uniform                               */
    double p;            /* exp(-beta dE)                                */
    int accept;          /* u1 < p                                       */
} orc_step;

static orc_step attempt(int Lx, int Ly, const double *theta, int64_t s,
                        double beta, double J, double delta, uint64_t seed,
                        uint32_t lattice_id, uint32_t sweep)
{
    /* the block of the pair (x - (x & 2), x - (x & 2) + 2) in row y */
    int64_t x = s % Lx;
    int upper = (x & 2) != 0;
    uint32_t w[4];
    site_words(seed, (uint32_t)(s - (x & 2)), sweep, lattice_id, 1u, w);
    double u0 = u24(w[2 * upper]);
    orc_step st;
    st.u1 = u24(w[2 * upper + 1]);
    double prop = theta[s] + delta * (2.0 * u0 - 1.0);
    if (prop < 0.0) prop += ORC_TWO_PI;
    else if (prop >= ORC_TWO_PI) prop -= ORC_TWO_PI;
    st.theta_prop = prop;
    double dE = orc_delta_energy(Lx, Ly, theta, s, prop, J);
    st.p = exp(-beta * dE);
    st.accept = st.u1 < st.p;
    return st;
}

/* Evaluate the Metropolis step of sweep `sweep` at each listed site against
 * the given state, without applying it.  Any output pointer may be NULL. */
void orc_attempt_sites(int Lx, int Ly, const double *theta, const int64_t *sites,
                       int64_t n, double beta, double J, double delta,
                       uint64_t seed, uint32_t lattice_id, uint32_t sweep,
                       int nthreads, double *theta_prop, double *u1, double *p,
                       uint8_t *accept)
{
#ifdef _OPENMP
    #pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t i = 0; i < n; ++i) {
        orc_step st = attempt(Lx, Ly, theta, sites[i], beta, J, delta, seed,
                              lattice_id, sweep);
        if (theta_prop) theta_prop[i] = st.theta_prop;
        if (u1) u1[i] = st.u1;
        if (p) p[i] = st.p;
        if (accept) accept[i] = (uint8_t)st.accept;
    }
    (void)nthreads;
}

/* Half-sweep of colour c ((x + y) mod 2 == c): every site of that colour
 * attempts one move against the same neighbours (they are all of the other
 * colour), then the accepted moves are applied.  Per-site outputs (indexed
 * by natural site id, NULL allowed) let a test compare each decision.
 * Returns the number of accepted moves. */
int64_t orc_half_sweep(int Lx, int Ly, double *theta, int colour, double beta,
                       double J, double delta, uint64_t seed, uint32_t lattice_id,
                       uint32_t sweep, int nthreads, double *theta_prop,
                       double *u1, double *p, uint8_t *accept)
{
    int64_t N = (int64_t)Lx * Ly;
    double *next = (double *)malloc(sizeof(double) * (size_t)N);
    if (!next) return -1;
    memcpy(next, theta, sizeof(double) * (size_t)N);
    int64_t count = 0;
#ifdef _OPENMP
    #pragma omp parallel for schedule(static) reduction(+:count) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t s = 0; s < N; ++s) {
        int64_t x = s % Lx, y = s / Lx;
        if ((int)((x + y) & 1) != colour) continue;
        orc_step st = attempt(Lx, Ly, theta, s, beta, J, delta, seed,
                              lattice_id, sweep);
        if (theta_prop) theta_prop[s] = st.theta_prop;
        if (u1) u1[s] = st.u1;
        if (p) p[s] = st.p;
        if (accept) accept[s] = (uint8_t)st.accept;
        /* Sec. 3.2 select: new = z * proposal + (1 - z) * old, z in {0, 1} */
        next[s] = st.accept ? st.theta_prop : theta[s];
        count += st.accept;
    }
    (void)nthreads;
    memcpy(theta, next, sizeof(double) * (size_t)N);
    free(next);
    return count;
}

/* One full sweep.  order 0: checkerboard (colour 0 then colour 1; needs even
 * Lx and Ly).  order 1: typewriter (sites in natural order, each move applied
 * at once).  Returns the number of accepted moves, or -1 on bad input. */
int64_t orc_sweep(int Lx, int Ly, double *theta, double beta, double J,
                  double delta, uint64_t seed, uint32_t lattice_id,
                  uint32_t sweep, int order, int nthreads)
{
    if (order == 0) {
        if ((Lx & 1) || (Ly & 1)) return -1;
        int64_t a = orc_half_sweep(Lx, Ly, theta, 0, beta, J, delta, seed,
                                   lattice_id, sweep, nthreads, NULL, NULL, NULL, NULL);
        int64_t b = orc_half_sweep(Lx, Ly, theta, 1, beta, J, delta, seed,
                                   lattice_id, sweep, nthreads, NULL, NULL, NULL, NULL);
        if (a < 0 || b < 0) return -1;
        return a + b;
    }
    int64_t N = (int64_t)Lx * Ly, count = 0;
    for (int64_t s = 0; s < N; ++s) {
        orc_step st = attempt(Lx, Ly, theta, s, beta, J, delta, seed,
                              lattice_id, sweep);
        if (st.accept) { theta[s] = st.theta_prop; ++count; }
    }
    return count;
}

/* Free-running chain: start (hot != 0: Philox hot start; 0: cold), then
 * n_sweeps sweeps numbered first_sweep, first_sweep + 1, ...  After each
 * sweep, records[6*i .. 6*i+5] = { C, Ix, Iy, Mx, My, accepted }.
 * If theta_io is non-NULL and start < 0, the chain starts from theta_io;
 * the final state is written back to theta_io when it is non-NULL. */
int orc_run(int Lx, int Ly, uint64_t seed, uint32_t lattice_id, double beta,
            double J, double delta, int start, int order, uint32_t first_sweep,
            int64_t n_sweeps, int nthreads, double *theta_io, double *records)
{
    int64_t N = (int64_t)Lx * Ly;
    double *theta = (double *)malloc(sizeof(double) * (size_t)N);
    if (!theta) return -1;
    if (start < 0) {
        if (!theta_io) { free(theta); return -1; }
        memcpy(theta, theta_io, sizeof(double) * (size_t)N);
    } else {
        orc_start(Lx, Ly, seed, lattice_id, start, theta);
    }
    for (int64_t i = 0; i < n_sweeps; ++i) {
        int64_t acc = orc_sweep(Lx, Ly, theta, beta, J, delta, seed, lattice_id,
                                first_sweep + (uint32_t)i, order, nthreads);
        if (acc < 0) { free(theta); return -1; }
        if (records) {
            orc_measure(Lx, Ly, theta, records + 6 * i);
            records[6 * i + 5] = (double)acc;
        }
    }
    if (theta_io) memcpy(theta_io, theta, sizeof(double) * (size_t)N);
    free(theta);
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Replica exchange (parallel tempering) between neighbouring          */
/* temperatures of a ladder.                                           */
/* ------------------------------------------------------------------ */

/* One exchange step.  Ladder l owns slots [ladder_start[l], ladder_start[l+1])
 * (the last ladder ends at n_slots); slot s holds lattice pos_lattice[s] at
 * temperature pos_beta[s] (ascending within a ladder).  In round r the pairs
 * of positions (p, p+1) with p = r mod 2, r mod 2 + 2, ... are tried: with
 * E = energy[lattice] (-J C of its last sweep) and w the Philox words of
 * counter (l * 65536 + p, r, lattice_id0, 2), the two lattices trade
 * temperatures iff u24(w0) < exp((beta_p - beta_{p+1}) (E_p - E_{p+1})),
 * the Metropolis rule for swapping two replicas.  beta_of_lattice and
 * pos_lattice are updated; swapped[slot] = 1 for the lower slot of a swap. */
void orc_exchange(int n_ladders, const int *ladder_start, int n_slots, int *pos_lattice,
                  const double *pos_beta, double *beta_of_lattice, const double *energy,
                  uint32_t round, uint64_t seed, uint32_t lattice_id0, uint8_t *swapped)
{
    for (int s = 0; s < n_slots; ++s) if (swapped) swapped[s] = 0;
    for (int l = 0; l < n_ladders; ++l) {
        int begin = ladder_start[l];
        int end = (l + 1 < n_ladders) ? ladder_start[l + 1] : n_slots;
        for (int p = (int)(round & 1u); begin + p + 1 < end; p += 2) {
            int a = pos_lattice[begin + p], b = pos_lattice[begin + p + 1];
            double ba = pos_beta[begin + p], bb = pos_beta[begin + p + 1];
            uint32_t w[4];
            site_words(seed, (uint32_t)l * 65536u + (uint32_t)p, round, lattice_id0, 2u, w);
            if (u24(w[0]) < exp((ba - bb) * (energy[a] - energy[b]))) {
                pos_lattice[begin + p] = b;
                pos_lattice[begin + p + 1] = a;
                beta_of_lattice[b] = ba;
                beta_of_lattice[a] = bb;
                if (swapped) swapped[begin + p] = 1;
            }
        }
    }
}

/* Parallel tempering of one ladder of n equal Lx x Ly lattices (checkerboard
 * sweeps): lattice i starts hot with lattice id lattice_id0 + i at beta[i]
 * (ascending); every round it runs sweeps_per_round sweeps at its current
 * temperature, then one exchange step (round r) on the energies of the last
 * sweep.  records[(i * total + t) * 7 + 0..6] = C, Ix, Iy, Mx, My, accepted,
 * beta after sweep t of lattice i, total = rounds * sweeps_per_round. */
int orc_pt_run(int Lx, int Ly, int n, const double *beta, double J, double delta,
               uint64_t seed, uint32_t lattice_id0, int sweeps_per_round, int rounds,
               double *records)
{
    int64_t N = (int64_t)Lx * Ly;
    int64_t total = (int64_t)rounds * sweeps_per_round;
    double *theta = (double *)malloc(sizeof(double) * (size_t)(N * n));
    double *bl = (double *)malloc(sizeof(double) * (size_t)n);
    double *energy = (double *)malloc(sizeof(double) * (size_t)n);
    int *pos = (int *)malloc(sizeof(int) * (size_t)n);
    int start0 = 0;
    if (!theta || !bl || !energy || !pos) {
        free(theta); free(bl); free(energy); free(pos);
        return -1;
    }
    for (int i = 0; i < n; ++i) {
        orc_start(Lx, Ly, seed, lattice_id0 + (uint32_t)i, 1, theta + N * i);
        bl[i] = beta[i];
        pos[i] = i;
    }
    for (int r = 0; r < rounds; ++r) {
        for (int i = 0; i < n; ++i) {
            for (int k = 0; k < sweeps_per_round; ++k) {
                int64_t t = (int64_t)r * sweeps_per_round + k;
                int64_t acc = orc_sweep(Lx, Ly, theta + N * i, bl[i], J, delta, seed,
                                        lattice_id0 + (uint32_t)i, (uint32_t)t, 0, 1);
                if (acc < 0) {
                    free(theta); free(bl); free(energy); free(pos);
                    return -1;
                }
                double *rec = records + (i * total + t) * 7;
                orc_measure(Lx, Ly, theta + N * i, rec);
                rec[5] = (double)acc;
                rec[6] = bl[i];
                if (k == sweeps_per_round - 1) energy[i] = -J * rec[0];
            }
        }
        orc_exchange(1, &start0, n, pos, beta, bl, energy, (uint32_t)r, seed, lattice_id0, NULL);
    }
    free(theta); free(bl); free(energy); free(pos);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Hybrid Monte Carlo, the method of Sec. 1.2: Gaussian momenta, the   */
/* leap-frog integration of the equations of motion, and a global      */
/* Metropolis test on the change of the fictitious Hamiltonian.        */
/*                                                                     */
/*   H_hmc(theta, p) = sum_s p_s^2 / 2 + beta H(theta)                 */
/*   F_s = -d(beta H)/d theta_s = -beta J sum_{4 nn j} sin(t_s - t_j)  */
/*                                                                     */
/* The paper does not fix the step size, the number of steps or the    */
/* Gaussian transform; here the momenta of trajectory t come from the  */
/* words of domain 3, counter (site, t, lattice id, 3), by Box-Muller: */
/*   u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1],  u2 = (w1 >> 8) 2^-24,      */
/*   p = sqrt(-2 ln u1) cos(2 pi u2),                                  */
/* and the test uses u = u24(w0) of counter (0, t, lattice id, 4):     */
/* accept iff u < exp(-dH).  Angles are wrapped into [0, 2pi) after    */
/* every drift (H depends only on angle differences mod 2pi).          */
/* ------------------------------------------------------------------ */

static double wrap_2pi(double t)
{
    double w = t - ORC_TWO_PI * floor(t / ORC_TWO_PI);
    if (w >= ORC_TWO_PI) w -= ORC_TWO_PI;   /* floor rounding at the edge */
    if (w < 0.0) w += ORC_TWO_PI;
    return w;
}

void orc_hmc_momenta(int Lx, int Ly, uint64_t seed, uint32_t traj, uint32_t lattice_id,
                     double *p)
{
    int64_t N = (int64_t)Lx * Ly;
    for (int64_t s = 0; s < N; ++s) {
        uint32_t w[4];
        site_words(seed, (uint32_t)s, traj, lattice_id, 3u, w);
        double u1 = (double)((w[0] >> 8) + 1u) * (1.0 / 16777216.0);
        double u2 = u24(w[1]);
        p[s] = sqrt(-2.0 * log(u1)) * cos(ORC_TWO_PI * u2);
    }
}

/* F_s = -beta J sum over the four neighbours of sin(theta_s - theta_j). */
void orc_hmc_force(int Lx, int Ly, const double *theta, double beta, double J, double *F)
{
    int64_t N = (int64_t)Lx * Ly;
    for (int64_t s = 0; s < N; ++s) {
        int64_t nb[4] = { site_right(Lx, s), site_left(Lx, s),
                          site_up(Lx, Ly, s), site_down(Lx, Ly, s) };
        double f = 0.0;
        for (int k = 0; k < 4; ++k) f -= sin(theta[s] - theta[nb[k]]);
        F[s] = beta * J * f;
    }
}

/* out = { K, V } with K = sum p^2 / 2 and V = beta H(theta) = -beta J C. */
void orc_hmc_hamiltonian(int Lx, int Ly, const double *theta, const double *p, double beta,
                         double J, double out[2])
{
    int64_t N = (int64_t)Lx * Ly;
    double K = 0.0, sums[5];
    for (int64_t s = 0; s < N; ++s) K += 0.5 * p[s] * p[s];
    orc_measure(Lx, Ly, theta, sums);
    out[0] = K;
    out[1] = -beta * J * sums[0];
}

/* n_steps leap-frog steps of size eps, in place:
 *   p += eps/2 F(theta);
 *   repeat n_steps times: theta += eps p (wrapped); p += eps F(theta),
 *   with eps/2 instead of eps in the last kick.
 * n_steps = 0 leaves both arrays unchanged.  Returns 0, or -1 on no memory. */
int orc_hmc_leapfrog(int Lx, int Ly, double *theta, double *p, double beta, double J,
                     double eps, int n_steps)
{
    int64_t N = (int64_t)Lx * Ly;
    if (n_steps <= 0) return 0;
    double *F = (double *)malloc(sizeof(double) * (size_t)N);
    if (!F) return -1;
    orc_hmc_force(Lx, Ly, theta, beta, J, F);
    for (int64_t s = 0; s < N; ++s) p[s] += 0.5 * eps * F[s];
    for (int k = 1; k <= n_steps; ++k) {
        for (int64_t s = 0; s < N; ++s) theta[s] = wrap_2pi(theta[s] + eps * p[s]);
        orc_hmc_force(Lx, Ly, theta, beta, J, F);
        double h = (k == n_steps) ? 0.5 * eps : eps;
        for (int64_t s = 0; s < N; ++s) p[s] += h * F[s];
    }
    free(F);
    return 0;
}

/* One trajectory from `theta` (in place): draw the momenta of trajectory
 * `traj`, integrate, test.  On rejection theta is restored.  out =
 * { dH, accepted, K0, V0, K1, V1 }.  If p_out is non-NULL it receives the
 * momenta at the end of the integration.  Returns 0 or -1. */
int orc_hmc_trajectory(int Lx, int Ly, double *theta, double beta, double J, double eps,
                       int n_steps, uint64_t seed, uint32_t traj, uint32_t lattice_id,
                       double out[6], double *p_out)
{
    int64_t N = (int64_t)Lx * Ly;
    double *p = (double *)malloc(sizeof(double) * (size_t)N);
    double *theta0 = (double *)malloc(sizeof(double) * (size_t)N);
    if (!p || !theta0) { free(p); free(theta0); return -1; }
    orc_hmc_momenta(Lx, Ly, seed, traj, lattice_id, p);
    memcpy(theta0, theta, sizeof(double) * (size_t)N);
    double h0[2], h1[2];
    orc_hmc_hamiltonian(Lx, Ly, theta, p, beta, J, h0);
    if (orc_hmc_leapfrog(Lx, Ly, theta, p, beta, J, eps, n_steps) != 0) {
        free(p); free(theta0);
        return -1;
    }
    orc_hmc_hamiltonian(Lx, Ly, theta, p, beta, J, h1);
    double dH = (h1[0] + h1[1]) - (h0[0] + h0[1]);
    uint32_t w[4];
    site_words(seed, 0u, traj, lattice_id, 4u, w);
    int accepted = u24(w[0]) < exp(-dH);
    if (!accepted) memcpy(theta, theta0, sizeof(double) * (size_t)N);
    if (p_out) memcpy(p_out, p, sizeof(double) * (size_t)N);
    out[0] = dH; out[1] = (double)accepted;
    out[2] = h0[0]; out[3] = h0[1]; out[4] = h1[0]; out[5] = h1[1];
    free(p); free(theta0);
    return 0;
}

/* A chain of n_traj trajectories numbered first_traj, first_traj + 1, ...
 * from a hot (start = 1) or cold (0) start, or from theta_io (start < 0).
 * After trajectory i, records[7*i .. 7*i+6] = { C, Ix, Iy, Mx, My, dH,
 * accepted } of the state after the test.  The final state goes back to
 * theta_io when it is non-NULL. */
int orc_hmc_run(int Lx, int Ly, uint64_t seed, uint32_t lattice_id, double beta, double J,
                double eps, int n_steps, int start, uint32_t first_traj, int64_t n_traj,
                double *theta_io, double *records)
{
    int64_t N = (int64_t)Lx * Ly;
    double *theta = (double *)malloc(sizeof(double) * (size_t)N);
    if (!theta) return -1;
    if (start < 0) {
        if (!theta_io) { free(theta); return -1; }
        memcpy(theta, theta_io, sizeof(double) * (size_t)N);
    } else {
        orc_start(Lx, Ly, seed, lattice_id, start, theta);
    }
    for (int64_t i = 0; i < n_traj; ++i) {
        double o[6];
        if (orc_hmc_trajectory(Lx, Ly, theta, beta, J, eps, n_steps, seed,
                               first_traj + (uint32_t)i, lattice_id, o, NULL) != 0) {
            free(theta);
            return -1;
        }
        if (records) {
            orc_measure(Lx, Ly, theta, records + 7 * i);
            records[7 * i + 5] = o[0];
            records[7 * i + 6] = o[1];
        }
    }
    if (theta_io) memcpy(theta_io, theta, sizeof(double) * (size_t)N);
    free(theta);
    return 0;
}
