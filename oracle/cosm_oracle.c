/*
 * Plain FP64 CPU oracle of Cosm (Collective Switched Motion).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the bench may load this library. It shares no code, header, table or
 * helper with the CUDA path.
 *
 * It follows the paper's statement of the method step by step, in the
 * paper's order, without blocking, fusion or reordering:
 *   - Ising/Max-Cut form: eq. (1) and Appendix A (w_ij = -J_ij).
 *   - Circular variables: x_i in [0, 360) degrees, held here in turns
 *     (x_turn = x_deg / 360), modular updates (Section II-A).
 *   - Pair update: eqs. (4)-(6), applied to the minimum angular difference
 *     (Fig. 1 caption), with the biased sign of eq. (4).
 *   - Sequential conflict-free search: eqs. (9)-(12), colours in order.
 *   - Dual window twist: Section II-D and Alg. 1 (every DWTperiod sweeps).
 *   - Step schedule: linear ramp alpha_0 -> 0, constant within a sweep
 *     (Section II-B, Appendix B, Table IX).
 *   - Binarization with equally spaced bisectors over a semicircle and the
 *     best cut (Alg. 1, Appendix B: 100 bisectors spaced 1.8 degrees).
 *   - Greedy edge colouring (Section II-B) and the regular lattice pattern.
 *   - Local fields h of eq. (1), the fixed-semicircle readout and a random
 *     twist direction (Sections II-A, II-B, II-D); the optimal bisector
 *     (Section II-B, after Burer, Monteiro and Zhang 2002); mid-anneal
 *     readouts with best tracking and an energy trace (Fig. 10).
 * Readings taken where the paper is silent are listed with each function.
 *
 * Random numbers: Philox4x32-10 written from Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of the 4x32 Philox S-box    */
/* with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments          */
/* 0x9E3779B9 / 0xBB67AE85 (golden ratio and sqrt(3)-1).                     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24-bit uniform in [0,1): top 24 bits of a Philox word, exact in FP32. */
static double orc_u24(uint32_t word) { return (double)(word >> 8) * 0x1p-24; }

/* Random initial state (Alg. 1 "Set x_i random"): key = (seed low, seed
 * high), counter = (vertex/4, replica, 0, 0); vertex v takes word v mod 4. */
void orc_init_phases(int32_t n, uint64_t seed, int64_t replica, double *x)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t v = 0; v < n; ++v) {
        uint32_t ctr[4] = {(uint32_t)(v >> 2), (uint32_t)replica, 0u, 0u};
        uint32_t o[4];
        orc_philox4x32_10(ctr, key, o);
        x[v] = orc_u24(o[v & 3]);
    }
}

/* DWT reference angle theta_ref for sweep s of a replica (Alg. 1: "Select
 * random reference angle"; Section II-E: one global random value per DWT
 * event): key = seed, counter = (s, replica, 0, 1); theta = top 24 bits of
 * word 0, in turns. */
double orc_theta(uint64_t seed, int64_t replica, int64_t sweep)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)sweep, (uint32_t)replica, 0u, 1u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return orc_u24(o[0]);
}

/* Step schedule (Section II-B; Table IX: initial alpha_0, final 0; updated
 * once per sweep, constant within it). Reading: alpha_s = alpha_0 (S-s)/(S-1)
 * for s = 1..S, so alpha_1 = alpha_0 and alpha_S = 0; a single-sweep run
 * uses alpha_0. */
double orc_alpha(int64_t s, int64_t S, double alpha0)
{
    if (S <= 1) return alpha0;
    return alpha0 * (double)(S - s) / (double)(S - 1);
}

/* Modular wrap onto [0,1) (Section II-A: "updates use modular arithmetic").
 * A result that rounds to 1.0 is the same point as 0.0 and becomes 0.0. */
double orc_wrap(double y)
{
    double r = y - floor(y);
    if (r >= 1.0) r = 0.0;
    return r;
}

/* Biased sign of eq. (4) applied to the minimum angular difference
 * (Fig. 1 caption): d = ((x_i - x_j + 1/2) mod 1) - 1/2 in [-1/2, 1/2);
 * +1 when d >= 0, -1 when d < 0. Equivalently +1 iff frac(x_i - x_j) < 1/2.
 * Exactly opposite points (d = -1/2) give -1. */
int orc_sgn_b(double xi, double xj)
{
    double f = (xi - xj) - floor(xi - xj);
    return (f < 0.5) ? 1 : -1;
}

/* Distance of the minimum angular difference from the two switching points
 * of eq. (4), d = 0 and d = -1/2; used to flag near-ties, where an FP32 and
 * an FP64 evaluation may legitimately take different branches. */
static double orc_tie_distance(double xi, double xj)
{
    double f = (xi - xj) - floor(xi - xj); /* in [0,1] */
    double a = fabs(f);
    double b = fabs(f - 0.5);
    double c = fabs(f - 1.0);
    double m = a < b ? a : b;
    return m < c ? m : c;
}

/* IEEE 754 binary16 round-to-nearest-even of a value with |y| <= 1/2:
 * 10 fraction bits in normal binades (exponent >= -14), quantum 2^-24 in
 * the subnormal range. */
double orc_round_binary16(double y)
{
    if (y == 0.0) return y;
    int E;
    frexp(y, &E);             /* |y| = f 2^E, f in [1/2, 1): binade exponent E-1 */
    int e = E - 1;
    if (e < -14) e = -14;     /* subnormals share the quantum of the lowest binade */
    double q = ldexp(1.0, e - 10);
    return nearbyint(y / q) * q; /* default rounding mode: to nearest, ties to even */
}

/* bfloat16 round-to-nearest-even of a value with |y| <= 1/2: 8 significant
 * bits (7 fraction bits), the exponent range of binary32 (no subnormal
 * quanta arise at these magnitudes above 2^-126). */
double orc_round_bfloat16(double y)
{
    if (y == 0.0) return y;
    int E;
    frexp(y, &E);             /* |y| = f 2^E, f in [1/2, 1): binade exponent E-1 */
    int e = E - 1;
    if (e < -126) e = -126;
    double q = ldexp(1.0, e - 7);
    return nearbyint(y / q) * q;
}

/* Fixed-point phases (storage 2): phases live on the grid of 2^-16 turn
 * and every step is rounded to that grid, a step a becoming
 * floor(a 2^16 + 1/2) 2^-16; sums and differences of grid values are then
 * exact in FP64, so the dynamics are exact integer arithmetic mod 2^16. */
static double orc_q16_step(double a) { return floor(a * 65536.0 + 0.5) / 65536.0; }

/* Storage rounding: 0 = none (FP64), 1 = binary16 of the phase's
 * representative in [-1/2, 1/2), 2 = fixed point (values already on the
 * grid), 3 = bfloat16 of the representative; 4 and 5 round as 1 and 3 (they
 * differ from them only in when a sweep rounds, orc_sweep_h). The result is
 * returned in [0,1). */
static double orc_store(double x, int32_t storage)
{
    if (storage != 1 && storage != 3 && storage != 4 && storage != 5) return x;
    double g = (x >= 0.5) ? x - 1.0 : x;
    g = (storage == 1 || storage == 4) ? orc_round_binary16(g) : orc_round_bfloat16(g);
    g = (g < 0.0) ? g + 1.0 : g;
    return g >= 1.0 ? 0.0 : g;
}

/* Dual-window membership (Section II-D, Alg. 1): two windows of width W
 * (turns) centred at theta and theta + 1/2, half-open [c - W/2, c + W/2).
 * Evaluated exactly on q = floor(x 2^32), qt = theta 2^32:
 *   ((q - qt + QW/2) mod 2^31) < QW,   QW = round(W 2^32).
 * Returns 1 inside, 0 outside; *dist gets the distance (turns) to the
 * nearest window edge. */
static int orc_in_window(double x, double theta, double W, double *dist)
{
    uint64_t QW = (uint64_t)floor(W * 4294967296.0 + 0.5);
    uint64_t Qh = QW >> 1;
    uint32_t q = (uint32_t)(uint64_t)floor(x * 4294967296.0);
    uint32_t qt = (uint32_t)(uint64_t)floor(theta * 4294967296.0);
    uint32_t rel = (uint32_t)(q - qt + (uint32_t)Qh) & 0x7FFFFFFFu;
    if (dist) {
        double r = (double)rel * 0x1p-32;           /* in [0, 1/2) */
        double w = (double)QW * 0x1p-32;
        double d1 = fabs(r - w), d2 = fabs(r), d3 = fabs(0.5 - r);
        double m = d1 < d2 ? d1 : d2;
        *dist = m < d3 ? m : d3;
    }
    return (uint64_t)rel < QW ? 1 : 0;
}

int orc_in_window_q(double x, double theta, double W) { return orc_in_window(x, theta, W, 0); }

#define ORC_NO_DWT 1
#define ORC_NO_SCS 2
#define ORC_DWT_RANDDIR 4
#define ORC_OPT_BISECTOR 8

/* Twist direction of the DWT event of sweep s of a replica when it is
 * randomised (Section II-D allows either direction): word 1 of the Philox
 * draw that gives theta_ref (counter (s, replica, 0, 1)); +1 when its top
 * bit is clear, -1 when set. */
int orc_twist_dir(uint64_t seed, int64_t replica, int64_t sweep)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)sweep, (uint32_t)replica, 0u, 1u};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return (o[1] >> 31) ? -1 : 1;
}

/*
 * One sweep of Alg. 1 on one replica, in place.
 *   Colour-major edge lists: colour c owns edges [off[c], off[c+1]); each
 *   edge (src < dst) with Max-Cut weight w = -J (Appendix A).
 *   Pair update, eq. (6) with J = -w, in turns:
 *     s = sgn_b(x_i - x_j);  x_i <- wrap(x_i - alpha J s);  x_j <- wrap(x_j + alpha J s)
 *   Sub-sweeps in colour order 1..C (eqs. (11)-(12)); edges of one colour are
 *   a matching, so their order inside the colour does not matter.
 *   With flag NO_SCS the sweep is one simultaneous generalized-gradient step
 *   over all edges (eq. (8)), the ablation "without SCS" of Table VII.
 *   Then, when sweep % dwt_period == 0 and DWT is on, every phase inside the
 *   dual windows moves by +dwt_ratio * alpha (Section II-D; one direction).
 * Local fields h (eq. (1); NULL = none). Reading: a field is a coupling
 * J = h_v to a reference variable frozen at 0, so it acts through the same
 * pair rule, eq. (6), on x_v alone. Its updates touch each vertex once and
 * the reference never moves, so together they form one more conflict-free
 * sub-sweep, taken after the C colours and before the DWT (with NO_SCS the
 * field forces join the simultaneous step).
 * With flag DWT_RANDDIR the twist direction of each DWT event is drawn
 * (orc_twist_dir) instead of always +1 (Section II-D).
 * storage: 0 FP64, 1 binary16 storage rounding, 2 fixed point on the
 * 2^-16-turn grid (alpha and the twist rounded to the grid), 3 bfloat16
 * storage rounding; modes 1 and 3 round every phase write (each pair update,
 * each twist move). Modes 4 (binary16) and 5 (bfloat16) store once per pass
 * of two consecutive colours instead: the phases stay unrounded inside a
 * pass and every phase is rounded when it ends, after colours 2, 4, ... and
 * at the end of the sweep; the last pass takes the field sub-sweep and the
 * twist, when due, before its rounding. (The paper fixes no phase storage
 * format; Section II-E only says that no double precision is needed. The
 * 16-bit storage forms are readings of that: a stored phase is rounded,
 * arithmetic stays exact between stores.)
 * Near-ties: an edge whose angular difference is within tie_eps of 0 or 1/2
 * when processed, a phase within tie_eps of a window edge, and a phase with
 * a field within tie_eps of 0 or 1/2, are recorded in ties[] (edge e as e,
 * DWT vertex v as m + v, field vertex v as m + n + v). force[], when given,
 * has m + n entries (m + 2n with fields): 0 = natural branch, +1/-1 = forced
 * sign (edges, fields) or forced inside/outside (DWT vertices).
 * Returns the number of near-ties found (ties[] holds at most max_ties).
 */
int64_t orc_sweep_h(int32_t n, int32_t C, const int64_t *off, const int32_t *src,
                    const int32_t *dst, const int32_t *w, const int32_t *h, double *x, double alpha,
                    int64_t sweep, int32_t dwt_period, double dwt_ratio, double window,
                    uint64_t seed, int64_t replica, int32_t flags, int32_t storage,
                    const int8_t *force, double tie_eps, int64_t *ties, int64_t max_ties)
{
    int64_t m = off[C];
    int64_t nt = 0;
    double step = dwt_ratio * alpha;
    if (storage == 2) {
        step = orc_q16_step(step);
        alpha = orc_q16_step(alpha);
    }
    /* modes 4, 5: no rounding at each write; every phase at each pass end */
    const int per_pass = (storage == 4 || storage == 5);
    const int32_t pass_store = storage;
    if (per_pass) storage = 0;
    if (!(flags & ORC_NO_SCS)) {
        for (int32_t c = 0; c < C; ++c) {
            if (per_pass && c > 0 && c % 2 == 0)
                for (int32_t v = 0; v < n; ++v) x[v] = orc_store(x[v], pass_store);
            for (int64_t e = off[c]; e < off[c + 1]; ++e) {
                int32_t i = src[e], j = dst[e];
                double J = -(double)w[e];
                int s = orc_sgn_b(x[i], x[j]);
                if (tie_eps > 0.0 && orc_tie_distance(x[i], x[j]) < tie_eps) {
                    if (nt < max_ties && ties) ties[nt] = e;
                    ++nt;
                }
                if (force && force[e]) s = force[e];
                double xi = x[i] - alpha * J * (double)s;
                double xj = x[j] + alpha * J * (double)s;
                x[i] = orc_store(orc_wrap(xi), storage);
                x[j] = orc_store(orc_wrap(xj), storage);
            }
        }
        if (h) {
            for (int32_t v = 0; v < n; ++v) {
                if (h[v] == 0) continue;
                double J = (double)h[v];
                int s = orc_sgn_b(x[v], 0.0);
                if (tie_eps > 0.0 && orc_tie_distance(x[v], 0.0) < tie_eps) {
                    if (nt < max_ties && ties) ties[nt] = m + n + v;
                    ++nt;
                }
                if (force && force[m + n + v]) s = force[m + n + v];
                x[v] = orc_store(orc_wrap(x[v] - alpha * J * (double)s), storage);
            }
        }
    } else {
        double *dx = (double *)calloc((size_t)n, sizeof(double));
        if (!dx) return -1;
        for (int64_t e = 0; e < m; ++e) {
            int32_t i = src[e], j = dst[e];
            double J = -(double)w[e];
            int s = orc_sgn_b(x[i], x[j]);
            if (tie_eps > 0.0 && orc_tie_distance(x[i], x[j]) < tie_eps) {
                if (nt < max_ties && ties) ties[nt] = e;
                ++nt;
            }
            if (force && force[e]) s = force[e];
            dx[i] -= alpha * J * (double)s;
            dx[j] += alpha * J * (double)s;
        }
        if (h) {
            for (int32_t v = 0; v < n; ++v) {
                if (h[v] == 0) continue;
                int s = orc_sgn_b(x[v], 0.0);
                if (tie_eps > 0.0 && orc_tie_distance(x[v], 0.0) < tie_eps) {
                    if (nt < max_ties && ties) ties[nt] = m + n + v;
                    ++nt;
                }
                if (force && force[m + n + v]) s = force[m + n + v];
                dx[v] -= alpha * (double)h[v] * (double)s;
            }
        }
        for (int32_t v = 0; v < n; ++v) x[v] = orc_store(orc_wrap(x[v] + dx[v]), storage);
        free(dx);
    }
    if (!(flags & ORC_NO_DWT) && dwt_period > 0 && (sweep % dwt_period) == 0) {
        double theta = orc_theta(seed, replica, sweep);
        double twist = step;
        if (flags & ORC_DWT_RANDDIR) twist = (double)orc_twist_dir(seed, replica, sweep) * step;
        for (int32_t v = 0; v < n; ++v) {
            double dist = 1.0;
            int in = orc_in_window(x[v], theta, window, &dist);
            if (tie_eps > 0.0 && dist < tie_eps) {
                if (nt < max_ties && ties) ties[nt] = m + v;
                ++nt;
            }
            if (force && force[m + v]) in = force[m + v] > 0;
            if (in) x[v] = orc_store(orc_wrap(x[v] + twist), storage);
        }
    }
    if (per_pass)
        for (int32_t v = 0; v < n; ++v) x[v] = orc_store(x[v], pass_store);
    return nt;
}

/* The sweep of Alg. 1 without local fields. */
int64_t orc_sweep(int32_t n, int32_t C, const int64_t *off, const int32_t *src,
                  const int32_t *dst, const int32_t *w, double *x, double alpha,
                  int64_t sweep, int32_t dwt_period, double dwt_ratio, double window,
                  uint64_t seed, int64_t replica, int32_t flags, int32_t storage,
                  const int8_t *force, double tie_eps, int64_t *ties, int64_t max_ties)
{
    return orc_sweep_h(n, C, off, src, dst, w, 0, x, alpha, sweep, dwt_period, dwt_ratio, window,
                       seed, replica, flags, storage, force, tie_eps, ties, max_ties);
}

/* Bisector binarization and exact cut (Alg. 1 final loop; Appendix B: P
 * bisectors spaced over a semicircle). Reading: bisector p sits at
 * B_p = floor(p 2^31 / P) on the 2^32 circle; s_v = +1 iff
 * ((q_v - B_p) mod 2^32) < 2^31 with q_v = floor(x_v 2^32).
 * cut_p = sum_e w_e [s_i != s_j] (Max-Cut form, Appendix A), in int64.
 * Writes all P cuts when cuts != NULL; returns the index of the best cut
 * (ties -> smallest p) and the spins of that bisector when spins != NULL. */
int32_t orc_binarize(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                     const int32_t *w, const double *x, int32_t P, int64_t *cuts,
                     int64_t *best_cut, int8_t *spins)
{
    uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    int8_t *s = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!q || !s) { free(q); free(s); return -1; }
    for (int32_t v = 0; v < n; ++v) q[v] = (uint32_t)(uint64_t)floor(x[v] * 4294967296.0);
    int32_t best_p = 0;
    int64_t best = INT64_MIN;
    for (int32_t p = 0; p < P; ++p) {
        uint32_t B = (uint32_t)(((uint64_t)p << 31) / (uint64_t)P);
        for (int32_t v = 0; v < n; ++v) s[v] = ((uint32_t)(q[v] - B) < 0x80000000u) ? 1 : -1;
        int64_t cut = 0;
        for (int64_t e = 0; e < m; ++e)
            if (s[src[e]] != s[dst[e]]) cut += (int64_t)w[e];
        if (cuts) cuts[p] = cut;
        if (cut > best) { best = cut; best_p = p; }
    }
    if (spins) {
        uint32_t B = (uint32_t)(((uint64_t)best_p << 31) / (uint64_t)P);
        for (int32_t v = 0; v < n; ++v) spins[v] = ((uint32_t)(q[v] - B) < 0x80000000u) ? 1 : -1;
    }
    if (best_cut) *best_cut = best;
    free(q); free(s);
    return best_p;
}

/* Cut of a spin assignment (Appendix A) and Ising energy eq. (1) with h = 0:
 * H = -sum J s_i s_j = sum w s_i s_j. */
int64_t orc_cut(int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w, const int8_t *s)
{
    int64_t cut = 0;
    for (int64_t e = 0; e < m; ++e)
        if (s[src[e]] != s[dst[e]]) cut += (int64_t)w[e];
    return cut;
}

int64_t orc_energy(int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w, const int8_t *s)
{
    int64_t H = 0;
    for (int64_t e = 0; e < m; ++e) H += (int64_t)w[e] * (int64_t)s[src[e]] * (int64_t)s[dst[e]];
    return H;
}

/* Ising energy eq. (1) with local fields, Max-Cut weights w = -J:
 * H = sum_e w_e s_i s_j - sum_v h_v s_v (h NULL = no fields). */
int64_t orc_energy_h(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *w,
                     const int32_t *h, const int8_t *s)
{
    int64_t H = orc_energy(m, src, dst, w, s);
    if (h)
        for (int32_t v = 0; v < n; ++v) H -= (int64_t)h[v] * (int64_t)s[v];
    return H;
}

static int64_t orc_total_weight(int64_t m, const int32_t *w)
{
    int64_t W = 0;
    for (int64_t e = 0; e < m; ++e) W += (int64_t)w[e];
    return W;
}

static uint32_t orc_q32(double x) { return (uint32_t)(uint64_t)floor(x * 4294967296.0); }

/* Spins of a bisector at position B (2^-32 turns) on the circle:
 * s_v = +1 iff ((q_v - B) mod 2^32) < 2^31, the half circle that starts at B. */
static void orc_spins_at(int32_t n, const double *x, uint32_t B, int8_t *s)
{
    for (int32_t v = 0; v < n; ++v) s[v] = ((uint32_t)(orc_q32(x[v]) - B) < 0x80000000u) ? 1 : -1;
}

/* Readout of a problem with local fields (Section II-B: the fields fix the
 * semicircles, so no bisector search is needed). Reading: the reference
 * variable sits at 0 and s_v = +1 iff x_v lies in the half circle centred on
 * it, [-1/4, 1/4) turns: the bisector at B = 3/4 turn (3 2^30). Returns H
 * (eq. (1)); writes the cut and the spins when asked. */
int64_t orc_readout_fields(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           const int32_t *w, const int32_t *h, const double *x, int64_t *cut,
                           int8_t *spins)
{
    int8_t *s = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!s) return INT64_MIN;
    orc_spins_at(n, x, 0xC0000000u, s);
    if (cut) *cut = orc_cut(m, src, dst, w, s);
    int64_t H = orc_energy_h(n, m, src, dst, w, h, s);
    if (spins) memcpy(spins, s, (size_t)n);
    free(s);
    return H;
}

/* Optimal bisector, brute force (the definition): the largest cut over
 * every bisector position B in [0, 2^31) (the half circle from B and its
 * complement give the same cut, so half a turn of positions covers all
 * bisectors). The spins at B change only where B passes a point of some
 * phase, so the cut is constant on [0, phi_1] and on every [phi_k + 1,
 * phi_{k+1}] (phi_v = q_v mod 2^31, sorted), and the candidates are
 * B = 0 and B = phi_v + 1 < 2^31; each is evaluated from scratch.
 * Returns the best B (ties -> smallest B), writes the cut and spins. */
int64_t orc_binarize_opt_brute(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                               const int32_t *w, const double *x, int64_t *best_cut, int8_t *spins)
{
    int8_t *s = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!s) return -1;
    int64_t best = INT64_MIN;
    uint32_t bestB = 0;
    for (int32_t k = -1; k < n; ++k) {
        uint32_t B = 0;
        if (k >= 0) {
            uint32_t phi = orc_q32(x[k]) & 0x7FFFFFFFu;
            if (phi + 1u >= 0x80000000u) continue;
            B = phi + 1u;
        }
        orc_spins_at(n, x, B, s);
        int64_t c = orc_cut(m, src, dst, w, s);
        if (c > best || (c == best && B < bestB)) { best = c; bestB = B; }
    }
    if (spins) orc_spins_at(n, x, bestB, spins);
    if (best_cut) *best_cut = best;
    free(s);
    return (int64_t)bestB;
}

typedef struct { uint32_t pos; int64_t delta; } orc_event;

static int orc_event_cmp(const void *a, const void *b)
{
    uint32_t pa = ((const orc_event *)a)->pos, pb = ((const orc_event *)b)->pos;
    return (pa > pb) - (pa < pb);
}

/* Optimal bisector by one sorted sweep over the bisector positions, the
 * procedure of Burer, Monteiro and Zhang (2002) (Section II-B cites it as
 * the exact alternative to equally spaced bisectors). With phi_v = q_v mod
 * 2^31 and t_v = q_v's top bit, s_v(B) = +1 iff [B <= phi_v] xor t_v, so edge
 * (i, j) is cut at B iff (t_i xor t_j) xor [lo < B <= hi] (lo, hi = the
 * smaller and larger of phi_i, phi_j). Starting from the cut at B = 0, every
 * edge contributes d_e = w_e (1 - 2 (t_i xor t_j)) on the interval
 * (lo, hi]: +d_e at position lo + 1, -d_e at hi + 1. Sorting these 2m
 * events (the library sort) and summing them in order gives the cut at
 * every position where it can change. Same result and tie rule as the brute
 * force above. */
int64_t orc_binarize_opt(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                         const int32_t *w, const double *x, int64_t *best_cut, int8_t *spins)
{
    orc_event *ev = (orc_event *)malloc(sizeof(orc_event) * (size_t)(2 * m > 0 ? 2 * m : 1));
    if (!ev) return -1;
    int64_t c0 = 0, k = 0;
    for (int64_t e = 0; e < m; ++e) {
        uint32_t qi = orc_q32(x[src[e]]), qj = orc_q32(x[dst[e]]);
        int cross = (int)((qi >> 31) ^ (qj >> 31));
        if (cross) c0 += (int64_t)w[e];
        uint32_t pi = qi & 0x7FFFFFFFu, pj = qj & 0x7FFFFFFFu;
        uint32_t lo = pi < pj ? pi : pj, hi = pi < pj ? pj : pi;
        if (lo == hi) continue;
        int64_t d = (int64_t)w[e] * (cross ? -1 : 1);
        ev[k].pos = lo + 1u; ev[k].delta = d; ++k;
        ev[k].pos = hi + 1u; ev[k].delta = -d; ++k;
    }
    qsort(ev, (size_t)k, sizeof(orc_event), orc_event_cmp);
    int64_t best = c0, cur = c0;
    uint32_t bestB = 0;
    for (int64_t a = 0; a < k;) {
        uint32_t pos = ev[a].pos;
        while (a < k && ev[a].pos == pos) cur += ev[a++].delta;
        if (pos < 0x80000000u && cur > best) { best = cur; bestB = pos; }
    }
    free(ev);
    if (spins) orc_spins_at(n, x, bestB, spins);
    if (best_cut) *best_cut = best;
    return (int64_t)bestB;
}

/* One readout of the current phases: with fields the fixed semicircle,
 * with opt the optimal bisector, else the P bisectors. out: [0] cut,
 * [1] energy H, [2] bisector position B, [3] bisector index p (-1 unless
 * the P bisectors chose). */
static void orc_readout(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                        const int32_t *w, const int32_t *h, int64_t W, const double *x, int32_t P,
                        int opt, int64_t out[4], int8_t *spins)
{
    if (h) {
        int64_t c = 0;
        out[1] = orc_readout_fields(n, m, src, dst, w, h, x, &c, spins);
        out[0] = c;
        out[2] = 0xC0000000u;
        out[3] = -1;
    } else if (opt) {
        int64_t c = 0;
        out[2] = orc_binarize_opt(n, m, src, dst, w, x, &c, spins);
        out[0] = c;
        out[1] = W - 2 * c;
        out[3] = -1;
    } else {
        int64_t c = 0;
        int32_t p = orc_binarize(n, m, src, dst, w, x, P, 0, &c, spins);
        out[0] = c;
        out[1] = W - 2 * c;
        out[2] = (int64_t)(((uint64_t)p << 31) / (uint64_t)P);
        out[3] = p;
    }
}

/* Readouts of one trial with mid-anneal best tracking: with track = T > 0
 * the phases are read out after every sweep s with s mod T = 0 and after
 * the last sweep S (the energy trajectories of Fig. 10 sample every 1000
 * sweeps), each readout's energy goes to trace[k] (k = 0 .. ceil(S/T) - 1),
 * and the replica keeps the readout of lowest energy (ties -> the earlier).
 * Readouts use the fixed semicircle with fields, else the P bisectors; with
 * flag OPT_BISECTOR a last readout at S with the optimal bisector competes
 * too (it replaces the final P-bisector readout when track = 0).
 * out: [0] cut, [1] energy, [2] B, [3] p or -1, [4] sweep of the kept
 * readout. Returns the kept energy. */
int64_t orc_trial_ex(int32_t n, int32_t C, const int64_t *off, const int32_t *src, const int32_t *dst,
                     const int32_t *w, const int32_t *h, int64_t S, double alpha0, int32_t dwt_period,
                     double dwt_ratio, double window, int32_t P, uint64_t seed, int64_t replica,
                     int32_t flags, int32_t storage, int32_t track, double *x, int8_t *spins,
                     int64_t *out, int64_t *trace)
{
    int64_t m = off[C], W = orc_total_weight(m, w);
    int8_t *s_cur = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!s_cur) return INT64_MIN;
    int opt = (flags & ORC_OPT_BISECTOR) && !h;
    orc_init_phases(n, seed, replica, x);
    for (int32_t v = 0; v < n; ++v) {
        x[v] = orc_store(x[v], storage);
        if (storage == 2) x[v] = floor(x[v] * 65536.0) / 65536.0; /* top 16 bits */
    }
    int64_t kept[5] = {0, INT64_MAX, 0, -1, 0};
    int64_t k = 0;
    for (int64_t s = 1; s <= S; ++s) {
        double a = orc_alpha(s, S, alpha0);
        orc_sweep_h(n, C, off, src, dst, w, h, x, a, s, dwt_period, dwt_ratio, window, seed, replica,
                    flags, storage, 0, 0.0, 0, 0);
        if (track > 0 && (s % track == 0 || s == S)) {
            int64_t r[4];
            orc_readout(n, m, src, dst, w, h, W, x, P, 0, r, s_cur);
            if (trace) trace[k] = r[1];
            ++k;
            if (r[1] < kept[1]) {
                memcpy(kept, r, sizeof(r));
                kept[4] = s;
                if (spins) memcpy(spins, s_cur, (size_t)n);
            }
        }
    }
    if (track <= 0 || opt) {
        int64_t r[4];
        orc_readout(n, m, src, dst, w, h, W, x, P, opt, r, s_cur);
        if (track <= 0 || r[1] < kept[1]) {
            memcpy(kept, r, sizeof(r));
            kept[4] = S;
            if (spins) memcpy(spins, s_cur, (size_t)n);
        }
    }
    if (out) memcpy(out, kept, sizeof(kept));
    free(s_cur);
    return kept[1];
}

/* One full trial of Alg. 1 for one replica: random x, sweeps 1..S with the
 * schedule, DWT and the bisector readout. x (n) receives the final phases,
 * cuts (P, optional) the bisector cuts; returns the best cut. */
int64_t orc_trial(int32_t n, int32_t C, const int64_t *off, const int32_t *src, const int32_t *dst,
                  const int32_t *w, int64_t S, double alpha0, int32_t dwt_period, double dwt_ratio,
                  double window, int32_t P, uint64_t seed, int64_t replica, int32_t flags,
                  int32_t storage, double *x, int8_t *spins, int32_t *best_p)
{
    orc_init_phases(n, seed, replica, x);
    for (int32_t v = 0; v < n; ++v) {
        x[v] = orc_store(x[v], storage);
        if (storage == 2) x[v] = floor(x[v] * 65536.0) / 65536.0; /* top 16 bits */
    }
    for (int64_t s = 1; s <= S; ++s) {
        double a = orc_alpha(s, S, alpha0);
        orc_sweep(n, C, off, src, dst, w, x, a, s, dwt_period, dwt_ratio, window, seed, replica,
                  flags, storage, 0, 0.0, 0, 0);
    }
    int64_t best = 0;
    int32_t bp = orc_binarize(n, off[C], src, dst, w, x, P, 0, &best, spins);
    if (best_p) *best_p = bp;
    return best;
}

/* Many replicas over host threads (replicas are independent trials). */
typedef struct {
    int32_t n, C; const int64_t *off; const int32_t *src, *dst, *w;
    int64_t S; double alpha0; int32_t dwt_period; double dwt_ratio, window; int32_t P;
    uint64_t seed; int32_t flags, storage;
    int64_t r0, r1, stride; int64_t *cuts; int32_t *best_p; double *x_out;
} orc_job;

static void *orc_worker(void *arg)
{
    orc_job *j = (orc_job *)arg;
    double *x = (double *)malloc(sizeof(double) * (size_t)(j->n > 0 ? j->n : 1));
    if (!x) return 0;
    for (int64_t r = j->r0; r < j->r1; r += j->stride) {
        int32_t bp = 0;
        j->cuts[r] = orc_trial(j->n, j->C, j->off, j->src, j->dst, j->w, j->S, j->alpha0,
                               j->dwt_period, j->dwt_ratio, j->window, j->P, j->seed, r,
                               j->flags, j->storage, x, 0, &bp);
        if (j->best_p) j->best_p[r] = bp;
        if (j->x_out) memcpy(j->x_out + (size_t)r * (size_t)j->n, x, sizeof(double) * (size_t)j->n);
    }
    free(x);
    return 0;
}

int32_t orc_trials(int32_t n, int32_t C, const int64_t *off, const int32_t *src, const int32_t *dst,
                   const int32_t *w, int64_t S, double alpha0, int32_t dwt_period, double dwt_ratio,
                   double window, int32_t P, uint64_t seed, int64_t replicas, int32_t flags,
                   int32_t storage, int32_t threads, int64_t *cuts, int32_t *best_p, double *x_out)
{
    if (threads < 1) threads = 1;
    if (threads > replicas) threads = (int32_t)(replicas > 0 ? replicas : 1);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    orc_job *jobs = (orc_job *)malloc(sizeof(orc_job) * (size_t)threads);
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    for (int32_t t = 0; t < threads; ++t) {
        orc_job j = {n, C, off, src, dst, w, S, alpha0, dwt_period, dwt_ratio, window, P,
                     seed, flags, storage, t, replicas, threads, cuts, best_p, x_out};
        jobs[t] = j;
        pthread_create(&th[t], 0, orc_worker, &jobs[t]);
    }
    for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], 0);
    free(th); free(jobs);
    return threads;
}

/* Many replicas of orc_trial_ex over host threads. out: [replicas][5],
 * trace: [replicas][ceil(S/track)] (may be NULL), x_out: [replicas][n]. */
typedef struct {
    int32_t n, C; const int64_t *off; const int32_t *src, *dst, *w, *h;
    int64_t S; double alpha0; int32_t dwt_period; double dwt_ratio, window; int32_t P;
    uint64_t seed; int32_t flags, storage, track;
    int64_t r0, r1, stride, n_trace; int64_t *out, *trace; double *x_out; int8_t *spins_out;
} orc_job_ex;

static void *orc_worker_ex(void *arg)
{
    orc_job_ex *j = (orc_job_ex *)arg;
    double *x = (double *)malloc(sizeof(double) * (size_t)(j->n > 0 ? j->n : 1));
    if (!x) return 0;
    for (int64_t r = j->r0; r < j->r1; r += j->stride) {
        orc_trial_ex(j->n, j->C, j->off, j->src, j->dst, j->w, j->h, j->S, j->alpha0, j->dwt_period,
                     j->dwt_ratio, j->window, j->P, j->seed, r, j->flags, j->storage, j->track, x,
                     j->spins_out ? j->spins_out + (size_t)r * (size_t)j->n : 0, j->out + 5 * r,
                     j->trace ? j->trace + (size_t)r * (size_t)j->n_trace : 0);
        if (j->x_out) memcpy(j->x_out + (size_t)r * (size_t)j->n, x, sizeof(double) * (size_t)j->n);
    }
    free(x);
    return 0;
}

int32_t orc_trials_ex(int32_t n, int32_t C, const int64_t *off, const int32_t *src, const int32_t *dst,
                      const int32_t *w, const int32_t *h, int64_t S, double alpha0, int32_t dwt_period,
                      double dwt_ratio, double window, int32_t P, uint64_t seed, int64_t replicas,
                      int32_t flags, int32_t storage, int32_t track, int32_t threads, int64_t *out,
                      int64_t *trace, double *x_out, int8_t *spins_out)
{
    if (threads < 1) threads = 1;
    if (threads > replicas) threads = (int32_t)(replicas > 0 ? replicas : 1);
    int64_t n_trace = track > 0 ? (S + track - 1) / track : 0;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    orc_job_ex *jobs = (orc_job_ex *)malloc(sizeof(orc_job_ex) * (size_t)threads);
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    for (int32_t t = 0; t < threads; ++t) {
        orc_job_ex j = {n, C, off, src, dst, w, h, S, alpha0, dwt_period, dwt_ratio, window, P,
                        seed, flags, storage, track, t, replicas, threads, n_trace, out, trace,
                        x_out, spins_out};
        jobs[t] = j;
        pthread_create(&th[t], 0, orc_worker_ex, &jobs[t]);
    }
    for (int32_t t = 0; t < threads; ++t) pthread_join(th[t], 0);
    free(th); free(jobs);
    return threads;
}

/* ------------------------------------------------------------------------ */
/* Edge colourings (Alg. 1 line "Assign a proper edge coloring")             */
/* ------------------------------------------------------------------------ */

/* Greedy heuristic of Section II-B: loop over the edges in order and give
 * each the lowest colour not yet used at either endpoint. Returns C. */
int32_t orc_color_greedy(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *color)
{
    int32_t *deg = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    if (!deg) return -1;
    int32_t D = 0;
    for (int64_t e = 0; e < m; ++e) { deg[src[e]]++; deg[dst[e]]++; }
    for (int32_t v = 0; v < n; ++v) if (deg[v] > D) D = deg[v];
    free(deg);
    int32_t K = 2 * D; /* greedy never needs more than 2D-1 colours */
    if (K < 1) K = 1;
    uint8_t *used = (uint8_t *)calloc((size_t)n * (size_t)K, 1);
    if (!used && n > 0) return -1;
    int32_t C = 0;
    for (int64_t e = 0; e < m; ++e) {
        int32_t i = src[e], j = dst[e];
        int32_t c = 0;
        while (used[(size_t)i * K + c] || used[(size_t)j * K + c]) ++c;
        color[e] = c;
        used[(size_t)i * K + c] = 1;
        used[(size_t)j * K + c] = 1;
        if (c + 1 > C) C = c + 1;
    }
    free(used);
    return C;
}

/* Regular 4-colour pattern of a 2D torus with even sides (Section II-B,
 * Appendix B). The paper fixes the pattern (horizontal and vertical edges,
 * each split by the parity of the lower end) but not the order of the
 * colours; the reading taken here is: colour 0 = horizontal edges leaving an
 * even column, 1 = vertical edges leaving an even row, 2 = horizontal edges
 * leaving an odd column, 3 = vertical edges leaving an odd row. Vertex
 * v = r L2 + c. Returns 4, or -1 if an edge is not a torus edge or a side is
 * odd. */
int32_t orc_color_torus2d(int32_t L1, int32_t L2, int64_t m, const int32_t *src, const int32_t *dst,
                          int32_t *color)
{
    if (L1 < 4 || L2 < 4 || (L1 & 1) || (L2 & 1)) return -1;
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = src[e], b = dst[e];
        int32_t ra = a / L2, ca = a % L2, rb = b / L2, cb = b % L2;
        if (ra == rb && (ca + 1) % L2 == cb) color[e] = (ca & 1) ? 2 : 0;
        else if (ra == rb && (cb + 1) % L2 == ca) color[e] = (cb & 1) ? 2 : 0;
        else if (ca == cb && (ra + 1) % L1 == rb) color[e] = (ra & 1) ? 3 : 1;
        else if (ca == cb && (rb + 1) % L1 == ra) color[e] = (rb & 1) ? 3 : 1;
        else return -1;
    }
    return 4;
}

/* 3D torus, six colours: colour = 3 (parity) + axis, where axis a (0,1,2)
 * is the edge's direction and parity that of the lower end's coordinate
 * along a (same ordering reading as in 2D: all even classes first).
 * Vertex v = (i L2 + j) L3 + k. */
int32_t orc_color_torus3d(int32_t L1, int32_t L2, int32_t L3, int64_t m, const int32_t *src,
                          const int32_t *dst, int32_t *color)
{
    int32_t L[3] = {L1, L2, L3};
    for (int a = 0; a < 3; ++a) if (L[a] < 4 || (L[a] & 1)) return -1;
    for (int64_t e = 0; e < m; ++e) {
        int32_t u[2] = {src[e], dst[e]};
        int32_t co[2][3];
        for (int t = 0; t < 2; ++t) {
            co[t][2] = u[t] % L3;
            co[t][1] = (u[t] / L3) % L2;
            co[t][0] = u[t] / (L2 * L3);
        }
        int found = 0;
        for (int a = 0; a < 3 && !found; ++a) {
            int same = 1;
            for (int b = 0; b < 3; ++b) if (b != a && co[0][b] != co[1][b]) same = 0;
            if (!same) continue;
            if ((co[0][a] + 1) % L[a] == co[1][a]) { color[e] = 3 * (co[0][a] & 1) + a; found = 1; }
            else if ((co[1][a] + 1) % L[a] == co[0][a]) { color[e] = 3 * (co[1][a] & 1) + a; found = 1; }
        }
        if (!found) return -1;
    }
    return 6;
}

/* Partition check (Section II-C: E = E_1 u ... u E_C, each E_c a matching):
 * returns 0 if every edge has a colour in [0,C) and no vertex meets two
 * edges of one colour; 1 if a colour is out of range; 2 if a colour class
 * is not a matching. */
int32_t orc_validate_partition(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                               int32_t C, const int32_t *color)
{
    if (C < 0) return 1;
    uint8_t *seen = (uint8_t *)calloc((size_t)n * (size_t)(C > 0 ? C : 1), 1);
    if (!seen && n > 0) return -1;
    int32_t rc = 0;
    for (int64_t e = 0; e < m && rc == 0; ++e) {
        int32_t c = color[e];
        if (c < 0 || c >= C) { rc = 1; break; }
        size_t a = (size_t)src[e] * (size_t)C + (size_t)c;
        size_t b = (size_t)dst[e] * (size_t)C + (size_t)c;
        if (seen[a] || seen[b]) { rc = 2; break; }
        seen[a] = seen[b] = 1;
    }
    free(seen);
    return rc;
}

/* Exhaustive Max-Cut for small n (n <= 26): every assignment with s_0 = +1
 * (a global flip leaves the cut unchanged). Returns the optimum cut and one
 * optimal assignment. */
int64_t orc_bruteforce_maxcut(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                              const int32_t *w, int8_t *best_spins)
{
    if (n <= 0) return 0;
    if (n > 26) return INT64_MIN;
    int8_t *s = (int8_t *)malloc((size_t)n);
    if (!s) return INT64_MIN;
    int64_t best = INT64_MIN;
    uint64_t total = (uint64_t)1 << (n - 1);
    for (uint64_t mask = 0; mask < total; ++mask) {
        s[0] = 1;
        for (int32_t v = 1; v < n; ++v) s[v] = ((mask >> (v - 1)) & 1u) ? -1 : 1;
        int64_t cut = orc_cut(m, src, dst, w, s);
        if (cut > best) {
            best = cut;
            if (best_spins) memcpy(best_spins, s, (size_t)n);
        }
    }
    free(s);
    return best;
}
