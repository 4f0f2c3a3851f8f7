/*
 * siminf_oracle.c -- plain, slow, serial CPU oracle for the SimInf split-step
 * method (Widgren, Bauer, Eriksson, Engblom, "SimInf: An R package for
 * Data-driven Stochastic Disease Spread Simulations", arXiv 1605.01421).
 *
 * TEST INFRASTRUCTURE ONLY.  This file defines the results that the CUDA
 * path must reproduce.  It is linked by the tests, by the smoke check and by
 * the CPU-baseline leg of the benchmark, never by the product path.  It
 * shares no source with the CUDA library: its random generator, logarithm,
 * bounded-integer routine, rate functions, event semantics and validation are
 * all written here, once, in plain C99.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fno-fast-math -fPIC -shared.
 * Every floating-point expression is evaluated left to right exactly as
 * written; no fused multiply-add is allowed (the CUDA side is built with
 * -fmad=false for the same reason), so the double results are bit-identical.
 * The same source compiled with -fopenmp is a timing build for the CPU
 * baseline only: the node loops of a day (SSA, each node's E1 events, post
 * time step) run in parallel as in the paper's solver (Sec. 3.4.2), E2
 * events stay serial, and the results are the serial build's.  The tests use
 * the serial build.
 *
 * What each part follows:
 *   - the split-step solver: Sec. 2.3 (Eq. numstep1-numstep3) and the solver
 *     pseudo-code of Appendix A: per node, direct SSA up to the next unit of
 *     time, then the node's E1 events, then all E2 events, then the post time
 *     step function, then recording at tspan points (Sec. 3.4.2);
 *   - the 'aem' solver of Sec. 3.4.2 (channels with private random streams),
 *     read as the next reaction method of Gibson and Bruck with one Philox
 *     stream per (node, transition) channel (see aem_node_day);
 *   - direct SSA step: Appendix A (rate sum, exponential waiting time with
 *     log of an open-interval uniform, inversion on lambda * r2, update by
 *     column n of S, recomputation of the rates that column n of G marks);
 *   - rate functions: SIR Eq. (SIR) and the C listing of the SIR rates in
 *     Appendix C (operation order kept); SIS Eq. (SIRstoich) of Sec. 2.1;
 *     SISe Eq. (vtectrans) and the environmental pressure ODE of Sec. 4.2
 *     without the spatial coupling term; SISe3 = SISe per age class;
 *     SISe_sp = SISe with the coupling term of that ODE (Eq.
 *     envInfPressure-local-spread), all nodes updated from the same old
 *     values;
 *   - scheduled events: Sec. 3.3 (enter, internal transfer, external
 *     transfer, exit; select matrix E, shift matrix N; same-time order exit,
 *     enter, internal transfer, external transfer) and Appendix B;
 *   - the random stream: Philox4x32-10 of Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3" (SC'11), counter based,
 *     so that every draw is a function of (seed, replicate, node, day,
 *     draw index) or (seed, replicate, event, draw index);
 *   - bounded integers: Lemire, "Fast random integer generation in an
 *     interval" (ACM TOMACS 2019), multiply-shift with rejection.
 *
 * Readings of points the paper leaves open are listed beside the code that
 * takes them (marked "Reading").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "siminf_oracle.h"

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4.2): ten rounds of a           */
/* multiply-xor bijection keyed by a Weyl sequence.                          */
/* ------------------------------------------------------------------------ */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    /* The two round multipliers and the key increments are the published
     * constants of Philox4x32. */
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    int r;
    for (r = 0; r < 10; r++) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* ------------------------------------------------------------------------ */
/* Open-interval uniform from two 32-bit words.  The paper requires r1, r2   */
/* uniform in (0, 1) (Appendix A).  Reading: take 52 random bits            */
/* k = (b << 20) | (a >> 12) and return (k + 1/2) * 2^-52, which is exact   */
/* and lies in [2^-53, 1 - 2^-53].                                            */
/* ------------------------------------------------------------------------ */

double oracle_u01(uint32_t a, uint32_t b)
{
    uint64_t k = ((uint64_t)b << 20) | (uint64_t)(a >> 12);
    double dk = (double)k;
    return (dk + 0.5) * (1.0 / 4503599627370496.0); /* 2^-52 */
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm written from the mathematics, so that both sides of    */
/* the parity check evaluate the same sequence of IEEE operations.          */
/*   x = 2^k * m, m in (sqrt(2)/2, sqrt(2)];  f = m - 1;  s = f / (2 + f);  */
/*   log(1 + f) = 2 atanh(s) = 2 s + s R(s^2),                              */
/*   R(z) = sum_{j=1..10} 2 z^j / (2 j + 1)   (Taylor series of atanh),     */
/*   evaluated in Estrin's scheme (depth 8 instead of Horner's 20),         */
/* rearranged with 2 s = f - hfsq + s hfsq, hfsq = f^2 / 2, into            */
/*   log(1 + f) = f - (hfsq - s (hfsq + R)),                                */
/* and log x = k ln2_hi + (f - (hfsq - (s (hfsq + R) + k ln2_lo))) with a   */
/* Cody-Waite split of ln 2 whose high part has 33 significant bits, so     */
/* k ln2_hi is exact.  |s| <= 0.1716, so ten terms leave a truncation       */
/* error below 2^-54 relative.  Every a + b c of the polynomial, hfsq + R,  */
/* s (hfsq + R) + k ln2_lo and the final k ln2_hi + (...) is one fused      */
/* multiply-add (C99 fma: a single rounding), the form with the fewest      */
/* IEEE operations.                                                          */
/* ------------------------------------------------------------------------ */

double oracle_log(double x)
{
    uint64_t bits;
    int k;
    double m, f, hfsq, s, z, t, dk;
    const double ln2_hi = 0.6931471804855391;      /* 33 significant bits */
    const double ln2_lo = 7.440617110012397e-11;   /* ln 2 - ln2_hi      */

    if (!(x > 0.0)) {
        if (x == 0.0) return -HUGE_VAL;
        return NAN;
    }
    if (isinf(x)) return x;
    k = 0;
    if (x < 2.2250738585072014e-308) {   /* subnormal: scale by 2^54 */
        x = x * 18014398509481984.0;
        k = -54;
    }
    memcpy(&bits, &x, sizeof bits);
    k += (int)((bits >> 52) & 0x7ff) - 1023;
    bits = (bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    memcpy(&m, &bits, sizeof m);
    if (m > 1.4142135623730951) {        /* sqrt(2) rounded to double */
        m = m * 0.5;
        k = k + 1;
    }
    f = m - 1.0;
    hfsq = (0.5 * f) * f;
    s = f / (2.0 + f);
    z = s * s;
    /* R(z) = z P(z), P(z) = sum_{j=1..10} c_j z^(j-1), c_j = 2 / (2 j + 1),
     * in Estrin's scheme: pairs c_j + c_(j+1) z, combined with z^2, z^4, z^8;
     * t = hfsq + R = hfsq + z P */
    {
        double z2 = z * z, z4 = z2 * z2, z8 = z4 * z4;
        double p01 = fma(2.0 / 5.0, z, 2.0 / 3.0);
        double p23 = fma(2.0 / 9.0, z, 2.0 / 7.0);
        double p45 = fma(2.0 / 13.0, z, 2.0 / 11.0);
        double p67 = fma(2.0 / 17.0, z, 2.0 / 15.0);
        double p89 = fma(2.0 / 21.0, z, 2.0 / 19.0);
        double q03 = fma(z2, p23, p01);
        double q47 = fma(z2, p67, p45);
        double P = fma(z8, p89, fma(z4, q47, q03));
        t = fma(z, P, hfsq);
    }
    dk = (double)k;
    return fma(dk, ln2_hi, f - (hfsq - fma(s, t, dk * ln2_lo)));
}

/* ------------------------------------------------------------------------ */
/* Word stream for the scheduled events: counter (c, idx_lo, idx_hi,         */
/* (1 << 24) | replicate), c = 0, 1, 2, ...; four words per Philox call,     */
/* used in order.                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t ctr[4];
    uint32_t key[2];
    uint32_t buf[4];
    int pos;
} word_stream;

static void ws_init(word_stream *ws, uint64_t seed, int64_t event_index, int rep)
{
    ws->key[0] = (uint32_t)seed;
    ws->key[1] = (uint32_t)(seed >> 32);
    ws->ctr[0] = 0;
    ws->ctr[1] = (uint32_t)(uint64_t)event_index;
    ws->ctr[2] = (uint32_t)((uint64_t)event_index >> 32);
    ws->ctr[3] = ((uint32_t)ORACLE_STREAM_EVENTS << 24) | (uint32_t)rep;
    ws->pos = 4;
}

static uint32_t ws_next(word_stream *ws)
{
    if (ws->pos == 4) {
        oracle_philox4x32_10(ws->ctr, ws->key, ws->buf);
        ws->ctr[0] += 1;
        ws->pos = 0;
    }
    return ws->buf[ws->pos++];
}

/* Lemire's unbiased multiply-shift: uniform integer in [0, s), s >= 1. */
static uint32_t ws_bounded(word_stream *ws, uint32_t s)
{
    uint32_t x = ws_next(ws);
    uint64_t m = (uint64_t)x * (uint64_t)s;
    uint32_t l = (uint32_t)m;
    if (l < s) {
        uint32_t t = (uint32_t)(0u - s) % s;
        while (l < t) {
            x = ws_next(ws);
            m = (uint64_t)x * (uint64_t)s;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

uint32_t oracle_bounded_sequence(uint64_t seed, int64_t event_index, int rep,
                                 const uint32_t *ranges, int n, uint32_t *out)
{
    word_stream ws;
    int i;
    ws_init(&ws, seed, event_index, rep);
    for (i = 0; i < n; i++) out[i] = ws_bounded(&ws, ranges[i]);
    return (uint32_t)ws.ctr[0];
}

/* ------------------------------------------------------------------------ */
/* Transition-rate functions (TRFun of Sec. 3.4.1) and post time step        */
/* functions (PTSFun).                                                       */
/* ------------------------------------------------------------------------ */

/* Seasonal decay beta(t) of Sec. 4.2: four seasons whose last day of year   */
/* is local data end_t1..end_t4.  Reading: day of year d = ((t - 1) mod 365) */
/* + 1 (floored); beta_t1 while d <= end_t1, beta_t2 while d <= end_t2,     */
/* beta_t3 while d <= end_t3, else beta_t4.                                  */
static double seasonal_beta(int t, const double *ldata, const double *beta4)
{
    int d = (t - 1) % 365;
    if (d < 0) d += 365;
    d = d + 1;
    if ((double)d <= ldata[0]) return beta4[0];
    if ((double)d <= ldata[1]) return beta4[1];
    if ((double)d <= ldata[2]) return beta4[2];
    return beta4[3];
}

/* rate j of the model for a node with counts u, continuous state v */
static double model_rate(const oracle_model *m, int j, const int *u,
                         const double *v, const double *ldata,
                         const double *gdata)
{
    (void)ldata;
    switch (m->kind) {
    case ORACLE_SIR: {
        /* Appendix C: S_n, I_n as doubles, n = S_n + I_n + R, then
         * (beta * S_n * I_n) / n when n > 0; recovery gamma * I. */
        const double S_n = (double)u[0];
        const double I_n = (double)u[1];
        const double n = S_n + I_n + (double)u[2];
        if (j == 0) {
            if (n > 0.0) return (gdata[0] * S_n * I_n) / n;
            return 0.0;
        }
        return gdata[1] * (double)u[1];
    }
    case ORACLE_SIS:
        /* Sec. 2.1: R(x) = [beta x1 x2, gamma x2] (no division by N). */
        if (j == 0) return gdata[0] * (double)u[0] * (double)u[1];
        return gdata[1] * (double)u[1];
    case ORACLE_SISE:
    case ORACLE_SISE_SP:
        /* Sec. 4.2: S -> I at upsilon * phi * S, I -> S at gamma * I. */
        if (j == 0) return gdata[0] * v[0] * (double)u[0];
        return gdata[1] * (double)u[1];
    case ORACLE_SISE3: {
        /* compartments [S1, I1, S2, I2, S3, I3]; transition 2a is
         * S_a -> I_a at upsilon_a * phi * S_a, transition 2a + 1 is
         * I_a -> S_a at gamma_a * I_a. */
        int a = j / 2;
        if ((j & 1) == 0) return gdata[a] * v[0] * (double)u[2 * a];
        return gdata[3 + a] * (double)u[2 * a + 1];
    }
    case ORACLE_GENERIC:
        /* a model from transition strings (Sec. 3.5, mparse): the
         * propensity functions are C code generated from the strings and
         * compiled separately */
        return m->rate_fn(j, u, gdata);
    default:
        return 0.0;
    }
}

/* Post time step (Eq. numstep3, Euler forward with dt = 1).  Returns > 0 if
 * the rates must be recomputed, < 0 on error, 0 otherwise (Appendix C).     */
static int model_pts(int kind, double *v_new, const int *u, const double *v,
                     const double *ldata, const double *gdata, int t)
{
    int a;
    double I_tot, N_tot, phi, shed, beta;
    const double *g;
    switch (kind) {
    case ORACLE_SISE:
        I_tot = (double)u[1];
        N_tot = (double)u[0] + (double)u[1];
        g = gdata + 2;            /* alpha, beta_t1..beta_t4 */
        break;
    case ORACLE_SISE3:
        I_tot = 0.0;
        N_tot = 0.0;
        for (a = 0; a < 3; a++) {
            I_tot = I_tot + (double)u[2 * a + 1];
            N_tot = N_tot + (double)u[2 * a] + (double)u[2 * a + 1];
        }
        g = gdata + 6;            /* alpha, beta_t1..beta_t4 */
        break;
    default:
        return 0;                 /* SIR, SIS: no continuous state */
    }
    phi = v[0];
    /* Reading: with an empty node the shedding term is zero. */
    shed = 0.0;
    if (N_tot > 0.0) shed = (g[0] * I_tot) / N_tot;
    beta = seasonal_beta(t, ldata, g + 1);
    v_new[0] = phi + (shed - beta * phi);
    if (!isfinite(v_new[0])) return ORACLE_ERR_PTS;
    return v_new[0] != phi ? 1 : 0;
}

/* SISe_sp post time step of node i (Sec. 4.2, environmental pressure with
 * spatial coupling), one Euler step of length 1 from the values of every
 * node before the update:
 *   phi_i' = phi_i + ((alpha I_i / N_i
 *                      + sum_k ((phi_k N_k - phi_i N_i) / N_i) (D / d_ik))
 *                     - beta(t) phi_i),
 * N = S + I, the sum in neighbour-list order.  Reading: both the shedding
 * and the coupling terms are 0 in an empty node. */
static int sise_sp_pts(const oracle_model *m, int node, const int *u_all,
                       const double *v_all, int t, double *phi_new)
{
    const int *u = u_all + (size_t)node * 2;
    const double *g = m->gdata;
    double N_i = (double)u[0] + (double)u[1];
    double phi = v_all[node];
    double shed = 0.0, coupling = 0.0, beta;
    int64_t k;
    if (N_i > 0.0) {
        shed = (g[2] * (double)u[1]) / N_i;
        if (m->nb_ptr) {
            for (k = m->nb_ptr[node]; k < m->nb_ptr[node + 1]; k++) {
                int j = m->nb_idx[k];
                double N_k = (double)u_all[(size_t)j * 2] + (double)u_all[(size_t)j * 2 + 1];
                double term = ((v_all[j] * N_k - phi * N_i) / N_i) * (g[7] / m->nb_dist[k]);
                coupling = coupling + term;
            }
        }
    }
    beta = seasonal_beta(t, m->ldata + (size_t)node * m->n_ldata, g + 3);
    *phi_new = phi + ((shed + coupling) - beta * phi);
    return isfinite(*phi_new) ? 0 : ORACLE_ERR_PTS;
}

/* ------------------------------------------------------------------------ */
/* Scheduled events (Sec. 3.3).                                              */
/* ------------------------------------------------------------------------ */

static int col_nonzero(const int *M, int n_rows, int col, int row)
{
    return M[(size_t)col * (size_t)n_rows + (size_t)row] != 0;
}

/* Number of individuals an exit / internal / external transfer moves:
 * n if n > 0, else proportion * (sum of the selected compartments).
 * Reading: the product is rounded half away from zero. */
static int64_t event_count(int n, double proportion, int64_t total)
{
    if (n > 0) return n;
    return (int64_t)round(proportion * (double)total);
}

int oracle_apply_event(int n_comp, const int *E, int n_select,
                       const int *N, int n_shift,
                       int type, int *u_node, int *u_dest, int n,
                       double proportion, int select, int shift,
                       uint64_t seed, int64_t event_index, int rep)
{
    int p;
    int64_t total = 0, k, j;
    int moved[ORACLE_MAX_COMP];
    word_stream ws;

    if (n_comp > ORACLE_MAX_COMP || select < 0 || select >= n_select)
        return ORACLE_ERR_ARG;

    if (type == ORACLE_EV_ENTER) {
        /* add n to the first compartment with a non-zero entry in E[, s] */
        for (p = 0; p < n_comp; p++) {
            if (col_nonzero(E, n_comp, select, p)) {
                u_node[p] += n;
                return 0;
            }
        }
        return ORACLE_ERR_ARG;
    }

    for (p = 0; p < n_comp; p++) {
        moved[p] = 0;
        if (col_nonzero(E, n_comp, select, p)) total += u_node[p];
    }
    k = event_count(n, proportion, total);
    if (k < 0 || k > total) return ORACLE_ERR_EVENT_UNDERFLOW;

    /* Sample k individuals without replacement, proportionally to the
     * selected compartments: one uniform index into the remaining
     * individuals per draw, resolved by walking the compartments in row
     * order (an urn; exact multivariate hypergeometric sampling). */
    ws_init(&ws, seed, event_index, rep);
    for (j = 0; j < k; j++) {
        uint32_t x = ws_bounded(&ws, (uint32_t)(total - j));
        for (p = 0; p < n_comp; p++) {
            uint32_t rem;
            if (!col_nonzero(E, n_comp, select, p)) continue;
            rem = (uint32_t)(u_node[p] - moved[p]);
            if (x < rem) {
                moved[p] += 1;
                break;
            }
            x -= rem;
        }
    }

    for (p = 0; p < n_comp; p++) u_node[p] -= moved[p];
    if (type == ORACLE_EV_EXIT) return 0;

    {
        int *target = (type == ORACLE_EV_INTERNAL) ? u_node : u_dest;
        for (p = 0; p < n_comp; p++) {
            int q = p;
            if (moved[p] == 0) continue;
            if (shift >= 0) {
                if (shift >= n_shift) return ORACLE_ERR_ARG;
                q = p + N[(size_t)shift * (size_t)n_comp + (size_t)p];
                if (q < 0 || q >= n_comp) return ORACLE_ERR_SHIFT_RANGE;
            }
            target[q] += moved[p];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The solver.                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t idx;
    int time;
    int type;
} ev_key;

static int ev_key_cmp(const void *a, const void *b)
{
    const ev_key *x = (const ev_key *)a, *y = (const ev_key *)b;
    if (x->time != y->time) return x->time < y->time ? -1 : 1;
    if (x->type != y->type) return x->type < y->type ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static void set_error(oracle_error *err, int code, int rep, int node,
                      int64_t event, int day)
{
    if (err && err->code == 0) {
        err->code = code;
        err->rep = rep;
        err->node = node;
        err->event = event;
        err->day = day;
    }
}

/* Validation of the model and event tables (the error checks of Sec. 3.4.2
 * and the event table constraints of Sec. 3.3). */
static int validate(const oracle_model *m, const oracle_events *ev,
                    const int *tspan, int n_tspan, int n_rep,
                    oracle_error *err)
{
    int64_t e;
    int i, p;
    static const int ncomp[5] = {3, 2, 2, 6, 2};
    static const int ntrans[5] = {2, 2, 2, 6, 2};
    static const int nv[5] = {0, 0, 1, 1, 1};
    static const int ngd[5] = {2, 2, 7, 11, 8};
    static const int nld[5] = {0, 0, 4, 4, 4};
    const int generic = m->kind == ORACLE_GENERIC;
    if (m->kind < 0 || m->kind > ORACLE_GENERIC || m->n_nodes < 0 || n_rep < 1
        || n_tspan < 1 || m->n_comp > ORACLE_MAX_COMP
        || m->n_trans > ORACLE_MAX_TRANS
        || (generic && (!m->rate_fn || m->n_v != 0 || m->n_comp < 1
                        || m->n_trans < 1 || m->n_gdata < 0))
        || (!generic && (m->n_comp != ncomp[m->kind]
                         || m->n_trans != ntrans[m->kind]
                         || m->n_v != nv[m->kind]
                         || m->n_gdata < ngd[m->kind]
                         || m->n_ldata < nld[m->kind]))) {
        set_error(err, ORACLE_ERR_ARG, -1, -1, -1, -1);
        return ORACLE_ERR_ARG;
    }
    for (i = 1; i < n_tspan; i++) {
        if (tspan[i] <= tspan[i - 1]) {
            set_error(err, ORACLE_ERR_ARG, -1, -1, -1, -1);
            return ORACLE_ERR_ARG;
        }
    }
    if (m->nb_ptr) {
        int64_t k;
        if (m->nb_ptr[0] != 0) {
            set_error(err, ORACLE_ERR_ARG, -1, -1, -1, -1);
            return ORACLE_ERR_ARG;
        }
        for (i = 0; i < m->n_nodes; i++) {
            if (m->nb_ptr[i + 1] < m->nb_ptr[i]) {
                set_error(err, ORACLE_ERR_ARG, -1, i, -1, -1);
                return ORACLE_ERR_ARG;
            }
            for (k = m->nb_ptr[i]; k < m->nb_ptr[i + 1]; k++) {
                if (m->nb_idx[k] < 0 || m->nb_idx[k] >= m->n_nodes
                    || !(m->nb_dist[k] > 0.0) || isinf(m->nb_dist[k])) {
                    set_error(err, ORACLE_ERR_ARG, -1, i, -1, -1);
                    return ORACLE_ERR_ARG;
                }
            }
        }
    }
    if (!ev) return 0;
    for (e = 0; e < ev->n; e++) {
        int type = ev->event[e], s = ev->select[e], q = ev->shift[e];
        int bad = 0;
        if (type < 0 || type > 3) bad = 1;
        if (ev->node[e] < 0 || ev->node[e] >= m->n_nodes) bad = 1;
        if (type == ORACLE_EV_EXTERNAL
            && (ev->dest[e] < 0 || ev->dest[e] >= m->n_nodes)) bad = 1;
        if (s < 0 || s >= m->n_select) bad = 1;
        if (ev->n_ind[e] < 0) bad = 1;
        if (!(ev->proportion[e] >= 0.0 && ev->proportion[e] <= 1.0)) bad = 1;
        if (type == ORACLE_EV_INTERNAL && q < 0) bad = 1;
        if (type != ORACLE_EV_ENTER && q >= m->n_shift) bad = 1;
        if (ev->rep && (ev->rep[e] < 0 || ev->rep[e] >= n_rep)) bad = 1;
        if (!bad && type == ORACLE_EV_ENTER) {
            int any = 0;
            for (p = 0; p < m->n_comp; p++)
                if (col_nonzero(m->E, m->n_comp, s, p)) any = 1;
            if (!any) bad = 1;
        }
        if (bad) {
            set_error(err, ORACLE_ERR_ARG, -1, ev->node[e], e, ev->time[e]);
            return ORACLE_ERR_ARG;
        }
        /* the shift must keep every selectable compartment in range */
        if (q >= 0 && type != ORACLE_EV_ENTER && type != ORACLE_EV_EXIT) {
            for (p = 0; p < m->n_comp; p++) {
                int dst;
                if (!col_nonzero(m->E, m->n_comp, s, p)) continue;
                dst = p + m->N[(size_t)q * (size_t)m->n_comp + (size_t)p];
                if (dst < 0 || dst >= m->n_comp) {
                    set_error(err, ORACLE_ERR_SHIFT_RANGE, -1, ev->node[e], e,
                              ev->time[e]);
                    return ORACLE_ERR_SHIFT_RANGE;
                }
            }
        }
    }
    return 0;
}

/* Test hook (not part of the method): when a trace buffer is set, the
 * direct method appends, for every node-day with lambda > 0, the waiting time
 * tau of its first draw (whether or not t + tau passes T) with the node-day's
 * replicate, node and T.  The waiting-time law of Appendix A is pinned on
 * these records.  Serial builds only. */
static oracle_tau_record *g_tau_trace = NULL;
static int64_t g_tau_cap = 0, g_tau_n = 0;

int64_t oracle_trace_first_tau(oracle_tau_record *buf, int64_t cap)
{
#ifdef _OPENMP
    (void)buf;
    (void)cap;
    return -1;
#else
    int64_t n = g_tau_n;
    g_tau_trace = cap > 0 ? buf : NULL;
    g_tau_cap = cap > 0 ? cap : 0;
    g_tau_n = 0;
    return n;
#endif
}

/* Direct SSA for one node from its current time t0 = T - 1 (or tspan[0])
 * up to the next unit of time T (Appendix A).  Returns an error code. */
static int ssa_node_day(const oracle_model *m, int node, int rep, int T,
                        double t0, int *u, const double *v, uint64_t seed,
                        int64_t *reactions)
{
    double w[ORACLE_MAX_TRANS];
    const double *ld = m->ldata + (size_t)node * (size_t)m->n_ldata;
    uint32_t ctr[4], key[2], x[4];
    double t = t0;
    int j, k;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    ctr[0] = 0;
    ctr[1] = (uint32_t)node;
    ctr[2] = (uint32_t)T;
    ctr[3] = ((uint32_t)ORACLE_STREAM_SSA << 24) | (uint32_t)rep;

    /* Reading: all rates are computed at the start of every day, so that
     * changes made by events and the post time step are always seen. */
    for (j = 0; j < m->n_trans; j++) {
        w[j] = model_rate(m, j, u, v, ld, m->gdata);
        if (!(w[j] >= 0.0) || isinf(w[j])) return ORACLE_ERR_RATE;
    }

    for (;;) {
        double lambda = 0.0, r1, r2, tau, target, cum;
        int n = -1, last_pos = -1;
        for (j = 0; j < m->n_trans; j++) lambda = lambda + w[j];
        /* Reading: with lambda = 0 no transition can fire; the node jumps
         * to T without consuming a draw. */
        if (!(lambda > 0.0)) break;
        /* Guard (not in the paper): rates so large that a node-day needs more
         * than 2^24 draws end the run with an error instead of running on. */
        if (ctr[0] >= ORACLE_MAX_DRAWS_PER_NODE_DAY) return ORACLE_ERR_STEP_LIMIT;
        oracle_philox4x32_10(ctr, key, x);
        ctr[0] += 1;
        r1 = oracle_u01(x[0], x[1]);
        r2 = oracle_u01(x[2], x[3]);
        tau = -oracle_log(r1) / lambda;
        if (g_tau_trace && ctr[0] == 1 && g_tau_n < g_tau_cap) {
            g_tau_trace[g_tau_n].rep = rep;
            g_tau_trace[g_tau_n].node = node;
            g_tau_trace[g_tau_n].T = T;
            g_tau_trace[g_tau_n].tau = tau;
            g_tau_n++;
        }
        if (t + tau >= (double)T) break;
        t = t + tau;
        /* Inversion: the smallest n with lambda r2 <= sum_{j<=n} w_j, summed
         * in index order over the positive rates.  Reading: if rounding
         * leaves no such n, take the last positive rate. */
        target = lambda * r2;
        cum = 0.0;
        for (j = 0; j < m->n_trans; j++) {
            if (!(w[j] > 0.0)) continue;
            cum = cum + w[j];
            last_pos = j;
            if (target <= cum) {
                n = j;
                break;
            }
        }
        if (n < 0) n = last_pos;
        for (k = 0; k < m->n_comp; k++)
            u[k] += m->S[(size_t)n * (size_t)m->n_comp + (size_t)k];
        for (k = 0; k < m->n_trans; k++) {
            if (m->G[(size_t)n * (size_t)m->n_trans + (size_t)k] == 0) continue;
            w[k] = model_rate(m, k, u, v, ld, m->gdata);
            if (!(w[k] >= 0.0) || isinf(w[k])) return ORACLE_ERR_RATE;
        }
        *reactions += 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The 'aem' solver (Sec. 3.4.2): transitions carried out in channels with   */
/* private random streams.  Reading: channel (node i, transition j) owns the */
/* Philox stream with counter (c_ij, i, j, (3 << 24) | replicate), c_ij the */
/* number of draws the channel has taken so far, and the channels are advanced by the next reaction method of   */
/* Gibson and Bruck (J. Phys. Chem. A 104, 2000): every channel holds an     */
/* absolute firing time tau_ij; the earliest one fires; the fired channel    */
/* draws a fresh exponential, and a channel whose rate changed from a_old > 0 */
/* to a_new > 0 rescales its residual waiting time by a_old / a_new, which   */
/* keeps it exponential with the new rate.  A channel whose rate drops to 0  */
/* sleeps (tau = +inf); one that wakes draws a fresh exponential (memoryless  */
/* property).  Residual times carry over from day to day: at the start of    */
/* every day the rates of all channels are recomputed (events and the post   */
/* time step may have changed u and v) and the same update rule is applied. */
/* ------------------------------------------------------------------------ */

/* Exponential(1) draw number *cnt of channel (node, j): -log u, u from the
 * first two words of Philox call (*cnt, node, j, (3 << 24) | rep). */
static int aem_draw(uint64_t seed, int node, int j, int rep, uint32_t *cnt,
                    double *E)
{
    uint32_t ctr[4], key[2], x[4];
    if (*cnt == UINT32_MAX) return ORACLE_ERR_STEP_LIMIT;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    ctr[0] = *cnt;
    ctr[1] = (uint32_t)node;
    ctr[2] = (uint32_t)j;
    ctr[3] = ((uint32_t)ORACLE_STREAM_AEM << 24) | (uint32_t)rep;
    oracle_philox4x32_10(ctr, key, x);
    *cnt += 1;
    *E = -oracle_log(oracle_u01(x[0], x[1]));
    return 0;
}

/* The update rule of channel j at time t when its rate becomes a_new. */
static int aem_update(uint64_t seed, int node, int j, int rep, double t,
                      double a_new, double *a, double *tau, uint32_t *cnt)
{
    double E;
    int rc;
    if (a_new == a[j]) return 0;  /* unchanged rate: nothing to do */
    if (a[j] > 0.0 && a_new > 0.0) {
        tau[j] = t + (a[j] / a_new) * (tau[j] - t);
    } else if (a_new > 0.0) {
        rc = aem_draw(seed, node, j, rep, &cnt[j], &E);
        if (rc) return rc;
        tau[j] = t + E / a_new;
    } else {
        tau[j] = INFINITY;
    }
    a[j] = a_new;
    return 0;
}

/* One node from t0 = T - 1 to T under the all events method.  a, tau, cnt
 * are the node's n_trans channel states (a = 0, tau = +inf, cnt = 0 before
 * the first day). */
static int aem_node_day(const oracle_model *m, int node, int rep, int T,
                        double t0, int *u, const double *v, double *a,
                        double *tau, uint32_t *cnt, uint64_t seed,
                        int64_t *reactions)
{
    const double *ld = m->ldata + (size_t)node * (size_t)m->n_ldata;
    double t = t0;
    uint32_t fired = 0;
    int j, k, rc;

    for (j = 0; j < m->n_trans; j++) {
        double w = model_rate(m, j, u, v, ld, m->gdata);
        if (!(w >= 0.0) || isinf(w)) return ORACLE_ERR_RATE;
        rc = aem_update(seed, node, j, rep, t, w, a, tau, cnt);
        if (rc) return rc;
    }
    for (;;) {
        /* the earliest channel; ties go to the lowest index */
        int mu = -1;
        double best = INFINITY, E;
        for (j = 0; j < m->n_trans; j++) {
            if (tau[j] < best) {
                best = tau[j];
                mu = j;
            }
        }
        if (mu < 0 || best >= (double)T) break;
        /* Guard (not in the paper), as for the direct method. */
        if (fired >= ORACLE_MAX_DRAWS_PER_NODE_DAY) return ORACLE_ERR_STEP_LIMIT;
        fired++;
        t = best;
        for (k = 0; k < m->n_comp; k++)
            u[k] += m->S[(size_t)mu * (size_t)m->n_comp + (size_t)k];
        *reactions += 1;
        /* the rates column mu of G marks; the fired channel itself always
         * draws a fresh waiting time */
        for (k = 0; k < m->n_trans; k++) {
            double w;
            if (k != mu && m->G[(size_t)mu * (size_t)m->n_trans + (size_t)k] == 0)
                continue;
            w = a[k];
            if (m->G[(size_t)mu * (size_t)m->n_trans + (size_t)k] != 0) {
                w = model_rate(m, k, u, v, ld, m->gdata);
                if (!(w >= 0.0) || isinf(w)) return ORACLE_ERR_RATE;
            }
            if (k == mu) {
                a[k] = w;
                if (w > 0.0) {
                    rc = aem_draw(seed, node, k, rep, &cnt[k], &E);
                    if (rc) return rc;
                    tau[k] = t + E / w;
                } else {
                    tau[k] = INFINITY;
                }
            } else {
                rc = aem_update(seed, node, k, rep, t, w, a, tau, cnt);
                if (rc) return rc;
            }
        }
    }
    return 0;
}

int oracle_run(const oracle_model *m, const oracle_events *ev,
               const int *tspan, int n_tspan, uint64_t seed, int n_rep,
               const int *u0, const double *v0, int *U, double *V,
               int64_t *reactions, oracle_error *err)
{
    return oracle_run_reps(m, ev, tspan, n_tspan, seed, 0, n_rep, n_rep, u0,
                           v0, U, V, reactions, err);
}

/* Replicates rep0 .. rep0 + n_rep - 1 of a run with n_rep_total replicates
 * (each replicate's random streams and events depend on its index only);
 * u0, v0, U, V, reactions hold those n_rep replicates. */
int oracle_run_reps(const oracle_model *m, const oracle_events *ev,
                    const int *tspan, int n_tspan, uint64_t seed, int rep0,
                    int n_rep, int n_rep_total, const int *u0, const double *v0,
                    int *U, double *V, int64_t *reactions, oracle_error *err)
{
    const int C = m->n_comp, Nv = m->n_v, Nn = m->n_nodes;
    const size_t ustride = (size_t)Nn * (size_t)C;
    const size_t vstride = (size_t)Nn * (size_t)Nv;
    ev_key *order = NULL;
    int64_t n_sorted = 0, e;
    int r, rc;
    int *u = NULL;
    double *v = NULL, *vtmp = NULL;
    double *aem_a = NULL, *aem_tau = NULL;
    uint32_t *aem_cnt = NULL;
    const size_t nch = (size_t)Nn * (size_t)m->n_trans;

    if (err) memset(err, 0, sizeof *err);
    if (rep0 < 0 || n_rep < 1 || rep0 + n_rep > n_rep_total) {
        set_error(err, ORACLE_ERR_ARG, -1, -1, -1, -1);
        return ORACLE_ERR_ARG;
    }
    rc = validate(m, ev, tspan, n_tspan, n_rep_total, err);
    if (rc) return rc;

    /* Events sorted by (time, type, list index): same-time events run in
     * the order exit, enter, internal transfer, external transfer (Sec. 3.3),
     * equal keys keep list order.  Events after tspan's end never run. */
    if (ev && ev->n > 0) {
        order = (ev_key *)malloc((size_t)ev->n * sizeof *order);
        if (!order) return ORACLE_ERR_NOMEM;
        for (e = 0; e < ev->n; e++) {
            if (ev->time[e] > tspan[n_tspan - 1]) continue;
            order[n_sorted].idx = e;
            order[n_sorted].time = ev->time[e];
            order[n_sorted].type = ev->event[e];
            n_sorted++;
        }
        qsort(order, (size_t)n_sorted, sizeof *order, ev_key_cmp);
    }

    u = (int *)malloc((ustride ? ustride : 1) * sizeof *u);
    v = (double *)malloc((vstride ? vstride : 1) * sizeof *v);
    vtmp = (double *)malloc((Nn ? Nn : 1) * sizeof *vtmp);
    if (m->solver == ORACLE_SOLVER_AEM) {
        aem_a = (double *)malloc((nch ? nch : 1) * sizeof *aem_a);
        aem_tau = (double *)malloc((nch ? nch : 1) * sizeof *aem_tau);
        aem_cnt = (uint32_t *)malloc((nch ? nch : 1) * sizeof *aem_cnt);
    }
    if (!u || !v || !vtmp ||
        (m->solver == ORACLE_SOLVER_AEM && (!aem_a || !aem_tau || !aem_cnt))) {
        free(order); free(u); free(v); free(vtmp);
        free(aem_a); free(aem_tau); free(aem_cnt);
        return ORACLE_ERR_NOMEM;
    }

    for (r = 0; r < n_rep; r++) {
        const int rep = rep0 + r;
        int T, m_rec = 1, node;
        int64_t cursor = 0;
        memcpy(u, u0 + (size_t)r * ustride, ustride * sizeof *u);
        if (vstride) memcpy(v, v0 + (size_t)r * vstride, vstride * sizeof *v);
        if (reactions) reactions[r] = 0;
        if (aem_a) {
            size_t q;
            for (q = 0; q < nch; q++) {
                aem_a[q] = 0.0;
                aem_tau[q] = INFINITY;
                aem_cnt[q] = 0;
            }
        }
        /* U[, 1] = u0 and V[, 1] = v0: the state at tspan[0]. */
        memcpy(U + (size_t)r * (size_t)n_tspan * ustride, u,
               ustride * sizeof *u);
        if (vstride)
            memcpy(V + (size_t)r * (size_t)n_tspan * vstride, v,
                   vstride * sizeof *v);

        for (T = tspan[0] + 1; T <= tspan[n_tspan - 1]; T++) {
            int64_t seg_begin = cursor, seg_end;
            double t0 = (double)(T - 1);
            int64_t nr = 0;

            /* (1) local stochastic step, Eq. numstep1, node by node.  The
             * nodes are independent; the timing build (OpenMP) runs them in
             * parallel as the paper's solver does (Sec. 3.4.2).  Either way
             * the failing node with the lowest index is reported. */
            {
                int bad_node = -1, bad_rc = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(guided) reduction(+ : nr)
#endif
                for (node = 0; node < Nn; node++) {
                    int64_t nr_node = 0;
                    int rc_node;
#ifndef _OPENMP
                    if (bad_node >= 0) continue;
#endif
                    if (aem_a) {
                        const size_t o = (size_t)node * (size_t)m->n_trans;
                        rc_node = aem_node_day(m, node, rep, T, t0, u + (size_t)node * C,
                                               v + (size_t)node * Nv, aem_a + o,
                                               aem_tau + o, aem_cnt + o, seed, &nr_node);
                    } else {
                        rc_node = ssa_node_day(m, node, rep, T, t0, u + (size_t)node * C,
                                               v + (size_t)node * Nv, seed, &nr_node);
                    }
                    nr += nr_node;
                    if (rc_node) {
#ifdef _OPENMP
#pragma omp critical(oracle_first_bad_node)
#endif
                        {
                            if (bad_node < 0 || node < bad_node) {
                                bad_node = node;
                                bad_rc = rc_node;
                            }
                        }
                    }
                }
                if (bad_node >= 0) {
                    set_error(err, bad_rc, rep, bad_node, -1, T);
                    rc = bad_rc;
                    goto done;
                }
            }
            if (reactions) reactions[r] += nr;

            /* Events whose time has been reached: time <= T.  Reading: the
             * events dated tspan[0] or earlier run at the first unit of
             * time. */
            seg_end = seg_begin;
            while (seg_end < n_sorted && order[seg_end].time <= T) seg_end++;
            cursor = seg_end;

            /* (2) data step, Eq. numstep2: E1 events in sorted order, then
             * E2 events in sorted order.  An E1 event touches one node only,
             * so in the timing build each thread applies the E1 events of
             * its own range of nodes (in sorted order, as the paper's node
             * threads do); E2 events stay serial (Sec. 3.4.2).  The first
             * failing E1 event in sorted order is reported. */
            {
                int64_t bad_e = -1;
                int bad_rc = 0;
#ifdef _OPENMP
#pragma omp parallel
#endif
                {
                    int nth = 1, me = 0, nd_lo, nd_hi;
                    int64_t e1;
#ifdef _OPENMP
                    nth = omp_get_num_threads();
                    me = omp_get_thread_num();
#endif
                    nd_lo = (int)(((int64_t)Nn * me) / nth);
                    nd_hi = (int)(((int64_t)Nn * (me + 1)) / nth);
                    for (e1 = seg_begin; e1 < seg_end; e1++) {
                        int64_t idx = order[e1].idx;
                        int type = ev->event[idx], nd = ev->node[idx], rc1;
                        if (type == ORACLE_EV_EXTERNAL) continue;
                        if (ev->rep && ev->rep[idx] != rep) continue;
                        if (nd < nd_lo || nd >= nd_hi) continue;
                        rc1 = oracle_apply_event(
                            C, m->E, m->n_select, m->N, m->n_shift, type,
                            u + (size_t)nd * C, NULL, ev->n_ind[idx],
                            ev->proportion[idx], ev->select[idx], ev->shift[idx],
                            seed, idx, rep);
                        if (rc1) {
#ifdef _OPENMP
#pragma omp critical(oracle_first_bad_event)
#endif
                            {
                                if (bad_e < 0 || e1 < bad_e) {
                                    bad_e = e1;
                                    bad_rc = rc1;
                                }
                            }
                            break;
                        }
                    }
                }
                if (bad_e >= 0) {
                    int64_t idx = order[bad_e].idx;
                    set_error(err, bad_rc, rep, ev->node[idx], idx, T);
                    rc = bad_rc;
                    goto done;
                }
            }
            for (e = seg_begin; e < seg_end; e++) {
                int64_t idx = order[e].idx;
                int type = ev->event[idx];
                int nd = ev->node[idx], ds = ev->dest[idx];
                if (type != ORACLE_EV_EXTERNAL) continue;
                if (ev->rep && ev->rep[idx] != rep) continue;
                rc = oracle_apply_event(
                    C, m->E, m->n_select, m->N, m->n_shift, type,
                    u + (size_t)nd * C, u + (size_t)ds * C,
                    ev->n_ind[idx], ev->proportion[idx], ev->select[idx],
                    ev->shift[idx], seed, idx, rep);
                if (rc) {
                    set_error(err, rc, rep, nd, idx, T);
                    goto done;
                }
            }

            /* (3) post time step, Eq. numstep3, on the state after events;
             * node-parallel in the timing build, the failing node with the
             * lowest index reported */
            if (m->kind == ORACLE_SISE_SP) {
                /* every node from the same old values: new values first */
                int bad_node = -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
                for (node = 0; node < Nn; node++) {
                    if (sise_sp_pts(m, node, u, v, T, &vtmp[node])) {
#ifdef _OPENMP
#pragma omp critical(oracle_first_bad_node)
#endif
                        {
                            if (bad_node < 0 || node < bad_node) bad_node = node;
                        }
                    }
                }
                if (bad_node >= 0) {
                    set_error(err, ORACLE_ERR_PTS, rep, bad_node, -1, T);
                    rc = ORACLE_ERR_PTS;
                    goto done;
                }
                memcpy(v, vtmp, (size_t)Nn * sizeof *v);
            }
            if (Nv > 0 && m->kind != ORACLE_SISE_SP) {
                int bad_node = -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
                for (node = 0; node < Nn; node++) {
                    double vn[ORACLE_MAX_V];
                    int ret;
                    memcpy(vn, v + (size_t)node * Nv, (size_t)Nv * sizeof *v);
                    ret = model_pts(m->kind, vn, u + (size_t)node * C,
                                    v + (size_t)node * Nv,
                                    m->ldata + (size_t)node * m->n_ldata,
                                    m->gdata, T);
                    if (ret < 0) {
#ifdef _OPENMP
#pragma omp critical(oracle_first_bad_node)
#endif
                        {
                            if (bad_node < 0 || node < bad_node) bad_node = node;
                        }
                        continue;
                    }
                    memcpy(v + (size_t)node * Nv, vn, (size_t)Nv * sizeof *v);
                }
                if (bad_node >= 0) {
                    set_error(err, ORACLE_ERR_PTS, rep, bad_node, -1, T);
                    rc = ORACLE_ERR_PTS;
                    goto done;
                }
            }

            /* (4) record when T reaches the next tspan point (Sec. 3.4.2) */
            if (m_rec < n_tspan && T == tspan[m_rec]) {
                memcpy(U + ((size_t)r * n_tspan + m_rec) * ustride, u,
                       ustride * sizeof *u);
                if (vstride)
                    memcpy(V + ((size_t)r * n_tspan + m_rec) * vstride, v,
                           vstride * sizeof *v);
                m_rec++;
            }
        }
    }
    rc = 0;
done:
    free(aem_a);
    free(aem_tau);
    free(aem_cnt);
    free(order);
    free(u);
    free(v);
    free(vtmp);
    return rc;
}
