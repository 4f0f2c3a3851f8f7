/*
 * siminf_oracle.h -- interface of the plain CPU oracle (test infrastructure
 * only; see siminf_oracle.c).  Shares nothing with the CUDA library.
 *
 * Layouts (all 0-based, all host memory, all owned by the caller):
 *   u0 [n_rep][n_nodes][n_comp] int, v0 [n_rep][n_nodes][n_v] double,
 *   U  [n_rep][n_tspan][n_nodes][n_comp] int,
 *   V  [n_rep][n_tspan][n_nodes][n_v] double   -- column m of the paper's U
 *   (Sec. 3.2) is U[rep][m], node-major with the compartments contiguous.
 *   S (n_comp x n_trans), G (n_trans x n_trans), E (n_comp x n_select),
 *   N (n_comp x n_shift) and ldata (n_ldata x n_nodes) are column-major, as
 *   in the paper's model slots (Sec. 3.2).
 * Event fields follow the event table of Sec. 3.3 with 0-based node, dest,
 * select and shift; shift < 0 means "no shift".  rep may be NULL (every
 * replicate runs every event) or give the replicate each event belongs to.
 */
#ifndef SIMINF_ORACLE_H
#define SIMINF_ORACLE_H

#include <stdint.h>

#define ORACLE_MAX_COMP 16
#define ORACLE_MAX_TRANS 16
#define ORACLE_MAX_V 16

enum {
    ORACLE_SIR = 0,
    ORACLE_SIS = 1,
    ORACLE_SISE = 2,
    ORACLE_SISE3 = 3,
    ORACLE_SISE_SP = 4,
    ORACLE_GENERIC = 5
};
enum {
    ORACLE_EV_EXIT = 0,
    ORACLE_EV_ENTER = 1,
    ORACLE_EV_INTERNAL = 2,
    ORACLE_EV_EXTERNAL = 3
};
enum { ORACLE_STREAM_SSA = 0, ORACLE_STREAM_EVENTS = 1, ORACLE_STREAM_AEM = 3 };
enum { ORACLE_SOLVER_SSM = 0, ORACLE_SOLVER_AEM = 1 };
enum {
    ORACLE_OK = 0,
    ORACLE_ERR_ARG = -1,
    ORACLE_ERR_EVENT_UNDERFLOW = -2,
    ORACLE_ERR_SHIFT_RANGE = -3,
    ORACLE_ERR_RATE = -4,
    ORACLE_ERR_PTS = -5,
    ORACLE_ERR_NOMEM = -8,
    ORACLE_ERR_STEP_LIMIT = -9
};

/* A node-day stops with ORACLE_ERR_STEP_LIMIT before its 2^24 + 1-th draw
 * (direct method) or firing ('aem'). */
#define ORACLE_MAX_DRAWS_PER_NODE_DAY (1u << 24)

typedef struct {
    int kind;
    int n_nodes, n_comp, n_trans;
    const int *S;
    const int *G;
    int n_select;
    const int *E;
    int n_shift;
    const int *N;
    int n_v;
    int n_ldata;
    const double *ldata;
    int n_gdata;
    const double *gdata;
    /* SISe_sp neighbours of node i: nb_idx[nb_ptr[i] .. nb_ptr[i+1]) with
     * distances nb_dist (NULL pointers: no neighbours) */
    const int64_t *nb_ptr;
    const int *nb_idx;
    const double *nb_dist;
    /* ORACLE_SOLVER_SSM (direct SSA per day) or ORACLE_SOLVER_AEM */
    int solver;
    /* ORACLE_GENERIC: propensity of transition j for counts u and global
     * data gdata (generated from transition strings, compiled separately) */
    double (*rate_fn)(int j, const int *u, const double *gdata);
} oracle_model;

typedef struct {
    int64_t n;
    const int *event, *time, *node, *dest, *n_ind;
    const double *proportion;
    const int *select, *shift, *rep;
} oracle_events;

typedef struct {
    int code, rep, node;
    int64_t event;
    int day;
} oracle_error;

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]);
double oracle_u01(uint32_t a, uint32_t b);
double oracle_log(double x);
uint32_t oracle_bounded_sequence(uint64_t seed, int64_t event_index, int rep,
                                 const uint32_t *ranges, int n, uint32_t *out);
int oracle_apply_event(int n_comp, const int *E, int n_select,
                       const int *N, int n_shift,
                       int type, int *u_node, int *u_dest, int n,
                       double proportion, int select, int shift,
                       uint64_t seed, int64_t event_index, int rep);
int oracle_run(const oracle_model *m, const oracle_events *ev,
               const int *tspan, int n_tspan, uint64_t seed, int n_rep,
               const int *u0, const double *v0, int *U, double *V,
               int64_t *reactions, oracle_error *err);
/* Replicates rep0 .. rep0 + n_rep - 1 of a run with n_rep_total replicates;
 * u0, v0, U, V and reactions hold only those. */
int oracle_run_reps(const oracle_model *m, const oracle_events *ev,
                    const int *tspan, int n_tspan, uint64_t seed, int rep0,
                    int n_rep, int n_rep_total, const int *u0, const double *v0,
                    int *U, double *V, int64_t *reactions, oracle_error *err);

/* Test hook: records of the first waiting time of every node-day with
 * lambda > 0 (direct method).  oracle_trace_first_tau(buf, cap) starts a
 * trace into buf (at most cap records; cap = 0 stops tracing) and returns
 * the number of records of the previous trace; -1 in the OpenMP build. */
typedef struct {
    int rep, node, T;
    double tau;
} oracle_tau_record;
int64_t oracle_trace_first_tau(oracle_tau_record *buf, int64_t cap);

#endif
