/*
 * siminf_gpu.h -- C ABI of the GB300 (sm_103a) engine for the SimInf
 * split-step method (Widgren, Bauer, Eriksson, Engblom, arXiv 1605.01421).
 *
 * The library runs, for every replicate and node, the direct-method SSA
 * between unit time points (Sec. 2.3 Eq. numstep1, Appendix A), the scheduled
 * events (Sec. 2.3 Eq. numstep2, Sec. 3.3), the post time step update of the
 * continuous state (Eq. numstep3) and the recording of U and V at the tspan
 * points (Sec. 3.2).  Every step runs in CUDA kernels on one GPU.
 *
 * Conventions for every call:
 *   - Indices are 0-based: node, dest, select and shift columns.  shift < 0
 *     means "no shift" (the paper's 1-based shift = 0).
 *   - Matrices S, G, E, N and ldata are column-major, as the paper's model
 *     slots (Sec. 3.2 table of SimInf_model slots): column j of S is the
 *     state change of transition j; ldata column i is node i's local data.
 *   - Return value: SG_OK (0) or a negative SG_ERR_* code.  No call aborts
 *     the process; a failed call leaves the model usable.
 *   - Host arrays passed to sg_model_create / sg_set_events are copied; the
 *     caller may free them after the call.  Device pointers passed to sg_run
 *     stay owned by the caller; the library never frees them.
 *   - The library owns the sg_model and the device memory behind it (model
 *     tables, event plan, working state); sg_model_destroy releases it.
 *   - One sg_model must not be used from two threads at once.
 */
#ifndef SIMINF_GPU_H
#define SIMINF_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SG_MAX_COMP 16   /* compartments per node */
#define SG_MAX_TRANS 16  /* transitions per node */
#define SG_MAX_SELECT 32 /* columns of E */
#define SG_MAX_SHIFT 32  /* columns of N */

/* Built-in models.  Transition-rate functions (TRFun) and the post time step
 * (PTSFun) of Sec. 3.4.1 are compiled device functions, one set per kind;
 * the model tables S, G, E, N are data.
 *   SG_SIR   Eq. (SIR) and the rate listing of Appendix C: S -> I at
 *            beta S I / (S + I + R), I -> R at gamma I.  gdata = [beta,
 *            gamma].  No continuous state.
 *   SG_SIS   Sec. 2.1 example: R(x) = [beta S I, gamma I].  gdata = [beta,
 *            gamma].
 *   SG_SISE  Sec. 4.2 without spatial coupling: S -> I at upsilon phi S,
 *            I -> S at gamma I; phi' = alpha I / N - beta(t) phi.  gdata =
 *            [upsilon, gamma, alpha, beta_t1..beta_t4]; ldata = [end_t1..
 *            end_t4] per node; v = [phi].
 *   SG_SISE3 SISe per age class, compartments [S1,I1,S2,I2,S3,I3]; gdata =
 *            [upsilon_1..3, gamma_1..3, alpha, beta_t1..beta_t4]; ldata and
 *            v as SG_SISE.
 *   SG_SISE_SP SISe with the spatial coupling term of the environmental
 *            pressure ODE of Sec. 4.2: phi_i' = alpha I_i / N_i + sum_k
 *            (phi_k N_k - phi_i N_i) / N_i * D / d_ik - beta(t) phi_i over the
 *            node's neighbours k (sg_set_neighbors), all nodes updated from the
 *            same old values (one Euler step of length 1); both terms are 0 in
 *            an empty node.  gdata = [upsilon, gamma, alpha, beta_t1..beta_t4,
 *            D]; ldata and v as SG_SISE.                                     */
typedef enum {
  SG_SIR = 0,
  SG_SIS = 1,
  SG_SISE = 2,
  SG_SISE3 = 3,
  SG_SISE_SP = 4,
  SG_GENERIC = 5 /* from transition strings, sg_model_create_parsed */
} sg_model_kind;

/* Solvers of Sec. 3.4.2.  Both process the scheduled events and the post
 * time step once per unit of time; they differ in how transitions fire
 * between those points.
 *   SG_SOLVER_SSM  split-step method: per node and day, direct SSA
 *                  (Appendix A) with one random stream for all transitions,
 *                  Philox counter (draw, node, day, (0 << 24) | replicate).
 *   SG_SOLVER_AEM  all events method: every (node, transition) is a channel
 *                  with its own random stream, Philox counter (draws taken by
 *                  the channel, node, transition, (3 << 24) | replicate),
 *                  advanced by the next reaction method of Gibson and Bruck
 *                  (absolute firing times; the earliest fires and redraws;
 *                  a channel whose rate changes from a > 0 to a' > 0 rescales
 *                  its residual time by a / a'; rate 0 sleeps, waking
 *                  redraws).  Firing times carry over between days, and every
 *                  rate is recomputed at each day start.  The draw is
 *                  E = -log u with u from the first two words of the call. */
typedef enum { SG_SOLVER_SSM = 0, SG_SOLVER_AEM = 1 } sg_solver;

/* Event types, coded as in the event table of Sec. 3.3. */
typedef enum {
  SG_EXIT = 0,
  SG_ENTER = 1,
  SG_INTERNAL_TRANSFER = 2,
  SG_EXTERNAL_TRANSFER = 3
} sg_event_type;

enum {
  SG_OK = 0,
  SG_ERR_ARG = -1,             /* invalid argument or table entry          */
  SG_ERR_EVENT_UNDERFLOW = -2, /* an event moves more individuals than the
                                  selected compartments hold (Sec. 4.1)     */
  SG_ERR_SHIFT_RANGE = -3,     /* p + N[p, q] outside the compartments     */
  SG_ERR_RATE = -4,            /* negative or non-finite transition rate   */
  SG_ERR_PTS = -5,             /* post time step returned an error         */
  SG_ERR_TIMEOUT = -6,         /* a bounded device wait gave up            */
  SG_ERR_CUDA = -7,            /* a CUDA runtime call failed               */
  SG_ERR_NOMEM = -8,           /* host or device allocation failed         */
  SG_ERR_STEP_LIMIT = -9,      /* a node needed more than SG_MAX_DRAWS draws
                                  in one unit step (rates far too large)    */
  SG_ERR_TOO_LARGE = -10,      /* the problem does not fit the fixed scratch
                                  of sg_run_noalloc                         */
  SG_ERR_PARSE = -11,          /* a transition string does not parse       */
  SG_ERR_JIT = -12             /* run-time compilation or loading failed   */
};

/* Draws one node may take in one unit step before the run stops with
 * SG_ERR_STEP_LIMIT: a bound on kernel run time, not part of the method. */
#define SG_MAX_DRAWS (1u << 24)

typedef struct sg_model sg_model; /* opaque, library-owned */

/* Model description: the slots of the SimInf_model class (Sec. 3.2). */
typedef struct {
  int32_t kind;     /* sg_model_kind                                        */
  int32_t n_nodes;  /* Nnodes >= 0                                          */
  int32_t n_comp;   /* Ncomp: must equal the kind's compartment count       */
  int32_t n_trans;  /* Ntrans: must equal the kind's transition count       */
  const int32_t *S; /* n_comp x n_trans state-change matrix (column-major)  */
  const int32_t *G; /* n_trans x n_trans dependency graph: G[k, j] != 0
                       means rate k is recomputed after transition j         */
  int32_t n_select; /* columns of E                                         */
  const int32_t *E; /* n_comp x n_select select matrix; non-zero = selected */
  int32_t n_shift;  /* columns of N (may be 0)                              */
  const int32_t *N; /* n_comp x n_shift shift matrix (compartment offsets)  */
  int32_t n_v;      /* continuous states per node: the kind's count         */
  int32_t n_ldata;  /* local data per node (>= the kind's requirement)      */
  const double *ldata; /* n_ldata x n_nodes                                 */
  int32_t n_gdata;  /* global data entries (>= the kind's requirement)      */
  const double *gdata;
} sg_desc;

/* First error seen by a run (code 0 if none); -1 marks "not applicable". */
typedef struct {
  int32_t code;
  int32_t rep;
  int32_t node;
  int32_t day; /* the unit time point T being simulated toward */
  int64_t event; /* index of the event in the list given to sg_set_events */
} sg_error;

typedef struct {
  int64_t reactions;      /* SSA transitions fired, all replicates         */
  int64_t draws;          /* SSA random draws (Philox calls), all replicates*/
  int64_t node_days;      /* replicates x nodes x unit time steps           */
  int64_t events_applied; /* scheduled events run, all replicates           */
  int64_t kernel_launches;/* kernels this run launched                      */
  int32_t e2_waves;       /* external-transfer waves over the run           */
  int32_t days;           /* unit time steps simulated                      */
  /* Per-kernel device time, filled only when kernel timing is enabled
   * (sg_set_kernel_timing): CUDA events around every launch.               */
  double ms_ssa;          /* SSA + post time step + recording kernels       */
  double ms_e1;           /* exit / enter / internal-transfer kernels       */
  double ms_e2;           /* external-transfer wave kernels                 */
  int64_t launches_ssa, launches_e1, launches_e2;
  double ms_mlp;          /* emulator kernels (features, GEMMs, sampling)    */
  int64_t launches_mlp;
  double ms_host_plan;    /* host time of this call spent sorting, planning
                             and uploading the events (0 when the plan of an
                             earlier run was reused)                        */
  double ms_host_total;   /* host time of the whole call                    */
  int64_t node_days_rated;/* node-days whose transition rates were evaluated:
                             all of them on the thread-per-node schedule, the
                             non-quiescent ones on the sparse-activity schedule
                             (see sg_set_tuning)                            */
} sg_stats;

/* Create a model from its tables (Sec. 3.2).  Validates the sizes against
 * the kind, copies every table to the device and returns the handle in
 * *out.  Errors: SG_ERR_ARG, SG_ERR_NOMEM, SG_ERR_CUDA. */
int sg_model_create(const sg_desc *desc, sg_model **out);

/* Create a model from transition strings (Sec. 3.5, the model parser):
 * transitions[j] = "LHS -> propensity -> RHS", LHS / RHS "@" (the empty
 * set) or compartment names joined by "+" (optionally "k*name"); the
 * propensity is an expression over compartment names (the node's counts),
 * the names in gdata_names (values gdata), decimal numbers, + - * /, unary
 * minus and parentheses; * and / bind tighter than + and -, all group left
 * to right, and each operation is one IEEE double operation.  The parser
 * builds S (S[p, j] = count of p on the RHS minus on the LHS) and G (G[k, j]
 * = 1 when propensity k reads a compartment transition j changes); the
 * propensities become CUDA code, compiled at run time with NVRTC for sm_103a
 * together with the engine's day and event kernels, and loaded on the
 * current device (the model must then run on that device).  E (n_comp x
 * n_select) and N (n_comp x n_shift) are the event tables of Sec. 3.3,
 * column-major.  The model has no continuous state and no local data.
 * Host arrays are copied.  msg (msg_len bytes, may be NULL) receives the
 * parse or compiler message.  Errors: SG_ERR_ARG, SG_ERR_PARSE, SG_ERR_JIT,
 * SG_ERR_NOMEM, SG_ERR_CUDA. */
int sg_model_create_parsed(const char *const *transitions, int32_t n_trans,
                           const char *const *compartments, int32_t n_comp,
                           const char *const *gdata_names, const double *gdata,
                           int32_t n_gdata, int32_t n_nodes, const int32_t *E,
                           int32_t n_select, const int32_t *N, int32_t n_shift,
                           sg_model **out, char *msg, int32_t msg_len);

/* The model's S (n_comp x n_trans) and G (n_trans x n_trans) as the engine
 * uses them, column-major, into caller arrays (either may be NULL). */
int sg_model_tables(const sg_model *m, int32_t *S, int32_t *G);

/* SG_SISE_SP neighbour lists (the distance matrix of Sec. 4.2 within a
 * cutoff), compressed rows: node i's neighbours are idx[ptr[i] .. ptr[i+1])
 * with distances dist[..] (> 0, finite), summed in that order.  ptr has
 * n_nodes + 1 entries, ptr[0] = 0.  Host arrays, copied.  Without a call the
 * nodes have no neighbours.  Errors: SG_ERR_ARG, SG_ERR_NOMEM. */
int sg_set_neighbors(sg_model *m, const int64_t *ptr, const int32_t *idx, const double *dist);

/* Replace the model's scheduled events (event table of Sec. 3.3): n_events
 * entries of type event[e] at integer time[e] on node[e] (and dest[e] for
 * external transfers), moving n[e] individuals, or, when n[e] == 0 and the
 * type samples, round(proportion[e] * selected total) (half away from zero),
 * sampled without replacement from the compartments of column select[e] of E
 * and shifted by column shift[e] of N.  rep may be NULL (every replicate runs
 * every event) or give each event's replicate.  The events are validated
 * (types, node and dest ranges, select / shift columns, n >= 0, 0 <=
 * proportion <= 1, internal transfers need a shift, shifts must keep every
 * selectable compartment in range), sorted and planned on the host, and
 * copied to the device.  Errors: SG_ERR_ARG, SG_ERR_SHIFT_RANGE,
 * SG_ERR_NOMEM, SG_ERR_CUDA. */
int sg_set_events(sg_model *m, int64_t n_events, const int32_t *event,
                  const int32_t *time, const int32_t *node, const int32_t *dest,
                  const int32_t *n, const double *proportion,
                  const int32_t *select, const int32_t *shift,
                  const int32_t *rep);

/* Host only (no device is touched): the schedule that sg_run builds from an
 * event table for the window of unit steps T = t0 + 1 .. t_end (Sec. 3.3 and
 * Appendix A, "Process E1 events" / "Process E2 events"), for inspection and
 * tests.  Day d = T - t0 - 1 runs the events with time in (T - 1, T]; day 0
 * also every earlier time; events after t_end never run.  Events as in
 * sg_set_events (type, time, node, dest; rep NULL for slots = 1, else each
 * event's replicate in 0 .. slots - 1).
 *   E1 events (exit, enter, internal transfer): per (slot, node), ordered by
 *     (day, time on day 0, type, list index);
 *   E2 events (external transfers): per (day, slot), split into waves: an
 *     event goes one wave after the last earlier event of its bucket that
 *     sampled its source, added to its source or sampled its destination,
 *     list order kept inside a wave.
 * Two calls: with order == NULL, counts[0..2] = (n_e1, n_e2, n_waves); then,
 * with caller arrays of those sizes, order[n_e1 + n_e2] (event indices: the
 * E1 part by (slot, node), then the E2 part by (day, slot) and wave),
 * e1_day[n_e1], e1_node_off[slots * n_nodes + 1] (into order),
 * e2_wave_off[days * slots + 1] (into wave_ev) and wave_ev[n_waves + 1]
 * (positions in order; wave w is wave_ev[w] .. wave_ev[w + 1]).  Errors:
 * SG_ERR_ARG (a node, dest, type or rep out of range, t_end < t0). */
int sg_plan_events(int64_t n_events, const int32_t *type, const int32_t *time,
                   const int32_t *node, const int32_t *dest, const int32_t *rep,
                   int32_t n_nodes, int32_t t0, int32_t t_end, int32_t slots, int64_t *counts,
                   int64_t *order, int32_t *e1_day, int64_t *e1_node_off,
                   int64_t *e2_wave_off, int64_t *wave_ev);

/* Run n_rep independent trajectories over tspan (n_tspan >= 1 strictly
 * increasing integers; the simulation covers unit steps T = tspan[0] + 1 ..
 * tspan[n_tspan - 1]) with Philox key `seed`, on the caller's CUDA stream
 * (cudaStream_t passed as void*, NULL = legacy default stream).
 *   d_u0 [n_rep][n_nodes][n_comp] int32   device, read
 *   d_v0 [n_rep][n_nodes][n_v]    double  device, read (NULL if n_v == 0)
 *   d_U  [n_rep][n_tspan][n_nodes][n_comp] int32  device, written: U[r][m]
 *        is column m of the paper's U (node-major, compartments contiguous)
 *   d_V  [n_rep][n_tspan][n_nodes][n_v]    double device, written (NULL if
 *        n_v == 0)
 * Events dated tspan[0] or earlier run at the first step; events after the
 * last tspan point never run.  The call enqueues all work, then waits for
 * the stream and reads back the error word and counters.  stats and err may
 * be NULL.  Errors: any SG_ERR_* (err says where). */
int sg_run(sg_model *m, const int32_t *tspan, int32_t n_tspan, uint64_t seed,
           int32_t n_rep, const int32_t *d_u0, const double *d_v0,
           int32_t *d_U, double *d_V, void *stream, sg_stats *stats,
           sg_error *err);

/* sg_run on host buffers (same shapes): copies u0 / v0 to the device,
 * runs, and copies U / V back, all on `stream`.  Device buffers for the
 * copies are allocated by the library and kept for reuse.  Host buffers in
 * page-locked memory give full copy bandwidth. */
int sg_run_host(sg_model *m, const int32_t *tspan, int32_t n_tspan,
                uint64_t seed, int32_t n_rep, const int32_t *u0,
                const double *v0, int32_t *U, double *V, void *stream,
                sg_stats *stats, sg_error *err);

/* Enable (1) or disable (0) per-kernel timing: sg_run then brackets every
 * kernel launch with CUDA events on its stream and fills the ms_* fields of
 * sg_stats.  Off by default (the events add host work per launch). */
int sg_set_kernel_timing(sg_model *m, int enable);

/* Run a shard of a job with several replicates (replicas only across GPUs:
 * replicates are independent trajectories, Sec. 3.4.2 runs one realisation
 * per call).  After this call, sg_run's n_rep replicates are the job's
 * global replicates rep0 .. rep0 + n_rep - 1 out of rep_total: every random
 * stream (SSA draws, event sampling, 'aem' channels) and every error report
 * uses the global index, so the shards of one job together reproduce the
 * whole job's run bit for bit; u0 / v0 / U / V hold the shard's n_rep
 * replicates only.  With per-replicate events (sg_set_events with a
 * replicate column) the event table may be the whole job's: the events of
 * other replicates are left out.  rep_total = 0 (and rep0 = 0) restores a
 * whole job (the default).  Returns SG_ERR_ARG for rep0 < 0, rep0 >=
 * rep_total, rep_total > 2^24, or a learned emulator set (the emulator
 * runs whole jobs only); sg_run returns SG_ERR_ARG when rep0 + n_rep >
 * rep_total or an event's replicate is >= rep_total. */
int sg_set_replicate_range(sg_model *m, int32_t rep0, int32_t rep_total);

/* Work split of the SSA day kernel.  With nodes_per_block in 1..128 each
 * block of 128 threads owns that many (replicate, node) pairs, one per
 * thread, kept in registers for a run of days; a node whose SSA needs more
 * than heavy_after draws in a day is handed to one of the block's warps,
 * whose 32 lanes compute 32 draws' random numbers at once.  With
 * nodes_per_block > 128 (up to 2^22; the direct method on the built-in
 * kinds without emulator or persistent schedule -- elsewhere it
 * means 128) the sparse-activity schedule runs instead: each block of 256
 * threads owns nodes_per_block pairs in device memory, skips the days that
 * are certainly empty (no infected animal and phi == +0, with finite model
 * parameters), and runs the SSA of the pairs with a positive total rate from
 * a compact list, one thread each, handing those that need more than
 * heavy_after draws to warps.  When nodes_per_block is also a multiple of
 * the node count (every block holds whole replicates) the whole run is one
 * launch: each block runs its replicates' external transfers itself and no
 * block waits for another.  Results are identical for every setting (the
 * random stream is a function of replicate, node, day and draw index only);
 * only speed changes.  nodes_per_block <= 0 or heavy_after < 0 restore the
 * size-based defaults: where the sparse-activity schedule applies and the
 * pairs exceed two full 128-pair blocks per SM, one replicate per block
 * and heavy_after 32 when there are at least as many replicates as SMs
 * (and more than 128 nodes), else two blocks per SM and heavy_after 8;
 * otherwise 128 pairs per block (fewer for small problems, so that about
 * two blocks per SM exist) and heavy_after 2. */
int sg_set_tuning(sg_model *m, int32_t nodes_per_block, int32_t heavy_after);

/* Autotuner: for each of nodes_per_block in {4, 8, 16, 32, 64, 128} x
 * heavy_after in {0, 1, 2, 4, 8}, and, where the sparse-activity schedule
 * applies, nodes_per_block = the pairs spread over 1, 2 or 4 blocks per SM,
 * 1,024, and one or two whole replicates (when above 128; replicates per
 * block such that at least half a block per SM exists) x heavy_after in
 * {2, 8, 16, 32, 128}, runs the given
 * workload (arguments as sg_run) once untimed (capturing its graph when
 * graphs are on) and twice timed, keeps the setting with the fastest timed
 * run in the model and reports it and its time (outputs may be NULL).  U and
 * V hold the last run's (identical) results.  A shorter tspan tunes a long
 * workload on a prefix. */
int sg_autotune(sg_model *m, const int32_t *tspan, int32_t n_tspan, uint64_t seed,
                int32_t n_rep, const int32_t *d_u0, const double *d_v0, int32_t *d_U,
                double *d_V, void *stream, int32_t *nodes_per_block,
                int32_t *heavy_after, double *ms);

/* CUDA graphs (on by default): sg_run captures its whole launch sequence
 * (counter resets, initial copy, every day and event kernel) into one CUDA
 * graph the first time, and replays it while the buffers, tspan window,
 * seed, replicate count, work split and events stay the same.  Runs on the
 * legacy default stream (stream NULL) or with kernel timing on are launched
 * directly.  enable = 0 turns capture off. */
int sg_set_graphs(sg_model *m, int enable);

/* Output selection of later sg_run calls.
 *
 * Sec. 3.2 (the model's result slots U, V, U_sparse, V_sparse): besides the
 * dense trajectories, the solver can write the state only where a sparse
 * pattern with the layout of U (rows node * n_comp + compartment) or of V
 * (rows node * n_v + index), one column per tspan point, has entries; this
 * saves memory when only a few points of many nodes and days matter.  The
 * prevalence summary (Sec. 4.2, prevalence with a formula cases ~ at risk)
 * is accumulated on the device at every tspan point.
 *
 *   dense        1: sg_run writes d_U and d_V as before; 0: they are not
 *                written and may be NULL (sg_run_host: U and V may be NULL).
 *   n_tspan      columns of the patterns and points of the prevalence
 *                counters; every later sg_run must use this many tspan
 *                points (SG_ERR_ARG otherwise) while a pattern or the
 *                prevalence is set.
 *   u_nnz, u_colptr, u_row   U_sparse pattern in compressed-column form:
 *                the entries of column m are u_colptr[m] .. u_colptr[m+1]-1
 *                (u_colptr[0] = 0, u_colptr[n_tspan] = u_nnz), u_row their
 *                rows, strictly increasing within a column.  Host memory,
 *                copied by this call.  u_nnz = 0: no U_sparse.
 *   d_u_val      device, int32 [n_rep][u_nnz]: U at the pattern's entries.
 *   v_nnz, v_colptr, v_row, d_v_val   the same for V_sparse (double).
 *   prev_cases, prev_at_risk   bit p set: compartment p is a case / at risk
 *                (both 0: no prevalence, else both nonzero).
 *   d_prev       device, int64 [n_rep][n_tspan][4]: per replicate and point
 *                the sum over nodes of the cases, the sum of those at risk,
 *                the number of nodes with a case and the number of nodes
 *                with anyone at risk.  "pop" prevalence = [0] / [1], "nop"
 *                (proportion of nodes with a case) = [2] / [3].
 * The d_ buffers are caller-owned and must stay valid for every later run.
 * o = NULL restores the default (dense only).  Returns SG_ERR_ARG for an
 * invalid pattern or mask (the selection is then reset to the default). */
typedef struct {
  int32_t dense;
  int32_t n_tspan;
  int64_t u_nnz;
  const int64_t *u_colptr;
  const int32_t *u_row;
  int32_t *d_u_val;
  int64_t v_nnz;
  const int64_t *v_colptr;
  const int32_t *v_row;
  double *d_v_val;
  uint32_t prev_cases, prev_at_risk;
  int64_t *d_prev;
} sg_output;

int sg_set_output(sg_model *m, const sg_output *o);

/* Persistent day loop (default off).  When the day kernel's grid fits on the
 * device at once (cooperative launch), the whole run is one launch: each
 * day's external transfers run inside it, between two grid-wide barriers
 * (block counter and generation word in device memory, polled with a 20 s
 * limit after which the run stops with SG_ERR_TIMEOUT), by the block that
 * holds the replicate's first node.  Otherwise, and for models from
 * transition strings, the run is split into day kernels and E2 kernels.
 * enable = 0 (default) always splits: on the SISe benchmark workload the two
 * grid barriers and the E2 block's unhidden event loads cost more per day
 * (10.0 vs 7.9 ms per 365-day run) than the two launches they replace, which
 * programmatic dependent launch already overlaps.  Results are identical. */
int sg_set_persistent(sg_model *m, int enable);

/* Where the external transfers of a day run.  enable = 0 (default): in a
 * separate kernel, one block per replicate, which stages the day's events
 * and their first random words while the day kernel is still running
 * (programmatic dependent launch).  enable = 1: at the end of the day
 * kernel, by the last block to finish each replicate's nodes (blocks count
 * themselves off with an atomic after a device-wide fence; no block ever
 * waits for another); one launch fewer per day, but the event loads are no
 * longer hidden, and on the SISe benchmark workload this is slower (9.6 vs
 * 8.0 ms per 365-day run).  Results are identical. */
int sg_set_fused_events(sg_model *m, int enable);

/* Select the solver of later sg_run calls (SG_SOLVER_SSM by default).
 * SG_SOLVER_AEM keeps 20 bytes of channel state per (replicate, node,
 * transition) on the device, allocated by sg_run.  It cannot be combined
 * with a learned emulator (sg_run returns SG_ERR_ARG).  Returns SG_ERR_ARG
 * for an unknown solver. */
int sg_set_solver(sg_model *m, int32_t solver);

/* Release the model and all its device memory. */
void sg_model_destroy(sg_model *m);

/* Static description of an error code. */
const char *sg_strerror(int code);

/* sg_run without any allocation, for callers that cannot allocate memory.
 *
 * Some callers cannot call cudaMalloc (or anything that allocates): code that
 * runs inside a host framework which owns the device memory pool and forbids
 * private allocations, and services that must not allocate after start-up so
 * that their memory footprint stays fixed.
 * This entry point needs neither an sg_model nor any allocation: the model
 * tables come from `desc` (host memory, read during the call; desc->ldata is
 * ignored and `d_ldata` gives the local data on the device, n_ldata x
 * n_nodes column-major), the caller passes every input and output buffer,
 * and the working memory (node states, tspan table, error word, counters)
 * lives in one fixed array of SG_NOALLOC_SCRATCH_BYTES bytes inside this
 * library, which every GPU that loads the library keeps until the process
 * exits.  It runs the model without scheduled events (the event schedule
 * needs memory proportional to the event table), with the direct-method
 * solver SG_SOLVER_SSM.
 *
 * Limits and behaviour:
 *   - needed scratch = 1024 + 4 (days + 1) + 4 n_tspan + 4 n_rep n_nodes
 *     n_comp + 8 n_rep n_nodes n_v bytes, each part rounded up to 256 bytes;
 *     a larger problem returns SG_ERR_TOO_LARGE before any device work;
 *   - the first call on a device (per process) looks up the array's device
 *     address with that device current; make that first call before any
 *     stream capture;
 *   - every call on a device uses the same array, which keeps the previous
 *     call's contents (each call clears what must start at zero); calls whose
 *     work overlaps on the GPU (several host threads, or several streams
 *     without ordering) race on it and must be serialised by the caller;
 *   - the call copies `tspan` from host memory to the array, reads the
 *     error word and counters back into host memory and waits for its
 *     stream (cudaStreamSynchronize) before it returns;
 *   - otherwise as sg_run: same results bit for bit, same errors. */
#define SG_NOALLOC_SCRATCH_BYTES (8u << 20)
int sg_run_noalloc(const sg_desc *desc, const double *d_ldata, const int32_t *tspan,
                   int32_t n_tspan, uint64_t seed, int32_t n_rep, const int32_t *d_u0,
                   const double *d_v0, int32_t *d_U, double *d_V, void *stream,
                   sg_stats *stats, sg_error *err);

/* Dense layer on the tensor cores (tcgen05, FP32 accumulators in tensor
 * memory), the building block of the learned one-day emulator (an extension
 * of the method; the paper has no emulator):
 *   C = act(A . Bt^T + bias)
 * A: M x K BF16 row-major (leading dimension lda), Bt: N x K BF16 row-major
 * (ldb), i.e. the weight in "out x in" layout; bias: N floats or NULL;
 * act: 0 identity, 1 GELU (tanh form, hardware tanh).  C32 (FP32, before the activation,
 * ldc32) and / or C16 (BF16, after it, ldc16) are written; either may be
 * NULL but not both.  K, lda and ldb must be multiples of 8 and A / Bt
 * 16-byte aligned (SG_ERR_ARG otherwise).  All pointers are device pointers;
 * the call waits for its stream.  SG_ERR_TIMEOUT if a tensor-core wait gave
 * up (the kernel bounds every wait). */
int sg_gemm_bf16(const void *A, int32_t lda, const void *Bt, int32_t ldb, int32_t M,
                 int32_t N, int32_t K, const float *bias, int32_t act, float *C32,
                 int32_t ldc32, void *C16, int32_t ldc16, void *stream);

/* C = act(A8 . B8^T * a_scale * b_scale[n] + bias) with FP8 E4M3 operands
 * on the tensor cores (tcgen05.mma kind::f8f6f4, FP32 accumulation in tensor
 * memory).  A8: M x K, B8: N x K, bytes, row-major with K contiguous (K % 16
 * == 0, lda and ldb multiples of 16, 16-byte aligned rows); a_scale scales
 * the whole of A, b_scale (N floats) each row of B (dequantisation factors).
 * Outputs (any may be NULL, not all): C32 (FP32, before the activation),
 * C16 (BF16, after it), C8 (E4M3 bytes of the activated value times
 * c8_inv_scale, rounded to nearest even and saturated to +-448).  act: 0
 * identity, 1 GELU (tanh form).  Device pointers; the call waits for its
 * stream.  SG_ERR_TIMEOUT if a tensor-core wait gave up. */
int sg_gemm_fp8(const void *A8, int32_t lda, const void *B8, int32_t ldb, int32_t M, int32_t N,
                int32_t K, float a_scale, const float *b_scale, const float *bias, int32_t act,
                float *C32, int32_t ldc32, void *C16, int32_t ldc16, void *C8, int32_t ldc8,
                float c8_inv_scale, void *stream);

/* The same layer with BF16 operands (as sg_gemm_bf16) whose only output is
 * C8: E4M3 bytes of act(A . Bt^T + bias) times c8_inv_scale, rounded to
 * nearest even and saturated to +-448 (the input layer of an FP8 chain).
 * Device pointers; the call waits for its stream. */
int sg_gemm_bf16_to_fp8(const void *A, int32_t lda, const void *Bt, int32_t ldb, int32_t M,
                        int32_t N, int32_t K, const float *bias, int32_t act, void *C8,
                        int32_t ldc8, float c8_inv_scale, void *stream);

/* FP8 quantisation helpers (device pointers, each waits for its stream):
 *   sg_quant_fp8_rows: per row r of W (rows x cols, FP32): scale[r] = max |w|
 *     / 448 (1 for a zero row), W8 = e4m3(w / scale[r]) (nearest even,
 *     saturated);
 *   sg_quant_fp8_bf16: out8[i] = e4m3(x[i] * inv_scale) for BF16 x;
 *   sg_absmax_bf16:    *out = max_i |x[i]| for BF16 x. */
int sg_quant_fp8_rows(const float *W, int32_t rows, int32_t cols, void *W8, float *scale,
                      void *stream);
int sg_quant_fp8_bf16(const void *x, int64_t n, float inv_scale, void *out8, void *stream);
int sg_absmax_bf16(const void *x, int64_t n, float *out, void *stream);

/* ---- Learned one-day emulator (an extension of the method: the paper has
 * no emulator).  For SISe3 nodes inside a validity range, a small MLP
 * predicts the distribution of each age class's one-day increment of I
 * (S moves opposite, so every age class keeps its size, as under the SSA),
 * and a sample from it replaces the node's SSA for that day; other nodes run
 * the SSA.  Network: 16 features -> 256 -> 256 -> 256 (GELU) -> 392 logits
 * (three heads of 129 bins for increments -64..64, 5 padding columns), BF16
 * weights and activations, FP32 accumulation on the tensor cores.
 * Features of a node: log1p of S1, I1, S2, I2, S3, I3; phi; 50 upsilon_1..3;
 * 10 gamma_1..3; three zeros.
 * All pointers below are device pointers; every call waits for its stream. */

/* Cross-entropy of the three 129-way heads of `B` rows of logits (FP32,
 * leading dimension ldl >= 387) against target bins (int32, B x 3, 0..128):
 * adds the summed loss to *loss_sum (device double) and writes
 * d loss / d logits / B as BF16 (leading dimension ldd; columns 387.. are 0). */
int sg_mlp_ce_loss(const float *logits, int32_t ldl, const int32_t *targets, int32_t B,
                   void *dlogits, int32_t ldd, double *loss_sum, void *stream);
/* dpre[i] = dpost[i] * GELU'(pre[i]) (tanh form; BF16 out), n elements. */
int sg_gelu_backward(const float *dpost, const float *pre, int64_t n, void *dpre, void *stream);
/* dst (cols x rows) = src (rows x cols) transposed, BF16. */
int sg_transpose_bf16(const void *src, int32_t rows, int32_t cols, void *dst, void *stream);
/* out[c] = sum over rows of src[r][c] (BF16 in, FP32 out). */
int sg_colsum_bf16(const void *src, int32_t rows, int32_t cols, float *out, void *stream);
/* One Adam step (Kingma and Ba) on n FP32 parameters with bias correction
 * for `step` (>= 1); params_bf16 (may be NULL) receives the BF16 copy. */
int sg_adam_step(float *params, const float *grads, float *m, float *v, int64_t n, float lr,
                 float beta1, float beta2, float eps, int32_t step, void *params_bf16,
                 void *stream);
/* Emulator features (units x 16 BF16) of SISe3 states u (units x 6 int32)
 * and phi (units doubles) with the model's gdata (11 host doubles); flag[i]
 * = 1 when herd <= max_herd, phi_lo <= phi <= phi_hi and the node's total
 * transition rate sum_a (upsilon_a phi S_a + gamma_a I_a) >= min_rate
 * (expected transitions per day), else 0. */
int sg_emu_features(const int32_t *u, const double *v, int64_t units, const double *gdata,
                    int32_t max_herd, double phi_lo, double phi_hi, double min_rate,
                    void *feat, int32_t *flag, void *stream);
/* Training targets: bins clamp(I_a(after) - I_a(before) + 64, 0, 128). */
int sg_emu_targets(const int32_t *u_before, const int32_t *u_after, int64_t units,
                   int32_t *targets, void *stream);
/* Sample increments for the flagged units from the logits: delta[i] =
 * (dI_1, dI_2, dI_3, used), each clamped to -I_a .. S_a; a head's softmax
 * weights are 2^(z - max z), z = logit log2 e (hardware 2^x), summed in
 * groups of 5 bins and scanned over the groups; the uniforms come
 * from Philox with counter (0, node, day, (2 << 24) | replicate), unit i =
 * replicate * n_nodes + node. */
int sg_emu_sample(const float *logits, int32_t ldl, const int32_t *u, const int32_t *flag,
                  int64_t units, int32_t n_nodes, uint64_t seed, int32_t day, int32_t *delta,
                  void *stream);
/* Use the emulator in sg_run (enable != 0; SISe3 models only): W[l] are the
 * BF16 weights in "out x in" layout (256 x 16, 256 x 256, 256 x 256,
 * 392 x 256) and b[l] the FP32 biases; both stay owned by the caller and
 * must outlive the runs.  Nodes with herd > max_herd (-1: every node) or phi outside
 * [phi_lo, phi_hi] fall back to the SSA.  enable = 0 turns it off. */
int sg_emulator_set(sg_model *m, const void *const *W, const float *const *b, int32_t max_herd,
                    double phi_lo, double phi_hi, int enable);

/* The emulator's activity threshold: a node whose total transition rate at
 * the start of a day (sum_a upsilon_a phi S_a + gamma_a I_a, expected
 * transitions per day) is below min_rate stays on the SSA that day (default
 * 0: only the herd size and phi decide).  Quiet nodes are cheap for the SSA,
 * and the emulator's rare-event probabilities are where its error
 * accumulates over long runs.  SG_ERR_ARG for a negative or NaN min_rate. */
int sg_emulator_set_min_rate(sg_model *m, double min_rate);

/* FP8 inference for the emulator set with sg_emulator_set: layers 2-4 run on
 * E4M3 operands (sg_gemm_fp8): W8[l] (E4M3 bytes, out x in, as W of layer l
 * + 1) with per-row scales w_scale[l], and the input activations of layers
 * 2-4 quantised with the static scales act_scale[0..2] (each = calibrated max
 * |activation| / 448); layer 1 stays BF16 and writes E4M3 directly.  Device
 * pointers (act_scale: 3 host floats), caller-owned, must outlive the runs.
 * enable = 0 returns to BF16.  SG_ERR_ARG without an emulator. */
int sg_emulator_set_fp8(sg_model *m, const void *const *W8, const float *const *w_scale,
                        const float *act_scale, int enable);

/* Device-side primitives, exported for parity checks of the random stream
 * and arithmetic (each fills a caller-owned device buffer on `stream` and
 * waits for it):
 *   sg_philox_batch: out[4 i .. 4 i + 3] = Philox4x32-10(ctr[4 i ..], key)
 *                    for i < n  (Salmon et al., SC'11)
 *   sg_log_batch:    y[i] = the library's natural logarithm of x[i]
 *   sg_u01_batch:    y[i] = open-interval uniform of words w[2 i], w[2 i+1]
 * All pointers are device pointers. */
int sg_philox_batch(const uint32_t *d_ctr, uint64_t key, uint32_t *d_out,
                    int64_t n, void *stream);
int sg_log_batch(const double *d_x, double *d_y, int64_t n, void *stream);
int sg_u01_batch(const uint32_t *d_w, double *d_y, int64_t n, void *stream);

/* FP64 throughput probe for roofline statements: runs independent chains of
 * fused multiply-adds on every SM for about `iters` steps and returns the
 * achieved rate in *tflops (2 flops per fused multiply-add). */
int sg_fp64_fma_probe(int32_t iters, double *tflops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SIMINF_GPU_H */
