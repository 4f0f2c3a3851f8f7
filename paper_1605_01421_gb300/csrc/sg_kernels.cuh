// sg_kernels.cuh -- the day kernel, the external-transfer kernel and the
// recording helpers of the SimInf GB300 engine, templated on the model kind.
//
// Compiled twice: by nvcc into the library for the built-in kinds, and by
// NVRTC at run time for a model given as transition strings (the generated
// ModelTraits<SG_GENERIC> is defined before this header is included).  So it
// holds device code only and includes nothing but the engine's own headers.
#pragma once

#include "sg_common.h"
#include "sg_device.cuh"

namespace sg {

constexpr int kDayBlock = 128;
constexpr int kE2Block = 256;

// Programmatic dependent launch: the day kernels and the E2 kernels are
// launched so that the next kernel in the stream may start while the
// previous one finishes.  Each kernel lets its successor launch at once,
// reads only static inputs (model tables, event plan) before pdl_wait, and
// waits for its predecessor (completion and memory) before it touches state.
// Every such kernel executes pdl_wait on all paths, so its completion implies
// its predecessor's.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Events of the plan, structure of arrays in planned order (E1 part first).
struct EvDev {
  const int8_t *type;
  const uint8_t *select;
  const int8_t *shift;       // -1 = no shift
  const int32_t *node, *dest, *n;
  const double *proportion;
  const int64_t *index;      // position in the caller's list (random stream key)
  const int32_t *e1_day;     // day index of each E1 event
  const int64_t *e1_node_off;  // [slots * Nn + 1]; nullptr when there are none
};

// Output selection (Sec. 3.2 result slots U_sparse and V_sparse, and the
// prevalence summary): compressed-column patterns with the layouts of U
// (rows node * C + compartment) and V (rows node * NV + index), one column
// per tspan point; values [R][nnz]; prevalence counters [R][M][4] (sum of
// cases, sum at risk, nodes with a case, nodes with anyone at risk).
struct OutDev {
  const int64_t *u_colptr = nullptr;
  const int32_t *u_row = nullptr;
  int32_t *u_val = nullptr;
  long long u_nnz = 0;
  const int64_t *v_colptr = nullptr;
  const int32_t *v_row = nullptr;
  double *v_val = nullptr;
  long long v_nnz = 0;
  uint32_t cases = 0, at_risk = 0;
  unsigned long long *prev = nullptr;
};

// First index in row[lo, hi) whose value is >= x.
__device__ __forceinline__ long long lower_bound_i32(const int32_t *row, long long lo,
                                                     long long hi, int32_t x) {
  while (lo < hi) {
    const long long mid = lo + ((hi - lo) >> 1);
    if (row[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The U_sparse / V_sparse entries of one node at tspan slot m.
template <int C, int NV>
__device__ __forceinline__ void record_sparse(const OutDev &o, int m, int rep, int node,
                                              const int *u, const double *v) {
  if (o.u_nnz > 0) {
    const long long hi = o.u_colptr[m + 1];
    long long e = lower_bound_i32(o.u_row, o.u_colptr[m], hi, node * C);
    for (; e < hi && o.u_row[e] < node * C + C; ++e) {
      const int p = o.u_row[e] - node * C;
      int x = 0;
#pragma unroll
      for (int q = 0; q < C; ++q)
        if (q == p) x = u[q];
      o.u_val[(long long)rep * o.u_nnz + e] = x;
    }
  }
  if (NV > 0 && o.v_nnz > 0) {
    const long long hi = o.v_colptr[m + 1];
    long long e = lower_bound_i32(o.v_row, o.v_colptr[m], hi, node * NV);
    for (; e < hi && o.v_row[e] < node * NV + NV; ++e) {
      const int p = o.v_row[e] - node * NV;
      double x = 0.0;
#pragma unroll
      for (int q = 0; q < NV; ++q)
        if (q == p) x = v[q];
      o.v_val[(long long)rep * o.v_nnz + e] = x;
    }
  }
}

// Adds recorded nodes to the prevalence counters of (replicate, slot m).
// Called by all 32 lanes of the warp together; `key` = rep * M + m for a
// thread that holds a unit (-1 otherwise; such lanes sit at the end of the
// warp, so equal keys are contiguous), `on` = its state is recorded.  A
// segmented inclusive scan over the warp, then one atomic per segment.
template <int C>
__device__ __forceinline__ void prevalence_add(const OutDev &o, long long key, bool on,
                                               const int *u) {
  long long cs = 0, rk = 0;
  int nc = 0, nr = 0;
  if (on) {
#pragma unroll
    for (int p = 0; p < C; ++p) {
      if ((o.cases >> p) & 1u) cs += u[p];
      if ((o.at_risk >> p) & 1u) rk += u[p];
    }
    nc = cs > 0;
    nr = rk > 0;
  }
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long k2 = __shfl_up_sync(full, key, d);
    const long long c2 = __shfl_up_sync(full, cs, d), r2 = __shfl_up_sync(full, rk, d);
    const int nc2 = __shfl_up_sync(full, nc, d), nr2 = __shfl_up_sync(full, nr, d);
    if (lane >= d && k2 == key) {
      cs += c2;
      rk += r2;
      nc += nc2;
      nr += nr2;
    }
  }
  const long long next = __shfl_down_sync(full, key, 1);
  if (key >= 0 && (lane == 31 || next != key)) {
    unsigned long long *q = o.prev + key * 4;
    if (cs) atomicAdd(q, (unsigned long long)cs);
    if (rk) atomicAdd(q + 1, (unsigned long long)rk);
    if (nc) atomicAdd(q + 2, (unsigned long long)nc);
    if (nr) atomicAdd(q + 3, (unsigned long long)nr);
  }
}

struct DayArgs {
  int *u;              // [R][Nn][C] working counts
  double *v;           // [R][Nn][NV] working continuous state
  const double *ldata; // [Nn][n_ldata]
  int32_t *U;          // [R][M][Nn][C]
  double *V;           // [R][M][Nn][NV]
  const int32_t *rec;  // [days + 1]: tspan slot of T = t0 + i, or -1
  int32_t *e1_cur;     // [R][Nn]: next E1 event, relative to the node's list
  int32_t *e1_next;    // [R][Nn]: day index of that event (sparse schedule)
  EvDev ev;
  int32_t t0, M, n_rep, slots;
  // global index of the run's replicate 0 (a shard of a larger job): every
  // random stream and error report uses rep0 + the local replicate, state
  // and outputs the local one
  int32_t rep0;
  // 1: the model's parameters are finite, so a unit without infected
  // animals and with phi == +0 has an empty day (k_days_sparse skips it)
  int32_t quiet;
  int32_t T_begin, T_end;  // SSA toward T = T_begin .. T_end - 1
  int32_t finish_first;    // finish unit step T_begin - 1 before the SSA
  int32_t finish_last;     // finish unit step T_end - 1 after the SSA
  int32_t heavy_after;     // draws a thread takes before its warp takes over
  int32_t npb;             // nodes per block (<= kDayBlock); the other
                           // threads of the block only serve heavy nodes
  const int32_t *emu;      // [R][Nn][4]: emulated increments of I_1..I_3 and
                           // a flag (1 = use them instead of the SSA), or null
  // the emulator's node split across two launches of a day: 0 every node;
  // 1 only the nodes outside the emulator's range (emu_flag[gid] == 0, the
  // SSA part, run beside the emulator); 2 only the emulated nodes (emu[gid]
  // flag set)
  const int32_t *emu_flag;
  int32_t emu_part;
  uint32_t k0, k1;         // Philox key (seed)
  SgDevError *err;
  SgCounters *cnt;
  // all events method: channel state [T][R * Nn] (rate, firing time, draws
  // taken); null for the direct method
  double *aem_a, *aem_tau;
  uint32_t *aem_cnt;
  OutDev out;            // sparse output and prevalence (U, V may be null)
  // external transfers of unit time T_end - 1 run inside this launch, by the
  // last block to finish each replicate's nodes (null: none or by the E2
  // kernel): wave bounds (wave_ev), the day's wave range [e2_wb, e2_we) when
  // the events are shared, else per replicate from wave_off[day][slot], and
  // a per-replicate count of finished blocks (zero between launches)
  const int64_t *wave_ev, *wave_off;
  long long e2_wb, e2_we;
  int32_t e2_day_index;
  int32_t *e2_done;
  // persistent run (cooperative launch, every block resident): the days'
  // external transfers run inside this launch between two grid barriers
  // (arrival count, generation); null: not persistent
  unsigned int *grid_bar;
  int32_t n_blocks;
  // sparse schedule with every block holding whole replicates (nodes per
  // block a multiple of the node count): each block runs its replicates'
  // external transfers of every day itself, between the day's E1 events and
  // its post time step, so one launch covers all days; 0: off
  int32_t e2_inblock;
};

// %globaltimer (ns).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Adds one recorded unit to the prevalence counters of `key` with its own
// atomics (for units taken from a list, whose lanes are in no order).
template <int C>
__device__ __forceinline__ void prevalence_add_unit(const OutDev &o, long long key,
                                                    const int *u) {
  long long cs = 0, rk = 0;
#pragma unroll
  for (int p = 0; p < C; ++p) {
    if ((o.cases >> p) & 1u) cs += u[p];
    if ((o.at_risk >> p) & 1u) rk += u[p];
  }
  unsigned long long *q = o.prev + key * 4;
  if (cs) atomicAdd(q, (unsigned long long)cs);
  if (rk) atomicAdd(q + 1, (unsigned long long)rk);
  if (cs > 0) atomicAdd(q + 2, 1ull);
  if (rk > 0) atomicAdd(q + 3, 1ull);
}

// A grid barrier must wait for the slowest block's whole day; a wait longer
// than this is taken as a failure (SG_ERR_TIMEOUT) instead of a hang.
constexpr unsigned long long kGridWaitNs = 20ull * 1000 * 1000 * 1000;

// Grid-wide barrier for a cooperative launch (all blocks resident): thread 0
// of each block reads the generation, fences, arrives; the last arrival
// resets the count and advances the generation; the others poll the
// generation with a time limit.  Returns false (the same in every thread of
// the block) if this block gave up; the kernel must then leave.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, int n_blocks, SgDevError *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == (unsigned int)n_blocks - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (global_ns() - t0 > kGridWaitNs) {
          ok = 0;
          report(err, SG_ERR_TIMEOUT, -1, -1, -1, -1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The external transfers (Sec. 3.3) of replicate `rep` at unit time T, wave by
// wave, by one block (a block barrier between waves), on the replicate's
// state in global memory.  The state was written by other blocks of the same
// launch, so it is read and written at L2 only (ld / st .cg) and added to
// with atomics; a wave never samples a node another event of the wave
// touches.  Same arithmetic and random stream as the E2 kernel.
template <int C>
__device__ void e2_rep_block(const SgTables &tb, const DayArgs &a, int rep, int T,
                             long long w0, long long w1) {
  // a run that already failed does nothing (one thread reads, the barrier
  // makes the answer the block's)
  if (__syncthreads_or(threadIdx.x == 0 && *(volatile int32_t *)&a.err->code != 0)) return;
  int *state = a.u + (long long)rep * tb.n_nodes * C;
  const uint64_t seed = ((uint64_t)a.k1 << 32) | a.k0;
  constexpr int kHv = 256;  // large transfers of a wave left to the warps
  __shared__ long long s_hv[kHv];
  __shared__ int s_nhv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned long long applied = 0;
  bool bad = false;
  if (threadIdx.x == 0) s_nhv = 0;
  __syncthreads();
  for (long long w = w0; w < w1; ++w) {
    const long long lo = a.wave_ev[w], hi = a.wave_ev[w + 1];
    for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
      const int src = a.ev.node[j];
      int *un = state + (long long)src * C;
      const uint32_t mask = tb.Emask[a.ev.select[j]];
      const long long idx = a.ev.index[j];
      int cur[C];
      long long total = 0;
#pragma unroll
      for (int p = 0; p < C; ++p) {
        cur[p] = __ldcg(un + p);
        if ((mask >> p) & 1u) total += cur[p];
      }
      const int n = a.ev.n[j];
      const long long k =
          n > 0 ? (long long)n : (long long)round(a.ev.proportion[j] * (double)total);
      if (k < 0 || k > total) {
        report(a.err, SG_ERR_EVENT_UNDERFLOW, a.rep0 + rep, src, T, idx);
        bad = true;
        continue;
      }
      if (k >= kUrnWarp) {
        // a large transfer: sampled by a warp after this pass (in this
        // thread when the list is full)
        const int slot = atomicAdd(&s_nhv, 1);
        if (slot < kHv) {
          s_hv[slot] = j;
          continue;
        }
      }
      int moved[C];
#pragma unroll
      for (int p = 0; p < C; ++p) moved[p] = 0;
      if (k > 0) {
        WordStream ws;
        ws.init(seed, idx, a.rep0 + rep);
        for (long long d = 0; d < k; ++d) {
          uint32_t x = ws.below((uint32_t)(total - d));
          bool taken = false;
#pragma unroll
          for (int p = 0; p < C; ++p) {
            if (taken || !((mask >> p) & 1u)) continue;
            const uint32_t rem = (uint32_t)(cur[p] - moved[p]);
            if (x < rem) {
              ++moved[p];
              taken = true;
            } else {
              x -= rem;
            }
          }
        }
      }
      const int q_sh = a.ev.shift[j];
      int *ud = state + (long long)a.ev.dest[j] * C;
#pragma unroll
      for (int p = 0; p < C; ++p)
        if (moved[p] != 0) __stcg(un + p, cur[p] - moved[p]);
#pragma unroll
      for (int p = 0; p < C; ++p)
        if (moved[p] != 0) atomicAdd(ud + (q_sh >= 0 ? p + tb.Nsh[q_sh][p] : p), moved[p]);
      ++applied;
    }
    // one barrier per wave; its result is the same for every thread
    if (__syncthreads_or(bad)) break;
    const int nhv = min(s_nhv, kHv);  // the same in every thread
    if (nhv > 0) {
      __syncthreads();  // every thread has read the count
      if (threadIdx.x == 0) s_nhv = 0;
      // the wave's large transfers, one warp each (no other event of the
      // wave touches their source nodes)
      for (int h = warp; h < nhv; h += nwarps) {
        const long long j = s_hv[h];
        const int src = a.ev.node[j];
        int *un = state + (long long)src * C;
        const uint32_t mask = tb.Emask[a.ev.select[j]];
        int cur[C];
        long long total = 0;
#pragma unroll
        for (int p = 0; p < C; ++p) {
          cur[p] = __ldcg(un + p);
          if ((mask >> p) & 1u) total += cur[p];
        }
        const int n = a.ev.n[j];
        const long long k =
            n > 0 ? (long long)n : (long long)round(a.ev.proportion[j] * (double)total);
        int moved[C];
        urn_warp<C>(cur, mask, (uint32_t)k, (uint32_t)total, seed, a.ev.index[j], a.rep0 + rep,
                    moved);
        if (lane == 0) {
          const int q_sh = a.ev.shift[j];
          int *ud = state + (long long)a.ev.dest[j] * C;
#pragma unroll
          for (int p = 0; p < C; ++p)
            if (moved[p] != 0) __stcg(un + p, cur[p] - moved[p]);
#pragma unroll
          for (int p = 0; p < C; ++p)
            if (moved[p] != 0) atomicAdd(ud + (q_sh >= 0 ? p + tb.Nsh[q_sh][p] : p), moved[p]);
          ++applied;
        }
        __syncwarp();
      }
      __syncthreads();
    }
  }
  if (applied) atomicAdd(&a.cnt->events, applied);
}

// One transition (Appendix A, inversion and update): the smallest n with
// target <= running sum of the positive rates (last positive one if rounding
// leaves none), u += S[, n], and the rates that column n of G marks are
// recomputed.  Returns 0 or SG_ERR_RATE.
// u += S[, n] and the rates that column n of G marks recomputed; 0 or
// SG_ERR_RATE.
template <int KIND>
__device__ __forceinline__ int apply_transition(int *u, double *w, int n, const double *kf,
                                                const SgTables &tb) {
  using M = ModelTraits<KIND>;
#pragma unroll
  for (int p = 0; p < M::C; ++p) u[p] += tb.S[n][p];
  const uint32_t dep = tb.dep[n];
  int code = 0;
#pragma unroll
  for (int k = 0; k < M::T; ++k) {
    if ((dep >> k) & 1u) {
      w[k] = M::rate_k(k, u, kf, tb.gdata);
      if (bad_rate(w[k])) code = SG_ERR_RATE;
    }
  }
  return code;
}

template <int KIND>
__device__ __forceinline__ int fire(int *u, double *w, double target, const double *kf,
                                    const SgTables &tb) {
  using M = ModelTraits<KIND>;
  // running sum over the positive rates in index order; the first term is
  // taken as is (0 + w == w exactly), the comparisons are exact integer
  // comparisons of non-negative doubles
  double cum = 0.0;
  int n = -1, last = -1;
#pragma unroll
  for (int j = 0; j < M::T; ++j) {
    if (n < 0 && gt0(w[j])) {
      cum = last < 0 ? w[j] : cum + w[j];
      last = j;
      if (le_nonneg(target, cum)) n = j;
    }
  }
  if (n < 0) n = last;
  return apply_transition<KIND>(u, w, n, kf, tb);
}

// Prefix sums P_j = (..(w_0 + w_1) + ..) + w_j of the rates in index order,
// recomputed from index j0 on (the rates below j0 unchanged).  P_(T-1) is
// lambda as the direct method sums it, and at every positive rate P_j is
// the running sum of the positive rates that fire() forms (adding a zero
// rate leaves a sum unchanged, and a sum of zeros plus w is w).
template <int T>
__device__ __forceinline__ void rate_prefix(const double *w, double *P, int j0) {
#pragma unroll
  for (int j = 0; j < T; ++j)
    if (j >= j0) P[j] = j == 0 ? w[0] : P[j - 1] + w[j];
}

// fire()'s choice of transition from the prefix sums.
template <int T>
__device__ __forceinline__ int select_prefix(const double *w, const double *P, double target) {
  int n = -1, last = -1;
#pragma unroll
  for (int j = 0; j < T; ++j) {
    if (gt0(w[j])) {
      if (n < 0) last = j;
      if (n < 0 && le_nonneg(target, P[j])) n = j;
    }
  }
  return n < 0 ? last : n;
}

enum { SSA_DONE = 0, SSA_HEAVY = 1 };

// Direct SSA of one node toward the unit time Tn in its own thread, for at
// most `budget` draws (Appendix A, one iteration per draw).  Returns SSA_DONE,
// SSA_HEAVY (budget spent, state and counter ready for the warp) or an error.
template <int KIND>
__device__ __forceinline__ int ssa_thread(int *u, double *w, const double *kf, double &t,
                                          uint32_t &c, double Tn, uint32_t node, uint32_t Td,
                                          uint32_t tag, uint32_t k0, uint32_t k1, int budget,
                                          const SgTables &tb, unsigned long long &fired) {
  using M = ModelTraits<KIND>;
  const long long Tkey = order_key(Tn);
  for (int b = 0;; ++b) {
    // lambda = ((0 + w_1) + w_2) + ...; the leading 0 + w_1 changes no
    // decision or value, so the sum starts at w_1
    double lam = w[0];
#pragma unroll
    for (int j = 1; j < M::T; ++j) lam = lam + w[j];
    if (!gt0(lam)) return SSA_DONE;  // nothing can fire: jump to Tn
    if (c >= SG_MAX_DRAWS) return SG_ERR_STEP_LIMIT;
    if (b == budget) return SSA_HEAVY;
    const U4 x = philox10(U4{c, node, Td, tag}, k0, k1);
    ++c;
    const double r1 = u01_open(x.x, x.y);
    const double r2 = u01_open(x.z, x.w);
    const double tau = -log_pos(r1) / lam;
    const double tt = t + tau;
    if (order_key(tt) >= Tkey) return SSA_DONE;
    t = tt;
    const int rc = fire<KIND>(u, w, lam * r2, kf, tb);
    ++fired;
    if (rc) return rc;
  }
}

// One iteration of ssa_thread's loop (one draw of the direct method,
// Appendix A): returns SSA_STEP_FIRED (a transition fired, t and u moved on),
// SSA_DONE (lambda = 0 or the next event falls at or after Tn),
// SSA_HEAVY (hand_off set and a draw is due: state unchanged, for a warp) or
// an error.  The same operations in the same order as ssa_thread.
enum { SSA_STEP_FIRED = 2 };
template <int KIND>
__device__ __forceinline__ int ssa_step(int *u, double *w, const double *kf, double &t,
                                        uint32_t &c, long long Tkey, uint32_t node, uint32_t Td,
                                        uint32_t tag, uint32_t k0, uint32_t k1, bool hand_off,
                                        const SgTables &tb, unsigned long long &fired) {
  using M = ModelTraits<KIND>;
  double lam = w[0];
#pragma unroll
  for (int j = 1; j < M::T; ++j) lam = lam + w[j];
  if (!gt0(lam)) return SSA_DONE;
  if (c >= SG_MAX_DRAWS) return SG_ERR_STEP_LIMIT;
  if (hand_off) return SSA_HEAVY;
  const U4 x = philox10(U4{c, node, Td, tag}, k0, k1);
  ++c;
  const double r1 = u01_open(x.x, x.y);
  const double r2 = u01_open(x.z, x.w);
  const double tau = -log_pos(r1) / lam;
  const double tt = t + tau;
  if (order_key(tt) >= Tkey) return SSA_DONE;
  t = tt;
  const int rc = fire<KIND>(u, w, lam * r2, kf, tb);
  ++fired;
  return rc ? rc : SSA_STEP_FIRED;
}

// A node handed from its thread to a warp.
template <int C, int NK>
struct HeavySlot {
  double t;
  double kf[NK];
  uint32_t c;
  int32_t node, rep, code;
  int32_t u[C];
};

// SISe3 heavy node-days, three draws per parallel round (see the comment
// inside); returns false, doing nothing, for other kinds or another
// dependency graph (the caller then takes the sequential loop).
template <int KIND>
__device__ __forceinline__ bool ssa_window3(int *u, double *w, const double *kf, double &t,
                                            uint32_t &c, uint32_t &c0, double &nE, double &r2,
                                            bool &have, unsigned long long &f, int &code,
                                            uint32_t node, uint32_t Td, uint32_t tag, uint32_t k0,
                                            uint32_t k1, long long Tkey, const SgTables &tb) {
  if constexpr (KIND != SG_SISE3) {
    return false;
  } else {
    using M = ModelTraits<KIND>;
    constexpr int C = M::C, T = M::T;
    if (!(tb.dep[0] == 3u && tb.dep[1] == 3u && tb.dep[2] == 12u && tb.dep[3] == 12u &&
          tb.dep[4] == 48u && tb.dep[5] == 48u))
      return false;
    const int lane = threadIdx.x & 31;
    // SISe3 with its block-diagonal dependency graph (each transition changes
    // and is changed by its own age class only), so the rates of a state are
    // the same however it was reached.  The states reachable within the next
    // J = 3 draws are u plus at most two columns of S: the root (lane 0), one
    // transition n (lanes 1 + n) and two transitions a <= b (lanes 7 +
    // pair(a, b)), 28 in all.  Every lane evaluates its state's draw (draw
    // c + depth): rates, lambda in index order, waiting-time divide and
    // inversion; the walk then follows the fired transitions through the
    // table.  Same operations and order as the sequential loop.
    constexpr int J = 3;
    constexpr int kT = ModelTraits<SG_SISE3>::T;  // 6
    auto pair = [](int a, int b) { return a * kT - a * (a - 1) / 2 + (b - a); };
    int depth = 0, ma = -1, mb = -1;  // this lane's state: root, {ma}, {ma, mb}
    if (lane >= 1 && lane <= kT) {
      depth = 1;
      ma = lane - 1;
    } else if (lane > kT && lane < 1 + kT + kT * (kT + 1) / 2) {
      depth = 2;
      int l = lane - 1 - kT, a = 0;
      while (l >= kT - a) {
        l -= kT - a;
        ++a;
      }
      ma = a;
      mb = a + l;
    }
    bool done = false;
    while (!done && code == 0) {
      if (!have || c + (uint32_t)J - c0 > 32u) {
        c0 = c;
        const U4 x = philox10(U4{c0 + (uint32_t)lane, node, Td, tag}, k0, k1);
        nE = -log_pos(u01_open(x.x, x.y));
        r2 = u01_open(x.z, x.w);
        have = true;
      }
      int us[C];
#pragma unroll
      for (int p = 0; p < C; ++p) {
        int x = u[p];
        if (ma >= 0) x += tb.S[ma][p];
        if (mb >= 0) x += tb.S[mb][p];
        us[p] = x;
      }
      double ws[T];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        ws[j] = M::rate_k(j, us, kf, tb.gdata);
        bad = bad || bad_rate(ws[j]);
      }
      const int src = (int)(c - c0) + depth;  // lane holding draw c + depth
      const double E = __shfl_sync(0xffffffffu, nE, src);
      const double R2 = __shfl_sync(0xffffffffu, r2, src);
      double lam = ws[0];
#pragma unroll
      for (int j = 1; j < T; ++j) lam = lam + ws[j];
      const double tau = E / lam;
      const double target = lam * R2;
      // inversion exactly as fire(): running sum over the positive rates
      double cum = 0.0;
      int nsel = -1, last = -1;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        if (nsel < 0 && gt0(ws[j])) {
          cum = last < 0 ? ws[j] : cum + ws[j];
          last = j;
          if (le_nonneg(target, cum)) nsel = j;
        }
      }
      if (nsel < 0) nsel = last;
      const unsigned pos_mask = __ballot_sync(0xffffffffu, gt0(lam));
      const unsigned bad_mask = __ballot_sync(0xffffffffu, bad);
      int L = 0, n1 = -1, j = 0;
      for (; j < J; ++j) {
        if (j > 0 && ((bad_mask >> L) & 1u)) {
          code = SG_ERR_RATE;  // the transition into this state gave a bad rate
          break;
        }
        if (!((pos_mask >> L) & 1u)) {
          done = true;  // nothing can fire: jump to Tn
          break;
        }
        if (c >= SG_MAX_DRAWS) {
          code = SG_ERR_STEP_LIMIT;
          break;
        }
        const double tauL = __shfl_sync(0xffffffffu, tau, L);
        const int n = __shfl_sync(0xffffffffu, nsel, L);
        ++c;
        const double tt = t + tauL;
        if (order_key(tt) >= Tkey) {
          done = true;
          break;
        }
        t = tt;
#pragma unroll
        for (int p = 0; p < C; ++p) u[p] += tb.S[n][p];
        ++f;
        if (j == 0) {
          n1 = n;
          L = 1 + n;
        } else if (j == 1) {
          L = 1 + kT + (n1 <= n ? pair(n1, n) : pair(n, n1));
        }
      }
      if (!done && code == 0) {
        // j == J: a new window starts from the state after J transitions
#pragma unroll
        for (int k = 0; k < T; ++k) {
          w[k] = M::rate_k(k, u, kf, tb.gdata);
          if (bad_rate(w[k])) code = SG_ERR_RATE;
        }
      }
    }
    return true;
  }
}

// Speculative window for heavy node-days of models from transition strings,
// whose dependency graph is complete (the parser derives it from what each
// propensity reads, so recomputing the rates G marks after a transition gives
// the same rates as recomputing every rate from the counts).  The states reachable
// within the next J draws are u plus a multiset of at most J - 1 columns of
// S; lane l holds one such multiset (sorted transition indices a_1 <= ... ),
// with J the largest for which they fit in a warp (T = 3: 4; T = 4..6: 3;
// T = 7..31: 2).  Every lane evaluates its state's draw (draw c + depth):
// rates from the counts, lambda in index order, waiting-time divide and
// inversion; the walk then follows the fired transitions, finding the lane
// of the state reached with a ballot, so J draws cost one parallel round
// instead of J dependent rate updates and divides.  Same operations and
// order as the sequential loop.  (SISe3 has a dedicated window with an
// arithmetic walk, ssa_window3.)  Returns false, doing nothing, for other
// kinds (the caller then takes the sequential loop).
template <int KIND>
__device__ __forceinline__ bool ssa_window(int *u, double *w, const double *kf, double &t,
                                           uint32_t &c, uint32_t &c0, double &nE, double &r2,
                                           bool &have, unsigned long long &f, int &code,
                                           uint32_t node, uint32_t Td, uint32_t tag, uint32_t k0,
                                           uint32_t k1, long long Tkey, const SgTables &tb) {
  using M = ModelTraits<KIND>;
  constexpr int C = M::C, T = M::T;
  if constexpr (KIND != SG_GENERIC || T < 3 || T > 31) {
    return false;
  } else {
    constexpr int J = T == 3 ? 4 : (T <= 6 ? 3 : 2);
    constexpr int D = J - 1;  // largest multiset held by a lane
    const int lane = threadIdx.x & 31;
    // this lane's multiset: enumerate by depth, then lexicographically
    int depth = 0, a[D > 0 ? D : 1];
#pragma unroll
    for (int i = 0; i < D; ++i) a[i] = -1;
    {
      int l = lane, d = 0, cur[D > 0 ? D : 1];
      bool found = false;
      // depth 0: lane 0
      if (l == 0) {
        found = true;
      } else {
        l -= 1;
        for (d = 1; d <= D && !found; ++d) {
          // multisets of size d in lexicographic order
#pragma unroll
          for (int i = 0; i < D; ++i) cur[i] = 0;
          for (;;) {
            if (l == 0) {
              found = true;
              depth = d;
#pragma unroll
              for (int i = 0; i < D; ++i) a[i] = i < d ? cur[i] : -1;
              break;
            }
            --l;
            // next non-decreasing tuple of length d over 0..T-1
            int i = d - 1;
            while (i >= 0 && cur[i] == T - 1) --i;
            if (i < 0) break;
            const int v = cur[i] + 1;
            for (int k = i; k < d; ++k) cur[k] = v;
          }
        }
      }
      if (!found) depth = -1;  // a spare lane: evaluates nothing used
    }
    const int ev_depth = depth < 0 ? 0 : depth;
    bool done = false;
    while (!done && code == 0) {
      if (!have || c + (uint32_t)J - c0 > 32u) {
        c0 = c;
        const U4 x = philox10(U4{c0 + (uint32_t)lane, node, Td, tag}, k0, k1);
        nE = -log_pos(u01_open(x.x, x.y));
        r2 = u01_open(x.z, x.w);
        have = true;
      }
      int us[C];
#pragma unroll
      for (int p = 0; p < C; ++p) {
        int x = u[p];
#pragma unroll
        for (int i = 0; i < D; ++i)
          if (a[i] >= 0) x += tb.S[a[i]][p];
        us[p] = x;
      }
      double ws[T];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        ws[j] = M::rate_k(j, us, kf, tb.gdata);
        bad = bad || bad_rate(ws[j]);
      }
      const int src = (int)(c - c0) + ev_depth;  // lane holding draw c + depth
      const double E = __shfl_sync(0xffffffffu, nE, src);
      const double R2 = __shfl_sync(0xffffffffu, r2, src);
      double lam = ws[0];
#pragma unroll
      for (int j = 1; j < T; ++j) lam = lam + ws[j];
      const double tau = E / lam;
      const double target = lam * R2;
      // inversion exactly as fire(): running sum over the positive rates
      double cum = 0.0;
      int nsel = -1, last = -1;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        if (nsel < 0 && gt0(ws[j])) {
          cum = last < 0 ? ws[j] : cum + ws[j];
          last = j;
          if (le_nonneg(target, cum)) nsel = j;
        }
      }
      if (nsel < 0) nsel = last;
      const unsigned pos_mask = __ballot_sync(0xffffffffu, gt0(lam));
      const unsigned bad_mask = __ballot_sync(0xffffffffu, bad);
      int L = 0, j = 0;
      int path[D > 0 ? D : 1];  // sorted transitions fired in this round
#pragma unroll
      for (int i = 0; i < D; ++i) path[i] = -1;
      for (; j < J; ++j) {
        if (j > 0 && ((bad_mask >> L) & 1u)) {
          code = SG_ERR_RATE;  // the transition into this state gave a bad rate
          break;
        }
        if (!((pos_mask >> L) & 1u)) {
          done = true;  // nothing can fire: jump to Tn
          break;
        }
        if (c >= SG_MAX_DRAWS) {
          code = SG_ERR_STEP_LIMIT;
          break;
        }
        const double tauL = __shfl_sync(0xffffffffu, tau, L);
        const int n = __shfl_sync(0xffffffffu, nsel, L);
        ++c;
        const double tt = t + tauL;
        if (order_key(tt) >= Tkey) {
          done = true;
          break;
        }
        t = tt;
#pragma unroll
        for (int p = 0; p < C; ++p) u[p] += tb.S[n][p];
        ++f;
        if (j + 1 < J) {
          // insert n into the sorted path, then find the lane holding it
          int x = n;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            if (i <= j && path[i] >= 0 && path[i] > x) {
              const int y = path[i];
              path[i] = x;
              x = y;
            } else if (i == j) {
              path[i] = x;
            }
          }
          bool match = depth == j + 1;
#pragma unroll
          for (int i = 0; i < D; ++i) match = match && a[i] == path[i];
          L = __ffs(__ballot_sync(0xffffffffu, match)) - 1;
        }
      }
      if (!done && code == 0) {
        // j == J: a new window starts from the state after J transitions
#pragma unroll
        for (int k = 0; k < T; ++k) {
          w[k] = M::rate_k(k, u, kf, tb.gdata);
          if (bad_rate(w[k])) code = SG_ERR_RATE;
        }
      }
    }
    return true;
  }
}

// Direct SSA of one heavy node by a whole warp.  The draws depend only on
// (seed, replicate, node, day, draw index), so lane l computes the Philox
// words, uniforms and logarithm of draw c0 + l for 32 draws at once; the
// sequential part (waiting time, boundary test, transition) then runs on all
// lanes in step, reading draw j from lane j.  The transition for a draw is
// evaluated alongside the waiting-time division and kept only if the draw
// falls before Tn.  Same operations, in the same order, as ssa_thread.
template <int KIND>
__device__ void ssa_warp(HeavySlot<ModelTraits<KIND>::C, ModelTraits<KIND>::NK> &hs, double Tn,
                         uint32_t Td, uint32_t k0, uint32_t k1, const SgTables &tb,
                         unsigned long long &fired, unsigned long long &drawn) {
  using M = ModelTraits<KIND>;
  constexpr int C = M::C, T = M::T, NK = M::NK;
  const int lane = threadIdx.x & 31;
  int u[C];
  double kf[NK], w[T];
#pragma unroll
  for (int p = 0; p < C; ++p) u[p] = hs.u[p];
#pragma unroll
  for (int i = 0; i < NK; ++i) kf[i] = hs.kf[i];
  double t = hs.t;
  uint32_t c = hs.c;
  const uint32_t c_in = c, node = (uint32_t)hs.node;
  const uint32_t tag = (SG_STREAM_SSA << 24) | (uint32_t)hs.rep;
  int code = 0;
#pragma unroll
  for (int j = 0; j < T; ++j) w[j] = M::rate_k(j, u, kf, tb.gdata);
  uint32_t c0 = c;
  double nE = 0.0, r2 = 0.0;
  bool have = false;
  unsigned long long f = 0;
  const long long Tkey = order_key(Tn);
  if (T == 2 && tb.dep[0] == 3u && tb.dep[1] == 3u) {
    // Two transitions, every rate recomputed after every transition: the
    // states reachable within the next J = 7 draws are u + (j - b) S0 + b S1,
    // 0 <= b <= j < 7 (28 of them).  Lane l = j (j + 1) / 2 + b evaluates
    // draw c + j at state (j, b): rates, lambda, waiting time, inversion.
    // The walk then follows the fired transitions through the table, so each
    // draw costs one addition (t + tau) and a branch.  Rates from scratch
    // equal the incrementally kept ones (pure functions of the counts).
    constexpr int J = 7;
    int lj = 0, lb = 0;
    {
      int l = lane < J * (J + 1) / 2 ? lane : 0;
      while (l > lj) { l -= lj + 1; ++lj; }
      lb = l;
    }
    bool done = false;
    while (!done && code == 0) {
      if (!have || c + (uint32_t)J - c0 > 32u) {
        c0 = c;
        const U4 x = philox10(U4{c0 + (uint32_t)lane, node, Td, tag}, k0, k1);
        nE = -log_pos(u01_open(x.x, x.y));
        r2 = u01_open(x.z, x.w);
        have = true;
      }
      // this lane's state and draw
      int us[C];
#pragma unroll
      for (int p = 0; p < C; ++p) us[p] = u[p] + (lj - lb) * tb.S[0][p] + lb * tb.S[1][p];
      double ws[T];
      bool bad = false;
#pragma unroll
      for (int j = 0; j < T; ++j) {
        ws[j] = M::rate_k(j, us, kf, tb.gdata);
        bad = bad || bad_rate(ws[j]);
      }
      const int src = (int)(c - c0) + lj;  // lane holding draw c + lj
      const double E = __shfl_sync(0xffffffffu, nE, src);
      const double R2 = __shfl_sync(0xffffffffu, r2, src);
      const double lam = ws[0] + ws[1];
      const double tau = E / lam;
      const double target = lam * R2;
      const int fire0 = gt0(ws[0]) && le_nonneg(target, ws[0]);
      // inversion: transition 0 if target <= w0 (w0 > 0), else 1 if w1 > 0,
      // else the last positive one (w0)
      const int nsel = fire0 ? 0 : (gt0(ws[1]) ? 1 : 0);
      const unsigned pos_mask = __ballot_sync(0xffffffffu, gt0(lam));
      const unsigned bad_mask = __ballot_sync(0xffffffffu, bad);
      const unsigned n1_mask = __ballot_sync(0xffffffffu, nsel == 1);
      int j = 0, b = 0;
      for (; j < J; ++j) {
        const int L = j * (j + 1) / 2 + b;
        if (j > 0 && ((bad_mask >> L) & 1u)) {
          code = SG_ERR_RATE;  // the transition into this state gave a bad rate
          break;
        }
        if (!((pos_mask >> L) & 1u)) {
          done = true;  // nothing can fire: jump to Tn
          break;
        }
        if (c >= SG_MAX_DRAWS) {
          code = SG_ERR_STEP_LIMIT;
          break;
        }
        const double tauL = __shfl_sync(0xffffffffu, tau, L);
        ++c;
        const double tt = t + tauL;
        if (order_key(tt) >= Tkey) {
          done = true;
          break;
        }
        t = tt;
        b += (int)((n1_mask >> L) & 1u);
        ++f;
      }
      // move to the state reached
#pragma unroll
      for (int p = 0; p < C; ++p) u[p] = u[p] + (j - b) * tb.S[0][p] + b * tb.S[1][p];
      if (!done && code == 0) {
        // j == J: a new window starts from the state after J transitions
#pragma unroll
        for (int k = 0; k < T; ++k) {
          w[k] = M::rate_k(k, u, kf, tb.gdata);
          if (bad_rate(w[k])) code = SG_ERR_RATE;
        }
      }
    }
  } else if (!ssa_window3<KIND>(u, w, kf, t, c, c0, nE, r2, have, f, code, node, Td, tag, k0,
                                 k1, Tkey, tb) &&
             !ssa_window<KIND>(u, w, kf, t, c, c0, nE, r2, have, f, code, node, Td, tag, k0,
                               k1, Tkey, tb)) {
  for (;;) {
    double lam = w[0];
#pragma unroll
    for (int j = 1; j < T; ++j) lam = lam + w[j];
    if (!gt0(lam)) break;
    if (c >= SG_MAX_DRAWS) {
      code = SG_ERR_STEP_LIMIT;
      break;
    }
    if (!have || c - c0 >= 32u) {
      c0 = c;
      const U4 x = philox10(U4{c0 + (uint32_t)lane, node, Td, tag}, k0, k1);
      nE = -log_pos(u01_open(x.x, x.y));
      r2 = u01_open(x.z, x.w);
      have = true;
    }
    const int jj = (int)(c - c0);
    const double E = __shfl_sync(0xffffffffu, nE, jj);
    const double R2 = __shfl_sync(0xffffffffu, r2, jj);
    ++c;
    const double tau = E / lam;
    int u2[C];
    double w2[T];
#pragma unroll
    for (int p = 0; p < C; ++p) u2[p] = u[p];
#pragma unroll
    for (int j = 0; j < T; ++j) w2[j] = w[j];
    const int rc = fire<KIND>(u2, w2, lam * R2, kf, tb);
    const double tt = t + tau;
    if (order_key(tt) >= Tkey) break;
    t = tt;
#pragma unroll
    for (int p = 0; p < C; ++p) u[p] = u2[p];
#pragma unroll
    for (int j = 0; j < T; ++j) w[j] = w2[j];
    ++f;
    if (rc) {
      code = rc;
      break;
    }
  }
  }
  __syncwarp();
  if (lane == 0) {
#pragma unroll
    for (int p = 0; p < C; ++p) hs.u[p] = u[p];
    hs.c = c;
    hs.code = code;
    fired += f;
    drawn += c - c_in;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// The all events method (solver 'aem' of Sec. 3.4.2): every transition of a
// node is a channel with its own random stream, Philox counter (draws taken
// by the channel, node, transition, (3 << 24) | replicate), and the channels
// advance by the next reaction method of Gibson and Bruck: each holds an
// absolute firing time, the earliest fires, the fired channel draws a fresh
// Exp(1) waiting time scaled by its rate, a channel whose rate changes from
// a > 0 to a' > 0 rescales its residual time by a / a', one whose rate drops
// to 0 sleeps (time +inf), one that wakes draws afresh.  Firing times carry
// over from day to day; at each day start every rate is recomputed and the
// same rule applied.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int aem_draw(uint32_t &c, uint32_t node, uint32_t j, uint32_t tag,
                                        uint32_t k0, uint32_t k1, double &E) {
  if (c == 0xffffffffu) return SG_ERR_STEP_LIMIT;
  const U4 x = philox10(U4{c, node, j, tag}, k0, k1);
  ++c;
  E = -log_pos(u01_open(x.x, x.y));
  return 0;
}

// Channel j's new rate a_new at time t (the update rule above).
__device__ __forceinline__ int aem_update(double t, double a_new, double &a, double &tau,
                                          uint32_t &c, uint32_t node, uint32_t j, uint32_t tag,
                                          uint32_t k0, uint32_t k1, unsigned long long &drawn) {
  if (a_new == a) return 0;
  if (gt0(a) && gt0(a_new)) {
    tau = t + (a / a_new) * (tau - t);
  } else if (gt0(a_new)) {
    double E;
    const int rc = aem_draw(c, node, j, tag, k0, k1, E);
    if (rc) return rc;
    ++drawn;
    tau = t + E / a_new;
  } else {
    tau = __longlong_as_double(0x7ff0000000000000ll);  // +inf
  }
  a = a_new;
  return 0;
}

// Day start (t = Tn - 1): every rate recomputed, the update rule applied.
template <int KIND>
__device__ __forceinline__ int aem_day_start(const int *u, const double *kf, double *a,
                                             double *tau, uint32_t *c, double Tn, uint32_t node,
                                             uint32_t tag, uint32_t k0, uint32_t k1,
                                             const SgTables &tb, unsigned long long &drawn) {
  using M = ModelTraits<KIND>;
  const double t = Tn - 1.0;
#pragma unroll
  for (int j = 0; j < M::T; ++j) {
    const double w = M::rate_k(j, u, kf, tb.gdata);
    if (bad_rate(w)) return SG_ERR_RATE;
    const int rc = aem_update(t, w, a[j], tau[j], c[j], node, (uint32_t)j, tag, k0, k1, drawn);
    if (rc) return rc;
  }
  return 0;
}

enum { AEM_DONE = 0, AEM_HEAVY = 1 };

// The earliest channel (ties to the lowest index); -1 if all sleep.
template <int T>
__device__ __forceinline__ int aem_earliest(const double *tau, double &best) {
  int mu = -1;
  best = __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
  for (int j = 0; j < T; ++j) {
    if (tau[j] < best) {
      best = tau[j];
      mu = j;
    }
  }
  return mu;
}

// Firings of one node until Tn, at most `budget` of them in this call.  The
// fired channel and the woken ones take their Exp(1) draws from `draw(j,
// E)` (computed on the spot by a thread, from a lane table by a warp).
// Returns AEM_DONE, AEM_HEAVY (budget spent; state ready for a warp) or an
// error.
template <int KIND, typename Draw>
__device__ __forceinline__ int aem_steps(int *u, const double *kf, double *a, double *tau,
                                         uint32_t *c, double &t, uint32_t &nfired, double Tn,
                                         const SgTables &tb, unsigned long long &fired,
                                         int budget, Draw &&draw) {
  using M = ModelTraits<KIND>;
  constexpr int T = M::T;
  const double inf = __longlong_as_double(0x7ff0000000000000ll);
  for (int b = 0;; ++b) {
    double best;
    const int mu = aem_earliest<T>(tau, best);
    if (mu < 0 || best >= Tn) return AEM_DONE;
    if (nfired >= SG_MAX_DRAWS) return SG_ERR_STEP_LIMIT;
    if (b == budget) return AEM_HEAVY;
    ++nfired;
    t = best;
#pragma unroll
    for (int p = 0; p < M::C; ++p) u[p] += tb.S[mu][p];
    ++fired;
    const uint32_t dep = tb.dep[mu];
#pragma unroll
    for (int k = 0; k < T; ++k) {
      const bool marked = (dep >> k) & 1u;
      if (k != mu && !marked) continue;
      double w = a[k];
      if (marked) {
        w = M::rate_k(k, u, kf, tb.gdata);
        if (bad_rate(w)) return SG_ERR_RATE;
      }
      if (k == mu) {
        // the fired channel always redraws
        a[k] = w;
        if (gt0(w)) {
          double E;
          const int rc = draw(k, E);
          if (rc) return rc;
          tau[k] = t + E / w;
        } else {
          tau[k] = inf;
        }
      } else if (!(w == a[k])) {
        if (gt0(a[k]) && gt0(w)) {
          tau[k] = t + (a[k] / w) * (tau[k] - t);
        } else if (gt0(w)) {
          double E;
          const int rc = draw(k, E);
          if (rc) return rc;
          tau[k] = t + E / w;
        } else {
          tau[k] = inf;
        }
        a[k] = w;
      }
    }
  }
}

// A node handed from its thread to a warp (all events method).
template <int C, int NK, int T>
struct AemSlot {
  double t;
  double kf[NK];
  double a[T], tau[T];
  uint32_t c[T];
  uint32_t nfired;
  int32_t node, rep, code;
  int32_t u[C];
};

// Shared-memory slots for hand-offs (at most 24 KB, at most one per thread).
template <int C, int NK, int T>
struct AemSlots {
  static constexpr int n = (int)(24576 / sizeof(AemSlot<C, NK, T>)) < kDayBlock
                               ? (int)(24576 / sizeof(AemSlot<C, NK, T>))
                               : kDayBlock;
};

// The rest of a heavy node-day by a whole warp.  Every channel's next draws
// depend only on its counter, so lane l holds the Exp(1) value of draw
// c_j + (l mod B) of channel j = l / B (B = 32 / T lanes per channel), all
// computed at once; the firing loop runs on all lanes in step and takes a
// channel's next value from its lane.  When a channel has used its B values
// the table is recomputed from the current counters.  Same operations, in
// the same order, as the thread path.
template <int KIND>
__device__ void aem_warp(AemSlot<ModelTraits<KIND>::C, ModelTraits<KIND>::NK,
                                 ModelTraits<KIND>::T> &hs,
                         double Tn, uint32_t k0, uint32_t k1, const SgTables &tb,
                         unsigned long long &fired, unsigned long long &drawn) {
  using M = ModelTraits<KIND>;
  constexpr int C = M::C, T = M::T, NK = M::NK;
  constexpr int B = 32 / T;
  const int lane = threadIdx.x & 31;
  const int jl = lane / B, il = lane - jl * B;
  int u[C];
  double kf[NK], a[T], tau[T];
  uint32_t c[T];
  int used[T];
#pragma unroll
  for (int p = 0; p < C; ++p) u[p] = hs.u[p];
#pragma unroll
  for (int i = 0; i < NK; ++i) kf[i] = hs.kf[i];
#pragma unroll
  for (int j = 0; j < T; ++j) {
    a[j] = hs.a[j];
    tau[j] = hs.tau[j];
    c[j] = hs.c[j];
    used[j] = B;  // no table yet
  }
  double t = hs.t;
  uint32_t nfired = hs.nfired;
  const uint32_t node = (uint32_t)hs.node;
  const uint32_t tag = (SG_STREAM_AEM << 24) | (uint32_t)hs.rep;
  double myE = 0.0;
  unsigned long long f = 0, dr = 0;
  auto draw = [&](int j, double &E) -> int {
    uint32_t cj = 0;
    int uj = 0;
#pragma unroll
    for (int q = 0; q < T; ++q)
      if (q == j) {
        cj = c[q];
        uj = used[q];
      }
    if (cj == 0xffffffffu) return SG_ERR_STEP_LIMIT;
    if (uj == B) {
      // recompute the table from every channel's current counter
      if (jl < T) {
        uint32_t cl = 0;
#pragma unroll
        for (int q = 0; q < T; ++q)
          if (q == jl) cl = c[q];
        const uint32_t ci = cl + (uint32_t)il;
        // draws past the counter's end are never used (the counter check
        // above stops first); compute something harmless for them
        const U4 x = philox10(U4{ci < cl ? cl : ci, node, (uint32_t)jl, tag}, k0, k1);
        myE = -log_pos(u01_open(x.x, x.y));
      }
#pragma unroll
      for (int q = 0; q < T; ++q) used[q] = 0;
      uj = 0;
    }
    E = __shfl_sync(0xffffffffu, myE, j * B + uj);
#pragma unroll
    for (int q = 0; q < T; ++q)
      if (q == j) {
        ++c[q];
        ++used[q];
      }
    ++dr;
    return 0;
  };
  const int rc = aem_steps<KIND>(u, kf, a, tau, c, t, nfired, Tn, tb, f, -1, draw);
  if (lane == 0) {
#pragma unroll
    for (int p = 0; p < C; ++p) hs.u[p] = u[p];
#pragma unroll
    for (int j = 0; j < T; ++j) {
      hs.a[j] = a[j];
      hs.tau[j] = tau[j];
      hs.c[j] = c[j];
    }
    hs.code = rc < 0 ? rc : 0;
    fired += f;
    drawn += dr;
  }
  __syncwarp();
}

// The fields of one planned event and the first Philox block of its word
// stream (a function of the seed, the list index and the replicate only), so
// that they can be fetched and computed ahead of the event.
struct E1Rec {
  int type, n, shift;
  uint32_t mask;
  long long idx;
  double prop;
  U4 first;
};

__device__ __forceinline__ E1Rec load_e1(const SgTables &tb, const EvDev &ev, long long j, int rep,
                                         uint32_t k0, uint32_t k1) {
  E1Rec r;
  r.type = ev.type[j];
  r.mask = tb.Emask[ev.select[j]];
  r.n = ev.n[j];
  r.shift = ev.shift[j];
  r.idx = ev.index[j];
  r.prop = ev.proportion[j];
  r.first = philox10(U4{0u, (uint32_t)(unsigned long long)r.idx,
                        (uint32_t)((unsigned long long)r.idx >> 32),
                        (SG_STREAM_EVENTS << 24) | (uint32_t)rep},
                     k0, k1);
  return r;
}

// One E1 event (exit, enter or internal transfer, Sec. 3.3) on a node whose
// counts are in the calling thread's registers.  Returns 0 or an error.
template <int C>
__device__ __forceinline__ int apply_e1(int *u, const SgTables &tb, const E1Rec &e, int rep,
                                        uint32_t k0, uint32_t k1) {
  const int type = e.type;
  const uint32_t mask = e.mask;
  const int n = e.n;
  if (type == SG_ENTER) {
    const int first = __ffs(mask) - 1;  // first selected compartment
#pragma unroll
    for (int p = 0; p < C; ++p)
      if (p == first) u[p] += n;
    return 0;
  }
  long long total = 0;
#pragma unroll
  for (int p = 0; p < C; ++p)
    if ((mask >> p) & 1u) total += u[p];
  const long long k = n > 0 ? (long long)n : (long long)round(e.prop * (double)total);
  if (k < 0 || k > total) return SG_ERR_EVENT_UNDERFLOW;
  int moved[C];
#pragma unroll
  for (int p = 0; p < C; ++p) moved[p] = 0;
  if (k > 0) {
    WordStream ws;
    ws.init_with_first(((uint64_t)k1 << 32) | k0, e.idx, rep, e.first);
    for (long long i = 0; i < k; ++i) {
      uint32_t x = ws.below((uint32_t)(total - i));
      bool taken = false;
#pragma unroll
      for (int p = 0; p < C; ++p) {
        if (taken || !((mask >> p) & 1u)) continue;
        const uint32_t rem = (uint32_t)(u[p] - moved[p]);
        if (x < rem) {
          ++moved[p];
          taken = true;
        } else {
          x -= rem;
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < C; ++p) u[p] -= moved[p];
  if (type == SG_EXIT) return 0;
  const int q = e.shift;  // internal transfer: validated q >= 0
#pragma unroll
  for (int dst = 0; dst < C; ++dst) {
    int add = 0;
#pragma unroll
    for (int p = 0; p < C; ++p)
      if (p + tb.Nsh[q][p] == dst) add += moved[p];
    u[dst] += add;
  }
  return 0;
}

// The number of individuals an E1 event draws (exit or internal transfer;
// 0 for an enter, -1 for one that moves more than exist).
template <int C>
__device__ __forceinline__ long long e1_draws(const int *u, const SgTables &tb, const E1Rec &e) {
  if (e.type == SG_ENTER) return 0;
  long long total = 0;
#pragma unroll
  for (int p = 0; p < C; ++p)
    if ((e.mask >> p) & 1u) total += u[p];
  const long long k = e.n > 0 ? (long long)e.n : (long long)round(e.prop * (double)total);
  return (k < 0 || k > total) ? -1 : k;
}

// The E1 event `e` of lane `owner` (an exit or internal transfer drawing at
// least kUrnWarp individuals), applied by the whole warp: the owner's counts
// and event fields are broadcast, the warp samples the urn (urn_warp, the
// same draws as apply_e1), and the owner's counts are updated.  Every lane
// calls it with the same owner; returns the owner's result in every lane.
template <int C>
__device__ __forceinline__ int apply_e1_warp(int *u, const SgTables &tb, const E1Rec &e,
                                             int owner, int rep, uint32_t k0, uint32_t k1) {
  const int lane = threadIdx.x & 31;
  int cu[C];
#pragma unroll
  for (int p = 0; p < C; ++p) cu[p] = __shfl_sync(0xffffffffu, u[p], owner);
  const int type = __shfl_sync(0xffffffffu, e.type, owner);
  const uint32_t mask = __shfl_sync(0xffffffffu, e.mask, owner);
  const int n = __shfl_sync(0xffffffffu, e.n, owner);
  const int shift = __shfl_sync(0xffffffffu, e.shift, owner);
  const long long idx = __shfl_sync(0xffffffffu, e.idx, owner);
  const double prop = __shfl_sync(0xffffffffu, e.prop, owner);
  const int r = __shfl_sync(0xffffffffu, rep, owner);
  long long total = 0;
#pragma unroll
  for (int p = 0; p < C; ++p)
    if ((mask >> p) & 1u) total += cu[p];
  const long long k = n > 0 ? (long long)n : (long long)round(prop * (double)total);
  if (k < 0 || k > total) return SG_ERR_EVENT_UNDERFLOW;
  int moved[C];
  urn_warp<C>(cu, mask, (uint32_t)k, (uint32_t)total, ((uint64_t)k1 << 32) | k0, idx, r, moved);
  if (lane == owner) {
#pragma unroll
    for (int p = 0; p < C; ++p) u[p] -= moved[p];
    if (type != SG_EXIT) {
#pragma unroll
      for (int dst = 0; dst < C; ++dst) {
        int add = 0;
#pragma unroll
        for (int p = 0; p < C; ++p)
          if (p + tb.Nsh[shift][p] == dst) add += moved[p];
        u[dst] += add;
      }
    }
  }
  return 0;
}

// Post time step and recording for unit time Tf (the state after its
// events).  Returns 0 or SG_ERR_PTS.
template <int KIND>
__device__ __forceinline__ int finish_step(int Tf, const int *u, double *v, const int *ends,
                                           const SgTables &tb, const DayArgs &a, int rep,
                                           int node) {
  using M = ModelTraits<KIND>;
  int code = 0;
  if (M::NV > 0) {
    const int r = post_step<KIND>(v, u, ends, tb.gdata, Tf);
    if (r < 0) code = r;
  }
  const int m = a.rec[Tf - a.t0];
  if (m >= 0) {
    const long long base = ((long long)rep * a.M + m) * tb.n_nodes + node;
    if (a.U) {
#pragma unroll
      for (int p = 0; p < M::C; ++p) a.U[base * M::C + p] = u[p];
    }
    if (a.V) {
#pragma unroll
      for (int q = 0; q < M::NV; ++q) a.V[base * M::NV + q] = v[q];
    }
    record_sparse<M::C, M::NV>(a.out, m, rep, node, u, v);
  }
  return code;
}

// The day kernel: one thread per (replicate, node) for a run of days
// T_begin .. T_end - 1 with no external transfers before T_end - 1.  Per day:
// rates, SSA (thread, then warp for heavy nodes), the node's E1 events, and
// (unless a kernel boundary follows) the post time step and recording.
template <int KIND, bool AEM>
__global__ void __launch_bounds__(kDayBlock)
k_days(const SgTables tb, const DayArgs a) {
  using M = ModelTraits<KIND>;
  constexpr int C = M::C, T = M::T, NV = M::NV, NK = M::NK;
  __shared__ HeavySlot<C, NK> s_heavy[AEM ? 1 : kDayBlock];
  constexpr int kAemSlots = AEM ? AemSlots<C, NK, T>::n : 1;
  __shared__ AemSlot<C, NK, T> s_aheavy[kAemSlots];
  __shared__ int s_nheavy;
  pdl_trigger();
  const int Nn = tb.n_nodes;
  const long long gid = (long long)blockIdx.x * a.npb + threadIdx.x;
  const long long total = (long long)Nn * a.n_rep;
  const bool in_range = (int)threadIdx.x < a.npb && gid < total;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned long long fired = 0, drawn = 0, applied = 0;
  int rep = 0, node = 0, code = 0, bad_day = 0;
  long long bad_event = -1;
  int u[C];
  double v[NV > 0 ? NV : 1];
  int ld[4] = {0, 0, 0, 0};  // season ends of the node (integer form)
#pragma unroll
  for (int p = 0; p < C; ++p) u[p] = 0;
  v[0] = 0.0;
  long long ecur = 0, ebase = 0, eend = 0;
  int next_day = 0x7fffffff;
  double ch_a[AEM ? T : 1], ch_tau[AEM ? T : 1];  // all events method channels
  uint32_t ch_c[AEM ? T : 1];
  // static inputs first (they overlap the previous kernel's tail)
  if (in_range) {
    rep = (int)(gid / Nn);
    node = (int)(gid - (long long)rep * Nn);
    if (NV > 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        ld[i] = season_end_int(a.ldata[(long long)node * tb.n_ldata + i]);
    }
    if (a.ev.e1_node_off) {
      const long long key = (long long)(a.slots > 1 ? rep : 0) * Nn + node;
      ebase = a.ev.e1_node_off[key];
      eend = a.ev.e1_node_off[key + 1];
    }
  }
  pdl_wait();
  bool live = in_range && *(volatile int32_t *)&a.err->code == 0;
  if (live && a.emu_part == 1) live = a.emu_flag[gid] == 0;
  if (live && a.emu_part == 2) live = a.emu[gid * 4 + 3] != 0;
  if (live) {
#pragma unroll
    for (int p = 0; p < C; ++p) u[p] = a.u[gid * C + p];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = a.v[gid * NV + q];
    if (a.ev.e1_node_off) {
      ecur = ebase + a.e1_cur[gid];
      if (ecur < eend) next_day = a.ev.e1_day[ecur];
    }
    if constexpr (AEM) {
#pragma unroll
      for (int j = 0; j < T; ++j) {
        ch_a[j] = a.aem_a[j * total + gid];
        ch_tau[j] = a.aem_tau[j * total + gid];
        ch_c[j] = a.aem_cnt[j * total + gid];
      }
    }
    if (a.finish_first) {
      code = finish_step<KIND>(a.T_begin - 1, u, v, ld, tb, a, rep, node);
      if (code) bad_day = a.T_begin - 1;
    }
  }
  if (a.finish_first && a.out.prev) {
    const int m = a.rec[a.T_begin - 1 - a.t0];
    if (m >= 0)
      prevalence_add<C>(a.out, in_range ? (long long)rep * a.M + m : -1, live && code == 0, u);
  }
  const int grep = a.rep0 + rep;  // global replicate: streams, error reports
  const uint32_t tag = (SG_STREAM_SSA << 24) | (uint32_t)grep;
  for (int Td = a.T_begin; Td < a.T_end; ++Td) {
    const double Tn = (double)Td;
    if (threadIdx.x == 0) s_nheavy = 0;
    __syncthreads();
    int my = -1;
    // the node's first E1 event of the day: fields and first random block
    // fetched now, so that their latency overlaps the SSA
    const int d = Td - a.t0 - 1;
    const bool e1_today = live && code == 0 && next_day == d;
    E1Rec pre;
    if (e1_today) pre = load_e1(tb, a.ev, ecur, grep, a.k0, a.k1);
    const bool emulated =
        !AEM && live && code == 0 && a.emu != nullptr && a.emu[gid * 4 + 3] != 0;
    if (emulated) {
      // the learned emulator's sampled one-day increments (SISe3 only):
      // I_a += d_a, S_a -= d_a, each age class keeps its size
#pragma unroll
      for (int h = 0; h < C / 2; ++h) {
        const int dlt = a.emu[gid * 4 + h];
        u[2 * h] -= dlt;
        u[2 * h + 1] += dlt;
      }
    }
    if (AEM && live && code == 0) {
      double kf[NK];
      M::prepare(v, tb.gdata, kf);
      const uint32_t tag = (SG_STREAM_AEM << 24) | (uint32_t)grep;
      code = aem_day_start<KIND>(u, kf, ch_a, ch_tau, ch_c, Tn, (uint32_t)node, tag, a.k0, a.k1,
                                 tb, drawn);
      double t = Tn - 1.0;
      uint32_t nfired = 0;
      if (code == 0) {
        auto draw = [&](int j, double &E) -> int {
          uint32_t cj = 0;
#pragma unroll
          for (int q = 0; q < T; ++q)
            if (q == j) cj = ch_c[q];
          const int rc = aem_draw(cj, (uint32_t)node, (uint32_t)j, tag, a.k0, a.k1, E);
#pragma unroll
          for (int q = 0; q < T; ++q)
            if (q == j) ch_c[q] = cj;
          if (rc == 0) ++drawn;
          return rc;
        };
        const int r = aem_steps<KIND>(u, kf, ch_a, ch_tau, ch_c, t, nfired, Tn, tb, fired,
                                      a.heavy_after, draw);
        if (r == AEM_HEAVY) {
          const int slot = atomicAdd(&s_nheavy, 1);
          if (slot < kAemSlots) {
            my = slot;
            AemSlot<C, NK, T> &hs = s_aheavy[slot];
            hs.t = t;
#pragma unroll
            for (int i = 0; i < NK; ++i) hs.kf[i] = kf[i];
#pragma unroll
            for (int j = 0; j < T; ++j) {
              hs.a[j] = ch_a[j];
              hs.tau[j] = ch_tau[j];
              hs.c[j] = ch_c[j];
            }
            hs.nfired = nfired;
            hs.node = node;
            hs.rep = grep;
            hs.code = 0;
#pragma unroll
            for (int p = 0; p < C; ++p) hs.u[p] = u[p];
          } else {
            // no slot left: the thread finishes its node itself
            const int r2 = aem_steps<KIND>(u, kf, ch_a, ch_tau, ch_c, t, nfired, Tn, tb, fired,
                                           -1, draw);
            if (r2 < 0) code = r2;
          }
        } else if (r < 0) {
          code = r;
        }
      }
      if (code) bad_day = Td;
    }
    if (!AEM && live && code == 0 && !emulated) {
      double kf[NK], w[T];
      M::prepare(v, tb.gdata, kf);
#pragma unroll
      for (int j = 0; j < T; ++j) {
        w[j] = M::rate_k(j, u, kf, tb.gdata);
        if (bad_rate(w[j])) code = SG_ERR_RATE;
      }
      if (code == 0) {
        double t = (double)(Td - 1);
        uint32_t c = 0;
        const int r = ssa_thread<KIND>(u, w, kf, t, c, Tn, (uint32_t)node, (uint32_t)Td, tag,
                                       a.k0, a.k1, a.heavy_after, tb, fired);
        drawn += c;
        if (r == SSA_HEAVY) {
          my = atomicAdd(&s_nheavy, 1);
          HeavySlot<C, NK> &hs = s_heavy[my];
          hs.t = t;
#pragma unroll
          for (int i = 0; i < NK; ++i) hs.kf[i] = kf[i];
          hs.c = c;
          hs.node = node;
          hs.rep = grep;
          hs.code = 0;
#pragma unroll
          for (int p = 0; p < C; ++p) hs.u[p] = u[p];
        } else if (r < 0) {
          code = r;
        }
      }
      if (code) bad_day = Td;
    }
    __syncthreads();
    if constexpr (!AEM) {
      const int nh = s_nheavy;
      for (int h = warp; h < nh; h += nwarps)
        ssa_warp<KIND>(s_heavy[h], Tn, (uint32_t)Td, a.k0, a.k1, tb, fired, drawn);
    } else {
      const int nh = min(s_nheavy, kAemSlots);
      for (int h = warp; h < nh; h += nwarps)
        aem_warp<KIND>(s_aheavy[h], Tn, a.k0, a.k1, tb, fired, drawn);
    }
    __syncthreads();
    if (AEM && my >= 0) {
#pragma unroll
      for (int p = 0; p < C; ++p) u[p] = s_aheavy[my].u[p];
#pragma unroll
      for (int j = 0; j < T; ++j) {
        ch_a[j] = s_aheavy[my].a[j];
        ch_tau[j] = s_aheavy[my].tau[j];
        ch_c[j] = s_aheavy[my].c[j];
      }
      if (s_aheavy[my].code) {
        code = s_aheavy[my].code;
        bad_day = Td;
      }
      my = -1;
    }
    if (my >= 0) {
#pragma unroll
      for (int p = 0; p < C; ++p) u[p] = s_heavy[my].u[p];
      if (s_heavy[my].code) {
        code = s_heavy[my].code;
        bad_day = Td;
      }
    }
    // this node's E1 events of day Td, in (time, type, list index) order:
    // each round every lane with an event left takes its next one, applied
    // in the thread, or by the whole warp when it draws kUrnWarp or more
    // individuals (every thread of the block reaches this loop)
    {
      bool pend = e1_today && code == 0;
      bool first = true;
      const int lane = threadIdx.x & 31;
      while (__any_sync(0xffffffffu, pend)) {
        E1Rec e;
        bool heavy = false;
        if (pend) {
          if (ecur < eend && a.ev.e1_day[ecur] == d) {
            e = first ? pre : load_e1(tb, a.ev, ecur, grep, a.k0, a.k1);
            first = false;
            heavy = e1_draws<C>(u, tb, e) >= kUrnWarp;
            if (!heavy) {
              const int rc = apply_e1<C>(u, tb, e, grep, a.k0, a.k1);
              if (rc) {
                code = rc;
                bad_day = Td;
                bad_event = a.ev.index[ecur];
                pend = false;
              } else {
                ++applied;
                ++ecur;
              }
            }
          } else {
            pend = false;
          }
        }
        unsigned hm = __ballot_sync(0xffffffffu, heavy);
        while (hm) {
          const int L = __ffs(hm) - 1;
          hm &= hm - 1;
          const int rc = apply_e1_warp<C>(u, tb, e, L, grep, a.k0, a.k1);
          if (lane == L) {
            if (rc) {
              code = rc;
              bad_day = Td;
              bad_event = a.ev.index[ecur];
              pend = false;
            } else {
              ++applied;
              ++ecur;
            }
          }
        }
      }
      if (e1_today) next_day = ecur < eend ? a.ev.e1_day[ecur] : 0x7fffffff;
    }
    if (a.grid_bar && a.wave_off) {
      // persistent run: the day's external transfers between two grid
      // barriers, by the block holding each replicate's first node, on the
      // state in global memory
      const long long wlo = a.wave_off[(long long)d * a.slots];
      const long long whi = a.wave_off[(long long)(d + 1) * a.slots];
      if (wlo < whi) {  // the same decision in every block
        if (live) {
#pragma unroll
          for (int p = 0; p < C; ++p) a.u[gid * C + p] = u[p];
        }
        __threadfence();
        if (!grid_barrier(a.grid_bar, a.n_blocks, a.err)) break;
        const long long g_lo = (long long)blockIdx.x * a.npb;
        const long long g_hi = min(total, g_lo + a.npb) - 1;
        for (int r = (int)((g_lo + Nn - 1) / Nn); (long long)r * Nn <= g_hi; ++r) {
          // this block holds node 0 of replicate r
          const long long k = (long long)d * a.slots + (a.slots > 1 ? r : 0);
          e2_rep_block<C>(tb, a, r, Td, a.wave_off[k], a.wave_off[k + 1]);
        }
        __threadfence();
        if (!grid_barrier(a.grid_bar, a.n_blocks, a.err)) break;
        if (live) {
#pragma unroll
          for (int p = 0; p < C; ++p) u[p] = __ldcg(a.u + gid * C + p);
        }
      }
    }
    if (live && code == 0 && (Td + 1 < a.T_end || a.finish_last)) {
      code = finish_step<KIND>(Td, u, v, ld, tb, a, rep, node);
      if (code) bad_day = Td;
    }
    if ((Td + 1 < a.T_end || a.finish_last) && a.out.prev) {
      const int m = a.rec[Td - a.t0];
      if (m >= 0)
        prevalence_add<C>(a.out, in_range ? (long long)rep * a.M + m : -1, live && code == 0,
                          u);
    }
  }
  if (live) {
    if (code) report(a.err, code, a.rep0 + rep, node, bad_day, bad_event);
#pragma unroll
    for (int p = 0; p < C; ++p) a.u[gid * C + p] = u[p];
#pragma unroll
    for (int q = 0; q < NV; ++q) a.v[gid * NV + q] = v[q];
    if (a.ev.e1_node_off) a.e1_cur[gid] = (int32_t)(ecur - ebase);
    if constexpr (AEM) {
#pragma unroll
      for (int j = 0; j < T; ++j) {
        a.aem_a[j * total + gid] = ch_a[j];
        a.aem_tau[j * total + gid] = ch_tau[j];
        a.aem_cnt[j * total + gid] = ch_c[j];
      }
    }
  }
  if (a.e2_done) {
    // the last block to finish a replicate's nodes runs its external
    // transfers of T_end - 1 (threadfence-reduction pattern: no block waits)
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    const long long g_lo = (long long)blockIdx.x * a.npb;
    const long long g_hi = min(total, g_lo + a.npb) - 1;
    for (int r = (int)(g_lo / Nn); r <= (int)(g_hi / Nn); ++r) {
      if (threadIdx.x == 0) {
        const long long b_first = (long long)r * Nn / a.npb;
        const long long b_last = ((long long)(r + 1) * Nn - 1) / a.npb;
        const int old = atomicAdd(&a.e2_done[r], 1);
        s_last = old == (int)(b_last - b_first);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        long long w0 = a.e2_wb, w1 = a.e2_we;
        if (a.slots > 1) {
          w0 = a.wave_off[(long long)a.e2_day_index * a.slots + r];
          w1 = a.wave_off[(long long)a.e2_day_index * a.slots + r + 1];
        }
        e2_rep_block<C>(tb, a, r, a.T_end - 1, w0, w1);
        if (threadIdx.x == 0) a.e2_done[r] = 0;
      }
      __syncthreads();
    }
  }
  // one atomic per warp for the counters
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fired += __shfl_down_sync(0xffffffffu, fired, off);
    drawn += __shfl_down_sync(0xffffffffu, drawn, off);
    applied += __shfl_down_sync(0xffffffffu, applied, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (drawn | fired) {
      atomicAdd(&a.cnt->reactions, fired);
      atomicAdd(&a.cnt->draws, drawn);
    }
    if (applied) atomicAdd(&a.cnt->events, applied);
  }
}

// ---------------------------------------------------------------------------
// Day kernel for sparse activity (the direct method on the built-in kinds).
// On cattle-shaped workloads only a few percent of the node-days have a
// positive total rate; the rest take no draw, and on the thread-per-node
// schedule above their threads still compute every rate and the post time
// step in FP64 (GB300's weakest pipe) and wait at block barriers for the
// block's few active nodes.  Here a block owns a contiguous range of
// `npb` (> kDayBlock) (replicate, node) units whose state stays in global
// memory (L2), and each day it
//   1. visits every unit: finishes the previous day when the launch starts
//      with it, and tests whether the unit's day is certainly empty
//      (quiescent<>: no infected animal and phi exactly +0, with finite
//      parameters every rate is then +-0 and the post time step leaves phi
//      at +0, so skipping them changes no bit); the other units get their
//      rates, and those with lambda > 0 go to a shared list;
//   2. runs the SSA of the listed units, one thread each (dense lanes), a
//      unit needing more than heavy_after draws handed to a warp (32 draws'
//      random numbers at once, as above);
//   3. visits every unit again: its E1 events of the day (per-unit cursor)
//      and, unless the day's external transfers follow in their own kernel,
//      the post time step and recording.
// Units are taken in chunks of kSparseChunk so that the list fits in shared
// memory.  Every unit's operations and random draws are the ones of the
// thread-per-node schedule, so the results are identical.
// ---------------------------------------------------------------------------
constexpr int kSparseBlock = 256;   // threads of the sparse-schedule day kernel
constexpr int kSparseChunk = 8192;  // units per pass through the active list
constexpr int kSparseHeavy = 64;    // warp hand-off slots per pass

// A unit whose day is certainly empty: no infected animal and phi == +0
// (bit pattern 0).  Exact only with finite model parameters (DayArgs::quiet).
template <int KIND>
__device__ __forceinline__ bool quiescent(const int *u, const double *v) {
  if constexpr (KIND == SG_SIR || KIND == SG_SIS) {
    return u[1] == 0;
  } else if constexpr (KIND == SG_SISE) {
    return u[1] == 0 && __double_as_longlong(v[0]) == 0;
  } else if constexpr (KIND == SG_SISE3) {
    return (u[1] | u[3] | u[5]) == 0 && __double_as_longlong(v[0]) == 0;
  } else {
    return false;
  }
}

__device__ __forceinline__ void load_ends(const DayArgs &a, const SgTables &tb, int node,
                                          int *ld) {
#pragma unroll
  for (int i = 0; i < 4; ++i) ld[i] = season_end_int(a.ldata[(long long)node * tb.n_ldata + i]);
}

// Recording of a unit whose post time step leaves it unchanged (tspan
// slot m >= 0): dense U / V and the sparse entries.
template <int C, int NV>
__device__ __forceinline__ void record_unit(const DayArgs &a, int Nn, int m, int rep, int node,
                                            const int *u, const double *v) {
  const long long base = ((long long)rep * a.M + m) * Nn + node;
  if (a.U) {
#pragma unroll
    for (int p = 0; p < C; ++p) a.U[base * C + p] = u[p];
  }
  if (a.V) {
#pragma unroll
    for (int q = 0; q < NV; ++q) a.V[base * NV + q] = v[q];
  }
  record_sparse<C, NV>(a.out, m, rep, node, u, v);
}

// Post time step and recording of unit time Tf for one unit of the sparse
// schedule (counts u, continuous state v, stored back); a quiescent unit's
// post time step is skipped (phi stays +0).  Returns 0 or SG_ERR_PTS.
template <int KIND>
__device__ __forceinline__ int sparse_finish(int Tf, const int *u, double *v, bool quiet,
                                             const SgTables &tb, const DayArgs &a, int rep,
                                             int node, long long gid) {
  using M = ModelTraits<KIND>;
  constexpr int C = M::C, NV = M::NV;
  if (quiet && quiescent<KIND>(u, v)) {
    const int m = a.rec[Tf - a.t0];
    if (m >= 0) {
      const long long base = ((long long)rep * a.M + m) * tb.n_nodes + node;
      if (a.U) {
#pragma unroll
        for (int p = 0; p < C; ++p) a.U[base * C + p] = u[p];
      }
      if (a.V) {
#pragma unroll
        for (int q = 0; q < NV; ++q) a.V[base * NV + q] = v[q];
      }
      record_sparse<C, NV>(a.out, m, rep, node, u, v);
    }
    return 0;
  }
  int ld[4] = {0, 0, 0, 0};
  if (NV > 0) load_ends(a, tb, node, ld);
  const int code = finish_step<KIND>(Tf, u, v, ld, tb, a, rep, node);
  if (code) report(a.err, code, a.rep0 + rep, node, Tf, -1);
#pragma unroll
  for (int q = 0; q < NV; ++q) a.v[gid * NV + q] = v[q];
  return code;
}

// E1 events of day index d (unit time Td) of the unit of every lane with
// `has`, in (time, type, list index) order, for the sparse schedule (state
// in device memory).  Warp-uniform: all 32 lanes call it.  Every round each
// lane with an event left takes its next one, applied in the thread or
// (kUrnWarp or more individuals drawn) by the whole warp.  Returns the
// lane's error code (0 if none).
template <int C>
__device__ __forceinline__ int sparse_e1(bool has, long long gid, int rep, int node, int Td,
                                         int d, const SgTables &tb, const DayArgs &a,
                                         uint32_t k0, uint32_t k1,
                                         unsigned long long &applied) {
  const int lane = threadIdx.x & 31;
  const int Nn = tb.n_nodes;
  long long ecur = 0, eend = 0, ebase = 0;
  int code = 0;
  int u[C];
#pragma unroll
  for (int p = 0; p < C; ++p) u[p] = 0;
  if (has) {
    const long long key = (long long)(a.slots > 1 ? rep : 0) * Nn + node;
    ebase = a.ev.e1_node_off[key];
    eend = a.ev.e1_node_off[key + 1];
    ecur = ebase + a.e1_cur[gid];
#pragma unroll
    for (int p = 0; p < C; ++p) u[p] = a.u[gid * C + p];
  }
  const int grep = a.rep0 + rep;
  bool pend = has;
  while (__any_sync(0xffffffffu, pend)) {
    E1Rec e;
    bool heavy = false;
    if (pend) {
      if (ecur < eend && a.ev.e1_day[ecur] == d) {
        e = load_e1(tb, a.ev, ecur, grep, k0, k1);
        heavy = e1_draws<C>(u, tb, e) >= kUrnWarp;
        if (!heavy) {
          const int rc = apply_e1<C>(u, tb, e, grep, k0, k1);
          if (rc) {
            code = rc;
            report(a.err, rc, grep, node, Td, a.ev.index[ecur]);
            pend = false;
          } else {
            ++applied;
            ++ecur;
          }
        }
      } else {
        pend = false;
      }
    }
    unsigned hm = __ballot_sync(0xffffffffu, heavy);
    while (hm) {
      const int L = __ffs(hm) - 1;
      hm &= hm - 1;
      const int rc = apply_e1_warp<C>(u, tb, e, L, grep, k0, k1);
      if (lane == L) {
        if (rc) {
          code = rc;
          report(a.err, rc, grep, node, Td, a.ev.index[ecur]);
          pend = false;
        } else {
          ++applied;
          ++ecur;
        }
      }
    }
  }
  if (has) {
#pragma unroll
    for (int p = 0; p < C; ++p) a.u[gid * C + p] = u[p];
    a.e1_cur[gid] = (int32_t)(ecur - ebase);
    a.e1_next[gid] = ecur < eend ? a.ev.e1_day[ecur] : 0x7fffffff;
  }
  return code;
}

// E1 events of day Td of the units marked in a chunk's bitmaps: units with
// events today (e1bits) that took SSA draws (actbits) when `act`, else those
// that did not.  A warp takes 32 words (1,024 units) at a time from *take,
// counts the marked units of each word, and gives the k-th marked unit of
// the take to lane k mod 32 in round k / 32 (word by a search over the
// warp's prefix counts, bit by halving), so the lanes stay full however
// sparse the marks are.  Warp-uniform; called by every lane of a warp.
template <int C>
__device__ __forceinline__ void sparse_e1_bits(const uint32_t *e1bits, const uint32_t *actbits,
                                               bool act, int *take, int nw, long long gbase,
                                               int Td, int d, const SgTables &tb,
                                               const DayArgs &a, uint32_t k0, uint32_t k1,
                                               unsigned long long &applied) {
  const int lane = threadIdx.x & 31;
  const int Nn = tb.n_nodes;
  for (;;) {
    int g = 0;
    if (lane == 0) g = atomicAdd(take, 32);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= nw) break;
    const int wi = g + lane;
    uint32_t m = 0;
    if (wi < nw) m = e1bits[wi] & (act ? actbits[wi] : ~actbits[wi]);
    const int cnt = __popc(m);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const int excl = incl - cnt;
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll 1
    for (int r0 = 0; r0 < tot; r0 += 32) {
      const int k = r0 + lane;
      // the last word whose count starts at or below k
      int w = 0;
#pragma unroll
      for (int sft = 16; sft > 0; sft >>= 1) {
        const int e = __shfl_sync(0xffffffffu, excl, w + sft);
        if (e <= k) w += sft;
      }
      uint32_t x = __shfl_sync(0xffffffffu, m, w);
      int n = k - __shfl_sync(0xffffffffu, excl, w);
      int pos = 0;
#pragma unroll
      for (int sft = 16; sft > 0; sft >>= 1) {
        const int c = __popc(x & ((1u << sft) - 1u));
        if (n >= c) {
          n -= c;
          x >>= sft;
          pos += sft;
        }
      }
      const bool has = k < tot;
      long long gid = 0;
      int rep = 0, node = 0;
      if (has) {
        gid = gbase + (long long)(g + w) * 32 + pos;
        rep = (int)(gid / Nn);
        node = (int)(gid - (long long)rep * Nn);
      }
      sparse_e1<C>(has, gid, rep, node, Td, d, tb, a, k0, k1, applied);
    }
  }
}

// (replicate, node) of a unit index, advanced by a stride without dividing
// (the passes over a block's units step by kSparseBlock).
struct UnitPos {
  int rep, node;
  __device__ __forceinline__ void set(long long gid, int Nn) {
    rep = (int)(gid / Nn);
    node = (int)(gid - (long long)rep * Nn);
  }
  __device__ __forceinline__ void advance(int by, int Nn) {
    node += by;
    while (node >= Nn) {
      node -= Nn;
      ++rep;
    }
  }
};

template <int KIND>
__global__ void __launch_bounds__(kSparseBlock)
k_days_sparse(const SgTables tb, const DayArgs a) {
  using M = ModelTraits<KIND>;
  constexpr int C = M::C, T = M::T, NV = M::NV, NK = M::NK;
  // lists of units of the current chunk (indices relative to the chunk)
  __shared__ uint16_t s_act[kSparseChunk];
  __shared__ uint16_t s_nq[kSparseChunk];  // units of the chunk that are not quiescent
  __shared__ HeavySlot<C, NK> s_heavy[kSparseHeavy];
  __shared__ uint32_t s_actbits[kSparseChunk / 32];  // units taking SSA draws today
  __shared__ uint32_t s_e1bits[kSparseChunk / 32];   // units with E1 events today
  __shared__ int s_nact, s_nheavy, s_stop, s_next, s_nnq, s_e1take, s_e1late, s_nshort;
  pdl_trigger();
  const int Nn = tb.n_nodes;
  const long long total = (long long)Nn * a.n_rep;
  const long long g0 = (long long)blockIdx.x * a.npb;
  const int nub = (int)max(0LL, min((long long)a.npb, total - g0));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const bool quiet = a.quiet != 0;
  const bool has_e1 = a.ev.e1_node_off != nullptr;
  const uint32_t k0 = a.k0, k1 = a.k1;
  unsigned long long rated = 0;  // units whose rates this thread evaluated
  // a unit whose expected transitions in the day (lambda times one day) reach
  // this goes to a warp at once
  const double heavy_rate = (double)max(a.heavy_after, 1);
  unsigned long long fired = 0, drawn = 0, applied = 0;
  pdl_wait();
  if (a.finish_first && a.T_begin >= a.T_end &&
      *(volatile int32_t *)&a.err->code == 0) {
    // a launch that only finishes unit time T_begin - 1 (the run's last
    // step after its external transfers)
    const int Tf = a.T_begin - 1;
    UnitPos pos;
    pos.set(g0 + tid, Nn);
    for (int i0 = 0; i0 < nub; i0 += kSparseBlock, pos.advance(kSparseBlock, Nn)) {
      const int i = i0 + tid;
      const bool in = i < nub;
      const long long gid = g0 + i;
      int u[C];
      double v[NV > 0 ? NV : 1];
      int rep = 0, node = 0, code = 0;
      v[0] = 0.0;
#pragma unroll
      for (int p = 0; p < C; ++p) u[p] = 0;
      if (in) {
        rep = pos.rep;
        node = pos.node;
#pragma unroll
        for (int p = 0; p < C; ++p) u[p] = a.u[gid * C + p];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = a.v[gid * NV + q];
        code = sparse_finish<KIND>(Tf, u, v, quiet, tb, a, rep, node, gid);
      }
      if (a.out.prev) {
        const int m = a.rec[Tf - a.t0];
        if (m >= 0)
          prevalence_add<C>(a.out, in ? (long long)rep * a.M + m : -1, in && code == 0, u);
      }
    }
  }
  for (int Td = a.T_begin; Td < a.T_end; ++Td) {
    // a failed run stops at the next day boundary (the block's verdict)
    if (tid == 0) s_stop = *(volatile int32_t *)&a.err->code != 0;
    __syncthreads();
    if (s_stop) break;
    const double Tn = (double)Td;
    const int d = Td - a.t0 - 1;
    // the post time step and recording of Td - 1 in this day's first
    // passes: at a launch that finishes the previous one's last day, and on
    // every day after the first when the block runs its replicates'
    // external transfers itself
    const bool fin_prev = (Td == a.T_begin && a.finish_first) ||
                          (a.e2_inblock && Td > a.T_begin);
    for (int c0 = 0; c0 < nub; c0 += kSparseChunk) {
      const int cn = min(kSparseChunk, nub - c0);
      if (tid == 0) {
        s_nact = 0;
        s_nheavy = 0;
        s_next = 0;
        s_nnq = 0;
        s_e1take = 0;
        s_e1late = 0;
        s_nshort = 0;
      }
      for (int q = tid; q < kSparseChunk / 32; q += kSparseBlock) s_actbits[q] = 0u;
      __syncthreads();
      // 1a. every unit of the chunk, four per thread per step (their loads
      //     issued together): a quiescent unit (no infected animal, phi ==
      //     +0) has an empty day and, at the launch's start, only its record
      //     of Td - 1 to write; the others are listed
      const int m_prev = fin_prev ? a.rec[Td - 1 - a.t0] : -1;
      {
        UnitPos pos;
        pos.set(g0 + c0 + tid, Nn);
#pragma unroll 1
        for (int b0 = 0; b0 < cn; b0 += 4 * kSparseBlock) {
          int uu[4][C];
          double vv[4][NV > 0 ? NV : 1];
          int nday[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int i = b0 + k * kSparseBlock + tid;
            vv[k][0] = 0.0;
            nday[k] = -1;
#pragma unroll
            for (int p = 0; p < C; ++p) uu[k][p] = 0;
            if (i < cn) {
              const long long gid = g0 + c0 + i;
#pragma unroll
              for (int p = 0; p < C; ++p) uu[k][p] = a.u[gid * C + p];
#pragma unroll
              for (int q = 0; q < NV; ++q) vv[k][q] = a.v[gid * NV + q];
              if (has_e1) nday[k] = a.e1_next[gid];
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int i = b0 + k * kSparseBlock + tid;
            const bool in = i < cn;
            // a warp's 32 units of step k are one word of the bitmap
            const uint32_t bw = __ballot_sync(0xffffffffu, nday[k] == d);
            if (lane == 0) s_e1bits[(b0 + k * kSparseBlock) / 32 + warp] = bw;
            const bool q0 = in && quiet && quiescent<KIND>(uu[k], vv[k]);
            if (in && !q0) s_nq[atomicAdd(&s_nnq, 1)] = (uint16_t)i;
            if (m_prev >= 0) {
              if (q0) record_unit<C, NV>(a, Nn, m_prev, pos.rep, pos.node, uu[k], vv[k]);
              if (a.out.prev)
                prevalence_add<C>(a.out, in ? (long long)pos.rep * a.M + m_prev : -1, q0,
                                  uu[k]);
            }
            pos.advance(kSparseBlock, Nn);
          }
        }
      }
      __syncthreads();
      // 1b. the listed units: finish of Td - 1 (launch start only), rates;
      //     units with lambda > 0 go to the thread list, or, expecting
      //     heavy_after transitions or more, straight to a warp slot
      {
        const int nq = s_nnq;
#pragma unroll 1
        for (int li = tid; li < nq; li += kSparseBlock) {
          const int i = c0 + s_nq[li];  // block-relative
          const long long gid = g0 + i;
          const int rep = (int)(gid / Nn);
          const int node = (int)(gid - (long long)rep * Nn);
          int u[C];
          double v[NV > 0 ? NV : 1];
          v[0] = 0.0;
#pragma unroll
          for (int p = 0; p < C; ++p) u[p] = a.u[gid * C + p];
#pragma unroll
          for (int q = 0; q < NV; ++q) v[q] = a.v[gid * NV + q];
          int code = 0;
          if (fin_prev) {
            code = sparse_finish<KIND>(Td - 1, u, v, quiet, tb, a, rep, node, gid);
            if (a.out.prev && m_prev >= 0 && code == 0)
              prevalence_add_unit<C>(a.out, (long long)rep * a.M + m_prev, u);
          }
          if (code == 0 && !(quiet && quiescent<KIND>(u, v))) {
            ++rated;
            double kf[NK], w[T];
            M::prepare(v, tb.gdata, kf);
            bool bad = false;
#pragma unroll
            for (int j = 0; j < T; ++j) {
              w[j] = M::rate_k(j, u, kf, tb.gdata);
              bad = bad || bad_rate(w[j]);
            }
            double lam = w[0];
#pragma unroll
            for (int j = 1; j < T; ++j) lam = lam + w[j];
            if (bad) {
              report(a.err, SG_ERR_RATE, a.rep0 + rep, node, Td, -1);
            } else if (gt0(lam)) {
              atomicOr(&s_actbits[(i - c0) >> 5], 1u << ((i - c0) & 31));
              int slot = kSparseHeavy;
              if (!(lam < heavy_rate)) slot = atomicAdd(&s_nheavy, 1);
              if (slot < kSparseHeavy) {
                HeavySlot<C, NK> &hs = s_heavy[slot];
                hs.t = (double)(Td - 1);
#pragma unroll
                for (int q = 0; q < NK; ++q) hs.kf[q] = kf[q];
                hs.c = 0;
                hs.node = node;
                hs.rep = a.rep0 + rep;
                hs.code = i;  // the unit, until the warp reports
#pragma unroll
                for (int p = 0; p < C; ++p) hs.u[p] = u[p];
              } else if (lam < 2.0) {
                // the thread list: units expecting two transitions or more
                // from the front, the others from the back, so that the
                // longer chains start first
                s_act[kSparseChunk - 1 - atomicAdd(&s_nshort, 1)] = (uint16_t)(i - c0);
              } else {
                s_act[atomicAdd(&s_nact, 1)] = (uint16_t)(i - c0);
              }
            }
          }
        }
      }
      __syncthreads();
      const int n_long = s_nact;
      const int na = n_long + s_nshort;
      const int n_direct = min(s_nheavy, kSparseHeavy);
      const int list_warps = min(nwarps, (na + 63) >> 6);
      if (warp >= list_warps) {
        for (int h = warp - list_warps; h < n_direct; h += nwarps - list_warps) {
          HeavySlot<C, NK> &hs = s_heavy[h];
          const long long gid = g0 + hs.code;
          __syncwarp();
          ssa_warp<KIND>(hs, Tn, (uint32_t)Td, k0, k1, tb, fired, drawn);
          if (lane == 0) {
            if (hs.code) report(a.err, hs.code, hs.rep, hs.node, Td, -1);
#pragma unroll
            for (int p = 0; p < C; ++p) a.u[gid * C + p] = hs.u[p];
          }
          __syncwarp();
        }
      } else {
        const long long Tkey = order_key(Tn);
        bool busy = false, drained = false;
        long long gid = 0;
        int rep = 0, node = 0, nb = 0;
        uint32_t tag = 0, c = 0;
        int u[C];
        double kf[NK], w[T];
        double t = 0.0;
        // draw buffer shared by the warp: after a refill with k busy lanes,
        // the busy lane of rank r finds draw cb + j of its unit in lane
        // r + j k (j < nbuf = 32 / k); bufE / bufR are this lane's entry
        uint32_t cb = 0;
        int nbuf = 0, rank = 0, kref = 1;
        double bufE = 0.0, bufR = 0.0;
        double P[T];  // prefix sums of w (rate_prefix)
#pragma unroll
        for (int j = 0; j < T; ++j) P[j] = 0.0;
#pragma unroll
        for (int p = 0; p < C; ++p) u[p] = 0;
#pragma unroll
        for (int q = 0; q < NK; ++q) kf[q] = 0.0;
#pragma unroll
        for (int j = 0; j < T; ++j) w[j] = 0.0;
        for (;;) {
          if (!busy && !drained) {
            const int i = atomicAdd(&s_next, 1);
            if (i < na) {
              gid = g0 + c0 + s_act[i < n_long ? i : kSparseChunk - 1 - (i - n_long)];
              rep = (int)(gid / Nn);
              node = (int)(gid - (long long)rep * Nn);
              tag = (SG_STREAM_SSA << 24) | (uint32_t)(a.rep0 + rep);
              double v[NV > 0 ? NV : 1];
              v[0] = 0.0;
#pragma unroll
              for (int p = 0; p < C; ++p) u[p] = a.u[gid * C + p];
#pragma unroll
              for (int q = 0; q < NV; ++q) v[q] = a.v[gid * NV + q];
              M::prepare(v, tb.gdata, kf);
#pragma unroll
              for (int j = 0; j < T; ++j) w[j] = M::rate_k(j, u, kf, tb.gdata);
              rate_prefix<T>(w, P, 0);
              t = (double)(Td - 1);
              c = 0;
              nb = 0;
              nbuf = 0;
              busy = true;
            } else {
              drained = true;
            }
          }
          const unsigned bm = __ballot_sync(0xffffffffu, busy);
          if (bm == 0u) break;
          // a busy lane without its next draw buffered: every lane computes
          // one draw (Philox, uniforms, logarithm) for the busy lanes, the
          // draws c .. c + 32 / k - 1 of each, so that in the list's tail one
          // logarithm sequence of the warp serves several rounds
          if (__any_sync(0xffffffffu, busy && (nbuf == 0 || c - cb >= (uint32_t)nbuf))) {
            const int k = __popc(bm);
            const int per = 32 / k;
            const int ro = lane % k, jo = lane / k;
            // the busy lane of rank ro (the ro-th set bit of bm, by halving)
            uint32_t x = bm;
            int n = ro, owner = 0;
#pragma unroll
            for (int sft = 16; sft > 0; sft >>= 1) {
              const int cnt = __popc(x & ((1u << sft) - 1u));
              if (n >= cnt) {
                n -= cnt;
                x >>= sft;
                owner += sft;
              }
            }
            const uint32_t oc = __shfl_sync(0xffffffffu, c, owner);
            const uint32_t on = (uint32_t)__shfl_sync(0xffffffffu, node, owner);
            const uint32_t ot = __shfl_sync(0xffffffffu, tag, owner);
            if (jo < per) {
              const U4 xr = philox10(U4{oc + (uint32_t)jo, on, (uint32_t)Td, ot}, k0, k1);
              bufE = -log_pos(u01_open(xr.x, xr.y));
              bufR = u01_open(xr.z, xr.w);
            }
            kref = k;
            cb = c;
            nbuf = per;
            rank = __popc(bm & ((1u << lane) - 1u));
          }
          const int src = (rank + (int)(c - cb) * kref) & 31;
          const double E = __shfl_sync(0xffffffffu, bufE, src);
          const double R2 = __shfl_sync(0xffffffffu, bufR, src);
          if (!busy) continue;
          // one draw: ssa_step's operations and order, with the draw's
          // random numbers from the buffer and lambda and the inversion's
          // running sums from the kept prefix sums
          int r;
          {
            const double lam = P[T - 1];
            if (!gt0(lam)) {
              r = SSA_DONE;
            } else if (c >= SG_MAX_DRAWS) {
              r = SG_ERR_STEP_LIMIT;
            } else if (nb == a.heavy_after) {
              r = SSA_HEAVY;
            } else {
              ++c;
              const double tt = t + E / lam;
              if (order_key(tt) >= Tkey) {
                r = SSA_DONE;
              } else {
                t = tt;
                const int n = select_prefix<T>(w, P, lam * R2);
                const int rc = apply_transition<KIND>(u, w, n, kf, tb);
                rate_prefix<T>(w, P, __ffs(tb.dep[n]) - 1);
                ++fired;
                r = rc ? rc : SSA_STEP_FIRED;
              }
            }
          }
          if (r == SSA_STEP_FIRED) {
            ++nb;
            continue;
          }
          if (r == SSA_HEAVY) {
            const int slot = atomicAdd(&s_nheavy, 1);
            if (slot < kSparseHeavy) {
              HeavySlot<C, NK> &hs = s_heavy[slot];
              hs.t = t;
#pragma unroll
              for (int q = 0; q < NK; ++q) hs.kf[q] = kf[q];
              hs.c = c;
              hs.node = node;
              hs.rep = a.rep0 + rep;
              hs.code = (int32_t)(gid - g0);  // the unit, until the warp reports
#pragma unroll
              for (int p = 0; p < C; ++p) hs.u[p] = u[p];
              drawn += c;
              busy = false;
              continue;
            }
            // no slot left: this lane goes on with its unit (no hand-off)
            nb = -(1 << 30);
            continue;
          }
          // done or an error
          drawn += c;
          if (r < 0) report(a.err, r, a.rep0 + rep, node, Td, -1);
#pragma unroll
          for (int p = 0; p < C; ++p) a.u[gid * C + p] = u[p];
          busy = false;
        }
      }
      // a warp with no SSA work left applies the E1 events of day Td of the
      // chunk's units that take no draw today (1,024 units per take, their
      // units with events compacted onto the lanes); the units that take
      // draws come after the SSA (their events follow their day's
      // transitions)
      if (has_e1) sparse_e1_bits<C>(s_e1bits, s_actbits, false, &s_e1take, (cn + 31) >> 5,
                                    g0 + c0, Td, d, tb, a, k0, k1, applied);
      __syncthreads();
      // the warp slots not run yet: all of them when every warp had list
      // units, else those the thread list handed over
      const int h0 = list_warps < nwarps ? n_direct : 0;
      const int nh = min(s_nheavy, kSparseHeavy);
      for (int h = h0 + warp; h < nh; h += nwarps) {
        HeavySlot<C, NK> &hs = s_heavy[h];
        const long long gid = g0 + hs.code;  // the unit (ssa_warp sets the code)
        __syncwarp();
        ssa_warp<KIND>(hs, Tn, (uint32_t)Td, k0, k1, tb, fired, drawn);
        if (lane == 0) {
          if (hs.code) report(a.err, hs.code, hs.rep, hs.node, Td, -1);
#pragma unroll
          for (int p = 0; p < C; ++p) a.u[gid * C + p] = hs.u[p];
        }
        __syncwarp();
      }
      __syncthreads();
      // 3. E1 events of day Td of the units that took draws today
      if (has_e1) {
        sparse_e1_bits<C>(s_e1bits, s_actbits, true, &s_e1late, (cn + 31) >> 5, g0 + c0, Td,
                          d, tb, a, k0, k1, applied);
        __syncthreads();
      }
    }
    if (a.e2_inblock) {
      // this block's replicates' external transfers of Td (the wave plan of
      // day d; no other block touches their nodes)
      for (long long r = g0 / Nn; nub > 0 && r * Nn < g0 + nub; ++r) {
        const long long k = (long long)d * a.slots + (a.slots > 1 ? r : 0);
        const long long w0 = a.wave_off[k], w1 = a.wave_off[k + 1];
        if (w0 < w1) e2_rep_block<C>(tb, a, (int)r, Td, w0, w1);
      }
      // a failed transfer ends the run before the day's post time step
      if (tid == 0) s_stop = *(volatile int32_t *)&a.err->code != 0;
      __syncthreads();
      if (s_stop) break;
    }
    // then, unless deferred to the next day's first passes or the next
    // launch, the post time step and recording of Td for every unit
    const bool fin = a.e2_inblock ? Td + 1 == a.T_end && a.finish_last
                                  : Td + 1 < a.T_end || a.finish_last;
    if (fin) {
      // post time step and recording of Td: quiescent units are recorded
      // by a scan (four per thread per step), the others listed (chunks of
      // kSparseChunk units) and finished from the list
      const int m_fin = a.rec[Td - a.t0];
      for (int c0 = 0; c0 < nub; c0 += kSparseChunk) {
        const int cn = min(kSparseChunk, nub - c0);
        if (tid == 0) s_nnq = 0;
        __syncthreads();
        UnitPos pos;
        pos.set(g0 + c0 + tid, Nn);
#pragma unroll 1
        for (int b0 = 0; b0 < cn; b0 += 4 * kSparseBlock) {
          int uu[4][C];
          double vv[4][NV > 0 ? NV : 1];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int i = b0 + k * kSparseBlock + tid;
            vv[k][0] = 0.0;
#pragma unroll
            for (int p = 0; p < C; ++p) uu[k][p] = 0;
            if (i < cn) {
              const long long gid = g0 + c0 + i;
#pragma unroll
              for (int p = 0; p < C; ++p) uu[k][p] = a.u[gid * C + p];
#pragma unroll
              for (int q = 0; q < NV; ++q) vv[k][q] = a.v[gid * NV + q];
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int i = b0 + k * kSparseBlock + tid;
            const bool in = i < cn;
            const bool q0 = in && quiet && quiescent<KIND>(uu[k], vv[k]);
            if (in && !q0) s_nq[atomicAdd(&s_nnq, 1)] = (uint16_t)i;
            if (m_fin >= 0) {
              if (q0) record_unit<C, NV>(a, Nn, m_fin, pos.rep, pos.node, uu[k], vv[k]);
              if (a.out.prev)
                prevalence_add<C>(a.out, in ? (long long)pos.rep * a.M + m_fin : -1, q0,
                                  uu[k]);
            }
            pos.advance(kSparseBlock, Nn);
          }
        }
        __syncthreads();
        const int nq = s_nnq;
#pragma unroll 1
        for (int li = tid; li < nq; li += kSparseBlock) {
          const long long gid = g0 + c0 + s_nq[li];
          const int rep = (int)(gid / Nn);
          const int node = (int)(gid - (long long)rep * Nn);
          int u[C];
          double v[NV > 0 ? NV : 1];
          v[0] = 0.0;
#pragma unroll
          for (int p = 0; p < C; ++p) u[p] = a.u[gid * C + p];
#pragma unroll
          for (int q = 0; q < NV; ++q) v[q] = a.v[gid * NV + q];
          const int code = sparse_finish<KIND>(Td, u, v, quiet, tb, a, rep, node, gid);
          if (a.out.prev && m_fin >= 0 && code == 0)
            prevalence_add_unit<C>(a.out, (long long)rep * a.M + m_fin, u);
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
  if (a.e2_done) {
    // the last block to finish a replicate's units runs its external
    // transfers of T_end - 1 (counted per replicate, no block waits)
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    const long long g_hi = g0 + nub - 1;
    for (int r = (int)(g0 / Nn); nub > 0 && (long long)r * Nn <= g_hi; ++r) {
      if (tid == 0) {
        const long long b_first = (long long)r * Nn / a.npb;
        const long long b_last = ((long long)(r + 1) * Nn - 1) / a.npb;
        const int old = atomicAdd(&a.e2_done[r], 1);
        s_last = old == (int)(b_last - b_first);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        long long w0 = a.e2_wb, w1 = a.e2_we;
        if (a.slots > 1) {
          w0 = a.wave_off[(long long)a.e2_day_index * a.slots + r];
          w1 = a.wave_off[(long long)a.e2_day_index * a.slots + r + 1];
        }
        e2_rep_block<C>(tb, a, r, a.T_end - 1, w0, w1);
        if (tid == 0) a.e2_done[r] = 0;
      }
      __syncthreads();
    }
  }
  // one atomic per warp for the counters
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fired += __shfl_down_sync(0xffffffffu, fired, off);
    drawn += __shfl_down_sync(0xffffffffu, drawn, off);
    applied += __shfl_down_sync(0xffffffffu, applied, off);
    rated += __shfl_down_sync(0xffffffffu, rated, off);
  }
  if ((tid & 31) == 0) {
    if (drawn | fired) {
      atomicAdd(&a.cnt->reactions, fired);
      atomicAdd(&a.cnt->draws, drawn);
    }
    if (applied) atomicAdd(&a.cnt->events, applied);
    if (rated) atomicAdd(&a.cnt->rated, rated);
  }
}

// Day index of each unit's first E1 event (or 0x7fffffff), the sparse
// schedule's per-unit test for "events today" (its E1 cursors start at 0).
__global__ void k_e1_next_init(const int64_t *__restrict__ e1_node_off,
                               const int32_t *__restrict__ e1_day, int Nn, int n_rep,
                               int slots, int32_t *e1_next) {
  const long long total = (long long)Nn * n_rep;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int rep = (int)(g / Nn), node = (int)(g - (long long)rep * Nn);
    const long long key = (long long)(slots > 1 ? rep : 0) * Nn + node;
    const long long b = e1_node_off[key], e = e1_node_off[key + 1];
    e1_next[g] = b < e ? e1_day[b] : 0x7fffffff;
  }
}

struct EvArgs {
  EvDev ev;
  int *u;
  int32_t n_rep;
  int32_t rep0;  // global index of local replicate 0 (streams, error reports)
  uint32_t k0, k1;
  int32_t day;  // unit time point T the events run at
  SgDevError *err;
  SgCounters *cnt;
};

// Block-wide copy of n 32-bit words with 16-byte accesses where both ends
// are aligned, several loads in flight per thread.
__device__ __forceinline__ void copy_words(int *dst, const int *src, int n) {
  int head = 0;
  if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    const int n4 = n >> 2;
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
#pragma unroll 4
    for (int i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = s4[i];
    head = n4 << 2;
  }
#pragma unroll 4
  for (int i = head + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

constexpr int kE2Cap = 512;      // events staged in shared memory per chunk
constexpr int kE2WaveCap = 128;  // wave bounds staged per chunk

// E2 events of one day: block r runs replicate r's external transfers
// (Sec. 3.3) wave by wave, with a block barrier between waves.  The block
// first stages a chunk of events in shared memory together with the first
// Philox block of each event's random stream (which does not depend on the
// state); with SMEM_STATE the replicate's whole node state is also held in
// shared memory for the day.  Several transfers of one wave may share a
// destination, so additions are atomic; a wave never samples a node that
// another event of the wave touches.
template <int KIND, bool SMEM_STATE>
__global__ void __launch_bounds__(kE2Block)
k_events_e2(const SgTables tb, const EvArgs a, const int64_t *__restrict__ wave_ev,
            long long w_begin_shared, long long w_end_shared,
            const int64_t *__restrict__ wave_off, int day_index, int slots) {
  constexpr int C = ModelTraits<KIND>::C;
  extern __shared__ __align__(16) int s_state[];
  __shared__ int32_t s_node[kE2Cap], s_dest[kE2Cap], s_n[kE2Cap];
  __shared__ uint8_t s_sel[kE2Cap];
  __shared__ int8_t s_shift[kE2Cap];
  __shared__ long long s_idx[kE2Cap];
  __shared__ double s_prop[kE2Cap];
  __shared__ uint4 s_w[kE2Cap];
  __shared__ long long s_wave[kE2WaveCap + 1];
  __shared__ int16_t s_hv[kE2Cap];  // the wave's events left to the warps
  __shared__ int s_nhv;
  pdl_trigger();
  const int rep = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) s_nhv = 0;
  const int Nn = tb.n_nodes;
  long long w0 = w_begin_shared, w1 = w_end_shared;
  if (slots > 1) {
    w0 = wave_off[(long long)day_index * slots + rep];
    w1 = wave_off[(long long)day_index * slots + rep + 1];
  }
  if (w0 >= w1) {
    pdl_wait();
    return;
  }
  int *gstate = a.u + (long long)rep * Nn * C;
  int *state = SMEM_STATE ? s_state : gstate;
  bool waited = false;
  // `bad`: this thread met an error; `stop`: the block's verdict, taken at a
  // barrier (__syncthreads_or), so every thread leaves the loops together
  bool bad = false, stop = false;
  const uint64_t seed = ((uint64_t)a.k1 << 32) | a.k0;
  const uint32_t tag = (SG_STREAM_EVENTS << 24) | (uint32_t)(a.rep0 + rep);
  unsigned long long applied = 0;
  long long w = w0;
  long long pos = wave_ev[w0];
  const long long pos_end = wave_ev[w1];
  while (pos < pos_end) {
    // stage the bounds of the next waves, then the events [pos, pend) they
    // hold (at most kE2Cap; a wave may continue into the next chunk)
    const long long wn = min(w1 - w, (long long)kE2WaveCap);
    __syncthreads();
    for (long long i = threadIdx.x; i <= wn; i += blockDim.x) s_wave[i] = wave_ev[w + i];
    __syncthreads();
    const long long pend = min(pos + (long long)kE2Cap, s_wave[wn]);
    for (long long i = threadIdx.x; i < pend - pos; i += blockDim.x) {
      const long long j = pos + i;
      s_node[i] = a.ev.node[j];
      s_dest[i] = a.ev.dest[j];
      s_n[i] = a.ev.n[j];
      s_sel[i] = a.ev.select[j];
      s_shift[i] = a.ev.shift[j];
      s_prop[i] = a.ev.proportion[j];
      const long long idx = a.ev.index[j];
      s_idx[i] = idx;
      const U4 f = philox10(U4{0u, (uint32_t)(unsigned long long)idx,
                               (uint32_t)((unsigned long long)idx >> 32), tag},
                            a.k0, a.k1);
      s_w[i] = make_uint4(f.x, f.y, f.z, f.w);
    }
    if (!waited) {
      // the first chunk is staged: now wait for the day kernel's state
      pdl_wait();
      waited = true;
      if (threadIdx.x == 0 && *(volatile int32_t *)&a.err->code != 0) bad = true;
      if (SMEM_STATE) copy_words(s_state, gstate, Nn * C);
    }
    stop = __syncthreads_or(bad);
    if (stop) break;
    // waves w .. (staged) intersecting [pos, pend)
    long long wi = 0;
    while (wi < wn && s_wave[wi] < pend) {
      const long long lo = max(pos, s_wave[wi]), hi = min(pend, s_wave[wi + 1]);
      for (long long q = lo + threadIdx.x; q < hi; q += blockDim.x) {
        const int i = (int)(q - pos);
        const int src = s_node[i];
        int *un = state + (long long)src * C;
        const uint32_t mask = tb.Emask[s_sel[i]];
        int cur[C];
        long long total = 0;
#pragma unroll
        for (int p = 0; p < C; ++p) {
          cur[p] = un[p];
          if ((mask >> p) & 1u) total += cur[p];
        }
        const long long k = s_n[i] > 0 ? (long long)s_n[i]
                                       : (long long)round(s_prop[i] * (double)total);
        if (k < 0 || k > total) {
          report(a.err, SG_ERR_EVENT_UNDERFLOW, a.rep0 + rep, src, a.day, s_idx[i]);
          bad = true;
          continue;
        }
        if (k >= kUrnWarp) {
          // a large transfer: sampled by a warp after this pass
          s_hv[atomicAdd(&s_nhv, 1)] = (int16_t)i;
          continue;
        }
        int moved[C];
#pragma unroll
        for (int p = 0; p < C; ++p) moved[p] = 0;
        if (k > 0) {
          WordStream ws;
          const uint4 f = s_w[i];
          ws.init_with_first(seed, s_idx[i], a.rep0 + rep, U4{f.x, f.y, f.z, f.w});
          for (long long d = 0; d < k; ++d) {
            uint32_t x = ws.below((uint32_t)(total - d));
            bool taken = false;
#pragma unroll
            for (int p = 0; p < C; ++p) {
              if (taken || !((mask >> p) & 1u)) continue;
              const uint32_t rem = (uint32_t)(cur[p] - moved[p]);
              if (x < rem) {
                ++moved[p];
                taken = true;
              } else {
                x -= rem;
              }
            }
          }
        }
        const int q_sh = s_shift[i];
        int *ud = state + (long long)s_dest[i] * C;
#pragma unroll
        for (int p = 0; p < C; ++p) {
          if (moved[p] == 0) continue;
          un[p] = cur[p] - moved[p];
        }
#pragma unroll
        for (int p = 0; p < C; ++p) {
          if (moved[p] == 0) continue;
          atomicAdd(ud + (q_sh >= 0 ? p + tb.Nsh[q_sh][p] : p), moved[p]);
        }
        ++applied;
      }
      stop = __syncthreads_or(bad);
      if (stop) break;
      const int nhv = s_nhv;  // the same in every thread (read after the barrier)
      if (nhv > 0) {
        __syncthreads();  // every thread has read the count
        if (threadIdx.x == 0) s_nhv = 0;
        // the wave's large transfers, one warp each: no other event of the
        // wave touches their source nodes, so the order does not matter
        for (int h = warp; h < nhv; h += nwarps) {
          const int i = s_hv[h];
          const int src = s_node[i];
          int *un = state + (long long)src * C;
          const uint32_t mask = tb.Emask[s_sel[i]];
          int cur[C];
          long long total = 0;
#pragma unroll
          for (int p = 0; p < C; ++p) {
            cur[p] = un[p];
            if ((mask >> p) & 1u) total += cur[p];
          }
          const long long k = s_n[i] > 0 ? (long long)s_n[i]
                                         : (long long)round(s_prop[i] * (double)total);
          int moved[C];
          urn_warp<C>(cur, mask, (uint32_t)k, (uint32_t)total, seed, s_idx[i], a.rep0 + rep,
                      moved);
          if (lane == 0) {
            const int q_sh = s_shift[i];
            int *ud = state + (long long)s_dest[i] * C;
#pragma unroll
            for (int p = 0; p < C; ++p)
              if (moved[p] != 0) un[p] = cur[p] - moved[p];
#pragma unroll
            for (int p = 0; p < C; ++p)
              if (moved[p] != 0) atomicAdd(ud + (q_sh >= 0 ? p + tb.Nsh[q_sh][p] : p), moved[p]);
            ++applied;
          }
          __syncwarp();
        }
        __syncthreads();
      }
      if (s_wave[wi + 1] <= pend) ++wi;
      else break;  // the wave continues in the next chunk
    }
    if (stop) break;
    w += wi;
    pos = pend;
  }
  if (!waited) pdl_wait();
  if (SMEM_STATE && waited) {
    __syncthreads();
    copy_words(gstate, s_state, Nn * C);
  }
  if (applied) atomicAdd(&a.cnt->events, applied);
}

// U_sparse / V_sparse entries and prevalence counters of tspan slot 0 (the
// initial state), one thread per (replicate, node).
template <int C, int NV>
__global__ void k_record0(const int32_t *__restrict__ u0, const double *__restrict__ v0, int Nn,
                          int n_rep, int M, const OutDev o) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in_range = gid < (long long)Nn * n_rep;
  int u[C];
  double v[NV > 0 ? NV : 1];
#pragma unroll
  for (int p = 0; p < C; ++p) u[p] = 0;
  v[0] = 0.0;
  int rep = 0;
  if (in_range) {
    rep = (int)(gid / Nn);
    const int node = (int)(gid - (long long)rep * Nn);
#pragma unroll
    for (int p = 0; p < C; ++p) u[p] = u0[gid * C + p];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = v0[gid * NV + q];
    record_sparse<C, NV>(o, 0, rep, node, u, v);
  }
  if (o.prev) prevalence_add<C>(o, in_range ? (long long)rep * M : -1, in_range, u);
}

}  // namespace sg
