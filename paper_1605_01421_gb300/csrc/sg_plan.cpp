// sg_plan.cpp -- host-side validation and scheduling of the scheduled events
// (Sec. 3.3, Appendix A "Process E1 events" / "Process E2 events").
#include "sg_plan.h"

#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <numeric>
#include <thread>

namespace sg {

// Checks of events lo .. hi - 1; the first offending one in *bad (-1: none).
static int validate_range(const SgTables &tb, const EventTable &ev, int64_t lo, int64_t hi,
                          int64_t *bad) {
  for (int64_t e = lo; e < hi; ++e) {
    const int type = ev.type[e], s = ev.select[e], q = ev.shift[e];
    bool ok = type >= SG_EXIT && type <= SG_EXTERNAL_TRANSFER;
    ok = ok && ev.node[e] >= 0 && ev.node[e] < tb.n_nodes;
    if (type == SG_EXTERNAL_TRANSFER)
      ok = ok && ev.dest[e] >= 0 && ev.dest[e] < tb.n_nodes;
    ok = ok && s >= 0 && s < tb.n_select;
    ok = ok && ev.n[e] >= 0;
    ok = ok && ev.proportion[e] >= 0.0 && ev.proportion[e] <= 1.0;
    // Reading: an internal transfer without a shift column is an error.
    if (type == SG_INTERNAL_TRANSFER) ok = ok && q >= 0;
    if (type != SG_ENTER) ok = ok && q < tb.n_shift;
    if (ev.per_rep) ok = ok && ev.rep[e] >= 0;
    if (ok && type == SG_ENTER) ok = tb.Emask[s] != 0;
    if (!ok) {
      *bad = e;
      return SG_ERR_ARG;
    }
    // a shift must keep every selectable compartment inside the node
    if (q >= 0 && (type == SG_INTERNAL_TRANSFER || type == SG_EXTERNAL_TRANSFER)) {
      for (int p = 0; p < tb.n_comp; ++p) {
        if (!((tb.Emask[s] >> p) & 1u)) continue;
        const int to = p + tb.Nsh[q][p];
        if (to < 0 || to >= tb.n_comp) {
          *bad = e;
          return SG_ERR_SHIFT_RANGE;
        }
      }
    }
  }
  *bad = -1;
  return SG_OK;
}

// Threads for a host pass over `work` items (one below 16,384 items).
static int plan_threads(int64_t work) {
  if (work < 16384) return 1;
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hc ? hc : 1u, 8u));
}

// Worker threads kept for the life of the process (created on first use,
// again after a fork): run(T, f) runs f(t) for t = 0 .. T - 1, the caller
// taking t = 0, and returns when every f(t) has returned.  One parallel
// region at a time.
class PlanPool {
 public:
  static PlanPool &get() {
    static PlanPool *pool = new PlanPool();  // never destroyed: workers are detached
    return *pool;
  }
  void run(int T, const std::function<void(int)> &f) {
    if (T <= 1) {
      f(0);
      return;
    }
    std::lock_guard<std::mutex> region(region_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (pid_ != getpid()) {  // a forked child has none of the parent's workers
        workers_ = 0;
        pid_ = getpid();
      }
      while (workers_ < T - 1) {
        const int id = ++workers_;
        std::thread([this, id] { loop(id); }).detach();
      }
      job_ = &f;
      active_ = T - 1;
      remaining_ = T - 1;
      ++gen_;
    }
    cv_.notify_all();
    f(0);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return remaining_ == 0; });
    job_ = nullptr;
  }

 private:
  void loop(int id) {
    const pid_t mine = getpid();
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(int)> *job = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        if (pid_ != mine || id > active_) continue;
        job = job_;
      }
      (*job)(id);
      std::lock_guard<std::mutex> lk(mu_);
      if (--remaining_ == 0) done_.notify_one();
    }
  }
  std::mutex region_mu_, mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)> *job_ = nullptr;
  int workers_ = 0, active_ = 0, remaining_ = 0;
  uint64_t gen_ = 0;
  pid_t pid_ = getpid();
};

template <class F>
static void run_threads(int T, F &&f) {
  const std::function<void(int)> fn = [&f](int t) { f(t); };
  PlanPool::get().run(T, fn);
}

// Split [0, nk) into T ranges of about equal weight, weight given by the
// prefix sums off[0 .. nk]; bounds[t] .. bounds[t + 1] is range t.
static std::vector<int64_t> weighted_ranges(const std::vector<int64_t> &off, int64_t nk, int T) {
  std::vector<int64_t> bounds(T + 1, nk);
  bounds[0] = 0;
  const int64_t total = off[nk];
  for (int t = 1; t < T; ++t) {
    const int64_t target = total * t / T;
    bounds[t] = std::lower_bound(off.begin(), off.begin() + nk + 1, target) - off.begin();
    bounds[t] = std::max(bounds[t - 1], std::min(bounds[t], nk));
  }
  return bounds;
}

int build_plan(const EventTable &ev, int32_t n_nodes, int32_t t0, int32_t t_end,
               int32_t slots, Plan *out, int32_t rep_lo, bool shard) {
  Plan &P = *out;
  P = Plan();
  P.t0 = t0;
  P.t_end = t_end;
  P.slots = slots;
  P.rep_lo = rep_lo;
  P.shard = shard;
  P.n_nodes = n_nodes;
  P.days = std::max(0, t_end - t0);
  const int64_t nb = (int64_t)P.days * slots;
  const int64_t nk = (int64_t)slots * n_nodes;
  P.e1_node_off.assign(nk + 1, 0);
  P.e2_wave_off.assign(nb + 1, 0);
  P.day_has_e2.assign(P.days, 0);
  P.wave_ev.assign(1, 0);
  if (P.days == 0) return SG_OK;

  // Events after t_end never run; events dated t0 or earlier run at the
  // first step.
  const int64_t n = ev.size();
  auto day_of = [&](int64_t e) {
    return (int32_t)std::max<int64_t>(0, (int64_t)ev.time[e] - t0 - 1);
  };
  // a shard plans the replicates rep_lo .. rep_lo + slots - 1 of a
  // per-replicate table (slot = replicate - rep_lo; the other replicates'
  // events are left out); otherwise slot = replicate when slots > 1
  auto slot_of = [&](int64_t e) -> int64_t {
    if (shard) return (int64_t)ev.rep[e] - rep_lo;
    return slots > 1 ? ev.rep[e] : 0;
  };

  // 1. E1 events bucketed by (slot, node), E2 events by (day, slot), both
  //    stable (list order kept inside a bucket): counts, offsets, scatter.
  //    With several threads each takes a chunk of the list and its own
  //    counts, so that its events land after those of the chunks before it.
  const int T = plan_threads(n);
  const bool par = T > 1 && n < ((int64_t)1 << 31) &&
                   (int64_t)T * (nk + nb) <= std::max<int64_t>(n, (int64_t)1 << 20);
  const int TB = par ? T : 1;
  std::vector<std::vector<int32_t>> c1(TB), c2(TB);
  std::vector<int> bad(TB, 0);
  run_threads(TB, [&](int t) {
    c1[t].assign(nk, 0);
    c2[t].assign(nb, 0);
    const int64_t lo = n * t / TB, hi = n * (t + 1) / TB;
    for (int64_t e = lo; e < hi; ++e) {
      if (ev.time[e] > t_end) continue;
      const int64_t s = slot_of(e);
      if (s < 0 || s >= slots) {
        if (!shard) bad[t] = 1;
        continue;
      }
      if (ev.type[e] == SG_EXTERNAL_TRANSFER)
        ++c2[t][(int64_t)day_of(e) * slots + s];
      else
        ++c1[t][s * n_nodes + ev.node[e]];
    }
  });
  for (int t = 0; t < TB; ++t)
    if (bad[t]) return SG_ERR_ARG;
  std::vector<int64_t> e1_count(nk + 1, 0), e2_count(nb + 1, 0);
  for (int t = 0; t < TB; ++t) {
    for (int64_t k = 0; k < nk; ++k) e1_count[k + 1] += c1[t][k];
    for (int64_t b = 0; b < nb; ++b) e2_count[b + 1] += c2[t][b];
  }
  std::partial_sum(e1_count.begin(), e1_count.end(), e1_count.begin());
  std::partial_sum(e2_count.begin(), e2_count.end(), e2_count.begin());
  const int64_t n_e1 = e1_count[nk], n_e2 = e2_count[nb];
  // each thread's first position in each bucket
  run_threads(TB, [&](int t) {
    const int64_t k0 = nk * t / TB, k1 = nk * (t + 1) / TB;
    for (int64_t k = k0; k < k1; ++k) {
      int64_t run = e1_count[k];
      for (int u = 0; u < TB; ++u) {
        const int32_t x = c1[u][k];
        c1[u][k] = (int32_t)run;
        run += x;
      }
    }
    const int64_t b0 = nb * t / TB, b1 = nb * (t + 1) / TB;
    for (int64_t b = b0; b < b1; ++b) {
      int64_t run = e2_count[b];
      for (int u = 0; u < TB; ++u) {
        const int32_t x = c2[u][b];
        c2[u][b] = (int32_t)run;
        run += x;
      }
    }
  });
  P.order.resize(n_e1 + n_e2);
  int64_t *e1 = P.order.data(), *e2 = P.order.data() + n_e1;
  // E1 events travel with their sort keys: (day, time on day 0, type)
  struct Rec1 {
    int64_t e;
    int32_t day, time0, type;  // time0: the time on day 0, else 0
  };
  std::unique_ptr<Rec1[]> rec1(new Rec1[n_e1 > 0 ? n_e1 : 1]);  // left unset: all written below
  run_threads(TB, [&](int t) {
    std::vector<int32_t> &f1 = c1[t], &f2 = c2[t];
    const int64_t lo = n * t / TB, hi = n * (t + 1) / TB;
    for (int64_t e = lo; e < hi; ++e) {
      const int32_t time = ev.time[e];
      if (time > t_end) continue;
      const int64_t s = slot_of(e);
      if (s < 0 || s >= slots) continue;  // another shard's replicate
      const int32_t day = day_of(e);
      if (ev.type[e] == SG_EXTERNAL_TRANSFER)
        e2[f2[(int64_t)day * slots + s]++] = e;
      else
        rec1[f1[s * n_nodes + ev.node[e]]++] = Rec1{e, day, day == 0 ? time : 0,
                                                    ev.type[e]};
    }
  });
  c1.clear();
  c2.clear();
  P.e1_day.resize(n_e1);

  // 2. In parallel over ranges of (slot, node) lists and of (day, slot)
  //    buckets:
  //    E1: each list ordered by (day, time on day 0, type, list index) --
  //    every event of a day d >= 1 has time t0 + 1 + d, day 0 also holds the
  //    earlier times;
  //    E2: the first day's buckets ordered by time (stable), then waves, and
  //    the bucket ordered by wave (stable).
  const std::vector<int64_t> r1 = weighted_ranges(e1_count, nk, T);
  const std::vector<int64_t> r2 = weighted_ranges(e2_count, nb, T);
  std::vector<std::vector<int64_t>> wave_ends(T);  // per thread: wave ends, bucket by bucket
  std::vector<int32_t> n_waves_of(nb, 0);
  run_threads(T, [&](int t) {
    // sort keys of a list: (day, time on day 0, type, position in the list)
    struct Key {
      int32_t day, time, type, pos;
      bool operator<(const Key &o) const {
        if (day != o.day) return day < o.day;
        if (time != o.time) return time < o.time;
        if (type != o.type) return type < o.type;
        return pos < o.pos;
      }
    };
    std::vector<Key> keys;
    for (int64_t k = r1[t]; k < r1[t + 1]; ++k) {
      const int64_t lo = e1_count[k];
      const int32_t m = (int32_t)(e1_count[k + 1] - lo);
      const Rec1 *rc = rec1.get() + lo;
      keys.resize(m);
      bool sorted = true;
      for (int32_t i = 0; i < m; ++i) {
        keys[i] = Key{rc[i].day, rc[i].time0, rc[i].type, i};
        if (i > 0 && keys[i] < keys[i - 1]) sorted = false;
      }
      if (!sorted) std::sort(keys.begin(), keys.end());
      for (int32_t i = 0; i < m; ++i) {
        e1[lo + i] = rc[keys[i].pos].e;
        P.e1_day[lo + i] = keys[i].day;
      }
    }
    std::vector<int32_t> last_sample(n_nodes, 0), last_add(n_nodes, 0);
    std::vector<int64_t> stamp(n_nodes, -1);
    std::vector<int32_t> wave_of;
    std::vector<int64_t> wc, tmp;
    std::vector<int64_t> &ends = wave_ends[t];
    for (int64_t b = r2[t]; b < r2[t + 1]; ++b) {
      int64_t *lo = e2 + e2_count[b], *hi = e2 + e2_count[b + 1];
      const size_t m = (size_t)(hi - lo);
      if (m == 0) continue;
      if (b < slots)
        std::stable_sort(lo, hi, [&](int64_t a, int64_t c) { return ev.time[a] < ev.time[c]; });
      wave_of.assign(m, 0);
      int32_t n_w = 0;
      for (size_t i = 0; i < m; ++i) {
        const int64_t e = lo[i];
        const int32_t s = ev.node[e], d = ev.dest[e];
        if (stamp[s] != b) { stamp[s] = b; last_sample[s] = 0; last_add[s] = 0; }
        if (stamp[d] != b) { stamp[d] = b; last_sample[d] = 0; last_add[d] = 0; }
        const int32_t w = std::max(std::max(last_sample[s], last_add[s]), last_sample[d]) + 1;
        last_sample[s] = w;
        last_add[d] = std::max(last_add[d], w);
        wave_of[i] = w;
        n_w = std::max(n_w, w);
      }
      // counting sort by wave, list order kept inside a wave
      wc.assign((size_t)n_w + 2, 0);
      for (size_t i = 0; i < m; ++i) ++wc[wave_of[i] + 1];
      std::partial_sum(wc.begin(), wc.end(), wc.begin());
      tmp.assign(lo, hi);
      for (size_t i = 0; i < m; ++i) lo[wc[wave_of[i]]++] = tmp[i];
      // wc[w] is now the end of wave w
      for (int32_t w = 1; w <= n_w; ++w) ends.push_back(wc[w]);
      n_waves_of[b] = n_w;
    }
  });

  // 3. Wave offsets, in bucket order (positions in order, past the E1 part).
  P.wave_ev[0] = n_e1;
  std::vector<size_t> pos(T, 0);
  int t = 0;
  for (int64_t b = 0; b < nb; ++b) {
    while (t + 1 < T && b >= r2[t + 1]) ++t;
    const int32_t n_w = n_waves_of[b];
    for (int32_t w = 0; w < n_w; ++w)
      P.wave_ev.push_back(n_e1 + e2_count[b] + wave_ends[t][pos[t]++]);
    P.e2_wave_off[b + 1] = (int64_t)P.wave_ev.size() - 1;
    if (e2_count[b + 1] > e2_count[b]) P.day_has_e2[b / slots] = 1;
    P.max_waves_per_day = std::max(P.max_waves_per_day, n_w);
  }
  P.e1_node_off = e1_count;
  P.n_e1 = n_e1;
  P.n_e2 = n_e2;
  P.n_waves = (int64_t)P.wave_ev.size() - 1;
  return SG_OK;
}

void gather_events(const EventTable &ev, const Plan &P, int8_t *type, int8_t *shift,
                   uint8_t *select, int32_t *node, int32_t *dest, int32_t *n, double *proportion,
                   int64_t *index) {
  const int64_t m = (int64_t)P.order.size();
  const int T = plan_threads(m);
  run_threads(T, [&](int t) {
    const int64_t lo = m * t / T, hi = m * (t + 1) / T;
    for (int64_t i = lo; i < hi; ++i) {
      const int64_t e = P.order[i];
      type[i] = (int8_t)ev.type[e];
      shift[i] = (int8_t)(ev.shift[e] < 0 ? -1 : ev.shift[e]);
      select[i] = (uint8_t)ev.select[e];
      node[i] = ev.node[e];
      dest[i] = ev.dest[e];
      n[i] = ev.n[e];
      proportion[i] = ev.proportion[e];
      index[i] = e;
    }
  });
}

int validate_events(const SgTables &tb, const EventTable &ev, int64_t *bad) {
  const int64_t n = ev.size();
  const int T = plan_threads(n);
  std::vector<int> rc(T, SG_OK);
  std::vector<int64_t> first(T, -1);
  run_threads(T, [&](int t) {
    rc[t] = validate_range(tb, ev, n * t / T, n * (t + 1) / T, &first[t]);
  });
  // the first offending event of the list: in the first slice that has one
  for (int t = 0; t < T; ++t)
    if (rc[t]) {
      *bad = first[t];
      return rc[t];
    }
  *bad = -1;
  return SG_OK;
}

void copy_events(EventTable *out, int64_t n, const int32_t *type, const int32_t *time,
                 const int32_t *node, const int32_t *dest, const int32_t *cnt,
                 const double *proportion, const int32_t *select, const int32_t *shift,
                 const int32_t *rep) {
  EventTable &ev = *out;
  plan_vector<int32_t> *cols[8] = {&ev.type, &ev.time, &ev.node, &ev.dest,
                                   &ev.n,    &ev.select, &ev.shift, &ev.rep};
  const int32_t *src[8] = {type, time, node, dest, cnt, select, shift, rep};
  for (int c = 0; c < 8; ++c) cols[c]->resize(src[c] ? (size_t)n : 0);
  ev.proportion.resize((size_t)n);
  ev.per_rep = rep != nullptr;
  const int T = plan_threads(n);
  std::vector<int32_t> max_rep(T, -1);
  run_threads(T, [&](int t) {
    const int64_t lo = n * t / T, hi = n * (t + 1) / T;
    for (int c = 0; c < 8; ++c)
      if (src[c] && hi > lo) std::copy(src[c] + lo, src[c] + hi, cols[c]->data() + lo);
    if (hi > lo) std::copy(proportion + lo, proportion + hi, ev.proportion.data() + lo);
    if (rep)
      for (int64_t e = lo; e < hi; ++e) max_rep[t] = std::max(max_rep[t], rep[e]);
  });
  ev.max_rep = -1;
  for (int t = 0; t < T; ++t) ev.max_rep = std::max(ev.max_rep, max_rep[t]);
}

}  // namespace sg

extern "C" int sg_plan_events(int64_t n_events, const int32_t *type, const int32_t *time,
                              const int32_t *node, const int32_t *dest, const int32_t *rep,
                              int32_t n_nodes, int32_t t0, int32_t t_end, int32_t slots,
                              int64_t *counts, int64_t *order, int32_t *e1_day,
                              int64_t *e1_node_off, int64_t *e2_wave_off, int64_t *wave_ev) {
  if (n_events < 0 || n_nodes < 0 || slots < 1 || t_end < t0 || !counts ||
      (n_events > 0 && (!type || !time || !node || !dest)) || (slots > 1 && !rep))
    return SG_ERR_ARG;
  sg::EventTable ev;
  ev.type.assign(type, type + n_events);
  ev.time.assign(time, time + n_events);
  ev.node.assign(node, node + n_events);
  ev.dest.assign(dest, dest + n_events);
  ev.per_rep = slots > 1;
  if (ev.per_rep) ev.rep.assign(rep, rep + n_events);
  for (int64_t e = 0; e < n_events; ++e) {
    const bool e2 = type[e] == SG_EXTERNAL_TRANSFER;
    if (type[e] < SG_EXIT || type[e] > SG_EXTERNAL_TRANSFER || node[e] < 0 ||
        node[e] >= n_nodes || (e2 && (dest[e] < 0 || dest[e] >= n_nodes)) ||
        (ev.per_rep && (rep[e] < 0 || rep[e] >= slots)))
      return SG_ERR_ARG;
  }
  sg::Plan P;
  const int rc = sg::build_plan(ev, n_nodes, t0, t_end, slots, &P);
  if (rc) return rc;
  counts[0] = P.n_e1;
  counts[1] = P.n_e2;
  counts[2] = P.n_waves;
  if (!order) return SG_OK;
  if ((P.n_e1 > 0 && !e1_day) || !e1_node_off || !e2_wave_off || !wave_ev) return SG_ERR_ARG;
  std::copy(P.order.begin(), P.order.end(), order);
  std::copy(P.e1_day.begin(), P.e1_day.end(), e1_day);
  std::copy(P.e1_node_off.begin(), P.e1_node_off.end(), e1_node_off);
  std::copy(P.e2_wave_off.begin(), P.e2_wave_off.end(), e2_wave_off);
  std::copy(P.wave_ev.begin(), P.wave_ev.end(), wave_ev);
  return SG_OK;
}
