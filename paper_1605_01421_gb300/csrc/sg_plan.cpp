// sg_plan.cpp -- host-side validation and scheduling of the scheduled events
// (Sec. 3.3, Appendix A "Process E1 events" / "Process E2 events").
#include "sg_plan.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>

namespace sg {

int validate_events(const SgTables &tb, const EventTable &ev, int64_t *bad) {
  const int64_t n = ev.size();
  for (int64_t e = 0; e < n; ++e) {
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

// f(t) for t = 0 .. T - 1, on T threads (the caller is thread 0).
template <class F>
static void run_threads(int T, F &&f) {
  std::vector<std::thread> th;
  th.reserve(T > 1 ? T - 1 : 0);
  for (int t = 1; t < T; ++t) th.emplace_back([&f, t] { f(t); });
  f(0);
  for (auto &x : th) x.join();
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
               int32_t slots, Plan *out) {
  Plan &P = *out;
  P = Plan();
  P.t0 = t0;
  P.t_end = t_end;
  P.slots = slots;
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
  auto slot_of = [&](int64_t e) -> int64_t { return slots > 1 ? ev.rep[e] : 0; };

  // 1. One pass in list order: E1 events bucketed by (slot, node), E2 events
  //    by (day, slot); both stable, so list order is kept inside a bucket.
  std::vector<int64_t> e1_count(nk + 1, 0), e2_count(nb + 1, 0);
  for (int64_t e = 0; e < n; ++e) {
    if (ev.time[e] > t_end) continue;
    const int64_t s = slot_of(e);
    if (s >= slots) return SG_ERR_ARG;
    if (ev.type[e] == SG_EXTERNAL_TRANSFER)
      ++e2_count[(int64_t)day_of(e) * slots + s + 1];
    else
      ++e1_count[s * n_nodes + ev.node[e] + 1];
  }
  std::partial_sum(e1_count.begin(), e1_count.end(), e1_count.begin());
  std::partial_sum(e2_count.begin(), e2_count.end(), e2_count.begin());
  const int64_t n_e1 = e1_count[nk], n_e2 = e2_count[nb];
  P.order.resize(n_e1 + n_e2);
  int64_t *e1 = P.order.data(), *e2 = P.order.data() + n_e1;
  {
    std::vector<int64_t> f1(e1_count.begin(), e1_count.end() - 1);
    std::vector<int64_t> f2(e2_count.begin(), e2_count.end() - 1);
    for (int64_t e = 0; e < n; ++e) {
      if (ev.time[e] > t_end) continue;
      if (ev.type[e] == SG_EXTERNAL_TRANSFER)
        e2[f2[(int64_t)day_of(e) * slots + slot_of(e)]++] = e;
      else
        e1[f1[slot_of(e) * n_nodes + ev.node[e]]++] = e;
    }
  }
  P.e1_day.resize(n_e1);

  // 2. In parallel over ranges of (slot, node) lists and of (day, slot)
  //    buckets:
  //    E1: each list ordered by (day, time on day 0, type, list index) --
  //    every event of a day d >= 1 has time t0 + 1 + d, day 0 also holds the
  //    earlier times;
  //    E2: the first day's buckets ordered by time (stable), then waves, and
  //    the bucket ordered by wave (stable).
  const int T = plan_threads(n_e1 + n_e2);
  const std::vector<int64_t> r1 = weighted_ranges(e1_count, nk, T);
  const std::vector<int64_t> r2 = weighted_ranges(e2_count, nb, T);
  std::vector<std::vector<int64_t>> wave_ends(T);  // per thread: wave ends, bucket by bucket
  std::vector<int32_t> n_waves_of(nb, 0);
  run_threads(T, [&](int t) {
    auto before = [&](int64_t a, int64_t b) {
      const int32_t da = day_of(a), db = day_of(b);
      if (da != db) return da < db;
      if (da == 0 && ev.time[a] != ev.time[b]) return ev.time[a] < ev.time[b];
      return ev.type[a] < ev.type[b];
    };
    for (int64_t k = r1[t]; k < r1[t + 1]; ++k) {
      int64_t *lo = e1 + e1_count[k], *hi = e1 + e1_count[k + 1];
      if (!std::is_sorted(lo, hi, before)) std::stable_sort(lo, hi, before);
      for (int64_t *q = lo; q != hi; ++q) P.e1_day[q - e1] = day_of(*q);
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

}  // namespace sg
