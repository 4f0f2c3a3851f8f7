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

  // The E1 and E2 parts write disjoint members of the plan and run in two
  // threads.
  int64_t n_e1 = 0;
  std::vector<int64_t> e1, e2;
  auto plan_e1 = [&]() -> int {
    // 1. E1: ordered by (slot, node), then (day, time, type, list index), by
    //    stable counting-sort passes over packed records taken in list order:
    //    by type, then by day, then by (slot, node).  Every event of a day
    //    d >= 1 has time t0 + 1 + d; day 0 also holds the earlier times, so
    //    its runs are then ordered by time (stable, keeping type and index).
    std::vector<int64_t> e1_count(nk + 1, 0);
    for (int64_t e = 0; e < n; ++e) {
      if (ev.time[e] > t_end || ev.type[e] == SG_EXTERNAL_TRANSFER) continue;
      const int64_t s = slot_of(e);
      if (s >= slots) return SG_ERR_ARG;
      ++e1_count[s * n_nodes + ev.node[e] + 1];
      ++n_e1;
    }
    std::partial_sum(e1_count.begin(), e1_count.end(), e1_count.begin());
    struct Rec {
      int64_t e;
      int32_t day, type, key, time;
    };
    std::vector<Rec> ra, rb(n_e1);
    ra.reserve(n_e1);
    for (int64_t e = 0; e < n; ++e)
      if (ev.time[e] <= t_end && ev.type[e] != SG_EXTERNAL_TRANSFER)
        ra.push_back(Rec{e, day_of(e), ev.type[e], (int32_t)(slot_of(e) * n_nodes + ev.node[e]),
                         ev.time[e]});
    int64_t tc[5] = {0, 0, 0, 0, 0};  // by type (0 .. 3)
    for (const Rec &r : ra) ++tc[r.type + 1];
    for (int k = 0; k < 4; ++k) tc[k + 1] += tc[k];
    for (const Rec &r : ra) rb[tc[r.type]++] = r;
    std::vector<int64_t> dc((size_t)P.days + 1, 0);  // by day
    for (const Rec &r : rb) ++dc[r.day + 1];
    std::partial_sum(dc.begin(), dc.end(), dc.begin());
    for (const Rec &r : rb) ra[dc[r.day]++] = r;
    std::vector<int64_t> fill(e1_count.begin(), e1_count.end() - 1);  // by (slot, node)
    for (const Rec &r : ra) rb[fill[r.key]++] = r;
    for (int64_t k = 0; k < nk; ++k) {
      auto lo = rb.begin() + e1_count[k], hi = rb.begin() + e1_count[k + 1];
      auto z = lo;
      while (z != hi && z->day == 0) ++z;
      if (z - lo > 1)
        std::stable_sort(lo, z, [](const Rec &x, const Rec &y) { return x.time < y.time; });
    }
    e1.resize(n_e1);
    P.e1_day.resize(n_e1);
    for (int64_t i = 0; i < n_e1; ++i) {
      e1[i] = rb[i].e;
      P.e1_day[i] = rb[i].day;
    }
    P.e1_node_off = e1_count;
    return SG_OK;
  };
  auto plan_e2 = [&]() -> int {
  // 2. E2: stable bucketing by (day, slot), waves inside each bucket.
  std::vector<int64_t> count(nb + 1, 0);
  for (int64_t e = 0; e < n; ++e) {
    if (ev.time[e] > t_end || ev.type[e] != SG_EXTERNAL_TRANSFER) continue;
    const int64_t s = slot_of(e);
    if (s >= slots) return SG_ERR_ARG;
    ++count[(int64_t)day_of(e) * slots + s + 1];
  }
  std::partial_sum(count.begin(), count.end(), count.begin());
  std::vector<int64_t> bucketed(count[nb]);
  {
    std::vector<int64_t> fill(count.begin(), count.end() - 1);
    for (int64_t e = 0; e < n; ++e) {
      if (ev.time[e] > t_end || ev.type[e] != SG_EXTERNAL_TRANSFER) continue;
      bucketed[fill[(int64_t)day_of(e) * slots + slot_of(e)]++] = e;
    }
  }
  e2.reserve(bucketed.size());
  std::vector<int32_t> last_sample(n_nodes, 0), last_add(n_nodes, 0);
  std::vector<int64_t> stamp(n_nodes, -1);
  std::vector<int64_t> tmp;
  std::vector<int32_t> wave_of;
  for (int64_t b = 0; b < nb; ++b) {
    tmp.assign(bucketed.begin() + count[b], bucketed.begin() + count[b + 1]);
    // list order is kept by the bucketing; only the first day can mix times
    if (b < slots)
      std::stable_sort(tmp.begin(), tmp.end(),
                       [&](int64_t a, int64_t c) { return ev.time[a] < ev.time[c]; });
    wave_of.assign(tmp.size(), 0);
    int32_t n_w = 0;
    for (size_t i = 0; i < tmp.size(); ++i) {
      const int64_t e = tmp[i];
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
    std::vector<int64_t> wc(n_w + 2, 0);
    for (size_t i = 0; i < tmp.size(); ++i) ++wc[wave_of[i] + 1];
    std::partial_sum(wc.begin(), wc.end(), wc.begin());
    std::vector<int64_t> sorted(tmp.size());
    {
      std::vector<int64_t> fill(wc.begin(), wc.end() - 1);
      for (size_t i = 0; i < tmp.size(); ++i) sorted[fill[wave_of[i]]++] = tmp[i];
    }
    const int64_t base = (int64_t)e2.size();
    e2.insert(e2.end(), sorted.begin(), sorted.end());
    for (int32_t w = 1; w <= n_w; ++w) P.wave_ev.push_back(base + wc[w + 1]);
    P.e2_wave_off[b + 1] = (int64_t)P.wave_ev.size() - 1;
    if (!tmp.empty()) P.day_has_e2[b / slots] = 1;
    P.max_waves_per_day = std::max(P.max_waves_per_day, n_w);
  }
    return SG_OK;
  };
  int rc2 = SG_OK;
  std::thread th([&] { rc2 = plan_e2(); });
  const int rc1 = plan_e1();
  th.join();
  if (rc1) return rc1;
  if (rc2) return rc2;
  P.n_e1 = n_e1;
  P.n_e2 = (int64_t)e2.size();
  P.n_waves = (int64_t)P.wave_ev.size() - 1;
  for (auto &x : P.wave_ev) x += P.n_e1;  // positions past the E1 part
  P.order.reserve(P.n_e1 + P.n_e2);
  P.order.insert(P.order.end(), e1.begin(), e1.end());
  P.order.insert(P.order.end(), e2.begin(), e2.end());
  return SG_OK;
}

}  // namespace sg
