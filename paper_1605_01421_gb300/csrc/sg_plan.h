// sg_plan.h -- host-side validation and scheduling of the scheduled events
// (Sec. 3.3) for the SimInf GB300 engine.
#pragma once

#include <stdint.h>

#include <memory>
#include <new>
#include <type_traits>
#include <utility>
#include <vector>

#include "sg_common.h"

namespace sg {

// Allocator whose default construction leaves trivial elements unset: the
// planner's large arrays are written exactly once by its threads, which then
// also touch their pages first (a value-initialised vector would zero them
// on one thread beforehand).
template <class T>
struct DefaultInitAllocator : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = DefaultInitAllocator<U>;
  };
  DefaultInitAllocator() noexcept = default;
  template <class U>
  DefaultInitAllocator(const DefaultInitAllocator<U> &) noexcept {}
  template <class U>
  void construct(U *p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void *>(p)) U;
  }
  template <class U, class... Args>
  void construct(U *p, Args &&...args) {
    ::new (static_cast<void *>(p)) U(std::forward<Args>(args)...);
  }
};
template <class T>
using plan_vector = std::vector<T, DefaultInitAllocator<T>>;

// The caller's event table, copied (0-based; shift < 0 = no shift).
struct EventTable {
  plan_vector<int32_t> type, time, node, dest, n, select, shift, rep;
  plan_vector<double> proportion;
  bool per_rep = false;  // rep[] given
  int32_t max_rep = -1;
  int64_t size() const { return (int64_t)type.size(); }
};

// The caller's columns copied into *ev (rep may be NULL), in parallel over
// slices of the table.
void copy_events(EventTable *ev, int64_t n, const int32_t *type, const int32_t *time,
                 const int32_t *node, const int32_t *dest, const int32_t *cnt,
                 const double *proportion, const int32_t *select, const int32_t *shift,
                 const int32_t *rep);

// Checks of the event table against the model (Sec. 3.3 constraints and the
// readings of the engine): returns SG_OK or the error code, and the index of
// the first offending event in *bad.
int validate_events(const SgTables &tb, const EventTable &ev, int64_t *bad);

// The device-ready schedule of the events for one simulation window
// (unit steps T = t0 + 1 .. t_end) and one number of replicate slots
// (1 when every replicate runs the same events, else n_rep).
//
// Day d (T = t0 + 1 + d) runs the events with time in (T - 1, T]; for d = 0
// also every earlier time.
//
// E1 events (exit, enter, internal transfer) are grouped per (slot, node) and
// sorted inside by (day, time, type, list index): the thread that owns a node
// walks its own list with a cursor, in the order of Sec. 3.3.
//
// E2 events (external transfers) of a (day, slot) keep their (time, list
// index) order and are split into waves: an event goes one wave after the last
// earlier event that sampled its source, added to its source, or sampled its
// destination.  So no two events of a wave touch the same node except as
// destinations (additions commute), and every node sees its samples and
// additions in list order.
struct Plan {
  int32_t t0 = 0, t_end = 0, slots = 1, days = 0, n_nodes = 0;
  int32_t rep_lo = 0;  // a shard's first replicate (slot = replicate - rep_lo)
  bool shard = false;
  plan_vector<int64_t> order;        // E1 part, then E2 part (EventTable indices)
  plan_vector<int32_t> e1_day;       // [n_e1] day index of each E1 event
  std::vector<int64_t> e1_node_off;  // [slots * n_nodes + 1] into order
  std::vector<int64_t> e2_wave_off;  // [days * slots + 1] into wave_ev
  std::vector<int64_t> wave_ev;      // [n_waves + 1] positions in order
  std::vector<uint8_t> day_has_e2;   // [days]
  int64_t n_e1 = 0, n_e2 = 0, n_waves = 0;
  int32_t max_waves_per_day = 0;
};

// shard: plan only the replicates rep_lo .. rep_lo + slots - 1 of a
// per-replicate table (the others' events are left out); otherwise an
// event whose replicate is >= slots (with slots > 1) is an argument error.
int build_plan(const EventTable &ev, int32_t n_nodes, int32_t t0, int32_t t_end,
               int32_t slots, Plan *out, int32_t rep_lo = 0, bool shard = false);

// The device image of the planned events, in plan order: type, shift (-1
// for none), select, node, dest, n, proportion and the list index.
void gather_events(const EventTable &ev, const Plan &P, int8_t *type, int8_t *shift,
                   uint8_t *select, int32_t *node, int32_t *dest, int32_t *n, double *proportion,
                   int64_t *index);

}  // namespace sg
