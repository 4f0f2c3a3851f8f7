// sg_common.h -- internal types shared by the host runtime and the kernels of
// the SimInf GB300 engine.  Not part of the public ABI (include/siminf_gpu.h).
#pragma once

#include <stdint.h>

#include "siminf_gpu.h"

#define SG_MAX_GDATA 32

// Counter-stream identifiers: the fourth Philox counter word is
// (stream << 24) | replicate, so replicates, SSA draws and event draws never
// share a counter.
#define SG_STREAM_SSA 0u
#define SG_STREAM_EVENTS 1u
#define SG_STREAM_EMU 2u
#define SG_STREAM_AEM 3u

// Model tables in the layout the kernels read (passed by value).
struct SgTables {
  int32_t kind, n_nodes, n_comp, n_trans, n_v, n_ldata, n_select, n_shift;
  int8_t S[SG_MAX_TRANS][SG_MAX_COMP];   // S[j][p]: change of p by transition j
  uint32_t dep[SG_MAX_TRANS];            // bit k: recompute rate k after j
  uint32_t Emask[SG_MAX_SELECT];         // bit p: compartment p in E[, s]
  int8_t Nsh[SG_MAX_SHIFT][SG_MAX_COMP]; // Nsh[q][p] = N[p, q]
  double gdata[SG_MAX_GDATA];
};

// Scheduled events in planned order, structure of arrays on the device.
struct SgEventsDev {
  const int8_t *type;
  const uint8_t *select;
  const int8_t *shift;     // -1 = no shift
  const int32_t *node;
  const int32_t *dest;
  const int32_t *n;
  const double *proportion;
  const int64_t *index;    // position in the caller's list (random stream key)
  const int32_t *rep;      // replicate of a replicate-specific event, or -1
};

// Error word written by kernels: the first error wins (atomicCAS on code).
struct SgDevError {
  int32_t code;
  int32_t rep;
  int32_t node;
  int32_t day;
  long long event;
};

struct SgCounters {
  unsigned long long reactions;
  unsigned long long draws;
  unsigned long long events;
  unsigned long long rated;  // node-days whose rates were evaluated (sparse schedule)
};
