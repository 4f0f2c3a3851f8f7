// sg_engine.cu -- kernels and C ABI of the SimInf GB300 engine.
//
// The split-step method of Sec. 2.3 runs as a chain of kernels on the
// caller's stream:
//   k_days<KIND>   one thread per (replicate, node): finishes the previous
//                  unit step (post time step + recording), then per day runs
//                  the direct SSA toward the next unit time point (Appendix A;
//                  a warp takes over nodes that need many draws) and the
//                  node's own exit / enter / internal-transfer events, for a
//                  whole run of days without external transfers;
//   k_events_e2    the external transfers of a day, one block per replicate,
//                  wave by wave (a block barrier between waves);
// and a last k_days launch finishes the final unit step.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "sg_common.h"
#include "sg_device.cuh"
#include "sg_kernels.cuh"
#include "sg_mlp.h"
#include "sg_mparse.h"
#include "sg_plan.h"

using namespace sg;

namespace {

// SISe_sp post time step of every node for unit time T from the same old
// values (Sec. 4.2 with the coupling term), one thread per (replicate, node):
//   phi' = phi + ((alpha I / N + sum_k ((phi_k N_k - phi N) / N) (D / d_k))
//                 - beta(T) phi),
// neighbours in list order, both terms 0 in an empty node; then recording.
struct PtsSpArgs {
  const int *u;
  const double *v_old;
  double *v_new;
  const double *ldata;
  const int64_t *nb_ptr;
  const int32_t *nb_idx;
  const double *nb_dist;
  int32_t *U;
  double *V;
  const int32_t *rec;
  int32_t t0, M, n_rep, T;
  int32_t rep0;  // global index of local replicate 0 (error reports)
  SgDevError *err;
  OutDev out;
};

// The coupled post time step of one (replicate, node) and its recording at
// slot m; the node's counts are returned in uu.
__device__ __forceinline__ void pts_sp_node(const SgTables &tb, const PtsSpArgs &a, long long gid,
                                          int m, int *uu) {
  const int Nn = tb.n_nodes;
  const int rep = (int)(gid / Nn), node = (int)(gid - (long long)rep * Nn);
  const int *ur = a.u + (long long)rep * Nn * 2;
  const double *vr = a.v_old + (long long)rep * Nn;
  const double *g = tb.gdata;
  const int S = ur[node * 2], I = ur[node * 2 + 1];
  const double Ni = i2d(S) + i2d(I);
  const double phi = vr[node];
  double shed = 0.0, coupling = 0.0;
  if (gt0(Ni)) {
    shed = (g[2] * i2d(I)) / Ni;
    if (a.nb_ptr) {
      const double DN = g[7];
      for (long long k = a.nb_ptr[node]; k < a.nb_ptr[node + 1]; ++k) {
        const int j = a.nb_idx[k];
        const double Nk = i2d(ur[j * 2]) + i2d(ur[j * 2 + 1]);
        const double term = ((vr[j] * Nk - phi * Ni) / Ni) * (DN / a.nb_dist[k]);
        coupling = coupling + term;
      }
    }
  }
  int ends[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) ends[i] = season_end_int(a.ldata[(long long)node * tb.n_ldata + i]);
  const double beta = season_decay(a.T, ends, g + 3);
  const double nv = phi + ((shed + coupling) - beta * phi);
  a.v_new[gid] = nv;
  if (!isfinite(nv)) report(a.err, SG_ERR_PTS, a.rep0 + rep, node, a.T, -1);
  uu[0] = S;
  uu[1] = I;
  if (m >= 0) {
    const long long base = ((long long)rep * a.M + m) * Nn + node;
    if (a.U) {
      a.U[base * 2] = S;
      a.U[base * 2 + 1] = I;
    }
    if (a.V) a.V[base] = nv;
    record_sparse<2, 1>(a.out, m, rep, node, uu, &nv);
  }
}

__global__ void __launch_bounds__(128) k_pts_sp(const SgTables tb, const PtsSpArgs a) {
  pdl_trigger();
  pdl_wait();
  const int Nn = tb.n_nodes;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in_range = gid < (long long)Nn * a.n_rep;
  const int m = a.rec[a.T - a.t0];
  int uu[2] = {0, 0};
  if (in_range) pts_sp_node(tb, a, gid, m, uu);
  if (m >= 0 && a.out.prev) {
    const int rep = in_range ? (int)(gid / Nn) : 0;
    prevalence_add<2>(a.out, in_range ? (long long)rep * a.M + m : -1, in_range, uu);
  }
}


// Channels of the all events method before the first day: rate 0, asleep
// (firing time +inf), no draws taken.
__global__ void k_aem_init(double *a, double *tau, uint32_t *c, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    a[i] = 0.0;
    tau[i] = __longlong_as_double(0x7ff0000000000000ll);
    c[i] = 0u;
  }
}

// U[r][0] = u0[r], V[r][0] = v0[r] (when recorded densely), working state =
// initial state.
__global__ void k_init(const int32_t *__restrict__ u0, const double *__restrict__ v0, int *u,
                       double *v, int32_t *U, double *V, long long per_rep_u,
                       long long per_rep_v, int M, int n_rep) {
  const long long nu = per_rep_u * n_rep, nv = per_rep_v * n_rep;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nu + nv;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nu) {
      const long long r = i / per_rep_u, k = i - r * per_rep_u;
      const int32_t x = u0[i];
      u[i] = x;
      if (U) U[r * M * per_rep_u + k] = x;
    } else {
      const long long ii = i - nu;
      const long long r = ii / per_rep_v, k = ii - r * per_rep_v;
      const double x = v0[ii];
      v[ii] = x;
      if (V) V[r * M * per_rep_v + k] = x;
    }
  }
}

__global__ void k_philox_batch(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                               long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const U4 c = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    const U4 r = philox10(c, k0, k1);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
  }
}

__global__ void k_log_batch(const double *x, double *y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = x[i];
    double r;
    if (!(a > 0.0)) r = a == 0.0 ? -INFINITY : NAN;
    else if (isinf(a)) r = a;
    else r = log_pos(a);
    y[i] = r;
  }
}

__global__ void k_u01_batch(const uint32_t *w, double *y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = u01_open(w[2 * i], w[2 * i + 1]);
}

// Independent fused multiply-add chains (8 per thread) for the FP64
// throughput probe; the result is stored so the chains are not removed.
__global__ void k_fp64_fma(double *out, int iters) {
  double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
  double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
  const double m = 0.999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
    a0 = __fma_rn(a0, m, c); a1 = __fma_rn(a1, m, c);
    a2 = __fma_rn(a2, m, c); a3 = __fma_rn(a3, m, c);
    a4 = __fma_rn(a4, m, c); a5 = __fma_rn(a5, m, c);
    a6 = __fma_rn(a6, m, c); a7 = __fma_rn(a7, m, c);
  }
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// ---------------------------------------------------------------------------
// Host runtime
// ---------------------------------------------------------------------------

// Memory kept for reuse by the models of the process: blocks freed by one
// model are handed to the next (creating and freeing CUDA memory costs tens
// to hundreds of microseconds a call and synchronises the device).  Blocks
// are matched by (device, size rounded up to 256 bytes), best fit up to
// twice the size asked for; at most kCap bytes stay cached, the rest is
// freed.  A block goes back to the pool only when its model is destroyed or
// grows it, after sg_run has synchronised its stream.
class MemPool {
 public:
  explicit MemPool(bool pinned) : pinned_(pinned) {}
  void *get(size_t bytes) {
    bytes = round(bytes);
    const int dev = device();
    {
      std::lock_guard<std::mutex> lock(mu_);
      auto it = free_.lower_bound(Key{dev, bytes});
      if (it != free_.end() && it->first.dev == dev && it->first.bytes <= 2 * bytes) {
        void *p = it->second;
        cached_ -= it->first.bytes;
        owner_[p] = it->first;
        free_.erase(it);
        return p;
      }
    }
    void *p = nullptr;
    const cudaError_t e = pinned_ ? cudaMallocHost(&p, bytes) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu_);
    owner_[p] = Key{dev, bytes};
    return p;
  }
  void put(void *p) {
    if (!p) return;
    std::unique_lock<std::mutex> lock(mu_);
    auto it = owner_.find(p);
    const Key k = it == owner_.end() ? Key{0, 0} : it->second;
    if (it != owner_.end()) owner_.erase(it);
    if (k.bytes && cached_ + k.bytes <= kCap) {
      free_.emplace(k, p);
      cached_ += k.bytes;
      return;
    }
    lock.unlock();
    if (pinned_)
      cudaFreeHost(p);
    else
      cudaFree(p);
  }

 private:
  struct Key {
    int dev;
    size_t bytes;
    bool operator<(const Key &o) const { return dev != o.dev ? dev < o.dev : bytes < o.bytes; }
  };
  static constexpr size_t kCap = (size_t)1 << 30;
  static size_t round(size_t b) { return ((b ? b : 1) + 255) & ~(size_t)255; }
  static int device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
      cudaGetLastError();
      d = 0;
    }
    return d;
  }
  const bool pinned_;
  std::mutex mu_;
  std::multimap<Key, void *> free_;
  std::map<void *, Key> owner_;  // blocks in use: device and size
  size_t cached_ = 0;
};

static MemPool &device_pool() {
  static MemPool *p = new MemPool(false);  // never destroyed (outlives every model)
  return *p;
}
static MemPool &pinned_pool() {
  static MemPool *p = new MemPool(true);
  return *p;
}

template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  int ensure(size_t want) {
    if (want <= n && p) return SG_OK;
    release();
    if (want == 0) want = 1;
    p = static_cast<T *>(device_pool().get(want * sizeof(T)));
    if (!p) return SG_ERR_NOMEM;
    n = want;
    return SG_OK;
  }
  void release() {
    device_pool().put(p);
    p = nullptr;
    n = 0;
  }
};

template <typename T>
int upload(DevBuf<T> &b, const std::vector<T> &h) {
  int rc = b.ensure(h.size());
  if (rc) return rc;
  if (!h.empty() &&
      cudaMemcpy(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  return SG_OK;
}

}  // namespace

// What a captured run depends on besides the model's tables and plan.
// Every pointer the captured kernels use is part of the key, so a buffer
// that was reallocated in between (by any call) forces a new capture.
struct GraphKey {
  const void *u0, *v0, *U, *V;
  const void *u, *v, *cur, *rec, *emu;
  uint64_t seed;
  int32_t n_rep, n_tspan, t0, t_end, npb, heavy_after, rep0;
  uint64_t plan_version;
  bool operator==(const GraphKey &o) const {
    return u0 == o.u0 && v0 == o.v0 && U == o.U && V == o.V && u == o.u && v == o.v &&
           cur == o.cur && rec == o.rec && emu == o.emu && seed == o.seed && n_rep == o.n_rep &&
           rep0 == o.rep0 &&
           n_tspan == o.n_tspan && t0 == o.t0 && t_end == o.t_end && npb == o.npb &&
           heavy_after == o.heavy_after && plan_version == o.plan_version;
  }
};

struct sg_model {
  SgTables tb;
  DevBuf<double> ldata;
  EventTable ev;
  // planned events for the cached window
  bool plan_ok = false;
  Plan plan;
  // the plan's device arrays: views into one arena (ev_arena), filled from
  // one host staging buffer (ev_stage)
  DevBuf<unsigned char> ev_arena;
  std::vector<unsigned char> ev_stage;
  int8_t *e_type = nullptr, *e_shift = nullptr;
  uint8_t *e_select = nullptr;
  int32_t *e_node = nullptr, *e_dest = nullptr, *e_n = nullptr, *e1_day = nullptr;
  double *e_prop = nullptr;
  int64_t *e_index = nullptr, *wave_ev = nullptr, *wave_off = nullptr, *e1_node_off = nullptr;
  int32_t heavy_after = -1;  // draws a thread takes before its warp takes
  int32_t npb = -1;          // nodes per block; -1 = chosen from the size
  // sg_set_replicate_range: the runs cover global replicates rep0 .. rep0 +
  // n_rep - 1 of a job with rep_total replicates (0: a whole job, rep0 = 0)
  int32_t rep0 = 0, rep_total = 0;
  // working memory
  DevBuf<int32_t> e1_cur;
  DevBuf<int32_t> e1_next;  // sparse schedule: day of each unit's next E1 event
  // the external transfers of a replicate-day touch a sizeable share of its
  // nodes (on average at least one node in 16 as a source): the E2 kernel
  // then stages the replicate's state in shared memory, else it works on
  // the state in device memory (L2)
  bool e2_dense = true;
  DevBuf<int> u;
  DevBuf<double> v;
  DevBuf<int32_t> rec;
  DevBuf<SgDevError> err;
  DevBuf<SgCounters> cnt;
  SgDevError *h_err = nullptr;
  SgCounters *h_cnt = nullptr;
  // per-kernel timing (sg_set_kernel_timing)
  bool timing = false;
  std::vector<cudaEvent_t> evpool;
  std::vector<int> ev_kind;  // per launch: 0 SSA, 1 E1, 2 E2, 3 emulator GEMM
  size_t ev_used = 0;
  // buffers of sg_run_host
  DevBuf<int32_t> hu0, hU;
  DevBuf<double> hv0, hV;
  // the tspan table on the device, as last uploaded
  std::vector<int32_t> rec_host;
  // the captured run (CUDA graph)
  bool graphs = true;
  bool graph_ok = false;
  GraphKey graph_key{};
  cudaGraphExec_t graph_exec = nullptr;
  long long graph_launches = 0;
  int32_t graph_waves = 0;
  uint64_t plan_version = 0;
  // learned one-day emulator (SISe3): caller-owned device weights, own buffers
  bool emu_on = false;
  const __nv_bfloat16 *emu_W[4] = {};
  const float *emu_b[4] = {};
  int32_t emu_max_herd = 2000;
  double emu_phi_lo = 0.0, emu_phi_hi = 0.0, emu_min_rate = 0.0;
  uint64_t emu_version = 0;
  DevBuf<__nv_bfloat16> emu_feat, emu_ha, emu_hb;
  // FP8 inference of layers 2-4 (sg_emulator_set_fp8)
  bool emu_fp8 = false;
  const uint8_t *emu_W8[3] = {};
  const float *emu_wscale[3] = {};
  float emu_act_scale[3] = {1.0f, 1.0f, 1.0f};
  DevBuf<uint8_t> emu_h8a, emu_h8b, emu_img;  // tiled E4M3 activations, weight images
  DevBuf<float> emu_hvec;                     // head-padded output-layer bias, scales
  // side stream of the emulator day (the SSA part beside the chain) and its
  // fork / join events
  cudaStream_t side_st = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
  DevBuf<float> emu_logits;
  DevBuf<int32_t> emu_flag, emu_delta;
  // SISe_sp neighbour lists and the second phi buffer of the coupled step
  DevBuf<int64_t> nb_ptr;
  DevBuf<int32_t> nb_idx;
  DevBuf<double> nb_dist, v2;
  bool has_nb = false;
  uint64_t nb_version = 0;
  // solver (SG_SOLVER_SSM or SG_SOLVER_AEM) and the channel state of 'aem'
  int32_t solver = SG_SOLVER_SSM;
  DevBuf<double> aem_a, aem_tau;
  DevBuf<uint32_t> aem_cnt;
  // output selection (sg_set_output)
  bool out_dense = true;
  int32_t out_cols = -1;  // tspan points the patterns were made for (-1: none)
  OutDev out;
  DevBuf<int64_t> out_u_colptr, out_v_colptr;
  DevBuf<int32_t> out_u_row, out_v_row;
  uint64_t out_version = 0;
  // SG_GENERIC: the kernels compiled at run time for the parsed model
  JitKernels jit;
  // external transfers inside the day kernel (sg_set_fused_events)
  bool fuse_e2 = false;
  DevBuf<int32_t> e2_done;
  // persistent day loop (sg_set_persistent) and its grid barrier words
  bool persistent = false;
  DevBuf<unsigned int> grid_bar;
};

extern "C" const char *sg_strerror(int code) {
  switch (code) {
    case SG_OK: return "ok";
    case SG_ERR_ARG: return "invalid argument";
    case SG_ERR_EVENT_UNDERFLOW: return "event moves more individuals than exist";
    case SG_ERR_SHIFT_RANGE: return "shift moves outside the compartments";
    case SG_ERR_RATE: return "negative or non-finite transition rate";
    case SG_ERR_PTS: return "post time step error";
    case SG_ERR_TIMEOUT: return "device wait timed out";
    case SG_ERR_CUDA: return "CUDA runtime error";
    case SG_ERR_NOMEM: return "out of memory";
    case SG_ERR_STEP_LIMIT: return "more than SG_MAX_DRAWS draws in one node-day";
    case SG_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of sg_run_noalloc";
    case SG_ERR_PARSE: return "transition string does not parse";
    case SG_ERR_JIT: return "run-time compilation or loading failed";
    default: return "unknown error";
  }
}

static const int kKindComp[5] = {3, 2, 2, 6, 2};
static const int kKindTrans[5] = {2, 2, 2, 6, 2};
static const int kKindNv[5] = {0, 0, 1, 1, 1};
static const int kKindGdata[5] = {2, 2, 7, 11, 8};
static const int kKindLdata[5] = {0, 0, 4, 4, 4};

static int model_create(const sg_desc *d, sg_model **out, bool generic);

extern "C" int sg_model_create(const sg_desc *d, sg_model **out) {
  return model_create(d, out, false);
}

static int model_create(const sg_desc *d, sg_model **out, bool generic) {
  if (!d || !out) return SG_ERR_ARG;
  *out = nullptr;
  const int k = d->kind;
  if (generic ? k != SG_GENERIC : (k < SG_SIR || k > SG_SISE_SP)) return SG_ERR_ARG;
  if (generic && (d->n_comp < 1 || d->n_comp > SG_MAX_COMP || d->n_trans < 1 ||
                  d->n_trans > SG_MAX_TRANS || d->n_v != 0 || d->n_ldata != 0 ||
                  d->n_gdata < 0))
    return SG_ERR_ARG;
  if (d->n_nodes < 0 ||
      (!generic && (d->n_comp != kKindComp[k] || d->n_trans != kKindTrans[k] ||
                    d->n_v != kKindNv[k] || d->n_gdata < kKindGdata[k] ||
                    d->n_ldata < kKindLdata[k])) ||
      d->n_gdata > SG_MAX_GDATA || d->n_select < 0 || d->n_select > SG_MAX_SELECT ||
      d->n_shift < 0 || d->n_shift > SG_MAX_SHIFT || !d->S || !d->G ||
      (d->n_select > 0 && !d->E) || (d->n_shift > 0 && !d->N) ||
      (d->n_gdata > 0 && !d->gdata) ||
      (d->n_ldata > 0 && d->n_nodes > 0 && !d->ldata))
    return SG_ERR_ARG;
  sg_model *m = new (std::nothrow) sg_model();
  if (!m) return SG_ERR_NOMEM;
  SgTables &tb = m->tb;
  std::memset(&tb, 0, sizeof tb);
  tb.kind = k;
  tb.n_nodes = d->n_nodes;
  tb.n_comp = d->n_comp;
  tb.n_trans = d->n_trans;
  tb.n_v = d->n_v;
  tb.n_ldata = d->n_ldata;
  tb.n_select = d->n_select;
  tb.n_shift = d->n_shift;
  const int C = d->n_comp, T = d->n_trans;
  for (int j = 0; j < T; ++j) {
    for (int p = 0; p < C; ++p) {
      const int s = d->S[(size_t)j * C + p];
      if (s < -127 || s > 127) { delete m; return SG_ERR_ARG; }
      tb.S[j][p] = (int8_t)s;
    }
    uint32_t dep = 0;
    for (int kk = 0; kk < T; ++kk)
      if (d->G[(size_t)j * T + kk] != 0) dep |= 1u << kk;
    tb.dep[j] = dep;
  }
  for (int s = 0; s < d->n_select; ++s) {
    uint32_t mask = 0;
    for (int p = 0; p < C; ++p)
      if (d->E[(size_t)s * C + p] != 0) mask |= 1u << p;
    tb.Emask[s] = mask;
  }
  for (int q = 0; q < d->n_shift; ++q)
    for (int p = 0; p < C; ++p) {
      const int x = d->N[(size_t)q * C + p];
      if (x < -127 || x > 127) { delete m; return SG_ERR_ARG; }
      tb.Nsh[q][p] = (int8_t)x;
    }
  for (int i = 0; i < d->n_gdata; ++i) tb.gdata[i] = d->gdata[i];
  const size_t nl = (size_t)d->n_ldata * d->n_nodes;
  std::vector<double> ld(d->ldata ? d->ldata : nullptr, d->ldata ? d->ldata + nl : nullptr);
  int rc = upload(m->ldata, ld);
  if (!rc) rc = m->err.ensure(1);
  if (!rc) rc = m->cnt.ensure(1);
  if (!rc && !(m->h_err = static_cast<SgDevError *>(pinned_pool().get(sizeof(SgDevError)))))
    rc = SG_ERR_NOMEM;
  if (!rc && !(m->h_cnt = static_cast<SgCounters *>(pinned_pool().get(sizeof(SgCounters)))))
    rc = SG_ERR_NOMEM;
  if (rc) {
    cudaGetLastError();
    sg_model_destroy(m);
    return rc;
  }
  *out = m;
  return SG_OK;
}

static void put_msg(char *msg, int32_t len, const std::string &text) {
  if (!msg || len <= 0) return;
  const size_t n = std::min<size_t>(text.size(), (size_t)len - 1);
  std::memcpy(msg, text.data(), n);
  msg[n] = 0;
}

extern "C" int sg_model_create_parsed(const char *const *transitions, int32_t n_trans,
                                      const char *const *compartments, int32_t n_comp,
                                      const char *const *gdata_names, const double *gdata,
                                      int32_t n_gdata, int32_t n_nodes, const int32_t *E,
                                      int32_t n_select, const int32_t *N, int32_t n_shift,
                                      sg_model **out, char *msg, int32_t msg_len) {
  put_msg(msg, msg_len, "");
  if (!out) return SG_ERR_ARG;
  *out = nullptr;
  ParsedModel pm;
  std::string text;
  int rc = mparse(transitions, n_trans, compartments, n_comp, gdata_names, n_gdata, pm, text);
  if (rc) {
    put_msg(msg, msg_len, text);
    return rc;
  }
  sg_desc d;
  std::memset(&d, 0, sizeof d);
  d.kind = SG_GENERIC;
  d.n_nodes = n_nodes;
  d.n_comp = pm.C;
  d.n_trans = pm.T;
  d.S = pm.S.data();
  d.G = pm.G.data();
  d.n_select = n_select;
  d.E = E;
  d.n_shift = n_shift;
  d.N = N;
  d.n_v = 0;
  d.n_ldata = 0;
  d.ldata = nullptr;
  d.n_gdata = n_gdata;
  d.gdata = gdata;
  sg_model *m = nullptr;
  rc = model_create(&d, &m, true);
  if (rc) return rc;
  rc = jit_build(pm, m->jit, text);
  if (rc) {
    put_msg(msg, msg_len, text);
    sg_model_destroy(m);
    return rc;
  }
  *out = m;
  return SG_OK;
}

extern "C" int sg_model_tables(const sg_model *m, int32_t *S, int32_t *G) {
  if (!m) return SG_ERR_ARG;
  const SgTables &tb = m->tb;
  for (int j = 0; j < tb.n_trans; ++j) {
    for (int p = 0; S && p < tb.n_comp; ++p) S[(size_t)j * tb.n_comp + p] = tb.S[j][p];
    for (int k = 0; G && k < tb.n_trans; ++k)
      G[(size_t)j * tb.n_trans + k] = (int32_t)((tb.dep[j] >> k) & 1u);
  }
  return SG_OK;
}

extern "C" void sg_model_destroy(sg_model *m) {
  if (!m) return;
  m->ldata.release();
  m->ev_arena.release();
  m->e1_cur.release();
  m->e1_next.release();
  m->u.release(); m->v.release(); m->rec.release(); m->err.release(); m->cnt.release();
  m->hu0.release(); m->hU.release(); m->hv0.release(); m->hV.release();
  m->emu_feat.release(); m->emu_ha.release(); m->emu_hb.release();
  m->emu_h8a.release(); m->emu_h8b.release(); m->emu_img.release(); m->emu_hvec.release();
  if (m->side_st) cudaStreamDestroy(m->side_st);
  if (m->side_fork) cudaEventDestroy(m->side_fork);
  if (m->side_join) cudaEventDestroy(m->side_join);
  m->emu_logits.release(); m->emu_flag.release(); m->emu_delta.release();
  m->nb_ptr.release(); m->nb_idx.release(); m->nb_dist.release(); m->v2.release();
  m->aem_a.release(); m->aem_tau.release(); m->aem_cnt.release();
  m->out_u_colptr.release(); m->out_v_colptr.release();
  m->out_u_row.release(); m->out_v_row.release();
  jit_release(m->jit);
  m->e2_done.release();
  m->grid_bar.release();
  pinned_pool().put(m->h_err);
  pinned_pool().put(m->h_cnt);
  for (cudaEvent_t e : m->evpool) cudaEventDestroy(e);
  if (m->graph_exec) cudaGraphExecDestroy(m->graph_exec);
  delete m;
}

extern "C" int sg_set_events(sg_model *m, int64_t n_events, const int32_t *event,
                             const int32_t *time, const int32_t *node, const int32_t *dest,
                             const int32_t *n, const double *proportion,
                             const int32_t *select, const int32_t *shift,
                             const int32_t *rep) {
  if (!m || n_events < 0) return SG_ERR_ARG;
  if (n_events > 0 && (!event || !time || !node || !dest || !n || !proportion || !select ||
                       !shift))
    return SG_ERR_ARG;
  EventTable ev;
  try {
    copy_events(&ev, n_events, event, time, node, dest, n, proportion, select, shift, rep);
  } catch (const std::bad_alloc &) {
    return SG_ERR_NOMEM;
  }
  int64_t bad = -1;
  const int rc = validate_events(m->tb, ev, &bad);
  if (rc) return rc;
  m->ev = std::move(ev);
  m->plan_ok = false;
  return SG_OK;
}

// Build (or reuse) the device schedule of the events for a window.
// Page-locked host staging for the plan upload, shared by every model of the
// process (the copy from it is a DMA transfer; pinning a new buffer per
// model would cost more than it saves).  Held under its lock from filling
// to the end of the copy.
static std::mutex g_stage_mu;
static unsigned char *g_stage = nullptr;
static size_t g_stage_cap = 0;

static unsigned char *pinned_stage(size_t bytes) {
  if (bytes <= g_stage_cap) return g_stage;
  if (g_stage) cudaFreeHost(g_stage);
  g_stage = nullptr;
  g_stage_cap = 0;
  const size_t cap = std::max<size_t>(bytes + bytes / 2, (size_t)1 << 20);
  if (cudaHostAlloc((void **)&g_stage, cap, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    g_stage = nullptr;
    return nullptr;
  }
  g_stage_cap = cap;
  return g_stage;
}

static int ensure_plan(sg_model *m, int32_t t0, int32_t t_end, int32_t slots) {
  // a shard of a job with per-replicate events plans its own replicates
  const bool shard = m->rep_total > 0 && m->ev.per_rep;
  const int32_t rep_lo = shard ? m->rep0 : 0;
  if (m->plan_ok && m->plan.t0 == t0 && m->plan.t_end == t_end && m->plan.slots == slots &&
      m->plan.rep_lo == rep_lo && m->plan.shard == shard)
    return SG_OK;
  m->plan_ok = false;
  Plan &P = m->plan;
  int rc = build_plan(m->ev, m->tb.n_nodes, t0, t_end, slots, &P, rep_lo, shard);
  if (rc) return rc;
  // every device array of the plan in one arena, filled in one host staging
  // buffer and copied with one transfer
  const size_t n = P.order.size();
  size_t off = 0;
  auto place = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_type = place(n), o_shift = place(n), o_sel = place(n),
               o_node = place(4 * n), o_dest = place(4 * n), o_cnt = place(4 * n),
               o_prop = place(8 * n), o_idx = place(8 * n),
               o_wev = place(8 * P.wave_ev.size()), o_woff = place(8 * P.e2_wave_off.size()),
               o_e1d = place(4 * P.e1_day.size()), o_e1o = place(8 * P.e1_node_off.size());
  const size_t total = std::max<size_t>(off, 256);
  std::lock_guard<std::mutex> stage_lock(g_stage_mu);
  unsigned char *h = pinned_stage(total);
  if (!h) {  // no page-locked memory: a pageable buffer of the model's own
    m->ev_stage.resize(total);
    h = m->ev_stage.data();
  }
  {
    gather_events(m->ev, P, (int8_t *)(h + o_type), (int8_t *)(h + o_shift), h + o_sel,
                  (int32_t *)(h + o_node), (int32_t *)(h + o_dest), (int32_t *)(h + o_cnt),
                  (double *)(h + o_prop), (int64_t *)(h + o_idx));
    auto put = [&](size_t o, const void *src, size_t bytes) {
      if (bytes) std::memcpy(h + o, src, bytes);
    };
    put(o_wev, P.wave_ev.data(), 8 * P.wave_ev.size());
    put(o_woff, P.e2_wave_off.data(), 8 * P.e2_wave_off.size());
    put(o_e1d, P.e1_day.data(), 4 * P.e1_day.size());
    put(o_e1o, P.e1_node_off.data(), 8 * P.e1_node_off.size());
  }
  if ((rc = m->ev_arena.ensure(total))) return rc;
  if (cudaMemcpy(m->ev_arena.p, h, total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  unsigned char *d = m->ev_arena.p;
  m->e_type = (int8_t *)(d + o_type);
  m->e_shift = (int8_t *)(d + o_shift);
  m->e_select = d + o_sel;
  m->e_node = (int32_t *)(d + o_node);
  m->e_dest = (int32_t *)(d + o_dest);
  m->e_n = (int32_t *)(d + o_cnt);
  m->e_prop = (double *)(d + o_prop);
  m->e_index = (int64_t *)(d + o_idx);
  m->wave_ev = (int64_t *)(d + o_wev);
  m->wave_off = (int64_t *)(d + o_woff);
  m->e1_day = (int32_t *)(d + o_e1d);
  m->e1_node_off = (int64_t *)(d + o_e1o);
  m->plan_ok = true;
  ++m->plan_version;
  return SG_OK;
}

// Launch with programmatic stream serialization (see pdl_wait).
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Nodes per block when not tuned: fill about two blocks per SM for small
// problems (so heavy nodes spread over many SMs and warps), full blocks
// otherwise.
static int32_t default_npb(long long units) {
  int32_t npb = kDayBlock;
  while (npb > 16 && (units + npb - 1) / npb < 2 * 152) npb >>= 1;
  return npb;
}

template <int KIND>
static void launch_days(sg_model *m, const DayArgs &a, cudaStream_t st) {
  const long long units = (long long)m->tb.n_nodes * a.n_rep;
  const unsigned grid = (unsigned)std::max<long long>(1, (units + a.npb - 1) / a.npb);
  if (a.aem_tau) {
    launch_pdl(k_days<KIND, true>, grid, kDayBlock, 0, st, m->tb, a);
  } else if (a.npb > kDayBlock) {
    // sparse-activity schedule (sg_run only sets npb > kDayBlock where it
    // applies: direct method, built-in kinds without a coupled post step)
    if constexpr (KIND == SG_SIR || KIND == SG_SIS || KIND == SG_SISE || KIND == SG_SISE3)
      launch_pdl(k_days_sparse<KIND>, grid, kSparseBlock, 0, st, m->tb, a);
  } else {
    launch_pdl(k_days<KIND, false>, grid, kDayBlock, 0, st, m->tb, a);
  }
}

// Launch of a kernel compiled at run time (SG_GENERIC), with programmatic
// stream serialization when `pdl`.
static void launch_jit(cudaKernel_t k, unsigned grid, unsigned block, size_t smem,
                       cudaStream_t st, void **args, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelExC(&cfg, (const void *)k, args);
}

// Persistent day loop: one cooperative launch (every block resident) runs
// every day, external transfers included.  Possible for the built-in kinds
// when the grid fits on the device at once.
template <int KIND>
static bool coop_fits(bool aem, unsigned grid) {
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const cudaError_t e =
      aem ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_days<KIND, true>, kDayBlock, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_days<KIND, false>, kDayBlock,
                                                          0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return coop != 0 && (long long)per_sm * sms >= (long long)grid;
}

template <int KIND>
static void launch_days_coop(sg_model *m, const DayArgs &a, unsigned grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kDayBlock);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (a.aem_tau)
    cudaLaunchKernelEx(&cfg, k_days<KIND, true>, m->tb, a);
  else
    cudaLaunchKernelEx(&cfg, k_days<KIND, false>, m->tb, a);
}

static unsigned day_grid(const sg_model *m, const DayArgs &a) {
  const long long units = (long long)m->tb.n_nodes * a.n_rep;
  return (unsigned)std::max<long long>(1, (units + a.npb - 1) / a.npb);
}

// Whether the persistent form applies (built-in kind, grid resident at once).
static bool persistent_fits(const sg_model *m, const DayArgs &a) {
  const unsigned grid = day_grid(m, a);
  const bool aem = a.aem_tau != nullptr;
  switch (m->tb.kind) {
    case SG_SIR: return coop_fits<SG_SIR>(aem, grid);
    case SG_SIS: return coop_fits<SG_SIS>(aem, grid);
    case SG_SISE: return coop_fits<SG_SISE>(aem, grid);
    case SG_SISE3: return coop_fits<SG_SISE3>(aem, grid);
    default: return false;
  }
}

static void launch_days_persistent(sg_model *m, const DayArgs &a, cudaStream_t st) {
  const unsigned grid = day_grid(m, a);
  switch (m->tb.kind) {
    case SG_SIR: launch_days_coop<SG_SIR>(m, a, grid, st); break;
    case SG_SIS: launch_days_coop<SG_SIS>(m, a, grid, st); break;
    case SG_SISE: launch_days_coop<SG_SISE>(m, a, grid, st); break;
    default: launch_days_coop<SG_SISE3>(m, a, grid, st); break;
  }
}

static void launch_days_kind(sg_model *m, const DayArgs &a, cudaStream_t st) {
  if (m->tb.kind == SG_GENERIC) {
    const long long units = (long long)m->tb.n_nodes * a.n_rep;
    const unsigned grid = (unsigned)std::max<long long>(1, (units + a.npb - 1) / a.npb);
    SgTables tb = m->tb;
    DayArgs da = a;
    void *args[] = {&tb, &da};
    launch_jit(m->jit.k[a.aem_tau ? JitKernels::kDaysAem : JitKernels::kDaysSsm], grid,
               kDayBlock, 0, st, args, true);
    return;
  }
  switch (m->tb.kind) {
    case SG_SIR: launch_days<SG_SIR>(m, a, st); break;
    case SG_SIS: launch_days<SG_SIS>(m, a, st); break;
    case SG_SISE: launch_days<SG_SISE>(m, a, st); break;
    case SG_SISE_SP: launch_days<SG_SISE_SP>(m, a, st); break;
    default: launch_days<SG_SISE3>(m, a, st); break;
  }
}

// Bracket one kernel launch with timing events (no-op unless timing is on).
struct LaunchTimer {
  sg_model *m;
  cudaStream_t st;
  int kind;
  bool on;
  LaunchTimer(sg_model *m_, cudaStream_t s_, int k_) : m(m_), st(s_), kind(k_), on(m_->timing) {
    if (!on) return;
    while (m->evpool.size() < m->ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); on = false; return; }
      m->evpool.push_back(e);
    }
    cudaEventRecord(m->evpool[m->ev_used], st);
  }
  ~LaunchTimer() {
    if (!on) return;
    cudaEventRecord(m->evpool[m->ev_used + 1], st);
    m->ev_kind.push_back(kind);
    m->ev_used += 2;
  }
};

// The E2 kernel keeps the replicate's node state in shared memory when it
// is at most this large.
constexpr size_t kE2SmemStateMax = 64 * 1024;

template <int KIND>
static void launch_e2(sg_model *m, const EvArgs &ea, long long wb, long long we, int day,
                      int slots, int n_rep, cudaStream_t st) {
  const size_t bytes = sizeof(int) * (size_t)m->tb.n_nodes * ModelTraits<KIND>::C;
  if (bytes <= kE2SmemStateMax && m->e2_dense) {
    static unsigned long long attr_set = 0;  // one bit per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !((attr_set >> dev) & 1ull)) {
      cudaFuncSetAttribute(k_events_e2<KIND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kE2SmemStateMax);
      attr_set |= 1ull << dev;
    }
    launch_pdl(k_events_e2<KIND, true>, (unsigned)n_rep, kE2Block, bytes, st, m->tb, ea,
               (const int64_t *)m->wave_ev, wb, we, (const int64_t *)m->wave_off, day, slots);
  } else {
    launch_pdl(k_events_e2<KIND, false>, (unsigned)n_rep, kE2Block, 0, st, m->tb, ea,
               (const int64_t *)m->wave_ev, wb, we, (const int64_t *)m->wave_off, day, slots);
  }
}

static void launch_e2_kind(sg_model *m, const EvArgs &ea, long long wb, long long we, int day,
                           int slots, int n_rep, cudaStream_t st) {
  if (m->tb.kind == SG_GENERIC) {
    const size_t bytes = sizeof(int) * (size_t)m->tb.n_nodes * m->tb.n_comp;
    const bool in_smem = bytes <= kE2SmemStateMax && m->e2_dense;
    cudaKernel_t k = m->jit.k[in_smem ? JitKernels::kE2Smem : JitKernels::kE2];
    if (in_smem)
      cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kE2SmemStateMax);
    SgTables tb = m->tb;
    EvArgs a = ea;
    const int64_t *wev = m->wave_ev, *woff = m->wave_off;
    long long b = wb, e = we;
    int dd = day, sl = slots;
    void *args[] = {&tb, &a, &wev, &b, &e, &woff, &dd, &sl};
    launch_jit(k, (unsigned)n_rep, kE2Block, in_smem ? bytes : 0, st, args, true);
    return;
  }
  switch (m->tb.kind) {
    case SG_SIR: launch_e2<SG_SIR>(m, ea, wb, we, day, slots, n_rep, st); break;
    case SG_SIS: launch_e2<SG_SIS>(m, ea, wb, we, day, slots, n_rep, st); break;
    case SG_SISE: launch_e2<SG_SISE>(m, ea, wb, we, day, slots, n_rep, st); break;
    case SG_SISE_SP: launch_e2<SG_SISE_SP>(m, ea, wb, we, day, slots, n_rep, st); break;
    default: launch_e2<SG_SISE3>(m, ea, wb, we, day, slots, n_rep, st); break;
  }
}

static void fill_error(sg_error *err, int code, int rep, int node, int day, int64_t ev) {
  if (!err) return;
  err->code = code;
  err->rep = rep;
  err->node = node;
  err->day = day;
  err->event = ev;
}

// Everything one run puts on the stream after the host set-up: counters and
// cursors cleared, initial state copied, then the day loop (day kernels and
// E2 kernels).  Returns the number of kernels and E2 waves enqueued.
static void enqueue_run(sg_model *m, const DayArgs &da0, const EvArgs &ea0, int32_t days,
                        int32_t t0, int32_t t_end, int32_t slots, int32_t n_rep, int32_t n_tspan,
                        const int32_t *d_u0, const double *d_v0, int32_t *d_U, double *d_V,
                        cudaStream_t st, long long *launches_out, int32_t *waves_out) {
  const SgTables &tb = m->tb;
  const Plan &P = m->plan;
  const int C = tb.n_comp, NV = tb.n_v, Nn = tb.n_nodes;
  const long long per_rep_u = (long long)Nn * C, per_rep_v = (long long)Nn * NV;
  long long launches = 0;
  int32_t waves = 0;
  cudaMemsetAsync(m->err.p, 0, sizeof(SgDevError), st);
  cudaMemsetAsync(m->cnt.p, 0, sizeof(SgCounters), st);
  cudaMemsetAsync(m->e1_cur.p, 0, sizeof(int32_t) * (size_t)std::max(1, Nn * n_rep), st);
  if (da0.npb > kDayBlock && da0.ev.e1_node_off && Nn > 0) {
    // the sparse schedule's per-unit day of the next E1 event
    const long long units = (long long)Nn * n_rep;
    const unsigned g = (unsigned)std::min<long long>(4096, (units + 255) / 256);
    k_e1_next_init<<<std::max(1u, g), 256, 0, st>>>(da0.ev.e1_node_off, da0.ev.e1_day, Nn,
                                                     n_rep, da0.slots, m->e1_next.p);
    ++launches;
  }
  cudaMemsetAsync(m->e2_done.p, 0, sizeof(int32_t) * (size_t)n_rep, st);
  if (Nn > 0) {
    const long long nthreads = per_rep_u * n_rep + per_rep_v * n_rep;
    const unsigned g = (unsigned)std::min<long long>(4096, (nthreads + 255) / 256);
    k_init<<<std::max(1u, g), 256, 0, st>>>(d_u0, NV ? d_v0 : nullptr, m->u.p,
                                            NV ? m->v.p : nullptr, da0.U, NV ? da0.V : nullptr,
                                            per_rep_u, per_rep_v, n_tspan, n_rep);
    ++launches;
    if (da0.out.prev)
      cudaMemsetAsync(da0.out.prev, 0, sizeof(unsigned long long) * 4 * (size_t)n_rep * n_tspan,
                      st);
    if (da0.out.prev || da0.out.u_nnz > 0 || da0.out.v_nnz > 0) {
      const long long units = (long long)Nn * n_rep;
      const unsigned g0 = (unsigned)((units + 255) / 256);
      switch (tb.kind) {
        case SG_GENERIC: {
          const int32_t *pu0 = d_u0;
          const double *pv0 = nullptr;
          int nn = Nn, nr = n_rep, mm = n_tspan;
          OutDev o = da0.out;
          void *args[] = {&pu0, &pv0, &nn, &nr, &mm, &o};
          launch_jit(m->jit.k[JitKernels::kRecord0], g0, 256, 0, st, args, false);
          break;
        }
        case SG_SIR: k_record0<3, 0><<<g0, 256, 0, st>>>(d_u0, d_v0, Nn, n_rep, n_tspan, da0.out); break;
        case SG_SIS: k_record0<2, 0><<<g0, 256, 0, st>>>(d_u0, d_v0, Nn, n_rep, n_tspan, da0.out); break;
        case SG_SISE3: k_record0<6, 1><<<g0, 256, 0, st>>>(d_u0, d_v0, Nn, n_rep, n_tspan, da0.out); break;
        default: k_record0<2, 1><<<g0, 256, 0, st>>>(d_u0, d_v0, Nn, n_rep, n_tspan, da0.out); break;
      }
      ++launches;
    }
    if (da0.aem_tau) {
      const long long n = (long long)Nn * n_rep * tb.n_trans;
      const unsigned ga = (unsigned)std::min<long long>(4096, (n + 255) / 256);
      k_aem_init<<<std::max(1u, ga), 256, 0, st>>>(da0.aem_a, da0.aem_tau, da0.aem_cnt, n);
      ++launches;
    }
  }
  DayArgs da = da0;
  EvArgs ea = ea0;
  if (Nn > 0 && days > 0 && tb.kind == SG_SISE_SP) {
    // Coupled post time step: it reads other nodes' phi and sizes, so every
    // day ends with its own kernel after the day's events (phi in two
    // buffers, old and new).
    double *vc = m->v.p, *vn = m->v2.p;
    PtsSpArgs pa;
    pa.u = m->u.p;
    pa.ldata = m->ldata.p;
    pa.nb_ptr = m->has_nb ? m->nb_ptr.p : nullptr;
    pa.nb_idx = m->nb_idx.p;
    pa.nb_dist = m->nb_dist.p;
    pa.U = da0.U;
    pa.V = da0.V;
    pa.out = da0.out;
    pa.rec = m->rec.p;
    pa.t0 = t0;
    pa.M = n_tspan;
    pa.n_rep = n_rep;
    pa.rep0 = da0.rep0;
    pa.err = m->err.p;
    const long long units = (long long)Nn * n_rep;
    for (int32_t d = 0; d < days; ++d) {
      const int32_t T = t0 + 1 + d;
      da.v = vc;
      da.T_begin = T;
      da.T_end = T + 1;
      da.finish_first = 0;
      da.finish_last = 0;
      {
        LaunchTimer lt(m, st, 0);
        launch_days_kind(m, da, st);
      }
      ++launches;
      if (P.day_has_e2[d]) {
        ea.day = T;
        const long long b0 = (long long)d * slots, b1 = b0 + slots;
        const long long wb = P.e2_wave_off[b0], we = P.e2_wave_off[b1];
        LaunchTimer lt(m, st, 2);
        launch_e2_kind(m, ea, wb, we, d, slots, n_rep, st);
        ++launches;
        waves += (int32_t)(we - wb);
      }
      pa.v_old = vc;
      pa.v_new = vn;
      pa.T = T;
      {
        LaunchTimer lt(m, st, 0);
        launch_pdl(k_pts_sp, (unsigned)((units + 127) / 128), 128, 0, st, tb, pa);
      }
      ++launches;
      std::swap(vc, vn);
    }
  } else if (Nn > 0 && days > 0 && m->emu_on) {
    // One day at a time: finish the previous day, emulator features and MLP
    // for every node, sampling, then the day kernel (SSA only for the nodes
    // outside the emulator's range) and the day's external transfers.
    const long long units = (long long)Nn * n_rep;
    EmuParams ep{};
    for (int i = 0; i < 11; ++i) ep.gdata[i] = tb.gdata[i];
    ep.max_herd = m->emu_max_herd;
    ep.phi_lo = m->emu_phi_lo;
    ep.phi_hi = m->emu_phi_hi;
    ep.min_rate = m->emu_min_rate;
    const unsigned gu = (unsigned)std::max<long long>(1, std::min<long long>(16384, (units + 255) / 256));
    const unsigned gw = (unsigned)std::max<long long>(1, std::min<long long>(1 << 20, (units * 32 + 255) / 256));
    EmuChainWeights cw{};
    if (m->emu_fp8) {
      // weight images of the E4M3 chain, from the caller's current weights
      cw.W0 = m->emu_W[0];
      for (int l = 0; l < 3; ++l) {
        cw.W8[l] = m->emu_W8[l];
        cw.wscale[l] = m->emu_wscale[l];
        cw.act_scale[l] = m->emu_act_scale[l];
      }
      for (int l = 0; l < 4; ++l) cw.b[l] = m->emu_b[l];
      LaunchTimer lt(m, st, 3);
      emu_chain_images(cw, m->emu_img.p, m->emu_hvec.p, st);
      launches += 5;
    }
    bool pending = false;
    for (int32_t d = 0; d < days; ++d) {
      const int32_t T = t0 + 1 + d;
      if (pending) {
        da.T_begin = T;
        da.T_end = T;
        da.finish_first = 1;
        da.finish_last = 0;
        da.emu = nullptr;
        launch_days_kind(m, da, st);
        ++launches;
      }
      const bool split = m->emu_fp8 && m->side_st != nullptr;
      if (m->emu_fp8) {
        // the persistent E4M3 chain: features, flags and layer 1; then the
        // SSA of the units outside the emulator's range on the side stream,
        // beside layers 2 and 3 and layer 4 with the sampler
        {
          LaunchTimer lt(m, st, 3);
          emu_chain_day(cw, m->emu_img.p, m->emu_hvec.p, m->emu_h8a.p, m->emu_h8b.p, m->u.p,
                        m->v.p, ep, units, Nn, da.k0, da.k1, T, m->emu_flag.p, m->emu_delta.p,
                        st, 0);
        }
        if (split) {
          cudaEventRecord(m->side_fork, st);
          cudaStreamWaitEvent(m->side_st, m->side_fork, 0);
          DayArgs db = da;
          db.T_begin = T;
          db.T_end = T + 1;
          db.finish_first = 0;
          db.finish_last = P.day_has_e2[d] != 0 ? 0 : 1;
          db.emu = nullptr;
          db.emu_flag = m->emu_flag.p;
          db.emu_part = 1;
          {
            LaunchTimer lt(m, m->side_st, 0);
            launch_days_kind(m, db, m->side_st);
          }
          cudaEventRecord(m->side_join, m->side_st);
          ++launches;
        }
        {
          LaunchTimer lt(m, st, 3);
          emu_chain_day(cw, m->emu_img.p, m->emu_hvec.p, m->emu_h8a.p, m->emu_h8b.p, m->u.p,
                        m->v.p, ep, units, Nn, da.k0, da.k1, T, m->emu_flag.p, m->emu_delta.p,
                        st, 1);
        }
        if (split) cudaStreamWaitEvent(st, m->side_join, 0);
        launches += 4;
      } else {
        {
          LaunchTimer lt(m, st, 3);
          k_emu_features<<<gu, 256, 0, st>>>(m->u.p, m->v.p, units, ep, m->emu_feat.p,
                                             m->emu_flag.p);
        }
        const __nv_bfloat16 *in = m->emu_feat.p;
        int kin = kEmuIn;
        __nv_bfloat16 *outs[3] = {m->emu_ha.p, m->emu_hb.p, m->emu_ha.p};
        for (int l = 0; l < 4; ++l) {
          GemmArgs g{};
          g.A = in;
          g.lda = kin;
          g.Bt = m->emu_W[l];
          g.ldb = kin;
          g.M = (int)units;
          g.N = l < 3 ? kEmuHidden : kEmuOut;
          g.K = kin;
          g.bias = m->emu_b[l];
          g.act = l < 3 ? 1 : 0;
          g.C32 = l < 3 ? nullptr : m->emu_logits.p;
          g.ldc32 = kEmuOut;
          g.C16 = l < 3 ? outs[l] : nullptr;
          g.ldc16 = kEmuHidden;
          g.err = nullptr;
          {
            LaunchTimer lt(m, st, 3);
            gemm_bf16(g, st);
          }
          ++launches;
          if (l < 3) {
            in = outs[l];
            kin = kEmuHidden;
          }
        }
        {
          LaunchTimer lt(m, st, 3);
          k_emu_sample<<<gw, 256, 0, st>>>(m->emu_logits.p, kEmuOut, m->u.p, m->emu_flag.p,
                                           units, Nn, da.k0, da.k1, T, m->emu_delta.p);
        }
        launches += 2;
      }
      const bool e2_today = P.day_has_e2[d] != 0;
      da.T_begin = T;
      da.T_end = T + 1;
      da.finish_first = 0;
      da.finish_last = e2_today ? 0 : 1;
      da.emu = m->emu_delta.p;
      da.emu_part = split ? 2 : 0;  // split: the SSA part ran on the side stream
      {
        LaunchTimer lt(m, st, 0);
        launch_days_kind(m, da, st);
      }
      da.emu_part = 0;
      ++launches;
      if (e2_today) {
        ea.day = T;
        const long long b0 = (long long)d * slots, b1 = b0 + slots;
        const long long wb = P.e2_wave_off[b0], we = P.e2_wave_off[b1];
        LaunchTimer lt(m, st, 2);
        launch_e2_kind(m, ea, wb, we, d, slots, n_rep, st);
        ++launches;
        waves += (int32_t)(we - wb);
      }
      pending = e2_today;
    }
    if (pending) {
      da.T_begin = t_end + 1;
      da.T_end = t_end + 1;
      da.finish_first = 1;
      da.finish_last = 0;
      da.emu = nullptr;
      launch_days_kind(m, da, st);
      ++launches;
    }
  } else if (Nn > 0 && days > 0 && m->persistent && persistent_fits(m, da)) {
    // the whole run in one persistent launch
    DayArgs dp = da;
    dp.T_begin = t0 + 1;
    dp.T_end = t_end + 1;
    dp.finish_first = 0;
    dp.finish_last = 1;
    dp.grid_bar = m->grid_bar.p;
    dp.n_blocks = (int32_t)std::max<long long>(1, ((long long)Nn * n_rep + da.npb - 1) / da.npb);
    cudaMemsetAsync(m->grid_bar.p, 0, 2 * sizeof(unsigned int), st);
    {
      LaunchTimer lt(m, st, 0);
      launch_days_persistent(m, dp, st);
    }
    ++launches;
    for (int32_t d = 0; d < days; ++d)
      waves += (int32_t)(P.e2_wave_off[(long long)(d + 1) * slots] -
                         P.e2_wave_off[(long long)d * slots]);
  } else if (Nn > 0 && days > 0 && da.npb > kDayBlock && da.npb % Nn == 0 &&
             m->tb.kind != SG_GENERIC && !da.aem_tau) {
    // sparse schedule with whole replicates per block: every day in one
    // launch, each block running its replicates' external transfers itself
    // (no block waits for another)
    DayArgs dr = da;
    dr.T_begin = t0 + 1;
    dr.T_end = t_end + 1;
    dr.finish_first = 0;
    dr.finish_last = 1;
    dr.e2_inblock = 1;
    {
      LaunchTimer lt(m, st, 0);
      launch_days_kind(m, dr, st);
    }
    ++launches;
    for (int32_t d = 0; d < days; ++d)
      waves += (int32_t)(P.e2_wave_off[(long long)(d + 1) * slots] -
                         P.e2_wave_off[(long long)d * slots]);
  } else if (Nn > 0 && days > 0) {
    bool pending = false;  // the previous unit step still needs finishing
    int32_t d = 0;
    while (d < days) {
      // days d .. last run in one kernel; only `last` may have external
      // transfers, which need every node's state first
      int32_t last = d;
      while (last < days - 1 && !P.day_has_e2[last]) ++last;
      const bool e2_today = P.day_has_e2[last] != 0;
      da.T_begin = t0 + 1 + d;
      da.T_end = t0 + 1 + last + 1;
      da.finish_first = pending ? 1 : 0;
      da.finish_last = e2_today ? 0 : 1;
      const bool fused = e2_today && m->fuse_e2;
      da.e2_done = fused ? m->e2_done.p : nullptr;
      if (fused) {
        const long long b0 = (long long)last * slots, b1 = b0 + slots;
        da.e2_wb = P.e2_wave_off[b0];
        da.e2_we = P.e2_wave_off[b1];
        da.e2_day_index = last;
        waves += (int32_t)(da.e2_we - da.e2_wb);
      }
      {
        LaunchTimer lt(m, st, 0);
        launch_days_kind(m, da, st);
      }
      ++launches;
      da.e2_done = nullptr;
      if (e2_today && !fused) {
        ea.day = t0 + 1 + last;
        const long long b0 = (long long)last * slots, b1 = b0 + slots;
        const long long wb = P.e2_wave_off[b0], we = P.e2_wave_off[b1];
        LaunchTimer lt(m, st, 2);
        launch_e2_kind(m, ea, wb, we, last, slots, n_rep, st);
        ++launches;
        waves += (int32_t)(we - wb);
      }
      pending = e2_today;
      d = last + 1;
    }
    if (pending) {
      da.T_begin = t_end + 1;
      da.T_end = t_end + 1;
      da.finish_first = 1;
      da.finish_last = 0;
      {
        LaunchTimer lt(m, st, 0);
        launch_days_kind(m, da, st);
      }
      ++launches;
    }
  }
  *launches_out = launches;
  *waves_out = waves;
}

extern "C" int sg_run(sg_model *m, const int32_t *tspan, int32_t n_tspan, uint64_t seed,
                      int32_t n_rep, const int32_t *d_u0, const double *d_v0, int32_t *d_U,
                      double *d_V, void *stream, sg_stats *stats, sg_error *err) {
  fill_error(err, 0, -1, -1, -1, -1);
  if (stats) std::memset(stats, 0, sizeof *stats);
  if (!m || !tspan || n_tspan < 1 || n_rep < 1 || n_rep >= (1 << 24)) return SG_ERR_ARG;
  for (int i = 1; i < n_tspan; ++i)
    if (tspan[i] <= tspan[i - 1]) return SG_ERR_ARG;
  const SgTables &tb = m->tb;
  const int C = tb.n_comp, NV = tb.n_v, Nn = tb.n_nodes;
  if (Nn > 0 && (!d_u0 || (NV > 0 && !d_v0))) return SG_ERR_ARG;
  if (Nn > 0 && m->out_dense && (!d_U || (NV > 0 && !d_V))) return SG_ERR_ARG;
  if (m->out_cols >= 0 && m->out_cols != n_tspan) return SG_ERR_ARG;
  // a shard (sg_set_replicate_range) runs global replicates rep0 .. rep0 +
  // n_rep - 1 of a job with rep_total; a whole job needs every event's
  // replicate below n_rep
  const int32_t rep_total = m->rep_total > 0 ? m->rep_total : n_rep;
  if (m->rep0 + (long long)n_rep > rep_total) return SG_ERR_ARG;
  if (m->ev.per_rep && m->ev.max_rep >= rep_total) {
    fill_error(err, SG_ERR_ARG, m->ev.max_rep, -1, -1, -1);
    return SG_ERR_ARG;
  }
  if (m->rep0 > 0 && m->emu_on) return SG_ERR_ARG;  // the emulator runs whole jobs only
  if (tb.kind == SG_GENERIC) {
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != m->jit.device) return SG_ERR_ARG;  // kernels loaded on another device
  }
  cudaStream_t st = (cudaStream_t)stream;
  const auto host_t0 = std::chrono::steady_clock::now();
  const int32_t t0 = tspan[0], t_end = tspan[n_tspan - 1];
  const int32_t days = t_end - t0;
  const int32_t slots = m->ev.per_rep ? n_rep : 1;
  int rc = ensure_plan(m, t0, t_end, slots);
  if (rc) return rc;
  const double plan_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - host_t0).count();
  const Plan &P = m->plan;
  m->e2_dense = days > 0 && P.n_e2 * 16 >= (long long)days * slots * Nn;

  const long long per_rep_u = (long long)Nn * C, per_rep_v = (long long)Nn * NV;
  if ((rc = m->u.ensure((size_t)(per_rep_u * n_rep))) ||
      (rc = m->v.ensure((size_t)std::max<long long>(1, per_rep_v * n_rep))) ||
      (rc = m->e1_cur.ensure((size_t)std::max(1, Nn * n_rep))) ||
      (rc = m->e1_next.ensure((size_t)std::max(1, Nn * n_rep))) ||
      (rc = m->rec.ensure((size_t)days + 1)))
    return rc;
  if (tb.kind == SG_SISE_SP && (rc = m->v2.ensure((size_t)std::max<long long>(1, per_rep_v * n_rep))))
    return rc;
  if ((rc = m->e2_done.ensure((size_t)n_rep)) || (rc = m->grid_bar.ensure(2))) return rc;
  const bool aem = m->solver == SG_SOLVER_AEM;
  if (aem && m->emu_on) return SG_ERR_ARG;  // the emulator replaces direct-method days only
  if (aem) {
    const size_t nch = (size_t)std::max<long long>(1, (long long)Nn * n_rep * tb.n_trans);
    if ((rc = m->aem_a.ensure(nch)) || (rc = m->aem_tau.ensure(nch)) ||
        (rc = m->aem_cnt.ensure(nch)))
      return rc;
  }
  if (m->emu_on) {
    const size_t units = (size_t)Nn * n_rep;
    const size_t tiles = (units + 127) / 128;
    if ((rc = m->emu_flag.ensure(units)) || (rc = m->emu_delta.ensure(units * 4)) ||
        (rc = gemm_prepare()))
      return rc;
    if (m->emu_fp8) {
      if ((rc = m->emu_h8a.ensure(tiles * kEmuTileBytes)) ||
          (rc = m->emu_h8b.ensure(tiles * kEmuTileBytes)) ||
          (rc = m->emu_img.ensure(kEmuImgBytes)) || (rc = m->emu_hvec.ensure(kEmuHeadVecFloats)))
        return rc;
      if (!m->side_st) {
        // side stream of the emulator day; without it the day runs in order
        if (cudaStreamCreateWithFlags(&m->side_st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&m->side_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&m->side_join, cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          if (m->side_st) cudaStreamDestroy(m->side_st);
          if (m->side_fork) cudaEventDestroy(m->side_fork);
          if (m->side_join) cudaEventDestroy(m->side_join);
          m->side_st = nullptr;
          m->side_fork = m->side_join = nullptr;
        }
      }
    } else if ((rc = m->emu_feat.ensure(units * kEmuIn)) ||
               (rc = m->emu_ha.ensure(units * kEmuHidden)) ||
               (rc = m->emu_hb.ensure(units * kEmuHidden)) ||
               (rc = m->emu_logits.ensure(units * kEmuOut))) {
      return rc;
    }
  }
  // tspan slot of every unit time, uploaded when it changes
  std::vector<int32_t> rec(days + 1, -1);
  for (int i = 0; i < n_tspan; ++i) rec[tspan[i] - t0] = i;
  if (rec != m->rec_host) {
    if (cudaMemcpy(m->rec.p, rec.data(), rec.size() * sizeof(int32_t),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return SG_ERR_CUDA;
    }
    m->rec_host.swap(rec);
    m->graph_ok = false;
  }

  const EvDev evd{m->e_type, m->e_select, m->e_shift, m->e_node, m->e_dest,
                  m->e_n,    m->e_prop,   m->e_index, m->e1_day,
                  P.n_e1 > 0 ? m->e1_node_off : nullptr};
  DayArgs da{};
  da.u = m->u.p;
  da.v = m->v.p;
  da.ldata = m->ldata.p;
  da.U = d_U;
  da.V = d_V;
  da.rec = m->rec.p;
  da.e1_cur = m->e1_cur.p;
  da.e1_next = m->e1_next.p;
  da.ev = evd;
  da.t0 = t0;
  da.M = n_tspan;
  da.n_rep = n_rep;
  da.slots = slots;
  da.rep0 = m->rep0;
  da.heavy_after = m->heavy_after >= 0 ? m->heavy_after : 2;
  da.npb = m->npb > 0 ? m->npb : default_npb((long long)Nn * n_rep);
  // the sparse-activity schedule (nodes_per_block > kDayBlock) is for the
  // direct method on the built-in kinds with the day / E2 kernel pair;
  // elsewhere such a split falls back to full thread-per-node blocks
  const bool sparse_ok = !aem && !m->emu_on && !m->persistent &&
                         (tb.kind == SG_SIR || tb.kind == SG_SIS || tb.kind == SG_SISE ||
                          tb.kind == SG_SISE3);
  if (da.npb > kDayBlock && !sparse_ok) da.npb = kDayBlock;
  if (m->npb <= 0 && sparse_ok) {
    // untuned: more units than two full thread-per-node blocks per SM take
    // the sparse-activity schedule: one replicate per block when there are
    // at least as many replicates as SMs (every day in one launch), else
    // the units spread over two blocks per SM
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    const long long units = (long long)Nn * n_rep;
    if (units > 2LL * kDayBlock * sms) {
      const bool whole = n_rep >= sms && Nn > kDayBlock;
      da.npb = whole ? Nn : (int32_t)((units + 2LL * sms - 1) / (2LL * sms));
      if (m->heavy_after < 0) da.heavy_after = whole ? 32 : 8;
    }
  }
  {
    // a unit with no infected animal and phi == +0 has an empty day only
    // when every parameter is finite (0 times inf or NaN is not 0)
    bool finite = true;
    for (int i = 0; i < SG_MAX_GDATA; ++i) finite = finite && std::isfinite(tb.gdata[i]);
    da.quiet = finite ? 1 : 0;
  }
  da.k0 = (uint32_t)seed;
  da.k1 = (uint32_t)(seed >> 32);
  da.err = m->err.p;
  da.cnt = m->cnt.p;
  da.T_begin = da.T_end = da.finish_first = da.finish_last = 0;
  da.emu = nullptr;
  if (!m->out_dense) {
    da.U = nullptr;
    da.V = nullptr;
  }
  da.out = m->out;
  da.wave_ev = m->wave_ev;
  da.wave_off = m->wave_off;
  da.e2_wb = da.e2_we = 0;
  da.e2_day_index = 0;
  da.e2_done = nullptr;
  da.grid_bar = nullptr;
  da.n_blocks = 0;
  da.e2_inblock = 0;
  da.aem_a = aem ? m->aem_a.p : nullptr;
  da.aem_tau = aem ? m->aem_tau.p : nullptr;
  da.aem_cnt = aem ? m->aem_cnt.p : nullptr;

  EvArgs ea;
  ea.ev = evd;
  ea.u = m->u.p;
  ea.n_rep = n_rep;
  ea.rep0 = m->rep0;
  ea.k0 = da.k0;
  ea.k1 = da.k1;
  ea.day = 0;
  ea.err = m->err.p;
  ea.cnt = m->cnt.p;

  m->ev_used = 0;
  m->ev_kind.clear();
  long long launches = 0;
  int32_t waves = 0;
  // The whole run is one CUDA graph, captured the first time and replayed
  // while nothing it depends on changes (not on the legacy default stream,
  // which cannot be captured, and not while kernels are being timed).
  const bool use_graph = m->graphs && st != nullptr && !m->timing;
  const GraphKey key{d_u0,
                     d_v0,
                     d_U,
                     d_V,
                     m->u.p,
                     m->v.p,
                     m->e1_cur.p,
                     m->rec.p,
                     m->emu_on ? (const void *)m->emu_delta.p : nullptr,
                     seed,
                     n_rep,
                     n_tspan,
                     t0,
                     t_end,
                     da.npb,
                     da.heavy_after,
                     m->rep0,
                     (m->plan_version * 1000003ull + (m->emu_on ? m->emu_version + 1 : 0)) *
                             1000033ull +
                         m->nb_version * 7ull + (uint64_t)(uintptr_t)m->v2.p +
                         ((uint64_t)(uintptr_t)m->e1_next.p << 7) +
                         m->out_version * 0x100000001b3ull +
                         ((uint64_t)(uintptr_t)m->e2_done.p << 3) + (m->fuse_e2 ? 5 : 0) +
                         ((uint64_t)(uintptr_t)m->grid_bar.p << 5) + (m->persistent ? 11 : 0) +
                         (aem ? 0x9e3779b97f4a7c15ull ^ (uint64_t)(uintptr_t)m->aem_tau.p ^
                                    ((uint64_t)(uintptr_t)m->aem_a.p << 1) ^
                                    ((uint64_t)(uintptr_t)m->aem_cnt.p << 2)
                              : 0)};
  if (use_graph) {
    if (!(m->graph_ok && m->graph_key == key)) {
      if (m->graph_exec) {
        cudaGraphExecDestroy(m->graph_exec);
        m->graph_exec = nullptr;
      }
      m->graph_ok = false;
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return SG_ERR_CUDA;
      }
      enqueue_run(m, da, ea, days, t0, t_end, slots, n_rep, n_tspan, d_u0, d_v0, d_U, d_V,
                  st, &launches, &waves);
      if (cudaStreamEndCapture(st, &g) != cudaSuccess ||
          cudaGraphInstantiate(&m->graph_exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        m->graph_exec = nullptr;
        return SG_ERR_CUDA;
      }
      cudaGraphDestroy(g);
      m->graph_key = key;
      m->graph_launches = launches;
      m->graph_waves = waves;
      m->graph_ok = true;
    }
    launches = m->graph_launches;
    waves = m->graph_waves;
    if (cudaGraphLaunch(m->graph_exec, st) != cudaSuccess) {
      cudaGetLastError();
      return SG_ERR_CUDA;
    }
  } else {
    enqueue_run(m, da, ea, days, t0, t_end, slots, n_rep, n_tspan, d_u0, d_v0, d_U, d_V, st,
                &launches, &waves);
  }
  if (cudaMemcpyAsync(m->h_err, m->err.p, sizeof(SgDevError), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(m->h_cnt, m->cnt.p, sizeof(SgCounters), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    fill_error(err, SG_ERR_CUDA, -1, -1, -1, -1);
    return SG_ERR_CUDA;
  }
  if (stats) {
    for (size_t i = 0; i < m->ev_kind.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, m->evpool[2 * i], m->evpool[2 * i + 1]);
      const int k = m->ev_kind[i];
      (k == 0 ? stats->ms_ssa : k == 1 ? stats->ms_e1 : k == 2 ? stats->ms_e2 : stats->ms_mlp) += ms;
      ++(k == 0 ? stats->launches_ssa
                : k == 1 ? stats->launches_e1 : k == 2 ? stats->launches_e2 : stats->launches_mlp);
    }
    cudaGetLastError();
    stats->draws = (int64_t)m->h_cnt->draws;
    stats->reactions = (int64_t)m->h_cnt->reactions;
    stats->events_applied = (int64_t)m->h_cnt->events;
    stats->node_days = (int64_t)Nn * n_rep * days;
    // the sparse schedule evaluates the rates of non-quiescent node-days only
    stats->node_days_rated =
        da.npb > kDayBlock ? (int64_t)m->h_cnt->rated : stats->node_days;
    stats->kernel_launches = launches;
    stats->e2_waves = waves;
    stats->days = days;
    stats->ms_host_plan = plan_ms;
    stats->ms_host_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - host_t0)
            .count();
  }
  const SgDevError &e = *m->h_err;
  if (e.code) {
    fill_error(err, e.code, e.rep, e.node, e.day, e.event);
    return e.code;
  }
  if (m->emu_on) {
    rc = gemm_check(st);
    if (rc) {
      fill_error(err, rc, -1, -1, -1, -1);
      return rc;
    }
  }
  return SG_OK;
}

extern "C" int sg_run_host(sg_model *m, const int32_t *tspan, int32_t n_tspan, uint64_t seed,
                           int32_t n_rep, const int32_t *u0, const double *v0, int32_t *U,
                           double *V, void *stream, sg_stats *stats, sg_error *err) {
  if (!m || !tspan || n_tspan < 1 || n_rep < 1) return SG_ERR_ARG;
  const SgTables &tb = m->tb;
  const size_t nu = (size_t)n_rep * tb.n_nodes * tb.n_comp;
  const size_t nv = (size_t)n_rep * tb.n_nodes * tb.n_v;
  const size_t M = (size_t)n_tspan;
  const bool dense = m->out_dense;
  if (tb.n_nodes > 0 && (!u0 || (tb.n_v > 0 && !v0))) return SG_ERR_ARG;
  if (tb.n_nodes > 0 && dense && (!U || (tb.n_v > 0 && !V))) return SG_ERR_ARG;
  int rc;
  if ((rc = m->hu0.ensure(nu)) || (rc = m->hv0.ensure(std::max<size_t>(1, nv))) ||
      (dense && ((rc = m->hU.ensure(nu * M)) || (rc = m->hV.ensure(std::max<size_t>(1, nv * M))))))
    return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((nu && cudaMemcpyAsync(m->hu0.p, u0, nu * sizeof(int32_t), cudaMemcpyHostToDevice, st) !=
                 cudaSuccess) ||
      (nv && cudaMemcpyAsync(m->hv0.p, v0, nv * sizeof(double), cudaMemcpyHostToDevice, st) !=
                 cudaSuccess)) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  rc = sg_run(m, tspan, n_tspan, seed, n_rep, m->hu0.p, nv ? m->hv0.p : nullptr,
              dense ? m->hU.p : nullptr, dense && nv ? m->hV.p : nullptr, stream, stats, err);
  if (rc) return rc;
  if ((dense && nu &&
       cudaMemcpyAsync(U, m->hU.p, nu * M * sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
           cudaSuccess) ||
      (dense && nv &&
       cudaMemcpyAsync(V, m->hV.p, nv * M * sizeof(double), cudaMemcpyDeviceToHost, st) !=
           cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  return SG_OK;
}

static unsigned grid_for(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>(8192, (n + 255) / 256));
}

extern "C" int sg_philox_batch(const uint32_t *d_ctr, uint64_t key, uint32_t *d_out, int64_t n,
                               void *stream) {
  if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n) k_philox_batch<<<grid_for(n), 256, 0, st>>>(d_ctr, (uint32_t)key, (uint32_t)(key >> 32),
                                                     d_out, n);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  return SG_OK;
}

extern "C" int sg_log_batch(const double *d_x, double *d_y, int64_t n, void *stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_y))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n) k_log_batch<<<grid_for(n), 256, 0, st>>>(d_x, d_y, n);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  return SG_OK;
}

extern "C" int sg_u01_batch(const uint32_t *d_w, double *d_y, int64_t n, void *stream) {
  if (n < 0 || (n > 0 && (!d_w || !d_y))) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n) k_u01_batch<<<grid_for(n), 256, 0, st>>>(d_w, d_y, n);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  return SG_OK;
}

extern "C" int sg_set_kernel_timing(sg_model *m, int enable) {
  if (!m) return SG_ERR_ARG;
  m->timing = enable != 0;
  return SG_OK;
}

extern "C" int sg_fp64_fma_probe(int32_t iters, double *tflops, void *stream) {
  if (iters < 1 || !tflops) return SG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  const int threads = 256, blocks = sms * 8;
  double *out = nullptr;
  cudaEvent_t e0, e1;
  if (cudaMallocAsync(&out, sizeof(double) * threads * blocks, st) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_NOMEM;
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fp64_fma<<<blocks, threads, 0, st>>>(out, 16);  // warm-up
  cudaEventRecord(e0, st);
  k_fp64_fma<<<blocks, threads, 0, st>>>(out, iters);
  cudaEventRecord(e1, st);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaFreeAsync(out, st);
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
  const double flops = 2.0 * 8.0 * (double)iters * threads * blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SG_OK;
}

// ---------------------------------------------------------------------------
// sg_run_noalloc: the event-free run with its working memory in a fixed
// device array instead of allocated buffers (see include/siminf_gpu.h for
// which callers need this and its limits).
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[SG_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_base[kNoallocMaxDevices] = {};

// The array's device address for the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device, with that device current.
int noalloc_base(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SG_ERR_CUDA;
    }
    g_noalloc_base[dev] = (unsigned char *)p;
  }
  *out = g_noalloc_base[dev];
  return SG_OK;
}

constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// rec[i] = tspan slot of unit time t0 + i, or -1
__global__ void k_noalloc_rec(const int32_t *tspan, int32_t n_tspan, int32_t *rec, int32_t days) {
  const int32_t t0 = tspan[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= days; i += gridDim.x * blockDim.x)
    rec[i] = -1;
  __syncthreads();
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < n_tspan; i += blockDim.x) rec[tspan[i] - t0] = i;
}

}  // namespace

extern "C" int sg_run_noalloc(const sg_desc *d, const double *d_ldata, const int32_t *tspan,
                              int32_t n_tspan, uint64_t seed, int32_t n_rep,
                              const int32_t *d_u0, const double *d_v0, int32_t *d_U,
                              double *d_V, void *stream, sg_stats *stats, sg_error *err) {
  fill_error(err, 0, -1, -1, -1, -1);
  if (stats) std::memset(stats, 0, sizeof *stats);
  if (!d || !tspan || n_tspan < 1 || n_rep < 1 || n_rep >= (1 << 24)) return SG_ERR_ARG;
  const int k = d->kind;
  if (k < SG_SIR || k > SG_SISE3) return SG_ERR_ARG;  // coupled kinds need neighbour lists
  if (d->n_nodes < 0 || d->n_comp != kKindComp[k] || d->n_trans != kKindTrans[k] ||
      d->n_v != kKindNv[k] || d->n_gdata < kKindGdata[k] || d->n_gdata > SG_MAX_GDATA ||
      d->n_ldata < kKindLdata[k] || !d->S || !d->G || (d->n_gdata > 0 && !d->gdata) ||
      (d->n_ldata > 0 && d->n_nodes > 0 && !d_ldata))
    return SG_ERR_ARG;
  for (int i = 1; i < n_tspan; ++i)
    if (tspan[i] <= tspan[i - 1]) return SG_ERR_ARG;
  const int C = d->n_comp, T = d->n_trans, NV = d->n_v, Nn = d->n_nodes;
  if (Nn > 0 && (!d_u0 || !d_U || (NV > 0 && (!d_v0 || !d_V)))) return SG_ERR_ARG;

  // tables passed by value to the kernels (no allocation)
  SgTables tb;
  std::memset(&tb, 0, sizeof tb);
  tb.kind = k;
  tb.n_nodes = Nn;
  tb.n_comp = C;
  tb.n_trans = T;
  tb.n_v = NV;
  tb.n_ldata = d->n_ldata;
  for (int j = 0; j < T; ++j) {
    for (int p = 0; p < C; ++p) {
      const int sv = d->S[(size_t)j * C + p];
      if (sv < -127 || sv > 127) return SG_ERR_ARG;
      tb.S[j][p] = (int8_t)sv;
    }
    uint32_t dep = 0;
    for (int kk = 0; kk < T; ++kk)
      if (d->G[(size_t)j * T + kk] != 0) dep |= 1u << kk;
    tb.dep[j] = dep;
  }
  for (int i = 0; i < d->n_gdata; ++i) tb.gdata[i] = d->gdata[i];

  // scratch layout: error word | counters | tspan | rec | u | v
  const int32_t t0 = tspan[0], t_end = tspan[n_tspan - 1], days = t_end - t0;
  const size_t units = (size_t)n_rep * (size_t)Nn;
  const size_t off_cnt = 256, off_tspan = 512;
  const size_t off_rec = off_tspan + round256(sizeof(int32_t) * (size_t)n_tspan);
  const size_t off_u = off_rec + round256(sizeof(int32_t) * ((size_t)days + 1));
  const size_t off_v = off_u + round256(sizeof(int32_t) * units * C);
  const size_t need = off_v + round256(sizeof(double) * units * NV) + 512;
  if (need > SG_NOALLOC_SCRATCH_BYTES) {
    fill_error(err, SG_ERR_TOO_LARGE, -1, -1, -1, -1);
    return SG_ERR_TOO_LARGE;
  }
  unsigned char *base = nullptr;
  int rc = noalloc_base(&base);
  if (rc) {
    fill_error(err, rc, -1, -1, -1, -1);
    return rc;
  }
  SgDevError *d_err = (SgDevError *)base;
  SgCounters *d_cnt = (SgCounters *)(base + off_cnt);
  int32_t *d_tspan = (int32_t *)(base + off_tspan);
  int32_t *d_rec = (int32_t *)(base + off_rec);
  int *d_u = (int *)(base + off_u);
  double *d_v = (double *)(base + off_v);
  cudaStream_t st = (cudaStream_t)stream;

  // clear what must start at zero; the rest is overwritten before use
  if (cudaMemsetAsync(d_err, 0, sizeof(SgDevError), st) != cudaSuccess ||
      cudaMemsetAsync(d_cnt, 0, sizeof(SgCounters), st) != cudaSuccess ||
      cudaMemcpyAsync(d_tspan, tspan, sizeof(int32_t) * (size_t)n_tspan,
                      cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    fill_error(err, SG_ERR_CUDA, -1, -1, -1, -1);
    return SG_ERR_CUDA;
  }
  k_noalloc_rec<<<1, 256, 0, st>>>(d_tspan, n_tspan, d_rec, days);
  long long launches = 1;
  const long long per_rep_u = (long long)Nn * C, per_rep_v = (long long)Nn * NV;
  if (Nn > 0) {
    const long long nthreads = per_rep_u * n_rep + per_rep_v * n_rep;
    const unsigned g = (unsigned)std::min<long long>(4096, (nthreads + 255) / 256);
    k_init<<<std::max(1u, g), 256, 0, st>>>(d_u0, NV ? d_v0 : nullptr, d_u, NV ? d_v : nullptr,
                                            d_U, NV ? d_V : nullptr, per_rep_u, per_rep_v,
                                            n_tspan, n_rep);
    ++launches;
    if (days > 0) {
      DayArgs da{};
      da.u = d_u;
      da.v = d_v;
      da.ldata = d_ldata;
      da.U = d_U;
      da.V = d_V;
      da.rec = d_rec;
      da.e1_cur = nullptr;
      da.ev = EvDev{};
      da.t0 = t0;
      da.M = n_tspan;
      da.n_rep = n_rep;
      da.slots = 1;
      da.heavy_after = 2;
      da.npb = default_npb((long long)Nn * n_rep);
      da.emu = nullptr;
      da.T_begin = t0 + 1;
      da.T_end = t_end + 1;
      da.finish_first = 0;
      da.finish_last = 1;
      da.k0 = (uint32_t)seed;
      da.k1 = (uint32_t)(seed >> 32);
      da.err = d_err;
      da.cnt = d_cnt;
      da.aem_a = da.aem_tau = nullptr;
      da.aem_cnt = nullptr;
      da.wave_ev = da.wave_off = nullptr;
      da.e2_wb = da.e2_we = 0;
      da.e2_day_index = 0;
      da.e2_done = nullptr;
      da.grid_bar = nullptr;
      da.n_blocks = 0;
      da.e2_inblock = 0;
      const long long units = (long long)Nn * n_rep;
      const unsigned grid = (unsigned)std::max<long long>(1, (units + da.npb - 1) / da.npb);
      switch (k) {
        case SG_SIR: k_days<SG_SIR, false><<<grid, kDayBlock, 0, st>>>(tb, da); break;
        case SG_SIS: k_days<SG_SIS, false><<<grid, kDayBlock, 0, st>>>(tb, da); break;
        case SG_SISE: k_days<SG_SISE, false><<<grid, kDayBlock, 0, st>>>(tb, da); break;
        default: k_days<SG_SISE3, false><<<grid, kDayBlock, 0, st>>>(tb, da); break;
      }
      ++launches;
    }
  }
  SgDevError h_err;
  SgCounters h_cnt;
  if (cudaMemcpyAsync(&h_err, d_err, sizeof h_err, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&h_cnt, d_cnt, sizeof h_cnt, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    fill_error(err, SG_ERR_CUDA, -1, -1, -1, -1);
    return SG_ERR_CUDA;
  }
  if (stats) {
    stats->reactions = (int64_t)h_cnt.reactions;
    stats->draws = (int64_t)h_cnt.draws;
    stats->node_days = (int64_t)Nn * n_rep * days;
    stats->node_days_rated = stats->node_days;
    stats->kernel_launches = launches;
    stats->days = days;
  }
  if (h_err.code) {
    fill_error(err, h_err.code, h_err.rep, h_err.node, h_err.day, h_err.event);
    return h_err.code;
  }
  return SG_OK;
}

extern "C" int sg_set_replicate_range(sg_model *m, int32_t rep0, int32_t rep_total) {
  if (!m || rep0 < 0 || rep_total < 0 || (rep_total > 0 && rep0 >= rep_total) ||
      (rep_total == 0 && rep0 != 0) || rep_total > (1 << 24))
    return SG_ERR_ARG;
  if (rep0 > 0 && m->emu_on) return SG_ERR_ARG;
  m->rep0 = rep0;
  m->rep_total = rep_total;
  return SG_OK;
}

extern "C" int sg_set_tuning(sg_model *m, int32_t nodes_per_block, int32_t heavy_after) {
  if (!m || nodes_per_block > (1 << 22) || heavy_after > (1 << 20)) return SG_ERR_ARG;
  m->npb = nodes_per_block > 0 ? nodes_per_block : -1;
  m->heavy_after = heavy_after >= 0 ? heavy_after : -1;
  return SG_OK;
}

extern "C" int sg_autotune(sg_model *m, const int32_t *tspan, int32_t n_tspan, uint64_t seed,
                           int32_t n_rep, const int32_t *d_u0, const double *d_v0,
                           int32_t *d_U, double *d_V, void *stream, int32_t *npb_out,
                           int32_t *heavy_after_out, double *ms_out) {
  if (!m) return SG_ERR_ARG;
  // 4 and 8 nodes per block give every heavy node its own warp (workloads
  // where most node-days take thousands of draws); more than kDayBlock
  // selects the sparse-activity schedule: units spread over 1, 2 or 4
  // blocks per SM, fixed 1,024-unit blocks, or one or two whole replicates
  // per block
  std::vector<std::pair<int32_t, int32_t>> cand;
  for (int32_t npb : {4, 8, 16, 32, 64, 128})
    for (int32_t h : {0, 1, 2, 4, 8}) cand.emplace_back(npb, h);
  {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    const long long units = (long long)m->tb.n_nodes * n_rep;
    std::vector<int32_t> sp;
    for (int per_sm : {1, 2, 4}) {
      const long long b = (units + (long long)sms * per_sm - 1) / ((long long)sms * per_sm);
      if (b > kDayBlock && b <= (1 << 22)) sp.push_back((int32_t)b);
    }
    if (units > 2LL * kDayBlock * sms) sp.push_back(1024);
    // whole replicates per block (one launch for every day, external
    // transfers in the blocks) when that still gives half a block per SM
    for (int per_block : {1, 2}) {
      const long long b = (long long)m->tb.n_nodes * per_block;
      if (b > kDayBlock && b <= (1 << 22) && (long long)n_rep / per_block >= sms / 2)
        sp.push_back((int32_t)b);
    }
    const int k = m->tb.kind;
    const bool sparse_ok = m->solver != SG_SOLVER_AEM && !m->emu_on && !m->persistent &&
                           (k == SG_SIR || k == SG_SIS || k == SG_SISE || k == SG_SISE3);
    if (!sparse_ok) sp.clear();
    for (int32_t npb : sp)
      for (int32_t h : {2, 8, 16, 32, 128}) cand.emplace_back(npb, h);
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return SG_ERR_CUDA;
  }
  const int32_t old_npb = m->npb, old_heavy = m->heavy_after;
  const bool old_timing = m->timing;
  m->timing = false;
  double best = 1e300;
  int32_t best_npb = -1, best_heavy = -1;
  int rc = SG_OK;
  for (const auto &ch : cand) {
    {
      const int32_t npb = ch.first, h = ch.second;
      m->npb = npb;
      m->heavy_after = h;
      // one untimed run (it captures the candidate's graph when graphs are
      // on), then the faster of two timed runs
      rc = sg_run(m, tspan, n_tspan, seed, n_rep, d_u0, d_v0, d_U, d_V, stream, nullptr,
                  nullptr);
      if (rc) break;
      float ms = 3.0e38f;
      for (int rep = 0; rep < 2 && rc == SG_OK; ++rep) {
        cudaEventRecord(e0, st);
        rc = sg_run(m, tspan, n_tspan, seed, n_rep, d_u0, d_v0, d_U, d_V, stream, nullptr,
                    nullptr);
        cudaEventRecord(e1, st);
        float t = 0.f;
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (rc) break;
      if (ms < best) {
        best = ms;
        best_npb = npb;
        best_heavy = h;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->timing = old_timing;
  if (rc) {
    m->npb = old_npb;
    m->heavy_after = old_heavy;
    return rc;
  }
  m->npb = best_npb;
  m->heavy_after = best_heavy;
  if (npb_out) *npb_out = best_npb;
  if (heavy_after_out) *heavy_after_out = best_heavy;
  if (ms_out) *ms_out = best;
  return SG_OK;
}

// Checks one compressed-column pattern (see sg_output) and uploads it.
static int upload_pattern(int32_t cols, int64_t nnz, const int64_t *colptr, const int32_t *row,
                          long long rows, DevBuf<int64_t> &dptr, DevBuf<int32_t> &drow) {
  if (nnz < 0 || (nnz > 0 && (!colptr || !row))) return SG_ERR_ARG;
  if (nnz == 0 && !colptr) return SG_OK;
  if (colptr[0] != 0 || colptr[cols] != nnz) return SG_ERR_ARG;
  for (int32_t c = 0; c < cols; ++c) {
    if (colptr[c + 1] < colptr[c]) return SG_ERR_ARG;
    for (int64_t e = colptr[c]; e < colptr[c + 1]; ++e) {
      if (row[e] < 0 || row[e] >= rows) return SG_ERR_ARG;
      if (e > colptr[c] && row[e] <= row[e - 1]) return SG_ERR_ARG;
    }
  }
  std::vector<int64_t> p(colptr, colptr + cols + 1);
  std::vector<int32_t> r(row, row + nnz);
  int rc = upload(dptr, p);
  if (!rc && nnz > 0) rc = upload(drow, r);
  return rc;
}

extern "C" int sg_set_output(sg_model *m, const sg_output *o) {
  if (!m) return SG_ERR_ARG;
  m->graph_ok = false;
  ++m->out_version;
  m->out = OutDev{};
  m->out_dense = true;
  m->out_cols = -1;
  if (!o) return SG_OK;
  const SgTables &tb = m->tb;
  const uint32_t all = tb.n_comp >= 32 ? 0xffffffffu : ((1u << tb.n_comp) - 1u);
  const bool sparse = o->u_nnz > 0 || o->v_nnz > 0;
  const bool prev = o->prev_cases != 0 || o->prev_at_risk != 0;
  if ((o->dense != 0 && o->dense != 1) || (o->prev_cases & ~all) || (o->prev_at_risk & ~all) ||
      (prev && (!o->prev_cases || !o->prev_at_risk || !o->d_prev)) ||
      ((sparse || prev) && o->n_tspan < 1) || (o->u_nnz > 0 && !o->d_u_val) ||
      (o->v_nnz > 0 && (!o->d_v_val || tb.n_v == 0)))
    return SG_ERR_ARG;
  int rc = SG_OK;
  if (o->u_nnz > 0)
    rc = upload_pattern(o->n_tspan, o->u_nnz, o->u_colptr, o->u_row,
                        (long long)tb.n_nodes * tb.n_comp, m->out_u_colptr, m->out_u_row);
  if (!rc && o->v_nnz > 0)
    rc = upload_pattern(o->n_tspan, o->v_nnz, o->v_colptr, o->v_row,
                        (long long)tb.n_nodes * tb.n_v, m->out_v_colptr, m->out_v_row);
  if (rc) return rc;
  OutDev d;
  if (o->u_nnz > 0) {
    d.u_colptr = m->out_u_colptr.p;
    d.u_row = m->out_u_row.p;
    d.u_val = o->d_u_val;
    d.u_nnz = o->u_nnz;
  }
  if (o->v_nnz > 0) {
    d.v_colptr = m->out_v_colptr.p;
    d.v_row = m->out_v_row.p;
    d.v_val = o->d_v_val;
    d.v_nnz = o->v_nnz;
  }
  if (prev) {
    d.cases = o->prev_cases;
    d.at_risk = o->prev_at_risk;
    d.prev = reinterpret_cast<unsigned long long *>(o->d_prev);
  }
  m->out = d;
  m->out_dense = o->dense != 0;
  m->out_cols = (sparse || prev) ? o->n_tspan : -1;
  return SG_OK;
}

extern "C" int sg_set_persistent(sg_model *m, int enable) {
  if (!m) return SG_ERR_ARG;
  if ((enable != 0) != m->persistent) {
    m->persistent = enable != 0;
    m->graph_ok = false;
  }
  return SG_OK;
}

extern "C" int sg_set_fused_events(sg_model *m, int enable) {
  if (!m) return SG_ERR_ARG;
  if ((enable != 0) != m->fuse_e2) {
    m->fuse_e2 = enable != 0;
    m->graph_ok = false;
  }
  return SG_OK;
}

extern "C" int sg_set_solver(sg_model *m, int32_t solver) {
  if (!m || (solver != SG_SOLVER_SSM && solver != SG_SOLVER_AEM)) return SG_ERR_ARG;
  if (solver != m->solver) {
    m->solver = solver;
    m->graph_ok = false;
  }
  return SG_OK;
}

extern "C" int sg_set_graphs(sg_model *m, int enable) {
  if (!m) return SG_ERR_ARG;
  m->graphs = enable != 0;
  if (!m->graphs) m->graph_ok = false;
  return SG_OK;
}

extern "C" int sg_emulator_set(sg_model *m, const void *const *W, const float *const *b,
                               int32_t max_herd, double phi_lo, double phi_hi, int enable) {
  if (!m) return SG_ERR_ARG;
  if (!enable) {
    m->emu_on = false;
    m->graph_ok = false;
    return SG_OK;
  }
  if (m->tb.kind != SG_SISE3 || !W || !b || max_herd < -1 || !(phi_lo <= phi_hi)) return SG_ERR_ARG;
  for (int l = 0; l < 4; ++l) {
    if (!W[l] || !b[l] || ((uintptr_t)W[l] & 15) != 0) return SG_ERR_ARG;
    m->emu_W[l] = (const __nv_bfloat16 *)W[l];
    m->emu_b[l] = b[l];
  }
  m->emu_max_herd = max_herd;
  m->emu_phi_lo = phi_lo;
  m->emu_phi_hi = phi_hi;
  m->emu_on = true;
  ++m->emu_version;
  m->graph_ok = false;
  return SG_OK;
}

extern "C" int sg_emulator_set_min_rate(sg_model *m, double min_rate) {
  if (!m || !(min_rate >= 0.0)) return SG_ERR_ARG;
  m->emu_min_rate = min_rate;
  ++m->emu_version;
  m->graph_ok = false;
  return SG_OK;
}

extern "C" int sg_emulator_set_fp8(sg_model *m, const void *const *W8,
                                   const float *const *w_scale, const float *act_scale,
                                   int enable) {
  if (!m) return SG_ERR_ARG;
  if (!enable) {
    m->emu_fp8 = false;
    ++m->emu_version;
    m->graph_ok = false;
    return SG_OK;
  }
  if (!m->emu_on || !W8 || !w_scale || !act_scale) return SG_ERR_ARG;
  for (int l = 0; l < 3; ++l) {
    if (!W8[l] || !w_scale[l] || ((uintptr_t)W8[l] & 15) != 0 || !(act_scale[l] > 0.0f))
      return SG_ERR_ARG;
    m->emu_W8[l] = (const uint8_t *)W8[l];
    m->emu_wscale[l] = w_scale[l];
    m->emu_act_scale[l] = act_scale[l];
  }
  m->emu_fp8 = true;
  ++m->emu_version;
  m->graph_ok = false;
  return SG_OK;
}

extern "C" int sg_set_neighbors(sg_model *m, const int64_t *ptr, const int32_t *idx,
                                const double *dist) {
  if (!m || !ptr) return SG_ERR_ARG;
  const int Nn = m->tb.n_nodes;
  if (ptr[0] != 0) return SG_ERR_ARG;
  for (int i = 0; i < Nn; ++i)
    if (ptr[i + 1] < ptr[i]) return SG_ERR_ARG;
  const int64_t nnz = ptr[Nn];
  if (nnz > 0 && (!idx || !dist)) return SG_ERR_ARG;
  for (int64_t k = 0; k < nnz; ++k)
    if (idx[k] < 0 || idx[k] >= Nn || !(dist[k] > 0.0) || std::isinf(dist[k])) return SG_ERR_ARG;
  int rc;
  try {
    std::vector<int64_t> p(ptr, ptr + Nn + 1);
    std::vector<int32_t> ix(idx ? idx : nullptr, idx ? idx + nnz : nullptr);
    std::vector<double> ds(dist ? dist : nullptr, dist ? dist + nnz : nullptr);
    if ((rc = upload(m->nb_ptr, p)) || (rc = upload(m->nb_idx, ix)) ||
        (rc = upload(m->nb_dist, ds)))
      return rc;
  } catch (const std::bad_alloc &) {
    return SG_ERR_NOMEM;
  }
  m->has_nb = true;
  ++m->nb_version;
  m->graph_ok = false;
  return SG_OK;
}
