// sg_device.cuh -- device primitives of the SimInf GB300 engine: the
// counter-based random stream, the open-interval uniform, the logarithm, the
// bounded integers, the transition-rate functions and the post time step.
//
// Every double expression is written in a fixed evaluation order and the
// library is compiled with -fmad=false, so no multiply-add is contracted:
// the results are the correctly rounded IEEE results of each written
// operation, in that order.
#pragma once

#include <stdint.h>

#include "sg_common.h"

namespace sg {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32 -> 64-bit products whose
// halves are xor-ed with the other counter words and the round key; the key
// is advanced by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform on (0, 1) from 52 random bits: k = (hi << 20) | (lo >> 12),
// r = (k + 1/2) 2^-52 = (2k + 1) 2^-53.  The value is exact, so it is built
// directly from its bits with integer instructions (normalise the odd 53-bit
// integer 2k + 1): no floating-point operation, same value as the product.
// The range is [2^-53, 1 - 2^-53].
__device__ __forceinline__ double u01_open(uint32_t lo, uint32_t hi) {
  const unsigned long long m =
      (((unsigned long long)hi << 21) | (unsigned long long)((lo >> 12) << 1)) | 1ull;
  const int p = 63 - __clzll((long long)m);  // msb position, 0..52
  const unsigned long long frac = (m << (52 - p)) & 0x000fffffffffffffull;
  const unsigned long long ex = (unsigned long long)(p + 970);  // 2^(p - 53)
  return __longlong_as_double((long long)((ex << 52) | frac));
}

// ---------------------------------------------------------------------------
// Exact helpers that replace FP64 instructions (each FP64 instruction costs
// tens of cycles of latency on GB300) by integer ones with identical results.
// ---------------------------------------------------------------------------

// (double)n for a 32-bit integer: positive values are normalised from their
// bits; zero and negatives (which counts never are) use the conversion.
__device__ __forceinline__ double i2d(int n) {
  if (n <= 0) return (double)n;
  const int p = 31 - __clz(n);
  const unsigned long long frac =
      ((unsigned long long)(unsigned)n << (52 - p)) & 0x000fffffffffffffull;
  return __longlong_as_double((long long)(((unsigned long long)(p + 1023) << 52) | frac));
}

// Order-preserving integer key of a double (for non-NaN values, including
// negatives): a < b  <=>  key(a) < key(b), except that -0 orders below +0.
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// x > 0 for a value that is not NaN (negative zero is not > 0).
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }

// a <= b for two values that are not NaN and not negative.
__device__ __forceinline__ bool le_nonneg(double a, double b) {
  return __double_as_longlong(a) <= __double_as_longlong(b);
}

// ---------------------------------------------------------------------------
// Natural logarithm from the argument reduction x = 2^k m, m in
// (sqrt(2)/2, sqrt(2)], and log(m) = 2 atanh(s), s = f / (2 + f), f = m - 1,
// evaluated as f - (h - s (h + R(s^2))) with h = f^2 / 2 and the atanh
// Taylor polynomial R(z) = sum_{j=1}^{10} 2 z^j / (2 j + 1) in Estrin form;
// k ln 2 is added through a split ln 2 = L_hi + L_lo whose high part has 33
// significant bits (k L_hi exact).  Every a + b c of the polynomial, h + R,
// s (h + R) + k L_lo and k L_hi + (...) is one fused multiply-add (one
// rounding): on GB300 each FP64 warp instruction occupies the
// sub-partition's FP64 pipe for ~76 cycles, so the count of operations is
// the cost.  Accuracy: within 1 ulp of the correctly rounded logarithm.
// Only positive finite arguments reach it here.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double log_pos(double x) {
  long long bits = __double_as_longlong(x);
  int k = 0;
  if (bits < 0x0010000000000000LL) {  // subnormal: scale by 2^54
    x = x * 0x1.0p54;
    bits = __double_as_longlong(x);
    k = -54;
  }
  k += (int)(bits >> 52) - 1023;
  double m = __longlong_as_double((bits & 0x000fffffffffffffLL) |
                                  0x3ff0000000000000LL);
  if (m > 0x1.6a09e667f3bcdp+0) {  // sqrt(2) rounded to nearest
    m = m * 0.5;
    k = k + 1;
  }
  const double f = m - 1.0;
  const double h = (0.5 * f) * f;
  const double s = f / (2.0 + f);
  const double z = s * s;
  // Estrin's scheme for z (c1 + c2 z + ... + c10 z^9): coefficient pairs,
  // then combined with z^2, z^4, z^8 (dependency depth 8 instead of 20)
  const double z2 = z * z, z4 = z2 * z2, z8 = z4 * z4;
  const double p01 = fma(0x1.999999999999ap-2, z, 0x1.5555555555555p-1);
  const double p23 = fma(0x1.c71c71c71c71cp-3, z, 0x1.2492492492492p-2);
  const double p45 = fma(0x1.3b13b13b13b14p-3, z, 0x1.745d1745d1746p-3);
  const double p67 = fma(0x1.e1e1e1e1e1e1ep-4, z, 0x1.1111111111111p-3);
  const double p89 = fma(0x1.8618618618618p-4, z, 0x1.af286bca1af28p-4);
  const double q03 = fma(z2, p23, p01);
  const double q47 = fma(z2, p67, p45);
  const double hR = fma(z, fma(z8, p89, fma(z4, q47, q03)), h);  // h + R
  const double dk = (double)k;
  return fma(dk, 0x1.62e42fefp-1, f - (h - fma(s, hR, dk * 0x1.473de6af278edp-34)));
}

// ---------------------------------------------------------------------------
// Event word stream: Philox counter (c, index_lo, index_hi,
// (SG_STREAM_EVENTS << 24) | rep), four words per call, consumed in order.
// ---------------------------------------------------------------------------
struct WordStream {
  uint32_t k0, k1, idx_lo, idx_hi, tag, c;
  U4 buf;
  int pos;
  __device__ __forceinline__ void init(uint64_t seed, long long index, int rep) {
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
    idx_lo = (uint32_t)(unsigned long long)index;
    idx_hi = (uint32_t)((unsigned long long)index >> 32);
    tag = (SG_STREAM_EVENTS << 24) | (uint32_t)rep;
    c = 0;
    pos = 4;
  }
  // Same stream with the first Philox block already computed (c = 0).
  __device__ __forceinline__ void init_with_first(uint64_t seed, long long index, int rep,
                                                  U4 first) {
    init(seed, index, rep);
    buf = first;
    c = 1;
    pos = 0;
  }
  __device__ __forceinline__ uint32_t next() {
    if (pos == 4) {
      buf = philox10(U4{c, idx_lo, idx_hi, tag}, k0, k1);
      ++c;
      pos = 0;
    }
    const uint32_t r = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
    ++pos;
    return r;
  }
  // Uniform integer on [0, s), s >= 1: Lemire's multiply-shift with
  // rejection of the low product words below 2^32 mod s (unbiased).
  __device__ __forceinline__ uint32_t below(uint32_t s) {
    unsigned long long m = (unsigned long long)next() * s;
    uint32_t lo = (uint32_t)m;
    if (lo < s) {
      const uint32_t thr = (0u - s) % s;
      while (lo < thr) {
        m = (unsigned long long)next() * s;
        lo = (uint32_t)m;
      }
    }
    return (uint32_t)(m >> 32);
  }
};

// Events that move at least this many individuals are sampled by a whole
// warp (urn_warp); smaller ones by one thread (WordStream::below + walk).
constexpr int kUrnWarp = 32;

// The urn of one event, sampled by the 32 lanes of a warp together (every
// lane passes the same arguments and gets the same moved[]).  k individuals
// are drawn without replacement from the compartments of `mask` with counts
// cur[] (total of them: `total`): draw j takes a uniform index below
// total - j from the event's word stream by Lemire's multiply-shift with
// rejection, and walks the compartments in row order -- the same words,
// the same indices and the same walk as the thread urn, so moved[] is
// identical.  Lane l tests draw j0 + l on word i0 + l (words i: component
// i % 4 of Philox block i / 4); a ballot finds the first rejected draw r,
// draws j0 .. j0 + r - 1 are final, the rejected word is skipped and the
// next round starts at draw j0 + r with word i0 + r + 1 (the thread urn's
// retry).  The walk then takes the final indices in order (a shuffle each).
template <int C>
__device__ __forceinline__ void urn_warp(const int *cur, uint32_t mask, uint32_t k,
                                         uint32_t total, uint64_t seed, long long index, int rep,
                                         int *moved) {
  const int lane = threadIdx.x & 31;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint32_t ilo = (uint32_t)(unsigned long long)index;
  const uint32_t ihi = (uint32_t)((unsigned long long)index >> 32);
  const uint32_t tag = (SG_STREAM_EVENTS << 24) | (uint32_t)rep;
  int rem[C];
#pragma unroll
  for (int p = 0; p < C; ++p) {
    moved[p] = 0;
    rem[p] = ((mask >> p) & 1u) ? cur[p] : 0;
  }
  uint32_t j0 = 0, i0 = 0;
  while (j0 < k) {
    const uint32_t j = j0 + (uint32_t)lane;
    const uint32_t wi = i0 + (uint32_t)lane;
    const U4 b = philox10(U4{wi >> 2, ilo, ihi, tag}, k0, k1);
    const uint32_t q = wi & 3u;
    const uint32_t word = q == 0 ? b.x : q == 1 ? b.y : q == 2 ? b.z : b.w;
    const bool live = j < k;
    const uint32_t s = live ? total - j : 1u;  // >= 1 for the draws of this event
    const unsigned long long m = (unsigned long long)word * s;
    const uint32_t lo = (uint32_t)m;
    const bool reject = live && lo < s && lo < (0u - s) % s;
    const unsigned rmask = __ballot_sync(0xffffffffu, reject);
    const uint32_t ok = rmask ? (uint32_t)(__ffs(rmask) - 1) : 32u;
    const uint32_t nd = min(ok, k - j0);
    const uint32_t x = (uint32_t)(m >> 32);
    for (uint32_t d = 0; d < nd; ++d) {
      uint32_t xd = __shfl_sync(0xffffffffu, x, (int)d);
      bool taken = false;
#pragma unroll
      for (int p = 0; p < C; ++p) {
        if (taken || !((mask >> p) & 1u)) continue;
        const uint32_t r = (uint32_t)rem[p];
        if (xd < r) {
          ++moved[p];
          --rem[p];
          taken = true;
        } else {
          xd -= r;
        }
      }
    }
    j0 += nd;
    i0 += nd + (ok < 32u && j0 < k ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// Transition-rate functions (TRFun, Sec. 3.4.1), one set per kind.
// ---------------------------------------------------------------------------
template <int KIND> struct ModelTraits;

// Each kind also has `prepare`, which evaluates once per node and day the
// factors of its rates that do not change within the day (they depend on v
// and gdata only), and `rate_k`, the same rate from those factors.  The
// factors are the leftmost products of the written expressions, so the
// values are identical to `rate`.

// SIR, Eq. (SIR); operation order of the SIR rate listing (Appendix C).
template <> struct ModelTraits<SG_SIR> {
  static constexpr int C = 3, T = 2, NV = 0, NK = 1;
  __device__ static __forceinline__ void prepare(const double *, const double *, double *) {}
  __device__ static __forceinline__ double rate_k(int j, const int *u, const double *,
                                                  const double *g) {
    return rate(j, u, nullptr, g);
  }
  __device__ static __forceinline__ double rate(int j, const int *u, const double *,
                                                const double *g) {
    if (j == 0) {
      const double Sn = i2d(u[0]), In = i2d(u[1]);
      const double n = Sn + In + i2d(u[2]);
      return gt0(n) ? (g[0] * Sn * In) / n : 0.0;
    }
    return g[1] * i2d(u[1]);
  }
};

// SIS of Sec. 2.1: [beta S I, gamma I].
template <> struct ModelTraits<SG_SIS> {
  static constexpr int C = 2, T = 2, NV = 0, NK = 1;
  __device__ static __forceinline__ void prepare(const double *, const double *, double *) {}
  __device__ static __forceinline__ double rate_k(int j, const int *u, const double *,
                                                  const double *g) {
    return rate(j, u, nullptr, g);
  }
  __device__ static __forceinline__ double rate(int j, const int *u, const double *,
                                                const double *g) {
    return j == 0 ? g[0] * i2d(u[0]) * i2d(u[1]) : g[1] * i2d(u[1]);
  }
};

// SISe (Sec. 4.2, no coupling): [upsilon phi S, gamma I].
template <> struct ModelTraits<SG_SISE> {
  static constexpr int C = 2, T = 2, NV = 1, NK = 1;
  __device__ static __forceinline__ void prepare(const double *v, const double *g, double *k) {
    k[0] = g[0] * v[0];
  }
  __device__ static __forceinline__ double rate_k(int j, const int *u, const double *k,
                                                  const double *g) {
    return j == 0 ? k[0] * i2d(u[0]) : g[1] * i2d(u[1]);
  }
  __device__ static __forceinline__ double rate(int j, const int *u, const double *v,
                                                const double *g) {
    return j == 0 ? g[0] * v[0] * (double)u[0] : g[1] * (double)u[1];
  }
};

// SISe_sp: the rates of SISe (the coupling acts on phi only).
template <> struct ModelTraits<SG_SISE_SP> : ModelTraits<SG_SISE> {};

// SISe3: transition 2a is S_a -> I_a at upsilon_a phi S_a, 2a + 1 is
// I_a -> S_a at gamma_a I_a.
template <> struct ModelTraits<SG_SISE3> {
  static constexpr int C = 6, T = 6, NV = 1, NK = 3;
  __device__ static __forceinline__ void prepare(const double *v, const double *g, double *k) {
    k[0] = g[0] * v[0];
    k[1] = g[1] * v[0];
    k[2] = g[2] * v[0];
  }
  __device__ static __forceinline__ double rate_k(int j, const int *u, const double *k,
                                                  const double *g) {
    const int a = j >> 1;
    return (j & 1) == 0 ? k[a] * i2d(u[2 * a]) : g[3 + a] * i2d(u[2 * a + 1]);
  }
  __device__ static __forceinline__ double rate(int j, const int *u, const double *v,
                                                const double *g) {
    const int a = j >> 1;
    return (j & 1) == 0 ? g[a] * v[0] * (double)u[2 * a] : g[3 + a] * (double)u[2 * a + 1];
  }
};

// !(w >= 0) || isinf(w) from the bits: bad unless w is -0 or a finite
// value >= +0.
__device__ __forceinline__ bool bad_rate(double w) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  return !(b == 0x8000000000000000ull || b < 0x7ff0000000000000ull);
}

// Season ends as integers: for an integer day d, d <= e exactly when
// d <= floor(e) (any finite e); NaN ends never hold.
__device__ __forceinline__ int season_end_int(double e) {
  if (e >= 2147483647.0) return 0x7fffffff;
  if (!(e >= -2147483648.0)) return (int)0x80000000;
  return (int)floor(e);
}

// beta(t) of Sec. 4.2: season of day-of-year ((t - 1) mod 365) + 1 against
// the node's season ends.
__device__ __forceinline__ double season_decay(int t, const int *ends, const double *b4) {
  int d = (t - 1) % 365;
  if (d < 0) d += 365;
  const int doy = d + 1;
  return doy <= ends[0] ? b4[0] : doy <= ends[1] ? b4[1] : doy <= ends[2] ? b4[2] : b4[3];
}

// Post time step (PTSFun; Eq. numstep3 as one Euler step of length 1) for
// the SISe kinds: phi_new = phi + (alpha I / N - beta(t) phi), shedding 0 in
// an empty node.  Returns 1 if phi changed, 0 if not, SG_ERR_PTS if the new
// value is not finite.
template <int KIND>
__device__ __forceinline__ int post_step(double *v, const int *u, const int *ends,
                                         const double *g, int t) {
  double I_tot, N_tot;
  const double *pg;
  if (KIND == SG_SISE) {
    I_tot = i2d(u[1]);
    N_tot = i2d(u[0]) + i2d(u[1]);
    pg = g + 2;
  } else if (KIND == SG_SISE3) {
    I_tot = 0.0;
    N_tot = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      I_tot = I_tot + i2d(u[2 * a + 1]);
      N_tot = N_tot + i2d(u[2 * a]) + i2d(u[2 * a + 1]);
    }
    pg = g + 6;
  } else {
    return 0;
  }
  const double phi = v[0];
  const double shed = gt0(N_tot) ? (pg[0] * I_tot) / N_tot : 0.0;
  const double beta = season_decay(t, ends, pg + 1);
  const double nv = phi + (shed - beta * phi);
  v[0] = nv;
  if (!isfinite(nv)) return SG_ERR_PTS;
  return __double_as_longlong(nv) != __double_as_longlong(phi) ? 1 : 0;
}

__device__ __forceinline__ void report(SgDevError *err, int code, int rep, int node,
                                       int day, long long event) {
  if (atomicCAS(&err->code, 0, code) == 0) {
    err->rep = rep;
    err->node = node;
    err->day = day;
    err->event = event;
  }
}

}  // namespace sg
