// device_math.cuh -- message arithmetic of the decoders (FP32 sum-product and
// 6-bit integer min-sum), check-team combination and warp argmax helpers.
#pragma once

#include <cstdint>

#include "graph.cuh"
#include "internal.h"

namespace ldpc {

constexpr unsigned kFull = 0xffffffffu;

template <int A> struct Arith;
template <> struct Arith<kFP32> {
  using msg = float;   // C2V messages L^C, L~^C
  using llr = float;   // lambda, L, L~
  using dval = float;  // CI metric D
};
template <> struct Arith<kINT6> {
  using msg = int8_t;
  using llr = int16_t;
  using dval = uint16_t;
};

// 1 - e^-x for 0 <= x < 1/4 by its Taylor polynomial to x^6 (relative error < 6e-8)
__device__ __forceinline__ float one_minus_exp_small(float x) {
  return x * (1.0f - x * (0.5f - x * (1.0f / 6.0f - x * (1.0f / 24.0f - x * (1.0f / 120.0f - x * (1.0f / 720.0f))))));
}

// phi(x) = -ln tanh(x/2) = 2 atanh(e^-x) for x >= 0; phi(0) = +inf, phi(inf) = 0.
// phi is its own inverse and turns eq. (2) into sums:
// 2 atanh(prod tanh(|V_k|/2)) = phi(sum phi(|V_k|)).
// With t = e^-x: for t <= 1/4 the odd series 2t(1 + t^2/3 + ... + t^10/11)
// (truncation < 5e-9 relative); above, ln((1+t)/(1-t)) with 1 - t from the Taylor
// polynomial when x < 1/4 (no cancellation) and MUFU lg2.  Relative error ~1e-6
// (the exponential itself is the accurate expf: MUFU ex2 alone loses |x| 1e-7).
// Both forms are evaluated and one selected: the lanes of a check team take
// both sides, and a branch would run them one after the other.
__device__ __forceinline__ float phi_f(float x) {
  const float t = expf(-x);
  const float t2 = t * t;
  float p = 1.0f / 11.0f;
  p = fmaf(p, t2, 1.0f / 9.0f);
  p = fmaf(p, t2, 1.0f / 7.0f);
  p = fmaf(p, t2, 0.2f);
  p = fmaf(p, t2, 1.0f / 3.0f);
  p = fmaf(p, t2, 1.0f);
  const float series = 2.0f * t * p;
  const float omt = x < 0.25f ? one_minus_exp_small(x) : 1.0f - t;
  const float lg = __logf(__fdividef(1.0f + t, omt));
  return t <= 0.25f ? series : lg;
}

// The encoded V2C input of a check: phi(|V| clipped) with the sign of V in the
// sign bit (V < 0 gives a set sign bit, also when phi is 0).
__device__ __forceinline__ float encode_fp(float v, float clip) {
  const float p = phi_f(fminf(fabsf(v), clip));
  return v < 0.0f ? -p : p;
}

// sign product and phi of the sum of phis, clamped to +-clip (eq. 2)
__device__ __forceinline__ float combine_fp(float sum_phi, unsigned neg, float clip) {
  const float m = fminf(phi_f(sum_phi), clip);
  return neg ? -m : m;
}

__device__ __forceinline__ int8_t encode_int(int v) { return (int8_t)max(-31, min(31, v)); }

// |p0(a) - p0(b)| of eq. (8), p0(L) = e^L/(1+e^L) = (1 + tanh(L/2))/2, without
// the cancellation of 1 - 1: with x = |a|, y = |b|, ex = e^-x, ey = e^-y and
// tanh(x/2) = (1 - ex)/(1 + ex), both sign cases share one denominator:
//   opposite signs : (tanh(x/2) + tanh(y/2)) / 2 = (1 - e^-(x+y)) / ((1+ex)(1+ey))
//   equal signs    : |tanh(x/2) - tanh(y/2)| / 2 = |ex - ey| / ((1+ex)(1+ey))
//                    with |ex - ey| = e^-min(x,y) (1 - e^-|x-y|)
// 1 - e^-u comes from its Taylor polynomial for u < 1/4 (no cancellation),
// else from the exponentials at hand.  Both numerators are evaluated and one
// selected (no divergent branch in a lane team).
__device__ __forceinline__ float ci_fp(float a, float b) {
  const float x = fabsf(a), y = fabsf(b);
  const float ex = expf(-x), ey = expf(-y);
  const float sum = x + y, d = fabsf(x - y);
  const float opposite = sum < 0.25f ? one_minus_exp_small(sum) : 1.0f - ex * ey;
  const float hi = fmaxf(ex, ey);
  const float equal = d < 0.25f ? hi * one_minus_exp_small(d) : hi - fminf(ex, ey);
  return __fdividef((a >= 0.0f) != (b >= 0.0f) ? opposite : equal, (1.0f + ex) * (1.0f + ey));
}

// Integer CI: |T[c(a)] - T[c(b)]| with c = clamp to [-127, 127].
__device__ __forceinline__ uint16_t ci_int(int a, int b, const int16_t* tab) {
  const int qa = max(-127, min(127, a)) + 127, qb = max(-127, min(127, b)) + 127;
  const int d = (int)tab[qa] - (int)tab[qb];
  return (uint16_t)(d < 0 ? -d : d);
}

// Syndrome-check cadence without a 64-bit division per step: `left` counts the
// updates until the next multiple of `interval` (1..interval; start it at
// interval).  Advances by `done` updates (0 <= done < 2^31) and returns true
// when a multiple of interval was reached, i.e. floor(count / interval) grew.
__device__ __forceinline__ bool check_due(int64_t& left, int64_t interval, int64_t done) {
  if (interval <= 0) return false;
  if (done < left) {
    left -= done;
    return false;
  }
  int64_t rest = done - left;  // updates past the first multiple reached
  if (rest >= interval) rest = (int64_t)((uint32_t)rest % (uint32_t)interval);  // here interval <= rest < 2^31
  left = interval - rest;
  return true;
}

// Order-preserving 32-bit keys of non-negative metric values.
__device__ __forceinline__ uint32_t mkey(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t mkey(int v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t mkey(uint16_t v) { return (uint32_t)v; }

// residual |L~^C - L^C| (eq. 4) as a key
__device__ __forceinline__ uint32_t rkey(float p, float c) { return mkey(fabsf(p - c)); }
__device__ __forceinline__ uint32_t rkey(int8_t p, int8_t c) { return (uint32_t)abs((int)p - (int)c); }

// Running argmax of (key, idx): larger key wins, equal keys go to the lower idx.
__device__ __forceinline__ void am_update(uint32_t& bk, uint32_t& bi, uint32_t k, uint32_t i) {
  if (k > bk || (k == bk && i < bi)) {
    bk = k;
    bi = i;
  }
}

// Warp-wide argmax; lanes without a candidate pass (0, 0xffffffff).  Returns the
// winning index (0xffffffff if no lane had a candidate) and its key.
__device__ __forceinline__ uint32_t warp_argmax(uint32_t key, uint32_t idx, uint32_t& best_key) {
  best_key = __reduce_max_sync(kFull, key);
  return __reduce_min_sync(kFull, key == best_key ? idx : 0xffffffffu);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Check team: W lanes (power of two) handle check m (m < 0: idle).  Lane r < dc
// owns edge e = base + r towards variable j; V2C = L_j - C[e] (eq. 1); `out`
// receives the exclude-one combination over the other edges (eq. 2 / min-sum).
// All lanes of the warp must call it (width-W shuffles).  Returns dc.  CA and
// LA index like arrays (pointers, or the decoders' array views).
template <int A, class G, class CA, class LA>
__device__ __forceinline__ int team_c2v(const G& g, const CA& C, const LA& L, int m, int r, int W,
                                        float clip, int& e, int& j, typename Arith<A>::msg& out) {
  int dc = 0;
  e = 0;
  j = 0;
  if (m >= 0) {
    const typename G::C cc = g.cn(m);
    dc = cc.d;
    if (r < dc) {
      e = cc.b + r;
      j = g.cvn(cc, r);
    }
  }
  // exclude-one combination by one butterfly over the team; the sign is the
  // team parity (one ballot) with r's own sign removed
  const int team0 = (int)(threadIdx.x & 31) - r;  // first lane of the team
  const unsigned tmask = W == 32 ? kFull : (((1u << W) - 1u) << team0);
  if (A == kFP32) {
    // idle lanes (e = j = 0) compute too and drop the value: no branch around phi
    const float enc0 = encode_fp((float)L[j] - (float)C[e], clip);
    const float enc = r < dc ? enc0 : 0.0f;
    const unsigned sg = __float_as_uint(enc) >> 31;
    const unsigned sall = __popc(__ballot_sync(kFull, sg) & tmask) & 1u;
    // the team's largest phi mx and the sum `rest` of the others (one copy of
    // mx left out): the sum over the other lanes is rest for a lane holding mx,
    // else (rest - phi_r) + mx, whose subtraction loses at most an ulp of
    // phi_r <= mx against a result >= mx (no cancellation of a dominant term;
    // phi = +inf for a zero input gives inf or the finite rest, never inf - inf)
    const float a0 = fabsf(enc);
    float mx = a0, rest = 0.0f;
    for (int o = 1; o < W; o <<= 1) {
      const float omx = __shfl_xor_sync(kFull, mx, o, W);
      const float ore = __shfl_xor_sync(kFull, rest, o, W);
      rest = (rest + ore) + fminf(mx, omx);
      mx = fmaxf(mx, omx);
    }
    const float sum = a0 == mx ? rest : (rest - a0) + mx;
    out = (typename Arith<A>::msg)combine_fp(sum, sall ^ sg, clip);
  } else {
    const int enc = r < dc ? (int)encode_int((int)L[j] - (int)C[e]) : 0;
    const unsigned sg = enc < 0;
    const unsigned sall = __popc(__ballot_sync(kFull, sg) & tmask) & 1u;
    // the team's smallest and second smallest magnitudes (idle lanes: 31),
    // packed in one word: the minimum over the other lanes is m2 for a lane
    // holding m1, else m1
    const int a0 = r < dc ? abs(enc) : 31;
    int m1 = a0, m2 = 31;
    for (int o = 1; o < W; o <<= 1) {
      const int pk = __shfl_xor_sync(kFull, m1 | (m2 << 8), o, W);
      const int o1 = pk & 0xff, o2 = pk >> 8;
      m2 = min(max(m1, o1), min(m2, o2));
      m1 = min(m1, o1);
    }
    const int mag = a0 == m1 ? m2 : m1;
    out = (typename Arith<A>::msg)((sall ^ sg) ? -mag : mag);
  }
  return dc;
}

// lam[n] + sum_{m in M(n)} X[e]  (eq. 3 with X = L^C, Sec. 2.B with X = L~^C)
template <int A, class G, typename X>
__device__ __forceinline__ typename Arith<A>::llr vn_total(const G& g, const typename Arith<A>::llr* lam,
                                                           const X* arr, int n) {
  using L_ = typename Arith<A>::llr;
  const typename G::V v = g.vn(n);
  L_ acc = lam[n];
  for (int k = 0; k < v.d; ++k) {
    int e, m;
    g.vedge(v, k, e, m);
    acc = (L_)(acc + arr[e]);
  }
  return acc;
}

}  // namespace ldpc
