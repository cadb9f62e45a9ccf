// device_math.cuh -- message arithmetic of the decoders (FP32 sum-product and
// 6-bit integer min-sum) and warp-level argmax helpers.
#pragma once

#include <cstdint>

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

// phi(x) = -ln tanh(x/2) = ln((e^x + 1)/(e^x - 1)) for x >= 0; phi is its own
// inverse and turns the product of tanh terms of eq. (2) into a sum:
// 2 atanh(prod tanh(|V_k|/2)) = phi(sum phi(|V_k|)).  phi(0) = +inf, phi(inf) = 0.
__device__ __forceinline__ float phi_f(float x) { return log1pf(2.0f / expm1f(x)); }

// The scratch value of one V2C input of a check: its phi with the sign of V
// in the sign bit (V < 0 gives a set sign bit, also when phi is 0).
__device__ __forceinline__ float encode_fp(float v, float clip) {
  const float a = fminf(fabsf(v), clip);
  const float p = phi_f(a);
  return v < 0.0f ? -p : p;
}

// Combine every other entry of a check (exclude-one): sign product and phi of
// the sum of phis, clamped to +-clip.  Matches eq. (2) with the V2C clip.
__device__ __forceinline__ float combine_fp(float sum_phi, unsigned neg, float clip) {
  float m = fminf(phi_f(sum_phi), clip);
  return neg ? -m : m;
}

__device__ __forceinline__ int8_t encode_int(int v) { return (int8_t)max(-31, min(31, v)); }

// |p0(a) - p0(b)| of eq. (8) with p0(L) = e^L/(1+e^L), written to avoid the
// cancellation of 1 - 1: for equal signs it is |e^-y - e^-x| / ((1+e^-x)(1+e^-y))
// with x = |a|, y = |b|; for opposite signs (tanh(|a|/2) + tanh(|b|/2)) / 2.
__device__ __forceinline__ float ci_fp(float a, float b) {
  const bool sa = a >= 0.0f, sb = b >= 0.0f;
  const float x = fabsf(a), y = fabsf(b);
  if (sa != sb) return 0.5f * (tanhf(0.5f * x) + tanhf(0.5f * y));
  const float lo = fminf(x, y), d = fabsf(x - y);
  const float num = -expf(-lo) * expm1f(-d);
  const float den = (1.0f + expf(-x)) * (1.0f + expf(-y));
  return num / den;
}

// Integer CI: |T[c(a)] - T[c(b)]| with c = clamp to [-127, 127].
__device__ __forceinline__ uint16_t ci_int(int a, int b, const int16_t* tab) {
  const int qa = max(-127, min(127, a)) + 127, qb = max(-127, min(127, b)) + 127;
  const int d = (int)tab[qa] - (int)tab[qb];
  return (uint16_t)(d < 0 ? -d : d);
}

// Order-preserving 32-bit keys of non-negative metric values.
__device__ __forceinline__ uint32_t mkey(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t mkey(int v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t mkey(uint16_t v) { return (uint32_t)v; }

// Running argmax of (key, idx): larger key wins, equal keys go to the lower idx.
__device__ __forceinline__ void am_update(uint32_t& bk, uint32_t& bi, uint32_t k, uint32_t i) {
  if (k > bk || (k == bk && i < bi)) { bk = k; bi = i; }
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

}  // namespace ldpc
