// decode_me.cu -- multi-edge schedules, one frame per CTA.
//
// ME-CIRBP (Algorithm 5) and ME-LMD-CIRBP (Algorithm 6) update N_P variable
// nodes per step, chosen by the CI group quantiser of Algorithm 4.  "In
// parallel" is taken as a two-phase step: every selected p picks
// m*_p = argmax_i R_{i->p} on the pre-step state, all commits are applied, then
// every check that received a new V2C message (i in M(p)\m*_p) recomputes all
// its precomputed C2V messages, and every variable node next to one of them
// (and every p) recomputes L~ and D.  Results do not depend on the order of
// the parallel work.
//
// Checks are processed by teams of W lanes (W = power of two >= max check
// degree): lane r of a team owns edge r of the check and gets the exclude-one
// combination of eq. (2) (or min-sum) by W width-limited shuffles.
//
// Algorithm 4's random fill takes, from the fill group, the members with the
// smallest Philox4x32-10 keys (key = seed, counter = (n, step, frame)); the
// k-th smallest key is found by an exact 4 x 8-bit radix select.
#include "device_math.cuh"

namespace ldpc {

namespace {

struct MELayout {
  int C, P, lam, L, Lt, D, par, key, sel, est, best, cnl, hist, cnt, bits, misc, total;
};

__host__ __device__ inline MELayout me_layout(int arith, int M, int N, int E, int n_p, int dvm, int n_g) {
  const int msg = arith == kINT6 ? 1 : 4;
  const int llr = arith == kINT6 ? 2 : 4;
  const int dv = arith == kINT6 ? 2 : 4;
  MELayout l;
  int o = 0;
  l.C = o; o = align16(o + E * msg);
  l.P = o; o = align16(o + E * msg);
  l.lam = o; o = align16(o + N * llr);
  l.L = o; o = align16(o + N * llr);
  l.Lt = o; o = align16(o + N * llr);
  l.D = o; o = align16(o + N * dv);
  l.par = o; o = align16(o + ((M + 31) / 32) * 4);
  l.key = o; o = align16(o + N * 4);
  l.sel = o; o = align16(o + n_p * 4);
  l.est = o; o = align16(o + n_p * 4);
  l.best = o; o = align16(o + n_p * 8);
  l.cnl = o; o = align16(o + n_p * (dvm > 1 ? dvm - 1 : 1) * 8);
  l.hist = o; o = align16(o + 256 * 4);
  l.cnt = o; o = align16(o + n_g * 4);
  l.bits = o; o = align16(o + ((N + 31) / 32) * 4);
  l.misc = o; o = align16(o + 16 * 8);
  l.total = o;
  return l;
}

// shared scalars (misc area)
struct MEMisc {
  int unsat;
  int ncn;       // affected checks this step
  int nsel;      // selected VNs
  int npp;       // |P'| (ME-LMD)
  int kstar, fill_g, need, take_all_eq;
  uint32_t thr;  // radix threshold key
  int cnt_eq;
  int sz;
  int pad[5];
};

template <int A>
struct MEState {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  M_* C;
  M_* P;
  L_* lam;
  L_* L;
  L_* Lt;
  D_* D;
  uint32_t* par;
  uint32_t* key;
  int32_t* sel;
  int32_t* est;
  unsigned long long* best;
  int2* cnl;  // (check, owner k)
  int32_t* hist;
  int32_t* cnt;
  uint32_t* bits;  // selection bitmap over VNs
  MEMisc* misc;
  int16_t* tab;
};

__device__ __forceinline__ uint32_t philox_word0(uint32_t n, uint32_t step, uint64_t frame, uint64_t seed) {
  uint32_t c0 = n, c1 = step, c2 = (uint32_t)frame, c3 = (uint32_t)(frame >> 32);
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c0;
}

__device__ __forceinline__ float ci_me(const MEState<kFP32>&, float a, float b) { return ci_fp(a, b); }
__device__ __forceinline__ uint16_t ci_me(const MEState<kINT6>& s, int a, int b) {
  return ci_int(a, b, s.tab);
}

__device__ __forceinline__ int group_of(float d, int ng) { return min((int)floorf(d * (float)ng), ng - 1); }
__device__ __forceinline__ int group_of(uint16_t d, int ng) { return min((int)(((int)d * ng) / 65534), ng - 1); }

__device__ __forceinline__ uint32_t rkey_me(float p, float c) { return mkey(fabsf(p - c)); }
__device__ __forceinline__ uint32_t rkey_me(int8_t p, int8_t c) { return (uint32_t)abs((int)p - (int)c); }

// Team C2V of check m: lane r (< W) of the team owns edge r.  V2C = L_j - C[e]
// (eq. 1), output P[e] for every edge of the check (eq. 2 / min-sum).
template <int A>
__device__ __forceinline__ void team_c2v(const DevCode& g, const MEState<A>& s, int m, int r, int W,
                                         float clip) {
  const int c0 = m >= 0 ? __ldg(g.cn_ptr + m) : 0;
  const int dc = m >= 0 ? __ldg(g.cn_ptr + m + 1) - c0 : 0;
  const int e = c0 + r;
  if (A == kFP32) {
    float enc = 0.0f;
    if (r < dc) {
      const int j = __ldg(g.e_vn + e);
      enc = encode_fp((float)s.L[j] - (float)s.C[e], clip);
    }
    float sum = 0.0f;
    unsigned neg = 0;
    for (int k = 0; k < W; ++k) {
      const float v = __shfl_sync(kFull, enc, k, W);
      if (k != r && k < dc) {
        sum += fabsf(v);
        neg ^= __float_as_uint(v) >> 31;
      }
    }
    if (r < dc) ((float*)s.P)[e] = combine_fp(sum, neg, clip);
  } else {
    int enc = 0;
    if (r < dc) {
      const int j = __ldg(g.e_vn + e);
      enc = encode_int((int)s.L[j] - (int)s.C[e]);
    }
    int mag = 31;
    unsigned neg = 0;
    for (int k = 0; k < W; ++k) {
      const int v = __shfl_sync(kFull, enc, k, W);
      if (k != r && k < dc) {
        neg ^= (v < 0);
        mag = min(mag, abs(v));
      }
    }
    if (r < dc) ((int8_t*)s.P)[e] = (int8_t)(neg ? -mag : mag);
  }
}

template <int A>
__device__ __forceinline__ typename Arith<A>::llr me_total(const DevCode& g, const MEState<A>& s,
                                                           const typename Arith<A>::msg* X, int n) {
  using L_ = typename Arith<A>::llr;
  const int b0 = __ldg(g.vn_ptr + n), b1 = __ldg(g.vn_ptr + n + 1);
  L_ acc = s.lam[n];
  for (int k = b0; k < b1; ++k) acc = (L_)(acc + X[__ldg(g.vn_e + k)]);
  return acc;
}

// Algorithm 4 over the set S = {n : bit n of `excl` clear}, selecting `np`
// VNs into the bitmap s.bits (which already holds the excluded set when
// `excl_is_bits`).  Uses s.key, s.hist, s.cnt and misc.  All threads call it.
template <int A>
__device__ void alg4(const DevCode& g, const MEState<A>& s, int np, int ng, uint32_t step,
                     uint64_t frame, uint64_t seed) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int N = g.N;
  MEMisc* ms = s.misc;
  for (int i = tid; i < ng; i += nt) s.cnt[i] = 0;
  if (tid == 0) ms->sz = 0;
  __syncthreads();
  int my_sz = 0;
  for (int n = tid; n < N; n += nt) {  // line 2: G_i <- G_i u {n}, i = floor(D_n N_G)
    if (s.bits[n >> 5] & (1u << (n & 31))) continue;
    atomicAdd(&s.cnt[group_of(s.D[n], ng)], 1);
    ++my_sz;
  }
  my_sz = __reduce_add_sync(kFull, my_sz);
  if (lane == 0) atomicAdd(&ms->sz, my_sz);
  __syncthreads();
  if (tid == 0) {  // line 3: k* = max{k : |Q(k)| <= N_P}
    int kstar = 0, q = 0;
    if (ms->sz <= np) {
      kstar = ng;
      q = ms->sz;
    } else {
      for (int k = 1; k < ng; ++k) {
        if (q + s.cnt[ng - k] <= np) {
          q += s.cnt[ng - k];
          kstar = k;
        } else {
          break;
        }
      }
    }
    ms->kstar = kstar;
    ms->need = (kstar < ng) ? np - q : 0;
    ms->fill_g = ng - kstar - 1;
    ms->thr = 0;
  }
  __syncthreads();
  const int kstar = ms->kstar, fg = ms->fill_g;
  int need = ms->need;
  const int top = ng - kstar;
  if (need > 0) {
    // keys of the fill group, then the need-th smallest key by radix select
    for (int n = tid; n < N; n += nt) {
      if (s.bits[n >> 5] & (1u << (n & 31))) continue;
      if (group_of(s.D[n], ng) == fg) s.key[n] = philox_word0((uint32_t)n, step, frame, seed);
    }
    uint32_t prefix = 0;
    for (int pass = 3; pass >= 0; --pass) {
      const int shift = 8 * pass;
      const uint32_t hmask = pass == 3 ? 0u : (0xffffffffu << (shift + 8));
      for (int i = tid; i < 256; i += nt) s.hist[i] = 0;
      __syncthreads();
      for (int n = tid; n < N; n += nt) {
        if (s.bits[n >> 5] & (1u << (n & 31))) continue;
        if (group_of(s.D[n], ng) != fg) continue;
        const uint32_t k = s.key[n];
        if ((k & hmask) == (prefix & hmask)) atomicAdd(&s.hist[(k >> shift) & 255], 1);
      }
      __syncthreads();
      if (warp == 0) {
        // digit d with cum(<d) < need <= cum(<=d); lane owns digits 8 lane .. 8 lane + 7
        int loc[8], tot = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          loc[i] = s.hist[8 * lane + i];
          tot += loc[i];
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        int before = incl - tot;
        int found = -1, fb = 0, fc = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (found < 0 && before < need && need <= before + loc[i]) {
            found = 8 * lane + i;
            fb = before;
            fc = loc[i];
          }
          before += loc[i];
        }
        const unsigned hit = __ballot_sync(kFull, found >= 0);
        const int src = __ffs(hit) - 1;
        const int d = __shfl_sync(kFull, found, src);
        const int b4 = __shfl_sync(kFull, fb, src);
        const int c4 = __shfl_sync(kFull, fc, src);
        if (lane == 0) {
          ms->thr = prefix | ((uint32_t)d << shift);
          ms->need = need - b4;
          ms->cnt_eq = c4;
        }
      }
      __syncthreads();
      prefix = ms->thr;
      need = ms->need;
    }
  }
  const uint32_t thr = ms->thr;
  const bool all_eq = need > 0 && ms->cnt_eq == need;
  // selection: groups >= N_G - k* (line 3), plus fill members with key < thr
  // (or == thr) (lines 4-6)
  for (int n = tid; n < N; n += nt) {
    if (s.bits[n >> 5] & (1u << (n & 31))) continue;
    const int gi = group_of(s.D[n], ng);
    bool take = gi >= top;
    if (!take && need > 0 && gi == fg) {
      const uint32_t k = s.key[n];
      take = k < thr || (k == thr && all_eq);
    }
    if (take) atomicOr(&s.bits[n >> 5], 1u << (n & 31));
  }
  __syncthreads();
  if (need > 0 && !all_eq && tid == 0) {  // rare: equal keys at the threshold -> lowest n
    int left = need;
    for (int n = 0; n < N && left > 0; ++n) {
      if (group_of(s.D[n], ng) != fg || s.key[n] != thr) continue;
      if (s.bits[n >> 5] & (1u << (n & 31))) continue;  // excluded set (never the case for members)
      s.bits[n >> 5] |= 1u << (n & 31);
      --left;
    }
  }
  __syncthreads();
}

// Compact the selection bitmap into s.sel (ascending) and clear it.
template <int A>
__device__ void compact_selection(const DevCode& g, const MEState<A>& s, int np) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int words = (g.N + 31) / 32;
  if (warp == 0) {
    int base = 0;
    for (int w0 = 0; w0 < words; w0 += 32) {
      const int w = w0 + lane;
      const uint32_t bw = w < words ? s.bits[w] : 0u;
      const int c = __popc(bw);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      int pos = base + incl - c;
      uint32_t x = bw;
      while (x) {
        const int bit = __ffs(x) - 1;
        x &= x - 1;
        if (pos < np) s.sel[pos] = w * 32 + bit;
        ++pos;
      }
      base += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) s.misc->nsel = min(base, np);
  }
  __syncthreads();
  for (int w = tid; w < words; w += nt) s.bits[w] = 0u;
  __syncthreads();
}

template <int A, int SCHED>
__global__ void __launch_bounds__(256) me_decode_kernel(const DecodeArgs a) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t b = blockIdx.x;
  const DevCode& g = a.g;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int N = g.N, E = g.E, M = g.M;
  const int np = a.n_p, ng = a.n_g;
  const MELayout ly = me_layout(A, M, N, E, np, g.dv_max, ng);
  MEState<A> s;
  s.C = (M_*)(smem_raw + ly.C);
  s.P = (M_*)(smem_raw + ly.P);
  s.lam = (L_*)(smem_raw + ly.lam);
  s.L = (L_*)(smem_raw + ly.L);
  s.Lt = (L_*)(smem_raw + ly.Lt);
  s.D = (D_*)(smem_raw + ly.D);
  s.par = (uint32_t*)(smem_raw + ly.par);
  s.key = (uint32_t*)(smem_raw + ly.key);
  s.sel = (int32_t*)(smem_raw + ly.sel);
  s.est = (int32_t*)(smem_raw + ly.est);
  s.best = (unsigned long long*)(smem_raw + ly.best);
  s.cnl = (int2*)(smem_raw + ly.cnl);
  s.hist = (int32_t*)(smem_raw + ly.hist);
  s.cnt = (int32_t*)(smem_raw + ly.cnt);
  s.bits = (uint32_t*)(smem_raw + ly.bits);
  s.misc = (MEMisc*)(smem_raw + ly.misc);
  __shared__ int16_t tab_int[256];
  s.tab = tab_int;
  MEMisc* ms = s.misc;
  const float clip = a.llr_clip;
  const uint64_t frame = a.frame_offset + (uint64_t)b;
  int W = 1;
  while (W < g.dc_max) W <<= 1;
  const int tpw = 32 / W;  // teams per warp
  const int team = lane / W, r = lane % W;

  if (A == kINT6)
    for (int i = tid; i < 256; i += nt) tab_int[i] = a.ci_table[i];
  int bad = 0;
  for (int n = tid; n < N; n += nt) {
    L_ v;
    if (A == kFP32) {
      const float x = ((const float*)a.llr)[b * N + n];
      bad |= !isfinite(x);
      v = (L_)x;
    } else {
      const int x = ((const int8_t*)a.llr)[b * N + n];
      bad |= (x < -31 || x > 31);
      v = (L_)x;
    }
    s.lam[n] = v;
    s.L[n] = v;
  }
  for (int e = tid; e < E; e += nt) s.C[e] = (M_)0;
  for (int w = tid; w < (N + 31) / 32; w += nt) s.bits[w] = 0u;
  for (int w = tid; w < (M + 31) / 32; w += nt) s.par[w] = 0u;
  if (tid == 0) ms->unsat = 0;
  if (__syncthreads_or(bad)) {
    for (int n = tid; n < N; n += nt) {
      if (a.hard) a.hard[b * N + n] = 0;
      if (a.llr_out) a.llr_out[b * N + n] = (float)s.lam[n];
    }
    if (tid == 0) {
      if (a.updates) a.updates[b] = 0;
      if (a.converged) a.converged[b] = 2;
      atomicOr(a.status, 1u);
    }
    return;
  }
  // ---- Alg. 5/6 lines 1-3: every L~^C, R, L~, D; syndrome of bsgn(lambda)
  for (int t0 = warp * tpw; t0 < M; t0 += nw * tpw) {
    const int m = t0 + team;
    team_c2v<A>(g, s, m < M ? m : -1, r, W, clip);
  }
  for (int m = tid; m < M; m += nt) {
    const int c0 = __ldg(g.cn_ptr + m), c1 = __ldg(g.cn_ptr + m + 1);
    unsigned p = 0;
    for (int e = c0; e < c1; ++e) p ^= (s.L[__ldg(g.e_vn + e)] < (L_)0);
    if (p) {
      atomicOr(&s.par[m >> 5], 1u << (m & 31));
      atomicAdd(&ms->unsat, 1);
    }
  }
  __syncthreads();
  for (int n = tid; n < N; n += nt) {
    const L_ lt = me_total<A>(g, s, s.P, n);
    s.Lt[n] = lt;
    s.D[n] = ci_me(s, s.L[n], lt);
  }
  __syncthreads();

  int64_t count = 0;
  uint32_t step = 0;
  bool stop = a.check_interval > 0 && ms->unsat == 0;
  if (!stop && a.max_updates > 0) {  // Alg. 5 line 4 / Alg. 6 line 4
    alg4<A>(g, s, np, ng, step, frame, a.seed);
    compact_selection<A>(g, s, np);
  }
  while (!stop && count < a.max_updates) {
    int nsel = ms->nsel;
    if (nsel <= 0) break;  // nothing selectable: the step would not advance
    if ((int64_t)nsel > a.max_updates - count) nsel = (int)(a.max_updates - count);
    // -- m*_p = argmax_i R_{i->p}, i in M(p), on the pre-step state
    for (int k = tid; k < nsel; k += nt) {
      const int p = s.sel[k];
      const int v0 = __ldg(g.vn_ptr + p), v1 = __ldg(g.vn_ptr + p + 1);
      uint32_t bk = 0, bi = 0xffffffffu;
      for (int q = v0; q < v1; ++q) {
        const int e = __ldg(g.vn_e + q);
        am_update(bk, bi, rkey_me(s.P[e], s.C[e]), (uint32_t)e);
      }
      s.est[k] = (int)bi;
      s.best[k] = 0ull;
    }
    if (tid == 0) ms->ncn = 0;
    __syncthreads();
    // -- commits, L_p, syndrome, trace, affected checks i in M(p)\m*_p
    for (int k = tid; k < nsel; k += nt) {
      const int p = s.sel[k], es = s.est[k], ms_ = __ldg(g.e_cn + es);
      s.C[es] = s.P[es];
      const L_ lold = s.L[p];
      const L_ lnew = me_total<A>(g, s, s.C, p);
      s.L[p] = lnew;
      const bool flip = (lold < (L_)0) != (lnew < (L_)0);
      const int v0 = __ldg(g.vn_ptr + p), v1 = __ldg(g.vn_ptr + p + 1);
      for (int q = v0; q < v1; ++q) {
        const int m = __ldg(g.e_cn + __ldg(g.vn_e + q));
        if (flip) {
          const uint32_t bit = 1u << (m & 31);
          const uint32_t old = atomicXor(&s.par[m >> 5], bit);
          atomicAdd(&ms->unsat, (old & bit) ? -1 : 1);
        }
        if (m != ms_) {
          const int pos = atomicAdd(&ms->ncn, 1);
          s.cnl[pos] = make_int2(m, k);
        }
      }
      if (a.trace) a.trace[b * a.max_updates + count + k] = es;
    }
    __syncthreads();
    const int ncn = ms->ncn;
    // -- precomputed C2V of every affected check
    for (int t0 = warp * tpw; t0 < ncn; t0 += nw * tpw) {
      const int t = t0 + team;
      team_c2v<A>(g, s, t < ncn ? s.cnl[t].x : -1, r, W, clip);
    }
    __syncthreads();
    // -- L~_j, D_j next to affected checks (and of every p); LMD candidates
    for (int t0 = warp * tpw; t0 < ncn; t0 += nw * tpw) {
      const int t = t0 + team;
      if (t >= ncn) continue;
      const int2 ck = s.cnl[t];
      const int c0 = __ldg(g.cn_ptr + ck.x), dc = __ldg(g.cn_ptr + ck.x + 1) - c0;
      if (r >= dc) continue;
      const int j = __ldg(g.e_vn + c0 + r);
      const L_ lt = me_total<A>(g, s, s.P, j);
      const D_ d = ci_me(s, s.L[j], lt);
      s.Lt[j] = lt;
      s.D[j] = d;
      if (SCHED == kMELMD && j != s.sel[ck.y]) {
        const unsigned long long key = ((unsigned long long)mkey(d) << 32) | (0xffffffffu - (uint32_t)j);
        atomicMax(&s.best[ck.y], key);
      }
    }
    for (int k = tid; k < nsel; k += nt) {
      const int p = s.sel[k];
      const L_ lt = me_total<A>(g, s, s.P, p);
      s.Lt[p] = lt;
      s.D[p] = ci_me(s, s.L[p], lt);
    }
    __syncthreads();
    count += nsel;
    ++step;
    if (a.check_interval > 0 && (count / a.check_interval) > ((count - nsel) / a.check_interval) &&
        ms->unsat == 0)
      break;
    if (count >= a.max_updates) break;
    if (SCHED == kMECIRBP) {
      alg4<A>(g, s, np, ng, step, frame, a.seed);  // Alg. 5 line 4
      compact_selection<A>(g, s, np);
      continue;
    }
    // -- Alg. 6 lines 6-10: P' = {argmax_{j in U(m*_p, p)} D_j}; degree-1 rule
    for (int k = tid; k < nsel; k += nt) {
      const int p = s.sel[k];
      if (__ldg(g.vn_ptr + p + 1) - __ldg(g.vn_ptr + p) == 1) {
        const int mm = __ldg(g.e_cn + s.est[k]);
        const int c0 = __ldg(g.cn_ptr + mm), c1 = __ldg(g.cn_ptr + mm + 1);
        unsigned long long bk = 0ull;
        for (int e = c0; e < c1; ++e) {
          const int j = __ldg(g.e_vn + e);
          if (j == p) continue;
          const unsigned long long key = ((unsigned long long)mkey(s.D[j]) << 32) | (0xffffffffu - (uint32_t)j);
          bk = key > bk ? key : bk;
        }
        s.best[k] = bk;
      }
    }
    if (tid == 0) ms->npp = 0;
    __syncthreads();
    int mine = 0;
    for (int k = tid; k < nsel; k += nt) {
      const unsigned long long bk = s.best[k];
      if (bk == 0ull) continue;  // empty candidate set
      const int j = (int)(0xffffffffu - (uint32_t)(bk & 0xffffffffull));
      const uint32_t bit = 1u << (j & 31);
      const uint32_t old = atomicOr(&s.bits[j >> 5], bit);
      mine += (old & bit) ? 0 : 1;
    }
    mine = __reduce_add_sync(kFull, mine);
    if (lane == 0 && mine) atomicAdd(&ms->npp, mine);
    __syncthreads();
    const int npp = ms->npp;
    if (npp < np) alg4<A>(g, s, np - npp, ng, step, frame, a.seed);  // lines 11-13
    compact_selection<A>(g, s, np);
  }

  for (int n = tid; n < N; n += nt) {
    if (a.hard) a.hard[b * N + n] = (uint8_t)(s.L[n] < (L_)0);
    if (a.llr_out) a.llr_out[b * N + n] = (float)s.L[n];
  }
  if (tid == 0) {
    if (a.updates) a.updates[b] = count;
    if (a.converged) a.converged[b] = ms->unsat == 0 ? 1 : 0;
  }
}

template <int A, int S>
cudaError_t launch_me_one(const DecodeArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)a.smem_per_frame;
  auto k = me_decode_kernel<A, S>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<(unsigned)a.batch, 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t me_smem_per_frame(int arith, int sched, const DevCode& g, int n_p, int n_g) {
  (void)sched;
  if (g.dc_max > 32) return 0;
  return (size_t)me_layout(arith, g.M, g.N, g.E, n_p, g.dv_max, n_g).total;
}

cudaError_t launch_me(const DecodeArgs& a, int arith, int sched, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  if (arith == kFP32) {
    if (sched == kMECIRBP) return launch_me_one<kFP32, kMECIRBP>(a, s);
    return launch_me_one<kFP32, kMELMD>(a, s);
  }
  if (sched == kMECIRBP) return launch_me_one<kINT6, kMECIRBP>(a, s);
  return launch_me_one<kINT6, kMELMD>(a, s);
}

}  // namespace ldpc
