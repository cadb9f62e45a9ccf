// decode_se.cu -- single-edge dynamic schedules, one frame per warp.
//
// Residual BP (Sec. 2.A, steps 1-4), CIRBP (Algorithm 1), LMD-CIRBP
// (Algorithm 3), LMDRBP and sLMDRBP (Algorithm 2, with and without its line 10)
// commit one check-to-variable (C2V) message per update.  The
// chain select -> commit -> refresh -> select is serial within a frame, so a
// frame is one warp; frames are the warps of the CTAs.  Per update:
//   - lanes k < d_v(n*) own the edges into the target n*: residual argmax
//     (Alg. 1 line 8 / Alg. 3 line 5), commit, L_{n*} as a warp sum;
//   - the d_v - 1 refreshed checks i in M(n*)\m* (Alg. 1 lines 10-13) are
//     handled by teams of W lanes, one lane per edge: new V2C inputs, the
//     exclude-one C2V of eq. (2) (or min-sum) by width-W shuffles, then
//     L~_j and D_j (eq. 8) of j in N(i)\n*, which are also the LMD candidates
//     (LMD-CIRBP by D_j, LMDRBP by the new residuals of those edges).
// Per-frame state (SELayout): the V region lam/L[N], D[N], Rmax/Ridx[M]
// (largest residual per check, for the global argmax of eq. (5): RBP and
// CIRBP's fallback), par (syndrome bits of the tentative decisions bsgn(L),
// Sec. 2.A) and the block maxima of D and Rmax; the E region C[E] L^C, P[E]
// L~^C.  Forms: both regions in shared memory (several frames per CTA), both in
// a global slot, or the V region in shared memory and the E region in a global
// slot (split form).  Where the V region is in shared memory, CIRBP's and RBP's
// global argmaxes read the block maxima (one key per 32 VNs or checks, kept
// exact) and one block instead of every entry.
// The graph is a QCGraph (protograph arithmetic) or TabGraph (CSR tables), both
// staged once per CTA in shared memory.
#include "device_math.cuh"

namespace ldpc {

namespace {

template <int A>
struct SEState {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  M_* C;
  M_* P;
  L_* lam;
  L_* L;
  D_* D;
  M_* Rmax;
  int32_t* Ridx;
  uint32_t* par;
  uint32_t* Dblk;    // largest key of D per block of 32 VNs (CIRBP)
  uint32_t* Ddirty;  // blocks whose largest D may have dropped
  uint32_t* Rblk;    // largest per-check residual key per block of 32 checks (RBP, CIRBP)
  uint32_t* Rdirty;
  int16_t* tab;
  int32_t* Lt;       // CIRBP, LMD-CIRBP: sum over the edges of each VN of L~^C, exact integer
  float fx, ifx;     // FP32 fixed point of those sums: 2^k and 2^-k
};

// message -> exact integer term of the L~ sum, and L~ = lambda + that sum
__device__ __forceinline__ int se_fix(const SEState<kFP32>& s, float x) { return __float2int_rn(x * s.fx); }
__device__ __forceinline__ int se_fix(const SEState<kINT6>&, int8_t x) { return (int)x; }
__device__ __forceinline__ float se_lt(const SEState<kFP32>& s, int n) { return s.lam[n] + (float)s.Lt[n] * s.ifx; }
__device__ __forceinline__ int16_t se_lt(const SEState<kINT6>& s, int n) { return (int16_t)(s.lam[n] + s.Lt[n]); }

// Upper level of the global argmaxes: blk[b] is the largest key of block b (32
// entries).  A key that grows raises its block's entry at once; a key that
// drops from a block's largest value marks the block dirty, and the block is
// recomputed before the next search (blk_fix).  The entry thus always equals
// the block's largest key when it is read.
__device__ __forceinline__ void blk_note(uint32_t* blk, uint32_t* dirty, int i, uint32_t kold, uint32_t knew) {
  const int b = i >> 5;
  if (knew > kold) atomicMax(&blk[b], knew);
  else if (knew < kold && kold == blk[b]) atomicOr(&dirty[b >> 5], 1u << (b & 31));
}

// recompute the dirty blocks (whole warp); key(i) is entry i's key, 0 past n
template <class K>
__device__ __forceinline__ void blk_fix(uint32_t* blk, uint32_t* dirty, int n, const K& key) {
  const int lane = threadIdx.x & 31, nb = (n + 31) >> 5;
  __syncwarp();
  for (int w = 0; w < ((nb + 31) >> 5); ++w) {
    uint32_t dm = dirty[w];
    if (dm == 0u) continue;
    __syncwarp();
    if (lane == 0) dirty[w] = 0u;
    while (dm != 0u) {
      const int b = w * 32 + __ffs(dm) - 1;
      dm &= dm - 1u;
      const int i = b * 32 + lane;
      const uint32_t mx = __reduce_max_sync(kFull, i < n ? key(i) : 0u);
      if (lane == 0) blk[b] = mx;
    }
  }
  __syncwarp();
}

// every block from scratch (whole warp)
template <class K>
__device__ __forceinline__ void blk_build(uint32_t* blk, uint32_t* dirty, int n, const K& key) {
  const int lane = threadIdx.x & 31, nb = (n + 31) >> 5;
  for (int b = 0; b < nb; ++b) {
    const int i = b * 32 + lane;
    const uint32_t mx = __reduce_max_sync(kFull, i < n ? key(i) : 0u);
    if (lane == 0) blk[b] = mx;
  }
  for (int w = lane; w < ((nb + 31) >> 5); w += 32) dirty[w] = 0u;
  __syncwarp();
}

__device__ __forceinline__ float ci_val(const SEState<kFP32>&, float a, float b) { return ci_fp(a, b); }
__device__ __forceinline__ uint16_t ci_val(const SEState<kINT6>& s, int a, int b) {
  return ci_int(a, b, s.tab);
}

// two warp sums at once (independent butterflies interleave)
__device__ __forceinline__ void warp_sum2(float& a, float& b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(kFull, a, o);
    b += __shfl_xor_sync(kFull, b, o);
  }
}
__device__ __forceinline__ void warp_sum2(int16_t& a, int16_t& b) {
  a = (int16_t)__reduce_add_sync(kFull, (int)a);
  b = (int16_t)__reduce_add_sync(kFull, (int)b);
}

// argmax over D of every VN, lowest index on ties (Alg. 1 line 4)
template <int A>
__device__ __forceinline__ int global_argmax_D(int N, const SEState<A>& s, uint32_t& key) {
  uint32_t bk = 0, bi = 0xffffffffu;
  for (int n = threadIdx.x & 31; n < N; n += 32) {
    const uint32_t k = mkey(s.D[n]);
    if (k > bk || bi == 0xffffffffu) {
      bk = k;
      bi = n;
    }
  }
  return (int)warp_argmax(bk, bi, key);
}

// the same through the block maxima: the first block holding the largest key,
// then the lowest index with that key in it
template <int A>
__device__ __forceinline__ int global_argmax_D_blk(int N, const SEState<A>& s, uint32_t& key) {
  const int lane = threadIdx.x & 31, nb = (N + 31) >> 5;
  blk_fix(s.Dblk, s.Ddirty, N, [&](int i) { return mkey(s.D[i]); });
  uint32_t bk = 0, bi = 0xffffffffu;
  for (int b = lane; b < nb; b += 32) {
    const uint32_t k = s.Dblk[b];
    if (k > bk || bi == 0xffffffffu) {
      bk = k;
      bi = (uint32_t)b;
    }
  }
  const int B = (int)warp_argmax(bk, bi, key);
  const int n = B * 32 + lane;
  const bool hit = n < N && mkey(s.D[n]) == key;
  const uint32_t r = __reduce_min_sync(kFull, hit ? (uint32_t)n : 0xffffffffu);
  return r != 0xffffffffu ? (int)r : global_argmax_D<A>(N, s, key);  // (the block entries are exact)
}

// argmax over the residual of every edge, eq. (5), via the per-check maxima
template <int A>
__device__ __forceinline__ int global_argmax_R(int M, const SEState<A>& s) {
  uint32_t bk = 0, bi = 0xffffffffu;
  for (int m = threadIdx.x & 31; m < M; m += 32) {
    const uint32_t k = rkey(s.Rmax[m], (typename Arith<A>::msg)0);
    if (k > bk || bi == 0xffffffffu) {
      bk = k;
      bi = (uint32_t)s.Ridx[m];
    }
  }
  uint32_t key;
  return (int)warp_argmax(bk, bi, key);
}

// the same through the block maxima of the per-check residual maxima (edge ids
// grow with the check index, so the lowest check holding the largest key has
// the lowest edge id among them)
template <int A>
__device__ __forceinline__ int global_argmax_R_blk(int M, const SEState<A>& s) {
  using M_ = typename Arith<A>::msg;
  const int lane = threadIdx.x & 31, mb = (M + 31) >> 5;
  blk_fix(s.Rblk, s.Rdirty, M, [&](int m) { return rkey(s.Rmax[m], (M_)0); });
  uint32_t bk = 0, bi = 0xffffffffu;
  for (int b = lane; b < mb; b += 32) {
    const uint32_t k = s.Rblk[b];
    if (k > bk || bi == 0xffffffffu) {
      bk = k;
      bi = (uint32_t)b;
    }
  }
  uint32_t key;
  const int B = (int)warp_argmax(bk, bi, key);
  const int m = B * 32 + lane;
  const bool hit = m < M && rkey(s.Rmax[m], (M_)0) == key;
  const uint32_t mm = __reduce_min_sync(kFull, hit ? (uint32_t)m : 0xffffffffu);
  return mm != 0xffffffffu ? s.Ridx[mm] : global_argmax_R<A>(M, s);  // (the block entries are exact)
}

// per-check largest residual (value, lowest edge id), one lane; with `blk` the
// block maxima follow
template <int A, class G>
__device__ __forceinline__ void refresh_rmax(const G& g, const SEState<A>& s, int m, bool blk = false) {
  const typename G::C cc = g.cn(m);
  uint32_t bk = 0, bi = (uint32_t)cc.b;
  for (int e = cc.b; e < cc.b + cc.d; ++e) {
    const uint32_t k = rkey(s.P[e], s.C[e]);
    if (k > bk) {
      bk = k;
      bi = e;
    }
  }
  using M_ = typename Arith<A>::msg;
  const uint32_t kold = blk ? rkey(s.Rmax[m], (M_)0) : 0u;
  if (A == kFP32) s.Rmax[m] = (M_)__uint_as_float(bk);
  else s.Rmax[m] = (M_)bk;
  s.Ridx[m] = (int32_t)bi;
  if (blk) blk_note(s.Rblk, s.Rdirty, m, kold, bk);
}

// Decode one frame of code `gd` with the V region of its state at `vbase` and
// the E region at `ebase` (shared or global memory; see SELayout).  kVs: the V
// region is in shared memory, where the block maxima of the global argmaxes
// pay (in global memory their atomics cost more than the plain scans save).
template <int A, int SCHED, class G, bool kVs>
__device__ __forceinline__ void se_frame(const DecodeArgs& a, const GraphDesc& gd, const G& g, const FrameIO& io,
                                         unsigned char* vbase, unsigned char* ebase) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  constexpr bool kNeedR = SCHED != kLMD;
  // L~_j of the refreshed VNs from sums kept up to date by the check updates
  // (integers: the sum does not depend on the order of the updates; FP32
  // messages in fixed point x 2^k, d_v,max * llr_clip * 2^k < 2^30) instead
  // of d_v(j) reads of L~^C per refreshed VN
  constexpr bool kLt = SCHED == kLMD || SCHED == kCIRBP;
  constexpr bool kDblk = kVs && SCHED == kCIRBP;                   // global argmax of D every update
  constexpr bool kRblk = kVs && (SCHED == kCIRBP || SCHED == kRBP);  // global argmax of the residuals
  const int lane = threadIdx.x & 31;
  const int N = gd.N, E = gd.E, M = gd.M;
  const SELayout ly = se_layout(A, M, N, E, SCHED);
  SEState<A> s;
  s.C = (M_*)(ebase + ly.C);
  s.P = (M_*)(ebase + ly.P);
  s.lam = (L_*)(vbase + ly.lam);
  s.L = (L_*)(vbase + ly.L);
  s.D = (D_*)(vbase + ly.D);
  s.Rmax = (M_*)(vbase + ly.Rmax);
  s.Ridx = (int32_t*)(vbase + ly.Ridx);
  s.par = (uint32_t*)(vbase + ly.par);
  s.Dblk = (uint32_t*)(vbase + ly.Dblk);
  s.Ddirty = (uint32_t*)(vbase + ly.Ddirty);
  s.Rblk = (uint32_t*)(vbase + ly.Rblk);
  s.Rdirty = (uint32_t*)(vbase + ly.Rdirty);
  s.tab = (int16_t*)(vbase + ly.tab);
  s.Lt = (int32_t*)(vbase + ly.Lt);
  {
    const int k = min(24, 29 - ilogbf((float)gd.dv_max * a.llr_clip));
    s.fx = __int_as_float((127 + k) << 23);
    s.ifx = __int_as_float((127 - k) << 23);
  }
  const float clip = a.llr_clip;
  const int W = team_width(gd.dc_max), tpw = 32 / W, team = lane / W, r = lane % W;

  if (A == kINT6)
    for (int i = lane; i < 256; i += 32) s.tab[i] = a.ci_table[i];
  __syncwarp();

  // ---- channel LLRs (coalesced) and input validation
  bool bad = false;
  for (int n = lane; n < N; n += 32) {
    L_ v;
    if (A == kFP32) {
      const float x = ((const float*)io.llr)[n];
      bad |= !isfinite(x);
      v = (L_)x;
    } else {
      const int x = ((const int8_t*)io.llr)[n];
      bad |= (x < -31 || x > 31);
      v = (L_)x;
    }
    s.lam[n] = v;
    s.L[n] = v;
  }
  for (int e = lane; e < E; e += 32) s.C[e] = (M_)0;
  if (__any_sync(kFull, bad)) {
    for (int n = lane; n < N; n += 32) {
      if (io.hard) io.hard[n] = 0;
      if (io.llr_out) io.llr_out[n] = (float)s.lam[n];
    }
    if (lane == 0) {
      if (io.updates) *io.updates = 0;
      if (io.converged) *io.converged = 2;
      atomicOr(a.status, 1u);
    }
    return;
  }
  __syncwarp();

  // ---- Alg. 1 lines 1-3: L^C = 0, L = L^V = lambda, every L~^C, R, L~, D
  for (int t0 = 0; t0 < M; t0 += tpw) {
    const int m = t0 + team;
    int e, j;
    M_ out;
    const int dc = team_c2v<A, G>(g, s.C, s.L, m < M ? m : -1, r, W, clip, e, j, out);
    if (r < dc) s.P[e] = out;
  }
  __syncwarp();
  for (int n = lane; n < N; n += 32) {
    if (kLt) {
      const typename G::V v = g.vn(n);
      int acc = 0;
      for (int k = 0; k < v.d; ++k) {
        int e, m;
        g.vedge(v, k, e, m);
        acc += se_fix(s, s.P[e]);
      }
      s.Lt[n] = acc;
      s.D[n] = ci_val(s, s.L[n], se_lt(s, n));
    } else {
      s.D[n] = ci_val(s, s.L[n], vn_total<A, G>(g, s.lam, s.P, n));
    }
  }
  uint32_t unsat = 0;
  for (int m0 = 0; m0 < M; m0 += 32) {
    const int m = m0 + lane;
    unsigned p = 0;
    if (m < M) {
      const typename G::C cc = g.cn(m);
      for (int k = 0; k < cc.d; ++k) p ^= (s.L[g.cvn(cc, k)] < (L_)0);
    }
    const unsigned bits = __ballot_sync(kFull, p);
    if (lane == 0) s.par[m0 >> 5] = bits;
    unsat += __popc(bits);
  }
  __syncwarp();
  if (kNeedR)
    for (int m = lane; m < M; m += 32) refresh_rmax<A, G>(g, s, m);
  __syncwarp();
  if (kDblk) blk_build(s.Dblk, s.Ddirty, N, [&](int i) { return mkey(s.D[i]); });
  if (kRblk) blk_build(s.Rblk, s.Rdirty, M, [&](int m) { return rkey(s.Rmax[m], (M_)0); });
  // D_j <- d, with the block maxima of CIRBP's global argmax
  auto set_D = [&](int j, D_ d) {
    if (kDblk) {
      const uint32_t ko = mkey(s.D[j]);
      s.D[j] = d;
      blk_note(s.Dblk, s.Ddirty, j, ko, mkey(d));
    } else {
      s.D[j] = d;
    }
  };

  // ---- schedule loop
  constexpr bool kLMDR = SCHED == kLMDRBP || SCHED == kSLMDRBP;
  int64_t count = 0, nfall = 0, left = a.check_interval;
  int nstar = 0;
  int enext = -1;  // LMDRBP: edge found by Alg. 2 line 9 for the next update (-1: none)
  bool stop = (a.check_interval > 0 && unsat == 0);
  if (!stop && SCHED == kLMD) {
    uint32_t k;
    nstar = global_argmax_D<A>(N, s, k);  // Alg. 3 line 4
  }
  while (!stop && count < io.max_updates) {
    // -- selection
    int eglob = -1;  // RBP / CIRBP fallback: the global residual argmax fixes e*
    if (SCHED == kRBP) {
      eglob = kRblk ? global_argmax_R_blk<A>(M, s) : global_argmax_R<A>(M, s);
      nstar = g.evn(eglob);
    } else if (kLMDR) {
      if (enext < 0) {  // Alg. 2 line 3, and an empty candidate set
        eglob = global_argmax_R<A>(M, s);
        nstar = g.evn(eglob);
      } else {
        nstar = g.evn(enext);  // n' of line 9; LMDRBP re-selects its check (line 10)
        if (SCHED == kSLMDRBP) eglob = enext;
      }
    } else if (SCHED == kCIRBP) {
      uint32_t dkey;
      nstar = kDblk ? global_argmax_D_blk<A>(N, s, dkey) : global_argmax_D<A>(N, s, dkey);
      const bool fallback = (A == kFP32) ? (__uint_as_float(dkey) < a.gamma_f) : ((int)dkey < a.gamma_i);
      if (fallback) {  // Alg. 1 line 6
        eglob = kRblk ? global_argmax_R_blk<A>(M, s) : global_argmax_R<A>(M, s);
        nstar = g.evn(eglob);
        ++nfall;
      }
    }
    // lane k < d_v owns the k-th edge into n* (d_v <= 32 for this form)
    const typename G::V vv = g.vn(nstar);
    const int dv = vv.d;
    int my_e = 0, my_m = -1;
    M_ my_p = (M_)0, my_c = (M_)0;
    uint32_t rk = 0, ri = 0xffffffffu;
    if (lane < dv) {
      g.vedge(vv, lane, my_e, my_m);
      my_p = s.P[my_e];
      my_c = s.C[my_e];
      rk = rkey(my_p, my_c);
      ri = (uint32_t)my_e;
    }
    uint32_t kk;
    const int estar = eglob >= 0 ? eglob : (int)warp_argmax(rk, ri, kk);  // Alg. 1 line 8 / Alg. 3 line 5
    const unsigned own = __ballot_sync(kFull, lane < dv && my_e == estar);
    const int kstar = __ffs(own) - 1;
    const int mstar = __shfl_sync(kFull, my_m, kstar);

    // -- commit (Alg. 1 line 9): L^C <- L~^C, update L_{n*}; L~_{n*} is unchanged
    //    by the commit and is summed alongside for D_{n*}
    const L_ Lold = s.L[nstar];
    L_ Lnew = (L_)0, Ltn = (L_)0;
    if (lane < dv) {
      Lnew = (L_)(lane == kstar ? my_p : my_c);
      Ltn = (L_)my_p;
    }
    if (A == kFP32 && lane == 0) {
      Lnew = (L_)(Lnew + s.lam[nstar]);
      Ltn = (L_)(Ltn + s.lam[nstar]);
    }
    warp_sum2(Lnew, Ltn);
    if (A == kINT6) {
      Lnew = (L_)(Lnew + s.lam[nstar]);
      Ltn = (L_)(Ltn + s.lam[nstar]);
    }
    if (lane == kstar) s.C[estar] = my_p;
    if (lane == 0) {
      s.L[nstar] = Lnew;
      set_D(nstar, ci_val(s, Lnew, Ltn));  // reading: D of n* follows L_{n*}
    }
    if ((Lold < (L_)0) != (Lnew < (L_)0)) {  // tentative decision flipped
      int delta = 0;
      if (lane < dv) {
        const uint32_t bit = 1u << (my_m & 31);
        const uint32_t old = atomicXor(s.par + (my_m >> 5), bit);
        delta = (old & bit) ? -1 : 1;
      }
      unsat += __reduce_add_sync(kFull, delta);
    }
    if (lane == 0 && io.trace) io.trace[count] = estar;
    __syncwarp();

    // -- refresh (Alg. 1 lines 10-13): team i handles the i-th check of M(n*)\m*:
    //    new V2C inputs and precomputed C2V (eq. 2), then L~_j and D_j of its
    //    variables j != n* (also the LMD candidates)
    const int nref = dv - 1;
    // new L~^C of edge e (towards j); with kLt its L~ sum follows by the exact delta
    auto put_p = [&](int e, int j, M_ out) {
      if (kLt) {
        const int delta = se_fix(s, out) - se_fix(s, s.P[e]);
        if (delta != 0) atomicAdd(&s.Lt[j], delta);
      }
      s.P[e] = out;
    };
    uint32_t ck = 0, cidx = 0xffffffffu;
    uint32_t rck = 0, rcidx = 0xffffffffu;
    if (nref <= tpw) {  // one pass of teams
      const int k = team < kstar ? team : team + 1;
      const int m = __shfl_sync(kFull, my_m, k & 31);
      int e, j;
      M_ out;
      const int dc = team_c2v<A, G>(g, s.C, s.L, team < nref ? m : -1, r, W, clip, e, j, out);
      const bool mine = r < dc && j != nstar;
      if (mine) {
        put_p(e, j, out);
        if (kLMDR) am_update(rck, rcidx, rkey(out, s.C[e]), (uint32_t)e);  // Alg. 2 line 9
      }
      __syncwarp();
      if (mine) {
        const D_ d = ci_val(s, s.L[j], kLt ? se_lt(s, j) : vn_total<A, G>(g, s.lam, s.P, j));
        set_D(j, d);
        am_update(ck, cidx, mkey(d), (uint32_t)j);
      }
    } else {
      for (int i0 = 0; i0 < nref; i0 += tpw) {
        const int i = i0 + team;
        const int k = i < kstar ? i : i + 1;
        const int m = __shfl_sync(kFull, my_m, k & 31);
        int e, j;
        M_ out;
        const int dc = team_c2v<A, G>(g, s.C, s.L, i < nref ? m : -1, r, W, clip, e, j, out);
        if (r < dc && j != nstar) {
          put_p(e, j, out);
          if (kLMDR) am_update(rck, rcidx, rkey(out, s.C[e]), (uint32_t)e);  // Alg. 2 line 9
        }
      }
      __syncwarp();
      for (int i0 = 0; i0 < nref; i0 += tpw) {
        const int i = i0 + team;
        const int k = i < kstar ? i : i + 1;
        const int m = __shfl_sync(kFull, my_m, k & 31);
        if (i >= nref) continue;
        const typename G::C cc = g.cn(m);
        if (r >= cc.d) continue;
        const int j = g.cvn(cc, r);
        if (j == nstar) continue;
        const D_ d = ci_val(s, s.L[j], kLt ? se_lt(s, j) : vn_total<A, G>(g, s.lam, s.P, j));
        set_D(j, d);
        am_update(ck, cidx, mkey(d), (uint32_t)j);
      }
    }
    __syncwarp();
    if (kNeedR && lane < dv) refresh_rmax<A, G>(g, s, my_m, kRblk);
    __syncwarp();

    ++count;
    if (check_due(left, a.check_interval, 1) && unsat == 0) break;

    // -- LMDRBP: next edge = argmax of the residuals just refreshed (Alg. 2 line
    //    9), or over the edges of m* to N(m*)\n* when d_v(n*) = 1 (Sec. 5.A);
    //    none: the global residual argmax next time
    if (kLMDR) {
      if (dv == 1) {
        rck = 0;
        rcidx = 0xffffffffu;
        const typename G::C cc = g.cn(mstar);
        for (int q = lane; q < cc.d; q += 32) {
          const int e = cc.b + q;
          if (g.cvn(cc, q) != nstar) am_update(rck, rcidx, rkey(s.P[e], s.C[e]), (uint32_t)e);
        }
      }
      uint32_t key;
      const uint32_t en = warp_argmax(rck, rcidx, key);
      enext = en == 0xffffffffu ? -1 : (int)en;
    }
    // -- LMD: next target = argmax D over U(m*, n*) (Alg. 3 line 11), or over
    //    N(m*)\n* when d_v(n*) = 1 (Sec. 5.A), else the global argmax.
    if (SCHED == kLMD) {
      if (dv == 1) {
        ck = 0;
        cidx = 0xffffffffu;
        const typename G::C cc = g.cn(mstar);
        for (int q = lane; q < cc.d; q += 32) {
          const int j = g.cvn(cc, q);
          if (j != nstar) am_update(ck, cidx, mkey(s.D[j]), (uint32_t)j);
        }
      }
      uint32_t key;
      const uint32_t nn = warp_argmax(ck, cidx, key);
      nstar = (nn == 0xffffffffu) ? global_argmax_D<A>(N, s, key) : (int)nn;
    }
  }

  // ---- outputs
  for (int n = lane; n < N; n += 32) {
    if (io.hard) io.hard[n] = (uint8_t)(s.L[n] < (L_)0);
    if (io.llr_out) io.llr_out[n] = (float)s.L[n];
  }
  for (int e = lane; e < E; e += 32) {
    if (io.c2v_out) io.c2v_out[e] = (float)s.C[e];
    if (io.pre_out) io.pre_out[e] = (float)s.P[e];
  }
  if (lane == 0) {
    if (io.updates) *io.updates = count;
    if (io.converged) *io.converged = unsat == 0 ? 1 : 0;
    if (io.fallbacks) *io.fallbacks = nfall;
  }
  __syncwarp();
}

// Shared-memory form: warp w of CTA c decodes frame c * frames_per_cta + w.
template <int A, int SCHED, class G>
__global__ void __launch_bounds__(512) se_decode_kernel(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);  // all threads, before any exit
  const int warp = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * a.frames_per_cta + warp;
  if (b >= a.batch) return;
  unsigned char* vbase = smem_raw + a.graph_smem + (size_t)warp * a.smem_per_frame;
  se_frame<A, SCHED, G, true>(a, a.g, g, batch_io(a, b, A == kINT6 ? 1 : 4), vbase,
                              vbase + se_layout(A, a.g.M, a.g.N, a.g.E, SCHED).vtotal);
}

// Global-memory form (frame state larger than shared memory): every warp owns
// one state slot of a.gstate and loops over the frames b = slot + k * slots.
// CTAs of at most 256 threads (8 frames), four per SM: the chain waits on L2,
// so more resident warps pay more than registers (64 instead of up to 122:
// 10-26 % faster on the WiFi-like code).
template <int A, int SCHED, class G>
__global__ void __launch_bounds__(256, 4) se_decode_kernel_gs(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  const int warp = threadIdx.x >> 5;
  const int64_t slot = (int64_t)blockIdx.x * a.frames_per_cta + warp;
  const int64_t slots = (int64_t)gridDim.x * a.frames_per_cta;
  unsigned char* base = (unsigned char*)a.gstate + slot * a.gstate_stride;
  unsigned char* ebase = base + se_layout(A, a.g.M, a.g.N, a.g.E, SCHED).vtotal;
  for (int64_t b = slot; b < a.batch; b += slots)
    se_frame<A, SCHED, G, false>(a, a.g, g, batch_io(a, b, A == kINT6 ? 1 : 4), base, ebase);
}

// Split form: the V region of a frame (VN- and check-sized arrays) in shared
// memory, its E region (the edge arrays) in a global-memory slot, small enough
// in total for L2 to hold.  Every warp owns one slot and loops over the frames
// b = slot + k * slots.
template <int A, int SCHED, class G>
__global__ void __launch_bounds__(512) se_decode_kernel_split(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  const int warp = threadIdx.x >> 5;
  const int64_t slot = (int64_t)blockIdx.x * a.frames_per_cta + warp;
  const int64_t slots = (int64_t)gridDim.x * a.frames_per_cta;
  unsigned char* vbase = smem_raw + a.graph_smem + (size_t)warp * a.smem_per_frame;
  unsigned char* ebase = (unsigned char*)a.gstate + slot * a.gstate_stride;
  for (int64_t b = slot; b < a.batch; b += slots)
    se_frame<A, SCHED, G, true>(a, a.g, g, batch_io(a, b, A == kINT6 ? 1 : 4), vbase, ebase);
}

// Queue form of the single-edge schedules: one warp per CTA takes work items
// until the queue is empty (see the multi-edge queue kernel).
template <int A, int SCHED>
__global__ void __launch_bounds__(32) se_queue_kernel(const QueueArgs q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ GraphDesc s_gd;
  const int lane = threadIdx.x & 31;
  unsigned char* sstate = smem_raw + q.graph_bytes;
  unsigned char* gslot = (unsigned char*)q.a.gstate + (int64_t)blockIdx.x * q.a.gstate_stride;
  int cur = -1;
  QCGraph g{};
  for (int64_t round = 0;; ++round) {
    long long idx = 0;
    if (lane == 0) idx = q.persistent ? (long long)atomicAdd(q.head, 1u) : (round == 0 ? (long long)blockIdx.x : q.n_items);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= q.n_items) break;
    const WorkItem it = q.items[idx];
    if (it.code < 0 || it.code >= q.n_codes) {  // not a code of this call: flag the item
      if (lane == 0) {
        if (q.a.updates) q.a.updates[idx] = 0;
        if (q.a.converged) q.a.converged[idx] = 2;
        atomicOr(q.a.status, 4u);
      }
      continue;
    }
    if (it.code != cur) {
      if (lane == 0) s_gd = q.codes[it.code];
      __syncwarp();
      g = GraphStage<QCGraph>::make(s_gd, (int32_t*)smem_raw);
      cur = it.code;
    }
    const int elem = A == kINT6 ? 1 : 4;
    FrameIO io = empty_io();
    io.llr = (const unsigned char*)q.a.llr + it.llr_offset * elem;
    io.hard = q.a.hard ? q.a.hard + it.out_offset : nullptr;
    io.llr_out = nullptr;
    io.updates = q.a.updates ? q.a.updates + idx : nullptr;
    io.converged = q.a.converged ? q.a.converged + idx : nullptr;
    io.trace = nullptr;
    io.max_updates = it.max_updates;
    io.frame = it.frame_index;
    const SELayout ly = se_layout(A, s_gd.M, s_gd.N, s_gd.E, SCHED);
    unsigned char* base = ly.total <= q.smem_state_bytes ? sstate : gslot;
    se_frame<A, SCHED, QCGraph, false>(q.a, s_gd, g, io, base, base + ly.vtotal);
  }
}

template <int A, int S>
cudaError_t launch_se_queue_t(const QueueArgs& q, int grid, size_t smem, cudaStream_t st) {
  auto k = se_queue_kernel<A, S>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<(unsigned)grid, 32, smem, st>>>(q);
  return cudaGetLastError();
}

template <int A, int S, class G>
cudaError_t launch_one(const DecodeArgs& a, cudaStream_t st) {
  if (a.se_split) {
    const size_t smem = (size_t)a.graph_smem + (size_t)a.smem_per_frame * a.frames_per_cta;
    auto k = se_decode_kernel_split<A, S, G>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k<<<(unsigned)a.gstate_ctas, 32 * a.frames_per_cta, smem, st>>>(a);
    return cudaGetLastError();
  }
  if (a.gstate) {
    const size_t smem = (size_t)a.graph_smem;
    auto k = se_decode_kernel_gs<A, S, G>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k<<<(unsigned)a.gstate_ctas, 32 * a.frames_per_cta, smem, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)a.graph_smem + (size_t)a.smem_per_frame * a.frames_per_cta;
  auto k = se_decode_kernel<A, S, G>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int64_t grid = (a.batch + a.frames_per_cta - 1) / a.frames_per_cta;
  k<<<(unsigned)grid, 32 * a.frames_per_cta, smem, st>>>(a);
  return cudaGetLastError();
}

template <int A, class G>
cudaError_t launch_sched(const DecodeArgs& a, int sched, cudaStream_t s) {
  if (sched == kRBP) return launch_one<A, kRBP, G>(a, s);
  if (sched == kCIRBP) return launch_one<A, kCIRBP, G>(a, s);
  if (sched == kLMDRBP) return launch_one<A, kLMDRBP, G>(a, s);
  if (sched == kSLMDRBP) return launch_one<A, kSLMDRBP, G>(a, s);
  return launch_one<A, kLMD, G>(a, s);
}

}  // namespace

namespace {
template <int A>
cudaError_t se_queue_occ(size_t smem, int* out) {
  auto k = se_queue_kernel<A, kLMD>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, 32, smem);
}
}  // namespace

cudaError_t se_queue_blocks_per_sm(int arith, size_t smem, int* out) {
  return arith == kFP32 ? se_queue_occ<kFP32>(smem, out) : se_queue_occ<kINT6>(smem, out);
}

cudaError_t launch_se_queue(const QueueArgs& q, int arith, int grid, size_t smem, cudaStream_t s) {
  if (q.n_items == 0) return cudaSuccess;
  return arith == kFP32 ? launch_se_queue_t<kFP32, kLMD>(q, grid, smem, s) : launch_se_queue_t<kINT6, kLMD>(q, grid, smem, s);
}

size_t se_smem_per_frame(int arith, int sched, const GraphDesc& g) {
  return (size_t)se_layout(arith, g.M, g.N, g.E, sched).total;
}

size_t se_vregion_bytes(int arith, int sched, const GraphDesc& g) {
  return (size_t)se_layout(arith, g.M, g.N, g.E, sched).vtotal;
}

cudaError_t launch_se(const DecodeArgs& a, int arith, int sched, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  if (arith == kFP32)
    return a.g.is_qc ? launch_sched<kFP32, QCGraph>(a, sched, s) : launch_sched<kFP32, TabGraph>(a, sched, s);
  return a.g.is_qc ? launch_sched<kINT6, QCGraph>(a, sched, s) : launch_sched<kINT6, TabGraph>(a, sched, s);
}

}  // namespace ldpc
