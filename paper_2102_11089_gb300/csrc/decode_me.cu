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
// Work layout of one step (CTA of 256 or 512 threads):
//  commit   a team of Wv lanes per selected p (Wv = power of two >= max VN
//           degree): lane q reads edge q of p; team argmax of the residual,
//           team sum of the new L_p.
//  checks   a team of W lanes per affected check (W = power of two >= max
//           check degree): lane r owns edge r; exclude-one combination of
//           eq. (2) (or min-sum) by width-W shuffles.
//  refresh  L~_j is kept as an exact integer sum: the 6-bit messages
//           themselves, or FP32 messages in fixed point (x 2^k with k chosen so
//           that d_v,max * llr_clip * 2^k < 2^30), updated by the checks
//           phase with atomic deltas; integer sums do not depend on the order
//           of the updates.  L~_j = lambda_j + that sum (x 2^-k).
//
// Algorithm 4 keeps the group index floor(D N_G) of every VN in shared memory
// and the group sizes up to date.  Its random fill takes the fill-group members
// with the smallest keys (word n mod 4 of Philox4x32-10 with counter (n/4,
// step, frame), key = seed; equal keys to the lower index): members with key
// <= T are gathered (T bisected until between `need` and kCap of them), then
// ranked exactly.
//
// Selection lists: the VNs of the next step (P' of Algorithm 6, Algorithm 4's
// top groups and fill winners) are appended to the other of two lists by slot
// atomics as they are chosen, in no particular order; every consumer is
// order-independent.  A VN's rank in index order (its trace position, and
// whether the budget keeps it in a truncated last step) is counted only when
// a trace is requested or the step is truncated.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "device_math.cuh"
#include "philox.cuh"

namespace ldpc {

namespace cg = cooperative_groups;

namespace {

constexpr int kCap = 512;  // candidate list of the random fill

// Array views of the frame state.  LArr: a plain array (this CTA's shared
// memory, or a global-memory slot).  DArr: an array spread over the shared
// memory of the CTAs of a thread-block cluster: element i lives in rank
// rank0 + (i >> shift) at the same offset in every rank, reached through
// distributed shared memory.
template <class T>
struct LArr {
  T* p;
  __device__ __forceinline__ T& operator[](int i) const { return p[i]; }
};
template <class T>
struct DArr {
  T* p;  // this CTA's address of the array's chunk
  int shift, rank0;
  __device__ __forceinline__ T& operator[](int i) const {
    return *cg::this_cluster().map_shared_rank(p + (i & ((1 << shift) - 1)), (unsigned)(rank0 + (i >> shift)));
  }
};

// Thread group decoding one frame: a CTA, or all CTAs of a cluster.  tid/nt
// number the group's threads; sync() is the group barrier (with the memory
// ordering of __syncthreads / barrier.cluster); sync_or() a barrier that ORs
// a flag over the group.
struct CtaX {
  template <class T>
  using Arr = LArr<T>;
  int tid, nt;
  __device__ __forceinline__ CtaX() : tid((int)threadIdx.x), nt((int)blockDim.x) {}
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ int sync_or(int v, int*) const { return __syncthreads_or(v); }
};
struct ClusterX {
  template <class T>
  using Arr = DArr<T>;
  int tid, nt;
  __device__ __forceinline__ ClusterX() {
    const cg::cluster_group c = cg::this_cluster();
    tid = (int)(c.block_rank() * blockDim.x + threadIdx.x);
    nt = (int)(c.num_blocks() * blockDim.x);
  }
  // release/acquire cluster barrier; the "memory" clobber also keeps the
  // compiler from moving shared-memory accesses across it.  Not the .aligned
  // form: the compiler does not know this asm needs a converged warp, and an
  // .aligned barrier reached by a diverged warp is undefined.
  __device__ __forceinline__ void sync() const {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
  }
  // `flag` (one int of the cluster, zero on entry) is reset by thread 0 after use
  __device__ __forceinline__ int sync_or(int v, int* flag) const {
    if (__syncthreads_or(v) && threadIdx.x == 0) atomicOr(flag, 1);
    sync();
    const int r = *(volatile int*)flag;
    sync();
    if (tid == 0) *flag = 0;
    return r;
  }
};

// Big per-frame arrays (shared memory, or a global-memory slot for large codes)
struct MEBig {
  int C, P, lam, L, D, Lt, grp, par, total;
};
// Per-CTA working set of one step (always shared memory).  The fill candidates
// of Algorithm 4 share storage with the affected-check list (not live then).
struct MESmall {
  int sel, est, best, cnl, cul, cbits, cnt, cntS, bits, touched, misc, total;
};

__host__ __device__ inline MEBig me_big(int arith, int M, int N, int E) {
  const int msg = arith == kINT6 ? 1 : 4;
  const int llr = arith == kINT6 ? 2 : 4;
  const int dv = arith == kINT6 ? 2 : 4;
  MEBig l;
  int o = 0;
  l.C = o; o = align16(o + E * msg);
  l.P = o; o = align16(o + E * msg);
  l.lam = o; o = align16(o + N * llr);
  l.L = o; o = align16(o + N * llr);
  l.D = o; o = align16(o + N * dv);
  l.Lt = o; o = align16(o + N * 4);
  l.grp = o; o = align16(o + N);
  l.par = o; o = align16(o + ((M + 31) / 32) * 4);
  l.total = o;
  return l;
}

__host__ __device__ inline MESmall me_small(int M, int N, int n_p, int dvm, int n_g) {
  MESmall l;
  int o = 0;
  const int ncnl = n_p * (dvm > 1 ? dvm - 1 : 1);
  l.sel = o; o = align16(o + 2 * n_p * 4);
  l.est = o; o = align16(o + n_p * 4);
  l.best = o; o = align16(o + n_p * 8);
  l.cnl = o; o = align16(o + (ncnl > kCap ? ncnl : kCap) * 8);
  l.cul = o; o = align16(o + ncnl * 4);
  l.cbits = o; o = align16(o + ((M + 31) / 32) * 4);
  l.cnt = o; o = align16(o + n_g * 4);
  l.cntS = o; o = align16(o + n_g * 4);
  l.bits = o; o = align16(o + ((N + 31) / 32) * 4);
  l.touched = o; o = align16(o + ((N + 31) / 32) * 4);
  l.misc = o; o = align16(o + 32 * 4);
  l.total = o;
  return l;
}

// shared scalars (misc area)
struct MEMisc {
  int unsat;
  int ncnu;   // affected (check, owner) pairs this step | distinct affected checks << 16: checks of degree <= 8
  int ncnu2;  // the same for checks of larger degree (kept from the back of the lists)
  int nsel[2];  // selected VNs of the two selection buffers (this step's, the next step's)
  int ncand;  // fill candidates gathered (reset at every step start)
  uint32_t thr, lo, hi;
  int hi_set;
  int orflag;  // cluster form: OR of the bad-input flags
};

template <int A, class X>
struct MEState {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  template <class T>
  using Arr = typename X::template Arr<T>;
  Arr<M_> C;
  Arr<M_> P;
  Arr<L_> lam;
  Arr<L_> L;
  Arr<D_> D;
  Arr<int32_t> Lt;   // sum over the edges of each VN of L~^C, exact integer (see top)
  Arr<uint8_t> grp;
  Arr<uint32_t> par;
  Arr<int32_t> sel;    // two selection lists of n_p slots: this step's and the next step's
  Arr<int32_t> est;
  Arr<unsigned long long> best;
  Arr<int2> cnl;       // (check, owner k) of every affected check
  Arr<unsigned long long> cand;  // aliases cnl
  Arr<int32_t> cul;    // distinct affected checks
  Arr<uint32_t> cbits;   // checks already listed this step
  Arr<int32_t> cnt;      // |G_i| over all VNs, kept up to date with grp
  Arr<int32_t> cntS;     // per-group count of the VNs excluded from Algorithm 4's search set
  Arr<uint32_t> bits;    // selection bitmap over VNs
  Arr<uint32_t> touched; // VNs whose D was rewritten in this step
  MEMisc* misc;
  const int16_t* tab;
  float fx, ifx;     // FP32 fixed point: 2^k and 2^-k
};

template <class X>
__device__ __forceinline__ float ci_me(const MEState<kFP32, X>&, float a, float b) { return ci_fp(a, b); }
template <class X>
__device__ __forceinline__ uint16_t ci_me(const MEState<kINT6, X>& s, int a, int b) { return ci_int(a, b, s.tab); }

// message -> exact integer term of the L~ sum, and the sum -> L~ contribution
template <class X>
__device__ __forceinline__ int fix_msg(const MEState<kFP32, X>& s, float x) { return __float2int_rn(x * s.fx); }
template <class X>
__device__ __forceinline__ int fix_msg(const MEState<kINT6, X>&, int8_t x) { return (int)x; }
template <class X>
__device__ __forceinline__ float lt_total(const MEState<kFP32, X>& s, int n) {
  return s.lam[n] + (float)s.Lt[n] * s.ifx;
}
template <class X>
__device__ __forceinline__ int16_t lt_total(const MEState<kINT6, X>& s, int n) { return (int16_t)(s.lam[n] + s.Lt[n]); }

// Algorithm 4 line 2: group i = floor(D N_G), clamped to N_G - 1
__device__ __forceinline__ int group_of(float d, int ng) { return min((int)floorf(d * (float)ng), ng - 1); }
__device__ __forceinline__ int group_of(uint16_t d, int ng) { return min((int)(((int)d * ng) / 65534), ng - 1); }

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// Algorithm 4 over S = O_N minus nexcl excluded VNs (their bits are set and
// s.cntS counts them per group): sets the bits of the selected VNs (at most
// np) and appends them, in no particular order, to the selection list at
// s.sel[sbase...] whose count is *nsel.  Group sizes come from the maintained
// s.cnt.  All threads call it.
template <int A, class X>
__device__ void alg4(const X& x, const MEState<A, X>& s, int N, int np, int ng, int nexcl, uint32_t step,
                     uint64_t frame, uint64_t seed, int sbase, int* nsel) {
  const int tid = x.tid, nt = x.nt, lane = tid & 31, warp = tid >> 5;
  MEMisc* ms = s.misc;
  // line 3: k* = max{k : |Q(k)| <= N_P} on the counts of S, by every warp from
  // the maintained counts (the same values everywhere, no barrier); warp 0
  // stores the state of the threshold search.  |G_i| over S = cnt[i] - cntS[i]
  // (cntS counts the excluded VNs per group); lane l of chunk b looks at group
  // ng - 1 - (b + l), i.e. k = b + l + 1
  const int sz = N - nexcl;
  int kstar = 0, q = 0;
  if (sz <= np) {
    kstar = ng;
    q = sz;
  } else {
    for (int b0 = 0; b0 < ng - 1; b0 += 32) {
      const int i = b0 + lane;
      const int c = i < ng - 1 ? s.cnt[ng - 1 - i] - s.cntS[ng - 1 - i] : np + 1;  // > np, no overflow
      int pre = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, pre, o);
        if (lane >= o) pre += y;
      }
      const unsigned ok = __ballot_sync(kFull, q + pre <= np);  // a prefix of the lanes
      const int nok = __popc(ok);
      kstar += nok;
      q += nok > 0 ? __shfl_sync(kFull, pre, nok - 1) : 0;
      if (nok < 32) break;
    }
  }
  const int need = kstar < ng ? np - q : 0;
  const int top = ng - kstar, fg = ng - kstar - 1;
  uint32_t thr0 = 0xffffffffu;
  if (need > 0) {
    // first threshold: need + 3 sqrt(need) + 8 expected members at or below
    // it, short of `need` with probability < 1e-3 (the selection does not
    // depend on it, so approximate arithmetic serves)
    const int members = s.cnt[fg] - s.cntS[fg];
    const float fn = (float)need;
    const float want = fn + 3.0f * fn * rsqrtf(fn) + 8.0f;
    if ((float)members > want) {
      const float t = __fdividef(want, (float)members) * 4294967296.0f;
      thr0 = t >= 4294967040.0f ? 0xffffffffu : (uint32_t)t;
    }
  }
  if (tid == 0) {  // read only after the pass's barrier
    ms->thr = thr0;
    ms->lo = 0;
    ms->hi = 0xffffffffu;
    ms->hi_set = 0;
  }
  const int nq = (N + 3) / 4;
  // one pass over VN quads: line 3 selects Q(k*); lines 4-6 gather fill candidates
  // (key = word i of the Philox block of quad q)
  bool fill = need > 0;
  for (int iter = 0; iter < 64; ++iter) {
    const uint32_t thr = iter == 0 ? thr0 : ms->thr;
    // two quads per lane (q0 + lane and q0 + 32 + lane): their Philox chains
    // are independent and interleave; warp-uniform trip count
    for (int q0 = warp * 64; q0 < nq; q0 += 2 * nt) {
      unsigned fm[2] = {0u, 0u}, gem[2] = {0u, 0u};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = q0 + 32 * u + lane;
        if (q < nq) {
          // the quad's four group bytes compared at once (per-byte SIMD compares,
          // then the byte masks packed to nibbles); VNs past N or already in
          // the bitmap are not live; Q(k*) members go in with one atomic
          const uint32_t g4 = *(const uint32_t*)&s.grp[4 * q];
          const int sh = (q & 7) * 4;
          const unsigned live = (N - 4 * q >= 4 ? 0xfu : ((1u << (N - 4 * q)) - 1u)) & ~((s.bits[q >> 3] >> sh) & 0xfu);
          const uint32_t ge = __vcmpgeu4(g4, (uint32_t)top * 0x01010101u);
          const uint32_t eq = __vcmpeq4(g4, (uint32_t)(fg & 0xff) * 0x01010101u);  // fg = -1: byte 255, no group
          gem[u] = ((((ge >> 7) & 0x01010101u) * 0x01020408u) >> 24) & live;
          fm[u] = ((((eq >> 7) & 0x01010101u) * 0x01020408u) >> 24) & live;
          if (iter == 0 && gem[u]) atomicOr(&s.bits[q >> 3], gem[u] << sh);
          if (iter != 0) gem[u] = 0u;
        }
      }
      if (__any_sync(kFull, (gem[0] | gem[1]) != 0u)) {  // Q(k*) members of the warp's quads: one slot atomic
        unsigned b[8];
        int tot = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          b[i] = __ballot_sync(kFull, (gem[i >> 2] >> (i & 3)) & 1u);
          tot += __popc(b[i]);
        }
        int base = 0;
        if (lane == 0) base = atomicAdd(nsel, tot);
        base = __shfl_sync(kFull, base, 0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if ((gem[i >> 2] >> (i & 3)) & 1u)
            s.sel[sbase + base + __popc(b[i] & lanemask_lt())] = 4 * (q0 + 32 * (i >> 2) + lane) + (i & 3);
          base += __popc(b[i]);
        }
      }
      if (!fill) continue;
      uint32_t w[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        w[u][0] = (uint32_t)(q0 + 32 * u + lane);
        w[u][1] = step;
        w[u][2] = (uint32_t)frame;
        w[u][3] = (uint32_t)(frame >> 32);
      }
      if (fm[0] | fm[1]) {
        philox4x32_10(w[0], seed);
        philox4x32_10(w[1], seed);
      }
      // fill candidates (key <= thr) of both quads: one slot atomic
      unsigned b[8];
      int tot = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        b[i] = __ballot_sync(kFull, ((fm[i >> 2] >> (i & 3)) & 1u) && w[i >> 2][i & 3] <= thr);
        tot += __popc(b[i]);
      }
      if (tot == 0) continue;
      int base = 0;
      if (lane == 0) base = atomicAdd(&ms->ncand, tot);
      base = __shfl_sync(kFull, base, 0);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int pos = base + __popc(b[i] & lanemask_lt());
        if (((b[i] >> lane) & 1u) && pos < kCap)
          s.cand[pos] = ((unsigned long long)w[i >> 2][i & 3] << 32) |
                        (unsigned)(4 * (q0 + 32 * (i >> 2) + lane) + (i & 3));
        base += __popc(b[i]);
      }
    }
    x.sync();
    if (!fill) break;
    const int nc = ms->ncand;
    if (nc >= need && nc <= kCap) {
      // exact rank among the candidates ((key, n) is unique): a thread per
      // candidate counts the keys below its own (the lanes of a warp read the
      // same key at a time: broadcast loads)
      for (int c = tid; c < nc; c += nt) {
        const unsigned long long kc = s.cand[c];
        int rank = 0;
        int c2 = 0;
        for (; c2 + 4 <= nc; c2 += 4)
          rank += (s.cand[c2] < kc) + (s.cand[c2 + 1] < kc) + (s.cand[c2 + 2] < kc) + (s.cand[c2 + 3] < kc);
        for (; c2 < nc; ++c2) rank += s.cand[c2] < kc;
        if (rank < need) {
          const int n = (int)(kc & 0xffffffffull);
          atomicOr(&s.bits[n >> 5], 1u << (n & 31));
          s.sel[sbase + atomicAdd(nsel, 1)] = n;
        }
      }
      x.sync();
      break;
    }
    x.sync();  // every thread has read ncand
    if (tid == 0) {
      if (nc < need) {  // bisect the threshold upwards
        ms->lo = thr;
        ms->thr = ms->hi_set ? thr + (ms->hi - thr + 1) / 2
                             : (thr > 0x7fffffffu ? 0xffffffffu : 2u * thr + 1u);
      } else {  // too many: downwards
        ms->hi = thr;
        ms->hi_set = 1;
        ms->thr = ms->lo + (thr - ms->lo) / 2;
      }
      ms->ncand = 0;
    }
    x.sync();
  }
}

// State views of a frame in one CTA: big arrays at `big` (shared memory or a
// global-memory slot), per-CTA working set at `small`.
template <int A>
__device__ __forceinline__ MEState<A, CtaX> cta_state(const GraphDesc& gd, const DecodeArgs& a, unsigned char* big,
                                                      unsigned char* small, const int16_t* tab_int) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  const MEBig lb = me_big(A, gd.M, gd.N, gd.E);
  const MESmall ls = me_small(gd.M, gd.N, a.n_p, gd.dv_max, a.n_g);
  MEState<A, CtaX> s;
  s.C.p = (M_*)(big + lb.C);
  s.P.p = (M_*)(big + lb.P);
  s.lam.p = (L_*)(big + lb.lam);
  s.L.p = (L_*)(big + lb.L);
  s.D.p = (D_*)(big + lb.D);
  s.Lt.p = (int32_t*)(big + lb.Lt);
  s.grp.p = (uint8_t*)(big + lb.grp);
  s.par.p = (uint32_t*)(big + lb.par);
  s.sel.p = (int32_t*)(small + ls.sel);
  s.est.p = (int32_t*)(small + ls.est);
  s.best.p = (unsigned long long*)(small + ls.best);
  s.cnl.p = (int2*)(small + ls.cnl);
  s.cul.p = (int32_t*)(small + ls.cul);
  s.cand.p = (unsigned long long*)(small + ls.cnl);
  s.cbits.p = (uint32_t*)(small + ls.cbits);
  s.cnt.p = (int32_t*)(small + ls.cnt);
  s.cntS.p = (int32_t*)(small + ls.cntS);
  s.bits.p = (uint32_t*)(small + ls.bits);
  s.touched.p = (uint32_t*)(small + ls.touched);
  s.misc = (MEMisc*)(small + ls.misc);
  s.tab = tab_int;
  return s;
}

// Decode one frame of code `gd` with thread group `x` on state `s`.  kPair: a
// check team takes two checks (and two LMD pairs) per loop iteration where its
// warp has them, so that their dependency chains interleave; taken for frames
// in shared memory only (with global-memory state the pairing measured 6-22 %
// slower on 26k-bit codes).
template <int A, int SCHED, class G, class X, bool kPair = false>
__device__ __forceinline__ void me_frame(const X& x, const DecodeArgs& a, const GraphDesc& gd, const G& g,
                                         const FrameIO& io, MEState<A, X>& s) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  const int tid = x.tid, nt = x.nt, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int N = gd.N, E = gd.E, M = gd.M;
  const int np = a.n_p, ng = a.n_g;
  {
    // fixed point of the FP32 L~ sums: d_v,max * llr_clip * 2^k < 2^30
    const int k = min(24, 29 - ilogbf((float)gd.dv_max * a.llr_clip));
    s.fx = __int_as_float((127 + k) << 23);
    s.ifx = __int_as_float((127 - k) << 23);
  }
  MEMisc* ms = s.misc;
  const float clip = a.llr_clip;
  const uint64_t frame = io.frame;
  const int W = team_width(gd.dc_max), tpw = 32 / W, team = lane / W, r = lane % W;
  const int Wv = team_width(gd.dv_max), tpv = 32 / Wv, vteam = lane / Wv, q = lane % Wv;
  const int Mw = (M + 31) / 32, Nw = (N + 31) / 32;
  // Affected checks and (check, owner) pairs are kept in two degree classes:
  // degree <= Ws from the front of their lists, handled by teams of Ws lanes,
  // larger degrees from the back (capL - 1 downwards), by teams of W lanes.
  // Codes whose checks all have degree <= 8 have one class, and so does the
  // shared-memory form (kPair), whose registers the second class would spill.
  constexpr bool kSplit = !kPair;
  const int Ws = kSplit && W > 8 ? 8 : W;
  const bool split = kSplit && W > Ws;
  const int capL = np * (gd.dv_max > 1 ? gd.dv_max - 1 : 1);  // pairs of one step, at most

  int bad = 0;
  for (int n = tid; n < N; n += nt) {
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
  for (int e = tid; e < E; e += nt) s.C[e] = (M_)0;
  for (int w = tid; w < Nw; w += nt) s.bits[w] = 0u;
  for (int w = tid; w < Mw; w += nt) {
    s.par[w] = 0u;
    s.cbits[w] = 0u;
  }
  for (int i = tid; i < ng; i += nt) {
    s.cnt[i] = 0;
    s.cntS[i] = 0;
  }
  if (tid == 0) {
    ms->unsat = 0;
    ms->ncnu = 0;
    ms->ncnu2 = 0;
    ms->nsel[0] = 0;
    ms->nsel[1] = 0;
    ms->ncand = 0;
  }
  if (x.sync_or(bad, &ms->orflag)) {
    for (int n = tid; n < N; n += nt) {
      if (io.hard) io.hard[n] = 0;
      if (io.llr_out) io.llr_out[n] = (float)s.lam[n];
    }
    if (tid == 0) {
      if (io.updates) *io.updates = 0;
      if (io.converged) *io.converged = 2;
      atomicOr(a.status, 1u);
    }
    return;
  }
  // ---- Alg. 5/6 lines 1-3: every L~^C, R, L~, D; syndrome of bsgn(lambda)
  for (int t0 = warp * tpw; t0 < M; t0 += nw * tpw) {
    const int m = t0 + team;
    int e, j;
    M_ out;
    const int dc = team_c2v<A, G>(g, s.C, s.L, m < M ? m : -1, r, W, clip, e, j, out);
    if (r < dc) s.P[e] = out;
    const unsigned neg = __ballot_sync(kFull, r < dc && s.L[j] < (L_)0);
    const unsigned tmask = (W == 32 ? kFull : ((1u << W) - 1u)) << (team * W);
    if (r == 0 && m < M && (__popc(neg & tmask) & 1)) {
      atomicOr(&s.par[m >> 5], 1u << (m & 31));
      atomicAdd(&ms->unsat, 1);
    }
  }
  x.sync();
  for (int n0 = warp * 32; n0 < N; n0 += nt) {  // warp-uniform trip count
    const int n = n0 + lane;
    const bool act = n < N;
    int gi = 0;
    if (act) {
      const typename G::V v = g.vn(n);
      int acc = 0;
      for (int k = 0; k < v.d; ++k) {
        int e, m;
        g.vedge(v, k, e, m);
        acc += fix_msg(s, s.P[e]);
      }
      s.Lt[n] = acc;
      const D_ d = ci_me(s, s.L[n], lt_total(s, n));
      gi = group_of(d, ng);
      s.D[n] = d;
      s.grp[n] = (uint8_t)gi;
    }
    if (act) atomicAdd(&s.cnt[gi], 1);
  }
  x.sync();

  int64_t count = 0, left = a.check_interval;
  uint32_t step = 0;
  int cur = 0;  // selection buffer of this step (s.sel[cur * np ...], ms->nsel[cur])
  bool stop = a.check_interval > 0 && ms->unsat == 0;
  if (!stop && io.max_updates > 0)  // Alg. 5 line 4 / Alg. 6 line 4
    alg4<A, X>(x, s, N, np, ng, 0, step, frame, a.seed, 0, &ms->nsel[0]);
  // L~_j, D_j of VN j (j < 0: idle lane) unless already rewritten in this
  // step; group and group sizes follow.  All lanes of the warp call it.
  // With `want` the new D_j is also returned when another lane rewrites it (its
  // inputs are final in this phase, so every lane computes the same value).
  auto refresh_vn = [&](int j, bool want) -> D_ {
    bool ch = false;
    int go = 0, gn = 0;
    D_ d = (D_)0;
    if (j >= 0) {
      const uint32_t bit = 1u << (j & 31);
      const bool first = !(atomicOr(&s.touched[j >> 5], bit) & bit);
      if (first || want) d = ci_me(s, s.L[j], lt_total(s, j));
      if (first) {
        s.D[j] = d;
        gn = group_of(d, ng);
        go = s.grp[j];
        if (gn != go) {
          s.grp[j] = (uint8_t)gn;
          ch = true;
        }
      }
    }
    if (ch) {  // per-lane atomics: aggregating equal groups first (match) costs more
      atomicAdd(&s.cnt[go], -1);
      atomicAdd(&s.cnt[gn], 1);
    }
    return d;
  };
  while (!stop && count < io.max_updates) {
    // The selection list is in no particular order.  A VN's rank in ascending
    // index order gives its trace position and, when the budget cuts the last
    // step, whether it is kept (the lowest indices are); it is computed only then.
    const int nsel = ms->nsel[cur];
    if (nsel <= 0) break;  // nothing selectable: the step would not advance
    const int64_t room = io.max_updates - count;
    const bool trunc = (int64_t)nsel > room;
    const bool ranked = trunc || io.trace != nullptr;
    const int done = trunc ? (int)room : nsel;
    const int so = cur * np, sn = (cur ^ 1) * np;
    if (tid == 0) {
      ms->nsel[cur ^ 1] = 0;  // read for the last time two steps ago
      ms->ncand = 0;          // read for the last time before the previous step's last barrier
    }
    // -- for each selected p (a team of Wv lanes, lane q on edge q of p):
    //    m*_p = argmax_i R_{i->p} on the pre-step state (the edges of p are
    //    disjoint from every other p's), commit L^C <- L~^C, L_p, syndrome,
    //    trace, and list the checks i in M(p)\m*_p whose inputs changed
    for (int w = tid; w < Nw; w += nt) {
      s.bits[w] = 0u;
      s.touched[w] = 0u;
    }
    for (int k0 = warp * tpv; k0 < nsel; k0 += nw * tpv) {  // warp-uniform trip count
      const int k = k0 + vteam;
      bool act = k < nsel;
      const int p = act ? s.sel[so + k] : 0;
      int rank = k;
      if (ranked) {  // team count of the selected VNs below p
        int c = 0;
        if (act)
          for (int i = q; i < nsel; i += Wv) c += s.sel[so + i] < p;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          if (o < Wv) c += __shfl_xor_sync(kFull, c, o);
        rank = c;
        act = act && rank < done;
      }
      int dv = 0, e = 0, m = 0;
      uint32_t bk = 0, bi = 0xffffffffu;
      M_ pk = (M_)0, ck = (M_)0;
      if (act) {
        const typename G::V v = g.vn(p);
        dv = v.d;
        if (q < dv) {
          g.vedge(v, q, e, m);
          pk = s.P[e];
          ck = s.C[e];
          bk = rkey(pk, ck);
          bi = (uint32_t)e;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {  // team argmax, ties to the lower edge id
        if (o >= Wv) continue;
        const uint32_t ok = __shfl_xor_sync(kFull, bk, o), oi = __shfl_xor_sync(kFull, bi, o);
        if (ok > bk || (ok == bk && oi < bi)) {
          bk = ok;
          bi = oi;
        }
      }
      const bool mine = act && q < dv;
      const bool isbest = mine && (uint32_t)e == bi;
      if (isbest) s.C[e] = pk;
      // L_p = lambda_p + sum of the committed C2V of p (butterfly sum: the same
      // value in every lane of the team)
      L_ lnew;
      if (A == kFP32) {
        float x = mine ? (float)(isbest ? pk : ck) : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          if (o < Wv) x += __shfl_xor_sync(kFull, x, o);
        lnew = act ? (L_)((float)s.lam[p] + x) : (L_)0;
      } else {
        int x = mine ? (int)(isbest ? pk : ck) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          if (o < Wv) x += __shfl_xor_sync(kFull, x, o);
        lnew = act ? (L_)((int)s.lam[p] + x) : (L_)0;
      }
      int flip = 0;
      if (act && q == 0) {
        const L_ lold = s.L[p];
        flip = (lold < (L_)0) != (lnew < (L_)0);
        s.L[p] = lnew;
        s.est[k] = (int)bi;
        if (io.trace) io.trace[count + rank] = (int)bi;
      }
      flip = __shfl_sync(kFull, flip, vteam * Wv);
      int du = 0;
      if (flip && mine) {  // tentative decision of p flipped: parity of every check of p
        const uint32_t bit = 1u << (m & 31);
        const uint32_t old = atomicXor(&s.par[m >> 5], bit);
        du = (old & bit) ? -1 : 1;
      }
      du = __reduce_add_sync(kFull, du);
      if (lane == 0 && du != 0) atomicAdd(&ms->unsat, du);
      const bool aff = mine && !isbest;
      bool first = false;
      if (aff) {
        const uint32_t bit = 1u << (m & 31);
        first = !(atomicOr(&s.cbits[m >> 5], bit) & bit);
      }
      // list slots of the warp's pairs and new checks from one atomic per
      // degree class on its packed counts (pairs in the low half, checks in
      // the high half)
      const bool big = split && aff && g.cn(m).d > Ws;
      const unsigned bs = __ballot_sync(kFull, aff && !big), bb = kSplit ? __ballot_sync(kFull, big) : 0u;
      const unsigned fs = __ballot_sync(kFull, first && !big), fb = kSplit ? __ballot_sync(kFull, first && big) : 0u;
      int bases = 0, bases2 = 0;
      if (lane == 0 && (bs | fs) != 0u) bases = atomicAdd(&ms->ncnu, __popc(bs) | (__popc(fs) << 16));
      if (kSplit && lane == 0 && (bb | fb) != 0u) bases2 = atomicAdd(&ms->ncnu2, __popc(bb) | (__popc(fb) << 16));
      bases = __shfl_sync(kFull, bases, 0);
      if (kSplit) bases2 = __shfl_sync(kFull, bases2, 0);
      const unsigned lt = lanemask_lt();
      if (aff)
        s.cnl[big ? capL - 1 - ((bases2 & 0xffff) + __popc(bb & lt)) : (bases & 0xffff) + __popc(bs & lt)] =
            make_int2(m, k);
      if (first) s.cul[big ? capL - 1 - ((bases2 >> 16) + __popc(fb & lt)) : (bases >> 16) + __popc(fs & lt)] = m;
      if (act && q == 0) {  // p's pairs are one block of each list: (first, count) of both, 16 bits each
        const unsigned tm = (Wv == 32 ? kFull : ((1u << Wv) - 1u)) << (vteam * Wv);
        const unsigned below = (1u << (vteam * Wv)) - 1u;
        const unsigned long long f0 = (unsigned)((bases & 0xffff) + __popc(bs & below)), n0 = __popc(bs & tm);
        const unsigned long long f1 = (unsigned)((bases2 & 0xffff) + __popc(bb & below)), n1 = __popc(bb & tm);
        s.best[k] = f0 | (n0 << 16) | (f1 << 32) | (n1 << 48);
      }
    }
    x.sync();
    const int ncn = ms->ncnu & 0xffff, ncu = ms->ncnu >> 16;
    const int ncn2 = ms->ncnu2 & 0xffff, ncu2 = ms->ncnu2 >> 16;
    // per-group counts of P': every warp summed them after the previous P'
    // barrier, and a warp that skipped the top-up met no barrier since; all
    // have passed the commit barrier now
    for (int i = tid; i < ng; i += nt) s.cntS[i] = 0;
    // -- precomputed C2V of every affected check (once per check); the L~ sums
    //    of its variables follow by exact deltas.  One list of a degree class:
    //    cnt checks, teams of Wc lanes (two checks per team and iteration
    //    with kPair)
    auto check_list = [&](int Wc, int cnt, bool back) {
      const int tpc = 32 / Wc, tc = lane / Wc, rc = lane % Wc;
      auto chk = [&](int t) { return t < cnt ? s.cul[back ? capL - 1 - t : t] : -1; };
      auto put = [&](int dc, int e, int j, M_ out) {
        if (rc < dc) {
          const int delta = fix_msg(s, out) - fix_msg(s, s.P[e]);
          s.P[e] = out;
          if (delta != 0) atomicAdd(&s.Lt[j], delta);
        }
      };
      if constexpr (kPair) {
        for (int t0 = warp * tpc; t0 < cnt; t0 += 2 * nw * tpc) {
          const int ta = t0 + tc, tb = ta + nw * tpc;
          int ea, ja, eb, jb;
          M_ oa, ob;
          if (__any_sync(kFull, tb < cnt)) {
            const int dca = team_c2v<A, G>(g, s.C, s.L, chk(ta), rc, Wc, clip, ea, ja, oa);
            const int dcb = team_c2v<A, G>(g, s.C, s.L, chk(tb), rc, Wc, clip, eb, jb, ob);
            put(dca, ea, ja, oa);
            put(dcb, eb, jb, ob);
          } else {
            const int dca = team_c2v<A, G>(g, s.C, s.L, chk(ta), rc, Wc, clip, ea, ja, oa);
            put(dca, ea, ja, oa);
          }
        }
      } else {
        for (int t0 = warp * tpc; t0 < cnt; t0 += nw * tpc) {
          int e, j;
          M_ out;
          const int dc = team_c2v<A, G>(g, s.C, s.L, chk(t0 + tc), rc, Wc, clip, e, j, out);
          put(dc, e, j, out);
        }
      }
    };
    check_list(Ws, ncu, false);
    if (kSplit && ncu2 > 0) check_list(W, ncu2, true);
    x.sync();
    // -- L~_j, D_j next to the affected checks and of every p.  ME-LMD-CIRBP runs
    //    this over the (check i, owner p) pairs and also forms Alg. 6 lines 6-10's
    //    candidate of each pair: the best j in N(i)\p by (D_j, lower index),
    //    written over the pair
    for (int w = tid; w < Mw; w += nt) s.cbits[w] = 0u;
    if (SCHED == kMELMD) {
      auto pair_key = [&](int j, int k, D_ d) -> unsigned long long {
        return (j >= 0 && j != s.sel[so + k]) ? (((unsigned long long)mkey(d) << 32) | (0xffffffffu - (uint32_t)j))
                                              : 0ull;
      };
      // one pair list of a degree class: cnt pairs, teams of Wc lanes
      auto pair_list = [&](int Wc, int cnt, bool back) {
        const int tpc = 32 / Wc, tc = lane / Wc, rc = lane % Wc;
        auto slot = [&](int t) { return back ? capL - 1 - t : t; };
        // VN of lane rc in pair t (-1: none) and the pair's owner k
        auto pair_vn = [&](int t, int& k) -> int {
          int j = -1;
          k = 0;
          if (t < cnt) {
            const int2 ck = s.cnl[slot(t)];
            k = ck.y;
            const typename G::C cc = g.cn(ck.x);
            if (rc < cc.d) j = g.cvn(cc, rc);
          }
          return j;
        };
        if constexpr (kPair) {  // two pairs per team and iteration (as above)
          for (int t0 = warp * tpc; t0 < cnt; t0 += 2 * nw * tpc) {
            const int ta = t0 + tc, tb = ta + nw * tpc;
            const bool two = __any_sync(kFull, tb < cnt);
            int ka, kb = 0;
            const int ja = pair_vn(ta, ka);
            const int jb = two ? pair_vn(tb, kb) : -1;
            const D_ da = refresh_vn(ja, true);
            const D_ db = two ? refresh_vn(jb, true) : (D_)0;
            unsigned long long keya = pair_key(ja, ka, da), keyb = pair_key(jb, kb, db);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {  // both team maxima at once (interleaved shuffles)
              if (o >= Wc) continue;
              const unsigned long long oa = __shfl_xor_sync(kFull, keya, o);
              const unsigned long long ob = __shfl_xor_sync(kFull, keyb, o);
              keya = oa > keya ? oa : keya;
              keyb = ob > keyb ? ob : keyb;
            }
            if (rc == 0 && ta < cnt) s.cand[slot(ta)] = keya;
            if (rc == 0 && two && tb < cnt) s.cand[slot(tb)] = keyb;
          }
        } else {
          for (int t0 = warp * tpc; t0 < cnt; t0 += nw * tpc) {
            const int t = t0 + tc;
            int k;
            const int j = pair_vn(t, k);
            unsigned long long key = pair_key(j, k, refresh_vn(j, true));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {  // team maximum
              if (o >= Wc) continue;
              const unsigned long long ok = __shfl_xor_sync(kFull, key, o);
              key = ok > key ? ok : key;
            }
            if (rc == 0 && t < cnt) s.cand[slot(t)] = key;
          }
        }
      };
      pair_list(Ws, ncn, false);
      if (kSplit && ncn2 > 0) pair_list(W, ncn2, true);
    } else {
      auto vn_list = [&](int Wc, int cnt, bool back) {
        const int tpc = 32 / Wc, tc = lane / Wc, rc = lane % Wc;
        for (int t0 = warp * tpc; t0 < cnt; t0 += nw * tpc) {
          const int t = t0 + tc;
          int j = -1;
          if (t < cnt) {
            const typename G::C cc = g.cn(s.cul[back ? capL - 1 - t : t]);
            if (rc < cc.d) j = g.cvn(cc, rc);
          }
          refresh_vn(j, false);
        }
      };
      vn_list(Ws, ncu, false);
      if (kSplit && ncu2 > 0) vn_list(W, ncu2, true);
    }
    // the selected VNs go to the last warps, which have the fewest pair teams
    for (int k0 = (nw - 1 - warp) * 32; k0 < nsel; k0 += nt) {
      const int k = k0 + lane;
      refresh_vn(k < nsel ? s.sel[so + k] : -1, false);
    }
    x.sync();
    // the pair and check counts were read after the commit barrier; the next
    // commit phase, which counts again, starts after at least one more barrier
    if (tid == 0) {
      ms->ncnu = 0;
      ms->ncnu2 = 0;
    }
    count += done;
    ++step;
    if (check_due(left, a.check_interval, done) && ms->unsat == 0) break;
    if (count >= io.max_updates) break;
    if constexpr (SCHED == kMECIRBP) {  // the selection bitmap is still clear from this step's start
      alg4<A, X>(x, s, N, np, ng, 0, step, frame, a.seed, sn, &ms->nsel[cur ^ 1]);  // Alg. 5 line 4
    } else {
      // -- P' = {argmax_{j in U(m*_p, p)} D_j} (degree-1 rule of Sec. 5.A:
      //    N(m*_p)\p), de-duplicated in the selection bitmap
      for (int k0 = warp * 32; k0 < nsel; k0 += nt) {  // warp-uniform trip count
        const int k = k0 + lane;
        bool add = false;
        int j = 0;
        if (k < nsel) {
          const int p = s.sel[so + k];
          const unsigned long long rg = s.best[k];  // p's pairs in both degree classes
          const int f0 = (int)(rg & 0xffff), n0 = (int)((rg >> 16) & 0xffff);
          const int f1 = (int)((rg >> 32) & 0xffff), n1 = (int)(rg >> 48);
          unsigned long long bk = 0ull;
          for (int i = f0; i < f0 + n0; ++i) {
            const unsigned long long v = s.cand[i];
            bk = v > bk ? v : bk;
          }
          for (int i = f1; kSplit && i < f1 + n1; ++i) {
            const unsigned long long v = s.cand[capL - 1 - i];
            bk = v > bk ? v : bk;
          }
          if (g.vn(p).d == 1) {
            const typename G::C cc = g.cn(g.ecn(s.est[k]));
            bk = 0ull;
            for (int qq = 0; qq < cc.d; ++qq) {
              const int jj = g.cvn(cc, qq);
              if (jj == p) continue;
              const unsigned long long key = ((unsigned long long)mkey(s.D[jj]) << 32) | (0xffffffffu - (uint32_t)jj);
              bk = key > bk ? key : bk;
            }
          }
          if (bk != 0ull) {  // else an empty candidate set
            j = (int)(0xffffffffu - (uint32_t)(bk & 0xffffffffull));
            const uint32_t bit = 1u << (j & 31);
            add = !(atomicOr(&s.bits[j >> 5], bit) & bit);
          }
        }
        if (add) atomicAdd(&s.cntS[s.grp[j]], 1);  // per-group count of P' for Algorithm 4's top-up
        const unsigned bal = __ballot_sync(kFull, add);  // P' joins the next selection list
        int base = 0;
        if (lane == 0 && bal != 0u) base = atomicAdd(&ms->nsel[cur ^ 1], __popc(bal));
        base = __shfl_sync(kFull, base, 0);
        if (add) s.sel[sn + base + __popc(bal & lanemask_lt())] = j;
      }
      x.sync();
      // |P'| = the sum of its per-group counts (every warp, same value)
      int npp = 0;
      for (int i = lane; i < ng; i += 32) npp += s.cntS[i];
      npp = __reduce_add_sync(kFull, npp);
      if (npp < np)  // lines 11-13
        alg4<A, X>(x, s, N, np - npp, ng, npp, step, frame, a.seed, sn, &ms->nsel[cur ^ 1]);
    }
    cur ^= 1;
  }

  for (int n = tid; n < N; n += nt) {
    if (io.hard) io.hard[n] = (uint8_t)(s.L[n] < (L_)0);
    if (io.llr_out) io.llr_out[n] = (float)s.L[n];
  }
  for (int e = tid; e < E; e += nt) {
    if (io.c2v_out) io.c2v_out[e] = (float)s.C[e];
    if (io.pre_out) io.pre_out[e] = (float)s.P[e];
  }
  if (tid == 0) {
    if (io.updates) *io.updates = count;
    if (io.converged) *io.converged = ms->unsat == 0 ? 1 : 0;
    if (io.fallbacks) *io.fallbacks = 0;
  }
  x.sync();
}

// Registers: FP32 frames are limited to two CTAs per SM by shared memory, so two
// resident CTAs are requested (up to 128 registers at 256 threads, 64 at 512);
// 6-bit frames fit more CTAs: four of 256 threads or two of 512 (64 registers).
template <int A, int TPB>
struct MEBounds {
  static constexpr int kMinBlocks = A == kFP32 ? 2 : (TPB == 256 ? 4 : 2);
};

// Shared-memory form: CTA b decodes frame b.
template <int A, int SCHED, class G, int TPB>
__global__ void __launch_bounds__(TPB, MEBounds<A, TPB>::kMinBlocks) me_decode_kernel(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int16_t tab_int[256];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  if (A == kINT6)
    for (int i = threadIdx.x; i < 256; i += blockDim.x) tab_int[i] = a.ci_table[i];
  unsigned char* big = smem_raw + a.graph_smem;
  const CtaX x;
  MEState<A, CtaX> s = cta_state<A>(a.g, a, big, big + a.smem_per_frame, tab_int);
  me_frame<A, SCHED, G, CtaX, true>(x, a, a.g, g, batch_io(a, blockIdx.x, A == kINT6 ? 1 : 4), s);
}

// Global-memory form: CTA c owns state slot c of a.gstate and decodes frames
// c, c + gridDim.x, ...
template <int A, int SCHED, class G, int TPB>
__global__ void __launch_bounds__(TPB, MEBounds<A, TPB>::kMinBlocks) me_decode_kernel_gs(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int16_t tab_int[256];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  if (A == kINT6)
    for (int i = threadIdx.x; i < 256; i += blockDim.x) tab_int[i] = a.ci_table[i];
  unsigned char* big = (unsigned char*)a.gstate + (int64_t)blockIdx.x * a.gstate_stride;
  const CtaX x;
  MEState<A, CtaX> s = cta_state<A>(a.g, a, big, smem_raw + a.graph_smem, tab_int);
  for (int64_t b = blockIdx.x; b < a.batch; b += gridDim.x)
    me_frame<A, SCHED, G, CtaX>(x, a, a.g, g, batch_io(a, b, A == kINT6 ? 1 : 4), s);
}

// Queue form: CTAs take work items (frames of any of up to 16 lifted codes, each
// with its own budget) until the queue is empty; a code's protograph view is
// staged when it changes; frame state sits in shared memory when it fits the
// CTA's reservation, else in the CTA's global slot.
template <int A, int SCHED, int TPB>
__global__ void __launch_bounds__(TPB, MEBounds<A, TPB>::kMinBlocks) me_queue_kernel(const QueueArgs q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int16_t tab_int[256];
  __shared__ GraphDesc s_gd;
  __shared__ long long s_item;
  const int tid = threadIdx.x;
  if (A == kINT6)
    for (int i = tid; i < 256; i += blockDim.x) tab_int[i] = q.a.ci_table[i];
  unsigned char* small = smem_raw + q.graph_bytes;
  unsigned char* sstate = small + q.small_bytes;
  unsigned char* gslot = (unsigned char*)q.a.gstate + (int64_t)blockIdx.x * q.a.gstate_stride;
  int cur = -1;
  QCGraph g{};
  for (int64_t round = 0;; ++round) {
    __syncthreads();  // every thread has read the previous item index
    if (tid == 0) s_item = q.persistent ? (long long)atomicAdd(q.head, 1u) : (round == 0 ? (long long)blockIdx.x : q.n_items);
    __syncthreads();
    const int64_t idx = s_item;
    if (idx >= q.n_items) break;
    const WorkItem it = q.items[idx];
    if (it.code < 0 || it.code >= q.n_codes) {  // not a code of this call: flag the item
      if (tid == 0) {
        if (q.a.updates) q.a.updates[idx] = 0;
        if (q.a.converged) q.a.converged[idx] = 2;
        atomicOr(q.a.status, 4u);
      }
      continue;
    }
    if (it.code != cur) {
      if (tid == 0) s_gd = q.codes[it.code];
      __syncthreads();
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
    const int big = me_big(A, s_gd.M, s_gd.N, s_gd.E).total;
    const CtaX x;
    MEState<A, CtaX> s = cta_state<A>(s_gd, q.a, big <= q.smem_state_bytes ? sstate : gslot, small, tab_int);
    me_frame<A, SCHED, QCGraph, CtaX>(x, q.a, s_gd, g, io, s);
  }
}

// State views of a frame spread over the CTAs of a cluster (plan a.cl); the
// state area starts at `base` in every CTA's shared memory.
template <int A>
__device__ __forceinline__ MEState<A, ClusterX> cluster_state(const DecodeArgs& a, unsigned char* base,
                                                              const int16_t* tab_int) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  const ClusterPlan& c = a.cl;
  MEState<A, ClusterX> s;
#define LDPC_DARR(field, T, k) s.field = DArr<T>{(T*)(base + c.off[k]), (int)c.shift[k], (int)c.rank0[k]}
  LDPC_DARR(C, M_, 0);
  LDPC_DARR(P, M_, 1);
  LDPC_DARR(lam, L_, 2);
  LDPC_DARR(L, L_, 3);
  LDPC_DARR(D, D_, 4);
  LDPC_DARR(Lt, int32_t, 5);
  LDPC_DARR(grp, uint8_t, 6);
  LDPC_DARR(par, uint32_t, 7);
  LDPC_DARR(sel, int32_t, 8);
  LDPC_DARR(est, int32_t, 9);
  LDPC_DARR(best, unsigned long long, 10);
  LDPC_DARR(cnl, int2, 11);
  LDPC_DARR(cand, unsigned long long, 11);
  LDPC_DARR(cul, int32_t, 12);
  LDPC_DARR(cbits, uint32_t, 13);
  LDPC_DARR(cnt, int32_t, 14);
  LDPC_DARR(cntS, int32_t, 15);
  LDPC_DARR(bits, uint32_t, 16);
  LDPC_DARR(touched, uint32_t, 17);
#undef LDPC_DARR
  s.misc = cg::this_cluster().map_shared_rank((MEMisc*)(base + c.off[18]), (unsigned)c.rank0[18]);
  s.tab = tab_int;
  return s;
}

// Cluster form: the CTAs of cluster c decode frames c, c + clusters, ... with
// the frame state spread over their shared memory (one CTA per SM).
template <int A, int SCHED, class G, int TPB>
__global__ void __launch_bounds__(TPB, 1) me_cluster_kernel(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int16_t tab_int[256];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  if (A == kINT6)
    for (int i = threadIdx.x; i < 256; i += blockDim.x) tab_int[i] = a.ci_table[i];
  const cg::cluster_group cl = cg::this_cluster();
  unsigned char* base = smem_raw + a.graph_smem;
  if (cl.block_rank() == (unsigned)a.cl.rank0[18] && threadIdx.x == 0)
    ((MEMisc*)(base + a.cl.off[18]))->orflag = 0;
  const ClusterX x;
  x.sync();  // every CTA of the cluster runs before any distributed address is formed
  MEState<A, ClusterX> s = cluster_state<A>(a, base, tab_int);
  const int64_t ncl = gridDim.x / a.cl.cs;
  for (int64_t b = blockIdx.x / a.cl.cs; b < a.batch; b += ncl)
    me_frame<A, SCHED, G, ClusterX>(x, a, a.g, g, batch_io(a, b, A == kINT6 ? 1 : 4), s);
  x.sync();  // no CTA leaves while another may still read its shared memory
}

template <int A, int S, class G, int TPB>
cudaError_t launch_me_cluster_t(const DecodeArgs& a, cudaStream_t st) {
  auto k = me_cluster_kernel<A, S, G, TPB>;
  const size_t smem = (size_t)a.graph_smem + (size_t)a.cl.bytes;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (a.cl.cs > 8) {
    err = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.cl.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(TPB, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)a.cl.cs, 1, 1);
  int clusters = 0;
  err = cudaOccupancyMaxActiveClusters(&clusters, (void*)k, &cfg);
  if (err != cudaSuccess) return err;
  if (clusters < 1) return cudaErrorInvalidConfiguration;
  const int64_t n = std::min<int64_t>(a.batch, clusters);
  cfg.gridDim = dim3((unsigned)(n * a.cl.cs), 1, 1);
  return cudaLaunchKernelEx(&cfg, k, a);
}

template <int A, int S, int TPB>
cudaError_t launch_me_queue_tpb(const QueueArgs& q, int grid, size_t smem, cudaStream_t st) {
  auto k = me_queue_kernel<A, S, TPB>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<(unsigned)grid, TPB, smem, st>>>(q);
  return cudaGetLastError();
}

template <int A, int S, class G, int TPB>
cudaError_t launch_me_tpb(const DecodeArgs& a, cudaStream_t st) {
  const MESmall ls = me_small(a.g.M, a.g.N, a.n_p, a.g.dv_max, a.n_g);
  if (a.gstate) {
    const size_t smem = (size_t)a.graph_smem + (size_t)ls.total;
    auto k = me_decode_kernel_gs<A, S, G, TPB>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k<<<(unsigned)a.gstate_ctas, TPB, smem, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)a.graph_smem + (size_t)a.smem_per_frame + (size_t)ls.total;
  auto k = me_decode_kernel<A, S, G, TPB>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<(unsigned)a.batch, TPB, smem, st>>>(a);
  return cudaGetLastError();
}

template <int A, int S, class G>
cudaError_t launch_me_one(const DecodeArgs& a, cudaStream_t st) {
  return a.cta_threads == 512 ? launch_me_tpb<A, S, G, 512>(a, st) : launch_me_tpb<A, S, G, 256>(a, st);
}

template <int A, class G>
cudaError_t launch_me_sched(const DecodeArgs& a, int sched, cudaStream_t s) {
  if (sched == kMECIRBP) return launch_me_one<A, kMECIRBP, G>(a, s);
  return launch_me_one<A, kMELMD, G>(a, s);
}

}  // namespace

cudaError_t launch_me_queue(const QueueArgs& q, int arith, int sched, int threads, int grid, size_t smem,
                            cudaStream_t s) {
  if (q.n_items == 0) return cudaSuccess;
  const bool lmd = sched == kMELMD, big = threads == 512;
  if (arith == kFP32) {
    if (lmd) return big ? launch_me_queue_tpb<kFP32, kMELMD, 512>(q, grid, smem, s) : launch_me_queue_tpb<kFP32, kMELMD, 256>(q, grid, smem, s);
    return big ? launch_me_queue_tpb<kFP32, kMECIRBP, 512>(q, grid, smem, s) : launch_me_queue_tpb<kFP32, kMECIRBP, 256>(q, grid, smem, s);
  }
  if (lmd) return big ? launch_me_queue_tpb<kINT6, kMELMD, 512>(q, grid, smem, s) : launch_me_queue_tpb<kINT6, kMELMD, 256>(q, grid, smem, s);
  return big ? launch_me_queue_tpb<kINT6, kMECIRBP, 512>(q, grid, smem, s) : launch_me_queue_tpb<kINT6, kMECIRBP, 256>(q, grid, smem, s);
}

namespace {
template <int A, int S, int TPB>
cudaError_t me_queue_occ(size_t smem, int* out) {
  auto k = me_queue_kernel<A, S, TPB>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, TPB, smem);
}
}  // namespace

cudaError_t me_queue_blocks_per_sm(int arith, int sched, int threads, size_t smem, int* out) {
  const bool lmd = sched == kMELMD, big = threads == 512;
  if (arith == kFP32) {
    if (lmd) return big ? me_queue_occ<kFP32, kMELMD, 512>(smem, out) : me_queue_occ<kFP32, kMELMD, 256>(smem, out);
    return big ? me_queue_occ<kFP32, kMECIRBP, 512>(smem, out) : me_queue_occ<kFP32, kMECIRBP, 256>(smem, out);
  }
  if (lmd) return big ? me_queue_occ<kINT6, kMELMD, 512>(smem, out) : me_queue_occ<kINT6, kMELMD, 256>(smem, out);
  return big ? me_queue_occ<kINT6, kMECIRBP, 512>(smem, out) : me_queue_occ<kINT6, kMECIRBP, 256>(smem, out);
}

bool me_cluster_plan(int arith, const GraphDesc& g, int n_p, int n_g, int cs, int64_t avail, ClusterPlan* out) {
  const int msg = arith == kINT6 ? 1 : 4, llr = arith == kINT6 ? 2 : 4, dv = arith == kINT6 ? 2 : 4;
  const int64_t ncnl = (int64_t)n_p * (g.dv_max > 1 ? g.dv_max - 1 : 1);
  const int64_t Mw = (g.M + 31) / 32, Nw = (g.N + 31) / 32;
  // elements and element sizes in array order
  const int64_t n[kClusterArrays] = {g.E, g.E, g.N, g.N, g.N, g.N, g.N, Mw,
                                     2 * (int64_t)n_p, n_p, n_p, std::max<int64_t>(ncnl, kCap), ncnl, Mw, n_g, n_g,
                                     Nw, Nw, 1};
  const int sz[kClusterArrays] = {msg, msg, llr, llr, dv, 4, 1, 4, 4, 4, 8, 8, 4, 4, 4, 4, 4, 4,
                                  (int)sizeof(MEMisc)};
  ClusterPlan p;
  std::memset(&p, 0, sizeof(p));
  p.cs = cs;
  std::vector<int64_t> used((size_t)cs, 0);
  auto a16 = [](int64_t x) { return (x + 15) & ~(int64_t)15; };
  auto spread = [&](int k) {  // same offset in every rank, 2^shift >= ceil(n / cs) elements each
    int sh = 2;
    while (((int64_t)1 << sh) * cs < n[k]) ++sh;
    int64_t at = 0;
    for (int64_t u : used) at = std::max(at, u);
    p.off[k] = (int32_t)at;
    p.shift[k] = (int8_t)sh;
    p.rank0[k] = 0;
    for (auto& u : used) u = at + a16(((int64_t)1 << sh) * sz[k]);
  };
  for (int k = 0; k < 8; ++k) spread(k);
  for (int k = 8; k < kClusterArrays; ++k) {
    int sh = 2;
    while (((int64_t)1 << sh) < n[k]) ++sh;
    const int64_t bytes = a16(((int64_t)1 << sh) * sz[k]);
    int best = 0;
    for (int r = 1; r < cs; ++r)
      if (used[(size_t)r] < used[(size_t)best]) best = r;
    if (used[(size_t)best] + bytes <= avail) {  // whole array in the least used rank
      p.off[k] = (int32_t)used[(size_t)best];
      p.shift[k] = (int8_t)sh;
      p.rank0[k] = (int8_t)best;
      used[(size_t)best] += bytes;
    } else {
      spread(k);
    }
  }
  int64_t mx = 0;
  for (int64_t u : used) mx = std::max(mx, u);
  if (mx > avail || mx > 0x7fffffff) return false;
  p.bytes = (int32_t)mx;
  *out = p;
  return true;
}

cudaError_t launch_me_cluster(const DecodeArgs& a, int arith, int sched, int threads, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  const bool lmd = sched == kMELMD, big = threads == 512;
#define LDPC_CL(AR, SC, GR) (big ? launch_me_cluster_t<AR, SC, GR, 512>(a, s) : launch_me_cluster_t<AR, SC, GR, 256>(a, s))
  if (arith == kFP32) {
    if (a.g.is_qc) return lmd ? LDPC_CL(kFP32, kMELMD, QCGraph) : LDPC_CL(kFP32, kMECIRBP, QCGraph);
    return lmd ? LDPC_CL(kFP32, kMELMD, TabGraph) : LDPC_CL(kFP32, kMECIRBP, TabGraph);
  }
  if (a.g.is_qc) return lmd ? LDPC_CL(kINT6, kMELMD, QCGraph) : LDPC_CL(kINT6, kMECIRBP, QCGraph);
  return lmd ? LDPC_CL(kINT6, kMELMD, TabGraph) : LDPC_CL(kINT6, kMECIRBP, TabGraph);
#undef LDPC_CL
}

size_t me_smem_per_frame(int arith, int sched, const GraphDesc& g, int n_p, int n_g) {
  (void)sched;
  (void)n_p;
  (void)n_g;
  return (size_t)me_big(arith, g.M, g.N, g.E).total;
}

size_t me_smem_per_cta(const GraphDesc& g, int n_p, int n_g) {
  return (size_t)me_small(g.M, g.N, n_p, g.dv_max, n_g).total;
}

cudaError_t launch_me(const DecodeArgs& a, int arith, int sched, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  if (arith == kFP32)
    return a.g.is_qc ? launch_me_sched<kFP32, QCGraph>(a, sched, s) : launch_me_sched<kFP32, TabGraph>(a, sched, s);
  return a.g.is_qc ? launch_me_sched<kINT6, QCGraph>(a, sched, s) : launch_me_sched<kINT6, TabGraph>(a, sched, s);
}

}  // namespace ldpc
