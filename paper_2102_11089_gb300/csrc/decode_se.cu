// decode_se.cu -- single-edge dynamic schedules, one frame per warp.
//
// Residual BP (Sec. 2.A, steps 1-4), CIRBP (Algorithm 1) and LMD-CIRBP
// (Algorithm 3) commit one check-to-variable (C2V) message per update.  The
// chain select -> commit -> refresh -> select is serial within a frame, so a
// frame is one warp: lanes cover the edges into the updated variable node and
// the flattened two-hop neighbourhood N(i)\n*, i in M(n*)\m*, that the
// algorithms refresh (Alg. 1 lines 10-13).  Frames are independent warps; all
// per-frame state lives in shared memory:
//   C[E]  committed messages L^C        P[E]  precomputed messages L~^C (eq. 2)
//   lam, L, Lt [N]  channel / total / precomputed LLR (eq. 3, Sec. 2.B)
//   D[N]  conditional innovation (eq. 8)
//   Rmax/Ridx[M]  per-check largest residual (eq. 4) for the global argmax of
//                 eq. (5) (RBP, and CIRBP's fallback, Alg. 1 line 6)
//   par[M/32]     syndrome bits (tentative decisions bsgn(L), Sec. 2.A)
// The graph (CSR/CSC maps) is read from global memory through the L1 cache;
// every warp of a CTA decodes another frame of the same code.
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
  L_* Lt;
  D_* D;
  M_* Rmax;
  int32_t* Ridx;
  uint32_t* par;
  int32_t* fe;   // flattened refresh list: edge id
  int32_t* fs;   // segment start | (segment length << 16)
  int32_t* fj;   // variable node of the entry
  void* scr;     // per-entry encoded V2C (float phi or int8 V)
  int16_t* tab;  // INT6 CI table
};

__device__ __forceinline__ float ci_val(const SEState<kFP32>&, float a, float b) { return ci_fp(a, b); }
__device__ __forceinline__ uint16_t ci_val(const SEState<kINT6>& s, int a, int b) {
  return ci_int(a, b, s.tab);
}

// residual |L~^C - L^C| (eq. 4) as an argmax key
__device__ __forceinline__ uint32_t rkey(float p, float c) { return mkey(fabsf(p - c)); }
__device__ __forceinline__ uint32_t rkey(int8_t p, int8_t c) { return (uint32_t)abs((int)p - (int)c); }

// Precomputed C2V of one flattened entry t from the encoded V2C entries of its
// check (exclude-one over [start, start + len), Eq. 2 / min-sum).
__device__ __forceinline__ float c2v_entry(const float* scr, int t, int start, int len, float clip) {
  float sum = 0.0f;
  unsigned neg = 0;
  for (int k = start; k < start + len; ++k) {
    if (k == t) continue;
    const float v = scr[k];
    sum += fabsf(v);
    neg ^= (__float_as_uint(v) >> 31);
  }
  return combine_fp(sum, neg, clip);
}
__device__ __forceinline__ int8_t c2v_entry(const int8_t* scr, int t, int start, int len, float) {
  int mag = 31;
  unsigned neg = 0;
  for (int k = start; k < start + len; ++k) {
    if (k == t) continue;
    const int v = scr[k];
    neg ^= (v < 0);
    mag = min(mag, abs(v));
  }
  return (int8_t)(neg ? -mag : mag);
}

template <int A>
__device__ __forceinline__ typename Arith<A>::llr warp_sum_llr(typename Arith<A>::llr v);
template <>
__device__ __forceinline__ float warp_sum_llr<kFP32>(float v) { return warp_sum_f(v); }
template <>
__device__ __forceinline__ int16_t warp_sum_llr<kINT6>(int16_t v) {
  return (int16_t)__reduce_add_sync(kFull, (int)v);
}

// total LLR from scratch: lam[n] + sum_{m in M(n)} X[e] (eq. 3 / Sec. 2.B), by one lane
template <int A, typename MT>
__device__ __forceinline__ typename Arith<A>::llr vn_total(const DevCode& g, const SEState<A>& s,
                                                           const MT* X, int n) {
  using L_ = typename Arith<A>::llr;
  const int b0 = __ldg(g.vn_ptr + n), b1 = __ldg(g.vn_ptr + n + 1);
  L_ acc = s.lam[n];
  for (int k = b0; k < b1; ++k) acc = (L_)(acc + X[__ldg(g.vn_e + k)]);
  return acc;
}

// argmax over D of every VN, lowest index on ties (Alg. 1 line 4)
template <int A>
__device__ __forceinline__ int global_argmax_D(const DevCode& g, const SEState<A>& s, uint32_t& key) {
  uint32_t bk = 0, bi = 0xffffffffu;
  for (int n = threadIdx.x & 31; n < g.N; n += 32) {
    const uint32_t k = mkey(s.D[n]);
    if (k > bk || bi == 0xffffffffu) { bk = k; bi = n; }
  }
  return (int)warp_argmax(bk, bi, key);
}

// argmax over the residual of every edge, eq. (5), via the per-check maxima
template <int A>
__device__ __forceinline__ int global_argmax_R(const DevCode& g, const SEState<A>& s) {
  uint32_t bk = 0, bi = 0xffffffffu;
  for (int m = threadIdx.x & 31; m < g.M; m += 32) {
    const uint32_t k = rkey(s.Rmax[m], (typename Arith<A>::msg)0);
    if (k > bk || bi == 0xffffffffu) { bk = k; bi = (uint32_t)s.Ridx[m]; }
  }
  uint32_t key;
  return (int)warp_argmax(bk, bi, key);
}

// argmax_i R_{i->n} over i in M(n), lowest edge id on ties (Alg. 1 line 8)
template <int A>
__device__ __forceinline__ int argmax_R_into(const DevCode& g, const SEState<A>& s, int n) {
  const int lane = threadIdx.x & 31;
  const int b0 = __ldg(g.vn_ptr + n), b1 = __ldg(g.vn_ptr + n + 1);
  uint32_t bk = 0, bi = 0xffffffffu;
  for (int k = b0 + lane; k < b1; k += 32) {
    const int e = __ldg(g.vn_e + k);
    am_update(bk, bi, rkey(s.P[e], s.C[e]), (uint32_t)e);
  }
  uint32_t key;
  return (int)warp_argmax(bk, bi, key);
}

// per-check largest residual (value, lowest edge id), one lane
template <int A>
__device__ __forceinline__ void refresh_rmax(const DevCode& g, const SEState<A>& s, int m) {
  const int b0 = __ldg(g.cn_ptr + m), b1 = __ldg(g.cn_ptr + m + 1);
  uint32_t bk = 0, bi = (uint32_t)b0;
  for (int e = b0; e < b1; ++e) {
    const uint32_t k = rkey(s.P[e], s.C[e]);
    if (k > bk) { bk = k; bi = e; }
  }
  using M_ = typename Arith<A>::msg;
  if (A == kFP32) s.Rmax[m] = (M_)__uint_as_float(bk);
  else s.Rmax[m] = (M_)bk;
  s.Ridx[m] = (int32_t)bi;
}

template <int A, int SCHED>
__global__ void __launch_bounds__(512) se_decode_kernel(const DecodeArgs a) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  using D_ = typename Arith<A>::dval;
  constexpr bool kNeedR = SCHED != kLMD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * a.frames_per_cta + warp;
  if (b >= a.batch) return;
  const DevCode& g = a.g;
  const SELayout ly = se_layout(A, g.M, g.N, g.E, g.maxr, kNeedR);
  unsigned char* base = smem_raw + (size_t)warp * ly.total;
  SEState<A> s;
  s.C = (M_*)(base + ly.C);
  s.P = (M_*)(base + ly.P);
  s.lam = (L_*)(base + ly.lam);
  s.L = (L_*)(base + ly.L);
  s.Lt = (L_*)(base + ly.Lt);
  s.D = (D_*)(base + ly.D);
  s.Rmax = (M_*)(base + ly.Rmax);
  s.Ridx = (int32_t*)(base + ly.Ridx);
  s.par = (uint32_t*)(base + ly.par);
  s.fe = (int32_t*)(base + ly.fe);
  s.fs = (int32_t*)(base + ly.fs);
  s.fj = (int32_t*)(base + ly.fj);
  s.scr = (void*)(base + ly.scr);
  s.tab = (int16_t*)(base + ly.tab);
  M_* scr = (M_*)s.scr;
  const float clip = a.llr_clip;
  const int N = g.N, E = g.E, M = g.M;

  if (A == kINT6)
    for (int i = lane; i < 256; i += 32) s.tab[i] = a.ci_table[i];

  // ---- channel LLRs (coalesced) and input validation
  bool bad = false;
  for (int n = lane; n < N; n += 32) {
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
  if (__any_sync(kFull, bad)) {
    for (int n = lane; n < N; n += 32) {
      if (a.hard) a.hard[b * N + n] = 0;
      if (a.llr_out) a.llr_out[b * N + n] = (float)s.lam[n];
    }
    if (lane == 0) {
      if (a.updates) a.updates[b] = 0;
      if (a.converged) a.converged[b] = 2;
      atomicOr(a.status, 1u);
    }
    return;
  }

  // ---- Alg. 1 lines 1-3: L^C = 0, L = L^V = lambda, all L~^C, R, L~, D.
  // C doubles as the scratch of encoded V2C values (V = lambda) first.
  for (int e = lane; e < E; e += 32) {
    const int j = __ldg(g.e_vn + e);
    if (A == kFP32) ((float*)s.C)[e] = encode_fp((float)s.lam[j], clip);
    else ((int8_t*)s.C)[e] = encode_int((int)s.lam[j]);
  }
  __syncwarp();
  for (int e = lane; e < E; e += 32) {
    const int m = __ldg(g.e_cn + e);
    const int c0 = __ldg(g.cn_ptr + m), c1 = __ldg(g.cn_ptr + m + 1);
    s.P[e] = c2v_entry((const M_*)s.C, e, c0, c1 - c0, clip);
  }
  __syncwarp();
  for (int e = lane; e < E; e += 32) s.C[e] = (M_)0;
  __syncwarp();
  for (int n = lane; n < N; n += 32) {
    const L_ lt = vn_total<A>(g, s, s.P, n);
    s.Lt[n] = lt;
    s.D[n] = ci_val(s, s.L[n], lt);
  }
  uint32_t unsat = 0;
  for (int m0 = 0; m0 < M; m0 += 32) {
    const int m = m0 + lane;
    unsigned p = 0;
    if (m < M) {
      const int c0 = __ldg(g.cn_ptr + m), c1 = __ldg(g.cn_ptr + m + 1);
      for (int e = c0; e < c1; ++e) p ^= (s.L[__ldg(g.e_vn + e)] < (L_)0);
    }
    const unsigned bits = __ballot_sync(kFull, p);
    if (lane == 0) s.par[m0 >> 5] = bits;
    unsat += __popc(bits);
  }
  __syncwarp();
  if (kNeedR)
    for (int m = lane; m < M; m += 32) refresh_rmax<A>(g, s, m);
  __syncwarp();

  // ---- schedule loop
  int64_t count = 0;
  int nstar = 0;
  bool stop = (a.check_interval > 0 && unsat == 0);
  if (!stop && SCHED == kLMD) {
    uint32_t k;
    nstar = global_argmax_D<A>(g, s, k);  // Alg. 3 line 4
  }
  while (!stop && count < a.max_updates) {
    int estar;
    // -- selection
    if (SCHED == kRBP) {
      estar = global_argmax_R<A>(g, s);
      nstar = __ldg(g.e_vn + estar);
    } else if (SCHED == kCIRBP) {
      uint32_t dkey;
      nstar = global_argmax_D<A>(g, s, dkey);
      const bool fallback = (A == kFP32) ? (__uint_as_float(dkey) < a.gamma_f)
                                         : ((int)dkey < a.gamma_i);
      if (fallback) {  // Alg. 1 line 6
        estar = global_argmax_R<A>(g, s);
        nstar = __ldg(g.e_vn + estar);
      } else {
        estar = argmax_R_into<A>(g, s, nstar);  // line 8
      }
    } else {
      estar = argmax_R_into<A>(g, s, nstar);  // Alg. 3 line 5
    }
    const int mstar = __ldg(g.e_cn + estar);
    const int vb = __ldg(g.vn_ptr + nstar), dv = __ldg(g.vn_ptr + nstar + 1) - vb;

    // -- commit (Alg. 1 line 9): L^C <- L~^C, update L_{n*}
    const L_ Lold = s.L[nstar];
    __syncwarp();
    if (lane == 0) s.C[estar] = s.P[estar];
    __syncwarp();
    // lane k < dv owns edge vn_e[vb + k] (dv <= 32 for this form)
    const int my_e = lane < dv ? __ldg(g.vn_e + vb + lane) : 0;
    const int my_m = lane < dv ? __ldg(g.e_cn + my_e) : 0;
    L_ part = lane < dv ? (L_)s.C[my_e] : (L_)0;
    if (A == kFP32 && lane == 0) part = (L_)(part + s.lam[nstar]);
    L_ Lnew = warp_sum_llr<A>(part);
    if (A == kINT6) Lnew = (L_)(Lnew + s.lam[nstar]);
    if (lane == 0) {
      s.L[nstar] = Lnew;
      s.D[nstar] = ci_val(s, Lnew, s.Lt[nstar]);  // reading: D of n* follows L_{n*}
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
    if (lane == 0 && a.trace) a.trace[b * a.max_updates + count] = estar;

    // -- refresh (Alg. 1 lines 10-13): for i in M(n*)\m*, V2C n*->i, then
    //    L~^C, R, L~_j, D_j for j in N(i)\n*
    int deg = 0, cbase = 0;
    if (lane < dv && my_m != mstar) {
      cbase = __ldg(g.cn_ptr + my_m);
      deg = __ldg(g.cn_ptr + my_m + 1) - cbase;
    }
    int off = deg;  // inclusive scan over lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, off, o);
      if (lane >= o) off += y;
    }
    const int T = __shfl_sync(kFull, off, 31);
    off -= deg;
    for (int k = 0; k < deg; ++k) {
      s.fe[off + k] = cbase + k;
      s.fs[off + k] = off | (deg << 16);
    }
    __syncwarp();
    for (int t = lane; t < T; t += 32) {  // new V2C inputs of the refreshed checks
      const int e = s.fe[t];
      const int j = __ldg(g.e_vn + e);
      s.fj[t] = j;
      if (A == kFP32) ((float*)scr)[t] = encode_fp((float)s.L[j] - (float)s.C[e], clip);
      else ((int8_t*)scr)[t] = encode_int((int)s.L[j] - (int)s.C[e]);
    }
    __syncwarp();
    for (int t = lane; t < T; t += 32) {  // precomputed C2V into j != n*
      if (s.fj[t] == nstar) continue;
      const int sg = s.fs[t];
      s.P[s.fe[t]] = c2v_entry((const M_*)scr, t, sg & 0xffff, sg >> 16, clip);
    }
    __syncwarp();
    uint32_t ck = 0, ci_ = 0xffffffffu;
    for (int t = lane; t < T; t += 32) {  // L~_j and D_j
      const int j = s.fj[t];
      if (j == nstar) continue;
      const L_ lt = vn_total<A>(g, s, s.P, j);
      const D_ d = ci_val(s, s.L[j], lt);
      s.Lt[j] = lt;
      s.D[j] = d;
      am_update(ck, ci_, mkey(d), (uint32_t)j);
    }
    __syncwarp();
    if (kNeedR && lane < dv) refresh_rmax<A>(g, s, my_m);
    __syncwarp();

    ++count;
    if (a.check_interval > 0 && (count % a.check_interval) == 0 && unsat == 0) break;

    // -- LMD: next target = argmax D over U(m*, n*) (Alg. 3 line 11), or over
    //    N(m*)\n* when d_v(n*) = 1 (Sec. 5.A), else the global argmax.
    if (SCHED == kLMD) {
      if (dv == 1) {
        ck = 0; ci_ = 0xffffffffu;
        const int c0 = __ldg(g.cn_ptr + mstar), c1 = __ldg(g.cn_ptr + mstar + 1);
        for (int e = c0 + lane; e < c1; e += 32) {
          const int j = __ldg(g.e_vn + e);
          if (j != nstar) am_update(ck, ci_, mkey(s.D[j]), (uint32_t)j);
        }
      }
      uint32_t key;
      const uint32_t nn = warp_argmax(ck, ci_, key);
      if (nn == 0xffffffffu) nstar = global_argmax_D<A>(g, s, key);
      else nstar = (int)nn;
    }
  }

  // ---- outputs
  for (int n = lane; n < N; n += 32) {
    if (a.hard) a.hard[b * N + n] = (uint8_t)(s.L[n] < (L_)0);
    if (a.llr_out) a.llr_out[b * N + n] = (float)s.L[n];
  }
  if (lane == 0) {
    if (a.updates) a.updates[b] = count;
    if (a.converged) a.converged[b] = unsat == 0 ? 1 : 0;
  }
}

template <int A, int S>
cudaError_t launch_one(const DecodeArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)a.smem_per_frame * a.frames_per_cta;
  auto k = se_decode_kernel<A, S>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int64_t grid = (a.batch + a.frames_per_cta - 1) / a.frames_per_cta;
  k<<<(unsigned)grid, 32 * a.frames_per_cta, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t se_smem_per_frame(int arith, int sched, const DevCode& g) {
  return (size_t)se_layout(arith, g.M, g.N, g.E, g.maxr, sched != kLMD).total;
}

cudaError_t launch_se(const DecodeArgs& a, int arith, int sched, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  if (arith == kFP32) {
    if (sched == kRBP) return launch_one<kFP32, kRBP>(a, s);
    if (sched == kCIRBP) return launch_one<kFP32, kCIRBP>(a, s);
    return launch_one<kFP32, kLMD>(a, s);
  }
  if (sched == kRBP) return launch_one<kINT6, kRBP>(a, s);
  if (sched == kCIRBP) return launch_one<kINT6, kCIRBP>(a, s);
  return launch_one<kINT6, kLMD>(a, s);
}

}  // namespace ldpc
