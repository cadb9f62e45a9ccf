// decode_flood.cu -- flooding BP (Sec. 1), one frame per CTA.
//
// One iteration computes every V2C message from the previous C2V messages
// (eq. 1, written as L_n - L^C_{m->n}) and every C2V message from those
// (eq. 2 or min-sum) in one pass of check teams (each edge is read and
// rewritten by the lane that owns it, so the update is in place), then the
// total LLRs (eq. 3).  An iteration propagates E messages (Sec. 2.A).
#include "device_math.cuh"

namespace ldpc {

namespace {

// Decode frame b with its state at `base` (shared or global memory).
template <int A, class G>
__device__ __forceinline__ void flood_frame(const DecodeArgs& a, const G& g, int64_t b, unsigned char* base) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  const int N = a.g.N, E = a.g.E, M = a.g.M;
  const FloodLayout ly = flood_layout(A, N, E);
  M_* C = (M_*)(base + ly.C);
  L_* lam = (L_*)(base + ly.lam);
  L_* L = (L_*)(base + ly.L);
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int W = a.team_w, tpw = 32 / W, team = lane / W, r = lane % W;
  const float clip = a.llr_clip;

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
    lam[n] = v;
    L[n] = v;
  }
  for (int e = tid; e < E; e += nt) C[e] = (M_)0;
  if (__syncthreads_or(bad)) {
    for (int n = tid; n < N; n += nt) {
      if (a.hard) a.hard[b * N + n] = 0;
      if (a.llr_out) a.llr_out[b * N + n] = (float)lam[n];
    }
    if (tid == 0) {
      if (a.updates) a.updates[b] = 0;
      if (a.converged) a.converged[b] = 2;
      atomicOr(a.status, 1u);
    }
    return;
  }

  auto syndrome_nonzero = [&]() -> int {
    int any = 0;
    for (int m = tid; m < M; m += nt) {
      const typename G::C cc = g.cn(m);
      unsigned p = 0;
      for (int k = 0; k < cc.d; ++k) p ^= (L[g.cvn(cc, k)] < (L_)0);
      any |= (int)p;
    }
    return __syncthreads_or(any);
  };

  int64_t count = 0, left = a.check_interval;
  bool ok = a.check_interval > 0 && !syndrome_nonzero();
  while (!ok && count + E <= a.max_updates) {
    for (int t0 = warp * tpw; t0 < M; t0 += nw * tpw) {  // every C2V from the previous V2C
      const int m = t0 + team;
      int e, j;
      M_ out;
      const int dc = team_c2v<A, G>(g, C, L, m < M ? m : -1, r, W, clip, e, j, out);
      if (r < dc) C[e] = out;
    }
    __syncthreads();
    for (int n = tid; n < N; n += nt) L[n] = vn_total<A, G>(g, lam, C, n);  // eq. (3)
    __syncthreads();
    count += E;
    if (check_due(left, a.check_interval, E)) ok = !syndrome_nonzero();
  }
  const int conv = !syndrome_nonzero();
  for (int n = tid; n < N; n += nt) {
    if (a.hard) a.hard[b * N + n] = (uint8_t)(L[n] < (L_)0);
    if (a.llr_out) a.llr_out[b * N + n] = (float)L[n];
  }
  if (a.c2v_out)
    for (int e = tid; e < E; e += nt) a.c2v_out[b * (int64_t)E + e] = (float)C[e];
  if (tid == 0) {
    if (a.updates) a.updates[b] = count;
    if (a.converged) a.converged[b] = (uint8_t)conv;
    if (a.fallbacks) a.fallbacks[b] = 0;
  }
  __syncthreads();
}

template <int A, class G>
__global__ void __launch_bounds__(512) flood_decode_kernel(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  flood_frame<A, G>(a, g, blockIdx.x, smem_raw + a.graph_smem);
}

// Global-memory form: CTA c owns state slot c and decodes frames c + k gridDim.x.
template <int A, class G>
__global__ void __launch_bounds__(512) flood_decode_kernel_gs(const DecodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  unsigned char* base = (unsigned char*)a.gstate + (int64_t)blockIdx.x * a.gstate_stride;
  for (int64_t b = blockIdx.x; b < a.batch; b += gridDim.x) flood_frame<A, G>(a, g, b, base);
}

int flood_threads(const DecodeArgs& a) { return a.g.E >= 4096 ? 512 : (a.g.E >= 1024 ? 256 : 128); }

template <int A, class G>
cudaError_t launch_g(const DecodeArgs& a, cudaStream_t s) {
  if (a.gstate) {
    auto k = flood_decode_kernel_gs<A, G>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.graph_smem);
    if (err != cudaSuccess) return err;
    k<<<(unsigned)a.gstate_ctas, flood_threads(a), a.graph_smem, s>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)a.graph_smem + (size_t)a.smem_per_frame;
  auto k = flood_decode_kernel<A, G>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k<<<(unsigned)a.batch, flood_threads(a), smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t flood_smem_per_frame(int arith, const GraphDesc& g) { return (size_t)flood_layout(arith, g.N, g.E).total; }

cudaError_t launch_flood(const DecodeArgs& a, int arith, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  if (arith == kFP32) return a.g.is_qc ? launch_g<kFP32, QCGraph>(a, s) : launch_g<kFP32, TabGraph>(a, s);
  return a.g.is_qc ? launch_g<kINT6, QCGraph>(a, s) : launch_g<kINT6, TabGraph>(a, s);
}

}  // namespace ldpc
