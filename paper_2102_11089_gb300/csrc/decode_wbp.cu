// decode_wbp.cu -- weighted BP along a recorded schedule, and its adjoint.
//
// Not a step of the paper: the differentiable decoder built on its schedules.
// A CI decoder records which edge it committed at each update (the trace); the
// weighted decoder replays that schedule with one FP32 weight per update:
// update t commits C[e_t] <- w[t] * P_t, where P_t is the clipped sum-product
// C2V of eq. (2) from the state before the update, and the output is
// L_n = lambda_n + sum_{m in M(n)} C[m->n] (eq. 3).  With unit weights the
// replay is the decoder's own message passing.
//
// Each update overwrites one entry of C, so the forward keeps the overwritten
// value (a 4-byte tape per update) and the adjoint walks the updates
// backwards, restoring every earlier state exactly instead of checkpointing
// and recomputing.  One warp per frame; lane k owns edge k of the committed
// edge's check.  For the C2V of edge e from the other inputs u_i of its check
// (phi(x) = -ln tanh(x/2), S = sum_i phi(|u_i|), |prod tanh(u_i/2)| = e^-S):
//   P = sign * phi(S),   dP/du_k = s_k (1 - e^(-2 phi_k)) e^-(S - phi_k) / (1 - e^(-2S)),
// s_k the sign of the other inputs, zero where u_k or P is clipped.
#include <algorithm>

#include "device_math.cuh"

namespace ldpc {

namespace {

// V2C of edge e2 (eq. 1): lambda_n + sum_{e3 in M(n)\e2} C[e3], in edge order
template <class G>
__device__ __forceinline__ float w_v2c(const G& g, const float* lam, const float* C, int n, int e2) {
  const typename G::V v = g.vn(n);
  float s = lam[n];
  for (int k = 0; k < v.d; ++k) {
    int e3, m3;
    g.vedge(v, k, e3, m3);
    if (e3 != e2) s += C[e3];
  }
  return s;
}

// The inputs of the C2V of edge e: lane k < dc holds edge k of e's check.
struct WInputs {
  int e2, n2;       // this lane's edge and variable (valid if in)
  bool in;          // an input of the C2V of e
  float u, ph;      // V2C input and phi(|u| clipped)
  unsigned neg;     // sign bit of u
  float S, Sx;      // sum of phi over the inputs, and without this lane's
  unsigned sgn;     // parity of the input signs (sign of P)
};

template <class G>
__device__ __forceinline__ WInputs w_inputs(const G& g, const float* lam, const float* C, int e, float clip) {
  const int lane = threadIdx.x & 31;
  const typename G::C cc = g.cn(g.ecn(e));
  WInputs w;
  w.in = lane < cc.d && cc.b + lane != e;
  w.e2 = cc.b + lane;
  w.n2 = lane < cc.d ? g.cvn(cc, lane) : 0;
  w.u = w.in ? w_v2c(g, lam, C, w.n2, w.e2) : 0.0f;
  w.ph = w.in ? phi_f(fminf(fabsf(w.u), clip)) : 0.0f;
  w.neg = w.in && w.u < 0.0f ? 1u : 0u;
  // inclusive prefix / suffix sums of phi over the lanes (fixed order)
  float pre = w.ph, suf = w.ph;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float a = __shfl_up_sync(kFull, pre, o), b = __shfl_down_sync(kFull, suf, o);
    if (lane >= o) pre += a;
    if (lane + o < 32) suf += b;
  }
  const float pl = __shfl_up_sync(kFull, pre, 1), sr = __shfl_down_sync(kFull, suf, 1);
  w.Sx = (lane > 0 ? pl : 0.0f) + (lane < 31 ? sr : 0.0f);
  w.S = __shfl_sync(kFull, pre, 31);
  w.sgn = __popc(__ballot_sync(kFull, w.neg)) & 1u;
  return w;
}

// Shared-memory layout of one frame (warp): C[E] | lam[N] (| Cb[E] | dlam[N] backward)
__host__ __device__ inline int wbp_frame_bytes(int N, int E, bool backward) {
  return align16(E * 4) + align16(N * 4) + (backward ? align16(E * 4) + align16(N * 4) : 0);
}

template <class G>
__global__ void __launch_bounds__(256) wbp_forward_kernel(const WbpArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= a.batch) return;
  const int N = a.g.N, E = a.g.E;
  unsigned char* base = smem_raw + a.graph_smem + (size_t)warp * a.frame_bytes;
  float* C = (float*)base;
  float* lam = (float*)(base + align16(E * 4));
  for (int n = lane; n < N; n += 32) lam[n] = a.llr[b * N + n];
  for (int e = lane; e < E; e += 32) C[e] = 0.0f;
  __syncwarp();
  const int32_t* tr = a.trace + b * a.T;
  const int64_t cnt = a.counts ? min(a.counts[b], a.T) : a.T;
  for (int64_t t = 0; t < cnt; ++t) {
    const int e = tr[t];
    if ((unsigned)e >= (unsigned)E) {  // not an edge id: flag it, leave the frame's outputs
      if (lane == 0) atomicOr(a.status, 4u);
      return;
    }
    const WInputs w = w_inputs<G>(g, lam, C, e, a.clip);
    const float P = fminf(phi_f(w.S), a.clip);
    __syncwarp();
    if (lane == 0) {
      if (a.tape) a.tape[b * a.T + t] = C[e];
      C[e] = a.w[t] * (w.sgn ? -P : P);
    }
    __syncwarp();
  }
  for (int n = lane; n < N; n += 32) {
    if (a.llr_out) a.llr_out[b * N + n] = w_v2c(g, lam, C, n, -1);
  }
  if (a.c_out)
    for (int e = lane; e < E; e += 32) a.c_out[b * E + e] = C[e];
}

template <class G>
__global__ void __launch_bounds__(512) wbp_backward_kernel(const WbpArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const G g = GraphStage<G>::make(a.g, (int32_t*)smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= a.batch) return;
  const int N = a.g.N, E = a.g.E;
  unsigned char* base = smem_raw + a.graph_smem + (size_t)warp * a.frame_bytes;
  float* C = (float*)base;
  float* lam = (float*)(base + align16(E * 4));
  float* Cb = (float*)(base + align16(E * 4) + align16(N * 4));
  float* lb = (float*)(base + 2 * align16(E * 4) + align16(N * 4));
  // final state of the forward; dloss/dC[e] = dloss/dL of its variable
  for (int n = lane; n < N; n += 32) {
    lam[n] = a.llr[b * N + n];
    lb[n] = a.dL[b * N + n];
  }
  for (int e = lane; e < E; e += 32) C[e] = a.c_in[b * E + e];
  __syncwarp();
  for (int e = lane; e < E; e += 32) Cb[e] = lb[g.evn(e)];
  float* dw = a.dw_frames + b * a.T;
  const int64_t cnt = a.counts ? min(a.counts[b], a.T) : a.T;
  for (int64_t t = cnt + lane; t < a.T; t += 32) dw[t] = 0.0f;
  __syncwarp();
  const int32_t* tr = a.trace + b * a.T;
  for (int64_t t = cnt - 1; t >= 0; --t) {
    const int e = tr[t];
    if ((unsigned)e >= (unsigned)E) {  // not an edge id: flag it, leave the frame's outputs
      if (lane == 0) atomicOr(a.status, 4u);
      return;
    }
    if (lane == 0) C[e] = a.tape_in[b * a.T + t];  // the state before update t
    __syncwarp();
    const WInputs w = w_inputs<G>(g, lam, C, e, a.clip);
    const float phiS = phi_f(w.S);
    const float P = fminf(phiS, a.clip);
    const float ab = Cb[e];
    __syncwarp();
    if (lane == 0) {
      dw[t] = ab * (w.sgn ? -P : P);
      Cb[e] = 0.0f;  // C[e] before the update does not reach the result
    }
    const float Pb = ab * a.w[t];
    if (Pb != 0.0f && phiS < a.clip && w.in && fabsf(w.u) < a.clip) {
      // dP/du_k, then u_k = lambda_n + sum_{e3 in M(n)\e2} C[e3]
      const float r = __fdividef(expm1f(-2.0f * w.ph), expm1f(-2.0f * w.S)) * expf(-w.Sx);
      const unsigned sk = w.sgn ^ w.neg;  // sign of the other inputs
      const float ub = Pb * (sk ? -r : r);
      lb[w.n2] += ub;
      const typename G::V v = g.vn(w.n2);
      for (int k = 0; k < v.d; ++k) {
        int e3, m3;
        g.vedge(v, k, e3, m3);
        if (e3 != w.e2) Cb[e3] += ub;
      }
    }
    __syncwarp();
  }
  if (a.dllr)
    for (int n = lane; n < N; n += 32) a.dllr[b * N + n] = lb[n];
}

// dw[t] = sum over frames of dw_frames[b][t] (fixed order over b)
__global__ void wbp_colsum_kernel(const float* dw_frames, int64_t batch, int64_t T, float* dw) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int64_t b = 0; b < batch; ++b) s += dw_frames[b * T + t];
    dw[t] = s;
  }
}

template <class G>
cudaError_t wbp_launch_t(const WbpArgs& a, bool backward, int fpc, cudaStream_t st) {
  const size_t smem = (size_t)a.graph_smem + (size_t)a.frame_bytes * fpc;
  auto k = backward ? wbp_backward_kernel<G> : wbp_forward_kernel<G>;
  cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int64_t grid = (a.batch + fpc - 1) / fpc;
  k<<<(unsigned)grid, 32 * fpc, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int wbp_state_bytes(const GraphDesc& g, bool backward) { return wbp_frame_bytes(g.N, g.E, backward); }

cudaError_t launch_wbp(const WbpArgs& a, bool backward, int fpc, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  cudaError_t e = a.g.is_qc ? wbp_launch_t<QCGraph>(a, backward, fpc, s) : wbp_launch_t<TabGraph>(a, backward, fpc, s);
  if (e != cudaSuccess || !backward || !a.dw) return e;
  wbp_colsum_kernel<<<(unsigned)std::min<int64_t>((a.T + 255) / 256, 4096), 256, 0, s>>>(a.dw_frames, a.batch, a.T, a.dw);
  return cudaGetLastError();
}

}  // namespace ldpc
