// decode_flood.cu -- flooding BP (Sec. 1), one frame per CTA.
//
// One iteration computes every V2C message from the previous C2V messages
// (eq. 1, written as L_n - L^C_{m->n}), then every C2V message (eq. 2 or
// min-sum) in parallel, then the total LLRs (eq. 3); it propagates E messages
// (the iteration unit of Sec. 2.A).  Messages, LLRs and the per-edge scratch of
// encoded V2C values sit in shared memory; threads stride over edges, then
// variable nodes, then checks (syndrome).
#include "device_math.cuh"

namespace ldpc {

namespace {

__device__ __forceinline__ float flood_c2v(const float* S, int e, int c0, int c1, float clip) {
  float sum = 0.0f;
  unsigned neg = 0;
  for (int k = c0; k < c1; ++k) {
    if (k == e) continue;
    const float v = S[k];
    sum += fabsf(v);
    neg ^= (__float_as_uint(v) >> 31);
  }
  return combine_fp(sum, neg, clip);
}

__device__ __forceinline__ int8_t flood_c2v(const int8_t* S, int e, int c0, int c1, float) {
  int mag = 31;
  unsigned neg = 0;
  for (int k = c0; k < c1; ++k) {
    if (k == e) continue;
    const int v = S[k];
    neg ^= (v < 0);
    mag = min(mag, abs(v));
  }
  return (int8_t)(neg ? -mag : mag);
}

template <int A>
__global__ void __launch_bounds__(512) flood_decode_kernel(const DecodeArgs a) {
  using M_ = typename Arith<A>::msg;
  using L_ = typename Arith<A>::llr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t b = blockIdx.x;
  const DevCode& g = a.g;
  const FloodLayout ly = flood_layout(A, g.N, g.E);
  M_* C = (M_*)(smem_raw + ly.C);
  M_* S = (M_*)(smem_raw + ly.S);
  L_* lam = (L_*)(smem_raw + ly.lam);
  L_* L = (L_*)(smem_raw + ly.L);
  const int N = g.N, E = g.E, M = g.M;
  const int tid = threadIdx.x, nt = blockDim.x;
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
      const int c0 = __ldg(g.cn_ptr + m), c1 = __ldg(g.cn_ptr + m + 1);
      unsigned p = 0;
      for (int e = c0; e < c1; ++e) p ^= (L[__ldg(g.e_vn + e)] < (L_)0);
      any |= (int)p;
    }
    return __syncthreads_or(any);
  };

  int64_t count = 0;
  bool ok = a.check_interval > 0 && !syndrome_nonzero();
  while (!ok && count + E <= a.max_updates) {
    const int64_t before = count;
    for (int e = tid; e < E; e += nt) {  // V2C from the previous C2V (eq. 1)
      const int j = __ldg(g.e_vn + e);
      if (A == kFP32) ((float*)S)[e] = encode_fp((float)L[j] - (float)C[e], clip);
      else ((int8_t*)S)[e] = encode_int((int)L[j] - (int)C[e]);
    }
    __syncthreads();
    for (int e = tid; e < E; e += nt) {  // every C2V (eq. 2 / min-sum)
      const int m = __ldg(g.e_cn + e);
      C[e] = flood_c2v((const M_*)S, e, __ldg(g.cn_ptr + m), __ldg(g.cn_ptr + m + 1), clip);
    }
    __syncthreads();
    for (int n = tid; n < N; n += nt) {  // total LLR (eq. 3)
      const int v0 = __ldg(g.vn_ptr + n), v1 = __ldg(g.vn_ptr + n + 1);
      L_ acc = lam[n];
      for (int k = v0; k < v1; ++k) acc = (L_)(acc + C[__ldg(g.vn_e + k)]);
      L[n] = acc;
    }
    __syncthreads();
    count += E;
    if (a.check_interval > 0 && (count / a.check_interval) > (before / a.check_interval))
      ok = !syndrome_nonzero();
  }
  const int conv = !syndrome_nonzero();
  for (int n = tid; n < N; n += nt) {
    if (a.hard) a.hard[b * N + n] = (uint8_t)(L[n] < (L_)0);
    if (a.llr_out) a.llr_out[b * N + n] = (float)L[n];
  }
  if (tid == 0) {
    if (a.updates) a.updates[b] = count;
    if (a.converged) a.converged[b] = (uint8_t)conv;
  }
}

}  // namespace

size_t flood_smem_per_frame(int arith, const DevCode& g) {
  return (size_t)flood_layout(arith, g.N, g.E).total;
}

cudaError_t launch_flood(const DecodeArgs& a, int arith, cudaStream_t s) {
  if (a.batch == 0) return cudaSuccess;
  const size_t smem = (size_t)a.smem_per_frame;
  const int threads = a.g.E >= 4096 ? 512 : (a.g.E >= 1024 ? 256 : 128);
  cudaError_t err;
  if (arith == kFP32) {
    err = cudaFuncSetAttribute(flood_decode_kernel<kFP32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err != cudaSuccess) return err;
    flood_decode_kernel<kFP32><<<(unsigned)a.batch, threads, smem, s>>>(a);
  } else {
    err = cudaFuncSetAttribute(flood_decode_kernel<kINT6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err != cudaSuccess) return err;
    flood_decode_kernel<kINT6><<<(unsigned)a.batch, threads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace ldpc
