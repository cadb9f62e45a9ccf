// channel.cu -- BPSK / AWGN channel LLRs (Sec. 2.A and Sec. 5).
//
// Codeword bits c (all-zero unless given): x = 1 - 2c, y = x + sigma w, N0/2 = sigma^2 with
// sigma^2 = 1 / (2 R 10^(EbN0/10)), LLR lambda = 2 y / sigma^2; punctured VNs
// are not transmitted and get lambda = 0.  Gaussian samples come from
// Box-Muller on Philox4x32-10 words (Salmon et al., SC'11): variable nodes
// 4k..4k+3 of frame f use one Philox block with counter (k, 0, f) and key =
// seed; (w0, w1) and (w2, w3) each give a uniform pair (u_a, u_b) with
// u = (x + 1/2) 2^-32, r = sqrt(-2 ln u_a), and the pair r cos(2 pi u_b),
// r sin(2 pi u_b).  One thread per Philox block, grid-stride; the 6-bit
// quantiser clamp(rint(lambda / step), -31, 31) runs in the same pass.
#include "internal.h"
#include "philox.cuh"

namespace ldpc {

namespace {

// -ln(u) * 2 with u = (x + 1/2) 2^-32, accurate near u = 1 as well
__device__ __forceinline__ float minus2_log_u(uint32_t x) {
  if (x < 0x80000000u) return -2.0f * logf(((float)x + 0.5f) * 2.3283064365386963e-10f);
  const float w = ((float)(~x) + 0.5f) * 2.3283064365386963e-10f;  // 1 - u
  return -2.0f * log1pf(-w);
}

__global__ void __launch_bounds__(256) awgn_kernel(int N, const uint8_t* __restrict__ punct,
                                                   const uint8_t* __restrict__ cw, float rate, const float* __restrict__ ebn0,
                                                   int64_t batch, uint64_t seed, uint64_t frame_offset,
                                                   float* __restrict__ llr, int8_t* __restrict__ qllr,
                                                   float q_step) {
  const int blocks = (N + 3) / 4;
  const int64_t total = batch * (int64_t)blocks;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / blocks;
    const int k = (int)(t - b * blocks);
    const uint64_t f = frame_offset + (uint64_t)b;
    uint32_t c[4] = {(uint32_t)k, 0u, (uint32_t)f, (uint32_t)(f >> 32)};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const float eb = ebn0[b];
    const float sigma2 = 1.0f / (2.0f * rate * exp10f(0.1f * eb));
    const float sigma = sqrtf(sigma2);
    const float scale = 2.0f / sigma2;
    float z[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float r = sqrtf(minus2_log_u(c[2 * p]));
      float sn, cs;
      sincospif(2.0f * (((float)c[2 * p + 1] + 0.5f) * 2.3283064365386963e-10f), &sn, &cs);
      z[2 * p] = r * cs;
      z[2 * p + 1] = r * sn;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = 4 * k + i;
      if (n >= N) break;
      const bool pn = punct != nullptr && punct[n];
      const float x = (cw != nullptr && (cw[b * N + n] & 1u)) ? -1.0f : 1.0f;
      const float lam = pn ? 0.0f : scale * (x + sigma * z[i]);
      llr[b * N + n] = lam;
      if (qllr) {
        const float q = fminf(31.0f, fmaxf(-31.0f, rintf(lam / q_step)));
        qllr[b * N + n] = (int8_t)q;
      }
    }
  }
}

}  // namespace

cudaError_t launch_channel(int N, const uint8_t* punct, const uint8_t* codewords, float rate, const float* ebn0,
                           int64_t batch, uint64_t seed, uint64_t frame_offset, float* llr, int8_t* qllr, float q_step,
                           cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  const int64_t work = batch * (int64_t)((N + 3) / 4);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (work + 255) / 256;
  const int grid = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  awgn_kernel<<<grid, 256, 0, s>>>(N, punct, codewords, rate, ebn0, batch, seed, frame_offset, llr, qllr, q_step);
  return cudaGetLastError();
}

}  // namespace ldpc
