// ci_stats.cu -- counters behind the CI metric's two properties (Sec. 3.A).
//
// For pairs (L, L~) of a variable node's current and precomputed total LLR
// (all-zero codeword sent), D = |p0(L) - p0(L~)| (eq. 8) is binned by
// b = min(floor(D * n_bins), n_bins - 1) and each bin counts
//   [0] decisions correct   (p0(L) >= 1/2, i.e. L >= 0)
//   [1] decisions incorrect (L < 0)
//   [2] incorrect and p0(L~) >= p0(L) (the update moves toward the truth)
//   [3] incorrect and p0(L~) <  p0(L).
// Cumulating bins from the top gives the empirical J(gamma) = [0]/[1] of
// Property 1 and F(gamma) = [2]/[3] of Property 2 at gamma = b / n_bins.
#include <algorithm>

#include "device_math.cuh"

namespace ldpc {

namespace {

__global__ void ci_stats_kernel(const float* La, const float* Lb, int64_t count, int n_bins,
                                unsigned long long* out) {
  extern __shared__ unsigned long long hist[];  // [n_bins][4]
  for (int i = threadIdx.x; i < 4 * n_bins; i += blockDim.x) hist[i] = 0ull;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = La[i], b = Lb[i];
    const float d = ci_fp(a, b);
    const int bin = min((int)floorf(d * (float)n_bins), n_bins - 1);
    const bool wrong = a < 0.0f;
    atomicAdd(&hist[4 * bin + (wrong ? 1 : 0)], 1ull);
    if (wrong) atomicAdd(&hist[4 * bin + (b >= a ? 2 : 3)], 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * n_bins; i += blockDim.x)
    if (hist[i]) atomicAdd(&out[i], hist[i]);
}

}  // namespace

cudaError_t launch_ci_stats(const float* La, const float* Lb, int64_t count, int n_bins, unsigned long long* out,
                            int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * 4 * (size_t)n_bins, s);
  if (e != cudaSuccess || count == 0) return e;
  const int64_t grid = std::min<int64_t>((count + 255) / 256, (int64_t)sms * 8);
  ci_stats_kernel<<<(unsigned)grid, 256, sizeof(unsigned long long) * 4 * (size_t)n_bins, s>>>(La, Lb, count, n_bins, out);
  return cudaGetLastError();
}

}  // namespace ldpc
