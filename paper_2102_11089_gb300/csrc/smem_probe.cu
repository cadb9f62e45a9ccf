// smem_probe.cu -- ldpc_smem_stream: a shared-memory read stream, the
// denominator of the decoders' roofline (their state lives in shared memory,
// and no vendor figure for its bandwidth is measured on this hardware).
//
// Every CTA fills 32 KB of shared memory, then each warp issues 128-bit loads
// (ld.shared.v4.u32, volatile so none is merged or hoisted) over consecutive
// 16-byte words: a warp instruction reads 512 contiguous bytes, free of bank
// conflicts.  The loaded words are folded into one value per thread and
// written to `sink`, so the loads have a use.  Bytes read = blocks x threads x
// iters x 4 loads x 16 B.
#include "internal.h"
#include "ldpc.h"

namespace {

constexpr int kWords = 2048;  // uint4 words: 32 KB

__global__ void __launch_bounds__(1024) smem_stream_kernel(int iters, uint32_t* __restrict__ sink) {
  __shared__ __align__(16) uint4 buf[kWords];
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    buf[i] = make_uint4((uint32_t)i, (uint32_t)i * 3u, (uint32_t)i ^ 5u, (uint32_t)i + 7u);
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
  uint32_t acc = 0;
  uint32_t idx = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t a, b, c, d;
      const uint32_t addr = base + (((idx + (uint32_t)k * 512u) & (kWords - 1)) << 4);
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "r"(addr));
      acc ^= a ^ b ^ c ^ d;
    }
    idx += 32u;
  }
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

extern "C" ldpc_status_t ldpc_smem_stream(int32_t blocks, int32_t threads, int32_t iters, uint32_t* sink,
                                          int64_t* bytes, void* cuda_stream) {
  if (blocks <= 0 || threads <= 0 || threads > 1024 || (threads & 31) != 0 || iters <= 0 || !sink) {
    ldpc::set_error_detail("blocks > 0, threads a multiple of 32 up to 1024, iters > 0 and sink are required");
    return LDPC_ERR_INVALID_ARG;
  }
  smem_stream_kernel<<<(unsigned)blocks, (unsigned)threads, 0, (cudaStream_t)cuda_stream>>>(iters, sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ldpc::set_error_detail(std::string("smem stream launch: ") + cudaGetErrorString(e));
    return LDPC_ERR_CUDA;
  }
  if (bytes) *bytes = (int64_t)blocks * threads * (int64_t)iters * 4 * 16;
  return LDPC_OK;
}
