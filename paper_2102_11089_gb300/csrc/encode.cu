// encode.cu -- systematic encoder of the lifted codes (random codewords).
//
// Not a step of the paper's decoders: it lets the channel send codewords
// other than the all-zero word.  Codes lifted from a protograph whose parity
// part has the dual-diagonal shape of the IEEE 802.11 / 5G NR core are encoded
// in linear time, Z-parallel over each block column.  With kb info block
// columns, a core of c rows and the blocks B[r][col] (circulant shift, or -1):
//   - within the core rows, parity column kb has shift s in rows 0 and c-1 and
//     shift 0 in a middle row x, and columns kb+k (k = 1..c-1) are a shift-0
//     staircase on rows k-1 and k; extension column kb+c+j is the identity on
//     row c+j alone (extension rows may also read the core columns);
//   - lambda_r = sum over info blocks of row r of the shifted info vectors
//     (block (r, col) with shift s maps vector v to v[(z + s) mod Z]);
//   - the sum of the core rows cancels everything but the middle entry of
//     column kb, so p0 = sum_{r < c} lambda_r; then q_1 = lambda_0 + P^s p0 and
//     q_{r+1} = lambda_r + q_r (+ p0 at r = x) along the staircase;
//   - extension row c+j gives its parity block as the sum of its other blocks.
// One CTA per frame; the codeword is built in shared memory (one byte per bit).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace ldpc {

namespace {

__global__ void __launch_bounds__(256) encode_kernel(const EncArgs a, const uint8_t* __restrict__ info,
                                                     uint8_t* __restrict__ cw_out, int64_t batch) {
  extern __shared__ uint8_t sm[];
  const int Z = a.Z, R = a.R, C = a.C, kb = a.kb, c = a.c;
  const int N = C * Z, K = kb * Z;
  uint8_t* cw = sm;
  uint8_t* lam = sm + ((N + 15) & ~15);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
    for (int i = tid; i < K; i += nt) cw[i] = info[b * K + i] & 1u;
    __syncthreads();
    for (int i = tid; i < c * Z; i += nt) {  // lambda_r of the core rows
      const int r = i / Z, z = i - r * Z;
      uint8_t v = 0;
      for (int col = 0; col < kb; ++col) {
        const int s = a.B[r * C + col];
        if (s >= 0) v ^= cw[col * Z + (z + s) % Z];
      }
      lam[i] = v;
    }
    __syncthreads();
    for (int z = tid; z < Z; z += nt) {  // p0 = sum of the core lambdas
      uint8_t p = 0;
      for (int r = 0; r < c; ++r) p ^= lam[r * Z + z];
      cw[kb * Z + z] = p;
    }
    __syncthreads();
    for (int z = tid; z < Z; z += nt) {  // the staircase, one z per thread
      uint8_t q = lam[z] ^ cw[kb * Z + (z + a.s) % Z];
      cw[(kb + 1) * Z + z] = q;
      for (int r = 1; r + 1 < c; ++r) {
        q ^= lam[r * Z + z] ^ (r == a.x ? cw[kb * Z + z] : 0);
        cw[(kb + 1 + r) * Z + z] = q;
      }
    }
    __syncthreads();
    for (int i = tid; i < (R - c) * Z; i += nt) {  // extension rows
      const int r = c + i / Z, z = i % Z;
      uint8_t v = 0;
      for (int col = 0; col < kb + c; ++col) {
        const int s = a.B[r * C + col];
        if (s >= 0) v ^= cw[col * Z + (z + s) % Z];
      }
      cw[(kb + r) * Z + z] = v;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) cw_out[b * N + i] = cw[i];
    __syncthreads();
  }
}

}  // namespace

bool encode_plan(const int32_t* base, int R, int C, int Z, int K, EncArgs* out) {
  if (Z <= 0 || K % Z != 0 || R * C > kEncMaxBlocks) return false;
  EncArgs a;
  std::memset(&a, 0, sizeof(a));
  a.Z = Z;
  a.R = R;
  a.C = C;
  a.kb = K / Z;
  const int kb = a.kb;
  if (kb <= 0 || C != kb + R) return false;
  auto B = [&](int r, int col) { return base[r * C + col]; };
  // first parity column: its first three blocks are the core's -- shift s in
  // rows 0 and c-1, 0 in a middle row x (extension rows may read it too)
  std::vector<int> rows;
  for (int r = 0; r < R && rows.size() < 3; ++r)
    if (B(r, kb) >= 0) rows.push_back(r);
  if (rows.size() != 3 || rows[0] != 0 || B(0, kb) != B(rows[2], kb) || B(rows[1], kb) != 0) return false;
  a.x = rows[1];
  a.c = rows[2] + 1;
  a.s = B(0, kb);
  const int c = a.c;
  if (c < 3 || c > kEncMaxCore || c > R) return false;
  for (int k = 1; k < c; ++k)  // staircase columns, within the core rows
    for (int r = 0; r < c; ++r) {
      const bool want = r == k - 1 || r == k;
      if ((B(r, kb + k) >= 0) != want || (want && B(r, kb + k) != 0)) return false;
    }
  for (int col = kb + c; col < C; ++col)  // extension columns: identity on their own row
    for (int r = 0; r < R; ++r) {
      const bool want = r == c + (col - kb - c);
      if ((B(r, col) >= 0) != want || (want && B(r, col) != 0)) return false;
    }
  for (int i = 0; i < R * C; ++i) a.B[i] = (int16_t)base[i];
  *out = a;
  return true;
}

cudaError_t launch_encode(const EncArgs& a, const uint8_t* info, uint8_t* cw, int64_t batch, int sms, cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  const size_t smem = (size_t)((a.C * a.Z + 15) & ~15) + (size_t)a.c * a.Z;
  cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>(batch, (int64_t)sms * 8);
  encode_kernel<<<(unsigned)grid, 256, smem, s>>>(a, info, cw, batch);
  return cudaGetLastError();
}

}  // namespace ldpc
