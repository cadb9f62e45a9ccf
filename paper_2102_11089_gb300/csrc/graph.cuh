// graph.cuh -- Tanner-graph access for the decode kernels.
//
// Two views of the same canonical graph (edge ids in (check, variable) order):
//
//  TabGraph  CSR/CSC tables (check pointers, edge->variable, edge->check,
//            variable pointers, variable->edges).  Staged into shared memory
//            when small, else read from global memory.
//
//  QCGraph   quasi-cyclic codes lifted from a protograph: every neighbour and
//            edge id is computed from the protograph's block list (a few
//            hundred entries in shared memory).  Check m = r Z + z has its
//            k-th edge (block (r, c_k), shift s_k) at edge id
//            rowbase[r] + z dc_r + k and variable c_k Z + (z + s_k) mod Z;
//            variable n = c Z + z meets check r Z + (z - s) mod Z of each block
//            (r, c) of column c.
//
// Both expose cursors: vn(n) -> edges of variable n (ascending check),
// cn(m) -> contiguous edge range of check m with its variables.
#pragma once

#include <cstdint>

#include "internal.h"

namespace ldpc {

struct TabGraph {
  const int32_t* cn_ptr;
  const int32_t* e_vn;
  const int32_t* e_cn;
  const int32_t* vn_ptr;
  const int32_t* vn_e;

  struct V {
    int b, d;
  };
  struct C {
    int b, d;
  };
  __device__ __forceinline__ V vn(int n) const {
    const int b = vn_ptr[n];
    return {b, vn_ptr[n + 1] - b};
  }
  __device__ __forceinline__ void vedge(const V& v, int k, int& e, int& m) const {
    e = vn_e[v.b + k];
    m = e_cn[e];
  }
  __device__ __forceinline__ C cn(int m) const {
    const int b = cn_ptr[m];
    return {b, cn_ptr[m + 1] - b};
  }
  __device__ __forceinline__ int cvn(const C& c, int k) const { return e_vn[c.b + k]; }
  __device__ __forceinline__ int ecn(int e) const { return e_cn[e]; }
  __device__ __forceinline__ int evn(int e) const { return e_vn[e]; }
};

struct QCGraph {
  const int32_t* rowbase;   // R+1 : first edge id of block row r
  const int32_t* rowfirst;  // R+1 : first entry of row r in rowblk
  const uint32_t* rowblk;   // nnz : (c << 16) | s, ascending c
  const int32_t* colfirst;  // C+1 : first entry of column c in colblk
  const uint32_t* colblk;   // nnz : (r << 24) | (k << 16) | s, ascending r
  int R, Z;
  uint32_t zmul, zshift;    // n / Z == __umulhi(n, zmul) >> zshift for n < R Z and C Z

  __device__ __forceinline__ int divZ(int n) const { return (int)(__umulhi((uint32_t)n, zmul) >> zshift); }

  struct V {
    int z, j0, d;
  };
  struct C {
    int b, d, z, i0;
  };
  __device__ __forceinline__ V vn(int n) const {
    const int c = divZ(n);
    const int j0 = colfirst[c];
    return {n - c * Z, j0, colfirst[c + 1] - j0};
  }
  __device__ __forceinline__ void vedge(const V& v, int k, int& e, int& m) const {
    const uint32_t blk = colblk[v.j0 + k];
    const int r = (int)(blk >> 24), kk = (int)((blk >> 16) & 255u), s = (int)(blk & 0xffffu);
    int zz = v.z - s;
    zz += zz < 0 ? Z : 0;
    m = r * Z + zz;
    e = rowbase[r] + zz * (rowfirst[r + 1] - rowfirst[r]) + kk;
  }
  __device__ __forceinline__ C cn(int m) const {
    const int r = divZ(m);
    const int z = m - r * Z;
    const int i0 = rowfirst[r], dc = rowfirst[r + 1] - i0;
    return {rowbase[r] + z * dc, dc, z, i0};
  }
  __device__ __forceinline__ int cvn(const C& c, int k) const {
    const uint32_t blk = rowblk[c.i0 + k];
    int zz = c.z + (int)(blk & 0xffffu);
    zz -= zz >= Z ? Z : 0;
    return (int)(blk >> 16) * Z + zz;
  }
  __device__ __forceinline__ int ecn(int e) const {
    int lo = 0, hi = R;  // rowbase[lo] <= e < rowbase[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (rowbase[mid] <= e) lo = mid;
      else hi = mid;
    }
    const int dc = rowfirst[lo + 1] - rowfirst[lo];
    return lo * Z + (e - rowbase[lo]) / dc;
  }
  __device__ __forceinline__ int evn(int e) const {
    const int m = ecn(e);
    const C c = cn(m);
    return cvn(c, e - c.b);
  }
};

// Copy the graph tables a kernel reads into shared memory (all threads of the
// CTA call this; ends with __syncthreads()).  `dst` must hold desc.smem_bytes.
__device__ __forceinline__ void stage_words(int32_t* dst, const int32_t* src, int words) {
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

template <class G>
struct GraphStage;

template <>
struct GraphStage<TabGraph> {
  // tables staged when desc.tab_in_smem, else read from global memory
  static __device__ __forceinline__ TabGraph make(const GraphDesc& d, int32_t* smem) {
    TabGraph g;
    if (d.tab_in_smem) {
      stage_words(smem, d.tab, d.tab_words);
      __syncthreads();
      const int32_t* p = smem;
      g.cn_ptr = p; p += d.M + 1;
      g.e_vn = p; p += d.E;
      g.e_cn = p; p += d.E;
      g.vn_ptr = p; p += d.N + 1;
      g.vn_e = p;
    } else {
      const int32_t* p = d.tab;
      g.cn_ptr = p; p += d.M + 1;
      g.e_vn = p; p += d.E;
      g.e_cn = p; p += d.E;
      g.vn_ptr = p; p += d.N + 1;
      g.vn_e = p;
    }
    return g;
  }
};

template <>
struct GraphStage<QCGraph> {
  static __device__ __forceinline__ QCGraph make(const GraphDesc& d, int32_t* smem) {
    stage_words(smem, d.qc, d.qc_words);
    __syncthreads();
    QCGraph g;
    const int32_t* p = smem;
    g.R = d.qc_R;
    g.Z = d.qc_Z;
    g.zmul = d.qc_zmul;
    g.zshift = d.qc_zshift;
    g.rowbase = p; p += d.qc_R + 1;
    g.rowfirst = p; p += d.qc_R + 1;
    g.colfirst = p; p += d.qc_C + 1;
    g.rowblk = (const uint32_t*)p; p += d.qc_nnz;
    g.colblk = (const uint32_t*)p;
    return g;
  }
};

}  // namespace ldpc
