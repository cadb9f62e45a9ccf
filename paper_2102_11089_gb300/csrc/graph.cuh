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
//            hundred 16-byte entries in shared memory, one load per edge).
//            Check m = r Z + z has its k-th edge (block (r, c_k), shift s_k) at
//            edge id rowbase[r] + z dc_r + k and variable c_k Z + (z + s_k) mod Z;
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
  const int4* rowinfo;  // R : {first edge id, first rowblk entry, d_c, r Z}
  const int4* colinfo;  // C : {first colblk entry, d_v, c Z, 0}
  const int4* colblk;   // nnz, by column then row: {s, r Z, rowbase[r] + k, d_c(r)}
  const int2* rowblk;   // nnz, by row then column: {c Z, s}
  int R, Z, E;
  uint32_t zmul, zshift;  // n / Z == __umulhi(n, zmul) >> zshift for n < R Z and C Z

  __device__ __forceinline__ int divZ(int n) const { return (int)(__umulhi((uint32_t)n, zmul) >> zshift); }

  struct V {
    int z, j0, d;
  };
  struct C {
    int b, d, z, i0;
  };
  __device__ __forceinline__ V vn(int n) const {
    const int4 ci = colinfo[divZ(n)];
    return {n - ci.z, ci.x, ci.y};
  }
  // k-th edge of variable c Z + z in block (r, c) with shift s: check r Z + (z - s) mod Z,
  // edge id rowbase[r] + ((z - s) mod Z) d_c(r) + k
  __device__ __forceinline__ void vedge(const V& v, int k, int& e, int& m) const {
    const int4 b = colblk[v.j0 + k];
    int zz = v.z - b.x;
    zz += zz < 0 ? Z : 0;
    m = b.y + zz;
    e = b.z + zz * b.w;
  }
  __device__ __forceinline__ C cn(int m) const {
    const int4 ri = rowinfo[divZ(m)];
    const int z = m - ri.w;
    return {ri.x + z * ri.z, ri.z, z, ri.y};
  }
  // k-th edge of check r Z + z, block (r, c_k) with shift s_k: variable c_k Z + (z + s_k) mod Z
  __device__ __forceinline__ int cvn(const C& c, int k) const {
    const int2 b = rowblk[c.i0 + k];
    int zz = c.z + b.y;
    zz -= zz >= Z ? Z : 0;
    return b.x + zz;
  }
  __device__ __forceinline__ int ecn(int e) const {
    int lo = 0, hi = R;  // rowinfo[lo].x <= e < rowinfo[hi].x (rowinfo[R].x = E)
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (rowinfo[mid].x <= e) lo = mid;
      else hi = mid;
    }
    const int4 ri = rowinfo[lo];
    return ri.w + (e - ri.x) / ri.z;
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
    g.E = d.E;
    g.zmul = d.qc_zmul;
    g.zshift = d.qc_zshift;
    g.rowinfo = (const int4*)p; p += 4 * d.qc_R;
    g.colinfo = (const int4*)p; p += 4 * d.qc_C;
    g.colblk = (const int4*)p; p += 4 * d.qc_nnz;
    g.rowblk = (const int2*)p;
    return g;
  }
};

}  // namespace ldpc
