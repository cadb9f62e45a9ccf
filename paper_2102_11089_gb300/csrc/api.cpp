// api.cpp -- the C ABI (include/ldpc.h): code handles, validation, dispatch.
#include "ldpc.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace {

thread_local std::string g_detail;

ldpc_status_t fail(ldpc_status_t st, const std::string& why) {
  g_detail = why;
  return st;
}

ldpc_status_t cuda_fail(cudaError_t e, const char* where) {
  return fail(LDPC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

struct DevCopy {
  int32_t* buf = nullptr;  // tab blob, then the QC blob (if any)
  uint8_t* punct = nullptr;
  ldpc::GraphDesc g{};
};

std::mutex g_status_mu;
std::map<int, uint32_t*> g_status;  // per-device status word

ldpc_status_t device_status_word(int dev, uint32_t** out) {
  std::lock_guard<std::mutex> lk(g_status_mu);
  auto it = g_status.find(dev);
  if (it != g_status.end()) {
    *out = it->second;
    return LDPC_OK;
  }
  uint32_t* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(status)");
  e = cudaMemset(p, 0, sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
  g_status[dev] = p;
  *out = p;
  return LDPC_OK;
}

}  // namespace

struct ldpc_code {
  int32_t M = 0, N = 0, E = 0, K = 0, Z = 0;
  int32_t dv_max = 0, dc_max = 0, maxr = 0, n_punct = 0;
  std::vector<int32_t> cn_ptr, e_vn, e_cn, vn_ptr, vn_e;
  std::vector<uint8_t> punct;
  // protograph view (codes from ldpc_code_build_qc): see graph.cuh
  std::vector<int32_t> qc;  // rowbase | rowfirst | colfirst | rowblk | colblk
  std::vector<int32_t> base;  // protograph shifts (codes from ldpc_code_build_qc)
  int32_t base_rows = 0, base_cols = 0;
  int32_t qc_R = 0, qc_C = 0, qc_nnz = 0;
  uint32_t qc_zmul = 0, qc_zshift = 0;
  std::mutex mu;
  std::map<int, DevCopy> dev;
};

namespace {

ldpc_status_t build_code(const int32_t* chk, const int32_t* var, int64_t n_edges, int32_t M, int32_t N,
                         const uint8_t* punct, int32_t k_info, int32_t Z, ldpc_code_t** out) {
  if (!out) return fail(LDPC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!chk || !var) return fail(LDPC_ERR_INVALID_ARG, "edge arrays are NULL");
  if (n_edges <= 0 || M <= 0 || N <= 0) return fail(LDPC_ERR_INVALID_ARG, "sizes must be positive");
  if (n_edges > (int64_t)M * (int64_t)N) return fail(LDPC_ERR_DUPLICATE_EDGE, "more edges than cells of H");
  if (n_edges > 0x7fffffff) return fail(LDPC_ERR_UNSUPPORTED, "more than 2^31-1 edges");
  if (k_info <= 0) return fail(LDPC_ERR_INVALID_ARG, "k_info must be positive");
  std::vector<int64_t> key;
  try {
    key.resize((size_t)n_edges);
  } catch (const std::bad_alloc&) {
    return fail(LDPC_ERR_NOMEM, "host allocation");
  }
  for (int64_t e = 0; e < n_edges; ++e) {
    if (chk[e] < 0 || chk[e] >= M || var[e] < 0 || var[e] >= N)
      return fail(LDPC_ERR_INDEX_RANGE, "edge " + std::to_string(e) + " out of range");
    key[(size_t)e] = (int64_t)chk[e] * N + var[e];
  }
  std::sort(key.begin(), key.end());
  for (size_t e = 1; e < key.size(); ++e)
    if (key[e] == key[e - 1])
      return fail(LDPC_ERR_DUPLICATE_EDGE, "edge (" + std::to_string(key[e] / N) + ", " +
                                               std::to_string(key[e] % N) + ") listed twice");
  ldpc_code_t* c = new (std::nothrow) ldpc_code_t();
  if (!c) return fail(LDPC_ERR_NOMEM, "host allocation");
  const int32_t E = (int32_t)n_edges;
  c->M = M; c->N = N; c->E = E; c->K = k_info; c->Z = Z;
  try {
    c->cn_ptr.assign((size_t)M + 1, 0);
    c->vn_ptr.assign((size_t)N + 1, 0);
    c->e_vn.resize(E);
    c->e_cn.resize(E);
    c->vn_e.resize(E);
    c->punct.assign((size_t)N, 0);
  } catch (const std::bad_alloc&) {
    delete c;
    return fail(LDPC_ERR_NOMEM, "host allocation");
  }
  for (int32_t e = 0; e < E; ++e) {
    const int32_t m = (int32_t)(key[e] / N), n = (int32_t)(key[e] % N);
    c->e_cn[e] = m;
    c->e_vn[e] = n;
    c->cn_ptr[m + 1]++;
    c->vn_ptr[n + 1]++;
  }
  for (int32_t m = 0; m < M; ++m) {
    if (c->cn_ptr[m + 1] == 0) {
      delete c;
      return fail(LDPC_ERR_EMPTY_NODE, "check " + std::to_string(m) + " has no edge");
    }
    c->dc_max = std::max(c->dc_max, c->cn_ptr[m + 1]);
    c->cn_ptr[m + 1] += c->cn_ptr[m];
  }
  for (int32_t n = 0; n < N; ++n) {
    if (c->vn_ptr[n + 1] == 0) {
      delete c;
      return fail(LDPC_ERR_EMPTY_NODE, "variable " + std::to_string(n) + " has no edge");
    }
    c->dv_max = std::max(c->dv_max, c->vn_ptr[n + 1]);
    c->vn_ptr[n + 1] += c->vn_ptr[n];
  }
  std::vector<int32_t> fill((size_t)N, 0);
  for (int32_t e = 0; e < E; ++e) {  // ascending e = ascending check within a VN
    const int32_t n = c->e_vn[e];
    c->vn_e[c->vn_ptr[n] + fill[n]++] = e;
  }
  for (int32_t n = 0; n < N; ++n) {
    int32_t r = 0;
    for (int32_t k = c->vn_ptr[n]; k < c->vn_ptr[n + 1]; ++k) {
      const int32_t m = c->e_cn[c->vn_e[k]];
      r += c->cn_ptr[m + 1] - c->cn_ptr[m];
    }
    c->maxr = std::max(c->maxr, r);
    if (punct && punct[n]) {
      c->punct[n] = 1;
      c->n_punct++;
    }
  }
  *out = c;
  return LDPC_OK;
}

ldpc_status_t ensure_device(ldpc_code_t* c, const ldpc::GraphDesc** out, const uint8_t** punct) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->dev.find(dev);
  if (it == c->dev.end()) {
    DevCopy d;
    const size_t tab_words = (size_t)(c->M + 1) + 3 * (size_t)c->E + (size_t)(c->N + 1);
    const size_t words = tab_words + c->qc.size();
    e = cudaMalloc(&d.buf, words * sizeof(int32_t));
    if (e != cudaSuccess) return fail(LDPC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMalloc(&d.punct, (size_t)c->N);
    if (e != cudaSuccess) {
      cudaFree(d.buf);
      return fail(LDPC_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    std::vector<int32_t> host;
    host.reserve(words);
    host.insert(host.end(), c->cn_ptr.begin(), c->cn_ptr.end());
    host.insert(host.end(), c->e_vn.begin(), c->e_vn.end());
    host.insert(host.end(), c->e_cn.begin(), c->e_cn.end());
    host.insert(host.end(), c->vn_ptr.begin(), c->vn_ptr.end());
    host.insert(host.end(), c->vn_e.begin(), c->vn_e.end());
    host.insert(host.end(), c->qc.begin(), c->qc.end());
    e = cudaMemcpy(d.buf, host.data(), words * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.punct, c->punct.data(), (size_t)c->N, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d.buf);
      cudaFree(d.punct);
      return cuda_fail(e, "cudaMemcpy(code)");
    }
    ldpc::GraphDesc& g = d.g;
    std::memset(&g, 0, sizeof(g));
    g.M = c->M; g.N = c->N; g.E = c->E;
    g.dv_max = c->dv_max; g.dc_max = c->dc_max; g.maxr = c->maxr;
    g.tab = d.buf;
    g.tab_words = (int32_t)tab_words;
    g.tab_in_smem = tab_words * 4 <= 32 * 1024;
    if (!c->qc.empty()) {
      g.is_qc = 1;
      g.qc = d.buf + tab_words;
      g.qc_words = (int32_t)c->qc.size();
      g.qc_R = c->qc_R; g.qc_C = c->qc_C; g.qc_Z = c->Z; g.qc_nnz = c->qc_nnz;
      g.qc_zmul = c->qc_zmul; g.qc_zshift = c->qc_zshift;
    }
    it = c->dev.emplace(dev, d).first;
  }
  *out = &it->second.g;
  if (punct) *punct = it->second.punct;
  return LDPC_OK;
}

// Protograph view of a lifted code (layout in graph.cuh), kept only when it
// reproduces the CSR maps exactly and fits the packed fields.
void build_qc_view(ldpc_code_t* c, const int32_t* base, int32_t R, int32_t Cc, int32_t Z) {
  c->qc.clear();
  if (Z <= 0) return;
  struct Blk { int32_t r, col, s, k; };
  std::vector<int32_t> rowbase(R + 1, 0), rowfirst(R + 1, 0), dcr(R, 0), colfirst(Cc + 1, 0), dvc(Cc, 0);
  std::vector<Blk> rows, cols;
  std::vector<int32_t> kpos((size_t)R * Cc, -1);
  for (int32_t r = 0; r < R; ++r) {
    rowfirst[r] = (int32_t)rows.size();
    int32_t k = 0;
    for (int32_t col = 0; col < Cc; ++col) {
      const int32_t sft = base[(int64_t)r * Cc + col];
      if (sft < 0) continue;
      rows.push_back({r, col, sft, k});
      kpos[(size_t)r * Cc + col] = k++;
    }
    dcr[r] = k;
    if ((int64_t)rowbase[r] + (int64_t)k * Z > 0x7fffffff) return;
    rowbase[r + 1] = rowbase[r] + k * Z;
  }
  rowfirst[R] = (int32_t)rows.size();
  for (int32_t col = 0; col < Cc; ++col) {
    colfirst[col] = (int32_t)cols.size();
    for (int32_t r = 0; r < R; ++r) {
      const int32_t sft = base[(int64_t)r * Cc + col];
      if (sft >= 0) cols.push_back({r, col, sft, kpos[(size_t)r * Cc + col]});
    }
    dvc[col] = (int32_t)cols.size() - colfirst[col];
  }
  colfirst[Cc] = (int32_t)cols.size();
  // n / Z == umulhi(n, mul) >> shift for every n < max(R, C) Z
  const uint32_t limit = (uint32_t)std::max(R, Cc) * (uint32_t)Z;
  uint32_t mul = 0, shift = 0;
  bool found = false;
  for (uint32_t sh = 0; sh < 32 && !found; ++sh) {
    const unsigned __int128 num = ((unsigned __int128)1) << (32 + sh);
    const unsigned __int128 m = (num + Z - 1) / Z;
    if (m >> 32) continue;
    bool ok = true;
    for (uint32_t n = 0; n < limit && ok; ++n)
      ok = (uint32_t)((((uint64_t)n * (uint64_t)m) >> 32) >> sh) == n / (uint32_t)Z;
    if (ok) {
      mul = (uint32_t)m;
      shift = sh;
      found = true;
    }
  }
  if (!found) return;
  // self-check with the kernels' formulas: the view must give the CSR ids and neighbours
  for (int32_t m = 0; m < c->M; ++m) {
    const int32_t r = m / Z, z = m - r * Z, dc = dcr[r];
    const int32_t b = rowbase[r] + z * dc;
    if (c->cn_ptr[m] != b || c->cn_ptr[m + 1] - c->cn_ptr[m] != dc) return;
    for (int32_t k = 0; k < dc; ++k) {
      const Blk& bb = rows[rowfirst[r] + k];
      int32_t zz = z + bb.s;
      zz -= zz >= Z ? Z : 0;
      if (zz < 0 || zz >= Z || c->e_vn[b + k] != bb.col * Z + zz) return;
    }
  }
  for (int32_t n = 0; n < c->N; ++n) {
    const int32_t col = n / Z, z = n - col * Z;
    if (c->vn_ptr[n + 1] - c->vn_ptr[n] != dvc[col]) return;
    for (int32_t k = 0; k < dvc[col]; ++k) {
      const Blk& bb = cols[colfirst[col] + k];
      int32_t zz = z - bb.s;
      zz += zz < 0 ? Z : 0;
      if (zz < 0 || zz >= Z) return;
      const int32_t e = rowbase[bb.r] + bb.k + zz * dcr[bb.r];
      if (c->vn_e[c->vn_ptr[n] + k] != e || c->e_cn[e] != bb.r * Z + zz) return;
    }
  }
  std::vector<int32_t>& q = c->qc;
  for (int32_t r = 0; r < R; ++r) q.insert(q.end(), {rowbase[r], rowfirst[r], dcr[r], r * Z});
  for (int32_t col = 0; col < Cc; ++col) q.insert(q.end(), {colfirst[col], dvc[col], col * Z, 0});
  for (const Blk& bb : cols) q.insert(q.end(), {bb.s, bb.r * Z, rowbase[bb.r] + bb.k, dcr[bb.r]});
  for (const Blk& bb : rows) q.insert(q.end(), {bb.col * Z, bb.s});
  c->qc_R = R;
  c->qc_C = Cc;
  c->qc_nnz = (int32_t)rows.size();
  c->qc_zmul = mul;
  c->qc_zshift = shift;
}

}  // namespace

namespace ldpc {

// Read-only host view of a code handle, for entry points that keep the graph in
// memory they manage themselves.
bool code_host_view(const void* code, CodeHostView* out) {
  const ldpc_code_t* c = (const ldpc_code_t*)code;
  if (!c || !out) return false;
  out->M = c->M; out->N = c->N; out->E = c->E; out->K = c->K; out->Z = c->Z;
  out->dv_max = c->dv_max; out->dc_max = c->dc_max; out->maxr = c->maxr;
  // the CSR arrays are separate vectors; callers copy them one by one
  out->tab = nullptr;
  out->tab_words = (c->M + 1) + 3 * c->E + (c->N + 1);
  out->qc = c->qc.empty() ? nullptr : c->qc.data();
  out->qc_words = (int32_t)c->qc.size();
  out->qc_R = c->qc_R; out->qc_C = c->qc_C; out->qc_nnz = c->qc_nnz;
  out->qc_zmul = c->qc_zmul; out->qc_zshift = c->qc_zshift;
  return true;
}

void set_error_detail(const std::string& why) { g_detail = why; }

// The five CSR arrays of a code in the order of GraphDesc::tab.
bool code_host_tab(const void* code, const int32_t* parts[5], int32_t sizes[5]) {
  const ldpc_code_t* c = (const ldpc_code_t*)code;
  if (!c) return false;
  parts[0] = c->cn_ptr.data(); sizes[0] = c->M + 1;
  parts[1] = c->e_vn.data(); sizes[1] = c->E;
  parts[2] = c->e_cn.data(); sizes[2] = c->E;
  parts[3] = c->vn_ptr.data(); sizes[3] = c->N + 1;
  parts[4] = c->vn_e.data(); sizes[4] = c->E;
  return true;
}

}  // namespace ldpc

namespace {

int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}

}  // namespace

extern "C" {

const char* ldpc_status_string(ldpc_status_t s) {
  switch (s) {
    case LDPC_OK: return "LDPC_OK";
    case LDPC_ERR_INVALID_ARG: return "LDPC_ERR_INVALID_ARG";
    case LDPC_ERR_DUPLICATE_EDGE: return "LDPC_ERR_DUPLICATE_EDGE";
    case LDPC_ERR_INDEX_RANGE: return "LDPC_ERR_INDEX_RANGE";
    case LDPC_ERR_EMPTY_NODE: return "LDPC_ERR_EMPTY_NODE";
    case LDPC_ERR_UNSUPPORTED: return "LDPC_ERR_UNSUPPORTED";
    case LDPC_ERR_CUDA: return "LDPC_ERR_CUDA";
    case LDPC_ERR_NOMEM: return "LDPC_ERR_NOMEM";
    case LDPC_ERR_TIMEOUT: return "LDPC_ERR_TIMEOUT";
    case LDPC_ERR_NONFINITE_LLR: return "LDPC_ERR_NONFINITE_LLR";
    default: return "LDPC_ERR_UNKNOWN";
  }
}

const char* ldpc_last_error_detail(void) { return g_detail.c_str(); }

ldpc_status_t ldpc_default_params(ldpc_decode_params_t* p) {
  if (!p) return fail(LDPC_ERR_INVALID_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->schedule = LDPC_LMD_CIRBP;
  p->arith = LDPC_FP32_SUMPRODUCT;
  p->gamma = 0.1;
  p->n_p = 16;
  p->n_g = 16;
  p->max_updates = 0;
  p->check_interval = 1;
  p->llr_clip = 25.0f;
  p->q_step = 0.5f;
  p->form = LDPC_FORM_AUTO;
  return LDPC_OK;
}

ldpc_status_t ldpc_code_create(const int32_t* check_idx, const int32_t* var_idx, int64_t n_edges,
                               int32_t n_checks, int32_t n_vars, const uint8_t* punctured, int32_t k_info,
                               ldpc_code_t** out) {
  return build_code(check_idx, var_idx, n_edges, n_checks, n_vars, punctured, k_info, 0, out);
}

ldpc_status_t ldpc_code_build_qc(const int32_t* base, int32_t rows, int32_t cols, int32_t Z,
                                 const uint8_t* punct_cols, int32_t k_info, ldpc_code_t** out) {
  if (!out) return fail(LDPC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!base || rows <= 0 || cols <= 0 || Z <= 0) return fail(LDPC_ERR_INVALID_ARG, "bad protograph");
  if ((int64_t)rows * Z > 0x7fffffff || (int64_t)cols * Z > 0x7fffffff)
    return fail(LDPC_ERR_UNSUPPORTED, "lifted code too large");
  int64_t nnz = 0;
  for (int64_t i = 0; i < (int64_t)rows * cols; ++i) {
    if (base[i] >= Z || base[i] < -1) return fail(LDPC_ERR_INVALID_ARG, "shift out of [-1, Z)");
    nnz += base[i] >= 0;
  }
  std::vector<int32_t> chk, var;
  std::vector<uint8_t> punct((size_t)cols * Z, 0);
  try {
    chk.reserve((size_t)(nnz * Z));
    var.reserve((size_t)(nnz * Z));
  } catch (const std::bad_alloc&) {
    return fail(LDPC_ERR_NOMEM, "host allocation");
  }
  // circulant block (r, c, s): row z of the block has its one in column (z + s) mod Z
  for (int32_t r = 0; r < rows; ++r)
    for (int32_t c = 0; c < cols; ++c) {
      const int32_t s = base[(int64_t)r * cols + c];
      if (s < 0) continue;
      for (int32_t z = 0; z < Z; ++z) {
        chk.push_back(r * Z + z);
        var.push_back(c * Z + (z + s) % Z);
      }
    }
  if (punct_cols)
    for (int32_t c = 0; c < cols; ++c)
      if (punct_cols[c]) std::fill(punct.begin() + (size_t)c * Z, punct.begin() + (size_t)(c + 1) * Z, 1);
  ldpc_status_t st = build_code(chk.data(), var.data(), (int64_t)chk.size(), rows * Z, cols * Z, punct.data(),
                                k_info, Z, out);
  if (st == LDPC_OK) {
    build_qc_view(*out, base, rows, cols, Z);
    (*out)->base.assign(base, base + (int64_t)rows * cols);
    (*out)->base_rows = rows;
    (*out)->base_cols = cols;
  }
  return st;
}

ldpc_status_t ldpc_code_destroy(ldpc_code_t* code) {
  if (!code) return LDPC_OK;
  for (auto& kv : code->dev) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first);
    cudaFree(kv.second.buf);
    cudaFree(kv.second.punct);
    cudaSetDevice(cur);
  }
  delete code;
  return LDPC_OK;
}

ldpc_status_t ldpc_code_info(const ldpc_code_t* c, ldpc_code_info_t* out) {
  if (!c || !out) return fail(LDPC_ERR_INVALID_ARG, "NULL argument");
  out->n_checks = c->M;
  out->n_vars = c->N;
  out->n_edges = c->E;
  out->k_info = c->K;
  out->n_punctured = c->n_punct;
  out->max_vn_degree = c->dv_max;
  out->max_cn_degree = c->dc_max;
  out->max_two_hop = c->maxr;
  out->qc_lifting = c->qc.empty() ? 0 : c->Z;
  return LDPC_OK;
}

ldpc_status_t ldpc_code_edges(const ldpc_code_t* c, int32_t* check_out, int32_t* var_out) {
  if (!c || !check_out || !var_out) return fail(LDPC_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(check_out, c->e_cn.data(), sizeof(int32_t) * (size_t)c->E);
  std::memcpy(var_out, c->e_vn.data(), sizeof(int32_t) * (size_t)c->E);
  return LDPC_OK;
}

ldpc_status_t ldpc_awgn_llr_codewords(const ldpc_code_t* code, const float* ebn0_db, int64_t batch, uint64_t seed,
                                      uint64_t frame_offset, const uint8_t* codewords, float* llr, int8_t* qllr,
                                      float q_step, void* cuda_stream) {
  if (!code) return fail(LDPC_ERR_INVALID_ARG, "code is NULL");
  if (batch < 0) return fail(LDPC_ERR_INVALID_ARG, "batch < 0");
  if (batch == 0) return LDPC_OK;
  if (!ebn0_db || !llr) return fail(LDPC_ERR_INVALID_ARG, "ebn0_db and llr are required");
  if (qllr && !(q_step > 0.0f && std::isfinite(q_step))) return fail(LDPC_ERR_INVALID_ARG, "q_step must be > 0");
  const ldpc::GraphDesc* g;
  const uint8_t* punct;
  ldpc_status_t st = ensure_device(const_cast<ldpc_code_t*>(code), &g, &punct);
  if (st) return st;
  const int32_t ntx = code->N - code->n_punct;
  if (ntx <= 0) return fail(LDPC_ERR_INVALID_ARG, "every VN is punctured");
  const float rate = (float)code->K / (float)ntx;
  cudaError_t e = ldpc::launch_channel(g->N, punct, codewords, rate, ebn0_db, batch, seed, frame_offset, llr, qllr,
                                       q_step, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "channel launch");
  return LDPC_OK;
}

ldpc_status_t ldpc_awgn_llr(const ldpc_code_t* code, const float* ebn0_db, int64_t batch, uint64_t seed,
                            uint64_t frame_offset, float* llr, int8_t* qllr, float q_step, void* cuda_stream) {
  return ldpc_awgn_llr_codewords(code, ebn0_db, batch, seed, frame_offset, nullptr, llr, qllr, q_step, cuda_stream);
}

ldpc_status_t ldpc_encode(const ldpc_code_t* code, const uint8_t* info, int64_t batch, uint8_t* codewords,
                          void* cuda_stream) {
  if (!code) return fail(LDPC_ERR_INVALID_ARG, "code is NULL");
  if (batch < 0) return fail(LDPC_ERR_INVALID_ARG, "batch < 0");
  if (code->base.empty()) return fail(LDPC_ERR_UNSUPPORTED, "encoding needs a code built by ldpc_code_build_qc");
  ldpc::EncArgs* plan = new (std::nothrow) ldpc::EncArgs;
  if (!plan) return fail(LDPC_ERR_NOMEM, "host allocation");
  if (!ldpc::encode_plan(code->base.data(), code->base_rows, code->base_cols, code->Z, code->K, plan)) {
    delete plan;
    return fail(LDPC_ERR_UNSUPPORTED, "the parity part is not the dual-diagonal core + extension shape");
  }
  if (batch == 0) {
    delete plan;
    return LDPC_OK;
  }
  if (!info || !codewords) {
    delete plan;
    return fail(LDPC_ERR_INVALID_ARG, "info and codewords are required");
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t e = ldpc::launch_encode(*plan, info, codewords, batch, sms, (cudaStream_t)cuda_stream);
  delete plan;
  if (e != cudaSuccess) return cuda_fail(e, "encode launch");
  return LDPC_OK;
}

ldpc_status_t ldpc_decode(const ldpc_code_t* code, const void* llr, int64_t batch,
                          const ldpc_decode_params_t* p, uint8_t* hard, int64_t* updates, uint8_t* converged,
                          int32_t* trace, float* llr_out, void* cuda_stream) {
  ldpc_decode_outputs_t o;
  std::memset(&o, 0, sizeof(o));
  o.hard = hard;
  o.updates = updates;
  o.converged = converged;
  o.trace = trace;
  o.llr_out = llr_out;
  return ldpc_decode_ex(code, llr, batch, p, &o, cuda_stream);
}

ldpc_status_t ldpc_decode_ex(const ldpc_code_t* code, const void* llr, int64_t batch,
                             const ldpc_decode_params_t* p, const ldpc_decode_outputs_t* o, void* cuda_stream) {
  if (!code || !p || !o) return fail(LDPC_ERR_INVALID_ARG, "code, params and outputs are required");
  if (o->pre_out && p->schedule == LDPC_FLOODING) return fail(LDPC_ERR_INVALID_ARG, "flooding keeps no L~^C");
  if (batch < 0) return fail(LDPC_ERR_INVALID_ARG, "batch < 0");
  if (p->schedule < LDPC_FLOODING || p->schedule > LDPC_SLMDRBP)
    return fail(LDPC_ERR_INVALID_ARG, "unknown schedule");
  if (p->arith != LDPC_FP32_SUMPRODUCT && p->arith != LDPC_INT6_MINSUM)
    return fail(LDPC_ERR_INVALID_ARG, "unknown arithmetic");
  if (p->max_updates < 0 || p->check_interval < 0) return fail(LDPC_ERR_INVALID_ARG, "negative budget");
  if (!(p->gamma >= 0.0 && p->gamma <= 1.0)) return fail(LDPC_ERR_INVALID_ARG, "gamma outside [0, 1]");
  if (!(p->llr_clip > 0.0f && p->llr_clip <= 1.0e4f)) return fail(LDPC_ERR_INVALID_ARG, "llr_clip outside (0, 1e4]");
  if (p->arith == LDPC_INT6_MINSUM && !(p->q_step > 0.0f && std::isfinite(p->q_step)))
    return fail(LDPC_ERR_INVALID_ARG, "q_step");
  if (ldpc::is_multi_edge(p->schedule) && (p->n_p <= 0 || p->n_p > 384 || p->n_g <= 0 || p->n_g > 1024))
    return fail(LDPC_ERR_INVALID_ARG, "0 < n_p <= 384 and 0 < n_g <= 1024 required");
  if (p->form < LDPC_FORM_AUTO || p->form > LDPC_FORM_SPLIT || (p->tune & ~0x1ff) != 0 || (p->tune & 3) == 3)
    return fail(LDPC_ERR_INVALID_ARG, "bad form / tune");
  if (p->form == LDPC_FORM_CLUSTER && !ldpc::is_multi_edge(p->schedule))
    return fail(LDPC_ERR_UNSUPPORTED, "the cluster form runs the multi-edge schedules");
  if (p->form == LDPC_FORM_SPLIT && !ldpc::is_single_edge(p->schedule))
    return fail(LDPC_ERR_UNSUPPORTED, "the split form runs the single-edge schedules");
  if (batch == 0) return LDPC_OK;
  if (!llr) return fail(LDPC_ERR_INVALID_ARG, "llr is NULL");
  // lane teams: a check (every schedule) or a variable (dynamic schedules) within one warp
  if (code->dc_max > 32) return fail(LDPC_ERR_UNSUPPORTED, "check degree > 32");
  if (p->schedule != LDPC_FLOODING && code->dv_max > 32) return fail(LDPC_ERR_UNSUPPORTED, "variable degree > 32");

  const ldpc::GraphDesc* g;
  ldpc_status_t st = ensure_device(const_cast<ldpc_code_t*>(code), &g, nullptr);
  if (st) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  uint32_t* status;
  st = device_status_word(dev, &status);
  if (st) return st;

  ldpc::DecodeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = *g;
  a.llr = llr;
  a.batch = batch;
  a.hard = o->hard;
  a.updates = o->updates;
  a.converged = o->converged;
  a.trace = o->trace;
  a.llr_out = o->llr_out;
  a.c2v_out = o->c2v_out;
  a.pre_out = o->pre_out;
  a.fallbacks = o->fallbacks;
  a.max_updates = p->max_updates;
  a.check_interval = p->check_interval;
  a.gamma_f = (float)p->gamma;
  a.gamma_i = (int32_t)std::round(p->gamma * 65534.0);
  a.llr_clip = p->llr_clip;
  a.n_p = p->n_p;
  a.n_g = p->n_g;
  a.seed = p->seed;
  a.frame_offset = p->frame_offset;
  a.status = status;
  a.graph_smem = ldpc::graph_smem_bytes(*g);
  a.team_w = 1;
  while (a.team_w < g->dc_max) a.team_w <<= 1;
  // multi-edge CTA size: FP32 frames run two CTAs per SM (shared memory), where 512
  // threads hide more latency; 6-bit frames run four 256-thread CTAs per SM
  a.cta_threads = p->arith == LDPC_INT6_MINSUM ? 256 : 512;
  if ((p->tune & 3) != 0) a.cta_threads = (p->tune & 3) == 2 ? 512 : 256;
  if (p->arith == LDPC_INT6_MINSUM)
    for (int q = -127; q <= 127; ++q)
      a.ci_table[q + 127] = (int16_t)std::round(32767.0 * std::tanh(q * (double)p->q_step / 2.0));

  const int arith = p->arith == LDPC_INT6_MINSUM ? ldpc::kINT6 : ldpc::kFP32;
  const int optin = max_optin_smem();
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e;
  const int gsm = a.graph_smem;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  // Form: frame state in shared memory when it fits (LDPC_FORM_AUTO / SMEM), else
  // (or on request) in global-memory slots that persistent CTAs/warps reuse.
  size_t per = 0, cta_fixed = 0;
  if (p->schedule == LDPC_FLOODING) {
    per = ldpc::flood_smem_per_frame(arith, *g);
  } else if (ldpc::is_single_edge(p->schedule)) {
    per = ldpc::se_smem_per_frame(arith, p->schedule, *g);
  } else {
    if (p->n_g > 255) return fail(LDPC_ERR_UNSUPPORTED, "n_g > 255 for the multi-edge kernel");
    per = ldpc::me_smem_per_frame(arith, p->schedule, *g, p->n_p, p->n_g);
    cta_fixed = ldpc::me_smem_per_cta(*g, p->n_p, p->n_g) + 1024;  // + static table headroom
  }
  const bool fits = (int64_t)per + (int64_t)cta_fixed + gsm <= optin;
  if (p->form == LDPC_FORM_SMEM && !fits) return fail(LDPC_ERR_UNSUPPORTED, "frame state exceeds shared memory");
  // Cluster form (multi-edge): on request (LDPC_FORM_CLUSTER, or a cluster
  // size in tune bits 6-7), or for frames too large for one CTA when the batch
  // is small and the step is wide or integer: on 38 frames of the 26,112-bit
  // code a cluster of 8 decodes 2.9x faster than the global-memory form in
  // 6-bit mode and 1.07x faster in FP32 at N_P = 256, but 1.2x slower in FP32
  // at N_P = 64; it holds cs SMs, so with auto sizing it is taken while the
  // batch is at most twice the resident clusters.  The smallest cluster (or
  // the requested size) whose shared memory holds the state and that can be
  // resident; else the global-memory form.
  const int req = (p->tune >> 6) & 3;
  const bool cluster_pays = p->arith == LDPC_INT6_MINSUM || p->n_p >= 128;
  if (ldpc::is_multi_edge(p->schedule) &&
      (p->form == LDPC_FORM_CLUSTER || (p->form == LDPC_FORM_AUTO && (req != 0 || (!fits && cluster_pays))))) {
    const int threads = (p->tune & 3) == 1 ? 256 : 512;
    const int64_t avail = (int64_t)optin - gsm - 1024;
    for (int cs = req ? (2 << req) : 2; cs <= (req ? (2 << req) : 16); cs *= 2) {
      if (!ldpc::me_cluster_plan(arith, *g, p->n_p, p->n_g, cs, avail, &a.cl)) continue;
      if (p->form == LDPC_FORM_AUTO && req == 0 && batch > 2 * (int64_t)(sms / cs)) {
        a.cl.cs = 0;  // large batch: the global-memory form keeps every SM busy
        break;
      }
      a.cta_threads = threads;
      e = ldpc::launch_me_cluster(a, arith, p->schedule, threads, s);
      if (e == cudaSuccess) return LDPC_OK;
      a.cl.cs = 0;
      if (e != cudaErrorInvalidConfiguration && e != cudaErrorInvalidValue && e != cudaErrorNotSupported &&
          e != cudaErrorInvalidClusterSize)
        return cuda_fail(e, "cluster decode launch");
      (void)cudaGetLastError();  // this size cannot be resident: try the next
    }
    if (p->form == LDPC_FORM_CLUSTER) return fail(LDPC_ERR_UNSUPPORTED, "frame state exceeds a resident cluster");
  }
  if ((int64_t)cta_fixed + gsm > optin) return fail(LDPC_ERR_UNSUPPORTED, "working set exceeds shared memory");
  // single-edge frames (a warp each) that shared memory holds fewer than eight
  // per SM run faster with all state in global memory and 32 warps per SM
  // (WiFi-like code, 1.5 dB, 3E: LMD-CIRBP 2.5x, CIRBP 1.7x, RBP 1.7x over two
  // FP32 frames per SM; the split form ties or trails it); tune bit 8 asks for it too
  const int64_t smem_per_sm = (int64_t)228 * 1024 / ((int64_t)per + 1024);
  const bool se_few = ldpc::is_single_edge(p->schedule) && fits && ((p->tune & 0x100) != 0 || smem_per_sm < 8);
  void* scratch = nullptr;
  // single-edge split form: the V region of a frame in shared memory, its edge
  // arrays in a global slot; one CTA per SM holds as many frames as fit
  const size_t vper = ldpc::is_single_edge(p->schedule) ? ldpc::se_vregion_bytes(arith, p->schedule, *g) : 0;
  const int split_fpc = vper > 0 ? (int)std::min<int64_t>(16, ((int64_t)optin - gsm) / (int64_t)vper) : 0;
  if (p->form == LDPC_FORM_SPLIT && split_fpc < 1)
    return fail(LDPC_ERR_UNSUPPORTED, "the VN arrays of a frame exceed shared memory");
  if (p->form == LDPC_FORM_SPLIT) {
    int fpc = split_fpc;
    if ((p->tune >> 2) & 3) fpc = std::min(fpc, 1 << ((p->tune >> 2) & 3));  // 2, 4 or 8 frames by request
    if ((int64_t)fpc > batch) fpc = (int)batch;
    const int64_t ctas = std::min<int64_t>((batch + fpc - 1) / fpc, (int64_t)sms);
    const int64_t estride = ((int64_t)(per - vper) + 255) & ~(int64_t)255;
    e = cudaMallocAsync(&scratch, (size_t)(ctas * fpc) * (size_t)estride, s);
    if (e != cudaSuccess) return fail(LDPC_ERR_NOMEM, std::string("cudaMallocAsync(state): ") + cudaGetErrorString(e));
    a.se_split = 1;
    a.gstate = scratch;
    a.gstate_stride = estride;
    a.gstate_ctas = (int32_t)ctas;
    a.frames_per_cta = fpc;
    a.smem_per_frame = (int32_t)(((int64_t)vper + 15) & ~(int64_t)15);
    e = ldpc::launch_se(a, arith, p->schedule, s);
    const cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    return LDPC_OK;
  }
  const bool global_form = p->form == LDPC_FORM_GLOBAL || !fits || (p->form == LDPC_FORM_AUTO && se_few);
  a.smem_per_frame = (int32_t)per;
  if (global_form) {
    const int64_t stride = ((int64_t)per + 255) & ~(int64_t)255;
    int fpc = 1;
    int64_t ctas;
    if (ldpc::is_single_edge(p->schedule)) {
      fpc = (int)std::min<int64_t>(8, batch);
      ctas = std::min<int64_t>((batch + fpc - 1) / fpc, (int64_t)sms * 4);
    } else {
      ctas = std::min<int64_t>(batch, (int64_t)sms * 2);
    }
    const size_t bytes = (size_t)(ctas * fpc) * (size_t)stride;
    e = cudaMallocAsync(&scratch, bytes, s);
    if (e != cudaSuccess) return fail(LDPC_ERR_NOMEM, std::string("cudaMallocAsync(state): ") + cudaGetErrorString(e));
    a.gstate = scratch;
    a.gstate_stride = stride;
    a.gstate_ctas = (int32_t)ctas;
    a.frames_per_cta = fpc;
  } else if (ldpc::is_single_edge(p->schedule)) {
    // frames per CTA: fill about half the opt-in shared memory so two CTAs share an SM
    int fpc = (int)std::max<size_t>(1, std::min<size_t>(16, (size_t)std::max(0, optin / 2 - gsm) / per));
    if ((p->tune >> 2) & 3) fpc = 1 << ((p->tune >> 2) & 3);  // 2, 4 or 8 frames by request
    while (fpc > 1 && (int)(fpc * per) + gsm > optin) --fpc;
    if ((int64_t)fpc > batch) fpc = (int)batch;
    a.frames_per_cta = fpc;
  } else {
    a.frames_per_cta = 1;
  }
  if (p->schedule == LDPC_FLOODING) e = ldpc::launch_flood(a, arith, s);
  else if (ldpc::is_single_edge(p->schedule)) e = ldpc::launch_se(a, arith, p->schedule, s);
  else e = ldpc::launch_me(a, arith, p->schedule, s);
  if (scratch) {
    const cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return cuda_fail(e, "decode launch");
  return LDPC_OK;
}

ldpc_status_t ldpc_decode_queue(const ldpc_code_t* const* codes, int32_t n_codes, const ldpc_work_item_t* items,
                                int64_t n_items, const void* llr, const ldpc_decode_params_t* p, uint8_t* hard,
                                int64_t* updates, uint8_t* converged, int32_t mode, void* cuda_stream) {
  static_assert(sizeof(ldpc_work_item_t) == sizeof(ldpc::WorkItem), "work item layout");
  if (!codes || !p || n_codes < 1 || n_codes > ldpc::kMaxQueueCodes)
    return fail(LDPC_ERR_INVALID_ARG, "1..16 codes and params are required");
  if (n_items < 0 || (mode != LDPC_QUEUE_STATIC && mode != LDPC_QUEUE_PERSISTENT))
    return fail(LDPC_ERR_INVALID_ARG, "bad item count or mode");
  // the head counter is 32-bit and each CTA takes one item past the end
  if (n_items > ((int64_t)1 << 31) - ((int64_t)1 << 20)) return fail(LDPC_ERR_UNSUPPORTED, "more than 2^31 - 2^20 items");
  if (p->schedule != LDPC_LMD_CIRBP && p->schedule != LDPC_ME_CIRBP && p->schedule != LDPC_ME_LMD_CIRBP)
    return fail(LDPC_ERR_UNSUPPORTED, "queue form: LMD-CIRBP, ME-CIRBP or ME-LMD-CIRBP");
  if (p->arith != LDPC_FP32_SUMPRODUCT && p->arith != LDPC_INT6_MINSUM)
    return fail(LDPC_ERR_INVALID_ARG, "unknown arithmetic");
  if (p->check_interval < 0 || !(p->gamma >= 0.0 && p->gamma <= 1.0) || !(p->llr_clip > 0.0f && p->llr_clip <= 1.0e4f) ||
      (p->arith == LDPC_INT6_MINSUM && !(p->q_step > 0.0f)) || (p->tune & ~0x1ff) != 0 || (p->tune & 3) == 3)
    return fail(LDPC_ERR_INVALID_ARG, "bad parameters");
  const bool me = p->schedule != LDPC_LMD_CIRBP;
  if (me && (p->n_p <= 0 || p->n_p > 384 || p->n_g <= 0 || p->n_g > 255)) return fail(LDPC_ERR_INVALID_ARG, "n_p, n_g");
  if (n_items == 0) return LDPC_OK;
  if (!items || !llr) return fail(LDPC_ERR_INVALID_ARG, "items and llr are required");
  int dev = 0;
  cudaGetDevice(&dev);
  uint32_t* status;
  ldpc_status_t st = device_status_word(dev, &status);
  if (st) return st;
  const int arith = p->arith == LDPC_INT6_MINSUM ? ldpc::kINT6 : ldpc::kFP32;
  ldpc::QueueArgs q;
  std::memset(&q, 0, sizeof(q));
  size_t graph_bytes = 0, small_bytes = 0, big_max = 0;
  std::vector<size_t> bigs;
  for (int i = 0; i < n_codes; ++i) {
    if (!codes[i]) return fail(LDPC_ERR_INVALID_ARG, "NULL code");
    const ldpc::GraphDesc* g;
    st = ensure_device(const_cast<ldpc_code_t*>(codes[i]), &g, nullptr);
    if (st) return st;
    if (!g->is_qc) return fail(LDPC_ERR_UNSUPPORTED, "queue form needs codes built by ldpc_code_build_qc");
    if (g->dc_max > 32 || g->dv_max > 32) return fail(LDPC_ERR_UNSUPPORTED, "degree > 32");
    q.codes[i] = *g;
    graph_bytes = std::max(graph_bytes, (size_t)ldpc::graph_smem_bytes(*g));
    const size_t big = me ? ldpc::me_smem_per_frame(arith, p->schedule, *g, p->n_p, p->n_g)
                          : ldpc::se_smem_per_frame(arith, p->schedule, *g);
    bigs.push_back(big);
    big_max = std::max(big_max, big);
    if (me) small_bytes = std::max(small_bytes, ldpc::me_smem_per_cta(*g, p->n_p, p->n_g));
  }
  const int optin = max_optin_smem();
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t fixed = graph_bytes + small_bytes + (me ? 1024 : 0);
  if ((int64_t)fixed > optin) return fail(LDPC_ERR_UNSUPPORTED, "working set exceeds shared memory");
  // frame state in shared memory for codes up to a size: two CTAs per SM by
  // default (three, one or none by tune bits 4-5); larger codes use global slots
  const int placement = (p->tune >> 4) & 3;
  const int64_t share = placement == 3 ? 0 : (placement == 2 ? optin : (placement == 1 ? optin / 3 - 1024 : optin / 2 - 1024));
  const size_t budget = share > (int64_t)fixed ? (size_t)(share - (int64_t)fixed) : 0;
  size_t sstate = 0;
  for (size_t b : bigs)
    if (b <= budget) sstate = std::max(sstate, b);
  const int threads = me ? ((p->tune & 3) == 1 ? 256 : ((p->tune & 3) == 2 ? 512 : (arith == ldpc::kINT6 ? 256 : 512))) : 32;
  const size_t smem = fixed + sstate;
  int grid;
  if (mode == LDPC_QUEUE_PERSISTENT) {
    // one CTA per resident slot: the occupancy of the kernel actually launched
    int per_sm = 0;
    const cudaError_t e = me ? ldpc::me_queue_blocks_per_sm(arith, p->schedule, threads, smem, &per_sm)
           : ldpc::se_queue_blocks_per_sm(arith, smem, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    if (per_sm < 1) return fail(LDPC_ERR_UNSUPPORTED, "queue kernel does not fit an SM");
    grid = (int)std::min<int64_t>(n_items, (int64_t)sms * per_sm);
  } else {
    if (n_items > 0x7fffffff) return fail(LDPC_ERR_UNSUPPORTED, "too many items for one launch");
    grid = (int)n_items;
  }
  const size_t stride = ((big_max + 255) / 256) * 256;
  const bool need_global = sstate < big_max;
  const size_t bytes = 256 + (need_global ? (size_t)grid * stride : 0);
  void* scratch = nullptr;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
  if (e != cudaSuccess) return fail(LDPC_ERR_NOMEM, std::string("cudaMallocAsync(queue): ") + cudaGetErrorString(e));
  e = cudaMemsetAsync(scratch, 0, 256, s);
  ldpc::DecodeArgs& a = q.a;
  a.llr = llr;
  a.batch = n_items;
  a.hard = hard;
  a.updates = updates;
  a.converged = converged;
  a.check_interval = p->check_interval;
  a.gamma_f = (float)p->gamma;
  a.gamma_i = (int32_t)std::round(p->gamma * 65534.0);
  a.llr_clip = p->llr_clip;
  a.n_p = p->n_p;
  a.n_g = p->n_g;
  a.seed = p->seed;
  a.status = status;
  a.gstate = need_global ? (unsigned char*)scratch + 256 : nullptr;
  a.gstate_stride = (int64_t)stride;
  if (arith == ldpc::kINT6)
    for (int qq = -127; qq <= 127; ++qq)
      a.ci_table[qq + 127] = (int16_t)std::round(32767.0 * std::tanh(qq * (double)p->q_step / 2.0));
  q.n_codes = n_codes;
  q.items = (const ldpc::WorkItem*)items;
  q.n_items = n_items;
  q.head = (unsigned int*)scratch;
  q.persistent = mode == LDPC_QUEUE_PERSISTENT;
  q.graph_bytes = (int32_t)graph_bytes;
  q.small_bytes = (int32_t)small_bytes;
  q.smem_state_bytes = (int32_t)sstate;
  if (e == cudaSuccess)
    e = me ? ldpc::launch_me_queue(q, arith, p->schedule, threads, grid, smem, s)
           : ldpc::launch_se_queue(q, arith, grid, smem, s);
  const cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "queue launch");
  return LDPC_OK;
}

namespace {
// Shared checks of the weighted-BP entry points; sets up `a` on success.
ldpc_status_t wbp_setup(const ldpc_code_t* code, const float* llr, int64_t batch, const int32_t* trace, int64_t T,
                        const float* weights, float llr_clip, bool backward, ldpc::WbpArgs* a, int* fpc) {
  if (!code) return fail(LDPC_ERR_INVALID_ARG, "code is required");
  if (batch < 0 || T < 0) return fail(LDPC_ERR_INVALID_ARG, "negative batch or T");
  if (!(llr_clip > 0.0f && llr_clip <= 1.0e4f)) return fail(LDPC_ERR_INVALID_ARG, "llr_clip outside (0, 1e4]");
  if (batch > 0 && (!llr || (T > 0 && (!trace || !weights))))
    return fail(LDPC_ERR_INVALID_ARG, "llr, trace and weights are required");
  std::memset(a, 0, sizeof(*a));
  if (batch == 0) return LDPC_OK;
  const ldpc::GraphDesc* g;
  ldpc_status_t st = ensure_device(const_cast<ldpc_code_t*>(code), &g, nullptr);
  if (st) return st;
  if (g->dc_max > 32) return fail(LDPC_ERR_UNSUPPORTED, "check degree > 32");
  int dev = 0;
  cudaGetDevice(&dev);
  uint32_t* status;
  st = device_status_word(dev, &status);
  if (st) return st;
  a->g = *g;
  a->llr = llr;
  a->batch = batch;
  a->trace = trace;
  a->T = T;
  a->w = weights;
  a->clip = llr_clip;
  a->status = status;
  a->graph_smem = ldpc::graph_smem_bytes(*g);
  a->frame_bytes = ldpc::wbp_state_bytes(*g, backward);
  const int64_t room = (int64_t)max_optin_smem() - a->graph_smem;
  // frames (warps) per CTA: as many as shared memory holds for the adjoint (a
  // serial chain per frame: more resident warps pay; 11 frames of the n = 576
  // code: -21 %), at most 8 for the forward (more gained nothing there)
  const int64_t f = std::min<int64_t>(backward ? 16 : 8, std::min<int64_t>(batch, room / a->frame_bytes));
  if (f < 1) return fail(LDPC_ERR_UNSUPPORTED, "frame state exceeds shared memory");
  *fpc = (int)f;
  return LDPC_OK;
}
}  // namespace

ldpc_status_t ldpc_wbp_forward(const ldpc_code_t* code, const float* llr, int64_t batch, const int32_t* trace,
                               const int64_t* counts, int64_t T, const float* weights, float llr_clip,
                               float* llr_out, float* c_out, float* tape, void* cuda_stream) {
  ldpc::WbpArgs a;
  int fpc = 0;
  ldpc_status_t st = wbp_setup(code, llr, batch, trace, T, weights, llr_clip, false, &a, &fpc);
  if (st || batch == 0) return st;
  a.counts = counts;
  a.llr_out = llr_out;
  a.c_out = c_out;
  a.tape = tape;
  const cudaError_t e = ldpc::launch_wbp(a, false, fpc, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "weighted BP forward");
  return LDPC_OK;
}

ldpc_status_t ldpc_wbp_backward(const ldpc_code_t* code, const float* llr, int64_t batch, const int32_t* trace,
                                const int64_t* counts, int64_t T, const float* weights, float llr_clip,
                                const float* c_final, const float* tape, const float* dL, float* dw_frames,
                                float* dw, float* dllr, void* cuda_stream) {
  if (batch > 0 && (!c_final || !dL || !dw_frames || (T > 0 && !tape)))
    return fail(LDPC_ERR_INVALID_ARG, "c_final, tape, dL and dw_frames are required");
  ldpc::WbpArgs a;
  int fpc = 0;
  ldpc_status_t st = wbp_setup(code, llr, batch, trace, T, weights, llr_clip, true, &a, &fpc);
  if (st || batch == 0) return st;
  a.counts = counts;
  a.c_in = c_final;
  a.tape_in = tape;
  a.dL = dL;
  a.dw_frames = dw_frames;
  a.dw = dw;
  a.dllr = dllr;
  const cudaError_t e = ldpc::launch_wbp(a, true, fpc, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "weighted BP backward");
  return LDPC_OK;
}

ldpc_status_t ldpc_ci_stats(const float* llr_now, const float* llr_pre, int64_t count, int32_t n_bins,
                            uint64_t* counts, void* cuda_stream) {
  if (count < 0 || n_bins < 1 || n_bins > 1024) return fail(LDPC_ERR_INVALID_ARG, "count >= 0 and 1 <= n_bins <= 1024");
  if (!counts || (count > 0 && (!llr_now || !llr_pre))) return fail(LDPC_ERR_INVALID_ARG, "NULL buffer");
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t e = ldpc::launch_ci_stats(llr_now, llr_pre, count, n_bins, (unsigned long long*)counts, sms,
                                              (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "ci_stats");
  return LDPC_OK;
}

ldpc_status_t ldpc_sync(void* cuda_stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int dev = 0;
  cudaGetDevice(&dev);
  uint32_t* status;
  ldpc_status_t st = device_status_word(dev, &status);
  if (st) return st;
  uint32_t v = 0;
  e = cudaMemcpy(&v, status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read status");
  if (v) {
    e = cudaMemset(status, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
  }
  if (v & 2u) return fail(LDPC_ERR_TIMEOUT, "a bounded device wait gave up");
  if (v & 4u) return fail(LDPC_ERR_INVALID_ARG, "a queue item named a code outside its call's code list, "
                                               "or a weighted-BP trace entry is not an edge id");
  if (v & 1u) return fail(LDPC_ERR_NONFINITE_LLR, "a decode saw a non-finite or out-of-range LLR");
  return LDPC_OK;
}

}  // extern "C"
