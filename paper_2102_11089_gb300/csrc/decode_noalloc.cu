// decode_noalloc.cu -- ldpc_decode_noalloc: decoding that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they decode:
// real-time loops that must not enter the CUDA allocator (its calls can block
// on the device or take locks for an unbounded time), processes whose device
// memory is all handed out up front to another allocator (a framework's
// caching pool) or capped by a fixed budget, and plug-ins that run inside a
// host application which owns every allocation.  ldpc_decode allocates the
// frame-state slots of its global-memory form (cudaMallocAsync) and uploads a
// code on its first use on a device (cudaMalloc); this entry point does
// neither.  It runs the same
// global-memory-form kernels on a file-scope device array of fixed size,
// holding the code's graph tables (copied from the host handle at each call)
// followed by the state slots.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"
#include "ldpc.h"

namespace {

// Size of the static scratch array.  Every GPU on which this library's code is
// loaded holds it until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];
__device__ __align__(256) uint32_t g_scratch_status;

struct DeviceScratch {
  unsigned char* scratch = nullptr;  // device address of g_scratch
  uint32_t* status = nullptr;        // device address of g_scratch_status
};

std::mutex g_mu;
std::map<int, DeviceScratch> g_dev;

// failures are reported through ldpc_last_error_detail()
ldpc_status_t fail(ldpc_status_t st, const std::string& why) {
  ldpc::set_error_detail(why);
  return st;
}

// Once per device, with that device current: resolve the device addresses of
// the static arrays (in host code their names are only host-side stand-ins).
ldpc_status_t scratch_for_device(int dev, DeviceScratch* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dev.find(dev);
  if (it == g_dev.end()) {
    DeviceScratch d;
    cudaError_t e = cudaGetSymbolAddress((void**)&d.scratch, g_scratch);
    if (e != cudaSuccess) return fail(LDPC_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress((void**)&d.status, g_scratch_status);
    if (e != cudaSuccess) return fail(LDPC_ERR_CUDA, std::string("cudaGetSymbolAddress(status): ") + cudaGetErrorString(e));
    it = g_dev.emplace(dev, d).first;
  }
  *out = it->second;
  return LDPC_OK;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" ldpc_status_t ldpc_decode_noalloc(const ldpc_code_t* code, const void* llr, int64_t batch,
                                             const ldpc_decode_params_t* p, uint8_t* hard, int64_t* updates,
                                             uint8_t* converged, int32_t* trace, float* llr_out,
                                             void* cuda_stream) {
  ldpc::CodeHostView v;
  if (!code || !p || !ldpc::code_host_view(code, &v)) return fail(LDPC_ERR_INVALID_ARG, "code and params are required");
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
  if (ldpc::is_multi_edge(p->schedule) && (p->n_p <= 0 || p->n_p > 384 || p->n_g <= 0 || p->n_g > 255))
    return fail(LDPC_ERR_INVALID_ARG, "0 < n_p <= 384 and 0 < n_g <= 255 required");
  if (p->form < LDPC_FORM_AUTO || p->form > LDPC_FORM_SPLIT || (p->tune & ~0x1ff) != 0 || (p->tune & 3) == 3)
    return fail(LDPC_ERR_INVALID_ARG, "bad form / tune");
  if (batch == 0) return LDPC_OK;
  if (!llr) return fail(LDPC_ERR_INVALID_ARG, "llr is NULL");
  if (v.dc_max > 32) return fail(LDPC_ERR_UNSUPPORTED, "check degree > 32");
  if (p->schedule != LDPC_FLOODING && v.dv_max > 32) return fail(LDPC_ERR_UNSUPPORTED, "variable degree > 32");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LDPC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  DeviceScratch sc;
  ldpc_status_t st = scratch_for_device(dev, &sc);
  if (st) return st;
  const cudaStream_t s = (cudaStream_t)cuda_stream;

  // graph tables at the start of the array: the protograph view of a lifted
  // code, else the CSR arrays
  ldpc::GraphDesc g;
  std::memset(&g, 0, sizeof(g));
  g.M = v.M; g.N = v.N; g.E = v.E;
  g.dv_max = v.dv_max; g.dc_max = v.dc_max; g.maxr = v.maxr;
  size_t graph_bytes;
  if (v.qc) {
    graph_bytes = round_up((size_t)v.qc_words * 4, 256);
    if (graph_bytes > kStaticScratchBytes) return fail(LDPC_ERR_UNSUPPORTED, "graph exceeds the static scratch");
    e = cudaMemcpyAsync(sc.scratch, v.qc, (size_t)v.qc_words * 4, cudaMemcpyHostToDevice, s);
    g.is_qc = 1;
    g.qc = (const int32_t*)sc.scratch;
    g.qc_words = v.qc_words;
    g.qc_R = v.qc_R; g.qc_C = v.qc_C; g.qc_Z = v.Z; g.qc_nnz = v.qc_nnz;
    g.qc_zmul = v.qc_zmul; g.qc_zshift = v.qc_zshift;
  } else {
    graph_bytes = round_up((size_t)v.tab_words * 4, 256);
    if (graph_bytes > kStaticScratchBytes) return fail(LDPC_ERR_UNSUPPORTED, "graph exceeds the static scratch");
    const int32_t* parts[5];
    int32_t sizes[5];
    ldpc::code_host_tab(code, parts, sizes);
    size_t off = 0;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
      e = cudaMemcpyAsync(sc.scratch + off, parts[i], (size_t)sizes[i] * 4, cudaMemcpyHostToDevice, s);
      off += (size_t)sizes[i] * 4;
    }
    g.tab = (const int32_t*)sc.scratch;
    g.tab_words = v.tab_words;
    g.tab_in_smem = (size_t)v.tab_words * 4 <= 32 * 1024;
  }
  if (e != cudaSuccess) return fail(LDPC_ERR_CUDA, std::string("cudaMemcpyAsync(graph): ") + cudaGetErrorString(e));
  // the status word is shared by every call: clear it
  e = cudaMemsetAsync(sc.status, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return fail(LDPC_ERR_CUDA, std::string("cudaMemsetAsync(status): ") + cudaGetErrorString(e));

  ldpc::DecodeArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = g;
  a.llr = llr;
  a.batch = batch;
  a.hard = hard;
  a.updates = updates;
  a.converged = converged;
  a.trace = trace;
  a.llr_out = llr_out;
  a.max_updates = p->max_updates;
  a.check_interval = p->check_interval;
  a.gamma_f = (float)p->gamma;
  a.gamma_i = (int32_t)std::round(p->gamma * 65534.0);
  a.llr_clip = p->llr_clip;
  a.n_p = p->n_p;
  a.n_g = p->n_g;
  a.seed = p->seed;
  a.frame_offset = p->frame_offset;
  a.status = sc.status;
  a.graph_smem = ldpc::graph_smem_bytes(g);
  a.team_w = 1;
  while (a.team_w < g.dc_max) a.team_w <<= 1;
  a.cta_threads = p->arith == LDPC_INT6_MINSUM ? 256 : 512;
  if ((p->tune & 3) != 0) a.cta_threads = (p->tune & 3) == 2 ? 512 : 256;
  const int arith = p->arith == LDPC_INT6_MINSUM ? ldpc::kINT6 : ldpc::kFP32;
  if (arith == ldpc::kINT6)
    for (int q = -127; q <= 127; ++q)
      a.ci_table[q + 127] = (int16_t)std::round(32767.0 * std::tanh(q * (double)p->q_step / 2.0));

  // state slots after the graph, as many as fit (at most the usual count)
  int sms = 1, optin = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(LDPC_ERR_CUDA, std::string("cudaDeviceGetAttribute(SM count): ") + cudaGetErrorString(e));
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess)
    return fail(LDPC_ERR_CUDA, std::string("cudaDeviceGetAttribute(shared memory): ") + cudaGetErrorString(e));
  if (sms < 1) sms = 1;
  size_t per, cta_fixed = 0;
  int fpc = 1;
  int64_t want;
  if (p->schedule == LDPC_FLOODING) {
    per = ldpc::flood_smem_per_frame(arith, g);
    want = std::min<int64_t>(batch, (int64_t)sms * 2);
  } else if (ldpc::is_single_edge(p->schedule)) {
    per = ldpc::se_smem_per_frame(arith, p->schedule, g);
    fpc = (int)std::min<int64_t>(8, batch);
    want = std::min<int64_t>((batch + fpc - 1) / fpc, (int64_t)sms * 4);
  } else {
    per = ldpc::me_smem_per_frame(arith, p->schedule, g, p->n_p, p->n_g);
    cta_fixed = ldpc::me_smem_per_cta(g, p->n_p, p->n_g) + 1024;
    want = std::min<int64_t>(batch, (int64_t)sms * 2);
  }
  if ((int64_t)cta_fixed + a.graph_smem > optin) return fail(LDPC_ERR_UNSUPPORTED, "working set exceeds shared memory");
  const size_t stride = round_up(per, 256);
  const int64_t cap_slots = (int64_t)((kStaticScratchBytes - graph_bytes) / stride);
  if (cap_slots < fpc)
    return fail(LDPC_ERR_UNSUPPORTED, "frame state of " + std::to_string(stride) + " bytes per frame exceeds the " +
                                          std::to_string(kStaticScratchBytes >> 20) + " MiB static scratch");
  const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(want, cap_slots / fpc));
  a.gstate = sc.scratch + graph_bytes;
  a.gstate_stride = (int64_t)stride;
  a.gstate_ctas = (int32_t)ctas;
  a.frames_per_cta = fpc;
  a.smem_per_frame = (int32_t)per;
  if (p->schedule == LDPC_FLOODING) e = ldpc::launch_flood(a, arith, s);
  else if (ldpc::is_single_edge(p->schedule)) e = ldpc::launch_se(a, arith, p->schedule, s);
  else e = ldpc::launch_me(a, arith, p->schedule, s);
  if (e != cudaSuccess) return fail(LDPC_ERR_CUDA, std::string("decode launch: ") + cudaGetErrorString(e));
  return LDPC_OK;
}
