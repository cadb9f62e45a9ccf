// internal.h -- structures shared by the host dispatcher and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

namespace ldpc {

constexpr int kFP32 = 0;
constexpr int kINT6 = 1;

constexpr int kFlooding = 0;
constexpr int kRBP = 1;
constexpr int kCIRBP = 2;
constexpr int kLMD = 3;
constexpr int kMECIRBP = 4;
constexpr int kMELMD = 5;
constexpr int kLMDRBP = 6;   // Algorithm 2
constexpr int kSLMDRBP = 7;  // Algorithm 2 without line 10

inline __host__ __device__ bool is_multi_edge(int s) { return s == kMECIRBP || s == kMELMD; }
inline __host__ __device__ bool is_single_edge(int s) { return s >= kRBP && !is_multi_edge(s) && s <= kSLMDRBP; }

// Device view of a code (canonical CSR edge order: by check, then variable).
// `tab` = cn_ptr[M+1] | e_vn[E] | e_cn[E] | vn_ptr[N+1] | vn_e[E] (int32), always
// present.  For codes lifted from a protograph `qc` holds (see graph.cuh)
// rowinfo[R] (int4) | colinfo[C] (int4) | colblk[nnz] (int4) | rowblk[nnz] (int2).
struct GraphDesc {
  int32_t M, N, E;
  int32_t dv_max, dc_max, maxr;  // maxr = max_n sum_{m in M(n)} |N(m)|
  const int32_t* tab;
  int32_t tab_words;
  int32_t tab_in_smem;  // stage the tables into shared memory
  const int32_t* qc;
  int32_t qc_words;
  int32_t qc_R, qc_C, qc_Z, qc_nnz;
  uint32_t qc_zmul, qc_zshift;
  int32_t is_qc;
};

// Everything a decode kernel needs, passed by value.
// Cluster form of the multi-edge decoders: where each frame-state array lives
// in the shared memory of the CTAs of a cluster.  Element i of array k is in
// rank rank0[k] + (i >> shift[k]), at byte off[k] + (i & (2^shift[k] - 1)) *
// element size from the start of that CTA's state area.
constexpr int kClusterArrays = 19;  // C P lam L D Lt grp par | sel est best cnl cul cbits cnt cntS bits touched misc
struct ClusterPlan {
  int32_t cs;     // CTAs per cluster (0: not the cluster form)
  int32_t bytes;  // state bytes per CTA
  int32_t off[kClusterArrays];
  int8_t shift[kClusterArrays];
  int8_t rank0[kClusterArrays];
};

struct DecodeArgs {
  GraphDesc g;
  const void* llr;  // [batch][N] float (FP32) or int8 (INT6)
  int64_t batch;
  uint8_t* hard;
  int64_t* updates;
  uint8_t* converged;
  int32_t* trace;
  float* llr_out;
  float* c2v_out;      // [batch][E] final L^C, or null
  float* pre_out;      // [batch][E] final L~^C, or null
  int64_t* fallbacks;  // [batch] CIRBP updates chosen by the residual fallback, or null
  int64_t max_updates;
  int64_t check_interval;
  float gamma_f;    // FP32 threshold on D
  int32_t gamma_i;  // INT6 threshold: round(gamma * 65534)
  float llr_clip;
  int32_t n_p, n_g;
  uint64_t seed;
  uint64_t frame_offset;
  uint32_t* status;  // device status word (bit 0: bad input seen)
  void* gstate;          // global-memory form: state slots (else null)
  int64_t gstate_stride;  // bytes per slot
  int32_t gstate_ctas;    // CTAs of the global-memory form
  int32_t frames_per_cta;
  int32_t smem_per_frame;  // shared-memory bytes per frame (single-edge split form: the V region)
  int32_t se_split;        // single-edge split form: E regions in global slots of gstate_stride bytes
  int32_t graph_smem;    // bytes of staged graph tables at the start of shared memory
  int32_t team_w;        // lanes per check team: power of two >= max check degree
  int32_t cta_threads;   // multi-edge CTA size (256 or 512)
  ClusterPlan cl;         // cluster form (cl.cs > 0)
  int16_t ci_table[256];  // INT6: round(32767 tanh(q * q_step / 2)), q = -127..127
};

// Per-frame inputs and outputs of one decode (built from DecodeArgs for frame b
// of a batch, or from a work item of the queue form).
struct FrameIO {
  const void* llr;     // this frame's N channel LLRs (float or int8)
  uint8_t* hard;       // N decisions, or null
  float* llr_out;      // N final LLRs, or null
  int64_t* updates;    // update count, or null
  uint8_t* converged;  // flags, or null
  int32_t* trace;      // max_updates edge ids, or null
  float* c2v_out;      // E final L^C, or null
  float* pre_out;      // E final L~^C, or null
  int64_t* fallbacks;  // CIRBP fallback count, or null
  int64_t max_updates;
  uint64_t frame;  // global frame index (Algorithm 4's Philox counter)
};

// FrameIO with every optional output absent (queue form)
inline __device__ FrameIO empty_io() {
  FrameIO io;
  io.llr = nullptr;
  io.hard = nullptr;
  io.llr_out = nullptr;
  io.updates = nullptr;
  io.converged = nullptr;
  io.trace = nullptr;
  io.c2v_out = nullptr;
  io.pre_out = nullptr;
  io.fallbacks = nullptr;
  io.max_updates = 0;
  io.frame = 0;
  return io;
}

inline __host__ __device__ int align16(int x) { return (x + 15) & ~15; }

inline __host__ __device__ int team_width(int dc_max) {
  int w = 1;
  while (w < dc_max) w <<= 1;
  return w;
}

// FrameIO of frame b of a batch decode
inline __device__ FrameIO batch_io(const DecodeArgs& a, int64_t b, int elem_bytes) {
  FrameIO io;
  const int64_t N = a.g.N;
  io.llr = (const unsigned char*)a.llr + b * N * elem_bytes;
  io.hard = a.hard ? a.hard + b * N : nullptr;
  io.llr_out = a.llr_out ? a.llr_out + b * N : nullptr;
  io.updates = a.updates ? a.updates + b : nullptr;
  io.converged = a.converged ? a.converged + b : nullptr;
  io.trace = a.trace ? a.trace + b * a.max_updates : nullptr;
  io.c2v_out = a.c2v_out ? a.c2v_out + b * (int64_t)a.g.E : nullptr;
  io.pre_out = a.pre_out ? a.pre_out + b * (int64_t)a.g.E : nullptr;
  io.fallbacks = a.fallbacks ? a.fallbacks + b : nullptr;
  io.max_updates = a.max_updates;
  io.frame = a.frame_offset + (uint64_t)b;
  return io;
}

inline __host__ __device__ int graph_smem_bytes(const GraphDesc& d) {
  if (d.is_qc) return align16(d.qc_words * 4);
  return d.tab_in_smem ? align16(d.tab_words * 4) : 0;
}

// Per-frame state layout of the single-edge (warp per frame) decoder, in two
// regions: the V region (VN- and check-sized arrays, `vtotal` bytes) and the E
// region (the edge arrays C, P: offsets relative to its start, `etotal`
// bytes).  Contiguous placement puts the E region right after the V region
// (`total` bytes); the split form keeps the V region in shared memory and the
// E region in global memory.  Dblk / Rblk: the largest metric key of each
// block of 32 VNs / 32 checks (the upper level of the global argmax of CIRBP
// and RBP), with dirty bits of blocks whose maximum may have dropped.
struct SELayout {
  int lam, L, D, Lt, Rmax, Ridx, par, Dblk, Ddirty, Rblk, Rdirty, tab, vtotal;
  int C, P, etotal;
  int total;
};

// Per-frame state of the single-edge schedules: the residual maxima for the
// schedules that search residuals, the exact L~ sums (Lt) for those that read D.
inline __host__ __device__ SELayout se_layout(int arith, int M, int N, int E, int sched) {
  const bool need_r = sched != kLMD;
  const bool need_lt = sched == kLMD || sched == kCIRBP;
  const int msg = arith == kINT6 ? 1 : 4;
  const int llr = arith == kINT6 ? 2 : 4;
  const int dv = arith == kINT6 ? 2 : 4;
  SELayout l;
  int o = 0;
  l.lam = o; o = align16(o + N * llr);
  l.L = o; o = align16(o + N * llr);
  l.D = o; o = align16(o + N * dv);
  l.Lt = o; o = align16(o + (need_lt ? N * 4 : 0));
  l.Rmax = o; o = align16(o + (need_r ? M * msg : 0));
  l.Ridx = o; o = align16(o + (need_r ? M * 4 : 0));
  l.par = o; o = align16(o + ((M + 31) / 32) * 4);
  const int nb = (N + 31) / 32, mb = (M + 31) / 32;
  l.Dblk = o; o = align16(o + nb * 4);
  l.Ddirty = o; o = align16(o + ((nb + 31) / 32) * 4);
  l.Rblk = o; o = align16(o + (need_r ? mb * 4 : 0));
  l.Rdirty = o; o = align16(o + (need_r ? ((mb + 31) / 32) * 4 : 0));
  l.tab = o; o = align16(o + (arith == kINT6 ? 256 * 2 : 0));
  l.vtotal = o;
  o = 0;
  l.C = o; o = align16(o + E * msg);
  l.P = o; o = align16(o + E * msg);
  l.etotal = o;
  l.total = l.vtotal + l.etotal;
  return l;
}

// Per-frame state layout of the flooding (CTA per frame) decoder.
struct FloodLayout {
  int C, lam, L, total;
};

inline __host__ __device__ FloodLayout flood_layout(int arith, int N, int E) {
  const int msg = arith == kINT6 ? 1 : 4;
  const int llr = arith == kINT6 ? 2 : 4;
  FloodLayout l;
  int o = 0;
  l.C = o; o = align16(o + E * msg);
  l.lam = o; o = align16(o + N * llr);
  l.L = o; o = align16(o + N * llr);
  l.total = o;
  return l;
}

// Work queue of the persistent form (layout of ldpc_work_item_t).
struct WorkItem {
  int32_t code;
  int32_t flags;
  int64_t llr_offset;  // elements
  int64_t out_offset;  // elements
  int64_t max_updates;
  uint64_t frame_index;
};
constexpr int kMaxQueueCodes = 16;

struct QueueArgs {
  DecodeArgs a;  // common parameters; llr/hard are base pointers, updates/converged per item
  GraphDesc codes[kMaxQueueCodes];
  int32_t n_codes;
  const WorkItem* items;
  int64_t n_items;
  unsigned int* head;        // persistent mode: next item (zeroed before the launch)
  int32_t persistent;        // 1: CTAs pop items until the queue is empty; 0: item = CTA index
  int32_t graph_bytes;       // staged graph area (max over codes)
  int32_t small_bytes;       // per-CTA working set (max over codes)
  int32_t smem_state_bytes;  // frame state kept in shared memory when it fits this, else global
};

// Weighted BP along a recorded schedule (decode_wbp.cu).
struct WbpArgs {
  GraphDesc g;
  const float* llr;      // [batch][N]
  int64_t batch;
  const int32_t* trace;  // [batch][T] committed edge ids
  const int64_t* counts; // [batch] updates used per frame, or null (all T)
  int64_t T;
  const float* w;        // [T] weight of update t
  float clip;
  float* llr_out;        // forward: [batch][N] final LLRs, or null
  float* c_out;          // forward: [batch][E] final C2V state, or null
  float* tape;           // forward: [batch][T] overwritten C2V values, or null
  const float* c_in;     // backward: the forward's final C2V state
  const float* tape_in;  // backward: the forward's tape
  const float* dL;       // backward: [batch][N] dloss/dL
  float* dw_frames;      // backward: [batch][T] dloss/dw per frame
  float* dw;             // backward: [T] summed over frames, or null
  float* dllr;           // backward: [batch][N] dloss/dllr, or null
  uint32_t* status;      // bit 2: a trace entry is not an edge id
  int32_t graph_smem;
  int32_t frame_bytes;
};
int wbp_state_bytes(const GraphDesc& g, bool backward);
cudaError_t launch_wbp(const WbpArgs& a, bool backward, int frames_per_cta, cudaStream_t s);

cudaError_t launch_ci_stats(const float* La, const float* Lb, int64_t count, int n_bins, unsigned long long* out,
                            int sms, cudaStream_t s);

// Systematic encoder of dual-diagonal lifted codes (encode.cu).
constexpr int kEncMaxBlocks = 4096;  // protograph cells
constexpr int kEncMaxCore = 64;
struct EncArgs {
  int32_t Z, R, C;  // lifting, protograph rows and columns
  int32_t kb;       // info block columns
  int32_t c, x, s;  // core rows, middle row of the first parity column, its shift
  int16_t B[kEncMaxBlocks];  // shifts, -1 for empty blocks (row-major R x C)
};
bool encode_plan(const int32_t* base, int R, int C, int Z, int K, EncArgs* out);
cudaError_t launch_encode(const EncArgs& a, const uint8_t* info, uint8_t* cw, int64_t batch, int sms, cudaStream_t s);

// Launchers (return a cudaError_t from the launch).
cudaError_t launch_me_queue(const QueueArgs& q, int arith, int sched, int threads, int grid, size_t smem,
                            cudaStream_t s);
cudaError_t launch_se_queue(const QueueArgs& q, int arith, int grid, size_t smem, cudaStream_t s);
// resident CTAs per SM of the queue kernels with `smem` bytes of dynamic shared memory
cudaError_t me_queue_blocks_per_sm(int arith, int sched, int threads, size_t smem, int* out);
cudaError_t se_queue_blocks_per_sm(int arith, size_t smem, int* out);
// Cluster form: plan the frame state of code g over `cs` CTAs with `avail`
// bytes of state each (false if it does not fit), and launch it (a.cl set).
bool me_cluster_plan(int arith, const GraphDesc& g, int n_p, int n_g, int cs, int64_t avail, ClusterPlan* out);
cudaError_t launch_me_cluster(const DecodeArgs& a, int arith, int sched, int threads, cudaStream_t s);
cudaError_t launch_se(const DecodeArgs& a, int arith, int sched, cudaStream_t s);
cudaError_t launch_flood(const DecodeArgs& a, int arith, cudaStream_t s);
cudaError_t launch_me(const DecodeArgs& a, int arith, int sched, cudaStream_t s);
cudaError_t launch_channel(int N, const uint8_t* punct, const uint8_t* codewords, float rate, const float* ebn0,
                           int64_t batch, uint64_t seed, uint64_t frame_offset, float* llr, int8_t* qllr, float q_step,
                           cudaStream_t s);

// Host-side view of a code handle (arrays owned by the handle).
struct CodeHostView {
  int32_t M, N, E, K, Z;
  int32_t dv_max, dc_max, maxr;
  const int32_t* tab;  // cn_ptr | e_vn | e_cn | vn_ptr | vn_e
  int32_t tab_words;
  const int32_t* qc;   // protograph view, or null
  int32_t qc_words, qc_R, qc_C, qc_nnz;
  uint32_t qc_zmul, qc_zshift;
};
bool code_host_view(const void* code, CodeHostView* out);
bool code_host_tab(const void* code, const int32_t* parts[5], int32_t sizes[5]);
void set_error_detail(const std::string& why);  // text returned by ldpc_last_error_detail()

size_t se_smem_per_frame(int arith, int sched, const GraphDesc& g);
size_t se_vregion_bytes(int arith, int sched, const GraphDesc& g);  // single-edge V region (split form)
size_t flood_smem_per_frame(int arith, const GraphDesc& g);
size_t me_smem_per_frame(int arith, int sched, const GraphDesc& g, int n_p, int n_g);  // big arrays
size_t me_smem_per_cta(const GraphDesc& g, int n_p, int n_g);  // per-CTA working set

}  // namespace ldpc
