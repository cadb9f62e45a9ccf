/*
 * ldpc.h -- C ABI of the GB300 (sm_103a) dynamic-schedule LDPC decoder.
 *
 * The library decodes binary LDPC codes by belief propagation (BP) under the
 * variable-node-centric dynamic schedules of T. C.-Y. Chang et al.,
 * "Belief-Propagation Decoding of LDPC Codes with Variable Node-Centric
 * Dynamic Schedules" (arXiv 2102.11089):
 *   - CIRBP (Algorithm 1), LMD-CIRBP (Algorithm 3),
 *   - the multi-edge ME-CIRBP (Algorithm 5) and ME-LMD-CIRBP (Algorithm 6)
 *     with the VN selection of Algorithm 4,
 * next to flooding BP (Sec. 1) and the original residual BP (Sec. 2.A).
 *
 * Conventions
 *   - Every function returns ldpc_status_t: 0 on success, a negative code on
 *     failure.  No function throws or aborts across this boundary.  A failed
 *     call leaves its outputs unspecified and records a one-line reason
 *     readable with ldpc_last_error_detail() (thread-local).
 *   - Host pointers ("host") are read during the call only; the caller keeps
 *     ownership.  Device pointers ("device") are CUDA global-memory addresses
 *     on the current device, owned by the caller, and must stay valid until the
 *     work enqueued on `cuda_stream` has finished.
 *   - `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Decode
 *     and channel calls are asynchronous on that stream; argument validation is
 *     synchronous.  Errors found by kernels (non-finite or out-of-range inputs)
 *     set per-frame flags and a per-device status word read by ldpc_sync().
 *   - Edge ids are positions in the canonical order: edges sorted by check
 *     index, then by variable index (the CSR order of H).
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ldpc_status_t;

#define LDPC_OK 0
#define LDPC_ERR_INVALID_ARG (-1)    /* NULL where not allowed, bad size or enum */
#define LDPC_ERR_DUPLICATE_EDGE (-2) /* an (m, n) pair listed twice             */
#define LDPC_ERR_INDEX_RANGE (-3)    /* check or variable index out of range    */
#define LDPC_ERR_EMPTY_NODE (-4)     /* a check or variable node without edges  */
#define LDPC_ERR_UNSUPPORTED (-5)    /* code or parameters beyond every form    */
#define LDPC_ERR_CUDA (-6)           /* a CUDA runtime call failed              */
#define LDPC_ERR_NOMEM (-7)          /* host or device allocation failed        */
#define LDPC_ERR_TIMEOUT (-8)        /* a bounded device wait gave up           */
#define LDPC_ERR_NONFINITE_LLR (-9)  /* a decode saw a NaN/Inf or out-of-range LLR */

/* schedules (ldpc_decode_params_t.schedule) */
#define LDPC_FLOODING 0     /* flooding BP: all V2C, then all C2V (Sec. 1)          */
#define LDPC_RBP 1          /* residual BP, steps 1-4 of Sec. 2.A, eq. (5)          */
#define LDPC_CIRBP 2        /* Algorithm 1 (CI metric eq. (8), threshold gamma)     */
#define LDPC_LMD_CIRBP 3    /* Algorithm 3 (latest-message-driven CIRBP)            */
#define LDPC_ME_CIRBP 4     /* Algorithm 5 (N_P edges per step, Algorithm 4)        */
#define LDPC_ME_LMD_CIRBP 5 /* Algorithm 6                                          */
#define LDPC_LMDRBP 6       /* Algorithm 2 (latest-message-driven RBP)              */
#define LDPC_SLMDRBP 7      /* Algorithm 2 without line 10 (simplified LMDRBP)      */

/* arithmetic (ldpc_decode_params_t.arith) */
#define LDPC_FP32_SUMPRODUCT 0 /* eq. (2) in FP32; input LLRs are float          */
#define LDPC_INT6_MINSUM 1     /* min-sum (Sec. 5) on 6-bit integer LLRs (int8)  */

/* execution forms (ldpc_decode_params_t.form) */
#define LDPC_FORM_AUTO 0   /* pick by code size                                   */
#define LDPC_FORM_SMEM 1   /* frame state in shared memory (warp or CTA / frame)  */
#define LDPC_FORM_GLOBAL 2 /* frame state in device global memory (large codes)   */
#define LDPC_FORM_CLUSTER 3 /* multi-edge: frame state spread over the shared memory
                             of a thread-block cluster (large codes)          */
#define LDPC_FORM_SPLIT 4   /* single-edge: VN- and check-sized arrays in shared
                             memory, the edge arrays in global memory (L2)    */

/* per-frame flag bits written to `converged` */
#define LDPC_FRAME_CONVERGED 1u /* final hard decision satisfies every check      */
#define LDPC_FRAME_BAD_INPUT 2u /* non-finite / out-of-range LLR: frame not decoded */

typedef struct ldpc_code ldpc_code_t;

typedef struct {
    int32_t n_checks;      /* M                                                  */
    int32_t n_vars;        /* N (all variable nodes, punctured ones included)    */
    int64_t n_edges;       /* E = number of h_mn = 1                             */
    int32_t k_info;        /* information bits per frame used for throughput     */
    int32_t n_punctured;   /* variable nodes flagged as not transmitted          */
    int32_t max_vn_degree; /* max |M(n)|                                         */
    int32_t max_cn_degree; /* max |N(m)|                                         */
    int32_t max_two_hop;   /* max over n of sum_{m in M(n)} |N(m)|               */
    int32_t qc_lifting;    /* Z when kernels use the protograph view of a code
                              built by ldpc_code_build_qc (graph neighbours computed
                              from the circulant shifts), else 0                  */
} ldpc_code_info_t;

typedef struct {
    int32_t schedule;       /* LDPC_FLOODING .. LDPC_SLMDRBP                      */
    int32_t arith;          /* LDPC_FP32_SUMPRODUCT or LDPC_INT6_MINSUM           */
    double gamma;           /* CIRBP threshold on D (Alg. 1 line 5), in [0, 1)    */
    int32_t n_p;            /* multi-edge: VNs updated per step (N_P, Sec. 6),
                               1..384                                             */
    int32_t n_g;            /* multi-edge: CI groups of Algorithm 4 (N_G)         */
    int64_t max_updates;    /* budget in committed C2V messages (E = 1 iteration,
                               Sec. 2.A); flooding uses whole iterations only     */
    int64_t check_interval; /* syndrome checked at 0 updates and whenever the
                               count crosses a multiple of this (0 = never)       */
    float llr_clip;         /* FP32: V2C inputs and C2V outputs clipped to +-this,
                               in (0, 1e4]; the multi-edge schedules keep the
                               sums L~ in fixed point with 2^-k resolution,
                               k = min(24, 29 - floor(log2(dv_max * llr_clip))) */
    float q_step;           /* INT6: LLR value of one quantisation step (Delta)   */
    uint64_t seed;          /* Algorithm 4 random fill (Philox4x32-10 key)         */
    uint64_t frame_offset;  /* global index of frame 0 of this batch (Philox ctr)  */
    int32_t form;           /* LDPC_FORM_*                                        */
    int32_t tune;           /* launch-shape hints (0 = library defaults), set by the
                               project's autotuner (paper_2102_11089_gb300.autotune):
                               bits 0-1 CTA size of the multi-edge kernels (1 = 256,
                               2 = 512 threads); bits 2-3 frames (warps) per CTA of
                               the single-edge kernels in shared memory (1 = 2,
                               2 = 4, 3 = 8, fewer when they do not fit); bits 4-5
                               frame state of the queue form (0 = shared memory for
                               codes whose state fits two CTAs per SM, 1 = three,
                               2 = one, 3 = global memory only); bits 6-7 CTAs per
                               cluster of the cluster form (0 = smallest that fits,
                               1 = 4, 2 = 8, 3 = 16); bit 8 single-edge state in
                               global memory (as LDPC_FORM_GLOBAL); other bits 0    */
} ldpc_decode_params_t;

/* One frame of the work queue of ldpc_decode_queue. */
typedef struct {
    int32_t code;          /* index into the call's array of codes               */
    int32_t flags;         /* must be 0                                          */
    int64_t llr_offset;    /* element offset of the frame's N LLRs in `llr`      */
    int64_t out_offset;    /* element offset of the frame's N decisions in `hard` */
    int64_t max_updates;   /* budget of this frame (committed C2V messages)      */
    uint64_t frame_index;  /* global frame index (Algorithm 4's Philox counter)  */
} ldpc_work_item_t;

#define LDPC_QUEUE_STATIC 0     /* one CTA (single-edge: one warp) per item         */
#define LDPC_QUEUE_PERSISTENT 1 /* resident CTAs take items until the queue is empty */

/* Name of a status code (static string). */
const char *ldpc_status_string(ldpc_status_t status);

/* One-line description of the last failure on this thread ("" if none). */
const char *ldpc_last_error_detail(void);

/* Fill `p` with the defaults: LMD-CIRBP, FP32, gamma 0.1 (Sec. 5.A), N_P 16,
 * N_G 16, budget 0 (caller must set), check_interval 1, llr_clip 25,
 * q_step 0.5, seed 0, frame_offset 0, form AUTO. */
ldpc_status_t ldpc_default_params(ldpc_decode_params_t *p);

/* Build a code from the edge list of H (Sec. 2.A: h_mn = 1 <=> edge (m, n)).
 * check_idx, var_idx : host int32[n_edges], 0 <= check < n_checks, 0 <= var < n_vars
 * punctured          : host uint8[n_vars] or NULL; nonzero = not transmitted
 *                      (the 5G NR codes of Sec. 5 puncture their first 2Z VNs)
 * k_info             : information bits per frame (> 0)
 * out                : receives the handle; the library copies every array.
 * Errors: INVALID_ARG (NULL arrays, sizes <= 0), INDEX_RANGE, DUPLICATE_EDGE,
 * EMPTY_NODE (every check and variable needs an edge), NOMEM.
 * Host only: no device memory is touched until the first decode on a device. */
ldpc_status_t ldpc_code_create(const int32_t *check_idx, const int32_t *var_idx, int64_t n_edges,
                               int32_t n_checks, int32_t n_vars, const uint8_t *punctured,
                               int32_t k_info, ldpc_code_t **out);

/* Seeded random (dv, dc)-regular code (the regular Tanner graphs of Sec. 2.A;
 * the (3,6) workload of the small experiments).  dv sockets per variable and dc
 * per check; the check sockets are shuffled (Fisher-Yates on SplitMix64 with the
 * given seed) and matched to the variable sockets in order; double edges, and
 * with girth6 != 0 the 4-cycles, are removed by seeded swaps of the check
 * endpoints of two edges (degrees are kept).  Deterministic for a seed.
 * n_checks = n dv / dc; k_info <= 0 takes the design value n - n_checks.
 * Host-side only.  Errors: INVALID_ARG (n dv not a multiple of dc, degrees
 * outside 1..32 or larger than the other side, n > 2^22), UNSUPPORTED (the
 * double edges / 4-cycles could not be removed in 200,000 trials), NOMEM. */
ldpc_status_t ldpc_code_build_regular(int32_t n, int32_t dv, int32_t dc, uint64_t seed, int32_t girth6,
                                      int32_t k_info, ldpc_code_t **out);

/* Build a quasi-cyclic code by circulant lifting of a protograph.
 * base       : host int32[rows * cols], row-major; -1 = zero block, s >= 0 =
 *              Z x Z circulant whose row z has its one in column (z + s) mod Z,
 *              i.e. edges (r Z + z, c Z + (z + s) mod Z) for z = 0..Z-1
 * punct_cols : host uint8[cols] or NULL; nonzero = every VN of that column punctured
 * k_info     : information bits per frame (> 0)
 * Errors as ldpc_code_create, plus INVALID_ARG for s >= Z or Z <= 0. */
ldpc_status_t ldpc_code_build_qc(const int32_t *base, int32_t rows, int32_t cols, int32_t Z,
                                 const uint8_t *punct_cols, int32_t k_info, ldpc_code_t **out);

/* Release a code and its device copies.  NULL is accepted. */
ldpc_status_t ldpc_code_destroy(ldpc_code_t *code);

/* Sizes and degree statistics of a code. */
ldpc_status_t ldpc_code_info(const ldpc_code_t *code, ldpc_code_info_t *out);

/* The canonical edge list: check_out, var_out are host int32[n_edges]
 * receiving edge e = (check_out[e], var_out[e]); used to decode traces. */
ldpc_status_t ldpc_code_edges(const ldpc_code_t *code, int32_t *check_out, int32_t *var_out);

/* BPSK/AWGN channel (Sec. 2.A, Sec. 5) for the all-zero codeword: x = +1,
 * y = 1 + sigma w, N0/2 = sigma^2 = 1 / (2 R 10^(EbN0/10)) with R = k_info / N_tx
 * (N_tx = unpunctured VNs), LLR lambda = 2 y / sigma^2, punctured VNs 0.
 * w: Box-Muller on Philox4x32-10 (key = seed, counter = (n / 4, 0, frame)),
 * frame = frame_offset + b; VNs 4k..4k+3 share one Philox block.
 * ebn0_db : device float[batch]       llr  : device float[batch][n_vars]
 * qllr    : device int8[batch][n_vars] or NULL: clamp(rint(lambda/q_step), -31, 31)
 * Errors: INVALID_ARG, CUDA. */
ldpc_status_t ldpc_awgn_llr(const ldpc_code_t *code, const float *ebn0_db, int64_t batch,
                            uint64_t seed, uint64_t frame_offset, float *llr, int8_t *qllr,
                            float q_step, void *cuda_stream);

/* As ldpc_awgn_llr for arbitrary codewords: x = 1 - 2c for the bits c of
 * `codewords` (device uint8[batch][n_vars], 0/1; NULL = the all-zero word). */
ldpc_status_t ldpc_awgn_llr_codewords(const ldpc_code_t *code, const float *ebn0_db, int64_t batch,
                                      uint64_t seed, uint64_t frame_offset, const uint8_t *codewords,
                                      float *llr, int8_t *qllr, float q_step, void *cuda_stream);

/* Systematic encoder (not a step of the paper's decoders: it lets the channel
 * send codewords other than the all-zero word).  For codes built by
 * ldpc_code_build_qc whose k_info is a whole number kb of block columns and
 * whose parity part has the dual-diagonal shape of the IEEE 802.11 / 5G NR
 * cores: first parity block column with shift s in rows 0 and c-1 and shift 0
 * in one middle row, a shift-0 staircase over the next c-1 columns, then one
 * identity column per remaining row.  codeword = info bits | parity bits.
 * info      : device uint8[batch][k_info] (bit 0 of each byte)
 * codewords : device uint8[batch][n_vars] (0/1)
 * Errors: INVALID_ARG, UNSUPPORTED (other codes, more than 4096 protograph
 * cells), NOMEM, CUDA. */
ldpc_status_t ldpc_encode(const ldpc_code_t *code, const uint8_t *info, int64_t batch, uint8_t *codewords,
                          void *cuda_stream);

/* Decode `batch` independent frames.
 * llr       : device [batch][n_vars]; float for FP32, int8 in [-31, 31] for INT6
 * params    : host; schedule, arithmetic and budget (see ldpc_decode_params_t)
 * hard      : device uint8[batch][n_vars] or NULL: bsgn(L_n), 0 if L_n >= 0 (Sec. 2.A)
 * updates   : device int64[batch] or NULL: committed C2V messages at the stop
 * converged : device uint8[batch] or NULL: LDPC_FRAME_* flags
 * trace     : device int32[batch][max_updates] or NULL: committed edge id per
 *             update (multi-edge: each step's ids in ascending VN order);
 *             entries past `updates` are left untouched; flooding writes none
 * llr_out   : device float[batch][n_vars] or NULL: final total LLR L_n, eq. (3)
 *             (INT6: the integer value)
 * Stops at a zero syndrome (checked per check_interval) or at the budget.
 * Execution form (params->form = LDPC_FORM_AUTO): frame state in shared
 * memory when it fits one CTA (single-edge frames: when shared memory holds
 * at least eight per SM, else global memory; the split form only on request);
 * else, for the multi-edge schedules in 6-bit mode or with n_p >= 128 and a batch
 * of at most twice the resident clusters (SMs / cluster size), spread over the
 * shared memory of a thread-block cluster (the smallest of 2, 4, 8 or 16 CTAs
 * that holds it and can be resident); else global memory.  A cluster size in
 * tune bits 6-7 selects the cluster form whenever it can run.  The form never
 * changes a result.
 * Errors: INVALID_ARG, UNSUPPORTED (no execution form fits; a check degree
 * above 32, or a variable degree above 32 for the dynamic schedules;
 * LDPC_FORM_CLUSTER with a single-edge or flooding schedule), CUDA, NOMEM. */
ldpc_status_t ldpc_decode(const ldpc_code_t *code, const void *llr, int64_t batch,
                          const ldpc_decode_params_t *params, uint8_t *hard, int64_t *updates,
                          uint8_t *converged, int32_t *trace, float *llr_out, void *cuda_stream);

/* Outputs of ldpc_decode_ex: every pointer is a device pointer or NULL.  The
 * first five are those of ldpc_decode; the others expose the decoder's final
 * message state and its fallback count, for checks against a reference
 * decoder and for the statistics of Sec. 3.A / Sec. 5.A.
 * c2v_out   : float[batch][n_edges]: final committed C2V messages L^C (the terms
 *             of eq. 3), edge ids as in ldpc_code_edges (INT6: integer values)
 * pre_out   : float[batch][n_edges]: final precomputed C2V messages L~^C of
 *             eq. (2) (dynamic schedules only; flooding keeps none)
 * fallbacks : int64[batch]: CIRBP updates whose edge came from the residual
 *             fallback of Alg. 1 line 6 (D_{n*} < gamma); 0 for the other
 *             schedules.  fallbacks / updates is the kappa of Sec. 5.A. */
typedef struct {
    uint8_t *hard;
    int64_t *updates;
    uint8_t *converged;
    int32_t *trace;
    float *llr_out;
    float *c2v_out;
    float *pre_out;
    int64_t *fallbacks;
} ldpc_decode_outputs_t;

/* ldpc_decode with the extended outputs above (out may not be NULL).  Same
 * arguments, forms and errors as ldpc_decode; pre_out with LDPC_FLOODING is
 * INVALID_ARG. */
ldpc_status_t ldpc_decode_ex(const ldpc_code_t *code, const void *llr, int64_t batch,
                             const ldpc_decode_params_t *params, const ldpc_decode_outputs_t *out,
                             void *cuda_stream);

/* Decode a work queue of frames from up to 16 codes lifted from protographs
 * (ldpc_code_build_qc), each frame with its own budget; the persistent form of
 * the batched decoder.  In LDPC_QUEUE_PERSISTENT mode one launch of resident
 * CTAs takes items through an atomic head counter, retires each frame at its
 * syndrome stop (or budget) and takes the next, whatever its code; a code's
 * protograph view is staged in shared memory when it changes.  In
 * LDPC_QUEUE_STATIC mode the launch has one CTA per item (the plain per-batch
 * form).  Schedules: LDPC_LMD_CIRBP, LDPC_ME_CIRBP, LDPC_ME_LMD_CIRBP.
 * codes   : host array of n_codes handles (1..16), each with a protograph view
 * items   : device ldpc_work_item_t[n_items]
 * llr     : device base of the LLR rows (float, or int8 for INT6)
 * hard    : device base of the decision rows, or NULL
 * updates : device int64[n_items] or NULL    converged : device uint8[n_items] or NULL
 * params  : as ldpc_decode (max_updates unused: each item carries its budget;
 *           form ignored; tune bits 0-1 and 4-5 apply)
 * The call is asynchronous and allocates only stream-ordered memory (the head
 * counter and global state slots, cudaMallocAsync / cudaFreeAsync on `stream`);
 * once every code has been used on the device (first call), it can be
 * recorded into a CUDA graph.
 * Offsets are not checked against the buffers (the caller sizes them); an
 * item whose code index is outside 0..n_codes-1 is not decoded: its
 * converged flag is LDPC_FRAME_BAD_INPUT, its updates 0, and the next
 * ldpc_sync returns LDPC_ERR_INVALID_ARG.
 * Errors: INVALID_ARG, UNSUPPORTED (a code without protograph view, schedule,
 * degrees, more than 2^31 - 2^20 items), CUDA, NOMEM. */
ldpc_status_t ldpc_decode_queue(const ldpc_code_t *const *codes, int32_t n_codes, const ldpc_work_item_t *items,
                                int64_t n_items, const void *llr, const ldpc_decode_params_t *params,
                                uint8_t *hard, int64_t *updates, uint8_t *converged, int32_t mode,
                                void *cuda_stream);

/* Decode like ldpc_decode, but without allocating any memory.  The paper has
 * no counterpart: this is a service of the library, not a step of the method.
 *
 * Who needs it: callers that must not allocate at the moment they decode --
 * real-time loops that must not enter the CUDA allocator (it can block on the
 * device or on locks for an unbounded time), processes whose device memory is
 * handed out up front to another allocator or capped by a fixed budget, and
 * plug-ins running inside a host application that owns every allocation.
 * ldpc_decode allocates the per-frame
 * state slots of its global-memory form and uploads a code on its first use
 * on a device; this entry point calls no cudaMalloc, cudaFree or other
 * allocating routine.  Instead it always uses the global-memory form on one
 * fixed device array of 32 MiB (declared static in the library, so every GPU
 * on which the library is loaded holds it until the process exits).  Each
 * call first copies the code's graph tables from the handle into the array
 * (the protograph view of a lifted code is a few KB), then runs the decode
 * with its frame-state slots after them.
 *
 * Arguments, outputs and results are those of ldpc_decode (params->form is
 * ignored).  Limits and errors: LDPC_ERR_UNSUPPORTED when the graph tables
 * plus one state slot (or, for the single-edge schedules, eight slots) do
 * not fit in the 32 MiB; fewer slots than ldpc_decode would use otherwise.
 * The first call on a device resolves the array's device address on that
 * device (it must be the current device); make that first call before any
 * stream capture.  Every call shares the one array, which keeps the contents
 * the last call left: the kernels initialise all state they read, and the
 * call clears its status word.  Calls that overlap on the GPU (on different
 * streams, or from different threads) race on the array.  Non-finite or
 * out-of-range LLRs are flagged per frame in `converged` only; ldpc_sync does
 * not report them for this entry point. */
ldpc_status_t ldpc_decode_noalloc(const ldpc_code_t *code, const void *llr, int64_t batch,
                                  const ldpc_decode_params_t *params, uint8_t *hard, int64_t *updates,
                                  uint8_t *converged, int32_t *trace, float *llr_out, void *cuda_stream);

/* Weighted BP along a recorded schedule, and its adjoint.  Not a step of the
 * paper: the differentiable decoder built on its schedules.  A decode with
 * `trace` records the edge committed at each update; the weighted decoder
 * replays that schedule in FP32 with one weight per update: update t commits
 * C[e_t] <- w[t] * P_t, P_t the C2V of eq. (2) (inputs and result clipped to
 * +-llr_clip) from the state before the update, and returns
 * L_n = lambda_n + sum_{m in M(n)} C[m->n] (eq. 3).  With unit weights this is
 * the decoder's own message passing; the selection itself is not replayed.
 * llr       : device float[batch][n_vars] channel LLRs
 * trace     : device int32[batch][T] edge ids (rows of an ldpc_decode trace)
 * counts    : device int64[batch] updates to replay per frame (<= T), or NULL (T)
 * weights   : device float[T]
 * llr_out   : device float[batch][n_vars] final L, or NULL
 * c_out     : device float[batch][n_edges] final C2V state, or NULL
 * tape      : device float[batch][T] value each update overwrote, or NULL
 * Frame state lives in shared memory (one warp per frame).  Errors:
 * INVALID_ARG, UNSUPPORTED (check degree > 32, or a frame's state larger than
 * one CTA's shared memory), CUDA.  A trace entry outside [0, n_edges) stops
 * that frame and makes the next ldpc_sync return LDPC_ERR_INVALID_ARG. */
ldpc_status_t ldpc_wbp_forward(const ldpc_code_t *code, const float *llr, int64_t batch, const int32_t *trace,
                               const int64_t *counts, int64_t T, const float *weights, float llr_clip,
                               float *llr_out, float *c_out, float *tape, void *cuda_stream);

/* Adjoint of ldpc_wbp_forward for a loss of the final LLRs: walks the updates
 * backwards from the forward's final state, restoring each overwritten C2V
 * value from the tape (no recomputation).
 * c_final, tape : the forward's c_out and tape (device)
 * dL        : device float[batch][n_vars] dloss/dL
 * dw_frames : device float[batch][T] dloss/dw[t] per frame (required)
 * dw        : device float[T] the same summed over frames, or NULL
 * dllr      : device float[batch][n_vars] dloss/dllr, or NULL
 * Same other arguments and errors as ldpc_wbp_forward. */
ldpc_status_t ldpc_wbp_backward(const ldpc_code_t *code, const float *llr, int64_t batch, const int32_t *trace,
                                const int64_t *counts, int64_t T, const float *weights, float llr_clip,
                                const float *c_final, const float *tape, const float *dL, float *dw_frames,
                                float *dw, float *dllr, void *cuda_stream);

/* Counters of the CI metric's Properties 1 and 2 (Sec. 3.A), for the
 * all-zero codeword: for each of `count` pairs (L, L~) -- a VN's current and
 * precomputed total LLR, e.g. consecutive flooding iterations -- bin
 * D = |p0(L) - p0(L~)| (eq. 8) by b = min(floor(D * n_bins), n_bins - 1) and
 * count per bin: [0] L >= 0 (decision correct), [1] L < 0, [2] L < 0 and
 * L~ >= L, [3] L < 0 and L~ < L.  Cumulated from the top bin, [0]/[1] is the
 * empirical J(gamma) and [2]/[3] F(gamma) at gamma = b / n_bins.
 * llr_now, llr_pre : device float[count]
 * counts           : device uint64[n_bins][4], overwritten (stream-ordered)
 * Errors: INVALID_ARG (n_bins outside 1..1024), CUDA. */
ldpc_status_t ldpc_ci_stats(const float *llr_now, const float *llr_pre, int64_t count, int32_t n_bins,
                            uint64_t *counts, void *cuda_stream);

/* Wait for `cuda_stream` and return the device status accumulated by decode
 * calls on the current device since the previous ldpc_sync (the status word
 * is then cleared): LDPC_OK, LDPC_ERR_NONFINITE_LLR, LDPC_ERR_TIMEOUT,
 * LDPC_ERR_INVALID_ARG (a queue item with a bad code index) or LDPC_ERR_CUDA
 * for a failed stream. */
ldpc_status_t ldpc_sync(void *cuda_stream);

/* Shared-memory read stream: the measured peak against which the decoders'
 * shared-memory traffic is compared (their frame state lives in shared
 * memory).  The paper has no counterpart; it is a measurement aid.  Launches
 * `blocks` CTAs of `threads` threads (a multiple of 32, at most 1024) on
 * `cuda_stream`; each thread issues `iters` x 4 conflict-free 128-bit loads
 * from a 32 KB shared array and writes one folded word to sink[block *
 * threads + thread] (device uint32, caller-owned).  *bytes (host, may be NULL)
 * receives the bytes read: blocks x threads x iters x 64.  Time it with events
 * on the same stream.  Errors: INVALID_ARG, CUDA. */
ldpc_status_t ldpc_smem_stream(int32_t blocks, int32_t threads, int32_t iters, uint32_t *sink, int64_t *bytes,
                               void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_GB300_H */
