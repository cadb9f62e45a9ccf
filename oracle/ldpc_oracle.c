/*
 * ldpc_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of the decoding schedules of
 * T. C.-Y. Chang, P.-H. Wang, J.-J. Weng, I-H. Lee and Y. T. Su,
 * "Belief-Propagation Decoding of LDPC Codes with Variable Node-Centric Dynamic
 * Schedules" (arXiv 2102.11089), in FP64 (sum-product) or exact integers
 * (6-bit min-sum).  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file.  It shares no code, header, table or
 * constant generator with the CUDA library; it reads the code as an edge list
 * and the channel LLRs as arrays.
 *
 * Every quantity is evaluated from its definition, in a fixed canonical order:
 * edge ids are the positions in (check, variable)-sorted order, N(m) is walked
 * in ascending variable index and M(n) in ascending check index.  In
 * "definitional" mode every derived array is recomputed after each step; in
 * the default incremental mode only the set the algorithms name is recomputed,
 * each value again from scratch (never by adding a delta), so the two modes
 * agree bit for bit.
 *
 * Readings of points the paper leaves open (each is a parameter or a fixed
 * rule here and is listed in the design notes of the repository):
 *  R1  After a commit, D of the updated variable node is refreshed too
 *      (it depends on L_{n*}); flag `stale_dn` keeps it stale instead.
 *  R2  Every argmax breaks ties toward the lowest variable index / edge id.
 *  R3  Algorithm 3 re-selects the check node (its line 5) for the new target.
 *  R4  Algorithm 6 uses, for each selected p, the check m*_p committed for p.
 *  R5  "In parallel" (Algorithms 5, 6) is a two-phase step: all selections on
 *      the pre-step state, all commits, then one refresh of everything touched.
 *  R6  Algorithm 4's random choice takes the members of the fill group with the
 *      smallest keys (key of n = word n mod 4 of Philox4x32-10 with key = seed,
 *      counter = (n / 4, step, frame)); equal keys go to the lower index.
 *  R7  Degree-1 rule (Sec. 5.A): if d_v(n*) = 1 the LMD candidate set is
 *      N(m*)\n*; if the candidate set is still empty, the global argmax of D.
 *      For LMDRBP the candidates are the edges of m* to N(m*)\n*, and an
 *      empty set falls back to the global residual argmax (its line 3).
 *  R8  Syndrome checked at update count 0 and whenever the count crosses a
 *      multiple of `check_interval` (0 = never); budget in edge updates.
 *  R9  Messages are clipped to +-llr_clip in FP mode (V2C before the tanh rule,
 *      and the C2V result); 6-bit mode saturates V2C to +-31 before min-sum.
 *  R10 Integer CI: D = |T[c(L)] - T[c(L~)]|, c = clamp to [-127,127],
 *      T[q] = round(32767 tanh(q*step/2)); D ranges over [0, 65534] and stands
 *      for 65534 * |p0(L) - p0(L~)|.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FLOODING 0
#define ORC_RBP 1
#define ORC_CIRBP 2
#define ORC_LMD_CIRBP 3
#define ORC_ME_CIRBP 4
#define ORC_ME_LMD_CIRBP 5
#define ORC_LMDRBP 6
#define ORC_SLMDRBP 7

#define ORC_ARITH_FP 0
#define ORC_ARITH_INT 1

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_DUP -2
#define ORC_ERR_RANGE -3
#define ORC_ERR_EMPTY -4
#define ORC_ERR_NOMEM -7

/* counters per frame (Tables I and II of the paper) */
enum {
    CT_PROP = 0,   /* C2V propagations (= committed updates)            */
    CT_V2C,        /* V2C updates                                       */
    CT_C2V_PRE,    /* C2V pre-updates (precomputed message + residual)   */
    CT_CI,         /* CI updates of the refreshed 2-hop set              */
    CT_CI_EXTRA,   /* CI refresh of the updated VN itself (reading R1)   */
    CT_CMP,        /* real-number comparisons for residual / CI argmax   */
    CT_ICMP,       /* integer comparisons inside Algorithm 4             */
    CT_STEPS,      /* schedule steps                                     */
    CT_SELFCHECK,  /* mismatches between incremental and definitional    */
    CT_FALLBACK,   /* CIRBP steps with D_{n*} < gamma                    */
    CT_N
};

typedef struct {
    int32_t schedule, arith;
    double gamma;
    int32_t n_p, n_g;
    int64_t max_updates;
    int64_t check_interval;
    double llr_clip;
    double q_step;
    uint64_t seed;
    uint64_t frame_offset;
    int32_t definitional;
    int32_t stale_dn;
    int32_t selfcheck;
    int32_t stop_on_quiescence;
} orc_params;

/* ------------------------------------------------------------------------ */
/* Tanner graph (Sec. 2.A): edges (m, n) with h_mn = 1                        */

typedef struct {
    int M, N, E;
    int *cn_ptr; /* M+1 : edges of check m are cn_ptr[m] .. cn_ptr[m+1]-1 */
    int *e_vn;   /* E   : variable node of edge e                        */
    int *e_cn;   /* E   : check node of edge e                           */
    int *vn_ptr; /* N+1                                                  */
    int *vn_e;   /* E   : edge ids of variable n, ascending check index  */
} og_t;

static int cmp_pair(const void *a, const void *b) {
    const int *x = (const int *)a, *y = (const int *)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
    return 0;
}

static void og_free(og_t *g) {
    free(g->cn_ptr); free(g->e_vn); free(g->e_cn); free(g->vn_ptr); free(g->vn_e);
    memset(g, 0, sizeof(*g));
}

static int og_build(og_t *g, const int32_t *chk, const int32_t *var, int64_t E, int M, int N) {
    memset(g, 0, sizeof(*g));
    if (E <= 0 || M <= 0 || N <= 0 || E > 0x7fffffff) return ORC_ERR_ARG;
    int *pairs = (int *)malloc(sizeof(int) * 2 * (size_t)E);
    if (!pairs) return ORC_ERR_NOMEM;
    for (int64_t e = 0; e < E; e++) {
        if (chk[e] < 0 || chk[e] >= M || var[e] < 0 || var[e] >= N) { free(pairs); return ORC_ERR_RANGE; }
        pairs[2 * e] = chk[e];
        pairs[2 * e + 1] = var[e];
    }
    qsort(pairs, (size_t)E, 2 * sizeof(int), cmp_pair);
    for (int64_t e = 1; e < E; e++)
        if (pairs[2 * e] == pairs[2 * e - 2] && pairs[2 * e + 1] == pairs[2 * e - 1]) { free(pairs); return ORC_ERR_DUP; }
    g->M = M; g->N = N; g->E = (int)E;
    g->cn_ptr = (int *)calloc((size_t)M + 1, sizeof(int));
    g->vn_ptr = (int *)calloc((size_t)N + 1, sizeof(int));
    g->e_vn = (int *)malloc(sizeof(int) * (size_t)E);
    g->e_cn = (int *)malloc(sizeof(int) * (size_t)E);
    g->vn_e = (int *)malloc(sizeof(int) * (size_t)E);
    if (!g->cn_ptr || !g->vn_ptr || !g->e_vn || !g->e_cn || !g->vn_e) { free(pairs); og_free(g); return ORC_ERR_NOMEM; }
    for (int e = 0; e < g->E; e++) {
        g->e_cn[e] = pairs[2 * e];
        g->e_vn[e] = pairs[2 * e + 1];
        g->cn_ptr[pairs[2 * e] + 1]++;
        g->vn_ptr[pairs[2 * e + 1] + 1]++;
    }
    free(pairs);
    for (int m = 0; m < M; m++) g->cn_ptr[m + 1] += g->cn_ptr[m];
    for (int n = 0; n < N; n++) g->vn_ptr[n + 1] += g->vn_ptr[n];
    for (int m = 0; m < M; m++) if (g->cn_ptr[m + 1] == g->cn_ptr[m]) { og_free(g); return ORC_ERR_EMPTY; }
    for (int n = 0; n < N; n++) if (g->vn_ptr[n + 1] == g->vn_ptr[n]) { og_free(g); return ORC_ERR_EMPTY; }
    int *fill = (int *)calloc((size_t)N, sizeof(int));
    if (!fill) { og_free(g); return ORC_ERR_NOMEM; }
    for (int e = 0; e < g->E; e++) { /* ascending e == ascending check index */
        int n = g->e_vn[e];
        g->vn_e[g->vn_ptr[n] + fill[n]++] = e;
    }
    free(fill);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition     */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random key of variable n for Algorithm 4's fill at a given step: word     */
/* (n mod 4) of Philox4x32-10 with counter (n / 4, step, frame), key = seed.  */
static uint32_t fill_key(uint32_t n, uint32_t step, uint64_t frame, uint64_t seed) {
    uint32_t ctr[4] = {n / 4u, step, (uint32_t)frame, (uint32_t)(frame >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return o[n % 4u];
}

/* ------------------------------------------------------------------------ */
/* Channel (Sec. 2.A and Sec. 5): BPSK x = 1 - 2u with u = 0, y = x + w,      */
/* w ~ N(0, sigma^2), N0/2 = sigma^2, sigma^2 = 1/(2 R Eb/N0), LLR 2y/sigma^2  */
/* Noise: Box-Muller on Philox words; VN 4k+i uses block k, counter          */
/* (k, 0, frame), key = seed; uniforms u = (x + 1/2) 2^-32; pairs (w0,w1),   */
/* (w2,w3) give r = sqrt(-2 ln u_a), z = r cos(2 pi u_b), r sin(2 pi u_b).    */

void orc_awgn_llr(int N, const uint8_t *punct, double rate, const double *ebn0_db, int64_t batch,
                  uint64_t seed, uint64_t frame_offset, double *llr) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t b = 0; b < batch; b++) {
        double sigma2 = 1.0 / (2.0 * rate * pow(10.0, ebn0_db[b] / 10.0));
        double sigma = sqrt(sigma2);
        uint64_t frame = frame_offset + (uint64_t)b;
        for (int n = 0; n < N; n++) {
            int k = n / 4, i = n % 4;
            uint32_t ctr[4] = {(uint32_t)k, 0u, (uint32_t)frame, (uint32_t)(frame >> 32)};
            uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
            uint32_t o[4];
            orc_philox4x32_10(ctr, key, o);
            int pair = i / 2;
            double ua = ((double)o[2 * pair] + 0.5) / 4294967296.0;
            double ub = ((double)o[2 * pair + 1] + 0.5) / 4294967296.0;
            double r = sqrt(-2.0 * log(ua));
            double z = (i % 2 == 0) ? r * cos(two_pi * ub) : r * sin(two_pi * ub);
            double y = 1.0 + sigma * z;
            llr[b * N + n] = (punct && punct[n]) ? 0.0 : 2.0 * y / sigma2;
        }
    }
}

/* 6-bit quantiser q = clamp(rint(lam/step), -31, 31); the rounding decision  */
/* is taken in float32, the precision of the channel kernel.                  */
void orc_quantize(const float *lam, int64_t count, float step, int8_t *q) {
    for (int64_t i = 0; i < count; i++) {
        float v = rintf(lam[i] / step);
        if (v > 31.f) v = 31.f;
        if (v < -31.f) v = -31.f;
        q[i] = (int8_t)v;
    }
}

/* ------------------------------------------------------------------------ */
/* One frame                                                                */

typedef struct {
    const og_t *g;
    const orc_params *pr;
    uint64_t frame;
    double *lam, *C, *P, *L, *Lt, *D;
    double T[255];    /* integer-mode table of round(32767 tanh(q step/2)) */
    double gamma;     /* threshold in the units of D                       */
    int64_t count;    /* committed edge updates so far                     */
    int64_t step;
    int64_t *ctr;     /* CT_N counters                                     */
    int32_t *trace;   /* [max_updates] or NULL                             */
    double *gap;      /* [max_updates] or NULL                             */
    /* scratch */
    int *mark_cn, *mark_vn, *list_a, *list_b;
    double *snapshot;
} fr_t;

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* eq. (1): L^V_{n->m} = lambda_n + sum_{m' in M(n)\m} L^C_{m'->n} (ascending m') */
static double v2c(const fr_t *f, int e) {
    const og_t *g = f->g;
    int n = g->e_vn[e];
    double v = f->lam[n];
    for (int k = g->vn_ptr[n]; k < g->vn_ptr[n + 1]; k++) {
        int e2 = g->vn_e[k];
        if (e2 != e) v += f->C[e2];
    }
    return v;
}

/* eq. (2): L~^C_{m->n} = 2 atanh( prod_{n' in N(m)\n} tanh(L^V_{n'->m}/2) ),   */
/* or, in 6-bit mode, the min-sum approximation named in Sec. 5:              */
/* (prod sgn V) * min |V| over N(m)\n, sgn(0) = +1, V saturated to +-31.      */
static double c2v(const fr_t *f, int e) {
    const og_t *g = f->g;
    int m = g->e_cn[e];
    if (f->pr->arith == ORC_ARITH_FP) {
        double lc = f->pr->llr_clip;
        double prod = 1.0;
        for (int e2 = g->cn_ptr[m]; e2 < g->cn_ptr[m + 1]; e2++) {
            if (e2 == e) continue;
            prod *= tanh(clampd(v2c(f, e2), -lc, lc) / 2.0);
        }
        return clampd(2.0 * atanh(prod), -lc, lc);
    } else {
        double mag = 31.0, sgn = 1.0;
        for (int e2 = g->cn_ptr[m]; e2 < g->cn_ptr[m + 1]; e2++) {
            if (e2 == e) continue;
            double v = clampd(v2c(f, e2), -31.0, 31.0);
            if (v < 0) sgn = -sgn;
            if (fabs(v) < mag) mag = fabs(v);
        }
        return sgn * mag;
    }
}

/* eq. (3): L_n = lambda_n + sum_{m in M(n)} L^C_{m->n}                       */
static double total_llr(const fr_t *f, int n) {
    const og_t *g = f->g;
    double s = f->lam[n];
    for (int k = g->vn_ptr[n]; k < g->vn_ptr[n + 1]; k++) s += f->C[g->vn_e[k]];
    return s;
}

/* Sec. 2.B: precomputed LLR L~_n = lambda_n + sum_{m in M(n)} L~^C_{m->n}     */
static double pre_llr(const fr_t *f, int n) {
    const og_t *g = f->g;
    double s = f->lam[n];
    for (int k = g->vn_ptr[n]; k < g->vn_ptr[n + 1]; k++) s += f->P[g->vn_e[k]];
    return s;
}

/* eq. (8): D_n = |p0(L_n) - p0(L~_n)| with p0(L) = e^L/(1+e^L).  Written      */
/* through p0(L) - 1/2 = tanh(L/2)/2, which is exact and odd-symmetric.        */
static double ci(const fr_t *f, int n) {
    double a = f->L[n], b = f->Lt[n];
    if (f->pr->arith == ORC_ARITH_FP) return fabs(tanh(a / 2.0) - tanh(b / 2.0)) / 2.0;
    int qa = (int)clampd(a, -127, 127), qb = (int)clampd(b, -127, 127);
    return fabs(f->T[qa + 127] - f->T[qb + 127]);
}

/* eq. (4): R_{m->n} = |L~^C - L^C|                                           */
static double resid(const fr_t *f, int e) { return fabs(f->P[e] - f->C[e]); }

/* bsgn of Sec. 2.A: 0 if a >= 0 else 1                                       */
static int bsgn(double a) { return a >= 0.0 ? 0 : 1; }

static int syndrome_weight(const fr_t *f) {
    const og_t *g = f->g;
    int w = 0;
    for (int m = 0; m < g->M; m++) {
        int par = 0;
        for (int e = g->cn_ptr[m]; e < g->cn_ptr[m + 1]; e++) par ^= bsgn(f->L[g->e_vn[e]]);
        w += par;
    }
    return w;
}

static void refresh_all(fr_t *f) {
    const og_t *g = f->g;
    for (int e = 0; e < g->E; e++) f->P[e] = c2v(f, e);
    for (int n = 0; n < g->N; n++) {
        f->L[n] = total_llr(f, n);
        f->Lt[n] = pre_llr(f, n);
        f->D[n] = ci(f, n);
    }
}

/* argmax helper with lowest-index tie-break and top-2 gap (for near-ties)   */
typedef struct { int idx; double best, second; int64_t ncand; } amax_t;
static void am_init(amax_t *a) { a->idx = -1; a->best = -INFINITY; a->second = -INFINITY; a->ncand = 0; }
static void am_push(amax_t *a, int idx, double v) {
    a->ncand++;
    if (a->idx == idx) return; /* the same candidate listed twice */
    if (v > a->best || (v == a->best && idx < a->idx)) {
        if (a->idx >= 0) a->second = a->best > a->second ? a->best : a->second;
        a->best = v; a->idx = idx;
    } else if (v > a->second) {
        a->second = v;
    }
}
/* top-2 gap relative to max(1, |best|): residuals scale with message          */
/* magnitudes (up to llr_clip), CI values lie in [0, 1) and keep an absolute gap */
static double am_gap(const amax_t *a) {
    if (a->second == -INFINITY) return INFINITY;
    return (a->best - a->second) / fmax(1.0, fabs(a->best));
}
static void am_count(fr_t *f, const amax_t *a) { if (a->ncand > 0) f->ctr[CT_CMP] += a->ncand - 1; }

/* argmax over D of all VNs (Alg. 1 line 4, Alg. 3 line 4)                    */
static amax_t argmax_D_all(fr_t *f) {
    amax_t a; am_init(&a);
    for (int n = 0; n < f->g->N; n++) am_push(&a, n, f->D[n]);
    am_count(f, &a);
    return a;
}
/* argmax over R of all edges, eq. (5)                                        */
static amax_t argmax_R_all(fr_t *f) {
    amax_t a; am_init(&a);
    for (int e = 0; e < f->g->E; e++) am_push(&a, e, resid(f, e));
    am_count(f, &a);
    return a;
}
/* argmax_i R_{i->n} over i in M(n) (Alg. 1 line 8, Alg. 3 line 5)           */
static amax_t argmax_R_into(fr_t *f, int n) {
    const og_t *g = f->g;
    amax_t a; am_init(&a);
    for (int k = g->vn_ptr[n]; k < g->vn_ptr[n + 1]; k++) am_push(&a, g->vn_e[k], resid(f, g->vn_e[k]));
    am_count(f, &a);
    return a;
}

/* The refresh of Alg. 1 lines 10-13 after the commit on edge (m*, n*):       */
/* for i in M(n*)\m*: new V2C n*->i, then L~^C, R, L~_j, D_j, j in N(i)\n*.   */
static void refresh_after_commit(fr_t *f, int nstar, int estar) {
    const og_t *g = f->g;
    int mstar = g->e_cn[estar];
    for (int k = g->vn_ptr[nstar]; k < g->vn_ptr[nstar + 1]; k++) {
        int ei = g->vn_e[k];
        int i = g->e_cn[ei];
        if (i == mstar) continue;
        f->ctr[CT_V2C]++;
        for (int e = g->cn_ptr[i]; e < g->cn_ptr[i + 1]; e++) {
            if (g->e_vn[e] == nstar) continue;
            f->P[e] = c2v(f, e);
            f->ctr[CT_C2V_PRE]++;
        }
    }
    for (int k = g->vn_ptr[nstar]; k < g->vn_ptr[nstar + 1]; k++) {
        int i = g->e_cn[g->vn_e[k]];
        if (i == mstar) continue;
        for (int e = g->cn_ptr[i]; e < g->cn_ptr[i + 1]; e++) {
            int j = g->e_vn[e];
            if (j == nstar) continue;
            f->Lt[j] = pre_llr(f, j);
            f->D[j] = ci(f, j);
            f->ctr[CT_CI]++;
        }
    }
    if (!f->pr->stale_dn) {
        f->D[nstar] = ci(f, nstar);
        f->ctr[CT_CI_EXTRA]++;
    }
}

/* Alg. 1 line 9 / Alg. 3 line 6: L^C <- L~^C on edge e, update L_{n*}.       */
static void commit(fr_t *f, int e) {
    f->C[e] = f->P[e];
    f->L[f->g->e_vn[e]] = total_llr(f, f->g->e_vn[e]);
    f->ctr[CT_PROP]++;
}

static size_t state_len(const og_t *g) { return 2 * (size_t)g->E + 3 * (size_t)g->N; }
static void state_copy(const fr_t *f, double *dst) {
    const og_t *g = f->g;
    memcpy(dst, f->C, sizeof(double) * g->E);
    memcpy(dst + g->E, f->P, sizeof(double) * g->E);
    memcpy(dst + 2 * g->E, f->L, sizeof(double) * g->N);
    memcpy(dst + 2 * g->E + g->N, f->Lt, sizeof(double) * g->N);
    memcpy(dst + 2 * g->E + 2 * g->N, f->D, sizeof(double) * g->N);
}

/* After each incremental step: recompute everything by definition and       */
/* compare bit for bit (invariant P4).                                        */
static void selfcheck(fr_t *f) {
    const og_t *g = f->g;
    size_t len = state_len(g);
    double *before = f->snapshot, *after = f->snapshot + len;
    state_copy(f, before);
    refresh_all(f);
    state_copy(f, after);
    if (memcmp(before, after, sizeof(double) * len) != 0) f->ctr[CT_SELFCHECK]++;
}

static void after_step(fr_t *f) {
    if (f->pr->definitional) refresh_all(f);
    else if (f->pr->selfcheck) selfcheck(f);
}

static int should_check(const fr_t *f, int64_t before) {
    int64_t ci = f->pr->check_interval;
    if (ci <= 0) return 0;
    return (f->count / ci) > (before / ci);
}

static int quiescent(const fr_t *f) {
    for (int e = 0; e < f->g->E; e++) if (resid(f, e) != 0.0) return 0;
    return 1;
}

static void record(fr_t *f, int e, double gap) {
    if (f->trace) f->trace[f->count] = e;
    if (f->gap) f->gap[f->count] = gap;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 4: VN selection by an N_G-level uniform quantiser of D          */

static int ci_group(const fr_t *f, double d) {
    int ng = f->pr->n_g;
    int gidx;
    if (f->pr->arith == ORC_ARITH_FP) gidx = (int)floor(d * ng);
    else gidx = (int)(((int64_t)d * ng) / 65534);
    return gidx < ng - 1 ? gidx : ng - 1;
}

typedef struct { uint32_t key; int n; } kn_t;
static int cmp_kn(const void *a, const void *b) {
    const kn_t *x = (const kn_t *)a, *y = (const kn_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->n < y->n ? -1 : (x->n > y->n);
}

/* Select from the set S (flag inS[n]) at most np VNs; output ascending in    */
/* out[], returns the count; *margin receives the distance of the nearest D   */
/* to a group boundary that decides membership (FP near-tie measure).         */
static int alg4(fr_t *f, const int *inS, int np, int *out, double *margin) {
    const og_t *g = f->g;
    int ng = f->pr->n_g;
    int *cnt = (int *)calloc((size_t)ng, sizeof(int));
    int *grp = f->list_b; /* per-VN group, -1 if not in S */
    int sz = 0;
    for (int n = 0; n < g->N; n++) {
        grp[n] = -1;
        if (!inS[n]) continue;
        grp[n] = ci_group(f, f->D[n]);
        cnt[grp[n]]++;
        sz++;
    }
    /* k* = max{k : |Q(k)| <= N_P}, Q(k) = union of the k top groups (line 3). */
    /* |Q(N_G)| = |S|: when |S| <= N_P, k* = N_G at once; otherwise at most    */
    /* N_G - 1 comparisons of the running union size decide k*.               */
    int kstar = 0, q = 0;
    f->ctr[CT_ICMP]++;
    if (sz <= np) {
        kstar = ng;
        q = sz;
    } else {
        for (int k = 1; k < ng; k++) {
            if (k > 1) f->ctr[CT_ICMP]++;
            if (q + cnt[ng - k] <= np) { q += cnt[ng - k]; kstar = k; }
            else break;
        }
    }
    f->ctr[CT_ICMP]++; /* |P| < N_P (line 4) */
    int outn = 0;
    for (int n = 0; n < g->N; n++) if (grp[n] >= ng - kstar) out[outn++] = n;
    *margin = INFINITY;
    if (outn < np && kstar < ng) {
        int fill = ng - kstar - 1, need = np - outn, nc = 0;
        kn_t *c = (kn_t *)malloc(sizeof(kn_t) * (size_t)cnt[fill]);
        for (int n = 0; n < g->N; n++)
            if (grp[n] == fill) {
                c[nc].key = fill_key((uint32_t)n, (uint32_t)f->step, f->frame, f->pr->seed);
                c[nc].n = n;
                nc++;
            }
        qsort(c, (size_t)nc, sizeof(kn_t), cmp_kn);
        for (int i = 0; i < need; i++) out[outn++] = c[i].n;
        free(c);
        /* keep out[] ascending */
        for (int i = 1; i < outn; i++) {
            int v = out[i], j = i - 1;
            while (j >= 0 && out[j] > v) { out[j + 1] = out[j]; j--; }
            out[j + 1] = v;
        }
        if (f->pr->arith == ORC_ARITH_FP) {
            double b1 = (double)(ng - kstar) / ng, b2 = (double)(ng - kstar - 1) / ng;
            for (int n = 0; n < g->N; n++) {
                if (!inS[n]) continue;
                double d1 = fabs(f->D[n] - b1), d2 = fabs(f->D[n] - b2);
                if (d1 < *margin) *margin = d1;
                if (d2 < *margin) *margin = d2;
            }
        }
    }
    (void)sz;
    free(cnt);
    return outn;
}

/* ------------------------------------------------------------------------ */
/* Schedules                                                                */

static int check_stop(fr_t *f, int64_t before) {
    if (f->pr->stop_on_quiescence && quiescent(f)) return 1;
    if (should_check(f, before) && syndrome_weight(f) == 0) return 1;
    return 0;
}

/* Flooding (Sec. 1): all V2C then all C2V per iteration; one iteration     */
/* propagates E messages.                                                    */
static void run_flooding(fr_t *f) {
    const og_t *g = f->g;
    double *Cn = (double *)malloc(sizeof(double) * g->E);
    while (f->count + g->E <= f->pr->max_updates) {
        int64_t before = f->count;
        for (int e = 0; e < g->E; e++) Cn[e] = c2v(f, e);
        int changed = 0;
        for (int e = 0; e < g->E; e++) { if (Cn[e] != f->C[e]) changed = 1; f->C[e] = Cn[e]; }
        for (int n = 0; n < g->N; n++) f->L[n] = total_llr(f, n);
        f->count += g->E;
        f->ctr[CT_PROP] += g->E;
        f->ctr[CT_STEPS]++;
        if (f->pr->stop_on_quiescence && !changed) break;
        if (should_check(f, before) && syndrome_weight(f) == 0) break;
    }
    free(Cn);
    /* keep P, Lt, D consistent with the final messages for state output */
    refresh_all(f);
}

/* Original RBP (Sec. 2.A, steps 1-4)                                        */
static void run_rbp(fr_t *f) {
    while (f->count < f->pr->max_updates) {
        int64_t before = f->count;
        amax_t a = argmax_R_all(f);
        int e = a.idx, n = f->g->e_vn[e];
        record(f, e, am_gap(&a));
        commit(f, e);
        refresh_after_commit(f, n, e);
        f->count++; f->ctr[CT_STEPS]++;
        after_step(f);
        if (check_stop(f, before)) break;
    }
}

/* Algorithm 1 (CIRBP)                                                        */
static void run_cirbp(fr_t *f) {
    while (f->count < f->pr->max_updates) {
        int64_t before = f->count;
        amax_t av = argmax_D_all(f); /* line 4 */
        int n = av.idx, e;
        double gap, thr = fabs(f->D[n] - f->gamma);
        f->ctr[CT_CMP]++;            /* line 5 */
        if (f->D[n] < f->gamma) {
            amax_t ar = argmax_R_all(f); /* line 6 */
            e = ar.idx; n = f->g->e_vn[e];
            gap = fmin(thr, am_gap(&ar));
            f->ctr[CT_FALLBACK]++;
        } else {
            amax_t ar = argmax_R_into(f, n); /* line 8 */
            e = ar.idx;
            gap = fmin(fmin(am_gap(&av), thr), am_gap(&ar));
        }
        record(f, e, gap);
        commit(f, e);                 /* line 9 */
        refresh_after_commit(f, n, e); /* lines 10-13 */
        f->count++; f->ctr[CT_STEPS]++;
        after_step(f);
        if (check_stop(f, before)) break;
    }
}

/* Candidate set U(m*, n*) of Alg. 3 line 11 with the degree-1 rule (R7).    */
static amax_t lmd_next(fr_t *f, int nstar, int estar) {
    const og_t *g = f->g;
    int mstar = g->e_cn[estar];
    amax_t a; am_init(&a);
    int dv = g->vn_ptr[nstar + 1] - g->vn_ptr[nstar];
    if (dv > 1) {
        for (int k = g->vn_ptr[nstar]; k < g->vn_ptr[nstar + 1]; k++) {
            int i = g->e_cn[g->vn_e[k]];
            if (i == mstar) continue;
            for (int e = g->cn_ptr[i]; e < g->cn_ptr[i + 1]; e++)
                if (g->e_vn[e] != nstar) am_push(&a, g->e_vn[e], f->D[g->e_vn[e]]);
        }
    } else {
        for (int e = g->cn_ptr[mstar]; e < g->cn_ptr[mstar + 1]; e++)
            if (g->e_vn[e] != nstar) am_push(&a, g->e_vn[e], f->D[g->e_vn[e]]);
    }
    am_count(f, &a);
    return a;
}

/* Algorithm 3 (LMD-CIRBP)                                                    */
static void run_lmd_cirbp(fr_t *f) {
    amax_t av = argmax_D_all(f); /* line 4 */
    int n = av.idx;
    double gap_vn = am_gap(&av);
    while (f->count < f->pr->max_updates) {
        int64_t before = f->count;
        amax_t ar = argmax_R_into(f, n); /* line 5 (reading R3) */
        int e = ar.idx;
        record(f, e, fmin(gap_vn, am_gap(&ar)));
        commit(f, e);                  /* line 6 */
        refresh_after_commit(f, n, e); /* lines 7-10 */
        f->count++; f->ctr[CT_STEPS]++;
        after_step(f);
        if (check_stop(f, before)) break;
        amax_t an = lmd_next(f, n, e); /* line 11 */
        if (an.idx < 0) an = argmax_D_all(f);
        n = an.idx;
        gap_vn = am_gap(&an);
    }
}

/* Candidate edges of Alg. 2 line 9: the residuals of i -> j for            */
/* i in M(n*)\m*, j in N(i)\n* (just recomputed), or, when d_v(n*) = 1, of  */
/* m* -> j for j in N(m*)\n* (Sec. 5.A).                                     */
static amax_t lmdrbp_next(fr_t *f, int nstar, int estar) {
    const og_t *g = f->g;
    int mstar = g->e_cn[estar];
    amax_t a; am_init(&a);
    int dv = g->vn_ptr[nstar + 1] - g->vn_ptr[nstar];
    for (int k = g->vn_ptr[nstar]; k < g->vn_ptr[nstar + 1]; k++) {
        int i = g->e_cn[g->vn_e[k]];
        if (dv > 1 && i == mstar) continue;
        for (int e = g->cn_ptr[i]; e < g->cn_ptr[i + 1]; e++)
            if (g->e_vn[e] != nstar) am_push(&a, e, resid(f, e));
    }
    am_count(f, &a);
    return a;
}

/* Algorithm 2 (LMDRBP); `simplified` bypasses its line 10 (sLMDRBP).        */
static void run_lmdrbp(fr_t *f, int simplified) {
    amax_t a = argmax_R_all(f); /* line 3 */
    int e = a.idx;
    double gap = am_gap(&a);
    while (f->count < f->pr->max_updates) {
        int64_t before = f->count;
        int n = f->g->e_vn[e];
        record(f, e, gap);
        commit(f, e);                  /* line 4 */
        refresh_after_commit(f, n, e); /* lines 5-8 */
        f->count++; f->ctr[CT_STEPS]++;
        after_step(f);
        if (check_stop(f, before)) break;
        a = lmdrbp_next(f, n, e);      /* line 9 */
        if (a.idx < 0) a = argmax_R_all(f);
        e = a.idx;
        gap = am_gap(&a);
        if (!simplified) {             /* line 10: the best check into n' */
            amax_t ar = argmax_R_into(f, f->g->e_vn[e]);
            e = ar.idx;
            gap = fmin(gap, am_gap(&ar));
        }
    }
}

/* Multi-edge step shared by Algorithms 5 and 6: for every p of the selected */
/* set, m*_p = argmax R into p on the pre-step state; commit all; then one   */
/* refresh of every check that received a new V2C and every VN next to one. */
static int me_step(fr_t *f, int *sel, int nsel, int *estar, double *gap) {
    const og_t *g = f->g;
    int64_t room = f->pr->max_updates - f->count;
    if (nsel > room) nsel = (int)room; /* truncate the last step (ascending p) */
    for (int k = 0; k < nsel; k++) {
        amax_t ar = argmax_R_into(f, sel[k]);
        estar[k] = ar.idx;
        if (am_gap(&ar) < *gap) *gap = am_gap(&ar);
    }
    for (int k = 0; k < nsel; k++) f->C[estar[k]] = f->P[estar[k]];
    for (int k = 0; k < nsel; k++) f->L[sel[k]] = total_llr(f, sel[k]);
    f->ctr[CT_PROP] += nsel;
    /* checks i in M(p)\m*_p */
    int ncn = 0;
    for (int k = 0; k < nsel; k++) {
        int p = sel[k], mstar = g->e_cn[estar[k]];
        for (int t = g->vn_ptr[p]; t < g->vn_ptr[p + 1]; t++) {
            int i = g->e_cn[g->vn_e[t]];
            if (i == mstar) continue;
            f->ctr[CT_V2C]++;
            if (!f->mark_cn[i]) { f->mark_cn[i] = 1; f->list_a[ncn++] = i; }
        }
    }
    int nvn = 0;
    int *vlist = (int *)malloc(sizeof(int) * (size_t)g->N);
    for (int t = 0; t < ncn; t++) {
        int i = f->list_a[t];
        for (int e = g->cn_ptr[i]; e < g->cn_ptr[i + 1]; e++) {
            f->P[e] = c2v(f, e);
            f->ctr[CT_C2V_PRE]++;
            int j = g->e_vn[e];
            if (!f->mark_vn[j]) { f->mark_vn[j] = 1; vlist[nvn++] = j; }
        }
    }
    for (int k = 0; k < nsel; k++) if (!f->mark_vn[sel[k]]) { f->mark_vn[sel[k]] = 1; vlist[nvn++] = sel[k]; }
    for (int t = 0; t < nvn; t++) {
        int j = vlist[t];
        f->Lt[j] = pre_llr(f, j);
        f->D[j] = ci(f, j);
        f->ctr[CT_CI]++;
        f->mark_vn[j] = 0;
    }
    for (int t = 0; t < ncn; t++) f->mark_cn[f->list_a[t]] = 0;
    free(vlist);
    for (int k = 0; k < nsel; k++) {
        if (f->trace) f->trace[f->count + k] = estar[k];
        if (f->gap) f->gap[f->count + k] = *gap;
    }
    return nsel;
}

/* Algorithm 5 (ME-CIRBP)                                                     */
static void run_me_cirbp(fr_t *f) {
    const og_t *g = f->g;
    int *all = (int *)malloc(sizeof(int) * (size_t)g->N);
    int *sel = (int *)malloc(sizeof(int) * (size_t)g->N);
    int *est = (int *)malloc(sizeof(int) * (size_t)g->N);
    for (int n = 0; n < g->N; n++) all[n] = 1;
    while (f->count < f->pr->max_updates) {
        int64_t before = f->count;
        double gap = INFINITY, margin;
        int nsel = alg4(f, all, f->pr->n_p, sel, &margin); /* line 4 */
        if (margin < gap) gap = margin;
        int done = me_step(f, sel, nsel, est, &gap); /* line 5 */
        f->count += done; f->ctr[CT_STEPS]++; f->step++;
        after_step(f);
        if (check_stop(f, before)) break;
    }
    free(all); free(sel); free(est);
}

/* Algorithm 6 (ME-LMD-CIRBP)                                                 */
static void run_me_lmd_cirbp(fr_t *f) {
    const og_t *g = f->g;
    int *inS = (int *)malloc(sizeof(int) * (size_t)g->N);
    int *sel = (int *)malloc(sizeof(int) * (size_t)g->N);
    int *nxt = (int *)malloc(sizeof(int) * (size_t)g->N);
    int *fill = (int *)malloc(sizeof(int) * (size_t)g->N);
    int *est = (int *)malloc(sizeof(int) * (size_t)g->N);
    int *inP = (int *)calloc((size_t)g->N, sizeof(int));
    for (int n = 0; n < g->N; n++) inS[n] = 1;
    double margin;
    int nsel = alg4(f, inS, f->pr->n_p, sel, &margin); /* line 4 */
    double carry_gap = margin;
    while (f->count < f->pr->max_updates) {
        int64_t before = f->count;
        double gap = carry_gap;
        int done = me_step(f, sel, nsel, est, &gap); /* line 5 */
        f->count += done; f->ctr[CT_STEPS]++; f->step++;
        after_step(f);
        if (check_stop(f, before)) break;
        /* lines 6-10: P' = { argmax_{j in U(m*_p, p)} D_j } (reading R4) */
        int nn = 0;
        carry_gap = INFINITY;
        for (int k = 0; k < done; k++) {
            amax_t a = lmd_next(f, sel[k], est[k]);
            if (a.idx < 0) continue;
            if (am_gap(&a) < carry_gap) carry_gap = am_gap(&a);
            if (!inP[a.idx]) { inP[a.idx] = 1; nxt[nn++] = a.idx; }
        }
        /* lines 11-14: top up with Algorithm 4 over O_N \ P' */
        int nf = 0;
        if (nn < f->pr->n_p) {
            for (int n = 0; n < g->N; n++) inS[n] = !inP[n];
            nf = alg4(f, inS, f->pr->n_p - nn, fill, &margin);
            if (margin < carry_gap) carry_gap = margin;
        }
        for (int k = 0; k < nn; k++) inP[nxt[k]] = 0;
        /* P <- P' u P, ascending */
        int a = 0, b = 0;
        nsel = 0;
        for (int k = 1; k < nn; k++) { /* sort P' */
            int v = nxt[k], j = k - 1;
            while (j >= 0 && nxt[j] > v) { nxt[j + 1] = nxt[j]; j--; }
            nxt[j + 1] = v;
        }
        while (a < nn || b < nf) {
            if (b >= nf || (a < nn && nxt[a] < fill[b])) sel[nsel++] = nxt[a++];
            else sel[nsel++] = fill[b++];
        }
    }
    free(inS); free(sel); free(nxt); free(fill); free(est); free(inP);
}

/* ------------------------------------------------------------------------ */
/* Batch entry point                                                        */

typedef struct {
    const og_t *g;
    const orc_params *pr;
    const double *llr;   /* [B][N] or NULL */
    const int8_t *qllr;  /* [B][N] or NULL */
    int64_t b0, b1;
    uint8_t *hard; int64_t *updates; uint8_t *converged;
    int32_t *trace; double *gap; double *llr_out; int64_t *counters; double *state_out;
    int rc;
} job_t;

static void decode_frame(job_t *J, int64_t b) {
    const og_t *g = J->g;
    const orc_params *pr = J->pr;
    fr_t f;
    memset(&f, 0, sizeof(f));
    f.g = g; f.pr = pr;
    f.frame = pr->frame_offset + (uint64_t)b;
    size_t E = (size_t)g->E, N = (size_t)g->N;
    f.lam = (double *)malloc(sizeof(double) * N);
    f.C = (double *)calloc(E, sizeof(double));
    f.P = (double *)malloc(sizeof(double) * E);
    f.L = (double *)malloc(sizeof(double) * N);
    f.Lt = (double *)malloc(sizeof(double) * N);
    f.D = (double *)malloc(sizeof(double) * N);
    f.mark_cn = (int *)calloc((size_t)g->M, sizeof(int));
    f.mark_vn = (int *)calloc(N, sizeof(int));
    f.list_a = (int *)malloc(sizeof(int) * ((size_t)g->M + 1));
    f.list_b = (int *)malloc(sizeof(int) * N);
    f.snapshot = pr->selfcheck ? (double *)malloc(sizeof(double) * 2 * state_len(g)) : NULL;
    int64_t ctr_local[CT_N];
    memset(ctr_local, 0, sizeof(ctr_local));
    f.ctr = J->counters ? J->counters + b * CT_N : ctr_local;
    f.trace = J->trace ? J->trace + b * pr->max_updates : NULL;
    f.gap = J->gap ? J->gap + b * pr->max_updates : NULL;
    for (size_t n = 0; n < N; n++)
        f.lam[n] = J->qllr ? (double)J->qllr[b * N + n] : J->llr[b * N + n];
    if (pr->arith == ORC_ARITH_INT) {
        for (int q = -127; q <= 127; q++) f.T[q + 127] = round(32767.0 * tanh(q * pr->q_step / 2.0));
        f.gamma = round(pr->gamma * 65534.0);
    } else {
        f.gamma = pr->gamma;
    }
    /* Alg. 1 lines 1-3: L^C = 0, L = L^V = lambda, all L~^C, R, L~, D */
    refresh_all(&f);
    if (pr->check_interval > 0 && syndrome_weight(&f) == 0) {
        /* valid codeword at count 0: no update */
    } else if (pr->max_updates > 0) {
        switch (pr->schedule) {
        case ORC_FLOODING: run_flooding(&f); break;
        case ORC_RBP: run_rbp(&f); break;
        case ORC_CIRBP: run_cirbp(&f); break;
        case ORC_LMD_CIRBP: run_lmd_cirbp(&f); break;
        case ORC_ME_CIRBP: run_me_cirbp(&f); break;
        case ORC_ME_LMD_CIRBP: run_me_lmd_cirbp(&f); break;
        case ORC_LMDRBP: run_lmdrbp(&f, 0); break;
        case ORC_SLMDRBP: run_lmdrbp(&f, 1); break;
        default: J->rc = ORC_ERR_ARG; break;
        }
    }
    for (size_t n = 0; n < N; n++) {
        if (J->hard) J->hard[b * N + n] = (uint8_t)bsgn(f.L[n]);
        if (J->llr_out) J->llr_out[b * N + n] = f.L[n];
    }
    if (J->updates) J->updates[b] = f.count;
    if (J->converged) J->converged[b] = syndrome_weight(&f) == 0;
    if (J->state_out) state_copy(&f, J->state_out + b * state_len(g));
    free(f.lam); free(f.C); free(f.P); free(f.L); free(f.Lt); free(f.D);
    free(f.mark_cn); free(f.mark_vn); free(f.list_a); free(f.list_b); free(f.snapshot);
}

static void *job_run(void *arg) {
    job_t *J = (job_t *)arg;
    for (int64_t b = J->b0; b < J->b1; b++) decode_frame(J, b);
    return NULL;
}

/* Decode `batch` frames with the schedule in `pr`.  `llr` (FP64) or `qllr`   */
/* (6-bit integers) holds [batch][N] channel values.  Outputs may be NULL:    */
/* hard [batch][N], updates [batch], converged [batch], trace and gap         */
/* [batch][max_updates], llr_out [batch][N], counters [batch][CT_N],          */
/* state_out [batch][2E+3N] (C, P, L, L~, D).  Frames are spread over         */
/* n_threads POSIX threads.                                                   */
int orc_decode(const int32_t *chk, const int32_t *var, int64_t E, int32_t M, int32_t N,
               const orc_params *pr, const double *llr, const int8_t *qllr, int64_t batch,
               uint8_t *hard, int64_t *updates, uint8_t *converged, int32_t *trace, double *gap,
               double *llr_out, int64_t *counters, double *state_out, int n_threads) {
    if (!pr || (!llr && !qllr) || batch < 0) return ORC_ERR_ARG;
    if (pr->schedule < 0 || pr->schedule > ORC_SLMDRBP) return ORC_ERR_ARG;
    if ((pr->schedule == ORC_ME_CIRBP || pr->schedule == ORC_ME_LMD_CIRBP) && (pr->n_p <= 0 || pr->n_g <= 0))
        return ORC_ERR_ARG;
    if (pr->max_updates < 0) return ORC_ERR_ARG;
    og_t g;
    int rc = og_build(&g, chk, var, E, M, N);
    if (rc) return rc;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > batch) n_threads = batch > 0 ? (int)batch : 1;
    job_t *jobs = (job_t *)calloc((size_t)n_threads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; t++) {
        job_t *J = &jobs[t];
        J->g = &g; J->pr = pr; J->llr = llr; J->qllr = qllr;
        J->b0 = batch * t / n_threads; J->b1 = batch * (t + 1) / n_threads;
        J->hard = hard; J->updates = updates; J->converged = converged; J->trace = trace;
        J->gap = gap; J->llr_out = llr_out; J->counters = counters; J->state_out = state_out;
    }
    if (n_threads == 1) job_run(&jobs[0]);
    else {
        for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, job_run, &jobs[t]);
        for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < n_threads; t++) if (jobs[t].rc) rc = jobs[t].rc;
    free(jobs); free(th);
    og_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Weighted BP along a recorded schedule, and its adjoint (not in the paper:  */
/* the differentiable decoder built on it).  Update t of a frame commits edge */
/* e_t = trace[t] as C[e_t] <- w[t] * P_t, where P_t is the clipped           */
/* sum-product C2V of eq. (2) from the state before the update; the final    */
/* L_n = lambda_n + sum C (eq. 3).  The adjoint runs the updates backwards,   */
/* restoring each overwritten C[e_t] from the tape the forward kept.         */

typedef struct {
    const og_t *g;
    const double *llr, *w, *dL;
    const int32_t *trace;
    const int64_t *counts;
    int64_t T, b0, b1;
    double clip;
    double *L_out, *dw_out, *dllr_out;
    int rc;
} wjob_t;

/* eq. (1) from the state C */
static double w_v2c(const og_t *g, const double *lam, const double *C, int e) {
    int n = g->e_vn[e];
    double v = lam[n];
    for (int k = g->vn_ptr[n]; k < g->vn_ptr[n + 1]; k++)
        if (g->vn_e[k] != e) v += C[g->vn_e[k]];
    return v;
}

static void *wjob_run(void *arg) {
    wjob_t *J = (wjob_t *)arg;
    const og_t *g = J->g;
    double *C = (double *)malloc(sizeof(double) * (size_t)g->E);
    double *Cb = (double *)malloc(sizeof(double) * (size_t)g->E);
    double *tape = (double *)malloc(sizeof(double) * (size_t)(J->T > 0 ? J->T : 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)g->E);
    double *th = (double *)malloc(sizeof(double) * (size_t)g->E);
    if (!C || !Cb || !tape || !u || !th) { J->rc = ORC_ERR_NOMEM; goto done; }
    for (int64_t b = J->b0; b < J->b1; b++) {
        const double *lam = J->llr + b * g->N;
        const int32_t *tr = J->trace + b * J->T;
        int64_t cnt = J->counts ? J->counts[b] : J->T;
        if (cnt > J->T) cnt = J->T;
        for (int e = 0; e < g->E; e++) C[e] = 0.0;
        for (int64_t t = 0; t < cnt; t++) { /* forward */
            int e = tr[t], m = g->e_cn[e];
            double prod = 1.0;
            for (int e2 = g->cn_ptr[m]; e2 < g->cn_ptr[m + 1]; e2++) {
                if (e2 == e) continue;
                prod *= tanh(clampd(w_v2c(g, lam, C, e2), -J->clip, J->clip) / 2.0);
            }
            tape[t] = C[e];
            C[e] = J->w[t] * clampd(2.0 * atanh(prod), -J->clip, J->clip);
        }
        for (int n = 0; n < g->N; n++) {
            double s = lam[n];
            for (int k = g->vn_ptr[n]; k < g->vn_ptr[n + 1]; k++) s += C[g->vn_e[k]];
            if (J->L_out) J->L_out[b * g->N + n] = s;
        }
        if (!J->dL) continue;
        /* adjoint: dloss/dC[e] = dloss/dL of its variable; dloss/dlambda likewise */
        const double *dL = J->dL + b * g->N;
        double *dw = J->dw_out ? J->dw_out + b * J->T : NULL;
        double *dlam = J->dllr_out ? J->dllr_out + b * g->N : NULL;
        for (int e = 0; e < g->E; e++) Cb[e] = dL[g->e_vn[e]];
        if (dlam) for (int n = 0; n < g->N; n++) dlam[n] = dL[n];
        if (dw) for (int64_t t = 0; t < J->T; t++) dw[t] = 0.0;
        for (int64_t t = cnt - 1; t >= 0; t--) {
            int e = tr[t], m = g->e_cn[e];
            C[e] = tape[t]; /* the state before update t */
            double prod = 1.0;
            for (int e2 = g->cn_ptr[m]; e2 < g->cn_ptr[m + 1]; e2++) {
                if (e2 == e) continue;
                u[e2] = w_v2c(g, lam, C, e2);
                th[e2] = tanh(clampd(u[e2], -J->clip, J->clip) / 2.0);
                prod *= th[e2];
            }
            double Praw = 2.0 * atanh(prod);
            double P = clampd(Praw, -J->clip, J->clip);
            double a = Cb[e];
            Cb[e] = 0.0; /* C[e] before the update does not reach the result */
            if (dw) dw[t] += a * P;
            double Pb = a * J->w[t];
            if (fabs(Praw) >= J->clip || Pb == 0.0) continue;
            /* dP/du_k = (1 - t_k^2) prod_{i != k} t_i / (1 - prod^2) for |u_k| < clip */
            for (int e2 = g->cn_ptr[m]; e2 < g->cn_ptr[m + 1]; e2++) {
                if (e2 == e || fabs(u[e2]) >= J->clip) continue;
                double others = 1.0;
                for (int e3 = g->cn_ptr[m]; e3 < g->cn_ptr[m + 1]; e3++)
                    if (e3 != e && e3 != e2) others *= th[e3];
                double ub = Pb * (1.0 - th[e2] * th[e2]) * others / (1.0 - prod * prod);
                /* u = lambda_n + sum_{e3 in M(n)\e2} C[e3] */
                int n = g->e_vn[e2];
                if (dlam) dlam[n] += ub;
                for (int k = g->vn_ptr[n]; k < g->vn_ptr[n + 1]; k++)
                    if (g->vn_e[k] != e2) Cb[g->vn_e[k]] += ub;
            }
        }
    }
done:
    free(C); free(Cb); free(tape); free(u); free(th);
    return NULL;
}

/* Weighted BP of `batch` frames along `trace` ([batch][T] edge ids, the      */
/* first counts[b] of each row used; counts NULL: all T), weights w[T], FP64. */
/* Writes L_out [batch][N] (may be NULL); with dL (dloss/dL, [batch][N]) also */
/* dw_out [batch][T] and dllr_out [batch][N] (either may be NULL).            */
int orc_wbp(const int32_t *chk, const int32_t *var, int64_t E, int32_t M, int32_t N, const double *llr,
            int64_t batch, const int32_t *trace, const int64_t *counts, int64_t T, const double *w,
            double clip, double *L_out, const double *dL, double *dw_out, double *dllr_out, int n_threads) {
    if (!llr || !trace || !w || batch < 0 || T < 0 || !(clip > 0.0)) return ORC_ERR_ARG;
    og_t g;
    int rc = og_build(&g, chk, var, E, M, N);
    if (rc) return rc;
    for (int64_t i = 0; i < batch * T; i++) {
        int64_t b = i / (T > 0 ? T : 1), t = i % (T > 0 ? T : 1);
        int64_t cnt = counts ? counts[b] : T;
        if (t < cnt && (trace[i] < 0 || trace[i] >= g.E)) { og_free(&g); return ORC_ERR_RANGE; }
    }
    if (n_threads < 1) n_threads = 1;
    if (n_threads > batch) n_threads = batch > 0 ? (int)batch : 1;
    wjob_t *jobs = (wjob_t *)calloc((size_t)n_threads, sizeof(wjob_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; t++) {
        wjob_t *J = &jobs[t];
        J->g = &g; J->llr = llr; J->w = w; J->dL = dL; J->trace = trace; J->counts = counts;
        J->T = T; J->clip = clip; J->L_out = L_out; J->dw_out = dw_out; J->dllr_out = dllr_out;
        J->b0 = batch * t / n_threads; J->b1 = batch * (t + 1) / n_threads;
    }
    if (n_threads == 1) wjob_run(&jobs[0]);
    else {
        for (int t = 0; t < n_threads; t++) pthread_create(&th[t], NULL, wjob_run, &jobs[t]);
        for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < n_threads; t++) if (jobs[t].rc) rc = jobs[t].rc;
    free(jobs); free(th);
    og_free(&g);
    return rc;
}

/* Algorithm 4 alone, for unit tests: D values of all N VNs, membership of S, */
/* returns |P| and writes P ascending.                                        */
int orc_alg4(const double *D, const uint8_t *inS, int32_t N, int32_t arith, int32_t n_g, int32_t n_p,
             uint64_t seed, uint64_t frame, int64_t step, int32_t *out, int64_t *icmp) {
    fr_t f;
    orc_params pr;
    memset(&f, 0, sizeof(f));
    memset(&pr, 0, sizeof(pr));
    og_t g;
    memset(&g, 0, sizeof(g));
    g.N = N;
    pr.arith = arith; pr.n_g = n_g; pr.n_p = n_p; pr.seed = seed;
    f.g = &g; f.pr = &pr; f.frame = frame; f.step = step;
    int64_t ctr[CT_N];
    memset(ctr, 0, sizeof(ctr));
    f.ctr = ctr;
    f.D = (double *)D;
    f.list_b = (int *)malloc(sizeof(int) * (size_t)N);
    int *s = (int *)malloc(sizeof(int) * (size_t)N);
    int *o = (int *)malloc(sizeof(int) * (size_t)N);
    for (int n = 0; n < N; n++) s[n] = inS[n];
    double margin;
    int k = alg4(&f, s, n_p, o, &margin);
    for (int i = 0; i < k; i++) out[i] = o[i];
    if (icmp) *icmp = ctr[CT_ICMP];
    free(f.list_b); free(s); free(o);
    return k;
}

/* Circulant lifting of a protograph: block (r, c) with shift s >= 0 gives    */
/* edges (r Z + z, c Z + (z + s) mod Z), z = 0..Z-1.  Returns the edge count. */
int64_t orc_qc_lift(const int32_t *base, int32_t rows, int32_t cols, int32_t Z, int32_t *chk, int32_t *var) {
    int64_t e = 0;
    for (int r = 0; r < rows; r++)
        for (int c = 0; c < cols; c++) {
            int s = base[r * cols + c];
            if (s < 0) continue;
            for (int z = 0; z < Z; z++) {
                if (chk) { chk[e] = r * Z + z; var[e] = c * Z + (z + s) % Z; }
                e++;
            }
        }
    return e;
}

int orc_counters_count(void) { return CT_N; }
