// cc_api.cu -- host driver and C ABI of libcc.so: the recursive CC split
// integrator evolve_cc (arXiv:1407.7105 Sec. 2.3, CC pseudocode figure)
// run level-synchronously on one GPU.
//
// All sets at recursion depth d that share the pivot h = dt / 2^d are
// processed as one batch (they are independent closed Hamiltonians,
// Sec. 2.2 Eq. for E_{h/2,H_C}).  process(d, h):
//   split   : tau + union-find over every set of the batch, compress,
//             segment components (stable, ascending ids);
//   for each half (before and after the DKD of this level):
//             two-body components -> batched Kepler (CC_KEPLER);
//             small components    -> persistent small-component kernel;
//             large components    -> gathered into level d+1, process(d+1, h/2),
//                                    scattered back;
//   DKD     : D_{h/2,T_R} K_{h,V_R+V_CC+V_CR} D_{h/2,T_R} on the batch.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cc_internal.cuh"

namespace cc {
unsigned long long g_launches = 0;
}

using namespace cc;

namespace {

constexpr int TAU_TILE = 128;   // must match the tau kernel

thread_local std::string g_init_err;

// set layout of a level batch: sizes -> aligned starts, the block
// prefixes of every launch-shape variant, the packed total
struct SetLayout {
    std::vector<int32_t> start, n;
    std::vector<int32_t> tau_off[N_TAU_VAR], k64_off[N_K64_VAR], mk_off[N_MK_VAR];
    long long tau_blocks[N_TAU_VAR] = {}, k64_blocks[N_K64_VAR] = {}, mk_blocks[N_MK_VAR] = {};
    int mk_chunks_max[N_MK_VAR] = {};
    long long pairs = 0;
    int total = 0;
};

struct LevelAlloc {
    Level L{};
    FFView F{};
    bool classified = false;  // the last split's segmenting CTA also wrote the integrator lists
    // launch-shape variants: block prefixes over the sets (device) and the
    // total blocks (host) of every tunable shape, for the current layout
    int32_t *tau_off[N_TAU_VAR] = {}, *k64_off[N_K64_VAR] = {}, *mk_off[N_MK_VAR] = {};
    long long tau_blocks[N_TAU_VAR] = {}, k64_blocks[N_K64_VAR] = {}, mk_blocks[N_MK_VAR] = {};
    int mk_chunks_max[N_MK_VAR] = {};
    long long pairs = 0;     // sum n(n-1)/2 over the sets (work unit of the tuner)
    int cap = 0;      // element capacity (excluding PAD_TAIL)
    int set_cap = 0;  // set-array capacity
    void *block = nullptr;
    void *setblock = nullptr;
    // split products of this level
    int32_t *root = nullptr, *members = nullptr, *comp_start = nullptr, *comp_size = nullptr, *d_ncomp = nullptr;
    // component lists handed to the children
    // (kqueue: the work-queue counters of the two small-kernel launches of a
    // split, zeroed by the same upload as the lists)
    int32_t *kqueue = nullptr, *klist = nullptr, *slist = nullptr, *lcomp_start = nullptr;
    void *listblock = nullptr;
    int list_cap = 0;
    std::vector<int32_t> h_size, h_start;
    std::vector<int32_t> h_set_n;  // set sizes of this level (host copy)
    // device split summary, one block: [ncomp, -, edge-record count (8 B), sizes[nd], starts[nd]];
    // h_info is its pinned host copy (one D2H per split)
    int32_t *h_info = nullptr;
    int32_t *h_sets = nullptr;     // pinned staging of the set arrays (one H2D)
    int32_t *h_lists = nullptr;    // pinned staging of the component lists (one H2D)
    int info_cap = 0;
    cudaEvent_t ev_ready = nullptr, ev_small = nullptr;  // side-stream joins
    cudaEvent_t ev_info = nullptr;                       // split summary copied
    // edge records of this level's last split (read by the first-half split
    // of the next level) and the parent -> child index map of the gather
    int32_t *inv = nullptr;
    EdgeList E{nullptr, nullptr, 0};
    void *eblock = nullptr;
    long long ecount = 0;  // records the last split offered (complete if <= E.cap)
    // host scratch of the classification, kept between splits (no reallocation)
    std::vector<int32_t> v_lstart, v_lsize;
    SetLayout child_layout;
    // centre-of-mass approximation (params.theta > 0): the eligible components
    // of the last split (host lists, built after the split) and their device
    // copies, centres, far matrices; grow-only
    int Ke = 0;
    long long far_bytes = 0;
    std::vector<int32_t> h_eq, h_eset, h_eloc, h_efirst, h_K;
    std::vector<long long> h_foff;
    void *comblock = nullptr;
    size_t com_cap = 0;
    void *h_comstage = nullptr;
    size_t h_comstage_cap = 0;
    int32_t *d_cl = nullptr;
    int cl_cap = 0;
    unsigned char *d_far = nullptr;
    long long far_cap = 0;
    ComView cv{nullptr, nullptr, nullptr, nullptr};
    int32_t *d_eq = nullptr, *d_eset = nullptr, *d_eloc = nullptr, *d_efirst = nullptr, *d_K = nullptr,
            *d_eany = nullptr;
    long long *d_foff = nullptr;
    double *d_cm = nullptr;
};

// ------------------------------------------------------------ autotuner
// Online tuner of launch shapes per (kernel, size bin): the first launches
// of a bin try each variant (preference order first) while CUDA events time
// them; once every variant has its trials (one for launches of at least
// 2^24 pairs, three below, where a launch lasts a few microseconds and a
// single timing is noisy), the one with the least time per pair over its
// fastest trial is kept for the bin.  Results do not depend on the
// choice except through the rounding order of the mixed kick's j-chunks.
enum TuneKind { TK_TAU64 = 0, TK_TAUMIX = 1, TK_K64 = 2, TK_MK = 3, TK_N = 4 };
constexpr int TUNE_BINS = 40, TUNE_MAXV = 3, TUNE_BIG_BIN = 24;
constexpr int TUNE_NVAR[TK_N] = {N_TAU64_VAR, N_TAU_VAR, N_K64_VAR, N_MK_VAR};

struct TuneCell {
    double qmin[TUNE_MAXV] = {0, 0, 0};  // fastest trial: ms per unit of work
    double work[TUNE_MAXV] = {0, 0, 0};
    int picked[TUNE_MAXV] = {0, 0, 0}, timed[TUNE_MAXV] = {0, 0, 0};
    int best = -1;
};

struct Tuner {
    TuneCell cell[TK_N][TUNE_BINS];
};

static int tune_bin(long long work)
{
    int b = 0;
    while (b < TUNE_BINS - 1 && (2ll << b) <= work) ++b;
    return b;
}

}  // namespace

struct cc_ctx {
    int64_t n = 0;
    cc_params p{};
    cudaStream_t stream = nullptr;
    double t = 0.0;
    double *d_x3 = nullptr, *d_v3 = nullptr, *d_m = nullptr;
    std::vector<int64_t> sys_off;
    int32_t *d_sys_off = nullptr;
    // mixed form, one system: level 0 in a Morton order of the positions
    // (perm[id] = offset), renewed every SPATIAL_RENEW outer steps
    int32_t *d_perm = nullptr;
    unsigned *d_box = nullptr;
    long long perm_age = -1;
    std::vector<LevelAlloc> lv;  // recursion levels
    LevelAlloc unit;             // staging level of the unit entry points
    void *seg_scratch = nullptr;
    size_t seg_scratch_sz = 0;
    DevCounters *d_ctr = nullptr;
    int32_t *d_near_ij = nullptr;
    double *d_near_tau = nullptr;
    long long near_cap = 4096;
    double *d_partial = nullptr;
    int partial_cap = 0;
    void *tmp = nullptr;  // staging for caller buffers
    size_t tmp_sz = 0;
    unsigned *d_bad = nullptr;
    // small-component kernels overlap the level recursion, one stream per
    // depth (a level's launch must not queue behind its parent level's:
    // they touch disjoint particles), highest priority, created on first use
    std::vector<cudaStream_t> sides;
    int prio_high = 0;
    int nsm = 152;
    double *d_kpart = nullptr;  // mixed-kick chunk partials
    size_t kpart_sz = 0;
    // FP64 kick: the precomputed r^-3 matrices of a level's sets and their
    // offsets (one buffer: the levels' kicks run one after another)
    double *pf_S = nullptr;
    size_t pf_bytes = 0;
    long long *pf_moff = nullptr;
    int pf_sets = 0;
    std::vector<long long> h_moff;
    cc_stats_t st{};
    std::string err;
    double eta_run = 0.03;
    // optional per-launch event timing of the tau and kick kernels
    bool timing = false;
    std::vector<cudaEvent_t> evs;
    struct EvRec {
        int kind;   // 0 = tau, 1 = kick, 2 = small-component kernel
        int tkind;  // tuner kernel (-1 = none)
        int bin, var;
        double work;
    };
    std::vector<EvRec> ev_rec;  // one per event pair
    Tuner tuner;
    bool p_autotune = true;
    size_t ev_used = 0;
    cc_timing_t tm{};
    unsigned long long launch_mark = 0;
    // batched small-component kernel: frame scratch (per resident CTA), and
    // the whole-batch mode of independent systems (every system a task of
    // the kernel: tlist, t_start, t_size, count, queue; identity member list)
    char *batch_scr = nullptr;
    bool sys_batch = false;
    int32_t *d_sys_tasks = nullptr;
    int32_t *d_iota = nullptr;
    // the whole-batch outer step captured as a CUDA graph (pack, queue reset,
    // the batched kernel, unpack), for the eta it was captured with, and
    // the kernels one replay launches
    cudaGraphExec_t sys_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    double sys_exec_eta = 0.0;
    unsigned long long sys_exec_launches = 0;
    // the OK split (split = CC_SPLIT_OK): the outer level's fast pairs and
    // their directed copy (ok_cap pairs each, grown on demand), the level's
    // inverse id map, row pointers and drift flags, each set's segment and
    // arena offset, the arena of the recursion, node stamps and positions
    int32_t *ok_edges = nullptr, *ok_dir = nullptr;
    EdgeRec *ok_rec = nullptr;                // the outer level's edge records (certified kernel)
    unsigned long long *ok_reccnt = nullptr;
    long long ok_cap = 0;
    void *ok_sort = nullptr;
    int32_t *ok_inv = nullptr, *ok_row = nullptr, *ok_rest = nullptr, *ok_loc = nullptr;
    unsigned long long *ok_stamp = nullptr, ok_launch = 0;
    long long *ok_seg = nullptr, *ok_aoff = nullptr;
    int ok_lvl_cap = 0, ok_set_cap = 0;
    char *ok_arena = nullptr;
    size_t ok_arena_cap = 0;
    std::vector<long long> ok_hseg, ok_haoff;
    // the OK split's GPU-wide nodes (lists too long for one CTA): per-depth
    // flags, prefix, child list, particle list and F flags; per-particle and
    // per-set stamps; the node counters; scan, directed-pair and sort scratch
    struct OkDepth {
        int *fast = nullptr, *pos = nullptr;
        int32_t *child = nullptr, *S = nullptr;
        unsigned char *isF = nullptr;
        long long cap = 0;
    };
    std::vector<OkDepth> okd;
    unsigned long long *ok_hst = nullptr;  // [4 * total + 2 * nsets] S, F stamps; set stamps
    int ok_hst_total = 0, ok_hst_sets = 0;
    unsigned long long ok_node_stamp = 0;
    unsigned long long *ok_cnt = nullptr;
    int *ok_scan = nullptr;
    long long ok_scan_cap = 0;
    int32_t *ok_ndir = nullptr;
    void *ok_nsort = nullptr;
    long long ok_ndir_cap = 0;
};

// components (and systems) of at most this many bodies run in the batched
// kernel; above 32 only without the centre-of-mass approximation (it acts in
// sets of more than 32 members, which the host levels run)
static int small_max(const cc_ctx *c)
{
    const int lim = c->p.theta > 0.0 ? 32 : BATCH_NMAX;
    return std::min(c->p.s_small, lim);
}

// record the start of a timed launch (user timing on, or a tuner sample);
// returns the pair index or -1
static int ev_begin(cc_ctx *c, int kind, cudaStream_t st = nullptr, int tkind = -1, int bin = 0, int var = 0,
                    double work = 0.0)
{
    if (!st) st = c->stream;
    if (!c->timing && tkind < 0) return -1;
    if (c->ev_used + 2 > c->evs.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->evs.push_back(e);
        }
        c->ev_rec.resize(c->evs.size() / 2);
    }
    const int pair = (int)(c->ev_used / 2);
    c->ev_rec[pair] = {kind, tkind, bin, var, work};
    cudaEventRecord(c->evs[c->ev_used], st);
    c->ev_used += 2;
    return pair;
}

static void ev_end(cc_ctx *c, int pair, cudaStream_t st = nullptr)
{
    if (pair >= 0) cudaEventRecord(c->evs[2 * pair + 1], st ? st : c->stream);
}

// fold the recorded event pairs into the totals (stream must be idle)
static void ev_resolve(cc_ctx *c)
{
    for (size_t q = 0; q < c->ev_used / 2; ++q) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->evs[2 * q], c->evs[2 * q + 1]);
        const cc_ctx::EvRec &r = c->ev_rec[q];
        if (r.tkind >= 0) {
            TuneCell &t = c->tuner.cell[r.tkind][r.bin];
            const double q = ms / (r.work > 0 ? r.work : 1.0);
            if (t.timed[r.var] == 0 || q < t.qmin[r.var]) t.qmin[r.var] = q;
            t.work[r.var] += r.work;
            t.timed[r.var]++;
        }
        if (!c->timing) continue;
        if (r.kind == 0) {
            c->tm.tau_ms += ms;
            c->tm.tau_launches++;
        } else if (r.kind == 1) {
            c->tm.kick_ms += ms;
            c->tm.kick_launches++;
        } else {
            c->tm.small_ms += ms;
            c->tm.small_launches++;
        }
    }
    c->ev_used = 0;
}

// ------------------------------------------------------------ utilities
#define CC_CUDA(ctx, call)                                                                             \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            (ctx)->err = std::string("CUDA error ") + cudaGetErrorString(e_) + " at " #call;            \
            return CC_E_CUDA;                                                                           \
        }                                                                                               \
    } while (0)

#define CC_TRY(expr)           \
    do {                       \
        int rc_ = (expr);      \
        if (rc_) return rc_;   \
    } while (0)

static int fail(cc_ctx *c, int code, const char *msg)
{
    c->err = msg;
    return code;
}

static int ensure_tmp(cc_ctx *c, size_t bytes)
{
    if (c->tmp_sz >= bytes) return CC_OK;
    if (c->tmp) cudaFree(c->tmp);
    c->tmp = nullptr;
    c->tmp_sz = 0;
    size_t sz = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&c->tmp, sz) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, CC_E_NOMEM, "device allocation failed (staging buffer)");
    }
    c->tmp_sz = sz;
    return CC_OK;
}

// copy `bytes` from a host or device pointer into device memory dst
static int copy_in(cc_ctx *c, void *dst, const void *src, size_t bytes)
{
    if (bytes == 0) return CC_OK;
    CC_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return CC_OK;
}

static int copy_out(cc_ctx *c, void *dst, const void *src, size_t bytes)
{
    if (bytes == 0 || !dst) return CC_OK;
    CC_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return CC_OK;
}

static int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Launch shape for a kernel of the given kind on a level.  Returns the
// variant; *timed tells whether this launch is a tuner sample.  Without
// autotuning (or before any sample) a rule picks the largest shape that
// still gives every SM a few blocks.
// Variants that split tile columns over more threads are only worth trying
// while the plain variant leaves the GPU short of blocks.
static bool tune_eligible(const cc_ctx *c, int tkind, const long long *blocks, int v)
{
    if (tkind == TK_TAUMIX && TAU_VAR_S[v] > 1) return blocks[0] < 16ll * c->nsm;
    if (tkind == TK_MK && MK_VAR_SLICE[v] > 1) return blocks[0] < 8ll * c->nsm;
    return true;
}

static int tune_pick(cc_ctx *c, int tkind, const long long *blocks, long long work, int *bin_out, bool *timed)
{
    const int nv = TUNE_NVAR[tkind];
    bool ok[TUNE_MAXV];
    for (int v = 0; v < nv; ++v) ok[v] = tune_eligible(c, tkind, blocks, v);
    int rule = 0;
    for (int v = nv - 1; v >= 0; --v)
        if (ok[v] && blocks[v] >= 3ll * c->nsm) {
            rule = v;
            break;
        }
    const int bin = tune_bin(work);
    *bin_out = bin;
    *timed = false;
    if (!c->p_autotune) return rule;
    TuneCell &t = c->tuner.cell[tkind][bin];
    if (t.best >= 0) return ok[t.best] ? t.best : rule;
    const int trials = bin >= TUNE_BIG_BIN ? 1 : 3;
    bool all = true;
    for (int v = 0; v < nv; ++v) all = all && (!ok[v] || t.timed[v] >= trials);
    if (all) {
        int best = rule;
        double bq = 1e300;
        for (int v = 0; v < nv; ++v) {
            if (!ok[v]) continue;
            const double q = t.qmin[v];
            if (q < bq) {
                bq = q;
                best = v;
            }
        }
        t.best = best;
        return best;
    }
    // explore: the rule's choice first, then the others, fewest picks first
    int pick = rule, fewest = t.picked[rule];
    for (int v = 0; v < nv; ++v)
        if (ok[v] && t.picked[v] < fewest) {
            fewest = t.picked[v];
            pick = v;
        }
    t.picked[pick]++;
    *timed = true;
    return pick;
}

static void free_level(LevelAlloc &a)
{
    if (a.h_info) cudaFreeHost(a.h_info);
    if (a.h_sets) cudaFreeHost(a.h_sets);
    if (a.h_lists) cudaFreeHost(a.h_lists);
    a.h_sets = a.h_lists = nullptr;
    if (a.ev_ready) cudaEventDestroy(a.ev_ready);
    if (a.ev_small) cudaEventDestroy(a.ev_small);
    if (a.ev_info) cudaEventDestroy(a.ev_info);
    a.ev_info = nullptr;
    a.h_info = nullptr;
    a.info_cap = 0;
    a.ev_ready = a.ev_small = nullptr;
    if (a.block) cudaFree(a.block);
    if (a.setblock) cudaFree(a.setblock);
    if (a.listblock) cudaFree(a.listblock);
    if (a.eblock) cudaFree(a.eblock);
    if (a.comblock) cudaFree(a.comblock);
    if (a.h_comstage) cudaFreeHost(a.h_comstage);
    if (a.d_cl) cudaFree(a.d_cl);
    if (a.d_far) cudaFree(a.d_far);
    a.comblock = a.h_comstage = nullptr;
    a.d_cl = nullptr;
    a.d_far = nullptr;
    a.com_cap = a.h_comstage_cap = 0;
    a.cl_cap = 0;
    a.far_cap = 0;
    a.block = a.setblock = a.listblock = a.eblock = nullptr;
    a.E = EdgeList{nullptr, nullptr, 0};
    a.cap = a.set_cap = a.list_cap = 0;
}

// (re)allocate a level for `need` packed elements and `nsets` sets
static int ensure_level(cc_ctx *c, LevelAlloc &a, int need, int nsets)
{
    if (need > a.cap) {
        if (a.block) cudaFree(a.block);
        a.block = nullptr;
        // sized once for the worst batch (every set padded): no reallocation,
        // and no cudaFree stall, once a level has been reached
        const long long worst = std::min<long long>(2 * (long long)c->n + 64, 0x3fffffff);
        int cap = align_up(std::max<int>(need, (int)std::max<long long>(64, worst)), 64);
        size_t nd = (size_t)cap + PAD_TAIL;
        size_t bytes = nd * 8 * 7 + (nd * 11 + 4) * 4 + nd * 64 + 4096;
        if (cudaMalloc(&a.block, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (level buffer)");
        }
        cudaMemsetAsync(a.block, 0, bytes, c->stream);
        char *q = (char *)a.block;
        double **dp[7] = {&a.L.x, &a.L.y, &a.L.z, &a.L.vx, &a.L.vy, &a.L.vz, &a.L.m};
        for (int k = 0; k < 7; ++k) { *dp[k] = (double *)q; q += nd * 8; }
        int32_t **ip[9] = {&a.L.gid, &a.L.sidx, &a.L.src, &a.L.parent, &a.L.cnt, &a.L.klab,
                           &a.root, &a.members, &a.inv};
        for (int k = 0; k < 9; ++k) { *ip[k] = (int32_t *)q; q += nd * 4; }
        a.d_ncomp = (int32_t *)q;
        a.comp_size = a.d_ncomp + 4;
        a.comp_start = a.d_ncomp + 4 + nd;
        q += (2 * nd + 4) * 4;
        if (a.h_info) cudaFreeHost(a.h_info);
        a.h_info = nullptr;
        if (cudaMallocHost(&a.h_info, (2 * nd + 4) * 4) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "pinned host allocation failed (split summary)");
        }
        a.info_cap = (int)nd;
        a.F.pq = (float4 *)q; q += nd * 32;
        a.F.vq = (float4 *)q; q += nd * 32;
        a.F.maxes = (float *)q;
        a.F.cap = (int)nd;
        a.cap = cap;
        // lists: at most cap/2 components
        if (a.listblock) cudaFree(a.listblock);
        a.listblock = nullptr;
        a.list_cap = cap / 2 + 8;
        if (cudaMalloc(&a.listblock, (size_t)a.list_cap * 4 * 5 + 1024) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (component lists)");
        }
        if (a.h_lists) cudaFreeHost(a.h_lists);
        a.h_lists = nullptr;
        if (cudaMallocHost(&a.h_lists, (size_t)a.list_cap * 4 * 5 + 1024) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "pinned host allocation failed (component lists)");
        }
        int32_t *lq = (int32_t *)a.listblock;
        a.kqueue = lq; lq += 4;
        a.klist = lq; lq += a.list_cap;
        a.slist = lq; lq += a.list_cap;
        a.lcomp_start = lq;
    }
    if (nsets + 2 > a.set_cap) {
        if (a.setblock) cudaFree(a.setblock);
        a.setblock = nullptr;
        int sc = align_up(nsets + 2, 256);
        if (cudaMalloc(&a.setblock, (size_t)sc * 4 * (2 + N_TAU_VAR + N_K64_VAR + N_MK_VAR)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (set arrays)");
        }
        if (a.h_sets) cudaFreeHost(a.h_sets);
        a.h_sets = nullptr;
        if (cudaMallocHost(&a.h_sets, (size_t)sc * 4 * (2 + N_TAU_VAR + N_K64_VAR + N_MK_VAR)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "pinned host allocation failed (set arrays)");
        }
        int32_t *sq = (int32_t *)a.setblock;
        a.L.set_start = sq; sq += sc;
        a.L.set_n = sq; sq += sc;
        for (int v = 0; v < N_TAU_VAR; ++v) { a.tau_off[v] = sq; sq += sc; }
        for (int v = 0; v < N_K64_VAR; ++v) { a.k64_off[v] = sq; sq += sc; }
        for (int v = 0; v < N_MK_VAR; ++v) { a.mk_off[v] = sq; sq += sc; }
        a.L.tile_off = a.tau_off[TAU_VAR_128];
        a.L.itile_off = a.k64_off[1];
        a.L.koff = a.mk_off[1];
        a.set_cap = sc;
    }
    // the segmentation scratch is shared by all levels: size for the largest
    size_t need_seg = seg_scratch_bytes(a.cap + PAD_TAIL);
    if (need_seg > c->seg_scratch_sz) {
        if (c->seg_scratch) cudaFree(c->seg_scratch);
        c->seg_scratch = nullptr;
        if (cudaMalloc(&c->seg_scratch, need_seg) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (segment scratch)");
        }
        c->seg_scratch_sz = need_seg;
    }
    return CC_OK;
}

// Edge-record list of a level: 4 records per element at first, grown to
// twice the last count when a split overflowed it (up to EDGE_CAP_MAX); an
// incomplete list only means the next first-half split evaluates tau itself.
constexpr long long EDGE_CAP_MAX = 1ll << 22;

static int ensure_edges(cc_ctx *c, LevelAlloc &a, long long at_least = 0)
{
    a.E.count = (unsigned long long *)(a.d_ncomp + 2);  // in the split summary block
    const long long cap_max = c->p.edge_rec_max > 0 ? (long long)c->p.edge_rec_max : EDGE_CAP_MAX;
    long long want = std::max<long long>(std::max<long long>(4096, 4ll * a.cap), at_least);
    if (a.ecount > a.E.cap) want = std::max(want, 2 * a.ecount);
    want = std::min(std::max(want, at_least), std::max(cap_max, at_least));
    if (a.eblock && want <= a.E.cap) return CC_OK;
    // grow geometrically: a reallocation synchronises the device
    if (a.eblock) want = std::max(want, std::min(a.E.cap + a.E.cap / 2, std::max(cap_max, at_least)));
    if (a.eblock) cudaFree(a.eblock);
    a.eblock = nullptr;
    a.E = EdgeList{nullptr, nullptr, 0};
    if (cudaMalloc(&a.eblock, 256 + (size_t)want * sizeof(EdgeRec)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, CC_E_NOMEM, "device allocation failed (edge records)");
    }
    a.E.rec = (EdgeRec *)((char *)a.eblock + 256);
    a.E.cap = want;
    a.E.count = (unsigned long long *)(a.d_ncomp + 2);
    return CC_OK;
}

// block prefixes of every launch-shape variant: triangular tau tiles,
// FP64-kick i-tiles, mixed-kick (i-tile, j-chunk) blocks
static void make_layout(const std::vector<int32_t> &sizes, SetLayout &S)
{
    const size_t ns = sizes.size();
    S.start.resize(ns);
    S.n = sizes;
    for (auto &v : S.tau_off) v.assign(ns + 1, 0);
    for (auto &v : S.k64_off) v.assign(ns + 1, 0);
    for (auto &v : S.mk_off) v.assign(ns + 1, 0);
    int pos = 0;
    long long tb[N_TAU_VAR] = {}, kb[N_K64_VAR] = {}, mb[N_MK_VAR] = {};
    S.pairs = 0;
    for (int v = 0; v < N_MK_VAR; ++v) S.mk_chunks_max[v] = 0;
    for (size_t s = 0; s < ns; ++s) {
        S.start[s] = pos;
        pos += align_up(sizes[s], SET_ALIGN);
        const long long n = sizes[s];
        S.pairs += n * (n - 1) / 2;
        for (int v = 0; v < N_TAU_VAR; ++v) {
            S.tau_off[v][s] = (int32_t)tb[v];
            const long long nt = (n + TAU_VAR_T[v] - 1) / TAU_VAR_T[v];
            tb[v] += nt * (nt + 1) / 2;
        }
        for (int v = 0; v < N_K64_VAR; ++v) {
            S.k64_off[v][s] = (int32_t)kb[v];
            kb[v] += (n + K64_VAR_T[v] - 1) / K64_VAR_T[v];
        }
        for (int v = 0; v < N_MK_VAR; ++v) {
            S.mk_off[v][s] = (int32_t)mb[v];
            mb[v] += mixed_kick_blocks((int)n, MK_VAR_CHUNK[v], MK_VAR_SLICE[v]);
            S.mk_chunks_max[v] = std::max(S.mk_chunks_max[v], mixed_kick_chunks((int)n, MK_VAR_CHUNK[v]));
        }
    }
    for (int v = 0; v < N_TAU_VAR; ++v) { S.tau_off[v][ns] = (int32_t)tb[v]; S.tau_blocks[v] = tb[v]; }
    for (int v = 0; v < N_K64_VAR; ++v) { S.k64_off[v][ns] = (int32_t)kb[v]; S.k64_blocks[v] = kb[v]; }
    for (int v = 0; v < N_MK_VAR; ++v) { S.mk_off[v][ns] = (int32_t)mb[v]; S.mk_blocks[v] = mb[v]; }
    S.total = pos;
}

static int upload_layout(cc_ctx *c, LevelAlloc &a, const SetLayout &S)
{
    const int ns = (int)S.n.size();
    CC_TRY(ensure_level(c, a, std::max(S.total, 1), ns));
    // one pinned staging block laid out like the device set arrays (stride
    // set_cap), copied in one asynchronous transfer
    const int sc = a.set_cap;
    int32_t *hq = a.h_sets;
    std::memcpy(hq, S.start.data(), ns * 4);
    hq += sc;
    std::memcpy(hq, S.n.data(), ns * 4);
    hq += sc;
    for (int v = 0; v < N_TAU_VAR; ++v, hq += sc) std::memcpy(hq, S.tau_off[v].data(), (ns + 1) * 4);
    for (int v = 0; v < N_K64_VAR; ++v, hq += sc) std::memcpy(hq, S.k64_off[v].data(), (ns + 1) * 4);
    for (int v = 0; v < N_MK_VAR; ++v, hq += sc) std::memcpy(hq, S.mk_off[v].data(), (ns + 1) * 4);
    const int narr = 2 + N_TAU_VAR + N_K64_VAR + N_MK_VAR;
    CC_CUDA(c, cudaMemcpyAsync(a.L.set_start, a.h_sets, (size_t)((narr - 1) * sc + ns + 1) * 4,
                               cudaMemcpyHostToDevice, c->stream));
    for (int v = 0; v < N_TAU_VAR; ++v) a.tau_blocks[v] = S.tau_blocks[v];
    for (int v = 0; v < N_K64_VAR; ++v) a.k64_blocks[v] = S.k64_blocks[v];
    for (int v = 0; v < N_MK_VAR; ++v) {
        a.mk_blocks[v] = S.mk_blocks[v];
        a.mk_chunks_max[v] = S.mk_chunks_max[v];
    }
    a.pairs = S.pairs;
    a.L.total = S.total;
    a.L.nsets = ns;
    a.h_set_n = S.n;
    return CC_OK;
}

static TauParams tau_params(const cc_ctx *c, double h)
{
    TauParams P;
    P.G = c->p.G;
    P.eps2 = c->p.eps * c->p.eps;
    P.eta = c->eta_run;
    P.eta_in = c->p.eta_outside ? 1.0 : c->eta_run;
    P.eta_outside = c->p.eta_outside;
    P.h = h;
    P.near_tol = c->p.near_tol;
    P.fault_test = c->p.fault_test;
    return P;
}

static int check_device_error(cc_ctx *c)
{
    unsigned e = 0;
    CC_CUDA(c, cudaMemcpyAsync(&e, &c->d_ctr->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (e == 0) return CC_OK;
    unsigned z = 0;
    cudaMemcpyAsync(&c->d_ctr->err, &z, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    switch (e) {
    case DERR_TMA_TIMEOUT: return fail(c, CC_E_TIMEOUT, "a bounded TMA/mbarrier wait timed out");
    case DERR_UF_RETRY: return fail(c, CC_E_TIMEOUT, "union-find retry limit reached");
    case DERR_KEPLER: return fail(c, CC_E_KEPLER, "Kepler solver did not converge");
    case DERR_DEPTH: return fail(c, CC_E_DEPTH, "recursion deeper than max_depth");
    default: return fail(c, CC_E_TIMEOUT, "device error");
    }
}

// ------------------------------------------------------------ recursion
static int process(cc_ctx *c, int d, double h, const LevelAlloc *parent);

// split the batch of level d at h: union-find components and segments.
// parent != null: this is the first half of the parent's components, whose
// split saw the same state at 2h, so the edges come from the parent's
// edge records (a pass over the records instead of all pairs).
static int split_launch(cc_ctx *c, LevelAlloc &a, double h, const LevelAlloc *parent)
{
    const cudaStream_t s = c->stream;
    const TauParams P = tau_params(c, h);
    // a first half's records are a subset of its parent's: room for all
    CC_TRY(ensure_edges(c, a, parent ? parent->ecount : 0));
    // Both forms decide the edge predicate tau(i,j) < h with the certified
    // FP32 kernel, the FP64 tau where the FP32 bounds leave it open: the
    // decisions are the FP64 predicate's, so the FP64 form's components,
    // and with them its state, stay the oracle's bit for bit.
    // (a fresh split initialises its forest in the float-float copy's pass)
    if (parent) launch_init_parent(a.L, a.E.count, s);
    bool hook_in_seg = false;  // a first half's child edges hooked by the one-CTA segmentation
    const bool hold = c->p.split == CC_SPLIT_HOLD;
    if (parent) {
        // (the HOLD merge needs the complete forest before the segmentation)
        hook_in_seg = segment_hooks_edges(a.L.total) && !hold;
        launch_edges_reuse(parent->E, parent->ecount, parent->L, parent->F, true, parent->inv, a.L, a.E, P, c->d_ctr,
                           c->d_near_ij, c->d_near_tau, c->near_cap, s, !hook_in_seg);
    } else {
        const int tk = TK_TAUMIX;
        int bin;
        bool timed;
        const int var = tune_pick(c, tk, a.tau_blocks, a.pairs, &bin, &timed);
        const long long ntiles = a.tau_blocks[var];
        if (ntiles > 0x7fffffff) return fail(c, CC_E_ARG, "set too large for the tile grid");
        Level L = a.L;
        L.tile_off = a.tau_off[var];
        launch_prep_ff(a.L, a.F, c->p.G, true, s, true, a.E.count);
        const int ev = ev_begin(c, 0, nullptr, timed ? tk : -1, bin, var, (double)a.pairs);
        launch_tau_mixed(L, a.F, (int)ntiles, P, var, c->d_ctr, c->d_near_ij, c->d_near_tau, c->near_cap, a.E, s);
        ev_end(c, ev);
    }
    // HOLD: the set's non-trivial components form one fast set
    if (hold) launch_hold_merge(a.L, (int32_t *)c->seg_scratch, s);
    const ClassifyArgs cls{small_max(c), c->p.kepler, a.kqueue, a.kqueue + 2, a.klist, a.slist};
    a.classified = launch_compress_segment(a.L, a.root, a.members, a.comp_start, a.comp_size, a.d_ncomp,
                                           c->seg_scratch, s, hook_in_seg ? &a.E : nullptr, c->d_ctr,
                                           a.klist && a.slist && a.kqueue ? &cls : nullptr);
    // one round trip: count, record count, sizes and (bounded by total/2) starts
    const int maxc = a.L.total / 2 + 1;
    CC_CUDA(c, cudaMemcpyAsync(a.h_info, a.d_ncomp, (size_t)(4 + a.info_cap + maxc) * 4, cudaMemcpyDeviceToHost, s));
    if (!a.ev_info) CC_CUDA(c, cudaEventCreateWithFlags(&a.ev_info, cudaEventDisableTiming));
    CC_CUDA(c, cudaEventRecord(a.ev_info, s));
    return CC_OK;
}

// wait for the split summary (only it: kernels queued after it keep
// running) and account the split
static int split_finish(cc_ctx *c, LevelAlloc &a, const LevelAlloc *parent, int &ncomp)
{
    CC_CUDA(c, cudaEventSynchronize(a.ev_info));
    const int32_t nc = a.h_info[0];
    ncomp = nc;
    std::memcpy(&a.ecount, a.h_info + 2, 8);
    a.h_size.assign(a.h_info + 4, a.h_info + 4 + nc);
    a.h_start.assign(a.h_info + 4 + a.info_cap, a.h_info + 4 + a.info_cap + nc);
    // statistics: n(n-1)/2 tau pairs per set, cross-component kick pairs
    unsigned long long tp = 0, inner = 0, memb = 0, all = 0;
    for (int32_t n : a.h_set_n) {
        tp += (unsigned long long)n * (n - 1) / 2;
        all += n;
    }
    for (int32_t k : a.h_size) {
        inner += (unsigned long long)k * (k - 1) / 2;
        memb += k;
    }
    c->st.splits += a.h_set_n.size();
    c->st.tau_pairs += tp;
    // (tau_fp64: the split kernels count the pairs whose FP64 tau they took)
    if (!parent) c->st.tau_evaluated += tp;
    if (c->timing) {
        if (!parent) c->tm.tau_pairs += tp;
        c->tm.kick_pairs += tp - inner;
    }
    c->st.components += nc;
    c->st.kick_pairs += tp - inner;
    c->st.drifts += 2 * (all - memb);
    return CC_OK;
}

// Centre-of-mass approximation: the eligible components of the split just
// taken (2..com_max members, in sets of at least COM_MIN_SET members), their
// local indices and the far-matrix layout, built on the host from the split
// summary and uploaded in one pinned transfer.  Components are ordered by
// root, so the eligible ones come grouped by set, ascending.
static int com_setup(cc_ctx *c, LevelAlloc &a, int ncomp)
{
    a.Ke = 0;
    a.cv = ComView{nullptr, nullptr, nullptr, nullptr};
    if (!(c->p.theta > 0.0)) return CC_OK;
    const int ns = (int)a.h_set_n.size();
    a.h_eq.clear();
    a.h_eset.clear();
    a.h_eloc.clear();
    a.h_K.assign(ns, 0);
    a.h_efirst.assign(ns, 0);
    a.h_foff.assign(ns, 0);
    std::vector<int32_t> starts(ns);
    {
        int pos = 0;
        for (int s = 0; s < ns; ++s) {
            starts[s] = pos;
            pos += align_up(a.h_set_n[s], SET_ALIGN);
        }
    }
    for (int q = 0; q < ncomp; ++q) {
        const int sz = a.h_size[q];
        if (sz < 2 || sz > c->p.com_max) continue;
        const int st = a.h_start[q];
        const int s = (int)(std::upper_bound(starts.begin(), starts.end(), st) - starts.begin()) - 1;
        if (s < 0 || a.h_set_n[s] < COM_MIN_SET) continue;
        if (a.h_K[s] == 0) a.h_efirst[s] = (int)a.h_eq.size();
        a.h_eq.push_back(q);
        a.h_eset.push_back(s);
        a.h_eloc.push_back(a.h_K[s]++);
    }
    const int Ke = (int)a.h_eq.size();
    if (Ke == 0) return CC_OK;
    long long fb = 0;
    for (int s = 0; s < ns; ++s) {
        a.h_foff[s] = fb;
        fb += (long long)a.h_K[s] * a.h_K[s];
    }
    // device buffers: ints (eq, eset, eloc, eany: Ke each; efirst, K: ns
    // each), foff (ns longs), cm (8 Ke doubles)
    const size_t ints = (size_t)4 * Ke + 2 * (size_t)ns;
    const size_t bytes = 256 + ints * 4 + 16 + (size_t)ns * 8 + 16 + (size_t)Ke * 64;
    if (bytes > a.com_cap) {
        if (a.comblock) cudaFree(a.comblock);
        a.comblock = nullptr;
        a.com_cap = 0;
        if (cudaMalloc(&a.comblock, 2 * bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (centre-of-mass lists)");
        }
        a.com_cap = 2 * bytes;
        if (a.h_comstage) cudaFreeHost(a.h_comstage);
        a.h_comstage = nullptr;
        if (cudaMallocHost(&a.h_comstage, 2 * bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "pinned host allocation failed (centre-of-mass lists)");
        }
        a.h_comstage_cap = 2 * bytes;
    }
    if (fb > a.far_cap) {
        if (a.d_far) cudaFree(a.d_far);
        a.d_far = nullptr;
        if (cudaMalloc(&a.d_far, (size_t)(2 * fb)) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (far matrices)");
        }
        a.far_cap = 2 * fb;
    }
    if (a.cl_cap < a.cap + PAD_TAIL) {
        if (a.d_cl) cudaFree(a.d_cl);
        a.d_cl = nullptr;
        if (cudaMalloc(&a.d_cl, (size_t)(a.cap + PAD_TAIL) * 4) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (centre-of-mass indices)");
        }
        a.cl_cap = a.cap + PAD_TAIL;
    }
    // staging laid out like the device block: the ints, then foff, then cm
    char *hq = (char *)a.h_comstage, *dq = (char *)a.comblock;
    int32_t *hi = (int32_t *)hq;
    std::memcpy(hi, a.h_eq.data(), Ke * 4);
    std::memcpy(hi + Ke, a.h_eset.data(), Ke * 4);
    std::memcpy(hi + 2 * Ke, a.h_eloc.data(), Ke * 4);
    std::memcpy(hi + 3 * Ke, a.h_efirst.data(), ns * 4);
    std::memcpy(hi + 3 * Ke + ns, a.h_K.data(), ns * 4);
    const size_t foff_at = (ints * 4 + 15) / 16 * 16;
    std::memcpy(hq + foff_at, a.h_foff.data(), ns * 8);
    const size_t cm_at = (foff_at + (size_t)ns * 8 + 15) / 16 * 16;
    int32_t *di = (int32_t *)dq;
    a.d_eq = di;
    a.d_eset = di + Ke;
    a.d_eloc = di + 2 * Ke;
    a.d_efirst = di + 3 * Ke;
    a.d_K = di + 3 * Ke + ns;
    a.d_eany = di + 3 * Ke + 2 * ns;
    a.d_foff = (long long *)(dq + foff_at);
    a.d_cm = (double *)(dq + cm_at);
    CC_CUDA(c, cudaMemcpyAsync(dq, hq, foff_at + (size_t)ns * 8, cudaMemcpyHostToDevice, c->stream));
    a.Ke = Ke;
    a.far_bytes = fb;
    a.cv = ComView{a.d_cl, a.d_foff, a.d_K, a.d_far};
    return CC_OK;
}

// the centres and far matrices of the eligible components, from the state
// at the DKD (their first half has moved them since the split)
static int com_prepare(cc_ctx *c, LevelAlloc &a)
{
    if (a.Ke == 0) return CC_OK;
    const cudaStream_t s = c->stream;
    CC_CUDA(c, cudaMemsetAsync(a.d_cl, 0xff, (size_t)a.L.total * 4, s));
    launch_com_prep(a.L, a.members, a.comp_start, a.comp_size, a.d_eq, a.d_eloc, a.Ke, a.d_cl, a.d_cm, s);
    launch_com_far(a.d_cm, a.d_eq, a.comp_size, a.d_eset, a.d_eloc, a.d_efirst, a.d_foff, a.d_K, a.Ke, c->p.theta,
                   c->p.G, c->p.eps * c->p.eps, a.d_far, a.d_eany, c->d_ctr, s, c->p.precision == CC_PREC_MIXED);
    return CC_OK;
}

// device memory the FP64 kick's precomputed pair-force matrices may take (a
// 16384-body set needs 6.4 GB, a 28000-body one 18.8 GB; larger levels
// compute the forces in the kick)
constexpr size_t PF_BUDGET = (size_t)24 << 30;
// levels with fewer pairs kick with the forces computed in place: the ~24
// FP64 operations a precomputed pair saves do not pay for the second launch
// and the offsets' upload (Plummer 256 and 1024: 20-35 % slower per step
// with the matrices at every level)
constexpr long long PF_MIN_PAIRS = 1LL << 18;

static int ensure_kpart(cc_ctx *c, int chunks, int fcap)
{
    const size_t need = (size_t)std::max(1, chunks) * 3 * (size_t)fcap * sizeof(double);
    if (chunks > 1 && need > c->kpart_sz) {
        if (c->d_kpart) cudaFree(c->d_kpart);
        c->d_kpart = nullptr;
        c->kpart_sz = 0;
        if (cudaMalloc(&c->d_kpart, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CC_E_NOMEM, "device allocation failed (kick partials)");
        }
        c->kpart_sz = need;
    }
    return CC_OK;
}

// Device matrices of the FP64 kick's pair forces G m_j r_ij^-3 (x_j - x_i)
// for the sets of level a (three n x n per set, row-major), when they fit
// PF_BUDGET; pf stays empty otherwise (the kick then computes the forces).
static int pair_factors(cc_ctx *c, LevelAlloc &a, PairFactors &pf)
{
    pf = PairFactors{nullptr, nullptr, 0};
    if (a.pairs < PF_MIN_PAIRS || a.tau_blocks[TAU_VAR_128] > 0x7fffffff) return CC_OK;
    const int ns = (int)a.h_set_n.size();
    c->h_moff.resize(ns + 1);
    long long tot = 0;
    for (int q = 0; q < ns; ++q) {
        c->h_moff[q] = tot;
        tot += 3LL * a.h_set_n[q] * a.h_set_n[q];
    }
    c->h_moff[ns] = tot;
    const size_t bytes = (size_t)tot * sizeof(double);
    if (tot <= 0 || bytes > PF_BUDGET) return CC_OK;
    if (bytes > c->pf_bytes) {
        if (c->pf_S) cudaFree(c->pf_S);
        c->pf_S = nullptr;
        c->pf_bytes = 0;
        if (cudaMalloc(&c->pf_S, bytes) == cudaSuccess) c->pf_bytes = bytes;
        else cudaGetLastError();
    }
    if (ns + 1 > c->pf_sets) {
        if (c->pf_moff) cudaFree(c->pf_moff);
        c->pf_moff = nullptr;
        c->pf_sets = 0;
        if (cudaMalloc(&c->pf_moff, (size_t)(ns + 1) * 8) == cudaSuccess) c->pf_sets = ns + 1;
        else cudaGetLastError();
    }
    if (!c->pf_S || !c->pf_moff || bytes > c->pf_bytes || ns + 1 > c->pf_sets) return CC_OK;
    CC_CUDA(c, cudaMemcpyAsync(c->pf_moff, c->h_moff.data(), (size_t)(ns + 1) * 8, cudaMemcpyHostToDevice,
                               c->stream));
    pf = PairFactors{c->pf_S, c->pf_moff, (int)a.tau_blocks[TAU_VAR_128]};
    return CC_OK;
}

// K_{h,V} on a level: labels lab (packed order); order = the root-sorted
// order of the mixed kick (its labels at L.klab, prepared by the caller)
static int level_kick(cc_ctx *c, LevelAlloc &a, const int32_t *lab, const int32_t *order, double h,
                      double drift_dt = 0.0)
{
    const cudaStream_t s = c->stream;
    int bin;
    bool timed;
    Level L = a.L;
    if (c->p.precision == CC_PREC_MIXED && !(h < c->p.h_fp64)) {
        const int var = tune_pick(c, TK_MK, a.mk_blocks, a.pairs, &bin, &timed);
        CC_TRY(ensure_kpart(c, a.mk_chunks_max[var], a.F.cap));
        const int ev = ev_begin(c, 1, nullptr, timed ? TK_MK : -1, bin, var, (double)a.pairs);
        launch_kick_mixed(L, a.F, order, a.mk_off[var], (int)a.mk_blocks[var], MK_VAR_CHUNK[var], MK_VAR_SLICE[var],
                          a.mk_chunks_max[var] > 1, c->p.eps * c->p.eps, h, c->d_ctr, c->d_kpart, lab, drift_dt, s,
                          a.Ke > 0 ? &a.cv : nullptr);
        ev_end(c, ev);
    } else {
        // FP64: one shape (32-body i-tiles; the row order fixes the rounding).
        // Without the centre-of-mass approximation each unordered pair's
        // force is computed once for both directions into per-set matrices
        // (while they fit PF_BUDGET), then summed by the kick in its row order.
        L.itile_off = a.k64_off[0];
        L.tile_off = a.tau_off[TAU_VAR_128];
        PairFactors pf{nullptr, nullptr, 0};
        if (a.Ke == 0) CC_TRY(pair_factors(c, a, pf));
        const int ev = ev_begin(c, 1, nullptr, -1, 0, 0, (double)a.pairs);
        launch_kick(L, lab, (int)a.k64_blocks[0], c->p.G, c->p.eps * c->p.eps, h, 0, c->d_ctr, s,
                    a.Ke > 0 ? &a.cv : nullptr, nullptr, pf.S ? &pf : nullptr);
        ev_end(c, ev);
    }
    return CC_OK;
}

static int dkd(cc_ctx *c, LevelAlloc &a, double h)
{
    const cudaStream_t s = c->stream;
    // the centre-of-mass approximation: the eligible components' centres and
    // far matrices at this state (component members are not drifted here)
    CC_TRY(com_prepare(c, a));
    if (c->p.precision == CC_PREC_MIXED && !(h < c->p.h_fp64)) {
        // positions in the root-sorted order of the split (members of one
        // component adjacent: tiles inside one component are skipped); both
        // drifts ride on the copy and on the partial reduce
        launch_prep_kick(a.L, a.F, a.members, a.root, c->p.G, 0.5 * h, s);
        CC_TRY(level_kick(c, a, a.root, a.members, h, 0.5 * h));
        // the FP32 kick left the far pairs out: the monopole kick instead
        if (a.Ke > 0)
            launch_com_apply(a.L, a.members, a.comp_start, a.comp_size, a.d_eq, a.d_cm, a.d_eany, a.Ke, h, s);
        return CC_OK;
    }
    launch_drift(a.L, a.root, 0.5 * h, s);
    CC_TRY(level_kick(c, a, a.root, a.members, h));
    if (a.Ke > 0)
        launch_com_apply(a.L, a.members, a.comp_start, a.comp_size, a.d_eq, a.d_cm, a.d_eany, a.Ke, h, s);
    launch_drift(a.L, a.root, 0.5 * h, s);
    return CC_OK;
}

static int side_stream(cc_ctx *c, int d, cudaStream_t *out)
{
    cudaStream_t &st = c->sides[d];
    if (!st) CC_CUDA(c, cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, c->prio_high));
    *out = st;
    return CC_OK;
}

static int ensure_batch_scratch(cc_ctx *c)
{
    if (c->batch_scr) return CC_OK;
    const size_t bytes = batch_scratch_bytes(c->nsm);
    if (cudaMalloc(&c->batch_scr, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->batch_scr = nullptr;
        return fail(c, CC_E_NOMEM, "device allocation failed (batched-kernel frames)");
    }
    CC_CUDA(c, cudaMemset(c->batch_scr, 0, bytes));  // every scratch slot free
    return CC_OK;
}

static SmallParams small_params(const cc_ctx *c, double h0, int depth0)
{
    SmallParams SP;
    SP.G = c->p.G;
    SP.eps2 = c->p.eps * c->p.eps;
    SP.eta = c->eta_run;
    SP.eta_in = c->p.eta_outside ? 1.0 : c->eta_run;
    SP.h0 = h0;
    SP.near_tol = c->p.near_tol;
    SP.h_fp64 = c->p.h_fp64;
    SP.eta_outside = c->p.eta_outside;
    SP.kepler = c->p.kepler;
    SP.precision = c->p.precision;
    SP.depth0 = depth0;
    SP.max_depth = c->p.max_depth;
    SP.hold = c->p.split == CC_SPLIT_HOLD;
    return SP;
}

static int process(cc_ctx *c, int d, double h, const LevelAlloc *parent)
{
    if (d > c->p.max_depth) return fail(c, CC_E_DEPTH, "recursion deeper than max_depth");
    if (d > c->st.max_depth_seen) c->st.max_depth_seen = d;
    // lv is sized once at init (max_depth + 2 levels) and never reallocates,
    // so references into it stay valid across the recursion
    LevelAlloc &a = c->lv[d];
    const cudaStream_t s = c->stream;
    CC_TRY(split_launch(c, a, h, parent));
    // The integrator lists of the components are built on the device, so the
    // small components' first half (side stream) and the Kepler pairs start
    // while the host waits for the split summary and lays out the large
    // components; they touch disjoint particles.
    const SmallParams SP = small_params(c, 0.5 * h, d + 1);
    const int smax = small_max(c);
    const int bound = a.L.total / 2 + 1;  // components of a split, at most
    const bool small_on = smax >= 2 && d + 1 <= c->p.max_depth;
    if (small_on && smax > 32) CC_TRY(ensure_batch_scratch(c));
    cudaStream_t side = nullptr;
    if (small_on) CC_TRY(side_stream(c, d, &side));
    if (!a.classified)
        launch_classify(a.comp_size, a.d_ncomp, smax, c->p.kepler, a.kqueue, a.kqueue + 2, a.klist, a.slist, s);
    if (small_on) {
        if (!a.ev_ready) {
            CC_CUDA(c, cudaEventCreateWithFlags(&a.ev_ready, cudaEventDisableTiming));
            CC_CUDA(c, cudaEventCreateWithFlags(&a.ev_small, cudaEventDisableTiming));
        }
        CC_CUDA(c, cudaEventRecord(a.ev_ready, s));
        CC_CUDA(c, cudaStreamWaitEvent(side, a.ev_ready, 0));
        const int ev = ev_begin(c, 2, side);
        if (smax > 32)
            launch_batch(a.L, a.members, a.comp_start, a.comp_size, a.slist, a.kqueue + 3, bound, SP, c->d_ctr,
                         a.kqueue + 0, c->d_near_ij, c->d_near_tau, c->near_cap, c->nsm, c->batch_scr, side, 8);
        else
            launch_small(a.L, a.members, a.comp_start, a.comp_size, a.slist, a.kqueue + 3, bound, SP, c->d_ctr,
                         a.kqueue + 0, c->d_near_ij, c->d_near_tau, c->near_cap, c->nsm, side);
        ev_end(c, ev, side);
        CC_CUDA(c, cudaEventRecord(a.ev_small, side));
    }
    if (c->p.kepler) launch_kepler(a.L, a.members, a.comp_start, a.klist, a.kqueue + 2, bound, c->p.G, 0.5 * h, c->d_ctr, s);
    int ncomp = 0;
    CC_TRY(split_finish(c, a, parent, ncomp));
    CC_TRY(com_setup(c, a, ncomp));
    // the host's part: counts, and the layout of the large components
    std::vector<int32_t> &lstart = a.v_lstart, &lsize = a.v_lsize;
    lstart.clear();
    lsize.clear();
    // (the classification's rule: a lone large component stays on the levels)
    int n_solo = 0;
    for (int q = 0; q < ncomp; ++q) n_solo += (a.h_size[q] > BATCH_SOLO && a.h_size[q] <= smax) ? 1 : 0;
    const int slim = batch_limit(smax, n_solo);
    int nk = 0, ns = 0;
    for (int q = 0; q < ncomp; ++q) {
        const int sz = a.h_size[q];
        if (c->p.kepler && sz == 2) ++nk;
        else if (sz <= slim) ++ns;
        else {
            lstart.push_back(a.h_start[q]);
            lsize.push_back(sz);
        }
    }
    const int nl = (int)lsize.size();
    if (ns && !small_on) return fail(c, CC_E_DEPTH, "recursion deeper than max_depth");
    c->st.kepler_calls += 2ull * nk;
    c->st.small_tasks += 2ull * ns;
    if (nl) {
        SetLayout &S = c->lv[d + 1].child_layout;
        make_layout(lsize, S);
        std::memcpy(a.h_lists, lstart.data(), nl * 4);
        CC_CUDA(c, cudaMemcpyAsync(a.lcomp_start, a.h_lists, (size_t)nl * 4, cudaMemcpyHostToDevice, s));
        CC_TRY(upload_layout(c, c->lv[d + 1], S));
    }
    for (int half = 0; half < 2; ++half) {
        if (half == 1) {
            if (small_on) CC_CUDA(c, cudaStreamWaitEvent(s, a.ev_small, 0));
            CC_TRY(dkd(c, a, h));
            if (ns) {
                // second half of the small components on the side stream,
                // overlapping the large components' second half
                CC_CUDA(c, cudaEventRecord(a.ev_ready, s));
                CC_CUDA(c, cudaStreamWaitEvent(side, a.ev_ready, 0));
                const int ev = ev_begin(c, 2, side);
                if (smax > 32)
                    launch_batch(a.L, a.members, a.comp_start, a.comp_size, a.slist, a.kqueue + 3, ns, SP, c->d_ctr,
                                 a.kqueue + 1, c->d_near_ij, c->d_near_tau, c->near_cap, c->nsm, c->batch_scr, side, 8);
                else
                    launch_small(a.L, a.members, a.comp_start, a.comp_size, a.slist, a.kqueue + 3, ns, SP,
                                 c->d_ctr, a.kqueue + 1, c->d_near_ij, c->d_near_tau, c->near_cap, c->nsm, side);
                ev_end(c, ev, side);
                CC_CUDA(c, cudaEventRecord(a.ev_small, side));
            }
            if (nk) launch_kepler(a.L, a.members, a.comp_start, a.klist, a.kqueue + 2, nk, c->p.G, 0.5 * h, c->d_ctr, s);
        }
        if (nl) {
            LevelAlloc &ch = c->lv[d + 1];
            launch_gather(a.L, ch.L, a.members, a.lcomp_start, a.inv, s);
            // first half: the state this split saw, so its edge records
            // (when complete) give the child's split; second half: fresh
            const bool reuse = half == 0 && a.ecount <= a.E.cap;
            CC_TRY(process(c, d + 1, 0.5 * h, reuse ? &a : nullptr));
            launch_scatter(a.L, ch.L, s);
        }
    }
    if (small_on) CC_CUDA(c, cudaStreamWaitEvent(s, a.ev_small, 0));
    return CC_OK;
}

// ------------------------------------------------------------ the OK split
// Bytes of one set's arena: a node of np pairs takes at most 55 np + 192
// bytes (fast flags, particle list, child list, flags, incoming lists and
// runs; nS <= 2 np), and a path of the tree holds at most max_depth + 1
// nodes, none larger than the set's outer-level fast list.
static size_t ok_arena_bytes(long long np, int max_depth)
{
    if (np <= 0) return 0;
    return (size_t)4096 + ((size_t)55 * (size_t)np + 192) * (size_t)(max_depth + 1);
}

static int ok_grow(cc_ctx *c, void **p, size_t bytes)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, CC_E_NOMEM, "device allocation failed (OK split)");
    }
    return CC_OK;
}

// Lists of at most this many pairs go to k_ok_tree (one CTA per set runs
// the rest of the set's tree); longer ones are GPU-wide nodes.
constexpr long long OK_NODE_MIN = 8192;

// evolve_ok of a sorted fast list (all sets) at pivot h, depth `depth`, by
// k_ok_tree: each set's segment of the list and its arena
static int ok_tree_small(cc_ctx *c, const int32_t *list, long long np, double h, int depth)
{
    LevelAlloc &a = c->lv[0];
    const cudaStream_t s = c->stream;
    const int ns = a.L.nsets;
    launch_ok_segments(a.L, list, np, c->ok_seg, s);
    c->ok_hseg.resize(ns + 1);
    c->ok_haoff.resize(ns + 1);
    CC_CUDA(c, cudaMemcpyAsync(c->ok_hseg.data(), c->ok_seg, (size_t)(ns + 1) * 8, cudaMemcpyDeviceToHost, s));
    CC_CUDA(c, cudaStreamSynchronize(s));
    size_t off = 0;
    for (int q = 0; q < ns; ++q) {
        c->ok_haoff[q] = (long long)off;
        off += (ok_arena_bytes(c->ok_hseg[q + 1] - c->ok_hseg[q], c->p.max_depth) + 255) / 256 * 256;
    }
    c->ok_haoff[ns] = (long long)off;
    if (off > c->ok_arena_cap) {
        CC_TRY(ok_grow(c, (void **)&c->ok_arena, off));
        c->ok_arena_cap = off;
    }
    CC_CUDA(c, cudaMemcpyAsync(c->ok_aoff, c->ok_haoff.data(), (size_t)(ns + 1) * 8, cudaMemcpyHostToDevice, s));
    launch_ok_tree(a.L, list, c->ok_seg, c->ok_aoff, c->ok_arena, c->ok_stamp, c->ok_loc, (++c->ok_launch) << 40, h,
                   depth, c->p.max_depth, tau_params(c, h), c->p.G, c->p.eps * c->p.eps, c->d_ctr, c->d_near_ij,
                   c->d_near_tau, c->near_cap, s);
    // (the host-side copies must outlive the asynchronous upload)
    CC_CUDA(c, cudaStreamSynchronize(s));
    return CC_OK;
}

// evolve_ok(F, I, h) of a sorted list I (all sets) at depth `depth`
static int ok_node(cc_ctx *c, const int32_t *list, long long np, double h, int depth)
{
    if (np <= 0) return CC_OK;
    if (depth > c->p.max_depth) return fail(c, CC_E_DEPTH, "recursion deeper than max_depth");
    if (np <= OK_NODE_MIN) return ok_tree_small(c, list, np, h, depth);
    if (np > (1ll << 30)) return fail(c, CC_E_ARG, "OK split: a fast list longer than 2^30 pairs");
    LevelAlloc &a = c->lv[0];
    const cudaStream_t s = c->stream;
    const int total = a.L.total, ns = a.L.nsets;
    if (c->okd.size() < (size_t)c->p.max_depth + 2) c->okd.resize((size_t)c->p.max_depth + 2);
    if (c->ok_hst_total < total + 1 || c->ok_hst_sets < ns + 1) {
        const size_t n8 = (size_t)2 * (total + 1) + 2 * (size_t)(ns + 1);
        CC_TRY(ok_grow(c, (void **)&c->ok_hst, n8 * 8));
        CC_CUDA(c, cudaMemsetAsync(c->ok_hst, 0, n8 * 8, s));
        c->ok_hst_total = total + 1;
        c->ok_hst_sets = ns + 1;
    }
    if (!c->ok_cnt) CC_TRY(ok_grow(c, (void **)&c->ok_cnt, 64));
    {
        cc_ctx::OkDepth &D = c->okd[depth];
        if (D.cap < np) {
            const long long cap = 2 * np;
            CC_TRY(ok_grow(c, (void **)&D.fast, (size_t)cap * 4));
            CC_TRY(ok_grow(c, (void **)&D.pos, (size_t)cap * 4));
            CC_TRY(ok_grow(c, (void **)&D.child, (size_t)cap * 8));
            CC_TRY(ok_grow(c, (void **)&D.S, (size_t)cap * 8));
            CC_TRY(ok_grow(c, (void **)&D.isF, (size_t)cap * 2));
            D.cap = cap;
        }
    }
    if (c->ok_scan_cap < scan_scratch_ints((int)np)) {
        c->ok_scan_cap = 2 * (long long)scan_scratch_ints((int)np);
        CC_TRY(ok_grow(c, (void **)&c->ok_scan, (size_t)c->ok_scan_cap * 4));
    }
    if (c->ok_ndir_cap < np) {
        c->ok_ndir_cap = 2 * np;
        CC_TRY(ok_grow(c, (void **)&c->ok_ndir, (size_t)c->ok_ndir_cap * 16));
        CC_TRY(ok_grow(c, &c->ok_nsort, edge_sort_scratch_bytes(2 * c->ok_ndir_cap)));
    }
    cc_ctx::OkDepth &D = c->okd[depth];  // (okd does not resize below this point)
    unsigned long long *sst = c->ok_hst, *fst = sst + c->ok_hst_total;
    unsigned long long *sys_st = fst + c->ok_hst_total, *sysf_st = sys_st + c->ok_hst_sets;
    const unsigned long long stamp = ++c->ok_node_stamp;
    const TauParams P = tau_params(c, h);
    CC_CUDA(c, cudaMemsetAsync(c->ok_cnt, 0, 32, s));
    launch_okh_split(a.L, list, np, P, stamp, D.fast, D.S, sst, fst, sys_st, sysf_st, c->ok_cnt, c->d_ctr,
                     c->d_near_ij, c->d_near_tau, c->near_cap, s);
    launch_exclusive_scan(D.fast, D.pos, (int)np, c->ok_scan, s);
    unsigned long long hc[4] = {0, 0, 0, 0};
    CC_CUDA(c, cudaMemcpyAsync(hc, c->ok_cnt, 32, cudaMemcpyDeviceToHost, s));
    CC_CUDA(c, cudaStreamSynchronize(s));
    const long long nf = (long long)hc[0], nS = (long long)hc[1];
    launch_okh_compact(list, np, D.fast, D.pos, D.child, D.S, nS, fst, stamp, D.isF, s);
    c->st.splits += hc[2];
    c->st.tau_pairs += (unsigned long long)np;
    c->st.tau_evaluated += (unsigned long long)np;
    c->st.components += hc[3];
    if (depth > c->st.max_depth_seen) c->st.max_depth_seen = depth;
    int32_t *child = D.child, *S = D.S;
    int *fast = D.fast, *pos = D.pos;
    unsigned char *isF = D.isF;
    const double G = c->p.G, eps2 = c->p.eps * c->p.eps;
    for (int half = 0; half < 2; ++half) {
        if (half == 1) {
            launch_okh_drift(a.L, S, nS, isF, 0.5 * h, c->d_ctr, true, s);
            launch_okh_kick(a.L, list, np, fast, pos, np - nf, c->ok_ndir, c->ok_nsort, G, eps2, h, s);
            launch_okh_drift(a.L, S, nS, isF, 0.5 * h, c->d_ctr, false, s);
            c->st.kick_pairs += (unsigned long long)(np - nf);
        }
        CC_TRY(ok_node(c, child, nf, 0.5 * h, depth + 1));
    }
    return CC_OK;
}

// One outer step of the OK split (Sec. 4.2) on level 0 (every set a system):
// the outer level here, the rest of the recursion in k_ok_tree.
static int ok_step(cc_ctx *c)
{
    LevelAlloc &a = c->lv[0];
    const cudaStream_t s = c->stream;
    const double dt = c->p.dt;
    const int total = a.L.total, ns = a.L.nsets;
    if (c->ok_lvl_cap < total + 1) {
        CC_TRY(ok_grow(c, (void **)&c->ok_inv, (size_t)(total + 1) * 4));
        CC_TRY(ok_grow(c, (void **)&c->ok_row, (size_t)(total + 1) * 4));
        CC_TRY(ok_grow(c, (void **)&c->ok_rest, (size_t)(total + 1) * 4));
        CC_TRY(ok_grow(c, (void **)&c->ok_loc, (size_t)(total + 1) * 4));
        CC_TRY(ok_grow(c, (void **)&c->ok_stamp, (size_t)(total + 1) * 8));
        CC_CUDA(c, cudaMemsetAsync(c->ok_stamp, 0, (size_t)(total + 1) * 8, s));
        c->ok_lvl_cap = total + 1;
    }
    if (c->ok_set_cap < ns + 1) {
        CC_TRY(ok_grow(c, (void **)&c->ok_seg, (size_t)(ns + 1) * 8));
        CC_TRY(ok_grow(c, (void **)&c->ok_aoff, (size_t)(ns + 1) * 8));
        c->ok_set_cap = ns + 1;
    }
    if (c->ok_cap == 0) {
        c->ok_cap = std::max<long long>(4096, (long long)total * 4);
        CC_TRY(ok_grow(c, (void **)&c->ok_edges, (size_t)c->ok_cap * 8));
        CC_TRY(ok_grow(c, (void **)&c->ok_rec, (size_t)c->ok_cap * sizeof(EdgeRec)));
        CC_TRY(ok_grow(c, (void **)&c->ok_dir, (size_t)c->ok_cap * 16));
        CC_TRY(ok_grow(c, &c->ok_sort, edge_sort_scratch_bytes(2 * c->ok_cap)));
    }
    if (!c->ok_reccnt) CC_TRY(ok_grow(c, (void **)&c->ok_reccnt, 8));
    // the outer level's tau over every pair of each set, its fast pairs
    const TauParams P = tau_params(c, dt);
    Level UL = a.L;
    UL.tile_off = a.tau_off[TAU_VAR_128];
    const long long ntiles = a.tau_blocks[TAU_VAR_128];
    if (ntiles > 0x7fffffff) return fail(c, CC_E_ARG, "set too large for the tile grid");
    // The certified tau kernel (every split's: the FP64 predicate's
    // decisions) records every fast pair; the record count is the list
    // length (the kernel's edge counter goes to the statistics from the host)
    long long ne = 0;
    for (int pass = 0; pass < 2; ++pass) {
        CC_CUDA(c, cudaMemsetAsync(&c->d_ctr->edges, 0, 8, s));
        // the float-float copy, the forest as singletons, the record count 0
        launch_prep_ff(a.L, a.F, c->p.G, true, s, true, c->ok_reccnt);
        launch_tau_mixed(UL, a.F, (int)ntiles, P, TAU_VAR_128, c->d_ctr, c->d_near_ij, c->d_near_tau, c->near_cap,
                         EdgeList{c->ok_rec, c->ok_reccnt, c->ok_cap}, s);
        unsigned long long e1 = 0;
        CC_CUDA(c, cudaMemcpyAsync(&e1, c->ok_reccnt, 8, cudaMemcpyDeviceToHost, s));
        CC_CUDA(c, cudaStreamSynchronize(s));
        CC_CUDA(c, cudaMemsetAsync(&c->d_ctr->edges, 0, 8, s));
        ne = (long long)e1;
        if (ne <= c->ok_cap) break;
        // more fast pairs than room: grow and redo
        c->ok_cap = 2 * ne;
        CC_TRY(ok_grow(c, (void **)&c->ok_edges, (size_t)c->ok_cap * 8));
        CC_TRY(ok_grow(c, (void **)&c->ok_rec, (size_t)c->ok_cap * sizeof(EdgeRec)));
        CC_TRY(ok_grow(c, (void **)&c->ok_dir, (size_t)c->ok_cap * 16));
        CC_TRY(ok_grow(c, &c->ok_sort, edge_sort_scratch_bytes(2 * c->ok_cap)));
    }
    launch_ok_rec_pairs(c->ok_rec, ne, a.L.gid, c->ok_edges, s);
    launch_ok_level(a.L, c->ok_edges, ne, c->ok_inv, c->ok_dir, c->ok_sort, c->ok_row, c->ok_rest, c->ok_seg,
                    c->d_ctr, s);
    unsigned long long nonempty = 0;
    {
        c->ok_hseg.resize(ns + 1);
        CC_CUDA(c, cudaMemcpyAsync(c->ok_hseg.data(), c->ok_seg, (size_t)(ns + 1) * 8, cudaMemcpyDeviceToHost, s));
        CC_CUDA(c, cudaStreamSynchronize(s));
        for (int q = 0; q < ns; ++q) nonempty += c->ok_hseg[q + 1] > c->ok_hseg[q] ? 1 : 0;
    }
    // the outer level's counts (the nodes below count their own)
    c->st.splits += (unsigned long long)ns;
    c->st.tau_pairs += (unsigned long long)a.pairs;
    c->st.tau_evaluated += (unsigned long long)a.pairs;
    c->st.kick_pairs += (unsigned long long)a.pairs - (unsigned long long)ne;
    c->st.components += nonempty;
    c->st.edges += (unsigned long long)ne;
    const OkView okv{c->ok_row, c->ok_dir};
    Level KL = a.L;
    KL.itile_off = a.k64_off[0];
    KL.tile_off = a.tau_off[TAU_VAR_128];
    PairFactors pf;
    CC_TRY(pair_factors(c, a, pf));
    const double G = c->p.G, eps2 = c->p.eps * c->p.eps;
    for (int half = 0; half < 2; ++half) {
        if (half == 1) {
            // D_{h/2} of the particles without a fast pair, K_h of every
            // slow pair of each set (the fast ones masked), D_{h/2}
            launch_drift_labels(a.L, c->ok_rest, 0.5 * dt, s);
            launch_kick(KL, a.L.gid, (int)a.k64_blocks[0], G, eps2, dt, 0, c->d_ctr, s, nullptr, &okv,
                        pf.S ? &pf : nullptr);
            launch_drift_labels(a.L, c->ok_rest, 0.5 * dt, s);
        }
        CC_TRY(ok_node(c, c->ok_edges, ne, 0.5 * dt, 1));
    }
    return CC_OK;
}

// level-0 layout of the systems
static int setup_systems(cc_ctx *c)
{
    std::vector<int32_t> sizes;
    for (size_t q = 0; q + 1 < c->sys_off.size(); ++q) sizes.push_back((int32_t)(c->sys_off[q + 1] - c->sys_off[q]));
    SetLayout S;
    make_layout(sizes, S);
    CC_TRY(upload_layout(c, c->lv[0], S));
    if (c->d_sys_off) cudaFree(c->d_sys_off);
    c->d_sys_off = nullptr;
    std::vector<int32_t> off(c->sys_off.begin(), c->sys_off.end());
    CC_CUDA(c, cudaMalloc(&c->d_sys_off, off.size() * 4));
    CC_CUDA(c, cudaMemcpyAsync(c->d_sys_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    // Whole-batch mode: when every system fits the batched kernel, an outer
    // step is evolve_cc(system, dt) of every system as one task of one
    // launch, largest first (no host level).  Kepler mode needs three
    // bodies or more (a two-body system's first split decides between the
    // Kepler flow and a kick, which the host level takes).
    if (c->sys_exec) cudaGraphExecDestroy(c->sys_exec);
    c->sys_exec = nullptr;
    if (c->d_sys_tasks) cudaFree(c->d_sys_tasks);
    if (c->d_iota) cudaFree(c->d_iota);
    c->d_sys_tasks = nullptr;
    c->d_iota = nullptr;
    c->sys_batch = false;
    const int smax = small_max(c);
    const int nmin = c->p.kepler ? 3 : 2;
    bool all = smax > 32 && c->p.max_depth >= 0 && c->p.split != CC_SPLIT_OK;
    for (int32_t z : sizes) all = all && z >= nmin && z <= smax;
    if (all) {
        const int ns = (int)sizes.size();
        std::vector<int32_t> order(ns);
        for (int q = 0; q < ns; ++q) order[q] = q;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return size_bucket(sizes[a]) > size_bucket(sizes[b]); });
        // tlist, t_start, t_size, [count, queue]
        std::vector<int32_t> blk(3 * (size_t)ns + 2);
        for (int q = 0; q < ns; ++q) {
            blk[q] = order[q];
            blk[ns + q] = S.start[q];
            blk[2 * ns + q] = sizes[q];
        }
        blk[3 * ns] = ns;
        blk[3 * ns + 1] = 0;
        CC_CUDA(c, cudaMalloc(&c->d_sys_tasks, blk.size() * 4));
        CC_CUDA(c, cudaMemcpy(c->d_sys_tasks, blk.data(), blk.size() * 4, cudaMemcpyHostToDevice));
        std::vector<int32_t> iota(S.total > 0 ? S.total : 1);
        for (size_t k = 0; k < iota.size(); ++k) iota[k] = (int32_t)k;
        CC_CUDA(c, cudaMalloc(&c->d_iota, iota.size() * 4));
        CC_CUDA(c, cudaMemcpy(c->d_iota, iota.data(), iota.size() * 4, cudaMemcpyHostToDevice));
        CC_TRY(ensure_batch_scratch(c));
        c->sys_batch = true;
    }
    return CC_OK;
}

// One outer step of the whole-batch mode on stream s: every system one task,
// evolve_cc(system, dt) split at depth 0 (8 warps per CTA while there are
// fewer systems than SMs: each task's CTA-level phases are then the step's
// critical path)
static void sys_step_launches(cc_ctx *c, cudaStream_t s)
{
    const int ns = (int)c->sys_off.size() - 1;
    int32_t *tk = c->d_sys_tasks;
    launch_pack_state(c->d_x3, c->d_v3, c->d_m, c->n, c->lv[0].L, c->d_sys_off, nullptr, s);
    cudaMemsetAsync(tk + 3 * ns + 1, 0, 4, s);
    const SmallParams SP = small_params(c, c->p.dt, 0);
    launch_batch(c->lv[0].L, c->d_iota, tk + ns, tk + 2 * ns, tk, tk + 3 * ns, ns, SP, c->d_ctr, tk + 3 * ns + 1,
                 c->d_near_ij, c->d_near_tau, c->near_cap, c->nsm, c->batch_scr, s, ns < c->nsm ? 8 : 4);
    launch_unpack_state(c->d_x3, c->d_v3, c->n, c->lv[0].L, s);
}

// The whole-batch step's launch sequence depends on nothing the step
// computes, so it is captured once into a CUDA graph (again when eta
// changes; set_systems drops it) and each outer step is one graph launch,
// with no host round trip between steps.
static int sys_step_graph(cc_ctx *c)
{
    if (c->sys_exec && c->sys_exec_eta == c->eta_run) return CC_OK;
    if (c->sys_exec) cudaGraphExecDestroy(c->sys_exec);
    c->sys_exec = nullptr;
    if (!c->cap_stream) CC_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const unsigned long long g0 = g_launches;
    CC_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    sys_step_launches(c, c->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &g);
    c->sys_exec_launches = g_launches - g0;
    g_launches = g0;  // (captured, not launched)
    if (ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(c, CC_E_CUDA, "capture of the whole-batch step failed");
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->sys_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        c->sys_exec = nullptr;
        cudaGetLastError();
        return fail(c, CC_E_CUDA, "instantiation of the whole-batch step graph failed");
    }
    c->sys_exec_eta = c->eta_run;
    return CC_OK;
}

static int reset_call_counters(cc_ctx *c)
{
    c->launch_mark = g_launches;
    CC_CUDA(c, cudaMemsetAsync(&c->d_ctr->edges, 0, sizeof(unsigned long long) * 2, c->stream));
    return CC_OK;
}

static int harvest_counters(cc_ctx *c)
{
    c->st.launches += g_launches - c->launch_mark;
    c->launch_mark = g_launches;
    DevCounters h;
    CC_CUDA(c, cudaMemcpyAsync(&h, c->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    c->st.edges += h.edges;
    c->st.near_pairs += h.near_pairs;
    c->st.tau_fp64 += h.tau_fp64;
    // sub-recursions run by the small-component kernel
    c->st.tau_pairs += h.small_tau_pairs;
    c->st.kick_pairs += h.small_kick_pairs;
    c->st.drifts += h.small_drifts;
    c->st.splits += h.small_splits;
    c->st.components += h.small_components;
    c->st.kepler_calls += h.small_kepler;
    c->st.tau_evaluated += h.tau_evals;
    if (h.max_depth_seen > c->st.max_depth_seen) c->st.max_depth_seen = h.max_depth_seen;
    if (c->timing) {
        c->tm.small_tau_evaluated += h.small_tau_evals;
        c->tm.small_kick_pairs += h.small_kick_pairs;
    }
    // the centre-of-mass approximation's pairs were counted as kick pairs by
    // the splits (n(n-1)/2 - inner pairs)
    c->st.kick_pairs -= h.com_pairs;
    c->st.com_pairs += h.com_pairs;
    // tau_fp64 .. com_pairs
    static_assert(offsetof(DevCounters, com_pairs) - offsetof(DevCounters, tau_fp64) ==
                      10 * sizeof(unsigned long long),
                  "counter block");
    CC_CUDA(c, cudaMemsetAsync(&c->d_ctr->tau_fp64, 0, sizeof(unsigned long long) * 11, c->stream));
    return CC_OK;
}

// ------------------------------------------------------------ C ABI
extern "C" {

int cc_default_params(cc_params *p)
{
    if (!p) return CC_E_ARG;
    std::memset(p, 0, sizeof(*p));
    p->G = 1.0;
    p->eps = 0.0;
    p->eta = 0.03;
    p->dt = 1.0 / 64.0;
    p->h_fp64 = 0.0;
    p->near_tol = 1e-12;
    p->precision = CC_PREC_FP64;
    p->kepler = 0;
    p->max_depth = 64;
    p->s_small = CC_SMALL_AUTO;
    p->eta_outside = 0;
    p->autotune = 1;
    p->com_max = 32;
    p->theta = 0.0;
    return CC_OK;
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int cc_init(cc_ctx **out, int64_t n, const double *m, const double *x3, const double *v3, const cc_params *p,
            void *stream)
{
    g_init_err.clear();
    if (!out || n < 1 || n > (1 << 28) || !m || !x3 || !v3 || !p) {
        g_init_err = "cc_init: invalid argument";
        return CC_E_ARG;
    }
    *out = nullptr;
    if (!(p->G > 0.0) || !(p->eps >= 0.0) || !finite_pos(p->eta) || !finite_pos(p->dt) || p->max_depth < 0 ||
        p->max_depth > 200 || (p->precision != CC_PREC_FP64 && p->precision != CC_PREC_MIXED) ||
        (p->kepler && p->eps != 0.0) || p->s_small < CC_SMALL_AUTO || p->s_small > BATCH_NMAX || p->edge_rec_max < 0 ||
        p->fault_test < 0 || p->fault_test > 2 ||
        (p->split != CC_SPLIT_CC && p->split != CC_SPLIT_HOLD && p->split != CC_SPLIT_OK) ||
        (p->split != CC_SPLIT_CC && p->kepler) ||
        (p->split == CC_SPLIT_OK && p->precision != CC_PREC_FP64) || !(p->theta >= 0.0) || !std::isfinite(p->theta) ||
        (p->theta > 0.0 && (p->split != CC_SPLIT_CC || p->com_max < 2 || p->com_max > COM_MAX_MEMBERS))) {
        g_init_err = "cc_init: invalid parameters";
        return CC_E_ARG;
    }
    cc_ctx *c = new cc_ctx();
    c->n = n;
    c->p = *p;
    // automatic size limit of the batched kernel: 512 for the mixed form; 32
    // for FP64, where one SM's FP64 rate makes a large on-chip task the
    // critical path of the step
    if (c->p.s_small == CC_SMALL_AUTO) c->p.s_small = c->p.precision == CC_PREC_MIXED ? BATCH_NMAX : 32;
    c->eta_run = p->eta;
    c->p_autotune = p->autotune != 0;
    c->stream = (cudaStream_t)stream;
    auto bail = [&](int code) {
        g_init_err = c->err;
        cc_destroy(c);
        return code;
    };
    if (cudaMalloc(&c->d_x3, 3 * n * 8) != cudaSuccess || cudaMalloc(&c->d_v3, 3 * n * 8) != cudaSuccess ||
        cudaMalloc(&c->d_m, n * 8) != cudaSuccess || cudaMalloc(&c->d_ctr, sizeof(DevCounters)) != cudaSuccess ||
        cudaMalloc(&c->d_near_ij, c->near_cap * 8) != cudaSuccess ||
        cudaMalloc(&c->d_near_tau, c->near_cap * 8) != cudaSuccess ||
        cudaMalloc(&c->d_bad, 16) != cudaSuccess) {
        cudaGetLastError();
        c->err = "cc_init: device allocation failed";
        return bail(CC_E_NOMEM);
    }
    cudaMemsetAsync(c->d_ctr, 0, sizeof(DevCounters), c->stream);
    {
        // the side streams of the small-component kernel get the highest
        // priority: its few long-running blocks take SM slots as soon as the
        // pair kernels' short blocks retire, instead of queueing behind them
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        c->prio_high = greatest;
        c->sides.assign((size_t)p->max_depth + 2, nullptr);
    }
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (c->nsm <= 0) c->nsm = 1;
    }
    c->lv.resize(p->max_depth + 2);
    int rc = cc_set_state(c, 0.0, m, x3, v3);
    if (rc) return bail(rc);
    c->sys_off = {0, n};
    rc = setup_systems(c);
    if (rc) return bail(rc);
    *out = c;
    return CC_OK;
}

int cc_set_systems(cc_ctx *c, const int64_t *sys_off, int64_t nsys)
{
    if (!c || !sys_off || nsys < 1) return c ? fail(c, CC_E_ARG, "cc_set_systems: invalid argument") : CC_E_ARG;
    if (sys_off[0] != 0 || sys_off[nsys] != c->n) return fail(c, CC_E_ARG, "cc_set_systems: bad offsets");
    for (int64_t q = 0; q < nsys; ++q)
        if (sys_off[q + 1] <= sys_off[q]) return fail(c, CC_E_ARG, "cc_set_systems: empty or decreasing system");
    c->sys_off.assign(sys_off, sys_off + nsys + 1);
    return setup_systems(c);
}

int cc_set_stream(cc_ctx *c, void *stream)
{
    if (!c) return CC_E_ARG;
    c->stream = (cudaStream_t)stream;
    return CC_OK;
}

int cc_set_state(cc_ctx *c, double t, const double *m, const double *x3, const double *v3)
{
    if (!c) return CC_E_ARG;
    const int64_t n = c->n;
    if (!std::isfinite(t)) return fail(c, CC_E_NONFINITE, "non-finite time");
    // stage into scratch, validate on the device, then commit
    CC_TRY(ensure_tmp(c, (size_t)n * 8 * 7 + 64));
    double *sm = (double *)c->tmp, *sx = sm + n, *sv = sx + 3 * n;
    if (m) CC_TRY(copy_in(c, sm, m, n * 8));
    if (x3) CC_TRY(copy_in(c, sx, x3, 3 * n * 8));
    if (v3) CC_TRY(copy_in(c, sv, v3, 3 * n * 8));
    CC_CUDA(c, cudaMemsetAsync(c->d_bad, 0, 4, c->stream));
    launch_check_state(m ? sm : nullptr, x3 ? sx : nullptr, v3 ? sv : nullptr, n, c->d_bad, c->stream);
    unsigned bad = 0;
    CC_CUDA(c, cudaMemcpyAsync(&bad, c->d_bad, 4, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad & 2u) return fail(c, CC_E_NONFINITE, "masses must be finite and > 0");
    if (bad) return fail(c, CC_E_NONFINITE, "non-finite position or velocity");
    if (m) CC_CUDA(c, cudaMemcpyAsync(c->d_m, sm, n * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (x3) CC_CUDA(c, cudaMemcpyAsync(c->d_x3, sx, 3 * n * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (v3) CC_CUDA(c, cudaMemcpyAsync(c->d_v3, sv, 3 * n * 8, cudaMemcpyDeviceToDevice, c->stream));
    c->t = t;
    c->perm_age = -1;  // a new state: renew the spatial order
    return CC_OK;
}

int cc_get_state(cc_ctx *c, double *t, double *m, double *x3, double *v3)
{
    if (!c) return CC_E_ARG;
    const int64_t n = c->n;
    if (t) *t = c->t;
    CC_TRY(copy_out(c, m, c->d_m, n * 8));
    CC_TRY(copy_out(c, x3, c->d_x3, 3 * n * 8));
    CC_TRY(copy_out(c, v3, c->d_v3, 3 * n * 8));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

int cc_evolve(cc_ctx *c, double t_end, double eta)
{
    if (!c) return CC_E_ARG;
    if (eta > 0.0) c->eta_run = eta;
    const double span = t_end - c->t;
    if (!(span >= -1e-15)) return fail(c, CC_E_ARG, "cc_evolve: t_end before current time");
    const double q = span / c->p.dt;
    const long long nsteps = std::llround(q);
    if (std::fabs(q - (double)nsteps) > 1e-9 * std::max(1.0, std::fabs(q)))
        return fail(c, CC_E_ARG, "cc_evolve: t_end - t is not a whole number of steps dt");
    CC_TRY(reset_call_counters(c));
    const double t0 = c->t;
    const bool spatial = c->p.precision == CC_PREC_MIXED && c->sys_off.size() == 2 && c->n >= SPATIAL_MIN_N;
    if (c->sys_batch && !spatial && nsteps > 0) {
        // every step one replay of the captured step; device errors are read
        // after the call's last step (the state is undefined after one, as
        // after an error of any step)
        CC_TRY(sys_step_graph(c));
        const unsigned long long ns = (unsigned long long)c->sys_off.size() - 1;
        for (long long k = 0; k < nsteps; ++k) {
            CC_CUDA(c, cudaGraphLaunch(c->sys_exec, c->stream));
            g_launches += c->sys_exec_launches;
            c->st.small_tasks += ns;
        }
        CC_TRY(check_device_error(c));
        c->t = t0 + (double)nsteps * c->p.dt;
        CC_CUDA(c, cudaGetLastError());
        CC_TRY(harvest_counters(c));
        return CC_OK;
    }
    for (long long k = 0; k < nsteps; ++k) {
        if (spatial && (c->perm_age < 0 || c->perm_age >= SPATIAL_RENEW)) {
            if (!c->d_perm) {
                CC_CUDA(c, cudaMalloc(&c->d_perm, (size_t)c->n * 4));
                CC_CUDA(c, cudaMalloc(&c->d_box, 8 * sizeof(unsigned)));
            }
            launch_spatial_order(c->d_x3, c->n, c->d_perm, c->d_box, c->seg_scratch, c->stream);
            c->perm_age = 0;
        }
        launch_pack_state(c->d_x3, c->d_v3, c->d_m, c->n, c->lv[0].L, c->d_sys_off, spatial ? c->d_perm : nullptr,
                          c->stream);
        if (spatial) ++c->perm_age;
        int rc = CC_OK;
        if (c->p.split == CC_SPLIT_OK) {
            rc = ok_step(c);
        } else {
            rc = process(c, 0, c->p.dt, nullptr);
        }
        if (rc) return rc;
        launch_unpack_state(c->d_x3, c->d_v3, c->n, c->lv[0].L, c->stream);
        CC_TRY(check_device_error(c));
        ev_resolve(c);
        c->t = t0 + (double)(k + 1) * c->p.dt;
    }
    CC_CUDA(c, cudaGetLastError());
    CC_TRY(harvest_counters(c));
    return CC_OK;
}

// stage a caller set (ascending ids) into the unit level as one set
static int stage_set(cc_ctx *c, const int32_t *set, int64_t n_set, const int32_t **dset_out)
{
    if (n_set < 1 || n_set > c->n) return fail(c, CC_E_ARG, "set size out of range");
    SetLayout S;
    make_layout(std::vector<int32_t>(1, (int32_t)n_set), S);
    CC_TRY(upload_layout(c, c->unit, S));
    CC_TRY(ensure_tmp(c, (size_t)n_set * 4 * 4 + 64));
    int32_t *dset = (int32_t *)c->tmp;
    if (set) {
        CC_TRY(copy_in(c, dset, set, n_set * 4));
    } else {
        if (n_set != c->n) return fail(c, CC_E_ARG, "NULL set requires n_set == n");
        std::vector<int32_t> all(n_set);
        for (int64_t k = 0; k < n_set; ++k) all[k] = (int32_t)k;
        CC_CUDA(c, cudaMemcpyAsync(dset, all.data(), n_set * 4, cudaMemcpyHostToDevice, c->stream));
        CC_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    CC_CUDA(c, cudaMemsetAsync(c->d_bad, 0, 4, c->stream));
    launch_gather_set(c->d_x3, c->d_v3, c->d_m, c->n, dset, (int)n_set, c->unit.L, c->d_bad, c->stream);
    unsigned bad = 0;
    CC_CUDA(c, cudaMemcpyAsync(&bad, c->d_bad, 4, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, CC_E_ARG, "set ids must be distinct, ascending and in [0, n)");
    if (dset_out) *dset_out = dset;
    return CC_OK;
}

int cc_components(cc_ctx *c, const int32_t *set, int64_t n_set, double h, int32_t *labels_out, int64_t *n_comp)
{
    if (!c || !(h > 0.0) || !std::isfinite(h)) return c ? fail(c, CC_E_ARG, "cc_components: bad argument") : CC_E_ARG;
    CC_TRY(stage_set(c, set, n_set, nullptr));
    CC_TRY(reset_call_counters(c));
    int nc = 0;
    CC_TRY(split_launch(c, c->unit, h, nullptr));
    CC_TRY(split_finish(c, c->unit, nullptr, nc));
    if (labels_out) {
        int32_t *dl = (int32_t *)c->tmp + n_set;
        launch_label_canon(c->unit.L, c->unit.root, dl, (int)n_set, c->stream);
        CC_TRY(copy_out(c, labels_out, dl, n_set * 4));
    }
    if (n_comp) *n_comp = nc;
    CC_TRY(check_device_error(c));
    CC_TRY(harvest_counters(c));
    return CC_OK;
}

int cc_timestep_graph(cc_ctx *c, const int32_t *set, int64_t n_set, double h, int64_t *n_edges, int32_t *edges_out,
                      int64_t cap, int64_t *n_near)
{
    if (!c || !(h > 0.0) || !std::isfinite(h) || cap < 0)
        return c ? fail(c, CC_E_ARG, "cc_timestep_graph: bad argument") : CC_E_ARG;
    CC_TRY(stage_set(c, set, n_set, nullptr));
    // pass 1: count edges (and split, which also fills the union-find)
    CC_TRY(reset_call_counters(c));
    LevelAlloc &u = c->unit;
    const TauParams P = tau_params(c, h);
    const long long nt = (n_set + TAU_TILE - 1) / TAU_TILE;
    Level UL = u.L;
    UL.tile_off = u.tau_off[TAU_VAR_128];  // 128-wide tiles
    launch_init_parent(u.L, nullptr, c->stream);
    launch_tau_hook(UL, (int)(nt * (nt + 1) / 2), P, TAU_VAR_128, c->d_ctr, nullptr, 0, c->d_near_ij,
                    c->d_near_tau, c->near_cap, c->stream);
    DevCounters h1;
    CC_CUDA(c, cudaMemcpyAsync(&h1, c->d_ctr, sizeof(h1), cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    const long long ne = (long long)h1.edges;
    if (n_edges) *n_edges = ne;
    if (n_near) *n_near = (long long)h1.near_pairs;
    c->st.edges += h1.edges;
    c->st.near_pairs += h1.near_pairs;
    c->st.tau_pairs += (unsigned long long)n_set * (n_set - 1) / 2;
    CC_TRY(check_device_error(c));
    if (edges_out && ne > 0) {
        // pass 2: write the edges, then sort them lexicographically
        const size_t need = (size_t)ne * 8 + edge_sort_scratch_bytes(ne) + (size_t)n_set * 16 + 1024;
        CC_TRY(ensure_tmp(c, need));
        int32_t *de = (int32_t *)((char *)c->tmp + (size_t)n_set * 16);
        void *ss = (void *)(de + 2 * ne);
        CC_TRY(reset_call_counters(c));
        launch_init_parent(u.L, nullptr, c->stream);
        launch_tau_hook(UL, (int)(nt * (nt + 1) / 2), P, TAU_VAR_128, c->d_ctr, de, ne, c->d_near_ij,
                        c->d_near_tau, c->near_cap, c->stream);
        int bits = 0;
        while (bits < 31 && (1ll << bits) <= c->n) ++bits;
        launch_sort_edges(de, ne, bits, ss, c->stream);
        CC_TRY(copy_out(c, edges_out, de, (size_t)std::min<long long>(ne, cap) * 8));
        CC_CUDA(c, cudaStreamSynchronize(c->stream));
        CC_TRY(check_device_error(c));
        if (ne > cap) return fail(c, CC_E_CAPACITY, "edges_out too small");
    }
    return CC_OK;
}

int cc_kick(cc_ctx *c, const int32_t *set, int64_t n_set, const int32_t *labels, double h)
{
    if (!c || !labels || !std::isfinite(h)) return c ? fail(c, CC_E_ARG, "cc_kick: bad argument") : CC_E_ARG;
    CC_TRY(stage_set(c, set, n_set, nullptr));
    int32_t *dl = (int32_t *)c->tmp + 2 * n_set + 8;
    dl = (int32_t *)(((uintptr_t)dl + 15) & ~(uintptr_t)15);
    CC_TRY(copy_in(c, dl, labels, n_set * 4));
    LevelAlloc &u = c->unit;
    int32_t *order = u.members;
    if (c->p.precision == CC_PREC_MIXED && !(h < c->p.h_fp64)) {
        // the mixed kick works in label-sorted order (members of a group adjacent)
        launch_label_order(dl, (int)n_set, u.L.total, order, c->seg_scratch, c->stream);
        launch_prep_kick(u.L, u.F, order, dl, c->p.G, 0.0, c->stream);
    }
    CC_TRY(level_kick(c, u, dl, order, h));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    ev_resolve(c);
    launch_scatter_set(c->d_x3, c->d_v3, c->n, u.L, (int)n_set, false, true, c->stream);
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int cc_drift(cc_ctx *c, const int32_t *set, int64_t n_set, const int32_t *labels, double h)
{
    if (!c || !labels || !std::isfinite(h)) return c ? fail(c, CC_E_ARG, "cc_drift: bad argument") : CC_E_ARG;
    CC_TRY(stage_set(c, set, n_set, nullptr));
    LevelAlloc &u = c->unit;
    // labels, singleton flags and sort scratch live after the staged set
    int32_t *dl = (int32_t *)c->tmp + 2 * n_set + 8;
    dl = (int32_t *)(((uintptr_t)dl + 15) & ~(uintptr_t)15);
    int32_t *single = dl + n_set + 4;
    void *ss = (void *)(single + n_set + 4);
    const size_t need = (size_t)((char *)ss - (char *)c->tmp) + sort_scratch_bytes(n_set) + (size_t)n_set * 8 + 256;
    if (need > c->tmp_sz) {
        // grow the staging buffer and restage (the set copy lives there)
        CC_TRY(ensure_tmp(c, need));
        CC_TRY(stage_set(c, set, n_set, nullptr));
        dl = (int32_t *)c->tmp + 2 * n_set + 8;
        dl = (int32_t *)(((uintptr_t)dl + 15) & ~(uintptr_t)15);
        single = dl + n_set + 4;
        ss = (void *)(single + n_set + 4);
    }
    CC_TRY(copy_in(c, dl, labels, n_set * 4));
    launch_singleton_from_labels(dl, (int)n_set, single, ss, c->stream);
    launch_drift_labels(u.L, single, h, c->stream);
    launch_scatter_set(c->d_x3, c->d_v3, c->n, u.L, (int)n_set, true, false, c->stream);
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int cc_stats(cc_ctx *c, cc_stats_t *out)
{
    if (!c || !out) return CC_E_ARG;
    *out = c->st;
    return CC_OK;
}

int cc_reset_stats(cc_ctx *c)
{
    if (!c) return CC_E_ARG;
    std::memset(&c->st, 0, sizeof(c->st));
    return CC_OK;
}

int cc_energy(cc_ctx *c, double *E, double *P3, double *L3)
{
    if (!c) return CC_E_ARG;
    const int nb = energy_blocks(c->n);
    if (nb > c->partial_cap) {
        if (c->d_partial) cudaFree(c->d_partial);
        c->d_partial = nullptr;
        CC_CUDA(c, cudaMalloc(&c->d_partial, (size_t)nb * 8 * 8));
        c->partial_cap = nb;
    }
    launch_energy(c->d_x3, c->d_v3, c->d_m, c->n, c->p.G, c->p.eps * c->p.eps, c->d_sys_off,
                  (int)c->sys_off.size() - 1, c->d_partial, nb, c->stream);
    std::vector<double> h((size_t)nb * 8);
    CC_CUDA(c, cudaMemcpyAsync(h.data(), c->d_partial, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 8; ++k) acc[k] += h[(size_t)b * 8 + k];
    if (E) *E = acc[0] + acc[1];
    if (P3) { P3[0] = acc[2]; P3[1] = acc[3]; P3[2] = acc[4]; }
    if (L3) { L3[0] = acc[5]; L3[1] = acc[6]; L3[2] = acc[7]; }
    return CC_OK;
}

int cc_near_pairs(cc_ctx *c, int32_t *pairs, double *tau, int64_t cap, int64_t *n)
{
    if (!c || cap < 0) return CC_E_ARG;
    unsigned long long cnt = 0;
    CC_CUDA(c, cudaMemcpyAsync(&cnt, &c->d_ctr->near_pairs, 8, cudaMemcpyDeviceToHost, c->stream));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    if (n) *n = (int64_t)cnt;
    const long long k = std::min<long long>(std::min<long long>((long long)cnt, cap), c->near_cap);
    if (pairs) CC_TRY(copy_out(c, pairs, c->d_near_ij, (size_t)k * 8));
    if (tau) CC_TRY(copy_out(c, tau, c->d_near_tau, (size_t)k * 8));
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    return CC_OK;
}

int cc_set_timing(cc_ctx *c, int on)
{
    if (!c) return CC_E_ARG;
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    ev_resolve(c);
    c->timing = on != 0;
    std::memset(&c->tm, 0, sizeof(c->tm));
    return CC_OK;
}

int cc_timing(cc_ctx *c, cc_timing_t *out)
{
    if (!c || !out) return CC_E_ARG;
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    ev_resolve(c);
    *out = c->tm;
    return CC_OK;
}

int cc_tuning(cc_ctx *c, cc_tune_entry_t *out, int64_t cap, int64_t *n_out)
{
    if (!c || !n_out || cap < 0 || (!out && cap > 0)) return CC_E_ARG;
    CC_CUDA(c, cudaStreamSynchronize(c->stream));
    ev_resolve(c);
    static_assert((int)TK_TAU64 == (int)CC_TUNE_TAU_FP64 && (int)TK_TAUMIX == (int)CC_TUNE_TAU_MIXED &&
                      (int)TK_K64 == (int)CC_TUNE_KICK_FP64 && (int)TK_MK == (int)CC_TUNE_KICK_MIXED,
                  "tuner kinds");
    int64_t n = 0;
    for (int k = 0; k < TK_N; ++k)
        for (int b = 0; b < TUNE_BINS; ++b) {
            const TuneCell &t = c->tuner.cell[k][b];
            const int nv = TUNE_NVAR[k];
            bool any = false;
            for (int v = 0; v < nv; ++v) any = any || t.timed[v] > 0;
            if (!any) continue;
            if (n < cap) {
                cc_tune_entry_t e{};
                e.kernel = k;
                e.bin = b;
                e.best = t.best;
                e.nvar = nv;
                for (int v = 0; v < nv; ++v) {
                    e.shape[v] = (k == TK_TAU64 || k == TK_TAUMIX) ? TAU_VAR_T[v]
                                 : k == TK_K64                    ? K64_VAR_T[v]
                                                                  : MK_VAR_CHUNK[v];
                    e.slices[v] = k == TK_TAUMIX ? TAU_VAR_S[v] : k == TK_MK ? MK_VAR_SLICE[v] : 1;
                    e.timed[v] = t.timed[v];
                    e.us_per_mpair[v] = t.timed[v] > 0 ? 1e9 * t.qmin[v] : 0.0;
                }
                out[n] = e;
            }
            ++n;
        }
    *n_out = n;
    return CC_OK;
}

int cc_destroy(cc_ctx *c)
{
    if (!c) return CC_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->sys_exec) cudaGraphExecDestroy(c->sys_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaStream_t st : c->sides)
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (cudaEvent_t e : c->evs) cudaEventDestroy(e);
    for (auto &a : c->lv) free_level(a);
    free_level(c->unit);
    void *ptrs[] = {c->d_x3, c->d_v3, c->d_m, c->d_ctr, c->d_near_ij, c->d_near_tau, c->d_partial,
                    c->tmp, c->seg_scratch, c->d_sys_off, c->d_bad, c->d_kpart, c->pf_S, c->pf_moff, c->d_perm, c->d_box,
                    c->batch_scr, c->d_sys_tasks, c->d_iota, c->ok_edges, c->ok_rec, c->ok_reccnt, c->ok_dir, c->ok_sort,
                    c->ok_inv, c->ok_row, c->ok_rest, c->ok_loc, c->ok_stamp, c->ok_seg, c->ok_aoff,
                    c->ok_arena, c->ok_hst, c->ok_cnt, c->ok_scan, c->ok_ndir, c->ok_nsort};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (auto &D : c->okd) {
        void *dp[] = {D.fast, D.pos, D.child, D.S, D.isF};
        for (void *q : dp)
            if (q) cudaFree(q);
    }
    delete c;
    return CC_OK;
}

int cc_probe_peaks(void *stream, double *fp64_flops, double *fp32_flops)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
        cudaGetLastError();
        g_init_err = "cc_probe_peaks: no CUDA device";
        return CC_E_CUDA;
    }
    if (fp64_flops) *fp64_flops = probe_fma(1, nsm, (cudaStream_t)stream);
    if (fp32_flops) *fp32_flops = probe_fma(0, nsm, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) {
        g_init_err = "cc_probe_peaks: kernel failed";
        return CC_E_CUDA;
    }
    return CC_OK;
}

const char *cc_last_error(cc_ctx *c)
{
    if (!c) return g_init_err.c_str();
    return c->err.c_str();
}

}  // extern "C"
