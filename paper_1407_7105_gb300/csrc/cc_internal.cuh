// cc_internal.cuh -- device helpers and kernel launchers shared by the
// translation units of libcc.so (CC split integrator, arXiv:1407.7105).
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "../../include/cc.h"

namespace cc {

// ---------------------------------------------------------------- layout
// A level buffer holds one batch of disjoint sets packed contiguously in
// SoA form.  Every set starts at a multiple of SET_ALIGN elements so that
// j-tiles of the double and int32 arrays start on 16-byte boundaries (TMA
// bulk copies).  Padding elements carry gid = -1.
constexpr int SET_ALIGN = 4;
constexpr int PAD_TAIL = 256;  // slack past the last element (tile over-reads)
// mixed form: level 0 of a single system of at least SPATIAL_MIN_N bodies is
// packed in a Morton order of the positions, renewed every SPATIAL_RENEW
// outer steps (the bodies move little in between; any order is correct)
constexpr long long SPATIAL_MIN_N = 2048;
constexpr long long SPATIAL_RENEW = 8;

struct Level {
    double *x, *y, *z, *vx, *vy, *vz, *m;  // packed state, cap entries each
    int32_t *gid;      // particle id, -1 = padding
    int32_t *sidx;     // set index of the element, -1 = padding
    int32_t *src;      // index in the parent level the element came from
    int32_t *parent;   // union-find forest over packed indices
    int32_t *cnt;      // component size, indexed by root
    int32_t *klab;     // mixed kick: label (root) by position of the root-sorted order
    int32_t *set_start, *set_n;      // [nsets]
    int32_t *tile_off;               // [nsets+1] triangular tau tiles prefix
    int32_t *itile_off;              // [nsets+1] i-tiles prefix (kick)
    int32_t *koff;                   // [nsets+1] mixed-kick blocks prefix
    int32_t total;                   // packed length including padding
    int32_t nsets;
};

// float-float copy of a level (mixed-precision kernels), two float4 per
// particle and quantity so that one j costs four 16-byte shared loads:
//   pq[2k] = (x_hi, y_hi, z_hi, G m),  pq[2k+1] = (x_lo, y_lo, z_lo, 0)
//   vq[2k] = (vx_hi, vy_hi, vz_hi, 0), vq[2k+1] = (vx_lo, vy_lo, vz_lo, 0)
// with hi = fl32(x), lo = fl32(x - hi); maxes = max |x|, max |v| of the
// level (float bit patterns, for the error bounds)
struct FFView {
    float4 *pq, *vq;
    float *maxes;
    int cap;
};

// Edge record of a split at pivot h: packed indices a < b of the level
// (tau(a,b) < h); tau in FP64 when it was evaluated (NaN when a certified
// FP32 decision settled the edge); e = the edge depth when known (the pair
// is an edge at h 2^-m exactly for m < e, saturating at EDGE_E_INF), -1
// when not.  The first-half split of a component at h/2 sees the same
// state, so its edges are the records that are edges at h/2, and its
// near-threshold pairs (tau within near_tol of h/2) are records too.
constexpr int EDGE_E_INF = 1 << 20;
struct EdgeRec {
    int32_t a, b, e, pad;
    double tau;
};
struct EdgeList {
    EdgeRec *rec;                  // [cap]
    unsigned long long *count;     // records offered (may exceed cap: list incomplete)
    long long cap;
};

// bounded-wait error codes written to the device error word
enum DevErr : unsigned {
    DERR_NONE = 0,
    DERR_TMA_TIMEOUT = 1,
    DERR_UF_RETRY = 2,
    DERR_KEPLER = 3,
    DERR_DEPTH = 4,
    DERR_SMALL_OVERFLOW = 5,
};

struct DevCounters {
    unsigned long long edges;
    unsigned long long near_pairs;
    unsigned long long tau_fp64;
    unsigned long long near_logged;
    unsigned long long small_tau_pairs;
    unsigned long long small_kick_pairs;
    unsigned long long small_drifts;
    unsigned long long small_kepler;
    unsigned long long small_splits;
    unsigned long long small_components;
    unsigned long long tau_evals;  // pairs whose tau the small kernel or the edge-record pass evaluated
    unsigned long long small_tau_evals;  // of those, the small kernel's
    unsigned long long com_pairs;        // body pairs the centre-of-mass approximation took
    unsigned int err;
    int max_depth_seen;
};

// parameters of the small-component kernel: h0 is the pivot of the
// components it receives (half the parent's), depth0 their recursion depth
struct SmallParams {
    double G, eps2, eta, eta_in, h0, near_tol, h_fp64;
    int eta_outside, kepler, precision, depth0, max_depth;
    int hold;  // HOLD split: a set's members with an edge form one fast set
};

struct TauParams {
    double G, eps2, eta_in, eta, h, near_tol;
    int eta_outside;
    int fault_test;  // failure-path test hooks of the tau kernels (cc_params.fault_test)
};

// --------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void raise_err(DevCounters *c, unsigned code)
{
    atomicCAS(&c->err, 0u, code);
}

// mbarrier + TMA bulk copy (sm_90+ PTX, used unchanged on sm_103a)
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// wait for the phase with the given parity; gives up after ~limit cycles
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit_cycles)
{
    unsigned a = smem_u32(bar);
    long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - t0 > limit_cycles) return false;
    }
}
constexpr long long TMA_WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
// the shortened wait of the fault_test = 1 hook: a copy that is never issued
constexpr long long FAULT_TEST_WAIT_CYCLES = 1LL << 20;
// union-find: compare-and-swap attempts before a hook gives up
constexpr int UF_RETRY_MAX = 1 << 24;

// ------------------------------------------------- FP64 tau(i,j), exact
// Eq. (tauij) with the free-fall / flyby times derived from first principles
// (T_ff = eta sqrt(r^3/mu), T_fb = eta r/|dv|, their time derivatives along
// the pair's own motion, dT/dt clamped at 1); the operations and their order are fixed (no FMA: explicit _rn intrinsics)
// so that the predicate tau < h is bit-identical to a plain IEEE-754
// evaluation of:
//   r2 = ((dx0*dx0 + dx1*dx1) + dx2*dx2) + eps2;  r = sqrt(r2)
//   v2 = (dv0*dv0 + dv1*dv1) + dv2*dv2;  rv = (dx0*dv0 + dx1*dv1) + dx2*dv2
//   mu = G*(mi + mj)
//   Tff = eta_in*sqrt((r2*r)/mu);  dTff = ((1.5*Tff)*rv)/r2
//   Tfb = eta_in*(r/sqrt(v2));  dTfb = (Tfb*(rv/r2))*(1 + mu/(r*v2))   [v2 > 0]
//   tau_x = T_x/(1 - 0.5*min(dT_x, 1));  tau = min(tau_ff, tau_fb) [* eta]
__device__ __forceinline__ double tau_fp64(double dx0, double dx1, double dx2, double dv0, double dv1,
                                           double dv2, double mi, double mj, const TauParams &P)
{
    double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)), __dmul_rn(dx2, dx2)),
                          P.eps2);
    double r = __dsqrt_rn(r2);
    double v2 = __dadd_rn(__dadd_rn(__dmul_rn(dv0, dv0), __dmul_rn(dv1, dv1)), __dmul_rn(dv2, dv2));
    double rv = __dadd_rn(__dadd_rn(__dmul_rn(dx0, dv0), __dmul_rn(dx1, dv1)), __dmul_rn(dx2, dv2));
    double mu = __dmul_rn(P.G, __dadd_rn(mi, mj));
    double Tff = __dmul_rn(P.eta_in, __dsqrt_rn(__ddiv_rn(__dmul_rn(r2, r), mu)));
    double dTff = __ddiv_rn(__dmul_rn(__dmul_rn(1.5, Tff), rv), r2);
    double c1 = dTff < 1.0 ? dTff : 1.0;
    double tff = __ddiv_rn(Tff, __dsub_rn(1.0, __dmul_rn(0.5, c1)));
    double tfb = CUDART_INF;
    if (v2 > 0.0) {
        double Tfb = __dmul_rn(P.eta_in, __ddiv_rn(r, __dsqrt_rn(v2)));
        double dTfb = __dmul_rn(__dmul_rn(Tfb, __ddiv_rn(rv, r2)), __dadd_rn(1.0, __ddiv_rn(mu, __dmul_rn(r, v2))));
        double c2 = dTfb < 1.0 ? dTfb : 1.0;
        tfb = __ddiv_rn(Tfb, __dsub_rn(1.0, __dmul_rn(0.5, c2)));
    }
    double t = tff < tfb ? tff : tfb;
    if (P.eta_outside) t = __dmul_rn(P.eta, t);
    return t;
}

// -------------------------------------------------------- union-find
// Forest over packed indices; every link goes from a larger root to a
// smaller one, so parent[x] <= x and a root is the smallest index of its
// tree.  find() halves paths; the halving stores only ever point a node
// to one of its own ancestors, so racing finds stay correct.
__device__ __forceinline__ int uf_find(int32_t *parent, int x)
{
    volatile int32_t *par = parent;
    int p = par[x];
    if (p != x) {
        int prev = x, nx;
        while (p > (nx = par[p])) {
            par[prev] = nx;
            prev = p;
            p = nx;
        }
    }
    return p;
}

// Union of the trees of a and b: link the larger root under the smaller one
// with compare-and-swap, retrying from the new parent on contention.
__device__ __forceinline__ bool uf_union(int32_t *parent, int a, int b, int retry_max = UF_RETRY_MAX)
{
    int ra = uf_find(parent, a), rb = uf_find(parent, b);
    for (int it = 0;; ++it) {
        if (ra == rb) return true;
        if (it >= retry_max) return false;
        if (ra < rb) {
            int old = atomicCAS(&parent[rb], rb, ra);
            if (old == rb) return true;
            rb = uf_find(parent, old);
        } else {
            int old = atomicCAS(&parent[ra], ra, rb);
            if (old == ra) return true;
            ra = uf_find(parent, old);
        }
    }
}

// The same forest operations reading through L1 (ld.global.ca), for passes
// in which thousands of finds end on one root: volatile reads all go to the
// L2 slice holding that root's line and queue there.  A stale read is safe:
// every pointer ever stored points to a smaller index of the same tree, so
// a find still terminates inside the tree, and the hook's compare-and-swap
// (performed at L2) rejects a root that is no longer one.  (Callers keep
// the trees shallow; see the min-neighbour links of the first-half split.)
__device__ __forceinline__ int uf_find_ca(const int32_t *parent, int x)
{
    // no path halving: its stores would queue at the same L2 lines
    int p = __ldca(parent + x), nx;
    while (p > (nx = __ldca(parent + p))) p = nx;
    return p;
}

__device__ __forceinline__ bool uf_union_ca(int32_t *parent, int a, int b)
{
    int ra = uf_find_ca(parent, a), rb = uf_find_ca(parent, b);
    for (int it = 0; it < UF_RETRY_MAX; ++it) {
        if (ra == rb) return true;
        if (ra < rb) {
            int old = atomicCAS(&parent[rb], rb, ra);
            if (old == rb) return true;
            rb = uf_find_ca(parent, old);
        } else {
            int old = atomicCAS(&parent[ra], ra, rb);
            if (old == ra) return true;
            ra = uf_find_ca(parent, old);
        }
    }
    return false;
}

// ----------------------------------------------------------- launchers
// Every launcher adds the number of kernels it launched to g_launches.
extern unsigned long long g_launches;
#define CC_COUNT_LAUNCH(k) (::cc::g_launches += (k))

// cc_pair.cu
void launch_init_parent(const Level &L, unsigned long long *edge_count, cudaStream_t s);
// tunable launch shapes (variant index): tau tiles {64, 128, 64 in two
// column slices}; FP64 kick tiles {32, 64, 128}; mixed kick (j-chunk in
// tiles of 128, column slices) {(1, 1), (4, 1), (1, 4)}
constexpr int N_TAU_VAR = 3, N_K64_VAR = 3, N_MK_VAR = 3;
// tau variants: tile edge T and column slices S per tile row (the FP64
// kernel takes the first two)
constexpr int TAU_VAR_T[N_TAU_VAR] = {64, 128, 64};
constexpr int TAU_VAR_S[N_TAU_VAR] = {1, 1, 2};
constexpr int N_TAU64_VAR = 2, TAU_VAR_128 = 1;
static_assert(TAU_VAR_T[TAU_VAR_128] == 128 && TAU_VAR_S[TAU_VAR_128] == 1, "128-wide tau tiles");
constexpr int K64_VAR_T[N_K64_VAR] = {32, 64, 128};
constexpr int MK_VAR_CHUNK[N_MK_VAR] = {1, 4, 1};
constexpr int MK_VAR_SLICE[N_MK_VAR] = {1, 1, 4};
constexpr int MK_TILE = 128;
void launch_tau_hook(const Level &L, int ntiles, const TauParams &P, int variant, DevCounters *ctr,
                     int32_t *edges, long long edge_cap, int32_t *near_ij, double *near_tau, long long near_cap,
                     cudaStream_t s, const EdgeList *rec = nullptr);
// first-half split from the parent split's edge records: the records that
// are edges at P.h and whose endpoints the gather moved to this level (inv =
// parent index -> child index) are hooked and recorded for this split
// (PF = the parent's float-float view, valid for records of a fresh mixed
// split: their FP32 decisions at h/2, h/4, ... are taken from it)
void launch_edges_reuse(const EdgeList &parent, long long pcount, const Level &PL, const FFView &PF, bool mixed,
                        const int32_t *inv, const Level &C, const EdgeList &child, const TauParams &P,
                        DevCounters *ctr, int32_t *near_ij, double *near_tau, long long near_cap, cudaStream_t s,
                        bool hook = true);
// centre-of-mass approximation of V_CC (Sec. 4.1): a level's eligible
// components (2..com_max members, in a set of more than COM_MIN_SET - 1
// members) have a local index within their set; two of them are far when
// R_a + R_b < theta |X_a - X_b| (far[foff[s] + a K[s] + b] = 1).  cl = null:
// the approximation is off.
constexpr int COM_MIN_SET = 33;
constexpr int COM_MAX_MEMBERS = 64;
struct ComView {
    const int32_t *cl;          // per packed element: local eligible index, -1
    const long long *foff;      // per set: offset of its far matrix
    const int32_t *K;           // per set: eligible components
    const unsigned char *far;   // far matrices, K x K bytes per set
};
// OK split (Sec. 4.2): the fast pairs of the outer level, both directions
// sorted by (row, partner) in col (pairs), rows delimited by row_ptr
struct OkView {
    const int32_t *row_ptr;  // [total + 1]
    const int32_t *col;      // (row, partner) pairs
};
// FP64 kick: the force G m_j r_ij^-3 (x_j - x_i) of every ordered pair (i, j)
// of each set, precomputed (k_pair_forces)
struct PairFactors {
    double *S;               // per set: three n x n matrices (x, y, z), row-major
    const long long *moff;   // per set: offset of its matrix in S
    int nblocks;             // k_pair_forces' grid: the level's 128-wide triangular tiles
};
void launch_kick(const Level &L, const int32_t *label, int nitiles, double G, double eps2, double h,
                 int variant, DevCounters *ctr, cudaStream_t s, const ComView *com = nullptr,
                 const OkView *okv = nullptr,
                 const PairFactors *pf = nullptr);
// the OK split's outer level after its tau kernel wrote the fast pairs
// (particle ids, count ne): pairs to packed indices and sorted, both
// directions sorted (dir, 2 ne pairs), row pointers, the drift flags of the
// particles without a fast partner (rest), each set's segment of the list
// the certified tau kernel's edge records -> particle-id pairs (OK split's outer level)
void launch_ok_rec_pairs(const EdgeRec *rec, long long ne, const int32_t *gid, int32_t *edges, cudaStream_t s);
void launch_ok_level(const Level &L, int32_t *edges, long long ne, int32_t *inv, int32_t *dir, void *sort_scratch,
                     int32_t *row_ptr, int32_t *rest, long long *seg, DevCounters *ctr, cudaStream_t s);
// a node of the OK recursion on the whole GPU (lists too long for one CTA):
// the split (fast flags, the node's particles S, per-set presence counts in
// counters = {nf, nS, nsys, nsysf}, u64, zeroed by the caller), the child
// list and the F flags of S, the drifts of S \ F, the kick of the slow pairs
void launch_okh_split(const Level &L, const int32_t *list, long long np, const TauParams &P, unsigned long long stamp,
                      int *fast, int32_t *S, unsigned long long *sst, unsigned long long *fst,
                      unsigned long long *sys_st, unsigned long long *sysf_st, void *counters, DevCounters *ctr,
                      int32_t *near_ij, double *near_tau, long long near_cap, cudaStream_t s);
void launch_okh_compact(const int32_t *list, long long np, const int *fast, const int *pos, int32_t *child,
                        const int32_t *S, long long nS, const unsigned long long *fst, unsigned long long stamp,
                        unsigned char *isF, cudaStream_t s);
void launch_okh_drift(const Level &L, const int32_t *S, long long nS, const unsigned char *isF, double dt,
                      DevCounters *ctr, bool count, cudaStream_t s);
void launch_okh_kick(const Level &L, const int32_t *list, long long np, const int *fast, const int *pos,
                     long long ns, int32_t *dir, void *sort_scratch, double G, double eps2, double h, cudaStream_t s);
void launch_ok_segments(const Level &L, const int32_t *list, long long np, long long *seg, cudaStream_t s);
// the rest of the OK recursion: one CTA per set evolves (F, I_F) of its
// segment of the sorted fast list at pivot h0 (depth depth0), node arrays in
// the set's arena [arena_off[s], arena_off[s+1])
void launch_ok_tree(const Level &L, const int32_t *list, const long long *seg, const long long *arena_off,
                    char *arena, unsigned long long *stamp, int32_t *loc, unsigned long long stamp_base, double h0,
                    int depth0, int max_depth, const TauParams &P, double G, double eps2, DevCounters *ctr,
                    int32_t *near_ij, double *near_tau, long long near_cap, cudaStream_t s);
void launch_energy(const double *x3, const double *v3, const double *m, long long n, double G, double eps2,
                   const int32_t *sys_off /* nsys + 1 offsets, or null */, int nsys, double *partial /*[nblk*8]*/,
                   int nblk, cudaStream_t s);
int energy_blocks(long long n);

// cc_graph.cu
void launch_compress(const Level &L, int32_t *root, cudaStream_t s);
void launch_drift(const Level &L, const int32_t *root, double dt, cudaStream_t s);
void launch_drift_labels(const Level &L, const int32_t *singleton, double dt, cudaStream_t s);
// stable segmentation of the components of a level; returns via device
// arrays: comp_start/comp_size (ncomp on device at *d_ncomp) and the sorted
// member list (packed indices).  scratch must hold seg_scratch_bytes(cap).
size_t seg_scratch_bytes(int cap);
void launch_segment(const Level &L, const int32_t *root, int32_t *members, int32_t *comp_start,
                    int32_t *comp_size, int32_t *d_ncomp, void *scratch, cudaStream_t s);
// Batches of at most a one-CTA size are segmented by one CTA with the
// level's union-find in shared memory; there it can also hook a first
// half's child edges (segment_hooks_edges(total) tells whether it will:
// then launch_edges_reuse leaves the hooks to it).
bool segment_hooks_edges(int total);
// The batched small-component kernel takes tasks (components, or whole
// systems) of up to BATCH_NMAX bodies; the classification orders them
// largest first by size_bucket (exact up to 32 bodies, bins of 16 above).
constexpr int BATCH_NMAX = 512;
__host__ __device__ constexpr int size_bucket(int sz) { return sz <= 32 ? sz : 32 + (sz - 17) / 16; }
constexpr int CLS_NB = size_bucket(BATCH_NMAX) + 1;
constexpr int CLS_SH = 2 * CLS_NB + 2;
// A component of more than BATCH_SOLO bodies goes to the batched kernel only
// when at least BATCH_SOLO_MIN such components of the split share its
// launch: alone, one CTA's whole recursion of a few hundred bodies is longer
// than the GPU-wide levels (the paper's 1024-body step: 1.19 s with every
// component of <= 512 bodies in the batched kernel, 0.70 s with <= 128).
// The device classification and the host's lists apply the same rule.
constexpr int BATCH_SOLO = 128, BATCH_SOLO_MIN = 8;
__host__ __device__ constexpr int batch_limit(int smax, int n_above_solo)
{
    return (smax > BATCH_SOLO && n_above_solo < BATCH_SOLO_MIN) ? BATCH_SOLO : smax;
}
// where the classification (see launch_classify) writes its lists
struct ClassifyArgs {
    int s_small, kepler;
    int32_t *queue, *counts, *klist, *slist;
};
// returns true when the segmenting CTA also classified the components
// (cls given and the batch segmented by one CTA)
bool launch_compress_segment(const Level &L, int32_t *root, int32_t *members, int32_t *comp_start,
                             int32_t *comp_size, int32_t *d_ncomp, void *scratch, cudaStream_t s,
                             const EdgeList *hook = nullptr, DevCounters *ctr = nullptr,
                             const ClassifyArgs *cls = nullptr);
// HOLD split (Sec. 2.1): join every non-trivial component of a set into one
// (the fast set F = the members with an edge), rooted at its smallest
// index; anchor: nsets ints of scratch
void launch_hold_merge(const Level &L, int32_t *anchor, cudaStream_t s);
void launch_gather(const Level &P, const Level &C, const int32_t *members, const int32_t *lcomp_start, int32_t *inv,
                   cudaStream_t s);
void launch_scatter(const Level &P, const Level &C, cudaStream_t s);
// integrator lists of a split's components on the device (Kepler pairs,
// small components largest first), their counts and the small kernel's
// zeroed queue counters
void launch_classify(const int32_t *comp_size, const int32_t *ncomp, int s_small, int kepler, int32_t *queue,
                     int32_t *counts, int32_t *klist, int32_t *slist, cudaStream_t s);
void launch_pack_state(const double *x3, const double *v3, const double *m, long long n, const Level &L,
                       const int32_t *sys_off, const int32_t *perm, cudaStream_t s);
// Morton ranking of the particles by position (perm[id] = rank); scratch
// holds 8 n bytes + sort_scratch_bytes(n); box: 6 unsigned of device memory
void launch_spatial_order(const double *x3, long long n, int32_t *perm, unsigned *box, void *scratch,
                          cudaStream_t s);
size_t sort_scratch_bytes(long long n);
void launch_unpack_state(double *x3, double *v3, long long n, const Level &L, cudaStream_t s);
void launch_gather_set(const double *x3, const double *v3, const double *m, long long n, const int32_t *set,
                       int nset, const Level &L, unsigned *bad, cudaStream_t s);
void launch_scatter_set(double *x3, double *v3, long long n, const Level &L, int nset, bool write_x,
                        bool write_v, cudaStream_t s);
void launch_label_canon(const Level &L, const int32_t *root, int32_t *labels_out, int nset, cudaStream_t s);
void launch_singleton_from_labels(const int32_t *labels, int n, int32_t *singleton, void *scratch,
                                  cudaStream_t s);
void launch_label_order(const int32_t *labels, int n, int total, int32_t *order, void *scratch, cudaStream_t s);
void launch_sort_edges(int32_t *edges, long long ne, int bits, void *scratch, cudaStream_t s);
// exclusive prefix sums of n ints (scratch: scan_scratch_ints(n) ints)
int scan_scratch_ints(int n);
void launch_exclusive_scan(const int *in, int *out, int n, int *scratch, cudaStream_t s);
size_t edge_sort_scratch_bytes(long long ne);
void launch_check_state(const double *m, const double *x3, const double *v3, long long n, unsigned *bad,
                        cudaStream_t s);
size_t sort_scratch_bytes(long long n);

double probe_fma(int fp64, int nsm, cudaStream_t s);

// cc_mixed.cu
// init_forest: the same pass also starts the split's union-find (parent[k]
// = k, sizes 0, *edge_count = 0), as launch_init_parent does
void launch_prep_ff(const Level &L, const FFView &F, double G, bool with_v, cudaStream_t s, bool init_forest = false,
                    unsigned long long *edge_count = nullptr);
void launch_tau_mixed(const Level &L, const FFView &F, int ntiles, const TauParams &P, int variant,
                      DevCounters *ctr, int32_t *near_ij, double *near_tau, long long near_cap, const EdgeList &rec,
                      cudaStream_t s);
int mixed_kick_blocks(int n, int chunk, int slices);
int mixed_kick_chunks(int n, int chunk);
// drift_dt > 0: the level's drift of rest-set members (component size 1 by
// root) fused in: before the positions are copied (prep), after the kick
// (the partial reduce, launched for it even without multi-chunk sets)
void launch_prep_kick(const Level &L, const FFView &F, const int32_t *order, const int32_t *root, double G,
                      double drift_dt, cudaStream_t s);
void launch_kick_mixed(const Level &L, const FFView &F, const int32_t *order, const int32_t *koff, int nblocks,
                       int chunk, int slices, bool multi_chunk, double eps2, double h, DevCounters *ctr,
                       double *partial, const int32_t *root, double drift_dt, cudaStream_t s,
                       const ComView *com = nullptr);

// cc_small.cu
// the batched kernel (k_batch): tasks tlist[0..*nt_ptr) (task c: packed
// indices members[t_start[c] ..][0..t_size[c]), ascending id), largest first;
// queue: a zeroed work counter; scratch: batch_scratch_bytes(nsm); warps: 4
// or 8 per CTA (8: shorter CTA-level phases, 4: more resident warp tasks)
size_t batch_scratch_bytes(int nsm);
void launch_batch(const Level &L, const int32_t *members, const int32_t *t_start, const int32_t *t_size,
                  const int32_t *tlist, const int32_t *nt_ptr, int nt_bound, const SmallParams &SP, DevCounters *ctr,
                  int *queue, int32_t *near_ij, double *near_tau, long long near_cap, int nsm, char *scratch,
                  cudaStream_t s, int warps);
void launch_small(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                  const int32_t *slist, const int32_t *ns_ptr, int ns_bound, const SmallParams &SP, DevCounters *ctr,
                  int *queue, int32_t *near_ij, double *near_tau, long long near_cap, int nsm, cudaStream_t s);

// cc_com.cu: the centre-of-mass approximation.  Eligible component g (of Ke)
// is component eq[g] (members[comp_start[q] ..]) of set eset[g] with local
// index eloc[g]; efirst[s] = the first g of set s.  cm: 8 doubles per g
// (M, X, Y, Z, R, Ax, Ay, Az), eany[g] = 1 if g has a far partner.
void launch_com_prep(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                     const int32_t *eq, const int32_t *eloc, int Ke, int32_t *cl, double *cm, cudaStream_t s);
void launch_com_far(double *cm, const int32_t *eq, const int32_t *comp_size, const int32_t *eset,
                    const int32_t *eloc, const int32_t *efirst, const long long *foff, const int32_t *K, int Ke,
                    double theta, double G, double eps2, unsigned char *far, int32_t *eany, DevCounters *ctr,
                    cudaStream_t s, bool mixed);
// v_i += h A_g for the members of every eligible component with a far partner
void launch_com_apply(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                      const int32_t *eq, const double *cm, const int32_t *eany, int Ke, double h, cudaStream_t s);

// cc_kepler.cu
void launch_kepler(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *klist,
                   const int32_t *nk_ptr, int nk_bound, double G, double dt, DevCounters *ctr, cudaStream_t s);

}  // namespace cc
