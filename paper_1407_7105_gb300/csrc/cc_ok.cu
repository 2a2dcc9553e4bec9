// cc_ok.cu -- the OK split (arXiv:1407.7105 Sec. 4.2): the interactions of a
// set, not its particles, partitioned by tau(i,j) against the pivot h.
//
// Reading: the interaction list I of a particle set S (at the outer step:
// every pair of S) splits at pivot h into the fast list I_F = {tau(i,j) < h}
// and the slow list I_S; F = the particles of I_F.  One step is
//     E_{h/2,T_F+V_{I_F}} D_{h/2,T_{S\F}} K_{h,V_{I_S}} D_{h/2,T_{S\F}} E_{h/2,T_F+V_{I_F}},
// each E the same split of (F, I_F) at h/2.  The outer step's level (every
// pair of each set) runs on the level kernels (tau with an edge list; the
// FP64 kick with the fast pairs masked); the rest of the recursion, whose
// lists are the fast pairs, runs in k_ok_tree: one CTA per set takes its
// set's whole recursion tree depth first, with an explicit stack of nodes
// and each node's arrays in the set's arena (stack discipline).
//
// FP64 only, every operation an explicit IEEE one in the oracle's order: a
// pair's tau from (x_a - x_b, v_a - v_b), a < b; a particle's kick sums its
// slow partners in ascending index (pairs (j, i), j < i, in the list's
// order, then (i, j)), then v += h a; drifts x += (h/2) v.  The pivot test
// tau(a,b) < h is decided as in every split: the certified FP32 decision,
// the FP64 tau where it stays open (the FP64 predicate's decisions).
#include "cc_device.cuh"

namespace cc {

// the FP32 decision's constants at the pivot P.h
__host__ __device__ inline MixedTauParams ok_q(const TauParams &P)
{
    MixedTauParams Q;
    Q.eta = (float)P.eta_in;
    Q.etah = (float)(P.eta_outside ? P.eta_in * P.eta / P.h : P.eta_in / P.h);
    Q.eps2 = (float)P.eps2;
    Q.G = (float)P.G;
    Q.hq = 0.f;
    return Q;
}

// tau(a,b) < P.h from the rounded FP64 differences (a < b): certified FP32,
// else the FP64 tau (logged when within near_tol of the pivot; ++nfp64)
__device__ __forceinline__ bool ok_fast(const double *x, const double *y, const double *z, const double *vx,
                                        const double *vy, const double *vz, const double *m, const int32_t *gid,
                                        int a, int b, const TauParams &P, const MixedTauParams &Q, DevCounters *ctr,
                                        int32_t *near_ij, double *near_tau, long long near_cap,
                                        unsigned long long &nfp64)
{
    const double dx0 = __dsub_rn(x[a], x[b]), dx1 = __dsub_rn(y[a], y[b]), dx2 = __dsub_rn(z[a], z[b]);
    const double dv0 = __dsub_rn(vx[a], vx[b]), dv1 = __dsub_rn(vy[a], vy[b]), dv2 = __dsub_rn(vz[a], vz[b]);
    const TauPrep32 t = tau_prep_fp32(fl32(dx0), fl32(dx1), fl32(dx2), fl32(dv0), fl32(dv1), fl32(dv2),
                                      Q.G * (fl32(m[a]) + fl32(m[b])), 0.f, 0.f, Q);
    const int dec = tau_decide_at(t, Q.etah);
    if (dec >= 0) return dec > 0;
    ++nfp64;
    const double tau = tau_fp64(dx0, dx1, dx2, dv0, dv1, dv2, m[a], m[b], P);
    if (fabs(tau - P.h) < P.near_tol * P.h) {
        const unsigned long long z = atomicAdd(&ctr->near_pairs, 1ull);
        if ((long long)z < near_cap) {
            const int ga = gid[a], gb = gid[b];
            near_ij[2 * z] = ga < gb ? ga : gb;
            near_ij[2 * z + 1] = ga < gb ? gb : ga;
            near_tau[z] = tau;
        }
    }
    return tau < P.h;
}

// the certified kernel's edge records (packed indices) -> particle-id pairs
__global__ void k_ok_rec_pairs(const EdgeRec *rec, long long ne, const int32_t *gid, int32_t *edges)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int ga = gid[rec[e].a], gb = gid[rec[e].b];
    edges[2 * e] = ga < gb ? ga : gb;
    edges[2 * e + 1] = ga < gb ? gb : ga;
}

void launch_ok_rec_pairs(const EdgeRec *rec, long long ne, const int32_t *gid, int32_t *edges, cudaStream_t s)
{
    if (ne <= 0) return;
    k_ok_rec_pairs<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(rec, ne, gid, edges);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ level helpers
__global__ void k_ok_inv(Level L, int32_t *inv)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.total) return;
    const int g = L.gid[k];
    if (g >= 0) inv[g] = k;
}

// particle-id pairs -> packed-index pairs (packing keeps id order in a set)
__global__ void k_ok_to_packed(int32_t *edges, long long ne, const int32_t *inv)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    edges[2 * e] = inv[edges[2 * e]];
    edges[2 * e + 1] = inv[edges[2 * e + 1]];
}

// both directions of each pair: (a, b) and (b, a)
__global__ void k_ok_directed(const int32_t *edges, long long ne, int32_t *dir)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int a = edges[2 * e], b = edges[2 * e + 1];
    dir[4 * e] = a;
    dir[4 * e + 1] = b;
    dir[4 * e + 2] = b;
    dir[4 * e + 3] = a;
}

// first entry >= key in the first column of a sorted pair list
__device__ __forceinline__ long long lower_first(const int32_t *p, long long n, int key)
{
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (p[2 * mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// row pointers of the directed adjacency (rows = packed indices 0..total)
// and the drift flags of the outer level: rest[k] = 1 for a particle with
// no fast partner (it drifts at this level)
__global__ void k_ok_rows(Level L, const int32_t *dir, long long nd, int32_t *row_ptr, int32_t *rest,
                          DevCounters *ctr)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > L.total) return;
    row_ptr[k] = (int32_t)lower_first(dir, nd, k);
    if (k == L.total) return;
    const bool in = L.gid[k] >= 0;
    const long long r1 = lower_first(dir, nd, k + 1);
    const int r = in && r1 == row_ptr[k] ? 1 : 0;
    rest[k] = r;
    if (r) atomicAdd(&ctr->small_drifts, 2ull);
}

// segment of each set in the sorted fast list (sets are packed in order)
__global__ void k_ok_segments(Level L, const int32_t *edges, long long ne, long long *seg)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > L.nsets) return;
    seg[s] = s == L.nsets ? ne : lower_first(edges, ne, L.set_start[s]);
}

void launch_ok_level(const Level &L, int32_t *edges, long long ne, int32_t *inv, int32_t *dir, void *sort_scratch,
                     int32_t *row_ptr, int32_t *rest, long long *seg, DevCounters *ctr, cudaStream_t s)
{
    k_ok_inv<<<(L.total + 255) / 256, 256, 0, s>>>(L, inv);
    int launches = 1;
    int bits = 0;
    while (bits < 31 && (1ll << bits) <= (long long)L.total) ++bits;
    if (ne > 0) {
        k_ok_to_packed<<<(int)((ne + 255) / 256), 256, 0, s>>>(edges, ne, inv);
        launch_sort_edges(edges, ne, bits, sort_scratch, s);
        k_ok_directed<<<(int)((ne + 255) / 256), 256, 0, s>>>(edges, ne, dir);
        launch_sort_edges(dir, 2 * ne, bits, sort_scratch, s);
        launches += 2;
    }
    k_ok_rows<<<(L.total + 1 + 255) / 256, 256, 0, s>>>(L, dir, 2 * ne, row_ptr, rest, ctr);
    k_ok_segments<<<(L.nsets + 1 + 255) / 256, 256, 0, s>>>(L, edges, ne, seg);
    CC_COUNT_LAUNCH(launches + 2);
}

// ------------------------------------------------------------ large nodes
// A node whose list is too long for one CTA runs on the whole GPU, driven
// by the host (ok_node in cc_api.cu): the split here, the child list by a
// scan, then the DKD.  The lists of all sets are processed together (sets
// never interact); per-set counts come from stamps on the set index.
struct OkNodeCounters {
    unsigned long long nf, nS, nsys, nsysf;
};

__global__ void k_okh_split(Level L, const int32_t *list, long long np, TauParams P, MixedTauParams Q,
                            unsigned long long stamp, int *fast, int32_t *S, unsigned long long *sst,
                            unsigned long long *fst, unsigned long long *sys_st, unsigned long long *sysf_st,
                            OkNodeCounters *cnt, DevCounters *ctr, int32_t *near_ij, double *near_tau,
                            long long near_cap)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool f = false;
    unsigned long long nfp64 = 0;
    if (k < np) {
        const int a = list[2 * k], b = list[2 * k + 1];
        f = ok_fast(L.x, L.y, L.z, L.vx, L.vy, L.vz, L.m, L.gid, a, b, P, Q, ctr, near_ij, near_tau, near_cap,
                    nfp64);
        fast[k] = f ? 1 : 0;
        for (int q = 0; q < 2; ++q) {
            const int e = q == 0 ? a : b;
            if (atomicExch(&sst[e], stamp) != stamp) S[atomicAdd(&cnt->nS, 1ull)] = e;
            if (f) fst[e] = stamp;
        }
        const int sy = L.sidx[a];
        if (atomicExch(&sys_st[sy], stamp) != stamp) atomicAdd(&cnt->nsys, 1ull);
        if (f && atomicExch(&sysf_st[sy], stamp) != stamp) atomicAdd(&cnt->nsysf, 1ull);
    }
    const unsigned fb = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && fb) atomicAdd(&cnt->nf, (unsigned long long)__popc(fb));
    const unsigned f64 = __ballot_sync(0xffffffffu, nfp64 != 0);
    if ((threadIdx.x & 31) == 0 && f64) atomicAdd(&ctr->tau_fp64, (unsigned long long)__popc(f64));
}

// the fast pairs in list order (pos = exclusive prefix of the flags)
__global__ void k_okh_compact(const int32_t *list, long long np, const int *fast, const int *pos, int32_t *child)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np || !fast[k]) return;
    const int at = pos[k];
    child[2 * at] = list[2 * k];
    child[2 * at + 1] = list[2 * k + 1];
}

// which particles of the node's list belong to a fast pair (read before a
// child node restamps them)
__global__ void k_okh_isf(const int32_t *S, long long nS, const unsigned long long *fst, unsigned long long stamp,
                          unsigned char *isF)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nS) isF[i] = fst[S[i]] == stamp ? 1 : 0;
}

__global__ void k_okh_drift(Level L, const int32_t *S, long long nS, const unsigned char *isF, double dt,
                            DevCounters *ctr, int count)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool d = false;
    if (i < nS && !isF[i]) {
        const int k = S[i];
        L.x[k] = __dadd_rn(L.x[k], __dmul_rn(dt, L.vx[k]));
        L.y[k] = __dadd_rn(L.y[k], __dmul_rn(dt, L.vy[k]));
        L.z[k] = __dadd_rn(L.z[k], __dmul_rn(dt, L.vz[k]));
        d = true;
    }
    const unsigned db = __ballot_sync(0xffffffffu, d);
    if (count && (threadIdx.x & 31) == 0 && db) atomicAdd(&ctr->small_drifts, 2ull * __popc(db));
}

// both directions of every slow pair (slow index = k - pos[k])
__global__ void k_okh_slow(const int32_t *list, long long np, const int *fast, const int *pos, int32_t *dir)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np || fast[k]) return;
    const long long si = k - pos[k];
    const int a = list[2 * k], b = list[2 * k + 1];
    dir[4 * si] = a;
    dir[4 * si + 1] = b;
    dir[4 * si + 2] = b;
    dir[4 * si + 3] = a;
}

// K_h over the slow pairs: the head of each row (sorted by (row, partner))
// sums its partners in ascending index, v += h a
__global__ void k_okh_kick(Level L, const int32_t *dir, long long nd, double G, double eps2, double h)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nd) return;
    const int i = dir[2 * q];
    if (q > 0 && dir[2 * (q - 1)] == i) return;
    double ax = 0.0, ay = 0.0, az = 0.0;
    const double xi = L.x[i], yi = L.y[i], zi = L.z[i];
    for (long long r = q; r < nd && dir[2 * r] == i; ++r) {
        const int j = dir[2 * r + 1];
        const double dx0 = __dsub_rn(L.x[j], xi), dx1 = __dsub_rn(L.y[j], yi), dx2 = __dsub_rn(L.z[j], zi);
        const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)),
                                              __dmul_rn(dx2, dx2)), eps2);
        const double rinv3 = __drcp_rn(__dmul_rn(r2, __dsqrt_rn(r2)));
        const double w = __dmul_rn(__dmul_rn(G, L.m[j]), rinv3);
        ax = __dadd_rn(ax, __dmul_rn(w, dx0));
        ay = __dadd_rn(ay, __dmul_rn(w, dx1));
        az = __dadd_rn(az, __dmul_rn(w, dx2));
    }
    L.vx[i] = __dadd_rn(L.vx[i], __dmul_rn(h, ax));
    L.vy[i] = __dadd_rn(L.vy[i], __dmul_rn(h, ay));
    L.vz[i] = __dadd_rn(L.vz[i], __dmul_rn(h, az));
}

static int okb(long long n) { return (int)((n + 255) / 256); }

void launch_okh_split(const Level &L, const int32_t *list, long long np, const TauParams &P, unsigned long long stamp,
                      int *fast, int32_t *S, unsigned long long *sst, unsigned long long *fst,
                      unsigned long long *sys_st, unsigned long long *sysf_st, void *counters, DevCounters *ctr,
                      int32_t *near_ij, double *near_tau, long long near_cap, cudaStream_t s)
{
    if (np <= 0) return;
    k_okh_split<<<okb(np), 256, 0, s>>>(L, list, np, P, ok_q(P), stamp, fast, S, sst, fst, sys_st, sysf_st,
                                        (OkNodeCounters *)counters, ctr, near_ij, near_tau, near_cap);
    CC_COUNT_LAUNCH(1);
}

void launch_okh_compact(const int32_t *list, long long np, const int *fast, const int *pos, int32_t *child,
                        const int32_t *S, long long nS, const unsigned long long *fst, unsigned long long stamp,
                        unsigned char *isF, cudaStream_t s)
{
    if (np > 0) k_okh_compact<<<okb(np), 256, 0, s>>>(list, np, fast, pos, child);
    if (nS > 0) k_okh_isf<<<okb(nS), 256, 0, s>>>(S, nS, fst, stamp, isF);
    CC_COUNT_LAUNCH(2);
}

void launch_okh_drift(const Level &L, const int32_t *S, long long nS, const unsigned char *isF, double dt,
                      DevCounters *ctr, bool count, cudaStream_t s)
{
    if (nS <= 0) return;
    k_okh_drift<<<okb(nS), 256, 0, s>>>(L, S, nS, isF, dt, ctr, count ? 1 : 0);
    CC_COUNT_LAUNCH(1);
}

void launch_okh_kick(const Level &L, const int32_t *list, long long np, const int *fast, const int *pos,
                     long long ns, int32_t *dir, void *sort_scratch, double G, double eps2, double h, cudaStream_t s)
{
    if (ns <= 0) return;
    int bits = 0;
    while (bits < 31 && (1ll << bits) <= (long long)L.total) ++bits;
    k_okh_slow<<<okb(np), 256, 0, s>>>(list, np, fast, pos, dir);
    launch_sort_edges(dir, 2 * ns, bits, sort_scratch, s);
    k_okh_kick<<<okb(2 * ns), 256, 0, s>>>(L, dir, 2 * ns, G, eps2, h);
    CC_COUNT_LAUNCH(2);
}

// segments of a sorted list by set (the tree takes one set per CTA)
void launch_ok_segments(const Level &L, const int32_t *list, long long np, long long *seg, cudaStream_t s)
{
    k_ok_segments<<<(L.nsets + 1 + 255) / 256, 256, 0, s>>>(L, list, np, seg);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ the tree
constexpr int KO_T = 256;
constexpr int KO_MAXF = 72;  // nested nodes of one tree (DERR_DEPTH beyond)

enum : int { KO_SPLIT = 0, KO_H1 = 1, KO_DKD = 2, KO_H2 = 3, KO_DONE = 4 };

struct OkNode {
    const int32_t *list;  // (a, b) pairs, packed indices, sorted
    unsigned char *fast;  // [np] tau < h
    int32_t *child;       // [2 nf] the fast pairs, in list order
    int32_t *S;           // [nS] the particles of the list
    unsigned char *isF;   // [nS] particle of a fast pair
    int32_t *in_start;    // [nS + 1] incoming slow pairs by particle
    int32_t *in_cur;      // [nS] placement cursor
    int32_t *in_list;     // [ns] their smaller partner, ascending
    int32_t *out_beg, *out_end;  // [nS] the particle's run of pairs (i, *) in the list
    double h;
    size_t mark;  // arena offset at entry
    int np, nf, nS, depth, ph;
};

struct OkShared {
    OkNode fr[KO_MAXF];
    size_t top, cap;
    unsigned long long stamp;
    int nf, nS, bad, wsum[KO_T / 32];
};

struct OkArgs {
    double *x, *y, *z, *vx, *vy, *vz;
    const double *m;
    const int32_t *gid;
    const int32_t *list;     // the outer level's fast list, sorted, all sets
    const long long *seg;    // [nsets + 1] each set's segment
    const long long *arena_off;  // [nsets + 1] bytes
    char *arena;
    unsigned long long *stamp;   // [total] node stamp of a particle's last claim
    int32_t *loc;                // [total] the particle's position in its node's S
    unsigned long long stamp_base;
    double h0;  // pivot of the tree's root (dt/2)
    int depth0, max_depth;
    TauParams P;
    double G, eps2;
    DevCounters *ctr;
    int32_t *near_ij;
    double *near_tau;
    long long near_cap;
};

// arena allocation by thread 0 (16-byte aligned); sets bad on overflow
__device__ __forceinline__ char *ok_alloc(OkShared &sh, char *base, size_t bytes, DevCounters *ctr)
{
    const size_t at = (sh.top + 15) & ~(size_t)15;
    if (at + bytes > sh.cap) {
        if (!sh.bad) raise_err(ctr, DERR_SMALL_OVERFLOW);
        sh.bad = 1;
        return base;
    }
    sh.top = at + bytes;
    return base + at;
}

// exclusive prefix of one value per thread over the CTA; total returned
__device__ __forceinline__ int ok_scan(OkShared &sh, int v, int &total)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh.wsum[w] = inc;
    __syncthreads();
    int off = 0;
    total = 0;
#pragma unroll
    for (int q = 0; q < KO_T / 32; ++q) {
        if (q < w) off += sh.wsum[q];
        total += sh.wsum[q];
    }
    __syncthreads();
    return off + inc - v;
}

__device__ __forceinline__ void ok_term(const OkArgs &A, int i, int j, double &ax, double &ay, double &az)
{
    const double dx0 = __dsub_rn(A.x[j], A.x[i]);
    const double dx1 = __dsub_rn(A.y[j], A.y[i]);
    const double dx2 = __dsub_rn(A.z[j], A.z[i]);
    const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)), __dmul_rn(dx2, dx2)),
                                A.eps2);
    const double rinv3 = __drcp_rn(__dmul_rn(r2, __dsqrt_rn(r2)));
    const double w = __dmul_rn(__dmul_rn(A.G, A.m[j]), rinv3);
    ax = __dadd_rn(ax, __dmul_rn(w, dx0));
    ay = __dadd_rn(ay, __dmul_rn(w, dx1));
    az = __dadd_rn(az, __dmul_rn(w, dx2));
}

__device__ __forceinline__ void ok_drift(const OkArgs &A, int i, double dt)
{
    A.x[i] = __dadd_rn(A.x[i], __dmul_rn(dt, A.vx[i]));
    A.y[i] = __dadd_rn(A.y[i], __dmul_rn(dt, A.vy[i]));
    A.z[i] = __dadd_rn(A.z[i], __dmul_rn(dt, A.vz[i]));
}

// the split of a node: fast flags, the child list (fast pairs in order), the
// particle list S with its F flags, outgoing runs, and the incoming slow
// pairs of each particle in ascending partner (a stable counting sort)
__device__ void ok_split(OkShared &sh, OkNode &N, const OkArgs &A, char *base, unsigned long long *cnt)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const int np = N.np;
    TauParams P = A.P;
    P.h = N.h;
    if (tid == 0) {
        sh.nf = 0;
        sh.nS = 0;
        sh.stamp += 1;
        N.fast = (unsigned char *)ok_alloc(sh, base, (size_t)np, A.ctr);
        N.S = (int32_t *)ok_alloc(sh, base, (size_t)8 * np, A.ctr);
    }
    __syncthreads();
    if (sh.bad) return;
    const unsigned long long stamp = sh.stamp;
    int nf_local = 0;
    const MixedTauParams Q = ok_q(P);
    unsigned long long nfp64 = 0;
    for (int k = tid; k < np; k += KO_T) {
        const int a = N.list[2 * k], b = N.list[2 * k + 1];
        const bool f = ok_fast(A.x, A.y, A.z, A.vx, A.vy, A.vz, A.m, A.gid, a, b, P, Q, A.ctr, A.near_ij,
                               A.near_tau, A.near_cap, nfp64);
        N.fast[k] = f ? 1 : 0;
        nf_local += f ? 1 : 0;
        // the particles of the list: the first claim of this node's stamp
        // appends the particle
        for (int q = 0; q < 2; ++q) {
            const int e = q == 0 ? a : b;
            if (atomicExch(&A.stamp[e], stamp) != stamp) {
                const int li = atomicAdd(&sh.nS, 1);
                N.S[li] = e;
                A.loc[e] = li;
            }
        }
    }
    atomicAdd(&sh.nf, nf_local);
    if (nfp64) atomicAdd(&A.ctr->tau_fp64, nfp64);
    __syncthreads();
    const int nf = sh.nf, nS = sh.nS;
    if (tid == 0) {
        N.nf = nf;
        N.nS = nS;
        N.child = (int32_t *)ok_alloc(sh, base, (size_t)8 * nf, A.ctr);
        N.isF = (unsigned char *)ok_alloc(sh, base, (size_t)nS, A.ctr);
        N.in_start = (int32_t *)ok_alloc(sh, base, (size_t)4 * (nS + 1), A.ctr);
        N.in_cur = (int32_t *)ok_alloc(sh, base, (size_t)4 * nS, A.ctr);
        N.in_list = (int32_t *)ok_alloc(sh, base, (size_t)4 * (np - nf), A.ctr);
        N.out_beg = (int32_t *)ok_alloc(sh, base, (size_t)4 * nS, A.ctr);
        N.out_end = (int32_t *)ok_alloc(sh, base, (size_t)4 * nS, A.ctr);
        cnt[0] += 1;                       // split
        cnt[1] += (unsigned long long)np;  // tau pairs
        cnt[2] += nf > 0 ? 1 : 0;          // components (non-empty fast lists)
        cnt[3] += (unsigned long long)np;  // tau evaluated
    }
    __syncthreads();
    if (sh.bad) return;
    for (int li = tid; li < nS; li += KO_T) {
        N.isF[li] = 0;
        N.in_start[li] = 0;
        N.out_beg[li] = 0;
        N.out_end[li] = 0;
    }
    __syncthreads();
    // fast flags of particles, outgoing runs, incoming slow counts
    for (int k = tid; k < np; k += KO_T) {
        const int a = N.list[2 * k], b = N.list[2 * k + 1];
        const int la = A.loc[a], lb = A.loc[b];
        if (N.fast[k]) {
            N.isF[la] = 1;
            N.isF[lb] = 1;
        } else {
            atomicAdd(&N.in_start[lb], 1);
        }
        if (k == 0 || N.list[2 * (k - 1)] != a) N.out_beg[la] = k;
        if (k == np - 1 || N.list[2 * (k + 1)] != a) N.out_end[la] = k + 1;
    }
    __syncthreads();
    // child list: the fast pairs in list order (chunks of KO_T, one per thread)
    int base_f = 0;
    for (int c0 = 0; c0 < np; c0 += KO_T) {
        const int k = c0 + tid;
        const int f = k < np ? N.fast[k] : 0;
        int tot;
        const int at = ok_scan(sh, f, tot) + base_f;
        if (f) {
            N.child[2 * at] = N.list[2 * k];
            N.child[2 * at + 1] = N.list[2 * k + 1];
        }
        base_f += tot;
    }
    // incoming starts: exclusive prefix of the counts over S
    int base_s = 0;
    for (int c0 = 0; c0 < nS; c0 += KO_T) {
        const int li = c0 + tid;
        const int v = li < nS ? N.in_start[li] : 0;
        int tot;
        const int at = ok_scan(sh, v, tot) + base_s;
        if (li < nS) {
            N.in_start[li] = at;
            N.in_cur[li] = at;
        }
        base_s += tot;
    }
    if (tid == 0) N.in_start[nS] = base_s;
    __syncthreads();
    // the incoming lists: one warp walks the list in order, ranking the slow
    // pairs of one particle by lane (stable: ascending smaller partner)
    if (tid < 32) {
        const unsigned lt = (1u << lane) - 1u;
        for (int c0 = 0; c0 < np; c0 += 32) {
            const int k = c0 + lane;
            const bool slow = k < np && !N.fast[k];
            const int key = slow ? A.loc[N.list[2 * k + 1]] : -1 - lane;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (slow) N.in_list[N.in_cur[key] + __popc(peers & lt)] = N.list[2 * k];
            __syncwarp();
            if (slow && lane == 31 - __clz(peers)) N.in_cur[key] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
}

// D_{h/2} K_{h, slow} D_{h/2} of a node
__device__ void ok_dkd(OkShared &sh, const OkNode &N, const OkArgs &A, unsigned long long *cnt)
{
    const int tid = threadIdx.x;
    const double hd = 0.5 * N.h;
    int drifts = 0;
    for (int li = tid; li < N.nS; li += KO_T)
        if (!N.isF[li]) {
            ok_drift(A, N.S[li], hd);
            ++drifts;
        }
    __syncthreads();
    for (int li = tid; li < N.nS; li += KO_T) {
        const int i = N.S[li];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int q = N.in_start[li]; q < N.in_start[li + 1]; ++q) ok_term(A, i, N.in_list[q], ax, ay, az);
        for (int k = N.out_beg[li]; k < N.out_end[li]; ++k)
            if (!N.fast[k]) ok_term(A, i, N.list[2 * k + 1], ax, ay, az);
        A.vx[i] = __dadd_rn(A.vx[i], __dmul_rn(N.h, ax));
        A.vy[i] = __dadd_rn(A.vy[i], __dmul_rn(N.h, ay));
        A.vz[i] = __dadd_rn(A.vz[i], __dmul_rn(N.h, az));
    }
    __syncthreads();
    for (int li = tid; li < N.nS; li += KO_T)
        if (!N.isF[li]) ok_drift(A, N.S[li], hd);
    atomicAdd((unsigned long long *)&cnt[5], (unsigned long long)(2 * drifts));
    if (tid == 0) cnt[4] += (unsigned long long)(N.np - N.nf);  // kick pairs
    __syncthreads();
}

__global__ void __launch_bounds__(KO_T) k_ok_tree(OkArgs A)
{
    __shared__ OkShared sh;
    __shared__ unsigned long long cnt[6];  // splits, tau, comps, evals, kicks, drifts
    const int s = blockIdx.x, tid = threadIdx.x;
    const long long l0 = A.seg[s], l1 = A.seg[s + 1];
    if (l1 <= l0) return;
    char *base = A.arena + A.arena_off[s];
    if (tid < 6) cnt[tid] = 0;
    if (tid == 0) {
        sh.top = 0;
        sh.cap = (size_t)(A.arena_off[s + 1] - A.arena_off[s]);
        sh.stamp = A.stamp_base + ((unsigned long long)s << 24);
        sh.bad = 0;
        OkNode &R = sh.fr[0];
        R.list = A.list + 2 * l0;
        R.np = (int)(l1 - l0);
        R.h = A.h0;
        R.depth = A.depth0;
        R.ph = KO_SPLIT;
        R.mark = 0;
    }
    int maxd = A.depth0;
    int top = 0;
    __syncthreads();
    if (A.depth0 > A.max_depth) {
        if (tid == 0) raise_err(A.ctr, DERR_DEPTH);
        return;
    }
    for (;;) {
        OkNode &N = sh.fr[top];
        const int ph = N.ph;
        __syncthreads();
        if (ph == KO_SPLIT) {
            ok_split(sh, N, A, base, cnt);
            if (tid == 0) N.ph = KO_H1;
        } else if (ph == KO_H1 || ph == KO_H2) {
            if (tid == 0) {
                N.ph = ph == KO_H1 ? KO_DKD : KO_DONE;
                if (N.nf > 0) {
                    if (N.depth + 1 > A.max_depth || top + 1 >= KO_MAXF) {
                        raise_err(A.ctr, DERR_DEPTH);
                        sh.bad = 1;
                    } else {
                        OkNode &C = sh.fr[top + 1];
                        C.list = N.child;
                        C.np = N.nf;
                        C.h = 0.5 * N.h;
                        C.depth = N.depth + 1;
                        C.ph = KO_SPLIT;
                        C.mark = sh.top;
                    }
                }
            }
            __syncthreads();
            if (!sh.bad && N.nf > 0) {
                ++top;
                if (top + A.depth0 > maxd) maxd = top + A.depth0;
            }
        } else if (ph == KO_DKD) {
            ok_dkd(sh, N, A, cnt);
            if (tid == 0) N.ph = KO_H2;
        } else {
            if (tid == 0) sh.top = N.mark;
            --top;
        }
        __syncthreads();
        if (sh.bad || top < 0) break;
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&A.ctr->small_splits, cnt[0]);
        atomicAdd(&A.ctr->small_tau_pairs, cnt[1]);
        atomicAdd(&A.ctr->small_components, cnt[2]);
        atomicAdd(&A.ctr->tau_evals, cnt[3]);
        atomicAdd(&A.ctr->small_kick_pairs, cnt[4]);
        atomicAdd(&A.ctr->small_drifts, cnt[5]);
        atomicMax(&A.ctr->max_depth_seen, maxd);
    }
}

void launch_ok_tree(const Level &L, const int32_t *list, const long long *seg, const long long *arena_off,
                    char *arena, unsigned long long *stamp, int32_t *loc, unsigned long long stamp_base, double h0,
                    int depth0, int max_depth, const TauParams &P, double G, double eps2, DevCounters *ctr,
                    int32_t *near_ij, double *near_tau, long long near_cap, cudaStream_t s)
{
    if (L.nsets <= 0) return;
    OkArgs A{L.x,      L.y,   L.z,    L.vx,       L.vy,  L.vz,      L.m,        L.gid,   list, seg, arena_off,
             arena,    stamp, loc,    stamp_base, h0,    depth0,    max_depth,  P,       G,    eps2, ctr,
             near_ij,  near_tau, near_cap};
    k_ok_tree<<<L.nsets, KO_T, 0, s>>>(A);
    CC_COUNT_LAUNCH(1);
}

}  // namespace cc
