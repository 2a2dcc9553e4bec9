// cc_pair.cu -- pairwise kernels of the CC split (arXiv:1407.7105):
//   * tau(i,j) over all pairs of each set fused with the edge test
//     tau < h (Sec. 2.2) and union-find hooking of every edge;
//   * the kick K_{h,V_ij} between members of different components
//     (Eqs. kickij, kickji; Sec. 2.2 K_{h, V_R + V_CC + V_CR});
//   * the energy diagnostic H (Eq. Hamiltonian).
// j-tiles are staged in shared memory by TMA bulk copies (cp.async.bulk)
// completing on an mbarrier; every wait is bounded.
#include "cc_device.cuh"

namespace cc {

// ------------------------------------------------------------ helpers
__device__ __forceinline__ int find_set(const int32_t *off, int nsets, int b)
{
    int lo = 0, hi = nsets;  // off[lo] <= b < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= b) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_init_parent(int32_t *parent, int32_t *cnt, int total, unsigned long long *edge_count)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < total) {
        parent[k] = k;
        cnt[k] = 0;
    }
    if (k == 0 && edge_count) *edge_count = 0ull;
}

void launch_init_parent(const Level &L, unsigned long long *edge_count, cudaStream_t s)
{
    if (L.total <= 0) return;
    k_init_parent<<<(L.total + 255) / 256, 256, 0, s>>>(L.parent, L.cnt, L.total, edge_count);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ tau + hook
// One CTA per (set, i-tile, j-tile) with i-tile <= j-tile: TAU_T threads,
// thread r owns particle i = i-tile*TAU_T + r and tests it against the
// j-tile staged in shared memory (pairs i < j only).
constexpr int TAU_T = 128;  // tile of the edge-list variant

template <int T>
struct __align__(16) TauSmem {
    double col[7][T + 4];  // x y z vx vy vz m of the j-tile
    uint64_t bar;
};

__device__ __forceinline__ void log_pair(const TauParams &P, double tau, int gi, int gj, DevCounters *ctr,
                                         int32_t *near_ij, double *near_tau, long long near_cap)
{
    if (fabs(tau - P.h) < P.near_tol * P.h) {
        unsigned long long k = atomicAdd(&ctr->near_pairs, 1ull);
        if ((long long)k < near_cap) {
            near_ij[2 * k] = gi < gj ? gi : gj;
            near_ij[2 * k + 1] = gi < gj ? gj : gi;
            near_tau[k] = tau;
        }
    }
}

template <int T>
__global__ void __launch_bounds__(T) k_tau_hook(Level L, TauParams P, DevCounters *ctr, int32_t *near_ij,
                                                     double *near_tau, long long near_cap, EdgeList E)
{
    __shared__ TauSmem<T> sm;
    const int tid = threadIdx.x;
    const int s = find_set(L.tile_off, L.nsets, blockIdx.x);
    int t = blockIdx.x - L.tile_off[s];
    const int n = L.set_n[s], start = L.set_start[s];
    const int nt = (n + T - 1) / T;
    int ti = 0;
    while (t >= nt - ti) {
        t -= nt - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int j0 = start + tj * T;
    const int jn = min(T, n - tj * T);

    if (tid == 0) {
        mbar_init(&sm.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // fault_test = 1: the copy is announced but never issued, so the wait
    // below runs out (a test of the bounded wait; no copy is in flight)
    const bool no_copy = P.fault_test == 1;
    const long long wait_cycles = no_copy ? FAULT_TEST_WAIT_CYCLES : TMA_WAIT_CYCLES;
    if (tid == 0) {
        const unsigned bytes = (unsigned)((jn + 3) & ~3) * 8u;
        mbar_expect_tx(&sm.bar, 7u * bytes);
        const double *src[7] = {L.x, L.y, L.z, L.vx, L.vy, L.vz, L.m};
        if (!no_copy) {
#pragma unroll
            for (int c = 0; c < 7; ++c) tma_load_1d(sm.col[c], src[c] + j0, bytes, &sm.bar);
        }
    }
    const int il = ti * T + tid;
    const bool iv = il < n;
    const int i = start + il;
    double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 0;
    int gi = -1;
    if (iv) {
        xi = L.x[i]; yi = L.y[i]; zi = L.z[i];
        vxi = L.vx[i]; vyi = L.vy[i]; vzi = L.vz[i];
        mi = L.m[i];
        gi = L.gid[i];
    }
    if (!mbar_wait(&sm.bar, 0, wait_cycles)) {
        raise_err(ctr, DERR_TMA_TIMEOUT);
        // let a copy still in flight land before the CTA exits
        mbar_wait(&sm.bar, 0, wait_cycles);
        return;
    }
    // fault_test = 2: every hook gives up at once (a test of the retry cap)
    const int uf_retry = P.fault_test == 2 ? 0 : UF_RETRY_MAX;
    unsigned long long my_edges = 0;
    if (iv) {
        const int kbeg = (ti == tj) ? tid + 1 : 0;
        auto tau_of = [&](int k) {
            return tau_fp64(__dsub_rn(xi, sm.col[0][k]), __dsub_rn(yi, sm.col[1][k]), __dsub_rn(zi, sm.col[2][k]),
                            __dsub_rn(vxi, sm.col[3][k]), __dsub_rn(vyi, sm.col[4][k]), __dsub_rn(vzi, sm.col[5][k]),
                            mi, sm.col[6][k], P);
        };
        // two pairs' tau in flight (its square roots and divisions are long
        // dependent chains); the second of the last pair may be a repeat
        double tnext = 0.0;
        for (int k = kbeg; k < jn; ++k) {
            double tau;
            if (((k - kbeg) & 1) == 0) {
                tau = tau_of(k);
                tnext = tau_of(k + 1 < jn ? k + 1 : k);
            } else {
                tau = tnext;
            }
            const int j = j0 + k;
            log_pair(P, tau, gi, L.gid[j], ctr, near_ij, near_tau, near_cap);
            if (tau < P.h) {
                ++my_edges;
                if (!uf_union(L.parent, i, j, uf_retry)) raise_err(ctr, DERR_UF_RETRY);
                // a record serves the first half at h/2: kept when the pair
                // is an edge there or near h/2
                if (E.rec && (tau < 0.5 * P.h || fabs(tau - 0.5 * P.h) < P.near_tol * 0.5 * P.h))
                    record_edge(E, i, j, -1, tau);
            }
        }
    }
    // warp-aggregated edge count: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_edges += __shfl_down_sync(0xffffffffu, my_edges, o);
    if ((tid & 31) == 0 && my_edges) atomicAdd(&ctr->edges, my_edges);
}

// ------------------------------------------------------------ first-half split
// The split of a component's first half (pivot h) sees the state its
// parent split saw at 2h, so tau(i,j) is unchanged: the edges are the
// parent's records that are edges at h, and every pair near h is a parent
// record too (tau < 2h).  Two passes:
//   k_edges_filter, one thread per parent record: records of components the
//   gather did not move to this level (small, Kepler) are skipped (inv[a] is
//   only meaningful where this level's src points back to a); the record's
//   edge depth comes from its e, else its FP64 tau, else (an FP32-certified
//   edge of a fresh mixed split) from certified FP32 decisions at 2h, h,
//   h/2, ... on the parent's float-float copy, which the first half leaves
//   untouched, with the FP64 tau from the parent level's state at the first
//   undecided threshold; near-threshold pairs are logged, and the edges at h
//   become this split's records (depth carried on, so deeper first halves
//   never need a float-float copy);
//   k_edges_hook: union-find hooking of this split's records, a compact list
//   (a fraction of the parent's), so the pointer chasing of the hooks runs
//   in about one wave (the list holds at least as many records as the
//   parent's, so none is dropped).  The filter pass also points each edge's larger
//   endpoint at its smallest neighbour (atomicMin): every union-find
//   invariant holds for that forest, and in a dense core, where many edges
//   share an endpoint, it spares the hooks their compare-and-swap retries.
__global__ void k_edges_filter(EdgeList PE, long long pcount, Level PL, FFView PF, MixedTauParams Q, int mixed,
                               const int32_t *inv, Level C, EdgeList CE, TauParams P, DevCounters *ctr,
                               int32_t *near_ij, double *near_tau, long long near_cap)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long my_edges = 0, my_evals = 0;
    if (t < pcount) {
        const EdgeRec r = PE.rec[t];
        const int a = inv[r.a], b = inv[r.b];
        const bool in = a >= 0 && a < C.total && b >= 0 && b < C.total && C.src[a] == r.a && C.src[b] == r.b &&
                        C.gid[a] >= 0 && C.gid[b] >= 0;
        if (in) {
            const double hp = 2.0 * P.h;  // the parent's pivot
            double tau = r.tau;
            int e = r.e;
            if (e < 0 && tau == tau) e = first_level_at_or_below(tau, hp, EDGE_E_INF);
            if (e < 0) {
                int m = 1, dec = 1;
                if (mixed) {
                    // the tau kernel's decision at hp, restated at hp 2^-m
                    const float4 ip0 = PF.pq[2 * r.a], ip1 = PF.pq[2 * r.a + 1];
                    const float4 iv0 = PF.vq[2 * r.a], iv1 = PF.vq[2 * r.a + 1];
                    const float4 jp0 = PF.pq[2 * r.b], jp1 = PF.pq[2 * r.b + 1];
                    const float4 jv0 = PF.vq[2 * r.b], jv1 = PF.vq[2 * r.b + 1];
                    const float cX = 11.f * U32 * U32 * PF.maxes[0];
                    const float cV = 11.f * U32 * U32 * PF.maxes[1];
                    const TauPrep32 tp = tau_prep_fp32(
                        (jp0.x - ip0.x) + (jp1.x - ip1.x), (jp0.y - ip0.y) + (jp1.y - ip1.y),
                        (jp0.z - ip0.z) + (jp1.z - ip1.z), (jv0.x - iv0.x) + (jv1.x - iv1.x),
                        (jv0.y - iv0.y) + (jv1.y - iv1.y), (jv0.z - iv0.z) + (jv1.z - iv1.z), ip0.w + jp0.w, cX, cV,
                        Q);
                    while (m < 100) {
                        dec = tau_decide_at(tp, Q.etah * pow2f(m));
                        if (dec != 1) break;
                        ++m;
                    }
                }
                if (mixed && dec == 0) {
                    e = m;
                } else {
                    const int i = r.a, j = r.b;
                    tau = tau_fp64(__dsub_rn(PL.x[i], PL.x[j]), __dsub_rn(PL.y[i], PL.y[j]),
                                   __dsub_rn(PL.z[i], PL.z[j]), __dsub_rn(PL.vx[i], PL.vx[j]),
                                   __dsub_rn(PL.vy[i], PL.vy[j]), __dsub_rn(PL.vz[i], PL.vz[j]), PL.m[i], PL.m[j], P);
                    ++my_evals;
                    const int e64 = first_level_at_or_below(tau, hp, EDGE_E_INF);
                    e = e64 > m ? e64 : m;
                }
            }
            if (tau == tau) log_pair(P, tau, C.gid[a], C.gid[b], ctr, near_ij, near_tau, near_cap);
            if (e >= 2) {
                ++my_edges;
                // link the larger endpoint to its smallest neighbour so far:
                // a forest with parent < self whose links are edges, built
                // without retries; the hook pass then finds most record
                // endpoints already in one tree
                atomicMin(&C.parent[max(a, b)], min(a, b));
                // the host sizes this list to the parent's record count, so
                // a record is never dropped (the hook pass must see every edge)
                if (!record_edge(CE, min(a, b), max(a, b), e >= EDGE_E_INF ? EDGE_E_INF : e - 1, tau))
                    raise_err(ctr, DERR_UF_RETRY);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_edges += __shfl_down_sync(0xffffffffu, my_edges, o);
        my_evals += __shfl_down_sync(0xffffffffu, my_evals, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (my_edges) atomicAdd(&ctr->edges, my_edges);
        if (my_evals) {
            atomicAdd(&ctr->tau_fp64, my_evals);
            atomicAdd(&ctr->tau_evals, my_evals);
        }
    }
}

__global__ void k_edges_hook(EdgeList E, int32_t *parent, DevCounters *ctr)
{
    const long long n = (long long)min(*E.count, (unsigned long long)E.cap);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const EdgeRec r = E.rec[t];
        // a shared parent, or the link itself, already puts a and b in one
        // tree (a parent is an ancestor, and trees only merge)
        const int pa = __ldca(parent + r.a), pb = __ldca(parent + r.b);
        if (pa == pb || pb == r.a || pa == r.b) continue;
        if (!uf_union_ca(parent, r.a, r.b)) raise_err(ctr, DERR_UF_RETRY);
    }
}

void launch_edges_reuse(const EdgeList &parent, long long pcount, const Level &PL, const FFView &PF, bool mixed,
                        const int32_t *inv, const Level &C, const EdgeList &child, const TauParams &P,
                        DevCounters *ctr, int32_t *near_ij, double *near_tau, long long near_cap, cudaStream_t s,
                        bool hook)
{
    if (pcount <= 0) return;
    const double hp = 2.0 * P.h;
    MixedTauParams Q;
    Q.eta = (float)P.eta_in;
    Q.etah = (float)(P.eta_outside ? P.eta_in * P.eta / hp : P.eta_in / hp);
    Q.eps2 = (float)P.eps2;
    Q.G = (float)P.G;
    Q.hq = 0.f;  // (the pre-test is not used here)
    const unsigned blocks = (unsigned)((pcount + 255) / 256);
    k_edges_filter<<<blocks, 256, 0, s>>>(parent, pcount, PL, PF, Q, mixed ? 1 : 0, inv, C, child, P, ctr, near_ij,
                                          near_tau, near_cap);
    CC_COUNT_LAUNCH(1);
    if (hook) {
        // the hooks: at most pcount records, usually far fewer (grid-stride)
        k_edges_hook<<<blocks < 1216u ? blocks : 1216u, 256, 0, s>>>(child, C.parent, ctr);
        CC_COUNT_LAUNCH(1);
    }
}

// Edge-list variant for the time-step-graph entry point: same predicate,
// each edge written as (gid_i, gid_j), gid_i < gid_j, at an atomically
// reserved slot (order fixed afterwards by a sort).
__global__ void __launch_bounds__(TAU_T) k_tau_edges(Level L, TauParams P, DevCounters *ctr, int32_t *edges,
                                                      long long edge_cap, int32_t *near_ij, double *near_tau,
                                                      long long near_cap)
{
    __shared__ TauSmem<TAU_T> sm;
    const int tid = threadIdx.x;
    const int s = find_set(L.tile_off, L.nsets, blockIdx.x);
    int t = blockIdx.x - L.tile_off[s];
    const int n = L.set_n[s], start = L.set_start[s];
    const int nt = (n + TAU_T - 1) / TAU_T;
    int ti = 0;
    while (t >= nt - ti) {
        t -= nt - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int j0 = start + tj * TAU_T;
    const int jn = min(TAU_T, n - tj * TAU_T);
    if (tid == 0) {
        mbar_init(&sm.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned bytes = (unsigned)((jn + 3) & ~3) * 8u;
        mbar_expect_tx(&sm.bar, 7u * bytes);
        const double *src[7] = {L.x, L.y, L.z, L.vx, L.vy, L.vz, L.m};
#pragma unroll
        for (int c = 0; c < 7; ++c) tma_load_1d(sm.col[c], src[c] + j0, bytes, &sm.bar);
    }
    const int il = ti * TAU_T + tid;
    const bool iv = il < n;
    const int i = start + il;
    double xi = 0, yi = 0, zi = 0, vxi = 0, vyi = 0, vzi = 0, mi = 0;
    int gi = -1;
    if (iv) {
        xi = L.x[i]; yi = L.y[i]; zi = L.z[i];
        vxi = L.vx[i]; vyi = L.vy[i]; vzi = L.vz[i];
        mi = L.m[i];
        gi = L.gid[i];
    }
    if (!mbar_wait(&sm.bar, 0, TMA_WAIT_CYCLES)) {
        raise_err(ctr, DERR_TMA_TIMEOUT);
        mbar_wait(&sm.bar, 0, TMA_WAIT_CYCLES);
        return;
    }
    if (!iv) return;
    const int kbeg = (ti == tj) ? tid + 1 : 0;
    for (int k = kbeg; k < jn; ++k) {
        const double tau = tau_fp64(__dsub_rn(xi, sm.col[0][k]), __dsub_rn(yi, sm.col[1][k]),
                                    __dsub_rn(zi, sm.col[2][k]), __dsub_rn(vxi, sm.col[3][k]),
                                    __dsub_rn(vyi, sm.col[4][k]), __dsub_rn(vzi, sm.col[5][k]), mi,
                                    sm.col[6][k], P);
        const int j = j0 + k;
        const int gj = L.gid[j];
        log_pair(P, tau, gi, gj, ctr, near_ij, near_tau, near_cap);
        if (tau < P.h) {
            if (!uf_union(L.parent, i, j)) raise_err(ctr, DERR_UF_RETRY);
            unsigned long long e = atomicAdd(&ctr->edges, 1ull);
            if ((long long)e < edge_cap) {
                edges[2 * e] = gi < gj ? gi : gj;
                edges[2 * e + 1] = gi < gj ? gj : gi;
            }
        }
    }
}

void launch_tau_hook(const Level &L, int ntiles, const TauParams &P, int variant, DevCounters *ctr,
                     int32_t *edges, long long edge_cap, int32_t *near_ij, double *near_tau, long long near_cap,
                     cudaStream_t s, const EdgeList *rec)
{
    if (ntiles <= 0) return;
    const EdgeList E = rec ? *rec : EdgeList{nullptr, nullptr, 0};
    if (edges) {
        k_tau_edges<<<ntiles, TAU_T, 0, s>>>(L, P, ctr, edges, edge_cap, near_ij, near_tau, near_cap);
        CC_COUNT_LAUNCH(1);
        return;
    }
    if (variant == 0)
        k_tau_hook<64><<<ntiles, 64, 0, s>>>(L, P, ctr, near_ij, near_tau, near_cap, E);
    else
        k_tau_hook<128><<<ntiles, 128, 0, s>>>(L, P, ctr, near_ij, near_tau, near_cap, E);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ kick (FP64)
// One CTA per (set, i-tile); thread r accumulates a_i over every j-tile of
// its set in ascending order (pairs with equal labels skipped), so the sum
// runs over j in ascending packed index = ascending particle id, the
// order of the plain definition; then v_i += h a_i.  Two-stage TMA ring.

template <int T>
struct __align__(16) KickSmem {
    double col[2][4][T];  // x y z m per stage
    int32_t lab[2][T];
    uint64_t bar[2];
};

template <int T>
__device__ __forceinline__ void kick_issue(KickSmem<T> &sm, int st, const Level &L, const int32_t *label, int j0,
                                           int jn)
{
    const unsigned cnt = (unsigned)((jn + 3) & ~3);
    fence_proxy_async_smem();
    mbar_expect_tx(&sm.bar[st], cnt * (4u * 8u + 4u));
    tma_load_1d(sm.col[st][0], L.x + j0, cnt * 8u, &sm.bar[st]);
    tma_load_1d(sm.col[st][1], L.y + j0, cnt * 8u, &sm.bar[st]);
    tma_load_1d(sm.col[st][2], L.z + j0, cnt * 8u, &sm.bar[st]);
    tma_load_1d(sm.col[st][3], L.m + j0, cnt * 8u, &sm.bar[st]);
    tma_load_1d(sm.lab[st], label + j0, cnt * 4u, &sm.bar[st]);
}

// One CTA (256 threads) per 32-body i-tile of a set.  For each 32-body
// j-tile (TMA, double-buffered) all threads first compute the tile's 1024
// pair forces (the square roots and divisions, the bulk of the FP64 work,
// spread over eight warps) into shared memory, then 96 threads each add one
// (row, component) over the tile in ascending j: a_i is still the sum over
// j in ascending id, term by term as in the plain definition (a skipped
// pair is an exact +0), so the result is the oracle's bit for bit, while the
// FP64 pipe sees eight warps per block instead of one thread per body.
constexpr int KB_T = 32;        // i-tile and j-tile
constexpr int KB_THREADS = 256;
constexpr int KB_Q = KB_T * KB_T / KB_THREADS;  // pairs of a tile per thread
static_assert(K64_VAR_T[0] == KB_T, "the FP64 kick runs on the 32-body i-tile prefix");

struct __align__(16) KickBSmem {
    KickSmem<KB_T> j;                // j tiles: x y z m, labels
    double f[3][KB_T][KB_T + 1];     // pair forces of the current tile (padded rows)
    double xi[3][KB_T];              // the i-tile
    int32_t li[KB_T];
    int32_t ci[KB_T], cj[KB_T];      // centre-of-mass approximation: local eligible indices
    int32_t okc[KB_T], oke[KB_T];    // OK split: each row's cursor / end in its sorted fast partners
    uint32_t okm[KB_T];              // OK split: fast partners of each row in the current j-tile
};

// MODE 1 (centre-of-mass approximation): pairs of far components (ComView)
// are left out; their kick is the centre-of-mass one that launch_com_apply
// adds afterwards.  MODE 2 (OK split): the fast pairs (OkView: each row's
// partners, sorted) are left out, every other pair of the set kicks.
// MODE 3: as MODE 0 with each pair's force G m_j r_ij^-3 (x_j - x_i) read
// from the matrices k_pair_forces filled (PairFactors) instead of computed;
// MODE 4: as MODE 2 with the forces read.
template <int MODE>
__global__ void __launch_bounds__(KB_THREADS) k_kick64(Level L, const int32_t *label, double G, double eps2, double h,
                                                       DevCounters *ctr, ComView cv, OkView okv, PairFactors pf)
{
    constexpr bool COM = MODE == 1, OKM = MODE == 2 || MODE == 4, PRE = MODE >= 3;
    __shared__ KickBSmem sm;
    const int tid = threadIdx.x;
    const int s = find_set(L.itile_off, L.nsets, blockIdx.x);
    const int ti = blockIdx.x - L.itile_off[s];
    const int n = L.set_n[s], start = L.set_start[s];
    const int nt = (n + KB_T - 1) / KB_T;
    const int il0 = ti * KB_T, ni = min(KB_T, n - il0);
    if (tid == 0) {
        mbar_init(&sm.j.bar[0], 1);
        mbar_init(&sm.j.bar[1], 1);
        fence_mbar_init();
    }
    if (tid < KB_T) {
        const bool v = tid < ni;
        const int i = start + il0 + tid;
        sm.xi[0][tid] = v ? L.x[i] : 0.0;
        sm.xi[1][tid] = v ? L.y[i] : 0.0;
        sm.xi[2][tid] = v ? L.z[i] : 0.0;
        sm.li[tid] = v ? label[i] : 0;
        if (COM) sm.ci[tid] = v ? cv.cl[i] : -1;
        if (OKM) {
            sm.okc[tid] = v ? okv.row_ptr[i] : 0;
            sm.oke[tid] = v ? okv.row_ptr[i + 1] : 0;
        }
    }
    long long fo = 0;
    int Ks = 0;
    if (COM) {
        fo = cv.foff[s];
        Ks = cv.K[s];
    }
    __syncthreads();
    if (tid == 0) kick_issue(sm.j, 0, L, label, start, min(KB_T, n));
    const int r = tid & 31, c = tid >> 5;  // summing threads: row r, component c (tid < 96)
    double acc = 0.0;
    bool ok = true;
    // MODE 3/4: this thread's pairs (row (tid >> 5) + 8 q, column tid & 31)
    // of a j-tile, all three components, loaded a tile ahead
    double fr[3][KB_Q];
    const long long nn = (long long)n * n;
    const double *F = PRE ? pf.S + pf.moff[s] : nullptr;
    auto load_f = [&](int tj) {
        const int jl0 = tj * KB_T, jn = min(KB_T, n - jl0);
#pragma unroll
        for (int q = 0; q < KB_Q; ++q) {
            const int ii = (tid >> 5) + q * (KB_THREADS / KB_T), jj = tid & 31;
            const bool v = ii < ni && jj < jn;
            const long long e = (long long)(il0 + ii) * n + (jl0 + jj);
            fr[0][q] = v ? F[e] : 0.0;
            fr[1][q] = v ? F[nn + e] : 0.0;
            fr[2][q] = v ? F[2 * nn + e] : 0.0;
        }
    };
    if (PRE) load_f(0);
    for (int tj = 0; tj < nt; ++tj) {
        const int st = tj & 1;
        if (tid == 0 && tj + 1 < nt)
            kick_issue(sm.j, st ^ 1, L, label, start + (tj + 1) * KB_T, min(KB_T, n - (tj + 1) * KB_T));
        const bool got = mbar_wait(&sm.j.bar[st], (tj >> 1) & 1, TMA_WAIT_CYCLES);
        if (__syncthreads_or(!got)) {  // uniform exit: no thread is left at a barrier
            ok = false;
            break;
        }
        const int jn = min(KB_T, n - tj * KB_T), jl0 = tj * KB_T;
        if (COM) {
            if (tid < KB_T) sm.cj[tid] = tid < jn ? cv.cl[start + jl0 + tid] : -1;
            __syncthreads();
        }
        if (OKM) {
            // the row's fast partners inside this j-tile (partners ascend, so
            // the cursor only moves forward)
            if (tid < KB_T) {
                const int jb = start + jl0;
                uint32_t mk = 0u;
                int q = sm.okc[tid];
                const int qe = sm.oke[tid];
                while (q < qe && okv.col[2 * q + 1] < jb + jn) {
                    const int d = okv.col[2 * q + 1] - jb;
                    if (d >= 0) mk |= 1u << d;
                    ++q;
                }
                sm.okc[tid] = q;
                sm.okm[tid] = mk;
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < KB_Q; ++q) {
            const int pidx = tid + q * KB_THREADS, ii = pidx >> 5, jj = pidx & 31;
            bool use = ii < ni && jj < jn && il0 + ii != jl0 + jj && sm.li[ii] != sm.j.lab[st][jj];
            if (COM && use && sm.ci[ii] >= 0 && sm.cj[jj] >= 0)
                use = cv.far[fo + (long long)sm.ci[ii] * Ks + sm.cj[jj]] == 0;
            if (OKM && use) use = ((sm.okm[ii] >> jj) & 1u) == 0u;
            if (PRE) {
                sm.f[0][ii][jj] = use ? fr[0][q] : 0.0;
                sm.f[1][ii][jj] = use ? fr[1][q] : 0.0;
                sm.f[2][ii][jj] = use ? fr[2][q] : 0.0;
                continue;
            }
            const double dx0 = __dsub_rn(sm.j.col[st][0][jj], sm.xi[0][ii]);
            const double dx1 = __dsub_rn(sm.j.col[st][1][jj], sm.xi[1][ii]);
            const double dx2 = __dsub_rn(sm.j.col[st][2][jj], sm.xi[2][ii]);
            const double r2 = __dadd_rn(
                __dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)), __dmul_rn(dx2, dx2)), eps2);
            const double rinv3 = __drcp_rn(__dmul_rn(r2, __dsqrt_rn(r2)));
            const double w = __dmul_rn(__dmul_rn(G, sm.j.col[st][3][jj]), rinv3);
            sm.f[0][ii][jj] = use ? __dmul_rn(w, dx0) : 0.0;
            sm.f[1][ii][jj] = use ? __dmul_rn(w, dx1) : 0.0;
            sm.f[2][ii][jj] = use ? __dmul_rn(w, dx2) : 0.0;
        }
        // the next j-tile's forces into registers while this one is summed
        if (PRE && tj + 1 < nt) load_f(tj + 1);
        __syncthreads();
        if (tid < 3 * KB_T)
            for (int jj = 0; jj < jn; ++jj) acc = __dadd_rn(acc, sm.f[c][r][jj]);
        __syncthreads();
    }
    if (!ok) {
        raise_err(ctr, DERR_TMA_TIMEOUT);
        // let any copy still in flight land before the CTA exits
        mbar_wait(&sm.j.bar[0], 0, TMA_WAIT_CYCLES);
        mbar_wait(&sm.j.bar[1], 0, TMA_WAIT_CYCLES);
        return;
    }
    if (tid < 3 * KB_T && r < ni) {
        const int i = start + il0 + r;
        double *v = c == 0 ? L.vx : (c == 1 ? L.vy : L.vz);
        v[i] = __dadd_rn(v[i], __dmul_rn(h, acc));
    }
}

// The force G m_j r_ij^-3 (x_j - x_i) of every ordered pair (i, j) of each
// set into its three n x n matrices (components x, y, z) at pf.moff[s] (row
// i, column j; the diagonal unused).  One block per 128-wide triangular tile
// (TI <= TJ; the grid and prefix L.tile_off of the 128-wide tau tiles), in
// 32 x 32 sub-tiles: every unordered pair is evaluated once with the kick's
// own operations (dx = x_j - x_i; the squares make r^2, and so r^-3, the same
// bits for (j, i), and x_i - x_j = -dx exactly); (G m_j) r^-3 dx goes to row
// i directly, -(G m_i) r^-3 dx to row j through shared memory.
constexpr int KR_T = 32, KR_W = 128;
static_assert(KR_T == KB_T, "the force sub-tiles are the kick's i-tiles");
static_assert(KR_W == TAU_VAR_T[TAU_VAR_128], "the force tiles are the 128-wide tau tiles");
__global__ void __launch_bounds__(KB_THREADS) k_pair_forces(Level L, double G, double eps2, PairFactors pf)
{
    __shared__ double xi[4][KR_W];  // x, y, z, G m
    __shared__ double xj[4][KR_W];
    __shared__ double t[3][KR_T][KR_T + 1];
    const int tid = threadIdx.x;
    const int s = find_set(L.tile_off, L.nsets, blockIdx.x);
    int tt = blockIdx.x - L.tile_off[s];
    const int n = L.set_n[s], start = L.set_start[s];
    const long long nn = (long long)n * n;
    const int nT = (n + KR_W - 1) / KR_W;
    const int TI = tri_tile_row(tt, nT), TJ = TI + tt;
    const int i0 = TI * KR_W, j0 = TJ * KR_W;
    const int ni = min(KR_W, n - i0), nj = min(KR_W, n - j0);
    double *S = pf.S + pf.moff[s];
    for (int e = tid; e < KR_W; e += KB_THREADS) {
        const bool vi = e < ni, vj = e < nj;
        xi[0][e] = vi ? L.x[start + i0 + e] : 0.0;
        xi[1][e] = vi ? L.y[start + i0 + e] : 0.0;
        xi[2][e] = vi ? L.z[start + i0 + e] : 0.0;
        xi[3][e] = vi ? __dmul_rn(G, L.m[start + i0 + e]) : 0.0;
        xj[0][e] = vj ? L.x[start + j0 + e] : 0.0;
        xj[1][e] = vj ? L.y[start + j0 + e] : 0.0;
        xj[2][e] = vj ? L.z[start + j0 + e] : 0.0;
        xj[3][e] = vj ? __dmul_rn(G, L.m[start + j0 + e]) : 0.0;
    }
    for (int a = 0; a < KR_W / KR_T; ++a) {
        for (int b = TI == TJ ? a : 0; b < KR_W / KR_T; ++b) {
            const int il = a * KR_T, jl = b * KR_T;
            if (il >= ni || jl >= nj) continue;  // (uniform over the block)
            __syncthreads();  // (the staged rows, or the previous sub-tile's transposed write)
#pragma unroll
            for (int q = 0; q < KB_Q; ++q) {
                const int pidx = tid + q * KB_THREADS, ii = pidx >> 5, jj = pidx & 31;
                const int gi = il + ii, gj = jl + jj;
                if (gi < ni && gj < nj && j0 + gj > i0 + gi) {
                    const double dx0 = __dsub_rn(xj[0][gj], xi[0][gi]);
                    const double dx1 = __dsub_rn(xj[1][gj], xi[1][gi]);
                    const double dx2 = __dsub_rn(xj[2][gj], xi[2][gi]);
                    const double r2 = __dadd_rn(
                        __dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)), __dmul_rn(dx2, dx2)), eps2);
                    const double v = __drcp_rn(__dmul_rn(r2, __dsqrt_rn(r2)));
                    const double wij = __dmul_rn(xj[3][gj], v), wji = __dmul_rn(xi[3][gi], v);
                    const long long e = (long long)(i0 + gi) * n + (j0 + gj);
                    S[e] = __dmul_rn(wij, dx0);
                    S[nn + e] = __dmul_rn(wij, dx1);
                    S[2 * nn + e] = __dmul_rn(wij, dx2);
                    t[0][ii][jj] = -__dmul_rn(wji, dx0);
                    t[1][ii][jj] = -__dmul_rn(wji, dx1);
                    t[2][ii][jj] = -__dmul_rn(wji, dx2);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < KB_Q; ++q) {
                const int pidx = tid + q * KB_THREADS, jj = pidx >> 5, ii = pidx & 31;
                const int gi = il + ii, gj = jl + jj;
                if (gi < ni && gj < nj && j0 + gj > i0 + gi) {
                    const long long e = (long long)(j0 + gj) * n + (i0 + gi);
                    S[e] = t[0][ii][jj];
                    S[nn + e] = t[1][ii][jj];
                    S[2 * nn + e] = t[2][ii][jj];
                }
            }
        }
    }
}

void launch_kick(const Level &L, const int32_t *label, int nitiles, double G, double eps2, double h,
                 int variant, DevCounters *ctr, cudaStream_t s, const ComView *com, const OkView *okv,
                 const PairFactors *pf)
{
    (void)variant;  // one shape: 32-body tiles (the prefix of variant 0)
    if (nitiles <= 0) return;
    const ComView nc{nullptr, nullptr, nullptr, nullptr};
    const OkView no{nullptr, nullptr};
    const PairFactors np{nullptr, nullptr, 0};
    if (okv && okv->row_ptr && pf && pf->S) {
        k_pair_forces<<<pf->nblocks, KB_THREADS, 0, s>>>(L, G, eps2, *pf);
        k_kick64<4><<<nitiles, KB_THREADS, 0, s>>>(L, label, G, eps2, h, ctr, nc, *okv, *pf);
        CC_COUNT_LAUNCH(1);
    } else if (okv && okv->row_ptr) {
        k_kick64<2><<<nitiles, KB_THREADS, 0, s>>>(L, label, G, eps2, h, ctr, nc, *okv, np);
    } else if (com && com->cl) {
        k_kick64<1><<<nitiles, KB_THREADS, 0, s>>>(L, label, G, eps2, h, ctr, *com, no, np);
    } else if (pf && pf->S) {
        k_pair_forces<<<pf->nblocks, KB_THREADS, 0, s>>>(L, G, eps2, *pf);
        k_kick64<3><<<nitiles, KB_THREADS, 0, s>>>(L, label, G, eps2, h, ctr, nc, no, *pf);
        CC_COUNT_LAUNCH(1);
    } else {
        k_kick64<0><<<nitiles, KB_THREADS, 0, s>>>(L, label, G, eps2, h, ctr, nc, no, np);
    }
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ energy
constexpr int EN_T = 128;

int energy_blocks(long long n) { return (int)((n + EN_T - 1) / EN_T); }

// Kinetic and potential energy, momentum and angular momentum.  With
// independent systems (sys_off, nsys + 1 offsets) the potential sums only
// pairs inside one system: systems never interact, so a pair of two
// systems belongs to no system's Hamiltonian.
__global__ void __launch_bounds__(EN_T) k_energy(const double *x3, const double *v3, const double *m,
                                                  long long n, double G, double eps2, const int32_t *sys_off,
                                                  int nsys, double *partial)
{
    __shared__ double sx[EN_T], sy[EN_T], sz[EN_T], smm[EN_T];
    __shared__ double red[8][EN_T / 32];
    __shared__ long long blk_hi;
    const long long i = (long long)blockIdx.x * EN_T + threadIdx.x;
    const bool iv = i < n;
    double xi = 0, yi = 0, zi = 0, mi = 0, vx = 0, vy = 0, vz = 0;
    if (iv) {
        xi = x3[i]; yi = x3[n + i]; zi = x3[2 * n + i];
        vx = v3[i]; vy = v3[n + i]; vz = v3[2 * n + i];
        mi = m[i];
    }
    // the end of i's system (binary search over the offsets)
    long long hi = n;
    if (iv && sys_off && nsys > 1) {
        int lo = 0, up = nsys;  // sys_off[lo] <= i < sys_off[up]
        while (up - lo > 1) {
            const int mid = (lo + up) >> 1;
            if ((long long)sys_off[mid] <= i) lo = mid;
            else up = mid;
        }
        hi = sys_off[up];
    }
    if (threadIdx.x == 0) blk_hi = 0;
    __syncthreads();
    if (iv) atomicMax((unsigned long long *)&blk_hi, (unsigned long long)hi);
    __syncthreads();
    const long long jend = blk_hi;
    double V = 0.0;
    for (long long j0 = (long long)blockIdx.x * EN_T; j0 < jend; j0 += EN_T) {
        const long long j = j0 + threadIdx.x;
        __syncthreads();
        if (j < n) {
            sx[threadIdx.x] = x3[j]; sy[threadIdx.x] = x3[n + j]; sz[threadIdx.x] = x3[2 * n + j];
            smm[threadIdx.x] = m[j];
        }
        __syncthreads();
        if (iv) {
            const int jn = (int)min((long long)EN_T, n - j0);
            for (int k = 0; k < jn; ++k) {
                if (j0 + k <= i || j0 + k >= hi) continue;
                const double dx = sx[k] - xi, dy = sy[k] - yi, dz = sz[k] - zi;
                V -= G * mi * smm[k] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
            }
        }
    }
    double q[8];
    q[0] = iv ? 0.5 * mi * (vx * vx + vy * vy + vz * vz) : 0.0;
    q[1] = V;
    q[2] = mi * vx; q[3] = mi * vy; q[4] = mi * vz;
    q[5] = mi * (yi * vz - zi * vy);
    q[6] = mi * (zi * vx - xi * vz);
    q[7] = mi * (xi * vy - yi * vx);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        double val = q[c];
        for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = val;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double acc = 0.0;
        for (int w = 0; w < EN_T / 32; ++w) acc += red[threadIdx.x][w];
        partial[blockIdx.x * 8 + threadIdx.x] = acc;
    }
}

void launch_energy(const double *x3, const double *v3, const double *m, long long n, double G, double eps2,
                   const int32_t *sys_off, int nsys, double *partial, int nblk, cudaStream_t s)
{
    if (n <= 0) return;
    k_energy<<<nblk, EN_T, 0, s>>>(x3, v3, m, n, G, eps2, sys_off, nsys, partial);
    CC_COUNT_LAUNCH(1);
}

}  // namespace cc

// ------------------------------------------------------------ peak probe
// FMA throughput microbenchmarks (the ALU roofline denominators): every
// thread advances 8 independent FMA chains; flops = 2 per FMA.
namespace cc {

template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(T b, T c, int iters, T *out)
{
    T a0 = (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    const T r = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (r == (T)-12345.678) out[blockIdx.x] = r;  // keeps the chains live
}

double probe_fma(int fp64, int nsm, cudaStream_t s)
{
    const int blocks = nsm * 8, threads = 256;
    const int iters = fp64 ? 512 : 16384;
    void *out = nullptr;
    cudaMalloc(&out, blocks * 8);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        if (fp64)
            k_probe_fma<double><<<blocks, threads, 0, s>>>(0.999999, 1e-7, iters, (double *)out);
        else
            k_probe_fma<float><<<blocks, threads, 0, s>>>(0.999999f, 1e-7f, iters, (float *)out);
        CC_COUNT_LAUNCH(1);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    return flops / (best * 1e-3);
}

}  // namespace cc
