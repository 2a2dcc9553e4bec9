// cc_mixed.cu -- mixed-precision forms of the two pair kernels of the CC
// split (arXiv:1407.7105, Eqs. tauij, kickij/kickji):
//
//  * k_tau_mixed: the edge predicate tau(i,j) < h decided in FP32 with a
//    rigorous per-pair error bound; a pair whose FP32 value is too close to
//    h for the bound to decide is re-evaluated with the exact FP64
//    predicate (tau_fp64), so the edge set is identical to the FP64 one.
//    Every split of both forms (and the OK split's outer level) runs it.
//  * k_kick_mixed: pair forces in FP32 from float-float position
//    differences, rsqrt plus one Newton step, Kahan-compensated FP32 sums,
//    partial sums over j-chunks combined in FP64; v stays FP64.
//
// Positions and velocities are carried as float pairs (hi = fl32(x),
// lo = fl32(x - hi)), so x_j - x_i = (hi_j - hi_i) + (lo_j - lo_i) is formed
// with relative error <= 2u + 11 u^2 X / r (u = 2^-24, X = max |x|),
// the accuracy of an FP64 difference rounded to FP32 up to one more
// rounding, at three FP32 additions instead of three FP64 subtractions
// (GB300 issues FP64 at 1/58 of the FP32 rate).
#include "cc_device.cuh"

namespace cc {

// ------------------------------------------------------------ prep
// float-float copy of the packed state; per-level maxima of |x| and |v|
__global__ void k_prep_ff(Level L, FFView F, float G, int with_v, int init_forest, unsigned long long *edge_count)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    float ax = 0.f, av = 0.f;
    if (init_forest) {
        // the split's union-find starts as singletons (what k_init_parent does)
        if (k < L.total) {
            L.parent[k] = k;
            L.cnt[k] = 0;
        }
        if (k == 0 && edge_count) *edge_count = 0ull;
    }
    if (k < L.total && L.gid[k] >= 0) {
        const double xs[3] = {L.x[k], L.y[k], L.z[k]};
        float hi[3], lo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ff_split(xs[c], hi[c], lo[c]);
            ax = fmaxf(ax, fabsf(hi[c]));
        }
        F.pq[2 * k] = make_float4(hi[0], hi[1], hi[2], G * fl32(L.m[k]));
        F.pq[2 * k + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
        if (with_v) {
            const double vs[3] = {L.vx[k], L.vy[k], L.vz[k]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ff_split(vs[c], hi[c], lo[c]);
                av = fmaxf(av, fabsf(hi[c]));
            }
            F.vq[2 * k] = make_float4(hi[0], hi[1], hi[2], 0.f);
            F.vq[2 * k + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
        }
    }
    // positive floats order like their bit patterns
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax = fmaxf(ax, __shfl_xor_sync(0xffffffffu, ax, o));
        av = fmaxf(av, __shfl_xor_sync(0xffffffffu, av, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (ax > 0.f) atomicMax((int *)&F.maxes[0], __float_as_int(ax));
        if (av > 0.f) atomicMax((int *)&F.maxes[1], __float_as_int(av));
    }
}

void launch_prep_ff(const Level &L, const FFView &F, double G, bool with_v, cudaStream_t s, bool init_forest,
                    unsigned long long *edge_count)
{
    if (L.total <= 0) return;
    cudaMemsetAsync(F.maxes, 0, 2 * sizeof(float), s);
    k_prep_ff<<<(L.total + 255) / 256, 256, 0, s>>>(L, F, (float)G, with_v ? 1 : 0, init_forest ? 1 : 0,
                                                    edge_count);
    CC_COUNT_LAUNCH(1);
}

// positions (hi, G m), (lo) and labels in the root-sorted order of the
// split: position t holds packed element order[t].  dt > 0: the level's
// first drift D_{h/2,T_R} of rest-set members (component size 1, Eq. drift,
// exact IEEE operations) is applied first, in the same pass.
__global__ void k_prep_kick(Level L, FFView F, const int32_t *order, const int32_t *root, float G, double dt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L.total) return;
    const int k = order[t];
    if (L.gid[k] < 0) {
        L.klab[t] = -1 - t;
        return;
    }
    if (dt > 0.0 && L.cnt[root[k]] == 1) {
        L.x[k] = __dadd_rn(L.x[k], __dmul_rn(dt, L.vx[k]));
        L.y[k] = __dadd_rn(L.y[k], __dmul_rn(dt, L.vy[k]));
        L.z[k] = __dadd_rn(L.z[k], __dmul_rn(dt, L.vz[k]));
    }
    const double xs[3] = {L.x[k], L.y[k], L.z[k]};
    float hi[3], lo[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ff_split(xs[c], hi[c], lo[c]);
    F.pq[2 * t] = make_float4(hi[0], hi[1], hi[2], G * fl32(L.m[k]));
    F.pq[2 * t + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    L.klab[t] = root[k];
}

void launch_prep_kick(const Level &L, const FFView &F, const int32_t *order, const int32_t *root, double G,
                      double drift_dt, cudaStream_t s)
{
    if (L.total <= 0) return;
    k_prep_kick<<<(L.total + 255) / 256, 256, 0, s>>>(L, F, order, root, (float)G, drift_dt);
    CC_COUNT_LAUNCH(1);
}


constexpr int TAU_JG = 8;  // columns per group of the group certificates (rows: a warp's 32)

template <int T, int S>
struct __align__(16) MixedTauSmem {
    float4 pq[2 * T];   // positions (hi, Gm), (lo) of the j-tile
    float4 vq[2 * T];   // velocities (hi), (lo)
    int32_t lp[2 * T];  // local union-find over the tile's particles
    uint32_t q[T * S / 32][64];  // per warp: pairs waiting for the certified decision
    uint32_t om[T * S / 32][T / S];       // per warp and column: lanes whose pair is still open
    uint32_t cm[T * S / 32][T / S / 32];  // per warp and 32 columns: columns with open pairs
    GroupBox jb[T / TAU_JG];               // boxes of the j-tile's TAU_JG-column groups
    float gthr[T * S / 32][T / S / TAU_JG];  // per warp and column group: |dv~|^2 threshold, < 0: none
    uint64_t bar;
};

// min / max over each aligned segment of W lanes
template <int W>
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int W>
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// box of the high parts held by the lanes with `on` in each aligned segment
// of W lanes (p = (x, y, z, G m), v = (vx, vy, vz)); returns false if no
// lane of the segment is on
template <int W>
__device__ __forceinline__ bool warp_group_box(bool on, float4 p, float4 v, GroupBox &B)
{
    const float inf = __int_as_float(0x7f800000);
    B.xlo[0] = warp_min<W>(on ? p.x : inf);
    B.xlo[1] = warp_min<W>(on ? p.y : inf);
    B.xlo[2] = warp_min<W>(on ? p.z : inf);
    B.xhi[0] = warp_max<W>(on ? p.x : -inf);
    B.xhi[1] = warp_max<W>(on ? p.y : -inf);
    B.xhi[2] = warp_max<W>(on ? p.z : -inf);
    B.vlo[0] = warp_min<W>(on ? v.x : inf);
    B.vlo[1] = warp_min<W>(on ? v.y : inf);
    B.vlo[2] = warp_min<W>(on ? v.z : inf);
    B.vhi[0] = warp_max<W>(on ? v.x : -inf);
    B.vhi[1] = warp_max<W>(on ? v.y : -inf);
    B.vhi[2] = warp_max<W>(on ? v.z : -inf);
    B.gm = warp_max<W>(on ? p.w : 0.f);
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a = fmaxf(a, fmaxf(fabsf(B.xlo[k]), fabsf(B.xhi[k])));
        b = fmaxf(b, fmaxf(fabsf(B.vlo[k]), fabsf(B.vhi[k])));
    }
    B.amax = a;
    B.vabs = b;
    const unsigned seg = (W == 32 ? 0xffffffffu : ((1u << W) - 1u)) << ((threadIdx.x & 31) & ~(W - 1));
    return (__ballot_sync(0xffffffffu, on) & seg) != 0u;
}

// local union-find in shared memory (indices 0..2T-1, links to the smaller)
__device__ __forceinline__ int luf_find(volatile int32_t *p, int x)
{
    while (true) {
        const int q = p[x];
        if (q == x) return x;
        const int g = p[q];
        if (g != q) p[x] = g;
        x = q;
    }
}

__device__ __forceinline__ bool luf_union(int32_t *p, int a, int b)
{
    volatile int32_t *vp = p;
    for (int it = 0; it < (1 << 20); ++it) {
        a = luf_find(vp, a);
        b = luf_find(vp, b);
        if (a == b) return true;
        if (a > b) {
            const int t = a; a = b; b = t;
        }
        if (atomicCAS(&p[b], b, a) == b) return true;
    }
    return false;
}

// Settles the warp's queued pairs sm.q[w][0..cnt), one per lane: the
// certified FP32 decision on the float-float differences, the exact FP64
// predicate when it is undecided, then the local union and the edge record
// (one counter update per batch).  Out of line: the pair loop keeps only the
// high parts and its queue in registers.
template <int T, int S>
__device__ __noinline__ uint2 tau_settle_batch(MixedTauSmem<T, S> &sm, int w, int cnt, int ibase, int j0, int joff,
                                              const Level &L, const FFView &F, const TauParams &P,
                                              const MixedTauParams &Q, DevCounters *ctr, int32_t *near_ij,
                                              double *near_tau, long long near_cap, const EdgeList &E)
{
    // returns (edges, FP64 evaluations) of this lane's pair
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const bool has = lane < cnt;
    const unsigned ent = has ? sm.q[w][lane] : 0u;
    const int ii = (int)(ent >> 8), kk = (int)(ent & 255u);
    int dec = 0;
    unsigned nfp64 = 0u;
    double tau = CUDART_NAN;
    if (has) {
        const int gi = ibase + ii, gj = j0 + kk;
        const float4 a0 = F.pq[2 * gi], a1 = F.pq[2 * gi + 1], b0 = F.vq[2 * gi], b1 = F.vq[2 * gi + 1];
        const float cX = 11.f * U32 * U32 * F.maxes[0], cV = 11.f * U32 * U32 * F.maxes[1];
        const float4 jp0 = sm.pq[2 * kk], jp1 = sm.pq[2 * kk + 1], jv0 = sm.vq[2 * kk], jv1 = sm.vq[2 * kk + 1];
        dec = tau_decide_fp32((jp0.x - a0.x) + (jp1.x - a1.x), (jp0.y - a0.y) + (jp1.y - a1.y),
                              (jp0.z - a0.z) + (jp1.z - a1.z), (jv0.x - b0.x) + (jv1.x - b1.x),
                              (jv0.y - b0.y) + (jv1.y - b1.y), (jv0.z - b0.z) + (jv1.z - b1.z), a0.w + jp0.w, cX, cV,
                              Q);
        if (dec < 0) {
            // undecided: the exact FP64 predicate
            tau = tau_fp64(__dsub_rn(L.x[gi], L.x[gj]), __dsub_rn(L.y[gi], L.y[gj]), __dsub_rn(L.z[gi], L.z[gj]),
                           __dsub_rn(L.vx[gi], L.vx[gj]), __dsub_rn(L.vy[gi], L.vy[gj]),
                           __dsub_rn(L.vz[gi], L.vz[gj]), L.m[gi], L.m[gj], P);
            nfp64 = 1u;
            if (fabs(tau - P.h) < P.near_tol * P.h) {
                const unsigned long long q = atomicAdd(&ctr->near_pairs, 1ull);
                if ((long long)q < near_cap) {
                    const int pi = L.gid[gi], pj = L.gid[gj];
                    near_ij[2 * q] = pi < pj ? pi : pj;
                    near_ij[2 * q + 1] = pi < pj ? pj : pi;
                    near_tau[q] = tau;
                }
            }
            dec = tau < P.h ? 1 : 0;
        }
    }
    const bool edge = dec > 0;
    const unsigned eb = __ballot_sync(0xffffffffu, edge);
    if (eb == 0u) return make_uint2(0u, nfp64);
    if (edge && !luf_union(sm.lp, ii, joff + kk)) raise_err(ctr, DERR_UF_RETRY);
    if (E.rec) {
        // every edge is recorded (the decision at h/2 is left to the first
        // half's pass); tau = the FP64 value or NaN
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(E.count, (unsigned long long)__popc(eb));
        base = __shfl_sync(0xffffffffu, base, 0);
        const unsigned long long q = base + (unsigned)__popc(eb & lt);
        if (edge && (long long)q < E.cap) {
            EdgeRec r;
            r.a = ibase + ii;
            r.b = j0 + kk;
            r.e = -1;
            r.pad = 0;
            r.tau = tau;
            E.rec[q] = r;
        }
    }
    return make_uint2(edge ? 1u : 0u, nfp64);
}

// Block = T x S threads: thread (row r, slice s) takes pairs (r, k) of the
// tile with k in the slice's T/S columns (S > 1 shortens each warp's chain
// for sets with few tiles).  Parameters are grid constants: the out-of-line
// settle takes them by reference without a copy.
template <int T, int S>
__global__ void __launch_bounds__(T * S, 1024 / (T * S))
    k_tau_mixed(const __grid_constant__ Level L, const __grid_constant__ FFView F,
                const __grid_constant__ TauParams P, const __grid_constant__ MixedTauParams Q, DevCounters *ctr,
                int32_t *near_ij, double *near_tau, long long near_cap, const __grid_constant__ EdgeList E)
{
    static_assert(T % 32 == 0 && T % S == 0, "tile shape");
    __shared__ MixedTauSmem<T, S> sm;
    const int tid = threadIdx.x, row = tid % T, slice = tid / T;
    int lo = 0, hi = L.nsets;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (L.tile_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
    }
    const int s = lo;
    int t = blockIdx.x - L.tile_off[s];
    const int n = L.set_n[s], start = L.set_start[s];
    const int nt = (n + T - 1) / T;
    const int ti = tri_tile_row(t, nt);
    const int tj = ti + t;
    const bool diag = ti == tj;
    const int j0 = start + tj * T;
    const int jn = min(T, n - tj * T);
    if (tid == 0) {
        mbar_init(&sm.bar, 1);
        fence_mbar_init();
    }
    for (int e = tid; e < 2 * T; e += T * S) sm.lp[e] = e;
    __syncthreads();
    // fault_test = 1: the copy is announced but never issued, so the wait
    // below runs out (a test of the bounded wait; no copy is in flight)
    const bool no_copy = P.fault_test == 1;
    const long long wait_cycles = no_copy ? FAULT_TEST_WAIT_CYCLES : TMA_WAIT_CYCLES;
    if (tid == 0) {
        const unsigned bytes = (unsigned)jn * 32u;
        mbar_expect_tx(&sm.bar, 2u * bytes);
        if (!no_copy) {
            tma_load_1d(sm.pq, F.pq + 2 * (size_t)j0, bytes, &sm.bar);
            tma_load_1d(sm.vq, F.vq + 2 * (size_t)j0, bytes, &sm.bar);
        }
    }
    const int il = ti * T + row;
    const bool iv = il < n;
    const int i = start + il;
    float4 ip0 = make_float4(0, 0, 0, 0), iv0 = ip0;
    if (iv) {
        ip0 = F.pq[2 * i];
        iv0 = F.vq[2 * i];
    }
    const bool got = mbar_wait(&sm.bar, 0, wait_cycles);
    if (__syncthreads_or(!got)) {
        raise_err(ctr, DERR_TMA_TIMEOUT);
        // let a copy still in flight land before the CTA exits
        mbar_wait(&sm.bar, 0, wait_cycles);
        return;
    }
    unsigned long long my_edges = 0, my_fp64 = 0;
    const int joff = diag ? 0 : T;  // local index base of the j-tile
    const int lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    // column groups per tile, per warp; groups whose boxes a warp computes
    constexpr int NG = T / TAU_JG, GW = T / S / TAU_JG, GPW = 32 / TAU_JG;
    // Group certificates: the warp's 32 rows against each TAU_JG-column group
    // of its columns (tau_groups_apart).  A certified group costs each pair
    // one velocity difference and a comparison.
    if (w * GPW < NG) {
        const int k = TAU_JG * (w * GPW) + lane;  // lane segment s: group w GPW + s
        GroupBox B;
        const bool any =
            warp_group_box<TAU_JG>(k < jn, k < jn ? sm.pq[2 * k] : ip0, k < jn ? sm.vq[2 * k] : iv0, B);
        if ((lane & (TAU_JG - 1)) == 0) {
            if (!any) B.gm = -1.f;  // empty group: no pairs
            sm.jb[w * GPW + lane / TAU_JG] = B;
        }
    }
    {
        GroupBox A;
        const bool any = warp_group_box<32>(iv, ip0, iv0, A);
        __syncthreads();
        if (lane < GW) {
            const GroupBox &B = sm.jb[slice * GW + lane];
            float thr = -1.f;
            if (any && B.gm >= 0.f && !diag && !tau_groups_apart(A, B, Q, thr)) thr = -1.f;
            sm.gthr[w][lane] = thr;
        }
        __syncwarp();
    }
    // the pre-test's error terms for high-part differences: per component
    // |x_j| <= |x_i| + r, so |dx~ - dx| <= u r + 3.5 u (2 max|x_i| + r): c_x =
    // 7 u max|x_i| per thread, and the remaining 3.5 u r goes to the
    // threshold (likewise for the velocities)
    const float cXh = 7.1f * U32 * fmaxf(fabsf(ip0.x), fmaxf(fabsf(ip0.y), fabsf(ip0.z)));
    const float cVh = 7.1f * U32 * fmaxf(fabsf(iv0.x), fmaxf(fabsf(iv0.y), fabsf(iv0.z)));
    // Pairs the certificates leave open are queued per warp and settled 32
    // at a time, one per lane: taken as they come, a single such pair would
    // run the certified decision (and possibly FP64) with one lane of 32
    // active.  Entry = (row in the i-tile << 8) | column in the j-tile.
    auto settle = [&](int cnt) {
        const uint2 c = tau_settle_batch<T, S>(sm, w, cnt, start + ti * T, j0, joff, L, F, P, Q, ctr, near_ij,
                                               near_tau, near_cap, E);
        my_edges += c.x;
        my_fp64 += c.y;
    };
    int qn = 0;  // entries queued by this warp (warp-uniform)
    // the warp's columns [kb, k1): one trip count for all its lanes, so each
    // column ends in a vote (the common case: no lane's pair left open)
    const int kb = slice * (T / S), k1 = min(jn, kb + T / S);
    // the full high-part certificate of pair (row, k)
    auto quick = [&](int k) {
        const float4 jp0 = sm.pq[2 * k], jv0 = sm.vq[2 * k];
        return tau_quick_apart(jp0.x - ip0.x, jp0.y - ip0.y, jp0.z - ip0.z, jv0.x - iv0.x, jv0.y - iv0.y,
                               jv0.z - iv0.z, ip0.w + jp0.w, cXh, cVh, Q);
    };
    // Pass 1, the hot loop: certificates only.  A column with open pairs
    // (rare) leaves its lane word in sm.om and its bit in sm.cm.
    if (lane < T / S / 32) sm.cm[w][lane] = 0u;
    __syncwarp();
#pragma unroll 1
    for (int g = 0; g < GW; ++g) {
        const int ka = kb + TAU_JG * g, kz = min(k1, ka + TAU_JG);
        const float thr = sm.gthr[w][g];
        if (thr >= 0.f) {
            // certified group: one velocity difference per pair; a pair
            // below the lower speed root takes the full certificate
            for (int k = ka; k < kz; ++k) {
                const bool mine = iv && (!diag || k > row);
                const float4 jv0 = sm.vq[2 * k];
                const float a = jv0.x - iv0.x, b = jv0.y - iv0.y, c = jv0.z - iv0.z;
                const bool slow = mine && fmaf(c, c, fmaf(b, b, a * a)) < thr;
                if (__ballot_sync(0xffffffffu, slow) == 0u) continue;
                const unsigned open = __ballot_sync(0xffffffffu, slow && !quick(k));
                if (open && lane == 0) {
                    sm.om[w][k - kb] = open;
                    sm.cm[w][(k - kb) >> 5] |= 1u << ((k - kb) & 31);
                }
            }
        } else {
            for (int k = ka; k < kz; ++k) {
                const unsigned open = __ballot_sync(0xffffffffu, iv && (!diag || k > row) && !quick(k));
                if (open && lane == 0) {
                    sm.om[w][k - kb] = open;
                    sm.cm[w][(k - kb) >> 5] |= 1u << ((k - kb) & 31);
                }
            }
        }
    }
    __syncwarp();
    // Pass 2: the open pairs, queued and settled 32 at a time
    for (int c = 0; c < T / S / 32; ++c) {
        unsigned cols = sm.cm[w][c];
        while (cols) {
            const int k = kb + 32 * c + __ffs(cols) - 1;
            cols &= cols - 1u;
            const unsigned open = sm.om[w][k - kb];
            if ((open >> lane) & 1u) sm.q[w][qn + __popc(open & lt)] = ((unsigned)row << 8) | (unsigned)k;
            qn += __popc(open);
            if (qn >= 32) {
                __syncwarp();
                settle(32);
                __syncwarp();
                if (lane < qn - 32) sm.q[w][lane] = sm.q[w][32 + lane];
                __syncwarp();
                qn -= 32;
            }
        }
    }
    if (qn > 0) {
        __syncwarp();
        settle(qn);
    }
    __syncthreads();
    // merge the tile's local components into the global forest: one union
    // per local non-root element instead of one per edge
    for (int e = tid; e < (diag ? T : 2 * T); e += T * S) {
        const int r = luf_find(sm.lp, e);
        if (r != e) {
            const int ge = (e < T) ? start + ti * T + e : j0 + (e - T);
            const int gr = (r < T) ? start + ti * T + r : j0 + (r - T);
            // (fault_test = 2: every hook gives up at once, a test of the retry cap)
            if (!uf_union(L.parent, ge, gr, P.fault_test == 2 ? 0 : UF_RETRY_MAX)) raise_err(ctr, DERR_UF_RETRY);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_edges += __shfl_down_sync(0xffffffffu, my_edges, o);
        my_fp64 += __shfl_down_sync(0xffffffffu, my_fp64, o);
    }
    if ((tid & 31) == 0) {
        if (my_edges) atomicAdd(&ctr->edges, my_edges);
        if (my_fp64) atomicAdd(&ctr->tau_fp64, my_fp64);
    }
}

void launch_tau_mixed(const Level &L, const FFView &F, int ntiles, const TauParams &P, int variant,
                      DevCounters *ctr, int32_t *near_ij, double *near_tau, long long near_cap, const EdgeList &E,
                      cudaStream_t s)
{
    if (ntiles <= 0) return;
    MixedTauParams Q;
    Q.eta = (float)P.eta_in;
    Q.etah = (float)(P.eta_outside ? P.eta_in * P.eta / P.h : P.eta_in / P.h);
    Q.eps2 = (float)P.eps2;
    Q.G = (float)P.G;
    Q.hq = (float)(P.eta_outside ? P.h / P.eta : P.h);  // h/eta_in in the units of T: eta_in/etah
    static_assert(TAU_VAR_T[0] == 64 && TAU_VAR_T[1] == 128 && TAU_VAR_T[2] == 64 && TAU_VAR_S[2] == 2,
                  "tau variants");
    if (variant == 0)
        k_tau_mixed<64, 1><<<ntiles, 64, 0, s>>>(L, F, P, Q, ctr, near_ij, near_tau, near_cap, E);
    else if (variant == 1)
        k_tau_mixed<128, 1><<<ntiles, 128, 0, s>>>(L, F, P, Q, ctr, near_ij, near_tau, near_cap, E);
    else
        k_tau_mixed<64, 2><<<ntiles, 128, 0, s>>>(L, F, P, Q, ctr, near_ij, near_tau, near_cap, E);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ kick, FP32
// Works in the root-sorted order of the split (members of a component are
// adjacent; rest-set members are their own components).  Grid: (set,
// i-tile, j-chunk).  Thread r of an i-tile accumulates
// sum_j G m_j (x_j - x_i) |x_j - x_i|^-3 over the chunk's j whose label
// differs in FP32 (groups of MK_GROUP terms, each group sum added with
// compensation); a j-tile whose labels and the i-tile's are
// all one component is skipped whole (sorted order: first == last label
// means a uniform tile).  Partials go to scratch in FP64 unless the set has
// a single chunk, in which case v is updated directly.
constexpr int MK_T = 128;
constexpr int MK_CHUNK_MAX = 4;  // j-tiles per chunk (tuned per size bin)
static_assert(MK_VAR_CHUNK[0] <= MK_CHUNK_MAX && MK_VAR_CHUNK[1] <= MK_CHUNK_MAX && MK_VAR_CHUNK[2] <= MK_CHUNK_MAX,
              "chunk variants");
constexpr int MK_GROUP = 8;       // j terms summed in plain FP32 per compensated addition

struct __align__(16) MixedKickSmem {
    float4 pq[2][2 * MK_T];  // (hi, Gm), (lo) per j, two stages
    int32_t lab[2][MK_T];
    int32_t cj[MK_T];        // centre-of-mass approximation: the j-tile's eligible components
    int32_t tiles[MK_CHUNK_MAX];
    int32_t apart[MK_CHUNK_MAX];  // 1: no label of the j-tile is one of the i-tile's
    int32_t ntiles;
    uint64_t bar[2];
};

__device__ __forceinline__ void mk_issue(MixedKickSmem &sm, int st, const FFView &F, const int32_t *label,
                                         int j0, int jn)
{
    const unsigned cnt = (unsigned)((jn + 3) & ~3);
    fence_proxy_async_smem();
    mbar_expect_tx(&sm.bar[st], (unsigned)jn * 32u + cnt * 4u);
    tma_load_1d(sm.pq[st], F.pq + 2 * (size_t)j0, (unsigned)jn * 32u, &sm.bar[st]);
    tma_load_1d(sm.lab[st], label + j0, cnt * 4u, &sm.bar[st]);
}

// Block = MK_T threads = (MK_T / S rows of the i-tile) x (S column slices of
// each j-tile); the S partial sums of a row are combined in slice order.
// COM: pairs of two far components (ComView, the centre-of-mass
// approximation) are left out, as in the FP64 kick.
template <int S, bool COM>
__global__ void __launch_bounds__(MK_T) k_kick_mixed(Level L, FFView F, const int32_t *order, const int32_t *koff,
                                                      int chunk, float eps2, double h, DevCounters *ctr,
                                                      double *partial, ComView cv)
{
    constexpr int R = MK_T / S;  // i rows per block
    static_assert(R % 32 == 0, "one slice per warp");
    __shared__ MixedKickSmem sm;
    __shared__ double red[S > 1 ? S : 1][3][R];
    const int tid = threadIdx.x, row = tid % R, slice = tid / R;
    int lo = 0, hi = L.nsets;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (koff[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
    }
    const int s = lo;
    const int b = blockIdx.x - koff[s];
    const int n = L.set_n[s], start = L.set_start[s];
    const int ntile = (n + MK_T - 1) / MK_T;
    const int nchunk = (ntile + chunk - 1) / chunk;
    const int ti = b / nchunk, ch = b % nchunk;
    const int tj0 = ch * chunk, tj1 = min(ntile, tj0 + chunk);
    const int il = ti * R + row;
    const bool iv = il < n;
    const int t = start + il;  // position in the sorted order
    const int32_t *label = L.klab;
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
        // tiles with at least one cross-component pair
        const int ia = start + ti * R, ib = start + min(n, (ti + 1) * R) - 1;
        const bool iu = label[ia] == label[ib];
        int q = 0;
        for (int tj = tj0; tj < tj1; ++tj) {
            const int ja = start + tj * MK_T, jb = start + min(n, (tj + 1) * MK_T) - 1;
            if (iu && label[ja] == label[jb] && label[ja] == label[ia]) continue;
            // labels ascend within a set: disjoint ranges share no component
            sm.apart[q] = (label[jb] < label[ia] || label[ib] < label[ja]) ? 1 : 0;
            sm.tiles[q++] = tj;
        }
        sm.ntiles = q;
    }
    __syncthreads();
    const int nt = sm.ntiles;
    if (tid == 0 && nt > 0) mk_issue(sm, 0, F, label, start + sm.tiles[0] * MK_T, min(MK_T, n - sm.tiles[0] * MK_T));
    float4 ip0 = make_float4(0, 0, 0, 0), ip1 = ip0;
    int li = 0, ci = -1;
    if (iv) {
        ip0 = F.pq[2 * t];
        ip1 = F.pq[2 * t + 1];
        li = label[t];
        if constexpr (COM) ci = cv.cl[order[t]];
    }
    long long fo = 0;
    int Ks = 0;
    bool iany = false;
    if constexpr (COM) {
        fo = cv.foff[s];
        Ks = cv.K[s];
        iany = __syncthreads_or(ci >= 0) != 0;
    }
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    bool ok = true;
    for (int q = 0; q < nt; ++q) {
        const int tj = sm.tiles[q], st = q & 1;
        if (tid == 0 && q + 1 < nt) {
            const int tn = sm.tiles[q + 1];
            mk_issue(sm, st ^ 1, F, label, start + tn * MK_T, min(MK_T, n - tn * MK_T));
        }
        const bool got = mbar_wait(&sm.bar[st], (q >> 1) & 1, TMA_WAIT_CYCLES);
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        const int jn = min(MK_T, n - tj * MK_T);
        bool fchk = false;  // far pairs possible in this tile
        if constexpr (COM) {
            int c = -1;
            if (tid < jn) c = cv.cl[order[start + tj * MK_T + tid]];
            sm.cj[tid] = c;
            fchk = (__syncthreads_or(c >= 0) != 0) && iany;
        }
        if (iv) {
            // g += G m_j r^-3 (x_j - x_i) over groups of MK_GROUP j in plain
            // FP32 (fused), each group sum then added to the compensated
            // total: the per-term roundings dominate the error either way,
            // and the compensation costs 4 operations per component
            float gx, gy, gz;
            auto term = [&](int k, bool check) {
                const float4 jp0 = sm.pq[st][2 * k], jp1 = sm.pq[st][2 * k + 1];
                const float dx = (jp0.x - ip0.x) + (jp1.x - ip1.x);
                const float dy = (jp0.y - ip0.y) + (jp1.y - ip1.y);
                const float dz = (jp0.z - ip0.z) + (jp1.z - ip1.z);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
                float ri = rsqrtf(r2);
                ri = ri * fmaf(-0.5f * r2, ri * ri, 1.5f);  // one Newton step
                float w = jp0.w * (ri * ri * ri);            // G m_j / r^3
                if (check && sm.lab[st][k] == li) w = 0.f;  // same component (and self)
                if constexpr (COM) {
                    const int c = sm.cj[k];
                    if (fchk && ci >= 0 && c >= 0 && cv.far[fo + (long long)ci * Ks + c]) w = 0.f;
                }
                gx = fmaf(w, dx, gx);
                gy = fmaf(w, dy, gy);
                gz = fmaf(w, dz, gz);
            };
            auto flush = [&]() {
                kahan_add(sx, cx, gx);
                kahan_add(sy, cy, gy);
                kahan_add(sz, cz, gz);
            };
            auto run = [&](bool check) {
                int k = slice * (MK_T / S);
                const int k1 = min(jn, k + MK_T / S);
                for (; k + MK_GROUP <= k1; k += MK_GROUP) {
                    gx = gy = gz = 0.f;
#pragma unroll
                    for (int u = 0; u < MK_GROUP; ++u) term(k + u, check);
                    flush();
                }
                if (k < k1) {
                    gx = gy = gz = 0.f;
                    for (; k < k1; ++k) term(k, check);
                    flush();
                }
            };
            if (sm.apart[q]) run(false);
            else run(true);
        }
        __syncthreads();
    }
    if (!ok) {
        raise_err(ctr, DERR_TMA_TIMEOUT);
        mbar_wait(&sm.bar[0], 0, TMA_WAIT_CYCLES);
        mbar_wait(&sm.bar[1], 0, TMA_WAIT_CYCLES);
        return;
    }
    double ax = (double)sx - (double)cx, ay = (double)sy - (double)cy, az = (double)sz - (double)cz;
    if constexpr (S > 1) {
        red[slice][0][row] = ax;
        red[slice][1][row] = ay;
        red[slice][2][row] = az;
        __syncthreads();
        if (slice != 0) return;
        for (int q = 1; q < S; ++q) {
            ax += red[q][0][row];
            ay += red[q][1][row];
            az += red[q][2][row];
        }
    }
    if (!iv) return;
    if (nchunk == 1) {
        const int k = order[t];
        L.vx[k] += h * ax;
        L.vy[k] += h * ay;
        L.vz[k] += h * az;
    } else {
        // partial[(chunk * 3 + c) * cap + t]
        const size_t cap = (size_t)F.cap;
        partial[((size_t)ch * 3 + 0) * cap + t] = ax;
        partial[((size_t)ch * 3 + 1) * cap + t] = ay;
        partial[((size_t)ch * 3 + 2) * cap + t] = az;
    }
}

// Sum the chunk partials of multi-chunk sets (FP64), v += h a.  KR_LANES
// lanes per body: lane s sums chunks s, s + KR_LANES, ... in order, then a
// fixed butterfly combines the lanes, so the rounding order is fixed (run to
// run identical) and the dependent FP64 chain is nchunk/KR_LANES + 3 adds
// long instead of nchunk (an FP64 add's latency dominates this kernel).
constexpr int KR_LANES = 8;

__global__ void k_kick_reduce(Level L, FFView F, const int32_t *order, int chunk, double h, const double *partial,
                              const int32_t *root, double drift_dt)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = (int)(g / KR_LANES), sub = (int)(g % KR_LANES);
    int k = -1, nchunk = 1;
    if (t < L.total) {
        k = order[t];
        if (L.sidx[k] >= 0) {
            const int n = L.set_n[L.sidx[k]];
            nchunk = ((n + MK_T - 1) / MK_T + chunk - 1) / chunk;
        }
    }
    const bool on = k >= 0 && L.sidx[k] >= 0 && nchunk > 1;
    const size_t cap = (size_t)F.cap;
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (on) {
        for (int c = sub; c < nchunk; c += KR_LANES) {
            ax += partial[((size_t)c * 3 + 0) * cap + t];
            ay += partial[((size_t)c * 3 + 1) * cap + t];
            az += partial[((size_t)c * 3 + 2) * cap + t];
        }
    }
#pragma unroll
    for (int o = KR_LANES / 2; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (on && sub == 0) {
        L.vx[k] += h * ax;
        L.vy[k] += h * ay;
        L.vz[k] += h * az;
    }
    // drift_dt > 0: the level's second drift of rest-set members, after their
    // kick (the kick kernels read the float-float copy, never x)
    if (drift_dt > 0.0 && sub == 0 && k >= 0 && L.gid[k] >= 0 && L.cnt[root[k]] == 1) {
        L.x[k] = __dadd_rn(L.x[k], __dmul_rn(drift_dt, L.vx[k]));
        L.y[k] = __dadd_rn(L.y[k], __dmul_rn(drift_dt, L.vy[k]));
        L.z[k] = __dadd_rn(L.z[k], __dmul_rn(drift_dt, L.vz[k]));
    }
}

int mixed_kick_blocks(int n, int chunk, int slices)
{
    const int ntile = (n + MK_T - 1) / MK_T, rows = MK_T / slices;
    return ((n + rows - 1) / rows) * ((ntile + chunk - 1) / chunk);
}

int mixed_kick_chunks(int n, int chunk)
{
    const int ntile = (n + MK_T - 1) / MK_T;
    return (ntile + chunk - 1) / chunk;
}

void launch_kick_mixed(const Level &L, const FFView &F, const int32_t *order, const int32_t *koff, int nblocks,
                       int chunk, int slices, bool multi_chunk, double eps2, double h, DevCounters *ctr,
                       double *partial, const int32_t *root, double drift_dt, cudaStream_t s, const ComView *com)
{
    if (nblocks > 0) {
        const ComView cv = com ? *com : ComView{nullptr, nullptr, nullptr, nullptr};
        const float e2 = (float)eps2;
        if (com) {
            if (slices == 4)
                k_kick_mixed<4, true><<<nblocks, MK_T, 0, s>>>(L, F, order, koff, chunk, e2, h, ctr, partial, cv);
            else
                k_kick_mixed<1, true><<<nblocks, MK_T, 0, s>>>(L, F, order, koff, chunk, e2, h, ctr, partial, cv);
        } else {
            if (slices == 4)
                k_kick_mixed<4, false><<<nblocks, MK_T, 0, s>>>(L, F, order, koff, chunk, e2, h, ctr, partial, cv);
            else
                k_kick_mixed<1, false><<<nblocks, MK_T, 0, s>>>(L, F, order, koff, chunk, e2, h, ctr, partial, cv);
        }
        CC_COUNT_LAUNCH(1);
    }
    if ((multi_chunk && nblocks > 0) || (drift_dt > 0.0 && L.total > 0)) {
        const long long threads = (long long)L.total * KR_LANES;
        k_kick_reduce<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(L, F, order, multi_chunk ? chunk : 1 << 30, h,
                                                                        partial, root, drift_dt);
        CC_COUNT_LAUNCH(1);
    }
}

}  // namespace cc
