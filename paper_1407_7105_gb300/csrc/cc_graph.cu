// cc_graph.cu -- graph and data-movement kernels of the CC split
// (arXiv:1407.7105 Sec. 2.2-2.3):
//   * union-find compression: root[k] = smallest packed index of k's
//     component, sizes by root;
//   * segmentation: a stable sort of component members by root, so every
//     non-trivial component C_i is a contiguous run of ascending members
//     (the paper's particle reshuffle into start/end ranges, Sec. 2.3);
//   * gathering components into the next level's packed buffer and back;
//   * the drift D_{h,T_i} of Eq. (drift) for rest-set members.
// Scans and the radix sort are written here (no library kernels).
#include "cc_internal.cuh"

namespace cc {

// ------------------------------------------------------------ scan
constexpr int SCAN_T = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int block_exclusive_scan(int v, int *tmp, int &total)
{
    // tmp: SCAN_T/32 ints
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < (int)(blockDim.x >> 5)) tmp[lane] = t;
    }
    __syncthreads();
    total = tmp[(blockDim.x >> 5) - 1];
    int base = w > 0 ? tmp[w - 1] : 0;
    __syncthreads();
    return base + x - v;
}

// out[k] = sum of in[0..k); block sums to bsum
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int *in, int *out, int n, int *bsum)
{
    __shared__ int tmp[SCAN_T / 32];
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int ex = block_exclusive_scan(s, tmp, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// single block: exclusive scan of bsum[0..nb) in place, chunked
__global__ void __launch_bounds__(SCAN_T) k_scan_sums(int *bsum, int nb, int *grand)
{
    __shared__ int tmp[SCAN_T / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nb; c0 += SCAN_T) {
        const int k = c0 + threadIdx.x;
        int v = k < nb ? bsum[k] : 0, total;
        int ex = block_exclusive_scan(v, tmp, total);
        if (k < nb) bsum[k] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0 && grand) *grand = carry;
}

__global__ void k_scan_add(int *out, int n, const int *bsum)
{
    const int k = blockIdx.x * SCAN_TILE + threadIdx.x;
    const int add = bsum[blockIdx.x];
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        const int idx = k + q * SCAN_T;
        if (idx < n && idx < (int)(blockIdx.x + 1) * SCAN_TILE) out[idx] += add;
    }
}

static int scan_blocks(int n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

// exclusive scan of n ints; scratch needs scan_blocks(n) ints; *grand = total
static void device_scan(const int *in, int *out, int n, int *bsum, int *grand, cudaStream_t s)
{
    if (n <= 0) return;
    const int nb = scan_blocks(n);
    k_scan_tiles<<<nb, SCAN_T, 0, s>>>(in, out, n, bsum);
    CC_COUNT_LAUNCH(1);
    k_scan_sums<<<1, SCAN_T, 0, s>>>(bsum, nb, grand);
    CC_COUNT_LAUNCH(1);
    if (nb > 1) {
        k_scan_add<<<nb, SCAN_T, 0, s>>>(out, n, bsum);
        CC_COUNT_LAUNCH(1);
    }
}

int scan_scratch_ints(int n) { return scan_blocks(n) + 1; }

void launch_exclusive_scan(const int *in, int *out, int n, int *scratch, cudaStream_t s)
{
    device_scan(in, out, n, scratch, nullptr, s);
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort of (key, val) pairs, 8-bit digits.  Per pass:
// per-tile digit histograms, one exclusive scan over [digit][tile], and a
// stable scatter whose in-tile ranks come from warp match + per-warp
// digit counts combined in warp order.
constexpr int RS_T = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_T * RS_ROUNDS;

__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint32_t *keys, int n, int shift, int *hist, int ntiles)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int b = blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int i = b + r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint32_t *kin, const int32_t *vin, uint32_t *kout,
                                                      int32_t *vout, int n, int shift, const int *offs,
                                                      int ntiles)
{
    __shared__ int base[256];
    __shared__ int wc[RS_T / 32][257];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    base[threadIdx.x] = offs[threadIdx.x * ntiles + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        for (int q = threadIdx.x; q < (RS_T / 32) * 257; q += RS_T) (&wc[0][0])[q] = 0;
        __syncthreads();
        const int i = blockIdx.x * RS_TILE + r * RS_T + threadIdx.x;
        const bool valid = i < n;
        uint32_t key = 0;
        int32_t val = 0;
        int d = 256;
        if (valid) {
            key = kin[i];
            val = vin[i];
            d = (key >> shift) & 255u;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wc[w][d] = __popc(peers);
        __syncthreads();
        int run = 0;
        for (int ww = 0; ww < RS_T / 32; ++ww) {
            const int c = wc[ww][threadIdx.x];
            wc[ww][threadIdx.x] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            const int pos = base[d] + wc[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        base[threadIdx.x] += run;
        __syncthreads();
    }
}

static int rs_tiles(long long n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

size_t sort_scratch_bytes(long long n)
{
    const long long nt = rs_tiles(n);
    const long long hist = 256 * nt;
    return (size_t)(4 * n + hist + scan_blocks((int)hist) + 16) * 4 + 256;
}

// sorts (k, v) in place by the low `bits` bits of k; scratch >= sort_scratch_bytes(n)
static void radix_sort(uint32_t *k, int32_t *v, int n, int bits, void *scratch, cudaStream_t s)
{
    if (n <= 1 || bits <= 0) return;
    const int nt = rs_tiles(n);
    uint32_t *k2 = (uint32_t *)scratch;
    int32_t *v2 = (int32_t *)(k2 + n);
    int *hist = (int *)(v2 + n);
    int *bsum = hist + 256 * nt;
    uint32_t *ka = k, *kb = k2;
    int32_t *va = v, *vb = v2;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<nt, RS_T, 0, s>>>(ka, n, shift, hist, nt);
        CC_COUNT_LAUNCH(1);
        device_scan(hist, hist, 256 * nt, bsum, nullptr, s);
        k_rs_scatter<<<nt, RS_T, 0, s>>>(ka, va, kb, vb, n, shift, hist, nt);
        CC_COUNT_LAUNCH(1);
        uint32_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != k) {
        cudaMemcpyAsync(k, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(v, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
}

static int bits_for(long long maxval)
{
    int b = 0;
    while (b < 32 && (1ll << b) <= maxval) ++b;
    return b;
}

// ------------------------------------------------------------ compress
// root of every element (the forest is final: finds read through L1, since
// thousands of them end on one root) and component sizes by root, with one
// atomic per distinct root in each warp (members of a giant component would
// otherwise queue on one counter)
__global__ void k_compress(Level L, int32_t *root)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = k < L.total;
    const bool valid = in && L.gid[k] >= 0;
    const int r = valid ? uf_find_ca(L.parent, k) : (in ? k : -1);
    if (in) root[k] = r;
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? r : -2 - (int)(threadIdx.x & 31));
    if (valid && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&L.cnt[r], __popc(peers));
}

void launch_compress(const Level &L, int32_t *root, cudaStream_t s)
{
    if (L.total <= 0) return;
    k_compress<<<(L.total + 255) / 256, 256, 0, s>>>(L, root);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ segment
// The order produced here ("members") is every packed element stably sorted
// by root (padding keyed by its own index): each set keeps its range, each
// component is a contiguous run of ascending members, and rest-set members
// sit between runs in ascending order.  comp_start indexes this order.
__global__ void k_seg_keys(Level L, const int32_t *root, uint32_t *key, int32_t *val)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.total) return;
    key[k] = L.gid[k] >= 0 ? (uint32_t)root[k] : (uint32_t)k;
    val[k] = k;
}

__global__ void k_seg_heads(Level L, const uint32_t *key, int n, int *flag)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    flag[t] = L.cnt[key[t]] >= 2 && (t == 0 || key[t] != key[t - 1]) ? 1 : 0;
}

__global__ void k_seg_bounds(Level L, const uint32_t *key, const int32_t *val, const int *flag, const int *cidx,
                             int n, int32_t *members, int32_t *comp_start, int32_t *comp_size, int32_t *ncomp)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    members[t] = val[t];
    if (flag[t]) {
        comp_start[cidx[t]] = t;
        comp_size[cidx[t]] = L.cnt[key[t]];
    }
    if (t == n - 1) *ncomp = cidx[t] + flag[t];
}

size_t seg_scratch_bytes(int cap)
{
    return (size_t)cap * 4 * 4 + sort_scratch_bytes(cap) + (size_t)(scan_blocks(cap) + 16) * 4 + 1024;
}

void launch_segment(const Level &L, const int32_t *root, int32_t *members, int32_t *comp_start,
                    int32_t *comp_size, int32_t *d_ncomp, void *scratch, cudaStream_t s)
{
    const int n = L.total;
    if (n <= 0) {
        cudaMemsetAsync(d_ncomp, 0, sizeof(int32_t), s);
        return;
    }
    uint32_t *key = (uint32_t *)scratch;
    int32_t *val = (int32_t *)(key + n);
    int *flag = (int *)(val + n);
    int *cidx = flag + n;
    int *bsum = cidx + n;
    void *sort_scratch = (void *)(bsum + scan_blocks(n) + 16);
    const int g = (n + 255) / 256;
    k_seg_keys<<<g, 256, 0, s>>>(L, root, key, val);
    CC_COUNT_LAUNCH(1);
    radix_sort(key, val, n, bits_for(n), sort_scratch, s);
    k_seg_heads<<<g, 256, 0, s>>>(L, key, n, flag);
    CC_COUNT_LAUNCH(1);
    device_scan(flag, cidx, n, bsum, nullptr, s);
    k_seg_bounds<<<g, 256, 0, s>>>(L, key, val, flag, cidx, n, members, comp_start, comp_size, d_ncomp);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ one-CTA path
// For a batch of at most SEG1_MAX packed elements one CTA does what the
// general path spreads over ~15 launches: union-find compression, sizes,
// run starts and component offsets (block scans over contiguous chunks),
// and the ordered scatter of members.  Order within a run must be index
// order (the input order): runs of at most SEG1_RUN members are scattered
// by shared-memory cursors and then sorted by index (one thread per run of at
// most SEG1_THR by insertion, one warp per longer run by counting ranks); each larger run (up to SEG1_BIG of them; the giant
// component of a dense cluster is one) is written by a stable compaction,
// a block scan of "key == its root" over the batch.  More large runs than
// that send the block to a stable single-warp scatter (one warp walks the
// indices in order; lanes with the same root are ranked by warp match).
// Shared memory: 8 bytes per element (dynamic).
constexpr int SEG1_T = 1024;
constexpr int SEG1_MAX = 16384;
constexpr int SEG1_RUN = 64;
constexpr int SEG1_THR = 16;  // runs up to this size are sorted by one thread
constexpr int SEG1_BIG = 8;

// Each warp owns the contiguous range [32 per w, 32 per (w + 1)) of the
// batch and walks it in rounds of 32 consecutive elements (lane = offset in
// the round), so shared-memory accesses and global writes are unit-stride.
// seg1_warp_base: the sum of v over the warp's lanes, exclusively scanned
// over the warps in order (the warp's base); *total = the block's sum.
// tmp: SEG1_T / 32 + 1 ints.
__device__ __forceinline__ int seg1_warp_base(int v, int *tmp, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) tmp[w] = v;
    __syncthreads();
    if (w == 0) {
        const int x = lane < (int)(blockDim.x >> 5) ? tmp[lane] : 0;
        int y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (lane < (int)(blockDim.x >> 5)) tmp[lane] = y - x;
        if (lane == 31) tmp[32] = y;
    }
    __syncthreads();
    const int base = tmp[w];
    *total = tmp[32];
    __syncthreads();
    return base;
}

// inclusive scan of v over the warp's lanes
__device__ __forceinline__ int warp_inclusive_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int z = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += z;
    }
    return v;
}

// The classification of a split's components (see k_classify below) by the
// CTA that segmented them; sh: CLS_SH ints of shared memory
__device__ void classify_components(const int32_t *comp_size, int nc, const ClassifyArgs &C, int *sh)
{
    int *s_cnt = sh, *s_pos = sh + CLS_NB, *s_nk = sh + 2 * CLS_NB, *s_solo = sh + 2 * CLS_NB + 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int z = tid; z < CLS_NB; z += nt) s_cnt[z] = 0;
    if (tid == 0) {
        *s_nk = 0;
        *s_solo = 0;
    }
    __syncthreads();
    // the components above BATCH_SOLO bodies that the batched kernel could take
    for (int q = tid; q < nc; q += nt) {
        const int sz = comp_size[q];
        if (sz > BATCH_SOLO && sz <= C.s_small) atomicAdd(s_solo, 1);
    }
    __syncthreads();
    const int smax = batch_limit(C.s_small, *s_solo);
    for (int q = tid; q < nc; q += nt) {
        const int sz = comp_size[q];
        if (C.kepler && sz == 2) C.klist[atomicAdd(s_nk, 1)] = q;
        else if (sz <= smax) atomicAdd(&s_cnt[size_bucket(sz)], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int pos = 0;
        for (int z = size_bucket(smax < 0 ? 0 : smax); z >= 0; --z) {
            s_pos[z] = pos;
            pos += s_cnt[z];
        }
        C.counts[0] = *s_nk;
        C.counts[1] = pos;
        C.queue[0] = 0;
        C.queue[1] = 0;
    }
    __syncthreads();
    for (int q = tid; q < nc; q += nt) {
        const int sz = comp_size[q];
        if (!(C.kepler && sz == 2) && sz <= smax) C.slist[atomicAdd(&s_pos[size_bucket(sz)], 1)] = q;
    }
}

// find with path halving in the shared-memory forest (links point to
// smaller indices)
__device__ __forceinline__ int seg1_find(volatile int *p, int x)
{
    while (true) {
        const int q = p[x];
        if (q == x) return x;
        const int g = p[q];
        if (g != q) p[x] = g;
        x = q;
    }
}

// union by compare-and-swap in the shared-memory forest (the larger root
// under the smaller)
__device__ __forceinline__ bool seg1_union(int *p, int a, int b)
{
    volatile int *vp = p;
    for (int it = 0; it < (1 << 20); ++it) {
        a = seg1_find(vp, a);
        b = seg1_find(vp, b);
        if (a == b) return true;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(&p[b], b, a) == b) return true;
    }
    return false;
}

__global__ void __launch_bounds__(SEG1_T) k_segment_small(Level L, int32_t *root_out, int32_t *members,
                                                          int32_t *comp_start, int32_t *comp_size, int32_t *ncomp,
                                                          EdgeList hook, DevCounters *ctr, ClassifyArgs cls)
{
    extern __shared__ int seg1_smem[];
    const int n = L.total, tid = threadIdx.x;
    int *s_root = seg1_smem;      // roots (-1: padding), then the member list being built
    int *s_cnt = seg1_smem + n;   // size by root, then run start / cursor by key
    __shared__ int tmp[SEG1_T / 32 + 1];
    __shared__ int s_nbig, s_big_root[SEG1_BIG], s_big_start[SEG1_BIG], s_big_size[SEG1_BIG];
    // warp ranges walked in rounds of 32 (seg1_warp_base)
    const int per = (n + SEG1_T - 1) / SEG1_T;
    const int lane = tid & 31, wid = tid >> 5, wb = 32 * per * wid;
    const unsigned lt = (1u << lane) - 1u;
    if (tid == 0) s_nbig = 0;
    // the level's forest into shared memory (padding: its own root), then
    // the first half's child edges when given (hooked here rather than in
    // global memory, where thousands of finds of one giant component queue
    // on its root's line), then every root by finds in shared memory
    for (int k = tid; k < n; k += SEG1_T) s_root[k] = L.gid[k] >= 0 ? L.parent[k] : k;
    __syncthreads();
    if (hook.rec) {
        const long long ne = (long long)min(*hook.count, (unsigned long long)hook.cap);
        for (long long t = tid; t < ne; t += SEG1_T) {
            const EdgeRec r = hook.rec[t];
            if (!seg1_union(s_root, r.a, r.b)) raise_err(ctr, DERR_UF_RETRY);
        }
        __syncthreads();
    }
    for (int k = tid; k < n; k += SEG1_T) s_cnt[k] = seg1_find(s_root, k);  // roots, parked in s_cnt
    __syncthreads();
    for (int k = tid; k < n; k += SEG1_T) {
        const int r = s_cnt[k];
        s_root[k] = L.gid[k] >= 0 ? r : -1;
        root_out[k] = r;
        s_cnt[k] = 0;
    }
    __syncthreads();
    for (int k = tid; k < n; k += SEG1_T)
        if (s_root[k] >= 0) atomicAdd(&s_cnt[s_root[k]], 1);
    __syncthreads();
    for (int k = tid; k < n; k += SEG1_T) L.cnt[k] = s_cnt[k];
    // run of key k: w = elements keyed k (key = root for valid elements, own
    // index for padding); a component head has w >= 2
    auto weight = [&](int k) {
        const int r = s_root[k];
        return r < 0 ? 1 : (r == k ? s_cnt[k] : 0);
    };
    int sw = 0, sc = 0;
    for (int j = 0; j < per; ++j) {
        const int k = wb + 32 * j + lane;
        if (k < n) {
            const int w = weight(k);
            sw += w;
            sc += (s_root[k] >= 0 && w >= 2) ? 1 : 0;
        }
    }
    int tot_w, tot_c;
    int ew = seg1_warp_base(sw, tmp, &tot_w);
    int ec = seg1_warp_base(sc, tmp, &tot_c);
    // (an element reads its own weight before writing its own cursor: a key's
    // cursor lives at the key's own index)
    for (int j = 0; j < per; ++j) {
        const int k = wb + 32 * j + lane;
        const bool in = k < n;
        const int w = in ? weight(k) : 0;
        const bool head = in && s_root[k] >= 0 && w >= 2;
        const int x = warp_inclusive_scan(w);
        const unsigned hb = __ballot_sync(0xffffffffu, head);
        const int my_w = ew + x - w, my_c = ec + __popc(hb & lt);
        if (head) {
            comp_start[my_c] = my_w;
            comp_size[my_c] = w;
            if (w > SEG1_RUN) {
                const int b = atomicAdd(&s_nbig, 1);
                if (b < SEG1_BIG) {
                    s_big_root[b] = k;
                    s_big_start[b] = my_w;
                    s_big_size[b] = w;
                }
            }
        }
        if (in) s_cnt[k] = my_w;  // run start of key k (cursor)
        ew += __shfl_sync(0xffffffffu, x, 31);
        ec += __popc(hb);
    }
    if (tid == 0) *ncomp = tot_c;
    __syncthreads();
    const int nbig = s_nbig;
    if (nbig <= SEG1_BIG) {
        // keys of the thread's strided elements, read before s_root turns
        // into the member list
        auto key_of = [&](int k) { return s_root[k] >= 0 ? s_root[k] : k; };
        auto is_big = [&](int key) { return s_root[key] == key && L.cnt[key] > SEG1_RUN; };
        // large runs first: stable compaction per run (reads s_root only)
        for (int b = 0; b < nbig; ++b) {
            const int rb = s_big_root[b];
            int cnt = 0;
            for (int j = 0; j < per; ++j) {
                const int k = wb + 32 * j + lane;
                cnt += (k < n && s_root[k] == rb) ? 1 : 0;
            }
            int tot;
            int pos = s_big_start[b] + seg1_warp_base(cnt, tmp, &tot);
            for (int j = 0; j < per; ++j) {
                const int k = wb + 32 * j + lane;
                const bool hit = k < n && s_root[k] == rb;
                const unsigned hb = __ballot_sync(0xffffffffu, hit);
                if (hit) members[pos + __popc(hb & lt)] = k;
                pos += __popc(hb);
            }
            __syncthreads();
        }
        // small runs: unordered scatter into shared memory
        int kk[SEG1_MAX / SEG1_T];
#pragma unroll
        for (int q = 0; q < SEG1_MAX / SEG1_T; ++q) {
            const int k = tid + q * SEG1_T;
            kk[q] = (k < n && !is_big(key_of(k))) ? key_of(k) : -1;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < SEG1_MAX / SEG1_T; ++q) {
            const int k = tid + q * SEG1_T;
            if (kk[q] >= 0) s_root[atomicAdd(&s_cnt[kk[q]], 1)] = k;
        }
        __syncthreads();
        // runs of at most SEG1_THR members: one thread each, insertion sort
        for (int c = tid; c < tot_c; c += SEG1_T) {
            const int st = comp_start[c], sz = comp_size[c];
            if (sz > SEG1_THR) continue;
            for (int a = 1; a < sz; ++a) {
                const int x = s_root[st + a];
                int b = a - 1;
                while (b >= 0 && s_root[st + b] > x) {
                    s_root[st + b + 1] = s_root[st + b];
                    --b;
                }
                s_root[st + b + 1] = x;
            }
        }
        // longer runs (up to SEG1_RUN): one warp each, ranks by counting
        for (int c = wid; c < tot_c; c += SEG1_T / 32) {
            const int st = comp_start[c], sz = comp_size[c];
            if (sz <= SEG1_THR || sz > SEG1_RUN) continue;
            const int x0 = lane < sz ? s_root[st + lane] : 0x7fffffff;
            const int x1 = lane + 32 < sz ? s_root[st + lane + 32] : 0x7fffffff;
            int r0 = 0, r1 = 0;
            for (int j = 0; j < sz; ++j) {
                const int y = s_root[st + j];
                r0 += y < x0;
                r1 += y < x1;
            }
            __syncwarp();
            if (lane < sz) s_root[st + r0] = x0;
            if (lane + 32 < sz) s_root[st + r1] = x1;
            __syncwarp();
        }
        __syncthreads();
        // copy out everything but the large runs (already in place)
        for (int k = tid; k < n; k += SEG1_T) {
            bool in_big = false;
            for (int b = 0; b < nbig; ++b) in_big |= (k >= s_big_start[b] && k < s_big_start[b] + s_big_size[b]);
            if (!in_big) members[k] = s_root[k];
        }
    } else if (tid < 32) {
        for (int base = 0; base < n; base += 32) {
            const int k = base + tid;
            const bool in = k < n;
            const int key = in ? (s_root[k] >= 0 ? s_root[k] : k) : -1 - tid;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const int rank = __popc(peers & lt);
            const int lead = __ffs(peers) - 1;
            int pos = 0;
            if (in && rank == 0) {
                pos = s_cnt[key];
                s_cnt[key] += __popc(peers);
            }
            pos = __shfl_sync(0xffffffffu, pos, lead) + rank;
            if (in) members[pos] = k;
            __syncwarp();
        }
    }
    if (cls.queue) {
        // the components' integrator lists (comp_size is this CTA's own
        // writes: visible after the barrier)
        __shared__ int cls_sh[CLS_SH];
        __syncthreads();
        classify_components(comp_size, tot_c, cls, cls_sh);
    }
}

// one CTA hooks the edges of small batches only: a big first half's edge
// list (tens of thousands of edges, most into one giant component) hooks
// faster spread over the GPU (k_edges_hook) than in one CTA
constexpr int SEG1_HOOK_MAX = 4096;

bool segment_hooks_edges(int total) { return total > 0 && total <= SEG1_HOOK_MAX; }

bool launch_compress_segment(const Level &L, int32_t *root, int32_t *members, int32_t *comp_start,
                             int32_t *comp_size, int32_t *d_ncomp, void *scratch, cudaStream_t s,
                             const EdgeList *hook, DevCounters *ctr, const ClassifyArgs *cls)
{
    if (L.total > 0 && L.total <= SEG1_MAX) {
        // opt in to the dynamic shared memory once per device
        static bool attr_set[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            cudaFuncSetAttribute(k_segment_small, cudaFuncAttributeMaxDynamicSharedMemorySize, SEG1_MAX * 8);
            attr_set[dev] = true;
        }
        const EdgeList none{nullptr, nullptr, 0};
        ClassifyArgs nc{};
        if (cls) nc = *cls;
        k_segment_small<<<1, SEG1_T, (size_t)L.total * 8, s>>>(L, root, members, comp_start, comp_size, d_ncomp,
                                                               hook ? *hook : none, ctr, nc);
        CC_COUNT_LAUNCH(1);
        return cls != nullptr;
    }
    launch_compress(L, root, s);
    launch_segment(L, root, members, comp_start, comp_size, d_ncomp, scratch, s);
    return false;
}

// ------------------------------------------------------------ HOLD merge
// The HOLD split's fast set F = {i : tau(i) < h}, tau(i) = min over the set
// of tau(i,j), is the set of members with at least one edge at h: the union
// of the set's non-trivial CC components.  After the edges are hooked, every
// non-trivial root of a set is linked under the smallest of them (links go
// from larger to smaller indices, so the forest stays valid while finds run).
__global__ void k_hold_init(int32_t *anchor, int nsets)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nsets) anchor[k] = 0x7fffffff;
}

__global__ void k_hold_min(Level L, int32_t *anchor)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.total) return;
    const int s = L.sidx[k];
    if (s < 0) return;  // padding
    const int r = uf_find(L.parent, k);
    if (r != k) atomicMin(&anchor[s], r);  // k is a non-root member: r's component is non-trivial
}

__global__ void k_hold_link(Level L, const int32_t *anchor)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.total) return;
    const int s = L.sidx[k];
    if (s < 0) return;
    const int r = uf_find(L.parent, k);
    const int a = anchor[s];
    if (r != k && r != a) L.parent[r] = a;  // a <= r: every non-trivial root of the set
}

void launch_hold_merge(const Level &L, int32_t *anchor, cudaStream_t s)
{
    if (L.total <= 0 || L.nsets <= 0) return;
    k_hold_init<<<(L.nsets + 255) / 256, 256, 0, s>>>(anchor, L.nsets);
    const int g = (L.total + 255) / 256;
    k_hold_min<<<g, 256, 0, s>>>(L, anchor);
    k_hold_link<<<g, 256, 0, s>>>(L, anchor);
    CC_COUNT_LAUNCH(3);
}

// ------------------------------------------------------------ classification
// Sorts the components of a split for their integrators (one CTA, after the
// segmentation): two-body components go to klist when Kepler mode is on,
// components of at most s_small members to slist, largest first (a counting
// sort by size, in bins of 16 above 32 bodies; order within one bin is
// immaterial: components are independent), larger ones stay for the next
// level.  Writes counts[0] =
// nk, counts[1] = ns and zeroes the two work-queue counters of the small
// kernel (queue[0..1]), so the kernels that read them can be launched
// before the host learns the sizes.
constexpr int CLS_T = 1024;

__global__ void __launch_bounds__(CLS_T) k_classify(const int32_t *comp_size, const int32_t *ncomp, ClassifyArgs C)
{
    __shared__ int sh[CLS_SH];
    classify_components(comp_size, *ncomp, C, sh);
}

void launch_classify(const int32_t *comp_size, const int32_t *ncomp, int s_small, int kepler, int32_t *queue,
                     int32_t *counts, int32_t *klist, int32_t *slist, cudaStream_t s)
{
    const ClassifyArgs C{s_small < BATCH_NMAX ? s_small : BATCH_NMAX, kepler, queue, counts, klist, slist};
    k_classify<<<1, CLS_T, 0, s>>>(comp_size, ncomp, C);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ movement
__global__ void k_fill_pad(Level L)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.total) return;
    L.gid[k] = -1;
    L.sidx[k] = -1;
}

static void fill_pad(const Level &L, cudaStream_t s)
{
    if (L.total > 0) {
        k_fill_pad<<<(L.total + 255) / 256, 256, 0, s>>>(L);
        CC_COUNT_LAUNCH(1);
    }
}

__device__ __forceinline__ int upper_find(const int32_t *off, int nsets, int t)
{
    int lo = 0, hi = nsets;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// One thread per position of the child level: a member of large component
// c (child set c) copies its state from the parent, a padding slot is
// marked (gid = -1); inv[k] = the child index of parent element k (written
// for the gathered elements only; a reader checks C.src[inv[k]] == k)
__global__ void k_gather(Level P, Level C, const int32_t *members, const int32_t *lcomp_start, int32_t *inv)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= C.total) return;
    const int c = upper_find(C.set_start, C.nsets, d);
    const int w = d - C.set_start[c];
    if (w >= C.set_n[c]) {
        C.gid[d] = -1;
        C.sidx[d] = -1;
        return;
    }
    const int k = members[lcomp_start[c] + w];
    C.x[d] = P.x[k]; C.y[d] = P.y[k]; C.z[d] = P.z[k];
    C.vx[d] = P.vx[k]; C.vy[d] = P.vy[k]; C.vz[d] = P.vz[k];
    C.m[d] = P.m[k];
    C.gid[d] = P.gid[k];
    C.src[d] = k;
    C.sidx[d] = c;
    inv[k] = d;
}

void launch_gather(const Level &P, const Level &C, const int32_t *members, const int32_t *lcomp_start, int32_t *inv,
                   cudaStream_t s)
{
    if (C.total > 0) {
        k_gather<<<(C.total + 255) / 256, 256, 0, s>>>(P, C, members, lcomp_start, inv);
        CC_COUNT_LAUNCH(1);
    }
}

__global__ void k_scatter(Level P, Level C)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= C.total || C.gid[d] < 0) return;
    const int k = C.src[d];
    P.x[k] = C.x[d]; P.y[k] = C.y[d]; P.z[k] = C.z[d];
    P.vx[k] = C.vx[d]; P.vy[k] = C.vy[d]; P.vz[k] = C.vz[d];
}

void launch_scatter(const Level &P, const Level &C, cudaStream_t s)
{
    if (C.total > 0) {
        k_scatter<<<(C.total + 255) / 256, 256, 0, s>>>(P, C);
        CC_COUNT_LAUNCH(1);
    }
}

// state (id order) -> level 0, system q at set_start[q]; perm (one system
// only, may be null): the particle's offset in its set
__global__ void k_pack_state(const double *x3, const double *v3, const double *m, long long n, Level L,
                             const int32_t *sys_off, const int32_t *perm)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int q = upper_find(sys_off, L.nsets, (int)t);
    const int d = L.set_start[q] + (perm ? perm[t] : (int)(t - sys_off[q]));
    L.x[d] = x3[t]; L.y[d] = x3[n + t]; L.z[d] = x3[2 * n + t];
    L.vx[d] = v3[t]; L.vy[d] = v3[n + t]; L.vz[d] = v3[2 * n + t];
    L.m[d] = m[t];
    L.gid[d] = (int)t;
    L.src[d] = (int)t;
    L.sidx[d] = q;
}

void launch_pack_state(const double *x3, const double *v3, const double *m, long long n, const Level &L,
                       const int32_t *sys_off, const int32_t *perm, cudaStream_t s)
{
    fill_pad(L, s);
    if (n > 0) {
        k_pack_state<<<(int)((n + 255) / 256), 256, 0, s>>>(x3, v3, m, n, L, sys_off, perm);
        CC_COUNT_LAUNCH(1);
    }
}

__global__ void k_unpack_state(double *x3, double *v3, long long n, Level L)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= L.total) return;
    const int g = L.gid[d];
    if (g < 0) return;
    x3[g] = L.x[d]; x3[n + g] = L.y[d]; x3[2 * n + g] = L.z[d];
    v3[g] = L.vx[d]; v3[n + g] = L.vy[d]; v3[2 * n + g] = L.vz[d];
}

void launch_unpack_state(double *x3, double *v3, long long n, const Level &L, cudaStream_t s)
{
    if (L.total > 0) {
        k_unpack_state<<<(L.total + 255) / 256, 256, 0, s>>>(x3, v3, n, L);
        CC_COUNT_LAUNCH(1);
    }
}

// a caller set (ids, ascending) -> one packed set at 0; flags bad ids
__global__ void k_gather_set(const double *x3, const double *v3, const double *m, long long n,
                             const int32_t *set, int nset, Level L, unsigned *bad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nset) return;
    const int g = set[k];
    if (g < 0 || g >= n || (k > 0 && set[k - 1] >= g)) {
        atomicExch(bad, 1u);
        L.gid[k] = -1;
        return;
    }
    L.x[k] = x3[g]; L.y[k] = x3[n + g]; L.z[k] = x3[2 * n + g];
    L.vx[k] = v3[g]; L.vy[k] = v3[n + g]; L.vz[k] = v3[2 * n + g];
    L.m[k] = m[g];
    L.gid[k] = g;
    L.src[k] = g;
    L.sidx[k] = 0;
}

void launch_gather_set(const double *x3, const double *v3, const double *m, long long n, const int32_t *set,
                       int nset, const Level &L, unsigned *bad, cudaStream_t s)
{
    fill_pad(L, s);
    if (nset > 0) {
        k_gather_set<<<(nset + 255) / 256, 256, 0, s>>>(x3, v3, m, n, set, nset, L, bad);
        CC_COUNT_LAUNCH(1);
    }
}

__global__ void k_scatter_set(double *x3, double *v3, long long n, Level L, int nset, int wx, int wv)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nset) return;
    const int g = L.gid[k];
    if (g < 0) return;
    if (wx) { x3[g] = L.x[k]; x3[n + g] = L.y[k]; x3[2 * n + g] = L.z[k]; }
    if (wv) { v3[g] = L.vx[k]; v3[n + g] = L.vy[k]; v3[2 * n + g] = L.vz[k]; }
}

void launch_scatter_set(double *x3, double *v3, long long n, const Level &L, int nset, bool write_x,
                        bool write_v, cudaStream_t s)
{
    if (nset > 0) {
        k_scatter_set<<<(nset + 255) / 256, 256, 0, s>>>(x3, v3, n, L, nset, write_x, write_v);
        CC_COUNT_LAUNCH(1);
    }
}

// labels_out[k] = particle id of the root of k (the smallest id of its
// component, since the set is ascending)
__global__ void k_label_canon(Level L, const int32_t *root, int32_t *labels_out, int nset)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nset) return;
    labels_out[k] = L.gid[root[k]];
}

void launch_label_canon(const Level &L, const int32_t *root, int32_t *labels_out, int nset, cudaStream_t s)
{
    if (nset > 0) {
        k_label_canon<<<(nset + 255) / 256, 256, 0, s>>>(L, root, labels_out, nset);
        CC_COUNT_LAUNCH(1);
    }
}

// ------------------------------------------------------------ drift
// x_i += dt * v_i (Eq. drift) for rest-set members: component size 1
__global__ void k_drift_root(Level L, const int32_t *root, double dt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.total || L.gid[k] < 0 || L.cnt[root[k]] != 1) return;
    L.x[k] = __dadd_rn(L.x[k], __dmul_rn(dt, L.vx[k]));
    L.y[k] = __dadd_rn(L.y[k], __dmul_rn(dt, L.vy[k]));
    L.z[k] = __dadd_rn(L.z[k], __dmul_rn(dt, L.vz[k]));
}

void launch_drift(const Level &L, const int32_t *root, double dt, cudaStream_t s)
{
    if (L.total > 0) {
        k_drift_root<<<(L.total + 255) / 256, 256, 0, s>>>(L, root, dt);
        CC_COUNT_LAUNCH(1);
    }
}

__global__ void k_drift_flag(Level L, const int32_t *single, double dt, int nset)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nset || L.gid[k] < 0 || !single[k]) return;
    L.x[k] = __dadd_rn(L.x[k], __dmul_rn(dt, L.vx[k]));
    L.y[k] = __dadd_rn(L.y[k], __dmul_rn(dt, L.vy[k]));
    L.z[k] = __dadd_rn(L.z[k], __dmul_rn(dt, L.vz[k]));
}

void launch_drift_labels(const Level &L, const int32_t *singleton, double dt, cudaStream_t s)
{
    if (L.total > 0) {
        k_drift_flag<<<(L.total + 255) / 256, 256, 0, s>>>(L, singleton, dt, L.total);
        CC_COUNT_LAUNCH(1);
    }
}

// singleton[k] = 1 iff no other entry of labels[0..n) equals labels[k]
__global__ void k_lab_keys(const int32_t *labels, int n, uint32_t *key, int32_t *val)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    key[k] = (uint32_t)labels[k] ^ 0x80000000u;
    val[k] = k;
}

__global__ void k_lab_single(const uint32_t *key, const int32_t *val, int n, int32_t *single)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const bool a = t > 0 && key[t - 1] == key[t];
    const bool b = t + 1 < n && key[t + 1] == key[t];
    single[val[t]] = (a || b) ? 0 : 1;
}

void launch_singleton_from_labels(const int32_t *labels, int n, int32_t *singleton, void *scratch,
                                  cudaStream_t s)
{
    if (n <= 0) return;
    uint32_t *key = (uint32_t *)scratch;
    int32_t *val = (int32_t *)(key + n);
    void *ss = (void *)(val + n);
    k_lab_keys<<<(n + 255) / 256, 256, 0, s>>>(labels, n, key, val);
    CC_COUNT_LAUNCH(1);
    radix_sort(key, val, n, 32, ss, s);
    k_lab_single<<<(n + 255) / 256, 256, 0, s>>>(key, val, n, singleton);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ validation
// bad |= 1 if any value is non-finite; |= 2 if a mass is not > 0
__global__ void k_check_state(const double *m, const double *x3, const double *v3, long long n, unsigned *bad)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    unsigned b = 0;
    if (m && !(isfinite(m[k]) && m[k] > 0.0)) b |= 2u;
    if (x3 && !(isfinite(x3[k]) && isfinite(x3[n + k]) && isfinite(x3[2 * n + k]))) b |= 1u;
    if (v3 && !(isfinite(v3[k]) && isfinite(v3[n + k]) && isfinite(v3[2 * n + k]))) b |= 1u;
    if (b) atomicOr(bad, b);
}

void launch_check_state(const double *m, const double *x3, const double *v3, long long n, unsigned *bad,
                        cudaStream_t s)
{
    if (n > 0) {
        k_check_state<<<(int)((n + 255) / 256), 256, 0, s>>>(m, x3, v3, n, bad);
        CC_COUNT_LAUNCH(1);
    }
}

// order[0..n) = indices of labels[0..n) stably sorted by label;
// order[t] = t for the padding positions n <= t < total
__global__ void k_order_from_sorted(const int32_t *val, int n, int total, int32_t *order)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < total) order[t] = t < n ? val[t] : t;
}

void launch_label_order(const int32_t *labels, int n, int total, int32_t *order, void *scratch, cudaStream_t s)
{
    if (total <= 0) return;
    uint32_t *key = (uint32_t *)scratch;
    int32_t *val = (int32_t *)(key + n);
    void *ss = (void *)(val + n);
    if (n > 0) {
        k_lab_keys<<<(n + 255) / 256, 256, 0, s>>>(labels, n, key, val);
        CC_COUNT_LAUNCH(1);
        radix_sort(key, val, n, 32, ss, s);
    }
    k_order_from_sorted<<<(total + 255) / 256, 256, 0, s>>>(val, n, total, order);
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ spatial order
// A Morton (Z-order) ranking of the particles by position, 10 bits per
// axis over their bounding box: neighbours in the ranking are neighbours in
// space, so 32-body groups of a set in this order have small boxes (the
// group certificates of the mixed tau kernel).  Any permutation gives the
// same partitions; this one only decides which pairs share a group.
__device__ __forceinline__ unsigned ordered_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_ordered(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_pos_box(const double *x3, long long n, unsigned *box)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    if (t < n) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const unsigned o = ordered_bits((float)x3[k * n + t]);
            lo[k] = o;
            hi[k] = o;
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&box[k], lo[k]);
            atomicMax(&box[3 + k], hi[k]);
        }
    }
}

__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton_keys(const double *x3, long long n, const unsigned *box, uint32_t *key, int32_t *val)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t code = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = from_ordered(box[k]), hi = from_ordered(box[3 + k]);
        const float w = hi - lo;
        float f = w > 0.f ? ((float)x3[k * n + t] - lo) / w * 1023.f : 0.f;
        f = fminf(fmaxf(f, 0.f), 1023.f);
        code |= spread3((uint32_t)f) << k;
    }
    key[t] = code;
    val[t] = (int32_t)t;
}

__global__ void k_perm_from_sorted(const int32_t *val, long long n, int32_t *perm)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) perm[val[p]] = (int32_t)p;
}

void launch_spatial_order(const double *x3, long long n, int32_t *perm, unsigned *box, void *scratch,
                          cudaStream_t s)
{
    if (n <= 0) return;
    const int g = (int)((n + 255) / 256);
    cudaMemsetAsync(box, 0xff, 3 * sizeof(unsigned), s);
    cudaMemsetAsync(box + 3, 0, 3 * sizeof(unsigned), s);
    k_pos_box<<<g, 256, 0, s>>>(x3, n, box);
    uint32_t *key = (uint32_t *)scratch;
    int32_t *val = (int32_t *)(key + n);
    k_morton_keys<<<g, 256, 0, s>>>(x3, n, box, key, val);
    radix_sort(key, val, (int)n, 30, (void *)(val + n), s);
    k_perm_from_sorted<<<g, 256, 0, s>>>(val, n, perm);
    CC_COUNT_LAUNCH(3);
}

// ------------------------------------------------------------ edge order
__global__ void k_edge_keys(const int32_t *edges, long long ne, int col, const int32_t *perm, uint32_t *key,
                            int32_t *val)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne) return;
    const int e = perm ? perm[t] : (int)t;
    key[t] = (uint32_t)edges[2 * e + col];
    val[t] = e;
}

__global__ void k_edge_apply(const int32_t *edges, long long ne, const int32_t *perm, int32_t *out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ne) return;
    out[2 * t] = edges[2 * perm[t]];
    out[2 * t + 1] = edges[2 * perm[t] + 1];
}

// lexicographic (i, j) order: stable sort by j, then by i
void launch_sort_edges(int32_t *edges, long long ne, int bits, void *scratch, cudaStream_t s)
{
    if (ne <= 1) return;
    const int n = (int)ne;
    uint32_t *key = (uint32_t *)scratch;
    int32_t *val = (int32_t *)(key + n);
    int32_t *tmp = val + n;  // 2n
    void *ss = (void *)(tmp + 2 * n);
    const int g = (n + 255) / 256;
    k_edge_keys<<<g, 256, 0, s>>>(edges, ne, 1, nullptr, key, val);
    CC_COUNT_LAUNCH(1);
    radix_sort(key, val, n, bits, ss, s);
    cudaMemcpyAsync(tmp, val, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
    k_edge_keys<<<g, 256, 0, s>>>(edges, ne, 0, tmp, key, val);
    CC_COUNT_LAUNCH(1);
    radix_sort(key, val, n, bits, ss, s);
    k_edge_apply<<<g, 256, 0, s>>>(edges, ne, val, tmp);
    CC_COUNT_LAUNCH(1);
    cudaMemcpyAsync(edges, tmp, sizeof(int32_t) * 2 * n, cudaMemcpyDeviceToDevice, s);
}

size_t edge_sort_scratch_bytes(long long ne) { return (size_t)ne * 16 + sort_scratch_bytes(ne) + 256; }

}  // namespace cc
