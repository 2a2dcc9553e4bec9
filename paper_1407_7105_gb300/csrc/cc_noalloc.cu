// cc_noalloc.cu -- cc_components_noalloc: the connected-component split of
// a caller-held particle state with no device allocation at all.
//
// Who needs it: a caller whose device memory is owned by another allocator
// (a framework's caching pool that has reserved the GPU's memory, or a
// fixed budget handed out up front) cannot count on a cudaMalloc from this
// library succeeding, and a caller in a latency-critical loop cannot accept
// the device-wide synchronisation that cudaMalloc and cudaFree imply.  The
// context-based entry points allocate on the first use of every level, so
// this entry point instead keeps its union-find scratch in a fixed,
// file-scope device array: every GPU that loads libcc.so holds
// CC_NOALLOC_MAX_N * 8 bytes (512 KiB) of it until the process exits.
//
// The array's name in host code is a host-side stand-in, not a device
// address: kernels get the address from cudaGetSymbolAddress, looked up once
// per device (with that device current) on the first call made there.
#include <mutex>

#include "cc_internal.cuh"

namespace cc {

// parent[] and component sizes, then one word for the device error and one
// for the component count
static __device__ __align__(256) int32_t g_noalloc_scratch[2 * CC_NOALLOC_MAX_N + 64];

namespace {

constexpr int NA_T = 128;
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
int32_t *g_na_ptr[NA_MAX_DEVICES] = {};

struct NaScratch {
    int32_t *parent, *cnt;
    unsigned *err;
    int32_t *ncomp;
};

NaScratch na_view(int32_t *base)
{
    NaScratch s;
    s.parent = base;
    s.cnt = base + CC_NOALLOC_MAX_N;
    s.err = (unsigned *)(base + 2 * CC_NOALLOC_MAX_N);
    s.ncomp = base + 2 * CC_NOALLOC_MAX_N + 1;
    return s;
}

}  // namespace

// every word this call reads must start fresh: the array keeps the previous
// call's contents
__global__ void k_na_init(NaScratch S, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        S.parent[k] = k;
        S.cnt[k] = 0;
    }
    if (k == 0) {
        *S.err = 0u;
        *S.ncomp = 0;
    }
}

// tau(i,j) < h over all pairs i < j, hooked into the union-find forest
// (the same FP64 predicate as the context path, tiles loaded with plain
// coalesced loads because caller arrays need not be 16-byte aligned)
__global__ void __launch_bounds__(NA_T) k_na_tau_hook(const double *m, const double *x3, const double *v3, int n,
                                                      TauParams P, NaScratch S)
{
    __shared__ double col[7][NA_T];
    const int nt = (n + NA_T - 1) / NA_T;
    int t = blockIdx.x, ti = 0;
    while (t >= nt - ti) {
        t -= nt - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int j = tj * NA_T + threadIdx.x;
    if (j < n) {
        col[0][threadIdx.x] = x3[j];
        col[1][threadIdx.x] = x3[(size_t)n + j];
        col[2][threadIdx.x] = x3[2 * (size_t)n + j];
        col[3][threadIdx.x] = v3[j];
        col[4][threadIdx.x] = v3[(size_t)n + j];
        col[5][threadIdx.x] = v3[2 * (size_t)n + j];
        col[6][threadIdx.x] = m[j];
    }
    __syncthreads();
    const int i = ti * NA_T + threadIdx.x;
    if (i >= n) return;
    const double xi = x3[i], yi = x3[(size_t)n + i], zi = x3[2 * (size_t)n + i];
    const double vxi = v3[i], vyi = v3[(size_t)n + i], vzi = v3[2 * (size_t)n + i], mi = m[i];
    const int jn = min(NA_T, n - tj * NA_T);
    for (int k = (ti == tj) ? threadIdx.x + 1 : 0; k < jn; ++k) {
        const double tau = tau_fp64(__dsub_rn(xi, col[0][k]), __dsub_rn(yi, col[1][k]), __dsub_rn(zi, col[2][k]),
                                    __dsub_rn(vxi, col[3][k]), __dsub_rn(vyi, col[4][k]),
                                    __dsub_rn(vzi, col[5][k]), mi, col[6][k], P);
        if (tau < P.h && !uf_union(S.parent, i, tj * NA_T + k)) atomicCAS(S.err, 0u, (unsigned)DERR_UF_RETRY);
    }
}

// label = root = smallest index of the component; sizes by root
__global__ void k_na_compress(int n, NaScratch S, int32_t *labels)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int r = uf_find(S.parent, k);
    labels[k] = r;
    atomicAdd(&S.cnt[r], 1);
}

__global__ void k_na_count(int n, NaScratch S, int64_t *n_comp_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && S.cnt[k] >= 2) atomicAdd(S.ncomp, 1);
}

__global__ void k_na_store(NaScratch S, int64_t *n_comp_out) { *n_comp_out = *S.ncomp; }

}  // namespace cc

using namespace cc;

// Can a kernel on the current device read and write `ptr`?  Device and
// managed memory, and pinned host memory mapped into the device's address
// space, can; pageable host memory is refused (a kernel touching it would
// fault instead of returning an error).
static bool device_reachable(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.devicePointer != nullptr;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer == ptr;
    return false;
}

// device address of the scratch array for the current device, looked up
// once per device (with that device current) and kept for the life of the
// process (a cudaDeviceReset invalidates it; calls after one are not
// supported)
static int na_scratch(int32_t **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return CC_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        int32_t *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CC_E_CUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return CC_OK;
}

extern "C" int cc_components_noalloc(const double *m, const double *x3, const double *v3, int64_t n,
                                     const cc_params *p, double h, int32_t *labels_out, int64_t *n_comp_out,
                                     void *stream)
{
    if (!m || !x3 || !v3 || !p || !labels_out || !n_comp_out || !(h > 0.0) || !isfinite(h) || n < 1)
        return CC_E_ARG;
    // the parameters cc_init accepts for the same threshold test
    if (!(p->G > 0.0) || !isfinite(p->G) || !(p->eps >= 0.0) || !isfinite(p->eps) || !(p->eta > 0.0) ||
        !isfinite(p->eta) || (p->eta_outside != 0 && p->eta_outside != 1))
        return CC_E_ARG;
    if (n > CC_NOALLOC_MAX_N) return CC_E_CAPACITY;  // beyond the fixed scratch array
    // every pointer is read or written by a kernel: refuse what it cannot reach
    const void *ptrs[5] = {m, x3, v3, labels_out, n_comp_out};
    for (const void *q : ptrs)
        if (!device_reachable(q)) return CC_E_ARG;
    int32_t *base = nullptr;
    if (na_scratch(&base)) return CC_E_CUDA;
    const cudaStream_t s = (cudaStream_t)stream;
    const NaScratch S = na_view(base);
    TauParams P;
    P.G = p->G;
    P.eps2 = p->eps * p->eps;
    P.eta = p->eta;
    P.eta_in = p->eta_outside ? 1.0 : p->eta;
    P.eta_outside = p->eta_outside;
    P.h = h;
    P.near_tol = 0.0;
    P.fault_test = 0;
    const int ni = (int)n, g = (ni + 255) / 256;
    const long long nt = (n + NA_T - 1) / NA_T;
    k_na_init<<<g, 256, 0, s>>>(S, ni);
    k_na_tau_hook<<<(int)(nt * (nt + 1) / 2), NA_T, 0, s>>>(m, x3, v3, ni, P, S);
    k_na_compress<<<g, 256, 0, s>>>(ni, S, labels_out);
    k_na_count<<<g, 256, 0, s>>>(ni, S, n_comp_out);
    k_na_store<<<1, 1, 0, s>>>(S, n_comp_out);
    CC_COUNT_LAUNCH(5);
    if (cudaPeekAtLastError() != cudaSuccess) {  // a launch was refused: nothing was written
        cudaGetLastError();
        return CC_E_CUDA;
    }
    unsigned err = 0;
    if (cudaMemcpyAsync(&err, S.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return CC_E_CUDA;
    }
    return err ? CC_E_TIMEOUT : CC_OK;
}
