// cc_kepler.cu -- batched two-body flow for the CC_KEPLER variant
// (arXiv:1407.7105 Sec. 3.2: a connected component of two particles is
// advanced by a Kepler solver instead of recursion; the paper's solver is
// the universal-variable formulation of Bate, Mueller & White 1971).
// One thread per two-body component, FP64, eps = 0 (Eq. kepler).
#include "cc_device.cuh"

namespace cc {

__global__ void k_kepler(Level L, const int32_t *members, const int32_t *comp_start, const int32_t *klist,
                         const int32_t *nk_ptr, double G, double dt, DevCounters *ctr)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *nk_ptr) return;
    const int c = klist[t];
    const int a = members[comp_start[c]], b = members[comp_start[c] + 1];
    double xa[3] = {L.x[a], L.y[a], L.z[a]}, xb[3] = {L.x[b], L.y[b], L.z[b]};
    double va[3] = {L.vx[a], L.vy[a], L.vz[a]}, vb[3] = {L.vx[b], L.vy[b], L.vz[b]};
    if (!kepler_pair(L.m[a], L.m[b], xa, xb, va, vb, G, dt)) {
        raise_err(ctr, DERR_KEPLER);
        return;
    }
    L.x[a] = xa[0]; L.y[a] = xa[1]; L.z[a] = xa[2];
    L.x[b] = xb[0]; L.y[b] = xb[1]; L.z[b] = xb[2];
    L.vx[a] = va[0]; L.vy[a] = va[1]; L.vz[a] = va[2];
    L.vx[b] = vb[0]; L.vy[b] = vb[1]; L.vz[b] = vb[2];
}

void launch_kepler(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *klist,
                   const int32_t *nk_ptr, int nk_bound, double G, double dt, DevCounters *ctr, cudaStream_t s)
{
    if (nk_bound > 0) {
        k_kepler<<<(nk_bound + 127) / 128, 128, 0, s>>>(L, members, comp_start, klist, nk_ptr, G, dt, ctr);
        CC_COUNT_LAUNCH(1);
    }
}

}  // namespace cc
