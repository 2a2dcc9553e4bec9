// cc_com.cu -- the centre-of-mass approximation of V_CC (arXiv:1407.7105,
// Sec. 4.1 Discussion: long-range kicks between different connected
// components through their centres of mass, evaluated symmetrically).
//
// In the DKD of a set of at least COM_MIN_SET members, components of
// 2..com_max members are eligible; two of them are far when R_a + R_b <
// theta |X_a - X_b| (X: centre of mass, R: the largest distance of a member
// from it).  The kick kernel leaves the pairs of far components out and
// every member of component a then receives A_a = sum over its far
// partners b (ascending) of (G M_b) (X_b - X_a) / (d2 sqrt(d2)), d2 =
// |X_b - X_a|^2 + eps^2, as v += h A_a.  The forces between two components
// are opposite and along the line of their centres: momentum and angular
// momentum are kept.  Every sum runs over members in ascending packed index
// (ascending particle id in the FP64 form) with explicit IEEE operations, so
// the FP64 form is bit-identical to a plain evaluation in that order.
#include "cc_internal.cuh"

namespace cc {

// one thread per eligible component: mass, centre of mass, radius, and the
// members' local index
__global__ void k_com_prep(Level L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                           const int32_t *eq, const int32_t *eloc, int Ke, int32_t *cl, double *cm)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ke) return;
    const int q = eq[g], b0 = comp_start[q], nb = comp_size[q];
    double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int k = 0; k < nb; ++k) {
        const int i = members[b0 + k];
        const double mi = L.m[i];
        M = __dadd_rn(M, mi);
        sx = __dadd_rn(sx, __dmul_rn(mi, L.x[i]));
        sy = __dadd_rn(sy, __dmul_rn(mi, L.y[i]));
        sz = __dadd_rn(sz, __dmul_rn(mi, L.z[i]));
        cl[i] = eloc[g];
    }
    const double X = __ddiv_rn(sx, M), Y = __ddiv_rn(sy, M), Z = __ddiv_rn(sz, M);
    double R = 0.0;
    for (int k = 0; k < nb; ++k) {
        const int i = members[b0 + k];
        const double dx = __dsub_rn(L.x[i], X), dy = __dsub_rn(L.y[i], Y), dz = __dsub_rn(L.z[i], Z);
        const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        if (r > R) R = r;
    }
    double *c = cm + 8 * (size_t)g;
    c[0] = M; c[1] = X; c[2] = Y; c[3] = Z; c[4] = R;
}

// one thread per eligible component a: its row of the far matrix and its
// monopole acceleration A_a (partners in ascending local index)
__global__ void k_com_far(double *cm, const int32_t *eq, const int32_t *comp_size, const int32_t *eset,
                          const int32_t *eloc, const int32_t *efirst, const long long *foff, const int32_t *K, int Ke,
                          double theta, double G, double eps2, unsigned char *far, int32_t *eany,
                          DevCounters *ctr)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Ke) return;
    const int s = eset[g], a = eloc[g], Ks = K[s], g0 = efirst[s];
    const double *ca = cm + 8 * (size_t)g;
    unsigned char *row = far + foff[s] + (long long)a * Ks;
    double Ax = 0.0, Ay = 0.0, Az = 0.0;
    int any = 0;
    unsigned long long pairs = 0;
    const int na = comp_size[eq[g]];
    for (int b = 0; b < Ks; ++b) {
        unsigned char f = 0;
        if (b != a) {
            const double *cb = cm + 8 * (size_t)(g0 + b);
            const double dx = __dsub_rn(cb[1], ca[1]), dy = __dsub_rn(cb[2], ca[2]), dz = __dsub_rn(cb[3], ca[3]);
            const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            const double d = __dsqrt_rn(dd);
            f = __dadd_rn(ca[4], cb[4]) < __dmul_rn(theta, d) ? 1 : 0;
            if (f) {
                const double d2 = __dadd_rn(dd, eps2);
                const double w = __dmul_rn(__dmul_rn(G, cb[0]), __drcp_rn(__dmul_rn(d2, __dsqrt_rn(d2))));
                Ax = __dadd_rn(Ax, __dmul_rn(w, dx));
                Ay = __dadd_rn(Ay, __dmul_rn(w, dy));
                Az = __dadd_rn(Az, __dmul_rn(w, dz));
                any = 1;
                if (b > a) pairs += (unsigned long long)na * (unsigned long long)comp_size[eq[g0 + b]];
            }
        }
        row[b] = f;
    }
    double *c = cm + 8 * (size_t)g;
    c[5] = Ax; c[6] = Ay; c[7] = Az;
    eany[g] = any;
    if (pairs) atomicAdd(&ctr->com_pairs, pairs);
}

// mixed form: one warp per eligible component a, its lanes over the
// partners b (the same far decisions in the same FP64 operations), the
// monopole sum reduced across the lanes (another FP64 rounding order: the
// mixed form is not bit-tied to the oracle); K rows of K partners on
// 32 K lanes instead of K
__global__ void k_com_far_warp(double *cm, const int32_t *eq, const int32_t *comp_size, const int32_t *eset,
                               const int32_t *eloc, const int32_t *efirst, const long long *foff, const int32_t *K,
                               int Ke, double theta, double G, double eps2, unsigned char *far, int32_t *eany,
                               DevCounters *ctr)
{
    const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (g >= Ke) return;  // (the whole warp)
    const int s = eset[g], a = eloc[g], Ks = K[s], g0 = efirst[s];
    const double *ca = cm + 8 * (size_t)g;
    unsigned char *row = far + foff[s] + (long long)a * Ks;
    double Ax = 0.0, Ay = 0.0, Az = 0.0;
    int any = 0;
    unsigned long long pairs = 0;
    const int na = comp_size[eq[g]];
    for (int b = lane; b < Ks; b += 32) {
        unsigned char f = 0;
        if (b != a) {
            const double *cb = cm + 8 * (size_t)(g0 + b);
            const double dx = __dsub_rn(cb[1], ca[1]), dy = __dsub_rn(cb[2], ca[2]), dz = __dsub_rn(cb[3], ca[3]);
            const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            const double d = __dsqrt_rn(dd);
            f = __dadd_rn(ca[4], cb[4]) < __dmul_rn(theta, d) ? 1 : 0;
            if (f) {
                const double d2 = __dadd_rn(dd, eps2);
                const double w = __dmul_rn(__dmul_rn(G, cb[0]), __drcp_rn(__dmul_rn(d2, __dsqrt_rn(d2))));
                Ax = __dadd_rn(Ax, __dmul_rn(w, dx));
                Ay = __dadd_rn(Ay, __dmul_rn(w, dy));
                Az = __dadd_rn(Az, __dmul_rn(w, dz));
                any = 1;
                if (b > a) pairs += (unsigned long long)na * (unsigned long long)comp_size[eq[g0 + b]];
            }
        }
        row[b] = f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Ax += __shfl_xor_sync(0xffffffffu, Ax, o);
        Ay += __shfl_xor_sync(0xffffffffu, Ay, o);
        Az += __shfl_xor_sync(0xffffffffu, Az, o);
        any |= __shfl_xor_sync(0xffffffffu, any, o);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    }
    if (lane == 0) {
        double *c = cm + 8 * (size_t)g;
        c[5] = Ax; c[6] = Ay; c[7] = Az;
        eany[g] = any;
        if (pairs) atomicAdd(&ctr->com_pairs, pairs);
    }
}

// one block per eligible component, one thread per member
__global__ void k_com_apply(Level L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                            const int32_t *eq, const double *cm, const int32_t *eany, double h)
{
    const int g = blockIdx.x;
    if (!eany[g]) return;
    const int q = eq[g];
    if ((int)threadIdx.x >= comp_size[q]) return;
    const int i = members[comp_start[q] + threadIdx.x];
    const double *c = cm + 8 * (size_t)g;
    L.vx[i] = __dadd_rn(L.vx[i], __dmul_rn(h, c[5]));
    L.vy[i] = __dadd_rn(L.vy[i], __dmul_rn(h, c[6]));
    L.vz[i] = __dadd_rn(L.vz[i], __dmul_rn(h, c[7]));
}

void launch_com_prep(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                     const int32_t *eq, const int32_t *eloc, int Ke, int32_t *cl, double *cm, cudaStream_t s)
{
    if (Ke <= 0) return;
    k_com_prep<<<(Ke + 127) / 128, 128, 0, s>>>(L, members, comp_start, comp_size, eq, eloc, Ke, cl, cm);
    CC_COUNT_LAUNCH(1);
}

void launch_com_far(double *cm, const int32_t *eq, const int32_t *comp_size, const int32_t *eset,
                    const int32_t *eloc, const int32_t *efirst, const long long *foff, const int32_t *K, int Ke,
                    double theta, double G, double eps2, unsigned char *far, int32_t *eany, DevCounters *ctr,
                    cudaStream_t s, bool mixed)
{
    if (Ke <= 0) return;
    if (mixed)
        k_com_far_warp<<<(unsigned)(((long long)Ke * 32 + 127) / 128), 128, 0, s>>>(
            cm, eq, comp_size, eset, eloc, efirst, foff, K, Ke, theta, G, eps2, far, eany, ctr);
    else
        k_com_far<<<(Ke + 127) / 128, 128, 0, s>>>(cm, eq, comp_size, eset, eloc, efirst, foff, K, Ke, theta, G,
                                                   eps2, far, eany, ctr);
    CC_COUNT_LAUNCH(1);
}

void launch_com_apply(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                      const int32_t *eq, const double *cm, const int32_t *eany, int Ke, double h, cudaStream_t s)
{
    if (Ke <= 0) return;
    k_com_apply<<<Ke, COM_MAX_MEMBERS, 0, s>>>(L, members, comp_start, comp_size, eq, cm, eany, h);
    CC_COUNT_LAUNCH(1);
}

}  // namespace cc
