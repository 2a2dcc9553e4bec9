// cc_kepler.cu -- batched two-body flow for the CC_KEPLER variant
// (arXiv:1407.7105 Sec. 3.2: a connected component of two particles is
// advanced by a Kepler solver instead of recursion; the paper's solver is
// the universal-variable formulation of Bate, Mueller & White 1971).
// One thread per two-body component, FP64, eps = 0 (Eq. kepler).
#include "cc_internal.cuh"

namespace cc {

// Stumpff functions c2(z) = (1 - cos sqrt z)/z, c3(z) = (sqrt z - sin sqrt z)/z^{3/2}
// (hyperbolic continuation for z < 0), by their Taylor series near 0.
__device__ __forceinline__ void stumpff(double z, double &c2, double &c3)
{
    if (fabs(z) < 0.1) {
        // c2 = sum (-z)^k/(2k+2)!, c3 = sum (-z)^k/(2k+3)!
        double t2 = 0.5, t3 = 1.0 / 6.0;
        c2 = 0.0;
        c3 = 0.0;
#pragma unroll
        for (int k = 0; k < 10; ++k) {
            c2 += t2;
            c3 += t3;
            t2 *= -z / ((2.0 * k + 3.0) * (2.0 * k + 4.0));
            t3 *= -z / ((2.0 * k + 4.0) * (2.0 * k + 5.0));
        }
    } else if (z > 0.0) {
        const double s = sqrt(z);
        double sn, cs;
        sincos(s, &sn, &cs);
        c2 = (1.0 - cs) / z;
        c3 = (s - sn) / (z * s);
    } else {
        const double s = sqrt(-z);
        c2 = (cosh(s) - 1.0) / (-z);
        c3 = (sinh(s) - s) / (-z * s);
    }
}

// Advance the relative orbit (r0, v0) under mu by dt; returns false when
// the iteration does not converge.
__device__ bool kepler_universal(const double r0[3], const double v0[3], double mu, double dt, double r1[3],
                                 double v1[3])
{
    const double r0n = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    const double v0s = v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2];
    const double sig = r0[0] * v0[0] + r0[1] * v0[1] + r0[2] * v0[2];
    const double smu = sqrt(mu);
    const double alpha = 2.0 / r0n - v0s / mu;
    if (!(r0n > 0.0) || !(mu > 0.0) || !isfinite(alpha)) return false;
    // whole periods of a bound orbit are the identity: reduce dt
    if (alpha > 0.0) {
        const double P = 2.0 * CUDART_PI * sqrt(1.0 / (mu * alpha * alpha * alpha));
        if (fabs(dt) > P) dt = dt - P * trunc(dt / P);
    }
    const double a1 = sig / smu, a2 = 1.0 - alpha * r0n;
    double chi = (alpha > 0.0) ? smu * alpha * dt : smu * dt / r0n;
    if (alpha > 0.0 && fabs(alpha * r0n) < 1e-3) chi = smu * dt / r0n;
    double c2 = 0.5, c3 = 1.0 / 6.0, F1 = r0n;
    bool conv = false;
    // Laguerre-Conway iteration (order n = 5) on the universal Kepler equation
    for (int it = 0; it < 200; ++it) {
        const double x2 = chi * chi, z = alpha * x2;
        stumpff(z, c2, c3);
        const double F = a1 * x2 * c2 + a2 * x2 * chi * c3 + r0n * chi - smu * dt;
        F1 = a1 * chi * (1.0 - z * c3) + a2 * x2 * c2 + r0n;
        const double F2 = a1 * (1.0 - z * c2) + a2 * chi * (1.0 - z * c3);
        const double disc = sqrt(fabs(16.0 * F1 * F1 - 20.0 * F * F2));
        const double den = F1 + copysign(disc, F1);
        const double d = (den != 0.0) ? 5.0 * F / den : F / F1;
        chi -= d;
        if (fabs(d) <= 1e-15 * fmax(1.0, fabs(chi))) {
            conv = true;
            break;
        }
    }
    if (!conv) return false;
    // one Newton polish at the converged point
    {
        const double x2 = chi * chi, z = alpha * x2;
        stumpff(z, c2, c3);
        const double F = a1 * x2 * c2 + a2 * x2 * chi * c3 + r0n * chi - smu * dt;
        F1 = a1 * chi * (1.0 - z * c3) + a2 * x2 * c2 + r0n;
        chi -= F / F1;
    }
    const double x2 = chi * chi, z = alpha * x2;
    stumpff(z, c2, c3);
    const double f = 1.0 - x2 * c2 / r0n;
    const double g = dt - x2 * chi * c3 / smu;
    for (int k = 0; k < 3; ++k) r1[k] = f * r0[k] + g * v0[k];
    const double r = sqrt(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
    const double fd = smu / (r * r0n) * chi * (z * c3 - 1.0);
    const double gd = 1.0 - x2 * c2 / r;
    for (int k = 0; k < 3; ++k) v1[k] = fd * r0[k] + gd * v0[k];
    return isfinite(r);
}

__global__ void k_kepler(Level L, const int32_t *members, const int32_t *comp_start, const int32_t *klist, int nk,
                         double G, double dt, DevCounters *ctr)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nk) return;
    const int c = klist[t];
    const int a = members[comp_start[c]], b = members[comp_start[c] + 1];
    const double ma = L.m[a], mb = L.m[b], M = ma + mb;
    const double xa[3] = {L.x[a], L.y[a], L.z[a]}, xb[3] = {L.x[b], L.y[b], L.z[b]};
    const double va[3] = {L.vx[a], L.vy[a], L.vz[a]}, vb[3] = {L.vx[b], L.vy[b], L.vz[b]};
    double r0[3], v0[3], xc[3], vc[3], r1[3], v1[3];
    for (int k = 0; k < 3; ++k) {
        xc[k] = (ma * xa[k] + mb * xb[k]) / M;
        vc[k] = (ma * va[k] + mb * vb[k]) / M;
        r0[k] = xa[k] - xb[k];
        v0[k] = va[k] - vb[k];
    }
    if (!kepler_universal(r0, v0, G * M, dt, r1, v1)) {
        raise_err(ctr, DERR_KEPLER);
        return;
    }
    double na[3], nb[3], ua[3], ub[3];
    for (int k = 0; k < 3; ++k) {
        const double xcn = xc[k] + vc[k] * dt;
        na[k] = xcn + (mb / M) * r1[k];
        nb[k] = xcn - (ma / M) * r1[k];
        ua[k] = vc[k] + (mb / M) * v1[k];
        ub[k] = vc[k] - (ma / M) * v1[k];
    }
    L.x[a] = na[0]; L.y[a] = na[1]; L.z[a] = na[2];
    L.x[b] = nb[0]; L.y[b] = nb[1]; L.z[b] = nb[2];
    L.vx[a] = ua[0]; L.vy[a] = ua[1]; L.vz[a] = ua[2];
    L.vx[b] = ub[0]; L.vy[b] = ub[1]; L.vz[b] = ub[2];
}

void launch_kepler(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *klist,
                   int nk, double G, double dt, DevCounters *ctr, cudaStream_t s)
{
    if (nk > 0) {
        k_kepler<<<(nk + 127) / 128, 128, 0, s>>>(L, members, comp_start, klist, nk, G, dt, ctr);
        CC_COUNT_LAUNCH(1);
    }
}

}  // namespace cc
