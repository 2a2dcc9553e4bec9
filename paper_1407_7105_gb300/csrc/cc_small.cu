// cc_small.cu -- persistent small-component integrator: one warp evolves a
// whole connected component of at most 32 bodies through the recursion of
// evolve_cc (arXiv:1407.7105 Sec. 2.3, CC pseudocode figure) on-chip.
//
// Lane l holds body l of the component (members are in ascending particle
// id, so lane order is id order).  A set at recursion level k is a lane mask;
// all sets of the same level are advanced in lockstep (they are independent
// closed Hamiltonians, Sec. 2.2), level by level with an explicit stack:
//   phase 0: split the lane's set at h_k: tau(i,j) < h_k over the set (the
//            certified FP32 decision, the exact FP64 predicate where it
//            stays open: both forms), components by mask closure; push level k+1 with
//            the non-trivial components (first half)
//   phase 1: Kepler half step of two-body components (CC_KEPLER), the DKD
//            of level k, the second Kepler half step; push level k+1 again
//   phase 2: pop
// Warps take components from a queue (largest first) until it is empty.
// The arithmetic of every step is the same as the level kernels', so the
// FP64 form stays bit-identical to the oracle.
#include "cc_device.cuh"
#include <algorithm>

namespace cc {

constexpr int K8_WARPS = 4;
constexpr int K8_MAXD = 64;
constexpr unsigned FULL = 0xffffffffu;

struct __align__(16) K8Warp {
    double d[7][32];  // x y z vx vy vz m
    float f[13][32];  // hi/lo of x y z vx vy vz, m (FP32 decision)
    float xm[32], vm[32];  // per body max |x_hi|, max |v_hi| (error bounds)
    int gid[32];           // particle ids (near-threshold log)
    unsigned char e[32][32];  // e[j][l]: edge depth of pair (l, j) at the level the state was split fresh
};

__device__ __forceinline__ void k8_publish(K8Warp &S, int lane, const double st[7], bool ff)
{
    __syncwarp();  // every lane is done reading the previous contents
#pragma unroll
    for (int c = 0; c < 7; ++c) S.d[c][lane] = st[c];
    if (ff) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float hi, lo;
            ff_split(st[c], hi, lo);
            S.f[c][lane] = hi;
            S.f[6 + c][lane] = lo;
        }
        S.f[12][lane] = fl32(st[6]);
        S.xm[lane] = fmaxf(fabsf(S.f[0][lane]), fmaxf(fabsf(S.f[1][lane]), fabsf(S.f[2][lane])));
        S.vm[lane] = fmaxf(fabsf(S.f[3][lane]), fmaxf(fabsf(S.f[4][lane]), fabsf(S.f[5][lane])));
    }
    __syncwarp();
}

// x += dt v: exact IEEE operations in the FP64 form (bit-identical to the
// oracle), fused multiply-add in the mixed form
__device__ __forceinline__ void k8_drift(double st[7], double dt, bool exact)
{
    if (exact) {
        st[0] = __dadd_rn(st[0], __dmul_rn(dt, st[3]));
        st[1] = __dadd_rn(st[1], __dmul_rn(dt, st[4]));
        st[2] = __dadd_rn(st[2], __dmul_rn(dt, st[5]));
    } else {
        st[0] = fma(dt, st[3], st[0]);
        st[1] = fma(dt, st[4], st[1]);
        st[2] = fma(dt, st[5], st[2]);
    }
}

// ------------------------------------------------------------ edge depth
// A split at pivot h and the first split of each component's first half
// (pivot h/2) see the same state, so tau(i,j) is the same number and only
// the threshold halves.  The kernels therefore take, for each pair of a
// fresh state, its edge depth e: the pair is an edge at h 2^-m for
// m = 0 .. e-1 and not at h 2^-e (tau < h 2^-m is monotone in m).  The
// decisions are the ones a node-by-node evaluation takes: the FP64
// predicate compares one tau with each threshold, and the FP32 decision at
// h 2^-m is tau_decide_at(prep, (eta/h) 2^m) exactly.

// Out-of-line copies of the FP64 work a mixed-form component rarely needs
// (undecided tau, Kepler pairs, FP64 kicks): kept out of the lockstep loop
// so that its hot code stays compact in the instruction cache (a warp of
// this kernel mostly runs alone on its scheduler and waits on fetches).
__device__ __noinline__ double tau_fp64_ool(double dx0, double dx1, double dx2, double dv0, double dv1, double dv2,
                                            double mi, double mj, const TauParams &P)
{
    return tau_fp64(dx0, dx1, dx2, dv0, dv1, dv2, mi, mj, P);
}

struct K8Acc {
    double x, y, z;
};

// the FP64 row sum of one lane (the level kernels' arithmetic): a_i =
// sum over j in `others`, ascending, of (G m_j) r^-3 (x_j - x_i)
__device__ __noinline__ K8Acc k8_kick64(const K8Warp &S, int n, uint32_t others, double xi, double yi, double zi,
                                        double G, double eps2)
{
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int j = 0; j < n; ++j) {
        if (!((others >> j) & 1u)) continue;
        const double dx0 = __dsub_rn(S.d[0][j], xi);
        const double dx1 = __dsub_rn(S.d[1][j], yi);
        const double dx2 = __dsub_rn(S.d[2][j], zi);
        const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)),
                                              __dmul_rn(dx2, dx2)), eps2);
        const double rinv3 = __drcp_rn(__dmul_rn(r2, __dsqrt_rn(r2)));
        const double ww = __dmul_rn(__dmul_rn(G, S.d[6][j]), rinv3);
        ax = __dadd_rn(ax, __dmul_rn(ww, dx0));
        ay = __dadd_rn(ay, __dmul_rn(ww, dx1));
        az = __dadd_rn(az, __dmul_rn(ww, dx2));
    }
    return K8Acc{ax, ay, az};
}

// the Kepler flow of a two-body component over dt (positions and
// velocities of both bodies in place); the one copy of the solver that
// every kernel of this file calls
__device__ __noinline__ bool k8_kepler(double ma, double mb, double *xa, double *xb, double *va, double *vb, double G,
                                       double dt)
{
    return kepler_pair(ma, mb, xa, xb, va, vb, G, dt);
}

// log (i, j, tau) when |tau - h| < near_tol h (FP64-decided pairs only)
__device__ __noinline__ void near_log(double tau, double h, double near_tol, DevCounters *ctr, int ga, int gb,
                                         int32_t *near_ij, double *near_tau, long long near_cap)
{
    if (fabs(tau - h) < near_tol * h) {
        const unsigned long long z = atomicAdd(&ctr->near_pairs, 1ull);
        if ((long long)z < near_cap) {
            near_ij[2 * z] = ga < gb ? ga : gb;
            near_ij[2 * z + 1] = ga < gb ? gb : ga;
            near_tau[z] = tau;
        }
    }
}

struct NearLog {
    DevCounters *ctr;
    int32_t *ij;
    double *tau;
    long long cap;
    double tol;
};

// The FP64 tau's edge depth over `levels` thresholds h 2^-m (returns levels when
// every one is an edge).  log(tau, h_m) runs at the thresholds next to tau
// (h_m just above and at or below it): the only ones a near-threshold pair
// can sit at.
template <class LogF>
__device__ __forceinline__ int edge_depth_fp64(double tau, double h, int levels, LogF log)
{
    const int e = first_level_at_or_below(tau, h, levels);
    if (e >= 1) log(tau, scale2m(h, e - 1));
    if (e < levels) log(tau, scale2m(h, e));
    return e;
}

// mixed form: certified FP32 decisions from one prep (etah = eta/h) while
// they settle the threshold; at the first undecided threshold the FP64 tau
// (tau64(), evaluated once) settles the rest.  used64 reports whether it ran.
// The FP32 decisions agree with the FP64 predicate wherever they are taken,
// so the result is the FP64 predicate's edge depth.
template <class TauF, class LogF>
__device__ __forceinline__ int edge_depth_mixed(const TauPrep32 &t, float etah, double h, int levels, TauF tau64,
                                                LogF log, bool &used64)
{
    used64 = false;
    for (int m = 0; m < levels; ++m) {
        const int dec = tau_decide_at(t, etah * pow2f(m));
        if (dec > 0) continue;
        if (dec == 0) return m;
        used64 = true;
        const int e = edge_depth_fp64(tau64(), h, levels, log);
        return e > m ? e : m;
    }
    return levels;
}

// ------------------------------------------------------------ pair path
// evolve_cc({a, b}, h0) of a two-body set in one thread.  The recursion of a
// pair is a binary tree: a node at pivot h splits {a,b} (one tau); an edge
// makes it a component visited twice at h/2 (its DKD is empty: no rest set,
// no cross pair); no edge makes it a leaf, where both bodies form the rest
// set: drift h/2, pair kick h, drift h/2.  The tree is walked with a bit
// stack (bit d: the node at depth d has finished its first child); from a
// fresh state the walk goes straight down to the leaf through the state's
// edge depth.  e0 = the edge depth of the initial state if the caller knows
// it, else -1.
struct PairCounters {
    unsigned long long tau = 0, kick = 0, drift = 0, split = 0, comp = 0, fp64 = 0, evals = 0;
    int maxd = 0;
};

constexpr long long PAIR_VISIT_LIMIT = 1ll << 26;  // work cap per pair path (error beyond)

// after a leaf at depth d: the next node is the second child of the deepest
// node whose first child is finishing; returns false when the tree is done
__device__ __forceinline__ bool pair_next(unsigned long long &pend, int &d)
{
    while (d > 0) {
        --d;
        if (!((pend >> d) & 1ull)) {
            pend |= 1ull << d;
            ++d;
            return true;
        }
        pend &= ~(1ull << d);
    }
    return false;
}

// FP64 form, in the bodies' own coordinates with the level kernels'
// arithmetic (bit-identical to the oracle): the leaf's row sums are
// a_a = (G m_b) r^-3 (x_b - x_a) and a_b with -dx.
// Returns 0, DERR_DEPTH or DERR_SMALL_OVERFLOW (work cap).
// The edge decisions are the certified FP32 ones from the rounded FP64
// differences (relative error u, as in the mixed pair path), the FP64 tau
// where they stay open: the FP64 predicate's decisions (Q.etah = eta/h0).
__device__ unsigned pair_path(double A[7], double B[7], double h0, int depth0, int e0, const SmallParams &SP,
                              const TauParams &P, const MixedTauParams &Q, PairCounters &pc, const NearLog &nl,
                              int ga, int gb)
{
    const int dmax = min(SP.max_depth - depth0, 61);  // an edge at node d needs d + 1 <= dmax
    const float muf = Q.G * (fl32(A[6]) + fl32(B[6]));
    unsigned long long pend = 0ull;
    int d = 0, e = e0;
    for (long long work = 0; work < PAIR_VISIT_LIMIT;) {
        if (e < 0) {
            const double dx0 = __dsub_rn(A[0], B[0]), dx1 = __dsub_rn(A[1], B[1]), dx2 = __dsub_rn(A[2], B[2]);
            const double dv0 = __dsub_rn(A[3], B[3]), dv1 = __dsub_rn(A[4], B[4]), dv2 = __dsub_rn(A[5], B[5]);
            const TauPrep32 t = tau_prep_fp32(fl32(dx0), fl32(dx1), fl32(dx2), fl32(dv0), fl32(dv1), fl32(dv2), muf,
                                              0.f, 0.f, Q);
            ++pc.evals;
            bool used64;
            e = edge_depth_mixed(
                t, Q.etah * pow2f(d), scale2m(h0, d), max(dmax - d + 1, 1),
                [&]() { return tau_fp64_ool(dx0, dx1, dx2, dv0, dv1, dv2, A[6], B[6], P); },
                [&](double tv, double hm) { near_log(tv, hm, nl.tol, nl.ctr, ga, gb, nl.ij, nl.tau, nl.cap); },
                used64);
            pc.fp64 += used64 ? 1 : 0;
        }
        if (e > 0 && d + e > dmax) return DERR_DEPTH;  // an edge at a node below the cap
        pc.split += e + 1;
        pc.tau += e + 1;
        pc.comp += e;
        work += e + 1;
        d += e;
        if (depth0 + d > pc.maxd) pc.maxd = depth0 + d;
        const double h = scale2m(h0, d), hd = scale2m(h0, d + 1);
        k8_drift(A, hd, true);
        k8_drift(B, hd, true);
        const double dx0 = __dsub_rn(B[0], A[0]), dx1 = __dsub_rn(B[1], A[1]), dx2 = __dsub_rn(B[2], A[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)),
                                              __dmul_rn(dx2, dx2)), SP.eps2);
        const double rinv3 = __drcp_rn(__dmul_rn(r2, __dsqrt_rn(r2)));
        const double wa = __dmul_rn(__dmul_rn(SP.G, B[6]), rinv3), wb = __dmul_rn(__dmul_rn(SP.G, A[6]), rinv3);
        A[3] = __dadd_rn(A[3], __dmul_rn(h, __dmul_rn(wa, dx0)));
        A[4] = __dadd_rn(A[4], __dmul_rn(h, __dmul_rn(wa, dx1)));
        A[5] = __dadd_rn(A[5], __dmul_rn(h, __dmul_rn(wa, dx2)));
        B[3] = __dadd_rn(B[3], __dmul_rn(h, __dmul_rn(wb, -dx0)));
        B[4] = __dadd_rn(B[4], __dmul_rn(h, __dmul_rn(wb, -dx1)));
        B[5] = __dadd_rn(B[5], __dmul_rn(h, __dmul_rn(wb, -dx2)));
        k8_drift(A, hd, true);
        k8_drift(B, hd, true);
        ++pc.kick;
        pc.drift += 4;
        e = -1;
        if (!pair_next(pend, d)) return 0u;
    }
    return DERR_SMALL_OVERFLOW;
}

// Mixed form, in the pair's own coordinates: inside evolve_cc({a,b}, .)
// only the pair's mutual force acts, so the centre of mass moves uniformly
// and the relative state (r = x_a - x_b, u = v_a - v_b, FP64) carries
// everything.  A leaf is r += h/2 u; u -= h G M r/|r|^3; r += h/2 u: nine
// FP64 FMAs.  The FP32 force takes the drifted position in FP32, fl32(r) +
// (h/2) fl32(u) (a few units of u off the drifted FP64 r, like the force's
// own rounding), so the first drift's FP64 FMAs run beside the force
// instead of before it.  The edge decision takes fl32(r), fl32(u)
// (relative error u) and falls back to the exact FP64 predicate on (r, u);
// below h_fp64 the force is FP64 as well.
// Returns 0, DERR_DEPTH or DERR_SMALL_OVERFLOW.
__device__ unsigned pair_path_rel(double A[7], double B[7], double h0, int depth0, int e0, const SmallParams &SP,
                                  const TauParams &P, const MixedTauParams &Q, PairCounters &pc, const NearLog &nl,
                                  int ga, int gb)
{
    // mass fractions from one reciprocal (an FP64 division is a chain of
    // ~10 dependent FP64 operations on this part)
    const double ma = A[6], mb = B[6], M = ma + mb, iM = 1.0 / M, wa = ma * iM, wb = mb * iM;
    double R[3], V[3], r[3], u[3];
    for (int k = 0; k < 3; ++k) {
        R[k] = fma(wa, A[k], wb * B[k]);
        V[k] = fma(wa, A[3 + k], wb * B[3 + k]);
        r[k] = A[k] - B[k];
        u[k] = A[3 + k] - B[3 + k];
    }
    const float muf = Q.G * (fl32(ma) + fl32(mb));
    const double GM = SP.G * M;
    const float e2 = fl32(SP.eps2);
    const float etah0 = Q.etah;  // eta/h0 in float (the caller's, exact power-of-two scaling of its own)
    const int dmax = min(SP.max_depth - depth0, 61);
    const double c0 = -GM * h0;
    // h0 in float: h0 2^-(d+1) by exponent subtraction while it stays normal
    const float h0f = fl32(h0);
    const int h0x = (__float_as_int(h0f) >> 23) & 0xFF;
    // depths whose pivot h0 2^-d is below h_fp64 take FP64 forces
    int d64 = 64;
    if (SP.h_fp64 > 0.0) {
        d64 = first_level_at_or_below(SP.h_fp64, h0, 64);
        if (d64 < 64 && scale2m(h0, d64) == SP.h_fp64) ++d64;
    }
    unsigned long long pend = 0ull;
    int d = 0, e = e0;
    for (long long work = 0; work < PAIR_VISIT_LIMIT;) {
        const float fr0 = fl32(r[0]), fr1 = fl32(r[1]), fr2 = fl32(r[2]);
        const float fu0 = fl32(u[0]), fu1 = fl32(u[1]), fu2 = fl32(u[2]);
        if (e < 0) {
            const TauPrep32 t = tau_prep_fp32(fr0, fr1, fr2, fu0, fu1, fu2, muf, 0.f, 0.f, Q);
            ++pc.evals;
            bool used64;
            e = edge_depth_mixed(
                t, etah0 * pow2f(d), scale2m(h0, d), max(dmax - d + 1, 1),
                [&]() { return tau_fp64_ool(r[0], r[1], r[2], u[0], u[1], u[2], ma, mb, P); },
                [&](double tv, double hm) { near_log(tv, hm, nl.tol, nl.ctr, ga, gb, nl.ij, nl.tau, nl.cap); },
                used64);
            pc.fp64 += used64 ? 1 : 0;
        }
        if (e > 0 && d + e > dmax) return DERR_DEPTH;  // an edge at a node below the cap
        pc.split += e + 1;
        pc.tau += e + 1;
        pc.comp += e;
        work += e + 1;
        d += e;
        if (depth0 + d > pc.maxd) pc.maxd = depth0 + d;
        const double hd = scale2m(h0, d + 1);
        r[0] = fma(hd, u[0], r[0]);
        r[1] = fma(hd, u[1], r[1]);
        r[2] = fma(hd, u[2], r[2]);
        const double c = scale2m(c0, d);  // -G M h
        if (d >= d64) {
            // below the FP64-force threshold: the force in FP64
            const double q2 = fma(r[2], r[2], fma(r[1], r[1], fma(r[0], r[0], SP.eps2)));
            const double w = c / (q2 * sqrt(q2));
            u[0] = fma(w, r[0], u[0]);
            u[1] = fma(w, r[1], u[1]);
            u[2] = fma(w, r[2], u[2]);
        } else {
            float gx, gy, gz;
            if (h0x - (d + 1) >= 1) {
                const float hdf = __int_as_float(__float_as_int(h0f) - ((d + 1) << 23));
                gx = fmaf(hdf, fu0, fr0);
                gy = fmaf(hdf, fu1, fr1);
                gz = fmaf(hdf, fu2, fr2);
            } else {
                gx = fl32(r[0]);
                gy = fl32(r[1]);
                gz = fl32(r[2]);
            }
            const float q2 = fmaf(gz, gz, fmaf(gy, gy, fmaf(gx, gx, e2)));
            float ri = rsqrtf(q2);
            ri = ri * fmaf(-0.5f * q2, ri * ri, 1.5f);
            const float r3 = ri * ri * ri;
            u[0] = fma(c, f2d(r3 * gx), u[0]);
            u[1] = fma(c, f2d(r3 * gy), u[1]);
            u[2] = fma(c, f2d(r3 * gz), u[2]);
        }
        r[0] = fma(hd, u[0], r[0]);
        r[1] = fma(hd, u[1], r[1]);
        r[2] = fma(hd, u[2], r[2]);
        ++pc.kick;
        pc.drift += 4;
        e = -1;
        if (!pair_next(pend, d)) {
            for (int k = 0; k < 3; ++k) {
                const double Rk = fma(h0, V[k], R[k]);
                A[k] = fma(wb, r[k], Rk);
                B[k] = fma(-wa, r[k], Rk);
                A[3 + k] = fma(wb, u[k], V[k]);
                B[3 + k] = fma(-wa, u[k], V[k]);
            }
            return 0u;
        }
    }
    return DERR_SMALL_OVERFLOW;
}

// Hand every two-body set {lane, partner} (leader = the lower lane) to the
// pair path for its sub-recursion at pivot hsub; states move through shared
// memory.  First halves (eoff >= 0) start from the edge depths of the
// split just taken: the pair's depth at hsub is S.e - eoff unless the stored
// value hit its scan cap ecap.  Returns a device error code (0 = ok)
// uniform over the warp.
__device__ __forceinline__ unsigned k8_pair_handoff(K8Warp &S, int lane, double st[7], uint32_t cm, bool is_sub,
                                                    double hsub, float etah_sub, int dsub, int eoff, int ecap,
                                                    const SmallParams &SP,
                                                    const TauParams &P, const MixedTauParams &Q, bool mixed,
                                                    PairCounters &pc, const NearLog &nl)
{
    k8_publish(S, lane, st, false);
    const uint32_t me = 1u << lane;
    const bool leader = is_sub && lane == __ffs(cm) - 1;
    unsigned err = 0u;
    if (leader) {
        const int j = __ffs(cm & ~me) - 1;
        double B[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) B[c] = S.d[c][j];
        const int ga = S.gid[lane], gb = S.gid[j];
        const int ec = S.e[j][lane];
        const int e0 = (eoff >= 0 && ec < ecap) ? ec - eoff : -1;
        MixedTauParams Qs = Q;
        Qs.etah = etah_sub;  // eta/hsub
        if (mixed)
            err = pair_path_rel(st, B, hsub, dsub, e0, SP, P, Qs, pc, nl, ga, gb);
        else
            err = pair_path(st, B, hsub, dsub, e0, SP, P, Qs, pc, nl, ga, gb);
#pragma unroll
        for (int c = 0; c < 6; ++c) S.d[c][j] = B[c];
    }
    __syncwarp();
    if (is_sub && !leader) {
#pragma unroll
        for (int c = 0; c < 6; ++c) st[c] = S.d[c][lane];
    }
    const unsigned e = __reduce_or_sync(0xffffffffu, err);
    return e;
}

// counters of the sub-recursions a thread took part in (one atomic per
// warp at the end of the kernel)
struct SmallCnt {
    unsigned long long tau = 0, kick = 0, drift = 0, split = 0, comp = 0, kep = 0, fp64 = 0, eval = 0;
    int maxd = 0;
};

// the packed state of a level (what the batched tasks read and write)
struct SView {
    double *x, *y, *z, *vx, *vy, *vz;
    const double *m;
    const int32_t *gid;
};

// evolve_cc(C, h0) of one component of n <= 32 bodies (packed indices
// mem[0..n), ascending particle id) by one warp, its first split at depth
// depth0.  Errors are raised on ctr; the warp returns early on one.
__device__ __forceinline__ void small_task(K8Warp &S, const SView V, const int32_t *mem, int n, double h0, int depth0,
                                        const SmallParams &SP, DevCounters *ctr, const NearLog &nl, SmallCnt &cn,
                                        PairCounters &pc)
{
    const int lane = threadIdx.x & 31;
    const uint32_t me = 1u << lane;
    uint32_t mk[K8_MAXD], cmk[K8_MAXD];
    unsigned char ph[K8_MAXD], pm[K8_MAXD];
    signed char cf[K8_MAXD];  // level whose fresh split filled S.e for level k's state (-1: none)
    const bool mixed = SP.precision == CC_PREC_MIXED;
    TauParams P;
    P.G = SP.G; P.eps2 = SP.eps2; P.eta = SP.eta; P.eta_in = SP.eta_in; P.eta_outside = SP.eta_outside;
    P.near_tol = SP.near_tol;
    P.fault_test = 0;
    P.h = h0;
    MixedTauParams Q;
    Q.eta = (float)SP.eta_in; Q.eps2 = (float)SP.eps2; Q.G = (float)SP.G;
    Q.hq = 0.f;  // (the pre-test is not used here)
    // eta/h0 in float, once: eta/(h0 2^-k) is this times 2^k exactly
    const float etah_c = (float)(SP.eta_outside ? SP.eta_in * SP.eta / h0 : SP.eta_in / h0);
    const bool act = lane < n;
    const int p = act ? mem[lane] : -1;
    double st[7] = {0, 0, 0, 0, 0, 0, 0};
    if (act) {
        st[0] = V.x[p]; st[1] = V.y[p]; st[2] = V.z[p];
        st[3] = V.vx[p]; st[4] = V.vy[p]; st[5] = V.vz[p];
        st[6] = V.m[p];
    }
    const uint32_t all = (n >= 32) ? FULL : ((1u << n) - 1u);
    int k = 0;
    mk[0] = act ? all : 0u;
    ph[0] = 0;
    cf[0] = -1;
    __syncwarp();
    S.gid[lane] = act ? V.gid[p] : -1;
    __syncwarp();
    bool bad = false;
    if (depth0 > cn.maxd) cn.maxd = depth0;
    if (n == 2) {
        // a two-body component: its whole recursion on the pair path
        const unsigned e = k8_pair_handoff(S, lane, st, 3u, act, h0, etah_c, depth0, -1, 0, SP, P, Q, mixed, pc,
                                           nl);
        if (e) {
            raise_err(ctr, e);
            bad = true;
        }
        k = -1;
    }
    while (k >= 0 && !bad) {
        const double h = scale2m(h0, k);
        const uint32_t mine = mk[k];
        if (ph[k] == 0) {
            // ---------------- split at h: tau(i,j) < h inside the lane's set.
            // A fresh state (the component's start, a second half) takes
            // every pair's edge depth; a first half reads them, since its
            // state is the one its parent split.
            if (cf[k] < 0) {
                // (both forms: the certified FP32 decisions need the
                // float-float state; the FP64 tau settles what they leave open)
                k8_publish(S, lane, st, true);
                P.h = h;
                const float etah = etah_c * pow2f(k);
                const float c11 = 11.f * U32 * U32;
                const int levels = K8_MAXD - k;
                // FP64 tau of pair (lane, j), in the pair's fixed order
                // (symmetric bit for bit)
                auto tau64_of = [&](int j) {
                    const int lo = lane < j ? lane : j, hi = lane < j ? j : lane;
                    return tau_fp64_ool(__dsub_rn(S.d[0][lo], S.d[0][hi]), __dsub_rn(S.d[1][lo], S.d[1][hi]),
                                    __dsub_rn(S.d[2][lo], S.d[2][hi]), __dsub_rn(S.d[3][lo], S.d[3][hi]),
                                    __dsub_rn(S.d[4][lo], S.d[4][hi]), __dsub_rn(S.d[5][lo], S.d[5][hi]),
                                    S.d[6][lo], S.d[6][hi], P);
                };
                auto log_of = [&](int j, double tv, double hm) {
                    if (lane < j) near_log(tv, hm, nl.tol, nl.ctr, S.gid[lane], S.gid[j], nl.ij, nl.tau, nl.cap);
                };
                // the warp's active lanes at this level: a lane's set is a
                // subset, so its pairs are among these (deep levels of a
                // big component leave few)
                const uint32_t act = __reduce_or_sync(FULL, mine);
                if (mine) {
                    // the lane's own float-float state in registers (the
                    // byte stores of the edge depths below may alias any
                    // shared word, so reads from S would be repeated)
                    float me_f[13];
#pragma unroll
                    for (int q = 0; q < 13; ++q) me_f[q] = S.f[q][lane];
                    const float me_xm = S.xm[lane], me_vm = S.vm[lane];
                    auto prep = [&](int j) {
                        return tau_prep_fp32((S.f[0][j] - me_f[0]) + (S.f[6][j] - me_f[6]),
                                             (S.f[1][j] - me_f[1]) + (S.f[7][j] - me_f[7]),
                                             (S.f[2][j] - me_f[2]) + (S.f[8][j] - me_f[8]),
                                             (S.f[3][j] - me_f[3]) + (S.f[9][j] - me_f[9]),
                                             (S.f[4][j] - me_f[4]) + (S.f[10][j] - me_f[10]),
                                             (S.f[5][j] - me_f[5]) + (S.f[11][j] - me_f[11]),
                                             Q.G * (me_f[12] + S.f[12][j]), c11 * fmaxf(me_xm, S.xm[j]),
                                             c11 * fmaxf(me_vm, S.vm[j]), Q);
                    };
                    auto finish = [&](int j, const TauPrep32 &t) {
                        if (j == lane || !((mine >> j) & 1u)) return;
                        int e = 0;
                        if (tau_decide_at(t, etah) != 0) {
                            bool used64;
                            e = edge_depth_mixed(
                                t, etah, h, levels, [&]() { return tau64_of(j); },
                                [&](double tv, double hm) { log_of(j, tv, hm); }, used64);
                            if (used64 && lane < j) ++cn.fp64;
                        }
                        S.e[j][lane] = (unsigned char)e;
                        if (lane < j) ++cn.eval;
                    };
                    // two preps in flight, over the active lanes (pairs
                    // outside the lane's set are computed and dropped)
                    for (uint32_t rem = act; rem;) {
                        const int j0 = __ffs(rem) - 1;
                        rem &= rem - 1u;
                        const bool two = rem != 0u;
                        const int j1 = two ? __ffs(rem) - 1 : j0;
                        if (two) rem &= rem - 1u;
                        const TauPrep32 t0 = prep(j0), t1 = prep(j1);
                        finish(j0, t0);
                        if (two) finish(j1, t1);
                    }
                }
                cf[k] = (signed char)k;
            }
            const int eoff = k - cf[k];
            uint32_t adj = 0;
            if (mine) {
                for (int j = 0; j < n; ++j)
                    if (j != lane && ((mine >> j) & 1u) && S.e[j][lane] > eoff) adj |= 1u << j;
            }
            // components: closure of the adjacency by mask doubling
            // (each lane ORs the masks of its own members only: as many
            // shuffles per round as the largest mask has bits)
            uint32_t cm = mine ? (adj | me) : 0u;
            // HOLD split: every member of the set with an edge (tau(i) <
            // h) is in the one fast set
            const uint32_t hasedge = __ballot_sync(FULL, mine && adj != 0u);
            if (SP.hold) cm = mine ? (adj ? (hasedge & mine) : me) : 0u;
            for (int it = 0; it < 6 && !SP.hold; ++it) {
                uint32_t nx = cm, rem = cm;
                const unsigned rounds = __reduce_max_sync(FULL, (unsigned)__popc(cm));
                for (unsigned t = 0; t < rounds; ++t) {
                    const int j = rem ? __ffs(rem) - 1 : lane;
                    rem &= rem - 1u;
                    nx |= __shfl_sync(FULL, cm, j);
                }
                const bool same = __all_sync(FULL, nx == cm);
                cm = nx;
                if (same) break;
            }
            cmk[k] = cm;
            const int csz = __popc(cm);
            if (mine && lane == __ffs(mine) - 1) {
                const unsigned long long ms = __popc(mine);
                ++cn.split;
                cn.tau += ms * (ms - 1) / 2;
            }
            if (csz >= 2 && lane == __ffs(cm) - 1) {
                ++cn.comp;
                if (SP.kepler && csz == 2) cn.kep += 2;
            }
            ph[k] = 1;
            const bool sub = csz >= 2 && !(SP.kepler && csz == 2);
            // every sub-recursion at this level is a pair: run them on the
            // pair path (first half now, second half after the DKD)
            pm[k] = __all_sync(FULL, !sub || csz == 2) ? 1 : 0;
            if (pm[k] && __any_sync(FULL, sub)) {
                const unsigned e = k8_pair_handoff(S, lane, st, cm, sub, 0.5 * h, etah_c * pow2f(k + 1),
                                                   depth0 + k + 1, k + 1 - cf[k], K8_MAXD - cf[k], SP, P, Q,
                                                   mixed, pc, nl);
                if (e) {
                    raise_err(ctr, e);
                    bad = true;
                    break;
                }
            } else if (__any_sync(FULL, sub)) {
                pm[k] = 0;
                if (depth0 + k + 1 > SP.max_depth || k + 1 >= K8_MAXD) {
                    bad = true;
                    raise_err(ctr, DERR_DEPTH);
                    break;
                }
                mk[k + 1] = sub ? cm : 0u;
                ph[k + 1] = 0;
                cf[k + 1] = cf[k];  // first half: the state this split saw
                ++k;
                if (depth0 + k > cn.maxd) cn.maxd = depth0 + k;
                continue;
            }
        }
        const uint32_t cm = cmk[k];
        const int csz = __popc(cm);
        const bool sub = csz >= 2 && !(SP.kepler && csz == 2);
        if (ph[k] == 1) {
            const bool kep = mine && SP.kepler && csz == 2;
            const bool any_kep = __any_sync(FULL, kep);
            // the level's DKD has work only where the lane's set holds a
            // rest-set member or more than one component
            const bool any_dkd = __any_sync(FULL, mine && (cm != mine || cm == me));
            for (int half = 0; half < 2; ++half) {
                if (half == 1 && any_dkd) {
                    // ------------- D_{h/2,T_R} K_{h,V} D_{h/2,T_R} on the lane's set
                    const bool single = mine && cm == me;
                    const double hd = 0.5 * h;
                    if (single) {
                        k8_drift(st, hd, !mixed);
                        cn.drift += 2;
                    }
                    const bool fp64_kick = !mixed || h < SP.h_fp64;
                    k8_publish(S, lane, st, !fp64_kick);
                    const uint32_t act = __reduce_or_sync(FULL, mine);
                    if (mine) {
                        const uint32_t others = mine & ~cm;
                        cn.kick += __popc(others & ~((me << 1) - 1u));
                        if (fp64_kick) {
                            const K8Acc a = k8_kick64(S, n, others, st[0], st[1], st[2], SP.G, SP.eps2);
                            st[3] = __dadd_rn(st[3], __dmul_rn(h, a.x));
                            st[4] = __dadd_rn(st[4], __dmul_rn(h, a.y));
                            st[5] = __dadd_rn(st[5], __dmul_rn(h, a.z));
                        } else {
                            // FP32 pair forces from float-float differences
                            const float xh = S.f[0][lane], yh = S.f[1][lane], zh = S.f[2][lane];
                            const float xl = S.f[6][lane], yl = S.f[7][lane], zl = S.f[8][lane];
                            // two compensated accumulators: two independent
                            // dependency chains for one warp that runs alone on
                            // its scheduler; j outside the lane's others add an
                            // exact 0
                            float sx0 = 0.f, sy0 = 0.f, sz0 = 0.f, cx0 = 0.f, cy0 = 0.f, cz0 = 0.f;
                            float sx1 = 0.f, sy1 = 0.f, sz1 = 0.f, cx1 = 0.f, cy1 = 0.f, cz1 = 0.f;
                            const float e2 = (float)SP.eps2;
                            auto term = [&](int j, float &sx, float &sy, float &sz, float &cx, float &cy,
                                            float &cz) {
                                const float dx = (S.f[0][j] - xh) + (S.f[6][j] - xl);
                                const float dy = (S.f[1][j] - yh) + (S.f[7][j] - yl);
                                const float dz = (S.f[2][j] - zh) + (S.f[8][j] - zl);
                                const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, e2)));
                                float ri = rsqrtf(r2);
                                ri = ri * fmaf(-0.5f * r2, ri * ri, 1.5f);
                                const float ww = ((others >> j) & 1u) ? S.f[12][j] * (ri * ri * ri) : 0.f;
                                kahan_add(sx, cx, ww * dx);
                                kahan_add(sy, cy, ww * dy);
                                kahan_add(sz, cz, ww * dz);
                            };
                            // over the warp's active lanes, two terms per round
                            for (uint32_t rem = act; rem;) {
                                const int j0 = __ffs(rem) - 1;
                                rem &= rem - 1u;
                                term(j0, sx0, sy0, sz0, cx0, cy0, cz0);
                                if (rem) {
                                    term(__ffs(rem) - 1, sx1, sy1, sz1, cx1, cy1, cz1);
                                    rem &= rem - 1u;
                                }
                            }
                            const double gh = SP.G * h;
                            st[3] = fma(gh, (f2d(sx0) - f2d(cx0)) + (f2d(sx1) - f2d(cx1)), st[3]);
                            st[4] = fma(gh, (f2d(sy0) - f2d(cy0)) + (f2d(sy1) - f2d(cy1)), st[4]);
                            st[5] = fma(gh, (f2d(sz0) - f2d(cz0)) + (f2d(sz1) - f2d(cz1)), st[5]);
                        }
                    }
                    if (single) k8_drift(st, hd, !mixed);
                }
                if (!any_kep) continue;
                // two-body components: the Kepler flow over h/2
                k8_publish(S, lane, st, false);
                if (kep) {
                    const int other = __ffs(cm & ~me) - 1;
                    const int a = lane < other ? lane : other, b = lane < other ? other : lane;
                    double xa[3] = {S.d[0][a], S.d[1][a], S.d[2][a]}, xb[3] = {S.d[0][b], S.d[1][b], S.d[2][b]};
                    double va[3] = {S.d[3][a], S.d[4][a], S.d[5][a]}, vb[3] = {S.d[3][b], S.d[4][b], S.d[5][b]};
                    if (!k8_kepler(S.d[6][a], S.d[6][b], xa, xb, va, vb, SP.G, 0.5 * h)) {
                        raise_err(ctr, DERR_KEPLER);
                    } else if (lane == a) {
                        st[0] = xa[0]; st[1] = xa[1]; st[2] = xa[2]; st[3] = va[0]; st[4] = va[1]; st[5] = va[2];
                    } else {
                        st[0] = xb[0]; st[1] = xb[1]; st[2] = xb[2]; st[3] = vb[0]; st[4] = vb[1]; st[5] = vb[2];
                    }
                }
            }
            ph[k] = 2;
            if (__any_sync(FULL, sub)) {
                if (pm[k]) {
                    const unsigned e = k8_pair_handoff(S, lane, st, cm, sub, 0.5 * h, etah_c * pow2f(k + 1),
                                                       depth0 + k + 1, -1, 0, SP, P, Q, mixed, pc, nl);
                    if (e) {
                        raise_err(ctr, e);
                        bad = true;
                        break;
                    }
                } else {
                    mk[k + 1] = sub ? cm : 0u;
                    ph[k + 1] = 0;
                    cf[k + 1] = -1;  // second half: the DKD moved the state
                    ++k;
                    continue;
                }
            }
        }
        --k;
    }
    if (act) {
        V.x[p] = st[0]; V.y[p] = st[1]; V.z[p] = st[2];
        V.vx[p] = st[3]; V.vy[p] = st[4]; V.vz[p] = st[5];
    }
    __syncwarp();
}

// per-lane counters (lockstep levels + pair paths) -> one atomic per warp
__device__ __forceinline__ void flush_counters(const SmallCnt &cn, const PairCounters &pc, DevCounters *ctr)
{
    const int lane = threadIdx.x & 31;
    int maxd = max(cn.maxd, pc.maxd);
    unsigned long long v[8] = {cn.tau + pc.tau, cn.kick + pc.kick, cn.drift + pc.drift, cn.split + pc.split,
                               cn.comp + pc.comp, cn.kep, cn.fp64 + pc.fp64, cn.eval + pc.evals};
#pragma unroll
    for (int i = 0; i < 8; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(FULL, v[i], o);
    for (int o = 16; o > 0; o >>= 1) maxd = max(maxd, __shfl_down_sync(FULL, maxd, o));
    if (lane == 0) {
        if (v[0]) atomicAdd(&ctr->small_tau_pairs, v[0]);
        if (v[1]) atomicAdd(&ctr->small_kick_pairs, v[1]);
        if (v[2]) atomicAdd(&ctr->small_drifts, v[2]);
        if (v[3]) atomicAdd(&ctr->small_splits, v[3]);
        if (v[4]) atomicAdd(&ctr->small_components, v[4]);
        if (v[5]) atomicAdd(&ctr->small_kepler, v[5]);
        if (v[6]) atomicAdd(&ctr->tau_fp64, v[6]);
        if (v[7]) {
            atomicAdd(&ctr->tau_evals, v[7]);
            atomicAdd(&ctr->small_tau_evals, v[7]);
        }
        atomicMax(&ctr->max_depth_seen, maxd);
    }
}

__global__ void __launch_bounds__(K8_WARPS * 32) k_small(Level L, const int32_t *members, const int32_t *comp_start,
                                                          const int32_t *comp_size, const int32_t *slist,
                                                          const int32_t *ns_ptr,
                                                          SmallParams SP, DevCounters *ctr, int *queue,
                                                          int32_t *near_ij, double *near_tau, long long near_cap)
{
    __shared__ K8Warp sw[K8_WARPS];
    const int ns = *ns_ptr;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SView V{L.x, L.y, L.z, L.vx, L.vy, L.vz, L.m, L.gid};
    const NearLog nl = {ctr, near_ij, near_tau, near_cap, SP.near_tol};
    SmallCnt cn;
    PairCounters pc;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(queue, 1);
        q = __shfl_sync(FULL, q, 0);
        if (q >= ns) break;
        const int c = slist[q];
        if (comp_size[c] > 32) {  // (a warp holds at most 32 bodies: a task list out of order)
            if (lane == 0) raise_err(ctr, DERR_SMALL_OVERFLOW);
            continue;
        }
        small_task(sw[w], V, members + comp_start[c], comp_size[c], SP.h0, SP.depth0, SP, ctr, nl, cn, pc);
    }
    flush_counters(cn, pc, ctr);
}

// ------------------------------------------------------------ batched tasks
// k_batch takes evolve_cc tasks of up to BATCH_NMAX bodies from one queue,
// largest first.  A task of more than 32 bodies is run by the whole CTA
// (medium_task): the set's split, DKD and sub-recursions on-chip, its
// components of at most 32 bodies handed to the CTA's warps (small_task),
// larger ones to nested frames of the same CTA.  When the queue reaches the
// tasks of at most 32 bodies the CTA's warps take them one each, as k_small.
//
// A frame holds one set of more than 32 bodies (ascending particle id, in
// `sl`).  Its split: tau(i,j) < h over the set's pairs (in both forms the
// certified FP32 decision, the FP64 predicate where it cannot decide),
// union-find over set positions in shared memory (root = the
// smallest position, so labels are the smallest particle id), then the
// members by component into `cl` (components in root order, ascending
// inside): every component is a contiguous, ascending member list, which is
// what a nested frame or a warp task reads.  The DKD runs in set order, the
// kick's sum over j ascending: the FP64 form adds the same terms in the same
// order as the level kernels and the oracle.
// A CTA has W warps (template): 8 where a launch holds few tasks (latency:
// the CTA-level phases of the largest tasks), 4 for the batch of systems
// (thousands of tasks: more resident warps for the warp tasks).
constexpr int KM_MAXF = 32;  // nested sets of more than 32 bodies in one task (DERR_DEPTH beyond)
constexpr size_t KM_FRAME_BYTES = (size_t)BATCH_NMAX * 8;  // cl (int32) + lab (int16) + comp (int16 pairs)
static_assert(BATCH_NMAX % (2 * 8 * 32) == 0, "zig-zag rows");

enum : int { KM_SPLIT = 0, KM_H1 = 1, KM_B1 = 2, KM_DKD = 3, KM_H2 = 4, KM_B2 = 5, KM_DONE = 6 };

struct KMFrame {
    const int32_t *sl;  // the set's packed indices, ascending particle id
    int32_t *cl;        // the same, by component (root order), ascending inside
    int16_t *lab;       // by set position: the root's position (components of >= 2), else -1 - position
    int16_t *comp;      // (start in cl, size) of the components of >= 2 bodies, root order
    double h;
    int n, depth, ph, ncomp, it;
    unsigned long long kick;  // cross-component pairs of the set
    int nsingle;
};

// A frame's set staged in shared memory, four 16-byte words per body (one
// vector load each in the pair loops):
//   split (both forms): (x, y, z hi, fl32 m) (x, y, z lo, max |x hi|) (v hi, max |v hi|) (v lo, -)
//   DKD, FP64: {x, y} {z, m};  DKD, mixed: (x, y, z hi, fl32 m) (x, y, z lo, label bits)
struct KMStage {
    union {
        double2 d[4][BATCH_NMAX];
        float4 q[4][BATCH_NMAX];
    };
    int par[BATCH_NMAX];  // union-find forest over set positions, then roots
    int cnt[BATCH_NMAX];  // component size by root
    int cst[BATCH_NMAX];  // HOLD edge flags, then component start in cl by root
    int run[BATCH_NMAX];  // members placed so far by root
};

// the slot flags, then the slots (256-byte aligned)
__host__ __device__ constexpr size_t batch_pool_offset(int nslots) { return ((size_t)nslots * 4 + 255) / 256 * 256; }

template <int W>
struct KMShared {
    union {
        K8Warp sw[W];  // warp tasks
        KMStage st;    // a frame's split or DKD
    } u;
    KMFrame fr[KM_MAXF];
    int wsum[2][W];
    int top, bad, qi, hmin, q;
};

// exclusive prefix sums of two per-entry values over entries 0..n-1 (n <=
// BATCH_NMAX, entry e = 4 tid + k); totals returned
template <int W>
__device__ __forceinline__ void km_scan2(KMShared<W> &sh, const int a[4], const int b[4], int ea[4], int eb[4],
                                         int &ta, int &tb)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int sa = 0, sb = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ea[k] = sa;
        eb[k] = sb;
        sa += a[k];
        sb += b[k];
    }
    int ia = sa, ib = sb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int xa = __shfl_up_sync(FULL, ia, o), xb = __shfl_up_sync(FULL, ib, o);
        if (lane >= o) {
            ia += xa;
            ib += xb;
        }
    }
    if (lane == 31) {
        sh.wsum[0][w] = ia;
        sh.wsum[1][w] = ib;
    }
    __syncthreads();
    int oa = 0, ob = 0;
    ta = 0;
    tb = 0;
#pragma unroll
    for (int q = 0; q < W; ++q) {
        if (q < w) {
            oa += sh.wsum[0][q];
            ob += sh.wsum[1][q];
        }
        ta += sh.wsum[0][q];
        tb += sh.wsum[1][q];
    }
    oa += ia - sa;
    ob += ib - sb;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ea[k] += oa;
        eb[k] += ob;
    }
    __syncthreads();  // wsum is free again
}

// the split of the frame's set at F.h (see above); fills cl, lab, comp and
// the frame's counts
template <int W>
__device__ void km_split(KMShared<W> &sh, KMFrame &F, const SView V, const SmallParams &SP, float etah,
                         DevCounters *ctr, const NearLog &nl, SmallCnt &cn)
{
    constexpr int KM_T = W * 32;
    KMStage &T = sh.u.st;
    const int tid = threadIdx.x, lane = tid & 31;
    const int n = F.n;
    const double h = F.h;
    // both forms: the certified FP32 decision from the float-float state,
    // the FP64 tau (from the FP64 state) where it stays open
    for (int p = tid; p < n; p += KM_T) {
        const int k = F.sl[p];
        const double st[7] = {V.x[k], V.y[k], V.z[k], V.vx[k], V.vy[k], V.vz[k], V.m[k]};
        float hi[6], lo[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) ff_split(st[c], hi[c], lo[c]);
        const float xm = fmaxf(fabsf(hi[0]), fmaxf(fabsf(hi[1]), fabsf(hi[2])));
        const float vm = fmaxf(fabsf(hi[3]), fmaxf(fabsf(hi[4]), fabsf(hi[5])));
        T.q[0][p] = make_float4(hi[0], hi[1], hi[2], fl32(st[6]));
        T.q[1][p] = make_float4(lo[0], lo[1], lo[2], xm);
        T.q[2][p] = make_float4(hi[3], hi[4], hi[5], vm);
        T.q[3][p] = make_float4(lo[3], lo[4], lo[5], 0.f);
        T.par[p] = p;
        T.cnt[p] = 0;
        T.cst[p] = 0;
        T.run[p] = 0;
    }
    if (tid == 0) sh.hmin = BATCH_NMAX;
    __syncthreads();
    TauParams P;
    P.G = SP.G; P.eps2 = SP.eps2; P.eta = SP.eta; P.eta_in = SP.eta_in; P.eta_outside = SP.eta_outside;
    P.near_tol = SP.near_tol;
    P.fault_test = 0;
    P.h = h;
    MixedTauParams Q;
    Q.eta = (float)SP.eta_in; Q.eps2 = (float)SP.eps2; Q.G = (float)SP.G;
    Q.hq = 0.f;
    const float c11 = 11.f * U32 * U32;
    // the FP64 tau of positions lo < hi, in that order (the other kernels'
    // pair order; symmetric bit for bit)
    auto tau64 = [&](int lo, int hi) {
        const int a = F.sl[lo], b = F.sl[hi];
        return tau_fp64_ool(__dsub_rn(V.x[a], V.x[b]), __dsub_rn(V.y[a], V.y[b]), __dsub_rn(V.z[a], V.z[b]),
                            __dsub_rn(V.vx[a], V.vx[b]), __dsub_rn(V.vy[a], V.vy[b]),
                            __dsub_rn(V.vz[a], V.vz[b]), V.m[a], V.m[b], P);
    };
    bool uf_ok = true;
    auto edge_found = [&](int p, int j) {
        if (SP.hold) {
            T.cst[p] = 1;
            T.cst[j] = 1;
        } else if (!uf_union(T.par, p, j)) {
            uf_ok = false;
        }
    };
    auto decide64 = [&](int p, int j) {
        const double tau = tau64(p, j);
        ++cn.fp64;
        near_log(tau, h, nl.tol, nl.ctr, V.gid[F.sl[p]], V.gid[F.sl[j]], nl.ij, nl.tau, nl.cap);
        return tau < h;
    };
    // rows p of the pair triangle, zig-zag over the threads (balanced)
    for (int base = 0; base < n; base += 2 * KM_T) {
        for (int side = 0; side < 2; ++side) {
            const int p = side == 0 ? base + tid : base + 2 * KM_T - 1 - tid;
            if (p >= n - 1) continue;
            cn.eval += (unsigned long long)(n - 1 - p);
            {
                const float4 a0 = T.q[0][p], a1 = T.q[1][p], a2 = T.q[2][p], a3 = T.q[3][p];
                auto prep = [&](int j) {
                    const float4 b0 = T.q[0][j], b1 = T.q[1][j], b2 = T.q[2][j], b3 = T.q[3][j];
                    return tau_prep_fp32((b0.x - a0.x) + (b1.x - a1.x), (b0.y - a0.y) + (b1.y - a1.y),
                                         (b0.z - a0.z) + (b1.z - a1.z), (b2.x - a2.x) + (b3.x - a3.x),
                                         (b2.y - a2.y) + (b3.y - a3.y), (b2.z - a2.z) + (b3.z - a3.z),
                                         Q.G * (a0.w + b0.w), c11 * fmaxf(a1.w, b1.w), c11 * fmaxf(a2.w, b2.w), Q);
                };
                auto finish = [&](int j, const TauPrep32 &t) {
                    const int dec = tau_decide_at(t, etah);
                    const bool edge = dec >= 0 ? dec > 0 : decide64(p, j);
                    if (edge) edge_found(p, j);
                };
                // one pair at a time: two in flight shortened a lone task's
                // split but cost throughput when every SM was busy with tasks
                for (int j = p + 1; j < n; ++j) finish(j, prep(j));
            }
        }
    }
    if (!uf_ok) {
        raise_err(ctr, DERR_UF_RETRY);
        sh.bad = 1;
    }
    __syncthreads();
    // roots (HOLD: every member with an edge joins the smallest such member)
    if (SP.hold) {
        for (int p = tid; p < n; p += KM_T)
            if (T.cst[p]) atomicMin(&sh.hmin, p);
        __syncthreads();
        for (int p = tid; p < n; p += KM_T) T.run[p] = T.cst[p] ? sh.hmin : p;
    } else {
        for (int p = tid; p < n; p += KM_T) T.run[p] = uf_find(T.par, p);
    }
    __syncthreads();
    for (int p = tid; p < n; p += KM_T) {
        T.par[p] = T.run[p];
        T.run[p] = 0;
        atomicAdd(&T.cnt[T.par[p]], 1);
    }
    __syncthreads();
    // component starts (sizes by root, in root order) and the table of
    // components of >= 2 bodies
    int a[4], b[4], ea[4], eb[4], ta, tb;
    unsigned long long inner = 0;
    int nkep = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = 4 * tid + k;
        const bool root = r < n && T.par[r] == r;
        a[k] = root ? T.cnt[r] : 0;
        b[k] = root && T.cnt[r] >= 2 ? 1 : 0;
        if (b[k]) {
            inner += (unsigned long long)T.cnt[r] * (T.cnt[r] - 1) / 2;
            if (SP.kepler && T.cnt[r] == 2) ++nkep;
        }
    }
    km_scan2(sh, a, b, ea, eb, ta, tb);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = 4 * tid + k;
        if (r < n && T.par[r] == r) {
            T.cst[r] = ea[k];
            if (b[k]) {
                F.comp[2 * eb[k]] = (int16_t)ea[k];
                F.comp[2 * eb[k] + 1] = (int16_t)T.cnt[r];
            }
        }
    }
    // (inner, nkep, singles) summed over the CTA
    int single = 0;
    for (int p = tid; p < n; p += KM_T) single += T.cnt[T.par[p]] == 1 ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) {
        inner += __shfl_down_sync(FULL, inner, o);
        nkep += __shfl_down_sync(FULL, nkep, o);
        single += __shfl_down_sync(FULL, single, o);
    }
    __shared__ unsigned long long s_inner[W];
    __shared__ int s_kep[W], s_single[W];
    if (lane == 0) {
        s_inner[tid >> 5] = inner;
        s_kep[tid >> 5] = nkep;
        s_single[tid >> 5] = single;
    }
    __syncthreads();
    // members by component: one warp, 32 positions a round (peers of one
    // root ranked by lane, so each component stays ascending)
    if (tid < 32) {
        const unsigned lt = (1u << lane) - 1u;
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int p = c0 + lane;
            const bool v = p < n;
            const int r = v ? T.par[p] : -1 - lane;
            const unsigned peers = __match_any_sync(FULL, r);
            if (v) {
                const int pos = T.cst[r] + T.run[r] + __popc(peers & lt);
                F.cl[pos] = F.sl[p];
                F.lab[p] = (int16_t)(T.cnt[r] >= 2 ? r : -1 - p);
            }
            __syncwarp();
            if (v && lane == 31 - __clz(peers)) T.run[r] += __popc(peers);
            __syncwarp();
        }
    }
    if (tid == 0) {
        unsigned long long in = 0;
        int kp = 0, sg = 0;
        for (int q = 0; q < W; ++q) {
            in += s_inner[q];
            kp += s_kep[q];
            sg += s_single[q];
        }
        const unsigned long long pairs = (unsigned long long)n * (n - 1) / 2;
        F.ncomp = tb;
        F.kick = pairs - in;
        F.nsingle = sg;
        ++cn.split;
        cn.tau += pairs;
        cn.comp += tb;
        cn.kep += 2ull * kp;
    }
    __syncthreads();
}

// D_{h/2,T_R} K_{h,V} D_{h/2,T_R} on the frame's set: rest-set members drift,
// every cross-component pair kicks (sum over j ascending)
template <int W>
__device__ void km_dkd(KMShared<W> &sh, const KMFrame &F, const SView V, const SmallParams &SP, SmallCnt &cn)
{
    constexpr int KM_T = W * 32;
    KMStage &T = sh.u.st;
    const int tid = threadIdx.x;
    const int n = F.n;
    const double h = F.h, hd = 0.5 * h;
    const bool mixed = SP.precision == CC_PREC_MIXED;
    const bool fp64_kick = !mixed || h < SP.h_fp64;
    for (int p = tid; p < n; p += KM_T) {
        const int k = F.sl[p];
        double st[7] = {V.x[k], V.y[k], V.z[k], V.vx[k], V.vy[k], V.vz[k], V.m[k]};
        const int lab = F.lab[p];
        T.par[p] = lab;  // labels in shared memory for the pair loops
        if (lab < 0) {
            k8_drift(st, hd, !mixed);
            V.x[k] = st[0];
            V.y[k] = st[1];
            V.z[k] = st[2];
        }
        if (fp64_kick) {
            T.d[0][p] = make_double2(st[0], st[1]);
            T.d[1][p] = make_double2(st[2], st[6]);
        } else {
            float hi[3], lo[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) ff_split(st[c], hi[c], lo[c]);
            T.q[0][p] = make_float4(hi[0], hi[1], hi[2], fl32(st[6]));
            T.q[1][p] = make_float4(lo[0], lo[1], lo[2], __int_as_float(lab));
        }
    }
    __syncthreads();
    for (int p = tid; p < n; p += KM_T) {
        const int k = F.sl[p];
        const int li = T.par[p];
        double st[7] = {V.x[k], V.y[k], V.z[k], V.vx[k], V.vy[k], V.vz[k], V.m[k]};
        if (fp64_kick) {
            // the level kernels' row sum: terms of two j computed side by
            // side, added in ascending j
            double ax = 0.0, ay = 0.0, az = 0.0;
            const double2 i0 = T.d[0][p], i1 = T.d[1][p];
            auto term = [&](int j, double &fx, double &fy, double &fz) {
                const double2 b0 = T.d[0][j], b1 = T.d[1][j];
                const double dx0 = __dsub_rn(b0.x, i0.x);
                const double dx1 = __dsub_rn(b0.y, i0.y);
                const double dx2 = __dsub_rn(b1.x, i1.x);
                const double r2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx0, dx0), __dmul_rn(dx1, dx1)),
                                                      __dmul_rn(dx2, dx2)), SP.eps2);
                const double rinv3 = __drcp_rn(__dmul_rn(r2, __dsqrt_rn(r2)));
                const double ww = __dmul_rn(__dmul_rn(SP.G, b1.y), rinv3);
                fx = __dmul_rn(ww, dx0);
                fy = __dmul_rn(ww, dx1);
                fz = __dmul_rn(ww, dx2);
            };
            for (int j = 0; j < n; j += 2) {
                const bool u0 = j != p && T.par[j] != li;
                const bool u1 = j + 1 < n && j + 1 != p && T.par[j + 1] != li;
                double f0x = 0.0, f0y = 0.0, f0z = 0.0, f1x = 0.0, f1y = 0.0, f1z = 0.0;
                if (u0) term(j, f0x, f0y, f0z);
                if (u1) term(j + 1, f1x, f1y, f1z);
                if (u0) {
                    ax = __dadd_rn(ax, f0x);
                    ay = __dadd_rn(ay, f0y);
                    az = __dadd_rn(az, f0z);
                }
                if (u1) {
                    ax = __dadd_rn(ax, f1x);
                    ay = __dadd_rn(ay, f1y);
                    az = __dadd_rn(az, f1z);
                }
            }
            st[3] = __dadd_rn(st[3], __dmul_rn(h, ax));
            st[4] = __dadd_rn(st[4], __dmul_rn(h, ay));
            st[5] = __dadd_rn(st[5], __dmul_rn(h, az));
        } else {
            const float4 a0 = T.q[0][p], a1 = T.q[1][p];
            const float e2 = (float)SP.eps2;
            // two compensated accumulators (even and odd j): two independent chains
            float sx0 = 0.f, sy0 = 0.f, sz0 = 0.f, cx0 = 0.f, cy0 = 0.f, cz0 = 0.f;
            float sx1 = 0.f, sy1 = 0.f, sz1 = 0.f, cx1 = 0.f, cy1 = 0.f, cz1 = 0.f;
            auto term = [&](int j, float &sx, float &sy, float &sz, float &cx, float &cy, float &cz) {
                const float4 b0 = T.q[0][j], b1 = T.q[1][j];
                const float dx = (b0.x - a0.x) + (b1.x - a1.x);
                const float dy = (b0.y - a0.y) + (b1.y - a1.y);
                const float dz = (b0.z - a0.z) + (b1.z - a1.z);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, e2)));
                float ri = rsqrtf(r2);
                ri = ri * fmaf(-0.5f * r2, ri * ri, 1.5f);
                const float ww = (j != p && __float_as_int(b1.w) != li) ? b0.w * (ri * ri * ri) : 0.f;
                kahan_add(sx, cx, ww * dx);
                kahan_add(sy, cy, ww * dy);
                kahan_add(sz, cz, ww * dz);
            };
            for (int j = 0; j < n; j += 2) {
                term(j, sx0, sy0, sz0, cx0, cy0, cz0);
                if (j + 1 < n) term(j + 1, sx1, sy1, sz1, cx1, cy1, cz1);
            }
            const double gh = SP.G * h;
            st[3] = fma(gh, (f2d(sx0) - f2d(cx0)) + (f2d(sx1) - f2d(cx1)), st[3]);
            st[4] = fma(gh, (f2d(sy0) - f2d(cy0)) + (f2d(sy1) - f2d(cy1)), st[4]);
            st[5] = fma(gh, (f2d(sz0) - f2d(cz0)) + (f2d(sz1) - f2d(cz1)), st[5]);
        }
        if (li < 0) k8_drift(st, hd, !mixed);
        V.x[k] = st[0];
        V.y[k] = st[1];
        V.z[k] = st[2];
        V.vx[k] = st[3];
        V.vy[k] = st[4];
        V.vz[k] = st[5];
    }
    if (tid == 0) {
        cn.kick += F.kick;
        cn.drift += 2ull * F.nsingle;
    }
    __syncthreads();
}

// evolve_cc(C, h0) of one task of 33..BATCH_NMAX bodies (packed indices
// mem[0..n0), ascending particle id) by the whole CTA, its first split at
// depth depth0; frame scratch at fs (KM_MAXF frames)
template <int W>
__device__ void medium_task(KMShared<W> &sh, const SView V, const int32_t *mem, int n0, double h0, int depth0,
                            const SmallParams &SP, DevCounters *ctr, const NearLog &nl, SmallCnt &cn,
                            PairCounters &pc, char *fs)
{
    constexpr int KM_T = W * 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const float etah0 = (float)(SP.eta_outside ? SP.eta_in * SP.eta / h0 : SP.eta_in / h0);
    auto frame_at = [&](int k, const int32_t *sl, int n, double h, int depth) {
        KMFrame &F = sh.fr[k];
        char *b = fs + (size_t)k * KM_FRAME_BYTES;
        F.sl = sl;
        F.cl = (int32_t *)b;
        F.lab = (int16_t *)(b + (size_t)BATCH_NMAX * 4);
        F.comp = (int16_t *)(b + (size_t)BATCH_NMAX * 6);
        F.n = n;
        F.h = h;
        F.depth = depth;
        F.ph = KM_SPLIT;
        F.ncomp = 0;
        F.it = 0;
    };
    if (tid == 0) {
        frame_at(0, mem, n0, h0, depth0);
        sh.top = 0;
        sh.bad = 0;
        if (depth0 > cn.maxd) cn.maxd = depth0;
    }
    __syncthreads();
    for (;;) {
        const int top = sh.top;
        if (top < 0) break;
        KMFrame &F = sh.fr[top];
        const int ph = F.ph;
        __syncthreads();  // every thread has read the control words
        if (ph == KM_SPLIT) {
            km_split(sh, F, V, SP, etah0 * pow2f(F.depth - depth0), ctr, nl, cn);
            if (tid == 0) F.ph = KM_H1;
        } else if (ph == KM_H1 || ph == KM_H2) {
            // the Kepler flow of two-body components over h/2 (CC_KEPLER),
            // then the sub-recursions of components of at most 32 bodies
            const int nc = F.ncomp;
            const double hh = 0.5 * F.h;
            if (SP.kepler) {
                for (int ci = tid; ci < nc; ci += KM_T) {
                    if (F.comp[2 * ci + 1] != 2) continue;
                    const int a = F.cl[F.comp[2 * ci]], b = F.cl[F.comp[2 * ci] + 1];
                    double xa[3] = {V.x[a], V.y[a], V.z[a]}, xb[3] = {V.x[b], V.y[b], V.z[b]};
                    double va[3] = {V.vx[a], V.vy[a], V.vz[a]}, vb[3] = {V.vx[b], V.vy[b], V.vz[b]};
                    if (!k8_kepler(V.m[a], V.m[b], xa, xb, va, vb, SP.G, hh)) {
                        raise_err(ctr, DERR_KEPLER);
                    } else {
                        V.x[a] = xa[0]; V.y[a] = xa[1]; V.z[a] = xa[2];
                        V.vx[a] = va[0]; V.vy[a] = va[1]; V.vz[a] = va[2];
                        V.x[b] = xb[0]; V.y[b] = xb[1]; V.z[b] = xb[2];
                        V.vx[b] = vb[0]; V.vy[b] = vb[1]; V.vz[b] = vb[2];
                    }
                }
            }
            bool subs = false;
            for (int ci = 0; ci < nc && !subs; ++ci) {
                const int z = F.comp[2 * ci + 1];
                subs = !(SP.kepler && z == 2);
            }
            if (subs && F.depth + 1 > SP.max_depth) {
                if (tid == 0) {
                    raise_err(ctr, DERR_DEPTH);
                    sh.bad = 1;
                }
            } else if (subs) {
                if (tid == 0) sh.qi = 0;
                __syncthreads();
                for (;;) {
                    int ci = 0;
                    if (lane == 0) ci = atomicAdd(&sh.qi, 1);
                    ci = __shfl_sync(FULL, ci, 0);
                    if (ci >= nc) break;
                    const int z = F.comp[2 * ci + 1];
                    if (z > 32 || (SP.kepler && z == 2)) continue;
                    small_task(sh.u.sw[w], V, F.cl + F.comp[2 * ci], z, hh, F.depth + 1, SP, ctr, nl, cn, pc);
                }
            }
            if (tid == 0) {
                F.ph = ph == KM_H1 ? KM_B1 : KM_B2;
                F.it = 0;
            }
        } else if (ph == KM_B1 || ph == KM_B2) {
            // the next component of more than 32 bodies: a nested frame
            if (tid == 0) {
                int ci = F.it;
                while (ci < F.ncomp && F.comp[2 * ci + 1] <= 32) ++ci;
                if (ci < F.ncomp) {
                    F.it = ci + 1;
                    if (top + 1 >= KM_MAXF || F.depth + 1 > SP.max_depth) {
                        raise_err(ctr, DERR_DEPTH);
                        sh.bad = 1;
                    } else {
                        frame_at(top + 1, F.cl + F.comp[2 * ci], F.comp[2 * ci + 1], 0.5 * F.h, F.depth + 1);
                        sh.top = top + 1;
                        if (F.depth + 1 > cn.maxd) cn.maxd = F.depth + 1;
                    }
                } else {
                    F.ph = ph == KM_B1 ? KM_DKD : KM_DONE;
                }
            }
        } else if (ph == KM_DKD) {
            if (F.kick > 0 || F.nsingle > 0) km_dkd(sh, F, V, SP, cn);
            if (tid == 0) F.ph = KM_H2;
        } else {
            if (tid == 0) sh.top = top - 1;
        }
        __syncthreads();
        if (sh.bad) {
            __syncthreads();
            if (tid == 0) sh.top = -1;
            __syncthreads();
            break;
        }
    }
    __syncthreads();
}

template <int W>
__global__ void __launch_bounds__(W * 32) k_batch(Level L, const int32_t *members, const int32_t *t_start,
                                                 const int32_t *t_size, const int32_t *tlist, const int32_t *nt_ptr,
                                                 SmallParams SP, DevCounters *ctr, int *queue, int32_t *near_ij,
                                                 double *near_tau, long long near_cap, char *scratch, int nslots)
{
    __shared__ KMShared<W> sh;
    __shared__ int s_slot;
    const int nt = *nt_ptr;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const SView V{L.x, L.y, L.z, L.vx, L.vy, L.vz, L.m, L.gid};
    const NearLog nl = {ctr, near_ij, near_tau, near_cap, SP.near_tol};
    // frame scratch: a slot of the pool, claimed at the first CTA task (the
    // pool holds as many slots as CTAs of this kernel can be resident, over
    // all launches in flight, so a resident CTA always finds one)
    int *slot_flag = (int *)scratch;
    char *pool = scratch + batch_pool_offset(nslots);
    if (tid == 0) s_slot = -1;
    SmallCnt cn;
    PairCounters pc;
    // CTA mode while the queue's head task has more than 32 bodies
    int first = -1;
    for (;;) {
        if (tid == 0) sh.q = atomicAdd(queue, 1);
        __syncthreads();
        const int q = sh.q;
        __syncthreads();
        if (q >= nt) break;
        const int c = tlist[q], n = t_size[c];
        if (n > 32) {
            if (tid == 0 && s_slot < 0) {
                for (int r = 0; r < 4 * nslots && s_slot < 0; ++r) {
                    const int k = (int)((blockIdx.x + (unsigned)r) % (unsigned)nslots);
                    if (atomicCAS(&slot_flag[k], 0, 1) == 0) s_slot = k;
                }
                if (s_slot < 0) raise_err(ctr, DERR_SMALL_OVERFLOW);
            }
            __syncthreads();
            if (s_slot < 0) break;
            medium_task(sh, V, members + t_start[c], n, SP.h0, SP.depth0, SP, ctr, nl, cn, pc,
                        pool + (size_t)s_slot * KM_MAXF * KM_FRAME_BYTES);
            continue;
        }
        first = q;  // warp mode from here: this task to warp 0, the rest from the queue
        break;
    }
    if (first >= 0) {
        for (int q = (w == 0) ? first : -1;;) {
            if (q < 0) {
                if (lane == 0) q = atomicAdd(queue, 1);
                q = __shfl_sync(FULL, q, 0);
            }
            if (q >= nt) break;
            const int c = tlist[q];
            if (t_size[c] > 32) {
                // warp mode assumes the queue holds the CTA tasks first (the
                // classification's order): a larger task here is an error,
                // never a silent partial step
                if (lane == 0) raise_err(ctr, DERR_SMALL_OVERFLOW);
            } else {
                small_task(sh.u.sw[w], V, members + t_start[c], t_size[c], SP.h0, SP.depth0, SP, ctr, nl, cn, pc);
            }
            q = -1;
        }
    }
    __syncthreads();
    if (tid == 0 && s_slot >= 0) {
        __threadfence();
        atomicExch(&slot_flag[s_slot], 0);
    }
    flush_counters(cn, pc, ctr);
}

// CTAs of k_batch<W> resident on the whole GPU (a launch's grid)
template <int W>
static int batch_grid(int nsm)
{
    static int occ = 0;
    if (occ == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batch<W>, W * 32, 0) != cudaSuccess || o < 1) {
            cudaGetLastError();
            o = 1;
        }
        occ = o;
    }
    return occ * (nsm > 0 ? nsm : 1);
}

// the frame-scratch pool: one slot per CTA that can be resident, for the
// variant with the most resident CTAs (several launches of either variant
// in flight at once hold at most that many)
static int batch_slots(int nsm) { return std::max(batch_grid<4>(nsm), batch_grid<8>(nsm)); }

size_t batch_scratch_bytes(int nsm)
{
    const int g = batch_slots(nsm);
    return batch_pool_offset(g) + (size_t)g * KM_MAXF * KM_FRAME_BYTES;
}

void launch_batch(const Level &L, const int32_t *members, const int32_t *t_start, const int32_t *t_size,
                  const int32_t *tlist, const int32_t *nt_ptr, int nt_bound, const SmallParams &SP, DevCounters *ctr,
                  int *queue, int32_t *near_ij, double *near_tau, long long near_cap, int nsm, char *scratch,
                  cudaStream_t s, int warps)
{
    if (nt_bound <= 0) return;
    // *queue is zero on entry; CTAs beyond the work exit at the first read
    const int slots = batch_slots(nsm);
    if (warps == 8) {
        const int g = batch_grid<8>(nsm), grid = nt_bound < g ? nt_bound : g;
        k_batch<8><<<grid, 8 * 32, 0, s>>>(L, members, t_start, t_size, tlist, nt_ptr, SP, ctr, queue, near_ij,
                                           near_tau, near_cap, scratch, slots);
    } else {
        const int g = batch_grid<4>(nsm), grid = nt_bound < g ? nt_bound : g;
        k_batch<4><<<grid, 4 * 32, 0, s>>>(L, members, t_start, t_size, tlist, nt_ptr, SP, ctr, queue, near_ij,
                                           near_tau, near_cap, scratch, slots);
    }
    CC_COUNT_LAUNCH(1);
}

// ------------------------------------------------------------ Kepler pairs
// CC_KEPLER (Sec. 3.2): a component of two particles is advanced by the
// universal-variable Kepler flow instead of recursion.  One thread per
// two-body component of a level.  The solver is the one out-of-line
// k8_kepler of this translation unit that the warp and CTA tasks call too,
// so a two-body component gets the same bits whichever kernel takes it.
__global__ void k_kepler(Level L, const int32_t *members, const int32_t *comp_start, const int32_t *klist,
                         const int32_t *nk_ptr, double G, double dt, DevCounters *ctr)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *nk_ptr) return;
    const int c = klist[t];
    const int a = members[comp_start[c]], b = members[comp_start[c] + 1];
    double xa[3] = {L.x[a], L.y[a], L.z[a]}, xb[3] = {L.x[b], L.y[b], L.z[b]};
    double va[3] = {L.vx[a], L.vy[a], L.vz[a]}, vb[3] = {L.vx[b], L.vy[b], L.vz[b]};
    if (!k8_kepler(L.m[a], L.m[b], xa, xb, va, vb, G, dt)) {
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

void launch_small(const Level &L, const int32_t *members, const int32_t *comp_start, const int32_t *comp_size,
                  const int32_t *slist, const int32_t *ns_ptr, int ns_bound, const SmallParams &SP, DevCounters *ctr,
                  int *queue, int32_t *near_ij, double *near_tau, long long near_cap, int nsm, cudaStream_t s)
{
    if (ns_bound <= 0) return;
    // *queue is zero on entry and *ns_ptr the component count (k_classify);
    // warps of blocks beyond the work exit at the first queue read
    const int want = (ns_bound + K8_WARPS - 1) / K8_WARPS;
    const int grid = want < nsm * 8 ? want : nsm * 8;
    k_small<<<grid, K8_WARPS * 32, 0, s>>>(L, members, comp_start, comp_size, slist, ns_ptr, SP, ctr, queue, near_ij,
                                           near_tau, near_cap);
    CC_COUNT_LAUNCH(1);
}

}  // namespace cc
