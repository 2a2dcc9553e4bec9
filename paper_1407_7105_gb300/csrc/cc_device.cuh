// cc_device.cuh -- device functions shared by several kernels of libcc.so:
// the certified FP32 decision of the edge predicate tau(i,j) < h
// (arXiv:1407.7105 Eq. tauij), compensated summation, and the universal-
// variable two-body flow of the CC_KEPLER variant (Sec. 3.2).
#pragma once
#include "cc_internal.cuh"

namespace cc {

// ------------------------------------------------------------ tau, FP32 certified
// Error model (u = 2^-24; +,-,*,fma round to nearest: u each; rsqrtf within
// 2 ulp, budgeted 8u; every bound below is budgeted generously):
//   |dx~ - dx| <= er r,  er = 2.05u + 11u^2 X / r      (float-float difference)
//   |dv~ - dv| <= ev |dv|, ev = 2.05u + 11u^2 V / |dv|
//   rinv = rsqrt(r2), s1 = rsqrt(r mu), s2 = rsqrt(v2)
//   T_ff = eta r2 s1          (= eta sqrt(r^3/mu)),      rel. error <= 40u + 3er
//   T_fb = eta r s2           (= eta r/|dv|),            rel. error <= 40u + 3er + 3ev
//   dT_ff = 1.5 eta rv s1,  dT_fb = eta rv s2 rinv (1 + mu s2^2 rinv)
//   rv = dx.dv has no relative bound (cancellation): |drv| <= (er+ev+4u) r |dv|,
//   so |d dT| <= 32u|dT_ff| + 1.5 eta s1 |drv|   (ff)
//              80u|dT_fb| + eta s2 rinv (1 + mu s2^2 rinv) |drv|   (fb)
//   D = 1 - min(dT,1)/2 >= 1/2,  |dD| <= |d dT|/2 + 2u D
// tau_x = T_x / D_x < h is certain when T~(1+eT)(1+s) < h (D~ - dD), and
// certainly false when T~(1-eT)(1-s) >= h (D~ + dD); the slack s = 2e-6
// covers the FP32 evaluation of the bounds and the FP64 predicate's own
// rounding.  Any NaN/Inf fails both tests: the pair is undecided.
constexpr float U32 = 5.9604645e-8f;  // 2^-24
constexpr float SLACK = 2e-6f;

// eta and eta/h in float (the decision compares T/h with D); c_x = 11 u^2 X
// and c_v = 11 u^2 V carry the float-float rounding of the differences
struct MixedTauParams {
    float eta, etah, eps2, G;
    float hq;  // eta/etah (h, or h/eta when eta multiplies the min): the pre-test's q = hq |dv|/r
};

// The h-independent part of the decision: everything except T/h.  The
// decision at a threshold h then costs two products and four comparisons,
// and since eta/h doubles exactly when h halves, T/h at h 2^-m is T/h at h
// times 2^m bit for bit: decide(prep, etah * 2^m) is the decision the full
// evaluation would take at h 2^-m for the same state.
struct TauPrep32 {
    float r2, s1, r, s2;         // Tff/h = (etah r2) s1, Tfb/h = (etah r) s2
    float ffA, ffB, ffLo, ffHi;  // ff edge certain: Tff ffA < ffLo; no edge certain: Tff ffB >= ffHi
    float fbA, fbB, fbLo, fbHi;  // the same for the flyby term
    bool fb;                     // flyby term usable (else only a certain ff edge decides)
};

__device__ __forceinline__ TauPrep32 tau_prep_fp32(float dx0, float dx1, float dx2, float dv0, float dv1, float dv2,
                                                   float mu, float c_x, float c_v, const MixedTauParams &Q)
{
    TauPrep32 t;
    const float A = 1.f + SLACK, B = 1.f - SLACK;
    const float r2 = fmaf(dx2, dx2, fmaf(dx1, dx1, fmaf(dx0, dx0, Q.eps2)));
    const float v2 = fmaf(dv2, dv2, fmaf(dv1, dv1, dv0 * dv0));
    const float rv = fmaf(dx2, dv2, fmaf(dx1, dv1, dx0 * dv0));
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float s1 = rsqrtf(r * mu);
    const float er = fmaf(c_x, rinv, 2.05f * U32);
    const float s2 = v2 > 0.f ? rsqrtf(v2) : 0.f;
    const float vn = v2 * s2;  // |dv|
    const float ev = fmaf(c_v, s2, 2.05f * U32);
    const float drv = (er + ev + 4.f * U32) * (r * vn);
    // free fall: T/h = (eta/h) r2 s1, dT/dt = 1.5 eta rv s1
    const float dTff = 1.5f * Q.eta * rv * s1;
    const float Dff = fmaf(-0.5f, fminf(dTff, 1.f), 1.f);
    const float dDff = fmaf(0.5f, fmaf(32.f * U32, fabsf(dTff), 1.5f * Q.eta * s1 * drv), 2.f * U32 * Dff);
    const float eff = fmaf(3.f, er, 40.f * U32);
    t.r2 = r2;
    t.s1 = s1;
    t.r = r;
    t.s2 = s2;
    t.ffA = fmaf(eff, A, A);
    t.ffB = fmaf(-eff, B, B);
    t.ffLo = Dff - dDff;
    t.ffHi = Dff + dDff;
    // an exactly zero (or unresolved) FP32 velocity difference may hide a
    // tiny nonzero FP64 one, whose flyby term can be small: only a certain
    // free-fall edge decides such a pair
    t.fb = (v2 > 0.f) && !(vn < 6.f * c_v);
    // flyby: T/h = (eta/h) r s2, dT/dt = eta rv s2 rinv (1 + mu s2^2 rinv)
    const float g = fmaf(mu * s2 * s2, rinv, 1.f);
    const float k = s2 * rinv * g;
    const float dTfb = Q.eta * rv * k;
    const float Dfb = fmaf(-0.5f, fminf(dTfb, 1.f), 1.f);
    const float dDfb = fmaf(0.5f, fmaf(80.f * U32, fabsf(dTfb), Q.eta * k * drv), 2.f * U32 * Dfb);
    const float efb = fmaf(3.f, er + ev, 40.f * U32);
    t.fbA = fmaf(efb, A, A);
    t.fbB = fmaf(-efb, B, B);
    t.fbLo = Dfb - dDfb;
    t.fbHi = Dfb + dDfb;
    return t;
}

// returns 1 = edge certain, 0 = no edge certain, -1 = undecided; etah =
// eta/h in float
__device__ __forceinline__ int tau_decide_at(const TauPrep32 &t, float etah)
{
    const float Tff = etah * t.r2 * t.s1;
    const bool ff_yes = Tff * t.ffA < t.ffLo;
    if (!t.fb) return ff_yes ? 1 : -1;
    const bool ff_no = Tff * t.ffB >= t.ffHi;
    const float Tfb = etah * t.r * t.s2;
    const bool fb_yes = Tfb * t.fbA < t.fbLo;
    const bool fb_no = Tfb * t.fbB >= t.fbHi;
    if (ff_yes || fb_yes) return 1;
    if (ff_no && fb_no) return 0;
    return -1;
}

// A sufficient test for "no edge" that skips the certified evaluation for
// the great majority of pairs (those whose tau is well above h).  With T =
// T_ff or T_fb and D = 1 - min(dT/dt, 1)/2, tau_x = T/D and D <= 1 + |dT/dt|/2:
//   free fall: |dT_ff/dt| = 1.5 T_ff |rv|/r^2 <= 1.5 T_ff |dv|/r, so
//     tau_ff >= h  if  (T_ff/h) (1 - 0.75 q) >= 1,  q = h|dv|/r (q < 4/3);
//   flyby:     |dT_fb/dt| <= eta (1 + mu/(r v^2))  (T_fb = eta r/|dv|), so
//     tau_fb >= h  if  T_fb/h >= 1 + eta (1 + mu/(r v^2))/2.
// (eta is the factor inside T: Q.eta; hq = h/eta_in, the same as
// eta/etah in both readings of the eta placement.)  The differences may be
// formed from the rounded high parts alone: then |dx~ - dx| <= u r + c_x
// + 3.5 u r with c_x = 7 u max|x_i| (per component |x_j| <= |x_i| + r),
// likewise c_v for the velocities.  Once (c_x + 3.5 u r)/r and the velocity
// analogue are below 1e-4, every FP32 quantity used has relative
// error below 1e-3 (the error model above: 40u + 3(er + ev) plus the rsqrt
// budget), so a 2 % margin on each inequality makes the test rigorous; a
// pair it does not settle goes to the certified decision.
// reciprocal square root, PTX rsqrt.approx.ftz.f32 (relative error below
// 2^-22.9 for normal inputs; a denormal input is flushed to zero and gives
// +inf, which the pre-test's comparisons reject)
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ bool tau_quick_apart(float dx0, float dx1, float dx2, float dv0, float dv1, float dv2,
                                                float mu, float c_x, float c_v, const MixedTauParams &Q)
{
    const float r2 = fmaf(dx2, dx2, fmaf(dx1, dx1, fmaf(dx0, dx0, Q.eps2)));
    const float v2 = fmaf(dv2, dv2, fmaf(dv1, dv1, dv0 * dv0));
    const float rinv = rsqrt_ftz(r2);
    const float r = r2 * rinv;
    const float s1 = rsqrt_ftz(r * mu);
    const float s2 = rsqrt_ftz(v2);   // inf for v2 = 0: rejected below
    const float vn = v2 * s2;         // |dv|
    const float Tff = Q.etah * r2 * s1;                  // T_ff / h
    const float q = Q.hq * vn * rinv;                    // h |dv| / r
    const float Tfb = Q.etah * r * s2;                   // T_fb / h
    const float g = mu * rinv * s2 * s2;                 // mu / (r v^2)
    const float M = 1.02f;
    // (the bounds below leave 3.5u for a relative part of c_x/r, c_v/|dv|;
    // all conditions are evaluated: no short-circuit branches)
    const bool ok = (c_x * rinv <= 0.99e-4f) & (v2 > 0.f) & (c_v * s2 <= 0.99e-4f) & (0.75f * M * q < 1.f) &
                    (Tff * fmaf(-0.75f * M, q, 1.f) >= M) & (Tfb >= M * fmaf(0.5f * Q.eta, 1.f + g, 1.f));
    return ok;
}

// The same bounds over every pair of two groups of bodies at once.  A group
// is summarised by the boxes of its high parts (positions, velocities) and
// its largest G m.  Over pairs (i in A, j in B): r >= d = the boxes'
// distance (softened), |dv| <= vmax (the velocity boxes' widest relative
// speed), mu <= muA + muB.  Free fall: T_ff/h = etah sqrt(r^3/mu) grows with
// r and falls with mu, q = hq |dv|/r grows with |dv| and falls with r, so
// (T_ff/h)(1 - 0.75 q) >= 1 for every pair once it holds at (d, vmax,
// mu_max).  Flyby: with T_fb/h = etah r/v and |dT/dt| <= eta (1 + mu/(r
// v^2)), tau_fb/h >= f(r, v) = 2 etah r^2 v / ((2 + eta) r v^2 + eta mu),
// which grows with r and falls with mu; f >= 1 holds for v between the two
// roots v- < v+ of (2 + eta) d v^2 - 2 etah d^2 v + eta mu_max = 0.  Slow
// pairs fall below v- (approaching bodies with |dv| -> 0 have tau -> 0 in
// this form), so the groups are certified apart only for pairs with
// |dv| >= v-: the function returns true when every pair has tau_ff >= h
// and vmax <= v+, and sets vthr2 so that a pair whose high-part velocity
// difference has |dv~|^2 >= vthr2 is certified apart (vthr adds 16 u max|v|
// for the high parts' rounding and that of their difference: at most
// sqrt(3) (2 u max|v| + u |dv~|) <= 9.5 u max|v|).  pad_x, pad_v bound |x - x_hi| + |x' - x'_hi|
// over the two groups (likewise v); the 2 % margin M absorbs the FP32
// rounding of these few operations.
struct GroupBox {
    float xlo[3], xhi[3], vlo[3], vhi[3];
    float gm;    // max G m of the group (high part)
    float amax;  // max |x_hi| component
    float vabs;  // max |v_hi| component
};

__device__ __forceinline__ bool tau_groups_apart(const GroupBox &A, const GroupBox &B, const MixedTauParams &Q,
                                                 float &vthr2)
{
    const float M = 1.02f;
    const float pad_x = 4.f * U32 * fmaxf(A.amax, B.amax);
    const float pad_v = 4.f * U32 * fmaxf(A.vabs, B.vabs);
    float d2 = Q.eps2, w2 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float g = fmaxf(0.f, fmaxf(B.xlo[k] - A.xhi[k], A.xlo[k] - B.xhi[k]) - pad_x);
        const float w = fmaxf(0.f, fmaxf(B.vhi[k] - A.vlo[k], A.vhi[k] - B.vlo[k])) + pad_v;
        d2 = fmaf(g, g, d2);
        w2 = fmaf(w, w, w2);
    }
    const float d = sqrtf(d2), vmax = sqrtf(w2);
    const float mu = (A.gm + B.gm) * 1.0001f;
    if (!(d > 0.f) || !(mu > 0.f)) return false;
    // free fall at (d, vmax, mu_max)
    const float X = Q.etah * d * sqrtf(d / mu);
    const float q = Q.hq * vmax / d;
    if (!(X * (1.f - 0.75f * M * q) >= M)) return false;
    // flyby: roots of a v^2 - b v + c with the margin M on f >= 1
    const float a = M * (2.f + Q.eta) * d, b = 2.f * Q.etah * d2, c = M * Q.eta * mu;
    const float disc = b * b - 4.f * a * c;
    if (!(disc > 0.f)) return false;
    const float vp = (b + sqrtf(disc)) / (2.f * a);
    const float vm = c / (a * vp);  // the product of the roots is c/a
    if (!(vmax <= vp * 0.9999f)) return false;
    const float vt = vm * 1.0001f + 4.f * pad_v;
    vthr2 = vt * vt;
    return true;
}

__device__ __forceinline__ int tau_decide_fp32(float dx0, float dx1, float dx2, float dv0, float dv1, float dv2,
                                               float mu, float c_x, float c_v, const MixedTauParams &Q)
{
    return tau_decide_at(tau_prep_fp32(dx0, dx1, dx2, dv0, dv1, dv2, mu, c_x, c_v, Q), Q.etah);
}

// 2^k as a float (0 <= k <= 127); 2^-k as a double (0 <= k <= 1022)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }
__device__ __forceinline__ double pow2m(int k) { return __longlong_as_double((long long)(1023 - k) << 52); }

// x 2^-k for a normal x whose result stays normal: an exponent-field
// subtraction (exact, and no FP64 instruction)
__device__ __forceinline__ double scale2m(double x, int k)
{
    return __longlong_as_double(__double_as_longlong(x) - ((long long)k << 52));
}

// The first m >= 0 with h 2^-m <= tau (the first threshold of the sequence
// h, h/2, h/4, ... at which tau < threshold fails), at most `levels`.  h is
// positive and normal; the comparison is exact: (exponent, significand) of
// h 2^-m against those of tau.  NaN tau: 0 (the predicate is false).
__device__ __forceinline__ int first_level_at_or_below(double tau, double h, int levels)
{
    if (!(tau < h)) return 0;
    if (!(tau >= 2.2250738585072014e-308)) return levels;  // 0, negative or subnormal: below every threshold
    const long long bt = __double_as_longlong(tau), bh = __double_as_longlong(h);
    const int et = (int)(bt >> 52), eh = (int)(bh >> 52);
    const long long mt = bt & 0xFFFFFFFFFFFFFll, mh = bh & 0xFFFFFFFFFFFFFll;
    const int m = eh - et + (mh <= mt ? 0 : 1);
    return m < levels ? m : levels;
}

// Float-float split of a double: hi = fl32(x) (round to nearest even),
// lo = fl32(x - hi).  For |x| in [2^-74, 2^127) it is computed with integer
// operations and int->float conversions (the significand rounded to 24
// bits by integer arithmetic, the remainder converted exactly-then-rounded),
// giving the same two floats as the FP64 route at a fraction of its cost on
// a part whose FP64 pipe is 1/58 of the FP32 rate; outside that range it
// takes the FP64 route.
__device__ __forceinline__ void ff_split(double x, float &hi, float &lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFull);
    if (e < 949 || e > 1150) {
        hi = __double2float_rn(x);
        lo = __double2float_rn(x - (double)hi);
        return;
    }
    const long long F = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);  // 53-bit significand
    const long long Fr = (F + 0x0FFFFFFFll + ((F >> 29) & 1ll)) >> 29;             // 24 bits, nearest even
    const int d = (int)(F - (Fr << 29));                                           // |d| <= 2^28
    const float s_hi = __int_as_float((e - 1046 + 127) << 23);                     // 2^(e-1046)
    const float s_lo = __int_as_float((e - 1075 + 127) << 23);                     // 2^(e-1075)
    const float h = __int2float_rn((int)Fr) * s_hi;
    const float l = __int2float_rn(d) * s_lo;
    const bool neg = (b >> 63) != 0ull;
    hi = neg ? -h : h;
    lo = neg ? -l : l;
}

// fl32(x) = round-to-nearest-even double -> float, by integer arithmetic for
// results in the normal float range (same value as __double2float_rn); the
// conversion instruction costs ~180 cycles per warp on GB300.
__device__ __forceinline__ float fl32(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FFull);
    if (e < 1023 - 126 || e > 1023 + 126) return __double2float_rn(x);
    const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long r = mag + 0x0FFFFFFFull + ((mag >> 29) & 1ull);  // drop 29 bits, nearest even
    const unsigned int fb = (unsigned int)((r >> 29) - (896ull << 23)) | ((unsigned int)(b >> 32) & 0x80000000u);
    return __uint_as_float(fb);
}

// f2d(f) = the exact double of a float, by integer arithmetic for normal
// floats and zeros (the conversion instruction costs ~140 cycles per warp)
__device__ __forceinline__ double f2d(float f)
{
    const unsigned int u = __float_as_uint(f);
    const unsigned int ex = (u >> 23) & 0xFFu;
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
    if (ex == 0u || ex == 255u) return (double)f;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(ex + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

// one edge record at an atomically reserved slot (dropped past cap; the
// count still tells the host the list is incomplete)
__device__ __forceinline__ bool record_edge(const EdgeList &E, int a, int b, int e, double tau)
{
    const unsigned long long q = atomicAdd(E.count, 1ull);
    if ((long long)q >= E.cap) return false;
    {
        EdgeRec r;
        r.a = a;
        r.b = b;
        r.e = e;
        r.pad = 0;
        r.tau = tau;
        E.rec[q] = r;
    }
    return true;
}

// Kahan-compensated accumulation: s + (-c) carries the running sum
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// ------------------------------------------------------------ Kepler
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

// The same functions in FP32 (the starter of the iteration below), every
// operation an explicit IEEE one so that every translation unit computes
// the same starter (a contracted multiply-add would move it by an ulp, and
// the FP64 iteration's stopping point with it)
__device__ __forceinline__ void stumpff_f(float z, float &c2, float &c3)
{
    if (fabsf(z) < 0.1f) {
        float t2 = 0.5f, t3 = 1.0f / 6.0f;
        c2 = 0.0f;
        c3 = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            c2 = __fadd_rn(c2, t2);
            c3 = __fadd_rn(c3, t3);
            t2 = __fmul_rn(t2, __fdiv_rn(-z, (float)((2 * k + 3) * (2 * k + 4))));
            t3 = __fmul_rn(t3, __fdiv_rn(-z, (float)((2 * k + 4) * (2 * k + 5))));
        }
    } else if (z > 0.0f) {
        const float s = __fsqrt_rn(z);
        float sn, cs;
        sincosf(s, &sn, &cs);
        c2 = __fdiv_rn(__fsub_rn(1.0f, cs), z);
        c3 = __fdiv_rn(__fsub_rn(s, sn), __fmul_rn(z, s));
    } else {
        const float s = __fsqrt_rn(-z);
        c2 = __fdiv_rn(__fsub_rn(coshf(s), 1.0f), -z);
        c3 = __fdiv_rn(__fsub_rn(sinhf(s), s), __fmul_rn(-z, s));
    }
}

// Advance the relative orbit (r0, v0) under mu by dt; returns false when
// the iteration does not converge.  The Laguerre-Conway iteration runs in
// FP32 first (a GB300 FP64 instruction costs the pipe ~64 cycles, an FP32
// one ~4) until its step falls to a few FP32 ulps of chi; the FP64
// iteration then converges from there in one or two steps to the same
// FP64 criterion (and starts from the usual guess if the FP32 pass left no
// finite value).
__device__ __forceinline__ bool kepler_universal(const double r0[3], const double v0[3], double mu, double dt, double r1[3],
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
    {
        const float af = (float)alpha, a1f = (float)a1, a2f = (float)a2, r0f = (float)r0n;
        const float tf = (float)(smu * dt);
        float xf = (float)chi;
        bool ok32 = false;
        for (int it = 0; it < 60; ++it) {
            const float x2 = __fmul_rn(xf, xf), z = __fmul_rn(af, x2);
            float c2f, c3f;
            stumpff_f(z, c2f, c3f);
            const float zc3 = __fsub_rn(1.0f, __fmul_rn(z, c3f)), zc2 = __fsub_rn(1.0f, __fmul_rn(z, c2f));
            const float F = __fsub_rn(__fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(a1f, x2), c2f),
                                                          __fmul_rn(__fmul_rn(__fmul_rn(a2f, x2), xf), c3f)),
                                                __fmul_rn(r0f, xf)),
                                      tf);
            const float G1 = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(a1f, xf), zc3), __fmul_rn(__fmul_rn(a2f, x2), c2f)),
                                       r0f);
            const float G2 = __fadd_rn(__fmul_rn(a1f, zc2), __fmul_rn(__fmul_rn(a2f, xf), zc3));
            const float disc = __fsqrt_rn(fabsf(__fsub_rn(__fmul_rn(__fmul_rn(16.0f, G1), G1),
                                                          __fmul_rn(__fmul_rn(20.0f, F), G2))));
            const float den = __fadd_rn(G1, copysignf(disc, G1));
            const float d = (den != 0.0f) ? __fdiv_rn(__fmul_rn(5.0f, F), den) : __fdiv_rn(F, G1);
            xf = __fsub_rn(xf, d);
            if (!isfinite(xf)) break;
            if (fabsf(d) <= 4e-7f * fabsf(xf)) {
                ok32 = true;
                break;
            }
        }
        if (ok32) chi = (double)xf;
    }
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

// Two-body flow of particles a and b over dt (Eq. kepler, eps = 0): the
// centre of mass moves uniformly, the relative orbit r = x_a - x_b follows
// kepler_universal.  xa.. are updated in place; false if unconverged.
__device__ __forceinline__ bool kepler_pair(double ma, double mb, double xa[3], double xb[3], double va[3],
                                            double vb[3], double G, double dt)
{
    const double M = ma + mb;
    double r0[3], v0[3], xc[3], vc[3], r1[3], v1[3];
    for (int k = 0; k < 3; ++k) {
        xc[k] = (ma * xa[k] + mb * xb[k]) / M;
        vc[k] = (ma * va[k] + mb * vb[k]) / M;
        r0[k] = xa[k] - xb[k];
        v0[k] = va[k] - vb[k];
    }
    if (!kepler_universal(r0, v0, G * M, dt, r1, v1)) return false;
    for (int k = 0; k < 3; ++k) {
        const double xcn = xc[k] + vc[k] * dt;
        xa[k] = xcn + (mb / M) * r1[k];
        xb[k] = xcn - (ma / M) * r1[k];
        va[k] = vc[k] + (mb / M) * v1[k];
        vb[k] = vc[k] - (ma / M) * v1[k];
    }
    return true;
}

// Row ti and column offset of triangular tile t (tiles (ti, tj), tj >= ti,
// numbered row by row; row ti starts at ti nt - ti (ti - 1) / 2): the root of
// the quadratic in single precision, then exact integer corrections.
__device__ __forceinline__ int tri_tile_row(int &t, int nt)
{
    auto off = [nt](int x) { return x * nt - (x * (x - 1)) / 2; };
    const float b = 2.f * (float)nt + 1.f;
    int ti = (int)(0.5f * (b - sqrtf(fmaxf(b * b - 8.f * (float)t, 0.f))));
    ti = max(0, min(ti, nt - 1));
    while (ti > 0 && off(ti) > t) --ti;
    while (ti + 1 < nt && off(ti + 1) <= t) ++ti;
    t -= off(ti);
    return ti;
}

}  // namespace cc
