/*
 * cc_oracle.c -- plain FP64 oracle of the CC split integrator
 * (arXiv:1407.7105, Sec. 2).  TEST INFRASTRUCTURE ONLY: used by tests/,
 * __graft_entry__.smoke() and bench.py's CPU baseline; never by the CUDA
 * product path.  Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp].
 *
 * With OpenMP the loops over independent rows run in parallel: the tau
 * evaluations of one breadth-first scan (every unassigned member against
 * the popped one; the assignments are then made in ascending order, as the
 * serial scan makes them), the kick's rows (each row summed in ascending j
 * by one thread) and the drift's rows.  The arithmetic and its order are
 * those of the serial code, so the results are bit-identical for any
 * thread count (orc_set_threads(1) gives the serial oracle).
 *
 * Readings of the paper taken here (the GPU kernels implement the same ones):
 *  R1  tau_freefall / tau_flyby are not defined in the paper (it defers to
 *      Pelupessy et al. 2012).  From first principles, for the pair
 *      dx = x_i - x_j, dv = v_i - v_j, r^2 = |dx|^2 + eps^2, mu = G(m_i+m_j):
 *        T_ff  = eta * sqrt(r^3 / mu)              (free-fall time)
 *        T_fb  = eta * r / |dv|                    (flyby time, +inf if dv = 0)
 *        dT_ff/dt = 3/2 * T_ff * (dx.dv) / r^2
 *        dT_fb/dt = T_fb * (dx.dv)/r^2 * (1 + mu / (r |dv|^2))
 *      the last from differentiating r/|dv| with the pair's own relative
 *      acceleration -mu dx / r^3.
 *  R2  eta sits inside T and dT/dt (the approximately time-symmetric step
 *      T/(1 - T'/2) needs the derivative of the actual step); the literal
 *      placement, eta multiplying the min of Eq. (tauij), is selectable.
 *  R3  dT/dt is clamped at 1 before the denominator, so tau <= 2T > 0.
 *  R4  the edge test is strict: tau(i,j) < h (Sec. 2.2).
 *  R5  kick order: for each i of the set in ascending id, a_i is summed
 *      over j in ascending id, then v_i += h a_i.
 *
 * Exact operation order (no FMA, IEEE sqrt and division), for the pair:
 *   r2  = ((dx0*dx0 + dx1*dx1) + dx2*dx2) + eps2,  eps2 = eps*eps
 *   r   = sqrt(r2)
 *   v2  = (dv0*dv0 + dv1*dv1) + dv2*dv2
 *   rv  = (dx0*dv0 + dx1*dv1) + dx2*dv2
 *   mu  = G * (mi + mj)
 *   Tff = eta * sqrt((r2 * r) / mu)
 *   dTff = ((1.5 * Tff) * rv) / r2
 *   Tfb = eta * (r / sqrt(v2))                         (v2 > 0)
 *   dTfb = (Tfb * (rv / r2)) * (1.0 + mu / (r * v2))
 *   c(d) = d < 1.0 ? d : 1.0
 *   tau_ff = Tff / (1.0 - 0.5 * c(dTff)),  tau_fb likewise (+inf if v2 == 0)
 *   tau = tau_ff < tau_fb ? tau_ff : tau_fb
 */
#include "cc_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* sets smaller than this are scanned serially (a parallel region costs
 * more than the work) */
#define ORC_PAR_MIN 256

int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* tau(i,j), Eq. (tauij)                                               */
/* ------------------------------------------------------------------ */
static double clamp1(double d) { return d < 1.0 ? d : 1.0; }

double orc_tau(const double *xi, const double *vi, double mi,
               const double *xj, const double *vj, double mj,
               const orc_params *p, double *parts)
{
    double dx0 = xi[0] - xj[0], dx1 = xi[1] - xj[1], dx2 = xi[2] - xj[2];
    double dv0 = vi[0] - vj[0], dv1 = vi[1] - vj[1], dv2 = vi[2] - vj[2];
    double eps2 = p->eps * p->eps;
    double r2 = ((dx0 * dx0 + dx1 * dx1) + dx2 * dx2) + eps2;
    double r = sqrt(r2);
    double v2 = (dv0 * dv0 + dv1 * dv1) + dv2 * dv2;
    double rv = (dx0 * dv0 + dx1 * dv1) + dx2 * dv2;
    double mu = p->G * (mi + mj);
    double e_in = p->eta_outside ? 1.0 : p->eta;

    double Tff = e_in * sqrt((r2 * r) / mu);
    double dTff = ((1.5 * Tff) * rv) / r2;
    double tau_ff = Tff / (1.0 - 0.5 * clamp1(dTff));

    double Tfb = INFINITY, dTfb = 0.0, tau_fb = INFINITY;
    if (v2 > 0.0) {
        Tfb = e_in * (r / sqrt(v2));
        dTfb = (Tfb * (rv / r2)) * (1.0 + mu / (r * v2));
        tau_fb = Tfb / (1.0 - 0.5 * clamp1(dTfb));
    }
    double tau = tau_ff < tau_fb ? tau_ff : tau_fb;
    if (p->eta_outside) tau = p->eta * tau;
    if (parts) {
        parts[0] = Tff; parts[1] = dTff; parts[2] = Tfb;
        parts[3] = dTfb; parts[4] = tau_ff; parts[5] = tau_fb;
    }
    return tau;
}

double orc_tau_ids(int64_t n, const double *x3, const double *v3, const double *m,
                   const orc_params *p, int64_t i, int64_t j)
{
    /* evaluate with the smaller id first so tau(i,j) and tau(j,i) take the
     * same path (they are equal bitwise anyway: negation is exact) */
    if (j < i) { int64_t t = i; i = j; j = t; }
    double xi[3] = {x3[i], x3[n + i], x3[2 * n + i]};
    double xj[3] = {x3[j], x3[n + j], x3[2 * n + j]};
    double vi[3] = {v3[i], v3[n + i], v3[2 * n + i]};
    double vj[3] = {v3[j], v3[n + j], v3[2 * n + j]};
    return orc_tau(xi, vi, m[i], xj, vj, m[j], p, NULL);
}

/* ------------------------------------------------------------------ */
/* split_cc: breadth-first search over lazily evaluated tau (Sec. 2.3)  */
/* ------------------------------------------------------------------ */
int64_t orc_components(int64_t n, const double *x3, const double *v3, const double *m,
                       const orc_params *p, const int32_t *set, int64_t nset,
                       double h, int32_t *labels_out, orc_stats *st)
{
    if (nset < 0) return ORC_E_ARG;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (nset > 0 ? nset : 1));
    char *assigned = (char *)calloc(nset > 0 ? nset : 1, 1);
    char *hit = (char *)calloc(nset > 0 ? nset : 1, 1);
    int64_t ncomp = 0;
    if (st) {
        st->splits++;
        st->tau_pairs += (uint64_t)(nset * (nset - 1) / 2);
    }
    /* seeds are taken in ascending id, so every member found from a seed
     * has a larger id and the seed id is the smallest id of the component */
    for (int64_t s = 0; s < nset; ++s) {
        if (assigned[s]) continue;
        assigned[s] = 1;
        labels_out[s] = set[s];
        int64_t qh = 0, qt = 0, size = 1;
        queue[qt++] = s;
        while (qh < qt) {
            int64_t X = queue[qh++];
            /* assign to X's component every unassigned U with tau(X,U) < h:
             * the tests first (independent), then the assignments in
             * ascending U */
            uint64_t evals = 0;
#pragma omp parallel for schedule(static) reduction(+ : evals) if (nset >= ORC_PAR_MIN)
            for (int64_t U = 0; U < nset; ++U) {
                hit[U] = 0;
                if (assigned[U]) continue;
                double t = orc_tau_ids(n, x3, v3, m, p, set[X], set[U]);
                evals++;
                hit[U] = t < h;
            }
            if (st) st->tau_evals += evals;
            for (int64_t U = 0; U < nset; ++U) {
                if (hit[U]) {
                    assigned[U] = 1;
                    labels_out[U] = set[s];
                    queue[qt++] = U;
                    size++;
                }
            }
        }
        if (size >= 2) ncomp++;
    }
    if (st) st->components += (uint64_t)ncomp;
    free(queue);
    free(assigned);
    free(hit);
    return ncomp;
}

int64_t orc_edges(int64_t n, const double *x3, const double *v3, const double *m,
                  const orc_params *p, const int32_t *set, int64_t nset, double h,
                  int32_t *edges_out, int64_t cap, double near_tol, int64_t *n_near)
{
    int64_t ne = 0, nn = 0;
    for (int64_t a = 0; a < nset; ++a) {
        for (int64_t b = a + 1; b < nset; ++b) {
            double t = orc_tau_ids(n, x3, v3, m, p, set[a], set[b]);
            if (fabs(t - h) < near_tol * h) nn++;
            if (t < h) {
                if (ne < cap && edges_out) {
                    int32_t i = set[a], j = set[b];
                    edges_out[2 * ne] = i < j ? i : j;
                    edges_out[2 * ne + 1] = i < j ? j : i;
                }
                ne++;
            }
        }
    }
    if (n_near) *n_near = nn;
    return ne;
}

/* ------------------------------------------------------------------ */
/* kick and drift (Eqs. drift, kickij, kickji)                          */
/* ------------------------------------------------------------------ */
static int cmp_i32_any(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void orc_kick(int64_t n, const double *x3, double *v3, const double *m,
              const orc_params *p, const int32_t *set, const int32_t *labels,
              int64_t nset, double h, orc_stats *st)
{
    double eps2 = p->eps * p->eps;
    double *acc = (double *)calloc((size_t)(3 * (nset > 0 ? nset : 1)), sizeof(double));
    uint64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs) if (nset >= ORC_PAR_MIN)
    for (int64_t a = 0; a < nset; ++a) {
        int64_t i = set[a];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t b = 0; b < nset; ++b) {
            if (b == a || labels[b] == labels[a]) continue;
            int64_t j = set[b];
            if (b > a) pairs++;
            double dx0 = x3[j] - x3[i];
            double dx1 = x3[n + j] - x3[n + i];
            double dx2 = x3[2 * n + j] - x3[2 * n + i];
            double r2 = ((dx0 * dx0 + dx1 * dx1) + dx2 * dx2) + eps2;
            double rinv3 = 1.0 / (r2 * sqrt(r2));
            double w = (p->G * m[j]) * rinv3;
            ax = ax + w * dx0;
            ay = ay + w * dx1;
            az = az + w * dx2;
        }
        acc[3 * a] = ax; acc[3 * a + 1] = ay; acc[3 * a + 2] = az;
    }
    for (int64_t a = 0; a < nset; ++a) {
        int64_t i = set[a];
        v3[i] = v3[i] + h * acc[3 * a];
        v3[n + i] = v3[n + i] + h * acc[3 * a + 1];
        v3[2 * n + i] = v3[2 * n + i] + h * acc[3 * a + 2];
    }
    if (st) st->kick_pairs += pairs;
    free(acc);
}

/* centre-of-mass approximation of V_CC (Sec. 4.1, Discussion) */
void orc_kick_com(int64_t n, const double *x3, double *v3, const double *m,
                  const orc_params *p, const int32_t *set, const int32_t *labels,
                  int64_t nset, double h, orc_stats *st)
{
    if (!(p->theta > 0.0) || nset < 2) {
        orc_kick(n, x3, v3, m, p, set, labels, nset, h, st);
        return;
    }
    /* the eligible components in ascending label: a sorted copy of the labels */
    int32_t *srt = (int32_t *)malloc(sizeof(int32_t) * nset);
    memcpy(srt, labels, sizeof(int32_t) * nset);
    qsort(srt, nset, sizeof(int32_t), cmp_i32_any);
    int64_t ke = 0;
    int32_t *elab = (int32_t *)malloc(sizeof(int32_t) * nset);
    for (int64_t a = 0; a < nset;) {
        int64_t b = a;
        while (b < nset && srt[b] == srt[a]) b++;
        if (b - a >= 2 && b - a <= p->com_max) elab[ke++] = srt[a];
        a = b;
    }
    free(srt);
    /* comp[k] = the eligible component of set[k], or -1 */
    int64_t *comp = (int64_t *)malloc(sizeof(int64_t) * nset);
    for (int64_t k = 0; k < nset; ++k) {
        comp[k] = -1;
        for (int64_t e = 0; e < ke; ++e)
            if (labels[k] == elab[e]) {
                comp[k] = e;
                break;
            }
    }
    double *cm = (double *)calloc((size_t)(ke > 0 ? ke : 1) * 5, sizeof(double)); /* M, X, Y, Z, R */
    for (int64_t e = 0; e < ke; ++e) {
        double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int64_t k = 0; k < nset; ++k) {
            if (comp[k] != e) continue;
            int64_t i = set[k];
            M = M + m[i];
            sx = sx + m[i] * x3[i];
            sy = sy + m[i] * x3[n + i];
            sz = sz + m[i] * x3[2 * n + i];
        }
        double X = sx / M, Y = sy / M, Z = sz / M, R = 0.0;
        for (int64_t k = 0; k < nset; ++k) {
            if (comp[k] != e) continue;
            int64_t i = set[k];
            double dx = x3[i] - X, dy = x3[n + i] - Y, dz = x3[2 * n + i] - Z;
            double r = sqrt((dx * dx + dy * dy) + dz * dz);
            if (r > R) R = r;
        }
        cm[5 * e] = M; cm[5 * e + 1] = X; cm[5 * e + 2] = Y; cm[5 * e + 3] = Z; cm[5 * e + 4] = R;
    }
    /* far[a*ke + b]: R_a + R_b < theta |X_a - X_b| */
    char *far = (char *)calloc((size_t)(ke > 0 ? ke * ke : 1), 1);
    for (int64_t a = 0; a < ke; ++a)
        for (int64_t b = 0; b < ke; ++b) {
            if (a == b) continue;
            double dx = cm[5 * b + 1] - cm[5 * a + 1], dy = cm[5 * b + 2] - cm[5 * a + 2];
            double dz = cm[5 * b + 3] - cm[5 * a + 3];
            double d = sqrt((dx * dx + dy * dy) + dz * dz);
            far[a * ke + b] = (cm[5 * a + 4] + cm[5 * b + 4]) < p->theta * d;
        }
    /* 1. exact pairs, the far ones left out (orc_kick's arithmetic) */
    double eps2 = p->eps * p->eps;
    double *acc = (double *)calloc((size_t)(3 * nset), sizeof(double));
    uint64_t pairs = 0, cpairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs, cpairs) if (nset >= ORC_PAR_MIN)
    for (int64_t a = 0; a < nset; ++a) {
        int64_t i = set[a];
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t b = 0; b < nset; ++b) {
            if (b == a || labels[b] == labels[a]) continue;
            if (comp[a] >= 0 && comp[b] >= 0 && far[comp[a] * ke + comp[b]]) {
                if (b > a) cpairs++;
                continue;
            }
            int64_t j = set[b];
            if (b > a) pairs++;
            double dx0 = x3[j] - x3[i];
            double dx1 = x3[n + j] - x3[n + i];
            double dx2 = x3[2 * n + j] - x3[2 * n + i];
            double r2 = ((dx0 * dx0 + dx1 * dx1) + dx2 * dx2) + eps2;
            double rinv3 = 1.0 / (r2 * sqrt(r2));
            double w = (p->G * m[j]) * rinv3;
            ax = ax + w * dx0;
            ay = ay + w * dx1;
            az = az + w * dx2;
        }
        acc[3 * a] = ax; acc[3 * a + 1] = ay; acc[3 * a + 2] = az;
    }
    for (int64_t a = 0; a < nset; ++a) {
        int64_t i = set[a];
        v3[i] = v3[i] + h * acc[3 * a];
        v3[n + i] = v3[n + i] + h * acc[3 * a + 1];
        v3[2 * n + i] = v3[2 * n + i] + h * acc[3 * a + 2];
    }
    /* 2. the monopole of every far component */
    for (int64_t a = 0; a < ke; ++a) {
        double Ax = 0.0, Ay = 0.0, Az = 0.0;
        int any = 0;
        for (int64_t b = 0; b < ke; ++b) {
            if (!far[a * ke + b]) continue;
            any = 1;
            double dx0 = cm[5 * b + 1] - cm[5 * a + 1];
            double dx1 = cm[5 * b + 2] - cm[5 * a + 2];
            double dx2 = cm[5 * b + 3] - cm[5 * a + 3];
            double d2 = ((dx0 * dx0 + dx1 * dx1) + dx2 * dx2) + eps2;
            double w = (p->G * cm[5 * b]) * (1.0 / (d2 * sqrt(d2)));
            Ax = Ax + w * dx0;
            Ay = Ay + w * dx1;
            Az = Az + w * dx2;
        }
        if (!any) continue;
        for (int64_t k = 0; k < nset; ++k) {
            if (comp[k] != a) continue;
            int64_t i = set[k];
            v3[i] = v3[i] + h * Ax;
            v3[n + i] = v3[n + i] + h * Ay;
            v3[2 * n + i] = v3[2 * n + i] + h * Az;
        }
    }
    if (st) {
        st->kick_pairs += pairs;
        st->com_pairs += cpairs;
    }
    free(acc);
    free(far);
    free(cm);
    free(comp);
    free(elab);
}

void orc_drift(int64_t n, double *x3, const double *v3,
               const int32_t *set, const int32_t *labels, int64_t nset,
               double dt, orc_stats *st)
{
    uint64_t drifts = 0;
#pragma omp parallel for schedule(static) reduction(+ : drifts) if (nset >= ORC_PAR_MIN)
    for (int64_t a = 0; a < nset; ++a) {
        /* a label shared with any other member marks a component member */
        int single = 1;
        for (int64_t b = 0; b < nset && single; ++b)
            if (b != a && labels[b] == labels[a]) single = 0;
        if (!single) continue;
        int64_t i = set[a];
        x3[i] = x3[i] + dt * v3[i];
        x3[n + i] = x3[n + i] + dt * v3[n + i];
        x3[2 * n + i] = x3[2 * n + i] + dt * v3[2 * n + i];
        drifts++;
    }
    if (st) st->drifts += drifts;
}

/* ------------------------------------------------------------------ */
/* Two-body flow (Eq. kepler, eps = 0) by the classical Kepler equation */
/* in difference form: eccentric anomaly for bound orbits, hyperbolic   */
/* anomaly for unbound ones, Barker's cubic for the exact parabola.     */
/* ------------------------------------------------------------------ */
/* x - sin x and sinh x - x without cancellation for small |x| */
static double x_minus_sin(double x)
{
    if (fabs(x) > 0.5) return x - sin(x);
    double x2 = x * x, term = x * x2 / 6.0, s = 0.0;
    for (int k = 1; k < 30 && term != 0.0; ++k) {
        s += term;
        term = -term * x2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    }
    return s;
}
static double sinh_minus_x(double x)
{
    if (fabs(x) > 0.5) return sinh(x) - x;
    double x2 = x * x, term = x * x2 / 6.0, s = 0.0;
    for (int k = 1; k < 30 && term != 0.0; ++k) {
        s += term;
        term = term * x2 / ((2.0 * k + 2.0) * (2.0 * k + 3.0));
    }
    return s;
}

/* safeguarded Newton on an increasing function on [lo, hi] */
typedef double (*fn_t)(double x, const double *c, double *df);
static int solve_increasing(fn_t f, const double *c, double lo, double hi,
                            double x0, double *root)
{
    double x = x0;
    if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        double df, fx = f(x, c, &df);
        if (fx == 0.0) { *root = x; return 0; }
        if (fx < 0.0) lo = x; else hi = x;
        double xn = x - fx / df;
        if (!(xn > lo && xn < hi) || !isfinite(xn)) xn = 0.5 * (lo + hi);
        double step = fabs(xn - x);
        x = xn;
        if (step <= 2e-16 * fabs(x) || hi - lo <= 2e-16 * fabs(x) || step == 0.0) {
            /* one polishing Newton step from the converged point */
            fx = f(x, c, &df);
            xn = x - fx / df;
            if (xn >= lo && xn <= hi && isfinite(xn)) x = xn;
            *root = x;
            return 0;
        }
    }
    *root = x;
    return -1;
}

/* c = {r0a, es, ndt}:  (x - sin x) + r0a sin x + es (1 - cos x) - ndt */
static double f_ell(double x, const double *c, double *df)
{
    double s = sin(x), hs = sin(0.5 * x), omc = 2.0 * hs * hs;
    *df = omc + c[0] * cos(x) + c[1] * s;
    return x_minus_sin(x) + c[0] * s + c[1] * omc - c[2];
}
/* c = {r0b, es, ndt}:  (sinh x - x) + r0b sinh x + es (cosh x - 1) - ndt */
static double f_hyp(double x, const double *c, double *df)
{
    double s = sinh(x), hs = sinh(0.5 * x), cm1 = 2.0 * hs * hs;
    *df = cm1 + c[0] * cosh(x) + c[1] * s;
    return sinh_minus_x(x) + c[0] * s + c[1] * cm1 - c[2];
}
/* c = {r0, sig = sigma/sqrt(mu), sqmu*dt}: Barker's equation in chi */
static double f_par(double x, const double *c, double *df)
{
    *df = c[0] + c[1] * x + 0.5 * x * x;
    return c[0] * x + 0.5 * c[1] * x * x + x * x * x / 6.0 - c[2];
}

int orc_kepler(int64_t n, double *x3, double *v3, const double *m,
               double G, int64_t i, int64_t j, double dt)
{
    double mi = m[i], mj = m[j], M = mi + mj, mu = G * M;
    double xc[3], vc[3], r0[3], v0[3];
    for (int k = 0; k < 3; ++k) {
        double xi = x3[k * n + i], xj = x3[k * n + j];
        double vi = v3[k * n + i], vj = v3[k * n + j];
        xc[k] = (mi * xi + mj * xj) / M;
        vc[k] = (mi * vi + mj * vj) / M;
        r0[k] = xi - xj;
        v0[k] = vi - vj;
    }
    double r0n = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    double vv = v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2];
    double sig = r0[0] * v0[0] + r0[1] * v0[1] + r0[2] * v0[2];
    double alpha = 2.0 / r0n - vv / mu; /* 1/a */
    double f, g, fd, gd;
    if (!(r0n > 0.0) || !(mu > 0.0) || !isfinite(alpha)) return ORC_E_KEPLER;
    if (dt == 0.0) {
        f = 1.0; g = 0.0; fd = 0.0; gd = 1.0;
    } else if (alpha > 0.0) {
        double a = 1.0 / alpha, nmm = sqrt(mu / (a * a * a));
        double c[3] = {r0n / a, sig / sqrt(mu * a), nmm * dt};
        double x;
        if (solve_increasing(f_ell, c, c[2] - 3.0, c[2] + 3.0, c[2], &x)) return ORC_E_KEPLER;
        double s = sin(x), hs = sin(0.5 * x), omc = 2.0 * hs * hs;
        double r = a * omc + r0n * cos(x) + a * c[1] * s;
        f = 1.0 - (a / r0n) * omc;
        g = dt - x_minus_sin(x) / nmm;
        fd = -sqrt(mu * a) * s / (r * r0n);
        gd = 1.0 - (a / r) * omc;
    } else if (alpha < 0.0) {
        double b = -1.0 / alpha, nmm = sqrt(mu / (b * b * b));
        double c[3] = {r0n / b, sig / sqrt(mu * b), nmm * dt};
        double lo = 0.0, hi = 1.0;
        if (dt < 0.0) { lo = -1.0; hi = 0.0; }
        double dfd;
        while (f_hyp(hi, c, &dfd) < 0.0) { lo = hi; hi *= 2.0; if (hi > 1e4) return ORC_E_KEPLER; }
        while (f_hyp(lo, c, &dfd) > 0.0) { hi = lo; lo *= 2.0; if (lo < -1e4) return ORC_E_KEPLER; }
        double x;
        if (solve_increasing(f_hyp, c, lo, hi, 0.5 * (lo + hi), &x)) return ORC_E_KEPLER;
        double s = sinh(x), hs = sinh(0.5 * x), cm1 = 2.0 * hs * hs;
        double r = b * cm1 + r0n * cosh(x) + b * c[1] * s;
        f = 1.0 - (b / r0n) * cm1;
        g = dt - sinh_minus_x(x) / nmm;
        fd = -sqrt(mu * b) * s / (r * r0n);
        gd = 1.0 - (b / r) * cm1;
    } else {
        double sqmu = sqrt(mu);
        double c[3] = {r0n, sig / sqmu, sqmu * dt};
        double lo = 0.0, hi = 1.0, dfd;
        if (dt < 0.0) { lo = -1.0; hi = 0.0; }
        while (f_par(hi, c, &dfd) < 0.0) { lo = hi; hi *= 2.0; }
        while (f_par(lo, c, &dfd) > 0.0) { hi = lo; lo *= 2.0; }
        double x;
        if (solve_increasing(f_par, c, lo, hi, 0.5 * (lo + hi), &x)) return ORC_E_KEPLER;
        double r = r0n + c[1] * x + 0.5 * x * x;
        f = 1.0 - x * x / (2.0 * r0n);
        g = dt - x * x * x / (6.0 * sqmu);
        fd = -sqmu * x / (r * r0n);
        gd = 1.0 - x * x / (2.0 * r);
    }
    for (int k = 0; k < 3; ++k) {
        double r1 = f * r0[k] + g * v0[k];
        double v1 = fd * r0[k] + gd * v0[k];
        double xcn = xc[k] + vc[k] * dt;
        x3[k * n + i] = xcn + (mj / M) * r1;
        x3[k * n + j] = xcn - (mi / M) * r1;
        v3[k * n + i] = vc[k] + (mj / M) * v1;
        v3[k * n + j] = vc[k] - (mi / M) * v1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* evolve_cc (CC pseudocode figure, Sec. 2.3)                           */
/* ------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int orc_evolve_cc(int64_t n, double *x3, double *v3, const double *m,
                  const orc_params *p, const int32_t *set, int64_t nset,
                  double h, int depth, orc_stats *st)
{
    if (depth > p->max_depth) return ORC_E_DEPTH;
    if (st && depth > st->max_depth_seen) st->max_depth_seen = depth;
    int32_t *labels = (int32_t *)malloc(sizeof(int32_t) * (nset > 0 ? nset : 1));
    /* 1) split_cc: C_1..C_K and R */
    int64_t K = orc_components(n, x3, v3, m, p, set, nset, h, labels, st);
    int rc = ORC_OK;
    /* gather each C_i as an ascending id list, components in ascending label */
    int32_t *members = NULL, *coff = NULL;
    int64_t nc = 0;
    if (K > 0) {
        members = (int32_t *)malloc(sizeof(int32_t) * nset);
        coff = (int32_t *)malloc(sizeof(int32_t) * (K + 1));
        int32_t *lab_sorted = (int32_t *)malloc(sizeof(int32_t) * nset);
        memcpy(lab_sorted, labels, sizeof(int32_t) * nset);
        qsort(lab_sorted, nset, sizeof(int32_t), cmp_i32);
        int64_t pos = 0;
        for (int64_t a = 0; a < nset;) {
            int64_t b = a;
            while (b < nset && lab_sorted[b] == lab_sorted[a]) b++;
            if (b - a >= 2) {
                coff[nc] = (int32_t)pos;
                for (int64_t k = 0; k < nset; ++k)
                    if (labels[k] == lab_sorted[a]) members[pos++] = set[k];
                nc++;
            }
            a = b;
        }
        coff[nc] = (int32_t)pos;
        free(lab_sorted);
    }
    /* 2) + 6) evolve every C_i at h/2 (Kepler for two-body C_i in CC_KEPLER);
     * the second pass re-enters the same C_i, which re-split themselves */
    for (int pass = 0; pass < 2 && rc == ORC_OK; ++pass) {
        if (pass == 1) {
            /* 3)-5) D_{h/2,T_R} K_{h,V_R+V_CC+V_CR} D_{h/2,T_R} */
            orc_drift(n, x3, v3, set, labels, nset, 0.5 * h, st);
            /* the centre-of-mass approximation applies in sets of at least 33 */
            if (nset >= 33)
                orc_kick_com(n, x3, v3, m, p, set, labels, nset, h, st);
            else
                orc_kick(n, x3, v3, m, p, set, labels, nset, h, st);
            orc_drift(n, x3, v3, set, labels, nset, 0.5 * h, st);
        }
        for (int64_t c = 0; c < nc && rc == ORC_OK; ++c) {
            const int32_t *cs = members + coff[c];
            int64_t cn = coff[c + 1] - coff[c];
            if (p->kepler && cn == 2) {
                rc = orc_kepler(n, x3, v3, m, p->G, cs[0], cs[1], 0.5 * h);
                if (st) st->kepler_calls++;
            } else {
                rc = orc_evolve_cc(n, x3, v3, m, p, cs, cn, 0.5 * h, depth + 1, st);
            }
        }
    }
    free(labels);
    free(members);
    free(coff);
    return rc;
}

/* ------------------------------------------------------------------ */
/* the HOLD split and evolve_hold (Sec. 2.1, Eq. HOLD)                  */
/* ------------------------------------------------------------------ */
int64_t orc_hold_split(int64_t n, const double *x3, const double *v3, const double *m,
                       const orc_params *p, const int32_t *set, int64_t nset,
                       double h, int32_t *labels_out, orc_stats *st)
{
    if (nset < 0) return ORC_E_ARG;
    double *tmin = (double *)malloc(sizeof(double) * (nset > 0 ? nset : 1));
    /* tau(i) = min over j != i of tau(i,j): a row minimum per member (tau is
     * symmetric bit for bit, so each row holds the pair's one value) */
#pragma omp parallel for schedule(dynamic, 16) if (nset >= ORC_PAR_MIN)
    for (int64_t a = 0; a < nset; ++a) {
        double t = INFINITY;
        for (int64_t b = 0; b < nset; ++b) {
            if (b == a) continue;
            double tab = orc_tau_ids(n, x3, v3, m, p, set[a], set[b]);
            if (tab < t) t = tab;
        }
        tmin[a] = t;
    }
    int32_t fmin = 0;
    int64_t nf = 0;
    for (int64_t a = 0; a < nset; ++a)
        if (tmin[a] < h) {
            if (nf == 0 || set[a] < fmin) fmin = set[a];
            nf++;
        }
    for (int64_t a = 0; a < nset; ++a) labels_out[a] = tmin[a] < h ? fmin : set[a];
    if (st) {
        st->splits++;
        st->tau_pairs += (uint64_t)(nset * (nset - 1) / 2);
        st->tau_evals += (uint64_t)(nset * (nset - 1) / 2);
        if (nf >= 2) st->components++;
    }
    free(tmin);
    return nf >= 2 ? 1 : 0;
}

int orc_evolve_hold(int64_t n, double *x3, double *v3, const double *m,
                    const orc_params *p, const int32_t *set, int64_t nset,
                    double h, int depth, orc_stats *st)
{
    if (depth > p->max_depth) return ORC_E_DEPTH;
    if (st && depth > st->max_depth_seen) st->max_depth_seen = depth;
    int32_t *labels = (int32_t *)malloc(sizeof(int32_t) * (nset > 0 ? nset : 1));
    int32_t *fast = (int32_t *)malloc(sizeof(int32_t) * (nset > 0 ? nset : 1));
    /* S and F at h: F is labelled with its smallest id, so a member whose
     * label is not its own id names F's label */
    const int64_t K = orc_hold_split(n, x3, v3, m, p, set, nset, h, labels, st);
    int32_t lf = -1;
    for (int64_t a = 0; a < nset && K; ++a)
        if (labels[a] != set[a]) {
            lf = labels[a];
            break;
        }
    int64_t nf = 0;
    for (int64_t a = 0; a < nset && K; ++a)
        if (labels[a] == lf) fast[nf++] = set[a];
    int rc = ORC_OK;
    for (int pass = 0; pass < 2 && rc == ORC_OK; ++pass) {
        if (pass == 1) {
            /* E_{h,H_S+V_SF} = D_{h/2,T_S} K_{h,V_S+V_SF} D_{h/2,T_S}: the
             * drift moves the members whose label no other member shares (S),
             * the kick every pair whose labels differ (not both in F) */
            orc_drift(n, x3, v3, set, labels, nset, 0.5 * h, st);
            orc_kick(n, x3, v3, m, p, set, labels, nset, h, st);
            orc_drift(n, x3, v3, set, labels, nset, 0.5 * h, st);
        }
        /* E_{h/2,H_F}: the same split, recursively, at pivot h/2 */
        if (nf >= 2) rc = orc_evolve_hold(n, x3, v3, m, p, fast, nf, 0.5 * h, depth + 1, st);
    }
    free(labels);
    free(fast);
    return rc;
}

/* ------------------------------------------------------------------ */
/* the OK split (Sec. 4.2): interactions partitioned by tau(i,j)        */
/* ------------------------------------------------------------------ */
/* Reading (R15): as HOLD partitions the particles of a set, the OK split
 * partitions its interactions.  The interaction list I of a particle set S
 * (at the outer step: every pair of S) splits at pivot h into the fast list
 * I_F = {(i,j) in I : tau(i,j) < h} and the slow list I_S = I \ I_F; F is the
 * set of particles of I_F.  With H_F = T_F + V_{I_F} and H_S = T_{S\F} +
 * V_{I_S}, one step is
 *     E_{h/2,H_F} D_{h/2,T_{S\F}} K_{h,V_{I_S}} D_{h/2,T_{S\F}} E_{h/2,H_F},
 * E_{h/2,H_F} = evolve_ok(F, I_F, h/2), the same split at half the pivot.
 * Every slow interaction is kicked at the pivot of the level where tau
 * first fails the threshold: the power of two at or below tau(i,j).
 * Pair lists hold (a, b), a < b particle ids, sorted by (a, b).  Kick order
 * (R5): a_i sums its slow partners j in ascending id. */

/* the pair term of body i from body j, orc_kick's arithmetic */
static inline void pair_term(int64_t n, const double *x3, const double *m, double G, double eps2,
                             int64_t i, int64_t j, double *ax, double *ay, double *az)
{
    double dx0 = x3[j] - x3[i];
    double dx1 = x3[n + j] - x3[n + i];
    double dx2 = x3[2 * n + j] - x3[2 * n + i];
    double r2 = ((dx0 * dx0 + dx1 * dx1) + dx2 * dx2) + eps2;
    double rinv3 = 1.0 / (r2 * sqrt(r2));
    double w = (G * m[j]) * rinv3;
    *ax = *ax + w * dx0;
    *ay = *ay + w * dx1;
    *az = *az + w * dx2;
}

static int cmp_pair(const void *x, const void *y)
{
    const int32_t *a = (const int32_t *)x, *b = (const int32_t *)y;
    if (a[0] != b[0]) return (a[0] > b[0]) - (a[0] < b[0]);
    return (a[1] > b[1]) - (a[1] < b[1]);
}

/* both directions (i, j) and (j, i) of each pair, sorted by (i, j) */
static int32_t *directed(const int32_t *pairs, int64_t np)
{
    int32_t *d = (int32_t *)malloc(sizeof(int32_t) * 4 * (np > 0 ? np : 1));
    for (int64_t k = 0; k < np; ++k) {
        d[4 * k] = pairs[2 * k];
        d[4 * k + 1] = pairs[2 * k + 1];
        d[4 * k + 2] = pairs[2 * k + 1];
        d[4 * k + 3] = pairs[2 * k];
    }
    qsort(d, (size_t)(2 * np), 2 * sizeof(int32_t), cmp_pair);
    return d;
}

int orc_evolve_ok(int64_t n, double *x3, double *v3, const double *m,
                  const orc_params *p, const int32_t *set, int64_t nset,
                  const int32_t *pairs, int64_t npairs, double h, int depth, orc_stats *st)
{
    if (depth > p->max_depth) return ORC_E_DEPTH;
    if (st && depth > st->max_depth_seen) st->max_depth_seen = depth;
    const double eps2 = p->eps * p->eps;
    const int all = pairs == NULL;
    const int64_t ni = all ? nset * (nset - 1) / 2 : npairs;
    /* 1) the fast list (in the order of I: sorted) and the slow count */
    int64_t cap = 16, nf = 0;
    int32_t *fast = (int32_t *)malloc(sizeof(int32_t) * 2 * cap);
    if (all) {
        for (int64_t a = 0; a < nset; ++a)
            for (int64_t b = a + 1; b < nset; ++b)
                if (orc_tau_ids(n, x3, v3, m, p, set[a], set[b]) < h) {
                    if (nf == cap) {
                        cap *= 2;
                        fast = (int32_t *)realloc(fast, sizeof(int32_t) * 2 * cap);
                    }
                    fast[2 * nf] = set[a];
                    fast[2 * nf + 1] = set[b];
                    nf++;
                }
    } else {
        for (int64_t k = 0; k < npairs; ++k)
            if (orc_tau_ids(n, x3, v3, m, p, pairs[2 * k], pairs[2 * k + 1]) < h) {
                if (nf == cap) {
                    cap *= 2;
                    fast = (int32_t *)realloc(fast, sizeof(int32_t) * 2 * cap);
                }
                fast[2 * nf] = pairs[2 * k];
                fast[2 * nf + 1] = pairs[2 * k + 1];
                nf++;
            }
    }
    if (st) {
        st->splits++;
        st->tau_pairs += (uint64_t)ni;
        st->tau_evals += (uint64_t)ni;
        if (nf > 0) st->components++;
    }
    /* F: the particles of the fast list, ascending */
    int32_t *F = (int32_t *)malloc(sizeof(int32_t) * (2 * nf > 0 ? 2 * nf : 1));
    for (int64_t k = 0; k < 2 * nf; ++k) F[k] = fast[k];
    qsort(F, (size_t)(2 * nf), sizeof(int32_t), cmp_i32);
    int64_t nF = 0;
    for (int64_t k = 0; k < 2 * nf; ++k)
        if (nF == 0 || F[nF - 1] != F[k]) F[nF++] = F[k];
    /* the fast partners of every particle, for the slow kick */
    int32_t *fd = directed(fast, nf);
    /* the slow list when I is explicit */
    int32_t *slow = NULL;
    int64_t ns = 0;
    if (!all) {
        slow = (int32_t *)malloc(sizeof(int32_t) * 2 * (npairs - nf > 0 ? npairs - nf : 1));
        int64_t kf = 0;
        for (int64_t k = 0; k < npairs; ++k) {
            if (kf < nf && fast[2 * kf] == pairs[2 * k] && fast[2 * kf + 1] == pairs[2 * k + 1]) {
                kf++;
                continue;
            }
            slow[2 * ns] = pairs[2 * k];
            slow[2 * ns + 1] = pairs[2 * k + 1];
            ns++;
        }
    }
    int rc = ORC_OK;
    for (int pass = 0; pass < 2 && rc == ORC_OK; ++pass) {
        if (pass == 1) {
            /* D_{h/2,T_{S\F}} K_{h,V_{I_S}} D_{h/2,T_{S\F}} */
            for (int half = 0; half < 2; ++half) {
                if (half == 1) {
                    double *acc = (double *)calloc((size_t)(3 * (nset > 0 ? nset : 1)), sizeof(double));
                    if (all) {
                        /* every pair of the set but the fast ones */
                        int64_t q = 0;
                        for (int64_t a = 0; a < nset; ++a) {
                            const int64_t i = set[a];
                            while (q < 2 * nf && fd[2 * q] < i) q++;
                            int64_t r = q;
                            double ax = 0.0, ay = 0.0, az = 0.0;
                            for (int64_t b = 0; b < nset; ++b) {
                                const int64_t j = set[b];
                                if (j == i) continue;
                                while (r < 2 * nf && fd[2 * r] == i && fd[2 * r + 1] < j) r++;
                                if (r < 2 * nf && fd[2 * r] == i && fd[2 * r + 1] == j) continue;
                                pair_term(n, x3, m, p->G, eps2, i, j, &ax, &ay, &az);
                            }
                            acc[3 * a] = ax; acc[3 * a + 1] = ay; acc[3 * a + 2] = az;
                        }
                        if (st) st->kick_pairs += (uint64_t)(ni - nf);
                    } else {
                        /* the slow partners of each member, ascending */
                        int32_t *sd = directed(slow, ns);
                        int64_t q = 0;
                        for (int64_t a = 0; a < nset; ++a) {
                            const int64_t i = set[a];
                            while (q < 2 * ns && sd[2 * q] < i) q++;
                            double ax = 0.0, ay = 0.0, az = 0.0;
                            for (int64_t r = q; r < 2 * ns && sd[2 * r] == i; ++r)
                                pair_term(n, x3, m, p->G, eps2, i, sd[2 * r + 1], &ax, &ay, &az);
                            acc[3 * a] = ax; acc[3 * a + 1] = ay; acc[3 * a + 2] = az;
                        }
                        free(sd);
                        if (st) st->kick_pairs += (uint64_t)ns;
                    }
                    for (int64_t a = 0; a < nset; ++a) {
                        const int64_t i = set[a];
                        v3[i] = v3[i] + h * acc[3 * a];
                        v3[n + i] = v3[n + i] + h * acc[3 * a + 1];
                        v3[2 * n + i] = v3[2 * n + i] + h * acc[3 * a + 2];
                    }
                    free(acc);
                }
                /* the drift of the members outside F */
                int64_t f = 0;
                for (int64_t a = 0; a < nset; ++a) {
                    const int32_t i = set[a];
                    while (f < nF && F[f] < i) f++;
                    if (f < nF && F[f] == i) continue;
                    const double dt = 0.5 * h;
                    x3[i] = x3[i] + dt * v3[i];
                    x3[n + i] = x3[n + i] + dt * v3[n + i];
                    x3[2 * n + i] = x3[2 * n + i] + dt * v3[2 * n + i];
                    if (st) st->drifts++;
                }
            }
        }
        /* E_{h/2,H_F}: the fast list's particles and interactions at h/2 */
        if (nf > 0) rc = orc_evolve_ok(n, x3, v3, m, p, F, nF, fast, nf, 0.5 * h, depth + 1, st);
    }
    free(fast);
    free(F);
    free(fd);
    free(slow);
    return rc;
}

static int check_state(int64_t n, const double *x3, const double *v3, const double *m)
{
    for (int64_t k = 0; k < 3 * n; ++k)
        if (!isfinite(x3[k]) || !isfinite(v3[k])) return ORC_E_NONFINITE;
    for (int64_t k = 0; k < n; ++k)
        if (!isfinite(m[k]) || !(m[k] > 0.0)) return ORC_E_NONFINITE;
    return ORC_OK;
}

int orc_evolve(int64_t n, double *x3, double *v3, const double *m,
               const orc_params *p, int64_t nsteps, orc_stats *st)
{
    int64_t off[2] = {0, n};
    return orc_evolve_systems(n, x3, v3, m, p, off, 1, nsteps, st);
}

int orc_evolve_systems(int64_t n, double *x3, double *v3, const double *m,
                       const orc_params *p, const int64_t *sys_off, int64_t nsys,
                       int64_t nsteps, orc_stats *st)
{
    if (n < 0 || nsteps < 0 || !(p->dt > 0.0)) return ORC_E_ARG;
    if (p->kepler && p->eps != 0.0) return ORC_E_ARG;
    if (p->split < 0 || p->split > 2 || (p->split != 0 && p->kepler))
        return ORC_E_ARG; /* HOLD and the OK split have no Kepler mode */
    if (p->theta < 0.0 || (p->theta > 0.0 && (p->split != 0 || p->com_max < 2))) return ORC_E_ARG;
    int rc = check_state(n, x3, v3, m);
    if (rc) return rc;
    int32_t *set = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k) set[k] = (int32_t)k;
    for (int64_t s = 0; s < nsteps && rc == ORC_OK; ++s)
        for (int64_t q = 0; q < nsys && rc == ORC_OK; ++q)
            rc = p->split == 1   ? orc_evolve_hold(n, x3, v3, m, p, set + sys_off[q],
                                                   sys_off[q + 1] - sys_off[q], p->dt, 0, st)
                 : p->split == 2 ? orc_evolve_ok(n, x3, v3, m, p, set + sys_off[q],
                                                 sys_off[q + 1] - sys_off[q], NULL, 0, p->dt, 0, st)
                                 : orc_evolve_cc(n, x3, v3, m, p, set + sys_off[q],
                                                 sys_off[q + 1] - sys_off[q], p->dt, 0, st);
    free(set);
    if (rc == ORC_OK) rc = check_state(n, x3, v3, m);
    return rc;
}

/* ------------------------------------------------------------------ */
/* diagnostics: H of Eq. (Hamiltonian), P, L                           */
/* ------------------------------------------------------------------ */
void orc_energy(int64_t n, const double *x3, const double *v3, const double *m,
                double G, double eps, double *E, double *P3, double *L3)
{
    double T = 0.0, V = 0.0, eps2 = eps * eps;
    double P[3] = {0, 0, 0}, L[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        double x = x3[i], y = x3[n + i], z = x3[2 * n + i];
        double vx = v3[i], vy = v3[n + i], vz = v3[2 * n + i];
        T += 0.5 * m[i] * ((vx * vx + vy * vy) + vz * vz);
        P[0] += m[i] * vx; P[1] += m[i] * vy; P[2] += m[i] * vz;
        L[0] += m[i] * (y * vz - z * vy);
        L[1] += m[i] * (z * vx - x * vz);
        L[2] += m[i] * (x * vy - y * vx);
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = x3[j] - x, dy = x3[n + j] - y, dz = x3[2 * n + j] - z;
            V -= G * m[i] * m[j] / sqrt(((dx * dx + dy * dy) + dz * dz) + eps2);
        }
    }
    if (E) *E = T + V;
    if (P3) { P3[0] = P[0]; P3[1] = P[1]; P3[2] = P[2]; }
    if (L3) { L3[0] = L[0]; L3[1] = L[1]; L3[2] = L[2]; }
}
