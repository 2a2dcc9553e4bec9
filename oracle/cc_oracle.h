/*
 * cc_oracle.h -- plain FP64 CPU oracle for the connected-component
 * (CC) Hamiltonian-splitting integrator of Jaenes, Pelupessy & Portegies
 * Zwart (arXiv:1407.7105).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this file: only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Layout: positions and velocities are SoA, x3[k*n + i] is component k of
 * particle i (k = 0,1,2); m[i] is the mass.  Particle ids are the indices
 * 0..n-1.  A "set" is a list of particle ids in ascending order.
 *
 * Numerics: every routine is plain IEEE-754 double with no fused
 * multiply-add (compile with -ffp-contract=off) and evaluates its formula
 * in the left-to-right order written in its comment.  Built with OpenMP,
 * independent rows run on several threads with the same arithmetic, so
 * every result is the serial one bit for bit.
 */
#ifndef CC_ORACLE_H
#define CC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double G;          /* gravitational constant (N-body units: 1)          */
    double eps;        /* Plummer softening length, enters V_ij (Sec. 2.1)  */
    double eta;        /* accuracy parameter of tau(i,j), Eq. (tauij)       */
    double dt;         /* outer (largest) pivot time step                   */
    int    kepler;     /* 1 = CC_KEPLER: 2-body components by Kepler (3.2)  */
    int    max_depth;  /* recursion depth cap; exceeding it is an error     */
    int    eta_outside;/* 0 = eta inside T and dT/dt (default reading),
                          1 = literal placement: eta multiplies the min     */
    int    split;      /* 0 = CC split (Sec. 2.2-2.3), 1 = HOLD split
                          (Sec. 2.1, Eq. HOLD), 2 = OK split (Sec. 4.2)     */
    double theta;      /* > 0: centre-of-mass approximation of V_CC (Sec.
                          4.1) between components whose radii satisfy
                          R_a + R_b < theta |X_a - X_b|; 0 = exact kicks    */
    int    com_max;    /* only components of 2..com_max members take part  */
    int    pad_;
} orc_params;

typedef struct {
    uint64_t tau_pairs;    /* n(n-1)/2 summed over every split             */
    uint64_t tau_evals;    /* tau evaluations the lazy BFS actually made   */
    uint64_t kick_pairs;   /* unordered cross-component pairs kicked       */
    uint64_t drifts;       /* particle drifts                               */
    uint64_t kepler_calls; /* two-body Kepler solves                        */
    uint64_t splits;       /* split_cc calls                                */
    uint64_t components;   /* non-trivial components found                  */
    uint64_t com_pairs;    /* body pairs whose kick the centre-of-mass
                              approximation replaced                         */
    int      max_depth_seen;
    int      pad_;
} orc_stats;

/* error codes */
#define ORC_OK          0
#define ORC_E_ARG      -1
#define ORC_E_DEPTH    -3
#define ORC_E_NONFINITE -5
#define ORC_E_KEPLER   -7

/* Interaction time step tau(i,j), Eq. (tauij) with the free-fall and flyby
 * times and their time derivatives (reading stated in the .c file).
 * parts (may be NULL) receives {T_ff, dT_ff, T_fb, dT_fb, tau_ff, tau_fb}. */
double orc_tau(const double *xi, const double *vi, double mi,
               const double *xj, const double *vj, double mj,
               const orc_params *p, double *parts);

/* tau for the pair (i, j) of the SoA state; i, j are particle ids. */
double orc_tau_ids(int64_t n, const double *x3, const double *v3, const double *m,
                   const orc_params *p, int64_t i, int64_t j);

/* split_cc (Sec. 2.3): BFS connected components of the graph with an edge
 * (i,j) iff tau(i,j) < h, restricted to `set`.  labels_out[k] = smallest id
 * of the component of set[k].  Returns the number of non-trivial
 * components (>= 2 members) or a negative error. */
int64_t orc_components(int64_t n, const double *x3, const double *v3, const double *m,
                       const orc_params *p, const int32_t *set, int64_t nset,
                       double h, int32_t *labels_out, orc_stats *st);

/* All edges (i<j, ids) of the time-step graph on `set`, all pairs
 * evaluated, lexicographic order.  Near-threshold pairs
 * |tau-h| < near_tol*h are counted in *n_near.  Returns the edge count
 * (entries beyond cap are counted but not written). */
int64_t orc_edges(int64_t n, const double *x3, const double *v3, const double *m,
                  const orc_params *p, const int32_t *set, int64_t nset, double h,
                  int32_t *edges_out, int64_t cap, double near_tol, int64_t *n_near);

/* K_{h,V_ij} for every pair of `set` with different labels (Eqs. kickij,
 * kickji): v_i += h * a_i with a_i summed over j in ascending id. */
void orc_kick(int64_t n, const double *x3, double *v3, const double *m,
              const orc_params *p, const int32_t *set, const int32_t *labels,
              int64_t nset, double h, orc_stats *st);

/* The kick K_{h,V} of a split with the centre-of-mass approximation of
 * V_CC (Sec. 4.1) when p->theta > 0, else orc_kick.  Components (labels
 * shared by 2..p->com_max members) have mass M_a, centre of mass X_a (sums
 * over members in ascending id) and radius R_a = max |x_i - X_a|; two of
 * them are far when R_a + R_b < theta |X_a - X_b|.  Then:
 *   1. the exact kick of orc_kick with the pairs of far components left out,
 *      v_i += h a_i;
 *   2. for each such component a, ascending label, A_a = sum over the far
 *      components b, ascending label, of (G M_b) (X_b - X_a) / (d2 sqrt(d2)),
 *      d2 = |X_b - X_a|^2 + eps^2, and v_i += h A_a for its members.
 * The forces between two components are G M_a M_b d/|d|^3 and its
 * opposite: momentum and angular momentum are kept.  orc_evolve_cc uses it
 * in the kick of sets of at least 33 members (orc_kick in smaller ones). */
void orc_kick_com(int64_t n, const double *x3, double *v3, const double *m,
                  const orc_params *p, const int32_t *set, const int32_t *labels,
                  int64_t nset, double h, orc_stats *st);

/* D_{dt,T_i} (Eq. drift) for members of `set` whose label is shared by no
 * other member: x_i += dt * v_i. */
void orc_drift(int64_t n, double *x3, const double *v3,
               const int32_t *set, const int32_t *labels, int64_t nset,
               double dt, orc_stats *st);

/* Two-body flow of particles i and j over dt (Eq. kepler, eps = 0) by the
 * classical Kepler equation in difference form. */
int orc_kepler(int64_t n, double *x3, double *v3, const double *m,
               double G, int64_t i, int64_t j, double dt);

/* The HOLD split of `set` at pivot h (Sec. 2.1): the particle time step
 * tau(i) is the minimum of tau(i,j) over the other members j of the set
 * (every pair evaluated); F = {i : tau(i) < h} is the fast set, S = the
 * rest.  labels_out[k] = the smallest id of F for members of F, set[k]
 * itself for members of S.  Returns 1 when F is not empty (it then has at
 * least two members: tau(i,j) = tau(j,i)), else 0. */
int64_t orc_hold_split(int64_t n, const double *x3, const double *v3, const double *m,
                       const orc_params *p, const int32_t *set, int64_t nset,
                       double h, int32_t *labels_out, orc_stats *st);

/* evolve_hold(S, h) of Sec. 2.1 (Eq. HOLD), recursive: E_{h/2,H_F}
 * D_{h/2,T_S} K_{h,V_S+V_SF} D_{h/2,T_S} E_{h/2,H_F}, H_F at pivot h/2. */
int orc_evolve_hold(int64_t n, double *x3, double *v3, const double *m,
                    const orc_params *p, const int32_t *set, int64_t nset,
                    double h, int depth, orc_stats *st);

/* evolve_ok(S, I, h) of the OK split (Sec. 4.2, reading R15 in the .c
 * file): the interaction list I of the set S (pairs == NULL: every pair of
 * S; else npairs pairs (a, b), a < b ids, sorted) split at pivot h into
 * fast (tau < h) and slow interactions; the fast ones and their particles
 * evolve at h/2 before and after D_{h/2} K_{h, slow} D_{h/2} of the rest. */
int orc_evolve_ok(int64_t n, double *x3, double *v3, const double *m,
                  const orc_params *p, const int32_t *set, int64_t nset,
                  const int32_t *pairs, int64_t npairs, double h, int depth, orc_stats *st);

/* evolve_cc(S, h) of the CC pseudocode figure (Sec. 2.3), recursive. */
int orc_evolve_cc(int64_t n, double *x3, double *v3, const double *m,
                  const orc_params *p, const int32_t *set, int64_t nset,
                  double h, int depth, orc_stats *st);

/* nsteps outer steps evolve_cc(all, p->dt) (evolve_hold when p->split = 1,
 * evolve_ok when p->split = 2). */
int orc_evolve(int64_t n, double *x3, double *v3, const double *m,
               const orc_params *p, int64_t nsteps, orc_stats *st);

/* Same outer loop over several independent systems: system s is the id
 * range [sys_off[s], sys_off[s+1]); pairs of different systems never
 * interact. */
int orc_evolve_systems(int64_t n, double *x3, double *v3, const double *m,
                       const orc_params *p, const int64_t *sys_off, int64_t nsys,
                       int64_t nsteps, orc_stats *st);

/* Threads of the parallel row loops (OpenMP builds; nthreads <= 0 leaves
 * the setting unchanged).  Returns the threads that loops will use (1
 * without OpenMP).  Results do not depend on it. */
int orc_set_threads(int nthreads);

/* Total energy H (Eq. Hamiltonian), linear and angular momentum. */
void orc_energy(int64_t n, const double *x3, const double *v3, const double *m,
                double G, double eps, double *E, double *P3, double *L3);

#ifdef __cplusplus
}
#endif
#endif
