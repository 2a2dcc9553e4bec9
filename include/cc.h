/*
 * cc.h -- C ABI of libcc.so, the GB300 (sm_103a) CUDA implementation of the
 * connected-component (CC) Hamiltonian-splitting N-body integrator of
 * Jaenes, Pelupessy & Portegies Zwart, "A connected component-based method
 * for efficiently integrating multiscale N-body systems" (arXiv:1407.7105).
 *
 * Conventions shared by every entry point
 *  - Every function returns 0 (CC_OK) or a negative CC_E_* code; none
 *    throws, traps or aborts.  cc_last_error(ctx) describes the last error.
 *  - Particle state is SoA: x3[k*n + i] is coordinate k (0,1,2) of particle
 *    i, likewise v3; m[i] is the mass.  Particle ids are 0..n-1.
 *  - Pointer arguments may point to host or device memory (the library asks
 *    cudaPointerGetAttributes); caller buffers stay caller-owned, the
 *    context owns all device memory it allocates.
 *  - Work is ordered on the CUDA stream given to cc_init / cc_set_stream.
 *    Functions that return host values synchronise that stream.
 *  - A "set" is an array of distinct particle ids in ascending order;
 *    NULL with n_set = n means all particles.
 *  - A context is not thread safe: one host thread at a time.
 */
#ifndef CC_H
#define CC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_OK            0
#define CC_E_ARG        -1  /* invalid argument                                */
#define CC_E_CUDA       -2  /* a CUDA runtime call failed                       */
#define CC_E_DEPTH      -3  /* recursion deeper than max_depth                  */
#define CC_E_TIMEOUT    -4  /* a bounded device wait or retry loop gave up       */
#define CC_E_NONFINITE  -5  /* non-finite or non-positive input                 */
#define CC_E_CAPACITY   -6  /* output buffer too small (counts still reported)  */
#define CC_E_KEPLER     -7  /* Kepler solver did not converge                   */
#define CC_E_NOMEM      -8  /* device allocation failed                         */

#define CC_SPLIT_CC    0    /* connected components of the time-step graph
                               (Sec. 2.2-2.3)                                   */
#define CC_SPLIT_HOLD  1    /* slow/fast split by the particle time step
                               tau(i) = min_j tau(i,j) (Sec. 2.1, Eq. HOLD)     */
#define CC_SPLIT_OK    2    /* the OK split (Sec. 4.2): interactions, not
                               particles, split by tau(i,j) < h; FP64 only      */

#define CC_SMALL_AUTO -1    /* cc_params.s_small: the library picks the limit    */

#define CC_PREC_FP64   0    /* every force and tau in FP64                      */
#define CC_PREC_MIXED  1    /* FP32 forces between components, certified FP32
                               tau pre-filter; FP64 state, drift, predicate     */

typedef struct {
    double G;          /* gravitational constant (N-body units: 1)                     */
    double eps;        /* softening length in V_ij (Sec. 2.1, Eq. Hamiltonian)         */
    double eta;        /* accuracy parameter of tau(i,j) (Eq. tauij)                   */
    double dt;         /* outer pivot time step h of evolve_cc(all, h)                 */
    double h_fp64;     /* CC_PREC_MIXED: sets split at a threshold h < h_fp64 take
                          FP64 forces (close subsystems where FP32 cancels)            */
    double near_tol;   /* pairs with |tau - h| < near_tol * h are logged (1e-12)       */
    int    precision;  /* CC_PREC_FP64 or CC_PREC_MIXED                                 */
    int    kepler;     /* 1: CC_KEPLER (Sec. 3.2), two-body components by Kepler flow   */
    int    max_depth;  /* recursion depth cap (levels below the outer step)            */
    int    s_small;    /* CC_SMALL_AUTO (-1, default): 512 in the mixed form, 32 in FP64.
                          Components of at most s_small (<= 512) members run entirely
                          on-chip in the persistent batched kernel: up to 32 members
                          one warp each, 33..512 one thread block each (its own
                          components of <= 32 members on its warps); 0 disables it.
                          With theta > 0 the limit is 32.  When every system of
                          cc_set_systems (or the one system of n bodies) has 2..s_small
                          members (3.. with kepler), an outer step is one launch:
                          every system one task                                       */
    int    eta_outside;/* 0: eta inside T and dT/dt (default reading); 1: eta
                          multiplies the min of Eq. (tauij) literally                  */
    int    autotune;   /* 1: launch shapes tuned online per size bin (default); 0: a
                          fixed rule (run-to-run identical rounding in mixed mode)   */
    int    edge_rec_max;/* 0: default; > 0: at most this many edge records kept per
                          level for the first-half splits of the next level.  A
                          split with more edges than that leaves an incomplete
                          list, and the first halves of its components then run
                          a fresh split (results are the same, only slower)    */
    int    fault_test; /* 0 in normal use.  Failure-path test hooks of the tau
                          kernels (the certified one of every split, the FP64
                          one of cc_timestep_graph), so that a test can see a
                          bounded wait or retry run out and the call return
                          CC_E_TIMEOUT without any GPU fault: 1 = the tile copy
                          is announced but never issued, so the mbarrier wait
                          gives up after ~2^20 cycles; 2 = the union-find hook
                          gives up at once                                      */
    int    split;      /* CC_SPLIT_CC (default); CC_SPLIT_HOLD: the HOLD method of
                          Sec. 2.1 on the same kernels -- the fast set F = {i :
                          tau(i) < h} is the union of the CC components, so it is
                          split as one set; CC_SPLIT_OK: the OK split of Sec.
                          4.2 -- the pairs with tau(i,j) < h and their particles
                          recurse at h/2 around D K D of the other particles and
                          pairs (FP64 form only); neither has a Kepler mode   */
    int    com_max;    /* centre-of-mass approximation: components of 2..com_max
                          (<= 64) members take part (default 32)              */
    double theta;      /* > 0: the centre-of-mass approximation of V_CC (Sec. 4.1)
                          in the DKD of every set of at least 33 members: two
                          eligible components with R_a + R_b < theta |X_a - X_b|
                          (X the centre of mass, R the largest distance of a member
                          from it) kick each other through their centres of mass,
                          G M_b (X_b - X_a)/|X_b - X_a|^3 on every member of a, in
                          place of their pair kicks; 0 (default): exact kicks  */
} cc_params;

typedef struct {
    uint64_t tau_pairs;     /* pairs whose tau the splits covered: n(n-1)/2 per set  */
    uint64_t tau_fp64;      /* pairs whose predicate was evaluated in FP64           */
    uint64_t kick_pairs;    /* unordered cross-component pairs kicked                 */
    uint64_t drifts;        /* particle drifts                                        */
    uint64_t kepler_calls;  /* two-body Kepler solves                                 */
    uint64_t splits;        /* set splits (split_cc calls)                            */
    uint64_t components;    /* non-trivial components found                           */
    uint64_t edges;         /* edges (tau < h) found                                  */
    uint64_t near_pairs;    /* pairs with |tau-h| < near_tol*h                        */
    uint64_t small_tasks;   /* components run by the small-component kernel          */
    uint64_t launches;      /* kernels this context launched                          */
    uint64_t tau_evaluated; /* pairs whose tau a kernel computed: tau_pairs counts every
                               pair a split decides, but the split of a component's
                               first half sees the state its parent split saw, and
                               takes the edges from the parent's tau values instead  */
    uint64_t com_pairs;     /* body pairs whose kick the centre-of-mass approximation
                               replaced (not in kick_pairs)                         */
    int32_t  max_depth_seen;
    int32_t  reserved;
} cc_stats_t;

/* Device time of the pairwise kernels, measured with CUDA events on the
 * context's stream while timing is on (cc_set_timing): the tau kernels of
 * the level splits, the kick kernels of the level DKDs, and the
 * small-component kernel (which runs whole sub-recursions).  pairs =
 * unordered pairs the tau and kick launches covered (tau: n(n-1)/2 per
 * set; kick: cross-component pairs). */
typedef struct {
    double   tau_ms, kick_ms, small_ms;
    int64_t  tau_launches, kick_launches, small_launches;
    uint64_t tau_pairs, kick_pairs;
    /* work of the small-component kernel while timing was on: tau pairs it
     * evaluated (its first-half splits reuse their fresh split's values)
     * and cross-component pairs it kicked */
    uint64_t small_tau_evaluated, small_kick_pairs;
} cc_timing_t;

typedef struct cc_ctx cc_ctx;

/* Fill *p with defaults: G=1, eps=0, eta=0.03, dt=1/64, h_fp64=0,
 * near_tol=1e-12, FP64, kepler off, max_depth=64, s_small=CC_SMALL_AUTO,
 * autotune on. */
int cc_default_params(cc_params *p);

/* Create a context holding n particles (Sec. 2.1: masses m_i, positions q_i,
 * velocities v_i = p_i/m_i).  m[n], x3[3n], v3[3n] host or device.
 * stream: a cudaStream_t (NULL = default stream).  Device memory grows with
 * the recursion: each depth's level buffers at first use, and for the FP64
 * kicks (the FP64 form; the mixed form below h_fp64) of levels with at least
 * 2^18 pairs and no centre-of-mass approximation, the pair forces of every
 * set (3 n^2 doubles per set; 6.4 GB for a 16384-body set), kept up to 24 GB
 * for the context's lifetime; when that allocation fails, or a level needs
 * more, the kick computes the forces in place (same results, no error).
 * Errors: CC_E_ARG (n < 1, bad params), CC_E_NONFINITE (non-finite state or
 * m <= 0), CC_E_NOMEM. */
int cc_init(cc_ctx **out, int64_t n, const double *m, const double *x3,
            const double *v3, const cc_params *p, void *stream);

/* Declare independent systems: system s is the id range
 * [sys_off[s], sys_off[s+1]) (host array, nsys+1 entries, sys_off[0] = 0,
 * sys_off[nsys] = n); pairs of different systems never interact, and each
 * outer step runs evolve_cc(system, dt) for every system.  Default: one
 * system.  Errors: CC_E_ARG. */
int cc_set_systems(cc_ctx *ctx, const int64_t *sys_off, int64_t nsys);

int cc_set_stream(cc_ctx *ctx, void *stream);

/* Time-step graph of Sec. 2.2 on `set` at threshold h: all pairs of the set,
 * tau(i,j) by Eq. (tauij) in FP64 (T_ff = eta sqrt(r^3/mu), T_fb = eta r/|dv|,
 * their time derivatives along the pair's motion, dT/dt clamped at 1), edge iff
 * tau(i,j) < h.  *n_edges = edge count.  edges_out (may be NULL) receives
 * min(cap, n_edges) pairs (i<j as particle ids, int32[cap][2]) in
 * lexicographic order.  *n_near = pairs with |tau-h| < near_tol*h (their
 * (i, j, tau) are readable with cc_near_pairs).  Returns CC_E_CAPACITY when
 * n_edges > cap and edges_out != NULL (the first cap edges of the sorted
 * order are not guaranteed then: only the count is). */
int cc_timestep_graph(cc_ctx *ctx, const int32_t *set, int64_t n_set, double h,
                      int64_t *n_edges, int32_t *edges_out, int64_t cap,
                      int64_t *n_near);

/* split_cc of Sec. 2.3 by union-find: labels_out[k] (int32[n_set]) = the
 * smallest particle id of the connected component of set[k] in the
 * time-step graph at h (singletons: their own id; they form the rest set
 * R).  *n_comp = number of non-trivial components (>= 2 members).  With
 * params.split = CC_SPLIT_HOLD, the HOLD split of Sec. 2.1 instead: the
 * fast set F (every member with an edge, i.e. tau(i) < h) labelled with
 * its smallest id, the slow set with their own ids; *n_comp = 1 if F is
 * not empty, else 0. */
int cc_components(cc_ctx *ctx, const int32_t *set, int64_t n_set, double h,
                  int32_t *labels_out, int64_t *n_comp);

/* K_{h,V} of Eqs. (kickij, kickji) for every pair of `set` whose labels
 * differ (labels int32[n_set], any values): v_i += h * a_i.  Sec. 2.2 splits
 * V_R + V_CC + V_CR this way.  Precision follows params.precision (mixed
 * forces unless h < h_fp64). */
int cc_kick(cc_ctx *ctx, const int32_t *set, int64_t n_set,
            const int32_t *labels, double h);

/* D_{h,T_i} of Eq. (drift), x_i += h * v_i, for the members of `set` whose
 * label no other member shares (the rest set R). */
int cc_drift(cc_ctx *ctx, const int32_t *set, int64_t n_set,
             const int32_t *labels, double h);

/* Outer loop: while t < t_end, evolve_cc(system, dt) for every system (CC
 * pseudocode figure, Sec. 2.3), then t += dt.  (t_end - t) must be a whole
 * number of steps dt (relative slack 1e-9) else CC_E_ARG.  eta > 0
 * overrides params.eta.  Errors: CC_E_DEPTH, CC_E_TIMEOUT, CC_E_KEPLER,
 * CC_E_NONFINITE (state became non-finite); the state is undefined after
 * one.  When every system fits the batched kernel (s_small) each step is
 * one launch of a CUDA graph captured from the step (again after an eta
 * change), and a device error is reported after the call's last step. */
int cc_evolve(cc_ctx *ctx, double t_end, double eta);

/* Copy out / replace the state (any pointer may be NULL to skip). */
int cc_get_state(cc_ctx *ctx, double *t, double *m, double *x3, double *v3);
int cc_set_state(cc_ctx *ctx, double t, const double *m, const double *x3,
                 const double *v3);

/* Counters accumulated since cc_init or the last cc_reset_stats. */
int cc_stats(cc_ctx *ctx, cc_stats_t *out);
int cc_reset_stats(cc_ctx *ctx);

/* Total energy H (Eq. Hamiltonian, FP64 all pairs), momentum P[3] and
 * angular momentum L[3] (host pointers, any may be NULL).  With independent
 * systems (cc_set_systems) H is the sum of the systems' own Hamiltonians:
 * pairs of two systems, which never interact, are left out. */
int cc_energy(cc_ctx *ctx, double *E, double *P3, double *L3);

/* Near-threshold pairs logged since the last cc_timestep_graph /
 * cc_components / cc_evolve call: ids int32[cap][2], tau double[cap]
 * (either may be NULL); *n = total logged (may exceed cap). */
int cc_near_pairs(cc_ctx *ctx, int32_t *pairs, double *tau, int64_t cap, int64_t *n);

/* Turn per-launch event timing of the tau and kick kernels on (1) or off
 * (0); turning it on clears the accumulated times. */
int cc_set_timing(cc_ctx *ctx, int on);
int cc_timing(cc_ctx *ctx, cc_timing_t *out);

/* One cell of the launch-shape autotuner: a kernel and a size bin (the
 * launch's pair count in [2^bin, 2^(bin+1))).  Variant v of the kernel is
 * the launch shape (shape[v], slices[v]): for the tau kernels the tile edge
 * (64, 128) and the threads per tile row (its columns split in slices); for
 * the FP64 kick the tile edge (32, 64, 128), slices 1; for the mixed kick
 * the j-chunk in tiles of 128 and the column slices of each tile. */
typedef struct {
    int32_t kernel;            /* CC_TUNE_TAU_FP64 .. CC_TUNE_KICK_MIXED           */
    int32_t bin;
    int32_t best;              /* chosen variant; -1 while variants are tried     */
    int32_t nvar;              /* variants of this kernel (<= 3)                 */
    int32_t shape[3];
    int32_t slices[3];
    int32_t timed[3];          /* timed launches per variant                      */
    int32_t reserved;
    double  us_per_mpair[3];   /* fastest timed launch: microseconds per 1e6 pairs (0: none) */
} cc_tune_entry_t;

enum { CC_TUNE_TAU_FP64 = 0, CC_TUNE_TAU_MIXED = 1, CC_TUNE_KICK_FP64 = 2, CC_TUNE_KICK_MIXED = 3 };

/* Copy the autotuner's cells that have at least one timed launch, in
 * (kernel, bin) order, into out[cap]; *n_out = the number of such cells
 * (may exceed cap: only cap are written).  Synchronises the context's
 * stream.  Errors: CC_E_ARG (ctx or n_out NULL, cap < 0, out NULL with
 * cap > 0), CC_E_CUDA. */
int cc_tuning(cc_ctx *ctx, cc_tune_entry_t *out, int64_t cap, int64_t *n_out);

/* FMA throughput of the current device, measured by a microbenchmark on
 * `stream` (flop/s, an FMA counting 2): the ALU roofline denominators of
 * the FP64 and FP32 pair kernels.  Errors (message via cc_last_error(NULL)):
 * CC_E_CUDA. */
int cc_probe_peaks(void *stream, double *fp64_flops, double *fp32_flops);

/* Component labels of a caller-held state without any device allocation.
 * No counterpart in the paper: it is cc_components over all n particles
 * for callers that cannot let this library call cudaMalloc -- their device
 * memory belongs to another allocator (a framework pool that has reserved
 * the GPU, or a fixed budget) or their loop cannot take the device-wide
 * synchronisation cudaMalloc/cudaFree imply.  Scratch lives in a fixed
 * file-scope device array of CC_NOALLOC_MAX_N entries (512 KiB held on
 * every GPU that loads libcc.so, until exit), so n <= CC_NOALLOC_MAX_N.
 *   m[n], x3[3n], v3[3n]: device-accessible state, SoA as above (read only)
 *   p: G, eps, eta, eta_outside are used; h: threshold of tau(i,j) < h
 *   labels_out[n] (device-accessible int32): smallest particle index of
 *     each particle's component, identical to cc_components on all n
 *   n_comp_out (device-accessible int64): number of components >= 2
 * "Device-accessible" means device or managed memory, or pinned host memory
 * mapped into the device's address space; the call checks each pointer
 * (cudaPointerGetAttributes) before any launch and refuses pageable host
 * memory.  It cannot check sizes: the arrays must hold the counts above.
 * The first call on a device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 * The address is kept until the process exits (a cudaDeviceReset
 * invalidates it; calls after one are not supported).
 * Calls share the one array per device: calls whose work overlaps on the
 * GPU race and give wrong labels, so serialise them (one stream, or
 * synchronise between calls).  The call synchronises `stream` before it
 * returns.  Errors: CC_E_ARG (NULL or unreachable pointer, n < 1, h not
 * > 0, or G, eps, eta, eta_outside out of the range cc_init accepts),
 * CC_E_CAPACITY (n > CC_NOALLOC_MAX_N), CC_E_CUDA (a CUDA call or launch
 * failed), CC_E_TIMEOUT (union-find retry limit reached). */
#define CC_NOALLOC_MAX_N 65536
int cc_components_noalloc(const double *m, const double *x3, const double *v3,
                          int64_t n, const cc_params *p, double h,
                          int32_t *labels_out, int64_t *n_comp_out, void *stream);

/* Release the context and all its device memory. */
int cc_destroy(cc_ctx *ctx);

/* Static description of the last error on ctx (or of the last failed
 * cc_init when ctx is NULL). */
const char *cc_last_error(cc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
