/*
 * hx — matrix-free Hermite-Galerkin operator and time stepper for GB300 (sm_103a).
 *
 * C ABI of the CUDA library libhx.so.  It implements, for
 *     i c'(t) = A(t) c(t),   A(t) = D_K + W^pol(X_K, t)          (Sec. 1.2, Eq. (ODECoefficientsPol))
 * of Brumm, "A fast matrix-free algorithm for spectral approximations to the
 * Schroedinger equation" (arXiv:1403.3511):
 *   - the hyperbolically reduced index set K = {k in N^N : prod_l (1 + k_l) <= B}
 *     (Sec. 1.2, with the paper's K + 1 written as B);
 *   - the matrix-free product y = A(t) c, with W replaced by its Chebyshev
 *     polynomial (Sec. 1.3) and the coordinate matrices X_K^{(l)} inserted into
 *     it through the three-term recurrence (Sec. 3.1-3.3);
 *   - time steps of the exponential midpoint rule (Eq. (expMPR), Sec. 2.1) with the
 *     exponential approximated by an m-step Hermitian Lanczos process (Sec. 2.2).
 *
 * General conventions
 *   - Every function returns an hx_status (0 = success, negative = error) unless
 *     stated otherwise; on error, hx_last_error() describes it (thread-local).
 *   - Multi-indices are int32 arrays of length N, axes counted from 0.
 *   - Coefficient vectors are in canonical order: the lexicographic order of K with
 *     the LAST coordinate varying fastest; position = hx_indexset_rank().
 *   - Vectors are interleaved complex: complex128 (2 x double) or complex64 (2 x float).
 *   - "device" pointers are CUDA global-memory pointers on the current device (for
 *     example torch tensor data pointers); "host" pointers are ordinary memory.
 *   - The caller owns every vector it passes.  The library owns the index tables,
 *     the compiled potential, the Krylov workspace and any CUDA graphs, and frees
 *     them in the matching *_destroy call.
 *   - All device work is ordered on the stream given in hx_config (0 = the legacy
 *     default stream); functions named *_host synchronise that stream before
 *     returning, the others do not unless stated.
 *   - Sizes: |K| < 2^31 and B <= 65535 (HX_EUNSUPPORTED otherwise), 1 <= N <= 16.
 */
#ifndef HX_H
#define HX_H

#include <stdint.h>

#if defined(__GNUC__)
#define HX_API __attribute__((visibility("default")))
#else
#define HX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HX_OK = 0,
    HX_EINVAL = -1,        /* invalid argument (null pointer, bad size, bad enum) */
    HX_ENOMEM = -2,        /* device or host allocation failed */
    HX_ECUDA = -3,         /* a CUDA call failed */
    HX_ENONFINITE = -4,    /* a NaN or Inf reached a norm */
    HX_EBREAKDOWN = -5,    /* informational: Lanczos stopped early (exact invariant subspace) */
    HX_ETIMEOUT = -6,      /* a bounded device wait ran out */
    HX_EUNSUPPORTED = -7   /* valid request outside what this build implements */
} hx_status;

/* Precision of the stencil arithmetic and of the Krylov vectors. */
typedef enum {
    HX_C128 = 0,           /* complex128 vectors, FP64 arithmetic throughout */
    HX_C64 = 1             /* complex64 vectors and stencil, FP64 reductions and state */
} hx_dtype;

/* Factor order inside a product of Chebyshev polynomials of different axes.
 * On a reduced index set the coordinate matrices of different axes do not commute,
 * and the paper writes the product in one order (Eq. (Horner)) and applies it in the
 * other (Algorithm fast_algorithm).  HX_ORDER_SYM (default) takes the mean of the two,
 * which keeps A(t) Hermitian; the other two reproduce one literal order each. */
typedef enum {
    HX_ORDER_SYM = 0,
    HX_ORDER_EQ = 1,       /* T_{r_1}(X1/L)( ... T_{r_N}(XN/L) v): the last axis acts first */
    HX_ORDER_ALG = 2       /* axis 0 acts on v first, then axis 1, ... */
} hx_order;

/* Exponent of one time step c^{n+1} = exp(Omega^n) c^n (Sec. 2.1). */
typedef enum {
    HX_SCHEME_EXPMPR = 0,  /* exponential midpoint rule, Eq. (expMPR): Omega = -i h A(t + h/2); order 2 */
    HX_SCHEME_MAGNUS4 = 1  /* 2-stage Gauss-Legendre Magnus method, Eq. (2stageMagnus):
                              Omega = -(i/2) h (A_1 + A_2) - (sqrt(3)/12) h^2 [A_2, A_1],
                              A_j = A(t + c_j h), c_{1,2} = 1/2 -+ sqrt(3)/6; order 4, four
                              products per Lanczos vector */
} hx_scheme;

/* Time dependence f(t) of one potential term. */
typedef enum {
    HX_MOD_CONST = 0,      /* f = 1 */
    HX_MOD_COS = 1,        /* f = cos(omega t + phase) */
    HX_MOD_SIN2 = 2,       /* f = sin^2(omega t) */
    HX_MOD_PWCONST = 3     /* f = pw_values[q] on the q-th of pw_n equal intervals of [pw_t0, pw_t1),
                              clamped to the first / last interval outside it */
} hx_mod_kind;

/* One term of W^pol(x, t) = sum_terms amp * f(t) * sum_r coef_r prod_i T_{r_i}(x_{axes[i]} / L)
 * (Sec. 1.3: the alpha_r(t) of the paper are amp * f(t) * coef_r).
 * n_axes = 1 or 2 (terms on more axes return HX_EUNSUPPORTED); axes strictly increasing;
 * deg[i] <= HX_MAX_DEG; coef has prod_i (deg[i] + 1) entries, row-major over the axes. */
#define HX_MAX_DEG 8
typedef struct {
    int n_axes;
    int axes[2];
    int deg[2];
    const double *coef;            /* host pointer, copied */
    int mod_kind;                  /* hx_mod_kind */
    double amp, omega, phase;
    const double *pw_values;       /* host pointer, copied (HX_MOD_PWCONST only) */
    int pw_n;
    double pw_t0, pw_t1;
} hx_term;

typedef struct {
    double L;                      /* half-width of the interpolation cube [-L, L]^N (Sec. 1.3-1.4) */
    int n_terms;
    const hx_term *terms;
} hx_potential;

typedef struct {
    int dtype;                     /* hx_dtype */
    int order;                     /* hx_order */
    int m;                         /* Lanczos steps per time step, 1 <= m <= 32 */
    void *stream;                  /* cudaStream_t, 0 for the legacy default stream */
    int scheme;                    /* hx_scheme */
    double tol;                    /* 0: every step is one Lanczos exponential of m steps.  > 0: each
                                    * step of hx_step is split into sub-steps until the a-posteriori
                                    * estimate of the relative error of every sub-step's Lanczos
                                    * exponential, |h| beta_m |e_m^T exp(-ihT_m) e_1| (Sec. 2.2),
                                    * is at most tol (hx_step_substeps reports the counts) */
    double scale;                  /* basis scaling S of the scaled Hermite functions phi_k(S x)
                                    * (Sec. 1.4); 0 means 1.  With S != 1 the product is
                                    * A = S^2 D_K + (1/S^2 - S^2)/2 sum_l X_l^2 + W(X / S), W given in
                                    * x as for S = 1 (its terms are evaluated on [-S L, S L]); the
                                    * paper asks S L >= sqrt(2 (K + 1)) + 1 for the interpolation box */
} hx_config;

typedef struct hx_indexset hx_indexset;
typedef struct hx_problem hx_problem;

/* ---- index set (Sec. 1.2) ------------------------------------------------------ */

/* Builds K = {k : prod (1 + k_l) <= B} and its device rank tables on the current device.
 * Synchronous.  Errors: HX_EINVAL (N < 1, N > 16, B < 1, out == NULL), HX_EUNSUPPORTED
 * (B > 65535 or |K| >= 2^31), HX_ENOMEM, HX_ECUDA. */
HX_API int hx_indexset_create(int N, int64_t B, hx_indexset **out);
/* |K|, or -1 for a NULL handle. */
/* A general downward-closed index set (Sec. 1.2: any K with k in K, j <= k => j in K) from a list of
 * count multi-indices k[count * N] (host, any order; copied).  Stored in lexicographic order, last
 * coordinate fastest, like the hyperbolic cross (hx_indexset_export gives that order).  Errors:
 * HX_EINVAL for a negative coordinate, a duplicate, a set that is not downward closed (a multi-index
 * whose neighbour k - e_l is missing) or count < 1; HX_EUNSUPPORTED for coordinates above 65534, a
 * coordinate sum above 65535, rows longer than 65535 or count >= 2^31 - 1.  Products on such sets
 * run the generic kernel (membership and fibre tops from the row tables). */
HX_API int hx_indexset_create_list(int N, int64_t count, const int32_t *k, hx_indexset **out);
HX_API int64_t hx_indexset_size(const hx_indexset *s);
/* Writes the multi-index of position rank into k_out[0..N-1] (host).  HX_EINVAL if out of range. */
HX_API int hx_indexset_unrank(const hx_indexset *s, int64_t rank, int32_t *k_out);
/* Position of multi-index k (host, length N) in canonical order, or -1 if k is not in K. */
HX_API int64_t hx_indexset_rank(const hx_indexset *s, const int32_t *k);
/* Writes all multi-indices, |K| x N int32 row-major, to the host buffer k_out (enumerated on
 * the device).  Synchronous. */
HX_API int hx_indexset_export(const hx_indexset *s, int32_t *k_out);
HX_API void hx_indexset_destroy(hx_indexset *s);

/* ---- problem: index set + potential + configuration -------------------------- */

/* cfg may be NULL: HX_C128, HX_ORDER_SYM, m = 7, default stream, HX_SCHEME_EXPMPR.  The index
 * set must outlive the problem.  Errors: HX_EINVAL (bad dtype, order, m or scheme), HX_ENOMEM
 * (host or device memory), HX_ECUDA (no usable CUDA device). */
HX_API int hx_problem_create(const hx_indexset *s, const hx_config *cfg, hx_problem **out);
HX_API void hx_problem_destroy(hx_problem *p);

/* Compiles W^pol (Sec. 1.3) into the coefficient tables the kernels read and sets the
 * problem time to t.  Terms are copied; the caller's arrays may be freed afterwards.
 * A constant term (all degrees 0) is folded into the diagonal.  With a product kernel
 * specialised to the potential's operator structure (hx_apply_specialised) it also packs each
 * element's fibre-top distances for that kernel (up to 16 bytes per coefficient of device memory,
 * kept while the structure stays the same).  Synchronous.
 * Errors: HX_EINVAL (L <= 0, bad axes or degrees, NULL coef), HX_EUNSUPPORTED (n_axes > 2,
 * more than 48 operators after compilation: rank-one pieces of two-axis terms, and for high
 * degrees their two stages, count separately), HX_ENOMEM / HX_ECUDA. */
HX_API int hx_potential_set(hx_problem *p, const hx_potential *pot, double t);
HX_API int hx_get_time(const hx_problem *p, double *t);
HX_API int hx_set_time(hx_problem *p, double t);

/* ---- the matrix-free product (Sec. 3) ------------------------------------------ */

/* c_out = A(t) c_in at the problem time t: D_K c_in + W^pol(X_K, t) c_in with the
 * configured factor order.  Device pointers of |K| elements of the problem dtype, aligned to
 * the element size (8 bytes for HX_C64, 16 for HX_C128; HX_EINVAL otherwise);
 * c_in and c_out must not overlap (HX_EINVAL).  Asynchronous on the problem stream. */
HX_API int hx_apply(hx_problem *p, const void *c_in, void *c_out);
/* The product of one Lanczos step with its first Gram-Schmidt projections (Sec. 2.2):
 * y = A(t) c and h_i = <basis_i, y> = sum_j conj(basis_i[j]) y[j] for i = 0..k.
 * c, y: device vectors of |K| elements of the problem dtype (c and y must not overlap, and y
 * must not overlap the basis).  basis: device, k + 1 vectors of the problem dtype, vector i at
 * basis + i * ld elements (ld >= |K|).  h: device array of 2 (k + 1) doubles, h[2i] + i h[2i+1].
 * 0 <= k < 8.  All vectors aligned to the element size as for hx_apply, h to 8 bytes.
 * With a specialised product kernel (hx_apply_specialised) and HX_C64 one kernel
 * computes both (the projections from the stored y, compensated FP32 partial sums); otherwise the
 * product is followed by a projection kernel (FP64 or compensated FP32 sums).  Asynchronous on
 * the problem stream; the first call allocates a small workspace and synchronises.
 * Errors: HX_EINVAL (NULL pointer, k out of range, ld < |K|, y overlapping c or the basis,
 * misaligned pointer, no potential). */
HX_API int hx_apply_project(hx_problem *p, const void *c, void *y, const void *basis, size_t ld, int k,
                            double *h);
/* Same with host buffers: copies in, applies, copies out, synchronises. */
HX_API int hx_apply_host(hx_problem *p, const void *c_in_host, void *c_out_host);

/* ---- time stepping (Sec. 2) ----------------------------------------------------- */

/* nsteps steps c <- exp(Omega^n) c with the problem's scheme: exp(-i dt A(t + dt/2)) c for
 * HX_SCHEME_EXPMPR (Eq. (expMPR)), exp(-i dt H) c with the Hermitian
 * H = (A_1 + A_2)/2 - i (sqrt(3) dt / 12)(A_2 A_1 - A_1 A_2) for HX_SCHEME_MAGNUS4
 * (Eq. (2stageMagnus)).  Each exponential by an m-step Hermitian Lanczos process with full
 * reorthogonalisation (classical Gram-Schmidt twice), c^{n+1} = ||c^n|| V_m exp(-i dt T_m) e_1
 * (Sec. 2.2).  c is a DEVICE complex128 vector of
 * |K| elements, updated in place, for both dtypes (HX_C64 runs the Krylov vectors and the
 * stencil in complex64, the state and all inner products in FP64; its first Krylov vector is the
 * state rounded to complex64 before normalisation, so the state's norm should lie well inside
 * the binary32 range, e.g. a normalised wave function).  Advances the problem
 * time by nsteps * dt.  One step is captured into a CUDA graph for the pair (c, dt) and replayed
 * nsteps times; a call with another vector or step size captures a new graph.  Asynchronous;
 * hx_step_info reports HX_EBREAKDOWN (informational) when some step needed fewer than m
 * Lanczos vectors, and HX_ENONFINITE when the norm became NaN/Inf or the eigensolver of T_m
 * did not converge.  c must be 16-byte aligned (HX_EINVAL otherwise). */
HX_API int hx_step(hx_problem *p, void *c, double dt, int nsteps);
/* Same with a host complex128 vector: copies in, steps, copies out, synchronises (the copies run
 * at full speed from page-locked memory). */
HX_API int hx_step_host(hx_problem *p, void *c_host, double dt, int nsteps);
/* Time-dependent potentials re-interpolated every step (the time-propagation algorithm of Sec. 2.2,
 * step (1): the coefficients alpha_r(t) of W^pol(., t) are computed anew for each step at the times
 * the integrator prescribes).  fn(t, user) returns the potential to use at time t, in the form
 * hx_potential_set takes; typically terms with HX_MOD_CONST whose Chebyshev coefficients the
 * caller interpolated at t (hx_cheb_nodes, hx_cheb_coeffs).  The returned potential (and the
 * arrays it points to) must stay valid until fn is called again or this function returns; the
 * library copies what it keeps.
 * Per step: HX_SCHEME_EXPMPR calls fn once, at t + dt/2; HX_SCHEME_MAGNUS4 calls fn at the two
 * Gauss-Legendre points t + (1/2 -+ sqrt(3)/6) dt, whose potentials must have the same L and
 * only HX_MOD_CONST terms (the library evaluates the first at the first point and the second at
 * the second by piecewise-constant modulations over [t, t + dt)).  Then one step as hx_step does
 * (same kernels; the step graph is captured anew each step since the coefficient tables change).
 * After the call the problem holds the potential of the last step.  c: DEVICE complex128, as for
 * hx_step.  Synchronises the problem stream once per step.  Errors: HX_EINVAL (NULL argument, fn
 * returned NULL, bad potential as for hx_potential_set, Magnus potentials with other
 * modulations or different L), HX_EUNSUPPORTED (more operators than one product kernel holds),
 * and the errors of hx_step. */
typedef const hx_potential *(*hx_potential_fn)(double t, void *user);
HX_API int hx_step_reinterp(hx_problem *p, void *c, double dt, int nsteps, hx_potential_fn fn, void *user);
/* Synchronises the stream and reports the last step: Lanczos size used, alpha/beta of T_m
 * (host arrays of at least m and m-1 doubles, either may be NULL) and the norm of c. */
HX_API int hx_step_info(hx_problem *p, int *m_used, double *alpha, double *beta, double *norm);
/* Sub-steps taken by the last hx_step of a problem with hx_config.tol > 0: sub-steps of its last
 * step (*last), in total (*total), and the largest a-posteriori error estimate over the accepted
 * sub-steps (*err_max; above tol only when a step reached 65536 sub-steps).  With tol = 0: 1, nsteps
 * and 0.  A step whose estimate exceeds tol is taken again from its start (the state is saved in a
 * device copy allocated at the first such call) with twice the sub-steps; after a step whose
 * estimate is below tol / 2^(m+1) the next one starts from half.  Any pointer may be NULL.  The
 * estimate follows from the Krylov relation A V_m = V_m T_m + beta_m v_{m+1} e_m^T (Sec. 2.2); the
 * automatic choice of sub-steps has no counterpart in the paper.  HX_EINVAL before the first step. */
HX_API int hx_step_substeps(hx_problem *p, int *last, int64_t *total, double *err_max);
/* 1 when the product runs a kernel compiled at hx_potential_set for this potential's operator
 * structure (NVRTC, sm_103a; every operator of the potential has a specialised stencil), 0 when it
 * runs the generic kernel; hx_last_error then says why (also when 1).  Both compute the same
 * product.  HX_EINVAL without a potential.  The paper has no counterpart: this reports how the
 * library runs the product.  Setting the environment variable HX_APPLY_SPECIALISE=0 before
 * hx_potential_set selects the generic kernel; HX_JIT_SOURCE_DUMP=<file> appends the source of
 * each newly compiled kernel set to that file before compiling it.  The steps of a batch (hx_batch_step)
 * run the generic kernel, except the large members of the HX_SCHED_SERIAL schedule. */
HX_API int hx_apply_specialised(const hx_problem *p);
/* Kernel launches of one product hx_apply (1, or 2 when some term is evaluated in two stages
 * through channel vectors) and of one time step of hx_step.  Per Lanczos vector: the product
 * (per_apply launches), one projection launch unless the product computes the projections itself
 * (HX_C64, a specialised product kernel (hx_apply_specialised), per_apply = 1, m <= 8), and the
 * Gram-Schmidt work: one sweep for m <= 8, two passes for m > 8 (the last vector's second pass only
 * with hx_config.tol > 0).  HX_SCHEME_MAGNUS4 takes, instead of the product, four products and
 * their combination into H v (4 per_apply + 1), or with a specialised kernel and per_apply = 1 two
 * launches (one gives A_1 v and A_2 v, the other A_2 A_1 v and A_1 A_2 v combined into H v), and
 * always the projection launch.  Then the start vector, the exponential and the recombination: 3
 * more (for m > 8 counted as 2, the last vector's skipped second pass taken off), and with
 * hx_config.tol > 0 the error estimate: 1 more (for m > 8 2, with that pass), per sub-step.  For
 * example m (per_apply + 1) + 3 for HX_C64 with a specialised kernel and m <= 8.
 * Needs a potential; either pointer may be NULL.  The paper has no counterpart: this reports how
 * the library maps its work onto kernels. */
HX_API int hx_step_launches(const hx_problem *p, int *per_apply, int *per_step);

/* ---- batches of independent problems ----------------------------------------------- */

/* A batch of independent problems of any N, B and potential, stepped together: one CUDA graph per
 * time step holds every problem's step (the same kernels as hx_step) as an independent branch, so
 * the GPU runs the problems concurrently; the graph is replayed nsteps times.  The problems keep
 * their own index sets, potentials, times and Krylov workspaces; they must stay alive while the
 * batch exists.  Work is ordered on the first problem's stream.  hx_batch_create: n >= 1 distinct
 * problems, each with a potential (HX_EINVAL otherwise).
 * hx_batch_step: c[i] is the DEVICE complex128 state of problem i (in place, 16-byte aligned, no two
 * states overlapping: HX_EINVAL otherwise); the graph is built on the first call and rebuilt when dt
 * or a state pointer changes or a member's hx_potential_set ran since.  Asynchronous. */
typedef struct hx_batch hx_batch;
HX_API int hx_batch_create(hx_problem *const *probs, int n, hx_batch **out);
HX_API int hx_batch_step(hx_batch *b, void *const *c, double dt, int nsteps);
HX_API void hx_batch_destroy(hx_batch *b);
/* Schedules of a batch step.  All three run the same kernels on each member and give the same bits:
 *   HX_SCHED_MEMBERS  one graph per step holding every member's step as an independent child graph,
 *                     each member's product its own launch;
 *   HX_SCHED_BATCHED  per Lanczos index one persistent product launch per (precision, degree <= 3 or
 *                     not) class over all members: blocks draw tiles of consecutive coefficients of any
 *                     member from a shared queue, largest members first; the members' projections,
 *                     Gram-Schmidt passes and exponentials stay their own kernels, forked from and
 *                     joined to those launches inside the graph;
 *   HX_SCHED_HYBRID   members with at least one wave of product blocks (|K| >= 4 x 256 x SM count)
 *                     step on their own streams as in HX_SCHED_MEMBERS, the others as in
 *                     HX_SCHED_BATCHED;
 *   HX_SCHED_SERIAL   members with a specialised kernel (hx_apply_specialised) and at least four
 *                     waves of product blocks take their own step's kernels (the specialised product,
 *                     in complex64 with fused projections) one member after another with nothing
 *                     running beside them, then the others as in HX_SCHED_BATCHED.  These members
 *                     get the bits of hx_step; the first three schedules give one another's bits.
 * The batched schedules need every member on the exponential midpoint rule with one product stage,
 * on a hyperbolic cross, with fixed sub-steps (tol = 0); otherwise only HX_SCHED_MEMBERS runs.  The
 * first steps after a (re)capture run each candidate once, timed between two events, and the rest
 * use the fastest (with fewer steps than candidates, the next call goes on timing).  The tile size
 * of the batched launches is chosen before that by timing 256, 512, 1024, 2048 and 4096 elements on
 * the product of the first Lanczos index.  HX_BATCH_BATCHED=0, 1, 2 or 3 in the environment forces
 * HX_SCHED_MEMBERS, HX_SCHED_BATCHED, HX_SCHED_HYBRID or HX_SCHED_SERIAL.
 *
 * hx_batch_set_budget: seconds >= 0 bounds each block of a batched product launch to that much
 * SM time (clock64 ticks at the device's clock rate); a block that runs over stops taking tiles and
 * sets a flag, so the launch ends early with an incomplete product instead of running on.
 * hx_batch_step then synchronises and returns HX_ETIMEOUT (the states are then not valid).
 * seconds < 0 (the default) removes the bound.  A change of budget re-captures the batch graphs.
 *
 * hx_batch_info: the state after the last hx_batch_step (all zero / -1 before the first). */
enum { HX_SCHED_MEMBERS = 0, HX_SCHED_BATCHED = 1, HX_SCHED_HYBRID = 2, HX_SCHED_SERIAL = 3 };
typedef struct {
    int schedule;        /* HX_SCHED_* in use, -1 while the candidates are still being timed */
    int tile;            /* elements per tile of the batched launches (0: not tuned) */
    int launches;        /* kernel launches of one step of the schedule in use */
    int ntiles;          /* tile-size candidates timed */
    int tiles[8];        /* their sizes ... */
    float tile_ms[8];    /* ... and the time of the first Lanczos index's batched products, ms */
    float step_ms[4];    /* one timed step of each schedule, ms (-1: not a candidate) */
} hx_batch_stats;
HX_API int hx_batch_set_budget(hx_batch *b, double seconds);
HX_API int hx_batch_info(const hx_batch *b, hx_batch_stats *out);

/* ---- gradient with respect to a control (adjoint) ---------------------------- */

/* A control u(t), constant on n_intervals equal intervals of [t0, t1), that enters the potential
 * as u(t) x_axis.  The time step is dt = (t1 - t0) / (n_intervals * substeps). */
typedef struct {
    int axis;
    int n_intervals;
    int substeps;
    double t0, t1;
    const double *u;               /* host, n_intervals values */
} hx_control;

/* J = |<phi, psi(t1)>|^2, psi(t0) = c0, propagated with the potential `fixed` plus u(t) x_axis by
 * the exponential midpoint rule with m-step Lanczos exponentials (Eq. (expMPR), Sec. 2.2), and its
 * gradient dJ/du_q (q < n_intervals) by the adjoint method: with a = <phi, psi_M>, lambda_M = phi,
 * lambda_{n-1} = U_n^H lambda_n, dJ/du_q = 2 Re(conj(a) sum_{n in q} lambda_n^H (dU_n/du) psi_{n-1}),
 * where dU_n/du is the Frechet derivative of the exponential; each term is evaluated exactly in the
 * Lanczos spaces of psi_{n-1} and lambda_n.  States at interval starts are kept, states inside an
 * interval are recomputed.  The computation is FP64 (cfg->dtype is ignored); cfg->m must be large
 * enough for the Lanczos exponential of one step to converge (the gradient is that of the
 * converged propagator), cfg->order and cfg->stream are honoured.  c0, phi: DEVICE complex128
 * vectors of |K|; grad_out: host array of n_intervals doubles, or NULL for J only; J_out: host.
 * Device memory: about (n_intervals + substeps + 2m + 8) vectors.  Synchronous.
 * cfg->tol is ignored and cfg->scale must be 0 or 1 (else HX_EUNSUPPORTED).
 * Errors: HX_EINVAL (NULL pointers, bad control), HX_EUNSUPPORTED (cfg->scheme other than
 * HX_SCHEME_EXPMPR), HX_ENOMEM, HX_ECUDA, as hx_potential_set. */
HX_API int hx_adjoint_grad(const hx_indexset *s, const hx_config *cfg, const hx_potential *fixed,
                           const hx_control *ctl, const void *c0, const void *phi, double *grad_out,
                           double *J_out);

/* ||c||_2 of a device vector of the problem dtype (aligned to the element size), accumulated in
 * FP64; synchronous.  HX_ENONFINITE when the result is not finite (*out is still written). */
HX_API int hx_norm(hx_problem *p, const void *c, double *out);
/* The energy <c, A(t) c> (real, since A(t) is Hermitian; not divided by ||c||^2) of a device vector
 * of the problem dtype at the problem time, for monitoring a propagation (Sec. 2.2 assumes a
 * Hermitian A(t); for a time-independent W the exponential midpoint rule keeps it up to the
 * Lanczos error).  One hx_apply_rayleigh into a temporary vector; synchronous.  Errors as hx_apply. */
HX_API int hx_energy(hx_problem *p, const void *c, double *out);
/* y = A(t) c and r = <c, y> = c^H A(t) c (r[0] real part, r[1] imaginary part, zero up to rounding
 * for a Hermitian A) at the problem time: the product of a Lanczos step together with the
 * diagonal entry of T_m (Sec. 2.2).  One launch when the product kernel is specialised
 * (hx_apply_specialised) and the dtype is HX_C64 (the product kernel sums conj(c_e) y_e itself in
 * compensated FP32 and the blocks' sums in FP64); otherwise the product and one reduction kernel.
 * c, y: DEVICE vectors of the problem dtype and size |K|, aligned to the element size, not
 * overlapping; r: DEVICE pointer to 2 doubles, 8-byte aligned, overlapping neither.  Asynchronous on
 * the problem stream; the first call of this or hx_apply_project on a problem allocates a small
 * workspace and synchronises.  Errors: HX_EINVAL (NULL or misaligned pointers, overlap, no
 * potential), HX_ECUDA.  Calls of this and hx_apply_project on one problem must not run
 * concurrently on different streams (they share that workspace; the problem stream orders them). */
HX_API int hx_apply_rayleigh(hx_problem *p, const void *c, void *y, double *r);

/* ---- allocation-free norm ------------------------------------------------------- */

/* Same result as hx_norm (||c||_2 in FP64 of a device vector of the problem dtype, synchronous),
 * but without allocating any device memory.  The paper has no counterpart: this entry point is for
 * callers that cannot call cudaMalloc at this point, for example an application whose device
 * memory is held entirely by its own pool (a caching allocator keeps the free memory, so a fresh
 * allocation would fail) or a latency-critical loop that must not enter an allocator.
 * Scratch: a fixed 1026-double device array inside libhx.so (1024 block partial sums, the result
 * and the reduction counter), held on every GPU that loads the library until the process exits.
 * hx_problem_create binds that array on the problem's device (it looks up its device address with
 * cudaGetSymbolAddress, which loads the module holding it and so reserves its memory there, and
 * fails the creation if that fails), so hx_norm_noalloc itself needs no set-up.  Every call shares
 * the array: calls that overlap on the GPU (from several threads or streams) race, so serialise
 * them.  Errors: as hx_norm (HX_EINVAL for a vector not aligned to its element size, checked before
 * anything runs), plus HX_EUNSUPPORTED when the reduction would need more than 1024 block partials
 * (a GPU with more than 256 SMs) and HX_EINVAL when the current device is not the problem's device. */
HX_API int hx_norm_noalloc(hx_problem *p, const void *c, double *out);

/* ---- Chebyshev helpers for building hx_term coefficients (Sec. 1.3) ----------- */

/* First-kind Chebyshev nodes u_i = cos(pi (2i + 1) / (2R + 2)), i = 0..R, into u_out[R+1]. */
HX_API int hx_cheb_nodes(int R, double *u_out);
/* Interpolation coefficients from values at the nodes: dims = 1 (values[R+1]) or
 * dims = 2 (values[(R+1)*(R+1)], values[i*(R+1)+j] = f(u_i, u_j)); coef_out has the same shape. */
HX_API int hx_cheb_coeffs(int R, int dims, const double *values, double *coef_out);
/* Exact Chebyshev coefficients of x^p on [-L, L]: x^p = sum_{r<=p} coef_out[r] T_r(x/L). */
HX_API int hx_cheb_monomial(int p, double L, double *coef_out);

/* ---- errors ---------------------------------------------------------------------- */

/* Message of the last failing call on this thread (never NULL). */
HX_API const char *hx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
