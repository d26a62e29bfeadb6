/*
 * dmk_stokes.h -- C ABI of the GB300 near-field library for the DMK method for
 * Stokes potentials (Jiang, Tornberg et al., arXiv 2509.21471).
 *
 * What it computes (the "near" component of the DMK sum, Sec. 5.3 Eq.
 * (three_part_sum) and Step 4 of Sec. 6.1): for every target t of the unit box
 * [lo, lo+1]^d (Sec. 1), d = 2 or 3, where the targets are the source points
 * themselves or a separate point set,
 *
 *   u_t = sum_{s near t, 0 < r < nu_ts}  S_R,nu_ts(x_t - x_s) f_s      (Stokeslet)
 *       + sum_{s near t, 0 < r < nu_ts}  T_R,nu_ts(x_t - x_s) g_s n_s  (stresslet)
 *       + u_self(t)
 *
 * with the prolate-split residual kernels S_R, T_R of Sec. 5.2 (Eqs.
 * (res_stokeslet), (Soffdiag), (res_stresslet), (T-offd)) at the residual scale
 *   nu_ts = 2^-(min(L_t, L_s) + 1),   L = level of the point's leaf,
 * and the Stokeslet self term u_self = -phi(0)/(2 pi nu_t) f_t (Eq. (S_self),
 * nu_t = 2^-(L_t+1); the stresslet's is zero; separate targets, which carry
 * no force, have none).  "near" = the sources of the
 * leaves touching t's leaf in the adaptive, level-restricted tree of Step 1
 * (periodic images included in the periodic case, Sec. 6.2).  In the periodic
 * stresslet case the k = 0 term u0(x_t) = -sum_s (x_t - x_s)(g_s . n_s)
 * (Sec. 5.3, after Eq. (ewald_far)) is added as well.
 *
 * Conventions
 *   - Every array argument is a DEVICE pointer owned by the caller, row-major,
 *     float64, on the device current when the plan was made.
 *   - Calls are asynchronous on the given CUDA stream (NULL = legacy default
 *     stream).  Argument errors are returned synchronously.  Errors found on the
 *     device (a free-space point outside the box, a non-finite coordinate) are
 *     latched in the plan and returned by dmk_stokes_sync_status().
 *   - Outputs are in the caller's original point order.
 *   - The plan copies everything it needs from the coordinates; the caller may
 *     reuse the coordinate buffer when dmk_stokes_plan has returned (it
 *     synchronises its stream before returning).
 *   - The stream given to dmk_stokes_plan must stay valid until
 *     dmk_stokes_destroy (device memory is released on it, after the work of
 *     the last stream an evaluation was queued on).
 *   - Functions are not thread-safe on the same plan.
 */
#ifndef DMK_STOKES_H_
#define DMK_STOKES_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmk_stokes_plan_s* dmk_stokes_plan_t; /* opaque, owned by the library */

typedef enum {
  DMK_OK = 0,
  DMK_ERR_INVALID_ARG = 1,  /* bad option, null pointer, size or NaN */
  DMK_ERR_OUT_OF_RANGE = 2, /* free-space point outside [lo, lo+1]^d */
  DMK_ERR_UNSUPPORTED = 3,  /* valid but not provided by this library */
  DMK_ERR_NOMEM = 4,        /* device allocation failed */
  DMK_ERR_CUDA = 5,         /* a CUDA runtime call failed */
  DMK_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
  DMK_ERR_BAD_PLAN = 7      /* null, destroyed or foreign plan handle */
} dmk_status_t;

enum { DMK_KERNEL_STOKESLET = 1, DMK_KERNEL_STRESSLET = 2 };
enum { DMK_PRECISION_FP64 = 0, DMK_PRECISION_MIXED = 1 };
enum { DMK_COMPONENTS_ALL = 0, DMK_COMPONENTS_NEAR = 1, DMK_COMPONENTS_EWALD = 2 };

typedef struct {
  int32_t dim;           /* 2 or 3 */
  int32_t periodic;      /* 0 free space; 1 periodic unit cell (Sec. 6.2) */
  int32_t kernels;       /* bitmask DMK_KERNEL_*; the stresslet and the gradient
                            need n_rhs == 1 */
  int32_t precision;     /* DMK_PRECISION_FP64: all arithmetic in float64.
                            DMK_PRECISION_MIXED: pair terms in float32 with
                            leaf-relative coordinates and compensated (two-sum)
                            accumulation; self term and output in float64.
                            FP32 pair terms carry a relative l2 error of about
                            1e-7..2e-6, so for eps < 2e-7 (one force column)
                            MIXED takes float-float pair terms (hi + lo floats,
                            about 48 bits; an FP32 test still selects the
                            candidate pairs) and meets eps like FP64; several
                            columns below 2e-7 take float64 pair terms.
                            Nearly coincident pairs, r <= nu/32 (FP32 pair
                            terms) or r <= nu/1024 (float-float), are taken in
                            float64 from the float64 coordinates, since
                            leaf-relative coordinates cannot resolve them.
                            The gradient and the adjoint take float-float pair
                            terms at every eps. */
  int32_t components;    /* DMK_COMPONENTS_NEAR: the near component (residual
                            pass + self term, + the periodic stresslet zero
                            mode).
                            DMK_COMPONENTS_ALL: the whole DMK sum, 2D or 3D,
                            one force column, free space or periodic,
                            Stokeslet and/or stresslet, sources or separate
                            targets: the near component plus the far field of
                            Sec. 6 (leaf proxy charges on p^d Chebyshev grids,
                            child merges, level-l plane waves with N1 modes a
                            side for the colleague difference kernels, the
                            root kernel K_M,0: periodic Fourier series with
                            N_per modes a side, or the truncated kernel of
                            Eq. (Bmollhat_trunc), R = 1 + sqrt(d), in free
                            space, interpolation to the leaves; App. B
                            kernels in 2D).  p, N1, N_per from Table 2 (p
                            interpolated in log10 eps, N1 = 2 (3c/pi) - 1,
                            N_per = 2 floor(c / 2pi) + 1).  The far field runs
                            in float32 where the pair terms do (MIXED, eps >=
                            2e-7) and in float64 otherwise; in 3D float32 its
                            leaf charges and leaf evaluation run on the
                            tensor cores (split-TF32 products), or on the
                            FP32 pipe when the environment variable
                            DMK_STOKES_FAR_TC=0 is set at plan time.  Single system;
                            eval_grad / adjoint / noalloc: UNSUPPORTED.
                            DMK_COMPONENTS_EWALD: the periodic 3D Stokeslet
                            summed by a single-level prolate Ewald split on a
                            uniform tree (near pass at the leaf scale + an FFT
                            far field, Sec. 5.3), one column, targets = sources. */
  int32_t leaf_capacity; /* n_s, max points per leaf; 0 = the paper's value for
                            eps (Sec. 8: 3D 600..3000, 2D 120..480) */
  int32_t n_rhs;         /* force columns, 1..16 */
  int32_t bandlimit;     /* 0: the prolate bandlimit c from eps (below);
                            2..36: c = bandlimit * pi / 3 (3c/pi given), for
                            parameter studies such as E(c) of Sec. 7 */
  double eps;            /* tolerance in [1e-12, 1e-3]; selects the prolate
                            bandlimit c from Table 2 (3c/pi interpolated in
                            log10 eps and rounded up) unless bandlimit is set,
                            the FP32 table length and the Ewald grid width */
  double box_lo[3];      /* lower corner lo of the unit box (side 1) */
} dmk_stokes_opts_t;

/* Builds the plan: Morton keys, sort, adaptive tree (leaves hold <= n_s points,
 * Step 1(a)), level restriction (Step 1(b)), near lists and tiles, and the
 * polynomial kernel tables for the bandlimit c of eps (remark closing Sec. 5.2).
 *   n_src   number of points (>= 0, < 2^31)
 *   d_src   [n_src][dim] coordinates
 *   n_trg, d_trg: d_trg == NULL with n_trg == n_src: the targets are the
 *           sources; d_trg == NULL with n_trg == 0 < n_src: an empty set of
 *           separate targets.  Otherwise d_trg [n_trg][dim] are separate targets
 *           (0 <= n_trg < 2^31; the sums of Sec. 1 at points that need not be
 *           sources): the tree is the sources' (leaf capacity counts sources,
 *           Step 1(a)), each target takes the leaf containing it (empty leaves
 *           included), its level L_t in nu_ts and that leaf's near list, and no
 *           self term.  Every output then has n_trg rows in the caller's target
 *           order.  The passes are one-sided (MIXED below eps 2e-7 takes FP64
 *           pair terms); dmk_stokes_eval_adjoint returns DMK_ERR_UNSUPPORTED.
 *   stream  cudaStream_t or NULL
 *   out     receives the plan handle (set to NULL on failure)
 * Host-synchronises the stream a few times (tree sizes are read back). */
dmk_status_t dmk_stokes_plan(const dmk_stokes_opts_t* opts, int64_t n_src, const double* d_src,
                             int64_t n_trg, const double* d_trg, void* stream,
                             dmk_stokes_plan_t* out);

/* Same for n_sys independent systems (each its own unit box, tree and sums)
 * stored back to back: system i owns points [h_offsets[i], h_offsets[i+1]).
 * h_offsets is a HOST array of n_sys + 1 nondecreasing values, h_offsets[0] = 0.
 * No paper counterpart (batching of many small systems).  eval / eval_grad /
 * destroy work on the result as on any plan. */
dmk_status_t dmk_stokes_plan_batched(const dmk_stokes_opts_t* opts, int32_t n_sys,
                                     const int64_t* h_offsets, const double* d_src, void* stream,
                                     dmk_stokes_plan_t* out);

/* Evaluates the near component (definition at the top of this file).
 *   d_f  [n][dim][n_rhs] Stokeslet forces (required if the Stokeslet bit is set)
 *   d_g  [n][dim] stresslet strengths, d_n [n][dim] orientation vectors
 *        (required if the stresslet bit is set; rho_s = g_s (x) n_s, Eq. (stokes_stress_sum))
 *   d_u  [n_trg][dim][n_rhs] output, overwritten (n_trg = n without separate targets)
 * Does not allocate; may be captured in a CUDA graph.  With one force column
 * the FP32 Stokeslet pass and the float-float and FP64 passes evaluate each
 * pair once for both of its points (the residual Stokeslet is even, the
 * stresslet odd); the two sides meet in an FP64 accumulator by atomic
 * additions, so repeated calls agree to within the order of those additions
 * (~1e-16 relative), not bit for bit.  The periodic stresslet zero mode is
 * also summed atomically.  Other configurations are bitwise reproducible. */
dmk_status_t dmk_stokes_eval(dmk_stokes_plan_t plan, const double* d_f, const double* d_g,
                             const double* d_n, double* d_u, void* stream);

/* The same evaluation as dmk_stokes_eval for callers that must not allocate
 * device memory when they evaluate (for example during a CUDA stream capture
 * that forbids allocation calls, or where another allocator owns the device
 * memory budget).  It calls no cudaMalloc / cudaMallocAsync / cudaFree and
 * does not touch the plan's own workspace: its scratch (sorted copies of the
 * densities, the periodic zero-mode sums) is one array of 64 MiB that the
 * library reserves statically on every GPU that loads it, until exit.
 * The paper has no counterpart; this is a deployment variant.
 *   Arguments, layouts and results: as dmk_stokes_eval.
 *   Limit: plans needing more than 64 MiB of scratch (with n_rhs = 1: mixed
 *   precision at eps >= 2e-7 136 bytes per point, about 493k points; mixed
 *   below 2e-7 296 bytes per point in 3D (200 in 2D), about 226k points;
 *   FP64 104 bytes per point, about 645k points; more with several force
 *   columns; plus 32 bytes per system) return DMK_ERR_INVALID_ARG before any
 *   work is queued.
 *   The plan's device must be current.
 *   Sharing: all calls on a device use the same array, which keeps the last
 *   call's contents (what must start at zero is cleared by every call); calls
 *   whose work overlaps on the GPU race on it, so queue them on one stream.
 *   The first call on a device looks the array's address up (with that device
 *   current); make it before any stream capture.  The address is kept for the
 *   life of the process: resetting the device after that call is not supported. */
dmk_status_t dmk_stokes_eval_noalloc(dmk_stokes_plan_t plan, const double* d_f, const double* d_g,
                                     const double* d_n, double* d_u, void* stream);

/* Velocity gradient of the 3D near component, Stokeslet and / or stresslet
 * (d_f, d_g, d_n as for dmk_stokes_eval; one density column; the 2D gradient
 * is not provided: DMK_ERR_UNSUPPORTED):
 *   d_gradu [n_trg][3][3], gradu[t][j][m] = d u_j / d x_m at x_t with the
 *   tree (and so every nu_ts) held fixed; the self term does not depend on x,
 *   the periodic stresslet k = 0 term adds -delta_jm sum_s g_s.n_s.
 *   d_u may be NULL; if not NULL it receives the velocity as dmk_stokes_eval does.
 * Stokeslet: the derivative of Eq. (res_stokeslet) (Sec. 5.2) with Phi' = -2 phi
 * (Eq. (def_erfc_like_fcn)):  S_R = A(r) I + C(r) x x^T gives
 *   d_m (S_R f)_j = A'(r) x_m/r f_j + C'(r) x_m/r x_j (x.f) + C (delta_jm (x.f) + x_j f_m).
 * Stresslet: the derivative of Eq. (res_stresslet) written as
 * u_j = D(r) [g_j (x.n) + x_j (g.n) + n_j (x.g)] + E(r) x_j (x.g)(x.n):
 *   d_m u_j = D'(r) x_m/r V_j + D (g_j n_m + delta_jm (g.n) + n_j g_m)
 *           + E'(r) x_m/r x_j (x.g)(x.n) + E (delta_jm (x.g)(x.n) + x_j (g_m (x.n) + (x.g) n_m)),
 * V_j the bracket of D; every precision takes FP64 pair terms for it.
 * MIXED plans take float-float pair terms for the gradient at every eps (FP32
 * gradient terms, ~1/r^3, would carry a relative l2 error near 2e-5); a plan
 * with FP32 velocity pair terms (eps >= 2e-7) allocates the gradient
 * workspace (208 bytes per point) on its first eval_grad or eval_adjoint call,
 * and host-synchronises that call. */
dmk_status_t dmk_stokes_eval_grad(dmk_stokes_plan_t plan, const double* d_f, const double* d_g,
                                  const double* d_n, double* d_u, double* d_gradu, void* stream);

/* Adjoint (reverse mode) of the 3D Stokeslet near component u = S[f] (eval
 * with one force column) with the tree, hence every nu_ts, held fixed:
 * for a scalar L with cotangent w = dL/du,
 *   d_v  [n][3]  dL/df = S[w]: S_R is even and symmetric, so the operator is
 *                its own transpose; the self term is the forward one on w;
 *   d_gx [n][3]  dL/dx_t = sum_s G(w_t, f_s; x) + G(f_t, w_s; x), x = x_t - x_s,
 *                G(a, b; x)_m = sum_j a_j d_m (S_R b)_j
 *                             = [A1 (a.b) + C1 (x.a)(x.b)] x_m + C [a_m (x.b) + b_m (x.a)]
 *                with A1 = A'/r, C1 = C'/r of the gradient above (the self term
 *                does not depend on x).
 *   d_f [n][3] forces, d_w [n][3] cotangents (device, caller order).
 * One symmetric pass evaluates each pair once for both points and recomputes
 * the pair terms (nothing is stored per pair); MIXED plans take float-float
 * pair terms (nearly coincident pairs in FP64), FP64 plans FP64.  The first
 * call allocates the adjoint workspace (128 bytes per point MIXED, 96 FP64)
 * and host-synchronises.  Both outputs come from FP64 atomic additions
 * (reproducible to the order of those additions).  Stresslet, 2D and several
 * force columns: DMK_ERR_UNSUPPORTED. */
dmk_status_t dmk_stokes_eval_adjoint(dmk_stokes_plan_t plan, const double* d_f, const double* d_w, double* d_v,
                                     double* d_gx, void* stream);

/* Autotuner (no paper counterpart; the paper fixes n_s per eps, Sec. 8):
 * builds and evaluates a plan (dmk_stokes_plan + dmk_stokes_eval + destroy,
 * targets = sources) for every candidate leaf capacity h_leaf_capacity[k],
 * times each `repeats` times on `stream` with CUDA events after one untimed
 * run, and returns the median times in h_ms[n_cand] (may be NULL) and the
 * index of the fastest in *h_best.  The leaf capacity sets the tree: for
 * components = DMK_COMPONENTS_ALL it sets the balance between the near pass
 * (work per target grows with n_s) and the far field (work per box); for
 * DMK_COMPONENTS_EWALD it sets the uniform level of the Ewald split (the
 * smallest level with at most that many points per box), i.e. the balance
 * between the near pass and the Fourier part; for the near component alone
 * the smallest leaves always win (the far field that balances them is not part
 * of that component).  d_u receives the velocity of the last run.
 * Host-synchronises. */
dmk_status_t dmk_stokes_autotune(const dmk_stokes_opts_t* opts, int64_t n_src, const double* d_src,
                                 const double* d_f, const double* d_g, const double* d_n, double* d_u,
                                 int32_t n_cand, const int32_t* h_leaf_capacity, int32_t repeats, void* stream,
                                 double* h_ms, int32_t* h_best);

/* dmk_stokes_eval with the time of each stage (tracing; no paper counterpart):
 * CUDA events on `stream` between the stages, read after the evaluation (the call
 * host-synchronises).  h_stage_ms[n_stages] (n_stages <= 9) receives, in ms:
 *   [0] near pass (residual pairs, self term, periodic stresslet zero mode),
 *   [1] source Lagrange weights and leaf proxy charges, [2] child merges,
 *   [3] outgoing plane waves with the kernel contraction, [4] colleague sums,
 *   [5] incoming plane waves to the potential grids, [6] root kernel,
 *   [7] interpolation to the children, [8] leaf grids at the targets.
 * Stages 1..8 are zero for plans without the far field.  Not for the gradient. */
dmk_status_t dmk_stokes_eval_traced(dmk_stokes_plan_t plan, const double* d_f, const double* d_g, const double* d_n,
                                    double* d_u, void* stream, double* h_stage_ms, int32_t n_stages);

/* Far-field sizes of a components = DMK_COMPONENTS_ALL plan (host values):
 *   info[0] proxy order p, [1] plane-wave modes a side N1, [2] root modes a
 *   side, [3] boxes of the tree (all levels), [4] boxes holding sources,
 *   [5] boxes holding targets, [6] finest level, [7] 1 if the far field runs
 *   in float32, 0 in float64.  All zero for other plans. */
dmk_status_t dmk_stokes_far_info(dmk_stokes_plan_t plan, int32_t info[8]);

/* Diagnostics of the far field's tensor-core kernels (no paper counterpart): runs
 * on `stream` one block that allocates tensor memory and waits on an mbarrier that
 * nothing completes, with a limit of ~1 ms of SM clock instead of the kernels' ~2 s,
 * and sets *h_timed_out = 1 when the wait ran out and was reported in the status
 * word the way the kernels report it (then freeing the tensor memory).  The device
 * stays usable afterwards.  Host-synchronises. */
dmk_status_t dmk_stokes_tc_wait_selftest(void* stream, int32_t* h_timed_out);

/* Synchronises the plan's last stream and returns the latched device status
 * (DMK_OK, DMK_ERR_OUT_OF_RANGE, DMK_ERR_INVALID_ARG for a non-finite point). */
dmk_status_t dmk_stokes_sync_status(dmk_stokes_plan_t plan);

/* Tree statistics (host values, valid after dmk_stokes_plan returned DMK_OK):
 *   stats[0] leaves, [1] max leaf level, [2] near-list entries,
 *   [3] tiles, [4] issued pairs (sum over targets of the points in their
 *   near leaves, the target itself excluded), [5] bandlimit c (as integer
 *   3c/pi), [6] leaf capacity n_s, [7] points,
 *   [8] useful pairs (0 < r < nu_ts, decided in float64; counted by a GPU
 *   kernel on the first call), [9] kernel launches issued by this library for
 *   this plan so far (plan build, evaluations and the pair count).
 * Host-synchronises. */
dmk_status_t dmk_stokes_plan_stats(dmk_stokes_plan_t plan, int64_t stats[10]);

/* Copies the plan's tree to HOST arrays (any pointer may be NULL):
 *   perm[n]        sorted position -> original index.  Points are sorted by
 *                  the Morton key of their finest cell; a plan with FP32 pair
 *                  terms (MIXED, eps >= 2e-7) then orders the points inside
 *                  each leaf by the Hilbert curve over the leaf's sub-cells
 *                  three levels down (four in 2D; Morton order inside a
 *                  sub-cell, leaves within that many levels of the maximum
 *                  level unchanged), which makes the 32-point tiles compact.
 *   leaf_level[L], leaf_start[L], leaf_count[L], leaf_coords[L][dim] (box
 *   coordinates at the leaf's level), near_off[L+1], near_leaf[E],
 *   near_q[E][dim] (periodic image offsets q, displacement (w_t - w_s) + q).
 * Sizes L, E from dmk_stokes_plan_stats.  Host-synchronises. */
dmk_status_t dmk_stokes_plan_tree(dmk_stokes_plan_t plan, int32_t* perm, int32_t* leaf_level,
                                  int32_t* leaf_start, int32_t* leaf_count, int64_t* leaf_coords,
                                  int32_t* near_off, int32_t* near_leaf, int32_t* near_q);

/* Host-only query of the kernel tables for (dim, eps, kernels): bandlimit c,
 * phi(0) and the polynomial coefficients (monomials in t = 2 rho^2 - 1) of the
 * residual functions; no GPU needed.
 *   out_c, out_phi0   scalars (may be NULL)
 *   which             3D: 0 gS, 1 hS, 2 pT, 3 qT, 4 dgS/ds, 5 dhS/ds, with
 *                     gS = (Sdiag-1)/rho, hS = (Soffd-1)/rho, pT = Tdiag/rho,
 *                     qT = (Toffd-1)/rho (Sec. 5.2 functions at rho = r/nu);
 *                     2D: 0 m_d, 1 m_o, 2 m_td, 3 m_to, the mollified App. B
 *                     functions Mdiag/r, Moffd/r^3, MTdiag/r^3, MToffd/r^5 at
 *                     unit scale, and 6 their limit Mdiag(r)/r at r = 0
 *                     (one value, Eq. (msdiag0))
 *   fp32              0 the float64 table, 1 the float32 table
 *   coef, max_terms   output buffer; returns the number of terms in *n_terms. */
dmk_status_t dmk_stokes_kernel_table(int32_t dim, double eps, int32_t kernels, int32_t which,
                                     int32_t fp32, double* out_c, double* out_phi0,
                                     double* coef, int32_t max_terms, int32_t* n_terms);

/* Sharding one system over n_ranks GPUs (host-only, no GPU needed; no paper
 * counterpart: the paper's code is single-threaded, Sec. 8).  The near pass
 * needs, for a target leaf, only the sources of its near list (FMM list 1,
 * remark after Step 4 of Sec. 6.1).  Leaves are in Morton order, so contiguous
 * leaf ranges are compact; dmk_stokes_partition_leaves splits [0, n_leaf) into
 * n_ranks contiguous ranges [leaf_begin[r], leaf_begin[r+1]) of about equal
 * issued pairs, cost(leaf) = targets(leaf) x sum_{X in near(leaf)} sources(X).
 *   leaf_count[n_leaf]   sources per leaf; leaf_tcount[n_leaf] targets per
 *                        leaf (NULL: the sources are the targets)
 *   near_off[n_leaf+1], near_leaf[E]   the near lists (dmk_stokes_plan_tree)
 *   leaf_begin[n_ranks+1] (out), rank_cost[n_ranks] (out, may be NULL)
 * dmk_stokes_halo_leaves lists, sorted and unique, the leaves outside
 * [begin, end) that appear in the near lists of the leaves inside: the
 * sources whose densities a rank owning [begin, end) receives before its pass.
 *   halo[max_halo] (out, may be NULL to query *n_halo), *n_halo (out).
 * Both return DMK_ERR_INVALID_ARG for bad sizes or NULL required pointers. */
dmk_status_t dmk_stokes_partition_leaves(int32_t n_leaf, const int32_t* leaf_count, const int32_t* leaf_tcount,
                                         const int32_t* near_off, const int32_t* near_leaf, int32_t n_ranks,
                                         int32_t* leaf_begin, int64_t* rank_cost);
dmk_status_t dmk_stokes_halo_leaves(int32_t n_leaf, const int32_t* near_off, const int32_t* near_leaf,
                                    int32_t begin, int32_t end, int32_t* halo, int32_t max_halo,
                                    int32_t* n_halo);

/* Releases the plan (device memory is freed on the plan's stream). NULL is ignored. */
void dmk_stokes_destroy(dmk_stokes_plan_t plan);

/* Message of the last error on this plan, or of the last failed call on this
 * thread when plan == NULL.  The string is owned by the library. */
const char* dmk_stokes_last_error(dmk_stokes_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* DMK_STOKES_H_ */
