/*
 * dmk.h -- C ABI of the B300-native periodized DMK library (libdmk_b300.so).
 *
 * Evaluates, for N points x_t in the cuboid [0,L1) x [0,L2) x [0,L3) with the first D
 * directions periodic, the sums of Eq. periodic_sum (Sec. 1):
 *
 *     u(x_t) = sum_s sum*_{p in P_D} K(x_t - x_s + p) rho_s ,
 *
 * where P_D is the lattice of periodic images of Eq. periodic-images and "*" drops p = 0
 * when x_t = x_s, by the periodized dual-space multilevel kernel-splitting method:
 * leaf residual sums over periodically wrapped neighbour lists (Sec. 2.3, Eq. u_local),
 * per-level difference-kernel plane-wave interactions (Sec. 2.3 Eq. Dl_int_discr,
 * Sec. 3.1.4) and the root-level Fourier far field (Sec. 4.3, 4.4, 5.3; on tilings of several
 * cubes the sums over the cubes as DFTs over the cube index, Sec. 3.4, 5.4).  In dmk_eval the
 * sources are the targets (Sec. 1); dmk_eval_targets takes a separate target set.  Kernels:
 * Laplace K = 1/(4 pi r) and the Stokeslet, stresslet and rotlet of App. B.
 *
 * Conventions shared by every entry point
 *   - Arrays are plain pointers, row-major, FP64, owned by the caller.  "device" pointers
 *     must be CUDA device (or managed) memory on the current device; "host" pointers are
 *     ordinary host memory (pinned memory gives faster copies).
 *   - Every call returns a dmk_status_t; nothing aborts, exits or traps.  On an error the
 *     outputs are left unspecified and dmk_last_error() gives a one-line detail.
 *   - A plan owns its tables and a device workspace that grows on demand; calls on one
 *     plan must not overlap (the plan is not thread-safe).  Work is enqueued on the plan's
 *     CUDA stream; the residual sums of the leaf stage (p <= 24; they need only the tree)
 *     go to a second stream the plan owns, beside the far field, ordered against the first
 *     by events (dmk_set_pair_overlap).  dmk_eval returns after all of it is complete (the
 *     host waits for the small readbacks of the tree build and for the device status word).
 *   - Environment, read when a plan is created: DMK_PAIR_OVERLAP=0 runs the residual sums
 *     in order on the plan's stream instead; DMK_PAIR_BLOCKS=n caps their resident blocks
 *     per SM beside the far field (default 0 = no cap).
 */
#ifndef DMK_B300_H
#define DMK_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DMK_LAPLACE = 0,    /* K = 1/(4 pi r); rho scalar; u scalar                                    */
    DMK_STOKESLET = 1,  /* App. B Eq. stokeslet_def_deriv; rho = force (3); u = velocity (3)        */
    DMK_STRESSLET = 2,  /* App. B Eq. stresslet_def_deriv; rho = Q_lm = q_l n_m, l-major (9); u (3) */
    DMK_ROTLET = 3      /* App. B Eq. rotlet_def_deriv; rho = torque (3); u (3)                     */
} dmk_kernel_t;

typedef enum {
    DMK_FP64 = 0,       /* plain path: every stage in FP64                                          */
    DMK_MIXED = 1       /* FP32 residual sums, expansions and Chebyshev stages with box-relative
                           coordinates; FP64 root Fourier sum, self correction, final accumulate  */
} dmk_precision_t;

typedef enum {
    DMK_OK = 0,
    DMK_ERR_INVALID_ARG = 1,   /* bad kernel, D, lengths, tol, n_s or a NULL pointer             */
    DMK_ERR_OUT_OF_DOMAIN = 2, /* a free (non-periodic) coordinate outside [0, L_i), or non-finite */
    DMK_ERR_NOT_NEUTRAL = 3,   /* Laplace with D = 1, 2 needs sum rho = 0 (Sec. 5.2)               */
    DMK_ERR_UNSUPPORTED = 4,   /* a tiling of more than 1024 cubes; dmk_eval_shard on a
                                  non-exact tiling                                               */
    DMK_ERR_TREE_DEPTH = 5,    /* reserved, never returned: a box at the depth cap (18 levels below
                                  a cube) that holds more than n_s points (coincident or nearly
                                  coincident points) stays a leaf, the result is still the
                                  method's, and dmk_stats_t.n_capped_leaves counts such boxes     */
    DMK_ERR_OOM = 6,           /* device allocation failed                                        */
    DMK_ERR_CUDA = 7,          /* a CUDA call failed; see dmk_last_error                          */
    DMK_ERR_TIMEOUT = 8        /* reserved: no device-side wait exists in this library            */
} dmk_status_t;

typedef struct dmk_plan_s* dmk_plan_t;

/* Plan for kernel k with D periodic directions (0..3) on the cell L1 x L2 x L3 and a
 * requested relative tolerance tol in [1e-12, 1e-3].  The tolerance selects the row of the
 * paper's parameter tables (Table 1 for Laplace, Table 5 for the Stokes kernels; Sec. 6.1):
 * the PSWF band limit c, the Chebyshev order p and n_f = ceil(3c/pi) - 1; a tol between
 * rows takes the next stricter row.  The cube side is s = min of the periodic lengths
 * (max L_i for D = 0); free lengths are rounded up to multiples of s (Sec. 4.1, Sec. 5).  A
 * periodic length that s does not divide is tiled by ceil(L_i / s) cubes, the last one cut,
 * plus one padding cube on each side; the periodic images of the sources in the padded
 * domain are added as sources and the structure factor counts the sources inside the cell
 * only (Sec. 4.1.1, 4.1.2, 4.3).
 * Defaults: precision DMK_MIXED, n_s = 250 (Sec. 6), the legacy default stream.
 * On success *out receives a plan to be released with dmk_destroy. */
dmk_status_t dmk_plan(dmk_kernel_t k, int D, double L1, double L2, double L3, double tol,
                      dmk_plan_t* out);

/* As dmk_plan, with the precision path, the leaf capacity n_s (>= 1; the maximum number of
 * points in a leaf box, Sec. 3.1.1, which changes speed but not accuracy, Sec. 6) and the
 * CUDA stream (a cudaStream_t, or NULL for the legacy default stream). */
dmk_status_t dmk_plan_ex(dmk_kernel_t k, int D, const double L[3], double tol,
                         dmk_precision_t prec, int n_s, void* cuda_stream, dmk_plan_t* out);

/* Evaluate the sums for N >= 0 points.
 *   points      device, N x 3: positions; periodic coordinates may lie anywhere (they are
 *               wrapped into [0, L_i)), free coordinates must lie in [0, L_i).
 *   strengths   device, N x d_rho (1, 3, 9, 3 for the four kernels).
 *   potentials  device, N x d_u (1, 3, 3, 3): u(x_t) in input order.
 *   grad        device, or NULL to skip: N x 3 x d_u with grad[t][i][j] = d u_j / d x_i at
 *               x_t (the field gradient at the target; for Laplace the force on t is
 *               -rho_t grad[t][.][0]).
 * D = 3 Laplace with non-zero net charge drops the k = 0 mode (neutralising background,
 * Sec. 1 footnote).  N = 0 returns DMK_OK without touching the arrays. */
dmk_status_t dmk_eval(dmk_plan_t plan, int64_t N, const double* points, const double* strengths,
                      double* potentials, double* grad);

/* Same as dmk_eval with HOST arrays: the library copies points and strengths to the device,
 * evaluates, and copies potentials (and grad) back before returning. */
dmk_status_t dmk_eval_host(dmk_plan_t plan, int64_t N, const double* points, const double* strengths,
                           double* potentials, double* grad);

/* Vector-Jacobian product of dmk_eval, the reverse-mode derivative used for training-style
 * differentiation (not in the paper).  For a scalar L(u) with upstream gradient g = dL/du
 * (N x d_u), u = dmk_eval(points, strengths):
 *   d_strengths[s][l] = dL/drho_s,l = sum_t sum_j K_jl(x_t - x_s) g_t,j = v_l(x_s),
 *   d_points[a][i]    = dL/dx_a,i  = sum_j grad_u[a][i][j] g_a,j + sum_l grad_v[a][i][l] rho_a,l,
 * where v is the sum of Eq. periodic_sum with strengths g.  This holds for the kernels with
 * K(-x) = K(x)^T -- Laplace, Stokeslet, rotlet -- so one more evaluation of the whole method
 * (residual sums, plane waves, root far field) with strengths g and target gradients gives
 * both; the assembly of d_points runs on the GPU too.
 *   points, strengths  device, as passed to dmk_eval (N x 3, N x d_rho).
 *   grad_u             device, N x 3 x d_u: the grad output of that dmk_eval.
 *   g                  device, N x d_u: upstream gradient; need not sum to zero.  For Laplace
 *                      with D = 1, 2 a net sum is allowed here: the free-direction zero mode is
 *                      then the truncated Green's function of Sec. 5.2, which differs from any
 *                      other regularisation by a constant, so d_points is exact and
 *                      d_strengths is exact up to an additive constant (which no neutral
 *                      change of the strengths sees).
 *   d_strengths        device, N x d_rho, or NULL to skip.
 *   d_points           device, N x 3, or NULL to skip.
 * The stresslet (d_rho = 9 != d_u = 3) is not self-adjoint, but its periodized kernel
 * T_jlm = -delta_jm P_l + d_m G_jl + d_j G_ml is fully symmetric in (j, l, m) and odd in x, so
 *   d_strengths[s][3 l + m] = -S[g (x) e_m]_l(x_s),
 *   d_points[a][i] = sum_j grad_u[a][i][j] g_a,j - sum_lm Q_a,lm d_i S[g (x) e_m]_l(x_a),
 * S[Q] the stresslet sum with strengths Q: three evaluations with the strengths g (x) e_m.
 * Workspace as dmk_eval; the call returns after the results are complete. */
dmk_status_t dmk_vjp(dmk_plan_t plan, int64_t N, const double* points, const double* strengths,
                     const double* grad_u, const double* g, double* d_strengths, double* d_points);

/* One rank's part of an evaluation split over cubes (spatial sharding; a multi-GPU use of the
 * method, not in the paper).  The structure factor of Sec. 4.3 (Eq. structurefac) is a sum
 * over the cubes of the tiling, and the near field of a target (plane waves and residual sums,
 * Sec. 3.1.4-3.1.5) reaches only the cubes adjacent to its own.  A rank that owns a set of
 * cubes therefore evaluates its own targets from its own points plus those of the adjacent
 * cubes ("ghosts"), once the partial structure factors of all ranks are summed.
 *   points, strengths  device, N x 3 and N x d_rho: the n_own points of the rank's cubes first,
 *                      then the ghost points (every point of every cube adjacent to an owned
 *                      cube that the rank does not own, periodic neighbours included).
 *   potentials, grad   device, n_own x d_u and n_own x 3 x d_u (grad may be NULL): the results
 *                      for the owned points, in their order.
 *   cube_owned         host, M1 M2 M3 ints, cube m1 + M1 (m2 + M2 m3) owned if nonzero: only
 *                      those cubes enter this rank's partial structure factor.
 *   reduce             called once per call with the rank's partial sums -- n doubles at chi,
 *                      pinned HOST memory owned by the plan, valid during the call: the structure
 *                      factor (n - 2 d_rho doubles, complex pairs), then the d_rho sums of the
 *                      owned strengths and the d_rho sums of their absolute values (the total
 *                      strength enters the constants of the truncated kernels, Sec. 5) -- and
 *                      ctx; it must replace the n doubles by their sum over all ranks (an
 *                      all-reduce over any host transport) and return 0.  Nonzero returns
 *                      DMK_ERR_CUDA.  Every rank's call reduces the same n, a rank with N = 0
 *                      included.
 * Exact tilings only (DMK_ERR_UNSUPPORTED otherwise).  The sum of the strengths is not checked
 * (no rank sees all of them).  The result for an owned point is that of dmk_eval on all points
 * when the forest of the owned and ghost cubes is that of the whole problem there (2:1 balance
 * of Sec. 3.1.1 propagating no further than one cube); the call returns when the results are
 * complete. */
typedef int (*dmk_chi_reduce_fn)(double* chi, int64_t n, void* ctx);

dmk_status_t dmk_eval_shard(dmk_plan_t plan, int64_t N, int64_t n_own, const double* points, const double* strengths,
                            double* potentials, double* grad, const int* cube_owned, dmk_chi_reduce_fn reduce,
                            void* ctx);

/* Separate target set: u(y_t) = sum_s sum*_p K(y_t - x_s + p) rho_s at M targets y_t that need
 * not be sources (Eq. periodic_sum with the targets apart from the sources; terms with
 * y_t - x_s + p = 0 are skipped).  The forest is built on sources and targets together (the
 * targets enter as points of zero strength), so a target's value is the one dmk_eval gives a
 * zero-strength point at y_t.
 *   sources, strengths  device, N x 3 and N x d_rho (N >= 0; N = 0 gives zeros)
 *   targets             device, M x 3, wrapped and checked like the sources
 *   potentials, grad    device, M x d_u and M x 3 x d_u (grad may be NULL), target order
 * A target on a source (or on one of its periodic images) meets a singular term: the residual
 * sum skips the pair, and the smooth part of that term, K_M(0) rho_s, stays in the value.
 * Workspace as dmk_eval, plus (N + M) x (3 + d_rho) doubles for the joined point set; the call
 * is stream-ordered on the plan's stream like dmk_eval.  Errors as dmk_eval (the neutrality
 * test of D = 1, 2 Laplace is over the sources). */
dmk_status_t dmk_eval_targets(dmk_plan_t plan, int64_t N, const double* sources, const double* strengths,
                              int64_t M, const double* targets, double* potentials, double* grad);

/* dmk_eval without any device allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc at evaluation time -- applications whose
 * device memory is fully reserved by their own pool allocator and that must not let a
 * library allocate behind their back.
 *   - Same arguments, layouts and results as dmk_eval (device arrays; the plan, created
 *     beforehand with dmk_plan/dmk_plan_ex, owns its tables).
 *   - All workspace comes from one file-scope static device array of 64 MiB (every GPU that
 *     loads the library holds it until the process exits); nothing is allocated or freed.
 *   - N must lie in [0, 16384]; a larger N returns DMK_ERR_INVALID_ARG, and a problem whose
 *     workspace does not fit in 64 MiB (large p, FP64, deep trees) returns DMK_ERR_OOM, both
 *     with a message in dmk_last_error.
 *   - Like dmk_eval, the call cannot be captured into a CUDA graph: it waits on the host for
 *     small device readbacks during the tree build.  Its first call on a device also looks up
 *     the device address of the static array (a CUDA runtime query).
 *   - Every call shares the one array, which keeps the previous call's contents; the call
 *     clears everything it needs to start at zero.  Calls that overlap on the GPU (on
 *     different streams, plans or threads) race on the array and must be serialised. */
dmk_status_t dmk_eval_static(dmk_plan_t plan, int64_t N, const double* points, const double* strengths,
                             double* potentials, double* grad);

typedef struct {
    int32_t c_times_1000;      /* PSWF band limit c, times 1000                                  */
    int32_t p;                 /* Chebyshev order                                                */
    int32_t n_f;               /* plane-wave half width; N_F = 2 n_f + 1                          */
    int32_t n_root_modes;      /* retained root Fourier modes (rectangle points with nonzero weight) */
    int32_t n_levels;          /* tree levels (root cubes are level 0)                           */
    int32_t n_boxes;           /* boxes in the forest                                            */
    int32_t n_leaves;          /* leaf boxes                                                     */
    int32_t n_nonleaf;         /* non-leaf boxes (carry plane-wave expansions)                   */
    int64_t n_pairs;           /* source-target pairs visited by the residual sums               */
    int64_t n_direct_entries;  /* (target leaf, source box) entries of the direct lists          */
    int32_t kernel_launches;   /* CUDA kernels launched by the last evaluation                   */
    int32_t fit_terms;         /* Chebyshev terms of the residual function q used by the path    */
    float stage_ms[10];        /* last eval: tree, upward, root, plane waves, shift, leaf, total,
                                  residual kernel, expansion kernel, 0 (stages 7 and 8: p <= 24) */
    int32_t n_capped_leaves;   /* boxes at the depth cap holding more than n_s points (kept as leaves) */
    int32_t reserved;
    int64_t n_device_allocs;   /* device allocations (cudaMalloc, cudaMallocAsync) made by this plan
                                  since it was created, tables included; current at every call   */
} dmk_stats_t;

/* Statistics of the last evaluation on this plan (n_device_allocs: as of this call). */
dmk_status_t dmk_get_stats(dmk_plan_t plan, dmk_stats_t* out);

/* Residual sums beside the far field: with enable = 1 (the default) the leaf residual kernel
 * runs on a plan-owned second stream while the upward pass, root, plane waves and shifts run on
 * the plan's stream (they need only the tree); the leaf expansions wait for it.  At most
 * max_blocks_per_sm resident blocks of it per SM (0: as many as fit, the default).  The results
 * are bitwise the same either way.  enable = 0 runs everything on the plan's stream in order
 * (per-kernel timing with dmk_set_timing then measures each kernel alone).  The environment
 * variables DMK_PAIR_OVERLAP and DMK_PAIR_BLOCKS, read at plan creation, set the same. */
dmk_status_t dmk_set_pair_overlap(dmk_plan_t plan, int enable, int max_blocks_per_sm);

/* Enables (1) or disables (0) per-stage CUDA-event timing inside dmk_eval (stage_ms). */
dmk_status_t dmk_set_timing(dmk_plan_t plan, int enable);

/* Plan parameters computed on the host only (no device call): the values dmk_plan would use.
 * n_axis[i] = wavenumbers on root axis i of the first root part (periodic: 2 ceil(L_i c/(2 pi
 * nu_0)) + 1 integers, Eq. kintmax; free: 2 N + 1 trapezoidal nodes of step dk = pi/R with N
 * the smallest integer such that N dk > c/nu_0, Eqs. k1set-1p, k1k2set-2p); R = truncation radius
 * (0 for D = 3); n_root_modes = retained modes of all root parts; fit_terms_fp64/fp32 =
 * Chebyshev terms of the residual function q per path.
 * Root parts (D = 1, 2; Sec. 5.3 and the error estimates of App. E): where the trapezoidal
 * error estimate of the original kernel at the smallest nonzero periodic wavenumber, with its
 * Nyquist step pi/L_j, is at most tol in every free direction j, the modes with a nonzero
 * periodic wavenumber use the original symbol on that step (the second part) and the first part
 * keeps only the zero periodic wavenumber with the truncated symbols; otherwise one part, the
 * truncated symbol for every mode.
 * Sums over the cubes (Sec. 3.4 Cases 1 and 2, Sec. 5.4): root_dft_len[3 part + a] = Q_a, the
 * length of the DFT over the cube index along axis a that replaces the direct sum of Eqs.
 * structurefac and eval_tensor over the cubes -- M_a on an exactly tiled periodic axis, on a free
 * axis of step h the oversampled length 2 pi / (h s) (Eq. kappaqdef; it must be an integer
 * >= M_a), 1 on an axis of one cube.  All six are 0 where the direct sums over the cubes are used
 * (a single cube, a non-exact tiling, or a free step without an integer length). */
typedef struct {
    double c, s, R, dk;
    int32_t p, n_f, n_root_modes, fit_terms_fp64, fit_terms_fp32;
    int32_t M[3];
    int32_t n_axis[3];
    int32_t d_rho, d_u;
    int32_t root_dft_len[6];
} dmk_plan_info_t;

dmk_status_t dmk_plan_info(dmk_kernel_t k, int D, const double L[3], double tol, dmk_plan_info_t* out);

/* Copies one host-side plan table into out (FP64, host memory), for inspection and testing;
 * *n receives the number of doubles available (copies min(cap, *n)).  No device call.
 *   which = 0: root wavenumber axes, concatenated (n_axis[0] + n_axis[1] + n_axis[2]);
 *   which = 1: root weights C^{DP} G-hat(k) gamma-hat(|k| nu_0) on the rectangle, complex as
 *              (re, im) pairs, index ((i1 n2 + i2) n3 + i3) d_u d_rho + j d_rho + a (Sec. 4.3, 5.3);
 *   which = 2: level-0 difference-kernel scalar w_0 h_0^ord G_0(|h_0 m|) on the half grid,
 *              index ((m1 + n_f) N_F + (m2 + n_f)) (n_f + 1) + m3 (Sec. 2.3, Eq. Dl_int_discr);
 *   which = 3: PSWF window values phi(0), phi''(0), phi-hat''(0), then phi-hat at k = 0.099 c j,
 *              j = 0..10 (Sec. 2.2, Eqs. wfunc_pswf, wfunchat);
 *   which = 4: the FP32 path's piecewise cubic residual tables (App. B residual functions, the
 *              "precomputed polynomial approximations"): series q, f, g, dq/ds, df/ds, dg/ds of
 *              s = r^2/nu^2, with q(s) = int_0^r phi / r, f(s) = phi(r), g(s) = phi'(r)/r; 256
 *              intervals each, 4 coefficients per interval, index ((series 256 + i) 4 + c);
 *              X(s) = c0 + u (c1 + u (c2 + u c3)) with u = 256 s - i;
 *   which = 5, 6: as 0 and 1 for the second root part (no doubles when there is none). */
dmk_status_t dmk_plan_table(dmk_kernel_t k, int D, const double L[3], double tol, int which, double* out,
                            int64_t cap, int64_t* n);

/* Releases the plan, its tables and workspace.  NULL is accepted. */
dmk_status_t dmk_destroy(dmk_plan_t plan);

/* Static text for a status code. */
const char* dmk_status_string(dmk_status_t s);

/* Detail of the last error on this plan (plan-owned text, valid until the next call on it);
 * with plan == NULL, the detail of the last failed dmk_plan/dmk_plan_ex in this thread. */
const char* dmk_last_error(dmk_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* DMK_B300_H */
