/*
 * nphc.h -- C ABI of the GB300 library for numerical polynomial homotopy continuation
 * (NPHC): all stationary points of the power-law XY ring, after D. Mehta, "Finding All
 * the Stationary Points of a Potential Energy Landscape via Numerical Polynomial
 * Homotopy Continuation Method", arXiv:1104.5497.
 *
 * The calls follow the paper's statement of the method:
 *   build the polynomial system from N, sigma and the couplings
 *       (section "A First Application", Eq. alg_dec_XY_model_poly, theta_N = 0),
 *   track every path of the total-degree gamma-trick homotopy
 *       (section "Numerical Polynomial Homotopy Continuation Method"),
 *   refine, apply the solution and real tolerances and certify with alpha-theory
 *       (same section: Delta_sol, Delta_R, alphaCertified),
 *   classify the real stationary points by Hessian index and energy
 *       (introduction: minima have no negative Hessian eigenvalue; section
 *       "A First Application": theta_k = atan2(s_k, c_k), V).
 *
 * Conventions (every call):
 *   - Every call returns an nphc_status; none aborts or exits.  On failure
 *     nphc_last_error() returns a message (thread-local, valid until the next call on
 *     the same thread).
 *   - Handles (nphc_system, nphc_result) are created and destroyed by the library.
 *     Buffers passed in are owned by the caller.
 *   - "Device" pointers are CUDA global-memory pointers on the current device; "host"
 *     pointers are ordinary CPU memory.  Which one is stated per argument.
 *   - Calls that take a stream (a cudaStream_t passed as void*, NULL = legacy default
 *     stream) are asynchronous and stream-ordered.  nphc_solve and the nphc_result_copy_*
 *     calls synchronise.
 *   - Per-path failures are statuses in the endpoint arrays, not call failures.
 *
 * Unknowns are ordered z = (c_1..c_m, s_1..s_m), m = N-1, c_k = cos theta_k,
 * s_k = sin theta_k; equation k (< m) is the gradient equation of site k and equation
 * m+k is c_k^2 + s_k^2 - 1.  Path p starts at z_i = -1 if bit i of p is set, else +1.
 * Device endpoint arrays are structure-of-arrays: component i of entry e is at
 * [i * count + e].
 */
#ifndef NPHC_H
#define NPHC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NPHC_MIN_N 3
#define NPHC_MAX_N 13

typedef enum nphc_status {
    NPHC_OK = 0,
    NPHC_EINVAL = 1,   /* invalid argument (N out of range, non-finite or asymmetric J, |gamma| = 0, NULL) */
    NPHC_ENOMEM = 2,   /* device or host allocation failed */
    NPHC_ECUDA = 3,    /* a CUDA call failed; nphc_last_error() has the CUDA message */
    NPHC_EBUDGET = 4,  /* a device-side iteration limit fired (the run's watchdog) */
    NPHC_ESTATE = 5    /* call out of order (e.g. results requested before a solve) */
} nphc_status;

typedef enum nphc_precision {
    NPHC_PREC_FP64 = 0,   /* plain: every step in FP64 */
    NPHC_PREC_MIXED = 1   /* FP32 tracking (compensated corrector residual), FP64 hand-off,
                             re-track, refinement, certification and classification */
} nphc_precision;

/* Tracking outcome of one path. */
enum {
    NPHC_PATH_RUNNING = 0,
    NPHC_PATH_REACHED = 1,      /* tracked to t = 1 */
    NPHC_PATH_DIVERGED = 2,     /* ||z||_inf beyond the divergence radius before t = 1 */
    NPHC_PATH_MIN_STEP = 3,     /* step size fell below h_min */
    NPHC_PATH_STEP_BUDGET = 4,  /* more than max_steps step attempts */
    NPHC_PATH_NONFINITE = 5,    /* NaN or Inf in the state */
    NPHC_PATH_HANDOFF = 6,      /* FP32 tracking stopped; FP64 continues from (z, t, h) */
    NPHC_PATH_HANDOFF_COND = 7  /* FP32 tracking stopped at a step whose condition estimate
                                   exceeded kappa_fp32; FP64 continues from (z, t, h) */
};

/* Class of one endpoint after refinement, certification and deduplication. */
enum {
    NPHC_END_NONE = 0,       /* diverged path: no endpoint */
    NPHC_END_SINGULAR = 1,   /* reached t = 1 but does not certify (singular or not a solution) */
    NPHC_END_REAL = 2,       /* certified approximate solution, certified real */
    NPHC_END_NONREAL = 3,    /* certified approximate solution, certified non-real */
    NPHC_END_UNDECIDED = 4,  /* certified approximate solution, reality undecided */
    NPHC_END_DUPLICATE = 5,  /* certified, but a lower path reached the same solution */
    NPHC_END_FAILED = 6      /* tracking stopped before t = 1 without diverging */
};

/* Tuning and tolerances.  nphc_options_default() fills the defaults given here. */
typedef struct nphc_options {
    nphc_precision precision;  /* NPHC_PREC_MIXED */
    double gamma_re, gamma_im; /* the homotopy's random complex gamma; default exp(0.5 i) */
    double tol_sol;            /* Delta_sol: ||P(z)||_inf at the refined point, 1e-10 */
    double tol_real;           /* Delta_R: max |Im z_k| of a real solution, 1e-7 */
    double h0, h_max, h_min;   /* first, largest and smallest step in t: 0.01, 0.05, 1e-14 */
    double eps_fp32;           /* FP32 corrector: accept when ||dz|| <= eps (1 + ||z||), 1e-5 */
    double eps_fp64;           /* FP64 corrector tolerance, 1e-9 */
    double trust;              /* FP64: reject when the first correction exceeds trust (1 + ||z||), 0.1 */
    double trust_fp32;         /* FP32: the same bound on the prediction error, 2e-3 (no wider
                                  than what the FP64 corrector's tolerance implies) */
    double r_div;              /* divergence radius: a path whose ||z||_inf exceeds it before
                                  t = 1 goes to infinity (both precisions), 1e8 */
    int max_newton_fp32;       /* corrector iterations per FP32 step, 3 */
    int max_newton_fp64;       /* corrector iterations per FP64 step, 3 */
    int max_steps;             /* step attempts per path, 5000 */
    int max_steps_fp32;        /* step attempts per path in the FP32 pass before hand-off, 400 */
    int crawl_steps_fp32;      /* FP32 hands a path off when, once 1 - t < 1e-3, 1 - t fails to
                                  halve within this many accepted steps, 32 (0: never) */
    int grow_after;            /* consecutive accepted steps before h doubles, 3 */
    int refine_iters;          /* Newton refinement steps at t = 1, 8 */
    double refine_eps;         /* refinement stops when ||dz|| <= eps (1 + ||z||), 1e-14 */
    int block_size;            /* threads per block of the FP32 tracker; 0 = automatic */
    int blocks_per_sm;         /* resident blocks per SM of the FP32 tracker; 0 = automatic */
    /* Cauchy endgame (nphc_endgame) */
    int endgame;               /* nphc_solve_into runs the endgame on every path that ends
                                  NPHC_END_SINGULAR or NPHC_END_FAILED, 0 (off) */
    double eg_r0;              /* first radius |1 - t| of the turns around t = 1, 1/16 */
    double eg_ratio;           /* ratio between successive radii, 1/4 */
    int eg_radii;              /* most radii tried, 8 */
    int eg_samples;            /* samples per turn, 16 */
    int eg_max_cycle;          /* largest cycle number tried, 8 */
    double eg_tol_close;       /* a turn closes when ||z - z_start|| <= tol (1 + ||z_start||), 1e-6 */
    double eg_tol_conv;        /* two estimates agree when ||e_k - e_k-1|| <= tol (1 + ||e_k||), 1e-9 */
    double eg_h_min;           /* smallest endgame step, in sample intervals, 1/4096 */
    int eg_max_attempts;       /* endgame step attempts per path, 4000 */
    int list_blocks_per_sm;    /* blocks (of 4 warps) per SM of the FP64 list tracker (hand-offs,
                                  re-tracks; one path per warp); 0 = automatic (2) */
    double kappa_sing;         /* an endpoint is singular (never certified) when its Jacobian's
                                  Frobenius condition number ||DP||_F ||DP^-1||_F exceeds
                                  kappa_sing max(1, ||z||_inf^2), 1e12 */
    int threads_per_path;      /* FP64 tracking of lists (hand-offs, re-tracks): 32 = one path
                                  per warp (the path's solve shared over the lanes), 1 = one
                                  path per thread (every lane a path); 0 = automatic (one path
                                  per warp) */
    double kappa_fp32;         /* FP32 pass: a converged step whose solves' condition estimate
                                  exceeds this is not taken and FP64 continues the path
                                  (NPHC_PATH_HANDOFF_COND, see nphc_track); FP32 solves lose
                                  about kappa x 6e-8 of their relative accuracy.  The
                                  estimate is max/min |U_kk| of the solve's pivoted LU
                                  factor.  0 = no such test; 3e5 */
} nphc_options;

typedef struct nphc_system nphc_system;   /* opaque; owns the device copy of the couplings */
typedef struct nphc_result nphc_result;   /* opaque; owns device buffers for all paths */

/* Device endpoint arrays, caller-owned, for the step-by-step calls below.  count
 * entries; n = 2(N-1) components per point.  Any output pointer may be NULL where a
 * call does not write it; with count = 0 every array may be NULL. */
typedef struct nphc_endpoints {
    int64_t count;
    int64_t *path;       /* [count] path index of each entry (input) */
    double *z_re;        /* [n * count] current or final point, real parts */
    double *z_im;        /* [n * count] imaginary parts */
    double *t;           /* [count] homotopy time reached */
    double *h;           /* [count] step size to resume with */
    int32_t *status;     /* [count] NPHC_PATH_* */
    int32_t *steps;      /* [count] accepted steps (cumulative over calls) */
    int32_t *solves;     /* [count] linear solves spent (cumulative; flop accounting) */
    int32_t *newton;     /* [count] of which corrector (Newton) solves */
    int32_t *cls;        /* [count] NPHC_END_* */
    double *alpha;       /* [count] alpha = beta * gamma bound at the certified point */
    double *beta;        /* [count] ||DP^-1 P|| */
    double *gamma;       /* [count] ||DP^-1||_F ||D^2 P / 2|| (bound on Smale's gamma) */
    double *resid;       /* [count] ||P(z)||_inf at the refined point */
} nphc_endpoints;

/* Fills *opt with the defaults listed in nphc_options.  NPHC_EINVAL if opt is NULL. */
nphc_status nphc_options_default(nphc_options *opt);

/* Couplings of the power-law ring (section "A First Application", the potential V):
 * J_ij = d_ij^-sigma with d_ij = min(|i-j|, N-|i-j|), J_ii = 0, each scaled by
 * (1 + eps * g_ij) when g (host, N*N row-major, symmetric) is not NULL.  J_out: host,
 * N*N row-major.  NPHC_EINVAL for N outside [NPHC_MIN_N, NPHC_MAX_N], non-finite sigma,
 * asymmetric g, or a scaled coupling <= 0. */
nphc_status nphc_xy_couplings(int N, double sigma, const double *g, double eps, double *J_out);

/* The couplings' vector-Jacobian product with respect to sigma: given dL/dJ (host, N*N
 * row-major: the gradient of a loss L with respect to every entry of the matrix that
 * nphc_xy_couplings returns for the same arguments), writes
 *   *dsigma = sum_{i != j} dL/dJ_ij dJ_ij/dsigma,  dJ_ij/dsigma = -ln(d_ij) J_ij
 * (J_ij = d_ij^-sigma (1 + eps g_ij); the paper's couplings with sigma its alpha, section
 * "A First Application").  The diagonal of dL/dJ is ignored.  Errors as for
 * nphc_xy_couplings, and NPHC_EINVAL for a NULL dL_dJ or dsigma. */
nphc_status nphc_xy_couplings_vjp(int N, double sigma, const double *g, double eps,
                                  const double *dL_dJ, double *dsigma);

/* Builds the polynomial system of Eq. (alg_dec_XY_model_poly) for the ring with
 * couplings J (host, N*N row-major, symmetric, zero diagonal, finite) or, when J is
 * NULL, J_ij = d_ij^-sigma.  Host only: the couplings travel to the device inside each
 * kernel launch (constant bank), so the system holds no device memory.
 * NPHC_EINVAL for N outside [NPHC_MIN_N, NPHC_MAX_N], bad J, or out == NULL. */
nphc_status nphc_system_create_xy(int N, double sigma, const double *J, nphc_system **out);

/* Largest number of unknowns of a generic quadratic system. */
#define NPHC_QUAD_MAX_N 12

/* A generic square system of (at most) quadratic polynomials in n unknowns, for the
 * paper's one-variable example (x^2 - 5, tracked from x^2 - 1, section "Numerical
 * Polynomial Homotopy Continuation Method") and for tests on systems with known roots:
 *   P_i(z) = sum over the terms t with eq[t] == i of coef_t * w(va[t]) * w(vb[t]),
 *   w(k) = z_k for 0 <= k < n, w(-1) = 1,
 * so a term is a constant (va = vb = -1), linear (one of them -1) or quadratic.  The
 * homotopy is the one of the XY ring, H = gamma (1-t) Q + t P with Q_i = z_i^2 - 1, over
 * the 2^n start points z in {+1, -1}^n (path p: z_i = -1 iff bit i of p is set); it is
 * tracked in FP64 whatever the precision option, then refined, certified (beta, gamma
 * bound with ||D^2P/2|| <= sqrt(sum_i ||M_i||_F^2), M_i the symmetric matrix of the
 * quadratic part of P_i) and deduplicated exactly as for the XY ring.  Classification
 * and stationary points do not apply (nphc_classify and nphc_result_copy_sps return
 * NPHC_EINVAL; nphc_system_info reports N = 0).
 *   eq, va, vb (host int32 [nterms]) and coef_re, coef_im (host [nterms]) are copied; the
 * system keeps the term list in device memory on the current device (freed by
 * nphc_system_destroy).
 *   NPHC_EINVAL for n outside [1, NPHC_QUAD_MAX_N], nterms < 1, NULL arrays, an index out
 * of range or a non-finite coefficient; NPHC_ENOMEM / NPHC_ECUDA when the device copy
 * fails. */
nphc_status nphc_system_create_quadratic(int n, int nterms, const int32_t *eq, const int32_t *va,
                                         const int32_t *vb, const double *coef_re,
                                         const double *coef_im, nphc_system **out);

/* Dimensions of a system: ring size N, unknowns n = 2(N-1), Bezout number 4^(N-1)
 * (the number of paths); for a generic quadratic system N = 0, n and 2^n.  Any output
 * may be NULL. */
nphc_status nphc_system_info(const nphc_system *sys, int *N, int *n, int64_t *npaths);

/* The couplings of a system (host, N*N row-major). */
nphc_status nphc_system_couplings(const nphc_system *sys, double *J_out);

void nphc_system_destroy(nphc_system *sys);

/* Bytes of device scratch the step-by-step calls need for `count` entries. */
nphc_status nphc_workspace_size(const nphc_system *sys, int64_t count, size_t *bytes);

/* Tracks entries of ep along H(z,t) = gamma (1-t) Q(z) + t P(z), Q_i = z_i^2 - 1
 * (section "Numerical Polynomial Homotopy Continuation Method"), with a predictor
 * (classical RK4 on dz/dt = -H_z^-1 H_t) and a Newton corrector, in precision prec:
 *   FP64:  plain FP64 tracking;
 *   MIXED: FP32 tracking; a path the FP32 tracker cannot finish ends with status
 *          NPHC_PATH_HANDOFF, or NPHC_PATH_HANDOFF_COND when a converged step's condition
 *          estimate (max |U_kk| / min |U_kk| of the pivoted LU factor of the step's Schur
 *          system) exceeded opt->kappa_fp32, and its (z, t, h) for an FP64 call with
 *          resume = 1.
 * list (device int32, may be NULL) selects entries list[0 .. *list_count - 1]
 * (list_count: device int32); NULL tracks every entry.  resume = 0 starts each selected
 * path at its start point; resume = 1 continues from ep's (z, t, h).  Writes z, t, h,
 * status, steps, solves.  workspace: device scratch of nphc_workspace_size bytes.
 * NPHC_EINVAL on NULL arrays, count outside [0, 4^(N-1)], or a small workspace. */
nphc_status nphc_track(const nphc_system *sys, const nphc_options *opt, nphc_precision prec,
                       const nphc_endpoints *ep, const int32_t *list, const int32_t *list_count,
                       int resume, void *workspace, size_t workspace_bytes, void *stream);

/* FP64 Newton refinement of every selected entry with status NPHC_PATH_REACHED, then
 * the paper's solution tolerance and alpha-theory certification: beta = ||DP^-1 P||,
 * gamma <= ||DP^-1||_F ||D^2P/2||, certified when beta * gamma < (13 - 3 sqrt 17)/8 (half
 * of Smale's constant: an FP64 test keeps a margin where alphaCertified is exact);
 * real when z and Re z share their zero (alpha < 0.03, ||Im z|| < 1/(20 gamma)) and the
 * same test passes at Re z, otherwise non-real when ||Im z|| > 2 beta, else undecided.
 * The certificate is taken at the iterate whose Newton correction met the refinement
 * tolerance, from that iteration's own factorisation (beta = the correction's norm); z is
 * its Newton iterate, closer still to the same zero.  Writes z
 * (refined), cls, alpha, beta, gamma, resid.  Other statuses get NPHC_END_NONE
 * (diverged) or NPHC_END_FAILED.  list / list_count as in nphc_track. */
nphc_status nphc_refine_certify(const nphc_system *sys, const nphc_options *opt,
                                const nphc_endpoints *ep, const int32_t *list,
                                const int32_t *list_count, void *stream);

/* Marks NPHC_END_DUPLICATE every certified entry whose solution a lower path index also
 * reached (alpha-theory: same when ||z1 - z2|| < 1/(20 gamma) with alpha < 0.03, or when
 * not provably distinct, ||z1 - z2|| <= 2 (beta1 + beta2)), using a device hash on the
 * endpoints rounded to a grid.  dup_list (device int32[count], may be NULL) receives the
 * entries of every solution reached more than once and *dup_count (device int32) their
 * number.  workspace as in nphc_track. */
nphc_status nphc_dedup(const nphc_system *sys, const nphc_options *opt, const nphc_endpoints *ep,
                       int32_t *dup_list, int32_t *dup_count, void *workspace,
                       size_t workspace_bytes, void *stream);

/* Largest endpoint count nphc_dedup_noalloc accepts. */
#define NPHC_DEDUP_NOALLOC_MAX 65536

/* nphc_dedup without a workspace, for callers that cannot allocate device memory: a
 * plugin or embedded solver inside a host program whose device memory all belongs to
 * that program's own pool, or a caller that cannot afford cudaMalloc / cudaFree because
 * they may synchronise the device and stall other streams.  The paper has no
 * counterpart; this is an interface convenience.
 *   Arguments, outputs and results are those of nphc_dedup (same flags, same dup_list
 * and dup_count) for ep->count <= NPHC_DEDUP_NOALLOC_MAX (every path of a ring up to
 * N = 9, or the reached endpoints of N = 10).  The scratch is one fixed device array
 * inside the library (about 7.3 MB, part of the library's device image, present in every
 * context that loads it); the call allocates nothing and calls no allocating routine.
 *   The first call on a device (with that device current) looks up the array's device
 * address and caches it for the device's current context; make that first call before
 * any stream capture.  A new context on the device (after cudaDeviceReset, say) holds a
 * new copy of the array, whose address the next call looks up again.
 *   Every call on a device shares the one array and leaves its contents behind; each
 * call clears the parts that must start at zero before use.  Calls whose work overlaps
 * on the GPU (other streams, other host threads) race on the array and give wrong
 * results: order them on one stream or synchronise between them.
 *   NPHC_EINVAL when ep->count > NPHC_DEDUP_NOALLOC_MAX (with a message naming the
 * limit), for the argument errors of nphc_dedup, or for a device ordinal >= 64;
 * NPHC_ECUDA when the address lookup or a launch fails. */
nphc_status nphc_dedup_noalloc(const nphc_system *sys, const nphc_options *opt,
                               const nphc_endpoints *ep, int32_t *dup_list, int32_t *dup_count,
                               void *stream);

/* For every entry with cls == NPHC_END_REAL: theta_k = atan2(s_k, c_k) in (-pi, pi]
 * (theta: device [(N-1) * count], SoA), the Hessian of V in theta_1..theta_{N-1}, its
 * index (device int32 [count]: number of negative eigenvalues), its smallest |eigenvalue|
 * (device [count], may be NULL), log |det H| (device [count], may be NULL: the paper's
 * |det H|^(1/N) is exp(log |det H| / N), section "A First Application") and
 * V = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)) (device [count]).  Other entries get
 * index -1. */
nphc_status nphc_classify(const nphc_system *sys, const nphc_endpoints *ep, double *theta,
                          int32_t *index, double *energy, double *min_abs_eig,
                          double *log_abs_det, void *stream);

/* Gradient with respect to the couplings of a loss L summed over real stationary points
 * (derivatives of the method's outputs; the paper computes none): given, per point,
 * dL/dV (g_energy) and dL/dtheta (g_theta), adds to dJ
 *   dL/dJ_ij = g_energy (1 - cos(theta_i - theta_j)) - (lambda_i - lambda_j) sin(theta_i - theta_j),
 * H lambda = g_theta (H the Hessian of V in theta_1..theta_{N-1}, lambda_N = 0): the
 * envelope theorem for V (grad V = 0 at the point) and the implicit function theorem for
 * theta*.  For couplings J_ij = d_ij^-sigma (1 + eps g_ij), dL/dsigma is
 * sum_{i<j} dL/dJ_ij (-ln d_ij) J_ij.
 *   theta: device [count * (N-1)], one row per point (as nphc_result_copy_sps writes it);
 * g_energy: device [count] or NULL (0); g_theta: device [count * (N-1)] or NULL (0);
 * dJ: device [N * N], accumulated (+=), symmetric (J_ij and J_ji both get the value of
 * the one parameter), diagonal untouched.  A point whose Hessian is singular adds
 * nothing.  NPHC_EINVAL for NULL arrays or a generic quadratic system. */
nphc_status nphc_xy_adjoint(const nphc_system *sys, int64_t count, const double *theta,
                            const double *g_energy, const double *g_theta, double *dJ,
                            void *stream);

/* Outcome of the Cauchy endgame for one entry (nphc_endgame). */
enum {
    NPHC_EG_NONE = 0,           /* not run */
    NPHC_EG_CONVERGED = 1,      /* estimates from two successive radii agree: z is the endpoint */
    NPHC_EG_NOT_CLOSED = 2,     /* at the last radius tried no turn closed within eg_max_cycle */
    NPHC_EG_NOT_CONVERGED = 3,  /* the estimates still disagree at the last radius; z the last one */
    NPHC_EG_TRACK_FAILED = 4,   /* tracking to 1 - eg_r0, a radial leg, or the last radius's
                                   steps failed */
    NPHC_EG_DIVERGED = 5,       /* ||z||_inf exceeded the divergence radius */
    NPHC_EG_AT_INFINITY = 6     /* the turns close, but the path grows as the radius shrinks:
                                   it goes to infinity */
};

/* The Cauchy endgame for endpoints where several paths meet (singular solutions, for
 * instance on the positive-dimensional solution sets of rings with N = 0 mod 4) and for
 * paths that go to infinity too slowly to cross the divergence radius.  The paper reports
 * that such endpoints are dealt with in practice (section "Numerical Polynomial Homotopy
 * Continuation Method"); the method is the Cauchy endgame of Morgan, Sommese and Wampler
 * (1991).  For each selected entry:
 *   1. its path is tracked in FP64 from its start point to t = 1 - eg_r0 (as nphc_track
 *      with resume = 0: z, t, h, status, steps, solves, newton are overwritten);
 *   2. with 1 - t = e^w, the path is continued around the circle |1 - t| = r (RK4 on dz/dw,
 *      Newton's corrector): it closes after c turns, c the cycle number (the path is a
 *      power series in (1 - t)^(1/c)), and the mean of its eg_samples * c equally spaced
 *      samples (the trapezoid rule for Cauchy's integral) estimates the endpoint;
 *   3. r shrinks by eg_ratio (a leg along real t) until two estimates from successive
 *      radii agree and the estimate e solves P within the solution tolerance
 *      (||P(e)||_inf <= tol_sol max(1, ||e||_inf^2): NPHC_EG_CONVERGED), or eg_radii radii
 *      are used.  A radius whose turns do not close within eg_max_cycle turns, or where a
 *      step fails, is left from the point where the path reached it.  Estimates that
 *      agree without solving P belong to a path to infinity when the distance from the
 *      radius's start point to the estimate grows by more than
 *      eg_ratio^(-1/(2 eg_max_cycle)) per radius (NPHC_EG_AT_INFINITY); otherwise the
 *      turns enclose another pair of paths' branch point too, and r shrinks on.
 * Writes z (the estimate for NPHC_EG_CONVERGED and NPHC_EG_NOT_CONVERGED, else the point
 * where the endgame stopped), cycle[e] (device int32 [count]: c of the last radius whose
 * turns closed, 0 if none), eg_status[e] (device int32 [count]: NPHC_EG_*), and adds its
 * solves to solves[e].  cls and the certification arrays are not touched.  list /
 * list_count select entries as in nphc_track; workspace as in nphc_track.  Both the XY
 * ring and generic quadratic systems.  NPHC_EINVAL on NULL arrays, endgame options out
 * of range (0 < eg_r0 < 1, 0 < eg_ratio < 1, eg_radii >= 1, 2 <= eg_samples <= 4096,
 * eg_max_cycle >= 1, positive tolerances, eg_h_min and eg_max_attempts) or a small
 * workspace. */
nphc_status nphc_endgame(const nphc_system *sys, const nphc_options *opt, const nphc_endpoints *ep,
                         const int32_t *list, const int32_t *list_count, int32_t *cycle,
                         int32_t *eg_status, void *workspace, size_t workspace_bytes,
                         void *stream);

/* Result counters (nphc_result_counts). */
enum {
    NPHC_COUNT_PATHS = 0,
    NPHC_COUNT_REACHED, NPHC_COUNT_DIVERGED, NPHC_COUNT_FAILED,
    NPHC_COUNT_REAL, NPHC_COUNT_NONREAL, NPHC_COUNT_UNDECIDED, NPHC_COUNT_SINGULAR,
    NPHC_COUNT_DUPLICATE,
    NPHC_COUNT_HANDOFF,        /* paths the FP32 tracker handed to FP64 */
    NPHC_COUNT_RETRACKED,      /* paths re-tracked in FP64 from t = 0 */
    NPHC_COUNT_SOLVES,         /* linear solves summed over all tracking calls */
    NPHC_COUNT_LAUNCHES,       /* kernels the last nphc_solve_into launched (host count) */
    NPHC_COUNT_INDEX0,         /* + i: real SPs of Hessian index i, i = 0 .. NPHC_MAX_N-1 */
    /* with opt.endgame (zero otherwise): */
    NPHC_COUNT_EG_RUN = NPHC_COUNT_INDEX0 + NPHC_MAX_N,   /* paths given to the endgame */
    NPHC_COUNT_EG_CONVERGED,   /* of which NPHC_EG_CONVERGED (a finite endpoint) */
    NPHC_COUNT_EG_MULTIPLE,    /* of which with cycle number >= 2 (a singular endpoint) */
    NPHC_COUNT_EG_AT_INFINITY, /* NPHC_EG_AT_INFINITY or NPHC_EG_DIVERGED */
    NPHC_COUNT_HANDOFF_COND,   /* of NPHC_COUNT_HANDOFF: handed off by the condition test */
    NPHC_NCOUNTS
};

/* Allocates device buffers for every path of sys (the result keeps a reference to no
 * host memory of the caller).  NPHC_ENOMEM when the device is full. */
nphc_status nphc_result_create(const nphc_system *sys, nphc_result **out);

/* The whole method into an existing result, asynchronously on stream: track every path
 * (MIXED: FP32, then FP64 for hand-offs and for endpoints that do not certify), refine
 * and certify, deduplicate (FP64 re-track of every duplicated solution's paths, then
 * deduplicate again), classify; with opt.endgame, the Cauchy endgame (nphc_endgame) on
 * every path that ends singular or failed.  No allocation, no host synchronisation. */
nphc_status nphc_solve_into(const nphc_system *sys, const nphc_options *opt, nphc_result *res,
                            void *stream);

/* nphc_result_create + nphc_solve_into + stream synchronisation. */
nphc_status nphc_solve(const nphc_system *sys, const nphc_options *opt, void *stream,
                       nphc_result **out);

/* Counters (host int64[NPHC_NCOUNTS]); synchronises with the result's last stream. */
nphc_status nphc_result_counts(const nphc_result *res, int64_t *counts);

/* Real stationary points, ordered by path index, into host buffers of capacity cap:
 * theta [cap * (N-1)] (row per SP), energy, index, alpha, path, log |det H|.  Any output
 * may be NULL.  *n_out = number of real SPs (may exceed cap; only cap are written). */
nphc_status nphc_result_copy_sps(const nphc_result *res, int64_t cap, double *theta,
                                 double *energy, int32_t *index, double *alpha, int64_t *path,
                                 double *log_abs_det, int64_t *n_out);

/* Every path's endpoint (host, path-major z [cap * n]), status and class.  Any output may
 * be NULL.  *n_out = number of paths.  With opt.endgame, entries of class
 * NPHC_END_SINGULAR or NPHC_END_FAILED hold what nphc_endgame wrote (z the endpoint
 * estimate, status that of the FP64 tracking to 1 - eg_r0). */
nphc_status nphc_result_copy_endpoints(const nphc_result *res, int64_t cap, double *z_re,
                                       double *z_im, int32_t *status, int32_t *cls,
                                       int64_t *n_out);

/* Every path's Cauchy endgame outcome (host int32 [cap]): cycle number and NPHC_EG_*
 * status (NPHC_EG_NONE where the endgame did not run).  Any output may be NULL.
 * *n_out = number of paths. */
nphc_status nphc_result_copy_endgame(const nphc_result *res, int64_t cap, int32_t *cycle,
                                     int32_t *eg_status, int64_t *n_out);

/* ---------------------------------------------------------------------------------
 * Batches: many independent systems solved together (the paper's method per system;
 * batching is a scheduling choice of this library).  By default the XY rings of a batch
 * are grouped by size, and each group's FP32 pass -- every path of every instance in it --
 * is one persistent launch that pulls (instance, path) items from one queue, so that
 * small rings fill the GPU together and no instance leaves a tail of idle SMs; the rest
 * of each instance's method (hand-offs, FP64 continuation, refinement, certification,
 * deduplication, classification) runs per instance on one of NPHC_BATCH_STREAMS internal
 * streams once its group's pass is done.  A group runs that way when all its members are
 * solved in mixed precision with the same FP32 step control (gamma and kappa_sing may
 * differ); otherwise, and for generic quadratic systems, each instance runs the whole of
 * nphc_solve_into on its stream.  Deduplication and classification stay per instance.
 * --------------------------------------------------------------------------------- */
#define NPHC_BATCH_STREAMS 8
#define NPHC_BATCH_GRAPH 1          /* nphc_batch_solve flag: capture / replay a CUDA graph */
#define NPHC_BATCH_PER_INSTANCE 2   /* nphc_batch_solve flag: every instance runs the whole
                                       solve on its stream (no group launches) */
typedef struct nphc_batch nphc_batch;   /* opaque; owns one nphc_result per instance */

/* A batch over systems[0 .. count-1] (borrowed: they must outlive the batch).  Creates
 * one result per instance (device memory as nphc_result_create), the internal streams,
 * and the device tables of the size groups (couplings rows, endpoint views, path offsets).
 * NPHC_EINVAL for count < 1 or a NULL system; NPHC_ENOMEM / NPHC_ECUDA on allocation. */
nphc_status nphc_batch_create(int count, const nphc_system *const *systems, nphc_batch **out);

/* Solves every instance with its options opts[i] (host array of count), asynchronously
 * on `stream`: the call returns once the work is enqueued; the caller's stream is
 * ordered after every instance.  flags: 0 = eager launches, grouped by size;
 * NPHC_BATCH_GRAPH: the first solve of the batch runs eagerly, the next one captures the
 * whole batch (fork, every launch, join) into one CUDA graph in relaxed capture mode and
 * launches it, and later solves with the same options and flags replay that graph (new
 * options capture a new one); NPHC_BATCH_PER_INSTANCE: no group launches.  When the
 * options differ from the previous solve's, the call first waits for the batch's earlier
 * work and rewrites the couplings table (a synchronous copy).  The caller must not
 * capture `stream` itself around this call.  NPHC_EINVAL for NULL arguments, invalid
 * options or unknown flags. */
nphc_status nphc_batch_solve(nphc_batch *batch, const nphc_options *opts, int flags, void *stream);

/* The result of instance i (borrowed; valid until nphc_batch_destroy).  Read it with
 * the nphc_result_* calls after the solve (they synchronise on the caller's stream). */
nphc_status nphc_batch_result(const nphc_batch *batch, int i, const nphc_result **out);

void nphc_batch_destroy(nphc_batch *batch);

/* Device endpoint arrays of a result (valid until nphc_result_destroy). */
nphc_status nphc_result_endpoints(const nphc_result *res, nphc_endpoints *ep);

void nphc_result_destroy(nphc_result *res);

/* Index checks of the debug build (the library compiled with NPHC_DEBUG; the paper has no
 * counterpart: this stands in for a memory checker).  Its kernels check every work-list
 * entry, list append, deduplication link and batch item against the bounds of the array
 * it indexes; a failed check records a code and the access is skipped, so the kernel
 * returns normally.  Writes the first recorded code since the last call and clears it:
 * 0 none, 1 a work-list entry outside the endpoint set, 2 an append beyond a list's
 * capacity, 3 a deduplication link outside the endpoint set, 4 a batch item outside its
 * group, 5 a gathered or listed-for-classification entry outside the set; -1 in a release
 * build (no checks).
 * Synchronous.  NPHC_EINVAL for a NULL code. */
nphc_status nphc_debug_check(int32_t *code);

/* Message of the last failed call on this thread ("" when none). */
const char *nphc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NPHC_H */
