/*
 * nphc_oracle.c -- plain, slow, FP64 CPU restatement of the numerical polynomial
 * homotopy continuation (NPHC) method of Mehta, "Finding All the Stationary Points
 * of a Potential Energy Landscape via Numerical Polynomial Homotopy Continuation
 * Method" (arXiv:1104.5497).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant generator with
 * the CUDA path, and it never calls it.
 *
 * What it computes, step by step and in the paper's order:
 *   - couplings of the power-law XY ring (section "A First Application", the potential
 *     V and its exponent), written as J_ij = d_ij^-sigma with d_ij the ring distance,
 *     optionally scaled by a per-pair disorder factor (1 + eps * g_ij);
 *   - the polynomial system of Eq. (alg_dec_XY_model_poly): for each free site k the
 *     gradient equation in s_k = sin(theta_k), c_k = cos(theta_k) and the constraint
 *     s_k^2 + c_k^2 - 1, with theta_N pinned to 0 (the gauge fixing of that section),
 *     stored as a plain list of quadratic terms;
 *   - the total-degree start system Q_i = z_i^2 - 1 with start points z_i = +-1 and the
 *     gamma-trick homotopy H = gamma (1-t) Q + t P (section "Numerical Polynomial
 *     Homotopy Continuation Method");
 *   - a predictor-corrector path tracker from t=0 to t=1 (same section: "Euler's
 *     predictor and Newton's corrector"; the predictor here is classical RK4 on
 *     dz/dt = -H_z^-1 H_t, the corrector evaluates H with compensated sums; a path whose
 *     ||z||_inf exceeds the divergence radius is taken to go to infinity);
 *   - refinement of endpoints by Newton's method on P to machine precision (P evaluated
 *     with compensated double-double sums, so that the refinement and beta are limited
 *     by the solution's conditioning and not by the rounding of ~||z||^2 terms), the
 *     solution tolerance Delta_sol and the real tolerance Delta_R (same section);
 *   - Smale alpha-theory certification (the alphaCertified step of the same section):
 *     beta = ||DP^-1 P||, gamma <= ||DP^-1|| * ||D^2 P / 2||, alpha = beta * gamma <
 *     (13 - 3 sqrt 17)/4, a real test at Re z (when z and Re z share their zero) and a
 *     non-real test ||Im z|| > 2 beta;
 *   - theta recovery theta_k = atan2(s_k, c_k) in (-pi, pi], the Hessian of V in
 *     theta_1..theta_{N-1}, its index (number of negative eigenvalues, introduction)
 *     and the energy V (section "A First Application").
 *
 * Linear algebra is textbook: LU with partial pivoting on the largest modulus (ties to
 * the lowest row), cyclic Jacobi for symmetric eigenvalues.  No blocking, no fusion.
 * Every function that has a fixed meaning is exported for the tests to pin.
 */
#define _DEFAULT_SOURCE
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- path statuses -- */
enum {
    OR_RUNNING = 0,
    OR_REACHED = 1,      /* tracked to t = 1 */
    OR_DIVERGED = 2,     /* ||z||_inf exceeded the divergence radius before t = 1 */
    OR_MIN_STEP = 3,     /* step size fell below h_min */
    OR_STEP_BUDGET = 4,  /* more than max_steps step attempts */
    OR_NONFINITE = 5     /* NaN/Inf appeared */
};

/* ------------------------------------------------------------ endpoint classes -- */
enum {
    OC_NONE = 0,         /* diverged or failed path: no endpoint */
    OC_SINGULAR = 1,     /* finite endpoint that does not certify (singular or not a solution) */
    OC_REAL = 2,         /* certified approximate solution, certified real */
    OC_NONREAL = 3,      /* certified approximate solution, certified non-real */
    OC_UNDECIDED = 4,    /* certified approximate solution, reality not decided */
    OC_DUPLICATE = 5,    /* certified, but another path reached the same solution */
    OC_FAILED = 6        /* tracking stopped before t = 1 without diverging */
};

/* ------------------------------------------------------------ quadratic system -- */
/* P_i(z) = sum over terms with eq == i of coef * w(a) * w(b), where w(-1) = 1 and
 * w(k) = z_k.  Every equation has degree <= 2 (the XY system has degree exactly 2). */
typedef struct {
    int n;
    int nterms;
    const int *eq, *va, *vb;
    const double *cre, *cim;
} qsys;

static inline cplx wvar(const cplx *z, int a) { return a < 0 ? 1.0 : z[a]; }

/* P(z) */
static void sys_eval(const qsys *S, const cplx *z, cplx *P) {
    for (int i = 0; i < S->n; i++) P[i] = 0;
    for (int t = 0; t < S->nterms; t++) {
        cplx c = S->cre[t] + I * S->cim[t];
        P[S->eq[t]] += c * wvar(z, S->va[t]) * wvar(z, S->vb[t]);
    }
}

/* P(z) with every product formed exactly and every sum carried in double-double
 * (Knuth's two-sum, fma two-product), rounded once at the end.  Used where the value of
 * P at a candidate solution is the quantity of interest (refinement, beta): at ||z|| >> 1
 * the terms are ~||z||^2 and their plain double sum would be dominated by rounding. */
typedef struct { double hi, lo; } dd;

static dd dd_two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    dd r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}

static dd dd_two_prod(double a, double b) {
    double p = a * b;
    dd r = {p, fma(a, b, -p)};
    return r;
}

static dd dd_add(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    double lo = s.lo + a.lo + b.lo, hi = s.hi + lo;
    dd r = {hi, lo - (hi - s.hi)};
    return r;
}

/* (a.hi + a.lo) * b */
static dd dd_mul_d(dd a, double b) {
    dd p = dd_two_prod(a.hi, b);
    double lo = p.lo + a.lo * b, hi = p.hi + lo;
    dd r = {hi, lo - (hi - p.hi)};
    return r;
}

static void sys_eval_acc(const qsys *S, const cplx *z, cplx *P) {
    int n = S->n;
    dd *re = calloc(n, sizeof(dd)), *im = calloc(n, sizeof(dd));
    for (int t = 0; t < S->nterms; t++) {
        cplx wa = wvar(z, S->va[t]), wb = wvar(z, S->vb[t]);
        /* wa * wb exactly: real = ar br - ai bi, imag = ar bi + ai br */
        dd pr = dd_add(dd_two_prod(creal(wa), creal(wb)), dd_two_prod(-cimag(wa), cimag(wb)));
        dd pi = dd_add(dd_two_prod(creal(wa), cimag(wb)), dd_two_prod(cimag(wa), creal(wb)));
        /* times the coefficient c = cr + i ci */
        double cr = S->cre[t], ci = S->cim[t];
        dd tr = dd_add(dd_mul_d(pr, cr), dd_mul_d(pi, -ci));
        dd ti = dd_add(dd_mul_d(pi, cr), dd_mul_d(pr, ci));
        int e = S->eq[t];
        re[e] = dd_add(re[e], tr);
        im[e] = dd_add(im[e], ti);
    }
    for (int i = 0; i < n; i++) P[i] = (re[i].hi + re[i].lo) + I * (im[i].hi + im[i].lo);
    free(re);
    free(im);
}

/* DP(z), row-major n x n: d/dz_c of c*w(a)*w(b) = c*(delta_ac w(b) + delta_bc w(a)) */
static void sys_jac(const qsys *S, const cplx *z, cplx *D) {
    int n = S->n;
    for (int i = 0; i < n * n; i++) D[i] = 0;
    for (int t = 0; t < S->nterms; t++) {
        cplx c = S->cre[t] + I * S->cim[t];
        int e = S->eq[t], a = S->va[t], b = S->vb[t];
        if (a >= 0) D[e * n + a] += c * wvar(z, b);
        if (b >= 0) D[e * n + b] += c * wvar(z, a);
    }
}

/* Exported for the tests: P(z) and DP(z) (row-major) of a term-list system. */
void oracle_sys_eval_jac(int n, int nterms, const int *eq, const int *va, const int *vb,
                         const double *cre, const double *cim, const double *zre,
                         const double *zim, double *pre, double *pim, double *dre, double *dim) {
    qsys S = {n, nterms, eq, va, vb, cre, cim};
    cplx *z = malloc(sizeof(cplx) * n), *P = malloc(sizeof(cplx) * n),
         *D = malloc(sizeof(cplx) * n * n);
    for (int i = 0; i < n; i++) z[i] = zre[i] + I * zim[i];
    sys_eval(&S, z, P);
    sys_jac(&S, z, D);
    for (int i = 0; i < n; i++) { pre[i] = creal(P[i]); pim[i] = cimag(P[i]); }
    for (int i = 0; i < n * n; i++) { dre[i] = creal(D[i]); dim[i] = cimag(D[i]); }
    free(z); free(P); free(D);
}

/* Exported for the tests: P(z) with compensated sums. */
void oracle_sys_eval_acc(int n, int nterms, const int *eq, const int *va, const int *vb,
                         const double *cre, const double *cim, const double *zre,
                         const double *zim, double *pre, double *pim) {
    qsys S = {n, nterms, eq, va, vb, cre, cim};
    cplx *z = malloc(sizeof(cplx) * n), *P = malloc(sizeof(cplx) * n);
    for (int i = 0; i < n; i++) z[i] = zre[i] + I * zim[i];
    sys_eval_acc(&S, z, P);
    for (int i = 0; i < n; i++) { pre[i] = creal(P[i]); pim[i] = cimag(P[i]); }
    free(z); free(P);
}

/* ---------------------------------------------------------------- LU (textbook) -- */
/* In-place LU with partial pivoting (largest modulus; ties keep the lowest row).
 * Returns 0, or 1 when a pivot is exactly zero.  piv[k] is the row swapped into k. */
static int lu_factor(int n, cplx *A, int *piv) {
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = cabs(A[k * n + k]);
        for (int r = k + 1; r < n; r++) {
            double v = cabs(A[r * n + k]);
            if (v > best) { best = v; p = r; }
        }
        piv[k] = p;
        if (best == 0.0 || !isfinite(best)) return 1;
        if (p != k)
            for (int c = 0; c < n; c++) {
                cplx tmp = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = tmp;
            }
        for (int r = k + 1; r < n; r++) {
            cplx l = A[r * n + k] / A[k * n + k];
            A[r * n + k] = l;
            for (int c = k + 1; c < n; c++) A[r * n + c] -= l * A[k * n + c];
        }
    }
    return 0;
}

/* Solve with the factors of lu_factor (P A = L U, P the interchanges in order k = 0..n-1,
 * applied to whole rows): b <- P b, then L y = b, then U x = y.  b is overwritten with x. */
static void lu_apply(int n, const cplx *A, const int *piv, cplx *b) {
    for (int k = 0; k < n; k++)
        if (piv[k] != k) { cplx tmp = b[k]; b[k] = b[piv[k]]; b[piv[k]] = tmp; }
    for (int k = 0; k < n; k++)
        for (int r = k + 1; r < n; r++) b[r] -= A[r * n + k] * b[k];
    for (int k = n - 1; k >= 0; k--) {
        cplx s = b[k];
        for (int c = k + 1; c < n; c++) s -= A[k * n + c] * b[c];
        b[k] = s / A[k * n + k];
    }
}

static double norm2(int n, const cplx *v) {
    double s = 0;
    for (int i = 0; i < n; i++) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return sqrt(s);
}

static double norminf(int n, const cplx *v) {
    double s = 0;
    for (int i = 0; i < n; i++) { double a = cabs(v[i]); if (a > s || isnan(a)) s = a; }
    return s;
}

/* Exported for the tests: solve A x = b (row-major A, split re/im).  Returns 0 or 1. */
int oracle_lu_solve(int n, const double *are, const double *aim, const double *bre,
                    const double *bim, double *xre, double *xim) {
    cplx *A = malloc(sizeof(cplx) * n * n), *b = malloc(sizeof(cplx) * n);
    int *piv = malloc(sizeof(int) * n);
    for (int i = 0; i < n * n; i++) A[i] = are[i] + I * aim[i];
    for (int i = 0; i < n; i++) b[i] = bre[i] + I * bim[i];
    int rc = lu_factor(n, A, piv);
    if (!rc) {
        lu_apply(n, A, piv, b);
        for (int i = 0; i < n; i++) { xre[i] = creal(b[i]); xim[i] = cimag(b[i]); }
    }
    free(A); free(b); free(piv);
    return rc;
}

/* ------------------------------------------------------- symmetric eigenvalues -- */
/* Cyclic Jacobi rotations on a real symmetric n x n matrix (row-major, destroyed);
 * eigenvalues, unsorted, in w.  Sweeps until the off-diagonal mass is negligible. */
static void jacobi_eig(int n, double *A, double *w) {
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0, tot = 0;
        for (int p = 0; p < n; p++)
            for (int q = 0; q < n; q++) {
                tot += A[p * n + q] * A[p * n + q];
                if (p != q) off += A[p * n + q] * A[p * n + q];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {   /* columns p, q */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {   /* rows p, q */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
            }
    }
    for (int i = 0; i < n; i++) w[i] = A[i * n + i];
}

/* Exported for the tests: eigenvalues of a real symmetric matrix (unsorted). */
void oracle_sym_eig(int n, const double *A, double *w) {
    double *B = malloc(sizeof(double) * n * n);
    memcpy(B, A, sizeof(double) * n * n);
    jacobi_eig(n, B, w);
    free(B);
}

/* -------------------------------------------------------------- XY power law -- */
/* Ring distance d_ij = min(|i-j|, N-|i-j|) and couplings J_ij = d_ij^-sigma, each
 * scaled by (1 + eps * g_ij) when g (an N x N matrix of per-pair draws, symmetric) is
 * given.  J_ii = 0.  Returns 0, or 1 for invalid arguments. */
int oracle_xy_couplings(int N, double sigma, const double *g, double eps, double *J) {
    if (N < 3) return 1;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            if (i == j) { J[i * N + j] = 0.0; continue; }
            int d = abs(i - j);
            if (N - d < d) d = N - d;
            double v = pow((double)d, -sigma);
            if (g) v *= 1.0 + eps * g[i * N + j];
            J[i * N + j] = v;
        }
    return 0;
}

/* Eq. (alg_dec_XY_model_poly) as a term list, with the unknowns ordered
 * z = (c_1..c_m, s_1..s_m), m = N-1, and theta_N = 0 pinned (c_N = 1, s_N = 0).
 * Equation k (0 <= k < m):  sum_{j != k} J_kj (s_k c_j - s_j c_k) = 0,
 * equation m+k:             c_k^2 + s_k^2 - 1 = 0.
 * The paper's overall factor K (and its split j = 1..(N-1)/2 in both directions) only
 * rescales each gradient equation; summing over all j != k with J_kj = J_jk is the same
 * sum.  The arrays must hold at least 2*m*(N-1) + 3*m terms.  Returns nterms. */
int oracle_xy_terms(int N, const double *J, int *eq, int *va, int *vb, double *cre, double *cim) {
    int m = N - 1, nt = 0;
#define TERM(E, A, B, C) do { eq[nt] = (E); va[nt] = (A); vb[nt] = (B); cre[nt] = (C); cim[nt] = 0.0; nt++; } while (0)
    for (int k = 0; k < m; k++) {
        int ck = k, sk = m + k;
        for (int j = 0; j < N; j++) {
            if (j == k) continue;
            double Jkj = J[k * N + j];
            if (j == N - 1) {           /* pinned site: c_N = 1, s_N = 0 */
                TERM(k, sk, -1, Jkj);   /* s_k * c_N */
            } else {
                TERM(k, sk, j, Jkj);        /*  J s_k c_j */
                TERM(k, m + j, ck, -Jkj);   /* -J s_j c_k */
            }
        }
    }
    for (int k = 0; k < m; k++) {
        TERM(m + k, k, k, 1.0);
        TERM(m + k, m + k, m + k, 1.0);
        TERM(m + k, -1, -1, -1.0);
    }
#undef TERM
    return nt;
}

/* ------------------------------------------------------------- path tracking -- */
typedef struct {
    double h0;          /* first step size */
    double h_max;       /* largest step size */
    double h_min;       /* smallest step size before giving up */
    double eps_corr;    /* Newton corrector: accept when ||dz|| <= eps (1 + ||z||) */
    double trust;       /* reject when the first correction exceeds trust (1 + ||z||) */
    double r_div;       /* divergence radius on ||z||_inf */
    int max_newton;     /* corrector iterations per step */
    int max_steps;      /* step attempts per path */
    int grow_after;     /* consecutive accepted steps before doubling h */
} oracle_track_opts;

typedef struct {
    int n;
    cplx *A, *b, *hz, *k1, *k2, *k3, *k4, *zs, *zp, *P, *Q;
    int *piv;
} work;

static void work_init(work *w, int n) {
    w->n = n;
    w->A = malloc(sizeof(cplx) * n * n);
    cplx **v[] = {&w->b, &w->hz, &w->k1, &w->k2, &w->k3, &w->k4, &w->zs, &w->zp, &w->P, &w->Q};
    for (unsigned i = 0; i < sizeof(v) / sizeof(v[0]); i++) *v[i] = malloc(sizeof(cplx) * n);
    w->piv = malloc(sizeof(int) * n);
}

static void work_free(work *w) {
    free(w->A); free(w->b); free(w->hz); free(w->k1); free(w->k2); free(w->k3); free(w->k4);
    free(w->zs); free(w->zp); free(w->P); free(w->Q); free(w->piv);
}

/* H_z(z,t) = gamma (1-t) diag(2 z) + t DP(z), written into w->A. */
static void hom_jac(const qsys *S, cplx gamma, const cplx *z, double t, work *w) {
    int n = S->n;
    sys_jac(S, z, w->A);
    for (int i = 0; i < n * n; i++) w->A[i] *= t;
    for (int i = 0; i < n; i++) w->A[i * n + i] += gamma * (1.0 - t) * 2.0 * z[i];
}

/* dz/dt = -H_z^-1 H_t with H_t = P - gamma Q.  Returns 0 or 1 (singular H_z). */
static int dzdt(const qsys *S, cplx gamma, const cplx *z, double t, work *w, cplx *out) {
    int n = S->n;
    sys_eval(S, z, w->P);
    for (int i = 0; i < n; i++) out[i] = -(w->P[i] - gamma * (z[i] * z[i] - 1.0));
    hom_jac(S, gamma, z, t, w);
    if (lu_factor(n, w->A, w->piv)) return 1;
    lu_apply(n, w->A, w->piv, out);
    return 0;
}

/* H(z, t) = gamma (1-t) (z^2 - 1) + t P(z) with compensated sums (exact products,
 * double-double accumulation, one rounding), for the corrector: near a point where the
 * terms of H are much larger than H itself (large ||z||) a plain double evaluation would
 * stall Newton's method at the rounding of the terms rather than at the solution. */
static void hom_eval_acc(const qsys *S, cplx gamma, const cplx *z, double t, cplx *Hout, cplx *P) {
    int n = S->n;
    sys_eval_acc(S, z, P);   /* P to double, then t P: one product, compensated below */
    double gr = creal(gamma) * (1.0 - t), gi = cimag(gamma) * (1.0 - t);
    for (int i = 0; i < n; i++) {
        double xr = creal(z[i]), xi = cimag(z[i]);
        /* q = z^2 - 1 exactly */
        dd qr = dd_add(dd_add(dd_two_prod(xr, xr), dd_two_prod(-xi, xi)), (dd){-1.0, 0.0});
        dd qi = dd_two_prod(2.0 * xr, xi);
        /* gamma (1-t) q + t P */
        dd hr = dd_add(dd_add(dd_mul_d(qr, gr), dd_mul_d(qi, -gi)), dd_two_prod(t, creal(P[i])));
        dd hi = dd_add(dd_add(dd_mul_d(qi, gr), dd_mul_d(qr, gi)), dd_two_prod(t, cimag(P[i])));
        Hout[i] = (hr.hi + hr.lo) + I * (hi.hi + hi.lo);
    }
}

/* One Newton step on H(., t): z += -H_z^-1 H.  Writes ||dz||_2 to *dn. */
static int newton_hom(const qsys *S, cplx gamma, cplx *z, double t, work *w, double *dn) {
    int n = S->n;
    hom_eval_acc(S, gamma, z, t, w->b, w->P);
    for (int i = 0; i < n; i++) w->b[i] = -w->b[i];
    hom_jac(S, gamma, z, t, w);
    if (lu_factor(n, w->A, w->piv)) return 1;
    lu_apply(n, w->A, w->piv, w->b);
    for (int i = 0; i < n; i++) z[i] += w->b[i];
    *dn = norm2(n, w->b);
    return 0;
}

static int all_finite(int n, const cplx *z) {
    for (int i = 0; i < n; i++)
        if (!isfinite(creal(z[i])) || !isfinite(cimag(z[i]))) return 0;
    return 1;
}

/* Track one path from its start point z (in) to t_end (out): t_end = 1 for the whole
 * path, below 1 where the Cauchy endgame takes over. */
static int track_path(const qsys *S, cplx gamma, const oracle_track_opts *o, double t_end,
                      cplx *z, int *steps_out, double *t_out, work *w) {
    int n = S->n, accepted = 0, attempts = 0, run = 0, status = OR_RUNNING;
    double t = 0.0, h = o->h0;
    while (status == OR_RUNNING) {
        if (t >= t_end) { status = OR_REACHED; break; }
        if (attempts >= o->max_steps) { status = OR_STEP_BUDGET; break; }
        attempts++;
        double t1 = t + h, hh = h;
        if (t1 >= t_end) { t1 = t_end; hh = t_end - t; }
        /* classical RK4 on dz/dt = -H_z^-1 H_t */
        int bad = dzdt(S, gamma, z, t, w, w->k1);
        if (!bad) { for (int i = 0; i < n; i++) w->zs[i] = z[i] + 0.5 * hh * w->k1[i];
                    bad = dzdt(S, gamma, w->zs, t + 0.5 * hh, w, w->k2); }
        if (!bad) { for (int i = 0; i < n; i++) w->zs[i] = z[i] + 0.5 * hh * w->k2[i];
                    bad = dzdt(S, gamma, w->zs, t + 0.5 * hh, w, w->k3); }
        if (!bad) { for (int i = 0; i < n; i++) w->zs[i] = z[i] + hh * w->k3[i];
                    bad = dzdt(S, gamma, w->zs, t1, w, w->k4); }
        int ok = 0;
        if (!bad) {
            for (int i = 0; i < n; i++)
                w->zp[i] = z[i] + hh / 6.0 * (w->k1[i] + 2.0 * w->k2[i] + 2.0 * w->k3[i] + w->k4[i]);
            /* Newton corrector at t1; a large first correction means the prediction
             * left the path's neighbourhood, so the step is rejected */
            double zn = norm2(n, w->zp);
            for (int it = 0; it < o->max_newton; it++) {
                double dn;
                if (newton_hom(S, gamma, w->zp, t1, w, &dn)) break;
                if (!all_finite(n, w->zp)) break;
                if (it == 0 && dn > o->trust * (1.0 + zn)) break;
                if (dn <= o->eps_corr * (1.0 + norm2(n, w->zp))) { ok = 1; break; }
            }
        }
        if (ok) {
            memcpy(z, w->zp, sizeof(cplx) * n);
            t = t1;
            accepted++;
            if (++run >= o->grow_after) { run = 0; h = fmin(2.0 * h, o->h_max); }
            if (norminf(n, z) > o->r_div) status = OR_DIVERGED;
        } else {
            run = 0;
            h *= 0.5;
            if (h < o->h_min) status = OR_MIN_STEP;
        }
    }
    if (status != OR_DIVERGED && !all_finite(n, z)) status = OR_NONFINITE;
    *steps_out = accepted;
    *t_out = t;
    return status;
}

typedef struct {
    const qsys *S;
    cplx gamma;
    const oracle_track_opts *o;
    int64_t path0, npaths;
    double *zre, *zim;
    int *status, *steps;
    double *tend;
    int64_t next;   /* shared work counter */
} track_job;

static void *track_worker(void *arg) {
    track_job *J = arg;
    int n = J->S->n;
    work w;
    work_init(&w, n);
    cplx *z = malloc(sizeof(cplx) * n);
    for (;;) {
        int64_t i = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (i >= J->npaths) break;
        int64_t p = J->path0 + i;
        /* start point of path p: z_i = -1 when bit i of p is set, else +1 (the roots of
         * z_i^2 - 1 = 0, one of the 2^n combinations per path) */
        for (int k = 0; k < n; k++) z[k] = ((p >> k) & 1) ? -1.0 : 1.0;
        int steps;
        double t;
        int st = track_path(J->S, J->gamma, J->o, 1.0, z, &steps, &t, &w);
        for (int k = 0; k < n; k++) {
            J->zre[i * n + k] = creal(z[k]);
            J->zim[i * n + k] = cimag(z[k]);
        }
        J->status[i] = st;
        J->steps[i] = steps;
        J->tend[i] = t;
    }
    free(z);
    work_free(&w);
    return NULL;
}

/* Track paths path0 .. path0+npaths-1 of the total-degree homotopy of the quadratic
 * system (terms), with nthreads host threads.  Endpoints are path-major:
 * z[i*n + k].  Returns 0, or 1 for invalid arguments. */
int oracle_track(int n, int nterms, const int *eq, const int *va, const int *vb,
                 const double *cre, const double *cim, double gamma_re, double gamma_im,
                 const oracle_track_opts *o, int64_t path0, int64_t npaths, int nthreads,
                 double *zre, double *zim, int *status, int *steps, double *tend) {
    if (n < 1 || n > 62 || nthreads < 1 || npaths < 0) return 1;
    qsys S = {n, nterms, eq, va, vb, cre, cim};
    track_job J = {&S, gamma_re + I * gamma_im, o, path0, npaths, zre, zim, status, steps, tend, 0};
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, track_worker, &J);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    free(th);
    return 0;
}

/* ------------------------------------------------------------ Cauchy endgame -- */
/* Endpoints that are singular (several paths meeting at t = 1) stall a tracker that
 * walks t along the real axis: H_z becomes singular at t = 1.  The paper reports that
 * such difficulties are resolved in practice; this is the Cauchy endgame of the
 * homotopy continuation literature (Morgan, Sommese and Wampler, 1991).  Near t = 1 a
 * path is a Puiseux series in s = (1 - t)^(1/c), analytic in s, with c the cycle
 * number.  Writing 1 - t = e^w, the path is continued around the circle |1 - t| = r
 * (w = ln r + i theta, theta from 0 upward); it closes after exactly c turns, and by
 * Cauchy's integral formula its value at s = 0 is the mean of z over one turn in s,
 * i.e. over the c turns in t.  With K equally spaced samples per turn the mean is the
 * trapezoid rule, exact up to the aliased term of order r^K / R^K (R the distance from
 * t = 1 to the nearest other branch point).  The radius shrinks by `ratio` until two
 * successive estimates agree.  Continuation between samples is the tracker's: RK4 on
 * dz/dw, Newton's corrector at the end of each step, the same step control. */
typedef struct {
    double r0;          /* first radius |1 - t|; tracking from t = 0 stops at 1 - r0 */
    double ratio;       /* radius ratio between successive turns (< 1) */
    int n_radii;        /* most radii tried */
    int samples;        /* K: samples per turn around t = 1 */
    int max_cycle;      /* largest cycle number tried */
    double tol_close;   /* a turn closes when ||z - z_start|| <= tol_close (1 + ||z_start||) */
    double tol_conv;    /* estimates agree when ||e_k - e_{k-1}|| <= tol_conv (1 + ||e_k||) */
    double h_min;       /* smallest step, as a fraction of one sample interval */
    int max_attempts;   /* step attempts per path in the endgame */
    double tol_res;     /* an estimate is a solution when ||P||_inf <= tol_res max(1, ||e||_inf^2)
                         * (the solution tolerance Delta_sol, as for certification) */
} oracle_eg_opts;

enum {
    OE_NONE = 0,
    OE_CONVERGED = 1,      /* two successive estimates agree */
    OE_NOT_CLOSED = 2,     /* no turn closed within max_cycle turns */
    OE_NOT_CONVERGED = 3,  /* estimates still disagree at the last radius (last one kept) */
    OE_TRACK_FAILED = 4,   /* tracking to 1 - r0, or a step of the endgame, failed */
    OE_DIVERGED = 5,       /* ||z||_inf exceeded the divergence radius */
    OE_AT_INFINITY = 6     /* turns close, but the path grows as the radius shrinks: a pole */
};

/* H_z(z, t) = gamma (1-t) diag(2 z) + t DP(z) at complex t (omt = 1 - t), into w->A. */
static void hom_jac_c(const qsys *S, cplx gamma, const cplx *z, cplx t, cplx omt, work *w) {
    int n = S->n;
    sys_jac(S, z, w->A);
    for (int i = 0; i < n * n; i++) w->A[i] *= t;
    for (int i = 0; i < n; i++) w->A[i * n + i] += gamma * omt * 2.0 * z[i];
}

/* dz/dw for 1 - t = e^w: dt/dw = -e^w, so dz/dw = -H_z^-1 H_t dt/dw = e^w H_z^-1 H_t,
 * H_t = P - gamma Q.  Returns 0 or 1 (singular H_z). */
static int dzdw(const qsys *S, cplx gamma, const cplx *z, cplx ew, work *w, cplx *out) {
    int n = S->n;
    sys_eval(S, z, w->P);
    for (int i = 0; i < n; i++) out[i] = w->P[i] - gamma * (z[i] * z[i] - 1.0);
    hom_jac_c(S, gamma, z, 1.0 - ew, ew, w);
    if (lu_factor(n, w->A, w->piv)) return 1;
    lu_apply(n, w->A, w->piv, out);
    for (int i = 0; i < n; i++) out[i] *= ew;
    return 0;
}

/* H(z, t) at complex t with the compensated sums of hom_eval_acc. */
static void hom_eval_acc_c(const qsys *S, cplx gamma, const cplx *z, cplx t, cplx omt,
                           cplx *Hout, cplx *P) {
    int n = S->n;
    sys_eval_acc(S, z, P);
    cplx g1 = gamma * omt;
    double gr = creal(g1), gi = cimag(g1), tr = creal(t), ti = cimag(t);
    for (int i = 0; i < n; i++) {
        double xr = creal(z[i]), xi = cimag(z[i]);
        dd qr = dd_add(dd_add(dd_two_prod(xr, xr), dd_two_prod(-xi, xi)), (dd){-1.0, 0.0});
        dd qi = dd_two_prod(2.0 * xr, xi);
        double pr = creal(P[i]), pi = cimag(P[i]);
        dd hr = dd_add(dd_add(dd_mul_d(qr, gr), dd_mul_d(qi, -gi)),
                       dd_add(dd_two_prod(tr, pr), dd_two_prod(-ti, pi)));
        dd hi = dd_add(dd_add(dd_mul_d(qi, gr), dd_mul_d(qr, gi)),
                       dd_add(dd_two_prod(tr, pi), dd_two_prod(ti, pr)));
        Hout[i] = (hr.hi + hr.lo) + I * (hi.hi + hi.lo);
    }
}

static int newton_hom_c(const qsys *S, cplx gamma, cplx *z, cplx ew, work *w, double *dn) {
    int n = S->n;
    cplx t = 1.0 - ew;
    hom_eval_acc_c(S, gamma, z, t, ew, w->b, w->P);
    for (int i = 0; i < n; i++) w->b[i] = -w->b[i];
    hom_jac_c(S, gamma, z, t, ew, w);
    if (lu_factor(n, w->A, w->piv)) return 1;
    lu_apply(n, w->A, w->piv, w->b);
    for (int i = 0; i < n; i++) z[i] += w->b[i];
    *dn = norm2(n, w->b);
    return 0;
}

/* e^w at the point v in [0, 1] of a sample interval: on a turn (radial == 0) w = lr +
 * i 2 pi (j + v) / K; on the radial leg w = lr + v ln(ratio). */
static cplx eg_ew(double lr, int radial, int j, int K, double lnratio, double v) {
    if (radial) return exp(lr + v * lnratio);
    return cexp(lr + I * (2.0 * M_PI * ((double)j + v) / (double)K));
}

/* Continue z across one sample interval (v from 0 to 1) with the tracker's step control
 * in v (RK4 on dz/dv = dw/dv dz/dw, Newton at the end of each step, h halves on a reject,
 * doubles after grow_after accepts, at most 1).  *h carries the step between intervals.
 * Returns OE_NONE on success, else OE_TRACK_FAILED or OE_DIVERGED. */
static int eg_interval(const qsys *S, cplx gamma, const oracle_track_opts *o,
                       const oracle_eg_opts *e, double lr, int radial, int j, double lnratio,
                       cplx *z, double *h, int *run, int *attempts, work *w) {
    int n = S->n, K = e->samples;
    cplx dw = radial ? (cplx)lnratio : I * (2.0 * M_PI / (double)K);
    double v = 0.0;
    while (v < 1.0) {
        if (*attempts >= e->max_attempts) return OE_TRACK_FAILED;
        (*attempts)++;
        double hh = fmin(*h, 1.0 - v), v1 = v + hh;
        if (v1 >= 1.0) { v1 = 1.0; hh = 1.0 - v; }
        cplx hd = hh * dw;
        int bad = dzdw(S, gamma, z, eg_ew(lr, radial, j, K, lnratio, v), w, w->k1);
        cplx em = eg_ew(lr, radial, j, K, lnratio, v + 0.5 * hh);
        if (!bad) { for (int i = 0; i < n; i++) w->zs[i] = z[i] + 0.5 * hd * w->k1[i];
                    bad = dzdw(S, gamma, w->zs, em, w, w->k2); }
        if (!bad) { for (int i = 0; i < n; i++) w->zs[i] = z[i] + 0.5 * hd * w->k2[i];
                    bad = dzdw(S, gamma, w->zs, em, w, w->k3); }
        cplx e1 = eg_ew(lr, radial, j, K, lnratio, v1);
        if (!bad) { for (int i = 0; i < n; i++) w->zs[i] = z[i] + hd * w->k3[i];
                    bad = dzdw(S, gamma, w->zs, e1, w, w->k4); }
        int ok = 0;
        if (!bad) {
            for (int i = 0; i < n; i++)
                w->zp[i] = z[i] + hd / 6.0 * (w->k1[i] + 2.0 * w->k2[i] + 2.0 * w->k3[i] + w->k4[i]);
            double zn = norm2(n, w->zp);
            for (int it = 0; it < o->max_newton; it++) {
                double dn;
                if (newton_hom_c(S, gamma, w->zp, e1, w, &dn)) break;
                if (!all_finite(n, w->zp)) break;
                if (it == 0 && dn > o->trust * (1.0 + zn)) break;
                if (dn <= o->eps_corr * (1.0 + norm2(n, w->zp))) { ok = 1; break; }
            }
        }
        if (ok) {
            memcpy(z, w->zp, sizeof(cplx) * n);
            v = v1;
            if (++*run >= o->grow_after) { *run = 0; *h = fmin(2.0 * *h, 1.0); }
            if (norminf(n, z) > o->r_div) return OE_DIVERGED;
        } else {
            *run = 0;
            *h *= 0.5;
            if (*h < e->h_min) return OE_TRACK_FAILED;
        }
    }
    return OE_NONE;
}

static double dist2(int n, const cplx *a, const cplx *b) {
    double s = 0;
    for (int i = 0; i < n; i++) { cplx d = a[i] - b[i]; s += creal(d) * creal(d) + cimag(d) * cimag(d); }
    return sqrt(s);
}

/* The endgame of one path: track from the start point to t = 1 - r0, then turns around
 * t = 1 at radii r0, r0 ratio, r0 ratio^2, ...  A radius whose turns do not close within
 * max_cycle turns, or where a step fails, encloses more than the endpoint's own branch
 * point (or too sharp a neighbourhood): the path goes back to the point where it reached
 * that radius and continues to the next one.  Two estimates from successive radii that
 * both closed must agree and the estimate must solve P; an estimate that does not,
 * while the distance from each radius's start point to its estimate grows, belongs to a
 * path to infinity.  z (in: start point; out: the last estimate, or the point
 * where it stopped).  Outputs the cycle number and radius of the last closed turns and
 * the distance between the last two estimates. */
static int endgame_path(const qsys *S, cplx gamma, const oracle_track_opts *o,
                        const oracle_eg_opts *e, cplx *z, int *cycle, double *r_last,
                        double *delta, work *w) {
    int n = S->n, K = e->samples, steps;
    double tend;
    *cycle = 0; *r_last = e->r0; *delta = INFINITY;
    int st = track_path(S, gamma, o, 1.0 - e->r0, z, &steps, &tend, w);
    if (st == OR_DIVERGED) return OE_DIVERGED;
    if (st != OR_REACHED) return OE_TRACK_FAILED;
    cplx *zs = malloc(sizeof(cplx) * n), *sum = malloc(sizeof(cplx) * n),
         *est = malloc(sizeof(cplx) * n), *prev = malloc(sizeof(cplx) * n);
    double lnratio = log(e->ratio), h = 1.0;
    int run = 0, attempts = 0, status = OE_NONE, have_prev = 0, last_fail = OE_NOT_CLOSED;
    double d_prev = INFINITY;
    for (int k = 0; k < e->n_radii && status == OE_NONE; k++) {
        double lr = log(e->r0) + k * lnratio;
        if (k > 0) {   /* radial leg from the previous radius */
            int rc = eg_interval(S, gamma, o, e, lr - lnratio, 1, 0, lnratio, z, &h, &run, &attempts, w);
            if (rc != OE_NONE) { status = rc; break; }
        }
        memcpy(zs, z, sizeof(cplx) * n);
        for (int i = 0; i < n; i++) sum[i] = 0;
        int c = 0, rc = OE_NONE;
        for (int turn = 1; turn <= e->max_cycle && !c && rc == OE_NONE; turn++) {
            for (int j = 0; j < K && rc == OE_NONE; j++) {
                for (int i = 0; i < n; i++) sum[i] += z[i];   /* sample at theta = 2 pi j / K */
                rc = eg_interval(S, gamma, o, e, lr, 0, j, lnratio, z, &h, &run, &attempts, w);
            }
            if (rc == OE_NONE && dist2(n, z, zs) <= e->tol_close * (1.0 + norm2(n, zs))) c = turn;
        }
        if (rc == OE_DIVERGED) { status = rc; break; }
        if (rc != OE_NONE || !c) {   /* back to where the path reached this radius */
            memcpy(z, zs, sizeof(cplx) * n);
            h = 1.0;
            run = 0;
            have_prev = 0;
            last_fail = rc != OE_NONE ? OE_TRACK_FAILED : OE_NOT_CLOSED;
            continue;
        }
        *cycle = c;
        *r_last = exp(lr);
        for (int i = 0; i < n; i++) est[i] = sum[i] / (double)(c * K);
        /* distance from the turns' start point to the estimate: ~ r^(1/c) towards a finite
         * endpoint; it grows as r shrinks on a path to infinity, whose mean over a turn is
         * the constant term of a Laurent series, the same at every radius */
        double d = dist2(n, zs, est);
        if (have_prev) {
            *delta = dist2(n, est, prev);
            if (*delta <= e->tol_conv * (1.0 + norm2(n, est))) {
                /* agreement alone is not enough: turns that also enclose the branch point
                 * of two paths with distinct endpoints close after two turns and average
                 * those endpoints, the same at every radius that encloses it.  The
                 * estimate must solve P; if it does not, a path to infinity shows growth
                 * by at least ratio^(-1/c) per radius (c <= max_cycle), and anything else
                 * goes on to smaller radii */
                sys_eval_acc(S, est, w->P);
                double zi = norminf(n, est), scale = zi > 1.0 ? zi * zi : 1.0;
                if (norminf(n, w->P) <= e->tol_res * scale) { status = OE_CONVERGED; break; }
                if (d > d_prev * pow(e->ratio, -0.5 / e->max_cycle)) { status = OE_AT_INFINITY; break; }
            }
        }
        memcpy(prev, est, sizeof(cplx) * n);
        d_prev = d;
        have_prev = 1;
    }
    if (status == OE_NONE) status = have_prev ? OE_NOT_CONVERGED : last_fail;
    if (status == OE_CONVERGED || status == OE_NOT_CONVERGED) memcpy(z, est, sizeof(cplx) * n);
    free(zs); free(sum); free(est); free(prev);
    return status;
}

typedef struct {
    const qsys *S;
    cplx gamma;
    const oracle_track_opts *o;
    const oracle_eg_opts *e;
    const int64_t *paths;
    int64_t npaths;
    double *zre, *zim, *r_last, *delta;
    int *status, *cycle;
    int64_t next;
} eg_job;

static void *eg_worker(void *arg) {
    eg_job *J = arg;
    int n = J->S->n;
    work w;
    work_init(&w, n);
    cplx *z = malloc(sizeof(cplx) * n);
    for (;;) {
        int64_t i = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (i >= J->npaths) break;
        int64_t p = J->paths[i];
        for (int k = 0; k < n; k++) z[k] = ((p >> k) & 1) ? -1.0 : 1.0;
        J->status[i] = endgame_path(J->S, J->gamma, J->o, J->e, z, &J->cycle[i], &J->r_last[i],
                                    &J->delta[i], &w);
        for (int k = 0; k < n; k++) {
            J->zre[i * n + k] = creal(z[k]);
            J->zim[i * n + k] = cimag(z[k]);
        }
    }
    free(z);
    work_free(&w);
    return NULL;
}

/* Cauchy endgame for the paths listed in paths[0 .. npaths-1] (path indices).  Outputs
 * (path-major z [i*n + k]): the estimate of each endpoint, OE_* status, cycle number,
 * radius of the last turn, distance between the last two estimates.  Returns 0, or 1
 * for invalid arguments. */
int oracle_endgame(int n, int nterms, const int *eq, const int *va, const int *vb,
                   const double *cre, const double *cim, double gamma_re, double gamma_im,
                   const oracle_track_opts *o, const oracle_eg_opts *e, const int64_t *paths,
                   int64_t npaths, int nthreads, double *zre, double *zim, int *status,
                   int *cycle, double *r_last, double *delta) {
    if (n < 1 || n > 62 || nthreads < 1 || npaths < 0) return 1;
    if (!(e->r0 > 0.0 && e->r0 < 1.0) || !(e->ratio > 0.0 && e->ratio < 1.0) || e->n_radii < 1 ||
        e->samples < 2 || e->max_cycle < 1)
        return 1;
    qsys S = {n, nterms, eq, va, vb, cre, cim};
    eg_job J = {&S, gamma_re + I * gamma_im, o, e, paths, npaths, zre, zim, r_last, delta,
                status, cycle, 0};
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, eg_worker, &J);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    free(th);
    return 0;
}

/* -------------------------------------------------------- refine and certify -- */
/* ||D^2 P / 2|| bound: the quadratic part of P_i is z^T M_i z with M_i symmetric
 * (a term c z_a z_b puts c on (a,a) when a == b, else c/2 on (a,b) and (b,a)); the
 * bilinear map (u,v) -> (u^T M_i v)_i has operator norm <= sqrt(sum_i ||M_i||_F^2). */
double oracle_d2_norm(int n, int nterms, const int *eq, const int *va, const int *vb,
                      const double *cre, const double *cim) {
    cplx *M = calloc((size_t)n * n * n, sizeof(cplx));
    for (int t = 0; t < nterms; t++) {
        int e = eq[t], a = va[t], b = vb[t];
        if (a < 0 || b < 0) continue;
        cplx c = cre[t] + I * cim[t];
        if (a == b) M[(size_t)e * n * n + a * n + a] += c;
        else { M[(size_t)e * n * n + a * n + b] += 0.5 * c; M[(size_t)e * n * n + b * n + a] += 0.5 * c; }
    }
    double s = 0;
    for (size_t i = 0; i < (size_t)n * n * n; i++) s += creal(M[i]) * creal(M[i]) + cimag(M[i]) * cimag(M[i]);
    free(M);
    return sqrt(s);
}

/* beta = ||DP(z)^-1 P(z)||_2 and ||DP(z)^-1||_F at z.  Returns 1 if DP(z) is singular. */
static int beta_and_inv_norm(const qsys *S, const cplx *z, double *beta, double *invF,
                             double *cond, work *w) {
    int n = S->n;
    sys_jac(S, z, w->A);
    double fro = 0;
    for (int i = 0; i < n * n; i++) fro += creal(w->A[i]) * creal(w->A[i]) + cimag(w->A[i]) * cimag(w->A[i]);
    if (lu_factor(n, w->A, w->piv)) return 1;
    sys_eval_acc(S, z, w->b);
    lu_apply(n, w->A, w->piv, w->b);
    *beta = norm2(n, w->b);
    double s = 0;
    for (int c = 0; c < n; c++) {
        for (int i = 0; i < n; i++) w->P[i] = (i == c) ? 1.0 : 0.0;
        lu_apply(n, w->A, w->piv, w->P);
        double v = norm2(n, w->P);
        s += v * v;
    }
    *invF = sqrt(s);
    *cond = sqrt(fro) * *invF;
    return 0;
}

typedef struct {
    double tol_sol;       /* Delta_sol: ||P(z)||_inf <= tol_sol * max(1, ||z||_inf^2) */
    double refine_eps;    /* Newton refinement stops when ||dz|| <= eps (1 + ||z||) */
    int refine_iters;     /* at most this many refinement steps */
    double alpha0;        /* alpha threshold: half of (13 - 3 sqrt 17) / 4 (FP64 soft test) */
    double kappa_sing;    /* singular when ||DP||_F ||DP^-1||_F > kappa_sing max(1, ||z||_inf^2) */
} oracle_cert_opts;

/* The singularity test.  At a point of a positive-dimensional solution set P vanishes
 * to double-double precision, so beta is tiny, while rounding leaves the computed DP^-1
 * merely huge: the soft FP64 alpha test alone can pass there, so an endpoint whose
 * Jacobian has a Frobenius condition number above kappa_sing is singular.  The bound
 * grows with ||z||_inf^2, as the solution tolerance does: every equation is quadratic,
 * the Jacobian's entries grow like ||z|| and a finite solution near the solution set at
 * infinity has a smallest singular value that shrinks like 1 / ||z||, so an isolated
 * solution of norm 1e6 has a condition number ~1e12 without being singular. */
static int cond_ok(double cond, int n, const cplx *z, double kappa_sing) {
    double zi = norminf(n, z);
    return cond <= kappa_sing * (zi > 1.0 ? zi * zi : 1.0);
}

/* Refine and certify one endpoint.  Outputs: class, alpha, beta, residual, alpha at
 * Re z (the real test).  z is refined in place. */
static int refine_certify_one(const qsys *S, double d2, const oracle_cert_opts *o, cplx *z,
                              double *alpha_out, double *beta_out, double *gam_out,
                              double *res_out, double *alpha_re_out, work *w) {
    int n = S->n;
    *alpha_out = INFINITY; *beta_out = INFINITY; *gam_out = INFINITY; *res_out = INFINITY;
    *alpha_re_out = INFINITY;
    /* Newton on P at t = 1, P evaluated with compensated sums */
    for (int it = 0; it < o->refine_iters; it++) {
        sys_jac(S, z, w->A);
        if (lu_factor(n, w->A, w->piv)) break;
        sys_eval_acc(S, z, w->b);
        lu_apply(n, w->A, w->piv, w->b);
        for (int i = 0; i < n; i++) z[i] -= w->b[i];
        if (!all_finite(n, z)) return OC_SINGULAR;
        if (norm2(n, w->b) <= o->refine_eps * (1.0 + norm2(n, z))) break;
    }
    sys_eval_acc(S, z, w->P);
    double res = norminf(n, w->P);
    *res_out = res;
    double beta, invF, cond;
    if (beta_and_inv_norm(S, z, &beta, &invF, &cond, w)) return OC_SINGULAR;
    double gam = invF * d2, alpha = beta * gam;
    *alpha_out = alpha; *beta_out = beta; *gam_out = gam;
    /* the solution tolerance is applied relative to the size of the equations' terms:
     * every equation is quadratic, so at ||z|| >> 1 its terms are ~||z||^2 and an absolute
     * 1e-10 would sit below the rounding of their sum */
    double zi = norminf(n, z), scale = zi > 1.0 ? zi * zi : 1.0;
    if (!(res <= o->tol_sol * scale) || !(alpha < o->alpha0) || !cond_ok(cond, n, z, o->kappa_sing))
        return OC_SINGULAR;
    double im = 0;
    for (int i = 0; i < n; i++) im += cimag(z[i]) * cimag(z[i]);
    im = sqrt(im);
    /* real test: alpha at x = Re z, a real point of a real system, so that Newton's
     * iterates from x stay real and converge to a real solution.  That solution is z's
     * own when z and x share their associated zero: alpha(z) < 0.03 and
     * ||z - x|| = ||Im z|| < 1 / (20 gamma(z)) (alpha theory's robust-zero bound) */
    if (alpha < 0.03 && im < 1.0 / (20.0 * gam)) {
        cplx *x = w->zs;
        for (int i = 0; i < n; i++) x[i] = creal(z[i]);
        double beta_r, invF_r, cond_r;
        if (!beta_and_inv_norm(S, x, &beta_r, &invF_r, &cond_r, w)) {
            double ar = beta_r * invF_r * d2;
            *alpha_re_out = ar;
            if (ar < o->alpha0 && cond_ok(cond_r, n, x, o->kappa_sing)) return OC_REAL;
        }
    }
    /* non-real test: z and conj(z) have distinct associated solutions when
     * ||z - conj z|| = 2 ||Im z|| > 2 (beta(z) + beta(conj z)) = 4 beta(z) */
    if (im > 2.0 * beta) return OC_NONREAL;
    return OC_UNDECIDED;
}

typedef struct {
    const qsys *S;
    double d2;
    const oracle_cert_opts *o;
    int64_t count;
    double *zre, *zim;
    const int *status;
    const double *tend;
    int *cls;
    double *alpha, *beta, *gam, *res, *alpha_re;
    int64_t next;
} cert_job;

static void *cert_worker(void *arg) {
    cert_job *C = arg;
    int n = C->S->n;
    work w;
    work_init(&w, n);
    cplx *z = malloc(sizeof(cplx) * n);
    for (;;) {
        int64_t i = __atomic_fetch_add(&C->next, 1, __ATOMIC_RELAXED);
        if (i >= C->count) break;
        int st = C->status[i];
        C->alpha[i] = INFINITY; C->beta[i] = INFINITY; C->gam[i] = INFINITY;
        C->res[i] = INFINITY; C->alpha_re[i] = INFINITY;
        if (st == OR_DIVERGED) { C->cls[i] = OC_NONE; continue; }
        if (st != OR_REACHED) { C->cls[i] = OC_FAILED; continue; }
        for (int k = 0; k < n; k++) z[k] = C->zre[i * n + k] + I * C->zim[i * n + k];
        C->cls[i] = refine_certify_one(C->S, C->d2, C->o, z, &C->alpha[i], &C->beta[i],
                                       &C->gam[i], &C->res[i], &C->alpha_re[i], &w);
        for (int k = 0; k < n; k++) { C->zre[i * n + k] = creal(z[k]); C->zim[i * n + k] = cimag(z[k]); }
    }
    free(z);
    work_free(&w);
    return NULL;
}

/* Refine (in place) and certify count endpoints (path-major z).  cls gets the
 * endpoint class; duplicates are marked by oracle_dedup afterwards. */
int oracle_refine_certify(int n, int nterms, const int *eq, const int *va, const int *vb,
                          const double *cre, const double *cim, const oracle_cert_opts *o,
                          int64_t count, int nthreads, double *zre, double *zim,
                          const int *status, const double *tend, int *cls, double *alpha,
                          double *beta, double *gam, double *res, double *alpha_re) {
    if (n < 1 || nthreads < 1 || count < 0) return 1;
    qsys S = {n, nterms, eq, va, vb, cre, cim};
    double d2 = oracle_d2_norm(n, nterms, eq, va, vb, cre, cim);
    cert_job C = {&S, d2, o, count, zre, zim, status, tend, cls, alpha, beta, gam, res, alpha_re, 0};
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int i = 0; i < nthreads; i++) pthread_create(&th[i], NULL, cert_worker, &C);
    for (int i = 0; i < nthreads; i++) pthread_join(th[i], NULL);
    free(th);
    return 0;
}

/* ------------------------------------------------------------------- dedup -- */
typedef struct { double key; int64_t idx; } keyed;

static int cmp_keyed(const void *a, const void *b) {
    double x = ((const keyed *)a)->key, y = ((const keyed *)b)->key;
    if (x < y) return -1;
    if (x > y) return 1;
    int64_t i = ((const keyed *)a)->idx, j = ((const keyed *)b)->idx;
    return (i > j) - (i < j);
}

/* alpha-theory decides whether two certified endpoints z1, z2 approximate the same
 * solution: they do when alpha(z1) < 0.03 and ||z1 - z2|| < 1 / (20 gamma(z1)), and they
 * do not when ||z1 - z2|| > 2 (beta1 + beta2) (each lies within 2 beta of its
 * solution).  A pair that is not proved distinct is counted as the same solution.
 * Within each such pair the higher path index becomes OC_DUPLICATE.  Candidates are
 * found by sorting on Re z_0 and comparing every pair whose keys differ by no more
 * than the largest radius in play.  Returns the number of duplicates. */
int64_t oracle_dedup(int n, int64_t count, const double *zre, const double *zim,
                     const double *beta, const double *gam, int *cls) {
    keyed *K = malloc(sizeof(keyed) * (count > 0 ? count : 1));
    int64_t nk = 0;
    double rmax = 0;
    for (int64_t i = 0; i < count; i++)
        if (cls[i] == OC_REAL || cls[i] == OC_NONREAL || cls[i] == OC_UNDECIDED) {
            K[nk].key = zre[i * n];
            K[nk].idx = i;
            nk++;
            double r = fmax(4.0 * beta[i], 1.0 / (20.0 * gam[i]));
            if (r > rmax) rmax = r;
        }
    qsort(K, nk, sizeof(keyed), cmp_keyed);
    int64_t dups = 0;
    for (int64_t a = 0; a < nk; a++) {
        int64_t i = K[a].idx;
        for (int64_t b = a + 1; b < nk && K[b].key - K[a].key <= rmax; b++) {
            int64_t j = K[b].idx;
            double d = 0;
            for (int k = 0; k < n; k++) {
                double dr = zre[i * n + k] - zre[j * n + k], di = zim[i * n + k] - zim[j * n + k];
                d += dr * dr + di * di;
            }
            d = sqrt(d);
            int same_i = beta[i] * gam[i] < 0.03 && d < 1.0 / (20.0 * gam[i]);
            int same_j = beta[j] * gam[j] < 0.03 && d < 1.0 / (20.0 * gam[j]);
            int distinct = d > 2.0 * (beta[i] + beta[j]);
            if (same_i || same_j || !distinct) {
                int64_t hi = i < j ? j : i;
                if (cls[hi] != OC_DUPLICATE) { cls[hi] = OC_DUPLICATE; dups++; }
            }
        }
    }
    free(K);
    return dups;
}

/* --------------------------------------------------------------- classify -- */
/* For a real stationary point (c, s) of the XY ring (m = N-1 free sites):
 * theta_k = atan2(s_k, c_k) in (-pi, pi] (theta_N = 0), the Hessian of
 * V = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)) in theta_1..theta_m,
 *   H_kk = sum_{j != k} J_kj cos(theta_k - theta_j),  H_kl = -J_kl cos(theta_k - theta_l),
 * its index (number of negative eigenvalues), its smallest |eigenvalue| and the energy V.
 * hess_out (m*m, may be NULL) receives H. */
int oracle_xy_classify(int N, const double *J, const double *c, const double *s,
                       double *theta, int *index, double *energy, double *min_abs_eig,
                       double *log_abs_det, double *hess_out) {
    int m = N - 1;
    double *th = malloc(sizeof(double) * N), *H = malloc(sizeof(double) * m * m),
           *w = malloc(sizeof(double) * m);
    for (int k = 0; k < m; k++) {
        double a = atan2(s[k], c[k]);
        if (a <= -M_PI) a = M_PI;
        th[k] = a;
        theta[k] = a;
    }
    th[m] = 0.0;
    for (int k = 0; k < m; k++)
        for (int l = 0; l < m; l++) {
            if (k == l) {
                double d = 0;
                for (int j = 0; j < N; j++) if (j != k) d += J[k * N + j] * cos(th[k] - th[j]);
                H[k * m + k] = d;
            } else {
                H[k * m + l] = -J[k * N + l] * cos(th[k] - th[l]);
            }
        }
    if (hess_out) memcpy(hess_out, H, sizeof(double) * m * m);
    double V = 0;
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) V += J[i * N + j] * (1.0 - cos(th[i] - th[j]));
    jacobi_eig(m, H, w);
    int neg = 0;
    double mn = INFINITY, ld = 0.0;
    for (int k = 0; k < m; k++) {
        if (w[k] < 0) neg++;
        if (fabs(w[k]) < mn) mn = fabs(w[k]);
        ld += log(fabs(w[k]));   /* log |det H| = sum of log |eigenvalue| */
    }
    *index = neg;
    *energy = V;
    *min_abs_eig = mn;
    *log_abs_det = ld;
    free(th); free(H); free(w);
    return 0;
}

/* ----------------------------------------------------------------- adjoint -- */
/* Gradient with respect to the couplings of a loss L(V*, theta*) at a real stationary
 * point theta* (theta_N = 0 pinned) of V = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)).
 * theta* solves G(theta; J) = grad_theta V = 0, so (implicit function theorem)
 * d(theta*) / dJ_ij = -H^-1 dG/dJ_ij with H the Hessian in theta_1..theta_m, and
 * d(V at theta*) / dJ_ij = dV/dJ_ij (G = 0).  With H lambda = dL/dtheta (lambda_N = 0) and
 * dG_i/dJ_ij = sin(theta_i - theta_j) = -dG_j/dJ_ij:
 *   dL/dJ_ij = gV (1 - cos(theta_i - theta_j)) - (lambda_i - lambda_j) sin(theta_i - theta_j).
 * gV = dL/dV; g = dL/dtheta (m entries, NULL = 0).  dJ (N x N, symmetric, zero diagonal)
 * receives dL/dJ_ij for the one parameter J_ij = J_ji.  Returns 1 if H is singular. */
int oracle_xy_adjoint(int N, const double *J, const double *theta, double gV, const double *g,
                      double *dJ) {
    int m = N - 1;
    double *th = malloc(sizeof(double) * N), *lam = calloc(N, sizeof(double));
    cplx *H = malloc(sizeof(cplx) * m * m), *b = malloc(sizeof(cplx) * m);
    int *piv = malloc(sizeof(int) * m), bad = 0;
    for (int k = 0; k < m; k++) th[k] = theta[k];
    th[m] = 0.0;
    if (g) {
        for (int k = 0; k < m; k++)
            for (int l = 0; l < m; l++) {
                double v;
                if (k == l) {
                    v = 0;
                    for (int j = 0; j < N; j++) if (j != k) v += J[k * N + j] * cos(th[k] - th[j]);
                } else {
                    v = -J[k * N + l] * cos(th[k] - th[l]);
                }
                H[k * m + l] = v;
            }
        for (int k = 0; k < m; k++) b[k] = g[k];
        if (lu_factor(m, H, piv)) bad = 1;
        else {
            lu_apply(m, H, piv, b);
            for (int k = 0; k < m; k++) lam[k] = creal(b[k]);
        }
    }
    for (int i = 0; i < N; i++) {
        dJ[i * N + i] = 0.0;
        for (int j = i + 1; j < N; j++) {
            double d = th[i] - th[j];
            double v = gV * (1.0 - cos(d)) - (lam[i] - lam[j]) * sin(d);
            dJ[i * N + j] = v;
            dJ[j * N + i] = v;
        }
    }
    free(th); free(lam); free(H); free(b); free(piv);
    return bad;
}

