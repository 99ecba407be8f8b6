// nphc_internal.cuh -- device-side building blocks shared by the NPHC kernels:
// complex arithmetic, float-float (compensated) accumulation, and the launch
// arguments of the XY-ring kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nphc.h"

#define NPHC_MAXN NPHC_MAX_N          // couplings are stored in NPHC_MAXN x NPHC_MAXN tables
#define NPHC_JSTRIDE NPHC_MAXN

// ------------------------------------------------------------------ complex --
template <class R>
struct alignas(2 * sizeof(R)) cx {
    R re, im;
};

template <class R>
__device__ __forceinline__ cx<R> cmake(R a, R b) { return cx<R>{a, b}; }
template <class R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return cx<R>{a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return cx<R>{a.re - b.re, a.im - b.im}; }
template <class R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    return cx<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
    return cx<R>{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <class R>
__device__ __forceinline__ cx<R> cscale(R s, cx<R> a) { return cx<R>{s * a.re, s * a.im}; }
template <class R>
__device__ __forceinline__ R cabs2(cx<R> a) { return a.re * a.re + a.im * a.im; }

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float recip_r(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip_r(double x) { return 1.0 / x; }

template <class R>
__device__ __forceinline__ cx<R> crecip(cx<R> a) {
    R s = recip_r(cabs2(a));
    return cx<R>{a.re * s, -a.im * s};
}

template <class R>
__device__ __forceinline__ bool finite_r(R v) { return isfinite(v); }

// ---------------------------------------------- compensated (two-word) sums --
// Error-free transformations (Knuth's two-sum, FMA two-product) with round-to-nearest
// intrinsics, so that the compiler can neither contract nor reassociate them.  R is
// float (float-float accumulation for the FP32 corrector) or double (double-double for
// the FP64 corrector).
template <class R>
struct EFT;
template <>
struct EFT<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <>
struct EFT<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

template <class R>
struct ext {   // hi + lo, |lo| ~ ulp(hi)
    R hi, lo;
};

template <class R>
__device__ __forceinline__ void two_prod(R a, R b, R &p, R &e) {
    p = EFT<R>::mul(a, b);
    e = EFT<R>::fma(a, b, -p);
}

template <class R>
__device__ __forceinline__ void two_sum(R a, R b, R &s, R &e) {
    s = EFT<R>::add(a, b);
    const R bb = EFT<R>::sub(s, a);
    e = EFT<R>::add(EFT<R>::sub(a, EFT<R>::sub(s, bb)), EFT<R>::sub(b, bb));
}

// acc += a * b; the rounding errors of the product and of the sum are collected in
// acc.lo (compensated dot product)
template <class R>
__device__ __forceinline__ void ext_acc(ext<R> &acc, R a, R b) {
    R p, e, s, e2;
    two_prod(a, b, p, e);
    two_sum(acc.hi, p, s, e2);
    acc.hi = s;
    acc.lo = EFT<R>::add(acc.lo, EFT<R>::add(e, e2));
}

// acc += a * (b.hi + b.lo)
template <class R>
__device__ __forceinline__ void ext_acc_ext(ext<R> &acc, R a, ext<R> b) {
    ext_acc(acc, a, b.hi);
    acc.lo = EFT<R>::fma(a, b.lo, acc.lo);
}

template <class R>
__device__ __forceinline__ R ext_val(ext<R> a) { return EFT<R>::add(a.hi, a.lo); }

// ------------------------------------------------------ launch arguments --
// Couplings and homotopy constants of one XY ring, passed by value so that the
// unrolled kernels read them as constant-bank operands.
struct XYSys {
    int N;                                  // ring size; M = N - 1 free sites
    float Jf[NPHC_MAXN * NPHC_MAXN];        // J in FP32 (row k, column j at k * NPHC_JSTRIDE + j)
    double Jd[NPHC_MAXN * NPHC_MAXN];       // J in FP64
    double gre, gim;                        // gamma
    double d2norm;                          // ||D^2 P / 2|| bound (alpha-theory gamma)
    double kappa_sing;                      // singular above kappa_sing max(1, ||z||_inf^2)
};

struct XYCtl {                              // step control of one tracking call
    double h0, hmax, hmin, eps, trust;
    double rdiv;                            // divergence radius on ||z||_inf
    int max_newton, max_steps, grow_after;
    int handoff;                            // 1: stops become NPHC_PATH_HANDOFF (FP32 pass)
    int resume;                             // 1: continue from (z, t, h) of the entry
    int accumulate;                         // 1: add to the entry's step/solve counters
    int sparse;                             // 1: spread a short list, ceil(list / warps) paths per warp
    int crawl_steps;                        // near t = 1, 1 - t must halve within this many
                                            // accepted steps (0: no crawl test)
    double t_end;                           // tracking stops here: 1, or 1 - r0 before the
                                            // Cauchy endgame
    double kappa;                           // FP32 pass: a step attempt whose solves' condition
                                            // estimate exceeds this hands the path to FP64
                                            // (NPHC_PATH_HANDOFF_COND); 0: no test
};

struct EGCtl {                              // the Cauchy endgame (cauchy.cuh)
    double lr0, lnratio;                    // ln of the first radius |1 - t| and of the ratio
    int n_radii, samples, max_cycle;        // radii, samples per turn, largest cycle number
    double tol_close, tol_conv;             // turn closure and estimate agreement (relative)
    double tol_res;                         // the estimate solves P: ||P||_inf <= tol max(1, ||e||^2)
    double grow_inf;                        // growth per radius of a pole: ratio^(-1/(2 max_cycle))
    double hmin;                            // smallest step, in sample intervals
    int max_attempts;                       // step attempts per path
    double eps, trust, rdiv;                // corrector tolerance, first-correction bound,
    int max_newton, grow_after;             // divergence radius, as for FP64 tracking
};

// Scratch vectors per thread of the Cauchy endgame (the trackers keep four).
#define NPHC_CAUCHY_STATE_VECTORS 6

struct EPView {                             // device endpoint arrays (see nphc_endpoints)
    int64_t count;
    const int64_t *path;
    double *z_re, *z_im, *t, *h;
    int32_t *status, *steps, *solves, *newton, *cls;  // cls may be NULL during tracking
    double *alpha, *beta, *gamma, *resid;
};

struct WorkList {                           // which entries a launch processes
    const int32_t *list;                    // NULL: all entries
    const int32_t *list_count;              // device count of list
    unsigned long long *queue;              // zeroed work counter (persistent kernels)
    void *state;                            // tracker scratch: per-thread path state
    int64_t state_threads;                  // threads the scratch holds state for
};

// Threads of a persistent tracker grid the tracker scratch is sized for (a grid never
// launches more threads than this).
#define NPHC_TRACK_MAX_THREADS 65536

// Index checks of the debug build (compiled with NPHC_DEBUG, relocatable device code):
// NPHC_VALID(cond, code) is cond, and a false cond records code in nphc_dbg_error (the
// first one wins; nphc_debug_check reads it) so that the caller skips the access.  In a
// release build it is true and cond is not evaluated.  Codes: 1 a work-list entry outside
// the endpoint set, 2 an append beyond a list's capacity, 3 a dedup link outside the
// endpoint set, 4 a batch item outside its group, 5 a gathered entry outside the set.
#ifdef NPHC_DEBUG
extern __device__ int nphc_dbg_error;
__device__ __forceinline__ bool nphc_dbg_fail(int code) {
    atomicCAS(&nphc_dbg_error, 0, code);
    return false;
}
#define NPHC_VALID(cond, code) ((cond) ? true : nphc_dbg_fail(code))
#else
#define NPHC_VALID(cond, code) true
#endif

__device__ __forceinline__ int64_t worklist_size(const WorkList &w, int64_t count) {
    return w.list ? (int64_t)(*w.list_count) : count;
}
// Entry i of the work list (i itself without a list); -1 when the debug build finds the
// entry outside [0, count).
__device__ __forceinline__ int64_t worklist_entry(const WorkList &w, int64_t i, int64_t count) {
    const int64_t e = w.list ? (int64_t)w.list[i] : i;
    (void)count;
    return NPHC_VALID(e >= 0 && e < count, 1) ? e : -1;
}

// A generic quadratic system (quad.cuh): P_i(z) = sum of c w(a) w(b), w(-1) = 1, terms
// sorted by equation.
struct QTerm {
    int32_t a, b;      // variable indices, -1 for the constant 1
    double cre, cim;   // coefficient
};

struct QSys {
    int n;
    const int32_t *row;    // [n + 1] term offsets per equation (device)
    const QTerm *terms;    // [row[n]] (device)
    double gre, gim;       // gamma
    double d2norm;         // ||D^2 P / 2|| bound
    double kappa_sing;     // singular above kappa_sing max(1, ||z||_inf^2)
};

// One group of a batch: instances of one ring size whose FP32 pass runs as one launch
// (device tables; off[g] = paths of instances 0 .. g-1 of the group, off[n] the total).
struct BatchGroup {
    const XYSys *sys;
    const EPView *ep;
    const int64_t *off;
    int n;
    int64_t total;   // off[n], on the host
};

// ------------------------------------------------------ kernel launchers --
// Implemented per precision / ring size in the .cu files; return cudaGetLastError().
cudaError_t launch_xy_track_f32(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                const WorkList &wl, int block, int grid, cudaStream_t st);
cudaError_t launch_xy_track_f64(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                const WorkList &wl, int block, int grid, cudaStream_t st);
// The FP32 pass over every path of a batch group (ring size M), one persistent launch.
cudaError_t launch_xy_track_f32_batch(int M, const BatchGroup &bg, const XYCtl &ctl,
                                      const WorkList &wl, int grid, cudaStream_t st);
// FP64 tracking with one path per warp (xy_track_warp.cuh), for short lists.
cudaError_t launch_xy_track_f64_warp(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                     const WorkList &wl, cudaStream_t st);
cudaError_t launch_xy_refine_certify(int M, const XYSys &sys, double tol_sol, double refine_eps,
                                     int refine_iters, const EPView &ep, int64_t cap,
                                     const WorkList &wl, int shortcut, cudaStream_t st);
// Classification of every entry, or (list, device list_count) of listed real entries only,
// 32 to a warp (the other entries' outputs are then left as they are).
cudaError_t launch_xy_classify(int M, const XYSys &sys, const EPView &ep, double *theta,
                               int32_t *index, double *energy, double *min_eig,
                               double *log_abs_det,
                               cudaStream_t st, const int32_t *list = nullptr,
                               const int32_t *list_count = nullptr);
cudaError_t launch_quad_track(int n, const QSys &sys, const XYCtl &ctl, const EPView &ep,
                              const WorkList &wl, int grid, cudaStream_t st);
cudaError_t launch_quad_refine_certify(int n, const QSys &sys, double tol_sol, double refine_eps,
                                       int refine_iters, const EPView &ep, int64_t cap,
                                       const WorkList &wl, cudaStream_t st);
cudaError_t launch_xy_adjoint(int M, const XYSys &sys, int64_t count, const double *theta,
                              const double *g_energy, const double *g_theta, double *dJ,
                              cudaStream_t st);
// The Cauchy endgame (cauchy.cuh) over the entries of wl, from points at t = 1 - r0.
cudaError_t launch_xy_cauchy(int M, const XYSys &sys, const EGCtl &ctl, const EPView &ep,
                             const WorkList &wl, int32_t *cyc, int32_t *egst, cudaStream_t st);
cudaError_t launch_quad_cauchy(int n, const QSys &sys, const EGCtl &ctl, const EPView &ep,
                               const WorkList &wl, int32_t *cyc, int32_t *egst, cudaStream_t st);
// Host-side count of kernel launches made by this library (for the result counters).
int64_t nphc_launch_counter(int64_t add);
int xy_track_f32_block(int M);
int xy_track_f64_block(int M);
