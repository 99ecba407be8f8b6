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

// ------------------------------------------------------ float-float sums --
// Error-free transformations (Knuth's two-sum, FMA two-product) with round-to-
// nearest intrinsics, so the compiler cannot contract or reassociate them.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += a * b with a, b floats; the rounding errors of the product and of the sum
// are collected in acc.lo (compensated dot product).
__device__ __forceinline__ void ff_acc(ff &acc, float a, float b) {
    float p, e, s, e2;
    two_prod(a, b, p, e);
    two_sum(acc.hi, p, s, e2);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, e2));
}

// acc += a * (b.hi + b.lo)
__device__ __forceinline__ void ff_acc_ff(ff &acc, float a, ff b) {
    ff_acc(acc, a, b.hi);
    acc.lo = __fmaf_rn(a, b.lo, acc.lo);
}

__device__ __forceinline__ float ff_val(ff a) { return __fadd_rn(a.hi, a.lo); }

// ------------------------------------------------------ launch arguments --
// Couplings and homotopy constants of one XY ring, passed by value so that the
// unrolled kernels read them as constant-bank operands.
struct XYSys {
    int N;                                  // ring size; M = N - 1 free sites
    float Jf[NPHC_MAXN * NPHC_MAXN];        // J in FP32 (row k, column j at k * NPHC_JSTRIDE + j)
    double Jd[NPHC_MAXN * NPHC_MAXN];       // J in FP64
    double gre, gim;                        // gamma
    double d2norm;                          // ||D^2 P / 2|| bound (alpha-theory gamma)
};

struct XYCtl {                              // step control of one tracking call
    double h0, hmax, hmin, eps, trust;
    double rdiv;                            // divergence radius (final)
    double rdiv_soft;                       // FP32: radius where the growth test decides
    double rho_div;                         // FP32: growth exponent meaning divergence
    int max_newton, max_steps, grow_after;
    int handoff;                            // 1: stops become NPHC_PATH_HANDOFF (FP32 pass)
    int resume;                             // 1: continue from (z, t, h) of the entry
    int accumulate;                         // 1: add to the entry's step/solve counters
    int sparse;                             // 1: one path per warp (lane 0 only)
};

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

__device__ __forceinline__ int64_t worklist_size(const WorkList &w, int64_t count) {
    return w.list ? (int64_t)(*w.list_count) : count;
}
__device__ __forceinline__ int64_t worklist_entry(const WorkList &w, int64_t i) {
    return w.list ? (int64_t)w.list[i] : i;
}

// ------------------------------------------------------ kernel launchers --
// Implemented per precision / ring size in the .cu files; return cudaGetLastError().
cudaError_t launch_xy_track_f32(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                const WorkList &wl, int block, int grid, cudaStream_t st);
cudaError_t launch_xy_track_f64(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                const WorkList &wl, int block, int grid, cudaStream_t st);
cudaError_t launch_xy_refine_certify(int M, const XYSys &sys, double tol_sol, double refine_eps,
                                     int refine_iters, const EPView &ep, int64_t cap,
                                     const WorkList &wl, cudaStream_t st);
cudaError_t launch_xy_classify(int M, const XYSys &sys, const EPView &ep, double *theta,
                               int32_t *index, double *energy, double *min_eig,
                               cudaStream_t st);
// Host-side count of kernel launches made by this library (for the result counters).
int64_t nphc_launch_counter(int64_t add);
int xy_track_f32_block(int M);
int xy_track_f64_block(int M);
