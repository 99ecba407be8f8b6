// xy_track.cuh -- path tracker for the XY-ring total-degree homotopy
// (section "Numerical Polynomial Homotopy Continuation Method": H = gamma (1-t) Q + t P,
// Q_i = z_i^2 - 1, start points z_i = +-1, tracked from t = 0 to t = 1 with a
// predictor and Newton's corrector).
//
// Layout: one path per thread; a persistent grid pulls paths from a device work
// counter (warp-aggregated atomics) until the list is drained.  The warp runs its 32
// paths in lockstep through the same phases of a step -- three RK4 stage solves, then
// up to max_newton corrector solves -- in a loop with a single call site of the solve,
// so the heavy solve is never divergent and its unrolled code is instantiated once
// (instruction-cache resident); lanes whose path has finished take the next one at
// the step boundary.  The M x M Schur matrix, the evaluation point and the solve
// output of each path live in shared memory (xy_solve.cuh); the accepted point, its
// derivative and the RK4 sum live in a global scratch (coalesced, L2-resident).
//
// Predictor: classical RK4 on dz/dt = -H_z^-1 H_t.  The derivative at the start of a
// step is taken from the previous step's last corrector solve (second right-hand
// side, same factorisation), and at t = 0 it is known in closed form
// (H_z = 2 gamma diag(z), H_t = P(z)), so each step costs 3 stage solves.
// Corrector: Newton at t + h, its residual evaluated with compensated sums
// (xy_residual_comp: float-float in FP32, double-double in FP64).  A step is accepted when ||dz|| <= eps (1 + ||z||)
// within max_newton iterations, and rejected when the first correction exceeds
// trust (1 + ||z||).  Step size doubles after grow_after consecutive accepts and halves
// on a reject; the final step lands exactly on t = t_end (1, or 1 - r0 before the Cauchy
// endgame).
//
// A path whose ||z||_inf exceeds rdiv (1e8 by default) is taken to go to infinity, in
// either precision, as in the oracle: finite solutions of large norm are approached with
// the same power-law growth as paths to infinity, so only a radius far beyond the
// solutions sought tells them apart.  The tracker's state is kept in light-cone
// coordinates (XYProblem, xy_solve.cuh), which FP32 resolves out to that radius.
// FP32 pass (ctl.handoff = 1): on a step size underflow, ten consecutive rejects, a
// crawl near t = 1 (1 - t failing to halve within crawl_steps accepted steps), its own
// (smaller) attempt budget or a radius crossing within RDIV_BAND close to t = 1, a path
// is handed to FP64 (NPHC_PATH_HANDOFF) with the (z, t, h) of its last clean accepted
// point in the end zone 1 - t < CRAWL_ZONE (accepted right after another accepted step),
// or of its last accepted point if it never got there; a converged step whose condition
// estimate exceeds ctl.kappa ends it the same way (NPHC_PATH_HANDOFF_COND).  FP64 tracks like
// the oracle: no crawl test, the same step budget and minimum step.  The FP32 bound on
// the first correction (trust_fp32) keeps its accepted steps no longer than the FP64
// tolerance allows, so that it does not step across a sharp turn of the path onto a
// neighbouring one.
#pragma once

#include "xy_solve.cuh"

template <class R>
struct JSel;
template <>
struct JSel<float> {
    static __device__ __forceinline__ const float *get(const XYSys &S) { return S.Jf; }
};
template <>
struct JSel<double> {
    static __device__ __forceinline__ const double *get(const XYSys &S) { return S.Jd; }
};

#define CRAWL_ZONE 1e-3   // the crawl test applies once 1 - t < CRAWL_ZONE
// A path in the end zone whose ||z||_inf exceeds FAR_NORM and grew by more than FAR_GROWTH
// on its last accepted step is heading out (to infinity, or to a finite solution of
// large norm it has not reached yet): its next step is at most KAPPA_FAR (1 - t), so that
// it does not try to land on t = 1 while it still grows (such a landing always fails,
// and halving back cost as many solves as the steps themselves).  The ratio is set by the
// trust bound on the first Newton correction: at 0.5 a third of the far attempts of the
// N = 10 ring's paths to infinity failed it (18 rejects per path, each three stage solves
// and a correction wasted), while a small ratio takes more steps per decade of 1 - t;
// measured over 0.25 .. 0.5 on the N = 10 and N = 12 rings, 0.38 took the fewest solves at
// both (-23% against 0.5), with the same certified sets.  Once the path stops growing the
// cap is off and the step to t = 1 is tried as usual.
#define FAR_NORM 10.0
#define FAR_GROWTH 1.01
#define KAPPA_FAR 0.38
#define NEAR_END 1e-5     // FP32 radius crossings with 1 - t below this ...
#define RDIV_BAND 1e-3    // ... and ||z||_inf within rdiv (1 + RDIV_BAND) go to FP64

template <int NV, class R, class V>
__device__ __forceinline__ R vnorm2(const V &v) {
    R s = R(0);
#pragma unroll 1
    for (int i = 0; i < NV; i++) s += cabs2(v.get(i));
    return sqrt_r(s);
}

template <int NV, class R, class V>
__device__ __forceinline__ R vnorminf(const V &v) {
    R s = R(0);
#pragma unroll 1
    for (int i = 0; i < NV; i++) s = fmax(s, sqrt_r(cabs2(v.get(i))));
    return s;
}

// The problem a tracker runs on, as a policy for track_body: the unknowns (NV), the
// per-thread shared matrix (MD x (MD + 2)), the start point with its dz/dt, the
// corrector residual -H, the linear solve, and the tracker state's relation to the
// endpoint arrays' z (load, store, the factor that turns the state's 2-norm into z's and
// z's inf-norm).  XYProblem: the XY ring (structured Schur solve, M = N - 1 free sites,
// NV = 2M), its state in light-cone coordinates p_k = x_k + i y_k, q_k = x_k - i y_k
// (xy_solve.cuh): a unitary map times sqrt(2), so 2-norms are the state's over sqrt(2).
template <int M, class RT, int BLK>
struct XYProblem {
    using R = RT;
    using Sys = XYSys;
    static constexpr int BLOCK = BLK;
    static constexpr int NV = 2 * M;
    static constexpr int MD = M;
    static constexpr R NORM_SCALE = R(0.70710678118654752440);   // sqrt(1/2)

    // (x, y) of the endpoint arrays (FP64) to (p, q), formed in FP64 and then rounded
    template <class V>
    static __device__ __forceinline__ void load(const EPView &ep, int64_t e, const V &Z) {
        const int64_t cnt = ep.count;
#pragma unroll 1
        for (int k = 0; k < M; k++) {
            const double xr = ep.z_re[k * cnt + e], xi = ep.z_im[k * cnt + e];
            const double yr = ep.z_re[(M + k) * cnt + e], yi = ep.z_im[(M + k) * cnt + e];
            Z.set(k, cx<R>{(R)(xr - yi), (R)(xi + yr)});
            Z.set(M + k, cx<R>{(R)(xr + yi), (R)(xi - yr)});
        }
    }
    // (p, q) to x = (p + q) / 2, y = -i (p - q) / 2, in FP64
    template <class V>
    static __device__ __forceinline__ void store(const EPView &ep, int64_t e, const V &Z) {
        const int64_t cnt = ep.count;
#pragma unroll 1
        for (int k = 0; k < M; k++) {
            const cx<R> pk = Z.get(k), qk = Z.get(M + k);
            const double pr = pk.re, pi = pk.im, qr = qk.re, qi = qk.im;
            ep.z_re[k * cnt + e] = 0.5 * (pr + qr);
            ep.z_im[k * cnt + e] = 0.5 * (pi + qi);
            ep.z_re[(M + k) * cnt + e] = 0.5 * (pi - qi);
            ep.z_im[(M + k) * cnt + e] = -0.5 * (pr - qr);
        }
    }
    // max_k max(|x_k|, |y_k|) = max_k max(|p_k + q_k|, |p_k - q_k|) / 2
    template <class V>
    static __device__ __forceinline__ R norminf(const V &Z) {
        R s = R(0);
#pragma unroll 1
        for (int k = 0; k < M; k++) {
            const cx<R> pk = Z.get(k), qk = Z.get(M + k);
            s = fmax(s, fmax(cabs2(cadd(pk, qk)), cabs2(csub(pk, qk))));
        }
        return R(0.5) * sqrt_r(s);
    }

    // start point of path p and its derivative: at t = 0, H_z = 2 gamma diag(z) and
    // H_t = P(z), so dz_i/dt = -P_i(z) / (2 gamma z_i); both in light-cone coordinates
    static __device__ __forceinline__ void start(const Sys &S, int64_t p, const GVec<R> &Z0,
                                                 const GVec<R> &K1) {
        const R *J = JSel<R>::get(S);
        const cx<R> gam = cx<R>{(R)S.gre, (R)S.gim};
        cx<R> x[M], y[M];
#pragma unroll
        for (int k = 0; k < M; k++) {
            x[k] = cx<R>{((p >> k) & 1) ? R(-1) : R(1), R(0)};
            y[k] = cx<R>{((p >> (M + k)) & 1) ? R(-1) : R(1), R(0)};
        }
        const cx<R> ig = crecip(gam);
#pragma unroll 1
        for (int k = 0; k < M; k++) {
            const cx<R> xk = cx<R>{((p >> k) & 1) ? R(-1) : R(1), R(0)};
            const cx<R> yk = cx<R>{((p >> (M + k)) & 1) ? R(-1) : R(1), R(0)};
            cx<R> u, w, rf, rg;
            xy_uw<M, R>(J, x, y, k, u, w);
            minus_ht_rows<R>(xk, yk, u, w, gam, rf, rg);
            const cx<R> dx = cscale(R(0.5) * xk.re, cmul(ig, rf));
            const cx<R> dy = cscale(R(0.5) * yk.re, cmul(ig, rg));
            Z0.set(k, cx<R>{xk.re, yk.re});    // p = x + i y (x, y real at the start)
            Z0.set(M + k, cx<R>{xk.re, -yk.re});
            K1.set(k, cadd(dx, cmul_i(dy)));
            K1.set(M + k, csub(dx, cmul_i(dy)));
        }
    }

    static __device__ __forceinline__ void residual(const Sys &S, const SVec<R, BLOCK> &pt, R s,
                                                    R omt, const SVec<R, BLOCK> &out, bool wr) {
        residual_g(S, pt, s, omt, cx<R>{(R)S.gre, (R)S.gim}, out, wr);
    }

    template <class Out2>
    static __device__ __forceinline__ bool solve(const Sys &S, const SMat<M, R, BLOCK> &A,
                                                 const SVec<R, BLOCK> &pt, R s, R omt,
                                                 bool two_rhs, const SVec<R, BLOCK> &res,
                                                 const SVec<R, BLOCK> &out1, const Out2 &out2,
                                                 bool wr, R *kest = nullptr) {
        return solve_g(S, A, pt, s, omt, cx<R>{(R)S.gre, (R)S.gim}, two_rhs, res, out1, out2, wr,
                       kest);
    }

    // the same with an explicit gamma (per thread: the Cauchy endgame's equivalent real-t
    // homotopy at a complex t)
    static __device__ __forceinline__ void residual_g(const Sys &S, const SVec<R, BLOCK> &pt, R s,
                                                      R omt, cx<R> gam,
                                                      const SVec<R, BLOCK> &out, bool wr) {
        xy_residual_comp<M, R, BLOCK>(JSel<R>::get(S), pt, s, omt, gam, out, wr);
    }

    template <class Out2>
    static __device__ __forceinline__ bool solve_g(const Sys &S, const SMat<M, R, BLOCK> &A,
                                                   const SVec<R, BLOCK> &pt, R s, R omt,
                                                   cx<R> gam, bool two_rhs,
                                                   const SVec<R, BLOCK> &res,
                                                   const SVec<R, BLOCK> &out1, const Out2 &out2,
                                                   bool wr, R *kest = nullptr) {
        return xy_solve<M, R, BLOCK>(JSel<R>::get(S), A, pt, s, omt, gam, two_rhs, res, out1, out2,
                                     wr, kest);
    }
};

// Shared memory per thread of a tracker on problem P: the augmented matrix and the
// evaluation point; the solve output / residual vector (NV entries) is the matrix's
// right-hand-side columns (see xy_smem_per_thread).
template <class P>
constexpr size_t track_smem_per_thread() {
    return sizeof(cx<typename P::R>) * (size_t)(P::MD * (P::MD + 2) + P::NV);
}

// Where a tracker's entries come from.  SingleSrc: one system and its endpoint arrays,
// optionally through a work list.  BatchSrc: instances of one ring size (a batch), their
// entries numbered one after another: item i of the launch's queue is entry i - off[g]
// of instance g, off[g] <= i < off[g + 1], whose couplings and endpoint arrays are
// sys[g] and ep[g] (device tables).
template <class Sys>
struct SingleSrc {
    const Sys &S;
    const EPView &ep;
    const WorkList &wl;
    __device__ __forceinline__ int64_t total() const { return worklist_size(wl, ep.count); }
    __device__ __forceinline__ void take(int64_t i, int &g, int64_t &e) const {
        g = 0;
        e = worklist_entry(wl, i, ep.count);
    }
    __device__ __forceinline__ const Sys &sys(int) const { return S; }
    __device__ __forceinline__ const EPView &eps(int) const { return ep; }
};

template <class Sys>
struct BatchSrc {
    const Sys *__restrict__ S;
    const EPView *__restrict__ ep;
    const int64_t *__restrict__ off;   // [n + 1] prefix sums of the instances' path counts
    int n;
    __device__ __forceinline__ int64_t total() const { return off[n]; }
    __device__ __forceinline__ void take(int64_t i, int &g, int64_t &e) const {
        int lo = 0, hi = n - 1;   // the last g with off[g] <= i
#pragma unroll 1
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        g = lo;
        e = i - off[lo];
        if (!NPHC_VALID(e >= 0 && e < ep[lo].count, 4)) e = -1;
    }
    __device__ __forceinline__ const Sys &sys(int g) const { return S[g]; }
    __device__ __forceinline__ const EPView &eps(int g) const { return ep[g]; }
};

template <class P, class Src>
__device__ __forceinline__ void track_body(const Src &src, const XYCtl &C, const WorkList &wl) {
    using R = typename P::R;
    constexpr int BLOCK = P::BLOCK, NV = P::NV, MD = P::MD;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31;
    const SMat<MD, R, BLOCK> A{sm + tid};
    const SVec<R, BLOCK> ZC{sm + MD * (MD + 2) * BLOCK + tid};   // evaluation point / iterate
    const SVec<R, BLOCK> W1{sm + MD * MD * BLOCK + tid};          // solve output / residual:
                                                                  // the right-hand-side columns
    const int64_t gtid = (int64_t)blockIdx.x * BLOCK + tid;
    const int64_t nth = wl.state_threads;
    cx<R> *st = reinterpret_cast<cx<R> *>(wl.state);
    const GVec<R> Z0{st + (0 * NV) * nth + gtid, nth};       // accepted point
    const GVec<R> K1{st + (1 * NV) * nth + gtid, nth};       // dz/dt at Z0
    const GVec<R> AC{st + (2 * NV) * nth + gtid, nth};       // RK4 sum; next K1 in correction
    const GVec<R> CK{st + (3 * NV) * nth + gtid, nth};       // FP32 pass: hand-off checkpoint
    const int64_t total = src.total();

    // short lists: at most `lanes` paths per warp, so that the list spreads over every SM
    // instead of filling the first warps 32 at a time (FP64 continuation of a few
    // thousand hand-offs would otherwise run on a third of the SMs)
    int lanes = 32;
    if (C.sparse) {
        const int64_t warps = (int64_t)gridDim.x * (BLOCK / 32);
        const int64_t per = (total + warps - 1) / warps;
        lanes = per < 1 ? 1 : (per > 32 ? 32 : (int)per);
    }
    int64_t e = (lane >= lanes) ? -2 : -1;   // entry index; -1 idle, -2 drained
    int g = 0;                                // instance of the entry (batches)
    double t = 0.0, h = 0.0, hacc = 0.0;
    double tck = 0.0, hck = 0.0;   // checkpoint: the last clean accepted point with 1 - t < CRAWL_ZONE
    bool have_ck = false;
    int clean = 0;                 // accepted steps in a row without a reject between them
    double tmark = 0.0;   // 1 - t recorded every CRAWL_STEPS accepted steps near t = 1
    int since = 0;
    int status = 0, run = 0, rejects = 0, attempts = 0, steps = 0, solves = 0, newton = 0;
    bool need_k1 = false;
    bool far = false;      // heading out: steps capped at KAPPA_FAR (1 - t)
    double zlast = 0.0;    // ||z||_inf at the last accepted point

    for (;;) {
        // ---- hand new entries to idle lanes
        const bool idle = (e == -1);
        const unsigned need = __ballot_sync(0xffffffffu, idle);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(wl.queue, (unsigned long long)__popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (idle) {
                const int64_t i = (int64_t)base + __popc(need & ((1u << lane) - 1u));
                if (i < total) src.take(i, g, e);   // -1 (skipped) if the debug build rejects it
                if (i >= total) {
                    e = -2;
                } else if (e >= 0) {
                    const EPView &ep = src.eps(g);
                    status = NPHC_PATH_RUNNING;
                    run = 0;
                    rejects = 0;
                    attempts = 0;
                    have_ck = false;
                    clean = 0;
                    if (C.resume) {
                        P::load(ep, e, Z0);
                        t = ep.t[e];
                        // restart with a step on the scale of 1 - t: the FP32 pass may have
                        // been crawling with a far smaller one
                        h = fmin(fmax(ep.h[e], 0.125 * (1.0 - t)), C.hmax);
                        h = fmax(h, C.hmin * 4.0);
                        steps = ep.steps[e];
                        solves = ep.solves[e];
                        newton = ep.newton[e];
                        need_k1 = true;
                    } else {
                        P::start(src.sys(g), ep.path[e], Z0, K1);
                        t = 0.0;
                        h = C.h0;
                        steps = C.accumulate ? ep.steps[e] : 0;
                        solves = C.accumulate ? ep.solves[e] : 0;
                        newton = C.accumulate ? ep.newton[e] : 0;
                        need_k1 = false;
                    }
                    hacc = h;
                    tmark = 1.0 - t;
                    since = 0;
                    far = false;
                    zlast = 0.0;
                }
            }
        }
        if (__all_sync(0xffffffffu, e < 0)) break;
        const bool act = (e >= 0);

        // ---- one step: phase 0 = a resumed point is first pulled onto this precision's
        // path (one Newton correction at the same t) and its dz/dt taken from the same
        // solve (only when some lane needs it), phases 1..3 = RK4 stages 2..4, phases
        // 4.. = Newton corrector iterations at t + h
        if (far && h > KAPPA_FAR * (1.0 - t)) h = KAPPA_FAR * (1.0 - t);
        double hh = h, t1 = t + h;
        if (t1 >= C.t_end) {
            t1 = C.t_end;
            hh = C.t_end - t;
        }
        const R hr = (R)hh;
        bool go = act && !need_k1;
        bool conv = false, bad = false;
        R zpn = R(0);
        R kstep = R(0);   // the largest condition estimate of this attempt's solves
        const int ph0 = __any_sync(0xffffffffu, act && need_k1) ? 0 : 1;
        const int nph = 4 + C.max_newton;
#pragma unroll 1
        for (int ph = ph0; ph < nph; ph++) {
            const bool corr = ph >= 4 || ph == 0;   // warp-uniform: residual + two solutions
            if (ph >= 4 && __all_sync(0xffffffffu, !go || conv || bad)) break;
            // participating lanes and the evaluation time of this phase
            bool w;
            double te;
            if (ph == 0) {
                w = act && need_k1;
                te = t;
            } else if (!corr) {
                w = go;
                te = (ph == 3) ? t1 : t + 0.5 * hh;
            } else {
                w = go && !conv && !bad;
                te = t1;
            }
            if (w && ph < 4) {
                // evaluation point of the phase: z0, z0 + h/2 k1, z0 + h/2 k2, z0 + h k3
                const R c = ph == 3 ? hr : R(0.5) * hr;
#pragma unroll 6
                for (int k = 0; k < NV; k++) {
                    if (ph == 0) {
                        ZC.set(k, Z0.get(k));
                    } else {
                        const cx<R> d = ph == 1 ? K1.get(k) : W1.get(k);
                        ZC.set(k, cadd(Z0.get(k), cscale(c, d)));
                    }
                }
            }
            const R tr = (R)te, omt = (R)(1.0 - te);
            if (corr) P::residual(src.sys(g), ZC, tr, omt, W1, w);
            R kest = R(0);
            const bool oks = P::solve(src.sys(g), A, ZC, tr, omt, corr, W1, W1, AC, w, &kest);
            if (!w) continue;
            solves++;
            kstep = fmax(kstep, kest);
            if (ph == 0) {
                // z0 += Newton correction at t; dz/dt from the second right-hand side
#pragma unroll 6
                for (int k = 0; k < NV; k++) {
                    Z0.set(k, cadd(ZC.get(k), W1.get(k)));
                    K1.set(k, AC.get(k));
                }
                newton++;
                need_k1 = false;
                if (!oks) status = C.handoff ? NPHC_PATH_HANDOFF : NPHC_PATH_NONFINITE;
            } else if (!corr) {
                bad = bad || !oks;
                if (ph == 1) {
#pragma unroll 6
                    for (int k = 0; k < NV; k++) AC.set(k, cadd(K1.get(k), cscale(R(2), W1.get(k))));
                } else if (ph == 2) {
#pragma unroll 6
                    for (int k = 0; k < NV; k++) AC.set(k, cadd(AC.get(k), cscale(R(2), W1.get(k))));
                } else {
                    // predicted point z0 + h/6 (k1 + 2 k2 + 2 k3 + k4)
                    R zz = R(0);
#pragma unroll 6
                    for (int k = 0; k < NV; k++) {
                        const cx<R> zp = cadd(Z0.get(k), cscale(hr / R(6), cadd(AC.get(k), W1.get(k))));
                        ZC.set(k, zp);
                        zz += cabs2(zp);
                    }
                    zpn = sqrt_r(zz) * P::NORM_SCALE;
                }
            } else {
                newton++;
                const R dn = vnorm2<NV, R>(W1) * P::NORM_SCALE;
                if (!oks || !finite_r(dn)) {
                    bad = true;
                } else if (ph == 4 && dn > (R)C.trust * (R(1) + zpn)) {
                    bad = true;
                } else {
                    R zz = R(0);
#pragma unroll 1
                    for (int k = 0; k < NV; k++) {
                        const cx<R> zn = cadd(ZC.get(k), W1.get(k));
                        ZC.set(k, zn);
                        zz += cabs2(zn);
                    }
                    if (dn <= (R)C.eps * (R(1) + sqrt_r(zz) * P::NORM_SCALE)) conv = true;
                }
            }
        }
        go = go && status == NPHC_PATH_RUNNING;

        // ---- FP32 pass: a converged step whose Schur systems' condition estimate exceeds
        // kappa (kappa = 0 outside the FP32 pass) is not taken; FP64 continues the path from
        // its last accepted point (or the end zone's clean checkpoint), where the estimate
        // was below kappa: the FP32 solve's relative error grows like the condition number
        // times 6e-8, and a step across an ill-conditioned stretch (two paths passing
        // close) can land on the neighbouring path.  A step that did not converge lands
        // nowhere: it is rejected and halved as usual, whatever its estimate (a poor
        // prediction far off the path can see a large one)
        if (go && conv && C.kappa > 0.0 && !((double)kstep <= C.kappa)) {
            status = NPHC_PATH_HANDOFF_COND;
            go = false;
        }

        // ---- accept or reject
        if (go) {
            attempts++;
            if (conv) {
#pragma unroll 6
                for (int k = 0; k < NV; k++) {
                    Z0.set(k, ZC.get(k));
                    K1.set(k, AC.get(k));
                }
                const R zi = P::norminf(ZC);
                clean = rejects == 0 ? clean + 1 : 1;
                t = t1;
                far = 1.0 - t < CRAWL_ZONE && (double)zi > FAR_NORM && (double)zi > FAR_GROWTH * zlast;
                zlast = (double)zi;
                steps++;
                rejects = 0;
                hacc = h;
                if (++run >= C.grow_after) {
                    run = 0;
                    h = fmin(2.0 * h, C.hmax);
                }
                if ((double)zi > C.rdiv)
                    // An FP32 point is accurate to ~eps relative, so a crossing by more
                    // than RDIV_BAND is one in FP64 too; FP32 leaves only the marginal
                    // crossings close to t = 1 to FP64
                    status = (C.handoff && 1.0 - t < NEAR_END &&
                              (double)zi <= C.rdiv * (1.0 + RDIV_BAND))
                                 ? NPHC_PATH_HANDOFF
                                 : NPHC_PATH_DIVERGED;
                else if (t >= C.t_end)
                    status = NPHC_PATH_REACHED;
                // FP32 pass: in the end zone keep the last clean point (accepted, with the
                // step before it accepted too); a path that the pass later hands off
                // resumes in FP64 from there, not from the point where FP32 precision ran
                // out, which can sit off the path.  A converged FP32 point in light-cone
                // coordinates is on its path to the corrector's tolerance; in (x, y) the
                // small light-cone coordinate of a far point was lost to cancellation, so
                // such points could look converged while off the path, and the checkpoint
                // then had to stay at the end zone's entry.
                if (C.handoff && (clean >= 2 || !have_ck) && status == NPHC_PATH_RUNNING &&
                    1.0 - t < CRAWL_ZONE) {
#pragma unroll 6
                    for (int k = 0; k < NV; k++) CK.set(k, Z0.get(k));
                    tck = t;
                    hck = hacc;
                    have_ck = true;
                }
                // crawl test near t = 1: 1 - t must at least halve every CRAWL_STEPS
                // accepted steps (paths to nonsingular endpoints finish in a few steps;
                // a crawl means a singular endpoint, infinity, or precision exhausted)
                if (status == NPHC_PATH_RUNNING && C.crawl_steps > 0 && 1.0 - t < CRAWL_ZONE) {
                    if (++since >= C.crawl_steps) {
                        if (1.0 - t > 0.5 * tmark)
                            status = C.handoff ? NPHC_PATH_HANDOFF : NPHC_PATH_MIN_STEP;
                        tmark = 1.0 - t;
                        since = 0;
                    }
                } else {
                    tmark = 1.0 - t;
                    since = 0;
                }
            } else {
                run = 0;
                rejects++;
                h *= 0.5;
                if (h < C.hmin)
                    status = C.handoff ? NPHC_PATH_HANDOFF : NPHC_PATH_MIN_STEP;
                else if (C.handoff && rejects >= 10)
                    status = NPHC_PATH_HANDOFF;
            }
            if (status == NPHC_PATH_RUNNING && attempts >= C.max_steps)
                status = C.handoff ? NPHC_PATH_HANDOFF : NPHC_PATH_STEP_BUDGET;
        }
        if (act && status != NPHC_PATH_RUNNING) {
            const EPView &ep = src.eps(g);
            const bool handed = status == NPHC_PATH_HANDOFF || status == NPHC_PATH_HANDOFF_COND;
            const bool from_ck = handed && have_ck;
            if (from_ck)
                P::store(ep, e, CK);
            else
                P::store(ep, e, Z0);
            ep.t[e] = from_ck ? tck : t;
            ep.h[e] = from_ck ? hck : (handed ? hacc : h);
            ep.status[e] = status;
            ep.steps[e] = steps;
            ep.solves[e] = solves;
            ep.newton[e] = newton;
            e = -1;
        }
    }
}

template <int M, class R, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    xy_track_kernel(const __grid_constant__ XYSys S, const __grid_constant__ XYCtl C,
                    const EPView ep, const WorkList wl) {
    track_body<XYProblem<M, R, BLOCK>>(SingleSrc<XYSys>{S, ep, wl}, C, wl);
}

// The FP32 pass of a batch: every path of every instance of one ring size in one
// persistent launch, pulled from one queue (BatchSrc).
template <int M, class R, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    xy_track_batch_kernel(const XYSys *__restrict__ sys, const EPView *__restrict__ eps,
                          const int64_t *__restrict__ off, int n,
                          const __grid_constant__ XYCtl C, const WorkList wl) {
    track_body<XYProblem<M, R, BLOCK>>(BatchSrc<XYSys>{sys, eps, off, n}, C, wl);
}
