// xy_track.cuh -- path tracker for the XY-ring total-degree homotopy
// (section "Numerical Polynomial Homotopy Continuation Method": H = gamma (1-t) Q + t P,
// Q_i = z_i^2 - 1, start points z_i = +-1, tracked from t = 0 to t = 1 with a
// predictor and Newton's corrector).
//
// Layout: one path per thread; a persistent grid pulls paths from a device work
// counter (warp-aggregated atomics) until the list is drained.  The warp runs its 32
// paths in lockstep through the same phases -- three RK4 stage solves, then up to
// max_newton corrector solves -- so the heavy solve is never divergent; lanes whose
// path has finished take the next one at the step boundary.  Per-path state (point,
// derivative, RK4 accumulator, evaluation point, solve output: five vectors of 2M
// complex) lives in shared memory, interleaved by thread; the M x M Schur matrix of
// each solve lives in registers (xy_solve.cuh).
//
// Predictor: classical RK4 on dz/dt = -H_z^-1 H_t.  The derivative at the start of a
// step is taken from the previous step's last corrector solve (second right-hand
// side, same factorisation), and at t = 0 it is known in closed form
// (H_z = 2 gamma diag(z), H_t = P(z)), so each step costs 3 stage solves.
// Corrector: Newton at t + h; in FP32 its residual is evaluated with compensated sums
// (xy_residual_ff), in FP64 directly.  A step is accepted when ||dz|| <= eps (1 + ||z||)
// within max_newton iterations, and rejected when the first correction exceeds
// trust (1 + ||z||).  Step size doubles after grow_after consecutive accepts and halves
// on a reject; the final step lands exactly on t = 1.
//
// FP32 pass (ctl.handoff = 1): a path whose ||z||_inf exceeds rdiv_soft is declared
// diverged when its growth exponent d ln||z|| / d ln(1/(1-t)) over the last step
// exceeds rho_div (paths at infinity grow like (1-t)^-rho); otherwise, and on a step
// size underflow, ten consecutive rejects or the step budget, it is handed to FP64
// (NPHC_PATH_HANDOFF) with its (z, t, h).
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

template <int M, class R, int BLOCK>
__device__ __forceinline__ R tvec_norm2(const TVec<R, BLOCK> &v) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 2 * M; i++) s += cabs2(v.get(i));
    return sqrt_r(s);
}

template <int M, class R, int BLOCK>
__device__ __forceinline__ R tvec_norminf(const TVec<R, BLOCK> &v) {
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 2 * M; i++) s = fmax(s, sqrt_r(cabs2(v.get(i))));
    return s;
}

template <int M, class R, bool FF, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    xy_track_kernel(const __grid_constant__ XYSys S, const __grid_constant__ XYCtl C,
                    const EPView ep, const WorkList wl) {
    constexpr int NV = 4 * M;   // reals per vector
    extern __shared__ __align__(16) unsigned char smraw[];
    R *sm = reinterpret_cast<R *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31;
    const TVec<R, BLOCK> Z0{sm + 0 * NV * BLOCK + tid};   // accepted point
    const TVec<R, BLOCK> K1{sm + 1 * NV * BLOCK + tid};   // dz/dt at Z0
    const TVec<R, BLOCK> AC{sm + 2 * NV * BLOCK + tid};   // RK4 sum; next K1 during correction
    const TVec<R, BLOCK> ZC{sm + 3 * NV * BLOCK + tid};   // evaluation point / Newton iterate
    const TVec<R, BLOCK> W1{sm + 4 * NV * BLOCK + tid};   // solve output / residual
    const R *J = JSel<R>::get(S);
    const cx<R> gam = cx<R>{(R)S.gre, (R)S.gim};
    const int64_t total = worklist_size(wl, ep.count);
    const int64_t cnt = ep.count;

    int64_t e = -1;   // entry index; -1 idle, -2 list drained
    double t = 0.0, h = 0.0, hacc = 0.0, tprev = 0.0;
    R zprev = R(1);
    int status = 0, run = 0, rejects = 0, attempts = 0, steps = 0, solves = 0, newton = 0;
    bool need_k1 = false;

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
                if (i < total) {
                    e = worklist_entry(wl, i);
                    const int64_t p = ep.path[e];
                    status = NPHC_PATH_RUNNING;
                    run = 0;
                    rejects = 0;
                    attempts = 0;
                    if (C.resume) {
#pragma unroll
                        for (int k = 0; k < 2 * M; k++)
                            Z0.set(k, cx<R>{(R)ep.z_re[k * cnt + e], (R)ep.z_im[k * cnt + e]});
                        t = ep.t[e];
                        h = fmax(ep.h[e], C.hmin * 4.0);
                        steps = ep.steps[e];
                        solves = ep.solves[e];
                        newton = ep.newton[e];
                        need_k1 = true;
                    } else {
                        // start point and its derivative: at t = 0, H_z = 2 gamma diag(z)
                        // and H_t = P(z), so dz_i/dt = -P_i(z) / (2 gamma z_i)
                        cx<R> x[M], y[M];
#pragma unroll
                        for (int k = 0; k < M; k++) {
                            x[k] = cx<R>{((p >> k) & 1) ? R(-1) : R(1), R(0)};
                            y[k] = cx<R>{((p >> (M + k)) & 1) ? R(-1) : R(1), R(0)};
                            Z0.set(k, x[k]);
                            Z0.set(M + k, y[k]);
                        }
                        const cx<R> ig = crecip(gam);
#pragma unroll
                        for (int k = 0; k < M; k++) {
                            cx<R> u, w, rf, rg;
                            xy_minus_ht<M, R>(J, x, y, k, gam, u, w, rf, rg);
                            // rf = -H_t row = -P_k (Q_k = 0 at a start point)
                            K1.set(k, cscale(R(0.5) * x[k].re, cmul(ig, rf)));
                            K1.set(M + k, cscale(R(0.5) * y[k].re, cmul(ig, rg)));
                        }
                        t = 0.0;
                        h = C.h0;
                        steps = C.accumulate ? ep.steps[e] : 0;
                        solves = C.accumulate ? ep.solves[e] : 0;
                        newton = C.accumulate ? ep.newton[e] : 0;
                        need_k1 = false;
                    }
                    hacc = h;
                    tprev = t;
                    zprev = tvec_norminf<M, R, BLOCK>(Z0);
                } else {
                    e = -2;
                }
            }
        }
        if (__all_sync(0xffffffffu, e < 0)) break;
        const bool act = (e >= 0);

        // ---- resumed paths need dz/dt at their current point
        if (__any_sync(0xffffffffu, act && need_k1)) {
            const bool w = act && need_k1;
            if (w) {
#pragma unroll
                for (int k = 0; k < 2 * M; k++) ZC.set(k, Z0.get(k));
            }
            const bool okk = xy_solve<M, R, 1, BLOCK>(J, ZC, t, gam, W1, W1, W1, w);
            if (w) {
                solves++;
#pragma unroll
                for (int k = 0; k < 2 * M; k++) K1.set(k, W1.get(k));
                need_k1 = false;
                if (!okk) status = C.handoff ? NPHC_PATH_HANDOFF : NPHC_PATH_NONFINITE;
            }
        }
        const bool go = act && status == NPHC_PATH_RUNNING;

        // ---- RK4 predictor: stages 2..4 (stage 1 is K1)
        double hh = h, t1 = t + h;
        if (t1 >= 1.0) {
            t1 = 1.0;
            hh = 1.0 - t;
        }
        const R hr = (R)hh;
        bool okp = true;
        if (go) {
#pragma unroll
            for (int k = 0; k < 2 * M; k++) ZC.set(k, cadd(Z0.get(k), cscale(R(0.5) * hr, K1.get(k))));
        }
        okp &= xy_solve<M, R, 1, BLOCK>(J, ZC, t + 0.5 * hh, gam, W1, W1, W1, go);
        if (go) {
#pragma unroll
            for (int k = 0; k < 2 * M; k++) {
                const cx<R> d = W1.get(k);
                AC.set(k, cadd(K1.get(k), cscale(R(2), d)));
                ZC.set(k, cadd(Z0.get(k), cscale(R(0.5) * hr, d)));
            }
        }
        okp &= xy_solve<M, R, 1, BLOCK>(J, ZC, t + 0.5 * hh, gam, W1, W1, W1, go);
        if (go) {
#pragma unroll
            for (int k = 0; k < 2 * M; k++) {
                const cx<R> d = W1.get(k);
                AC.set(k, cadd(AC.get(k), cscale(R(2), d)));
                ZC.set(k, cadd(Z0.get(k), cscale(hr, d)));
            }
        }
        okp &= xy_solve<M, R, 1, BLOCK>(J, ZC, t1, gam, W1, W1, W1, go);
        if (go) {
            solves += 3;
#pragma unroll
            for (int k = 0; k < 2 * M; k++) {
                const cx<R> acc = cadd(AC.get(k), W1.get(k));
                ZC.set(k, cadd(Z0.get(k), cscale(hr / R(6), acc)));
            }
        }

        // ---- Newton corrector at t1
        bool conv = false, bad = !go || !okp;
        const R zpn = go ? tvec_norm2<M, R, BLOCK>(ZC) : R(0);
        for (int it = 0; it < C.max_newton; it++) {
            if (__all_sync(0xffffffffu, conv || bad)) break;
            const bool w = !conv && !bad;
            if constexpr (FF)
                xy_residual_ff<M, BLOCK>(J, ZC, t1, gam, W1, w);
            else
                xy_residual_plain<M, R, BLOCK>(J, ZC, t1, gam, W1, w);
            const bool oks = xy_solve<M, R, 2, BLOCK>(J, ZC, t1, gam, W1, W1, AC, w);
            if (w) {
                solves++;
                newton++;
                const R dn = tvec_norm2<M, R, BLOCK>(W1);
                if (!oks || !finite_r(dn)) {
                    bad = true;
                } else if (it == 0 && dn > (R)C.trust * (R(1) + zpn)) {
                    bad = true;
                } else {
#pragma unroll
                    for (int k = 0; k < 2 * M; k++) ZC.set(k, cadd(ZC.get(k), W1.get(k)));
                    if (dn <= (R)C.eps * (R(1) + tvec_norm2<M, R, BLOCK>(ZC))) conv = true;
                }
            }
        }

        // ---- accept or reject
        if (go) {
            attempts++;
            if (conv) {
#pragma unroll
                for (int k = 0; k < 2 * M; k++) {
                    Z0.set(k, ZC.get(k));
                    K1.set(k, AC.get(k));
                }
                t = t1;
                steps++;
                rejects = 0;
                hacc = h;
                if (++run >= C.grow_after) {
                    run = 0;
                    h = fmin(2.0 * h, C.hmax);
                }
                const R zi = tvec_norminf<M, R, BLOCK>(Z0);
                if (t >= 1.0) {
                    status = NPHC_PATH_REACHED;
                } else if ((double)zi > C.rdiv) {
                    status = NPHC_PATH_DIVERGED;
                } else if (C.handoff && (double)zi > C.rdiv_soft) {
                    double rho = 0.0;
                    if (tprev < t && zprev > R(0))
                        rho = log((double)zi / (double)zprev) / log((1.0 - tprev) / (1.0 - t));
                    status = rho > C.rho_div ? NPHC_PATH_DIVERGED : NPHC_PATH_HANDOFF;
                }
                zprev = zi;
                tprev = t;
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
#pragma unroll
            for (int k = 0; k < 2 * M; k++) {
                const cx<R> v = Z0.get(k);
                ep.z_re[k * cnt + e] = (double)v.re;
                ep.z_im[k * cnt + e] = (double)v.im;
            }
            ep.t[e] = t;
            ep.h[e] = status == NPHC_PATH_HANDOFF ? hacc : h;
            ep.status[e] = status;
            ep.steps[e] = steps;
            ep.solves[e] = solves;
            ep.newton[e] = newton;
            e = -1;
        }
    }
}
