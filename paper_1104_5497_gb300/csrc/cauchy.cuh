// cauchy.cuh -- the Cauchy endgame for endpoints where several paths meet (singular
// solutions) or where a path goes to infinity slowly.  The paper reports that such
// endpoints are handled in practice; the method here is the Cauchy endgame of the
// homotopy continuation literature (Morgan, Sommese and Wampler, 1991).
//
// Near t = 1 a path is a Puiseux series in s = (1 - t)^(1/c), c its cycle number.  With
// 1 - t = e^w the path is continued around |1 - t| = r (w = ln r + i theta): it closes
// after exactly c turns, and the mean of z over the c turns (K equally spaced samples
// per turn, the trapezoid rule for Cauchy's integral in s) is its value at t = 1.  The
// radius shrinks by `ratio` (a radial leg along real t) until two estimates from
// successive radii agree and the estimate solves P (the solution tolerance); radii whose
// turns do not close within max_cycle, or where a step fails, are skipped from the point
// where the path reached them.  Agreement without a solution is either a path to
// infinity (the mean is the constant Laurent coefficient, the same at every radius, while
// the distance from a radius's start point to it grows like a pole's, by at least
// ratio^(-1/c)) or turns that also enclose the branch point of two paths with distinct
// endpoints (they average them): the latter go on to smaller radii.
//
// Complex t without a complex-t solver: for t off the real axis,
//   H(z, t) = gamma (1-t) Q + t P = (t / s) [gamma' (1-s) Q + s P],
// with rho = gamma (1-t)/t, s = |gamma| / (|gamma| + |rho|) in (0, 1) and
// gamma' = rho |gamma| / |rho|, i.e. the real-t homotopy of the trackers at time s with
// gamma' in place of gamma has the same zeros and the same Newton corrections.  On the
// path, H_t = P/(1-t) and the real-t system's d = -H_z'^-1 H_t' gives
//   dz/dw = -(s (1-s) / t) d,
// so the predictor uses the trackers' solve too (same integral curve; off the path the
// two vector fields differ by terms in H, which the corrector removes).
//
// cauchy_body: layout as the per-thread tracker (xy_track.cuh), for any tracker policy
// (the generic quadratic systems use it): one path per thread, lockstep phases of a step
// (ph 0: Newton at the current point and dz/dw, for a point just taken over; 1..3: RK4
// stages; 4..: corrector), the matrix and the evaluation point in shared memory (the
// solve output shares the right-hand-side columns), six state vectors in global scratch.  The XY ring runs the same endgame with one path per warp
// (cauchy_warp.cuh).
#pragma once

#include "xy_track.cuh"

#define NPHC_TWO_PI 6.283185307179586

// The real-t homotopy equivalent to complex t = 1 - ew: time s, 1 - s, gamma', and the
// factor cw that turns its d into dz/dw.
struct EffPoint {
    double s, omt;
    cx<double> g, cw;
};

__device__ __forceinline__ EffPoint eff_point(cx<double> ew, cx<double> gam, double ag) {
    const cx<double> t = cx<double>{1.0 - ew.re, -ew.im};
    const cx<double> it = crecip(t);
    const cx<double> rho = cmul(cmul(gam, ew), it);
    const double ar = sqrt(cabs2(rho));
    EffPoint p;
    p.s = ag / (ag + ar);
    p.omt = ar / (ag + ar);
    p.g = cscale(ag / ar, rho);
    p.cw = cscale(-p.s * p.omt, it);
    return p;
}

// e^w at the point v in [0, 1] of a sample interval: on a turn w = lr + i 2 pi (j + v) / K,
// on a radial leg w = lr + v ln(ratio).
__device__ __forceinline__ cx<double> eg_ew(double lr, bool radial, int j, int K, double lnratio,
                                            double v) {
    if (radial) return cx<double>{exp(lr + v * lnratio), 0.0};
    double sn, cs;
    sincos(NPHC_TWO_PI * ((double)j + v) / (double)K, &sn, &cs);
    const double er = exp(lr);
    return cx<double>{er * cs, er * sn};
}

template <class V>
__device__ __forceinline__ double eg_norm(const V &a, int n) {
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < n; i++) s += cabs2(a.get(i));
    return sqrt(s);
}

template <class P>
__device__ __forceinline__ void cauchy_body(const typename P::Sys &S, const EGCtl &C,
                                            const EPView &ep, const WorkList &wl,
                                            int32_t *__restrict__ cyc_out,
                                            int32_t *__restrict__ eg_out) {
    using R = double;
    constexpr int BLOCK = P::BLOCK, NV = P::NV, MD = P::MD;
    extern __shared__ __align__(16) unsigned char smraw[];
    cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);
    const int tid = threadIdx.x, lane = tid & 31;
    const SMat<MD, R, BLOCK> A{sm + tid};
    const SVec<R, BLOCK> ZC{sm + MD * (MD + 2) * BLOCK + tid};
    const SVec<R, BLOCK> W1{sm + MD * MD * BLOCK + tid};   // the right-hand-side columns
    const int64_t gtid = (int64_t)blockIdx.x * BLOCK + tid;
    const int64_t nth = wl.state_threads;
    cx<R> *st = reinterpret_cast<cx<R> *>(wl.state);
    const GVec<R> Z0{st + (0 * NV) * nth + gtid, nth};   // accepted point
    const GVec<R> K1{st + (1 * NV) * nth + gtid, nth};   // dz/dw at Z0
    const GVec<R> AC{st + (2 * NV) * nth + gtid, nth};   // RK4 sum; the corrector's d
    const GVec<R> ZS{st + (3 * NV) * nth + gtid, nth};   // where the turns at this radius began
    const GVec<R> SU{st + (4 * NV) * nth + gtid, nth};   // sum of this radius's samples
    const GVec<R> PV{st + (5 * NV) * nth + gtid, nth};   // last estimate
    const int64_t total = worklist_size(wl, ep.count);
    const int64_t cnt = ep.count;
    const cx<R> gam = cx<R>{S.gre, S.gim};
    const double ag = sqrt(cabs2(gam));
    const int K = C.samples;

    int64_t e = -1;   // entry index; -1 idle, -2 drained
    int status = 0, k = 0, j = 0, turn = 1, run = 0, attempts = 0, cyc = 0, solves = 0;
    int last_fail = NPHC_EG_NOT_CLOSED;
    bool radial = false, have_prev = false, need_k1 = false;
    double v = 0.0, h = 1.0, d_prev = 0.0;

    for (;;) {
        // ---- hand new entries to idle lanes (again while one drew an entry whose tracking
        // to 1 - r0 failed: -2 must mean drained before the exit test below)
        for (;;) {
            const bool idle = (e == -1);
            const unsigned need = __ballot_sync(0xffffffffu, idle);
            if (!need) break;
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(wl.queue, (unsigned long long)__popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (idle) {
                const int64_t i = (int64_t)base + __popc(need & ((1u << lane) - 1u));
                if (i < total) e = worklist_entry(wl, i, ep.count);   // -1: rejected (debug)
                if (i < total && e >= 0) {
                    const int ts = ep.status[e];
                    if (ts != NPHC_PATH_REACHED) {   // tracking to 1 - r0 did not get there
                        cyc_out[e] = 0;
                        eg_out[e] = ts == NPHC_PATH_DIVERGED ? NPHC_EG_DIVERGED : NPHC_EG_TRACK_FAILED;
                        e = -1;
                    } else {
#pragma unroll 1
                        for (int q = 0; q < NV; q++) {
                            const cx<R> z = cx<R>{ep.z_re[q * cnt + e], ep.z_im[q * cnt + e]};
                            Z0.set(q, z);
                            ZS.set(q, z);
                            SU.set(q, z);   // sample 0 of the first turn
                        }
                        status = 0;
                        k = 0;
                        j = 0;
                        turn = 1;
                        run = 0;
                        attempts = 0;
                        cyc = 0;
                        solves = 0;
                        last_fail = NPHC_EG_NOT_CLOSED;
                        radial = false;
                        have_prev = false;
                        need_k1 = true;
                        v = 0.0;
                        h = 1.0;
                        d_prev = 0.0;
                    }
                } else {
                    e = -2;
                }
            }
        }
        if (__all_sync(0xffffffffu, e < 0)) break;
        const bool act = (e >= 0);

        // ---- one step attempt across part of the current sample interval
        bool budget = act && !need_k1 && attempts >= C.max_attempts;
        bool go = act && !need_k1 && !budget;
        double hh = fmin(h, 1.0 - v), v1 = v + hh;
        if (v1 >= 1.0) {
            v1 = 1.0;
            hh = 1.0 - v;
        }
        const double lrk = C.lr0 + k * C.lnratio;
        const double lr = radial ? lrk - C.lnratio : lrk;
        const cx<R> dw = radial ? cx<R>{C.lnratio, 0.0} : cx<R>{0.0, NPHC_TWO_PI / (double)K};
        const cx<R> hd = cscale(hh, dw);
        cx<R> cwm = cx<R>{0.0, 0.0}, cwe = cwm;   // dz/dw factors at v + hh/2 and at v1
        bool conv = false, bad = false;
        R zpn = R(0);
        const int ph0 = __any_sync(0xffffffffu, act && need_k1) ? 0 : 1;
        const int nph = 4 + C.max_newton;
#pragma unroll 1
        for (int ph = ph0; ph < nph; ph++) {
            const bool corr = ph >= 4 || ph == 0;
            if (ph >= 4 && __all_sync(0xffffffffu, !go || conv || bad)) break;
            bool w;
            if (ph == 0) w = act && need_k1;
            else if (!corr) w = go;
            else w = go && !conv && !bad;
            // the phase's evaluation time: v (ph 0), v + hh/2 (RK4 stages 2, 3), v1
            const double ve = ph == 0 ? v : (ph == 1 || ph == 2) ? v + 0.5 * hh : v1;
            const EffPoint pe =
                eff_point(act ? eg_ew(lr, radial, j, K, C.lnratio, ve) : cx<R>{0.5, 0.0}, gam, ag);
            if (ph == 1) cwm = pe.cw;
            else if (ph >= 3) cwe = pe.cw;
            if (w && ph < 4) {
                // evaluation point: z0, z0 + hd/2 k1, z0 + hd/2 k2, z0 + hd k3 (k = dz/dw)
#pragma unroll 1
                for (int q = 0; q < NV; q++) {
                    if (ph == 0) {
                        ZC.set(q, Z0.get(q));
                    } else {
                        const cx<R> d = ph == 1 ? K1.get(q) : cmul(cwm, W1.get(q));
                        const cx<R> c = ph == 3 ? hd : cscale(0.5, hd);
                        ZC.set(q, cadd(Z0.get(q), cmul(c, d)));
                    }
                }
            }
            if (corr) P::residual_g(S, ZC, pe.s, pe.omt, pe.g, W1, w);
            const bool oks = P::solve_g(S, A, ZC, pe.s, pe.omt, pe.g, corr, W1, W1, AC, w);
            if (!w) continue;
            solves++;
            if (ph == 0) {
#pragma unroll 1
                for (int q = 0; q < NV; q++) {
                    Z0.set(q, cadd(ZC.get(q), W1.get(q)));
                    K1.set(q, cmul(pe.cw, AC.get(q)));
                }
                need_k1 = false;
                if (!oks) status = NPHC_EG_TRACK_FAILED;
            } else if (!corr) {
                bad = bad || !oks;
                if (ph == 1) {
#pragma unroll 1
                    for (int q = 0; q < NV; q++)
                        AC.set(q, cadd(K1.get(q), cscale(R(2), cmul(cwm, W1.get(q)))));
                } else if (ph == 2) {
#pragma unroll 1
                    for (int q = 0; q < NV; q++)
                        AC.set(q, cadd(AC.get(q), cscale(R(2), cmul(cwm, W1.get(q)))));
                } else {
                    // predicted point z0 + hd/6 (k1 + 2 k2 + 2 k3 + k4)
                    const cx<R> c6 = cscale(R(1) / R(6), hd);
                    R zz = R(0);
#pragma unroll 1
                    for (int q = 0; q < NV; q++) {
                        const cx<R> k4 = cmul(cwe, W1.get(q));
                        const cx<R> zp = cadd(Z0.get(q), cmul(c6, cadd(AC.get(q), k4)));
                        ZC.set(q, zp);
                        zz += cabs2(zp);
                    }
                    zpn = sqrt(zz);
                }
            } else {
                const R dn = eg_norm(W1, NV);
                if (!oks || !isfinite(dn)) {
                    bad = true;
                } else if (ph == 4 && dn > C.trust * (R(1) + zpn)) {
                    bad = true;
                } else {
                    R zz = R(0);
#pragma unroll 1
                    for (int q = 0; q < NV; q++) {
                        const cx<R> zn = cadd(ZC.get(q), W1.get(q));
                        ZC.set(q, zn);
                        zz += cabs2(zn);
                    }
                    if (dn <= C.eps * (R(1) + sqrt(zz))) conv = true;
                }
            }
        }
        go = go && status == 0;

        // ---- accept or reject, then the events of the interval, turn and radius
        bool fail_step = budget;
        bool restart = false;   // back to ZS, on to the next radius
        if (go) {
            attempts++;
            if (conv) {
                R zi = R(0);
#pragma unroll 1
                for (int q = 0; q < NV; q++) {
                    const cx<R> z = ZC.get(q);
                    Z0.set(q, z);
                    K1.set(q, cmul(cwe, AC.get(q)));
                    zi = fmax(zi, sqrt(cabs2(z)));
                }
                v = v1;
                if (++run >= C.grow_after) {
                    run = 0;
                    h = fmin(2.0 * h, 1.0);
                }
                if (zi > C.rdiv) {
                    status = NPHC_EG_DIVERGED;
                } else if (v >= 1.0) {   // end of the sample interval
                    v = 0.0;
                    if (radial) {        // reached radius k: its turns start here
                        radial = false;
#pragma unroll 1
                        for (int q = 0; q < NV; q++) {
                            const cx<R> z = Z0.get(q);
                            ZS.set(q, z);
                            SU.set(q, z);
                        }
                        j = 0;
                        turn = 1;
                    } else if (++j < K) {
#pragma unroll 1
                        for (int q = 0; q < NV; q++) SU.set(q, cadd(SU.get(q), Z0.get(q)));
                    } else {             // end of a turn
                        double dd = 0.0;
#pragma unroll 1
                        for (int q = 0; q < NV; q++) dd += cabs2(csub(Z0.get(q), ZS.get(q)));
                        if (sqrt(dd) <= C.tol_close * (1.0 + eg_norm(ZS, NV))) {
                            // closed after c = turn turns: the estimate at this radius
                            cyc = turn;
                            const double inv = 1.0 / (double)(turn * K);
                            double dz = 0.0, de = 0.0, ne = 0.0;
#pragma unroll 1
                            for (int q = 0; q < NV; q++) {
                                const cx<R> est = cscale(inv, SU.get(q));
                                dz += cabs2(csub(ZS.get(q), est));
                                de += cabs2(csub(est, PV.get(q)));
                                ne += cabs2(est);
                                PV.set(q, est);
                            }
                            const double d = sqrt(dz);
                            if (have_prev && sqrt(de) <= C.tol_conv * (1.0 + sqrt(ne))) {
                                // agreement: a solution of P is the endpoint; an estimate
                                // that is none, with the start point's distance growing as a
                                // pole's would, is a path to infinity; anything else means
                                // the turns also enclose another branch point (two sheets
                                // with distinct endpoints average): on to smaller radii
                                double zi = 0.0;
#pragma unroll 1
                                for (int q = 0; q < NV; q++) {
                                    const cx<R> est = PV.get(q);
                                    ZC.set(q, est);
                                    zi = fmax(zi, sqrt(cabs2(est)));
                                }
                                P::residual_g(S, ZC, 1.0, 0.0, gam, W1, true);   // W1 = -P(est)
                                double res = 0.0;
#pragma unroll 1
                                for (int q = 0; q < NV; q++) res = fmax(res, sqrt(cabs2(W1.get(q))));
                                if (res <= C.tol_res * (zi > 1.0 ? zi * zi : 1.0))
                                    status = NPHC_EG_CONVERGED;
                                else if (d > d_prev * C.grow_inf)
                                    status = NPHC_EG_AT_INFINITY;
                            }
                            if (status == 0) {
                                d_prev = d;
                                have_prev = true;
                                if (++k >= C.n_radii) status = NPHC_EG_NOT_CONVERGED;
                                else radial = true;
                            }
                        } else if (turn < C.max_cycle) {
                            turn++;
                            j = 0;
#pragma unroll 1
                            for (int q = 0; q < NV; q++) SU.set(q, cadd(SU.get(q), Z0.get(q)));
                        } else {
                            last_fail = NPHC_EG_NOT_CLOSED;
                            restart = true;
                        }
                    }
                }
            } else {
                run = 0;
                h *= 0.5;
                if (h < C.hmin) fail_step = true;
            }
        }
        if (fail_step) {
            if (radial) {
                status = NPHC_EG_TRACK_FAILED;
            } else {
                last_fail = NPHC_EG_TRACK_FAILED;
                restart = true;
            }
        }
        if (restart) {   // skip this radius from where the path reached it
#pragma unroll 1
            for (int q = 0; q < NV; q++) Z0.set(q, ZS.get(q));
            need_k1 = true;
            h = 1.0;
            run = 0;
            v = 0.0;
            have_prev = false;
            if (++k >= C.n_radii) status = last_fail;
            else radial = true;
        }
        if (act && status != 0) {
            const bool est = status == NPHC_EG_CONVERGED || status == NPHC_EG_NOT_CONVERGED;
#pragma unroll 1
            for (int q = 0; q < NV; q++) {
                const cx<R> z = est ? PV.get(q) : Z0.get(q);
                ep.z_re[q * cnt + e] = z.re;
                ep.z_im[q * cnt + e] = z.im;
            }
            cyc_out[e] = cyc;
            eg_out[e] = status;
            ep.solves[e] += solves;
            e = -1;
        }
    }
}
