// cauchy_warp.cuh -- the Cauchy endgame of cauchy.cuh for the XY ring with one path per
// warp: the FP64 tracker's warp-cooperative solve and residual (xy_track_warp.cuh) at the
// real-t equivalent of each complex t (eff_point), the turns, radii, restarts and
// acceptance rule of cauchy_body.  The endgame's lists are short (the paths that end
// singular or fail) and each path is a long chain of dependent FP64 solves, so the
// latency of one solve sets the time: sharing it over the lanes cuts that chain ~10x
// against one path per thread.  Control flow is uniform over the warp (every branch is
// on values broadcast from lane 0); lane i < 2M holds component i of the vectors.
#pragma once

#include "cauchy.cuh"
#include "xy_track_warp.cuh"

template <int M>
struct CauchyWarpLayout {
    static constexpr int NV = 2 * M;
    static constexpr int ZS = WarpLayout<M>::TOTAL;   // where the turns at this radius began
    static constexpr int SU = ZS + NV;                // sum of this radius's samples
    static constexpr int PV = SU + NV;                // last estimate
    static constexpr int TOTAL = PV + NV;
};

template <int M>
constexpr size_t cauchy_warp_smem_per_warp() {
    return sizeof(cx<double>) * (size_t)CauchyWarpLayout<M>::TOTAL;
}

template <int M, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
    xy_cauchy_warp_kernel(const __grid_constant__ XYSys S, const __grid_constant__ EGCtl C,
                          const EPView ep, const WorkList wl, int32_t *__restrict__ cyc_out,
                          int32_t *__restrict__ eg_out) {
    using L = WarpLayout<M>;
    using CL = CauchyWarpLayout<M>;
    constexpr int NV = 2 * M;
    extern __shared__ __align__(16) unsigned char wraw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const WarpPath<M> P{reinterpret_cast<cx<double> *>(wraw) + (size_t)wid * CL::TOTAL, lane};
    const double *J = S.Jd;
    const cx<double> gam = cx<double>{S.gre, S.gim};
    const double ag = sqrt(cabs2(gam));
    const int64_t total = worklist_size(wl, ep.count);
    const int64_t cnt = ep.count;
    const int K = C.samples;
    const int i = lane;   // vector component of this lane (i < NV)
    const bool vl = i < NV;
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(wl.queue, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= total) break;
        const int64_t e = worklist_entry(wl, (int64_t)q, ep.count);
        if (e < 0) continue;   // rejected by the debug build's check
        const int ts = ep.status[e];
        if (ts != NPHC_PATH_REACHED) {   // tracking to 1 - r0 did not get there
            if (lane == 0) {
                cyc_out[e] = 0;
                eg_out[e] = ts == NPHC_PATH_DIVERGED ? NPHC_EG_DIVERGED : NPHC_EG_TRACK_FAILED;
            }
            continue;
        }
        if (vl) {
            const cx<double> z = cx<double>{ep.z_re[i * cnt + e], ep.z_im[i * cnt + e]};
            P.at(L::Z0, i) = z;
            P.at(CL::ZS, i) = z;
            P.at(CL::SU, i) = z;   // sample 0 of the first turn
        }
        __syncwarp();
        int status = 0, k = 0, j = 0, turn = 1, run = 0, attempts = 0, cyc = 0, solves = 0;
        int last_fail = NPHC_EG_NOT_CLOSED;
        bool radial = false, have_prev = false, need_k1 = true;
        double v = 0.0, h = 1.0, d_prev = 0.0;
        while (status == 0) {
            const double lrk = C.lr0 + k * C.lnratio;
            const double lr = radial ? lrk - C.lnratio : lrk;
            if (need_k1) {   // Newton at the point just taken over, and dz/dw there
                const EffPoint pe = eff_point(eg_ew(lr, radial, j, K, C.lnratio, v), gam, ag);
                if (vl) P.at(L::ZC, i) = P.at(L::Z0, i);
                __syncwarp();
                warp_residual<M>(P, J, pe.s, pe.omt, pe.g);
                const bool ok = warp_solve<M>(P, J, pe.s, pe.omt, pe.g, true, L::AC);
                solves++;
                if (vl) {
                    P.at(L::Z0, i) = cadd(P.at(L::ZC, i), P.at(L::W1, i));
                    P.at(L::K1, i) = cmul(pe.cw, P.at(L::AC, i));
                }
                __syncwarp();
                need_k1 = false;
                if (!ok) status = NPHC_EG_TRACK_FAILED;
                continue;
            }
            bool fail_step = false, restart = false;
            if (attempts >= C.max_attempts) {
                fail_step = true;
            } else {
                attempts++;
                double hh = fmin(h, 1.0 - v), v1 = v + hh;
                if (v1 >= 1.0) {
                    v1 = 1.0;
                    hh = 1.0 - v;
                }
                const cx<double> dw =
                    radial ? cx<double>{C.lnratio, 0.0} : cx<double>{0.0, NPHC_TWO_PI / (double)K};
                const cx<double> hd = cscale(hh, dw);
                const cx<double> hd2 = cscale(0.5, hd);
                const EffPoint pm = eff_point(eg_ew(lr, radial, j, K, C.lnratio, v + 0.5 * hh), gam, ag);
                const EffPoint p1 = eff_point(eg_ew(lr, radial, j, K, C.lnratio, v1), gam, ag);
                bool bad = false, conv = false;
                // RK4 stages 2..4 on dz/dw (k = cw d of the solve at each stage point)
                if (vl) P.at(L::ZC, i) = cadd(P.at(L::Z0, i), cmul(hd2, P.at(L::K1, i)));
                __syncwarp();
                bad = !warp_solve<M>(P, J, pm.s, pm.omt, pm.g, false, L::AC) || bad;
                solves++;
                if (vl) {
                    const cx<double> k2 = cmul(pm.cw, P.at(L::W1, i));
                    P.at(L::AC, i) = cadd(P.at(L::K1, i), cscale(2.0, k2));
                    P.at(L::ZC, i) = cadd(P.at(L::Z0, i), cmul(hd2, k2));
                }
                __syncwarp();
                bad = !warp_solve<M>(P, J, pm.s, pm.omt, pm.g, false, L::AC) || bad;
                solves++;
                if (vl) {
                    const cx<double> k3 = cmul(pm.cw, P.at(L::W1, i));
                    P.at(L::AC, i) = cadd(P.at(L::AC, i), cscale(2.0, k3));
                    P.at(L::ZC, i) = cadd(P.at(L::Z0, i), cmul(hd, k3));
                }
                __syncwarp();
                bad = !warp_solve<M>(P, J, p1.s, p1.omt, p1.g, false, L::AC) || bad;
                solves++;
                double zz = 0.0;
                if (vl) {   // predicted point z0 + hd/6 (k1 + 2 k2 + 2 k3 + k4)
                    const cx<double> k4 = cmul(p1.cw, P.at(L::W1, i));
                    const cx<double> zp = cadd(P.at(L::Z0, i),
                                               cmul(cscale(1.0 / 6.0, hd), cadd(P.at(L::AC, i), k4)));
                    P.at(L::ZC, i) = zp;
                    zz = cabs2(zp);
                }
                const double zpn = sqrt(warp_sum(zz));
                __syncwarp();
                // Newton's corrector at v1
#pragma unroll 1
                for (int it = 0; it < C.max_newton && !bad; it++) {
                    warp_residual<M>(P, J, p1.s, p1.omt, p1.g);
                    const bool oks = warp_solve<M>(P, J, p1.s, p1.omt, p1.g, true, L::AC);
                    solves++;
                    const double dn = sqrt(warp_sum(vl ? cabs2(P.at(L::W1, i)) : 0.0));
                    if (!oks || !isfinite(dn) || (it == 0 && dn > C.trust * (1.0 + zpn))) {
                        bad = true;
                        break;
                    }
                    double z2 = 0.0;
                    if (vl) {
                        const cx<double> zn = cadd(P.at(L::ZC, i), P.at(L::W1, i));
                        P.at(L::ZC, i) = zn;
                        z2 = cabs2(zn);
                    }
                    z2 = warp_sum(z2);
                    __syncwarp();
                    if (dn <= C.eps * (1.0 + sqrt(z2))) {
                        conv = true;
                        break;
                    }
                }
                if (conv) {
                    double zi = 0.0;
                    if (vl) {
                        const cx<double> z = P.at(L::ZC, i);
                        P.at(L::Z0, i) = z;
                        P.at(L::K1, i) = cmul(p1.cw, P.at(L::AC, i));
                        zi = sqrt(cabs2(z));
                    }
                    zi = warp_max(zi);
                    __syncwarp();
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
                            if (vl) {
                                const cx<double> z = P.at(L::Z0, i);
                                P.at(CL::ZS, i) = z;
                                P.at(CL::SU, i) = z;
                            }
                            __syncwarp();
                            j = 0;
                            turn = 1;
                        } else if (++j < K) {
                            if (vl) P.at(CL::SU, i) = cadd(P.at(CL::SU, i), P.at(L::Z0, i));
                            __syncwarp();
                        } else {             // end of a turn
                            const double dd = sqrt(warp_sum(vl ? cabs2(csub(P.at(L::Z0, i), P.at(CL::ZS, i))) : 0.0));
                            const double nzs = sqrt(warp_sum(vl ? cabs2(P.at(CL::ZS, i)) : 0.0));
                            if (dd <= C.tol_close * (1.0 + nzs)) {
                                // closed after c = turn turns: the estimate at this radius
                                cyc = turn;
                                const double inv = 1.0 / (double)(turn * K);
                                double dz = 0.0, de = 0.0, ne = 0.0;
                                if (vl) {
                                    const cx<double> est = cscale(inv, P.at(CL::SU, i));
                                    dz = cabs2(csub(P.at(CL::ZS, i), est));
                                    de = cabs2(csub(est, P.at(CL::PV, i)));
                                    ne = cabs2(est);
                                    P.at(CL::PV, i) = est;
                                    P.at(L::ZC, i) = est;
                                }
                                const double d = sqrt(warp_sum(dz));
                                de = sqrt(warp_sum(de));
                                ne = sqrt(warp_sum(ne));
                                __syncwarp();
                                if (have_prev && de <= C.tol_conv * (1.0 + ne)) {
                                    // a solution of P is the endpoint; otherwise a pole
                                    // (growing distance) or an enclosed branch point of
                                    // two other sheets (on to smaller radii)
                                    warp_residual<M>(P, J, 1.0, 0.0, gam);   // W1 = -P(est)
                                    const double res = warp_max(vl ? sqrt(cabs2(P.at(L::W1, i))) : 0.0);
                                    const double zi2 = warp_max(vl ? sqrt(cabs2(P.at(L::ZC, i))) : 0.0);
                                    if (res <= C.tol_res * (zi2 > 1.0 ? zi2 * zi2 : 1.0))
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
                                if (vl) P.at(CL::SU, i) = cadd(P.at(CL::SU, i), P.at(L::Z0, i));
                                __syncwarp();
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
                if (vl) P.at(L::Z0, i) = P.at(CL::ZS, i);
                __syncwarp();
                need_k1 = true;
                h = 1.0;
                run = 0;
                v = 0.0;
                have_prev = false;
                if (++k >= C.n_radii) status = last_fail;
                else radial = true;
            }
        }
        const bool est = status == NPHC_EG_CONVERGED || status == NPHC_EG_NOT_CONVERGED;
        if (vl) {
            const cx<double> z = est ? P.at(CL::PV, i) : P.at(L::Z0, i);
            ep.z_re[i * cnt + e] = z.re;
            ep.z_im[i * cnt + e] = z.im;
        }
        if (lane == 0) {
            cyc_out[e] = cyc;
            eg_out[e] = status;
            ep.solves[e] += solves;
        }
        __syncwarp();
    }
}
