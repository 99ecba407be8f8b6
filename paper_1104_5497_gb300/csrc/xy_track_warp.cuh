// xy_track_warp.cuh -- FP64 path tracking of the XY ring with one path per warp, for
// short lists (paths handed off by the FP32 pass, re-tracks).
//
// GB300 runs FP64 at 1/64 of the FP32 rate, and the per-thread tracker (xy_track.cuh)
// runs every solve on all 32 lanes of a warp whatever the number of paths in it: a
// list of a few thousand paths then costs the latency of ~12k dependent FP64
// instructions per solve.  Here the 32 lanes share one path: the per-site quantities
// (frames, u, w, right-hand sides) are computed by lane j for site j, column j of the
// Schur matrix is built by lane j, each Householder step updates one column per lane,
// the back substitution updates one row per lane, and the compensated residual is one
// row pair per lane.  The step logic (RK4 predictor, Newton corrector, step control,
// divergence radius, budget) is the one of the per-thread FP64 tracker: the same
// algorithm, so the same endpoints.
//
// Storage: everything of a path in per-warp shared memory (complex doubles): the
// augmented Schur matrix [S | b0 | b1] (column-major, M x (M + 2)), the five step
// vectors Z0, K1, AC, ZC, W1 (2M each) and nine per-site arrays.
#pragma once

#include "xy_track.cuh"

template <int M>
struct WarpLayout {
    static constexpr int NV = 2 * M;
    static constexpr int A = 0;
    static constexpr int Z0 = A + M * (M + 2);
    static constexpr int K1 = Z0 + NV;
    static constexpr int AC = K1 + NV;
    static constexpr int ZC = AC + NV;
    static constexpr int W1 = ZC + NV;
    static constexpr int AH = W1 + NV;    // frame a^_j
    static constexpr int BH = AH + M;     // frame b^_j
    static constexpr int IV = BH + M;     // 1 / |(a_j, b_j)| (real part)
    static constexpr int AJ = IV + M;     // diagonal entries A_jj, B_jj of the gradient rows
    static constexpr int BJ = AJ + M;
    static constexpr int P0 = BJ + M;     // conj(a^) q0, conj(b^) q0, conj(a^) q1, conj(b^) q1
    static constexpr int Q0 = P0 + M;
    static constexpr int P1 = Q0 + M;
    static constexpr int Q1 = P1 + M;
    static constexpr int SS = Q1 + M;     // light-cone scales (sp, sq) of each site
    static constexpr int SC = SS + M;     // reflector scalars of the current Householder step
    static constexpr int TOTAL = SC + 2;
};

template <int M>
constexpr size_t warp_track_smem_per_warp() {
    return sizeof(cx<double>) * (size_t)WarpLayout<M>::TOTAL;
}

// Warp reductions whose result is lane 0's, broadcast: the butterfly leaves each lane a
// sum in its own association order, and the step logic branches on these values, so
// every lane must see the same bits.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return __shfl_sync(0xffffffffu, v, 0);
}

template <int M>
struct WarpPath {
    cx<double> *s;   // this warp's shared memory
    int lane;
    __device__ __forceinline__ cx<double> &at(int off, int i) const { return s[off + i]; }
    __device__ __forceinline__ cx<double> &A(int i, int c) const { return s[WarpLayout<M>::A + c * M + i]; }
};

// -H(z, t) at ZC into W1 with compensated sums (the per-thread tracker's xy_residual_comp,
// rows k and M + k on lane k).
template <int M>
__device__ void warp_residual(const WarpPath<M> &P, const double *__restrict__ J, double s,
                              double omt, cx<double> gam) {
    using L = WarpLayout<M>;
    using E = EFT<double>;
    const int k = P.lane;
    if (k < M) {
        const cx<double> gomt = cx<double>{E::mul(omt, gam.re), E::mul(omt, gam.im)};
        const cx<double> xk = P.at(L::ZC, k), yk = P.at(L::ZC, M + k);
        const double *Jk = J + k * NPHC_JSTRIDE;
        const ext<double> zero = {0.0, 0.0};
        ext<double> ure = {Jk[M], 0.0}, uim = zero, wre = zero, wim = zero;
#pragma unroll 1
        for (int l = 0; l < M; l++) {   // J_kk = 0 adds exact zeros
            const cx<double> xl = P.at(L::ZC, l), yl = P.at(L::ZC, M + l);
            ext_acc(ure, Jk[l], xl.re);
            ext_acc(uim, Jk[l], xl.im);
            ext_acc(wre, Jk[l], yl.re);
            ext_acc(wim, Jk[l], yl.im);
        }
        ext<double> fre = zero, fim = zero;
        ext_acc_ext(fre, yk.re, ure);
        ext_acc_ext(fre, -yk.im, uim);
        ext_acc_ext(fre, -xk.re, wre);
        ext_acc_ext(fre, xk.im, wim);
        ext_acc_ext(fim, yk.re, uim);
        ext_acc_ext(fim, yk.im, ure);
        ext_acc_ext(fim, -xk.re, wim);
        ext_acc_ext(fim, -xk.im, wre);
        ext<double> qxr = {-1.0, 0.0}, qxi = zero, qyr = {-1.0, 0.0}, qyi = zero;
        ext_acc(qxr, xk.re, xk.re);
        ext_acc(qxr, -xk.im, xk.im);
        ext_acc(qxi, 2.0 * xk.re, xk.im);
        ext_acc(qyr, yk.re, yk.re);
        ext_acc(qyr, -yk.im, yk.im);
        ext_acc(qyi, 2.0 * yk.re, yk.im);
        ext<double> hfr = zero, hfi = zero, hgr = zero, hgi = zero;
        ext_acc_ext(hfr, gomt.re, qxr);
        ext_acc_ext(hfr, -gomt.im, qxi);
        ext_acc_ext(hfr, s, fre);
        ext_acc_ext(hfi, gomt.re, qxi);
        ext_acc_ext(hfi, gomt.im, qxr);
        ext_acc_ext(hfi, s, fim);
        ext_acc_ext(hgr, gomt.re, qyr);
        ext_acc_ext(hgr, -gomt.im, qyi);
        ext_acc_ext(hgr, s, qxr);
        ext_acc_ext(hgr, s, qyr);
        ext_acc(hgr, s, 1.0);
        ext_acc_ext(hgi, gomt.re, qyi);
        ext_acc_ext(hgi, gomt.im, qyr);
        ext_acc_ext(hgi, s, qxi);
        ext_acc_ext(hgi, s, qyi);
        P.at(L::W1, k) = cx<double>{-ext_val(hfr), -ext_val(hfi)};
        P.at(L::W1, M + k) = cx<double>{-ext_val(hgr), -ext_val(hgi)};
    }
    __syncwarp();
}

// H_z(ZC, t) d = r, the per-thread xy_solve shared out over the warp.
//   two_rhs false: r = -H_t, d into W1.
//   two_rhs true:  r1 = W1 (the residual), d1 into W1; r2 = -H_t, d2 into `out2`.
// Returns false (in every lane) when S is singular or the result is not finite.
template <int M>
__device__ bool warp_solve(const WarpPath<M> &P, const double *__restrict__ J, double s,
                           double omt, cx<double> gam, bool two_rhs, int out2) {
    using L = WarpLayout<M>;
    const int lane = P.lane;
    const cx<double> gomt = cscale(omt, gam);
    const cx<double> sg = cx<double>{s + gomt.re, gomt.im};   // t + gamma (1 - t)
    // ---- per-site quantities (lane j = site j)
    if (lane < M) {
        const int j = lane;
        const cx<double> xj = P.at(L::ZC, j), yj = P.at(L::ZC, M + j);
        const double *Jj = J + j * NPHC_JSTRIDE;
        cx<double> u = cx<double>{Jj[M], 0.0}, w = cx<double>{0.0, 0.0};
#pragma unroll 1
        for (int l = 0; l < M; l++) {
            const cx<double> xl = P.at(L::ZC, l), yl = P.at(L::ZC, M + l);
            u.re += Jj[l] * xl.re;
            u.im += Jj[l] * xl.im;
            w.re += Jj[l] * yl.re;
            w.im += Jj[l] * yl.im;
        }
        cx<double> htf, htg;
        minus_ht_rows<double>(xj, yj, u, w, gam, htf, htg);
        const cx<double> rg0 = two_rhs ? P.at(L::W1, M + j) : htg;
        cx<double> ah, bh;
        double iv, sp, sq;
        g_frame<double>(xj, yj, s, sg, ah, bh, iv, sp, sq);
        cx<double> Ajj, Bjj;   // diagonal entries of gradient row j on (dwp_j, dwq_j)
        lc_coef<double>(cx<double>{-s * w.re + 2.0 * (gomt.re * xj.re - gomt.im * xj.im),
                                   -s * w.im + 2.0 * (gomt.re * xj.im + gomt.im * xj.re)},
                        cscale(s, u), sp, sq, Ajj, Bjj);
        const cx<double> q0 = cscale(iv, rg0), q1 = cscale(iv, htg);
        P.at(L::AH, j) = ah;
        P.at(L::BH, j) = bh;
        P.at(L::IV, j) = cx<double>{iv, 0.0};
        P.at(L::SS, j) = cx<double>{sp, sq};
        P.at(L::AJ, j) = Ajj;
        P.at(L::BJ, j) = Bjj;
        P.at(L::P0, j) = cmulc(ah, q0);
        P.at(L::Q0, j) = cmulc(bh, q0);
        P.at(L::P1, j) = cmulc(ah, q1);
        P.at(L::Q1, j) = cmulc(bh, q1);
        // the f-row right-hand sides wait in the right-hand-side columns
        P.A(j, M) = two_rhs ? P.at(L::W1, j) : htf;
        if (two_rhs) P.A(j, M + 1) = htf;
    }
    __syncwarp();
    // ---- column j of S (lane j), right-hand-side row k (lane k)
    // (off-diagonal: (i t J_kj / 2) (sp_j q_k b^_j + sq_j p_k a^_j) and right-hand-side terms
    // (i t J_kj / 2) (sp_j q_k px_j - sq_j p_k py_j), p = x + i y, q = x - i y; see xy_solve.cuh)
    if (lane < M) {
        const int j = lane;
        const cx<double> ah = P.at(L::AH, j), bh = P.at(L::BH, j);
        const cx<double> sc = P.at(L::SS, j);
        const double hs = 0.5 * s;
        const cx<double> cb = cmul_i(cscale(hs * sc.re, bh)), ca = cmul_i(cscale(hs * sc.im, ah));
#pragma unroll 1
        for (int k = 0; k < M; k++) {
            cx<double> e;
            if (k == j) {
                e = csub(cmul(P.at(L::AJ, j), bh), cmul(P.at(L::BJ, j), ah));
            } else {
                const cx<double> xk = P.at(L::ZC, k), yk = P.at(L::ZC, M + k);
                const cx<double> pk = cx<double>{xk.re - yk.im, xk.im + yk.re};
                const cx<double> qk = cx<double>{xk.re + yk.im, xk.im - yk.re};
                e = cscale(J[k * NPHC_JSTRIDE + j], cadd(cmul(qk, cb), cmul(pk, ca)));
            }
            P.A(k, j) = e;
        }
        const int k = lane;
        const cx<double> xk = P.at(L::ZC, k), yk = P.at(L::ZC, M + k);
        const cx<double> pk = cx<double>{xk.re - yk.im, xk.im + yk.re};
        const cx<double> qk = cx<double>{xk.re + yk.im, xk.im - yk.re};
        cx<double> b0 = P.A(k, M), b1 = two_rhs ? P.A(k, M + 1) : cx<double>{0.0, 0.0};
#pragma unroll 1
        for (int jj = 0; jj < M; jj++) {
            const cx<double> px0 = P.at(L::P0, jj), py0 = P.at(L::Q0, jj);
            const cx<double> px1 = P.at(L::P1, jj), py1 = P.at(L::Q1, jj);
            if (jj == k) {
                const cx<double> Ak = P.at(L::AJ, k), Bk = P.at(L::BJ, k);
                b0 = csub(b0, cadd(cmul(Ak, px0), cmul(Bk, py0)));
                if (two_rhs) b1 = csub(b1, cadd(cmul(Ak, px1), cmul(Bk, py1)));
            } else {
                const cx<double> scj = P.at(L::SS, jj);
                const double hJ = hs * J[k * NPHC_JSTRIDE + jj];
                const cx<double> qs = cscale(hJ * scj.re, qk), ps = cscale(hJ * scj.im, pk);
                b0 = csub(b0, cmul_i(csub(cmul(qs, px0), cmul(ps, py0))));
                if (two_rhs) b1 = csub(b1, cmul_i(csub(cmul(qs, px1), cmul(ps, py1))));
            }
        }
        P.A(k, M) = b0;
        if (two_rhs) P.A(k, M + 1) = b1;
    }
    __syncwarp();
    // ---- Householder QR, one column per lane; lane k forms the reflector of step k
    // (FP64 work is paid per active lane: the other lanes read its scalars)
    const int ncol = two_rhs ? M + 2 : M + 1;
    bool ok = true;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        if (lane == k) {
            const cx<double> al = P.A(k, k);
            double xn2 = 0.0;
#pragma unroll 1
            for (int i = k + 1; i < M; i++) xn2 += cabs2(P.A(i, k));
            const double an = sqrt(cabs2(al) + xn2);
            const double beta = al.re >= 0.0 ? -an : an;
            const double ib = 1.0 / beta;
            P.at(L::SC, 0) = cx<double>{(beta - al.re) * ib, al.im * ib};   // conj(tau)
            P.at(L::SC, 1) = crecip(cx<double>{al.re - beta, al.im});        // 1 / (al - beta)
            P.A(k, k) = cx<double>{beta, an > 0.0 ? 1.0 : 0.0};              // flag in .im
        }
        __syncwarp();
        ok = ok && P.A(k, k).im != 0.0;
        const cx<double> tauc = P.at(L::SC, 0);
        // the reflector (1, v_{k+1}, .., v_{M-1}) replaces column k below the diagonal
        if (lane > k && lane < M) P.A(lane, k) = cmul(P.A(lane, k), P.at(L::SC, 1));
        __syncwarp();
        const int c = lane;
        if (c > k && c < ncol) {
            cx<double> wv = P.A(k, c);
#pragma unroll 1
            for (int i = k + 1; i < M; i++) wv = cadd(wv, cmulc(P.A(i, k), P.A(i, c)));
            wv = cmul(tauc, wv);
            P.A(k, c) = csub(P.A(k, c), wv);
#pragma unroll 1
            for (int i = k + 1; i < M; i++) P.A(i, c) = csub(P.A(i, c), cmul(P.A(i, k), wv));
        }
        __syncwarp();
        if (lane == k) P.A(k, k).im = 0.0;   // R_kk = beta, real
        __syncwarp();
    }
    // ---- back substitution: lane k scales row k, lanes i < k eliminate it
#pragma unroll 1
    for (int k = M - 1; k >= 0; k--) {
        if (lane == k) {
            const double ir = 1.0 / P.A(k, k).re;
            P.A(k, M) = cscale(ir, P.A(k, M));
            if (two_rhs) P.A(k, M + 1) = cscale(ir, P.A(k, M + 1));
        }
        __syncwarp();
        if (lane < k) {
            const cx<double> Rik = P.A(lane, k);
            P.A(lane, M) = csub(P.A(lane, M), cmul(Rik, P.A(k, M)));
            if (two_rhs) P.A(lane, M + 1) = csub(P.A(lane, M + 1), cmul(Rik, P.A(k, M + 1)));
        }
        __syncwarp();
    }
    // ---- back to (dx, dy) (lane j = site j)
    double chk = 0.0;
    if (lane < M) {
        const int j = lane;
        const cx<double> ah = P.at(L::AH, j), bh = P.at(L::BH, j);
        const double iv = P.at(L::IV, j).re;
        const cx<double> sc = P.at(L::SS, j);
        const cx<double> xj = P.at(L::ZC, j), yj = P.at(L::ZC, M + j);
        const cx<double> htg = minus_ht_g<double>(xj, yj, gam);
        const cx<double> q0 = cscale(iv, two_rhs ? P.at(L::W1, M + j) : htg);
        cx<double> dx0, dy0;
        lc_step<double>(ah, bh, sc.re, sc.im, q0, P.A(j, M), dx0, dy0);
        chk += cabs2(dx0) + cabs2(dy0);
        cx<double> dx1 = cx<double>{0.0, 0.0}, dy1 = dx1;
        if (two_rhs) {
            const cx<double> q1 = cscale(iv, htg);
            lc_step<double>(ah, bh, sc.re, sc.im, q1, P.A(j, M + 1), dx1, dy1);
            chk += cabs2(dx1) + cabs2(dy1);
        }
        P.at(L::W1, j) = dx0;   // lane j reads and writes only entries j and M + j
        P.at(L::W1, M + j) = dy0;
        if (two_rhs) {
            P.at(out2, j) = dx1;
            P.at(out2, M + j) = dy1;
        }
    }
    __syncwarp();
    chk = warp_sum(chk);
    return ok && isfinite(chk);
}

// One path per warp; the control flow of track_body in FP64, uniform over the warp.
template <int M, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
    xy_track_warp64_kernel(const __grid_constant__ XYSys S, const __grid_constant__ XYCtl C,
                           const EPView ep, const WorkList wl) {
    using L = WarpLayout<M>;
    constexpr int NV = 2 * M;
    extern __shared__ __align__(16) unsigned char wraw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const WarpPath<M> P{reinterpret_cast<cx<double> *>(wraw) + (size_t)wid * L::TOTAL, lane};
    const double *J = S.Jd;
    const cx<double> gam = cx<double>{S.gre, S.gim};
    const int64_t total = worklist_size(wl, ep.count);
    const int64_t cnt = ep.count;
    const int i = lane;   // vector component of this lane (i < NV)
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(wl.queue, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= total) break;
        const int64_t e = worklist_entry(wl, (int64_t)q, ep.count);
        if (e < 0) continue;   // rejected by the debug build's check
        int status = NPHC_PATH_RUNNING, run = 0, rejects = 0, attempts = 0, steps, solves, newton;
        double t, h, hacc;
        bool need_k1;
        if (C.resume) {
            if (i < NV) P.at(L::Z0, i) = cx<double>{ep.z_re[i * cnt + e], ep.z_im[i * cnt + e]};
            t = ep.t[e];
            h = fmin(fmax(ep.h[e], 0.125 * (1.0 - t)), C.hmax);
            h = fmax(h, C.hmin * 4.0);
            steps = ep.steps[e];
            solves = ep.solves[e];
            newton = ep.newton[e];
            need_k1 = true;
        } else {
            const int64_t p = ep.path[e];
            if (i < NV) P.at(L::Z0, i) = cx<double>{((p >> i) & 1) ? -1.0 : 1.0, 0.0};
            __syncwarp();
            if (lane < M) {   // dz/dt at t = 0: -P_i(z) / (2 gamma z_i)
                const int k = lane;
                const cx<double> xk = P.at(L::Z0, k), yk = P.at(L::Z0, M + k);
                const double *Jk = J + k * NPHC_JSTRIDE;
                cx<double> u = cx<double>{Jk[M], 0.0}, w = cx<double>{0.0, 0.0};
#pragma unroll 1
                for (int l = 0; l < M; l++) {
                    u.re += Jk[l] * P.at(L::Z0, l).re;
                    w.re += Jk[l] * P.at(L::Z0, M + l).re;
                }
                cx<double> rf, rg;
                minus_ht_rows<double>(xk, yk, u, w, gam, rf, rg);
                const cx<double> ig = crecip(gam);
                P.at(L::K1, k) = cscale(0.5 * xk.re, cmul(ig, rf));
                P.at(L::K1, M + k) = cscale(0.5 * yk.re, cmul(ig, rg));
            }
            t = 0.0;
            h = C.h0;
            steps = C.accumulate ? ep.steps[e] : 0;
            solves = C.accumulate ? ep.solves[e] : 0;
            newton = C.accumulate ? ep.newton[e] : 0;
            need_k1 = false;
        }
        hacc = h;
        bool far = false;      // heading out: steps capped at KAPPA_FAR (1 - t) (xy_track.cuh)
        double zlast = 0.0;
        __syncwarp();
        while (status == NPHC_PATH_RUNNING) {
            if (far && h > KAPPA_FAR * (1.0 - t)) h = KAPPA_FAR * (1.0 - t);
            double hh = h, t1 = t + h;
            if (t1 >= C.t_end) {
                t1 = C.t_end;
                hh = C.t_end - t;
            }
            bool conv = false, bad = false;
            double zpn = 0.0;
            const int ph0 = need_k1 ? 0 : 1;
            const int nph = 4 + C.max_newton;
#pragma unroll 1
            for (int ph = ph0; ph < nph; ph++) {
                const bool corr = ph >= 4 || ph == 0;
                if (ph >= 4 && (conv || bad)) break;
                const double te = ph == 0 ? t : (ph >= 4 || ph == 3) ? t1 : t + 0.5 * hh;
                if (ph < 4) {   // evaluation point: z0, z0 + h/2 k1, z0 + h/2 k2, z0 + h k3
                    const double c = ph == 3 ? hh : 0.5 * hh;
                    if (i < NV) {
                        const cx<double> z0 = P.at(L::Z0, i);
                        P.at(L::ZC, i) = ph == 0 ? z0
                                                 : cadd(z0, cscale(c, ph == 1 ? P.at(L::K1, i) : P.at(L::W1, i)));
                    }
                    __syncwarp();
                }
                if (corr) warp_residual<M>(P, J, te, 1.0 - te, gam);
                const bool oks = warp_solve<M>(P, J, te, 1.0 - te, gam, corr, L::AC);
                solves++;
                if (ph == 0) {   // pull the resumed point onto the FP64 path; dz/dt there
                    if (i < NV) {
                        P.at(L::Z0, i) = cadd(P.at(L::ZC, i), P.at(L::W1, i));
                        P.at(L::K1, i) = P.at(L::AC, i);
                    }
                    __syncwarp();
                    newton++;
                    need_k1 = false;
                    if (!oks) status = NPHC_PATH_NONFINITE;
                    if (status != NPHC_PATH_RUNNING) break;
                } else if (!corr) {
                    bad = bad || !oks;
                    if (i < NV) {
                        const cx<double> w1 = P.at(L::W1, i);
                        if (ph == 1) P.at(L::AC, i) = cadd(P.at(L::K1, i), cscale(2.0, w1));
                        else if (ph == 2) P.at(L::AC, i) = cadd(P.at(L::AC, i), cscale(2.0, w1));
                    }
                    if (ph == 3) {   // predicted point z0 + h/6 (k1 + 2 k2 + 2 k3 + k4)
                        double zz = 0.0;
                        if (i < NV) {
                            const cx<double> zp = cadd(P.at(L::Z0, i),
                                                       cscale(hh / 6.0, cadd(P.at(L::AC, i), P.at(L::W1, i))));
                            P.at(L::ZC, i) = zp;
                            zz = cabs2(zp);
                        }
                        zpn = sqrt(warp_sum(zz));
                    }
                    __syncwarp();
                } else {
                    newton++;
                    const double dn = sqrt(warp_sum(i < NV ? cabs2(P.at(L::W1, i)) : 0.0));
                    if (!oks || !isfinite(dn)) {
                        bad = true;
                    } else if (ph == 4 && dn > C.trust * (1.0 + zpn)) {
                        bad = true;
                    } else {
                        double zz = 0.0;
                        if (i < NV) {
                            const cx<double> zn = cadd(P.at(L::ZC, i), P.at(L::W1, i));
                            P.at(L::ZC, i) = zn;
                            zz = cabs2(zn);
                        }
                        zz = warp_sum(zz);
                        if (dn <= C.eps * (1.0 + sqrt(zz))) conv = true;
                    }
                    __syncwarp();
                }
            }
            if (status != NPHC_PATH_RUNNING) break;
            attempts++;
            if (conv) {
                double zi = 0.0;
                if (i < NV) {
                    const cx<double> v = P.at(L::ZC, i);
                    P.at(L::Z0, i) = v;
                    P.at(L::K1, i) = P.at(L::AC, i);
                    zi = sqrt(cabs2(v));
                }
                zi = warp_max(zi);
                __syncwarp();
                t = t1;
                far = 1.0 - t < CRAWL_ZONE && zi > FAR_NORM && zi > FAR_GROWTH * zlast;
                zlast = zi;
                steps++;
                rejects = 0;
                hacc = h;
                if (++run >= C.grow_after) {
                    run = 0;
                    h = fmin(2.0 * h, C.hmax);
                }
                if (zi > C.rdiv) status = NPHC_PATH_DIVERGED;
                else if (t >= C.t_end) status = NPHC_PATH_REACHED;
            } else {
                run = 0;
                rejects++;
                h *= 0.5;
                if (h < C.hmin) status = NPHC_PATH_MIN_STEP;
            }
            if (status == NPHC_PATH_RUNNING && attempts >= C.max_steps) status = NPHC_PATH_STEP_BUDGET;
        }
        if (i < NV) {
            const cx<double> v = P.at(L::Z0, i);
            ep.z_re[i * cnt + e] = v.re;
            ep.z_im[i * cnt + e] = v.im;
        }
        if (lane == 0) {
            ep.t[e] = t;
            ep.h[e] = h;
            ep.status[e] = status;
            ep.steps[e] = steps;
            ep.solves[e] = solves;
            ep.newton[e] = newton;
        }
        __syncwarp();
    }
}
