// xy_track_warp.cuh -- FP64 path tracking of the XY ring with one path per warp, for
// short lists (paths handed off by the FP32 pass, re-tracks).
//
// GB300 runs FP64 at 1/64 of the FP32 rate, and its FP64 pipe takes a warp instruction
// at the same cost whatever the number of active lanes: a solve costs about 76 cycles of
// an SM sub-partition per FP64 instruction on the longest chain that any lane runs.  So
// the 32 lanes share one path, and every stage is laid out to keep each lane's own FP64
// chain short rather than to save lanes:
//   * per-site quantities (couplings sums, frames, the diagonal's terms): lane j for
//     site j, the sums u_j and w_j on lanes j and 16 + j;
//   * the off-diagonal Schur entries: one entry per lane, strided over the M x M matrix;
//   * the right-hand sides: sums of J times per-site vectors, right-hand side r on the
//     lanes 16 r + k (row k);
//   * the factorisation: LU with partial pivoting (one reciprocal per column and no
//     square root; the pivot search compares the bit patterns of |re| + |im| as integers
//     and costs one FP64 add), the rank-one update strided over the trailing block;
//   * the back substitution in registers (right-hand side r on lanes 16 r + row);
//   * the compensated residual of row pair k on lanes k and 16 + k.
// The step logic (RK4 predictor, Newton corrector, step control, divergence radius,
// budget) is the per-thread FP64 tracker's, as are the state in light-cone coordinates,
// the equations and the scaled light-cone frames of the Schur reduction (xy_solve.cuh):
// the same algorithm with a different linear solver, so the endpoints agree to the
// tracking tolerance.  The Cauchy endgame (cauchy_warp.cuh) calls the same solve and
// residual on points in (x, y).
//
// Storage: everything of a path in per-warp shared memory (complex doubles): the
// augmented Schur matrix [S | b0 | b1] (column-major, M x (M + 2)), the five step
// vectors Z0, K1, AC, ZC, W1 (2M each) and thirteen per-site arrays.
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
    static constexpr int SS = BH + M;     // light-cone scales (sp, sq) of site j
    static constexpr int CB = SS + M;     // (i t / 2) sp_j b^_j: Schur column j is J_kj (q_k CB_j + p_k CA_j)
    static constexpr int CA = CB + M;     // (i t / 2) sq_j a^_j
    static constexpr int X0 = CA + M;     // sp_j conj(a^_j) q0_j, sq_j conj(b^_j) q0_j (right-hand side 0),
    static constexpr int Y0 = X0 + M;
    static constexpr int X1 = Y0 + M;     // the same with q1_j (right-hand side 1)
    static constexpr int Y1 = X1 + M;
    static constexpr int PK = Y1 + M;     // p_j = x_j + i y_j, q_j = x_j - i y_j
    static constexpr int QK = PK + M;
    static constexpr int QS0 = QK + M;    // the constraint rows' components q0_j, q1_j
    static constexpr int QS1 = QS0 + M;
    static constexpr int TOTAL = QS1 + M;
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

// c - a b with four fused multiply-adds
__device__ __forceinline__ cx<double> cfnms(cx<double> c, cx<double> a, cx<double> b) {
    return cx<double>{fma(a.im, b.im, fma(-a.re, b.re, c.re)), fma(-a.im, b.re, fma(-a.re, b.im, c.im))};
}

__device__ __forceinline__ cx<double> shfl_down16(cx<double> v) {
    return cx<double>{__shfl_down_sync(0xffffffffu, v.re, 16), __shfl_down_sync(0xffffffffu, v.im, 16)};
}

__device__ __forceinline__ ext<double> shfl_down16(ext<double> v) {
    return ext<double>{__shfl_down_sync(0xffffffffu, v.hi, 16), __shfl_down_sync(0xffffffffu, v.lo, 16)};
}

// (a.hi + a.lo) + (b.hi + b.lo), the rounding error of the leading sum kept in lo
__device__ __forceinline__ ext<double> ext_add(ext<double> a, ext<double> b) {
    double s, e;
    two_sum(a.hi, b.hi, s, e);
    return ext<double>{s, EFT<double>::add(e, EFT<double>::add(a.lo, b.lo))};
}

template <int M>
struct WarpPath {
    cx<double> *s;   // this warp's shared memory
    int lane;
    __device__ __forceinline__ cx<double> &at(int off, int i) const { return s[off + i]; }
    __device__ __forceinline__ cx<double> &A(int i, int c) const { return s[WarpLayout<M>::A + c * M + i]; }
};

// -H(z, t) at ZC into W1 with compensated sums (the per-thread trackers' residuals).
// LC == false: ZC holds (x, y) (the Cauchy endgame); row pair k: lane k sums
// u_k = J_kN + sum_l J_kl x_l and forms the f row, lane 16 + k sums w_k = sum_l J_kl y_l,
// forms the g row (which needs no sums) and hands its share of f_k = y_k u_k - x_k w_k to
// lane k.  LC == true: ZC holds the light-cone coordinates (p, q) (xy_residual_comp in
// xy_solve.cuh); lane k sums U_p,k, lane 16 + k sums U_q,k, and D_k = q_k U_p,k - p_k U_q,k
// is formed the same way.
template <int M, bool LC = false>
__device__ void warp_residual(const WarpPath<M> &P, const double *__restrict__ J, double s,
                              double omt, cx<double> gam) {
    static_assert(M <= 16, "one row pair per lane pair");
    using L = WarpLayout<M>;
    using E = EFT<double>;
    const int k = P.lane & 15;
    const bool hi = P.lane >= 16;
    const ext<double> zero = {0.0, 0.0};
    ext<double> fre = zero, fim = zero;   // lane k's and lane 16 + k's shares of f (or D)
    cx<double> zk = cx<double>{0.0, 0.0}, wk = zk;   // (x_k, y_k) or (p_k, q_k)
    const cx<double> gomt = cx<double>{E::mul(omt, gam.re), E::mul(omt, gam.im)};
    if (k < M) {
        zk = P.at(L::ZC, k);
        wk = P.at(L::ZC, M + k);
        const double *Jk = J + k * NPHC_JSTRIDE;
        const int off = hi ? L::ZC + M : L::ZC;
        ext<double> sre = {(hi && !LC) ? 0.0 : Jk[M], 0.0}, sim = zero;
#pragma unroll 1
        for (int l = 0; l < M; l++) {   // J_kk = 0 adds exact zeros
            const cx<double> v = P.at(off, l);
            ext_acc(sre, Jk[l], v.re);
            ext_acc(sim, Jk[l], v.im);
        }
        // (x, y): lane k y_k u_k, lane 16 + k -x_k w_k;  (p, q): lane k q_k U_p, lane 16 + k -p_k U_q
        const cx<double> c = hi ? cx<double>{-zk.re, -zk.im} : wk;
        ext_acc_ext(fre, c.re, sre);
        ext_acc_ext(fre, -c.im, sim);
        ext_acc_ext(fim, c.re, sim);
        ext_acc_ext(fim, c.im, sre);
    }
    const ext<double> ore = shfl_down16(fre), oim = shfl_down16(fim);
    if (k < M) {
        if (!LC) {
            const cx<double> xk = zk, yk = wk;
            ext<double> qxr = {-1.0, 0.0}, qxi = zero;
            ext_acc(qxr, xk.re, xk.re);
            ext_acc(qxr, -xk.im, xk.im);
            ext_acc(qxi, 2.0 * xk.re, xk.im);
            if (!hi) {
                fre = ext_add(fre, ore);
                fim = ext_add(fim, oim);
                ext<double> hfr = zero, hfi = zero;
                ext_acc_ext(hfr, gomt.re, qxr);
                ext_acc_ext(hfr, -gomt.im, qxi);
                ext_acc_ext(hfr, s, fre);
                ext_acc_ext(hfi, gomt.re, qxi);
                ext_acc_ext(hfi, gomt.im, qxr);
                ext_acc_ext(hfi, s, fim);
                P.at(L::W1, k) = cx<double>{-ext_val(hfr), -ext_val(hfi)};
            } else {
                ext<double> qyr = {-1.0, 0.0}, qyi = zero;
                ext_acc(qyr, yk.re, yk.re);
                ext_acc(qyr, -yk.im, yk.im);
                ext_acc(qyi, 2.0 * yk.re, yk.im);
                ext<double> hgr = zero, hgi = zero;
                ext_acc_ext(hgr, gomt.re, qyr);
                ext_acc_ext(hgr, -gomt.im, qyi);
                ext_acc_ext(hgr, s, qxr);
                ext_acc_ext(hgr, s, qyr);
                ext_acc(hgr, s, 1.0);
                ext_acc_ext(hgi, gomt.re, qyi);
                ext_acc_ext(hgi, gomt.im, qyr);
                ext_acc_ext(hgi, s, qxi);
                ext_acc_ext(hgi, s, qyi);
                P.at(L::W1, M + k) = cx<double>{-ext_val(hgr), -ext_val(hgi)};
            }
        } else {
            const cx<double> pk = zk, qk = wk;
            const double hs = 0.5 * s;
            if (!hi) {
                // H_f = gomt X + t f, f = i D / 2, X = x^2 - 1 = (p^2 + 2 p q + q^2) / 4 - 1
                const ext<double> dr = ext_add(fre, ore), di = ext_add(fim, oim);
                ext<double> xr = {-1.0, 0.0}, xi = zero;
                ext_acc(xr, 0.25 * pk.re, pk.re);
                ext_acc(xr, -0.25 * pk.im, pk.im);
                ext_acc(xr, 0.5 * pk.re, qk.re);
                ext_acc(xr, -0.5 * pk.im, qk.im);
                ext_acc(xr, 0.25 * qk.re, qk.re);
                ext_acc(xr, -0.25 * qk.im, qk.im);
                ext_acc(xi, 0.5 * pk.re, pk.im);
                ext_acc(xi, 0.5 * pk.re, qk.im);
                ext_acc(xi, 0.5 * pk.im, qk.re);
                ext_acc(xi, 0.5 * qk.re, qk.im);
                ext<double> hfr = zero, hfi = zero;
                ext_acc_ext(hfr, gomt.re, xr);
                ext_acc_ext(hfr, -gomt.im, xi);
                ext_acc_ext(hfr, -hs, di);
                ext_acc_ext(hfi, gomt.re, xi);
                ext_acc_ext(hfi, gomt.im, xr);
                ext_acc_ext(hfi, hs, dr);
                P.at(L::W1, k) = cx<double>{-ext_val(hfr), -ext_val(hfi)};
            } else {
                // H_g = gomt Y + t G, Y = y^2 - 1 = -(p^2 - 2 p q + q^2) / 4 - 1, G = p q - 1
                ext<double> yr = {-1.0, 0.0}, yi = zero, gr = {-1.0, 0.0}, gi = zero;
                ext_acc(yr, -0.25 * pk.re, pk.re);
                ext_acc(yr, 0.25 * pk.im, pk.im);
                ext_acc(yr, 0.5 * pk.re, qk.re);
                ext_acc(yr, -0.5 * pk.im, qk.im);
                ext_acc(yr, -0.25 * qk.re, qk.re);
                ext_acc(yr, 0.25 * qk.im, qk.im);
                ext_acc(yi, -0.5 * pk.re, pk.im);
                ext_acc(yi, 0.5 * pk.re, qk.im);
                ext_acc(yi, 0.5 * pk.im, qk.re);
                ext_acc(yi, -0.5 * qk.re, qk.im);
                ext_acc(gr, pk.re, qk.re);
                ext_acc(gr, -pk.im, qk.im);
                ext_acc(gi, pk.re, qk.im);
                ext_acc(gi, pk.im, qk.re);
                ext<double> hgr = zero, hgi = zero;
                ext_acc_ext(hgr, gomt.re, yr);
                ext_acc_ext(hgr, -gomt.im, yi);
                ext_acc_ext(hgr, s, gr);
                ext_acc_ext(hgi, gomt.re, yi);
                ext_acc_ext(hgi, gomt.im, yr);
                ext_acc_ext(hgi, s, gi);
                P.at(L::W1, M + k) = cx<double>{-ext_val(hgr), -ext_val(hgi)};
            }
        }
    }
    __syncwarp();
}

// H_z(ZC, t) d = r, the per-thread xy_solve's Schur reduction shared out over the warp;
// ZC and d in (x, y) (LC == false) or in the light-cone coordinates (p, q).
//   two_rhs false: r = -H_t, d into W1.
//   two_rhs true:  r1 = W1 (the residual), d1 into W1; r2 = -H_t, d2 into `out2`.
// Returns false (in every lane) when S is singular or the result is not finite.
template <int M, bool LC = false>
__device__ bool warp_solve(const WarpPath<M> &P, const double *__restrict__ J, double s,
                           double omt, cx<double> gam, bool two_rhs, int out2) {
    static_assert(M <= 16, "one site per lane of each half-warp");
    using L = WarpLayout<M>;
    const int lane = P.lane;
    const int hrow = lane & 15, r = lane >> 4;   // row and right-hand side of the half-warp layout
    const cx<double> gomt = cscale(omt, gam);
    const cx<double> sg = cx<double>{s + gomt.re, gomt.im};   // t + gamma (1 - t)
    const double hs = 0.5 * s;

    // ---- per-site quantities: u_j (U_p,j) on lane j, w_j (U_q,j) on lane 16 + j, the
    // rest on lane j
    cx<double> uw = cx<double>{0.0, 0.0};
    if (hrow < M) {
        const int j = hrow;
        const double *Jj = J + j * NPHC_JSTRIDE;
        const int off = r ? L::ZC + M : L::ZC;
        uw = cx<double>{(r && !LC) ? 0.0 : Jj[M], 0.0};
#pragma unroll 1
        for (int l = 0; l < M; l++) {
            const cx<double> v = P.at(off, l);
            uw.re = fma(Jj[l], v.re, uw.re);
            uw.im = fma(Jj[l], v.im, uw.im);
        }
    }
    const cx<double> w = shfl_down16(uw);
    if (lane < M) {
        const int j = lane;
        const cx<double> u = uw;
        const cx<double> zj = P.at(L::ZC, j), wj = P.at(L::ZC, M + j);
        cx<double> htf, htg, ah, bh, Ajj, Bjj, pj, qj;   // Ajj, Bjj: gradient row j on (dwp_j, dwq_j)
        double iv, sp, sq;
        if (LC) {
            pj = zj;
            qj = wj;
            lc_minus_ht_rows<double>(pj, qj, u, w, gam, htf, htg);
            g_frame_lc<double>(pj, qj, s, gomt, ah, bh, iv, sp, sq);
            const cx<double> gpq = cmul(gomt, cadd(pj, qj));
            Ajj = cscale(0.5 * sp, csub(gpq, cmul_i(cscale(s, w))));
            Bjj = cscale(0.5 * sq, cadd(gpq, cmul_i(cscale(s, u))));
        } else {
            const cx<double> xj = zj, yj = wj;
            pj = cx<double>{xj.re - yj.im, xj.im + yj.re};
            qj = cx<double>{xj.re + yj.im, xj.im - yj.re};
            minus_ht_rows<double>(xj, yj, u, w, gam, htf, htg);
            g_frame<double>(xj, yj, s, sg, ah, bh, iv, sp, sq);
            lc_coef<double>(cx<double>{-s * w.re + 2.0 * (gomt.re * xj.re - gomt.im * xj.im),
                                       -s * w.im + 2.0 * (gomt.re * xj.im + gomt.im * xj.re)},
                            cscale(s, u), sp, sq, Ajj, Bjj);
        }
        const cx<double> rf0 = two_rhs ? P.at(L::W1, j) : htf;
        const cx<double> rg0 = two_rhs ? P.at(L::W1, M + j) : htg;
        const cx<double> q0 = cscale(iv, rg0), q1 = cscale(iv, htg);
        const cx<double> px0 = cmulc(ah, q0), py0 = cmulc(bh, q0);
        P.at(L::AH, j) = ah;
        P.at(L::BH, j) = bh;
        P.at(L::SS, j) = cx<double>{sp, sq};
        P.at(L::CB, j) = cmul_i(cscale(hs * sp, bh));
        P.at(L::CA, j) = cmul_i(cscale(hs * sq, ah));
        P.at(L::X0, j) = cscale(sp, px0);
        P.at(L::Y0, j) = cscale(sq, py0);
        P.at(L::PK, j) = pj;
        P.at(L::QK, j) = qj;
        P.at(L::QS0, j) = q0;
        // the diagonal entry, and the diagonal's own terms of the right-hand sides
        P.A(j, j) = csub(cmul(Ajj, bh), cmul(Bjj, ah));
        P.A(j, M) = csub(rf0, cadd(cmul(Ajj, px0), cmul(Bjj, py0)));
        if (two_rhs) {
            const cx<double> px1 = cmulc(ah, q1), py1 = cmulc(bh, q1);
            P.at(L::X1, j) = cscale(sp, px1);
            P.at(L::Y1, j) = cscale(sq, py1);
            P.at(L::QS1, j) = q1;
            P.A(j, M + 1) = csub(htf, cadd(cmul(Ajj, px1), cmul(Bjj, py1)));
        }
    }
    __syncwarp();

    // ---- off-diagonal entries of S, one per lane (consecutive lanes: consecutive rows);
    // right-hand side r of row k on lane 16 r + k:
    //   b_k -= (i t / 2) (q_k sum_j J_kj X_j - p_k sum_j J_kj Y_j)   (J_kk = 0)
#pragma unroll 1
    for (int e = lane; e < M * M; e += 32) {
        const int j = e / M, k = e - j * M;
        if (k != j)
            P.A(k, j) = cscale(J[k * NPHC_JSTRIDE + j],
                               cadd(cmul(P.at(L::QK, k), P.at(L::CB, j)), cmul(P.at(L::PK, k), P.at(L::CA, j))));
    }
    if (hrow < M && (r == 0 || two_rhs)) {
        const int k = hrow;
        const double *Jk = J + k * NPHC_JSTRIDE;
        const int ox = r ? L::X1 : L::X0, oy = r ? L::Y1 : L::Y0;
        cx<double> sx = cx<double>{0.0, 0.0}, sy = sx;
#pragma unroll 1
        for (int j = 0; j < M; j++) {
            const double Jkj = Jk[j];
            const cx<double> xv = P.at(ox, j), yv = P.at(oy, j);
            sx.re = fma(Jkj, xv.re, sx.re);
            sx.im = fma(Jkj, xv.im, sx.im);
            sy.re = fma(Jkj, yv.re, sy.re);
            sy.im = fma(Jkj, yv.im, sy.im);
        }
        const cx<double> d = csub(cmul(P.at(L::QK, k), sx), cmul(P.at(L::PK, k), sy));
        P.A(k, M + r) = csub(P.A(k, M + r), cmul_i(cscale(hs, d)));
    }
    __syncwarp();

    // ---- LU with partial pivoting of [S | b0 | b1]; the pivot's reciprocal replaces it
    const int ncol = two_rhs ? M + 2 : M + 1;
    bool ok = true;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        // the row of the largest |re| + |im| at or below k (ties: the lowest row); the
        // bit patterns of non-negative doubles order as the values do
        unsigned long long key = 0ull;
        int idx = lane;
        if (lane >= k && lane < M) {
            const cx<double> a = P.A(lane, k);
            key = (unsigned long long)__double_as_longlong(fabs(a.re) + fabs(a.im));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ko = __shfl_xor_sync(0xffffffffu, key, o);
            const int io = __shfl_xor_sync(0xffffffffu, idx, o);
            if (ko > key || (ko == key && io < idx)) {
                key = ko;
                idx = io;
            }
        }
        int p = idx;
        if (key == 0ull) {   // the column is zero from row k down: S is singular
            ok = false;
            p = k;
        }
        if (p != k) {   // uniform
            if (lane >= k && lane < ncol) {
                const cx<double> a = P.A(k, lane);
                P.A(k, lane) = P.A(p, lane);
                P.A(p, lane) = a;
            }
            __syncwarp();
        }
        const cx<double> a = P.A(k, k);
        const double rd = 1.0 / fma(a.re, a.re, a.im * a.im);
        const cx<double> ip = cx<double>{a.re * rd, -a.im * rd};
        if (lane > k && lane < M) P.A(lane, k) = cmul(P.A(lane, k), ip);
        __syncwarp();
        const int nr = M - 1 - k, nc = ncol - 1 - k;
#pragma unroll 1
        for (int e = lane; e < nr * nc; e += 32) {
            const int c = k + 1 + e / nr, i = k + 1 + (e - (e / nr) * nr);
            P.A(i, c) = cfnms(P.A(i, c), P.A(i, k), P.A(k, c));
        }
        if (lane == 31) P.A(k, k) = ip;   // nothing reads the pivot in this step's update
        __syncwarp();
    }

    // ---- back substitution U x = b in registers: right-hand side r, row hrow
    const bool act = r == 0 || two_rhs;
    cx<double> cur = cx<double>{0.0, 0.0};
    if (act && hrow < M) cur = P.A(hrow, M + r);
#pragma unroll 1
    for (int k = M - 1; k >= 0; k--) {
        const int src = (lane & 16) | k;
        const cx<double> bk = cx<double>{__shfl_sync(0xffffffffu, cur.re, src),
                                         __shfl_sync(0xffffffffu, cur.im, src)};
        if (hrow <= k) {
            const cx<double> xk = cmul(bk, P.A(k, k));   // the pivot's reciprocal
            cur = hrow == k ? xk : cfnms(cur, P.A(hrow, k), xk);
        }
    }

    // ---- back to (dx, dy) or (dp, dq) = (sp dwp, sq dwq): site j of right-hand side r on
    // lane 16 r + j, (dwp, dwq) = conj(a^, b^) q_j + (b^, -a^) s_j
    double chk = 0.0;
    if (act && hrow < M) {
        const int j = hrow;
        const cx<double> sc = P.at(L::SS, j), ah = P.at(L::AH, j), bh = P.at(L::BH, j);
        const cx<double> qv = P.at(r ? L::QS1 : L::QS0, j);
        cx<double> dx, dy;
        if (LC) {
            dx = cscale(sc.re, cadd(cmulc(ah, qv), cmul(bh, cur)));
            dy = cscale(sc.im, csub(cmulc(bh, qv), cmul(ah, cur)));
        } else {
            lc_step<double>(ah, bh, sc.re, sc.im, qv, cur, dx, dy);
        }
        chk = cabs2(dx) + cabs2(dy);
        const int o = r ? out2 : L::W1;   // W1's entries j and M + j were read above only
        P.at(o, j) = dx;
        P.at(o, M + j) = dy;
    }
    __syncwarp();
    chk = warp_sum(chk);
    return ok && isfinite(chk);
}

// One path per warp; the control flow of track_body in FP64, uniform over the warp.  The
// path's state is in light-cone coordinates (p_k, q_k) = (x_k + i y_k, x_k - i y_k), like
// the per-thread trackers' (xy_track.cuh): near infinity one of them is far below x_k and
// y_k, and in (x, y) FP64 would lose it to cancellation.  Norms are those of (x, y):
// ||(x, y)||_2 = sqrt(1/2) ||(p, q)||_2 and ||(x, y)||_inf = max_k max(|p + q|, |p - q|) / 2.
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
            if (lane < M) {   // (x, y) to (p, q)
                const int k = lane;
                const double xr = ep.z_re[k * cnt + e], xi = ep.z_im[k * cnt + e];
                const double yr = ep.z_re[(M + k) * cnt + e], yi = ep.z_im[(M + k) * cnt + e];
                P.at(L::Z0, k) = cx<double>{xr - yi, xi + yr};
                P.at(L::Z0, M + k) = cx<double>{xr + yi, xi - yr};
            }
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
                const cx<double> dx = cscale(0.5 * xk.re, cmul(ig, rf));
                const cx<double> dy = cscale(0.5 * yk.re, cmul(ig, rg));
                P.at(L::K1, k) = cadd(dx, cmul_i(dy));       // dp = dx + i dy
                P.at(L::K1, M + k) = csub(dx, cmul_i(dy));   // dq = dx - i dy
            }
            __syncwarp();
            if (lane < M) {   // p = x + i y, q = x - i y (x, y real at the start)
                const int k = lane;
                const double xk = P.at(L::Z0, k).re, yk = P.at(L::Z0, M + k).re;
                P.at(L::Z0, k) = cx<double>{xk, yk};
                P.at(L::Z0, M + k) = cx<double>{xk, -yk};
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
                if (corr) warp_residual<M, true>(P, J, te, 1.0 - te, gam);
                const bool oks = warp_solve<M, true>(P, J, te, 1.0 - te, gam, corr, L::AC);
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
                        zpn = sqrt(0.5 * warp_sum(zz));
                    }
                    __syncwarp();
                } else {
                    newton++;
                    const double dn = sqrt(0.5 * warp_sum(i < NV ? cabs2(P.at(L::W1, i)) : 0.0));
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
                        zz = 0.5 * warp_sum(zz);
                        if (dn <= C.eps * (1.0 + sqrt(zz))) conv = true;
                    }
                    __syncwarp();
                }
            }
            if (status != NPHC_PATH_RUNNING) break;
            attempts++;
            if (conv) {
                double zi = 0.0;   // ||(x, y)||_inf
                if (i < NV) {
                    P.at(L::Z0, i) = P.at(L::ZC, i);
                    P.at(L::K1, i) = P.at(L::AC, i);
                }
                if (lane < M) {
                    const cx<double> pk = P.at(L::ZC, lane), qk = P.at(L::ZC, M + lane);
                    zi = 0.5 * sqrt(fmax(cabs2(cadd(pk, qk)), cabs2(csub(pk, qk))));
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
        if (lane < M) {   // x = (p + q) / 2, y = -i (p - q) / 2
            const int k = lane;
            const cx<double> pk = P.at(L::Z0, k), qk = P.at(L::Z0, M + k);
            ep.z_re[k * cnt + e] = 0.5 * (pk.re + qk.re);
            ep.z_im[k * cnt + e] = 0.5 * (pk.im + qk.im);
            ep.z_re[(M + k) * cnt + e] = 0.5 * (pk.im - qk.im);
            ep.z_im[(M + k) * cnt + e] = -0.5 * (pk.re - qk.re);
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
