// quad.cuh -- a generic square system of quadratics, P_i(z) = sum_t c_t w(a_t) w(b_t)
// with w(-1) = 1 (a term list), tracked along the same total-degree gamma-trick homotopy
//   H(z, t) = gamma (1 - t) Q(z) + t P(z),  Q_i = z_i^2 - 1,
// from the 2^n start points z in {+1, -1}^n (section "Numerical Polynomial Homotopy
// Continuation Method", including its one-variable example x^2 - 5 from x^2 - 1), in
// FP64, then refined, certified (alpha-theory) and deduplicated like the XY ring.
//
// The terms are sorted by equation on the host (row offsets in QSys.row) and live in
// device memory owned by the system; every thread reads them in the same order
// (broadcast loads).  The Jacobian is dense here: H_z is built in the per-thread shared
// matrix of the tracker and factored by the same augmented Householder QR as the XY
// ring's Schur system (aug_qr_solve); the endgame uses the stored-reflector QR of
// xy_endgame.cuh on DP.
#pragma once

#include "cauchy.cuh"
#include "xy_endgame.cuh"
#include "xy_track.cuh"

// Tracker policy (see XYProblem): FP64, one dense NV x NV Jacobian per thread.
template <int NVT>
struct QuadProblem {
    using R = double;
    using Sys = QSys;
    static constexpr int BLOCK = 32;
    static constexpr int NV = NVT;
    static constexpr int MD = NVT;

    // the tracker's state is z itself (see XYProblem for the hooks)
    static constexpr double NORM_SCALE = 1.0;
    template <class V>
    static __device__ __forceinline__ void load(const EPView &ep, int64_t e, const V &Z) {
#pragma unroll 1
        for (int k = 0; k < NV; k++)
            Z.set(k, cx<double>{ep.z_re[k * ep.count + e], ep.z_im[k * ep.count + e]});
    }
    template <class V>
    static __device__ __forceinline__ void store(const EPView &ep, int64_t e, const V &Z) {
#pragma unroll 1
        for (int k = 0; k < NV; k++) {
            const cx<double> v = Z.get(k);
            ep.z_re[k * ep.count + e] = v.re;
            ep.z_im[k * ep.count + e] = v.im;
        }
    }
    template <class V>
    static __device__ __forceinline__ double norminf(const V &Z) {
        double s = 0.0;
#pragma unroll 1
        for (int k = 0; k < NV; k++) s = fmax(s, sqrt(cabs2(Z.get(k))));
        return s;
    }

    template <class V>
    static __device__ __forceinline__ cx<double> w(const V &z, int a) {
        return a < 0 ? cx<double>{1.0, 0.0} : z.get(a);
    }

    // P_i at the point z (plain FP64)
    template <class V>
    static __device__ __forceinline__ cx<double> p_row(const Sys &S, const V &z, int i) {
        cx<double> acc = cx<double>{0.0, 0.0};
#pragma unroll 1
        for (int t = S.row[i]; t < S.row[i + 1]; t++) {
            const QTerm T = S.terms[t];
            acc = cadd(acc, cmul(cx<double>{T.cre, T.cim}, cmul(w(z, T.a), w(z, T.b))));
        }
        return acc;
    }

    // start point of path p: z_i = -1 if bit i of p is set, else +1; dz_i/dt at t = 0 is
    // -P_i(z) / (2 gamma z_i) (H_z = 2 gamma diag(z), H_t = P(z) - gamma Q(z) = P(z))
    static __device__ __forceinline__ void start(const Sys &S, int64_t p, const GVec<double> &Z0,
                                                 const GVec<double> &K1) {
#pragma unroll 1
        for (int i = 0; i < NV; i++) Z0.set(i, cx<double>{((p >> i) & 1) ? -1.0 : 1.0, 0.0});
        const cx<double> ig = crecip(cx<double>{S.gre, S.gim});
#pragma unroll 1
        for (int i = 0; i < NV; i++) {
            const double zi = Z0.get(i).re;
            K1.set(i, cscale(-0.5 * zi, cmul(ig, p_row(S, Z0, i))));
        }
    }

    // -H(z, t) with exact products and double-double sums, rounded once (as for the XY ring)
    static __device__ __forceinline__ void residual(const Sys &S, const SVec<double, BLOCK> &pt,
                                                    double s, double omt,
                                                    const SVec<double, BLOCK> &out, bool wr) {
        residual_g(S, pt, s, omt, cx<double>{S.gre, S.gim}, out, wr);
    }

    template <class Out2>
    static __device__ __forceinline__ bool solve(const Sys &S, const SMat<NV, double, BLOCK> &A,
                                                 const SVec<double, BLOCK> &pt, double s,
                                                 double omt, bool two_rhs,
                                                 const SVec<double, BLOCK> &res,
                                                 const SVec<double, BLOCK> &out1, const Out2 &out2,
                                                 bool wr, double *kest = nullptr) {
        return solve_g(S, A, pt, s, omt, cx<double>{S.gre, S.gim}, two_rhs, res, out1, out2, wr,
                       kest);
    }

    // the same with an explicit gamma (see XYProblem::residual_g)
    static __device__ __forceinline__ void residual_g(const Sys &S, const SVec<double, BLOCK> &pt,
                                                      double s, double omt, cx<double> gam,
                                                      const SVec<double, BLOCK> &out, bool wr) {
        using E = EFT<double>;
        const ext<double> zero = {0.0, 0.0};
        const double g1r = E::mul(omt, gam.re), g1i = E::mul(omt, gam.im);
#pragma unroll 1
        for (int i = 0; i < NV; i++) {
            ext<double> pr = zero, pi = zero;
#pragma unroll 1
            for (int t = S.row[i]; t < S.row[i + 1]; t++) {
                const QTerm T = S.terms[t];
                const cx<double> wa = w(pt, T.a), wb = w(pt, T.b);
                ext<double> mr = zero, mi = zero;   // wa * wb
                ext_acc(mr, wa.re, wb.re);
                ext_acc(mr, -wa.im, wb.im);
                ext_acc(mi, wa.re, wb.im);
                ext_acc(mi, wa.im, wb.re);
                ext_acc_ext(pr, T.cre, mr);
                ext_acc_ext(pr, -T.cim, mi);
                ext_acc_ext(pi, T.cre, mi);
                ext_acc_ext(pi, T.cim, mr);
            }
            const cx<double> zi = pt.get(i);
            ext<double> qr = {-1.0, 0.0}, qi = zero;   // z_i^2 - 1
            ext_acc(qr, zi.re, zi.re);
            ext_acc(qr, -zi.im, zi.im);
            ext_acc(qi, 2.0 * zi.re, zi.im);
            ext<double> hr = zero, hi = zero;
            ext_acc_ext(hr, g1r, qr);
            ext_acc_ext(hr, -g1i, qi);
            ext_acc_ext(hr, s, pr);
            ext_acc_ext(hi, g1r, qi);
            ext_acc_ext(hi, g1i, qr);
            ext_acc_ext(hi, s, pi);
            if (wr) out.set(i, cx<double>{-ext_val(hr), -ext_val(hi)});
        }
    }

    // H_z d = r: r = -H_t (two_rhs false) or r1 = res and r2 = -H_t (two_rhs true)
    template <class Out2>
    static __device__ __forceinline__ bool solve_g(const Sys &S, const SMat<NV, double, BLOCK> &A,
                                                   const SVec<double, BLOCK> &pt, double s,
                                                   double omt, cx<double> gam, bool two_rhs,
                                                   const SVec<double, BLOCK> &res,
                                                   const SVec<double, BLOCK> &out1,
                                                   const Out2 &out2, bool wr,
                                                   double *kest = nullptr) {
        const cx<double> g2 = cscale(2.0 * omt, gam);
#pragma unroll 1
        for (int c = 0; c < NV; c++)
#pragma unroll 1
            for (int i = 0; i < NV; i++) A.set(i, c, cx<double>{0.0, 0.0});
#pragma unroll 1
        for (int i = 0; i < NV; i++) {
            const cx<double> zi = pt.get(i);
            A.set(i, i, cmul(g2, zi));
            cx<double> p = cx<double>{0.0, 0.0};
#pragma unroll 1
            for (int t = S.row[i]; t < S.row[i + 1]; t++) {
                const QTerm T = S.terms[t];
                const cx<double> c = cx<double>{T.cre, T.cim};
                const cx<double> wa = w(pt, T.a), wb = w(pt, T.b);
                p = cadd(p, cmul(c, cmul(wa, wb)));
                if (T.a >= 0) A.set(i, T.a, cadd(A.get(i, T.a), cscale(s, cmul(c, wb))));
                if (T.b >= 0) A.set(i, T.b, cadd(A.get(i, T.b), cscale(s, cmul(c, wa))));
            }
            // -H_t = gamma Q - P
            const cx<double> z2 = cmul(zi, zi);
            const cx<double> mht = csub(cmul(gam, cx<double>{z2.re - 1.0, z2.im}), p);
            A.set(i, NV, two_rhs ? res.get(i) : mht);
            if (two_rhs) A.set(i, NV + 1, mht);
        }
        const bool ok = aug_qr_solve<NV, double, BLOCK>(A, two_rhs, kest);
        double chk = 0.0;
#pragma unroll 1
        for (int i = 0; i < NV; i++) {
            const cx<double> d0 = A.get(i, NV);
            chk += cabs2(d0);
            if (two_rhs) {
                const cx<double> d1 = A.get(i, NV + 1);
                chk += cabs2(d1);
                if (wr) out2.set(i, d1);
            }
            if (wr) out1.set(i, d0);
        }
        return ok && isfinite(chk);
    }
};

// Endgame policy (see EGXY): P, DP dense from the terms, z in G's X.
template <int NV>
struct EGQuad {
    using Sys = QSys;
    static constexpr int DIM = NV;
    static constexpr int NZ = NV;
    static __device__ __forceinline__ cx<double> zget(const EG<NV> &G, int k) {
        return G.v(EGLayout<NV>::X).get(k);
    }
    static __device__ __forceinline__ void zset(const EG<NV> &G, int k, cx<double> v) {
        G.v(EGLayout<NV>::X).set(k, v);
    }
    static __device__ __forceinline__ double minus_p(const EG<NV> &G, const Sys &S) {
        const EGVec X = G.v(EGLayout<NV>::X), R = G.v(EGLayout<NV>::R);
        const ext<double> zero = {0.0, 0.0};
        double res = 0.0;
#pragma unroll 1
        for (int i = 0; i < NV; i++) {
            ext<double> pr = zero, pi = zero;
#pragma unroll 1
            for (int t = S.row[i]; t < S.row[i + 1]; t++) {
                const QTerm T = S.terms[t];
                const cx<double> wa = T.a < 0 ? cx<double>{1.0, 0.0} : X.get(T.a);
                const cx<double> wb = T.b < 0 ? cx<double>{1.0, 0.0} : X.get(T.b);
                ext<double> mr = zero, mi = zero;
                ext_acc(mr, wa.re, wb.re);
                ext_acc(mr, -wa.im, wb.im);
                ext_acc(mi, wa.re, wb.im);
                ext_acc(mi, wa.im, wb.re);
                ext_acc_ext(pr, T.cre, mr);
                ext_acc_ext(pr, -T.cim, mi);
                ext_acc_ext(pi, T.cre, mi);
                ext_acc_ext(pi, T.cim, mr);
            }
            const cx<double> p = cx<double>{ext_val(pr), ext_val(pi)};
            res = fmax(res, sqrt(cabs2(p)));
            R.set(i, cx<double>{-p.re, -p.im});
        }
        return res;
    }
    static __device__ __forceinline__ bool factor(const EG<NV> &G, const Sys &S) {
        const EGVec X = G.v(EGLayout<NV>::X);
#pragma unroll 1
        for (int c = 0; c < NV; c++)
#pragma unroll 1
            for (int i = 0; i < NV; i++) G.setS(i, c, cx<double>{0.0, 0.0});
#pragma unroll 1
        for (int i = 0; i < NV; i++) {
#pragma unroll 1
            for (int t = S.row[i]; t < S.row[i + 1]; t++) {
                const QTerm T = S.terms[t];
                const cx<double> c = cx<double>{T.cre, T.cim};
                const cx<double> wa = T.a < 0 ? cx<double>{1.0, 0.0} : X.get(T.a);
                const cx<double> wb = T.b < 0 ? cx<double>{1.0, 0.0} : X.get(T.b);
                if (T.a >= 0) G.setS(i, T.a, cadd(G.S(i, T.a), cmul(c, wb)));
                if (T.b >= 0) G.setS(i, T.b, cadd(G.S(i, T.b), cmul(c, wa)));
            }
        }
        // ||DP||_F, kept in the unused second half of R for jac_fro
        double f = 0.0;
#pragma unroll 1
        for (int c = 0; c < NV; c++)
#pragma unroll 1
            for (int i = 0; i < NV; i++) f += cabs2(G.S(i, c));
        G.v(EGLayout<NV>::R).set(NV, cx<double>{sqrt(f), 0.0});
        return eg_qr<NV>(G);
    }
    static __device__ __forceinline__ double jac_fro(const EG<NV> &G, const Sys &S) {
        return G.v(EGLayout<NV>::R).get(NV).re;
    }
    static __device__ __forceinline__ double solve(const EG<NV> &G, const Sys &S) {
        const EGVec R = G.v(EGLayout<NV>::R), Dv = G.v(EGLayout<NV>::D);
#pragma unroll 1
        for (int i = 0; i < NV; i++) Dv.set(i, R.get(i));
        return eg_schur_solve<NV>(G, Dv);
    }
    static __device__ __forceinline__ double inv_fro(const EG<NV> &G, const Sys &S) {
        const EGVec Dv = G.v(EGLayout<NV>::D);
        double s = 0.0;
#pragma unroll 1
        for (int j = 0; j < NV; j++) {
#pragma unroll 1
            for (int k = 0; k < NV; k++) Dv.set(k, cx<double>{k == j ? 1.0 : 0.0, 0.0});
            s += eg_schur_solve<NV>(G, Dv);
        }
        return sqrt(s);
    }
    static __device__ __forceinline__ double d2norm(const Sys &S) { return S.d2norm; }
};

template <int NV>
__global__ void __launch_bounds__(32)
    quad_track_kernel(const __grid_constant__ QSys S, const __grid_constant__ XYCtl C,
                      const EPView ep, const WorkList wl) {
    track_body<QuadProblem<NV>>(SingleSrc<QSys>{S, ep, wl}, C, wl);
}

template <int NV>
__global__ void __launch_bounds__(EG_BLOCK)
    quad_refine_certify_kernel(const __grid_constant__ QSys S, double tol_sol, double refine_eps,
                               int refine_iters, const EPView ep, const WorkList wl) {
    refine_body<EGQuad<NV>>(S, tol_sol, refine_eps, refine_iters, ep, wl, 0);
}

template <int NV>
__global__ void __launch_bounds__(32)
    quad_cauchy_kernel(const __grid_constant__ QSys S, const __grid_constant__ EGCtl C,
                       const EPView ep, const WorkList wl, int32_t *cyc, int32_t *egst) {
    cauchy_body<QuadProblem<NV>>(S, C, ep, wl, cyc, egst);
}
