// xy_dispatch.cu -- runtime ring size -> kernel instantiated for it.
#include "xy_dispatch.cuh"

cudaError_t launch_xy_track_f32(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                const WorkList &wl, int block, int grid, cudaStream_t st) {
    (void)block;
#define C(MM) case MM: return launch_xy_track_f32_m##MM(sys, ctl, ep, wl, grid, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_xy_track_f32_batch(int M, const BatchGroup &bg, const XYCtl &ctl,
                                      const WorkList &wl, int grid, cudaStream_t st) {
#define C(MM) case MM: return launch_xy_track_f32_batch_m##MM(bg, ctl, wl, grid, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_xy_track_f64(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                const WorkList &wl, int block, int grid, cudaStream_t st) {
    (void)block;
#define C(MM) case MM: return launch_xy_track_f64_m##MM(sys, ctl, ep, wl, grid, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_xy_track_f64_warp_bps(int M, const XYSys &sys, const XYCtl &ctl,
                                         const EPView &ep, const WorkList &wl, int blocks_per_sm,
                                         cudaStream_t st) {
#define C(MM) case MM: return launch_xy_track_f64w_m##MM(sys, ctl, ep, wl, blocks_per_sm, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_xy_track_f64_warp(int M, const XYSys &sys, const XYCtl &ctl, const EPView &ep,
                                     const WorkList &wl, cudaStream_t st) {
    return launch_xy_track_f64_warp_bps(M, sys, ctl, ep, wl, 0, st);
}

cudaError_t launch_xy_refine_certify(int M, const XYSys &sys, double tol_sol, double refine_eps,
                                     int refine_iters, const EPView &ep, int64_t cap,
                                     const WorkList &wl, int shortcut, cudaStream_t st) {
#define C(MM) case MM: return launch_xy_refine_certify_m##MM(sys, tol_sol, refine_eps, refine_iters, ep, cap, wl, shortcut, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_xy_adjoint(int M, const XYSys &sys, int64_t count, const double *theta,
                              const double *g_energy, const double *g_theta, double *dJ,
                              cudaStream_t st) {
#define C(MM) case MM: return launch_xy_adjoint_m##MM(sys, count, theta, g_energy, g_theta, dJ, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_xy_classify(int M, const XYSys &sys, const EPView &ep, double *theta,
                               int32_t *index, double *energy, double *min_eig,
                               double *log_abs_det, cudaStream_t st, const int32_t *list,
                               const int32_t *list_count) {
#define C(MM) case MM: return launch_xy_classify_m##MM(sys, ep, theta, index, energy, min_eig, log_abs_det, list, list_count, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

int xy_track_f32_block(int M) { (void)M; return NPHC_TRACK_BLOCK; }
int xy_track_f64_block(int M) { (void)M; return NPHC_TRACK_BLOCK; }

cudaError_t launch_quad_track(int n, const QSys &sys, const XYCtl &ctl, const EPView &ep,
                              const WorkList &wl, int grid, cudaStream_t st) {
#define C(NN) case NN: return launch_quad_track_n##NN(sys, ctl, ep, wl, grid, st);
    switch (n) { NPHC_FOR_EACH_QN(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_quad_refine_certify(int n, const QSys &sys, double tol_sol, double refine_eps,
                                       int refine_iters, const EPView &ep, int64_t cap,
                                       const WorkList &wl, cudaStream_t st) {
#define C(NN) case NN: return launch_quad_refine_certify_n##NN(sys, tol_sol, refine_eps, refine_iters, ep, cap, wl, st);
    switch (n) { NPHC_FOR_EACH_QN(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_xy_cauchy(int M, const XYSys &sys, const EGCtl &ctl, const EPView &ep,
                             const WorkList &wl, int32_t *cyc, int32_t *egst, cudaStream_t st) {
#define C(MM) case MM: return launch_xy_cauchy_m##MM(sys, ctl, ep, wl, cyc, egst, st);
    switch (M) { NPHC_FOR_EACH_M(C) default: return cudaErrorInvalidValue; }
#undef C
}

cudaError_t launch_quad_cauchy(int n, const QSys &sys, const EGCtl &ctl, const EPView &ep,
                               const WorkList &wl, int32_t *cyc, int32_t *egst, cudaStream_t st) {
#define C(NN) case NN: return launch_quad_cauchy_n##NN(sys, ctl, ep, wl, cyc, egst, st);
    switch (n) { NPHC_FOR_EACH_QN(C) default: return cudaErrorInvalidValue; }
#undef C
}
