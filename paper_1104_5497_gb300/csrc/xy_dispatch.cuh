// xy_dispatch.cuh -- declarations of the per-size launchers and the runtime dispatch.
#pragma once

#include "nphc_internal.cuh"

#define NPHC_CAT2(a, b) a##b
#define NPHC_CAT(a, b) NPHC_CAT2(a, b)

#define NPHC_TRACK_BLOCK 32   // one warp per block: per-thread shared memory, no block sync
#define NPHC_M_MIN 2
#define NPHC_M_MAX 12
#define NPHC_FOR_EACH_M(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

#define NPHC_DECL(MM)                                                                         \
    cudaError_t launch_xy_track_f32_m##MM(const XYSys &, const XYCtl &, const EPView &,     \
                                          const WorkList &, int, cudaStream_t);              \
    cudaError_t launch_xy_track_f32_batch_m##MM(const BatchGroup &, const XYCtl &,          \
                                                const WorkList &, int, cudaStream_t);        \
    cudaError_t launch_xy_track_f64_m##MM(const XYSys &, const XYCtl &, const EPView &,     \
                                          const WorkList &, int, cudaStream_t);              \
    cudaError_t launch_xy_track_f64w_m##MM(const XYSys &, const XYCtl &, const EPView &,    \
                                           const WorkList &, int, cudaStream_t);            \
    cudaError_t launch_xy_refine_certify_m##MM(const XYSys &, double, double, int,          \
                                               const EPView &, int64_t, const WorkList &,   \
                                               int, cudaStream_t);                          \
    cudaError_t launch_xy_adjoint_m##MM(const XYSys &, int64_t, const double *, const double *, \
                                        const double *, double *, cudaStream_t);              \
    cudaError_t launch_xy_classify_m##MM(const XYSys &, const EPView &, double *, int32_t *, \
                                         double *, double *, double *, const int32_t *,      \
                                         const int32_t *, cudaStream_t);                      \
    cudaError_t launch_xy_cauchy_m##MM(const XYSys &, const EGCtl &, const EPView &,        \
                                       const WorkList &, int32_t *, int32_t *, cudaStream_t);
NPHC_FOR_EACH_M(NPHC_DECL)
#undef NPHC_DECL

#define NPHC_FOR_EACH_QN(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)
#define NPHC_QDECL(NN)                                                                        \
    cudaError_t launch_quad_track_n##NN(const QSys &, const XYCtl &, const EPView &,         \
                                        const WorkList &, int, cudaStream_t);                 \
    cudaError_t launch_quad_refine_certify_n##NN(const QSys &, double, double, int,          \
                                                 const EPView &, int64_t, const WorkList &,  \
                                                 cudaStream_t);                               \
    cudaError_t launch_quad_cauchy_n##NN(const QSys &, const EGCtl &, const EPView &,        \
                                         const WorkList &, int32_t *, int32_t *, cudaStream_t);
NPHC_FOR_EACH_QN(NPHC_QDECL)
#undef NPHC_QDECL

// The FP64 list tracker with a chosen number of blocks per SM (0: automatic); the
// launcher of nphc_internal.cuh is this one with 0.
cudaError_t launch_xy_track_f64_warp_bps(int M, const XYSys &sys, const XYCtl &ctl,
                                         const EPView &ep, const WorkList &wl, int blocks_per_sm,
                                         cudaStream_t st);
