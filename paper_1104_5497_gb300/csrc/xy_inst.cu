// xy_inst.cu -- one ring size of one kernel family per compilation, so that the build
// compiles the heavily unrolled kernels in parallel.  Compiled with
//   -DNPHC_INST_M=<M>  (free sites, N = M + 1)
//   -DNPHC_INST_KIND=0 (FP32 tracker), 1 (FP64 tracker), 2 (FP64 refinement,
//   certification, classification, adjoint) or 3 (Cauchy endgame)
#include "xy_dispatch.cuh"

#if NPHC_INST_KIND == 3
#include "cauchy_warp.cuh"

// one path per warp, 4 warps per block
cudaError_t NPHC_CAT(launch_xy_cauchy_m, NPHC_INST_M)(const XYSys &sys, const EGCtl &ctl,
                                                      const EPView &ep, const WorkList &wl,
                                                      int32_t *cyc, int32_t *egst,
                                                      cudaStream_t st) {
    constexpr int M = NPHC_INST_M, WARPS = 4;
    if (ep.count <= 0) return cudaSuccess;
    const size_t smem = cauchy_warp_smem_per_warp<M>() * WARPS;
    auto k = xy_cauchy_warp_kernel<M, WARPS>;
    static bool attr_set = false;   // once per process for this instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 32 * WARPS, smem);
    if (e != cudaSuccess) return e;
    const int64_t full = (int64_t)sms * (per > 0 ? per : 1);
    const int64_t need = (ep.count + WARPS - 1) / WARPS;   // the list is at most ep.count long
    const int grid = (int)(need < full ? need : full);
    k<<<grid, 32 * WARPS, smem, st>>>(sys, ctl, ep, wl, cyc, egst);
    nphc_launch_counter(1);
    return cudaGetLastError();
}
#endif

#if NPHC_INST_KIND == 0 || NPHC_INST_KIND == 1
#include "xy_track.cuh"
#if NPHC_INST_KIND == 1
#include "xy_track_warp.cuh"

// one path per warp (short FP64 lists), 4 warps per block, blocks_per_sm blocks per SM
// (0: two)
cudaError_t NPHC_CAT(launch_xy_track_f64w_m, NPHC_INST_M)(const XYSys &sys, const XYCtl &ctl,
                                                          const EPView &ep, const WorkList &wl,
                                                          int blocks_per_sm, cudaStream_t st) {
    constexpr int M = NPHC_INST_M, WARPS = 4;
    if (ep.count <= 0) return cudaSuccess;
    const size_t smem = warp_track_smem_per_warp<M>() * WARPS;
    auto k = xy_track_warp64_kernel<M, WARPS>;
    static bool attr_set = false;   // once per process for this instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 32 * WARPS, smem);
    if (e != cudaSuccess) return e;
    // by default two blocks (8 warps) per SM, each warp pulling paths until the list is
    // drained: the FP64 pipe is already busy at 8 warps, and with more warps than paths
    // each warp would take at most one path, whose SM is then chance (some SMs got twice
    // the mean and the others idled half the launch)
    const int want = blocks_per_sm > 0 ? blocks_per_sm : 2;
    const int64_t full = (int64_t)sms * (per < want ? (per > 0 ? per : 1) : want);
    const int64_t need = (ep.count + WARPS - 1) / WARPS;   // the list is at most ep.count long
    const int grid = (int)(need < full ? need : full);
    k<<<grid, 32 * WARPS, smem, st>>>(sys, ctl, ep, wl);
    nphc_launch_counter(1);
    return cudaGetLastError();
}
#endif

#if NPHC_INST_KIND == 0
using RT = float;
constexpr int BLK = NPHC_TRACK_BLOCK;
#define NPHC_FN NPHC_CAT(launch_xy_track_f32_m, NPHC_INST_M)
#else
using RT = double;
constexpr int BLK = NPHC_TRACK_BLOCK;
#define NPHC_FN NPHC_CAT(launch_xy_track_f64_m, NPHC_INST_M)
#endif

cudaError_t NPHC_FN(const XYSys &sys, const XYCtl &ctl, const EPView &ep, const WorkList &wl,
                    int grid, cudaStream_t st) {
    constexpr int M = NPHC_INST_M;
    const size_t smem = xy_smem_per_thread<M, RT>() * BLK;
    auto k = xy_track_kernel<M, RT, BLK>;
    static bool attr_set = false;   // once per process for this instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BLK, smem);
    if (e != cudaSuccess) return e;
    const int full = sms * (per > 0 ? per : 1);   // persistent grid: every SM filled
    if (grid <= 0 || grid > full) grid = full;
    const int cap = (int)(wl.state_threads / BLK);  // the scratch holds state for this many
    if (grid > cap) grid = cap;
    if (grid <= 0) return cudaErrorInvalidValue;
    k<<<grid, BLK, smem, st>>>(sys, ctl, ep, wl);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

#if NPHC_INST_KIND == 0
// The FP32 pass of a batch group: one persistent grid over every path of the group's
// instances (one queue), at most every SM filled.
cudaError_t NPHC_CAT(launch_xy_track_f32_batch_m, NPHC_INST_M)(const BatchGroup &bg,
                                                               const XYCtl &ctl,
                                                               const WorkList &wl, int grid,
                                                               cudaStream_t st) {
    constexpr int M = NPHC_INST_M;
    if (bg.total <= 0) return cudaSuccess;
    const size_t smem = xy_smem_per_thread<M, RT>() * BLK;
    auto k = xy_track_batch_kernel<M, RT, BLK>;
    static bool attr_set = false;   // once per process for this instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BLK, smem);
    if (e != cudaSuccess) return e;
    const int full = sms * (per > 0 ? per : 1);
    if (grid <= 0 || grid > full) grid = full;
    const int64_t need = (bg.total + BLK - 1) / BLK;   // no more threads than paths
    if (grid > need) grid = (int)need;
    const int cap = (int)(wl.state_threads / BLK);
    if (grid > cap) grid = cap;
    if (grid <= 0) return cudaErrorInvalidValue;
    k<<<grid, BLK, smem, st>>>(bg.sys, bg.ep, bg.off, bg.n, ctl, wl);
    nphc_launch_counter(1);
    return cudaGetLastError();
}
#endif

#elif NPHC_INST_KIND == 2
#include "xy_endgame.cuh"

cudaError_t NPHC_CAT(launch_xy_refine_certify_m, NPHC_INST_M)(const XYSys &sys, double tol_sol,
                                                             double refine_eps, int refine_iters,
                                                             const EPView &ep, int64_t cap,
                                                             const WorkList &wl, int shortcut,
                                                             cudaStream_t st) {
    if (cap <= 0) return cudaSuccess;
    constexpr int M = NPHC_INST_M;
    // with a scratch buffer (wl.state, wl.state_threads threads) S lives there and the
    // shared memory holds the rest only
    const bool gs = wl.state != nullptr && wl.state_threads >= EG_BLOCK;
    const size_t smem = eg_smem_per_thread<M>(!gs) * EG_BLOCK;
    auto k = xy_refine_certify_kernel<M>;
    static bool attr_set = false;   // once per process for this instantiation (the larger size)
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(eg_smem_per_thread<M>() * EG_BLOCK));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, EG_BLOCK, smem);
    if (e != cudaSuccess) return e;
    // grid-stride over the entries: at most every SM filled, at most one entry per thread,
    // and no more threads than the scratch buffer holds
    const int64_t need = (cap + EG_BLOCK - 1) / EG_BLOCK;
    int64_t full = (int64_t)sms * (per > 0 ? per : 1);
    if (gs && full > wl.state_threads / EG_BLOCK) full = wl.state_threads / EG_BLOCK;
    const int grid = (int)(need < full ? need : full);
    WorkList w = wl;
    if (!gs) w.state = nullptr;
    k<<<grid, EG_BLOCK, smem, st>>>(sys, tol_sol, refine_eps, refine_iters, ep, w, shortcut);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t NPHC_CAT(launch_xy_adjoint_m, NPHC_INST_M)(const XYSys &sys, int64_t count,
                                                      const double *theta, const double *g_energy,
                                                      const double *g_theta, double *dJ,
                                                      cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int grid = (int)((count + 127) / 128);
    xy_adjoint_kernel<NPHC_INST_M><<<grid, 128, 0, st>>>(sys, count, theta, g_energy, g_theta, dJ);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t NPHC_CAT(launch_xy_classify_m, NPHC_INST_M)(const XYSys &sys, const EPView &ep,
                                                       double *theta, int32_t *index,
                                                       double *energy, double *min_eig,
                                                       double *log_abs_det, const int32_t *list,
                                                       const int32_t *list_count,
                                                       cudaStream_t st) {
    if (ep.count <= 0) return cudaSuccess;
    // a list is at most ep.count long (its length is on the device)
    const int grid = (int)((ep.count + 127) / 128);
    xy_classify_kernel<NPHC_INST_M><<<grid, 128, 0, st>>>(sys, ep, theta, index, energy, min_eig,
                                                                   log_abs_det, list, list_count);
    nphc_launch_counter(1);
    return cudaGetLastError();
}
#endif
