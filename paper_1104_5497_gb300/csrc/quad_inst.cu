// quad_inst.cu -- the generic quadratic-system kernels for one system size per
// compilation.  Compiled with -DNPHC_QUAD_NV=<n> (unknowns, 1 .. NPHC_QUAD_MAX_N).
#include "quad.cuh"
#include "xy_dispatch.cuh"

namespace {

template <class K>
cudaError_t persistent_grid(K k, int block, size_t smem, int &grid) {
    static bool attr_set = false;   // once per process for this instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, block, smem);
    if (e != cudaSuccess) return e;
    grid = sms * (per > 0 ? per : 1);
    return cudaSuccess;
}

}  // namespace

cudaError_t NPHC_CAT(launch_quad_track_n, NPHC_QUAD_NV)(const QSys &sys, const XYCtl &ctl,
                                                        const EPView &ep, const WorkList &wl,
                                                        int grid, cudaStream_t st) {
    using P = QuadProblem<NPHC_QUAD_NV>;
    const size_t smem = track_smem_per_thread<P>() * P::BLOCK;
    auto k = quad_track_kernel<NPHC_QUAD_NV>;
    int full = 0;
    cudaError_t e = persistent_grid(k, P::BLOCK, smem, full);
    if (e != cudaSuccess) return e;
    if (grid <= 0 || grid > full) grid = full;
    const int cap = (int)(wl.state_threads / P::BLOCK);   // the scratch holds state for this many
    if (grid > cap) grid = cap;
    if (grid <= 0) return cudaErrorInvalidValue;
    k<<<grid, P::BLOCK, smem, st>>>(sys, ctl, ep, wl);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t NPHC_CAT(launch_quad_refine_certify_n, NPHC_QUAD_NV)(const QSys &sys, double tol_sol,
                                                                 double refine_eps,
                                                                 int refine_iters,
                                                                 const EPView &ep, int64_t cap,
                                                                 const WorkList &wl,
                                                                 cudaStream_t st) {
    if (cap <= 0) return cudaSuccess;
    const size_t smem = eg_smem_per_thread<NPHC_QUAD_NV>() * EG_BLOCK;
    auto k = quad_refine_certify_kernel<NPHC_QUAD_NV>;
    int full = 0;
    cudaError_t e = persistent_grid(k, EG_BLOCK, smem, full);
    if (e != cudaSuccess) return e;
    const int64_t need = (cap + EG_BLOCK - 1) / EG_BLOCK;
    const int grid = (int)(need < full ? need : full);
    WorkList w = wl;
    w.state = nullptr;   // S in shared memory (the launch is sized for it)
    k<<<grid, EG_BLOCK, smem, st>>>(sys, tol_sol, refine_eps, refine_iters, ep, w);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t NPHC_CAT(launch_quad_cauchy_n, NPHC_QUAD_NV)(const QSys &sys, const EGCtl &ctl,
                                                         const EPView &ep, const WorkList &wl,
                                                         int32_t *cyc, int32_t *egst,
                                                         cudaStream_t st) {
    using P = QuadProblem<NPHC_QUAD_NV>;
    if (ep.count <= 0) return cudaSuccess;
    const size_t smem = track_smem_per_thread<P>() * P::BLOCK;
    auto k = quad_cauchy_kernel<NPHC_QUAD_NV>;
    int full = 0;
    cudaError_t e = persistent_grid(k, P::BLOCK, smem, full);
    if (e != cudaSuccess) return e;
    const int64_t need = (ep.count + P::BLOCK - 1) / P::BLOCK;   // the list is at most ep.count long
    const int64_t cap = wl.state_threads / P::BLOCK;
    int64_t grid = need < full ? need : full;
    if (grid > cap) grid = cap;
    if (grid <= 0) return cudaErrorInvalidValue;
    k<<<(int)grid, P::BLOCK, smem, st>>>(sys, ctl, ep, wl, cyc, egst);
    nphc_launch_counter(1);
    return cudaGetLastError();
}
