// nphc_kernels.cu -- kernels that do not depend on the ring size: work-list
// compaction, deduplication of certified endpoints, and result counters.
#include "nphc_kernels.cuh"

// ------------------------------------------------------------- compaction --
__global__ void compact_kernel(const EPView ep, int pred, int32_t *flags, int32_t *list,
                               int32_t *count) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ep.count) return;
    bool take = false;
    if (pred == PRED_HANDOFF) {
        take = ep.status[e] == NPHC_PATH_HANDOFF;
        if (take) flags[e] |= FLAG_FP64_CONTINUED;
    } else if (pred == PRED_UNCERTIFIED_FP32) {
        take = ep.cls[e] == NPHC_END_SINGULAR && !(flags[e] & (FLAG_FP64_CONTINUED | FLAG_RETRACKED));
        if (take) flags[e] |= FLAG_RETRACKED;
    }
    if (take) list[atomicAdd(count, 1)] = (int32_t)e;
}

// Marks the entries of a list re-tracked (used for the duplicate re-track).
__global__ void flag_list_kernel(const int32_t *list, const int32_t *count, int32_t *flags,
                                 int32_t bit) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    flags[list[i]] |= bit;
}

// ------------------------------------------------------------------ dedup --
// Certified endpoints are rounded to a grid of pitch delta.  Two certified endpoints of
// one solution lie within 2 (beta_a + beta_b) of each other (each is within 2 beta of
// it), so when both betas are <= BETA_HASH and no coordinate lies within
// BAND = 4 BETA_HASH (< BAND_FRAC delta) of a cell boundary, they fall in the same cell.
// An endpoint that fails either condition is "ambiguous" and is compared with every
// certified endpoint instead (rare: ~2 n BAND_FRAC of the endpoints).  Cells live in an
// open-addressing table; inside a cell the alpha-theory test decides.

#define BETA_HASH 1e-12
#define BAND_FRAC 1e-5

__device__ __forceinline__ bool is_certified(int c) {
    return c == NPHC_END_REAL || c == NPHC_END_NONREAL || c == NPHC_END_UNDECIDED;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t cell_hash(const EPView &ep, int n, int64_t e, double inv_delta,
                                              bool &amb) {
    uint64_t hsh = 0x2545F4914F6CDD1Dull;
    amb = false;
    const int64_t cnt = ep.count;
    for (int i = 0; i < n; i++) {
        const double v[2] = {ep.z_re[i * cnt + e] * inv_delta, ep.z_im[i * cnt + e] * inv_delta};
        for (int p = 0; p < 2; p++) {
            const double r = rint(v[p]);
            if (fabs(v[p] - r) > 0.5 - BAND_FRAC) amb = true;
            hsh = mix64(hsh ^ (uint64_t)(long long)r);
        }
    }
    return hsh;
}

__device__ __forceinline__ bool same_cell(const EPView &ep, int n, int64_t a, int64_t b,
                                          double inv_delta) {
    const int64_t cnt = ep.count;
    for (int i = 0; i < n; i++) {
        if (rint(ep.z_re[i * cnt + a] * inv_delta) != rint(ep.z_re[i * cnt + b] * inv_delta)) return false;
        if (rint(ep.z_im[i * cnt + a] * inv_delta) != rint(ep.z_im[i * cnt + b] * inv_delta)) return false;
    }
    return true;
}

// alpha-theory: the same solution when alpha < 0.03 and ||za - zb|| < 1 / (20 gamma) for
// either point; a pair that is not provably distinct (||za - zb|| > 2 (beta_a + beta_b))
// counts as the same solution too.
__device__ __forceinline__ bool same_solution(const EPView &ep, int n, int64_t a, int64_t b) {
    const int64_t cnt = ep.count;
    double d2 = 0.0;
    for (int i = 0; i < n; i++) {
        const double dr = ep.z_re[i * cnt + a] - ep.z_re[i * cnt + b];
        const double di = ep.z_im[i * cnt + a] - ep.z_im[i * cnt + b];
        d2 += dr * dr + di * di;
    }
    const double d = sqrt(d2);
    const bool sa = ep.beta[a] * ep.gamma[a] < 0.03 && d * 20.0 * ep.gamma[a] < 1.0;
    const bool sb = ep.beta[b] * ep.gamma[b] < 0.03 && d * 20.0 * ep.gamma[b] < 1.0;
    const bool distinct = d > 2.0 * (ep.beta[a] + ep.beta[b]);
    return sa || sb || !distinct;
}

__global__ void dedup_insert_kernel(const EPView ep, int n, double inv_delta, DedupScratch w) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ep.count) return;
    w.rep[e] = -1;
    if (!is_certified(ep.cls[e])) return;
    bool amb;
    const uint64_t hsh = cell_hash(ep, n, e, inv_delta, amb);
    if (amb || !(ep.beta[e] <= BETA_HASH)) {
        w.amb[e] = 1;
        return;
    }
    const uint64_t mask = (uint64_t)w.table_size - 1;
    uint64_t slot = hsh & mask;
    int32_t rep = -1;
    for (int64_t probe = 0; probe < w.table_size; probe++) {
        int32_t cur = w.table[slot];
        if (cur == -1) {
            const int32_t prev = atomicCAS(&w.table[slot], -1, (int32_t)e);
            if (prev == -1) {
                rep = (int32_t)e;
                break;
            }
            cur = prev;
        }
        if (same_cell(ep, n, cur, e, inv_delta) && same_solution(ep, n, cur, e)) {
            rep = cur;
            break;
        }
        slot = (slot + 1) & mask;
    }
    w.rep[e] = rep;
    if (rep >= 0) {
        atomicMin(reinterpret_cast<unsigned long long *>(&w.minpath[rep]),
                  (unsigned long long)ep.path[e]);
        atomicAdd(&w.gsize[rep], 1);
    }
}

__device__ __forceinline__ void push_once(DedupScratch &w, int32_t *list, int32_t *count,
                                          int64_t e) {
    if (atomicExch(&w.inlist[e], 1) == 0 && list) list[atomicAdd(count, 1)] = (int32_t)e;
}

__global__ void dedup_resolve_kernel(const EPView ep, DedupScratch w, int32_t *list,
                                     int32_t *count) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ep.count) return;
    const int32_t r = w.rep[e];
    if (r < 0) return;
    if (w.gsize[r] > 1) {
        if ((unsigned long long)ep.path[e] != (unsigned long long)w.minpath[r])
            ep.cls[e] = NPHC_END_DUPLICATE;
        push_once(w, list, count, e);
    }
}

// Ambiguous endpoints: compared with every certified endpoint.
__global__ void dedup_ambiguous_kernel(const EPView ep, int n, DedupScratch w, int32_t *list,
                                       int32_t *count) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ep.count || !w.amb[e]) return;
    for (int64_t j = 0; j < ep.count; j++) {
        if (j == e || !is_certified(ep.cls[j])) continue;
        if (!same_solution(ep, n, e, j)) continue;
        if (ep.path[j] < ep.path[e])
            ep.cls[e] = NPHC_END_DUPLICATE;
        else
            ep.cls[j] = NPHC_END_DUPLICATE;
        push_once(w, list, count, e);
        push_once(w, list, count, j);
    }
}

// ---------------------------------------------------------------- counters --
__global__ void counts_kernel(const EPView ep, const int32_t *flags, const int32_t *index,
                              int64_t *counts) {
    __shared__ unsigned long long loc[NPHC_NCOUNTS];
    for (int i = threadIdx.x; i < NPHC_NCOUNTS; i += blockDim.x) loc[i] = 0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ep.count) {
        atomicAdd(&loc[NPHC_COUNT_PATHS], 1ull);
        const int st = ep.status[e];
        if (st == NPHC_PATH_REACHED) atomicAdd(&loc[NPHC_COUNT_REACHED], 1ull);
        else if (st == NPHC_PATH_DIVERGED) atomicAdd(&loc[NPHC_COUNT_DIVERGED], 1ull);
        else atomicAdd(&loc[NPHC_COUNT_FAILED], 1ull);
        const int c = ep.cls[e];
        if (c == NPHC_END_REAL) atomicAdd(&loc[NPHC_COUNT_REAL], 1ull);
        else if (c == NPHC_END_NONREAL) atomicAdd(&loc[NPHC_COUNT_NONREAL], 1ull);
        else if (c == NPHC_END_UNDECIDED) atomicAdd(&loc[NPHC_COUNT_UNDECIDED], 1ull);
        else if (c == NPHC_END_SINGULAR) atomicAdd(&loc[NPHC_COUNT_SINGULAR], 1ull);
        else if (c == NPHC_END_DUPLICATE) atomicAdd(&loc[NPHC_COUNT_DUPLICATE], 1ull);
        if (flags) {
            if (flags[e] & FLAG_FP64_CONTINUED) atomicAdd(&loc[NPHC_COUNT_HANDOFF], 1ull);
            if (flags[e] & (FLAG_RETRACKED | FLAG_RETRACKED_DUP)) atomicAdd(&loc[NPHC_COUNT_RETRACKED], 1ull);
        }
        atomicAdd(&loc[NPHC_COUNT_SOLVES], (unsigned long long)ep.solves[e]);
        if (c == NPHC_END_REAL && index) {
            const int ix = index[e];
            if (ix >= 0 && ix < NPHC_MAX_N - 1) atomicAdd(&loc[NPHC_COUNT_INDEX0 + ix], 1ull);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NPHC_NCOUNTS; i += blockDim.x)
        if (loc[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&counts[i]), loc[i]);
}

// Compacts the real stationary points (entry indices) for the copy-out.
__global__ void real_list_kernel(const EPView ep, int32_t *list, int32_t *count) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ep.count) return;
    if (ep.cls[e] == NPHC_END_REAL) list[atomicAdd(count, 1)] = (int32_t)e;
}

__global__ void iota_kernel(int64_t *path, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) path[e] = e;
}

__global__ void gather_sps_kernel(const EPView ep, int M, const int32_t *list, const int32_t *count,
                                  const double *theta, const int32_t *index, const double *energy,
                                  double *o_theta, int32_t *o_index, double *o_energy,
                                  double *o_alpha, int64_t *o_path) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const int64_t e = list[i];
    const int64_t cnt = ep.count;
    for (int k = 0; k < M; k++) o_theta[i * M + k] = theta[k * cnt + e];
    o_index[i] = index[e];
    o_energy[i] = energy[e];
    o_alpha[i] = ep.alpha[e];
    o_path[i] = ep.path[e];
}

// ------------------------------------------------------------- launchers --
static inline int blocks_for(int64_t n, int b) { return (int)((n + b - 1) / b); }

cudaError_t launch_compact(const EPView &ep, int pred, int32_t *flags, int32_t *list,
                           int32_t *count, cudaStream_t st) {
    if (ep.count == 0) return cudaSuccess;
    compact_kernel<<<blocks_for(ep.count, 256), 256, 0, st>>>(ep, pred, flags, list, count);
    return cudaGetLastError();
}

cudaError_t launch_flag_list(const int32_t *list, const int32_t *count, int64_t cap,
                             int32_t *flags, int32_t bit, cudaStream_t st) {
    if (cap == 0) return cudaSuccess;
    flag_list_kernel<<<blocks_for(cap, 256), 256, 0, st>>>(list, count, flags, bit);
    return cudaGetLastError();
}

cudaError_t launch_dedup(const EPView &ep, int n, double delta, DedupScratch w, int32_t *list,
                         int32_t *count, cudaStream_t st) {
    if (ep.count == 0) return cudaSuccess;
    cudaError_t err;
    if ((err = cudaMemsetAsync(w.table, 0xff, sizeof(int32_t) * w.table_size, st))) return err;
    if ((err = cudaMemsetAsync(w.minpath, 0xff, sizeof(int64_t) * ep.count, st))) return err;
    if ((err = cudaMemsetAsync(w.gsize, 0, sizeof(int32_t) * ep.count, st))) return err;
    if ((err = cudaMemsetAsync(w.amb, 0, sizeof(int32_t) * ep.count, st))) return err;
    if ((err = cudaMemsetAsync(w.inlist, 0, sizeof(int32_t) * ep.count, st))) return err;
    if (count && (err = cudaMemsetAsync(count, 0, sizeof(int32_t), st))) return err;
    const int g = blocks_for(ep.count, 256);
    dedup_insert_kernel<<<g, 256, 0, st>>>(ep, n, 1.0 / delta, w);
    dedup_resolve_kernel<<<g, 256, 0, st>>>(ep, w, list, count);
    dedup_ambiguous_kernel<<<g, 256, 0, st>>>(ep, n, w, list, count);
    return cudaGetLastError();
}

cudaError_t launch_counts(const EPView &ep, const int32_t *flags, const int32_t *index,
                          int64_t *counts, cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(counts, 0, sizeof(int64_t) * NPHC_NCOUNTS, st);
    if (err || ep.count == 0) return err;
    counts_kernel<<<blocks_for(ep.count, 256), 256, 0, st>>>(ep, flags, index, counts);
    return cudaGetLastError();
}

cudaError_t launch_real_list(const EPView &ep, int32_t *list, int32_t *count, cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
    if (err || ep.count == 0) return err;
    real_list_kernel<<<blocks_for(ep.count, 256), 256, 0, st>>>(ep, list, count);
    return cudaGetLastError();
}

cudaError_t launch_iota(int64_t *path, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    iota_kernel<<<blocks_for(n, 256), 256, 0, st>>>(path, n);
    return cudaGetLastError();
}

cudaError_t launch_gather_sps(const EPView &ep, int M, const int32_t *list, const int32_t *count,
                              int64_t cap, const double *theta, const int32_t *index,
                              const double *energy, double *o_theta, int32_t *o_index,
                              double *o_energy, double *o_alpha, int64_t *o_path, cudaStream_t st) {
    if (cap == 0) return cudaSuccess;
    gather_sps_kernel<<<blocks_for(cap, 256), 256, 0, st>>>(ep, M, list, count, theta, index, energy,
                                                          o_theta, o_index, o_energy, o_alpha, o_path);
    return cudaGetLastError();
}
