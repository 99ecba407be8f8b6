// nphc_kernels.cu -- kernels that do not depend on the ring size: work-list
// compaction, deduplication of certified endpoints, and result counters.
#include "nphc_kernels.cuh"

#include <atomic>

#ifdef NPHC_DEBUG
__device__ int nphc_dbg_error = 0;   // the first failed index check's code (debug build)

cudaError_t nphc_debug_read(int *code) {
    cudaError_t e = cudaMemcpyFromSymbol(code, nphc_dbg_error, sizeof(int));
    if (e != cudaSuccess) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(nphc_dbg_error, &zero, sizeof(int));
}
#else
cudaError_t nphc_debug_read(int *code) {
    *code = -1;   // a release build has no checks
    return cudaSuccess;
}
#endif

int64_t nphc_launch_counter(int64_t add) {
    static std::atomic<int64_t> n{0};
    return n.fetch_add(add) + add;
}

// ------------------------------------------------------------- compaction --
__global__ void compact_kernel(const EPView ep, int pred, int32_t *flags, int32_t *list,
                               int32_t *count) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ep.count) return;
    bool take = false;
    if (pred == PRED_HANDOFF) {
        const int st = ep.status[e];
        take = st == NPHC_PATH_HANDOFF || st == NPHC_PATH_HANDOFF_COND;
        if (take) flags[e] |= FLAG_FP64_CONTINUED | (st == NPHC_PATH_HANDOFF_COND ? FLAG_COND : 0);
    } else if (pred == PRED_UNCERTIFIED_FP32) {
        // FP32 endpoints that do not certify are tracked again from t = 0 in FP64 (hand-offs
        // already continued in FP64 from where they entered the end zone)
        take = ep.cls[e] == NPHC_END_SINGULAR && !(flags[e] & (FLAG_FP64_CONTINUED | FLAG_RETRACKED));
        if (take) flags[e] |= FLAG_RETRACKED;
    } else if (pred == PRED_ENDGAME) {
        // endpoints for the Cauchy endgame: finite but not certified, or tracking failed
        const int c = ep.cls[e];
        take = c == NPHC_END_SINGULAR || c == NPHC_END_FAILED;
    } else if (pred == PRED_REACHED || pred == PRED_REACHED_DIRECT || pred == PRED_REACHED_CONTINUED) {
        // endpoints to refine; every other path gets its final class here.  The split forms
        // touch only the entries on their side of the hand-off flag (the other side may be
        // in flight on another stream)
        const bool cont = (flags[e] & FLAG_FP64_CONTINUED) != 0;
        if (pred == PRED_REACHED || cont == (pred == PRED_REACHED_CONTINUED)) {
            const int st = ep.status[e];
            take = st == NPHC_PATH_REACHED;
            if (!take) {
                ep.cls[e] = st == NPHC_PATH_DIVERGED ? NPHC_END_NONE : NPHC_END_FAILED;
                ep.alpha[e] = ep.beta[e] = ep.gamma[e] = ep.resid[e] = INFINITY;
            }
        }
    }
    if (take) {
        const int32_t k = atomicAdd(count, 1);
        if (NPHC_VALID(k < ep.count, 2)) list[k] = (int32_t)e;
    }
}

// Marks the entries of a list re-tracked (used for the duplicate re-track).
__global__ void flag_list_kernel(const int32_t *list, const int32_t *count, int32_t *flags,
                                 int32_t bit, int64_t cap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const int64_t e = list[i];
    (void)cap;
    if (NPHC_VALID(e >= 0 && e < cap, 1)) flags[e] |= bit;
}

// ------------------------------------------------------------------ dedup --
// Two certified endpoints of one solution lie within 2 (beta_a + beta_b) of each other
// (each is within 2 beta of it).  Candidates are found through grids on four
// coordinates at DD_LEVELS pitches delta_L = delta_0 100^L: the projections of the point
// (Re z, Im z) in R^(2n) onto four fixed pseudo-random unit vectors.  A projection onto a
// unit vector moves by at most the distance between two points, so every bound below
// holds for them as for single coordinates; projections of the whole point, unlike
// (c_1, s_1), do not put the many solutions that the ring's symmetries give equal first
// coordinates into one cell (on the N = 9 ring up to 48 per cell, each pair then compared
// in FP64).
// Every hashed endpoint is listed under its cell at every level; an endpoint e looks up
// level L(e), the finest with 4 beta_e <= DD_BAND delta_L, in its own cell plus, in
// each coordinate within DD_BAND cells of a boundary, the neighbour across it.  A copy
// o with beta_o <= beta_e lies within 4 beta_e of e, so e finds it; a copy with a larger
// beta finds e at its own level.  Each match marks the higher path index a duplicate,
// so the lowest path of every solution keeps its class.  The alpha-theory test decides
// each candidate pair.  Endpoints whose beta exceeds the coarsest level are compared
// with every certified endpoint instead.
#define DD_BAND 0.05

__device__ __forceinline__ bool is_certified(int c) {
    return c == NPHC_END_REAL || c == NPHC_END_NONREAL || c == NPHC_END_UNDECIDED;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double dd_pitch(double delta0, int level) {
    double d = delta0;
    for (int l = 0; l < level; l++) d *= 100.0;
    return d;
}

// The projections' weights, fixed pseudo-random numbers in [-1, 1) (splitmix64 of (i, r),
// r = 2k: Re z_k, 2k + 1: Im z_k), and the prefix sums of their squares that normalise a
// projection over the first 2n real coordinates; built at compile time.  A point has at
// most DD_MAXR real coordinates (24 unknowns: the N = 13 ring).
#define DD_MAXR 48
struct DDTable {
    double w[4][DD_MAXR];
    double n2[4][DD_MAXR + 1];
};
constexpr uint64_t dd_splitmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
constexpr DDTable dd_make_table() {
    DDTable t{};
    for (int i = 0; i < 4; i++) {
        t.n2[i][0] = 0.0;
        for (int r = 0; r < DD_MAXR; r++) {
            const uint64_t h = dd_splitmix(0x5851F42D4C957F2Dull ^ ((uint64_t)i << 32) ^ (uint64_t)r);
            const double w = (double)(int64_t)h * (1.0 / 9223372036854775808.0);
            t.w[i][r] = w;
            t.n2[i][r + 1] = t.n2[i][r] + w * w;
        }
    }
    return t;
}
__constant__ DDTable dd_tab = dd_make_table();

// The four grid coordinates of entry e at pitch 1: its projections onto the four unit
// vectors (the weights over the 2n real coordinates, normalised).
__device__ __forceinline__ void dd_project(const EPView &ep, int n, int64_t e, double (&u)[4]) {
    const int64_t cnt = ep.count;
    double dot[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < n; k++) {
        const double re = ep.z_re[k * cnt + e], im = ep.z_im[k * cnt + e];
#pragma unroll
        for (int i = 0; i < 4; i++)
            dot[i] = fma(dd_tab.w[i][2 * k], re, fma(dd_tab.w[i][2 * k + 1], im, dot[i]));
    }
#pragma unroll
    for (int i = 0; i < 4; i++) u[i] = dot[i] / sqrt(dd_tab.n2[i][2 * n]);
}

__device__ __forceinline__ uint64_t dd_cell_key(int level, const long long (&q)[4]) {
    uint64_t h = 0x2545F4914F6CDD1Dull ^ (uint64_t)level;
    for (int i = 0; i < 4; i++) h = mix64(h ^ (uint64_t)q[i]);
    return h | 1ull;   // 0 marks an empty slot
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

// finest level at which e's copies with smaller beta are within the band; DD_LEVELS if none
__device__ __forceinline__ int dd_level(double beta, double delta0) {
    for (int L = 0; L < DD_LEVELS; L++)
        if (4.0 * beta <= DD_BAND * dd_pitch(delta0, L)) return L;
    return DD_LEVELS;
}

// phase 1: list every certified endpoint under its cell at every level
__global__ void dedup_insert_kernel(const EPView ep, int n, double delta0, DedupScratch w) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ep.count) return;
    for (int L = 0; L < DD_LEVELS; L++) w.next[L * ep.count + e] = -1;
    if (!is_certified(ep.cls[e])) return;
    const uint64_t mask = (uint64_t)w.table_size - 1;
    double u[4];
    dd_project(ep, n, e, u);
    for (int L = 0; L < DD_LEVELS; L++) {
        const double inv = 1.0 / dd_pitch(delta0, L);
        long long q[4];
        for (int i = 0; i < 4; i++) q[i] = (long long)floor(u[i] * inv);
        const unsigned long long key = dd_cell_key(L, q);
        unsigned long long *keys = w.keys + L * w.table_size;
        int32_t *head = w.head + L * w.table_size;
        uint64_t slot = key & mask;
        for (int64_t probe = 0; probe < w.table_size; probe++) {
            const unsigned long long cur = atomicCAS(&keys[slot], 0ull, key);
            if (cur == 0ull || cur == key) {
                w.next[L * ep.count + e] = atomicExch(&head[slot], (int32_t)e);
                break;
            }
            slot = (slot + 1) & mask;
        }
    }
}

__device__ __forceinline__ void push_once(DedupScratch &w, int32_t *list, int32_t *count,
                                          int64_t e, int64_t cap) {
    if (atomicExch(&w.inlist[e], 1) == 0 && list) {
        const int32_t k = atomicAdd(count, 1);
        (void)cap;
        if (NPHC_VALID(k < cap, 2)) list[k] = (int32_t)e;
    }
}

__device__ __forceinline__ void dd_pair(const EPView &ep, DedupScratch &w, int32_t *list,
                                        int32_t *count, int64_t e, int64_t o) {
    if (ep.path[o] < ep.path[e])
        ep.cls[e] = NPHC_END_DUPLICATE;
    else
        ep.cls[o] = NPHC_END_DUPLICATE;
    push_once(w, list, count, e, ep.count);
    push_once(w, list, count, o, ep.count);
}

// phase 2: compare with the endpoints of the own and the neighbouring cells at level L(e)
// The entry a dedup thread matches: every entry, or only those of mlist (entries whose
// solution may have changed since the last dedup, e.g. after a re-track).
__device__ __forceinline__ int64_t dd_entry(const EPView &ep, const int32_t *mlist,
                                            const int32_t *mcount) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mlist) {
        if (i >= *mcount) return -1;
        const int64_t e = mlist[i];
        return NPHC_VALID(e >= 0 && e < ep.count, 1) ? e : -1;
    }
    return i < ep.count ? i : -1;
}

__global__ void dedup_match_kernel(const EPView ep, int n, double delta0, DedupScratch w,
                                   int32_t *list, int32_t *count, const int32_t *mlist,
                                   const int32_t *mcount) {
    const int64_t e = dd_entry(ep, mlist, mcount);
    if (e < 0 || !is_certified(ep.cls[e])) return;
    const int L = dd_level(ep.beta[e], delta0);
    if (L >= DD_LEVELS) return;   // phase 3
    double v[4];
    long long q0[4];
    int dir[4];
    dd_project(ep, n, e, v);
    const double inv = 1.0 / dd_pitch(delta0, L);
    for (int i = 0; i < 4; i++) v[i] *= inv;
    for (int i = 0; i < 4; i++) {
        q0[i] = (long long)floor(v[i]);
        const double f = v[i] - (double)q0[i];
        dir[i] = f < DD_BAND ? -1 : (f > 1.0 - DD_BAND ? 1 : 0);
    }
    const uint64_t mask = (uint64_t)w.table_size - 1;
    const unsigned long long *keys = w.keys + L * w.table_size;
    const int32_t *head = w.head + L * w.table_size;
    const int32_t *next = w.next + L * ep.count;
    for (int combo = 0; combo < 16; combo++) {
        long long q[4];
        bool skip = false;
        for (int i = 0; i < 4; i++) {
            const int bit = (combo >> i) & 1;
            if (bit && dir[i] == 0) skip = true;
            q[i] = q0[i] + (bit ? dir[i] : 0);
        }
        if (skip) continue;
        const unsigned long long key = dd_cell_key(L, q);
        uint64_t slot = key & mask;
        int32_t o = -1;
        for (int64_t probe = 0; probe < w.table_size; probe++) {
            const unsigned long long cur = keys[slot];
            if (cur == 0ull) break;
            if (cur == key) {
                o = head[slot];
                break;
            }
            slot = (slot + 1) & mask;
        }
        for (int64_t guard = 0; o >= 0 && guard < ep.count; guard++) {
            if (!NPHC_VALID(o < ep.count, 3)) break;
            if (o != e && same_solution(ep, n, e, o)) dd_pair(ep, w, list, count, e, o);
            o = next[o];
        }
    }
}

__global__ void dedup_unhashed_kernel(const EPView ep, int n, double delta0, DedupScratch w,
                                      int32_t *list, int32_t *count, const int32_t *mlist,
                                      const int32_t *mcount) {
    const int64_t e = dd_entry(ep, mlist, mcount);
    if (e < 0 || !is_certified(ep.cls[e]) || dd_level(ep.beta[e], delta0) < DD_LEVELS) return;
    for (int64_t j = 0; j < ep.count; j++) {
        if (j == e) continue;
        const int cj = ep.cls[j];
        if (!is_certified(cj) && cj != NPHC_END_DUPLICATE) continue;
        if (same_solution(ep, n, e, j)) dd_pair(ep, w, list, count, e, j);
    }
}

// ---------------------------------------------------------------- counters --
__global__ void counts_kernel(const EPView ep, const int32_t *flags, const int32_t *index,
                              int64_t *counts, const int32_t *egst, const int32_t *cycle) {
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
            if (flags[e] & FLAG_COND) atomicAdd(&loc[NPHC_COUNT_HANDOFF_COND], 1ull);
            if (flags[e] & (FLAG_RETRACKED | FLAG_RETRACKED_DUP)) atomicAdd(&loc[NPHC_COUNT_RETRACKED], 1ull);
        }
        atomicAdd(&loc[NPHC_COUNT_SOLVES], (unsigned long long)ep.solves[e]);
        if (c == NPHC_END_REAL && index) {
            const int ix = index[e];
            if (ix >= 0 && ix < NPHC_MAX_N) atomicAdd(&loc[NPHC_COUNT_INDEX0 + ix], 1ull);
        }
        if (egst && egst[e] != NPHC_EG_NONE) {
            const int g = egst[e];
            atomicAdd(&loc[NPHC_COUNT_EG_RUN], 1ull);
            if (g == NPHC_EG_CONVERGED) {
                atomicAdd(&loc[NPHC_COUNT_EG_CONVERGED], 1ull);
                if (cycle[e] >= 2) atomicAdd(&loc[NPHC_COUNT_EG_MULTIPLE], 1ull);
            } else if (g == NPHC_EG_AT_INFINITY || g == NPHC_EG_DIVERGED) {
                atomicAdd(&loc[NPHC_COUNT_EG_AT_INFINITY], 1ull);
            }
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
    if (ep.cls[e] == NPHC_END_REAL) {
        const int32_t k = atomicAdd(count, 1);
        if (NPHC_VALID(k < ep.count, 2)) list[k] = (int32_t)e;
    }
}

__global__ void iota_kernel(int64_t *path, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) path[e] = e;
}

__global__ void gather_sps_kernel(const EPView ep, int M, const int32_t *list, const int32_t *count,
                                  const double *theta, const int32_t *index, const double *energy,
                                  double *o_theta, int32_t *o_index, double *o_energy,
                                  double *o_alpha, int64_t *o_path, const double *logdet,
                                  double *o_logdet) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const int64_t e = list[i];
    const int64_t cnt = ep.count;
    if (!NPHC_VALID(e >= 0 && e < cnt, 5)) return;
    for (int k = 0; k < M; k++) o_theta[i * M + k] = theta[k * cnt + e];
    o_index[i] = index[e];
    o_energy[i] = energy[e];
    o_alpha[i] = ep.alpha[e];
    o_path[i] = ep.path[e];
    o_logdet[i] = logdet[e];
}

// ------------------------------------------------------------- launchers --
static inline int blocks_for(int64_t n, int b) { return (int)((n + b - 1) / b); }

cudaError_t launch_compact(const EPView &ep, int pred, int32_t *flags, int32_t *list,
                           int32_t *count, cudaStream_t st) {
    if (ep.count == 0) return cudaSuccess;
    compact_kernel<<<blocks_for(ep.count, 256), 256, 0, st>>>(ep, pred, flags, list, count);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t launch_flag_list(const int32_t *list, const int32_t *count, int64_t cap,
                             int32_t *flags, int32_t bit, cudaStream_t st) {
    if (cap == 0) return cudaSuccess;
    flag_list_kernel<<<blocks_for(cap, 256), 256, 0, st>>>(list, count, flags, bit, cap);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t launch_dedup(const EPView &ep, int n, double delta, DedupScratch w, int32_t *list,
                         int32_t *count, cudaStream_t st, const int32_t *mlist,
                         const int32_t *mcount) {
    cudaError_t err;
    // *count is an output of every call, an empty set included
    if (count && (err = cudaMemsetAsync(count, 0, sizeof(int32_t), st))) return err;
    if (ep.count == 0) return cudaSuccess;
    const size_t slots = (size_t)DD_LEVELS * w.table_size;
    if ((err = cudaMemsetAsync(w.keys, 0, sizeof(unsigned long long) * slots, st))) return err;
    if ((err = cudaMemsetAsync(w.head, 0xff, sizeof(int32_t) * slots, st))) return err;
    if ((err = cudaMemsetAsync(w.inlist, 0, sizeof(int32_t) * ep.count, st))) return err;
    const int g = blocks_for(ep.count, 256);
    dedup_insert_kernel<<<g, 256, 0, st>>>(ep, n, delta, w);
    nphc_launch_counter(1);
    dedup_match_kernel<<<g, 256, 0, st>>>(ep, n, delta, w, list, count, mlist, mcount);
    nphc_launch_counter(1);
    dedup_unhashed_kernel<<<g, 256, 0, st>>>(ep, n, delta, w, list, count, mlist, mcount);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t launch_counts(const EPView &ep, const int32_t *flags, const int32_t *index,
                          int64_t *counts, cudaStream_t st, const int32_t *egst,
                          const int32_t *cycle) {
    cudaError_t err = cudaMemsetAsync(counts, 0, sizeof(int64_t) * NPHC_NCOUNTS, st);
    if (err || ep.count == 0) return err;
    counts_kernel<<<blocks_for(ep.count, 256), 256, 0, st>>>(ep, flags, index, counts, egst, cycle);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t launch_real_list(const EPView &ep, int32_t *list, int32_t *count, cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
    if (err || ep.count == 0) return err;
    real_list_kernel<<<blocks_for(ep.count, 256), 256, 0, st>>>(ep, list, count);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t launch_iota(int64_t *path, int64_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    iota_kernel<<<blocks_for(n, 256), 256, 0, st>>>(path, n);
    nphc_launch_counter(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_sps(const EPView &ep, int M, const int32_t *list, const int32_t *count,
                              int64_t cap, const double *theta, const int32_t *index,
                              const double *energy, double *o_theta, int32_t *o_index,
                              double *o_energy, double *o_alpha, int64_t *o_path,
                              const double *logdet, double *o_logdet, cudaStream_t st) {
    if (cap == 0) return cudaSuccess;
    gather_sps_kernel<<<blocks_for(cap, 256), 256, 0, st>>>(ep, M, list, count, theta, index, energy,
                                                          o_theta, o_index, o_energy, o_alpha, o_path,
                                                          logdet, o_logdet);
    nphc_launch_counter(1);
    return cudaGetLastError();
}
