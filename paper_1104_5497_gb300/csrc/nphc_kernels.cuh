// nphc_kernels.cuh -- declarations of the size-independent kernels' launchers.
#pragma once

#include "nphc_internal.cuh"

enum {
    PRED_HANDOFF = 1,
    PRED_UNCERTIFIED_FP32 = 2,
    PRED_REACHED = 3,             // reached entries to refine; every other entry gets its class
    PRED_ENDGAME = 4,
    PRED_REACHED_DIRECT = 5,      // PRED_REACHED over the entries without FLAG_FP64_CONTINUED
    PRED_REACHED_CONTINUED = 6    // PRED_REACHED over the entries with FLAG_FP64_CONTINUED
};
enum { FLAG_FP64_CONTINUED = 1, FLAG_RETRACKED = 2, FLAG_RETRACKED_DUP = 4, FLAG_COND = 8 };

#define DD_LEVELS 4   // grid pitches 1e-6, 1e-4, 1e-2, 1

// Device scratch of the deduplication: per level, an open-addressing table of grid
// cells (keys, list heads; a power of two >= 2 x count slots) and per-entry list links.
struct DedupScratch {
    unsigned long long *keys;
    int32_t *head;
    int64_t table_size;
    int32_t *next;
    int32_t *inlist;
};

// The debug build's first failed index check (0 if none), cleared; -1 in a release build.
cudaError_t nphc_debug_read(int *code);

cudaError_t launch_compact(const EPView &ep, int pred, int32_t *flags, int32_t *list,
                           int32_t *count, cudaStream_t st);
cudaError_t launch_flag_list(const int32_t *list, const int32_t *count, int64_t cap,
                             int32_t *flags, int32_t bit, cudaStream_t st);
// Marks duplicates among the certified entries of ep.  mlist / mcount (device, may be
// NULL): only the pairs with an entry of mlist are examined (every other pair was
// settled by an earlier dedup and its entries left unchanged since).
cudaError_t launch_dedup(const EPView &ep, int n, double delta, DedupScratch w, int32_t *list,
                         int32_t *count, cudaStream_t st, const int32_t *mlist = nullptr,
                         const int32_t *mcount = nullptr);
// egst / cycle (may be NULL): the Cauchy endgame's outcome, for its counters.
cudaError_t launch_counts(const EPView &ep, const int32_t *flags, const int32_t *index,
                          int64_t *counts, cudaStream_t st, const int32_t *egst = nullptr,
                          const int32_t *cycle = nullptr);
cudaError_t launch_real_list(const EPView &ep, int32_t *list, int32_t *count, cudaStream_t st);
cudaError_t launch_iota(int64_t *path, int64_t n, cudaStream_t st);
cudaError_t launch_gather_sps(const EPView &ep, int M, const int32_t *list, const int32_t *count,
                              int64_t cap, const double *theta, const int32_t *index,
                              const double *energy, double *o_theta, int32_t *o_index,
                              double *o_energy, double *o_alpha, int64_t *o_path,
                              const double *logdet, double *o_logdet, cudaStream_t st);
