// nphc_api.cu -- host implementation of the C ABI declared in include/nphc.h.
//
// The system builder (couplings, FP32/FP64 coupling tables, ||D^2 P/2||) runs on the
// host; the couplings reach the kernels as launch parameters (constant bank), so a
// system owns no device memory.  A result owns one device allocation that holds every
// per-path array, the work lists, the counters and the deduplication scratch.
#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "nphc.h"
#include "nphc_internal.cuh"
#include "xy_dispatch.cuh"
#include "nphc_kernels.cuh"

namespace {

// A named range around a stage of the pipeline (NVTX, for profilers and tracers; it marks
// the host thread's enqueueing of the stage's launches and costs nothing when no tool is
// attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

}  // namespace

namespace {

thread_local std::string g_err;

nphc_status fail(nphc_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define NPHC_CK(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(NPHC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

constexpr double kDedupDelta = 1e-6;   // pitch of the deduplication grid

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int64_t table_size_for(int64_t count) {
    int64_t t = 1024;
    while (t < 2 * count) t <<= 1;
    return t;
}

// Device scratch: [queue counters | tracker path state | dedup cell keys | cell list
// heads | list links | flags].  The tracker state holds four vectors of n complex
// doubles for each of NPHC_TRACK_MAX_THREADS threads (enough for either precision).
struct WsLayout {
    size_t queue, state, keys, head, next, inlist, total;
    int64_t tsize;
};

WsLayout ws_layout(int n, int64_t count) {
    WsLayout L;
    L.tsize = table_size_for(count);
    size_t o = 0;
    L.queue = o;  o += align256(64);
    L.state = o;  o += align256((size_t)4 * n * NPHC_TRACK_MAX_THREADS * 2 * sizeof(double));
    L.keys = o;   o += align256(sizeof(unsigned long long) * L.tsize * DD_LEVELS);
    L.head = o;   o += align256(sizeof(int32_t) * L.tsize * DD_LEVELS);
    L.next = o;   o += align256(sizeof(int32_t) * count * DD_LEVELS);
    L.inlist = o; o += align256(sizeof(int32_t) * count);
    L.total = o;
    return L;
}

DedupScratch dedup_scratch(void *ws, const WsLayout &L) {
    char *b = static_cast<char *>(ws);
    DedupScratch w;
    w.keys = reinterpret_cast<unsigned long long *>(b + L.keys);
    w.head = reinterpret_cast<int32_t *>(b + L.head);
    w.table_size = L.tsize;
    w.next = reinterpret_cast<int32_t *>(b + L.next);
    w.inlist = reinterpret_cast<int32_t *>(b + L.inlist);
    return w;
}

unsigned long long *ws_queue(void *ws, int slot) {
    return reinterpret_cast<unsigned long long *>(static_cast<char *>(ws)) + slot;
}

}  // namespace

struct nphc_system {
    int N, M, n;             // a generic quadratic system has N = M = 0
    int64_t npaths;
    std::vector<double> J;   // N x N
    XYSys xs;                // coupling tables; gamma is filled per call
    bool quad = false;       // generic quadratic system (nphc_system_create_quadratic)
    QSys qs;                 // its device term list; gamma is filled per call
    void *qdev = nullptr;    // device allocation holding qs.row and qs.terms
};

struct nphc_result {
    int N, M, n;
    int64_t P;
    void *block;             // single device allocation
    size_t bytes;
    nphc_endpoints ep;       // device arrays for all paths
    double *theta, *energy, *mineig, *logdet;
    int32_t *index, *flags, *list[4], *lcount, *real_list;
    int64_t *counts;
    double *o_theta, *o_energy, *o_alpha, *o_logdet;
    int32_t *o_index;
    int32_t *cycle, *egst;   // Cauchy endgame outcome per path
    int32_t *egtrack;        // status of the endgame's tracking to 1 - r0 (keeps ep.status)
    int64_t *o_path;
    void *ws;
    size_t ws_bytes;
    void *eg_s;              // the refinement's Schur matrices (XY rings), eg_s_threads of them
    int64_t eg_s_threads;
    cudaStream_t stream;
    cudaStream_t side;        // second stream of the mixed pipeline (refinement beside the
    cudaEvent_t ev_fork, ev_join;   // FP64 continuation), forked and joined by events
    bool solved;
    int64_t launches;        // kernels launched by the last solve (host count)
};

extern "C" {

const char *nphc_last_error(void) { return g_err.c_str(); }

nphc_status nphc_debug_check(int32_t *code) {
    if (!code) return fail(NPHC_EINVAL, "code is NULL");
    int c = 0;
    NPHC_CK(nphc_debug_read(&c));
    *code = c;
    return NPHC_OK;
}

nphc_status nphc_options_default(nphc_options *o) {
    if (!o) return fail(NPHC_EINVAL, "nphc_options_default: NULL");
    std::memset(o, 0, sizeof(*o));
    o->precision = NPHC_PREC_MIXED;
    o->gamma_re = std::cos(0.5);
    o->gamma_im = std::sin(0.5);
    o->tol_sol = 1e-10;
    o->tol_real = 1e-7;
    o->h0 = 0.01;
    o->h_max = 0.05;
    o->h_min = 1e-14;
    o->eps_fp32 = 1e-5;
    o->eps_fp64 = 1e-9;
    o->trust = 0.1;
    o->trust_fp32 = 2e-3;
    o->r_div = 1e8;
    o->max_newton_fp32 = 3;
    o->max_newton_fp64 = 3;
    o->max_steps = 5000;
    o->max_steps_fp32 = 400;
    o->crawl_steps_fp32 = 32;
    o->grow_after = 3;
    o->refine_iters = 8;
    o->refine_eps = 1e-14;
    o->endgame = 0;
    o->eg_r0 = 1.0 / 16.0;
    o->eg_ratio = 0.25;
    o->eg_radii = 8;
    o->eg_samples = 16;
    o->eg_max_cycle = 8;
    o->eg_tol_close = 1e-6;
    o->eg_tol_conv = 1e-9;
    o->eg_h_min = 1.0 / 4096.0;
    o->eg_max_attempts = 4000;
    o->list_blocks_per_sm = 0;
    o->block_size = 0;
    o->blocks_per_sm = 0;
    o->kappa_sing = 1e12;
    o->threads_per_path = 0;
    o->kappa_fp32 = 3e5;
    return NPHC_OK;
}

nphc_status nphc_xy_couplings(int N, double sigma, const double *g, double eps, double *J) {
    if (N < NPHC_MIN_N || N > NPHC_MAX_N) return fail(NPHC_EINVAL, "N outside [3, 13]");
    if (!std::isfinite(sigma)) return fail(NPHC_EINVAL, "sigma not finite");
    if (!J) return fail(NPHC_EINVAL, "J_out is NULL");
    if (g) {
        if (!std::isfinite(eps)) return fail(NPHC_EINVAL, "eps not finite");
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++)
                if (!std::isfinite(g[i * N + j]) || g[i * N + j] != g[j * N + i])
                    return fail(NPHC_EINVAL, "g not finite and symmetric");
    }
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            if (i == j) {
                J[i * N + j] = 0.0;
                continue;
            }
            const int d = std::min(std::abs(i - j), N - std::abs(i - j));
            double v = std::pow((double)d, -sigma);
            if (g) v *= 1.0 + eps * g[i * N + j];
            if (!(v > 0.0) || !std::isfinite(v)) return fail(NPHC_EINVAL, "coupling <= 0 or not finite");
            J[i * N + j] = v;
        }
    return NPHC_OK;
}

nphc_status nphc_xy_couplings_vjp(int N, double sigma, const double *g, double eps,
                                  const double *dL_dJ, double *dsigma) {
    if (!dL_dJ || !dsigma) return fail(NPHC_EINVAL, "dL_dJ or dsigma is NULL");
    if (N < NPHC_MIN_N || N > NPHC_MAX_N) return fail(NPHC_EINVAL, "N outside [3, 13]");
    std::vector<double> J(N * N);
    nphc_status s = nphc_xy_couplings(N, sigma, g, eps, J.data());
    if (s != NPHC_OK) return s;
    double acc = 0.0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            if (i == j) continue;
            const int d = std::min(std::abs(i - j), N - std::abs(i - j));
            acc += dL_dJ[i * N + j] * (-std::log((double)d)) * J[i * N + j];
        }
    if (!std::isfinite(acc)) return fail(NPHC_EINVAL, "dL_dJ not finite");
    *dsigma = acc;
    return NPHC_OK;
}

nphc_status nphc_system_create_xy(int N, double sigma, const double *J, nphc_system **out) {
    if (!out) return fail(NPHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < NPHC_MIN_N || N > NPHC_MAX_N) return fail(NPHC_EINVAL, "N outside [3, 13]");
    std::vector<double> Jv(N * N);
    if (J) {
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                const double v = J[i * N + j];
                if (!std::isfinite(v)) return fail(NPHC_EINVAL, "J not finite");
                if (v != J[j * N + i]) return fail(NPHC_EINVAL, "J not symmetric");
                if (i == j && v != 0.0) return fail(NPHC_EINVAL, "J diagonal not zero");
                Jv[i * N + j] = v;
            }
    } else {
        nphc_status s = nphc_xy_couplings(N, sigma, nullptr, 0.0, Jv.data());
        if (s != NPHC_OK) return s;
    }
    nphc_system *S = new (std::nothrow) nphc_system;
    if (!S) return fail(NPHC_ENOMEM, "host allocation");
    S->N = N;
    S->M = N - 1;
    S->n = 2 * (N - 1);
    S->npaths = (int64_t)1 << S->n;
    S->J = Jv;
    std::memset(&S->xs, 0, sizeof(S->xs));
    S->xs.N = N;
    double d2 = 2.0 * S->M;   // each constraint c^2 + s^2 - 1 contributes ||M_g||_F^2 = 2
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            S->xs.Jf[i * NPHC_JSTRIDE + j] = (float)Jv[i * N + j];
            S->xs.Jd[i * NPHC_JSTRIDE + j] = Jv[i * N + j];
            // gradient row i: J_ij (s_i c_j - s_j c_i) puts J_ij / 2 on four symmetric
            // entries when j is free, so ||M_fi||_F^2 gains J_ij^2
            if (i < S->M && j < S->M && i != j) d2 += Jv[i * N + j] * Jv[i * N + j];
        }
    S->xs.d2norm = std::sqrt(d2);
    S->xs.kappa_sing = 1e12;
    *out = S;
    return NPHC_OK;
}

nphc_status nphc_system_info(const nphc_system *S, int *N, int *n, int64_t *npaths) {
    if (!S) return fail(NPHC_EINVAL, "system is NULL");
    if (N) *N = S->N;
    if (n) *n = S->n;
    if (npaths) *npaths = S->npaths;
    return NPHC_OK;
}

nphc_status nphc_system_couplings(const nphc_system *S, double *J) {
    if (!S || !J) return fail(NPHC_EINVAL, "NULL argument");
    if (S->quad) return fail(NPHC_EINVAL, "a generic quadratic system has no couplings");
    std::memcpy(J, S->J.data(), sizeof(double) * S->J.size());
    return NPHC_OK;
}

void nphc_system_destroy(nphc_system *S) {
    if (!S) return;
    if (S->qdev) cudaFree(S->qdev);
    delete S;
}

nphc_status nphc_system_create_quadratic(int n, int nterms, const int32_t *eq, const int32_t *va,
                                         const int32_t *vb, const double *coef_re,
                                         const double *coef_im, nphc_system **out) {
    if (!out) return fail(NPHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > NPHC_QUAD_MAX_N) return fail(NPHC_EINVAL, "n outside [1, NPHC_QUAD_MAX_N]");
    if (nterms < 1 || !eq || !va || !vb || !coef_re || !coef_im)
        return fail(NPHC_EINVAL, "empty or missing term arrays");
    // terms sorted by equation (stable), row offsets, ||D^2 P / 2|| from the symmetric
    // coefficient matrices M_i of the quadratic parts: z^T M_i z
    std::vector<int32_t> row(n + 1, 0);
    std::vector<QTerm> terms(nterms);
    std::vector<std::vector<double>> m2(n, std::vector<double>((size_t)n * n * 2, 0.0));
    for (int t = 0; t < nterms; t++) {
        if (eq[t] < 0 || eq[t] >= n) return fail(NPHC_EINVAL, "term equation index out of range");
        if (va[t] < -1 || va[t] >= n || vb[t] < -1 || vb[t] >= n)
            return fail(NPHC_EINVAL, "term variable index out of range");
        if (!std::isfinite(coef_re[t]) || !std::isfinite(coef_im[t]))
            return fail(NPHC_EINVAL, "term coefficient not finite");
        row[eq[t] + 1]++;
    }
    for (int i = 0; i < n; i++) row[i + 1] += row[i];
    std::vector<int32_t> fill(row.begin(), row.end() - 1);
    for (int t = 0; t < nterms; t++) {
        QTerm q;
        q.a = va[t];
        q.b = vb[t];
        q.cre = coef_re[t];
        q.cim = coef_im[t];
        terms[fill[eq[t]]++] = q;
        if (q.a >= 0 && q.b >= 0) {
            std::vector<double> &Mi = m2[eq[t]];
            const double h = q.a == q.b ? 1.0 : 0.5;
            for (int rep = 0; rep < (q.a == q.b ? 1 : 2); rep++) {
                const size_t k = rep == 0 ? ((size_t)q.a * n + q.b) : ((size_t)q.b * n + q.a);
                Mi[2 * k] += h * q.cre;
                Mi[2 * k + 1] += h * q.cim;
            }
        }
    }
    double d2 = 0.0;
    for (int i = 0; i < n; i++)
        for (double v : m2[i]) d2 += v * v;
    nphc_system *S = new (std::nothrow) nphc_system;
    if (!S) return fail(NPHC_ENOMEM, "host allocation");
    S->N = 0;
    S->M = 0;
    S->n = n;
    S->npaths = (int64_t)1 << n;
    std::memset(&S->xs, 0, sizeof(S->xs));
    S->quad = true;
    const size_t rbytes = align256(sizeof(int32_t) * (n + 1));
    const size_t bytes = rbytes + sizeof(QTerm) * nterms;
    if (cudaMalloc(&S->qdev, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return fail(NPHC_ENOMEM, "device allocation for the term list");
    }
    char *d = static_cast<char *>(S->qdev);
    cudaError_t e = cudaMemcpy(d, row.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d + rbytes, terms.data(), sizeof(QTerm) * nterms, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        nphc_system_destroy(S);
        return fail(NPHC_ECUDA, std::string("term list upload: ") + cudaGetErrorString(e));
    }
    S->qs.n = n;
    S->qs.row = reinterpret_cast<const int32_t *>(d);
    S->qs.terms = reinterpret_cast<const QTerm *>(d + rbytes);
    S->qs.gre = 1.0;
    S->qs.gim = 0.0;
    S->qs.d2norm = std::sqrt(d2);
    S->qs.kappa_sing = 1e12;
    *out = S;
    return NPHC_OK;
}

nphc_status nphc_workspace_size(const nphc_system *S, int64_t count, size_t *bytes) {
    if (!S || !bytes || count < 0) return fail(NPHC_EINVAL, "invalid argument");
    *bytes = ws_layout(S->n, count).total;
    return NPHC_OK;
}

}  // extern "C"

// ------------------------------------------------------------ internals --
namespace {

nphc_status check_opt(const nphc_options *o) {
    if (!o) return fail(NPHC_EINVAL, "options are NULL");
    const double g2 = o->gamma_re * o->gamma_re + o->gamma_im * o->gamma_im;
    if (!(g2 > 0.0) || !std::isfinite(g2)) return fail(NPHC_EINVAL, "|gamma| = 0 or not finite");
    if (!(o->h0 > 0 && o->h_max >= o->h0 && o->h_min > 0 && o->eps_fp32 > 0 && o->eps_fp64 > 0 &&
          o->trust > 0 && o->trust_fp32 > 0 && o->r_div > 0 && o->max_newton_fp32 > 0 &&
          o->max_newton_fp64 > 0 && o->max_steps > 0 && o->max_steps_fp32 > 0 && o->crawl_steps_fp32 >= 0 && o->grow_after > 0 &&
          o->refine_iters >= 0 && o->kappa_sing > 0 && o->kappa_fp32 >= 0))
        return fail(NPHC_EINVAL, "options out of range");
    if (!(o->eg_r0 > 0.0 && o->eg_r0 < 1.0 && o->eg_ratio > 0.0 && o->eg_ratio < 1.0 &&
          o->eg_radii >= 1 && o->eg_samples >= 2 && o->eg_samples <= 4096 && o->eg_max_cycle >= 1 &&
          o->eg_tol_close > 0.0 && o->eg_tol_conv > 0.0 && o->eg_h_min > 0.0 &&
          o->eg_max_attempts > 0))
        return fail(NPHC_EINVAL, "endgame options out of range");
    if (o->blocks_per_sm < 0 || o->list_blocks_per_sm < 0 || o->block_size < 0 ||
        !(o->threads_per_path == 0 || o->threads_per_path == 1 || o->threads_per_path == 32))
        return fail(NPHC_EINVAL, "launch options out of range");
    return NPHC_OK;
}

// The system with the run's gamma and singularity bound.
QSys quad_with_gamma(const nphc_system *S, const nphc_options *o) {
    QSys q = S->qs;
    q.gre = o->gamma_re;
    q.gim = o->gamma_im;
    q.kappa_sing = o->kappa_sing;
    return q;
}

XYSys sys_with_gamma(const nphc_system *S, const nphc_options *o) {
    XYSys x = S->xs;
    x.gre = o->gamma_re;
    x.gim = o->gamma_im;
    x.kappa_sing = o->kappa_sing;
    return x;
}

XYCtl make_ctl(const nphc_options *o, bool fp32, bool resume, bool accumulate) {
    XYCtl c;
    c.h0 = o->h0;
    c.hmax = o->h_max;
    c.hmin = o->h_min;
    c.eps = fp32 ? o->eps_fp32 : o->eps_fp64;
    c.trust = fp32 ? o->trust_fp32 : o->trust;
    c.rdiv = o->r_div;
    c.max_newton = fp32 ? o->max_newton_fp32 : o->max_newton_fp64;
    c.max_steps = fp32 ? o->max_steps_fp32 : o->max_steps;
    c.grow_after = o->grow_after;
    c.handoff = fp32 ? 1 : 0;
    c.resume = resume ? 1 : 0;
    c.accumulate = accumulate ? 1 : 0;
    c.sparse = 0;
    c.crawl_steps = fp32 ? o->crawl_steps_fp32 : 0;
    c.t_end = 1.0;
    c.kappa = fp32 ? o->kappa_fp32 : 0.0;
    return c;
}

EPView view(const nphc_endpoints *e) {
    EPView v;
    v.count = e->count;
    v.path = e->path;
    v.z_re = e->z_re;
    v.z_im = e->z_im;
    v.t = e->t;
    v.h = e->h;
    v.status = e->status;
    v.steps = e->steps;
    v.solves = e->solves;
    v.newton = e->newton;
    v.cls = e->cls;
    v.alpha = e->alpha;
    v.beta = e->beta;
    v.gamma = e->gamma;
    v.resid = e->resid;
    return v;
}

nphc_status track_impl(const nphc_system *S, const nphc_options *o, nphc_precision prec,
                       const nphc_endpoints *ep, const int32_t *list, const int32_t *list_count,
                       bool resume, bool accumulate, void *ws, int queue_slot, cudaStream_t st,
                       double t_end = 1.0) {
    const bool f32 = prec == NPHC_PREC_MIXED && !S->quad;   // generic systems: FP64
    const XYSys xs = sys_with_gamma(S, o);
    XYCtl ctl = make_ctl(o, f32, resume, accumulate);
    ctl.t_end = t_end;
    // FP64 lists (hand-offs, re-tracks) spread over every SM: ceil(list / warps) paths
    // per warp, up to 32
    ctl.sparse = (!f32 && list != nullptr) ? 1 : 0;
    WorkList wl;
    wl.list = list;
    wl.list_count = list_count;
    wl.queue = ws_queue(ws, queue_slot);
    wl.state = static_cast<char *>(ws) + ws_layout(S->n, 0).state;
    wl.state_threads = NPHC_TRACK_MAX_THREADS;
    NPHC_CK(cudaMemsetAsync(wl.queue, 0, sizeof(unsigned long long), st));
    int grid = 0;
    if (f32 && o->blocks_per_sm > 0) {
        int dev = 0, sms = 0;
        NPHC_CK(cudaGetDevice(&dev));
        NPHC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        grid = sms * o->blocks_per_sm;
    }
    const EPView v = view(ep);
    if (S->quad)
        NPHC_CK(launch_quad_track(S->n, quad_with_gamma(S, o), ctl, v, wl, 0, st));
    else if (!f32 && list != nullptr && o->threads_per_path != 1)   // one path per warp
        NPHC_CK(launch_xy_track_f64_warp_bps(S->M, xs, ctl, v, wl, o->list_blocks_per_sm, st));
    else if (!f32 && list != nullptr)   // FP64 lists, one path per thread, full warps
        NPHC_CK(launch_xy_track_f64(S->M, xs, ctl, v, wl, 0, 0, st));
    else if (f32)
        NPHC_CK(launch_xy_track_f32(S->M, xs, ctl, v, wl, 0, grid, st));
    else
        NPHC_CK(launch_xy_track_f64(S->M, xs, ctl, v, wl, 0, 0, st));
    return NPHC_OK;
}

// The Cauchy endgame on the selected entries: FP64 tracking to 1 - eg_r0 (queue slot 6),
// then the turns around t = 1 (queue slot 7).  The tracking writes its statuses where ep
// says (the pipeline points them at a scratch array to keep the result's statuses).
nphc_status endgame_impl(const nphc_system *S, const nphc_options *o, const nphc_endpoints *ep,
                         const int32_t *list, const int32_t *list_count, int32_t *cycle,
                         int32_t *egst, bool accumulate, void *ws, cudaStream_t st) {
    nphc_status s = track_impl(S, o, NPHC_PREC_FP64, ep, list, list_count, false, accumulate, ws,
                               6, st, 1.0 - o->eg_r0);
    if (s != NPHC_OK) return s;
    EGCtl c;
    c.lr0 = std::log(o->eg_r0);
    c.lnratio = std::log(o->eg_ratio);
    c.n_radii = o->eg_radii;
    c.samples = o->eg_samples;
    c.max_cycle = o->eg_max_cycle;
    c.tol_close = o->eg_tol_close;
    c.tol_conv = o->eg_tol_conv;
    c.tol_res = o->tol_sol;
    c.grow_inf = std::pow(o->eg_ratio, -0.5 / o->eg_max_cycle);
    c.hmin = o->eg_h_min;
    c.max_attempts = o->eg_max_attempts;
    c.eps = o->eps_fp64;
    c.trust = o->trust;
    c.rdiv = o->r_div;
    c.max_newton = o->max_newton_fp64;
    c.grow_after = o->grow_after;
    WorkList wl;
    wl.list = list;
    wl.list_count = list_count;
    wl.queue = ws_queue(ws, 7);
    wl.state = static_cast<char *>(ws) + ws_layout(S->n, 0).state;
    // the tracker scratch holds 4 vectors per thread for NPHC_TRACK_MAX_THREADS threads
    wl.state_threads = (int64_t)4 * NPHC_TRACK_MAX_THREADS / NPHC_CAUCHY_STATE_VECTORS / 32 * 32;
    NPHC_CK(cudaMemsetAsync(wl.queue, 0, sizeof(unsigned long long), st));
    const EPView v = view(ep);
    if (S->quad)
        NPHC_CK(launch_quad_cauchy(S->n, quad_with_gamma(S, o), c, v, wl, cycle, egst, st));
    else
        NPHC_CK(launch_xy_cauchy(S->M, sys_with_gamma(S, o), c, v, wl, cycle, egst, st));
    return NPHC_OK;
}

nphc_status check_ep(const nphc_system *S, const nphc_endpoints *ep, bool certify) {
    if (!S || !ep) return fail(NPHC_EINVAL, "NULL argument");
    if (ep->count < 0 || ep->count > S->npaths || ep->count > INT32_MAX)
        return fail(NPHC_EINVAL, "endpoint count out of range");
    if (ep->count == 0) return NPHC_OK;   // nothing is read or written
    if (!ep->path || !ep->z_re || !ep->z_im || !ep->t || !ep->h || !ep->status || !ep->steps ||
        !ep->solves || !ep->newton)
        return fail(NPHC_EINVAL, "endpoint arrays missing");
    if (certify && (!ep->cls || !ep->alpha || !ep->beta || !ep->gamma || !ep->resid))
        return fail(NPHC_EINVAL, "certification arrays missing");
    return NPHC_OK;
}

}  // namespace

extern "C" {

nphc_status nphc_track(const nphc_system *S, const nphc_options *o, nphc_precision prec,
                       const nphc_endpoints *ep, const int32_t *list, const int32_t *list_count,
                       int resume, void *ws, size_t ws_bytes, void *stream) {
    nphc_status s;
    if ((s = check_ep(S, ep, false)) != NPHC_OK) return s;
    if ((s = check_opt(o)) != NPHC_OK) return s;
    if (prec != NPHC_PREC_FP64 && prec != NPHC_PREC_MIXED) return fail(NPHC_EINVAL, "precision");
    if ((list == nullptr) != (list_count == nullptr)) return fail(NPHC_EINVAL, "list without count");
    if (!ws || ws_bytes < ws_layout(S->n, ep->count).total) return fail(NPHC_EINVAL, "workspace too small");
    return track_impl(S, o, prec, ep, list, list_count, resume != 0, resume != 0, ws, 0,
                      (cudaStream_t)stream);
}

nphc_status nphc_endgame(const nphc_system *S, const nphc_options *o, const nphc_endpoints *ep,
                         const int32_t *list, const int32_t *list_count, int32_t *cycle,
                         int32_t *eg_status, void *ws, size_t ws_bytes, void *stream) {
    nphc_status s;
    if ((s = check_ep(S, ep, false)) != NPHC_OK) return s;
    if ((s = check_opt(o)) != NPHC_OK) return s;
    if (!cycle || !eg_status) return fail(NPHC_EINVAL, "cycle / eg_status arrays missing");
    if ((list == nullptr) != (list_count == nullptr)) return fail(NPHC_EINVAL, "list without count");
    if (!ws || ws_bytes < ws_layout(S->n, ep->count).total) return fail(NPHC_EINVAL, "workspace too small");
    return endgame_impl(S, o, ep, list, list_count, cycle, eg_status, false, ws,
                        (cudaStream_t)stream);
}

nphc_status nphc_refine_certify(const nphc_system *S, const nphc_options *o,
                                const nphc_endpoints *ep, const int32_t *list,
                                const int32_t *list_count, void *stream) {
    nphc_status s;
    if ((s = check_ep(S, ep, true)) != NPHC_OK) return s;
    if ((s = check_opt(o)) != NPHC_OK) return s;
    if ((list == nullptr) != (list_count == nullptr)) return fail(NPHC_EINVAL, "list without count");
    WorkList wl;
    wl.list = list;
    wl.list_count = list_count;
    wl.queue = nullptr;
    wl.state = nullptr;
    wl.state_threads = 0;
    if (S->quad)
        NPHC_CK(launch_quad_refine_certify(S->n, quad_with_gamma(S, o), o->tol_sol, o->refine_eps,
                                           o->refine_iters, view(ep), ep->count, wl,
                                           (cudaStream_t)stream));
    else
        NPHC_CK(launch_xy_refine_certify(S->M, sys_with_gamma(S, o), o->tol_sol, o->refine_eps,
                                         o->refine_iters, view(ep), ep->count, wl, 0,
                                         (cudaStream_t)stream));
    return NPHC_OK;
}

nphc_status nphc_dedup(const nphc_system *S, const nphc_options *o, const nphc_endpoints *ep,
                       int32_t *dup_list, int32_t *dup_count, void *ws, size_t ws_bytes,
                       void *stream) {
    nphc_status s;
    if ((s = check_ep(S, ep, true)) != NPHC_OK) return s;
    (void)o;
    if ((dup_list == nullptr) != (dup_count == nullptr)) return fail(NPHC_EINVAL, "list without count");
    const WsLayout L = ws_layout(S->n, ep->count);
    if (!ws || ws_bytes < L.total) return fail(NPHC_EINVAL, "workspace too small");
    NPHC_CK(launch_dedup(view(ep), S->n, kDedupDelta, dedup_scratch(ws, L), dup_list, dup_count,
                         (cudaStream_t)stream));
    return NPHC_OK;
}

nphc_status nphc_classify(const nphc_system *S, const nphc_endpoints *ep, double *theta,
                          int32_t *index, double *energy, double *min_abs_eig,
                          double *log_abs_det, void *stream) {
    nphc_status s;
    if ((s = check_ep(S, ep, true)) != NPHC_OK) return s;
    if (!theta || !index || !energy) return fail(NPHC_EINVAL, "output arrays missing");
    if (S->quad) return fail(NPHC_EINVAL, "classification needs an XY system");
    XYSys xs = S->xs;
    NPHC_CK(launch_xy_classify(S->M, xs, view(ep), theta, index, energy, min_abs_eig, log_abs_det,
                               (cudaStream_t)stream));
    return NPHC_OK;
}

nphc_status nphc_xy_adjoint(const nphc_system *S, int64_t count, const double *theta,
                            const double *g_energy, const double *g_theta, double *dJ,
                            void *stream) {
    if (!S || count < 0 || (count > 0 && !theta) || !dJ) return fail(NPHC_EINVAL, "NULL argument");
    if (S->quad) return fail(NPHC_EINVAL, "the adjoint needs an XY system");
    NPHC_CK(launch_xy_adjoint(S->M, S->xs, count, theta, g_energy, g_theta, dJ,
                              (cudaStream_t)stream));
    return NPHC_OK;
}

nphc_status nphc_result_create(const nphc_system *S, nphc_result **out) {
    if (!S || !out) return fail(NPHC_EINVAL, "NULL argument");
    *out = nullptr;
    const int64_t P = S->npaths;
    const int n = S->n, M = S->M;
    const WsLayout L = ws_layout(n, P);
    // the refinement's M x M Schur matrices in global memory, one per thread of its largest
    // launch (four one-warp blocks per SM, at most one thread per path)
    int64_t eg_threads = 0;
    if (!S->quad) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return fail(NPHC_ECUDA, "no CUDA device");
        }
        eg_threads = std::min<int64_t>((P + 31) / 32 * 32, (int64_t)4 * 32 * sms);
    }
    // sub-allocation plan
    std::vector<size_t> sz = {
        sizeof(int64_t) * P,            // 0 path
        sizeof(double) * n * P,         // 1 z_re
        sizeof(double) * n * P,         // 2 z_im
        sizeof(double) * P,             // 3 t
        sizeof(double) * P,             // 4 h
        sizeof(int32_t) * P,            // 5 status
        sizeof(int32_t) * P,            // 6 steps
        sizeof(int32_t) * P,            // 7 solves
        sizeof(int32_t) * P,            // 8 newton
        sizeof(int32_t) * P,            // 9 cls
        sizeof(double) * P,             // 10 alpha
        sizeof(double) * P,             // 11 beta
        sizeof(double) * P,             // 12 gamma
        sizeof(double) * P,             // 13 resid
        sizeof(double) * M * P,         // 14 theta
        sizeof(double) * P,             // 15 energy
        sizeof(double) * P,             // 16 mineig
        sizeof(int32_t) * P,            // 17 index
        sizeof(int32_t) * P,            // 18 flags
        sizeof(int32_t) * P,            // 19 list0
        sizeof(int32_t) * P,            // 20 list1
        sizeof(int32_t) * P,            // 21 list2
        sizeof(int32_t) * 8,            // 22 lcount
        sizeof(int32_t) * P,            // 23 list3
        sizeof(int32_t) * P,            // 24 real_list
        sizeof(int64_t) * NPHC_NCOUNTS, // 25 counts
        sizeof(double) * M * P,         // 26 o_theta
        sizeof(double) * P,             // 27 o_energy
        sizeof(double) * P,             // 28 o_alpha
        sizeof(int32_t) * P,            // 29 o_index
        sizeof(int64_t) * P,            // 30 o_path
        L.total,                        // 31 workspace
        sizeof(double) * P,             // 32 logdet
        sizeof(double) * P,             // 33 o_logdet
        sizeof(int32_t) * P,            // 34 cycle
        sizeof(int32_t) * P,            // 35 egst
        sizeof(int32_t) * P,            // 36 egtrack
        sizeof(double) * 2 * M * M * eg_threads};   // 37 refinement Schur matrices
    std::vector<size_t> off(sz.size());
    size_t tot = 0;
    for (size_t i = 0; i < sz.size(); i++) {
        off[i] = tot;
        tot += align256(sz[i]);
    }
    nphc_result *R = new (std::nothrow) nphc_result;
    if (!R) return fail(NPHC_ENOMEM, "host allocation");
    std::memset(R, 0, sizeof(*R));
    cudaError_t e = cudaMalloc(&R->block, tot);
    if (e != cudaSuccess) {
        delete R;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NPHC_ENOMEM : NPHC_ECUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    char *b = static_cast<char *>(R->block);
    auto at = [&](int i) { return static_cast<void *>(b + off[i]); };
    R->N = S->N;
    R->M = M;
    R->n = n;
    R->P = P;
    R->bytes = tot;
    R->ep.count = P;
    R->ep.path = (int64_t *)at(0);
    R->ep.z_re = (double *)at(1);
    R->ep.z_im = (double *)at(2);
    R->ep.t = (double *)at(3);
    R->ep.h = (double *)at(4);
    R->ep.status = (int32_t *)at(5);
    R->ep.steps = (int32_t *)at(6);
    R->ep.solves = (int32_t *)at(7);
    R->ep.newton = (int32_t *)at(8);
    R->ep.cls = (int32_t *)at(9);
    R->ep.alpha = (double *)at(10);
    R->ep.beta = (double *)at(11);
    R->ep.gamma = (double *)at(12);
    R->ep.resid = (double *)at(13);
    R->theta = (double *)at(14);
    R->energy = (double *)at(15);
    R->mineig = (double *)at(16);
    R->index = (int32_t *)at(17);
    R->flags = (int32_t *)at(18);
    R->list[0] = (int32_t *)at(19);
    R->list[1] = (int32_t *)at(20);
    R->list[2] = (int32_t *)at(21);
    R->lcount = (int32_t *)at(22);
    R->list[3] = (int32_t *)at(23);
    R->real_list = (int32_t *)at(24);
    R->counts = (int64_t *)at(25);
    R->o_theta = (double *)at(26);
    R->o_energy = (double *)at(27);
    R->o_alpha = (double *)at(28);
    R->o_index = (int32_t *)at(29);
    R->o_path = (int64_t *)at(30);
    R->ws = at(31);
    R->logdet = (double *)at(32);
    R->o_logdet = (double *)at(33);
    R->cycle = (int32_t *)at(34);
    R->egst = (int32_t *)at(35);
    R->egtrack = (int32_t *)at(36);
    R->eg_s = eg_threads > 0 ? at(37) : nullptr;
    R->eg_s_threads = eg_threads;
    R->ws_bytes = L.total;
    R->stream = nullptr;
    R->solved = false;
    e = launch_iota(R->ep.path, P, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&R->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (R->ev_fork) cudaEventDestroy(R->ev_fork);
        if (R->side) cudaStreamDestroy(R->side);
        cudaFree(R->block);
        delete R;
        return fail(NPHC_ECUDA, std::string("result init: ") + cudaGetErrorString(e));
    }
    *out = R;
    return NPHC_OK;
}

}  // extern "C"

namespace {

// The whole method into R on `stream`; with fp32_done the FP32 pass of a mixed-precision
// solve has already run (a batch group's launch) and the pipeline starts after it.
nphc_status solve_into_impl(const nphc_system *S, const nphc_options *o, nphc_result *R,
                            void *stream, bool fp32_done) {
    const Range whole("nphc_solve_into");
    if (!S || !R) return fail(NPHC_EINVAL, "NULL argument");
    if (R->P != S->npaths || R->N != S->N) return fail(NPHC_EINVAL, "result does not match system");
    nphc_status s;
    if ((s = check_opt(o)) != NPHC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const nphc_endpoints *ep = &R->ep;
    const EPView v = view(ep);
    const XYSys xs = sys_with_gamma(S, o);
    const WsLayout L = ws_layout(R->n, R->P);
    const DedupScratch dsc = dedup_scratch(R->ws, L);
    R->solved = false;
    const int64_t launches0 = nphc_launch_counter(0);
    NPHC_CK(cudaMemsetAsync(R->flags, 0, sizeof(int32_t) * R->P, st));
    NPHC_CK(cudaMemsetAsync(R->lcount, 0, sizeof(int32_t) * 8, st));
    NPHC_CK(cudaMemsetAsync(R->cycle, 0, sizeof(int32_t) * R->P, st));
    NPHC_CK(cudaMemsetAsync(R->egst, 0, sizeof(int32_t) * R->P, st));
    const bool mixed = o->precision == NPHC_PREC_MIXED;
    // the Cauchy endgame on the paths that end singular or failed; the result keeps its
    // tracking statuses (the endgame's own go to a scratch array)
    auto endgame = [&]() -> nphc_status {
        if (!o->endgame) return NPHC_OK;
        NPHC_CK(launch_compact(v, PRED_ENDGAME, R->flags, R->list[1], R->lcount + 6, st));
        nphc_endpoints eg = *ep;
        eg.status = R->egtrack;
        return endgame_impl(S, o, &eg, R->list[1], R->lcount + 6, R->cycle, R->egst, true, R->ws, st);
    };
    if (S->quad) {
        // generic quadratic system: FP64 tracking, refinement, certification, dedup; no
        // classification (index -1 everywhere)
        if ((s = track_impl(S, o, NPHC_PREC_FP64, ep, nullptr, nullptr, false, false, R->ws, 0, st)))
            return s;
        NPHC_CK(launch_compact(v, PRED_REACHED, R->flags, R->list[3], R->lcount + 3, st));
        WorkList l3 = {R->list[3], R->lcount + 3, nullptr, nullptr, 0};
        NPHC_CK(launch_quad_refine_certify(S->n, quad_with_gamma(S, o), o->tol_sol, o->refine_eps,
                                           o->refine_iters, v, R->P, l3, st));
        NPHC_CK(launch_dedup(v, R->n, kDedupDelta, dsc, nullptr, nullptr, st));
        NPHC_CK(cudaMemsetAsync(R->index, 0xff, sizeof(int32_t) * R->P, st));
        if ((s = endgame())) return s;
        NPHC_CK(launch_counts(v, R->flags, R->index, R->counts, st, R->egst, R->cycle));
        R->stream = st;
        R->solved = true;
        R->launches = nphc_launch_counter(0) - launches0;
        return NPHC_OK;
    }
    if (mixed) {
        // FP32 pass over every path
        if (!fp32_done) {
            const Range r("fp32 pass");
            if ((s = track_impl(S, o, NPHC_PREC_MIXED, ep, nullptr, nullptr, false, false, R->ws, 0, st)))
                return s;
        }
        Range r_tail("fp64 hand-offs, refinement, certification");
        // hand-offs: refinement at t = 1 straight from the hand-off point (certified ones
        // are done), then FP64 continuation of the others
        NPHC_CK(launch_compact(v, PRED_HANDOFF, R->flags, R->list[0], R->lcount + 0, st));
        WorkList l0 = {R->list[0], R->lcount + 0, nullptr, R->eg_s, R->eg_s_threads};
        NPHC_CK(launch_xy_refine_certify(S->M, xs, o->tol_sol, o->refine_eps, o->refine_iters, v,
                                         R->P, l0, 1, st));
        NPHC_CK(launch_compact(v, PRED_HANDOFF, R->flags, R->list[0], R->lcount + 5, st));
        // the FP64 continuation of the hand-offs is imbalanced (a few long paths; SMs idle
        // about half its time) and touches only hand-off entries: the refinement of the
        // endpoints the FP32 pass reached (every other entry) runs beside it on the side
        // stream, selected by the hand-off flag so that it never reads an entry the
        // continuation writes
        NPHC_CK(cudaEventRecord(R->ev_fork, st));
        NPHC_CK(cudaStreamWaitEvent(R->side, R->ev_fork, 0));
        NPHC_CK(launch_compact(v, PRED_REACHED_DIRECT, R->flags, R->list[3], R->lcount + 3, R->side));
        WorkList l3 = {R->list[3], R->lcount + 3, nullptr, R->eg_s, R->eg_s_threads};
        NPHC_CK(launch_xy_refine_certify(S->M, xs, o->tol_sol, o->refine_eps, o->refine_iters, v,
                                         R->P, l3, 0, R->side));
        NPHC_CK(cudaEventRecord(R->ev_join, R->side));
        if ((s = track_impl(S, o, NPHC_PREC_FP64, ep, R->list[0], R->lcount + 5, true, true, R->ws, 1, st)))
            return s;
        NPHC_CK(cudaStreamWaitEvent(st, R->ev_join, 0));
        // then the continued entries (the shortcut's certified ones included) that reached t = 1
        NPHC_CK(launch_compact(v, PRED_REACHED_CONTINUED, R->flags, R->list[0], R->lcount + 7, st));
        WorkList l0c = {R->list[0], R->lcount + 7, nullptr, R->eg_s, R->eg_s_threads};
        NPHC_CK(launch_xy_refine_certify(S->M, xs, o->tol_sol, o->refine_eps, o->refine_iters, v,
                                         R->P, l0c, 0, st));
        // FP64 re-track from t = 0 of FP32 endpoints that did not certify
        NPHC_CK(launch_compact(v, PRED_UNCERTIFIED_FP32, R->flags, R->list[1], R->lcount + 1, st));
        if ((s = track_impl(S, o, NPHC_PREC_FP64, ep, R->list[1], R->lcount + 1, false, true, R->ws, 2, st)))
            return s;
        WorkList l1 = {R->list[1], R->lcount + 1, nullptr, R->eg_s, R->eg_s_threads};
        NPHC_CK(launch_xy_refine_certify(S->M, xs, o->tol_sol, o->refine_eps, o->refine_iters, v,
                                         R->P, l1, 0, st));
        // deduplicate; every path of a solution reached more than once is re-tracked in
        // FP64 and the endpoints are deduplicated again
        const Range r_dedup("dedup and re-track of duplicates");
        NPHC_CK(launch_dedup(v, R->n, kDedupDelta, dsc, R->list[2], R->lcount + 2, st));
        NPHC_CK(launch_flag_list(R->list[2], R->lcount + 2, R->P, R->flags, FLAG_RETRACKED_DUP, st));
        if ((s = track_impl(S, o, NPHC_PREC_FP64, ep, R->list[2], R->lcount + 2, false, true, R->ws, 3, st)))
            return s;
        WorkList l2 = {R->list[2], R->lcount + 2, nullptr, R->eg_s, R->eg_s_threads};
        NPHC_CK(launch_xy_refine_certify(S->M, xs, o->tol_sol, o->refine_eps, o->refine_iters, v,
                                         R->P, l2, 0, st));
        // a solution still reached twice means a path jumped in FP64 too: its paths are
        // tracked once more with an 8x smaller step ceiling and trust bound (only the
        // re-tracked entries can have changed: the dedups match just those)
        NPHC_CK(launch_dedup(v, R->n, kDedupDelta, dsc, R->list[0], R->lcount + 0, st, R->list[2],
                             R->lcount + 2));
        NPHC_CK(launch_flag_list(R->list[0], R->lcount + 0, R->P, R->flags, FLAG_RETRACKED_DUP, st));
        nphc_options strict = *o;
        strict.h_max = o->h_max / 8.0;
        strict.h0 = std::min(o->h0, strict.h_max);
        strict.trust = o->trust / 8.0;
        if ((s = track_impl(S, &strict, NPHC_PREC_FP64, ep, R->list[0], R->lcount + 0, false, true, R->ws, 4, st)))
            return s;
        WorkList l0s = {R->list[0], R->lcount + 0, nullptr, R->eg_s, R->eg_s_threads};
        NPHC_CK(launch_xy_refine_certify(S->M, xs, o->tol_sol, o->refine_eps, o->refine_iters, v,
                                         R->P, l0s, 0, st));
        NPHC_CK(launch_dedup(v, R->n, kDedupDelta, dsc, nullptr, nullptr, st, R->list[0], R->lcount + 0));
    } else {
        if ((s = track_impl(S, o, NPHC_PREC_FP64, ep, nullptr, nullptr, false, false, R->ws, 0, st)))
            return s;
        NPHC_CK(launch_compact(v, PRED_REACHED, R->flags, R->list[3], R->lcount + 3, st));
        WorkList l3 = {R->list[3], R->lcount + 3, nullptr, R->eg_s, R->eg_s_threads};
        NPHC_CK(launch_xy_refine_certify(S->M, xs, o->tol_sol, o->refine_eps, o->refine_iters, v,
                                         R->P, l3, 0, st));
        NPHC_CK(launch_dedup(v, R->n, kDedupDelta, dsc, nullptr, nullptr, st));
    }
    {
        const Range r("classify");
        // defaults for every entry (theta, energy, |lambda|_min, log|det H| 0; index -1), then
        // the real stationary points, compacted so that they fill whole warps
        NPHC_CK(cudaMemsetAsync(R->theta, 0, sizeof(double) * R->M * R->P, st));
        NPHC_CK(cudaMemsetAsync(R->energy, 0, sizeof(double) * R->P, st));
        NPHC_CK(cudaMemsetAsync(R->mineig, 0, sizeof(double) * R->P, st));
        NPHC_CK(cudaMemsetAsync(R->logdet, 0, sizeof(double) * R->P, st));
        NPHC_CK(cudaMemsetAsync(R->index, 0xff, sizeof(int32_t) * R->P, st));
        NPHC_CK(launch_real_list(v, R->real_list, R->lcount + 4, st));
        NPHC_CK(launch_xy_classify(S->M, xs, v, R->theta, R->index, R->energy, R->mineig, R->logdet, st,
                                   R->real_list, R->lcount + 4));
    }
    if ((s = endgame())) return s;
    NPHC_CK(launch_counts(v, R->flags, R->index, R->counts, st, R->egst, R->cycle));
    R->stream = st;
    R->solved = true;
    R->launches = nphc_launch_counter(0) - launches0;
    return NPHC_OK;
}

}  // namespace

extern "C" {

nphc_status nphc_solve_into(const nphc_system *S, const nphc_options *o, nphc_result *R,
                            void *stream) {
    return solve_into_impl(S, o, R, stream, false);
}

nphc_status nphc_solve(const nphc_system *S, const nphc_options *o, void *stream, nphc_result **out) {
    if (!out) return fail(NPHC_EINVAL, "out is NULL");
    nphc_result *R = nullptr;
    nphc_status s = nphc_result_create(S, &R);
    if (s != NPHC_OK) return s;
    s = nphc_solve_into(S, o, R, stream);
    if (s == NPHC_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) s = fail(NPHC_ECUDA, std::string("solve: ") + cudaGetErrorString(e));
    }
    if (s != NPHC_OK) {
        nphc_result_destroy(R);
        return s;
    }
    *out = R;
    return NPHC_OK;
}

nphc_status nphc_result_counts(const nphc_result *R, int64_t *counts) {
    if (!R || !counts) return fail(NPHC_EINVAL, "NULL argument");
    if (!R->solved) return fail(NPHC_ESTATE, "no solve on this result");
    NPHC_CK(cudaStreamSynchronize(R->stream));
    NPHC_CK(cudaMemcpy(counts, R->counts, sizeof(int64_t) * NPHC_NCOUNTS, cudaMemcpyDeviceToHost));
    counts[NPHC_COUNT_LAUNCHES] = R->launches;
    return NPHC_OK;
}

nphc_status nphc_result_copy_sps(const nphc_result *R, int64_t cap, double *theta, double *energy,
                                 int32_t *index, double *alpha, int64_t *path, double *log_abs_det,
                                 int64_t *n_out) {
    if (!R || !n_out || cap < 0) return fail(NPHC_EINVAL, "invalid argument");
    if (!R->solved) return fail(NPHC_ESTATE, "no solve on this result");
    if (R->M == 0) return fail(NPHC_EINVAL, "a generic quadratic system has no stationary points; copy its endpoints");
    cudaStream_t st = R->stream;
    NPHC_CK(launch_real_list(view(&R->ep), R->real_list, R->lcount + 4, st));
    NPHC_CK(launch_gather_sps(view(&R->ep), R->M, R->real_list, R->lcount + 4, R->P, R->theta,
                              R->index, R->energy, R->o_theta, R->o_index, R->o_energy, R->o_alpha,
                              R->o_path, R->logdet, R->o_logdet, st));
    int32_t cnt = 0;
    NPHC_CK(cudaMemcpyAsync(&cnt, R->lcount + 4, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    NPHC_CK(cudaStreamSynchronize(st));
    *n_out = cnt;
    const int64_t k = std::min<int64_t>(cnt, cap);
    if (k == 0) return NPHC_OK;
    const int M = R->M;
    std::vector<double> th(k * M), en(k), al(k);
    std::vector<int32_t> ix(k);
    std::vector<int64_t> pa(cnt);
    NPHC_CK(cudaMemcpy(pa.data(), R->o_path, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost));
    // the device list is unordered: order by path index, keep the first cap
    std::vector<int64_t> ord(cnt);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return pa[a] < pa[b]; });
    std::vector<double> th_all(cnt * M), en_all(cnt), al_all(cnt), ld_all(cnt);
    std::vector<int32_t> ix_all(cnt);
    NPHC_CK(cudaMemcpy(th_all.data(), R->o_theta, sizeof(double) * cnt * M, cudaMemcpyDeviceToHost));
    NPHC_CK(cudaMemcpy(en_all.data(), R->o_energy, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    NPHC_CK(cudaMemcpy(al_all.data(), R->o_alpha, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    NPHC_CK(cudaMemcpy(ld_all.data(), R->o_logdet, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    NPHC_CK(cudaMemcpy(ix_all.data(), R->o_index, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < k; i++) {
        const int64_t j = ord[i];
        if (theta) std::memcpy(theta + i * M, th_all.data() + j * M, sizeof(double) * M);
        if (energy) energy[i] = en_all[j];
        if (index) index[i] = ix_all[j];
        if (alpha) alpha[i] = al_all[j];
        if (path) path[i] = pa[j];
        if (log_abs_det) log_abs_det[i] = ld_all[j];
    }
    return NPHC_OK;
}

nphc_status nphc_result_copy_endgame(const nphc_result *R, int64_t cap, int32_t *cycle,
                                     int32_t *eg_status, int64_t *n_out) {
    if (!R || !n_out || cap < 0) return fail(NPHC_EINVAL, "invalid argument");
    if (!R->solved) return fail(NPHC_ESTATE, "no solve on this result");
    NPHC_CK(cudaStreamSynchronize(R->stream));
    *n_out = R->P;
    const int64_t k = std::min<int64_t>(R->P, cap);
    if (k == 0) return NPHC_OK;
    if (cycle) NPHC_CK(cudaMemcpy(cycle, R->cycle, sizeof(int32_t) * k, cudaMemcpyDeviceToHost));
    if (eg_status) NPHC_CK(cudaMemcpy(eg_status, R->egst, sizeof(int32_t) * k, cudaMemcpyDeviceToHost));
    return NPHC_OK;
}

nphc_status nphc_result_copy_endpoints(const nphc_result *R, int64_t cap, double *z_re,
                                       double *z_im, int32_t *status, int32_t *cls,
                                       int64_t *n_out) {
    if (!R || !n_out || cap < 0) return fail(NPHC_EINVAL, "invalid argument");
    if (!R->solved) return fail(NPHC_ESTATE, "no solve on this result");
    NPHC_CK(cudaStreamSynchronize(R->stream));
    *n_out = R->P;
    const int64_t k = std::min<int64_t>(cap, R->P);
    if (k == 0) return NPHC_OK;
    const int n = R->n;
    if (z_re || z_im) {
        std::vector<double> buf(R->P);
        for (int part = 0; part < 2; part++) {
            double *dst = part ? z_im : z_re;
            if (!dst) continue;
            const double *src = part ? R->ep.z_im : R->ep.z_re;
            for (int i = 0; i < n; i++) {
                NPHC_CK(cudaMemcpy(buf.data(), src + (size_t)i * R->P, sizeof(double) * k,
                                   cudaMemcpyDeviceToHost));
                for (int64_t e = 0; e < k; e++) dst[e * n + i] = buf[e];
            }
        }
    }
    if (status) NPHC_CK(cudaMemcpy(status, R->ep.status, sizeof(int32_t) * k, cudaMemcpyDeviceToHost));
    if (cls) NPHC_CK(cudaMemcpy(cls, R->ep.cls, sizeof(int32_t) * k, cudaMemcpyDeviceToHost));
    return NPHC_OK;
}

nphc_status nphc_result_endpoints(const nphc_result *R, nphc_endpoints *ep) {
    if (!R || !ep) return fail(NPHC_EINVAL, "NULL argument");
    *ep = R->ep;
    return NPHC_OK;
}

void nphc_result_destroy(nphc_result *R) {
    if (!R) return;
    if (R->block) {
        if (R->stream) cudaStreamSynchronize(R->stream);
        if (R->side) cudaStreamSynchronize(R->side);
        cudaFree(R->block);
    }
    if (R->ev_join) cudaEventDestroy(R->ev_join);
    if (R->ev_fork) cudaEventDestroy(R->ev_fork);
    if (R->side) cudaStreamDestroy(R->side);
    delete R;
}

}  // extern "C"

// ------------------------------------------------- allocation-free dedup --
// nphc_dedup_noalloc: the deduplication of nphc_dedup with its scratch in a fixed
// device array of this file instead of a caller workspace.  The array is sized for
// NPHC_DEDUP_NOALLOC_MAX entries with the same table layout as the workspace path:
// per level a power-of-two cell table of 2 x NPHC_DEDUP_NOALLOC_MAX slots (keys, list
// heads), per-entry list links and flags.
namespace {

constexpr int64_t kNoallocTable = 2 * (int64_t)NPHC_DEDUP_NOALLOC_MAX;
static_assert((kNoallocTable & (kNoallocTable - 1)) == 0 && kNoallocTable >= 1024,
              "the cell table must be a power of two of at least 1024 slots");
constexpr size_t noalloc_align(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kNoallocBytes =
    noalloc_align(sizeof(unsigned long long) * kNoallocTable * DD_LEVELS) +
    noalloc_align(sizeof(int32_t) * kNoallocTable * DD_LEVELS) +
    noalloc_align(sizeof(int32_t) * (size_t)NPHC_DEDUP_NOALLOC_MAX * DD_LEVELS) +
    noalloc_align(sizeof(int32_t) * (size_t)NPHC_DEDUP_NOALLOC_MAX);

static __device__ __align__(256) unsigned char g_dedup_noalloc_scratch[kNoallocBytes];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoallocMaxDevices] = {};
CUcontext g_noalloc_ctx[kNoallocMaxDevices] = {};

// The calling thread's current driver context, through the runtime's driver entry point
// (the library does not link the driver library itself); NULL when it cannot be queried.
CUcontext current_context() {
    using Fn = CUresult(CUDAAPI *)(CUcontext *);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(f);
        else
            cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Device address of the array in the current device's current context, looked up on the
// first call in that context and cached; a new context (after cudaDeviceReset, say) holds
// a new copy of the array and gets its own lookup.
nphc_status noalloc_scratch(void **out) {
    int dev = -1;
    NPHC_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(NPHC_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    CUcontext ctx = current_context();
    if (!g_noalloc_ptr[dev] || !ctx || ctx != g_noalloc_ctx[dev]) {
        void *p = nullptr;
        NPHC_CK(cudaGetSymbolAddress(&p, g_dedup_noalloc_scratch));
        if (!p) return fail(NPHC_ECUDA, "cudaGetSymbolAddress returned NULL");
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = current_context();   // the lookup may have created the context
    }
    *out = g_noalloc_ptr[dev];
    return NPHC_OK;
}

}  // namespace

extern "C" {

nphc_status nphc_dedup_noalloc(const nphc_system *S, const nphc_options *o,
                               const nphc_endpoints *ep, int32_t *dup_list, int32_t *dup_count,
                               void *stream) {
    nphc_status s;
    if ((s = check_ep(S, ep, true)) != NPHC_OK) return s;
    (void)o;
    if ((dup_list == nullptr) != (dup_count == nullptr)) return fail(NPHC_EINVAL, "list without count");
    if (ep->count > NPHC_DEDUP_NOALLOC_MAX)
        return fail(NPHC_EINVAL, "nphc_dedup_noalloc: " + std::to_string(ep->count) +
                                     " entries exceed NPHC_DEDUP_NOALLOC_MAX (" +
                                     std::to_string(NPHC_DEDUP_NOALLOC_MAX) +
                                     "); use nphc_dedup with a workspace");
    void *base = nullptr;
    if ((s = noalloc_scratch(&base)) != NPHC_OK) return s;
    if (ep->count == 0) {   // nothing to deduplicate; *dup_count is still an output
        if (dup_count) NPHC_CK(cudaMemsetAsync(dup_count, 0, sizeof(int32_t), (cudaStream_t)stream));
        return NPHC_OK;
    }
    // Same layout as the workspace path for this count, so both paths hash alike.
    const int64_t tsize = table_size_for(ep->count);
    char *b = static_cast<char *>(base);
    size_t off = 0;
    DedupScratch w;
    w.keys = reinterpret_cast<unsigned long long *>(b + off);
    off += align256(sizeof(unsigned long long) * tsize * DD_LEVELS);
    w.head = reinterpret_cast<int32_t *>(b + off);
    off += align256(sizeof(int32_t) * tsize * DD_LEVELS);
    w.next = reinterpret_cast<int32_t *>(b + off);
    off += align256(sizeof(int32_t) * ep->count * DD_LEVELS);
    w.inlist = reinterpret_cast<int32_t *>(b + off);
    off += align256(sizeof(int32_t) * ep->count);
    w.table_size = tsize;
    if (tsize > kNoallocTable || off > kNoallocBytes) return fail(NPHC_EINVAL, "scratch layout overflow");
    // launch_dedup clears the cell keys, list heads, flags and *dup_count itself with
    // cudaMemsetAsync on `stream`; the list links are written before they are read.
    NPHC_CK(launch_dedup(view(ep), S->n, kDedupDelta, w, dup_list, dup_count, (cudaStream_t)stream));
    return NPHC_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- batch --
// Independent systems solved together.  Default mode: the instances are grouped by ring
// size; each group's FP32 pass (every path of every instance in it) is one persistent
// launch pulling (instance, path) items from one queue, on internal stream g % 8, and the
// rest of each instance's method (hand-offs, FP64 continuation, refinement, certification,
// dedup, classification) runs on internal stream i % NPHC_BATCH_STREAMS once its group's
// pass is done.  NPHC_BATCH_PER_INSTANCE: every instance runs the whole of
// nphc_solve_into on its stream.  Streams are forked from the caller's stream and joined
// back with events.  The first solve of a batch runs eagerly (it also sets each kernel's
// attributes once); with NPHC_BATCH_GRAPH the second solve captures the whole fork /
// solve / join sequence into one CUDA graph (relaxed capture mode), and later solves with
// the same options replay it.
struct nphc_batch {
    struct Group {
        int M = 0;
        std::vector<int> members;   // instance indices
        int base = 0;               // first row of the group in the device tables
        cudaEvent_t done = nullptr;
    };
    std::vector<const nphc_system *> sys;
    std::vector<nphc_result *> res;
    std::vector<nphc_options> opts;   // options of the captured solve
    std::vector<Group> groups;
    void *tab = nullptr;              // device: XYSys[count] | EPView[count] | int64_t[count + groups]
    XYSys *d_sys = nullptr;
    EPView *d_ep = nullptr;
    int64_t *d_off = nullptr;
    std::vector<nphc_options> tab_opts;   // options the XYSys rows were written with
    bool tab_valid = false;
    cudaStream_t streams[NPHC_BATCH_STREAMS] = {};
    cudaStream_t origin = nullptr;    // the captured stream (the caller's may be the legacy one)
    cudaEvent_t start = nullptr, done = nullptr;
    cudaEvent_t fork = nullptr, join[NPHC_BATCH_STREAMS] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int solves = 0;
    int mode = -1;                    // flags of the captured solve
    int64_t launches = 0;
};

namespace {

bool same_options(const std::vector<nphc_options> &a, const nphc_options *b) {
    for (size_t i = 0; i < a.size(); i++)
        if (std::memcmp(&a[i], &b[i], sizeof(nphc_options)) != 0) return false;
    return true;
}

// A group's FP32 pass can be one launch when every member is an XY ring solved in mixed
// precision with the same FP32 step control (gamma and kappa_sing live in each member's
// couplings row).
bool group_batchable(const nphc_batch *B, const nphc_batch::Group &G, const nphc_options *opts) {
    const XYCtl c0 = make_ctl(&opts[G.members[0]], true, false, false);
    for (int i : G.members) {
        if (B->sys[i]->quad || opts[i].precision != NPHC_PREC_MIXED) return false;
        const XYCtl c = make_ctl(&opts[i], true, false, false);
        if (std::memcmp(&c, &c0, sizeof(XYCtl)) != 0) return false;
        if (opts[i].blocks_per_sm != opts[G.members[0]].blocks_per_sm) return false;
    }
    return true;
}

// Writes every instance's couplings row (with its own gamma and kappa_sing) to the device
// table when the options changed since the last write.  The rows are read by the group
// launches of earlier solves, so every stream of the batch is drained first.
nphc_status batch_tables(nphc_batch *B, const nphc_options *opts, cudaStream_t st) {
    if (B->tab_valid && same_options(B->tab_opts, opts)) return NPHC_OK;
    const size_t n = B->sys.size();
    std::vector<XYSys> rows(n);
    for (const auto &G : B->groups)
        for (size_t r = 0; r < G.members.size(); r++) {
            const int i = G.members[r];
            rows[G.base + r] = sys_with_gamma(B->sys[i], &opts[i]);
        }
    NPHC_CK(cudaStreamSynchronize(st));
    NPHC_CK(cudaStreamSynchronize(B->origin));
    for (int k = 0; k < NPHC_BATCH_STREAMS; k++) NPHC_CK(cudaStreamSynchronize(B->streams[k]));
    NPHC_CK(cudaMemcpy(B->d_sys, rows.data(), sizeof(XYSys) * n, cudaMemcpyHostToDevice));
    B->tab_opts.assign(opts, opts + n);
    B->tab_valid = true;
    return NPHC_OK;
}

nphc_status batch_enqueue(nphc_batch *B, const nphc_options *opts, int mode, cudaStream_t st) {
    const Range whole("nphc_batch_solve");
    NPHC_CK(cudaEventRecord(B->fork, st));
    for (int k = 0; k < NPHC_BATCH_STREAMS; k++) NPHC_CK(cudaStreamWaitEvent(B->streams[k], B->fork, 0));
    std::vector<int> group_of(B->sys.size(), -1);   // -1: the instance runs the whole solve
    if (!(mode & NPHC_BATCH_PER_INSTANCE)) {
        for (size_t g = 0; g < B->groups.size(); g++) {
            const nphc_batch::Group &G = B->groups[g];
            if (!group_batchable(B, G, opts)) continue;
            nphc_result *R0 = B->res[G.members[0]];
            const nphc_options *o0 = &opts[G.members[0]];
            cudaStream_t gs = B->streams[g % NPHC_BATCH_STREAMS];
            XYCtl ctl = make_ctl(o0, true, false, false);
            WorkList wl;
            wl.list = nullptr;
            wl.list_count = nullptr;
            wl.queue = ws_queue(R0->ws, 0);
            wl.state = static_cast<char *>(R0->ws) + ws_layout(R0->n, 0).state;
            wl.state_threads = NPHC_TRACK_MAX_THREADS;
            BatchGroup bg;
            bg.sys = B->d_sys + G.base;
            bg.ep = B->d_ep + G.base;
            bg.off = B->d_off + G.base + g;
            bg.n = (int)G.members.size();
            bg.total = 0;
            for (int i : G.members) bg.total += B->sys[i]->npaths;
            int grid = 0;
            if (o0->blocks_per_sm > 0) {
                int dev = 0, sms = 0;
                NPHC_CK(cudaGetDevice(&dev));
                NPHC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
                grid = sms * o0->blocks_per_sm;
            }
            const Range r("batch group fp32 pass");
            NPHC_CK(cudaMemsetAsync(wl.queue, 0, sizeof(unsigned long long), gs));
            NPHC_CK(launch_xy_track_f32_batch(G.M, bg, ctl, wl, grid, gs));
            NPHC_CK(cudaEventRecord(G.done, gs));
            for (int i : G.members) group_of[i] = (int)g;
        }
    }
    for (size_t i = 0; i < B->sys.size(); i++) {
        cudaStream_t is = B->streams[i % NPHC_BATCH_STREAMS];
        if (group_of[i] >= 0) NPHC_CK(cudaStreamWaitEvent(is, B->groups[group_of[i]].done, 0));
        nphc_status s = solve_into_impl(B->sys[i], &opts[i], B->res[i], is, group_of[i] >= 0);
        if (s != NPHC_OK) return s;
    }
    for (int k = 0; k < NPHC_BATCH_STREAMS; k++) {
        NPHC_CK(cudaEventRecord(B->join[k], B->streams[k]));
        NPHC_CK(cudaStreamWaitEvent(st, B->join[k], 0));
    }
    return NPHC_OK;
}

}  // namespace

extern "C" {

void nphc_batch_destroy(nphc_batch *B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (int k = 0; k < NPHC_BATCH_STREAMS; k++) {
        if (B->streams[k]) {
            cudaStreamSynchronize(B->streams[k]);
            cudaStreamDestroy(B->streams[k]);
        }
        if (B->join[k]) cudaEventDestroy(B->join[k]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->origin) {
        cudaStreamSynchronize(B->origin);
        cudaStreamDestroy(B->origin);
    }
    if (B->start) cudaEventDestroy(B->start);
    if (B->done) cudaEventDestroy(B->done);
    for (auto &G : B->groups)
        if (G.done) cudaEventDestroy(G.done);
    if (B->tab) cudaFree(B->tab);
    for (nphc_result *R : B->res) nphc_result_destroy(R);
    delete B;
}

nphc_status nphc_batch_create(int count, const nphc_system *const *systems, nphc_batch **out) {
    if (!out) return fail(NPHC_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !systems) return fail(NPHC_EINVAL, "empty batch");
    for (int i = 0; i < count; i++)
        if (!systems[i]) return fail(NPHC_EINVAL, "NULL system in the batch");
    nphc_batch *B = new (std::nothrow) nphc_batch;
    if (!B) return fail(NPHC_ENOMEM, "host allocation");
    auto bail = [&](nphc_status s) {
        nphc_batch_destroy(B);
        return s;
    };
    for (int k = 0; k < NPHC_BATCH_STREAMS; k++) {
        if (cudaStreamCreateWithFlags(&B->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->join[k], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(NPHC_ECUDA, "batch streams"));
    }
    if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(NPHC_ECUDA, "batch events"));
    for (int i = 0; i < count; i++) {
        nphc_result *R = nullptr;
        nphc_status s = nphc_result_create(systems[i], &R);
        if (s != NPHC_OK) return bail(s);
        B->sys.push_back(systems[i]);
        B->res.push_back(R);
    }
    // groups of XY rings by size (generic quadratic systems always run alone)
    for (int i = 0; i < count; i++) {
        if (systems[i]->quad) continue;
        auto it = std::find_if(B->groups.begin(), B->groups.end(),
                               [&](const nphc_batch::Group &G) { return G.M == systems[i]->M; });
        if (it == B->groups.end()) {
            B->groups.emplace_back();
            B->groups.back().M = systems[i]->M;
            it = B->groups.end() - 1;
        }
        it->members.push_back(i);
    }
    int row = 0;
    for (auto &G : B->groups) {
        G.base = row;
        row += (int)G.members.size();
        if (cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(NPHC_ECUDA, "batch events"));
    }
    // device tables: couplings rows (written per solve), endpoint views, path offsets
    const size_t nrow = (size_t)(row > 0 ? row : 1), ng = B->groups.size();
    const size_t b_sys = align256(sizeof(XYSys) * nrow), b_ep = align256(sizeof(EPView) * nrow);
    const size_t b_off = align256(sizeof(int64_t) * (nrow + ng + 1));
    cudaError_t e = cudaMalloc(&B->tab, b_sys + b_ep + b_off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(e == cudaErrorMemoryAllocation ? NPHC_ENOMEM : NPHC_ECUDA,
                         std::string("batch tables: ") + cudaGetErrorString(e)));
    }
    B->d_sys = reinterpret_cast<XYSys *>(B->tab);
    B->d_ep = reinterpret_cast<EPView *>(static_cast<char *>(B->tab) + b_sys);
    B->d_off = reinterpret_cast<int64_t *>(static_cast<char *>(B->tab) + b_sys + b_ep);
    std::vector<EPView> eps(nrow);
    std::vector<int64_t> off;
    for (const auto &G : B->groups) {
        int64_t acc = 0;
        for (size_t r = 0; r < G.members.size(); r++) {
            const int i = G.members[r];
            eps[G.base + r] = view(&B->res[i]->ep);
            off.push_back(acc);
            acc += systems[i]->npaths;
        }
        off.push_back(acc);   // group g's offsets start at row base + g
    }
    if (row > 0) {
        e = cudaMemcpy(B->d_ep, eps.data(), sizeof(EPView) * row, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(B->d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(fail(NPHC_ECUDA, std::string("batch tables: ") + cudaGetErrorString(e)));
    }
    *out = B;
    return NPHC_OK;
}

nphc_status nphc_batch_solve(nphc_batch *B, const nphc_options *opts, int flags, void *stream) {
    if (!B || !opts) return fail(NPHC_EINVAL, "NULL argument");
    if (flags & ~(NPHC_BATCH_GRAPH | NPHC_BATCH_PER_INSTANCE)) return fail(NPHC_EINVAL, "unknown batch flags");
    for (size_t i = 0; i < B->sys.size(); i++) {
        nphc_status s = check_opt(&opts[i]);
        if (s != NPHC_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int mode = flags & NPHC_BATCH_PER_INSTANCE;
    if (B->exec && (!same_options(B->opts, opts) || B->mode != mode)) {   // capture again
        cudaGraphExecDestroy(B->exec);
        cudaGraphDestroy(B->graph);
        B->exec = nullptr;
        B->graph = nullptr;
    }
    nphc_status s;
    if (!mode && (s = batch_tables(B, opts, st)) != NPHC_OK) return s;
    const bool graph = (flags & NPHC_BATCH_GRAPH) != 0;
    if (graph && B->exec) {
        NPHC_CK(cudaGraphLaunch(B->exec, st));
        nphc_launch_counter(B->launches);
    } else if (graph && B->solves > 0) {
        // capture on the batch's own stream: the graph then runs on the caller's
        NPHC_CK(cudaEventRecord(B->start, st));
        NPHC_CK(cudaStreamWaitEvent(B->origin, B->start, 0));
        NPHC_CK(cudaStreamSynchronize(B->origin));
        const int64_t l0 = nphc_launch_counter(0);
        NPHC_CK(cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeRelaxed));
        s = batch_enqueue(B, opts, mode, B->origin);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(B->origin, &g);
        if (s != NPHC_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        NPHC_CK(e);
        B->graph = g;
        NPHC_CK(cudaGraphInstantiate(&B->exec, g, 0));
        B->launches = nphc_launch_counter(0) - l0;
        B->opts.assign(opts, opts + B->sys.size());
        B->mode = mode;
        NPHC_CK(cudaGraphLaunch(B->exec, st));
    } else {
        if ((s = batch_enqueue(B, opts, mode, st)) != NPHC_OK) return s;
    }
    for (nphc_result *R : B->res) R->stream = st;   // results are read after the join
    B->solves++;
    return NPHC_OK;
}

nphc_status nphc_batch_result(const nphc_batch *B, int i, const nphc_result **out) {
    if (!B || !out || i < 0 || i >= (int)B->res.size()) return fail(NPHC_EINVAL, "invalid argument");
    *out = B->res[i];
    return NPHC_OK;
}

}  // extern "C"

