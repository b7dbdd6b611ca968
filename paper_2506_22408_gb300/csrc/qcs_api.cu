// qcs_api.cu -- the C ABI of libqcs (declared in include/qcs.h).
//
// Host-side argument checking, the per-device context and its workspace, the
// interpolation-node plan, and the kernel launch sequence of each entry point.
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "qcs_gauss_nodes.h"
#include "qcs_internal.h"

// ------------------------------------------------------------ helpers

int qcs_log_level() {
    static const int level = [] {
        const char *e = std::getenv("QCS_LOG");
        const int v = e ? std::atoi(e) : 0;
        return v < 0 ? 0 : (v > 3 ? 3 : v);
    }();
    return level;
}

void qcs_log(int level, const char *fmt, ...) {
    if (level > qcs_log_level()) return;
    va_list ap;
    va_start(ap, fmt);
    std::fputs("[qcs] ", stderr);
    std::vfprintf(stderr, fmt, ap);
    std::fputc('\n', stderr);
    va_end(ap);
}

QcsRange::QcsRange(const char *name) {
    nvtxRangePushA(name);
    qcs_log(2, "%s", name);
}
QcsRange::~QcsRange() { nvtxRangePop(); }

qcs_status qcs_fail(qcs_ctx *ctx, qcs_status code, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    qcs_log(1, "error %d: %s", (int)code, msg.c_str());
    return code;
}

qcs_status qcs_check_launch(qcs_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    qcs_log(3, "launched %s", what);
    return QCS_OK;
}

qcs_status qcs_set_smem(qcs_ctx *ctx, const void *func, size_t bytes) {
    if (bytes > ctx->smem_optin) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "shared memory request too large");
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    // prefer the largest shared-memory carveout so that the blocks the occupancy
    // calculation allows are actually co-resident
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    return QCS_OK;
}

qcs_status qcs_dev_alloc(const qcs_allocator &a, void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (a.alloc) {
        *p = a.alloc(bytes, (void *)st, a.user);
        return *p ? QCS_OK : QCS_ERR_CUDA;
    }
    return cudaMalloc(p, bytes) == cudaSuccess ? QCS_OK : QCS_ERR_CUDA;
}

void qcs_dev_free(const qcs_allocator &a, void *p, size_t bytes) {
    if (!p) return;
    if (a.free) a.free(p, bytes, nullptr, a.user);
    else cudaFree(p);
}

qcs_status qcs_workspace(qcs_ctx *ctx, size_t bytes, void **out, cudaStream_t st) {
    bytes = align16(bytes < 16 ? 16 : bytes);
    if (bytes > ctx->work_bytes) {
        if (ctx->work) {
            cudaDeviceSynchronize();
            qcs_dev_free(ctx->alloc, ctx->work, ctx->work_bytes);
            ctx->work = nullptr;
            ctx->work_bytes = 0;
        }
        if (qcs_dev_alloc(ctx->alloc, &ctx->work, bytes, st) != QCS_OK)
            return qcs_fail(ctx, QCS_ERR_CUDA, ctx->alloc.alloc ? "workspace: the allocator callback returned NULL"
                                                                 : "workspace: cudaMalloc failed");
        ctx->work_bytes = bytes;
    }
    *out = ctx->work;
    return QCS_OK;
}

extern "C" qcs_status qcs_set_allocator(qcs_ctx *ctx, qcs_alloc_fn alloc_fn, qcs_free_fn free_fn, void *user) {
    if (!ctx) return QCS_ERR_ARG;
    if ((alloc_fn == nullptr) != (free_fn == nullptr))
        return qcs_fail(ctx, QCS_ERR_ARG, "qcs_set_allocator: give both functions or neither");
    DeviceGuard g(ctx->device);
    if (ctx->work) {  // later growth comes from the new allocator
        if (cudaDeviceSynchronize() != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, "qcs_set_allocator: synchronise");
        qcs_dev_free(ctx->alloc, ctx->work, ctx->work_bytes);
        ctx->work = nullptr;
        ctx->work_bytes = 0;
    }
    ctx->alloc.alloc = alloc_fn;
    ctx->alloc.free = free_fn;
    ctx->alloc.user = user;
    return QCS_OK;
}

void qcs_prof_begin(qcs_ctx *ctx, cudaStream_t st) {
    if (!ctx->profiling) return;
    std::pair<cudaEvent_t, cudaEvent_t> ev;
    if (!ctx->prof_pool.empty()) {
        ev = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
    } else {
        cudaEventCreate(&ev.first);
        cudaEventCreate(&ev.second);
    }
    cudaEventRecord(ev.first, st);
    ctx->prof_events.push_back(ev);
}

void qcs_prof_end(qcs_ctx *ctx, cudaStream_t st) {
    if (!ctx->profiling || ctx->prof_events.empty()) return;
    cudaEventRecord(ctx->prof_events.back().second, st);
}

namespace {

double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return std::floor(r + 0.5);
}

qcs_status check_sizes(qcs_ctx *ctx, int n, int ne) {
    if (n < 1 || n > QCS_MAX_N) return qcs_fail(ctx, QCS_ERR_ARG, "n must be in [1, QCS_MAX_N]");
    if (ne < 2 || ne > n) return qcs_fail(ctx, QCS_ERR_ARG, "ne must satisfy 2 <= ne <= n");
    if (ne & 1) return qcs_fail(ctx, QCS_ERR_ARG, "ne must be even (odd-particle shadow overlaps vanish)");
    return QCS_OK;
}

}  // namespace

// Node plans.  pf(A(z)) = z^{ne/2} q(z) with deg q <= d = n - ne, and the
// estimator needs L(q) = sum_t w'_t c'_t, w'_t = C(2n, ne+2t)/C(n, ne/2+t).
// The kernels evaluate pf'_k = pf(B + wnode_k D) and sum gamma_k pf'_k.
//
// Default plan (Gauss): for parity +1 snapshots q is palindromic, so L is a
// linear functional on a space of dimension D = floor(d/2)+1 and a Gauss rule
// with ceil(D/2) nodes on the unit circle computes it exactly; the nodes and
// weights are tabulated in qcs_gauss_nodes.h (derivation in gen_gauss_nodes.py).
//
// Roots-of-unity plan (nodes > 0 or QCS_FLAG_DFT_NODES): N >= d+1
// roots of unity z_k = w^k determine q exactly: c'_t = (1/N) sum_k q_k w^{-kt}.  The
// estimator needs sum_t w'_t c'_t with w'_t = C(2n, ne+2t)/C(n, ne/2+t), i.e.
// sum_k beta_k q_k with beta_k = (1/N) sum_t w'_t w^{-kt}.  The kernels evaluate
// pf'_k = pf(B + conj(z_k) D) = z_k^{-m/2} pf(A(z_k)), so q_k = z_k^d pf'_k.
// For parity +1 snapshots c'_{d-t} = c'_t gives q_{N-k} = w^{-kd} q_k, and the
// pairs (k, N-k) merge: only k = 0..floor(N/2) are evaluated.
qcs_status qcs_make_node_plan(int n, int ne, int nodes, unsigned flags, qcs_node_plan *plan) {
    const int d = n - ne;
    if (n < 2 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1)) return QCS_ERR_ARG;
    if (nodes < 0) return QCS_ERR_ARG;
    if (nodes == 0 && !(flags & (QCS_FLAG_ALL_NODES | QCS_FLAG_DFT_NODES))) {
        const qcs_gauss_rule &g = qcs_gauss_rules[n][ne];
        if (g.k < 1 || g.k > QCS_MAX_NODES) return QCS_ERR_ARG;
        plan->N = 0;
        plan->all = 0;
        plan->nev = g.k;
        for (int k = 0; k < g.k; ++k) {
            plan->wnode[k] = cmk(g.node[k][0], g.node[k][1]);
            plan->gamma[k] = cmk(g.node[k][2], g.node[k][3]);
        }
        return QCS_OK;
    }
    int N = nodes > 0 ? nodes : d + 1;
    if (N < d + 1 || N > QCS_MAX_NODES) return QCS_ERR_ARG;
    typedef std::complex<double> C;
    const double tw = 2.0 * M_PI / (double)N;
    std::vector<C> beta(N);
    for (int k = 0; k < N; ++k) {
        C s = 0.0;
        for (int t = 0; t <= d; ++t) {
            double wt = binom(2 * n, ne + 2 * t) / binom(n, ne / 2 + t);
            double ang = -tw * (double)(((long long)k * t) % N);
            s += wt * C(std::cos(ang), std::sin(ang));
        }
        beta[k] = s / (double)N;
    }
    auto wpow = [&](long long e) {
        long long r = ((e % N) + N) % N;
        double ang = tw * (double)r;
        return C(std::cos(ang), std::sin(ang));
    };
    plan->N = N;
    plan->all = (flags & QCS_FLAG_ALL_NODES) ? 1 : 0;
    if (plan->all) {
        plan->nev = N;
        for (int k = 0; k < N; ++k) {
            C wn = wpow(-k), g = beta[k] * wpow((long long)k * d);
            plan->wnode[k] = cmk(wn.real(), wn.imag());
            plan->gamma[k] = cmk(g.real(), g.imag());
        }
    } else {
        const int K = N / 2;
        plan->nev = K + 1;
        for (int k = 0; k <= K; ++k) {
            C wn = wpow(-k), g;
            if (k == 0) g = beta[0];
            else if (2 * k == N) g = beta[k] * wpow((long long)k * d);
            else g = beta[k] * wpow((long long)k * d) + beta[N - k];
            plan->wnode[k] = cmk(wn.real(), wn.imag());
            plan->gamma[k] = cmk(g.real(), g.imag());
        }
    }
    return QCS_OK;
}

// ------------------------------------------------------------ context

extern "C" qcs_status qcs_create(qcs_ctx **ctx, int device) {
    if (!ctx) return QCS_ERR_ARG;
    *ctx = nullptr;
    qcs_ctx *c = new qcs_ctx();
    c->device = device;
    DeviceGuard g(device);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)optin;
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    c->smem_per_sm = (size_t)per_sm;
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_status, sizeof(unsigned));
    if (e != cudaSuccess) {
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        qcs_log(1, "qcs_create(device %d): %s", device, cudaGetErrorString(e));
        return QCS_ERR_CUDA;
    }
    *ctx = c;
    qcs_log(2, "qcs_create(device %d): %d SMs, %zu bytes of shared memory per block", device, c->num_sms,
            c->smem_optin);
    return QCS_OK;
}

extern "C" qcs_status qcs_destroy(qcs_ctx *ctx) {
    if (!ctx) return QCS_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    qcs_dev_free(ctx->alloc, ctx->work, ctx->work_bytes);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    for (auto &ev : ctx->prof_events) ctx->prof_pool.push_back(ev);
    for (auto &ev : ctx->prof_pool) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    delete ctx;
    return QCS_OK;
}

extern "C" qcs_status qcs_profile_enable(qcs_ctx *ctx, int enable) {
    if (!ctx) return QCS_ERR_ARG;
    ctx->profiling = enable != 0;
    return QCS_OK;
}

extern "C" qcs_status qcs_profile_read(qcs_ctx *ctx, double *total_ms, int64_t *launches) {
    if (!ctx || !total_ms || !launches) return QCS_ERR_ARG;
    DeviceGuard g(ctx->device);
    double tot = 0.0;
    for (auto &ev : ctx->prof_events) {
        cudaError_t e = cudaEventSynchronize(ev.second);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.first, ev.second);
        if (e != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, std::string("qcs_profile_read: ") + cudaGetErrorString(e));
        tot += ms;
        ctx->prof_pool.push_back(ev);
    }
    *launches = (int64_t)ctx->prof_events.size();
    *total_ms = tot;
    ctx->prof_events.clear();
    return QCS_OK;
}

extern "C" const char *qcs_last_error(const qcs_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

extern "C" size_t qcs_workspace_bytes(const qcs_ctx *ctx) { return ctx ? ctx->work_bytes : 0; }

extern "C" qcs_status qcs_sync_status(qcs_ctx *ctx, void *stream) {
    if (!ctx) return QCS_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, std::string("qcs_sync_status: ") + cudaGetErrorString(e));
    return (qcs_status)(*ctx->h_status);
}

// ------------------------------------------------------------ snapshots

extern "C" qcs_status qcs_build_snapshots(qcs_ctx *ctx, int n, int64_t P, const double *d_Q, const uint8_t *d_b,
                                          qcs_snapshots **out, void *stream) {
    QcsRange range_("qcs_build_snapshots");
    if (!ctx || !out) return QCS_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > QCS_MAX_N) return qcs_fail(ctx, QCS_ERR_ARG, "n must be in [1, QCS_MAX_N]");
    if (P < 0 || P > (int64_t)INT32_MAX) return qcs_fail(ctx, QCS_ERR_ARG, "P out of range");
    if (P > 0 && (!d_Q || !d_b)) return qcs_fail(ctx, QCS_ERR_ARG, "null snapshot input");
    DeviceGuard g(ctx->device);
    qcs_snapshots *s = new qcs_snapshots();
    s->n = n;
    s->P = P;
    s->device = ctx->device;
    s->alloc = ctx->alloc;
    const int64_t Pa = P > 0 ? P : 1;
    const cudaStream_t cs = (cudaStream_t)stream;
    qcs_status ae = qcs_dev_alloc(s->alloc, (void **)&s->Qt, sizeof(cd) * (size_t)Pa * 2 * n * n, cs);
    if (ae == QCS_OK) ae = qcs_dev_alloc(s->alloc, (void **)&s->parity, (size_t)Pa, cs);
    if (ae == QCS_OK) ae = qcs_dev_alloc(s->alloc, (void **)&s->idx, sizeof(int) * (size_t)Pa, cs);
    if (ae == QCS_OK) ae = qcs_dev_alloc(s->alloc, (void **)&s->d_count, 2 * sizeof(int), cs);
    if (ae == QCS_OK) ae = qcs_dev_alloc(s->alloc, (void **)&s->gth, (size_t)Pa * 2 * n, cs);
    if (ae != QCS_OK) {
        qcs_snapshots_free(s);
        return qcs_fail(ctx, QCS_ERR_CUDA, "snapshot set: device allocation failed");
    }
    qcs_status st = qcs_launch_snapshot_build(ctx, s, d_Q, d_b, (cudaStream_t)stream);
    // the tensor-core congruence is the default FP64 path at n = 16: its per-snapshot
    // records are formed with the set
    if (st == QCS_OK && n == 16) st = qcs_tc_prepare_snapshots(ctx, s, (cudaStream_t)stream);
    if (st != QCS_OK) {
        qcs_snapshots_free(s);
        return st;
    }
    *out = s;
    return QCS_OK;
}

extern "C" qcs_status qcs_snapshots_signed_perm_count(const qcs_snapshots *s, int64_t *count, void *stream) {
    if (!s || !count) return QCS_ERR_ARG;
    DeviceGuard g(s->device);
    int h = 0;
    if (cudaMemcpyAsync(&h, s->d_count + 1, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return QCS_ERR_CUDA;
    *count = s->P > 0 ? (int64_t)h : 0;
    return QCS_OK;
}

extern "C" qcs_status qcs_snapshots_free(qcs_snapshots *s) {
    if (!s) return QCS_ERR_ARG;
    DeviceGuard g(s->device);
    cudaDeviceSynchronize();
    const int n = s->n;
    const size_t Pa = (size_t)(s->P > 0 ? s->P : 1);
    qcs_dev_free(s->alloc, s->Qt, sizeof(cd) * Pa * 2 * n * n);
    qcs_dev_free(s->alloc, s->parity, Pa);
    qcs_dev_free(s->alloc, s->idx, sizeof(int) * Pa);
    qcs_dev_free(s->alloc, s->d_count, 2 * sizeof(int));
    qcs_dev_free(s->alloc, s->gth, Pa * 2 * n);
    qcs_dev_free(s->alloc, s->split_hi, s->split_bytes);
    qcs_dev_free(s->alloc, s->split_lo, s->split_bytes);
    qcs_dev_free(s->alloc, s->tc_rec, s->tc_bytes);
    qcs_dev_free(s->alloc, s->Qh, s->qh_bytes);
    delete s;
    return QCS_OK;
}

extern "C" qcs_status qcs_snapshots_parity(const qcs_snapshots *s, int8_t *d_parity, void *stream) {
    if (!s || (!d_parity && s->P > 0)) return QCS_ERR_ARG;
    if (s->P == 0) return QCS_OK;
    DeviceGuard g(s->device);
    cudaError_t e = cudaMemcpyAsync(d_parity, s->parity, (size_t)s->P, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? QCS_OK : QCS_ERR_CUDA;
}

extern "C" int64_t qcs_snapshots_count(const qcs_snapshots *s) { return s ? s->P : -1; }
extern "C" int qcs_snapshots_modes(const qcs_snapshots *s) { return s ? s->n : -1; }

// ------------------------------------------------------------ overlaps

namespace {

const int kChunk = 4;  // snapshots per warp in an overlap tile

struct OverlapWork {
    cd *Ut, *pref, *partial;
    unsigned long long *counter;
    float *Mhi, *Mlo;          // split precision: walker operand slabs
    unsigned char *walk_rec;   // tensor-core congruence: walker slice records
    int *mode;                 // FP64 ALU path: per-walker form of the occupied rows (walker prep)
    int nchunks, nparts;
    int config, chunk;         // resolved kernel configuration, ALU snapshots per warp in a tile
    bool split, tc;
};

// The configuration of an overlap call: opts->config, else the context's tuned entry for
// these sizes and options, else 0 (built-in defaults).
int resolve_config(qcs_ctx *ctx, int n, int ne, const qcs_opts &o) {
    if (o.config > 0) return o.config;
    auto it = ctx->tuned.find(std::make_tuple(n, ne, o.nodes, o.flags));
    return it != ctx->tuned.end() ? it->second : 0;
}

// The FP64 overlap runs its congruence on tensor cores (qcs_tcpair.cu) by default at
// n = 16, on request (QCS_FLAG_FP64_TC) for any n <= 16, and on the FP64 ALU
// otherwise (QCS_FLAG_FP64_ALU, n > 16, or every node of every snapshot).
// A configured path (qcs_config.path, from the autotuner) applies when no flag names one.
qcs_status choose_tc(qcs_ctx *ctx, int n, const qcs_opts &o, int config, bool *tc) {
    *tc = false;
    if (o.precision != QCS_FP64) return QCS_OK;
    if ((o.flags & QCS_FLAG_FP64_TC) && (o.flags & QCS_FLAG_FP64_ALU))
        return qcs_fail(ctx, QCS_ERR_ARG, "QCS_FLAG_FP64_TC and QCS_FLAG_FP64_ALU exclude each other");
    const bool possible = qcs_tc_supported(n) && !(o.flags & QCS_FLAG_ALL_NODES);
    if (o.flags & QCS_FLAG_FP64_TC) {
        if (!possible)
            return qcs_fail(ctx, QCS_ERR_UNSUPPORTED,
                            "the tensor-core congruence needs n <= 16 and the parity-compacted snapshot list");
        *tc = true;
        return QCS_OK;
    }
    if (o.flags & QCS_FLAG_FP64_ALU) return QCS_OK;
    const int path = qcs_decode_config(config).path;
    *tc = possible && (path == 2 || (path == 0 && n == 16));
    return QCS_OK;
}

qcs_status overlap_common(qcs_ctx *ctx, const qcs_snapshots *s, int ne, int64_t W, const double *d_walkers,
                          const qcs_opts *opts, cudaStream_t st, qcs_node_plan *plan, OverlapWork *wk) {
    if (!ctx) return QCS_ERR_ARG;
    if (!s) return qcs_fail(ctx, QCS_ERR_ARG, "null snapshot set");
    if (s->device != ctx->device) return qcs_fail(ctx, QCS_ERR_ARG, "snapshot set lives on another device");
    const int n = s->n;
    qcs_status c = check_sizes(ctx, n, ne);
    if (c != QCS_OK) return c;
    if (W < 0) return qcs_fail(ctx, QCS_ERR_ARG, "W < 0");
    if (W > 0 && !d_walkers) return qcs_fail(ctx, QCS_ERR_ARG, "null walkers");
    qcs_opts o = {QCS_FP64, 0, 0u, 0};
    if (opts) o = *opts;
    if (o.precision != QCS_FP64 && o.precision != QCS_TF32X3)
        return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "unknown precision mode");
    if (qcs_make_node_plan(n, ne, o.nodes, o.flags, plan) != QCS_OK)
        return qcs_fail(ctx, QCS_ERR_ARG, "nodes must be 0 or in [n-ne+1, QCS_MAX_NODES]");
    const bool split = o.precision == QCS_TF32X3;
    // the tuned table belongs to the FP64 pair kernels
    wk->config = split ? o.config : resolve_config(ctx, n, ne, o);
    const qcs_config cfg = qcs_decode_config(wk->config);
    bool tc = false;
    c = choose_tc(ctx, n, o, wk->config, &tc);
    if (c != QCS_OK) return c;
    wk->split = split;
    wk->tc = tc;
    wk->chunk = cfg.chunk > 0 ? cfg.chunk : kChunk;
    // partial sums: FP64 ALU path one per (walker, tile, warp); split path one per
    // (walker, tile of snapshots); tensor-core path one per (walker, tile)
    const int span = split ? qcs_split_snaps_per_tile(n, cfg.subs) : tc ? qcs_tc_snaps_per_tile(cfg.subs)
                                                             : wk->chunk * qcs_pair_warps_per_block();
    wk->nchunks = (int)((s->P + span - 1) / span);
    if (wk->nchunks < 1) wk->nchunks = 1;
    wk->nparts = (split || tc) ? wk->nchunks : wk->nchunks * qcs_pair_warps_per_block();
    qcs_log(2, "  n=%d ne=%d W=%lld P=%lld nodes=%d path=%s config=0x%x tiles of %d snapshots", n, ne, (long long)W,
            (long long)s->P, plan->nev, split ? "split-tf32x3" : (tc ? "fp64-tensor-core" : "fp64-alu"),
            (unsigned)wk->config, span);
    size_t b_ut = align16(sizeof(cd) * (size_t)W * n * n);
    size_t b_pref = align16(sizeof(cd) * (size_t)W);
    size_t b_part = align16(sizeof(cd) * (size_t)W * wk->nparts);
    size_t b_slab = split ? align16(qcs_split_walker_bytes(n, W)) : 0;
    size_t b_rec = tc ? align16(qcs_tc_walker_bytes(W)) : 0;
    size_t b_mode = (split || tc) ? 0 : align16(sizeof(int) * (size_t)(W > 0 ? W : 1));
    void *base = nullptr;
    qcs_status ws = qcs_workspace(ctx, 16 + b_ut + b_pref + b_part + 2 * b_slab + b_rec + b_mode, &base, st);
    if (ws != QCS_OK) return ws;
    char *pb = (char *)base;
    wk->counter = (unsigned long long *)pb;
    wk->Ut = (cd *)(pb + 16);
    wk->pref = (cd *)(pb + 16 + b_ut);
    wk->partial = (cd *)(pb + 16 + b_ut + b_pref);
    wk->Mhi = split ? (float *)(pb + 16 + b_ut + b_pref + b_part) : nullptr;
    wk->Mlo = split ? (float *)(pb + 16 + b_ut + b_pref + b_part + b_slab) : nullptr;
    wk->walk_rec = tc ? (unsigned char *)(pb + 16 + b_ut + b_pref + b_part + 2 * b_slab) : nullptr;
    // the reduced form of the occupied rows serves the FP64 ALU pair kernel; the tensor
    // paths keep the orthonormal echelon form
    wk->mode = (split || tc) ? nullptr : (int *)(pb + 16 + b_ut + b_pref + b_part + 2 * b_slab + b_rec);
    return qcs_launch_walker_prep(ctx, n, ne, W, (const cd *)d_walkers, wk->Ut, wk->pref, st, nullptr, nullptr,
                                  true, wk->mode);
}

}  // namespace

extern "C" qcs_status qcs_overlap(qcs_ctx *ctx, const qcs_snapshots *s, int ne, int64_t W, const double *d_walkers,
                                  double *d_overlap, double *d_per_pair, const qcs_opts *opts, void *stream) {
    QcsRange range_("qcs_overlap");
    if (!ctx) return QCS_ERR_ARG;
    if (W > 0 && !d_overlap) return qcs_fail(ctx, QCS_ERR_ARG, "null overlap output");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    qcs_node_plan plan;
    OverlapWork wk;
    qcs_status r = overlap_common(ctx, s, ne, W, d_walkers, opts, st, &plan, &wk);
    if (r != QCS_OK) return r;
    if (W == 0) return QCS_OK;
    if (d_per_pair && s->P > 0) {
        cudaError_t e = cudaMemsetAsync(d_per_pair, 0, sizeof(cd) * (size_t)W * s->P, st);
        if (e != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, "memset per-pair output");
    }
    qcs_pair_launch L;
    L.n = s->n;
    L.ne = ne;
    L.W = W;
    L.P = s->P;
    L.chunk = wk.chunk;
    L.nchunks = wk.nchunks;
    L.Ut = wk.Ut;
    L.pref = wk.pref;
    L.mode = wk.mode;
    L.s = s;
    L.partial = wk.partial;
    L.per_pair = (cd *)d_per_pair;
    L.plan = plan;
    L.counter = wk.counter;
    L.config = wk.config;
    if (wk.split) {
        r = qcs_split_prepare_snapshots(ctx, const_cast<qcs_snapshots *>(s), st);
        if (r != QCS_OK) return r;
        r = qcs_launch_split(ctx, L, wk.Mhi, wk.Mlo, st);
    } else if (wk.tc) {
        r = qcs_tc_prepare_snapshots(ctx, const_cast<qcs_snapshots *>(s), st);
        if (r != QCS_OK) return r;
        r = qcs_launch_tc_pairs(ctx, L, wk.walk_rec, st);
    } else {
        if (qcs_pair_forms_K(s->n, L.config)) {
            r = qcs_hform_prepare_snapshots(ctx, const_cast<qcs_snapshots *>(s), st);
            if (r != QCS_OK) return r;
        }
        r = qcs_launch_pairs(ctx, L, st);
    }
    if (r != QCS_OK) return r;
    return qcs_launch_reduce(ctx, W, s->P, wk.nparts, wk.partial, wk.pref, (cd *)d_overlap, st);
}

extern "C" qcs_status qcs_overlap_batched(qcs_ctx *ctx, int nsys, const qcs_system *systems, const qcs_opts *opts,
                                          void *stream) {
    QcsRange range_("qcs_overlap_batched");
    if (!ctx) return QCS_ERR_ARG;
    if (nsys < 1 || nsys > QCS_MAX_SYSTEMS || !systems)
        return qcs_fail(ctx, QCS_ERR_ARG, "nsys must be in [1, QCS_MAX_SYSTEMS]");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    qcs_opts o = {QCS_FP64, 0, 0u, 0};
    if (opts) o = *opts;
    if (o.precision != QCS_FP64) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "batched calls are FP64");
    qcs_pair_launch Ls[QCS_MAX_SYSTEMS];
    size_t off[QCS_MAX_SYSTEMS][4];
    size_t total = 16;  // the tile counter first
    const int wpb = qcs_pair_warps_per_block();
    for (int i = 0; i < nsys; ++i) {
        const qcs_system &y = systems[i];
        const qcs_snapshots *s = y.snapshots;
        if (!s) return qcs_fail(ctx, QCS_ERR_ARG, "null snapshot set in batch");
        if (s->device != ctx->device) return qcs_fail(ctx, QCS_ERR_ARG, "snapshot set lives on another device");
        qcs_status c = check_sizes(ctx, s->n, y.ne);
        if (c != QCS_OK) return c;
        if (y.W < 0 || (y.W > 0 && (!y.d_walkers || !y.d_overlap)))
            return qcs_fail(ctx, QCS_ERR_ARG, "bad walkers or output in batch");
        qcs_pair_launch &L = Ls[i];
        if (qcs_make_node_plan(s->n, y.ne, o.nodes, o.flags, &L.plan) != QCS_OK)
            return qcs_fail(ctx, QCS_ERR_ARG, "nodes must be 0 or in [n-ne+1, QCS_MAX_NODES] for every system");
        L.n = s->n;
        L.ne = y.ne;
        L.W = y.W;
        L.P = s->P;
        // the batched launch runs the FP64 ALU pair kernel: a configuration tuned for that
        // path first, then one tuned for these options
        qcs_opts oa = o;
        oa.flags |= QCS_FLAG_FP64_ALU;
        L.config = o.config > 0 ? o.config : resolve_config(ctx, s->n, y.ne, oa);
        if (L.config == 0) L.config = resolve_config(ctx, s->n, y.ne, o);
        const qcs_config cfg = qcs_decode_config(L.config);
        L.chunk = cfg.chunk > 0 ? cfg.chunk : kChunk;
        L.nchunks = (int)((s->P + L.chunk * wpb - 1) / (L.chunk * wpb));
        if (L.nchunks < 1) L.nchunks = 1;
        L.s = s;
        L.per_pair = nullptr;
        L.counter = nullptr;
        if (qcs_pair_forms_K(s->n, L.config)) {
            qcs_status hr = qcs_hform_prepare_snapshots(ctx, const_cast<qcs_snapshots *>(s), st);
            if (hr != QCS_OK) return hr;
        }
        off[i][0] = total;
        total += align16(sizeof(cd) * (size_t)y.W * s->n * s->n);
        off[i][1] = total;
        total += align16(sizeof(cd) * (size_t)y.W);
        off[i][2] = total;
        total += align16(sizeof(cd) * (size_t)y.W * L.nchunks * wpb);
        off[i][3] = total;
        total += align16(sizeof(int) * (size_t)(y.W > 0 ? y.W : 1));
    }
    void *base = nullptr;
    qcs_status r = qcs_workspace(ctx, total, &base, st);
    if (r != QCS_OK) return r;
    char *pb = (char *)base;
    for (int i = 0; i < nsys; ++i) {
        Ls[i].Ut = (cd *)(pb + off[i][0]);
        Ls[i].pref = (cd *)(pb + off[i][1]);
        Ls[i].partial = (cd *)(pb + off[i][2]);
        int *mode = (int *)(pb + off[i][3]);
        Ls[i].mode = mode;
        r = qcs_launch_walker_prep(ctx, Ls[i].n, Ls[i].ne, Ls[i].W, (const cd *)systems[i].d_walkers,
                                   (cd *)Ls[i].Ut, (cd *)Ls[i].pref, st, nullptr, nullptr, true, mode);
        if (r != QCS_OK) return r;
    }
    r = qcs_launch_pairs_batched(ctx, nsys, Ls, (unsigned long long *)pb, st);
    if (r != QCS_OK) return r;
    for (int i = 0; i < nsys; ++i) {
        r = qcs_launch_reduce(ctx, Ls[i].W, Ls[i].P, Ls[i].nchunks * wpb, Ls[i].partial, Ls[i].pref,
                              (cd *)systems[i].d_overlap, st);
        if (r != QCS_OK) return r;
    }
    return QCS_OK;
}

extern "C" qcs_status qcs_overlap_grad(qcs_ctx *ctx, const qcs_snapshots *s, int ne, int64_t W,
                                       const double *d_walkers, double *d_overlap, double *d_grad,
                                       const qcs_opts *opts, void *stream) {
    QcsRange range_("qcs_overlap_grad");
    if (!ctx) return QCS_ERR_ARG;
    if (W > 0 && (!d_overlap || !d_grad)) return qcs_fail(ctx, QCS_ERR_ARG, "null overlap or gradient output");
    if (!s) return qcs_fail(ctx, QCS_ERR_ARG, "null snapshot set");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = s->n;
    qcs_status c = check_sizes(ctx, n, ne);
    if (c != QCS_OK) return c;
    if (W < 0) return qcs_fail(ctx, QCS_ERR_ARG, "W < 0");
    if (W == 0) return QCS_OK;
    if (!d_walkers) return qcs_fail(ctx, QCS_ERR_ARG, "null walkers");
    if (s->device != ctx->device) return qcs_fail(ctx, QCS_ERR_ARG, "snapshot set lives on another device");
    qcs_opts o = {QCS_FP64, 0, 0u, 0};
    if (opts) o = *opts;
    if (o.precision != QCS_FP64) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "the gradient is FP64 only");
    qcs_node_plan plan;
    if (qcs_make_node_plan(n, ne, o.nodes, o.flags, &plan) != QCS_OK)
        return qcs_fail(ctx, QCS_ERR_ARG, "nodes must be 0 or in [n-ne+1, QCS_MAX_NODES]");
    // tiles: about 32 per resident warp, at least 8 snapshots per tile
    int64_t target = (int64_t)ctx->num_sms * 4 * 32;
    int64_t nch = (target + W - 1) / W;
    int64_t maxch = (s->P + 7) / 8;
    if (nch > maxch) nch = maxch;
    if (nch < 1) nch = 1;
    int chunk = (int)((s->P + nch - 1) / nch);
    if (chunk < 1) chunk = 1;
    int nchunks = (int)((s->P + chunk - 1) / chunk);
    if (nchunks < 1) nchunks = 1;
    size_t b_ut = align16(sizeof(cd) * (size_t)W * n * n);
    size_t b_pref = align16(sizeof(cd) * (size_t)W);
    size_t b_u = b_ut;
    size_t b_r = align16(sizeof(cd) * (size_t)W * ne * ne);
    size_t b_w = align16(sizeof(cd) * (size_t)W * ((size_t)ne * ne + 1));
    size_t b_part = align16(sizeof(cd) * (size_t)W * nchunks * (1 + (size_t)n * n));
    void *base = nullptr;
    qcs_status ws = qcs_workspace(ctx, 16 + b_ut + b_pref + b_u + b_r + b_part + b_w, &base, st);
    if (ws != QCS_OK) return ws;
    unsigned long long *gcounter = (unsigned long long *)base;
    char *pb = (char *)base + 16;
    cd *Ut = (cd *)pb;
    cd *pref = (cd *)(pb + b_ut);
    cd *U = (cd *)(pb + b_ut + b_pref);
    cd *R = (cd *)(pb + b_ut + b_pref + b_u);
    cd *part = (cd *)(pb + b_ut + b_pref + b_u + b_r);
    cd *Wrot = (cd *)(pb + b_ut + b_pref + b_u + b_r + b_part);
    // echelon-form walker rows (the congruence skips their zeros); U is the rotated unitary,
    // R the QR's triangular factor and Wrot the occupied columns' rotation for the epilogue
    qcs_status r = qcs_launch_walker_prep(ctx, n, ne, W, (const cd *)d_walkers, Ut, pref, st, U, R, true, nullptr,
                                          Wrot);
    if (r != QCS_OK) return r;
    r = qcs_hform_prepare_snapshots(ctx, const_cast<qcs_snapshots *>(s), st);
    if (r != QCS_OK) return r;
    qcs_grad_launch L;
    L.n = n;
    L.ne = ne;
    L.W = W;
    L.P = s->P;
    L.chunk = chunk;
    L.nchunks = nchunks;
    L.Ut = Ut;
    L.U = U;
    L.R = R;
    L.Wrot = Wrot;
    L.pref = pref;
    L.s = s;
    L.partial = part;
    L.overlap = (cd *)d_overlap;
    L.grad = (cd *)d_grad;
    L.plan = plan;
    L.counter = gcounter;
    return qcs_launch_grad(ctx, L, st);
}

extern "C" qcs_status qcs_force_bias(qcs_ctx *ctx, int n, int ne, int64_t W, int nchol, const double *d_L,
                                     const double *d_walkers, const double *d_overlap, const double *d_grad,
                                     double sqrt_dt, double *d_xbar, void *stream) {
    QcsRange range_("qcs_force_bias");
    if (!ctx) return QCS_ERR_ARG;
    DeviceGuard g(ctx->device);
    qcs_status c = check_sizes(ctx, n, ne);
    if (c != QCS_OK) return c;
    if (W < 0 || nchol < 0) return qcs_fail(ctx, QCS_ERR_ARG, "W and nchol must be >= 0");
    if (W == 0 || nchol == 0) return QCS_OK;
    if (!d_L || !d_walkers || !d_overlap || !d_grad || !d_xbar) return qcs_fail(ctx, QCS_ERR_ARG, "null pointer");
    return qcs_launch_force_bias(ctx, n, ne, W, nchol, (const cd *)d_L, (const cd *)d_walkers,
                                 (const cd *)d_overlap, (const cd *)d_grad, sqrt_dt, (cd *)d_xbar,
                                 (cudaStream_t)stream);
}

// ------------------------------------------------------------ accounting

static void overlap_flops_parts(int n, int ne, int nev, bool overlap_kernel, double *part);

// T over the echelon-form walker rows as the gradient kernel forms it (and K = Ut Qh^T, the
// same product with the snapshot's rows [H1^T; G2^T] in place of Qt): at n = 16 three real
// products per complex multiply-add (with re + im of each snapshot entry and the two sums
// per entry), else four.
static double grad_T_flops(int n, int ne) {
    const double macs = 2.0 * n * ((double)n * n - tri_count(ne) - tri_count(n - ne));
    return n == 16 ? 6.0 * macs + 3.0 * 2.0 * n * n + 2.0 * n * n : 8.0 * macs;
}

// B from T (build_B): occupied x occupied, occupied x empty, empty x empty.
static double grad_B_from_T_flops(int n, int ne) {
    const int d = n - ne;
    return 8.0 * 2.0 * n * tri_count(ne) + 4.0 * 2.0 * n * ne * 2 * d + 2.0 * 2.0 * n * tri_count(2 * d);
}

// B from K in the two-warp overlap kernel above 16 modes (build_B_from_K of qcs_pair.cuh):
// each sum runs over the non-zero columns of its walker row with three real products per
// term (6 flop) and three additions per sum: occupied pairs W1 alone over the reduced row's
// 1 + d columns; completion row ne + j carries ne + j + 1 items of W1 and W2 over n - j
// columns; 8 flop of halved sums and differences per occupied-empty or distinct empty pair,
// 1 per mode; re + im of K's 2n^2 entries.
static double alu_B_from_K_flops(int n, int ne) {
    const int d = n - ne;
    double rows = 0.0;
    for (int j = 0; j < d; ++j) rows += (ne + j + 1.0) * (12.0 * (n - j) + 6.0);
    return tri_count(ne) * (6.0 * (1 + d) + 3.0) + rows + 8.0 * ne * d + 8.0 * tri_count(d) + d +
           2.0 * n * n;
}

// B from K in the gradient (build_B_from_K3): two n-term complex sums per work item (tri(ne) occupied
// pairs, ne d occupied-empty pairs, tri(d + 1) empty pairs j1 <= j2) with three real
// products per term and three additions per sum, then the halved sums and differences of
// the occupied-empty (8 flop) and distinct empty pairs (8 flop) and one product per mode;
// the staged sums re - im of Ut (n^2), re + im of K (2 n^2) and re - im of K's empty rows.
static double grad_B_from_K_flops(int n, int ne) {
    const int d = n - ne;
    const double items = (double)tri_count(ne) + (double)ne * d + (double)tri_count(d + 1);
    return (12.0 * n + 6.0) * items + 8.0 * ne * d + 8.0 * tri_count(d) + d + 3.0 * n * n + 2.0 * d * n;
}

// Cotangents from K: the coefficient rows (Yh = Y[ne+2i] - i Y[ne+2i+1] and the halved
// combinations of each empty pair) and their sums re + im, then n x n entries of m
// complex multiply-adds with three real products each and five additions per entry.
static double grad_gamma_from_K_flops(int n, int ne) {
    const int d = n - ne, m = 2 * n - ne;
    return 8.0 * ne * d + d * (16.0 * d + 2.0 * ne) + (double)n * m + 6.0 * n * n * m + 5.0 * n * n;
}

// Signed-permutation snapshots: Yh (d x m), G_X on the occupied rows and Ht on the empty
// modes (n rows of 2n, ne complex and 2d real terms each), two complex additions per
// cotangent entry.
static double grad_gamma_signed_perm_flops(int n, int ne) {
    const int d = n - ne, m = 2 * n - ne;
    return 2.0 * d * m + (double)n * 2 * n * (8.0 * ne + 4.0 * (m - ne)) + 4.0 * n * n;
}

extern "C" double qcs_grad_flops_per_pair(int n, int ne, int nodes, unsigned flags) {
    qcs_node_plan plan;
    if (n < 1 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1)) return 0.0;
    if (qcs_make_node_plan(n, ne, nodes, flags, &plan) != QCS_OK) return 0.0;
    const int d = n - ne, m = 2 * n - ne;
    // forward: K over the echelon-form walker rows, B from K, the occupied block once,
    // each node's 2d x 2d complement
    double f = qcs_overlap_flops_nev(n, ne, plan.nev, false);
    f += grad_T_flops(n, ne) - 16.0 * n * n * n;                 // instead of a dense T
    f += grad_B_from_K_flops(n, ne) - grad_B_from_T_flops(n, ne);  // B from K, not from T
    f -= (double)(plan.nev - 1) * qcs_pf_elim_flops(m, 2 * d);  // the occupied steps once, not per node
    // backward step with rv later indices: g1, g2 (12 rv), Z g1 and Z g2 (16 rv^2), corner (8 rv)
    auto bstep = [](int rv) { return 16.0 * rv * rv + 20.0 * rv; };
    double node = 0.0;                                              // each node's complement inverse
    for (int rv = 2 * d - 2; rv > 0; rv -= 2) node += bstep(rv);
    f += (node + 8.0 * tri_count(2 * d)) * plan.nev;                // + the weighted sum of the Z_k
    for (int rv = 2 * d; rv <= m - 2; rv += 2) f += bstep(rv);      // backward over the shared steps
    f += grad_gamma_from_K_flops(n, ne);                            // Gamma1 / Gamma2
    return f;
}

extern "C" double qcs_overlap_flops_per_pair_signed_perm(int n, int ne, int nodes, unsigned flags) {
    qcs_node_plan plan;
    if (n < 1 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1)) return 0.0;
    if (qcs_make_node_plan(n, ne, nodes, flags, &plan) != QCS_OK) return 0.0;
    double part[3];
    overlap_flops_parts(n, ne, plan.nev, true, part);
    return grad_B_from_T_flops(n, ne) + part[2];  // T is a gather, B is formed from it
}

extern "C" double qcs_grad_flops_per_pair_signed_perm(int n, int ne, int nodes, unsigned flags) {
    const double f = qcs_grad_flops_per_pair(n, ne, nodes, flags);
    if (!(f > 0.0)) return 0.0;
    // T is a gather and B is formed from it; G_X and gathers of Qt give the cotangents
    return f - grad_T_flops(n, ne) - grad_B_from_K_flops(n, ne) + grad_B_from_T_flops(n, ne) -
           grad_gamma_from_K_flops(n, ne) + grad_gamma_signed_perm_flops(n, ne);
}

extern "C" double qcs_overlap_flops_per_pair(int n, int ne, int nodes, unsigned flags) {
    qcs_node_plan plan;
    if (n < 1 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1)) return 0.0;
    if (qcs_make_node_plan(n, ne, nodes, flags, &plan) != QCS_OK) return 0.0;
    return qcs_overlap_flops_nev(n, ne, plan.nev, true);
}

namespace {
// One elimination step of an r x r Pfaffian (r > 2): Gauss vectors and rank-2 update.
double pf_step_flops(int r) { return 16.0 * tri_count(r - 2) + 6.0 * (r - 2); }
}  // namespace

// Elimination steps of an m x m Pfaffian from r = m down to r > stop.
double qcs_pf_elim_flops(int m, int stop) {
    double f = 0.0;
    for (int r = m; r > stop && r > 2; r -= 2) f += pf_step_flops(r);
    return f;
}

// Parts of the count: [0] congruence T, [1] covariance B, [2] Pfaffian eliminations.
static void overlap_flops_parts(int n, int ne, int nev, bool overlap_kernel, double *part) {
    const int d = n - ne, m = 2 * n - ne;
    // skipped entries of Ut: the reduced form of the occupied rows ([I; X], all but one of
    // the columns k < ne zero) and the echelon form of the completion; three real products
    // per complex multiply-add (every T of the overlap kernel in its default
    // configuration; n > 16 configured to one warp per pair takes four)
    const bool three = overlap_kernel;
    const double occ_zeros = three ? (double)ne * (ne - 1) : (double)tri_count(ne);
    const double zeros = overlap_kernel ? occ_zeros + tri_count(d) : 0.0;
    const double macs = 2.0 * n * ((double)n * n - zeros);   // complex multiply-adds of T
    if (three)
        // three real products per complex multiply-add, then Re = p1 - p2 and
        // Im = p3 - p1 - p2 per entry and re + im of each snapshot entry
        part[0] = 6.0 * macs + 3.0 * 2.0 * n * n + 2.0 * n * n;
    else
        part[0] = 8.0 * macs;
    // B: from K on the two-warp path above 16 modes, from T elsewhere
    part[1] = overlap_kernel && n > 16 ? alu_B_from_K_flops(n, ne) : grad_B_from_T_flops(n, ne);
    double node = 0.0;
    if (overlap_kernel) {  // occupied block once, then each node's 2d x 2d complement
        part[2] = qcs_pf_elim_flops(m, 2 * d);
        for (int r = 2 * d; r > 2; r -= 2) node += pf_step_flops(r);
    } else {
        part[2] = 0.0;
        for (int r = m; r > 2; r -= 2) node += pf_step_flops(r);
    }
    part[2] += node * nev;
}

double qcs_overlap_flops_nev(int n, int ne, int nev, bool overlap_kernel) {
    double part[3];
    overlap_flops_parts(n, ne, nev, overlap_kernel, part);
    return part[0] + part[1] + part[2];
}

extern "C" qcs_status qcs_overlap_flops_breakdown(int n, int ne, int nodes, unsigned flags, double *parts) {
    qcs_node_plan plan;
    if (!parts || n < 1 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1)) return QCS_ERR_ARG;
    qcs_status r = qcs_make_node_plan(n, ne, nodes, flags, &plan);
    if (r != QCS_OK) return r;
    overlap_flops_parts(n, ne, plan.nev, true, parts);
    return QCS_OK;
}

extern "C" qcs_status qcs_overlap_tc_work_per_pair(int n, int ne, int nodes, unsigned flags, double *fp64,
                                                   double *tensor) {
    if (!fp64 || !tensor || n < 1 || !qcs_tc_supported(n) || ne < 2 || ne > n || (ne & 1)) return QCS_ERR_ARG;
    qcs_node_plan plan;
    qcs_status r = qcs_make_node_plan(n, ne, nodes, flags, &plan);
    if (r != QCS_OK) return r;
    double part[3];
    overlap_flops_parts(n, ne, plan.nev, true, part);
    // B^(s) from P: each occupied x occupied entry takes two real additions; the rest are
    // copies and sign changes
    *fp64 = part[2] + 2.0 * tri_count(ne);
    // two sliced products per pair, 28 slice products each of a 32 x 32 x 32 BF16
    // multiply-add (rows and contraction padded to 32)
    *tensor = 2.0 * 28.0 * 2.0 * 32.0 * 32.0 * 32.0;
    return QCS_OK;
}

extern "C" qcs_status qcs_node_plan_get(int n, int ne, int nodes, unsigned flags, int *nev, double *wnode,
                                        double *gamma) {
    if (!nev || !wnode || !gamma) return QCS_ERR_ARG;
    qcs_node_plan plan;
    qcs_status r = qcs_make_node_plan(n, ne, nodes, flags, &plan);
    if (r != QCS_OK) return r;
    *nev = plan.nev;
    for (int k = 0; k < plan.nev; ++k) {
        wnode[2 * k] = plan.wnode[k].x;
        wnode[2 * k + 1] = plan.wnode[k].y;
        gamma[2 * k] = plan.gamma[k].x;
        gamma[2 * k + 1] = plan.gamma[k].y;
    }
    return QCS_OK;
}
