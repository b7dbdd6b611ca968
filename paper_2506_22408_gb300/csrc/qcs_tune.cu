// qcs_tune.cu -- autotuner of the overlap kernels' configuration.
//
// The choices (qcs_config) trade shared memory, resident warps and per-step work:
//  - the congruence path at n <= 16: on the FP64 ALU or on tensor cores;
//  - node matrices per warp round: more share the per-step pivot and reciprocal work
//    and fill more lanes, but need more shared memory per warp;
//  - the tile: snapshots per warp in an FP64 ALU tile (longer tiles amortise the walker's
//    staging, shorter ones balance the tail), sub-tiles per tensor-core tile (the walker's
//    slice record is loaded once per tile);
//  - warps per pair for n > 16 on the ALU kernel: one warp (more pairs in flight) or two
//    (half the shared memory per warp, more blocks per SM).
// The best choice depends on n, ne, the node plan and the GPU, so it is measured: a staged
// search (the path with its defaults, then node rounds, then the tile, then warps per pair,
// each stage keeping the best so far) times each configuration of qcs_overlap on a synthetic
// sample, and the fastest is recorded in the context.
#include <chrono>
#include <cmath>
#include <vector>

#include "qcs_internal.h"

namespace {

// Deterministic host fill: entries in [-1, 1).  Timing does not depend on the
// values (every pair runs the same instruction sequence), so the sample needs
// no orthogonality; parities come out mixed as for uniform bits.
void fill(std::vector<double> &v, uint64_t seed) {
    uint64_t x = seed * 6364136223846793005ull + 1442695040888963407ull;
    for (auto &e : v) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        e = (double)((x >> 11) & ((1ull << 53) - 1)) / (double)(1ull << 52) - 1.0;
    }
}

}  // namespace

extern "C" qcs_status qcs_set_config(qcs_ctx *ctx, int n, int ne, int nodes, unsigned flags, int config) {
    if (!ctx || config < 0) return QCS_ERR_ARG;
    auto key = std::make_tuple(n, ne, nodes, flags);
    if (config == 0) ctx->tuned.erase(key);
    else ctx->tuned[key] = config;
    return QCS_OK;
}

extern "C" qcs_status qcs_autotune(qcs_ctx *ctx, int n, int ne, int nodes, unsigned flags, int *config) {
    QcsRange range_("qcs_autotune");
    if (!ctx) return QCS_ERR_ARG;
    if (n < 1 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1)) return qcs_fail(ctx, QCS_ERR_ARG, "bad sizes");
    qcs_node_plan plan;
    if (qcs_make_node_plan(n, ne, nodes, flags, &plan) != QCS_OK) return qcs_fail(ctx, QCS_ERR_ARG, "bad nodes");
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != ctx->device) cudaSetDevice(ctx->device);
    const int64_t W = 4 * (int64_t)ctx->num_sms, P = 256;  // a few tiles per warp
    std::vector<double> hQ((size_t)P * 4 * n * n), hPhi((size_t)W * n * ne * 2);
    std::vector<uint8_t> hb((size_t)P * n);
    fill(hQ, 1);
    fill(hPhi, 2);
    for (size_t i = 0; i < hb.size(); ++i) hb[i] = (uint8_t)((i * 2654435761u >> 7) & 1);
    double *dQ = nullptr, *dPhi = nullptr, *dOv = nullptr;
    uint8_t *db = nullptr;
    qcs_snapshots *s = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    qcs_status rc = QCS_OK;
    int best = 1;
    float best_ms = 1e30f;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) {  // the sample comes from the context's allocator
        const bool got = qcs_dev_alloc(ctx->alloc, (void **)&dQ, sizeof(double) * hQ.size(), st) == QCS_OK &&
                         qcs_dev_alloc(ctx->alloc, (void **)&dPhi, sizeof(double) * hPhi.size(), st) == QCS_OK &&
                         qcs_dev_alloc(ctx->alloc, (void **)&dOv, sizeof(double) * 2 * W, st) == QCS_OK &&
                         qcs_dev_alloc(ctx->alloc, (void **)&db, hb.size(), st) == QCS_OK;
        if (!got) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpy(dQ, hQ.data(), sizeof(double) * hQ.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dPhi, hPhi.data(), sizeof(double) * hPhi.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db, hb.data(), hb.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        rc = qcs_fail(ctx, QCS_ERR_CUDA, std::string("autotune setup: ") + cudaGetErrorString(e));
        goto done;
    }
    rc = qcs_build_snapshots(ctx, n, P, dQ, db, &s, st);
    if (rc != QCS_OK) goto done;
    {
        // minimum over three timed calls after a warm-up; a configuration the kernels
        // cannot run (shared memory) counts as infinitely slow
        auto time_cfg = [&](int cfg, float *ms_out) -> qcs_status {
            qcs_opts o = {QCS_FP64, nodes, flags, cfg};
            *ms_out = 1e30f;
            qcs_status r = qcs_overlap(ctx, s, ne, W, dPhi, dOv, nullptr, &o, st);
            if (r == QCS_ERR_UNSUPPORTED) return QCS_OK;
            if (r != QCS_OK) return r;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                r = qcs_overlap(ctx, s, ne, W, dPhi, dOv, nullptr, &o, st);
                cudaEventRecord(e1, st);
                if (r != QCS_OK) return r;
                if (cudaEventSynchronize(e1) != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, "autotune: event");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < *ms_out) *ms_out = ms;
            }
            return QCS_OK;
        };
        auto try_cfg = [&](const qcs_config &c) -> qcs_status {
            float ms = 0.f;
            qcs_status r = time_cfg(qcs_encode_config(c), &ms);
            if (r == QCS_OK && ms < best_ms) {
                best_ms = ms;
                best = qcs_encode_config(c);
            }
            return r;
        };
        const bool path_free = !(flags & (QCS_FLAG_FP64_ALU | QCS_FLAG_FP64_TC | QCS_FLAG_ALL_NODES)) && n <= 16;
        const bool tc_forced = (flags & QCS_FLAG_FP64_TC) != 0;
        const int maxnb = plan.nev < 8 ? plan.nev : 8;
        qcs_config cand[2];
        int ncand = 0;
        // stage 1: the path with its defaults
        if (path_free) {
            cand[ncand++] = {0, 0, 0, 1, 0};
            cand[ncand++] = {0, 0, 0, 2, 0};
        } else {
            cand[ncand++] = {0, 0, 0, 0, 0};
        }
        qcs_config bc = cand[0];
        for (int i = 0; i < ncand; ++i) {
            const float before = best_ms;
            rc = try_cfg(cand[i]);
            if (rc != QCS_OK) goto done;
            if (best_ms < before) bc = cand[i];
        }
        const bool on_tc = tc_forced || bc.path == 2;
        // stage 2: node matrices per round
        for (int nb = 1; nb <= maxnb; ++nb) {
            qcs_config c = bc;
            c.nb = nb;
            const float before = best_ms;
            rc = try_cfg(c);
            if (rc != QCS_OK) goto done;
            if (best_ms < before) bc = c;
        }
        // stage 3: the tile
        if (on_tc) {
            for (int subs : {2, 4, 8, 15}) {
                qcs_config c = bc;
                c.subs = subs;
                const float before = best_ms;
                rc = try_cfg(c);
                if (rc != QCS_OK) goto done;
                if (best_ms < before) bc = c;
            }
        } else {
            for (int chunk : {2, 4, 8}) {
                qcs_config c = bc;
                c.chunk = chunk;
                const float before = best_ms;
                rc = try_cfg(c);
                if (rc != QCS_OK) goto done;
                if (best_ms < before) bc = c;
            }
            // stage 4: warps per pair (n > 16)
            if (n > 16)
                for (int warps : {1, 2}) {
                    qcs_config c = bc;
                    c.warps = warps;
                    const float before = best_ms;
                    rc = try_cfg(c);
                    if (rc != QCS_OK) goto done;
                    if (best_ms < before) bc = c;
                }
        }
        best = qcs_encode_config(bc);
        // 0 would clear the entry: name the default tile explicitly instead
        if (best == 0) best = qcs_encode_config(on_tc ? qcs_config{0, 0, 0, 0, 8} : qcs_config{0, 4, 0, 0, 0});
    }
    ctx->tuned[std::make_tuple(n, ne, nodes, flags)] = best;
    if (config) *config = best;
done:
    if (s) qcs_snapshots_free(s);
    if (st) cudaStreamSynchronize(st);
    qcs_dev_free(ctx->alloc, dQ, sizeof(double) * hQ.size());
    qcs_dev_free(ctx->alloc, dPhi, sizeof(double) * hPhi.size());
    qcs_dev_free(ctx->alloc, dOv, sizeof(double) * 2 * W);
    qcs_dev_free(ctx->alloc, db, hb.size());
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}
