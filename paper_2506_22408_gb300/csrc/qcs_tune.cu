// qcs_tune.cu -- autotuner of the pair kernel's configuration.
//
// The pair kernel evaluates nb node matrices per warp round.  More matrices
// per round share the per-step pivot and reciprocal work and fill more lanes,
// but need more shared memory per warp, which lowers the number of resident
// warps that hide latency.  The best trade-off depends on n, ne and the node
// count, so it is measured: every nb in 1..min(nodes evaluated, 8) is timed on
// a synthetic sample and the fastest is recorded in the context.
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
    cudaError_t e = cudaMalloc(&dQ, sizeof(double) * hQ.size());
    if (e == cudaSuccess) e = cudaMalloc(&dPhi, sizeof(double) * hPhi.size());
    if (e == cudaSuccess) e = cudaMalloc(&dOv, sizeof(double) * 2 * W);
    if (e == cudaSuccess) e = cudaMalloc(&db, hb.size());
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
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
        const int maxnb = plan.nev < 8 ? plan.nev : 8;
        for (int cfg = 1; cfg <= maxnb; ++cfg) {
            qcs_opts o = {QCS_FP64, nodes, flags, cfg};
            rc = qcs_overlap(ctx, s, ne, W, dPhi, dOv, nullptr, &o, st);  // warm-up
            if (rc != QCS_OK) goto done;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, st);
                rc = qcs_overlap(ctx, s, ne, W, dPhi, dOv, nullptr, &o, st);
                cudaEventRecord(e1, st);
                if (rc != QCS_OK) goto done;
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = qcs_fail(ctx, QCS_ERR_CUDA, "autotune: event");
                    goto done;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < ms_min) ms_min = ms;
            }
            if (ms_min < best_ms) {
                best_ms = ms_min;
                best = cfg;
            }
        }
    }
    ctx->tuned[std::make_tuple(n, ne, nodes, flags)] = best;
    if (config) *config = best;
done:
    if (s) qcs_snapshots_free(s);
    if (dQ) cudaFree(dQ);
    if (dPhi) cudaFree(dPhi);
    if (dOv) cudaFree(dOv);
    if (db) cudaFree(db);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}
