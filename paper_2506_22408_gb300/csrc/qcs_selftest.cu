// qcs_selftest.cu -- self-tests of the device time-out path and of the pivot
// reciprocal, and the FP64 FMA rate.
//
// The split-precision kernel waits for its bulk copies and tensor-core MMAs on
// mbarriers, each wait bounded by an iteration limit after which the kernel raises
// QCS_ERR_TIMEOUT, drains and returns instead of hanging.  That path never runs on
// healthy hardware, so this entry point exercises the same bounded wait on an
// mbarrier whose single expected arrival nothing ever performs: the wait expires
// after max_iter polls and the block raises the status bit.  No copy or MMA is
// issued, so nothing is in flight when the block returns.
//
// qcs_fp64_fma_rate measures the sustained FP64 fused multiply-add throughput of the
// device: register-only chains x <- fma(x, a, c), eight independent chains per
// thread, eight warps per SM (the rate is the same from 8 to 32 warps per SM), timed
// with CUDA events after a warm-up that lets the clocks settle under load.  The FP64
// kernels of the library are bound by this pipe; their roofline fractions are read
// against the measured rate beside the unit-count peak.
#include "qcs_internal.h"
#include "qcs_tc.cuh"

using namespace qcs_tc;

namespace {

__global__ void bounded_wait_selftest_kernel(uint32_t max_iter, unsigned *status) {
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x == 0) mbar_init(&mbar, 1);  // one arrival expected, none will come
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&mbar, 0, max_iter)) raise_status(status, QCS_ERR_TIMEOUT);
}

// One thread per value: r[i] = recip_nonneg(d[i]), the reciprocal of the eliminations.
__global__ void reciprocal_selftest_kernel(const double *__restrict__ d, double *__restrict__ r, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = recip_nonneg(d[i]);
}

constexpr int kRateChains = 8;
constexpr int kRateThreads = 256;  // eight warps per block, one block per SM

// Every thread writes one double to out[gid] (one entry per launched thread).
__global__ void __launch_bounds__(kRateThreads) fp64_fma_rate_kernel(double *out, int iters) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    double x[kRateChains];
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) x[i] = 1.0 + 1e-9 * (double)(gid + i);
    const double a = 0.9999999, c = 1e-8;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kRateChains; ++i) x[i] = fma(x[i], a, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) s += x[i];
    out[gid] = s;
}

}  // namespace

extern "C" qcs_status qcs_selftest_bounded_wait(qcs_ctx *ctx, uint32_t max_iter, void *stream) {
    if (!ctx) return QCS_ERR_ARG;
    if (max_iter < 1 || max_iter > (1u << 20)) return qcs_fail(ctx, QCS_ERR_ARG, "max_iter must be in [1, 2^20]");
    DeviceGuard g(ctx->device);
    bounded_wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(max_iter, ctx->d_status);
    return qcs_check_launch(ctx, "bounded_wait_selftest_kernel");
}

extern "C" qcs_status qcs_selftest_reciprocal(qcs_ctx *ctx, const double *d, double *r, int64_t n, void *stream) {
    if (!ctx) return QCS_ERR_ARG;
    if (n < 0 || (n > 0 && (!d || !r))) return qcs_fail(ctx, QCS_ERR_ARG, "qcs_selftest_reciprocal: n < 0 or null array");
    if (n == 0) return QCS_OK;
    DeviceGuard g(ctx->device);
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)ctx->num_sms * 8) blocks = (int64_t)ctx->num_sms * 8;
    reciprocal_selftest_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d, r, n);
    return qcs_check_launch(ctx, "reciprocal_selftest_kernel");
}

extern "C" qcs_status qcs_fp64_fma_rate(qcs_ctx *ctx, double *tflops, void *stream) {
    if (!ctx || !tflops) return QCS_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = ctx->num_sms;
    void *buf = nullptr;
    qcs_status r = qcs_workspace(ctx, sizeof(double) * (size_t)blocks * kRateThreads, &buf, st);
    if (r != QCS_OK) return r;
    double *out = (double *)buf;
    const int iters = 1 << 16;  // about 0.1 s per launch at 1 TFLOP/s on 152 SMs
    for (int i = 0; i < 20; ++i) fp64_fma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, iters);  // warm-up
    r = qcs_check_launch(ctx, "fp64_fma_rate_kernel");
    if (r != QCS_OK) return r;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int reps = 5;
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) fp64_fma_rate_kernel<<<blocks, kRateThreads, 0, st>>>(out, iters);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, std::string("qcs_fp64_fma_rate: ") + cudaGetErrorString(e));
    const double flops = 2.0 * kRateChains * (double)iters * blocks * kRateThreads * reps;
    *tflops = ms > 0.f ? flops / ((double)ms * 1e-3) / 1e12 : 0.0;
    return QCS_OK;
}
