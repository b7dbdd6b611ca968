// qcs_selftest.cu -- self-test of the device time-out path.
//
// The split-precision kernel waits for its bulk copies and tensor-core MMAs on
// mbarriers, each wait bounded by an iteration limit after which the kernel raises
// QCS_ERR_TIMEOUT, drains and returns instead of hanging.  That path never runs on
// healthy hardware, so this entry point exercises the same bounded wait on an
// mbarrier whose single expected arrival nothing ever performs: the wait expires
// after max_iter polls and the block raises the status bit.  No copy or MMA is
// issued, so nothing is in flight when the block returns.
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

}  // namespace

extern "C" qcs_status qcs_selftest_bounded_wait(qcs_ctx *ctx, uint32_t max_iter, void *stream) {
    if (!ctx) return QCS_ERR_ARG;
    if (max_iter < 1 || max_iter > (1u << 20)) return qcs_fail(ctx, QCS_ERR_ARG, "max_iter must be in [1, 2^20]");
    DeviceGuard g(ctx->device);
    bounded_wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(max_iter, ctx->d_status);
    return qcs_check_launch(ctx, "bounded_wait_selftest_kernel");
}
