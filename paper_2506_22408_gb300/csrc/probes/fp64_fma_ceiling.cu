// fp64_fma_ceiling.cu -- measurement aid (not part of libqcs): the sustained FP64
// FMA throughput of the GPU, for reading the FP64 kernels' roofline fractions.
//
// Each thread runs CH independent chains x = fma(x, a, c) in registers; warps per SM
// (8, 16, 32) and chains per thread (4, 8, 16) are swept after a warm-up of about
// three seconds so that the clocks have settled under load.  Every thread writes one
// double to out[gid] (the buffer holds one entry per launched thread).
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_fma_ceiling fp64_fma_ceiling.cu
#include <cstdio>
#include <cuda_runtime.h>

template <int CH>
__global__ void dfma_chains(double *out, int iters) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    double x[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) x[i] = 1.0 + 1e-9 * (gid + i);
    const double a = 0.9999999, c = 1e-8;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = fma(x[i], a, c);
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += x[i];
    out[gid] = s;
}

template <int CH>
static void sweep(double *out, int sms, int warps_per_sm, int clk_khz) {
    const int threads = 128, blocks = sms * (warps_per_sm / 4);
    const int iters = 8192 / CH * 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    dfma_chains<CH><<<blocks, threads>>>(out, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double tf = 2.0 * CH * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    printf("warps/SM %2d  chains/thread %2d  %8.3f ms  %.3f TFLOP/s  (%.3f of 4 flop/clk/SM at %d MHz)\n",
           warps_per_sm, CH, ms, tf, tf / (sms * 4.0 * clk_khz * 1e-9), clk_khz / 1000);
}

int main() {
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);  // kHz, the maximum SM clock
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * sms * 32 * 32) != cudaSuccess) return 1;  // 32 warps per SM at most
    for (int i = 0; i < 150; ++i) dfma_chains<8><<<sms * 4, 128>>>(out, 2048 * 16);  // warm-up
    cudaDeviceSynchronize();
    for (int w : {8, 16, 32}) {
        sweep<4>(out, sms, w, clk);
        sweep<8>(out, sms, w, clk);
        sweep<16>(out, sms, w, clk);
    }
    const cudaError_t e = cudaGetLastError();
    printf("%s\n", cudaGetErrorString(e));
    cudaFree(out);
    return e == cudaSuccess ? 0 : 2;
}
