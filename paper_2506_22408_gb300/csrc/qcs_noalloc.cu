// qcs_noalloc.cu -- qcs_overlap_noalloc: the overlap path without any device allocation.
//
// Some callers cannot let a library allocate device memory at the point where they
// need overlaps: hosts whose device memory is owned by their own pool allocator and
// that forbid libraries from allocating behind their back, plug-ins that run inside
// such hosts, and real-time loops that must not stall on the implicit
// synchronisation of cudaMalloc.  For them this entry point runs the same kernels
// as qcs_build_snapshots + qcs_overlap, but every intermediate buffer (snapshot
// rows, parity list, walker rows, tile partial sums) lives in one file-scope device
// array of fixed size, and no context is needed.
//
// The device address of the array is looked up once per device, with that device
// current, by cudaGetSymbolAddress on the first call made on that device.  The
// call runs on the current device; every pointer passed must be on it.
#include <mutex>

#include "qcs_internal.h"

namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QCS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_ptr[kMaxDevices] = {};

qcs_status scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return QCS_ERR_ARG;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return QCS_ERR_CUDA;
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return QCS_OK;
}

// Bytes of the static scratch that a call with these sizes uses.
size_t noalloc_bytes(int n, int64_t P, int64_t W) {
    const int span = 4 * qcs_pair_warps_per_block();
    int64_t nchunks = (P + span - 1) / span;
    if (nchunks < 1) nchunks = 1;
    const int64_t Pa = P > 0 ? P : 1;
    size_t b = 0;
    b += align16(sizeof(cd) * (size_t)Pa * 2 * n * n);
    b += align16((size_t)Pa);
    b += align16(sizeof(int) * (size_t)Pa);
    b += 16;
    b += align16(sizeof(cd) * (size_t)W * n * n);
    b += align16(sizeof(cd) * (size_t)W);
    b += align16(sizeof(cd) * (size_t)W * nchunks * qcs_pair_warps_per_block());
    b += 16;  // tile counter
    return b;
}

}  // namespace

extern "C" qcs_status qcs_overlap_noalloc(int n, int ne, int64_t P, const double *d_Q, const uint8_t *d_b, int64_t W,
                                          const double *d_walkers, double *d_overlap, unsigned *d_status,
                                          void *stream) {
    if (n < 1 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1) || P < 0 || W < 0) return QCS_ERR_ARG;
    if ((P > 0 && (!d_Q || !d_b)) || (W > 0 && (!d_walkers || !d_overlap))) return QCS_ERR_ARG;
    if (P > (int64_t)INT32_MAX) return QCS_ERR_ARG;
    // a walker alone needs 16 n^2 bytes of scratch: larger W cannot fit, and bounding it
    // here keeps the byte count below from overflowing
    if (W > (int64_t)(QCS_NOALLOC_SCRATCH_BYTES / (16u * (unsigned)n * (unsigned)n))) return QCS_ERR_ARG;
    const size_t need = noalloc_bytes(n, P, W);
    if (need > (size_t)QCS_NOALLOC_SCRATCH_BYTES) return QCS_ERR_ARG;  // beyond the static scratch
    if (W == 0) return QCS_OK;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return QCS_ERR_CUDA;
    void *base = nullptr;
    qcs_status r = scratch_address(device, &base);
    if (r != QCS_OK) return r;
    // A context on the stack: no workspace, the caller's status word, no profiling.
    qcs_ctx ctx;
    ctx.device = device;
    int optin = 0;
    if (cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
        return QCS_ERR_CUDA;
    ctx.smem_optin = (size_t)optin;
    int per_sm_smem = 0;
    if (cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess)
        return QCS_ERR_CUDA;
    ctx.smem_per_sm = (size_t)per_sm_smem;
    ctx.d_status = d_status;
    cudaStream_t st = (cudaStream_t)stream;

    const int span = 4 * qcs_pair_warps_per_block();  // snapshots per overlap tile
    int nchunks = (int)((P + span - 1) / span);
    if (nchunks < 1) nchunks = 1;
    const int64_t Pa = P > 0 ? P : 1;
    char *p = (char *)base;
    qcs_snapshots s;
    s.n = n;
    s.P = P;
    s.device = device;
    s.Qt = (cd *)p;
    p += align16(sizeof(cd) * (size_t)Pa * 2 * n * n);
    s.parity = (int8_t *)p;
    p += align16((size_t)Pa);
    s.idx = (int *)p;
    p += align16(sizeof(int) * (size_t)Pa);
    s.d_count = (int *)p;
    p += 16;
    cd *Ut = (cd *)p;
    p += align16(sizeof(cd) * (size_t)W * n * n);
    cd *pref = (cd *)p;
    p += align16(sizeof(cd) * (size_t)W);
    cd *partial = (cd *)p;
    p += align16(sizeof(cd) * (size_t)W * nchunks * qcs_pair_warps_per_block());
    unsigned long long *counter = (unsigned long long *)p;

    r = qcs_launch_snapshot_build(&ctx, &s, d_Q, d_b, st);
    if (r != QCS_OK) return r;
    r = qcs_launch_walker_prep(&ctx, n, ne, W, (const cd *)d_walkers, Ut, pref, st, nullptr, nullptr, true);
    if (r != QCS_OK) return r;
    qcs_pair_launch L;
    L.n = n;
    L.ne = ne;
    L.W = W;
    L.P = P;
    L.chunk = 4;
    L.nchunks = nchunks;
    L.Ut = Ut;
    L.pref = pref;
    L.mode = nullptr;  // echelon form only (no scratch for the per-walker form flags)
    L.s = &s;
    L.partial = partial;
    L.per_pair = nullptr;
    L.config = 0;
    L.counter = counter;
    if (qcs_make_node_plan(n, ne, 0, 0u, &L.plan) != QCS_OK) return QCS_ERR_ARG;
    r = qcs_launch_pairs(&ctx, L, st);
    if (r != QCS_OK) return r;
    return qcs_launch_reduce(&ctx, W, P, nchunks * qcs_pair_warps_per_block(), partial, pref, (cd *)d_overlap, st);
}

