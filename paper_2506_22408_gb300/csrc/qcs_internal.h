// qcs_internal.h -- host-side structures shared by the translation units of libqcs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "qcs_common.cuh"

// The device allocator of a context or snapshot set: the caller's callbacks, or (both
// null) cudaMalloc / cudaFree.
struct qcs_allocator {
    qcs_alloc_fn alloc = nullptr;
    qcs_free_fn free = nullptr;
    void *user = nullptr;
};
qcs_status qcs_dev_alloc(const qcs_allocator &a, void **p, size_t bytes, cudaStream_t st);
void qcs_dev_free(const qcs_allocator &a, void *p, size_t bytes);

struct qcs_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;     // per block
    size_t smem_per_sm = 0;    // per SM
    unsigned *d_status = nullptr;  // device status word (OR of qcs_status bits)
    unsigned *h_status = nullptr;  // pinned host mirror
    void *work = nullptr;          // device workspace
    size_t work_bytes = 0;
    qcs_allocator alloc;           // where the workspace and snapshot buffers come from
    std::string last_error;
    std::map<std::tuple<int, int, int, unsigned>, int> tuned;  // (n, ne, nodes, flags) -> config
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;  // recorded around dominant kernels
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pool;    // reusable event pairs
};

// Record the opening / closing event of a profiled launch (no-ops unless profiling).
void qcs_prof_begin(qcs_ctx *ctx, cudaStream_t st);
void qcs_prof_end(qcs_ctx *ctx, cudaStream_t st);

struct qcs_snapshots {
    int n = 0;
    int64_t P = 0;
    int device = 0;
    cd *Qt = nullptr;         // P x 2n x n complexified sign-folded rows
    int8_t *parity = nullptr; // P: +1 / -1 (0: singular or non-finite Q)
    int *idx = nullptr;       // P: indices with parity +1, ascending (first *d_count valid)
    int *d_count = nullptr;   // 2: number of parity +1 snapshots, number of signed permutations
    uint8_t *gth = nullptr;   // P x 2n gather codes of signed-permutation snapshots (row c of Qt:
                              // (k << 2) | phase, phase 0..3 = 1, i, -1, -i); first code 0xFF: dense
    void *split_hi = nullptr; // P x 4 KB TF32 operand slabs (split precision), built on first use
    void *split_lo = nullptr;
    void *tc_rec = nullptr;   // tensor-core congruence: BF16 slices of H_p = N^T J N for the parity +1
                              // list, four snapshots per record (57,856 bytes), built once
    cd *Qh = nullptr;         // P x 2n x n rows [H1^T; G2^T], H1 = Qt^T J Qt, G2 = Qt^T J conj(Qt), of
                              // each dense snapshot (FP64 ALU overlaps, gradient), built on first use
    size_t split_bytes = 0, tc_bytes = 0, qh_bytes = 0;  // sizes of the lazily built buffers (for the allocator)
    qcs_allocator alloc;      // the allocator the set's buffers came from
};

// Makes `dev` current for the scope of the guard, then restores the previous device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Helpers implemented in qcs_api.cu
qcs_status qcs_fail(qcs_ctx *ctx, qcs_status code, const std::string &msg);
qcs_status qcs_check_launch(qcs_ctx *ctx, const char *what);

// Observability.  QCS_LOG (environment, read once per process) sets what goes to
// stderr: 0 nothing (default), 1 every error message, 2 also one line per entry-point
// call (sizes, the path and configuration chosen), 3 also one line per kernel launch.
// QcsRange brackets an entry point in an NVTX range (header-only NVTX 3: inert unless
// a profiler that reads NVTX is attached) and logs the call at level 2.
int qcs_log_level();
void qcs_log(int level, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
struct QcsRange {
    explicit QcsRange(const char *name);
    ~QcsRange();
    QcsRange(const QcsRange &) = delete;
    QcsRange &operator=(const QcsRange &) = delete;
};
qcs_status qcs_set_smem(qcs_ctx *ctx, const void *func, size_t bytes);
qcs_status qcs_workspace(qcs_ctx *ctx, size_t bytes, void **out, cudaStream_t st = nullptr);

// Launchers implemented in the kernel translation units
qcs_status qcs_launch_snapshot_build(qcs_ctx *ctx, qcs_snapshots *s, const double *d_Q, const uint8_t *d_b,
                                     cudaStream_t st);

struct qcs_node_plan {
    int N;                       // roots of unity used (0: Gauss rule)
    int nev;                     // nodes evaluated
    int all;                     // 1: every node, every snapshot
    cd wnode[QCS_MAX_NODES];     // multiplier of D at each evaluated node: conj(z_k)
    cd gamma[QCS_MAX_NODES];     // weight of pf(B + conj(z_k) D) in sum_x w_x c_x
};

qcs_status qcs_make_node_plan(int n, int ne, int nodes, unsigned flags, qcs_node_plan *plan);
// algorithmic FP64 flops per parity +1 pair.  overlap_kernel: as the overlap kernels
// compute it (the congruence skips the zeros of the echelon-form walker rows; the
// occupied block is eliminated once for all nodes); otherwise a dense congruence and a
// full elimination per node, as the adjoint and local-energy kernels compute it.
double qcs_overlap_flops_nev(int n, int ne, int nev, bool overlap_kernel = false);
double qcs_pf_elim_flops(int m, int stop);  // Pfaffian elimination steps from r = m down to r > stop

qcs_status qcs_launch_walker_prep(qcs_ctx *ctx, int n, int ne, int64_t W, const cd *walkers, cd *Ut, cd *pref,
                                  cudaStream_t st, cd *Uout = nullptr, cd *Rout = nullptr, bool echelon = false,
                                  int *mode = nullptr, cd *Wout = nullptr);

struct qcs_grad_launch {
    int n, ne;
    int64_t W, P;
    int chunk, nchunks;
    const cd *Ut;
    const cd *U;      // the walker's unitary with its occupied and empty columns in echelon form
    const cd *R;      // the QR's triangular factor
    const cd *Wrot;   // per walker: det(conj W) W (ne x ne), then det(conj W); U_occ = U_qr W
    const cd *pref;
    const qcs_snapshots *s;
    cd *partial;     // W x nchunks x (1 + n*n)
    cd *overlap;     // W
    cd *grad;        // W x n x ne
    qcs_node_plan plan;
    unsigned long long *counter;  // device tile counter (reset by the launcher)
};

qcs_status qcs_launch_grad(qcs_ctx *ctx, const qcs_grad_launch &L, cudaStream_t st);

qcs_status qcs_launch_force_bias(qcs_ctx *ctx, int n, int ne, int64_t W, int nchol, const cd *L, const cd *walkers,
                                 const cd *overlap, const cd *grad, double sqrt_dt, cd *xbar, cudaStream_t st);

// A kernel configuration (qcs_opts.config, the autotuner's result), field by field; 0 in a
// field takes the built-in default.  Encoded as nb | chunk << 4 | warps << 8 | path << 10 |
// subs << 12, so that a plain k (1..8) keeps its meaning of k node matrices per round.
struct qcs_config {
    int nb;     // node matrices per warp round (pair kernels), 1..8
    int chunk;  // FP64 ALU pair kernel: snapshots per warp in a tile, 1..15 (default 4)
    int warps;  // FP64 ALU pair kernel, n > 16: 1 = one warp per pair, 2 = two (default)
    int path;   // FP64 overlaps, n <= 16: 1 = congruence on the FP64 ALU, 2 = on tensor cores
    int subs;   // tensor-core pair kernel: sub-tiles of four snapshots per tile, 1..15 (default 8)
};
inline qcs_config qcs_decode_config(int c) {
    qcs_config r;
    r.nb = c & 15;
    r.chunk = (c >> 4) & 15;
    r.warps = (c >> 8) & 3;
    r.path = (c >> 10) & 3;
    r.subs = (c >> 12) & 15;
    return r;
}
inline int qcs_encode_config(const qcs_config &r) {
    return (r.nb & 15) | ((r.chunk & 15) << 4) | ((r.warps & 3) << 8) | ((r.path & 3) << 10) | ((r.subs & 15) << 12);
}

struct qcs_pair_launch {
    int n, ne;
    int64_t W, P;
    int chunk, nchunks;
    const cd *Ut;
    const cd *pref;
    const int *mode;  // per walker: 1 = occupied rows in reduced form (walker prep), or null
    const qcs_snapshots *s;
    cd *partial;     // W x nchunks x warps-per-block
    cd *per_pair;    // W x P or null
    qcs_node_plan plan;
    int config;      // qcs_config encoding; 0 = heuristic
    unsigned long long *counter;  // device tile counter (reset by the launcher)
};

qcs_status qcs_launch_pairs(qcs_ctx *ctx, const qcs_pair_launch &L, cudaStream_t st);
int qcs_pair_warps_per_block();  // partial sums per overlap tile
// Split precision (qcs_split.cu)
qcs_status qcs_split_prepare_snapshots(qcs_ctx *ctx, qcs_snapshots *s, cudaStream_t st);
size_t qcs_split_walker_bytes(int n, int64_t W);
int qcs_split_snaps_per_tile(int n, int subs);  // snapshots per split-precision tile (subs sub-chunks; 0 = default)
qcs_status qcs_launch_split(qcs_ctx *ctx, const qcs_pair_launch &L, float *Mhi, float *Mlo, cudaStream_t st);
// FP64-accurate congruence on tensor cores (qcs_tcpair.cu)
bool qcs_tc_supported(int n);      // n <= 16
size_t qcs_tc_walker_bytes(int64_t W);
int qcs_tc_snaps_per_tile(int subs);  // parity +1 snapshots per tile (subs sub-tiles; 0 = default)
qcs_status qcs_tc_prepare_snapshots(qcs_ctx *ctx, qcs_snapshots *s, cudaStream_t st);
// Whether the FP64 ALU pair kernel runs (n, config) on its two-warp path, which forms
// K = Ut [H1 | G2] from the set's rows [H1^T; G2^T] and B from K.
bool qcs_pair_forms_K(int n, int config);
// The rows [H1^T; G2^T] of every dense snapshot into s->Qh (allocated and formed once).
qcs_status qcs_hform_prepare_snapshots(qcs_ctx *ctx, qcs_snapshots *s, cudaStream_t st);
qcs_status qcs_launch_tc_pairs(qcs_ctx *ctx, const qcs_pair_launch &L, unsigned char *walk_rec, cudaStream_t st);
qcs_status qcs_launch_pairs_batched(qcs_ctx *ctx, int nsys, const qcs_pair_launch *Ls, unsigned long long *counter,
                                    cudaStream_t st);
extern "C" double qcs_overlap_flops_per_pair(int n, int ne, int nodes, unsigned flags);
qcs_status qcs_launch_reduce(qcs_ctx *ctx, int64_t W, int64_t P, int nparts, const cd *partial, const cd *pref,
                             cd *overlap, cudaStream_t st);
