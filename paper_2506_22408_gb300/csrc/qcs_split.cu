// qcs_split.cu -- split-precision overlaps: the congruence on tensor cores.
//
// The congruence of Eq. (b_mat), T = Ut Qt^T (walker rows times the snapshot's
// complexified rows), is a dense contraction.  In real form, with Ut = A + iB and
// Qt = C + iD,
//     [T_re; T_im] = M_w N_q^T,   M_w = [[A, -B], [B, A]]  (2n x 2n),
//                                 N_q = [C, D]             (2n x 2n, rows c),
// so 4 walkers x 4 snapshots are one 128 x 128 x 32 GEMM (n <= 16, rows and K padded
// to 32).  A tile is 4 walkers x subs such sub-chunks of consecutive snapshots (8 by
// default, tuned by qcs_autotune); each warp keeps its walker's sum over the tile in
// registers and writes one partial sum per tile.  It runs on the 5th-generation tensor cores as three
// tcgen05.mma kind::tf32 passes over TF32 hi/lo splits of both operands
// (hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory).  The operand
// slabs are precomputed once per walker and per snapshot in the K-major core-matrix
// layout and staged into shared memory by bulk asynchronous copies that complete
// on an mbarrier.  Each warp then reads its walker's 32 accumulator lanes, forms
// the selected covariance B^(s) in FP32, and evaluates the Pfaffians of the node
// matrices in FP64 exactly as the FP64 path does.
//
// Accuracy: T carries the ~2^-21 relative error of the split TF32 products
// accumulated in FP32, B^(s) an FP32 rounding of its 2n-term sums; the Pfaffian
// elimination, its pivoting and the node sums stay FP64.
#include "qcs_internal.h"
#include "qcs_group.cuh"
#include "qcs_tc.cuh"

using namespace qcs_tc;

namespace {

constexpr int kK = 32;           // padded contraction length (2n <= 32)
constexpr int kRows = 32;        // padded rows per walker / snapshot
constexpr int kSlabBytes = kRows * kK * 4;  // one operand slab (4 KB)
// 16 < n <= 24: rows padded to 64 (a walker's rows are the lanes of two warps) and the
// contraction to 48; a sub-chunk is 2 walkers x 2 snapshots (M = N = 128)
constexpr int kKG = 48;
constexpr int kRowsG = 64;
constexpr int kSlabBytesG = kRowsG * kKG * 4;  // 12 KB
constexpr int kWalkersPerTileG = 2;
constexpr int kSnapsPerSubG = 2;
constexpr int kWalkersPerTile = 4;          // M = 128
constexpr int kSnapsPerSub = 4;             // N = 128: snapshots per MMA sub-chunk
constexpr int kSubPerTile = 8;              // default sub-chunks per tile (32 snapshots)
constexpr uint32_t kTmemCols = 128;         // 4 blocks x 128 columns fit the SM's 512
constexpr uint32_t kWaitIter = 1u << 26;     // bounded mbarrier waits

// hi/lo TF32 split of x written to slabs at (row, k)
__device__ __forceinline__ void put_split(float *hi, float *lo, int row, int k, int K, double x) {
    const float h = to_tf32((float)x);
    const float l = to_tf32((float)(x - (double)h));
    const uint32_t o = kmajor_offset(row, k, K) / 4;
    hi[o] = h;
    lo[o] = l;
}

// Snapshot slabs N_q (rows c < 2n: [Re Qt[c][0..n), Im Qt[c][0..n)]); zero padding.
// Slabs of R rows x K (K-major core matrices), R x K floats each.
__global__ void split_snapshots_kernel(int n, int64_t P, int R, int K, const cd *__restrict__ Qt,
                                       float *__restrict__ hi, float *__restrict__ lo) {
    const int64_t slab = (int64_t)R * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P * slab;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / slab;
        const int r = (int)((e % slab) / K), k = (int)(e % K);
        double x = 0.0;
        if (r < 2 * n && k < 2 * n) {
            const cd v = Qt[q * 2 * n * n + r * n + (k % n)];
            x = k < n ? v.x : v.y;
        }
        put_split(hi + q * slab, lo + q * slab, r, k, K, x);
    }
}

// Walker slabs M_w: row j < n: [A_j, -B_j], row n + j: [B_j, A_j] with Ut = A + iB.
__global__ void split_walkers_kernel(int n, int64_t W, int R, int K, const cd *__restrict__ Ut,
                                     float *__restrict__ hi, float *__restrict__ lo) {
    const int64_t slab = (int64_t)R * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < W * slab;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = e / slab;
        const int r = (int)((e % slab) / K), k = (int)(e % K);
        double x = 0.0;
        if (r < 2 * n && k < 2 * n) {
            const int j = r % n, kk = k % n;
            const cd u = Ut[w * n * n + j * n + kk];
            if (r < n) x = k < n ? u.x : -u.y;
            else x = k < n ? u.y : u.x;
        }
        put_split(hi + w * slab, lo + w * slab, r, k, K, x);
    }
}

struct SplitArgs {
    int n, ne, m, d, nev, NB, all;
    int64_t W, P;
    int nchunks;                 // snapshot chunks of kSnapsPerSub * subs
    int subs;                    // MMA sub-chunks per tile
    int64_t ngroups;             // walker groups of kWalkersPerTile
    int region_bytes;            // operand / workspace union
    int warp_bytes;
    int off_T, off_B, off_U, off_V, off_pf, off_act, off_pv;
    int vm;                      // entries per Gauss-vector buffer (the full matrix or NB complements)
    int off_inv, off_int, off_kh, off_ph, off_scr, gz, off_pvg;  // group kernel (16 < n <= 24): step history,
                                                        // scratch, S0 offset (entries) in Ns
    const float *Mhi, *Mlo;      // walker slabs
    const float *Nhi, *Nlo;      // snapshot slabs
    const cd *pref;
    const int *idx;
    const int *d_count;
    cd *partial;                 // W x nchunks
    cd *per_pair;
    unsigned long long *counter;
    unsigned *status;
    cd wnode[QCS_MAX_NODES];
    cd gamma[QCS_MAX_NODES];
};

// B^(s) (FP64 packed upper) from T (FP32 complex, row stride ld) in FP32 arithmetic.
__device__ void build_B_f32(int n, int ne, const float2 *__restrict__ Ts, int ld, cd *__restrict__ Bs,
                            const uint16_t *__restrict__ tab, int lane, int nthr = 32) {
    const int d = n - ne;
    const int c1 = tri_count(ne);
    for (int e = lane; e < c1; e += nthr) {
        int a, b;
        pair_of(tab, e, a, b);
        const float2 *Ta = Ts + a * ld, *Tb = Ts + b * ld;
        float ax = 0.f, ay = 0.f;
        for (int k = 0; k < n; ++k) {
            const float2 p = Ta[2 * k], q = Tb[2 * k + 1], r = Ta[2 * k + 1], s = Tb[2 * k];
            ax = fmaf(p.x, q.x, ax);
            ax = fmaf(-p.y, q.y, ax);
            ay = fmaf(p.x, q.y, ay);
            ay = fmaf(p.y, q.x, ay);
            ax = fmaf(-r.x, s.x, ax);
            ax = fmaf(r.y, s.y, ax);
            ay = fmaf(-r.x, s.y, ay);
            ay = fmaf(-r.y, s.x, ay);
        }
        Bs[tri_index(a, b)] = cmk(ax, ay);
    }
    const int twod = 2 * d, c2 = ne * twod;
    for (int e = lane; e < c2; e += nthr) {
        const int a = e / twod, r = e - a * twod, j = ne + (r >> 1);
        const bool odd = r & 1;
        const float2 *Ta = Ts + a * ld, *Tj = Ts + j * ld;
        float ax = 0.f, ay = 0.f;
        for (int k = 0; k < n; ++k) {
            const float2 t0 = Tj[2 * k], t1 = Tj[2 * k + 1];
            const float x0 = odd ? t0.y : t0.x, x1 = odd ? t1.y : t1.x;
            const float2 a0 = Ta[2 * k], a1 = Ta[2 * k + 1];
            ax = fmaf(a0.x, x1, ax);
            ay = fmaf(a0.y, x1, ay);
            ax = fmaf(-a1.x, x0, ax);
            ay = fmaf(-a1.y, x0, ay);
        }
        Bs[tri_index(a, ne + r)] = odd ? cmk(-ax, -ay) : cmk(ax, ay);
    }
    const int c3 = tri_count(twod);
    for (int e = lane; e < c3; e += nthr) {
        int a, b;
        pair_of(tab, e, a, b);
        const float2 *Ta = Ts + (ne + (a >> 1)) * ld, *Tb = Ts + (ne + (b >> 1)) * ld;
        const bool oa = a & 1, ob = b & 1;
        float acc = 0.f;
        for (int k = 0; k < n; ++k) {
            const float2 a0 = Ta[2 * k], a1 = Ta[2 * k + 1], b0 = Tb[2 * k], b1 = Tb[2 * k + 1];
            acc = fmaf(oa ? a0.y : a0.x, ob ? b1.y : b1.x, acc);
            acc = fmaf(-(oa ? a1.y : a1.x), ob ? b0.y : b0.x, acc);
        }
        Bs[tri_index(ne + a, ne + b)] = cmk((oa != ob) ? -acc : acc, 0.0);
    }
}

__global__ void __launch_bounds__(128) split_pair_kernel(const __grid_constant__ SplitArgs A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar_load, mbar_mma;
    __shared__ long long next_tile;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = A.n;
    // region: operands [A_hi 16K | A_lo 16K | B_hi 16K | B_lo 16K], later the warps' workspaces
    unsigned char *region = smem_raw;
    float *Ahi = reinterpret_cast<float *>(region);
    float *Alo = Ahi + kWalkersPerTile * kSlabBytes / 4;
    float *Bhi = Alo + kWalkersPerTile * kSlabBytes / 4;
    float *Blo = Bhi + kSnapsPerSub * kSlabBytes / 4;
    // operands, workspaces and the pair table fit the launch's shared memory
    if (!QCS_IN_BOUNDS((2 * kWalkersPerTile + 2 * kSnapsPerSub) * kSlabBytes <= A.region_bytes &&
                           kWalkersPerTile * A.warp_bytes <= A.region_bytes &&
                           A.region_bytes + tri_count(A.m) * (int)sizeof(uint16_t) <= (int)dyn_smem_bytes(),
                       A.status))
        return;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw + A.region_bytes);
    build_pair_table(tab, tri_count(A.m));
    unsigned char *wbase = region + (size_t)warp * A.warp_bytes;
    float2 *Ts = reinterpret_cast<float2 *>(wbase + A.off_T);
    cd *Bs = reinterpret_cast<cd *>(wbase + A.off_B);
    cd *Ns = reinterpret_cast<cd *>(wbase);  // node matrices start the warp region (T is consumed first)
    cd *Uv = reinterpret_cast<cd *>(wbase + A.off_U);
    cd *Vv = reinterpret_cast<cd *>(wbase + A.off_V);
    cd *pf = reinterpret_cast<cd *>(wbase + A.off_pf);
    uint8_t *act0 = wbase + A.off_act;
    uint8_t *act1 = act0 + A.vm;
    cd *pv = reinterpret_cast<cd *>(wbase + A.off_pv);
    const int ldT = 2 * n + 1;

    if (warp == 0) {
        tmem_alloc(&tmem_base, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&mbar_load, 1);
        mbar_init(&mbar_mma, 1);
        abort_flag = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = tmem_base;
    const int64_t L = A.all ? A.P : (int64_t)(*A.d_count);
    const int64_t ntiles = A.ngroups * A.nchunks;
    uint32_t phase = 0;
    bool load_pending = false, mma_pending = false;
    for (;;) {
        fence_proxy_async_smem();  // this thread's workspace writes precede the next bulk copies
        __syncthreads();           // previous tile fully consumed (workspaces overlay the operands)
        if (tid == 0) next_tile = abort_flag ? (long long)ntiles : (long long)atomicAdd(A.counter, 1ull);
        __syncthreads();
        const int64_t t = next_tile;
        if (t >= ntiles) break;
        const int ch = (int)(t / A.ngroups);  // chunk-major: a snapshot chunk stays in L2 over the walkers
        const int64_t g = t - (int64_t)ch * A.ngroups;
        const int64_t p0 = (int64_t)ch * kSnapsPerSub * A.subs;
        const int64_t w = g * kWalkersPerTile + warp;
        if (!QCS_IN_BOUNDS(ch < A.nchunks && L >= 0 && L <= A.P, A.status)) continue;  // block-uniform
        cd acc = cmk(0.0, 0.0);
        bool ok = true;
        for (int sc = 0; sc < A.subs; ++sc) {
            const int64_t pb = p0 + (int64_t)sc * kSnapsPerSub;
            if (pb >= L) break;  // no parity +1 snapshot left in this chunk
            if (sc > 0) {
                fence_proxy_async_smem();  // the workspaces of the last sub-chunk overlay the operands
                __syncthreads();
            }
            const int nq = (int)((L - pb) < kSnapsPerSub ? (L - pb) : kSnapsPerSub);
            // stage the operand slabs (bulk asynchronous copies on mbar_load); the
            // walkers' slabs come again from L2 for every sub-chunk
            if (tid == 0) {
                uint32_t bytes = 0;
                for (int s = 0; s < kWalkersPerTile; ++s) bytes += (g * kWalkersPerTile + s < A.W) ? 2 * kSlabBytes : 0;
                for (int q = 0; q < nq; ++q) {
                    const int64_t sq = A.all ? pb + q : (int64_t)A.idx[pb + q];
                    const bool okq = sq >= 0 && sq < A.P;  // a bad index is skipped, in both loops
                    (void)QCS_IN_BOUNDS(okq, A.status);
                    bytes += okq ? 2 * kSlabBytes : 0;
                }
                mbar_expect_tx(&mbar_load, bytes);
                for (int s = 0; s < kWalkersPerTile; ++s) {
                    const int64_t ws = g * kWalkersPerTile + s;
                    if (ws >= A.W) continue;
                    bulk_copy(Ahi + s * kSlabBytes / 4, A.Mhi + ws * (kSlabBytes / 4), kSlabBytes, &mbar_load);
                    bulk_copy(Alo + s * kSlabBytes / 4, A.Mlo + ws * (kSlabBytes / 4), kSlabBytes, &mbar_load);
                }
                for (int q = 0; q < nq; ++q) {
                    const int64_t sq = A.all ? pb + q : (int64_t)A.idx[pb + q];
                    if (!(sq >= 0 && sq < A.P)) continue;
                    bulk_copy(Bhi + q * kSlabBytes / 4, A.Nhi + sq * (kSlabBytes / 4), kSlabBytes, &mbar_load);
                    bulk_copy(Blo + q * kSlabBytes / 4, A.Nlo + sq * (kSlabBytes / 4), kSlabBytes, &mbar_load);
                }
            }
            load_pending = true;
            ok = __syncthreads_and(mbar_wait_bounded(&mbar_load, phase, kWaitIter));
            if (!ok) break;
            load_pending = false;
            if (tid == 0) {
                fence_after_sync();
                const uint32_t id = idesc_tf32(kWalkersPerTile * kRows, kSnapsPerSub * kRows);
                const float *Ap[3] = {Ahi, Ahi, Alo};
                const float *Bp[3] = {Bhi, Blo, Bhi};
                for (int pass = 0; pass < 3; ++pass)
                    for (int s = 0; s < kK / 8; ++s) {
                        const uint64_t ad = desc_kmajor(Ap[pass] + 64 * s, 128, 32 * kK);
                        const uint64_t bd = desc_kmajor(Bp[pass] + 64 * s, 128, 32 * kK);
                        mma_tf32(tbase, ad, bd, id, (pass > 0 || s > 0) ? 1u : 0u);
                    }
                mma_commit(&mbar_mma);
            }
            mma_pending = true;
            ok = __syncthreads_and(mbar_wait_bounded(&mbar_mma, phase, kWaitIter));
            if (!ok) break;
            mma_pending = false;
            phase ^= 1u;
            fence_after_sync();  // all MMAs complete: the operand region becomes the warps' workspaces
            for (int q = 0; q < nq; ++q) {
                // T rows of this warp's walker for snapshot q: lane r holds row r of [T_re; T_im]
                float v0[16], v1[16];
                const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * q);
                tmem_ld16(ta, v0);
                tmem_ld16(ta + 16, v1);
                tmem_ld_wait();
                __syncwarp();
                if (lane < 2 * n) {
                    const int j = lane % n;
                    const bool im = lane >= n;
                    for (int c = 0; c < 2 * n; ++c) {
                        const float x = c < 16 ? v0[c] : v1[c - 16];
                        if (im) Ts[j * ldT + c].y = x;
                        else Ts[j * ldT + c].x = x;
                    }
                }
                __syncwarp();
                if (w >= A.W) continue;
                build_B_f32(n, A.ne, Ts, ldT, Bs, tab, lane);
                __syncwarp();
                // occupied block eliminated once for all nodes when that is stable
                cd *pvo = pv + pv_records(A.vm, A.NB, A.ne);  // the occupied pivots
                const bool shared = schur_occupied(A.m, A.ne, Bs, Ns, Uv, Vv, act0, act1, tab, pvo, lane);
                const int mm = shared ? A.m - A.ne : A.m, nee = shared ? 0 : A.ne;
                const int NBr = shared ? A.NB : 1;  // the rare full eliminations run one node per round
                cd S = cmk(0.0, 0.0);
                for (int k0 = 0; k0 < A.nev; k0 += NBr) {
                    const int nb = A.nev - k0 < NBr ? A.nev - k0 : NBr;
                    node_pfaffians(mm, nee, A.wnode + k0, A.gamma + k0, nb, Bs, Ns, Uv, Vv, pf, act0, act1, tab, pv,
                                   shared ? A.ne / 2 : 0, pvo, lane);
                    if (lane == 0)
                        for (int vv = 0; vv < nb; ++vv) S = cadd(S, pf[vv]);  // pf[vv] carries gamma
                    __syncwarp();
                }
                if (lane == 0) {
                    if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                    acc = cadd(acc, S);
                    if (A.per_pair) {
                        const int64_t sq = A.all ? pb + q : (int64_t)A.idx[pb + q];
                        A.per_pair[w * A.P + sq] = cmul(A.pref[w], S);
                    }
                }
            }
            fence_before_sync();  // this warp's tensor-memory reads precede the next sub-chunk's MMAs
        }
        if (!ok) {
            if (tid == 0) {
                abort_flag = 1;
                raise_status(A.status, QCS_ERR_TIMEOUT);
            }
            continue;  // every thread leaves through the abort check at the top
        }
        if (lane == 0 && w < A.W) A.partial[w * A.nchunks + ch] = acc;
    }
    if (abort_flag && tid == 0) {  // a wait gave up: let a copy or MMAs in flight land first
        if (load_pending) mbar_wait_bounded(&mbar_load, phase, kWaitIter);
        if (mma_pending) mbar_wait_bounded(&mbar_mma, phase, kWaitIter);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tbase, kTmemCols);
}

// 16 < n <= 24: a sub-chunk of 2 walkers x 2 snapshots is one 128 x 128 x 48 GEMM per
// TF32 pass; walker i of the tile is the tensor-memory lanes of warps 2i and 2i+1, which
// form a 64-thread group (named barrier 1 + i) that reads the walker's T blocks, forms
// B^(s) in FP32 and evaluates the Pfaffians in FP64 with the group form of the
// eliminations (qcs_group.cuh), one pair at a time.  Partial sums as in
// split_pair_kernel: per walker and tile, kept in registers over the sub-chunks.
__global__ void __launch_bounds__(128, 2) split_group_kernel(const __grid_constant__ SplitArgs A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar_load, mbar_mma;
    __shared__ long long next_tile;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = warp >> 1, t = tid & (kGroup - 1), bar = 1 + gi;
    const int n = A.n, m = A.m, ne = A.ne, d2 = m - ne, Tn = tri_count(d2);
    unsigned char *region = smem_raw;
    float *Ahi = reinterpret_cast<float *>(region);
    float *Alo = Ahi + kWalkersPerTileG * kSlabBytesG / 4;
    float *Bhi = Alo + kWalkersPerTileG * kSlabBytesG / 4;
    float *Blo = Bhi + kSnapsPerSubG * kSlabBytesG / 4;
    // operands, the two groups' workspaces and the pair table fit the launch's shared memory
    if (!QCS_IN_BOUNDS(blockDim.x == 2 * kGroup &&
                           (2 * kWalkersPerTileG + 2 * kSnapsPerSubG) * kSlabBytesG <= A.region_bytes &&
                           2 * A.warp_bytes <= A.region_bytes &&
                           A.region_bytes + tri_count(m) * (int)sizeof(uint16_t) <= (int)dyn_smem_bytes(),
                       A.status))
        return;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw + A.region_bytes);
    build_pair_table(tab, tri_count(m));
    unsigned char *gb = region + (size_t)gi * A.warp_bytes;  // this group's workspace
    float2 *Ts = reinterpret_cast<float2 *>(gb + A.off_T);
    cd *Ns = reinterpret_cast<cd *>(gb);  // node matrices, once T is consumed into B
    cd *Sc = Ns + A.gz;                   // S0 of the shared elimination
    cd *Bs = reinterpret_cast<cd *>(gb + A.off_B);
    cd *Uv = reinterpret_cast<cd *>(gb + A.off_U);
    cd *Vv = reinterpret_cast<cd *>(gb + A.off_V);
    cd *pf = reinterpret_cast<cd *>(gb + A.off_pf);
    cd *invh = reinterpret_cast<cd *>(gb + A.off_inv);
    uint8_t *acth = gb + A.off_act;
    uint8_t *kh = gb + A.off_kh;
    uint8_t *ph = gb + A.off_ph;
    SharedScratch *scr = reinterpret_cast<SharedScratch *>(gb + A.off_scr);
    cd *pvg = reinterpret_cast<cd *>(gb + A.off_pvg);
    const int ldT = 2 * n + 1;

    if (warp == 0) {
        tmem_alloc(&tmem_base, kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&mbar_load, 1);
        mbar_init(&mbar_mma, 1);
        abort_flag = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = tmem_base;
    const int64_t L = A.all ? A.P : (int64_t)(*A.d_count);
    const int64_t ntiles = A.ngroups * A.nchunks;
    uint32_t phase = 0;
    bool load_pending = false, mma_pending = false;
    for (;;) {
        fence_proxy_async_smem();
        __syncthreads();  // previous tile fully consumed (workspaces overlay the operands)
        if (tid == 0) next_tile = abort_flag ? (long long)ntiles : (long long)atomicAdd(A.counter, 1ull);
        __syncthreads();
        const int64_t tile = next_tile;
        if (tile >= ntiles) break;
        const int ch = (int)(tile / A.ngroups);
        const int64_t g = tile - (int64_t)ch * A.ngroups;
        const int64_t p0 = (int64_t)ch * kSnapsPerSubG * A.subs;
        const int64_t w = g * kWalkersPerTileG + gi;
        if (!QCS_IN_BOUNDS(ch < A.nchunks && L >= 0 && L <= A.P, A.status)) continue;  // block-uniform
        cd acc = cmk(0.0, 0.0);
        bool ok = true;
        for (int sc = 0; sc < A.subs; ++sc) {
            const int64_t pb = p0 + (int64_t)sc * kSnapsPerSubG;
            if (pb >= L) break;
            if (sc > 0) {
                fence_proxy_async_smem();
                __syncthreads();
            }
            const int nq = (int)((L - pb) < kSnapsPerSubG ? (L - pb) : kSnapsPerSubG);
            if (tid == 0) {
                uint32_t bytes = 0;
                for (int s = 0; s < kWalkersPerTileG; ++s)
                    bytes += (g * kWalkersPerTileG + s < A.W) ? 2 * kSlabBytesG : 0;
                for (int q = 0; q < nq; ++q) {
                    const int64_t sq = A.all ? pb + q : (int64_t)A.idx[pb + q];
                    const bool okq = sq >= 0 && sq < A.P;  // a bad index is skipped, in both loops
                    (void)QCS_IN_BOUNDS(okq, A.status);
                    bytes += okq ? 2 * kSlabBytesG : 0;
                }
                mbar_expect_tx(&mbar_load, bytes);
                for (int s = 0; s < kWalkersPerTileG; ++s) {
                    const int64_t ws = g * kWalkersPerTileG + s;
                    if (ws >= A.W) continue;
                    bulk_copy(Ahi + s * kSlabBytesG / 4, A.Mhi + ws * (kSlabBytesG / 4), kSlabBytesG, &mbar_load);
                    bulk_copy(Alo + s * kSlabBytesG / 4, A.Mlo + ws * (kSlabBytesG / 4), kSlabBytesG, &mbar_load);
                }
                for (int q = 0; q < nq; ++q) {
                    const int64_t sq = A.all ? pb + q : (int64_t)A.idx[pb + q];
                    if (!(sq >= 0 && sq < A.P)) continue;
                    bulk_copy(Bhi + q * kSlabBytesG / 4, A.Nhi + sq * (kSlabBytesG / 4), kSlabBytesG, &mbar_load);
                    bulk_copy(Blo + q * kSlabBytesG / 4, A.Nlo + sq * (kSlabBytesG / 4), kSlabBytesG, &mbar_load);
                }
            }
            load_pending = true;
            ok = __syncthreads_and(mbar_wait_bounded(&mbar_load, phase, kWaitIter));
            if (!ok) break;
            load_pending = false;
            if (tid == 0) {
                fence_after_sync();
                const uint32_t id = idesc_tf32(kWalkersPerTileG * kRowsG, kSnapsPerSubG * kRowsG);
                const float *Ap[3] = {Ahi, Ahi, Alo};
                const float *Bp[3] = {Bhi, Blo, Bhi};
                for (int pass = 0; pass < 3; ++pass)
                    for (int s = 0; s < kKG / 8; ++s) {  // K = 8 per instruction: 2 core matrices, 256 bytes
                        const uint64_t ad = desc_kmajor(Ap[pass] + 64 * s, 128, 32 * kKG);
                        const uint64_t bd = desc_kmajor(Bp[pass] + 64 * s, 128, 32 * kKG);
                        mma_tf32(tbase, ad, bd, id, (pass > 0 || s > 0) ? 1u : 0u);
                    }
                mma_commit(&mbar_mma);
            }
            mma_pending = true;
            ok = __syncthreads_and(mbar_wait_bounded(&mbar_mma, phase, kWaitIter));
            if (!ok) break;
            mma_pending = false;
            phase ^= 1u;
            fence_after_sync();  // all MMAs complete: the operand region becomes the groups' workspaces
            for (int q = 0; q < nq; ++q) {
                // rows r = 32 (warp & 1) + lane of [T_re; T_im] for this group's walker and
                // snapshot q: columns 64 q .. 64 q + 2n - 1
                float v0[16], v1[16], v2[16];
                const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(kRowsG * q);
                tmem_ld16(ta, v0);
                tmem_ld16(ta + 16, v1);
                tmem_ld16(ta + 32, v2);
                tmem_ld_wait();
                const int r = 32 * (warp & 1) + lane;
                if (r < 2 * n) {
                    const int j = r % n;
                    const bool im = r >= n;
#pragma unroll
                    for (int c = 0; c < kKG; ++c) {
                        if (c >= 2 * n) break;
                        const float x = c < 16 ? v0[c] : (c < 32 ? v1[c - 16] : v2[c - 32]);
                        if (im) Ts[j * ldT + c].y = x;
                        else Ts[j * ldT + c].x = x;
                    }
                }
                group_sync(bar);
                if (w < A.W) {  // group-uniform
                    build_B_f32(n, ne, Ts, ldT, Bs, tab, t, kGroup);
                    group_sync(bar);
                    cd S = cmk(0.0, 0.0);
                    if (shared_factor(m, ne, Bs, Ns, Uv, Vv, invh, acth, kh, ph, scr, tab, t, bar)) {
                        const cd pf0 = scr->pf0;
                        for (int e = t; e < Tn; e += kGroup) {
                            int a, b;
                            pair_of(tab, e, a, b);
                            Sc[e] = Ns[tri_index(ne + a, ne + b)];
                        }
                        group_sync(bar);
                        for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                            const int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                            group_node_pfaffians(d2, 0, A.wnode + k0, A.gamma + k0, nb, Sc, Ns, Uv, Vv, pf, acth,
                                                 acth + A.vm, pvg, tab, t, bar);
                            if (t == 0)
                                for (int v = 0; v < nb; ++v) S = cadd(S, pf[v]);  // pf[v] carries gamma
                            group_sync(bar);
                        }
                        S = cmul(S, pf0);
                    } else {  // the rare full eliminations: one node matrix per round
                        for (int k0 = 0; k0 < A.nev; ++k0) {
                            group_node_pfaffians(m, ne, A.wnode + k0, A.gamma + k0, 1, Bs, Ns, Uv, Vv, pf, acth,
                                                 acth + A.vm, pvg, tab, t, bar);
                            if (t == 0) S = cadd(S, pf[0]);
                            group_sync(bar);
                        }
                    }
                    if (t == 0) {
                        if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                        acc = cadd(acc, S);
                        if (A.per_pair) {
                            const int64_t sq = A.all ? pb + q : (int64_t)A.idx[pb + q];
                            A.per_pair[w * A.P + sq] = cmul(A.pref[w], S);
                        }
                    }
                }
                group_sync(bar);  // Ts and the workspace are free for the next snapshot
            }
            fence_before_sync();  // tensor-memory reads precede the next sub-chunk's MMAs
        }
        if (!ok) {
            if (tid == 0) {
                abort_flag = 1;
                raise_status(A.status, QCS_ERR_TIMEOUT);
            }
            continue;
        }
        if (t == 0 && w < A.W) A.partial[w * A.nchunks + ch] = acc;
    }
    if (abort_flag && tid == 0) {
        if (load_pending) mbar_wait_bounded(&mbar_load, phase, kWaitIter);
        if (mma_pending) mbar_wait_bounded(&mbar_mma, phase, kWaitIter);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tbase, kTmemCols);
}

// Workspace of one 64-thread group of split_group_kernel: T (FP32) aliased by the node
// matrices (a full copy of B for the shared elimination, NB complements, S0 after
// them), then B, the Gauss vectors and the step history of qcs_group.cuh.
size_t split_group_layout(SplitArgs &A, int NB) {
    const int n = A.n, m = A.m, ne = A.ne, T = tri_count(m), d2 = m - ne, Tn = tri_count(d2), S = m / 2;
    const size_t tbytes = (size_t)n * (2 * n + 1) * sizeof(float2);
    A.gz = T > NB * Tn ? T : NB * Tn;
    size_t R = (size_t)(A.gz + Tn) * sizeof(cd);
    if (tbytes > R) R = tbytes;
    A.vm = m > NB * d2 ? m : NB * d2;
    A.off_T = 0;
    size_t o = align16(R);
    A.off_B = (int)o;
    o = align16(o + (size_t)T * sizeof(cd));
    A.off_U = (int)o;
    o = align16(o + (size_t)A.vm * sizeof(cd));
    A.off_V = (int)o;
    o = align16(o + (size_t)A.vm * sizeof(cd));
    A.off_pf = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    const int hs = S > NB * (d2 / 2) ? S : NB * (d2 / 2);  // history steps
    A.off_inv = (int)o;
    o = align16(o + (size_t)hs * sizeof(cd));
    A.off_int = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(int));
    size_t ha = (size_t)(S + 1) * m;  // active lists: full matrix, one node
    if ((size_t)NB * (d2 / 2 + 1) * d2 > ha) ha = (size_t)NB * (d2 / 2 + 1) * d2;
    A.off_act = (int)o;
    o = align16(o + ha);
    A.off_kh = (int)o;
    o = align16(o + (size_t)hs);
    A.off_ph = (int)o;
    o = align16(o + (size_t)hs);
    A.off_scr = (int)o;
    o = align16(o + sizeof(SharedScratch));
    A.off_pvg = (int)o;  // records of the node products: NB (d2/2 + 1) or, for a full round, m/2 + 1
    o = align16(o + (size_t)(NB * (d2 / 2 + 1) > S + 1 ? NB * (d2 / 2 + 1) : S + 1) * sizeof(cd));
    return o;
}

// Per-warp workspace of the split kernel for nb node matrices.
size_t split_warp_layout(SplitArgs &A, int NB) {
    const int n = A.n, m = A.m, T = tri_count(m), d2 = m - A.ne;
    // node matrices: one full copy of B (shared elimination; the rare full eliminations,
    // one node per round) or NB complements of 2d x 2d
    size_t nodes = (size_t)(T > NB * tri_count(d2) ? T : NB * tri_count(d2)) * sizeof(cd);
    A.vm = m > NB * d2 ? m : NB * d2;
    size_t tbytes = (size_t)n * (2 * n + 1) * sizeof(float2);
    // T is consumed (into B) before the node matrices are written: they may share
    size_t o = align16(nodes > tbytes ? nodes : tbytes);
    A.off_T = 0;
    A.off_B = (int)o;
    o = align16(o + (size_t)T * sizeof(cd));
    A.off_U = (int)o;
    o = align16(o + (size_t)A.vm * sizeof(cd));
    A.off_V = (int)o;
    o = align16(o + (size_t)A.vm * sizeof(cd));
    A.off_pf = (int)o;
    o = align16(o + (size_t)kMaxNB * sizeof(cd));
    A.off_act = (int)o;
    o = align16(o + (size_t)2 * A.vm);
    A.off_pv = (int)o;  // node products (gamma and the occupied pivots included), then those pivots
    o = align16(o + (size_t)(pv_records(A.vm, NB, A.ne) + A.ne / 2) * sizeof(cd));
    return o;
}

}  // namespace

namespace {
// operand slab geometry for n modes: rows x contraction, bytes
struct SlabGeom {
    int R, K;
    size_t bytes;
};
SlabGeom slab_geom(int n) {
    return n <= 16 ? SlabGeom{kRows, kK, (size_t)kSlabBytes} : SlabGeom{kRowsG, kKG, (size_t)kSlabBytesG};
}
}  // namespace

qcs_status qcs_split_prepare_snapshots(qcs_ctx *ctx, qcs_snapshots *s, cudaStream_t st) {
    if (s->split_hi) return QCS_OK;
    if (s->n > QCS_MAX_N) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "split precision supports n <= 24");
    const SlabGeom sg = slab_geom(s->n);
    const size_t bytes = (size_t)(s->P > 0 ? s->P : 1) * sg.bytes;
    qcs_status e = qcs_dev_alloc(s->alloc, &s->split_hi, bytes, st);
    if (e == QCS_OK) e = qcs_dev_alloc(s->alloc, &s->split_lo, bytes, st);
    s->split_bytes = bytes;
    if (e != QCS_OK) return qcs_fail(ctx, QCS_ERR_CUDA, "split snapshot slabs: device allocation failed");
    if (s->P > 0) {
        int64_t tot = s->P * sg.R * sg.K;
        int64_t blocks = (tot + 255) / 256;
        if (blocks > (int64_t)ctx->num_sms * 32) blocks = (int64_t)ctx->num_sms * 32;
        split_snapshots_kernel<<<(unsigned)blocks, 256, 0, st>>>(s->n, s->P, sg.R, sg.K, s->Qt,
                                                                 (float *)s->split_hi, (float *)s->split_lo);
    }
    return qcs_check_launch(ctx, "split_snapshots_kernel");
}

size_t qcs_split_walker_bytes(int n, int64_t W) { return (size_t)(W > 0 ? W : 1) * slab_geom(n).bytes; }

int qcs_split_snaps_per_tile(int n, int subs) {
    return (n <= 16 ? kSnapsPerSub : kSnapsPerSubG) * (subs > 0 ? subs : kSubPerTile);
}

namespace {
// 16 < n <= 24: split_group_kernel, two 64-thread groups per block.
qcs_status qcs_launch_split_group(qcs_ctx *ctx, const qcs_pair_launch &L, const float *Mhi, const float *Mlo,
                                  cudaStream_t st) {
    SplitArgs A;
    memset(&A, 0, sizeof(A));
    A.n = L.n;
    A.ne = L.ne;
    A.m = 2 * L.n - L.ne;
    A.d = L.n - L.ne;
    A.nev = L.plan.nev;
    A.all = L.plan.all;
    A.W = L.W;
    A.P = L.P;
    A.nchunks = L.nchunks;
    {
        const int cs = qcs_decode_config(L.config).subs;
        A.subs = cs > 0 ? cs : kSubPerTile;
    }
    A.ngroups = (L.W + kWalkersPerTileG - 1) / kWalkersPerTileG;
    const size_t operands = (size_t)(2 * kWalkersPerTileG + 2 * kSnapsPerSubG) * kSlabBytesG;
    const size_t tab = align16((size_t)tri_count(A.m) * sizeof(uint16_t));
    // largest balanced node round (<= kMaxNBG) whose two group workspaces fit in the
    // operand region, else one node per round with the workspaces beside it
    int NB = 1;
    for (int rounds = 1; rounds <= A.nev; ++rounds) {
        const int nb = (A.nev + rounds - 1) / rounds;
        if (nb > kMaxNBG) continue;
        if (2 * split_group_layout(A, nb) <= operands) {
            NB = nb;
            break;
        }
    }
    const int cnb = qcs_decode_config(L.config).nb;
    if (cnb > 0) NB = cnb < A.nev ? (cnb < kMaxNBG ? cnb : kMaxNBG) : A.nev;
    A.NB = NB;
    A.warp_bytes = (int)split_group_layout(A, NB);  // bytes per group
    size_t region = 2 * (size_t)A.warp_bytes;
    if (region < operands) region = operands;
    A.region_bytes = (int)align16(region);
    A.Mhi = Mhi;
    A.Mlo = Mlo;
    A.Nhi = (const float *)L.s->split_hi;
    A.Nlo = (const float *)L.s->split_lo;
    A.pref = L.pref;
    A.idx = L.s->idx;
    A.d_count = L.s->d_count;
    A.partial = L.partial;
    A.per_pair = L.per_pair;
    A.counter = L.counter;
    A.status = ctx->d_status;
    for (int k = 0; k < L.plan.nev; ++k) {
        A.wnode[k] = L.plan.wnode[k];
        A.gamma[k] = L.plan.gamma[k];
    }
    const size_t smem = (size_t)A.region_bytes + tab;
    if (smem + 1024 > ctx->smem_optin) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "split kernel: shared memory");
    if (qcs_set_smem(ctx, (const void *)split_group_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int per_sm = (int)(ctx->smem_per_sm / (smem + 1024 + 1024));
    if (per_sm > (int)(512 / kTmemCols)) per_sm = (int)(512 / kTmemCols);
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = A.ngroups * A.nchunks;
    int64_t blocks = (int64_t)ctx->num_sms * per_sm;
    if (blocks > ntiles) blocks = ntiles;
    if (blocks < 1) blocks = 1;
    if (cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return qcs_fail(ctx, QCS_ERR_CUDA, "split tile counter reset");
    qcs_prof_begin(ctx, st);
    split_group_kernel<<<(unsigned)blocks, 2 * kGroup, smem, st>>>(A);
    qcs_prof_end(ctx, st);
    return qcs_check_launch(ctx, "split_group_kernel");
}
}  // namespace

qcs_status qcs_launch_split(qcs_ctx *ctx, const qcs_pair_launch &L, float *Mhi, float *Mlo, cudaStream_t st) {
    const int n = L.n;
    if (n > QCS_MAX_N) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "split precision supports n <= 24");
    const SlabGeom sg = slab_geom(n);
    {
        int64_t tot = L.W * sg.R * sg.K;
        int64_t blocks = (tot + 255) / 256;
        if (blocks > (int64_t)ctx->num_sms * 32) blocks = (int64_t)ctx->num_sms * 32;
        if (blocks > 0) split_walkers_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, L.W, sg.R, sg.K, L.Ut, Mhi, Mlo);
        qcs_status r = qcs_check_launch(ctx, "split_walkers_kernel");
        if (r != QCS_OK) return r;
    }
    if (n > 16) return qcs_launch_split_group(ctx, L, Mhi, Mlo, st);
    SplitArgs A;
    memset(&A, 0, sizeof(A));
    A.n = n;
    A.ne = L.ne;
    A.m = 2 * n - L.ne;
    A.d = n - L.ne;
    A.nev = L.plan.nev;
    A.all = L.plan.all;
    A.W = L.W;
    A.P = L.P;
    A.nchunks = L.nchunks;
    {
        const int cs = qcs_decode_config(L.config).subs;
        A.subs = cs > 0 ? cs : kSubPerTile;
    }
    A.ngroups = (L.W + kWalkersPerTile - 1) / kWalkersPerTile;
    const int T = tri_count(A.m);
    const size_t operands = (size_t)(2 * kWalkersPerTile + 2 * kSnapsPerSub) * kSlabBytes;
    const size_t tab = align16((size_t)T * sizeof(uint16_t));
    // largest node round (<= kMaxNB, balanced) whose four workspaces fit in the operand
    // region
    int NB = 1;
    for (int rounds = 1; rounds <= A.nev; ++rounds) {
        int nb = (A.nev + rounds - 1) / rounds;
        if (nb > kMaxNB) continue;
        if ((size_t)kWalkersPerTile * split_warp_layout(A, nb) <= operands) {
            NB = nb;
            break;
        }
    }
    const int cnb = qcs_decode_config(L.config).nb;
    if (cnb > 0) NB = cnb < A.nev ? (cnb < kMaxNB ? cnb : kMaxNB) : A.nev;
    A.NB = NB;
    A.warp_bytes = (int)split_warp_layout(A, NB);
    size_t region = (size_t)kWalkersPerTile * A.warp_bytes;
    if (region < operands) region = operands;
    A.region_bytes = (int)align16(region);
    A.Mhi = Mhi;
    A.Mlo = Mlo;
    A.Nhi = (const float *)L.s->split_hi;
    A.Nlo = (const float *)L.s->split_lo;
    A.pref = L.pref;
    A.idx = L.s->idx;
    A.d_count = L.s->d_count;
    A.partial = L.partial;
    A.per_pair = L.per_pair;
    A.counter = L.counter;
    A.status = ctx->d_status;
    for (int k = 0; k < L.plan.nev; ++k) {
        A.wnode[k] = L.plan.wnode[k];
        A.gamma[k] = L.plan.gamma[k];
    }
    const size_t smem = (size_t)A.region_bytes + tab;
    if (smem + 1024 > ctx->smem_optin) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "split kernel: shared memory");
    if (qcs_set_smem(ctx, (const void *)split_pair_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    // blocks per SM from the SM's shared memory (static words and the 1 KB the driver
    // reserves per block included), and at most 512 / kTmemCols so that every block's
    // tensor-memory allocation is granted at once
    int per_sm = (int)(ctx->smem_per_sm / (smem + 1024 + 1024));
    if (per_sm > (int)(512 / kTmemCols)) per_sm = (int)(512 / kTmemCols);
    if (per_sm < 1) per_sm = 1;
    const int64_t ntiles = A.ngroups * A.nchunks;
    int64_t blocks = (int64_t)ctx->num_sms * per_sm;
    if (blocks > ntiles) blocks = ntiles;
    if (blocks < 1) blocks = 1;
    if (cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return qcs_fail(ctx, QCS_ERR_CUDA, "split tile counter reset");
    qcs_prof_begin(ctx, st);
    split_pair_kernel<<<(unsigned)blocks, 128, smem, st>>>(A);
    qcs_prof_end(ctx, st);
    return qcs_check_launch(ctx, "split_pair_kernel");
}
