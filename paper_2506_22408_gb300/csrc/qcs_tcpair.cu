// qcs_tcpair.cu -- FP64-accurate overlaps with the congruence on tensor cores.
//
// For a pair (walker w, snapshot p) the Pfaffians of Eq. (a_mat) need B^(s), the
// selected rows of the rotated covariance of Eq. (b_mat).  In real form, with the
// walker's rows Ut = A + iB and the snapshot's complexified sign-folded rows
// Qt = C + iD (see qcs_snapshots.cu),
//     R = [Re T; Im T] = M N^T,   M = [[A, -B], [B, A]],  N = [C, D]   (2n x 2n each),
// and every entry of B^(s) is a signed sum of entries of
//     P = R J R^T = M H M^T,      H = N^T J N                          (2n x 2n, skew),
// J the canonical skew form on the Majorana index.  H belongs to the snapshot alone
// and is formed once per snapshot; per pair only the two products Z = H M^T and
// P = M Z remain, two dense 32 x 32 x 32 contractions (n <= 16, padded with zeros).
//
// Both run on the 5th-generation tensor cores at FP64 accuracy by error-free operand
// slicing (qcs_ozaki.cuh): each FP64 row is cut into seven 8-bit integer slices held
// exactly in BF16, the 28 slice products of levels 2..8 are accumulated exactly in
// FP32 in tensor memory (one accumulator per level), and the levels are combined
// exactly into 64-bit fixed point on the integer pipe.  The walker's slices are
// formed once per walker, the snapshot's once per snapshot; Z is re-sliced per pair
// between the two products.  The FP64 pipe is left with the Pfaffians alone.
//
// Tiles: one walker and 4 subs consecutive parity +1 snapshots (subs sub-tiles of four,
// 8 by default, tuned by qcs_autotune);
// a team of four warps owns a tile, warp i the pair of snapshot i of each sub-tile, and
// a block (one per SM) runs three teams that share the SM's tensor memory as two
// 256-column accumulators, each held from the first product of a sub-tile to the end
// of the readout of P.
//  1. bulk copies bring the four snapshots' H slices (the A operand, M = 128 rows)
//     and, once per tile, the walker's M slices (the B operand, N = 32) into shared
//     memory;
//  2. 14 tcgen05.mma kind::f16 (the 28 slice products, one N = 32 (8 - i) instruction
//     per A slice i and K = 16 step) form Z_i = H_i M^T, level L in tensor-memory
//     columns 32(L-2) .. 32(L-2)+31;
//  3. each warp reads its 32 lanes (row k of Z_i), combines the levels into fixed
//     point, takes the row scale of each row b of Z_i^T by a warp max-reduction and
//     writes the seven slices straight from the lanes as the next A operand, laid out
//     MN-major (lane k owns column k of Z_i^T);
//  4. 14 more MMAs form P_i = M Z_i (lane b of warp i, column a: P_i[a][b]); each warp
//     converts its lanes to FP64, keeps the upper triangle of P_i, assembles B^(s) and
//     runs the node Pfaffians of the FP64 path (qcs_pair.cuh).
// Every wait is bounded: a time-out raises QCS_ERR_TIMEOUT, drains and frees the
// tensor memory.
#include "qcs_internal.h"
#include "qcs_ozaki.cuh"
#include "qcs_pair.cuh"
#include "qcs_tc.cuh"

using namespace qcs_tc;
using namespace qcs_oz;

namespace {

constexpr int kSnapsPerSub = 4;                               // M = 128 rows of the first product
constexpr int kSubPerTile = 8;                                // default sub-tiles per tile: 32 snapshots
constexpr uint32_t kTmemCols = 256;                           // 7 levels x 32 columns, power of two
constexpr int kTeamThreads = 128;                             // a team: four warps, one per lane quarter
constexpr int kMaxTeams = 3;                                  // teams per block (one block per SM)
constexpr uint32_t kTmemSlots = 2;                            // 256-column accumulators per block
constexpr uint32_t kWaitIter = 1u << 26;                      // bounded mbarrier waits
constexpr int kSnapSlab = kSnapsPerSub * kSliceBytes;         // one slice of 4 snapshots: 8 KB
constexpr int kSnapRecBytes = kSlices * kSnapSlab + kSnapsPerSub * kRowsPer * 4;  // + row exponents
constexpr int kWalkRecBytes = kSlices * kSliceBytes + kRowsPer * 4;
constexpr int kOperandBytes = kSlices * kSnapSlab;           // operand region: later four warp workspaces
constexpr int kPuBytes = (kRowsPer * (kRowsPer - 1) / 2) * 8; // upper triangle of P (32 x 32), FP64

static_assert(kSnapRecBytes % 16 == 0 && kWalkRecBytes % 16 == 0, "bulk copies move multiples of 16 bytes");

// ---------------------------------------------------------------- operand records

// Walker records: warp per walker, lane r = row r of M (zero beyond 2n).
__global__ void tc_walker_prep_kernel(int n, int64_t W, const cd *__restrict__ Ut, unsigned char *__restrict__ rec) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int64_t w = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); w < W; w += (int64_t)gridDim.x * wpb) {
        const cd *U = Ut + w * n * n;
        double x[kRowsPer];
        const int r = lane;
#pragma unroll
        for (int kk = 0; kk < kRowsPer; ++kk) {
            double v = 0.0;
            if (r < 2 * n && kk < 2 * n) {
                const int j = r < n ? r : r - n, k = kk < n ? kk : kk - n;
                const cd u = U[j * n + k];
                if (r < n) v = kk < n ? u.x : -u.y;  // [A_j, -B_j]
                else v = kk < n ? u.y : u.x;         // [B_j,  A_j]
            }
            x[kk] = v;
        }
        int e = kNoRow;
#pragma unroll
        for (int kk = 0; kk < kRowsPer; ++kk)
            if (x[kk] != 0.0) e = max(e, row_exp_of(x[kk]));
        uint64_t u[kRowsPer];
        uint32_t neg = 0u;
#pragma unroll
        for (int kk = 0; kk < kRowsPer; ++kk) {
            u[kk] = e == kNoRow ? 0ull : fixed_of(x[kk], e);
            neg |= (x[kk] < 0.0 ? 1u : 0u) << kk;
        }
        unsigned char *base = rec + (size_t)w * kWalkRecBytes;
        store_row_slices(base, kSliceBytes, r, u, neg);
        reinterpret_cast<int *>(base + kSlices * kSliceBytes)[r] = e;
    }
}

// Snapshot records in the order of the parity +1 list, four per record: warp per list
// slot, lane k = row k of H = N^T J N; slots at or beyond the list's length get zero
// slices.  Shared memory: per warp the 32 x 32 matrix N (zero-padded), 8 KB.
__global__ void tc_snapshot_prep_kernel(int n, int64_t nslots, const cd *__restrict__ Qt, const int *__restrict__ idx,
                                        const int *__restrict__ d_count, unsigned char *__restrict__ rec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double *N = reinterpret_cast<double *>(smem_raw) + (size_t)warp * kRowsPer * kRowsPer;
    const int64_t L = *d_count;
    for (int64_t p = (int64_t)blockIdx.x * wpb + warp; p < nslots; p += (int64_t)gridDim.x * wpb) {
        const bool live = p < L;
        if (live) {
            const cd *Qp = Qt + (int64_t)idx[p] * 2 * n * n;
            for (int e = lane; e < kRowsPer * kRowsPer; e += 32) {
                const int c = e / kRowsPer, kk = e - c * kRowsPer;
                double v = 0.0;
                if (c < 2 * n && kk < 2 * n) {
                    const cd q = Qp[c * n + (kk < n ? kk : kk - n)];
                    v = kk < n ? q.x : q.y;
                }
                N[e] = v;
            }
        }
        __syncwarp();
        double h[kRowsPer];
        const int k = lane;
#pragma unroll
        for (int l = 0; l < kRowsPer; ++l) h[l] = 0.0;
        if (live) {
            // H[k][l] = sum_i N[2i][k] N[2i+1][l] - N[2i+1][k] N[2i][l]
            for (int i = 0; i < n; ++i) {
                const double a = N[(2 * i) * kRowsPer + k], b = N[(2 * i + 1) * kRowsPer + k];
#pragma unroll
                for (int l = 0; l < kRowsPer; ++l)
                    h[l] = fma(a, N[(2 * i + 1) * kRowsPer + l], fma(-b, N[(2 * i) * kRowsPer + l], h[l]));
            }
        }
        int e = kNoRow;
#pragma unroll
        for (int l = 0; l < kRowsPer; ++l)
            if (h[l] != 0.0) e = max(e, row_exp_of(h[l]));
        uint64_t u[kRowsPer];
        uint32_t neg = 0u;
#pragma unroll
        for (int l = 0; l < kRowsPer; ++l) {
            u[l] = e == kNoRow ? 0ull : fixed_of(h[l], e);
            neg |= (h[l] < 0.0 ? 1u : 0u) << l;
        }
        unsigned char *base = rec + (size_t)(p / kSnapsPerSub) * kSnapRecBytes;
        const int row = (int)(p % kSnapsPerSub) * kRowsPer + k;
        store_row_slices(base, kSnapSlab, row, u, neg);
        reinterpret_cast<int *>(base + kSlices * kSnapSlab)[row] = e;
        __syncwarp();
    }
}

// ---------------------------------------------------------------- pair kernel

struct TcArgs {
    int n, ne, m, d, nev, NB;
    int64_t W, P;
    int64_t nrec;     // snapshot records allocated (4 list slots each)
    int nchunks;      // tiles per walker (chunks of 4 subs list positions)
    int subs;         // sub-tiles of kSnapsPerSub snapshots per tile
    int ws_bytes;     // Pfaffian workspace per warp
    int ws_in_operands;  // 1: the workspaces are quarters of the operand region
    int teams;        // four-warp teams in the block
    int team_bytes;   // shared bytes per team: records (and workspaces if not in them)
    int tslots;       // tensor-memory accumulators of 256 columns
    int off_P, off_N, off_U, off_V, off_pf, off_act, off_pv;  // B^(s) at offset 0
    int vm;
    int smem_tab;     // byte offset of the pair table (after the teams' regions)
    const unsigned char *snap_rec;
    const unsigned char *walk_rec;
    const cd *pref;
    const int *idx;
    const int *d_count;
    cd *partial;      // W x nchunks
    cd *per_pair;
    unsigned long long *counter;
    unsigned *status;
    cd wnode[QCS_MAX_NODES];
    cd gamma[QCS_MAX_NODES];
};

// The MMAs of one sliced product, levels 2..8: per A slice i one instruction pair
// (K = 32 as two K = 16 steps, 2 core matrices = 256 bytes apart) against the B slices
// j = 1 .. 8 - i taken as one operand of N = 32 (8 - i) rows (the B slabs are
// contiguous, so slab j continues the row groups of slab j - 1), with D at column
// 32 (i - 1): the columns of slice j land in 32 (i + j - 2), the accumulator of level
// i + j.  Slice 1 spans all seven levels and starts them (no accumulate on its first
// step).  A slabs kSnapSlab apart (M = 128), K-major (H slices) or MN-major (slices of
// Z^T).
__device__ __forceinline__ void issue_products(uint32_t tbase, const unsigned char *A, const unsigned char *B,
                                               bool a_mn_major) {
    const uint32_t tr = a_mn_major ? (1u << 15) : 0u;
#pragma unroll
    for (int i = 1; i <= kSlices; ++i) {
        const uint32_t id = idesc_bf16(kSnapsPerSub * kRowsPer, kRowsPer * (kSlices + 1 - i)) | tr;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const uint64_t ad = desc_kmajor(A + (size_t)(i - 1) * kSnapSlab + 256 * ks, 128, 512);
            const uint64_t bd = desc_kmajor(B + 256 * ks, 128, 512);
            mma_f16(tbase + (uint32_t)(kRowsPer * (i - 1)), ad, bd, id, (i > 1 || ks > 0) ? 1u : 0u);
        }
    }
}

// Columns cb*8 .. cb*8+7 of the seven level accumulators of this thread's lane (level L
// in columns 32 (L - 2)), combined into fixed point: one wait for the seven loads.
__device__ __forceinline__ void read_levels8(uint32_t taddr, int cb, long long (&z)[8]) {
    float v[kLevels][8];
#pragma unroll
    for (int L = 0; L < kLevels; ++L) tmem_ld8(taddr + (uint32_t)(32 * L + 8 * cb), v[L]);
    tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float a[kLevels];
#pragma unroll
        for (int L = 0; L < kLevels; ++L) a[L] = v[L][c];
        z[c] = combine_levels(a);
    }
}

// P[a][b] (a != b) from the upper triangle Pu (P is skew-symmetric): the sign of the
// lower triangle flipped on the bit pattern, without a branch or an FP64 instruction.
__device__ __forceinline__ double pget(const double *__restrict__ Pu, int a, int b) {
    const bool sw = a > b;
    const long long v = __double_as_longlong(Pu[tri_index(sw ? b : a, sw ? a : b)]);
    return __longlong_as_double(sw ? v ^ (long long)0x8000000000000000ull : v);
}

// B^(s) (packed upper, m x m) from P = R J R^T, R = [Re T; Im T]: selected row x < ne is
// T_x (= R[x] + i R[n+x]); x >= ne is Re T_j (even offset) or -Im T_j (odd offset) for
// the empty mode j = ne + (x - ne)/2.  One loop per block (occupied x occupied, occupied
// x empty, empty x empty), so that no pass of the warp diverges across the three forms.
__device__ void build_B_from_P(int n, int ne, int m, const double *__restrict__ Pu, cd *__restrict__ Bs,
                               const uint16_t *__restrict__ tab, int lane) {
    // occupied x occupied: (R_x + i R_nx) J (R_y + i R_ny)^T, the first tri(ne) entries
    for (int t = lane; t < tri_count(ne); t += 32) {
        int x, y;
        pair_of(tab, t, x, y);  // x < y
        const double prr = pget(Pu, x, y), pii = pget(Pu, n + x, n + y);
        const double pri = pget(Pu, x, n + y), pir = pget(Pu, n + x, y);
        Bs[t] = cmk(prr - pii, pri + pir);
    }
    // occupied x empty: (R_x + i R_nx) J (+-R_ry)^T, column y = ne + c, row x < ne
    const int d2 = m - ne;
    for (int e = lane; e < d2 * ne; e += 32) {
        const int c = e / ne, x = e - c * ne;
        const int jy = ne + (c >> 1);
        const bool yim = c & 1;
        const int ry = yim ? n + jy : jy;
        cd v = cmk(pget(Pu, x, ry), pget(Pu, n + x, ry));
        Bs[tri_index(x, ne + c)] = flip_if(v, yim);
    }
    // empty x empty: (+-R_rx) J (+-R_ry)^T, real
    for (int t = lane; t < tri_count(d2); t += 32) {
        int cx, cy;
        pair_of(tab, t, cx, cy);  // cx < cy
        const int jx = ne + (cx >> 1), jy = ne + (cy >> 1);
        const bool xim = cx & 1, yim = cy & 1;
        const long long re = __double_as_longlong(pget(Pu, xim ? n + jx : jx, yim ? n + jy : jy));
        Bs[tri_index(ne + cx, ne + cy)] =
            cmk(__longlong_as_double(xim != yim ? re ^ (long long)0x8000000000000000ull : re), 0.0);
    }
}

// Byte offset of element (row, k) of a 16-bit MN-major operand of 128 rows x 32 (K) with
// no swizzle: 8 (rows) x 8 (K) core matrices with the rows contiguous (16 bytes per K
// index), K-adjacent core matrices 128 bytes apart (LBO), row-adjacent ones 512 bytes
// apart (SBO), as the descriptor of the K-major operands.
__host__ __device__ __forceinline__ uint32_t mnmajor16(int row, int k) {
    return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (k & 7) * 16 + (row & 7) * 2);
}

// Slices of Z_i^T, read from tensor memory (lane k holds row k of Z_i, z_kb worth
// z 2^{g_k + e_b - 56}): row b of Z_i^T gets the scale 2^{F_b}, F_b = e_b + G_b - 56 with
// G_b = max_k (g_k + bitlen z_kb) (a warp max-reduction); the slices go MN-major into
// the A operand rows row0 + b.  Returns F_b for b = lane (kNoRow for a zero row).
__device__ __forceinline__ int slice_zt(uint32_t tlane, int gk, int eb_lane, unsigned char *Abase, int row0, int lane) {
    int Gl = kNoRow;
#pragma unroll 1
    for (int cb = 0; cb < 4; ++cb) {
        long long z[8];
        read_levels8(tlane, cb, z);
        uint64_t u[8];
        SliceSign g[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int t = z[c] != 0 ? gk + bitlen64(z[c]) : kNoRow;
            const int G = __reduce_max_sync(QCS_FULL, t);
            if (8 * cb + c == lane) Gl = G;
            u[c] = (z[c] == 0 || G == kNoRow) ? 0ull : rescale_mag(z[c], 56 + gk - G);
            g[c] = slice_sign(z[c] < 0);
        }
#pragma unroll
        for (int i = 1; i <= kSlices; ++i) {
            uint4 w;
            w.x = bf16x2_of(slice_f32(u[0], i, g[0]), slice_f32(u[1], i, g[1]));
            w.y = bf16x2_of(slice_f32(u[2], i, g[2]), slice_f32(u[3], i, g[3]));
            w.z = bf16x2_of(slice_f32(u[4], i, g[4]), slice_f32(u[5], i, g[5]));
            w.w = bf16x2_of(slice_f32(u[6], i, g[6]), slice_f32(u[7], i, g[7]));
            *reinterpret_cast<uint4 *>(Abase + (size_t)(i - 1) * kSnapSlab + mnmajor16(row0 + 8 * cb, lane)) = w;
        }
    }
    return (Gl != kNoRow && eb_lane != kNoRow) ? eb_lane + Gl - 56 : kNoRow;
}

// Team barrier (named barrier 1 + team over the team's 128 threads) and the same
// barrier with an AND over a predicate, so that every thread of a team takes the same
// branch after a bounded wait.
__device__ __forceinline__ void team_sync(int team) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "n"(kTeamThreads) : "memory");
}
__device__ __forceinline__ bool team_and(int team, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + team), "n"(kTeamThreads)
        : "memory");
    return r != 0;
}

// One block per SM holds up to kMaxTeams teams of four warps.  Each team has its own
// operand records (and, in them, its warps' Pfaffian workspaces) and runs the tile loop
// of the header on its own: a team is what a block of four warps would be, except that
// the tensor memory of the SM (512 columns) is shared as two 256-column accumulators.
// A team holds one from its first product of a sub-tile to the end of the readout of
// P (a bounded spin on a lock word in shared memory), so three teams, twelve warps per
// SM, keep the FP64 pipe fed while the tensor memory would only allow two blocks of four.
__global__ void __launch_bounds__(kTeamThreads * kMaxTeams, 1) tc_pair_kernel(const __grid_constant__ TcArgs A) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar_load[kMaxTeams], mbar_mma[kMaxTeams];
    __shared__ long long next_tile[kMaxTeams];
    __shared__ int slot_of[kMaxTeams];
    __shared__ int slot_owner[kTmemSlots];
    __shared__ int abort_flag;
    __shared__ cd red[kMaxTeams][4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int team = warp >> 2, wt = warp & 3, ttid = tid & (kTeamThreads - 1);
    const int n = A.n;
    unsigned char *X = smem_tc + (size_t)team * A.team_bytes;     // operands, then (usually) workspaces
    unsigned char *Wrec = X + kSnapRecBytes;                      // walker record
    const int *g_exp = reinterpret_cast<const int *>(X + kOperandBytes);              // snapshot row exponents
    const int *e_exp = reinterpret_cast<const int *>(Wrec + kSlices * kSliceBytes);  // walker row exponents
    // the teams' records, their workspaces and the pair table fit the launch's shared
    // memory, and the block is a whole number of teams (block-uniform: nothing is
    // allocated or issued yet)
    if (!QCS_IN_BOUNDS((int)blockDim.x == kTeamThreads * A.teams && A.teams <= kMaxTeams &&
                           A.tslots >= 1 && A.tslots <= (int)kTmemSlots &&
                           A.teams * A.team_bytes <= A.smem_tab &&
                           A.smem_tab + tri_count(A.m) * (int)sizeof(uint16_t) <= (int)dyn_smem_bytes() &&
                           (A.ws_in_operands ? 4 * A.ws_bytes <= kOperandBytes
                                             : kSnapRecBytes + kWalkRecBytes + 4 * A.ws_bytes <= A.team_bytes),
                       A.status))
        return;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_tc + A.smem_tab);
    build_pair_table(tab, tri_count(A.m));
    unsigned char *wbase = (A.ws_in_operands ? X : X + kSnapRecBytes + kWalkRecBytes) + (size_t)wt * A.ws_bytes;
    cd *Bs = reinterpret_cast<cd *>(wbase);
    double *Pu = reinterpret_cast<double *>(wbase + A.off_P);
    cd *Ns = reinterpret_cast<cd *>(wbase + A.off_N);  // aliases Pu: written once B^(s) is assembled
    cd *Uv = reinterpret_cast<cd *>(wbase + A.off_U);
    cd *Vv = reinterpret_cast<cd *>(wbase + A.off_V);
    cd *pf = reinterpret_cast<cd *>(wbase + A.off_pf);
    uint8_t *act0 = wbase + A.off_act;
    uint8_t *act1 = act0 + A.vm;
    cd *pv = reinterpret_cast<cd *>(wbase + A.off_pv);

    if (warp == 0) {
        tmem_alloc(&tmem_base, (uint32_t)A.tslots * kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int k = 0; k < kMaxTeams; ++k) {
            mbar_init(&mbar_load[k], 1);
            mbar_init(&mbar_mma[k], 1);
        }
        for (int k = 0; k < (int)kTmemSlots; ++k) slot_owner[k] = -1;
        abort_flag = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem0 = tmem_base;
    const int64_t L = *A.d_count;
    const int64_t ntiles = A.W * (int64_t)A.nchunks;
    uint32_t ph_load = 0, ph_mma = 0;
    bool load_pending = false, mma_pending = false;
    bool ok = true;
    int held = -1;  // tensor-memory slot this team holds
    // one sliced product issued by the team's first thread into the held slot, then a
    // bounded wait whose outcome the team shares
    auto product = [&](bool mn, uint32_t tbase) {
        if (ttid == 0) {
            fence_after_sync();
            issue_products(tbase, X, Wrec, mn);
            mma_commit(&mbar_mma[team]);
        }
        mma_pending = true;
        const bool r = team_and(team, mbar_wait_bounded(&mbar_mma[team], ph_mma, kWaitIter));
        if (r) {
            ph_mma ^= 1u;
            mma_pending = false;
            fence_after_sync();
        }
        return r;
    };
    // a free accumulator slot for the team (bounded spin), shared with the team
    auto acquire = [&]() {
        if (ttid == 0) {
            int got = -1;
            for (uint32_t it = 0; it < kWaitIter && got < 0; ++it) {
                if (*(volatile int *)&abort_flag) break;
                for (int k = 0; k < A.tslots && got < 0; ++k)
                    if (atomicCAS(&slot_owner[k], -1, team) == -1) got = k;
                if (got < 0) __nanosleep(64);
            }
            __threadfence_block();
            slot_of[team] = got;
        }
        team_sync(team);
        held = slot_of[team];
        return team_and(team, held >= 0);
    };
    // every warp's tensor-memory reads of the slot are done: hand it back
    auto release = [&]() {
        fence_before_sync();
        team_sync(team);
        if (ttid == 0 && held >= 0) {
            __threadfence_block();
            atomicExch(&slot_owner[held], -1);
        }
        held = -1;
    };
    for (;;) {
        fence_proxy_async_smem();  // generic writes to the operand region precede the next bulk copies
        team_sync(team);
        if (ttid == 0)
            next_tile[team] = *(volatile int *)&abort_flag ? (long long)ntiles : (long long)atomicAdd(A.counter, 1ull);
        team_sync(team);
        const int64_t t = next_tile[team];
        if (t >= ntiles) break;
        const int ch = (int)(t / A.W);  // chunk-major: a chunk's records stay in L2 over the walkers
        const int64_t w = t - (int64_t)ch * A.W;
        const int64_t p0 = (int64_t)ch * (kSnapsPerSub * A.subs);
        if (!QCS_IN_BOUNDS(ch < A.nchunks && L >= 0 && L <= A.P, A.status)) continue;  // team-uniform
        if (p0 >= L) {
            if (ttid == 0) A.partial[w * A.nchunks + ch] = cmk(0.0, 0.0);
            continue;
        }
        const cd prefw = A.pref[w];
        cd acc = cmk(0.0, 0.0);
        for (int s = 0; s < A.subs; ++s) {
            const int64_t pb = p0 + (int64_t)s * kSnapsPerSub;
            if (pb >= L) break;
            if (!QCS_IN_BOUNDS(pb / kSnapsPerSub < A.nrec, A.status)) break;  // the record to copy exists
            if (ttid == 0) {
                const uint32_t bytes = kSnapRecBytes + (s == 0 ? kWalkRecBytes : 0);
                mbar_expect_tx(&mbar_load[team], bytes);
                bulk_copy(X, A.snap_rec + (size_t)(pb / kSnapsPerSub) * kSnapRecBytes, kSnapRecBytes,
                          &mbar_load[team]);
                if (s == 0) bulk_copy(Wrec, A.walk_rec + (size_t)w * kWalkRecBytes, kWalkRecBytes, &mbar_load[team]);
            }
            load_pending = true;
            ok = team_and(team, mbar_wait_bounded(&mbar_load[team], ph_load, kWaitIter));
            if (!ok) break;
            ph_load ^= 1u;
            load_pending = false;
            if (!(ok = acquire())) break;
            fence_after_sync();
            const uint32_t tbase = tmem0 + (uint32_t)held * kTmemCols;
            const uint32_t tlane = tbase + ((uint32_t)(32 * wt) << 16);  // this warp's 32 lanes
            // ---- Z_i = H_i M^T: lane k holds row k; sliced by rows of Z^T (MN-major)
            if (!(ok = product(false, tbase))) break;
            // the operand region held H_i, which the completed MMAs no longer read
            const int Fb = slice_zt(tlane, g_exp[wt * kRowsPer + lane], e_exp[lane], X, wt * kRowsPer, lane);
            fence_proxy_async_smem();
            fence_before_sync();
            team_sync(team);  // every warp's tensor-memory reads and operand writes are done
            // ---- P_i = M Z_i: lane b, column a holds P_i[a][b] = z 2^{e_a + F_b - 56}
            if (!(ok = product(true, tbase))) break;
#pragma unroll 1
            for (int cb = 0; cb < 4; ++cb) {
                long long z[8];
                read_levels8(tlane, cb, z);
                // every lane converts all eight entries (no divergence); the upper
                // triangle of P_i (a < lane) is stored into the free operand region
                bool in_range = true;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int a = 8 * cb + c;
                    const int ea = e_exp[a];
                    const bool zero = Fb == kNoRow || ea == kNoRow;
                    const double val = fixed_to_f64(zero ? 0ll : z[c], ea + Fb - 56, in_range);
                    if (a < lane) Pu[tri_index(a, lane)] = val;
                }
                if (!__all_sync(QCS_FULL, in_range)) {  // an exponent outside the normal range
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int a = 8 * cb + c;
                        const int ea = e_exp[a];
                        if (a < lane && Fb != kNoRow && ea != kNoRow)
                            Pu[tri_index(a, lane)] = fixed_to_f64_exact(z[c], ea + Fb - 56);
                    }
                }
            }
            release();  // this team's tensor-memory reads are done; another team may use the slot
            const int64_t slot = pb + wt;
            if (slot < L && QCS_IN_BOUNDS(A.idx[slot] >= 0 && A.idx[slot] < A.P, A.status)) {
                build_B_from_P(n, A.ne, A.m, Pu, Bs, tab, lane);
                __syncwarp();
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
                        for (int v = 0; v < nb; ++v) S = cadd(S, pf[v]);  // pf[v] carries gamma
                    __syncwarp();
                }
                if (lane == 0) {
                    if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                    acc = cadd(acc, S);
                    if (A.per_pair) A.per_pair[w * A.P + A.idx[slot]] = cmul(prefw, S);
                }
            }
            fence_proxy_async_smem();  // workspace writes precede the next sub-tile's bulk copy
            team_sync(team);
        }
        if (!ok) {
            if (ttid == 0) {
                atomicExch(&abort_flag, 1);
                raise_status(A.status, QCS_ERR_TIMEOUT);
            }
            // a held slot stays held: MMAs that missed their wait may still write it, and
            // the other teams stop at the abort flag instead of waiting for it
            continue;  // every thread of the team leaves through the abort check at the top
        }
        if (lane == 0) red[team][wt] = acc;
        team_sync(team);
        if (ttid == 0) A.partial[w * A.nchunks + ch] = cadd(cadd(red[team][0], red[team][1]), cadd(red[team][2], red[team][3]));
    }
    if (ttid == 0 && (load_pending || mma_pending)) {  // a wait gave up: let a copy or MMAs in flight land first
        if (load_pending) mbar_wait_bounded(&mbar_load[team], ph_load, kWaitIter);
        if (mma_pending) mbar_wait_bounded(&mbar_mma[team], ph_mma, kWaitIter);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem0, (uint32_t)A.tslots * kTmemCols);
}

// Pfaffian workspace of one warp for nb node matrices: B^(s), then the upper triangle
// of P aliased by the node matrices (written once B^(s) is assembled), then the Gauss
// vectors and the step records; returns its bytes.
size_t tc_warp_layout(TcArgs &A, int NB) {
    const int m = A.m, T = tri_count(m), d2 = m - A.ne;
    const size_t nodes = (size_t)(T > NB * tri_count(d2) ? T : NB * tri_count(d2)) * sizeof(cd);
    A.vm = m > NB * d2 ? m : NB * d2;
    size_t o = align16((size_t)T * sizeof(cd));
    A.off_P = A.off_N = (int)o;
    o = align16(o + (nodes > (size_t)kPuBytes ? nodes : (size_t)kPuBytes));
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

size_t qcs_tc_walker_bytes(int64_t W) { return (size_t)(W > 0 ? W : 1) * kWalkRecBytes; }

int qcs_tc_snaps_per_tile(int subs) { return kSnapsPerSub * (subs > 0 ? subs : kSubPerTile); }

bool qcs_tc_supported(int n) { return n >= 2 && 2 * n <= kRowsPer; }

qcs_status qcs_tc_prepare_snapshots(qcs_ctx *ctx, qcs_snapshots *s, cudaStream_t st) {
    if (s->tc_rec) return QCS_OK;
    if (!qcs_tc_supported(s->n)) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "tensor-core congruence needs n <= 16");
    const int64_t nsub = (s->P + kSnapsPerSub - 1) / kSnapsPerSub;
    const size_t bytes = (size_t)(nsub > 0 ? nsub : 1) * kSnapRecBytes;
    if (qcs_dev_alloc(s->alloc, &s->tc_rec, bytes, st) != QCS_OK) {
        s->tc_rec = nullptr;
        return qcs_fail(ctx, QCS_ERR_CUDA, "tensor-core snapshot records: device allocation failed");
    }
    s->tc_bytes = bytes;
    if (nsub == 0) return QCS_OK;
    const int wpb = 4;
    const size_t smem = (size_t)wpb * kRowsPer * kRowsPer * sizeof(double);
    if (qcs_set_smem(ctx, (const void *)tc_snapshot_prep_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    const int64_t nslots = nsub * kSnapsPerSub;
    int64_t blocks = (nslots + wpb - 1) / wpb;
    if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
    tc_snapshot_prep_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(s->n, nslots, s->Qt, s->idx, s->d_count,
                                                                       (unsigned char *)s->tc_rec);
    return qcs_check_launch(ctx, "tc_snapshot_prep_kernel");
}

qcs_status qcs_launch_tc_pairs(qcs_ctx *ctx, const qcs_pair_launch &L, unsigned char *walk_rec, cudaStream_t st) {
    const int n = L.n;
    if (!qcs_tc_supported(n)) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "tensor-core congruence needs n <= 16");
    if (!L.s->tc_rec) return qcs_fail(ctx, QCS_ERR_ARG, "snapshot records for the tensor-core path are missing");
    if (L.W == 0) return QCS_OK;
    {
        const int wpb = 4;
        int64_t blocks = (L.W + wpb - 1) / wpb;
        if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
        tc_walker_prep_kernel<<<(unsigned)blocks, wpb * 32, 0, st>>>(n, L.W, L.Ut, walk_rec);
        qcs_status r = qcs_check_launch(ctx, "tc_walker_prep_kernel");
        if (r != QCS_OK) return r;
    }
    TcArgs A;
    memset(&A, 0, sizeof(A));
    A.n = n;
    A.ne = L.ne;
    A.m = 2 * n - L.ne;
    A.d = n - L.ne;
    A.nev = L.plan.nev;
    A.W = L.W;
    A.P = L.P;
    A.nrec = (L.P + kSnapsPerSub - 1) / kSnapsPerSub;
    A.nchunks = L.nchunks;
    // node matrices per round: the requested count, or the largest balanced count whose
    // four workspaces fit in the operand region; when even one node per round does not
    // fit there (large m), the workspaces get their own shared memory
    auto fits = [&](int nb) { return 4 * tc_warp_layout(A, nb) <= (size_t)kOperandBytes; };
    int NB = 1;
    const qcs_config cfg = qcs_decode_config(L.config);
    A.subs = cfg.subs > 0 ? cfg.subs : kSubPerTile;
    if (cfg.nb > 0) {
        NB = cfg.nb < A.nev ? cfg.nb : A.nev;
        if (NB > kMaxNB) NB = kMaxNB;
        while (NB > 1 && !fits(NB)) --NB;
    } else {
        for (int rounds = 1; rounds <= A.nev; ++rounds) {
            const int nb = (A.nev + rounds - 1) / rounds;
            if (nb > kMaxNB) continue;
            if (fits(nb)) {
                NB = nb;
                break;
            }
        }
    }
    A.NB = NB;
    A.ws_in_operands = fits(NB) ? 1 : 0;
    A.ws_bytes = (int)tc_warp_layout(A, NB);
    // teams per block: as many as the block's shared memory holds (about 1 KB kept for
    // the static words), at most kMaxTeams; one block per SM
    A.team_bytes = kSnapRecBytes + kWalkRecBytes + (A.ws_in_operands ? 0 : 4 * A.ws_bytes);
    const size_t tab = align16((size_t)tri_count(A.m) * sizeof(uint16_t));
    int teams = (int)((ctx->smem_optin - 1024 - tab) / (size_t)A.team_bytes);
    if (teams > kMaxTeams) teams = kMaxTeams;
    if (teams < 1) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "tc kernel: shared memory");
    A.teams = teams;
    A.tslots = teams >= 2 ? 2 : 1;
    A.smem_tab = teams * A.team_bytes;
    const size_t smem = (size_t)A.smem_tab + tab;
    A.snap_rec = (const unsigned char *)L.s->tc_rec;
    A.walk_rec = walk_rec;
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
    if (smem + 1024 > ctx->smem_optin) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "tc kernel: shared memory");
    if (qcs_set_smem(ctx, (const void *)tc_pair_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    // one block per SM (its shared memory and its 2 x 256 tensor-memory columns take the
    // SM), fewer when there are fewer tiles than teams
    const int64_t ntiles = A.W * (int64_t)A.nchunks;
    int64_t blocks = (int64_t)ctx->num_sms;
    if (blocks > (ntiles + teams - 1) / teams) blocks = (ntiles + teams - 1) / teams;
    if (blocks < 1) blocks = 1;
    if (cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return qcs_fail(ctx, QCS_ERR_CUDA, "tc tile counter reset");
    qcs_log(3, "tc_pair_kernel: %lld blocks x %d teams, %zu bytes of shared memory, %d tensor-memory slots",
            (long long)blocks, teams, smem, A.tslots);
    qcs_prof_begin(ctx, st);
    tc_pair_kernel<<<(unsigned)blocks, kTeamThreads * teams, smem, st>>>(A);
    qcs_prof_end(ctx, st);
    return qcs_check_launch(ctx, "tc_pair_kernel");
}
