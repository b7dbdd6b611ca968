// qcs_overlap.cu -- walker x snapshot shadow overlaps on the FP64 pipe.
//
// For a pair (walker w, snapshot p) the estimator of Sec. "Classical shadows
// and the evaluation of overlaps" needs the coefficients of
// pf(A(z)), A(z) = C_0^(s) + z B^(s)  (Eqs. a_mat, b_mat).  The kernel forms:
//
//  1. T = Ut Qt^T (n x 2n complex): Ut holds the walker's orbitals (rows of
//     U^T, occupied rows / sqrt2), Qt the snapshot's complexified sign-folded
//     rows.  Row j of T is the selected row of W^* M_phi Q'^T for an occupied
//     mode j; for an empty mode the two selected real rows are (Re T_j, -Im T_j).
//  2. B^(s)_ab = sum_k X_a,2k X_b,2k+1 - X_a,2k+1 X_b,2k  (X = selected rows),
//     i.e. X J X^T with J the canonical skew form (C_b was folded into Qt).
//     Computed as three classes (complex x complex, complex x real, real x real)
//     so that every FP64 instruction runs with all 32 lanes busy.
//  3. pf(B + conj(z_k) D) at the evaluated roots of unity z_k, D = C_0^(s)
//     (pf(A(z_k)) = z_k^{m/2} pf(B + conj(z_k) D) on |z| = 1): a warp runs
//     Parlett-Reid elimination with partial pivoting on several node matrices
//     in lockstep.  The matrices (packed upper triangles) stay in shared memory;
//     the elimination keeps the original index order (no physical swaps) and
//     tracks the sign (-1)^{(position of the pivot) - 1}; every rank-2 update
//     step spreads (node, entry) items over the 32 lanes.  Pivot magnitudes are
//     compared as integer keys (no FP64 work).
//  4. S_p = sum_k gamma_k pf_k, where gamma_k folds the inverse DFT, the
//     inverse-channel weights C(2n,2x)/C(n,x) and, by default, the palindromic
//     symmetry c_{n-x} = c_x of parity +1 snapshots (only floor(N/2)+1 of the
//     N nodes are evaluated; parity -1 snapshots are exactly zero and skipped).
//
// Tiles are (walker, chunk of snapshots); each warp owns a tile at a time and
// writes one partial sum per tile, reduced in a fixed order afterwards, so the
// result does not depend on scheduling.
#include "qcs_internal.h"
#include "qcs_pair.cuh"

namespace {

constexpr int kMaxNB = 8;

struct PairArgs {
    int n, ne, m, d, nev, NB, all, chunk, nchunks;
    int64_t W, P;
    int warp_bytes;   // shared bytes per warp
    int tab_bytes;    // shared bytes of the pair table (per block)
    int ut_bytes;     // shared bytes of the walker rows Ut (per block)
    int off_R, off_B, off_U, off_V, off_pf, off_inv, off_best, off_int, off_act;  // byte offsets in a warp region
    const cd *Ut;
    const cd *pref;
    const cd *Qt;
    const int *idx;
    const int *d_count;
    cd *partial;
    cd *per_pair;
    unsigned *status;
    cd wnode[QCS_MAX_NODES];
    cd gamma[QCS_MAX_NODES];
};

// Pfaffians of nb node matrices B + wnode[k0 + v] D held in Ns (packed upper).
// On return pf[v] holds pf(B + conj(z_{k0+v}) D).
__device__ void node_pfaffians(const PairArgs &A, int k0, int nb, const cd *__restrict__ Bs, cd *__restrict__ Ns,
                               cd *__restrict__ Uv, cd *__restrict__ Vv, cd *__restrict__ pf, cd *__restrict__ inv,
                               unsigned long long *__restrict__ best, int *__restrict__ ints,
                               uint8_t *__restrict__ act0, uint8_t *__restrict__ act1, const uint16_t *__restrict__ tab,
                               int lane) {
    const int m = A.m, ne = A.ne, d = A.d;
    const int T = tri_count(m);
    int *pos = ints, *kk = ints + kMaxNB, *pp = ints + 2 * kMaxNB;
    for (int e = lane; e < nb * T; e += 32) {
        int v = e / T, t = e - v * T;
        Ns[v * T + t] = Bs[t];
    }
    for (int e = lane; e < nb * m; e += 32) {
        int v = e / m, a = e - v * m;
        act0[v * m + a] = (uint8_t)a;
    }
    if (lane < nb) pf[lane] = cmk(1.0, 0.0);
    __syncwarp();
    for (int e = lane; e < nb * d; e += 32) {
        int v = e / d, i = e - v * d;
        cd *x = Ns + v * T + tri_index(ne + 2 * i, ne + 2 * i + 1);
        *x = cadd(*x, A.wnode[k0 + v]);
    }
    __syncwarp();
    uint8_t *cur = act0, *nxt = act1;
    for (int r = m; r >= 2; r -= 2) {
        // pivot: largest |A_{k,i}| over the active row of k = cur[0]
        if (lane < nb) best[lane] = 0ull;
        __syncwarp();
        const int rc = r - 1;
        for (int e = lane; e < nb * rc; e += 32) {
            int v = e / rc, a = 1 + (e - v * rc);
            int k = cur[v * m], i = cur[v * m + a];
            unsigned key = pivot_key(Ns[v * T + tri_index(k, i)]);
            atomicMax(&best[v], ((unsigned long long)key << 32) | (unsigned long long)(0xffffu - (unsigned)a));
        }
        __syncwarp();
        if (lane < nb) {
            int a = 0xffff - (int)(best[lane] & 0xffffull);
            int k = cur[lane * m], p = cur[lane * m + a];
            cd piv = Ns[lane * T + tri_index(k, p)];
            cd f = cmul(pf[lane], piv);
            pf[lane] = ((a - 1) & 1) ? cneg(f) : f;
            inv[lane] = cinv(piv);
            pos[lane] = a;
            kk[lane] = k;
            pp[lane] = p;
        }
        __syncwarp();
        if (r == 2) break;
        // Gauss vectors over the remaining indices (original order kept)
        const int rv = r - 2;
        for (int e = lane; e < nb * rv; e += 32) {
            int v = e / rv, a2 = e - v * rv;
            int a = a2 + 1 + ((a2 + 1 >= pos[v]) ? 1 : 0);
            int i = cur[v * m + a], k = kk[v], p = pp[v];
            const cd *Nv = Ns + v * T;
            cd u = Nv[tri_index(k, i)];          // A_{k,i}; A_{i,k} = -u
            cd ut = cneg(cmul(u, inv[v]));       // A_{i,k} / A_{k,p}
            cd vv = (i < p) ? Nv[tri_index(i, p)] : cneg(Nv[tri_index(p, i)]);  // A_{i,p}
            Uv[v * m + a2] = ut;
            Vv[v * m + a2] = vv;
            nxt[v * m + a2] = (uint8_t)i;
        }
        __syncwarp();
        // rank-2 update A_ij -= ut_i v_j - v_i ut_j on the remaining pairs
        const int Tr = tri_count(rv);
        for (int e = lane; e < nb * Tr; e += 32) {
            int v = e / Tr, t = e - v * Tr;
            int a, b;
            pair_of(tab, t, a, b);
            int i = nxt[v * m + a], j = nxt[v * m + b];
            cd *x = Ns + v * T + tri_index(i, j);
            cd y = *x;
            const cd *U_ = Uv + v * m, *V_ = Vv + v * m;
            cfms(y, U_[a], V_[b]);
            cfma(y, V_[a], U_[b]);
            *x = y;
        }
        __syncwarp();
        uint8_t *t = cur;
        cur = nxt;
        nxt = t;
    }
}

__global__ void __launch_bounds__(128) pair_overlap_kernel(const __grid_constant__ PairArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int n = A.n, n2 = 2 * n;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw);
    build_pair_table(tab, tri_count(A.m));
    cd *Uts = reinterpret_cast<cd *>(smem_raw + A.tab_bytes);  // shared by the block's warps
    unsigned char *wbase = smem_raw + A.tab_bytes + A.ut_bytes + (size_t)warp * A.warp_bytes;
    cd *Rg = reinterpret_cast<cd *>(wbase);
    cd *Qs = Rg;
    cd *Ts = Rg + (size_t)n2 * ld_qt(n);
    cd *Ns = Rg;
    cd *Bs = reinterpret_cast<cd *>(wbase + A.off_B);
    cd *Uv = reinterpret_cast<cd *>(wbase + A.off_U);
    cd *Vv = reinterpret_cast<cd *>(wbase + A.off_V);
    cd *pf = reinterpret_cast<cd *>(wbase + A.off_pf);
    cd *inv = reinterpret_cast<cd *>(wbase + A.off_inv);
    unsigned long long *best = reinterpret_cast<unsigned long long *>(wbase + A.off_best);
    int *ints = reinterpret_cast<int *>(wbase + A.off_int);
    uint8_t *act0 = reinterpret_cast<uint8_t *>(wbase + A.off_act);
    uint8_t *act1 = act0 + A.NB * A.m;

    const int64_t L = A.all ? A.P : (int64_t)(*A.d_count);
    const int64_t ntiles = A.W * A.nchunks;
    const int span = A.chunk * wpb;  // snapshots per tile; warp w takes every wpb-th
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t w = tile / A.nchunks;
        const int ch = (int)(tile - w * A.nchunks);
        const int64_t p0 = (int64_t)ch * span;
        const int64_t p1 = p0 + span < L ? p0 + span : L;
        __syncthreads();  // previous tile's readers of Uts are done
        if (p0 < L) {
            const cd *Utw = A.Ut + w * n * n;
            const int lu = ld_ut(n);
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) Uts[(e / n) * lu + (e % n)] = Utw[e];
        }
        __syncthreads();
        cd acc = cmk(0.0, 0.0);
        if (p0 < L) {
            const cd prefw = A.pref[w];
            for (int64_t pq = p0 + warp; pq < p1; pq += wpb) {
                const int64_t q = A.all ? pq : (int64_t)A.idx[pq];
                __syncwarp();
                load_Qt(n, A.Qt + q * n2 * n, Qs, lane);
                __syncwarp();
                build_T(n, Uts, Qs, Ts, lane);
                __syncwarp();
                build_B(A.n, A.ne, Ts, Bs, tab, lane);
                __syncwarp();
                cd S = cmk(0.0, 0.0);
                for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                    int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                    node_pfaffians(A, k0, nb, Bs, Ns, Uv, Vv, pf, inv, best, ints, act0, act1, tab, lane);
                    if (lane == 0)
                        for (int v = 0; v < nb; ++v) cfma(S, A.gamma[k0 + v], pf[v]);
                    __syncwarp();
                }
                if (lane == 0) {
                    if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                    acc = cadd(acc, S);
                    if (A.per_pair) A.per_pair[w * A.P + q] = cmul(prefw, S);
                }
            }
        }
        if (lane == 0) A.partial[tile * wpb + warp] = acc;
    }
}

// One warp per walker: lanes sum strided partials, then a fixed-order tree.
__global__ void reduce_kernel(int64_t W, int64_t P, int nparts, const cd *__restrict__ partial,
                              const cd *__restrict__ pref, cd *__restrict__ overlap) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= W) return;
    cd s = cmk(0.0, 0.0);
    for (int c = lane; c < nparts; c += 32) s = cadd(s, partial[w * nparts + c]);
    s = warp_csum(s);
    if (lane != 0) return;
    double inv = P > 0 ? 1.0 / (double)P : 0.0;
    overlap[w] = cscale(cmul(pref[w], s), inv);
}

}  // namespace

namespace {

// Per-warp shared layout for nb node matrices; returns bytes per warp.
size_t pair_warp_layout(PairArgs &A, int NB) {
    const int n = A.n, m = A.m, T = tri_count(m);
    size_t R = (size_t)2 * n * ld_qt(n) + (size_t)n * ld_t(n);  // Qt + T
    if ((size_t)NB * T > R) R = (size_t)NB * T;
    size_t o = align16(R * sizeof(cd));
    A.off_B = (int)o;
    o = align16(o + (size_t)T * sizeof(cd));
    A.off_U = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_V = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_pf = (int)o;
    o = align16(o + (size_t)kMaxNB * sizeof(cd));
    A.off_inv = (int)o;
    o = align16(o + (size_t)kMaxNB * sizeof(cd));
    A.off_best = (int)o;
    o = align16(o + (size_t)kMaxNB * sizeof(unsigned long long));
    A.off_int = (int)o;
    o = align16(o + (size_t)3 * kMaxNB * sizeof(int));
    A.off_act = (int)o;
    o = align16(o + (size_t)2 * NB * m);
    return o;
}

}  // namespace

int qcs_pair_warps_per_block() { return 4; }

qcs_status qcs_launch_pairs(qcs_ctx *ctx, const qcs_pair_launch &L, cudaStream_t st) {
    PairArgs A;
    memset(&A, 0, sizeof(A));
    A.n = L.n;
    A.ne = L.ne;
    A.m = 2 * L.n - L.ne;
    A.d = L.n - L.ne;
    A.nev = L.plan.nev;
    A.all = L.plan.all;
    A.chunk = L.chunk;
    A.nchunks = L.nchunks;
    A.W = L.W;
    A.P = L.P;
    const int n = A.n, m = A.m, T = tri_count(m);
    const int wpb = qcs_pair_warps_per_block();
    A.tab_bytes = (int)align16((size_t)T * sizeof(uint16_t));
    A.ut_bytes = (int)align16((size_t)n * ld_ut(n) * sizeof(cd));
    // Node matrices per round: the largest count (at most kMaxNB, balanced rounds)
    // for which two blocks of wpb warps fit on an SM, else one block.
    const size_t sm_budget = ctx->smem_optin;  // per block
    int NB = 1;
    for (int rounds = 1; rounds <= A.nev; ++rounds) {
        int nb = (A.nev + rounds - 1) / rounds;
        if (nb > kMaxNB) continue;
        size_t wb = pair_warp_layout(A, nb);
        size_t blk = (size_t)A.tab_bytes + A.ut_bytes + (size_t)wpb * wb + 1024;
        if (2 * blk <= sm_budget + 1024) {
            NB = nb;
            break;
        }
        if (rounds == A.nev) NB = 1;
    }
    A.NB = NB;
    A.warp_bytes = (int)pair_warp_layout(A, NB);
    A.Ut = L.Ut;
    A.pref = L.pref;
    A.Qt = L.s->Qt;
    A.idx = L.s->idx;
    A.d_count = L.s->d_count;
    A.partial = L.partial;
    A.per_pair = L.per_pair;
    A.status = ctx->d_status;
    for (int k = 0; k < L.plan.nev; ++k) {
        A.wnode[k] = L.plan.wnode[k];
        A.gamma[k] = L.plan.gamma[k];
    }
    size_t smem = (size_t)A.tab_bytes + A.ut_bytes + (size_t)wpb * A.warp_bytes;
    if (smem > ctx->smem_optin) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "pair kernel: shared memory too large");
    if (qcs_set_smem(ctx, (const void *)pair_overlap_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_overlap_kernel, wpb * 32, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t ntiles = L.W * L.nchunks;
    int64_t blocks = (int64_t)ctx->num_sms * per_sm;
    if (blocks > ntiles) blocks = ntiles;
    if (blocks < 1) blocks = 1;
    qcs_prof_begin(ctx, st);
    pair_overlap_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(A);
    qcs_prof_end(ctx, st);
    return qcs_check_launch(ctx, "pair_overlap_kernel");
}

qcs_status qcs_launch_reduce(qcs_ctx *ctx, int64_t W, int64_t P, int nparts, const cd *partial, const cd *pref,
                             cd *overlap, cudaStream_t st) {
    if (W == 0) return QCS_OK;
    int64_t blocks = (W * 32 + 127) / 128;
    reduce_kernel<<<(unsigned)blocks, 128, 0, st>>>(W, P, nparts, partial, pref, overlap);
    return qcs_check_launch(ctx, "reduce_kernel");
}
