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
//     The walker prep leaves the orbitals in echelon form, so T skips the exact
//     zeros of Ut; at n = 16 each lane holds one snapshot row in registers and
//     takes three real products per complex multiply-add (build_T_reg).
//  2. B^(s)_ab = sum_k X_a,2k X_b,2k+1 - X_a,2k+1 X_b,2k  (X = selected rows),
//     i.e. X J X^T with J the canonical skew form (C_b was folded into Qt).
//     Computed as three classes (complex x complex, complex x real, real x real)
//     so that every FP64 instruction runs with all 32 lanes busy.
//  3. pf(B + w_k D) at the node plan's evaluation points w_k (a Gauss rule on the
//     unit circle by default, roots of unity on request), D = C_0^(s): the node
//     matrices differ only in their empty x empty block, so the occupied block is
//     eliminated once (schur_occupied, pivots inside that block) and each node's
//     2d x 2d complement is eliminated by Parlett-Reid with partial pivoting, the
//     nodes in lockstep.  The matrices (packed upper triangles) stay in shared
//     memory; the elimination keeps the original index order (no physical swaps)
//     and tracks the sign of each pivot's position; every rank-2 update step
//     spreads (node, entry) items over the lanes.  Pivot magnitudes are compared
//     as integer keys (no FP64 work).
//  4. S_p = sum_k gamma_k pf_k, where gamma_k folds the node plan's weights, the
//     inverse-channel weights C(2n,2x)/C(n,x) and the palindromic symmetry
//     c_{n-x} = c_x of parity +1 snapshots (parity -1 snapshots are exactly zero
//     and skipped).
//
// Tiles are (walker, chunk of snapshots) owned by a block of four warps; each warp
// (n <= 16) or each pair of warps (n > 16, 64-thread groups) takes every
// snapshot of the tile in turn and writes one partial sum per warp slot, reduced
// in a fixed order afterwards, so the result does not depend on scheduling.
#include "qcs_internal.h"
#include "qcs_group.cuh"

namespace {


struct PairArgs {
    int n, ne, m, d, nev, NB, all, chunk, nchunks;
    int reg;          // n = 16: snapshot rows in registers, T by three real products (build_T_reg)
    int grp;          // n > 16: two warps share a pair (64-thread groups, qcs_group.cuh)
    int t3;           // n < 16: T by three real products from staged rows and their sums
    int vm;           // entries per Gauss-vector buffer (the full matrix or NB node complements)
    int off_kh, off_ph, off_scr, gz;  // group path: pivot history, scratch, S0 offset (entries) in Ns
    int off_pvg;      // group path: the node products' records
    int off_qs;       // re + im of the staged snapshot rows (warp and group paths)
    int64_t W, P;
    int warp_bytes;   // shared bytes per warp
    int tab_bytes;    // shared bytes of the pair table (per block)
    int ut_bytes;     // shared bytes of the walker rows Ut (per block)
    int off_T, off_B, off_U, off_V, off_pf, off_inv, off_int, off_act, off_pv;  // byte offsets in a warp region
    const cd *Ut;
    const cd *pref;
    const int *wmode;  // per walker: occupied rows in reduced form (register path), or null
    const cd *Qt;
    const cd *Qh;        // rows [H1^T; G2^T] of the dense snapshots (null: T and B from Qt)
    const uint8_t *gth;  // gather codes of signed-permutation snapshots (or null)
    const int *idx;
    const int *d_count;
    cd *partial;
    cd *per_pair;
    unsigned *status;
    cd wnode[QCS_MAX_NODES];
    cd gamma[QCS_MAX_NODES];
};

// One tile of system A: walker w = tile / nchunks, the tile's snapshots spread
// over the block's warps; each warp writes one partial sum.  Every thread of the
// block calls this (it contains block barriers around the shared walker rows).
// GRP: the launch holds a system on the two-warp group path (n > 16); without one
// the group code is left out of the kernel and its registers.
template <bool GRP>
__device__ void run_tile(const PairArgs &A, int64_t tile, int64_t L, unsigned char *wbase, size_t wstride, cd *Uts,
                         const uint16_t *tab, int warp, int wpb, int lane) {
    const int n = A.n, n2 = 2 * n;
    cd *Rg = reinterpret_cast<cd *>(wbase);
    cd *Qs = Rg;  // staged snapshot rows (shared-memory path only)
    cd *Ts = reinterpret_cast<cd *>(wbase + A.off_T);
    cd *Ns = Rg;  // node matrices, once T is consumed
    double *Uss = reinterpret_cast<double *>(Uts + n * ld_ut(n));  // re + im of Ut
    cd *Bs = reinterpret_cast<cd *>(wbase + A.off_B);
    cd *Uv = reinterpret_cast<cd *>(wbase + A.off_U);
    cd *Vv = reinterpret_cast<cd *>(wbase + A.off_V);
    cd *pf = reinterpret_cast<cd *>(wbase + A.off_pf);
    uint8_t *act0 = reinterpret_cast<uint8_t *>(wbase + A.off_act);
    uint8_t *act1 = act0 + A.vm;
    cd *pv = reinterpret_cast<cd *>(wbase + A.off_pv);
    const int span = A.chunk * wpb;  // snapshots per tile; warp w takes every wpb-th
    // chunk-major tile order: consecutive tiles share one snapshot chunk and run over
    // the walkers (whose rows all fit in L2), so each snapshot is fetched from HBM once
    const int ch = (int)(tile / A.W);
    const int64_t w = tile - (int64_t)ch * A.W;
    const int64_t p0 = (int64_t)ch * span;
    const int64_t p1 = p0 + span < L ? p0 + span : L;
    // the tile from the queue and the parity +1 count address this system's buffers
    // (block-uniform: every thread leaves before the first barrier)
    if (!QCS_IN_BOUNDS(tile >= 0 && ch < A.nchunks && L >= 0 && L <= A.P, A.status)) return;
    __syncthreads();  // previous tile's readers of Uts are done
    if (p0 < L) {
        const cd *Utw = A.Ut + w * n * n;
        const int lu = ld_ut(n);
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const cd u = Utw[e];
            Uts[(e / n) * lu + (e % n)] = u;
            Uss[(e / n) * lu + (e % n)] = u.x + u.y;
        }
    }
    __syncthreads();
    cd acc = cmk(0.0, 0.0);
    const bool redw = A.wmode != nullptr && A.wmode[w] != 0;
    if (GRP && A.grp) {
        // two warps per pair: group g = warps 2g, 2g+1 with the two warp regions as its
        // workspace; group g takes every (wpb/2)-th snapshot of the tile
        const int g = warp >> 1, t = ((warp & 1) << 5) + lane, bar = 1 + g, ng = wpb >> 1;
        unsigned char *gb = wbase - (size_t)(warp & 1) * wstride;
        cd *gQs = reinterpret_cast<cd *>(gb);
        cd *gTs = reinterpret_cast<cd *>(gb + A.off_T);
        double *gqs = reinterpret_cast<double *>(gb + A.off_qs);  // re + im of the staged rows
        cd *gNs = reinterpret_cast<cd *>(gb);
        cd *gSc = gNs + A.gz;
        cd *gBs = reinterpret_cast<cd *>(gb + A.off_B);
        cd *gUv = reinterpret_cast<cd *>(gb + A.off_U);
        cd *gVv = reinterpret_cast<cd *>(gb + A.off_V);
        cd *gpf = reinterpret_cast<cd *>(gb + A.off_pf);
        cd *ginvh = reinterpret_cast<cd *>(gb + A.off_inv);
        uint8_t *gacth = gb + A.off_act;
        uint8_t *gkh = gb + A.off_kh;
        uint8_t *gph = gb + A.off_ph;
        SharedScratch *gscr = reinterpret_cast<SharedScratch *>(gb + A.off_scr);
        cd *gpv = reinterpret_cast<cd *>(gb + A.off_pvg);
        const int m = A.m, ne = A.ne, d2 = A.m - A.ne, Tn = tri_count(d2);
        if (p0 < L) {
            const cd prefw = A.pref[w];
            for (int64_t pq = p0 + g; pq < p1; pq += ng) {
                const int64_t q = A.all ? pq : (int64_t)A.idx[pq];
                if (!QCS_IN_BOUNDS(q >= 0 && q < A.P, A.status)) continue;  // group-uniform
                const uint8_t *gq = A.gth ? A.gth + q * n2 : nullptr;
                group_sync(bar);
                const bool gat = gq && gq[0] != 0xFF;
                if (gat) {
                    build_T_gather(n, Uts, gq, gTs, t, kGroup);
                } else {
                    // T (or K = Ut [H1 | G2] from the rows Qh) by column halves: half of the
                    // snapshot's rows staged at a time
                    const cd *Qr = (A.Qh ? A.Qh : A.Qt) + q * n2 * n;
                    for (int h = 0; h < 2; ++h) {
                        load_Qt_rows_sums(n, Qr + (int64_t)h * n * n, gQs, gqs, t, kGroup);
                        group_sync(bar);
                        build_T_half3(n, ne, redw, Uts, Uss, gQs, gqs, gTs, h * n, t, kGroup);
                        group_sync(bar);
                    }
                }
                group_sync(bar);
                if (!gat && A.Qh) {
                    // B from K: re + im of K1 and re - im of K2 into the staging region (free now)
                    double *gks = reinterpret_cast<double *>(gQs);
                    for (int e = t; e < n * n2; e += kGroup) {
                        const int j = e / n2, c = e - j * n2;
                        const cd k = gTs[j * ld_t(n) + c];
                        gks[e] = c < n ? k.x + k.y : k.x - k.y;
                    }
                    group_sync(bar);
                    build_B_from_K(n, ne, redw, Uts, Uss, gTs, gks, gBs, tab, t, kGroup);
                } else {
                    build_B(n, ne, gTs, gBs, tab, t, kGroup);
                }
                group_sync(bar);
                cd S = cmk(0.0, 0.0);
                if (shared_factor(m, ne, gBs, gNs, gUv, gVv, ginvh, gacth, gkh, gph, gscr, tab, t, bar)) {
                    const cd pf0 = gscr->pf0;
                    for (int e = t; e < Tn; e += kGroup) {
                        int a, b;
                        pair_of(tab, e, a, b);
                        gSc[e] = gNs[tri_index(ne + a, ne + b)];
                    }
                    group_sync(bar);
                    for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                        const int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                        group_node_pfaffians(d2, 0, A.wnode + k0, A.gamma + k0, nb, gSc, gNs, gUv, gVv, gpf, gacth,
                                             gacth + A.vm, gpv, tab, t, bar);
                        if (t == 0)
                            for (int v = 0; v < nb; ++v) S = cadd(S, gpf[v]);  // gpf[v] carries gamma
                        group_sync(bar);
                    }
                    S = cmul(S, pf0);
                } else {  // the rare full eliminations: one node matrix per round
                    for (int k0 = 0; k0 < A.nev; ++k0) {
                        group_node_pfaffians(m, ne, A.wnode + k0, A.gamma + k0, 1, gBs, gNs, gUv, gVv, gpf, gacth,
                                             gacth + A.vm, gpv, tab, t, bar);
                        if (t == 0) S = cadd(S, gpf[0]);
                        group_sync(bar);
                    }
                }
                if (t == 0) {
                    if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                    acc = cadd(acc, S);
                    if (A.per_pair) A.per_pair[w * A.P + q] = cmul(prefw, S);
                }
            }
        }
        // one partial per warp slot: the group's sum in its first warp's slot, zero in the second
        if (lane == 0) A.partial[(w * A.nchunks + ch) * wpb + warp] = (warp & 1) ? cmk(0.0, 0.0) : acc;
        return;
    }
    if (p0 < L) {
        const cd prefw = A.pref[w];
        for (int64_t pq = p0 + warp; pq < p1; pq += wpb) {
            const int64_t q = A.all ? pq : (int64_t)A.idx[pq];
            if (!QCS_IN_BOUNDS(q >= 0 && q < A.P, A.status)) continue;  // warp-uniform
            const uint8_t *gq = A.gth ? A.gth + q * n2 : nullptr;
            const bool gat = gq && gq[0] != 0xFF;
            const cd *Qr = A.Qt + q * n2 * n;
            __syncwarp();
            if (gat) {
                build_T_gather(n, Uts, gq, Ts, lane);  // signed permutation: no products
            } else if (A.reg) {
                build_T_reg<16>(A.ne, Uts, Uss, Qr, Ts, lane, redw);
            } else if (A.t3) {
                // staged rows and their re + im sums; T by three real products per
                // complex multiply-add, skipping the zeros of the echelon or reduced form
                double *qs = reinterpret_cast<double *>(wbase + A.off_qs);
                load_Qt_rows_sums(n, Qr, Qs, qs, lane, 32);
                load_Qt_rows_sums(n, Qr + n * n, Qs + n * ld_qt(n), qs + n * n, lane, 32);
                __syncwarp();
                build_T_half3(n, A.ne, redw, Uts, Uss, Qs, qs, Ts, 0, lane, 32);
                build_T_half3(n, A.ne, redw, Uts, Uss, Qs + n * ld_qt(n), qs + n * n, Ts, n, lane, 32);
            } else {  // n > 16 configured to one warp per pair: no room for the sums
                load_Qt(n, Qr, Qs, lane);
                __syncwarp();
                build_T_echelon(n, A.ne, Uts, Qs, Ts, lane);  // walker rows in echelon form
            }
            __syncwarp();
            build_B(A.n, A.ne, Ts, Bs, tab, lane);
            __syncwarp();
            // occupied block eliminated once for all nodes when that is stable
            cd *pvo = pv + pv_records(A.vm, A.NB, A.ne);  // the occupied pivots
            const bool shared = schur_occupied(A.m, A.ne, Bs, Ns, Uv, Vv, act0, act1, tab, pvo, lane);
            const int mm = shared ? A.m - A.ne : A.m, nee = shared ? 0 : A.ne;
            const int NBr = shared ? A.NB : 1;  // the rare full eliminations run one node per round
            cd S = cmk(0.0, 0.0);
            for (int k0 = 0; k0 < A.nev; k0 += NBr) {
                int nb = A.nev - k0 < NBr ? A.nev - k0 : NBr;
                node_pfaffians(mm, nee, A.wnode + k0, A.gamma + k0, nb, Bs, Ns, Uv, Vv, pf, act0, act1, tab, pv,
                               shared ? A.ne / 2 : 0, pvo, lane);
                if (lane == 0)
                    for (int v = 0; v < nb; ++v) S = cadd(S, pf[v]);  // pf[v] carries gamma
                __syncwarp();
            }
            if (lane == 0) {
                if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                acc = cadd(acc, S);
                if (A.per_pair) A.per_pair[w * A.P + q] = cmul(prefw, S);
            }
        }
    }
    if (lane == 0) A.partial[(w * A.nchunks + ch) * wpb + warp] = acc;
}

// One or several systems (different n, ne, walkers, snapshots) in one persistent
// launch.  Blocks pull tiles from a global counter (no fixed stride, so no block
// can be dealt only empty tiles); the tile space lists the systems in decreasing
// cost per tile, so the largest tiles are handed out first and the small ones
// fill the tail.
struct BatchArgs {
    int nsys;
    int tab_bytes, ut_bytes, warp_bytes;  // maxima over the systems
    int max_m;
    int64_t tile_end[QCS_MAX_SYSTEMS];    // cumulative tile counts in queue order
    unsigned long long *counter;
    PairArgs sys[QCS_MAX_SYSTEMS];         // in queue order
};

template <bool GRP>
__global__ void __launch_bounds__(128, GRP ? 2 : 3) pair_overlap_kernel(const __grid_constant__ BatchArgs B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long next_tile;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    // the pair table, the walker rows and the warps' workspaces fit the launch's shared memory
    if (!QCS_IN_BOUNDS(tri_count(B.max_m) * (int)sizeof(uint16_t) <= B.tab_bytes &&
                           (size_t)B.tab_bytes + B.ut_bytes + (size_t)wpb * B.warp_bytes <= dyn_smem_bytes(),
                       B.sys[0].status))
        return;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw);
    build_pair_table(tab, tri_count(B.max_m));
    cd *Uts = reinterpret_cast<cd *>(smem_raw + B.tab_bytes);
    unsigned char *wbase = smem_raw + B.tab_bytes + B.ut_bytes + (size_t)warp * B.warp_bytes;
    const int64_t total = B.tile_end[B.nsys - 1];
    for (;;) {
        __syncthreads();  // every thread has read the previous tile index
        if (threadIdx.x == 0) next_tile = (long long)atomicAdd(B.counter, 1ull);
        __syncthreads();
        const int64_t t = next_tile;
        if (t >= total) break;
        int s = 0;
        while (t >= B.tile_end[s]) ++s;
        const int64_t local = t - (s > 0 ? B.tile_end[s - 1] : 0);
        const PairArgs &A = B.sys[s];
        const int64_t L = A.all ? A.P : (int64_t)(*A.d_count);
        run_tile<GRP>(A, local, L, wbase, B.warp_bytes, Uts, tab, warp, wpb, lane);
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

// Per-warp shared layout for nb node matrices; returns bytes per warp.  The first
// region holds the staged snapshot rows and T (T alone on the register path), then
// the node matrices: one full copy of B (shared elimination; the rare full
// eliminations, one node per round) or NB complements of 2d x 2d.
size_t pair_group_layout(PairArgs &A, int NB);

size_t pair_warp_layout(PairArgs &A, int NB) {
    if (A.grp) return align16((pair_group_layout(A, NB) + 1) / 2);  // a group spans two warp regions
    const int n = A.n, m = A.m, T = tri_count(m), d2 = m - A.ne;
    const size_t qbytes = A.reg ? 0 : (size_t)2 * n * ld_qt(n) * sizeof(cd);
    size_t R = qbytes + (size_t)n * ld_t(n) * sizeof(cd);
    A.off_qs = (int)align16(R);  // staged rows' re + im sums (shared-memory path)
    if (A.t3) R = (size_t)A.off_qs + (size_t)2 * n * n * sizeof(double);
    if ((size_t)T * sizeof(cd) > R) R = (size_t)T * sizeof(cd);
    if ((size_t)NB * tri_count(d2) * sizeof(cd) > R) R = (size_t)NB * tri_count(d2) * sizeof(cd);
    A.vm = m > NB * d2 ? m : NB * d2;
    A.off_T = (int)qbytes;
    size_t o = align16(R);
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

// Workspace of one 64-thread group (two warp regions) on the group path: half of the
// snapshot rows and T, aliased by the node matrices (a full copy of B for the shared
// elimination, NB complements, S0 after them), then B, the Gauss vectors and the
// step history of qcs_group.cuh; returns bytes per group.
size_t pair_group_layout(PairArgs &A, int NB) {
    const int n = A.n, m = A.m, ne = A.ne, T = tri_count(m), d2 = m - ne, Tn = tri_count(d2), S = m / 2;
    const size_t qbytes = (size_t)n * ld_qt(n) * sizeof(cd);
    A.off_T = (int)align16(qbytes);
    A.off_qs = (int)align16((size_t)A.off_T + (size_t)n * ld_t(n) * sizeof(cd));
    size_t R = (size_t)A.off_qs + (size_t)n * n * sizeof(double);
    A.gz = T > NB * Tn ? T : NB * Tn;
    if ((size_t)(A.gz + Tn) * sizeof(cd) > R) R = (size_t)(A.gz + Tn) * sizeof(cd);
    A.vm = m > NB * d2 ? m : NB * d2;
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

}  // namespace

int qcs_pair_warps_per_block() { return 4; }

bool qcs_pair_forms_K(int n, int config) { return n > 16 && qcs_decode_config(config).warps != 1; }

namespace {

// Fill the per-system arguments and shared layout of one pair launch.
void setup_pair_args(qcs_ctx *ctx, const qcs_pair_launch &L, PairArgs &A) {
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
    const qcs_config cfg = qcs_decode_config(L.config);
    A.reg = L.n == 16;
    A.grp = qcs_pair_forms_K(L.n, L.config);  // n > 16: two warps per pair unless one is configured
    A.t3 = L.n < 16;
    const int n = A.n, m = A.m, T = tri_count(m);
    const int wpb = qcs_pair_warps_per_block();
    A.tab_bytes = (int)align16((size_t)T * sizeof(uint16_t));
    A.ut_bytes = (int)align16((size_t)n * ld_ut(n) * (sizeof(cd) + sizeof(double)));  // rows and re + im
    // Node matrices per round: the requested count, or by default the largest
    // count (balanced rounds, at most kMaxNB) for which three blocks (register
    // path) or two blocks fit on an SM.
    int NB = 1;
    const int nbmax = A.grp ? kMaxNBG : kMaxNB;
    if (cfg.nb > 0) {
        NB = cfg.nb < A.nev ? cfg.nb : A.nev;
        if (NB > nbmax) NB = nbmax;
        while (NB > 1 && (size_t)A.tab_bytes + A.ut_bytes + (size_t)wpb * pair_warp_layout(A, NB) > ctx->smem_optin)
            --NB;
    } else {
        const size_t sm_budget = ctx->smem_optin;
        for (int rounds = 1; rounds <= A.nev; ++rounds) {
            int nb = (A.nev + rounds - 1) / rounds;
            if (nb > nbmax) continue;
            size_t blk = (size_t)A.tab_bytes + A.ut_bytes + (size_t)wpb * pair_warp_layout(A, nb) + 1024;
            if ((A.reg ? 3 : 2) * blk <= sm_budget + 1024) {
                NB = nb;
                break;
            }
        }
    }
    A.NB = NB;
    A.warp_bytes = (int)pair_warp_layout(A, NB);
    A.Ut = L.Ut;
    A.pref = L.pref;
    A.wmode = L.mode;
    A.Qt = L.s->Qt;
    A.Qh = A.grp ? L.s->Qh : nullptr;  // the group path forms K and B from K; the warp path T
    A.gth = L.s->gth;
    A.idx = L.s->idx;
    A.d_count = L.s->d_count;
    A.partial = L.partial;
    A.per_pair = L.per_pair;
    A.status = ctx->d_status;
    for (int k = 0; k < L.plan.nev; ++k) {
        A.wnode[k] = L.plan.wnode[k];
        A.gamma[k] = L.plan.gamma[k];
    }
}

}  // namespace

qcs_status qcs_launch_pairs(qcs_ctx *ctx, const qcs_pair_launch &L, cudaStream_t st) {
    return qcs_launch_pairs_batched(ctx, 1, &L, L.counter, st);
}

qcs_status qcs_launch_pairs_batched(qcs_ctx *ctx, int nsys, const qcs_pair_launch *Ls, unsigned long long *counter,
                                    cudaStream_t st) {
    if (nsys < 1 || nsys > QCS_MAX_SYSTEMS) return QCS_ERR_ARG;
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    B.nsys = nsys;
    B.counter = counter;
    // queue order: decreasing estimated cost of one tile
    int order[QCS_MAX_SYSTEMS];
    double cost[QCS_MAX_SYSTEMS];
    for (int i = 0; i < nsys; ++i) {
        order[i] = i;
        cost[i] = qcs_overlap_flops_nev(Ls[i].n, Ls[i].ne, Ls[i].plan.nev, true) *
                  (double)Ls[i].chunk;
    }
    for (int i = 0; i < nsys; ++i)
        for (int j = i + 1; j < nsys; ++j)
            if (cost[order[j]] > cost[order[i]]) {
                int t = order[i];
                order[i] = order[j];
                order[j] = t;
            }
    int64_t acc = 0;
    for (int q = 0; q < nsys; ++q) {
        const qcs_pair_launch &L = Ls[order[q]];
        setup_pair_args(ctx, L, B.sys[q]);
        acc += L.W * L.nchunks;
        B.tile_end[q] = acc;
        if (B.sys[q].tab_bytes > B.tab_bytes) B.tab_bytes = B.sys[q].tab_bytes;
        if (B.sys[q].ut_bytes > B.ut_bytes) B.ut_bytes = B.sys[q].ut_bytes;
        if (B.sys[q].warp_bytes > B.warp_bytes) B.warp_bytes = B.sys[q].warp_bytes;
        if (B.sys[q].m > B.max_m) B.max_m = B.sys[q].m;
    }
    if (acc == 0) return QCS_OK;
    const int wpb = qcs_pair_warps_per_block();
    size_t smem = (size_t)B.tab_bytes + B.ut_bytes + (size_t)wpb * B.warp_bytes;
    if (smem + 64 > ctx->smem_optin)  // + the kernel's static tile index
        return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "batched kernel: shared memory too large");
    bool grp = false;
    for (int q = 0; q < nsys; ++q) grp |= B.sys[q].grp != 0;
    const void *kfn = grp ? (const void *)pair_overlap_kernel<true> : (const void *)pair_overlap_kernel<false>;
    if (qcs_set_smem(ctx, kfn, smem) != QCS_OK) return QCS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, wpb * 32, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t blocks = (int64_t)ctx->num_sms * per_sm;
    if (blocks > acc) blocks = acc;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, "batched counter reset");
    qcs_prof_begin(ctx, st);
    if (grp) pair_overlap_kernel<true><<<(unsigned)blocks, wpb * 32, smem, st>>>(B);
    else pair_overlap_kernel<false><<<(unsigned)blocks, wpb * 32, smem, st>>>(B);
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
