// qcs_grad.cu -- holomorphic walker gradient of the shadow overlap and the force bias.
//
// Per pair the overlap term is pref_w * S_p with S_p = sum_k gamma_k pf(A'_k),
// A'_k = B + conj(z_k) D and B = X J X^T (X = selected rows of the walker-rotated
// snapshot, see qcs_overlap.cu).  Eq. (Pfaffian_der), d pf(A) = pf(A) tr(A^{-1} dA)/2,
// gives dS_p = tr(Y_p dB) with Y_p = (1/2) sum_k gamma_k pf_k A'_k^{-1}, hence
// dS_p = 2 tr(J X^T Y_p dX): the pair's cotangent on X is G_X = 2 Y_p X J.  The
// occupied rows of X are T_j, the empty ones (Re T_j, -Im T_j), T = Ut Qt^T, so
// G_X maps to a holomorphic part on the occupied rows of Ut and an
// antiholomorphic part on its empty rows:
//     Gamma1 += G_X[occ] Qt          (ne x n)
//     Gamma2 += Ht[empty] conj(Qt),  Ht_j = (G_X[2j'] - i G_X[2j'+1]) / 2   (d x n).
// The walker then moves by a unitary rotation of its orbitals (the column
// space part) plus a change of R (the in-span part); with Lambda =
// Gamma1/sqrt2 - U_occ^dagger Gamma2^T U^dagger (the antiholomorphic terms of the
// rotation cancel because the overlap is holomorphic in Phi):
//     g^T = (c0 / P) adj(R) [ S U_occ^dagger + Lambda (I - U_occ U_occ^dagger) ],
//     c0 = 2 i^{ne/2} / 2^{n - ne/2},  S = sum_p S_p,
// with adj(R) = det(R) R^{-1} formed without divisions, so rank-deficient
// walkers need no special case.  The walker rows of Ut are in echelon form
// (qcs_walker.cu): U_occ = U_qr W, and R above is W^H R_qr, so the epilogue
// takes adj(R_qr) det(conj W) W and det(conj W) det(R_qr).
//
// A'_k^{-1} is recomputed per pair and node, never stored in global memory: the
// Parlett-Reid elimination (as in the overlap kernel, original index order)
// leaves its Gauss vectors in place, and a backward recursion over the
// elimination steps assembles the inverse from the 2x2 pivot blocks:
//     (A^{-1})_{rest,k} = -Z g1,  (A^{-1})_{rest,p} = -Z g2,
//     (A^{-1})_{k,p} = -1/a + g1^T Z g2,  g1 = v/a, g2 = -u/a,
// where Z is the inverse of the step's Schur complement and (u, v, a) the
// step's pivot columns and pivot.  The node matrices share their occupied block, so
// its steps are taken once per pair (shared_factor); each node then factors and
// inverts only its 2d x 2d complement, and since every backward step is affine in Z,
// one backward pass over the shared steps, started from sum_k c_k Z_k, gives
// Y_p = sum_k c_k A'_k^{-1} (shared_inverse).  Pairs whose occupied block would grow
// the complement beyond 2^8 of max|B| take the full elimination per node.
#include "qcs_internal.h"
#include "qcs_group.cuh"

namespace {


struct GradArgs {
    int n, ne, m, d, nev, NB, all, chunk, nchunks;
    int64_t W, P;
    int group_bytes, tab_bytes;
    int off_Q, off_T, off_B, off_Y, off_G, off_NZ, off_g1, off_g2, off_y1, off_y2, off_pf, off_cf, off_invh,
        off_int, off_tile, off_acth, off_kh, off_ph, off_kc, off_sacth, off_skh, off_sph, off_sinvh, off_scr;
    const cd *Ut;
    const cd *Qt;
    const cd *Qh;        // per dense snapshot of the set: the rows [H1^T; G2^T] (2n x n, the layout of Qt)
    const uint8_t *gth;  // gather codes of signed-permutation snapshots (or null)
    const int *idx;
    const int *d_count;
    cd *partial;
    unsigned long long *counter;  // tile counter: groups pull tiles dynamically
    unsigned *status;
    cd wnode[QCS_MAX_NODES];
    cd gamma[QCS_MAX_NODES];
};

// B (packed upper, m x m) from K = [Ut H1 | Ut G2] (rows of Ks, stride ld_t) and the walker
// rows Ut: with W1 = (Ut H1) Ut^T = T J T^T and W2 = (Ut G2) Ut^H = T J conj(T)^T, and the
// empty rows R_j = Re T_j, I_j = -Im T_j of X,
//     occupied a, b:          W1[a][b]
//     occupied a, empty j:    (a, R_j) = (W1 + W2)[a][j] / 2,   (a, I_j) = i (W1 - W2)[a][j] / 2
//     empty j1 <= j2, al = W1[j1][j2], be = W2[j1][j2]:
//         (R, R) = Re(al + be)/2,  (R, I) = Im(be - al)/2,  (I, R) = -Im(al + be)/2,
//         (I, I) = Re(be - al)/2;  within one mode (al = 0) only (R_j, I_j) = Im(be)/2.
// Work items: the tri(ne) occupied pairs, the ne x d occupied-empty pairs and the
// tri(d + 1) empty pairs j1 <= j2, each two n-term sums (the echelon zeros of Ut included,
// so that every lane runs the same loop).
__device__ inline void build_B_from_K3(int n, int ne, const cd *__restrict__ Uts, const double *__restrict__ Uss,
                                      const double *__restrict__ Usd, const cd *__restrict__ Ks,
                                      const double *__restrict__ Ksum, cd *__restrict__ Bs,
                                      const uint16_t *__restrict__ tab, int t, int nthr) {
    const int d = n - ne, lu = ld_ut(n), lt = ld_t(n), n2 = 2 * n;
    const int c1 = tri_count(ne), c2 = c1 + ne * d, c3 = c2 + tri_count(d + 1);
    for (int it = t; it < c3; it += nthr) {
        int a, b, kind;  // K row a, walker row b
        if (it < c1) {
            pair_of(tab, it, a, b);
            kind = 0;
        } else if (it < c2) {
            const int e = it - c1, jj = e / ne;
            a = e - jj * ne;
            b = ne + jj;
            kind = 1;
        } else {
            int x, y;
            pair_of(tab, it - c2, x, y);  // x < y: empty modes x <= y - 1
            a = ne + x;
            b = ne + y - 1;
            kind = 2;
        }
        // three real products per complex term: K1 u with the sums re + im of both factors,
        // K2 conj(u) with re + im of K2 and re - im of u
        const cd *kr = Ks + a * lt, *ur = Uts + b * lu;
        const double *ks = Ksum + a * n2, *us = Uss + b * lu, *ud = Usd + b * lu;
        double p1 = 0.0, p2 = 0.0, p3 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
        for (int k = 0; k < n; ++k) {
            const cd u = ur[k], k1 = kr[k], k2 = kr[n + k];
            p1 = fma(k1.x, u.x, p1);
            p2 = fma(k1.y, u.y, p2);
            p3 = fma(ks[k], us[k], p3);
            q1 = fma(k2.x, u.x, q1);
            q2 = fma(k2.y, u.y, q2);
            q3 = fma(ks[n + k], ud[k], q3);
        }
        const cd w1 = cmk(p1 - p2, p3 - p1 - p2), w2 = cmk(q1 + q2, q3 - q1 + q2);
        if (kind == 0) {
            Bs[tri_index(a, b)] = w1;
        } else if (kind == 1) {
            const int r = 2 * (b - ne);
            const cd sp = cadd(w1, w2), dm = csub(w1, w2);
            Bs[tri_index(a, ne + r)] = cscale(sp, 0.5);
            Bs[tri_index(a, ne + r + 1)] = cmk(-0.5 * dm.y, 0.5 * dm.x);
        } else {
            const int r1 = 2 * (a - ne), r2 = 2 * (b - ne);
            if (r1 < r2) {
                Bs[tri_index(ne + r1, ne + r2)] = cmk(0.5 * (w1.x + w2.x), 0.0);
                Bs[tri_index(ne + r1, ne + r2 + 1)] = cmk(0.5 * (w2.y - w1.y), 0.0);
                Bs[tri_index(ne + r1 + 1, ne + r2)] = cmk(-0.5 * (w1.y + w2.y), 0.0);
                Bs[tri_index(ne + r1 + 1, ne + r2 + 1)] = cmk(0.5 * (w2.x - w1.x), 0.0);
            } else {
                Bs[tri_index(ne + r1, ne + r1 + 1)] = cmk(0.5 * w2.y, 0.0);
            }
        }
    }
}

// Two warps (a group of 64 threads) per pair; a block holds blockDim/64 groups,
// each with its own workspace and named barrier.  Groups pull (walker, chunk)
// tiles from a device counter in chunk-major order.
__global__ void __launch_bounds__(128, 2) grad_pair_kernel(const __grid_constant__ GradArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / kGroup;
    const int t = threadIdx.x - gid * kGroup;
    const int bar = 1 + gid;
    const int n = A.n, n2 = 2 * n, ne = A.ne, m = A.m, T = tri_count(m);
    const int lu = ld_ut(n), lq = ld_qt(n), lt = ld_t(n);
    // the pair table and the groups' workspaces fit the launch's shared memory
    if (!QCS_IN_BOUNDS(T * (int)sizeof(uint16_t) <= A.tab_bytes &&
                           (size_t)A.tab_bytes + (size_t)(blockDim.x / kGroup) * A.group_bytes <= dyn_smem_bytes(),
                       A.status))
        return;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw);
    build_pair_table(tab, T);
    __syncthreads();
    unsigned char *wb = smem_raw + A.tab_bytes + (size_t)gid * A.group_bytes;
    cd *Uts = reinterpret_cast<cd *>(wb);
    cd *Qs = reinterpret_cast<cd *>(wb + A.off_Q);
    cd *Ts = reinterpret_cast<cd *>(wb + A.off_T);
    cd *Bs = reinterpret_cast<cd *>(wb + A.off_B);
    cd *Ys = reinterpret_cast<cd *>(wb + A.off_Y);
    cd *Gs = reinterpret_cast<cd *>(wb + A.off_G);
    cd *Ns = reinterpret_cast<cd *>(wb + A.off_NZ);  // node factors, then their inverses, then G_X
    cd *GX = Ns;
    double *Uss = reinterpret_cast<double *>(Ns);  // while T (or K) and B are formed: re + im of Ut
    double *Usd = Uss + n * lu;                     // and re - im of Ut
    double *Ksum = reinterpret_cast<double *>(Qs);  // once K is formed: re + im of K (n x 2n)
    double *Kdif = Ksum + n * n2;                   // and re - im of K's empty rows (d x 2n)
    cd *g1v = reinterpret_cast<cd *>(wb + A.off_g1);  // forward: U vectors
    cd *g2v = reinterpret_cast<cd *>(wb + A.off_g2);  // forward: V vectors
    cd *y1v = reinterpret_cast<cd *>(wb + A.off_y1);
    cd *y2v = reinterpret_cast<cd *>(wb + A.off_y2);
    cd *pf = reinterpret_cast<cd *>(wb + A.off_pf);
    cd *cf = reinterpret_cast<cd *>(wb + A.off_cf);
    cd *invh = reinterpret_cast<cd *>(wb + A.off_invh);
    int *pos = reinterpret_cast<int *>(wb + A.off_int);
    long long *slot = reinterpret_cast<long long *>(wb + A.off_tile);
    uint8_t *acth = wb + A.off_acth;
    uint8_t *kh = wb + A.off_kh;
    uint8_t *ph = wb + A.off_ph;
    uint8_t *kc = wb + A.off_kc;  // signed-permutation snapshots: the two rows of each column of Qt
    uint8_t *sacth = wb + A.off_sacth;  // history of the shared occupied-block elimination
    uint8_t *skh = wb + A.off_skh;
    uint8_t *sph = wb + A.off_sph;
    cd *sinvh = reinterpret_cast<cd *>(wb + A.off_sinvh);
    SharedScratch *scr = reinterpret_cast<SharedScratch *>(wb + A.off_scr);

    const int64_t L = A.all ? A.P : (int64_t)(*A.d_count);
    const int64_t ntiles = A.W * A.nchunks;
    const size_t rec = 1 + (size_t)n * n;
    for (;;) {
        if (t == 0) *slot = (long long)atomicAdd(A.counter, 1ull);
        group_sync(bar);
        const int64_t tile = (int64_t)*slot;  // rewritten only after the barriers below
        if (tile >= ntiles) break;
        const int ch = (int)(tile / A.W);  // chunk-major: a snapshot chunk is fetched once
        const int64_t w = tile - (int64_t)ch * A.W;
        const int64_t p0 = (int64_t)ch * A.chunk;
        const int64_t p1 = p0 + A.chunk < L ? p0 + A.chunk : L;
        if (!QCS_IN_BOUNDS(ch < A.nchunks && L >= 0 && L <= A.P, A.status)) {  // group-uniform
            group_sync(bar);  // every thread has read the slot before it is rewritten
            continue;
        }
        cd *out = A.partial + (w * A.nchunks + ch) * rec;
        cd Ssum = cmk(0.0, 0.0);
        for (int e = t; e < n * n; e += kGroup) Gs[e] = cmk(0.0, 0.0);
        if (p0 < L) {
            const cd *Utw = A.Ut + w * n * n;
            for (int e = t; e < n * n; e += kGroup) Uts[(e / n) * lu + (e % n)] = Utw[e];
            for (int64_t pq = p0; pq < p1; ++pq) {
                const int64_t q = A.all ? pq : (int64_t)A.idx[pq];
                if (!QCS_IN_BOUNDS(q >= 0 && q < A.P, A.status)) continue;  // group-uniform
                const uint8_t *gq = A.gth ? A.gth + q * n2 : nullptr;
                const bool sp = gq && gq[0] != 0xFF;  // signed permutation: gathers instead of products
                group_sync(bar);
                if (sp) {
                    // column k of Qt has exactly two nonzeros, in rows kc[2k] < kc[2k+1]
                    for (int c = t; c < n2; c += kGroup) {
                        const int k = gq[c] >> 2;
                        int slot = 0;
                        for (int c2 = 0; c2 < c; ++c2) slot += ((gq[c2] >> 2) == k) ? 1 : 0;
                        kc[2 * k + slot] = (uint8_t)c;
                    }
                } else {
                    load_Qt(n, A.Qh + q * n2 * n, Qs, t, kGroup);  // [H1^T; G2^T]: K = Ut Qh^T in T's place
                    // re + im (for build_T_reg and B) and re - im (for B's conjugate products) of
                    // the walker rows, in the node region (free here)
                    for (int e = t; e < n * n; e += kGroup) {
                        const int j = e / n, k = e - j * n;
                        const cd u = Uts[j * lu + k];
                        Uss[j * lu + k] = u.x + u.y;
                        Usd[j * lu + k] = u.x - u.y;
                    }
                }
                group_sync(bar);
                if (sp) build_T_gather(n, Uts, gq, Ts, t, kGroup);
                else if (n == 16)  // lane = column of T, the two warps take alternate rows
                    build_T_reg<16>(ne, Uts, Uss, Qs, Ts, t & 31, false, lq, t >> 5, kGroup / 32);
                else build_T_echelon(n, ne, Uts, Qs, Ts, t, kGroup);  // walker rows in echelon form
                group_sync(bar);
                if (sp) {
                    build_B(n, ne, Ts, Bs, tab, t, kGroup);
                } else {
                    for (int e = t; e < n * n2; e += kGroup) {  // Qh is no longer needed
                        const int j = e / n2, c = e - j * n2;
                        const cd k = Ts[j * lt + c];
                        Ksum[e] = k.x + k.y;
                        if (j >= ne) Kdif[e - ne * n2] = k.x - k.y;
                    }
                    group_sync(bar);
                    build_B_from_K3(n, ne, Uts, Uss, Usd, Ts, Ksum, Bs, tab, t, kGroup);
                }
                group_sync(bar);
                cd S = cmk(0.0, 0.0);
                // Y = (1/2) sum_k gamma_k pf_k A_k^{-1}: block form when the occupied block
                // eliminates stably (shared_factor), else every node matrix in full
                if (shared_factor(m, ne, Bs, Ys, g1v, g2v, sinvh, sacth, skh, sph, scr, tab, t, bar)) {
                    const int md = m - ne, Tn = tri_count(md);
                    const cd pf0 = scr->pf0;
                    for (int e = t; e < Tn; e += kGroup) {  // S0 to Bs; Zc accumulates in its place
                        int a, b;
                        pair_of(tab, e, a, b);
                        cd *y = Ys + tri_index(ne + a, ne + b);
                        Bs[e] = *y;
                        *y = cmk(0.0, 0.0);
                    }
                    group_sync(bar);
                    cd csum = cmk(0.0, 0.0);
                    for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                        const int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                        node_factor(md, 0, A.wnode + k0, nb, Bs, Ns, g1v, g2v, pf, invh, pos, acth, kh, ph, tab, t,
                                    bar, A.status);
                        node_inverse(md, nb, Ns, g1v, g2v, y1v, y2v, invh, acth, kh, ph, t, bar);
                        if (t < nb) cf[t] = cscale(cmul(A.gamma[k0 + t], cmul(pf0, pf[t])), 0.5);
                        if (t == 0)
                            for (int v = 0; v < nb; ++v) cfma(S, A.gamma[k0 + v], cmul(pf0, pf[v]));
                        group_sync(bar);
                        for (int v = 0; v < nb; ++v) csum = cadd(csum, cf[v]);
                        for (int e = t; e < Tn; e += kGroup) {
                            int a, b;
                            pair_of(tab, e, a, b);
                            cd *yp = Ys + tri_index(ne + a, ne + b);
                            cd y = *yp;
                            for (int v = 0; v < nb; ++v) cfma(y, cf[v], Ns[v * Tn + e]);
                            *yp = y;
                        }
                        group_sync(bar);
                    }
                    shared_inverse(m, ne, Ys, g1v, g2v, y1v, y2v, sinvh, sacth, skh, sph, csum, scr, t, bar);
                } else {
                    for (int e = t; e < T; e += kGroup) Ys[e] = cmk(0.0, 0.0);
                    group_sync(bar);
                    for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                        const int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                        node_factor(m, ne, A.wnode + k0, nb, Bs, Ns, g1v, g2v, pf, invh, pos, acth, kh, ph, tab, t,
                                    bar, A.status);
                        node_inverse(m, nb, Ns, g1v, g2v, y1v, y2v, invh, acth, kh, ph, t, bar);
                        if (t < nb) cf[t] = cscale(cmul(A.gamma[k0 + t], pf[t]), 0.5);
                        if (t == 0)
                            for (int v = 0; v < nb; ++v) cfma(S, A.gamma[k0 + v], pf[v]);
                        group_sync(bar);
                        for (int e = t; e < T; e += kGroup) {
                            cd y = Ys[e];
                            for (int v = 0; v < nb; ++v) cfma(y, cf[v], Ns[v * T + e]);
                            Ys[e] = y;
                        }
                        group_sync(bar);
                    }
                }
                if (t == 0) {
                    if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                    Ssum = cadd(Ssum, S);
                }
                // Cotangents: Gamma1 (rows < ne) += G_X[occ] Qt and Gamma2 (rows >= ne) += Ht conj(Qt),
                // G_X / 2 = Y (X J) and Ht_i = G[ne+2i] - i G[ne+2i+1] = Yh_i (X J), where
                // Yh_i = Y[ne+2i] - i Y[ne+2i+1] (G_X is linear in Y's rows).
                if (sp) {
                    // signed permutation: G_X on the occupied rows and Ht, then gathers of Qt
                    cd *Yh = GX + n * n2;  // d x m, after G_X's n x 2n entries
                    for (int e = t; e < A.d * m; e += kGroup) {
                        const int i = e / m, b = e - i * m;
                        const cd y0 = skew_at(Ys, ne + 2 * i, b), y1 = skew_at(Ys, ne + 2 * i + 1, b);
                        Yh[e] = cmk(y0.x + y1.y, y0.y - y1.x);
                    }
                    group_sync(bar);
                    // (XJ)[b][2k] = -X[b][2k+1], (XJ)[b][2k+1] = X[b][2k]; row ne + i of GX is Ht_i
                    for (int e = t; e < n * n2; e += kGroup) {
                        const int a = e / n2, c = e - a * n2;
                        const int cx = c ^ 1;
                        const bool occ = a < ne;
                        const cd *yh = Yh + (occ ? 0 : (a - ne) * m);
                        cd acc = cmk(0.0, 0.0);
                        for (int b = 0; b < ne; ++b) cfma(acc, occ ? skew_at(Ys, a, b) : yh[b], Ts[b * lt + cx]);
                        for (int r = 0; r < m - ne; ++r) {
                            const cd tt = Ts[(ne + (r >> 1)) * lt + cx];
                            crfma(acc, occ ? skew_at(Ys, a, ne + r) : yh[ne + r], (r & 1) ? -tt.y : tt.x);
                        }
                        GX[e] = flip_if(acc, !(c & 1));
                    }
                    group_sync(bar);
                    for (int e = t; e < n * n; e += kGroup) {
                        const int j = e / n, k = e - j * n;
                        const cd *g = GX + j * n2;
                        cd acc = Gs[e];
                        for (int h = 0; h < 2; ++h) {
                            const int c = kc[2 * k + h];
                            const unsigned ph = gq[c] & 3u;
                            acc = cadd(acc, mul_phase(g[c], j < ne ? ph : ((4u - ph) & 3u)));
                        }
                        Gs[e] = acc;
                    }
                } else {
                    // dense: X J Qt and X J conj(Qt) are rows of K = [Ut H1 | Ut G2]: occupied row b
                    // gives K1_b and K2_b; the empty rows R_j, I_j give (K1_j + conj K2_j)/2,
                    // i (K1_j - conj K2_j)/2 and their conjugates.  So with the source row y (Y[r]
                    // for r < ne, Yh_{r-ne} else) and c_j = (y[R_j] + i y[I_j])/2,
                    // c'_j = (y[R_j] - i y[I_j])/2,
                    //     Gamma1[r] += sum_b y[b] K1_b + sum_j (c_j K1_j + c'_j conj K2_j)
                    //     Gamma2[r] += sum_b y[b] K2_b + sum_j (c_j K2_j + c'_j conj K1_j)
                    // (n x m coefficients Cf and their sums re + im in the node region, then n x n
                    // entries of m terms, three real products each: with the sums of K's entries
                    // (re - im for the conjugated ones), Re = p1 - p2 and Im = p3 - p1 - p2).
                    cd *Cf = Ns;
                    double *Cs = reinterpret_cast<double *>(Ns + n * m);
                    for (int e = t; e < n * m; e += kGroup) {
                        const int r = e / m, b = e - r * m;
                        const bool occ = r < ne;
                        const int r0 = occ ? r : ne + 2 * (r - ne), r1 = occ ? r : r0 + 1;
                        const bool pair = b >= ne;
                        const int b0 = pair ? ne + ((b - ne) & ~1) : b;
                        // y at columns b0 and bi = b0 + 1 (the second only for an empty pair)
                        const int bi = pair ? b0 + 1 : b0;
                        cd y0 = skew_at(Ys, r0, b0), y1 = skew_at(Ys, r1, b0);
                        const cd yb = occ ? y0 : cmk(y0.x + y1.y, y0.y - y1.x);
                        y0 = skew_at(Ys, r0, bi);
                        y1 = skew_at(Ys, r1, bi);
                        const cd yi = occ ? y0 : cmk(y0.x + y1.y, y0.y - y1.x);
                        // c = (yb + i yi) / 2 at even offsets, c' = (yb - i yi) / 2 at odd ones
                        const bool odd = (b - ne) & 1;
                        const cd iy = flip_if(cmk(-yi.y, yi.x), odd);
                        const cd c = pair ? cmk(0.5 * (yb.x + iy.x), 0.5 * (yb.y + iy.y)) : yb;
                        Cf[e] = c;
                        Cs[e] = c.x + c.y;
                    }
                    group_sync(bar);
                    for (int e = t; e < n * n; e += kGroup) {
                        const int r = e / n, k = e - r * n;
                        const int o1 = r < ne ? 0 : n, o2 = n - o1;
                        const cd *cf = Cf + r * m;
                        const double *cs = Cs + r * m;
                        double p1 = 0.0, p2 = 0.0, p3 = 0.0;
                        for (int b = 0; b < ne; ++b) {
                            const cd c = cf[b], v = Ts[b * lt + o1 + k];
                            p1 = fma(c.x, v.x, p1);
                            p2 = fma(c.y, v.y, p2);
                            p3 = fma(cs[b], Ksum[b * n2 + o1 + k], p3);
                        }
                        for (int j = 0; j < A.d; ++j) {
                            const cd *kr = Ts + (ne + j) * lt;
                            const cd c = cf[ne + 2 * j], v = kr[o1 + k];
                            p1 = fma(c.x, v.x, p1);
                            p2 = fma(c.y, v.y, p2);
                            p3 = fma(cs[ne + 2 * j], Ksum[(ne + j) * n2 + o1 + k], p3);
                            const cd c2 = cf[ne + 2 * j + 1], w = kr[o2 + k];  // c2 conj(w)
                            p1 = fma(c2.x, w.x, p1);
                            p2 = fma(-c2.y, w.y, p2);
                            p3 = fma(cs[ne + 2 * j + 1], Kdif[j * n2 + o2 + k], p3);
                        }
                        const cd acc = Gs[e];
                        Gs[e] = cmk(acc.x + (p1 - p2), acc.y + (p3 - p1 - p2));
                    }
                }
            }
        }
        group_sync(bar);
        for (int e = t; e < n * n; e += kGroup) out[1 + e] = Gs[e];
        if (t == 0) out[0] = Ssum;
    }
}

// Per walker: sum the tile records in order, then
//   O = c0 det(R) S / P,   g^T = (c0/P) adj(R) [S U_occ^dagger + Lambda (I - U_occ U_occ^dagger)],
//   Lambda = sqrt2 Gacc1 - U_occ^dagger Gacc2^T U^dagger
// where Gacc1 = Gamma1 / 2 and Gacc2 = Gamma2 as accumulated by grad_pair_kernel.
__global__ void grad_epilogue_kernel(int n, int ne, int64_t W, int64_t P, int nchunks, const cd *__restrict__ partial,
                                     const cd *__restrict__ U, const cd *__restrict__ R,
                                     const cd *__restrict__ Wrot, cd *__restrict__ overlap,
                                     cd *__restrict__ grad, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int nn = n * n;
    cd *G = reinterpret_cast<cd *>(smem_raw) + (size_t)warp * (4 * nn + 2 * ne * n + 2 * ne * ne + 2);
    cd *Us = G + nn;           // U (n x n)
    cd *V1 = Us + nn;          // Gamma2^T U^dagger (n x n)
    cd *Lm = V1 + nn;          // Lambda (ne x n)
    cd *Mm = Lm + ne * n;      // S U_occ^dagger + Lambda'  (ne x n)
    cd *Rs = Mm + ne * n;      // R (ne x ne)
    cd *Ad = Rs + ne * ne;     // adj(R)
    cd *Sv = Ad + ne * ne;     // S
    const double sq2 = 1.41421356237309504880;
    const size_t rec = 1 + (size_t)nn;
    for (int64_t w = (int64_t)blockIdx.x * wpb + warp; w < W; w += (int64_t)gridDim.x * wpb) {
        cd s = cmk(0.0, 0.0);
        for (int e = lane; e < nn; e += 32) {
            cd acc = cmk(0.0, 0.0);
            for (int c = 0; c < nchunks; ++c) acc = cadd(acc, partial[(w * nchunks + c) * rec + 1 + e]);
            G[e] = acc;
            Us[e] = U[w * nn + e];
        }
        if (lane == 0) {
            for (int c = 0; c < nchunks; ++c) s = cadd(s, partial[(w * nchunks + c) * rec]);
            Sv[0] = s;
        }
        for (int e = lane; e < ne * ne; e += 32) Rs[e] = R[w * ne * ne + e];
        __syncwarp();
        // V1[k][l] = sum_{j >= ne} Gacc[j][k] conj(U[l][j])
        for (int e = lane; e < nn; e += 32) {
            int k = e / n, l = e - k * n;
            cd acc = cmk(0.0, 0.0);
            for (int j = ne; j < n; ++j) cfma(acc, G[j * n + k], cconj(Us[l * n + j]));
            V1[e] = acc;
        }
        __syncwarp();
        // Lambda[a][l] = sqrt2 Gacc[a][l] - sum_k conj(U[k][a]) V1[k][l]
        for (int e = lane; e < ne * n; e += 32) {
            int a = e / n, l = e - a * n;
            cd acc = cscale(G[a * n + l], sq2);
            for (int k = 0; k < n; ++k) cfms(acc, cconj(Us[k * n + a]), V1[k * n + l]);
            Lm[e] = acc;
        }
        __syncwarp();
        // (Lambda U_occ)[a][b] -> V1 (reused), then Mm = S U_occ^dagger + Lambda - (Lambda U_occ) U_occ^dagger
        for (int e = lane; e < ne * ne; e += 32) {
            int a = e / ne, b = e - a * ne;
            cd acc = cmk(0.0, 0.0);
            for (int k = 0; k < n; ++k) cfma(acc, Lm[a * n + k], Us[k * n + b]);
            V1[e] = acc;
        }
        __syncwarp();
        const cd S = Sv[0];
        for (int e = lane; e < ne * n; e += 32) {
            int a = e / n, l = e - a * n;
            cd acc = cadd(Lm[e], cmul(S, cconj(Us[l * n + a])));
            for (int b = 0; b < ne; ++b) cfms(acc, V1[a * ne + b], cconj(Us[l * n + b]));
            Mm[e] = acc;
        }
        // adj(R) of the upper-triangular R without divisions:
        //   N_jj = 1, N_ij = -sum_{k=i+1..j} R_ik D(i+1..k-1) N_kj,  adj_ij = D(0..i-1) D(j+1..ne-1) N_ij
        // with D(a..b) the product of the diagonal entries; one lane per column j.
        if (lane < ne) {
            const int j = lane;
            cd Ncol[QCS_MAX_N];
            for (int i = 0; i < ne; ++i) Ncol[i] = cmk(0.0, 0.0);
            Ncol[j] = cmk(1.0, 0.0);
            for (int i = j - 1; i >= 0; --i) {
                cd acc = cmk(0.0, 0.0), Dp = cmk(1.0, 0.0);
                for (int k = i + 1; k <= j; ++k) {
                    cfma(acc, cmul(Rs[i * ne + k], Dp), Ncol[k]);
                    Dp = cmul(Dp, Rs[k * ne + k]);
                }
                Ncol[i] = flip_if(acc, true);
            }
            cd post = cmk(1.0, 0.0);
            for (int k = j + 1; k < ne; ++k) post = cmul(post, Rs[k * ne + k]);
            cd pre = cmk(1.0, 0.0);
            for (int i = 0; i < ne; ++i) {
                Ad[i * ne + j] = (i <= j) ? cmul(cmul(pre, post), Ncol[i]) : cmk(0.0, 0.0);
                pre = cmul(pre, Rs[i * ne + i]);
            }
        }
        __syncwarp();
        cd ip;
        switch ((ne / 2) & 3) {
            case 0: ip = cmk(1, 0); break;
            case 1: ip = cmk(0, 1); break;
            case 2: ip = cmk(-1, 0); break;
            default: ip = cmk(0, -1); break;
        }
        const double invP = P > 0 ? 1.0 / (double)P : 0.0;
        const cd c0 = cscale(ip, 2.0 * ldexp(1.0, -(n - ne / 2)) * invP);
        // The kernel's rows are those of U_occ = U_qr W (echelon form), so the factor is
        // W^H R: adj(W^H R) = adj(R) det(conj W) W, with det(conj W) W stored in Wrot.
        const cd *Ww = Wrot + w * ((size_t)ne * ne + 1);
        cd *Ad2 = V1;  // free again
        for (int e = lane; e < ne * ne; e += 32) {
            const int a = e / ne, b = e - a * ne;
            cd acc = cmk(0.0, 0.0);
            for (int c = a; c < ne; ++c) cfma(acc, Ad[a * ne + c], Ww[c * ne + b]);
            Ad2[e] = acc;
        }
        __syncwarp();
        // grad[w][l][a] = (g^T)[a][l] = c0 sum_b adj(W^H R)[a][b] Mm[b][l]
        for (int e = lane; e < n * ne; e += 32) {
            int l = e / ne, a = e - l * ne;
            cd acc = cmk(0.0, 0.0);
            for (int b = 0; b < ne; ++b) cfma(acc, Ad2[a * ne + b], Mm[b * n + l]);
            acc = cmul(c0, acc);
            if (!cfinite(acc)) raise_status(status, QCS_ERR_NONFINITE);
            grad[w * n * ne + e] = acc;
        }
        if (lane == 0) {
            cd detR = cmk(1.0, 0.0);  // det(W^H R) = det(conj W) det R
            for (int i = 0; i < ne; ++i) detR = cmul(detR, Rs[i * ne + i]);
            overlap[w] = cmul(c0, cscale(cmul(detR, S), Ww[ne * ne].x));
        }
        __syncwarp();
    }
}

// xbar[w][g] = -sqrt_dt * i * sum_pq L[g][p][q] (Phi g^T)[q][p] / O   (sqrt_dt = 0: <v_gamma>)
__global__ void force_bias_kernel(int n, int ne, int64_t W, int nchol, const cd *__restrict__ L,
                                  const cd *__restrict__ Phi, const cd *__restrict__ ov, const cd *__restrict__ grad,
                                  double sqrt_dt, cd *__restrict__ xbar) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cd *Gf = reinterpret_cast<cd *>(smem_raw);  // Phi g^T (n x n)
    for (int64_t w = blockIdx.x; w < W; w += gridDim.x) {
        const cd *Pw = Phi + w * n * ne, *gw = grad + w * n * ne;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int q = e / n, p = e - q * n;
            cd acc = cmk(0.0, 0.0);
            for (int j = 0; j < ne; ++j) cfma(acc, Pw[q * ne + j], gw[p * ne + j]);
            Gf[e] = acc;  // (Phi g^T)[q][p]
        }
        __syncthreads();
        const cd io = cinv(ov[w]);
        for (int g = threadIdx.x; g < nchol; g += blockDim.x) {
            const cd *Lg = L + (size_t)g * n * n;
            cd acc = cmk(0.0, 0.0);
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) cfma(acc, Lg[p * n + q], Gf[q * n + p]);
            acc = cmul(acc, io);
            cd v = cmk(-acc.y, acc.x);  // i * tr(L G)
            xbar[w * nchol + g] = (sqrt_dt != 0.0) ? cscale(v, -sqrt_dt) : v;
        }
        __syncthreads();
    }
}

size_t grad_group_layout(GradArgs &A) {
    const int n = A.n, m = A.m, T = tri_count(m), NB = A.NB, S = m / 2;
    size_t o = align16((size_t)n * ld_ut(n) * sizeof(cd));
    A.off_Q = (int)o;
    o = align16(o + (size_t)2 * n * ld_qt(n) * sizeof(cd));
    A.off_T = (int)o;
    o = align16(o + (size_t)n * ld_t(n) * sizeof(cd));
    A.off_B = (int)o;
    o = align16(o + (size_t)T * sizeof(cd));
    A.off_Y = (int)o;
    o = align16(o + (size_t)T * sizeof(cd));
    A.off_G = (int)o;
    o = align16(o + (size_t)n * n * sizeof(cd));
    A.off_NZ = (int)o;
    size_t nz = (size_t)NB * T;
    if ((size_t)m * 2 * n > nz) nz = (size_t)m * 2 * n;
    o = align16(o + nz * sizeof(cd));
    A.off_g1 = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_g2 = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_y1 = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_y2 = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_pf = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    A.off_cf = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    A.off_invh = (int)o;
    o = align16(o + (size_t)NB * S * sizeof(cd));
    A.off_int = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(int));
    A.off_tile = (int)o;
    o = align16(o + sizeof(long long));
    A.off_acth = (int)o;
    o = align16(o + (size_t)NB * (S + 1) * m);
    A.off_kh = (int)o;
    o = align16(o + (size_t)NB * S);
    A.off_ph = (int)o;
    o = align16(o + (size_t)NB * S);
    A.off_kc = (int)o;
    o = align16(o + (size_t)2 * n);
    A.off_sacth = (int)o;
    o = align16(o + (size_t)(A.ne / 2 + 1) * m);
    A.off_skh = (int)o;
    o = align16(o + (size_t)A.ne / 2);
    A.off_sph = (int)o;
    o = align16(o + (size_t)A.ne / 2);
    A.off_sinvh = (int)o;
    o = align16(o + (size_t)(A.ne / 2) * sizeof(cd));
    A.off_scr = (int)o;
    o = align16(o + sizeof(SharedScratch));
    return o;
}

}  // namespace

qcs_status qcs_launch_grad(qcs_ctx *ctx, const qcs_grad_launch &L, cudaStream_t st) {
    GradArgs A;
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
    A.tab_bytes = (int)align16((size_t)tri_count(A.m) * sizeof(uint16_t));
    A.Ut = L.Ut;
    A.Qt = L.s->Qt;
    A.Qh = L.s->Qh;
    A.gth = L.s->gth;
    A.idx = L.s->idx;
    A.d_count = L.s->d_count;
    A.partial = L.partial;
    A.counter = L.counter;
    A.status = ctx->d_status;
    for (int k = 0; k < L.plan.nev; ++k) {
        A.wnode[k] = L.plan.wnode[k];
        A.gamma[k] = L.plan.gamma[k];
    }
    // Node matrices per round (NB) and groups per block: the most resident groups
    // (at most 4 per SM, i.e. two warps per SM sub-partition), then the largest NB.
    int best_nb = 0, best_g = 1, best_score = -1;
    const int nbmax = L.plan.nev < kMaxNBG ? L.plan.nev : kMaxNBG;
    for (int nb = nbmax; nb >= 1; --nb) {
        A.NB = nb;
        const size_t gb = grad_group_layout(A);
        for (int g = 2; g >= 1; --g) {
            const size_t sm = (size_t)A.tab_bytes + (size_t)g * gb;
            if (sm > ctx->smem_optin) continue;
            int per_sm = (int)(ctx->smem_per_sm / (sm + 1024));
            if (per_sm > 2) per_sm = 2;
            int groups = per_sm * g;
            if (groups > 4) groups = 4;
            const int score = groups * 16 + nb;
            if (per_sm >= 1 && score > best_score) {
                best_score = score;
                best_nb = nb;
                best_g = g;
            }
        }
    }
    if (best_nb == 0) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "grad kernel: shared memory too large");
    A.NB = best_nb;
    A.group_bytes = (int)grad_group_layout(A);
    const int threads = best_g * kGroup;
    size_t smem = (size_t)A.tab_bytes + (size_t)best_g * A.group_bytes;
    if (qcs_set_smem(ctx, (const void *)grad_pair_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_pair_kernel, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t ntiles = L.W * L.nchunks;
    int64_t blocks = (int64_t)ctx->num_sms * per_sm;
    int64_t need = (ntiles + best_g - 1) / best_g;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return qcs_fail(ctx, QCS_ERR_CUDA, "grad tile counter reset");
    qcs_prof_begin(ctx, st);
    grad_pair_kernel<<<(unsigned)blocks, threads, smem, st>>>(A);
    qcs_prof_end(ctx, st);
    qcs_status r = qcs_check_launch(ctx, "grad_pair_kernel");
    if (r != QCS_OK) return r;
    const int n = L.n, ne = L.ne;
    const int ewpb = 4;
    size_t esm = (size_t)ewpb * (4 * n * n + 2 * ne * n + 2 * ne * ne + 2) * sizeof(cd);
    if (qcs_set_smem(ctx, (const void *)grad_epilogue_kernel, esm) != QCS_OK) return QCS_ERR_CUDA;
    int64_t eb = (L.W + ewpb - 1) / ewpb;
    if (eb > (int64_t)ctx->num_sms * 8) eb = (int64_t)ctx->num_sms * 8;
    grad_epilogue_kernel<<<(unsigned)eb, ewpb * 32, esm, st>>>(n, ne, L.W, L.P, L.nchunks, L.partial, L.U, L.R, L.Wrot,
                                                               L.overlap, L.grad, ctx->d_status);
    return qcs_check_launch(ctx, "grad_epilogue_kernel");
}

qcs_status qcs_launch_force_bias(qcs_ctx *ctx, int n, int ne, int64_t W, int nchol, const cd *L, const cd *walkers,
                                 const cd *overlap, const cd *grad, double sqrt_dt, cd *xbar, cudaStream_t st) {
    if (W == 0 || nchol == 0) return QCS_OK;
    size_t smem = (size_t)n * n * sizeof(cd);
    int64_t blocks = W < (int64_t)ctx->num_sms * 8 ? W : (int64_t)ctx->num_sms * 8;
    force_bias_kernel<<<(unsigned)blocks, 128, smem, st>>>(n, ne, W, nchol, L, walkers, overlap, grad, sqrt_dt, xbar);
    return qcs_check_launch(ctx, "force_bias_kernel");
}
