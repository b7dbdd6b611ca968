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
// walkers need no special case.
//
// A'_k^{-1} is recomputed per pair and node, never stored in global memory: the
// Parlett-Reid elimination (as in the overlap kernel, original index order)
// leaves its Gauss vectors in place, and a backward recursion over the
// elimination steps assembles the inverse from the 2x2 pivot blocks:
//     (A^{-1})_{rest,k} = -Z g1,  (A^{-1})_{rest,p} = -Z g2,
//     (A^{-1})_{k,p} = -1/a + g1^T Z g2,  g1 = v/a, g2 = -u/a,
// where Z is the inverse of the step's Schur complement and (u, v, a) the
// step's pivot columns and pivot.
#include "qcs_internal.h"
#include "qcs_pair.cuh"

namespace {

constexpr int kMaxNBG = 4;

struct GradArgs {
    int n, ne, m, d, nev, NB, all, chunk, nchunks;
    int64_t W, P;
    int warp_bytes, tab_bytes;
    int off_Q, off_T, off_B, off_Y, off_G, off_NZ, off_U, off_V, off_y1, off_y2, off_pf, off_inv, off_cf,
        off_best, off_int, off_acth, off_kh, off_ph;
    const cd *Ut;
    const cd *Qt;
    const int *idx;
    const int *d_count;
    cd *partial;
    unsigned long long *counter;  // tile counter: warps pull tiles dynamically
    unsigned *status;
    cd wnode[QCS_MAX_NODES];
    cd gamma[QCS_MAX_NODES];
};

// Skew matrix entry (i, j) from its packed upper triangle.
__device__ __forceinline__ cd skew_at(const cd *P, int i, int j) {
    if (i == j) return cmk(0.0, 0.0);
    int lo = i < j ? i : j, hi = i < j ? j : i;
    return flip_if(P[tri_index(lo, hi)], i > j);
}

// Forward Parlett-Reid elimination of nb node matrices with the step history
// kept for the backward inverse.  pf[v] receives pf(B + wnode[k0+v] D).
__device__ void node_factor(const GradArgs &A, int k0, int nb, const cd *__restrict__ Bs, cd *__restrict__ Ns,
                            cd *__restrict__ Uv, cd *__restrict__ Vv, cd *__restrict__ pf, cd *__restrict__ inv,
                            unsigned long long *__restrict__ best, int *__restrict__ ints, uint8_t *__restrict__ acth,
                            uint8_t *__restrict__ kh, uint8_t *__restrict__ ph, const uint16_t *__restrict__ tab,
                            int lane) {
    const int m = A.m, ne = A.ne, d = A.d, T = tri_count(m), S = m / 2;
    const int hstride = (S + 1) * m;
    int *pos = ints;
    for (int e = lane; e < nb * T; e += 32) {
        int v = e / T, t = e - v * T;
        Ns[v * T + t] = Bs[t];
    }
    for (int e = lane; e < nb * m; e += 32) {
        int v = e / m, a = e - v * m;
        acth[v * hstride + a] = (uint8_t)a;
    }
    if (lane < nb) pf[lane] = cmk(1.0, 0.0);
    __syncwarp();
    for (int e = lane; e < nb * d; e += 32) {
        int v = e / d, i = e - v * d;
        cd *x = Ns + v * T + tri_index(ne + 2 * i, ne + 2 * i + 1);
        *x = cadd(*x, A.wnode[k0 + v]);
    }
    __syncwarp();
    for (int s = 0; s < S; ++s) {
        const int r = m - 2 * s;
        const uint8_t *cur = acth + s * m;
        uint8_t *nxt = acth + (s + 1) * m;
        // pivot: largest |A_{k,i}| over the active row of k = cur[0].  Lanes form nb
        // segments of seg lanes; each lane scans every seg-th candidate, then a
        // shuffle reduction inside the segment (no atomics, no shared round trip).
        const int seg = nb <= 1 ? 32 : nb <= 2 ? 16 : nb <= 4 ? 8 : 4;
        unsigned long long bk = 0ull;
        {
            const int v = lane / seg, sl = lane - (lane / seg) * seg;
            if (v < nb) {
                const int k = cur[v * hstride];
                for (int a = 1 + sl; a < r; a += seg) {
                    const unsigned key = pivot_key(Ns[v * T + tri_index(k, cur[v * hstride + a])]);
                    const unsigned long long c =
                        ((unsigned long long)key << 32) | (unsigned long long)(0xffffu - (unsigned)a);
                    bk = c > bk ? c : bk;
                }
            }
            for (int o = seg >> 1; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(QCS_FULL, bk, o);
                bk = ob > bk ? ob : bk;
            }
            bk = __shfl_sync(QCS_FULL, bk, (lane < nb ? lane : 0) * seg);
        }
        if (lane < nb) {
            int a = 0xffff - (int)(bk & 0xffffull);
            int k = cur[lane * hstride], p = cur[lane * hstride + a];
            cd piv = Ns[lane * T + tri_index(k, p)];
            cd f = cmul(pf[lane], piv);
            pf[lane] = ((a - 1) & 1) ? cneg(f) : f;
            inv[lane] = cinv(piv);
            pos[lane] = a;
            kh[lane * S + s] = (uint8_t)k;
            ph[lane * S + s] = (uint8_t)p;
        }
        __syncwarp();
        const int rv = r - 2;
        for (int e = lane; e < nb * rv; e += 32) {
            int v = e / rv, a2 = e - v * rv;
            int a = a2 + 1 + ((a2 + 1 >= pos[v]) ? 1 : 0);
            int i = cur[v * hstride + a], k = kh[v * S + s], p = ph[v * S + s];
            const cd *Nv = Ns + v * T;
            cd u = Nv[tri_index(k, i)];
            Uv[v * m + a2] = cneg(cmul(u, inv[v]));
            Vv[v * m + a2] = (i < p) ? Nv[tri_index(i, p)] : cneg(Nv[tri_index(p, i)]);
            nxt[v * hstride + a2] = (uint8_t)i;
        }
        __syncwarp();
        const int Tr = tri_count(rv);
        for (int e = lane; e < nb * Tr; e += 32) {
            int v = e / Tr, t = e - v * Tr;
            int a, b;
            pair_of(tab, t, a, b);
            int i = nxt[v * hstride + a], j = nxt[v * hstride + b];
            cd *x = Ns + v * T + tri_index(i, j);
            cd y = *x;
            cfms(y, Uv[v * m + a], Vv[v * m + b]);
            cfma(y, Vv[v * m + a], Uv[v * m + b]);
            *x = y;
        }
        __syncwarp();
    }
}

// Backward recursion: Zs[v] (packed upper) <- inverse of node matrix v from its factors.
// Lanes are split into nb segments of 32/nb lanes; segment v serves node v.
__device__ void node_inverse(const GradArgs &A, int nb, const cd *__restrict__ Ns, cd *__restrict__ Zs,
                             cd *__restrict__ g1v, cd *__restrict__ g2v, cd *__restrict__ y1v, cd *__restrict__ y2v,
                             const uint8_t *__restrict__ acth, const uint8_t *__restrict__ kh,
                             const uint8_t *__restrict__ ph, int lane) {
    const int m = A.m, T = tri_count(m), S = m / 2;
    const int hstride = (S + 1) * m;
    const int seg = 32 / nb;  // nb in {1, 2, 4}
    const int v = lane / seg, sl = lane - v * seg;
    const bool live = v < nb;
    for (int s = S - 1; s >= 0; --s) {
        const int rv = m - 2 * s - 2;
        const cd *Nv = Ns + (live ? v : 0) * T;
        cd *Zv = Zs + (live ? v : 0) * T;
        const uint8_t *rest = acth + (live ? v : 0) * hstride + (s + 1) * m;
        const int k = kh[(live ? v : 0) * S + s], p = ph[(live ? v : 0) * S + s];
        const cd ia = cinv(Nv[tri_index(k, p)]);
        // g1 = v/a, g2 = -u/a with u_i = A_{i,k} = -N(k,i), v_i = A_{i,p}
        for (int a = sl; a < rv && live; a += seg) {
            int i = rest[a];
            cd vi = (i < p) ? Nv[tri_index(i, p)] : cneg(Nv[tri_index(p, i)]);
            g1v[v * m + a] = cmul(vi, ia);
            g2v[v * m + a] = cmul(Nv[tri_index(k, i)], ia);
        }
        __syncwarp();
        cd corner = cmk(0.0, 0.0);
        for (int a = sl; a < rv && live; a += seg) {
            int i = rest[a];
            cd y1 = cmk(0.0, 0.0), y2 = cmk(0.0, 0.0);
            for (int b = 0; b < rv; ++b) {
                int j = rest[b];
                cd z = (j == i) ? cmk(0.0, 0.0) : flip_if(Zv[tri_index(i < j ? i : j, i < j ? j : i)], j < i);
                cfma(y1, z, g1v[v * m + b]);
                cfma(y2, z, g2v[v * m + b]);
            }
            y1v[v * m + a] = y1;
            y2v[v * m + a] = y2;
            cfma(corner, g1v[v * m + a], y2);
        }
        // segmented sum of the corner term over the segment's lanes
        for (int o = seg / 2; o > 0; o >>= 1) {
            corner.x += __shfl_xor_sync(QCS_FULL, corner.x, o);
            corner.y += __shfl_xor_sync(QCS_FULL, corner.y, o);
        }
        __syncwarp();
        for (int a = sl; a < rv && live; a += seg) {
            int i = rest[a];
            Zv[tri_index(k, i)] = y1v[v * m + a];  // Z(k,i) = -Z(i,k) = (Z g1)_i
            cd y2 = y2v[v * m + a];                 // Z(i,p) = -y2_i
            if (i < p) Zv[tri_index(i, p)] = cneg(y2);
            else Zv[tri_index(p, i)] = y2;
        }
        if (live && sl == 0) Zv[tri_index(k, p)] = csub(corner, ia);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(128) grad_pair_kernel(const __grid_constant__ GradArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int n = A.n, n2 = 2 * n, ne = A.ne, m = A.m, T = tri_count(m);
    const int lu = ld_ut(n), lq = ld_qt(n), lt = ld_t(n);
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw);
    build_pair_table(tab, T);
    __syncthreads();
    unsigned char *wb = smem_raw + A.tab_bytes + (size_t)warp * A.warp_bytes;
    cd *Uts = reinterpret_cast<cd *>(wb);
    cd *Qs = reinterpret_cast<cd *>(wb + A.off_Q);
    cd *Ts = reinterpret_cast<cd *>(wb + A.off_T);
    cd *Bs = reinterpret_cast<cd *>(wb + A.off_B);
    cd *Ys = reinterpret_cast<cd *>(wb + A.off_Y);
    cd *Gs = reinterpret_cast<cd *>(wb + A.off_G);
    cd *NZ = reinterpret_cast<cd *>(wb + A.off_NZ);
    cd *Ns = NZ, *Zs = NZ + (size_t)A.NB * T, *GX = NZ;
    cd *Uv = reinterpret_cast<cd *>(wb + A.off_U);
    cd *Vv = reinterpret_cast<cd *>(wb + A.off_V);
    cd *y1v = reinterpret_cast<cd *>(wb + A.off_y1);
    cd *y2v = reinterpret_cast<cd *>(wb + A.off_y2);
    cd *pf = reinterpret_cast<cd *>(wb + A.off_pf);
    cd *inv = reinterpret_cast<cd *>(wb + A.off_inv);
    cd *cf = reinterpret_cast<cd *>(wb + A.off_cf);
    unsigned long long *best = reinterpret_cast<unsigned long long *>(wb + A.off_best);
    int *ints = reinterpret_cast<int *>(wb + A.off_int);
    uint8_t *acth = wb + A.off_acth;
    uint8_t *kh = wb + A.off_kh;
    uint8_t *ph = wb + A.off_ph;

    const int64_t L = A.all ? A.P : (int64_t)(*A.d_count);
    const int64_t ntiles = A.W * A.nchunks;
    const size_t rec = 1 + (size_t)n * n;
    (void)wpb;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(A.counter, 1ull);
        const int64_t tile = (int64_t)__shfl_sync(QCS_FULL, tk, 0);
        if (tile >= ntiles) break;
        const int ch = (int)(tile / A.W);  // chunk-major: a snapshot chunk is fetched once
        const int64_t w = tile - (int64_t)ch * A.W;
        const int64_t p0 = (int64_t)ch * A.chunk;
        const int64_t p1 = p0 + A.chunk < L ? p0 + A.chunk : L;
        cd *out = A.partial + (w * A.nchunks + ch) * rec;
        cd Ssum = cmk(0.0, 0.0);
        for (int e = lane; e < n * n; e += 32) Gs[e] = cmk(0.0, 0.0);
        if (p0 < L) {
            const cd *Utw = A.Ut + w * n * n;
            for (int e = lane; e < n * n; e += 32) Uts[(e / n) * lu + (e % n)] = Utw[e];
            for (int64_t pq = p0; pq < p1; ++pq) {
                const int64_t q = A.all ? pq : (int64_t)A.idx[pq];
                __syncwarp();
                load_Qt(n, A.Qt + q * n2 * n, Qs, lane);
                for (int e = lane; e < T; e += 32) Ys[e] = cmk(0.0, 0.0);
                __syncwarp();
                build_T(n, Uts, Qs, Ts, lane);
                __syncwarp();
                build_B(n, ne, Ts, Bs, tab, lane);
                __syncwarp();
                cd S = cmk(0.0, 0.0);
                for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                    const int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                    node_factor(A, k0, nb, Bs, Ns, Uv, Vv, pf, inv, best, ints, acth, kh, ph, tab, lane);
                    node_inverse(A, nb, Ns, Zs, Uv, Vv, y1v, y2v, acth, kh, ph, lane);
                    if (lane < nb) cf[lane] = cscale(cmul(A.gamma[k0 + lane], pf[lane]), 0.5);
                    if (lane == 0)
                        for (int v = 0; v < nb; ++v) cfma(S, A.gamma[k0 + v], pf[v]);
                    __syncwarp();
                    for (int e = lane; e < T; e += 32) {
                        cd y = Ys[e];
                        for (int v = 0; v < nb; ++v) cfma(y, cf[v], Zs[v * T + e]);
                        Ys[e] = y;
                    }
                    __syncwarp();
                }
                if (lane == 0) {
                    if (!cfinite(S)) raise_status(A.status, QCS_ERR_NONFINITE);
                    Ssum = cadd(Ssum, S);
                }
                // G_X / 2 = Y (X J): (XJ)[b][2k] = -X[b][2k+1], (XJ)[b][2k+1] = X[b][2k]
                for (int e = lane; e < m * n2; e += 32) {
                    const int a = e / n2, c = e - a * n2;
                    const int cx = c ^ 1;
                    const bool neg = !(c & 1);
                    cd acc = cmk(0.0, 0.0);
                    for (int b = 0; b < ne; ++b) cfma(acc, skew_at(Ys, a, b), Ts[b * lt + cx]);
                    for (int r = 0; r < m - ne; ++r) {
                        cd t = Ts[(ne + (r >> 1)) * lt + cx];
                        double x = (r & 1) ? -t.y : t.x;
                        crfma(acc, skew_at(Ys, a, ne + r), x);
                    }
                    GX[e] = neg ? cneg(acc) : acc;
                }
                __syncwarp();
                // empty rows: Ht_i = G[ne+2i] - i G[ne+2i+1] into row ne+2i (factor 1/2 applied at the end)
                for (int e = lane; e < A.d * n2; e += 32) {
                    const int i = e / n2, c = e - i * n2;
                    cd g0 = GX[(ne + 2 * i) * n2 + c], g1 = GX[(ne + 2 * i + 1) * n2 + c];
                    GX[(ne + 2 * i) * n2 + c] = cmk(g0.x + g1.y, g0.y - g1.x);
                }
                __syncwarp();
                // Gamma1 (rows < ne) += G[occ] Qt ; Gamma2 (rows >= ne) += Ht conj(Qt)
                for (int e = lane; e < n * n; e += 32) {
                    const int j = e / n, k = e - j * n;
                    cd acc = Gs[e];
                    if (j < ne) {
                        const cd *g = GX + j * n2;
                        for (int c = 0; c < n2; ++c) cfma(acc, g[c], Qs[c * lq + k]);
                    } else {
                        const cd *g = GX + (ne + 2 * (j - ne)) * n2;
                        for (int c = 0; c < n2; ++c) cfma(acc, g[c], cconj(Qs[c * lq + k]));
                    }
                    Gs[e] = acc;
                }
                __syncwarp();
            }
        }
        __syncwarp();
        for (int e = lane; e < n * n; e += 32) out[1 + e] = Gs[e];
        if (lane == 0) out[0] = Ssum;
    }
}

// Per walker: sum the tile records in order, then
//   O = c0 det(R) S / P,   g^T = (c0/P) adj(R) [S U_occ^dagger + Lambda (I - U_occ U_occ^dagger)],
//   Lambda = sqrt2 Gacc1 - U_occ^dagger Gacc2^T U^dagger
// where Gacc1 = Gamma1 / 2 and Gacc2 = Gamma2 as accumulated by grad_pair_kernel.
__global__ void grad_epilogue_kernel(int n, int ne, int64_t W, int64_t P, int nchunks, const cd *__restrict__ partial,
                                     const cd *__restrict__ U, const cd *__restrict__ R, cd *__restrict__ overlap,
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
    cd *LU = Sv + 1;           // (Lambda U_occ) scratch (ne x ne) stored in V1 later
    (void)LU;
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
                Ncol[i] = cneg(acc);
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
        // grad[w][l][a] = (g^T)[a][l] = c0 sum_b adj[a][b] Mm[b][l]
        for (int e = lane; e < n * ne; e += 32) {
            int l = e / ne, a = e - l * ne;
            cd acc = cmk(0.0, 0.0);
            for (int b = a; b < ne; ++b) cfma(acc, Ad[a * ne + b], Mm[b * n + l]);
            acc = cmul(c0, acc);
            if (!cfinite(acc)) raise_status(status, QCS_ERR_NONFINITE);
            grad[w * n * ne + e] = acc;
        }
        if (lane == 0) {
            cd detR = cmk(1.0, 0.0);
            for (int i = 0; i < ne; ++i) detR = cmul(detR, Rs[i * ne + i]);
            overlap[w] = cmul(c0, cmul(detR, S));
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

size_t grad_warp_layout(GradArgs &A) {
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
    size_t nz = (size_t)2 * NB * T;
    if ((size_t)m * 2 * n > nz) nz = (size_t)m * 2 * n;
    o = align16(o + nz * sizeof(cd));
    A.off_U = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_V = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_y1 = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_y2 = (int)o;
    o = align16(o + (size_t)NB * m * sizeof(cd));
    A.off_pf = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    A.off_inv = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    A.off_cf = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    A.off_best = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(unsigned long long));
    A.off_int = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(int));
    A.off_acth = (int)o;
    o = align16(o + (size_t)NB * (S + 1) * m);
    A.off_kh = (int)o;
    o = align16(o + (size_t)NB * S);
    A.off_ph = (int)o;
    o = align16(o + (size_t)NB * S);
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
    A.NB = L.plan.nev >= 2 ? 2 : 1;
    A.warp_bytes = (int)grad_warp_layout(A);
    A.tab_bytes = (int)align16((size_t)tri_count(A.m) * sizeof(uint16_t));
    A.Ut = L.Ut;
    A.Qt = L.s->Qt;
    A.idx = L.s->idx;
    A.d_count = L.s->d_count;
    A.partial = L.partial;
    A.counter = L.counter;
    A.status = ctx->d_status;
    for (int k = 0; k < L.plan.nev; ++k) {
        A.wnode[k] = L.plan.wnode[k];
        A.gamma[k] = L.plan.gamma[k];
    }
    int wpb = 4;
    while (wpb > 1 && (size_t)A.tab_bytes + (size_t)wpb * A.warp_bytes > ctx->smem_optin) --wpb;
    size_t smem = (size_t)A.tab_bytes + (size_t)wpb * A.warp_bytes;
    if (smem > ctx->smem_optin) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "grad kernel: shared memory too large");
    if (qcs_set_smem(ctx, (const void *)grad_pair_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_pair_kernel, wpb * 32, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t ntiles = L.W * L.nchunks;
    int64_t blocks = (int64_t)ctx->num_sms * per_sm;
    int64_t need = (ntiles + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return qcs_fail(ctx, QCS_ERR_CUDA, "grad tile counter reset");
    qcs_prof_begin(ctx, st);
    grad_pair_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(A);
    qcs_prof_end(ctx, st);
    qcs_status r = qcs_check_launch(ctx, "grad_pair_kernel");
    if (r != QCS_OK) return r;
    const int n = L.n, ne = L.ne;
    const int ewpb = 4;
    size_t esm = (size_t)ewpb * (4 * n * n + 2 * ne * n + 2 * ne * ne + 2) * sizeof(cd);
    if (qcs_set_smem(ctx, (const void *)grad_epilogue_kernel, esm) != QCS_OK) return QCS_ERR_CUDA;
    int64_t eb = (L.W + ewpb - 1) / ewpb;
    if (eb > (int64_t)ctx->num_sms * 8) eb = (int64_t)ctx->num_sms * 8;
    grad_epilogue_kernel<<<(unsigned)eb, ewpb * 32, esm, st>>>(n, ne, L.W, L.P, L.nchunks, L.partial, L.U, L.R,
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
