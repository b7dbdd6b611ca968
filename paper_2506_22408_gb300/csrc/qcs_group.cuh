// qcs_group.cuh -- per-pair building blocks for kernels in which two warps (a group
// of 64 threads with its own named barrier) share one walker-snapshot pair: the
// forward Parlett-Reid elimination of a round of node matrices that keeps its step
// history, and the backward recursion that assembles each node matrix's inverse in
// place over its factors (used by the adjoint and the local-energy kernels).
#pragma once
#include "qcs_pair.cuh"

constexpr int kMaxNBG = 4;  // node matrices per round, at most
constexpr int kGroup = 64;  // threads (two warps) that share one pair

// Barrier of the two warps that share a pair (named barrier `id`, 64 threads).
__device__ __forceinline__ void group_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kGroup) : "memory");
}

// Skew matrix entry (i, j) from its packed upper triangle.
__device__ __forceinline__ cd skew_at(const cd *P, int i, int j) { return skew_get0(P, i, j); }

// Forward Parlett-Reid elimination of nb node matrices B + wnode D (packed upper,
// original index order) by the pair's 64 threads, keeping the step history (active
// index lists, pivot rows and columns, pivot reciprocals) for the backward inverse.
// pf[v] receives pf(B + wnode[v] D).  An exactly singular node matrix (a pivot row
// that is zero) has no inverse; it raises QCS_ERR_SINGULAR in *status, and its
// contribution pf A^{-1} is taken as zero (the callers scale the inverse by pf = 0).
__device__ inline void node_factor(int m, int ne, const cd *__restrict__ wnode, int nb, const cd *__restrict__ Bs,
                                   cd *__restrict__ Ns,
                            cd *__restrict__ Uv, cd *__restrict__ Vv, cd *__restrict__ pf, cd *__restrict__ invh,
                            int *__restrict__ pos, uint8_t *__restrict__ acth, uint8_t *__restrict__ kh,
                            uint8_t *__restrict__ ph, const uint16_t *__restrict__ tab, int t, int bar,
                            unsigned *status) {
    const int d = (m - ne) / 2, T = tri_count(m), S = m / 2;
    const int hstride = (S + 1) * m;
    const int lane = t & 31;
    for (int e = t; e < nb * T; e += kGroup) {
        int v = e / T, u = e - v * T;
        Ns[v * T + u] = Bs[u];
    }
    for (int e = t; e < nb * m; e += kGroup) {
        int v = e / m, a = e - v * m;
        acth[v * hstride + a] = (uint8_t)a;
    }
    if (t < nb) pf[t] = cmk(1.0, 0.0);
    group_sync(bar);
    for (int e = t; e < nb * d; e += kGroup) {
        int v = e / d, i = e - v * d;
        cd *x = Ns + v * T + tri_index(ne + 2 * i, ne + 2 * i + 1);
        *x = cadd(*x, wnode[v]);
    }
    group_sync(bar);
    for (int s = 0; s < S; ++s) {
        const int r = m - 2 * s;
        const uint8_t *cur = acth + s * m;
        uint8_t *nxt = acth + (s + 1) * m;
        if (t < 32) {
            // pivot: largest |A_{k,i}| over the active row of k = cur[0].  Warp 0 alone:
            // nb segments of seg lanes, a shuffle reduction inside each segment.
            const int seg = nb <= 1 ? 32 : nb <= 2 ? 16 : 8;
            const int v = lane / seg, sl = lane - v * seg;
            unsigned long long bk = 0ull;
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
            if (lane < nb) {
                if ((bk >> 32) == 0ull) raise_status(status, QCS_ERR_SINGULAR);
                const int a = 0xffff - (int)(bk & 0xffffull);
                const int k = cur[lane * hstride], p = cur[lane * hstride + a];
                const cd piv = Ns[lane * T + tri_index(k, p)];
                const cd f = cmul(pf[lane], piv);
                pf[lane] = flip_if(f, (a - 1) & 1);
                invh[lane * S + s] = cinv(piv);
                pos[lane] = a;
                kh[lane * S + s] = (uint8_t)k;
                ph[lane * S + s] = (uint8_t)p;
            }
        }
        group_sync(bar);
        const int rv = r - 2;
        for (int e = t; e < nb * rv; e += kGroup) {
            const int v = e / rv, a2 = e - v * rv;
            const int a = a2 + 1 + ((a2 + 1 >= pos[v]) ? 1 : 0);
            const int i = cur[v * hstride + a], k = kh[v * S + s], p = ph[v * S + s];
            const cd *Nv = Ns + v * T;
            Uv[v * m + a2] = cnegmul(Nv[tri_index(k, i)], invh[v * S + s]);
            Vv[v * m + a2] = skew_get(Nv, i, p);
            nxt[v * hstride + a2] = (uint8_t)i;
        }
        group_sync(bar);
        const int Tr = tri_count(rv);
        for (int e = t; e < nb * Tr; e += kGroup) {
            const int v = e / Tr, u = e - v * Tr;
            int a, b;
            pair_of(tab, u, a, b);
            const int i = nxt[v * hstride + a], j = nxt[v * hstride + b];
            cd *x = Ns + v * T + tri_index(i, j);
            cd y = *x;
            cfms(y, Uv[v * m + a], Vv[v * m + b]);
            cfma(y, Vv[v * m + a], Uv[v * m + b]);
            *x = y;
        }
        group_sync(bar);
    }
}

// Pfaffians of nb <= kMaxNBG node matrices B + wnode[v] D (packed upper in Ns, m x m with
// ne occupied rows first) by the pair's 64 threads, for callers that need no inverse:
// no step history is kept.  Node v belongs to warp v & 1, where a segment of seg lanes
// owns it through each step (pivot of the active first row, reciprocal on every lane of
// the segment, Gauss vectors); the rank-2 updates of all nodes are spread over the 64
// threads.  The steps stop at four active indices, closed by the three-term Pfaffian.
// On return pf[v] = gamma[v] pf(B + wnode[v] D) (the weight is one more factor of the
// product tree).  Workspace: Ns (nb x tri(m)), Uv and Vv (nb x m), act0 and act1
// (nb x m), pv (nb (m/2 + 1)).
__device__ inline void group_node_pfaffians(int m, int ne, const cd *__restrict__ wnode, const cd *__restrict__ gamma,
                                            int nb, const cd *__restrict__ Bs, cd *__restrict__ Ns,
                                            cd *__restrict__ Uv, cd *__restrict__ Vv, cd *__restrict__ pf,
                                            uint8_t *__restrict__ act0, uint8_t *__restrict__ act1,
                                            cd *__restrict__ pv, const uint16_t *__restrict__ tab, int t, int bar) {
    if (m == 0) {
        if (t < nb) pf[t] = gamma[t];
        group_sync(bar);
        return;
    }
    const int S = (m >= 4 ? m / 2 - 1 : 1) + 1;  // pivots, the closing Pfaffian, the weight
    const int d = (m - ne) / 2;
    const int T = tri_count(m);
    for (int e = t; e < nb * T; e += kGroup) {
        const int v = e / T, u = e - v * T;
        Ns[v * T + u] = Bs[u];
    }
    for (int e = t; e < nb * m; e += kGroup) {
        const int v = e / m, a = e - v * m;
        act0[v * m + a] = (uint8_t)a;
    }
    group_sync(bar);
    for (int e = t; e < nb * d; e += kGroup) {
        const int v = e / d, i = e - v * d;
        cd *x = Ns + v * T + tri_index(ne + 2 * i, ne + 2 * i + 1);
        *x = cadd(*x, wnode[v]);
    }
    group_sync(bar);
    const int wg = t >> 5, lane = t & 31;
    const int npw = (nb + 1) >> 1;  // nodes per warp
    const int seg = npw <= 1 ? 32 : 16;
    const int slot = lane / seg, sl = lane - slot * seg;
    const int v = 2 * slot + wg;
    const bool live = slot < npw && v < nb;
    const int vr = live ? v : 0;  // lanes without a node read node 0 and write nothing
    const cd *__restrict__ Nv = Ns + vr * T;
    uint8_t *cur = act0, *nxt = act1;
    int s = 0;
    for (int r = m; r > 4; r -= 2, ++s) {
        const int k = cur[vr * m];
        unsigned long long bk = 0ull;
        for (int a = 1 + sl; a < r; a += seg) {
            const unsigned key = pivot_key(Nv[tri_index(k, cur[vr * m + a])]);
            const unsigned long long c = ((unsigned long long)key << 32) | (unsigned long long)(0xffffu - (unsigned)a);
            bk = c > bk ? c : bk;
        }
        for (int o = seg >> 1; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(QCS_FULL, bk, o);
            bk = ob > bk ? ob : bk;
        }
        const int a = 0xffff - (int)(bk & 0xffffull);  // 1 .. r - 1
        const int p = cur[vr * m + a];
        const cd piv = Nv[tri_index(k, p)];
        if (live && sl == 0) pv[v * S + s] = flip_if(piv, (a - 1) & 1);
        const int rv = r - 2;
        const bool g0 = live && sl < rv;
        int i0 = 0;
        cd u0 = cmk(0.0, 0.0), v0 = cmk(0.0, 0.0);
        if (g0) {
            i0 = cur[v * m + sl + 1 + ((sl + 1 >= a) ? 1 : 0)];
            u0 = Nv[tri_index(k, i0)];
            v0 = skew_get(Nv, i0, p);
        }
        const cd iv = cinv(piv);
        if (g0) {
            Uv[v * m + sl] = cnegmul(u0, iv);  // A_{i,k} / A_{k,p}, A_{i,k} = -A_{k,i}
            Vv[v * m + sl] = v0;               // A_{i,p}
            nxt[v * m + sl] = (uint8_t)i0;
        }
        if (live) {
            for (int a2 = sl + seg; a2 < rv; a2 += seg) {
                const int i = cur[v * m + a2 + 1 + ((a2 + 1 >= a) ? 1 : 0)];
                Uv[v * m + a2] = cnegmul(Nv[tri_index(k, i)], iv);
                Vv[v * m + a2] = skew_get(Nv, i, p);
                nxt[v * m + a2] = (uint8_t)i;
            }
        }
        group_sync(bar);
        const int Tr = tri_count(rv);
        for (int e = t; e < nb * Tr; e += kGroup) {
            const int w = e / Tr, u = e - w * Tr;
            int ia, ib;
            pair_of(tab, u, ia, ib);
            cd *x = Ns + w * T + tri_index(nxt[w * m + ia], nxt[w * m + ib]);
            cd y = *x;
            const cd *U_ = Uv + w * m, *V_ = Vv + w * m;
            cfms(y, U_[ia], V_[ib]);
            cfma(y, V_[ia], U_[ib]);
            *x = y;
        }
        group_sync(bar);
        uint8_t *tt = cur;
        cur = nxt;
        nxt = tt;
    }
    if (live && sl == 0) {
        const uint8_t *c = cur + v * m;
        cd q;
        if (m >= 4) {
            q = cmul(Nv[tri_index(c[0], c[1])], Nv[tri_index(c[2], c[3])]);
            cfms(q, Nv[tri_index(c[0], c[2])], Nv[tri_index(c[1], c[3])]);
            cfma(q, Nv[tri_index(c[0], c[3])], Nv[tri_index(c[1], c[2])]);
        } else {
            q = Nv[tri_index(c[0], c[1])];
        }
        pv[v * S + s] = q;
        pv[v * S + s + 1] = gamma[v];
    }
    group_sync(bar);
    // pf[v] = prod of the S records of node v: pairwise tree, one item per thread
    // (nb * half <= 4 * 13 < 64)
    for (int len = S; len > 1; len = (len + 1) / 2) {
        const int half = len / 2;
        cd r = cmk(0.0, 0.0);
        const bool act = t < nb * half;
        if (act) {
            const int w = t / half, i = t - w * half;
            r = cmul(pv[w * S + 2 * i], pv[w * S + 2 * i + 1]);
        }
        cd tail = cmk(0.0, 0.0);
        if ((len & 1) && t < nb) tail = pv[t * S + len - 1];
        group_sync(bar);
        if (act) {
            const int w = t / half, i = t - w * half;
            pv[w * S + i] = r;
        }
        if ((len & 1) && t < nb) pv[t * S + half] = tail;
        group_sync(bar);
    }
    if (t < nb) pf[t] = pv[t * S];
    group_sync(bar);
}

// Backward recursion, in place: the factors of node v in Ns become the packed
// upper triangle of the inverse of node matrix v.  Step s first reads its pivot
// row and column (entries (k,i) and (i,p) for the indices i still active after
// the step), then overwrites exactly those entries, and (k,p), with entries of the
// inverse; the entries among the later indices already hold the inverse of the
// step's Schur complement Z.
__device__ inline void node_inverse(int m, int nb, cd *__restrict__ Ns, cd *__restrict__ g1v,
                             cd *__restrict__ g2v, cd *__restrict__ y1v, cd *__restrict__ y2v,
                             const cd *__restrict__ invh, const uint8_t *__restrict__ acth,
                             const uint8_t *__restrict__ kh, const uint8_t *__restrict__ ph, int t, int bar) {
    const int T = tri_count(m), S = m / 2;
    const int hstride = (S + 1) * m;
    const int lane = t & 31;
    for (int s = S - 1; s >= 0; --s) {
        const int rv = m - 2 * s - 2;
        // g1 = v/a, g2 = -u/a with u_i = A_{i,k} = -N(k,i), v_i = A_{i,p}
        for (int e = t; e < nb * rv; e += kGroup) {
            const int v = e / rv, a = e - v * rv;
            const cd *Nv = Ns + v * T;
            const int i = acth[v * hstride + (s + 1) * m + a], k = kh[v * S + s], p = ph[v * S + s];
            const cd ia = invh[v * S + s];
            const cd vi = skew_get(Nv, i, p);
            g1v[v * m + a] = cmul(vi, ia);
            g2v[v * m + a] = cmul(Nv[tri_index(k, i)], ia);
        }
        group_sync(bar);
        // y1 = Z g1 and y2 = Z g2 over the later indices: one (node, vector, row) item per thread
        const int per = 2 * rv;
        for (int e = t; e < nb * per; e += kGroup) {
            const int v = e / per, r2 = e - v * per;
            const int vec = r2 >= rv ? 1 : 0, a = r2 - vec * rv;
            const cd *Zv = Ns + v * T;
            const uint8_t *rest = acth + v * hstride + (s + 1) * m;
            const cd *g = (vec ? g2v : g1v) + v * m;
            const int i = rest[a];
            cd y = cmk(0.0, 0.0);
            for (int b = 0; b < rv; ++b) cfma(y, skew_get0(Zv, i, rest[b]), g[b]);  // Z(i,i) = 0
            (vec ? y2v : y1v)[v * m + a] = y;
        }
        group_sync(bar);
        // corner g1^T Z g2 per node (warp 0: segmented shuffle sums), then the new entries
        if (t < 32) {
            const int seg = nb <= 1 ? 32 : nb <= 2 ? 16 : 8;
            const int v = lane / seg, sl = lane - v * seg;
            cd corner = cmk(0.0, 0.0);
            if (v < nb)
                for (int a = sl; a < rv; a += seg) cfma(corner, g1v[v * m + a], y2v[v * m + a]);
            for (int o = seg >> 1; o > 0; o >>= 1) {
                corner.x += __shfl_xor_sync(QCS_FULL, corner.x, o);
                corner.y += __shfl_xor_sync(QCS_FULL, corner.y, o);
            }
            if (v < nb && sl == 0) Ns[v * T + tri_index(kh[v * S + s], ph[v * S + s])] = csub(corner, invh[v * S + s]);
        }
        for (int e = t; e < nb * rv; e += kGroup) {
            const int v = e / rv, a = e - v * rv;
            cd *Zv = Ns + v * T;
            const int i = acth[v * hstride + (s + 1) * m + a], k = kh[v * S + s], p = ph[v * S + s];
            Zv[tri_index(k, i)] = y1v[v * m + a];  // Z(k,i) = -Z(i,k) = (Z g1)_i
            const cd y2 = y2v[v * m + a];          // Z(i,p) = -y2_i
            Zv[i < p ? tri_index(i, p) : tri_index(p, i)] = flip_if(y2, i < p);
        }
        group_sync(bar);
    }
}

// ---------------------------------------------------------------------------
// Block form for the adjoint: the node matrices A_k = B + w_k D differ only in their
// empty x empty block, so with the occupied block eliminated once (Schur complement
// S0 on the empty indices) A_k = [[P, Boe], [-Boe^T, S0 + w_k D + ...]] and
//     A_k^{-1} = F(Z_k),  Z_k = (S0 + w_k D)^{-1},
// where F is the backward recursion over the occupied steps.  Every backward step is
// affine in Z (new entries -Z g1, -Z g2 and -1/a + g1^T Z g2), so a weighted sum over
// the nodes is one recursion: sum_k c_k A_k^{-1} = F_c(sum_k c_k Z_k) with the
// constant -1/a of each step scaled by c = sum_k c_k.

struct SharedScratch {  // per-group scalars exchanged between the two warps
    unsigned key[2];
    int flag, ak, ap, pad_;
    cd pf0;
};

__device__ __forceinline__ void skew_put(cd *N, int i, int j, cd x) {  // A(i, j) = x, A(j, i) = -x
    N[i < j ? tri_index(i, j) : tri_index(j, i)] = flip_if(x, i > j);
}

// Forward elimination of the ne occupied indices of Ns (a copy of B, m x m packed) by
// the pair's 64 threads; pivots: the largest entry of the active occupied block (ties
// to the first pair in packed order), a pair at list positions ak < ap contributing
// (-1)^(ak+ap-1) A_kp to pf0.  Keeps the step history (active lists acth, pivot
// indices kh/ph, pivot reciprocals invh) for shared_inverse.  Returns false (the same
// on every thread) when a pivot is zero or the complement's largest entry exceeds
// 2^8 times that of B; on success the empty x empty block of Ns holds S0 and sc->pf0
// the product of the signed pivots.
__device__ inline bool shared_factor(int m, int ne, const cd *__restrict__ Bs, cd *__restrict__ Ns,
                                     cd *__restrict__ Uv, cd *__restrict__ Vv, cd *__restrict__ invh,
                                     uint8_t *__restrict__ acth, uint8_t *__restrict__ kh, uint8_t *__restrict__ ph,
                                     SharedScratch *sc, const uint16_t *__restrict__ tab, int t, int bar) {
    const int T = tri_count(m), S = ne / 2, lane = t & 31;
    unsigned kb = 0u;
    for (int e = t; e < T; e += kGroup) {
        const cd x = Bs[e];
        Ns[e] = x;
        const unsigned k = pivot_key(x);
        kb = k > kb ? k : kb;
    }
    for (int a = t; a < m; a += kGroup) acth[a] = (uint8_t)a;
    kb = __reduce_max_sync(QCS_FULL, kb);
    if (lane == 0) sc->key[t >> 5] = kb;
    if (t == 0) {
        sc->flag = 1;
        sc->pf0 = cmk(1.0, 0.0);
    }
    group_sync(bar);
    kb = sc->key[0] > sc->key[1] ? sc->key[0] : sc->key[1];
    for (int s = 0; s < S; ++s) {
        const int r = m - 2 * s, ro = ne - 2 * s;
        const uint8_t *cur = acth + s * m;
        uint8_t *nxt = acth + (s + 1) * m;
        if (t < 32) {
            unsigned long long bk = 0ull;
            for (int u = lane; u < tri_count(ro); u += 32) {
                int a, b;
                pair_of(tab, u, a, b);
                const unsigned key = pivot_key(Ns[tri_index(cur[a], cur[b])]);
                const unsigned long long c =
                    ((unsigned long long)key << 32) | (unsigned long long)(0xffffffffu - (unsigned)u);
                bk = c > bk ? c : bk;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(QCS_FULL, bk, o);
                bk = ob > bk ? ob : bk;
            }
            if (lane == 0) {
                if ((bk >> 32) == 0ull) {
                    sc->flag = 0;
                } else {
                    int ak, ap;
                    pair_of(tab, (int)(0xffffffffu - (unsigned)(bk & 0xffffffffull)), ak, ap);
                    const int k = cur[ak], p = cur[ap];
                    const cd piv = Ns[tri_index(k, p)];
                    sc->pf0 = cmul(sc->pf0, flip_if(piv, ((ak + ap - 1) & 1) != 0));
                    invh[s] = cinv(piv);
                    kh[s] = (uint8_t)k;
                    ph[s] = (uint8_t)p;
                    sc->ak = ak;
                    sc->ap = ap;
                }
            }
        }
        group_sync(bar);
        if (!sc->flag) return false;
        const int rv = r - 2;
        if (rv == 0) break;
        const int ak = sc->ak, ap = sc->ap, k = kh[s], p = ph[s];
        const cd ia = invh[s];
        for (int a2 = t; a2 < rv; a2 += kGroup) {
            int a = a2;
            if (a >= ak) ++a;
            if (a >= ap) ++a;
            const int i = cur[a];
            Uv[a2] = cmul(skew_get(Ns, i, k), ia);  // A_{i,k} / A_{k,p}
            Vv[a2] = skew_get(Ns, i, p);            // A_{i,p}
            nxt[a2] = (uint8_t)i;
        }
        group_sync(bar);
        const int Tr = tri_count(rv);
        for (int u = t; u < Tr; u += kGroup) {
            int a, b;
            pair_of(tab, u, a, b);
            cd *x = Ns + tri_index(nxt[a], nxt[b]);
            cd y = *x;
            cfms(y, Uv[a], Vv[b]);
            cfma(y, Vv[a], Uv[b]);
            *x = y;
        }
        group_sync(bar);
    }
    // growth of the complement on the empty indices ne .. m-1
    const int T2 = tri_count(m - ne);
    unsigned ks = 0u;
    for (int u = t; u < T2; u += kGroup) {
        int a, b;
        pair_of(tab, u, a, b);
        const unsigned k = pivot_key(Ns[tri_index(ne + a, ne + b)]);
        ks = k > ks ? k : ks;
    }
    ks = __reduce_max_sync(QCS_FULL, ks);
    group_sync(bar);  // every thread has read sc->key for kb
    if (lane == 0) sc->key[t >> 5] = ks;
    group_sync(bar);
    ks = sc->key[0] > sc->key[1] ? sc->key[0] : sc->key[1];
    return ks <= kb + (8u << 20);
}

// Backward recursion over the occupied steps of shared_factor, in place on Ns, whose
// empty x empty block must hold Zc = sum_k c_k Z_k on entry; c = sum_k c_k scales
// the constant -1/a of each step.  On return Ns holds sum_k c_k A_k^{-1}.
__device__ inline void shared_inverse(int m, int ne, cd *__restrict__ Ns, cd *__restrict__ g1v,
                                      cd *__restrict__ g2v, cd *__restrict__ y1v, cd *__restrict__ y2v,
                                      const cd *__restrict__ invh, const uint8_t *__restrict__ acth,
                                      const uint8_t *__restrict__ kh, const uint8_t *__restrict__ ph, cd c,
                                      SharedScratch *sc, int t, int bar) {
    const int S = ne / 2, lane = t & 31;
    for (int s = S - 1; s >= 0; --s) {
        const int rv = m - 2 * s - 2;
        const uint8_t *rest = acth + (s + 1) * m;
        const int k = kh[s], p = ph[s];
        const cd ia = invh[s];
        // g1 = v/a, g2 = -u/a with u_i = A_{i,k}, v_i = A_{i,p}
        for (int a = t; a < rv; a += kGroup) {
            const int i = rest[a];
            g1v[a] = cmul(skew_get(Ns, i, p), ia);
            g2v[a] = cmul(skew_get(Ns, k, i), ia);
        }
        group_sync(bar);
        // y1 = Z g1 and y2 = Z g2 over the later indices: one (vector, row) item per thread
        for (int e = t; e < 2 * rv; e += kGroup) {
            const int vec = e >= rv ? 1 : 0, a = e - vec * rv;
            const cd *g = vec ? g2v : g1v;
            const int i = rest[a];
            cd y = cmk(0.0, 0.0);
            for (int b = 0; b < rv; ++b) cfma(y, skew_get0(Ns, i, rest[b]), g[b]);  // Z(i,i) = 0
            (vec ? y2v : y1v)[a] = y;
        }
        group_sync(bar);
        if (t < 32) {  // corner g1^T Z g2 - c/a
            cd corner = cmk(0.0, 0.0);
            for (int a = lane; a < rv; a += 32) cfma(corner, g1v[a], y2v[a]);
            corner.x = warp_sum(corner.x);
            corner.y = warp_sum(corner.y);
            if (lane == 0) Ns[tri_index(k, p)] = csub(corner, cmul(c, ia));
        }
        for (int a = t; a < rv; a += kGroup) {
            const int i = rest[a];
            skew_put(Ns, k, i, y1v[a]);        // A^{-1}(k, i) = (Z g1)_i
            skew_put(Ns, i, p, flip_if(y2v[a], true));  // A^{-1}(i, p) = -(Z g2)_i
        }
        group_sync(bar);
    }
    (void)sc;
}
