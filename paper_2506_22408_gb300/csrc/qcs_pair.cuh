// qcs_pair.cuh -- per-pair device building blocks shared by the overlap and
// adjoint kernels: the packed-pair table, the congruence T = Ut Qt^T and the
// selected covariance B^(s) of Eqs. (a_mat), (b_mat).
#pragma once
#include "qcs_common.cuh"

constexpr int kMaxNB = 8;  // node matrices per warp round, at most

// tab[t] = (b << 8) | a for t = b(b-1)/2 + a, a < b  (pairs in packed-upper order).
__device__ inline void build_pair_table(uint16_t *tab, int count) {
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
        int b = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
        while (b * (b - 1) / 2 > t) --b;
        while ((b + 1) * b / 2 <= t) ++b;
        int a = t - b * (b - 1) / 2;
        tab[t] = (uint16_t)((b << 8) | a);
    }
}

// Shared-memory row strides: one complex entry of padding per row keeps rows
// that different lanes read in the same step on different banks.
__host__ __device__ __forceinline__ int ld_ut(int n) { return n + 1; }   // Ut: n rows of n
__host__ __device__ __forceinline__ int ld_qt(int n) { return n + 1; }   // Qt: 2n rows of n
__host__ __device__ __forceinline__ int ld_t(int n) { return 2 * n + 1; }  // T: n rows of 2n

// T[j][c] = sum_k Ut[j][k] Qt[c][k]  (n x 2n; entries spread over the nthr
// threads that share the pair, lane = this thread's index among them)
__device__ inline void build_T(int n, const cd *__restrict__ Uts, const cd *__restrict__ Qs, cd *__restrict__ Ts,
                               int lane, int nthr = 32) {
    const int n2 = 2 * n, lu = ld_ut(n), lq = ld_qt(n), lt = ld_t(n);
    for (int e = lane; e < n * n2; e += nthr) {
        int j = e / n2, c = e - j * n2;
        const cd *ur = Uts + j * lu, *qr = Qs + c * lq;
        cd s = cmk(0.0, 0.0);
        for (int k = 0; k < n; ++k) cfma(s, ur[k], qr[k]);
        Ts[j * lt + c] = s;
    }
}

// T from walker rows in echelon form (see qcs_walker.cu): row j < ne of Ut is zero in
// columns k < j, row ne + j' zero in columns [ne, ne + j'); those products are skipped.
// With 2n = 32 every warp pass covers one row, so the loop bounds are warp-uniform.
__device__ inline void build_T_echelon(int n, int ne, const cd *__restrict__ Uts, const cd *__restrict__ Qs,
                                       cd *__restrict__ Ts, int lane, int nthr = 32) {
    const int n2 = 2 * n, lu = ld_ut(n), lq = ld_qt(n), lt = ld_t(n);
    for (int e = lane; e < n * n2; e += nthr) {
        const int j = e / n2, c = e - j * n2;
        const cd *ur = Uts + j * lu, *qr = Qs + c * lq;
        cd s = cmk(0.0, 0.0);
        if (j < ne) {
            for (int k = j; k < n; ++k) cfma(s, ur[k], qr[k]);
        } else {
            for (int k = 0; k < ne; ++k) cfma(s, ur[k], qr[k]);
            for (int k = j; k < n; ++k) cfma(s, ur[k], qr[k]);  // j = ne + j'
        }
        Ts[j * lt + c] = s;
    }
}

// T from echelon-form walker rows for n = N (2N = 32 lanes): lane c holds row c of the
// snapshot's Qt in registers and owns column c of T.  Each complex multiply-add takes
// three real products (Gauss's 3-multiplication form): with s = re + im of both
// factors, Re = sum ur qr - sum ui qi and Im = sum us qs - sum ur qr - sum ui qi, so
// the sums us of the walker rows (Uss, per block) and qs of the snapshot row (here)
// are formed once.  The skipped zeros follow build_T_echelon, or for a walker in
// reduced form (occupied rows [I; X]: row j < ne has its one entry at column j
// among the columns k < ne) that single entry and the columns k >= ne; the row loop
// is warp-uniform and enters the unrolled k sequences by a switch, so the register
// arrays are indexed by constants.
#define QCS_T3M(K)                            \
    case K: {                                 \
        const cd u_ = ur[K];                  \
        p1 = fma(u_.x, qr[K], p1);            \
        p2 = fma(u_.y, qi[K], p2);            \
        p3 = fma(us[K], qs[K], p3);           \
    }
#define QCS_T3M1(K)                           \
    case K: {                                 \
        const cd u_ = ur[K];                  \
        p1 = fma(u_.x, qr[K], p1);            \
        p2 = fma(u_.y, qi[K], p2);            \
        p3 = fma(us[K], qs[K], p3);           \
        break;                                \
    }
// Qg holds the snapshot's rows with stride ldq (global memory or staged); rows
// j0, j0 + jstep, ... of T are formed, so that several warps can share one T.
template <int N>
__device__ inline void build_T_reg(int ne, const cd *__restrict__ Uts, const double *__restrict__ Uss,
                                   const cd *__restrict__ Qg, cd *__restrict__ Ts, int lane, bool reduced,
                                   int ldq = N, int j0 = 0, int jstep = 1) {
    static_assert(N == 16, "one lane per column of T: 2N must be the warp width");
    const int lu = ld_ut(N), lt = ld_t(N);
    double qr[N], qi[N], qs[N];
    const cd *qrow = Qg + lane * ldq;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const cd q = qrow[k];
        qr[k] = q.x;
        qi[k] = q.y;
        qs[k] = q.x + q.y;
    }
    for (int j = j0; j < N; j += jstep) {
        const cd *ur = Uts + j * lu;
        const double *us = Uss + j * lu;
        double p1 = 0.0, p2 = 0.0, p3 = 0.0;
        int kstart = j;
        if (j < ne && reduced) {
            switch (j) {  // the single entry among the columns k < ne
                QCS_T3M1(0) QCS_T3M1(1) QCS_T3M1(2) QCS_T3M1(3) QCS_T3M1(4) QCS_T3M1(5) QCS_T3M1(6) QCS_T3M1(7)
                QCS_T3M1(8) QCS_T3M1(9) QCS_T3M1(10) QCS_T3M1(11) QCS_T3M1(12) QCS_T3M1(13) QCS_T3M1(14)
                QCS_T3M1(15)
                default: break;
            }
            kstart = ne;
        }
        if (j >= ne) {
            switch (ne - 1) {  // k = ne-1 down to 0
                QCS_T3M(15) QCS_T3M(14) QCS_T3M(13) QCS_T3M(12) QCS_T3M(11) QCS_T3M(10) QCS_T3M(9) QCS_T3M(8)
                QCS_T3M(7) QCS_T3M(6) QCS_T3M(5) QCS_T3M(4) QCS_T3M(3) QCS_T3M(2) QCS_T3M(1) QCS_T3M(0)
                default: break;
            }
        }
        switch (kstart) {  // k = kstart up to N-1
            QCS_T3M(0) QCS_T3M(1) QCS_T3M(2) QCS_T3M(3) QCS_T3M(4) QCS_T3M(5) QCS_T3M(6) QCS_T3M(7)
            QCS_T3M(8) QCS_T3M(9) QCS_T3M(10) QCS_T3M(11) QCS_T3M(12) QCS_T3M(13) QCS_T3M(14) QCS_T3M(15)
            default: break;
        }
        Ts[j * lt + lane] = cmk(p1 - p2, p3 - p1 - p2);
    }
}
#undef QCS_T3M
#undef QCS_T3M1

// Columns c0 .. c0+n-1 of T from n staged rows of Qt (Qs, stride ld_qt) and their
// re + im sums (qs, n x n), with three real products per complex multiply-add as in
// build_T_reg (Uss: re + im of the walker rows): Re = sum ur qr - sum ui qi,
// Im = sum us qs - sum ur qr - sum ui qi.  Walker rows in echelon form skip their zeros
// (occupied row j: columns k < j; completion row ne + j': columns ne .. ne + j' - 1);
// in reduced form (red: occupied rows [I; X] / sqrt2) an occupied row j has one entry,
// at column j, among the columns k < ne.
__device__ inline void build_T_half3(int n, int ne, bool red, const cd *__restrict__ Uts,
                                     const double *__restrict__ Uss, const cd *__restrict__ Qs,
                                     const double *__restrict__ qs, cd *__restrict__ Ts, int c0, int lane,
                                     int nthr) {
    const int lu = ld_ut(n), lq = ld_qt(n), lt = ld_t(n);
    for (int e = lane; e < n * n; e += nthr) {
        const int j = e / n, c = e - j * n;
        const cd *ur = Uts + j * lu, *qr = Qs + c * lq;
        const double *us = Uss + j * lu, *qsr = qs + c * n;
        double p1 = 0.0, p2 = 0.0, p3 = 0.0;
        int k0 = 0, k1 = 0;  // columns [k0, k1) before the tail, then [kt, n)
        int kt = j;
        if (j < ne) {
            if (red) {
                k0 = j;
                k1 = j + 1;
                kt = ne;
            }
        } else {
            k1 = ne;  // the occupied columns, then the completion's tail from j = ne + j'
        }
        for (int k = k0; k < k1; ++k) {
            const cd u = ur[k], q = qr[k];
            p1 = fma(u.x, q.x, p1);
            p2 = fma(u.y, q.y, p2);
            p3 = fma(us[k], qsr[k], p3);
        }
        for (int k = kt; k < n; ++k) {
            const cd u = ur[k], q = qr[k];
            p1 = fma(u.x, q.x, p1);
            p2 = fma(u.y, q.y, p2);
            p3 = fma(us[k], qsr[k], p3);
        }
        Ts[j * lt + c0 + c] = cmk(p1 - p2, p3 - p1 - p2);
    }
}

// x * ph for a phase code ph = 0..3 (1, i, -1, -i): a swap of the parts and sign
// flips of the bit patterns, no floating-point arithmetic.
__device__ __forceinline__ cd mul_phase(cd x, unsigned ph) {
    cd r = (ph & 1u) ? cmk(x.y, x.x) : x;
    const bool fre = ph == 1u || ph == 2u, fim = ph >= 2u;
    if (fre) r.x = __longlong_as_double(__double_as_longlong(r.x) ^ (long long)0x8000000000000000ull);
    if (fim) r.y = __longlong_as_double(__double_as_longlong(r.y) ^ (long long)0x8000000000000000ull);
    return r;
}

// Signed-permutation snapshot: row c of Qt has one nonzero entry, the phase
// code & 3 at column code >> 2, so T[j][c] = Ut[j][k_c] ph_c is a gather.
__device__ inline void build_T_gather(int n, const cd *__restrict__ Uts, const uint8_t *__restrict__ code,
                                      cd *__restrict__ Ts, int lane, int nthr = 32) {
    const int n2 = 2 * n, lu = ld_ut(n), lt = ld_t(n);
    for (int e = lane; e < n * n2; e += nthr) {
        const int j = e / n2, c = e - j * n2;
        const unsigned q = code[c];
        Ts[j * lt + c] = mul_phase(Uts[j * lu + (int)(q >> 2)], q & 3u);
    }
}

// Stage a snapshot's rows Qt (2n x n, global) into padded shared rows.
__device__ inline void load_Qt(int n, const cd *__restrict__ Qg, cd *__restrict__ Qs, int lane, int nthr = 32) {
    const int lq = ld_qt(n);
    for (int e = lane; e < 2 * n * n; e += nthr) {
        int c = e / n, k = e - c * n;
        Qs[c * lq + k] = Qg[e];
    }
}

// Stage n consecutive rows of a snapshot's Qt (n x n, global) into padded shared rows.
__device__ inline void load_Qt_rows(int n, const cd *__restrict__ Qg, cd *__restrict__ Qs, int lane, int nthr) {
    const int lq = ld_qt(n);
    for (int e = lane; e < n * n; e += nthr) {
        int c = e / n, k = e - c * n;
        Qs[c * lq + k] = Qg[e];
    }
}

// The same, also writing re + im of every staged entry to qs (n x n, row stride n).
__device__ inline void load_Qt_rows_sums(int n, const cd *__restrict__ Qg, cd *__restrict__ Qs,
                                         double *__restrict__ qs, int lane, int nthr) {
    const int lq = ld_qt(n);
    for (int e = lane; e < n * n; e += nthr) {
        const int c = e / n, k = e - c * n;
        const cd q = Qg[e];
        Qs[c * lq + k] = q;
        qs[e] = q.x + q.y;
    }
}

__device__ __forceinline__ void pair_of(const uint16_t *tab, int t, int &a, int &b) {
    unsigned v = tab[t];
    a = v & 0xff;
    b = v >> 8;
}

// B^(s) (packed upper, m x m) from T (n x 2n).
__device__ inline void build_B(int n, int ne, const cd *__restrict__ Ts, cd *__restrict__ Bs,
                               const uint16_t *__restrict__ tab, int lane, int nthr = 32) {
    const int d = n - ne, n2 = ld_t(n);
    // occupied x occupied: complex x complex
    const int c1 = tri_count(ne);
    for (int e = lane; e < c1; e += nthr) {
        int a, b;
        pair_of(tab, e, a, b);
        const cd *Ta = Ts + a * n2, *Tb = Ts + b * n2;
        cd acc = cmk(0.0, 0.0);
        for (int k = 0; k < n; ++k) {
            cfma(acc, Ta[2 * k], Tb[2 * k + 1]);
            cfms(acc, Ta[2 * k + 1], Tb[2 * k]);
        }
        Bs[tri_index(a, b)] = acc;
    }
    // occupied x empty: complex x real.  Empty row r of mode j = ne + r/2 is
    // Re T_j (r even) or -Im T_j (r odd); the sign is applied once at the end.
    const int twod = 2 * d;
    const int c2 = ne * twod;
    for (int e = lane; e < c2; e += nthr) {
        int a = e / twod, r = e - a * twod;
        int j = ne + (r >> 1);
        bool odd = r & 1;
        const cd *Ta = Ts + a * n2, *Tj = Ts + j * n2;
        cd acc = cmk(0.0, 0.0);
        for (int k = 0; k < n; ++k) {
            cd t0 = Tj[2 * k], t1 = Tj[2 * k + 1];
            double x0 = odd ? t0.y : t0.x, x1 = odd ? t1.y : t1.x;
            crfma(acc, Ta[2 * k], x1);
            crfma(acc, Ta[2 * k + 1], -x0);
        }
        Bs[tri_index(a, ne + r)] = flip_if(acc, odd);
    }
    // empty x empty: real x real
    const int c3 = tri_count(twod);
    for (int e = lane; e < c3; e += nthr) {
        int a, b;
        pair_of(tab, e, a, b);
        const cd *Ta = Ts + (ne + (a >> 1)) * n2, *Tb = Ts + (ne + (b >> 1)) * n2;
        bool oa = a & 1, ob = b & 1;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) {
            cd a0 = Ta[2 * k], a1 = Ta[2 * k + 1], b0 = Tb[2 * k], b1 = Tb[2 * k + 1];
            double xa0 = oa ? a0.y : a0.x, xa1 = oa ? a1.y : a1.x;
            double xb0 = ob ? b0.y : b0.x, xb1 = ob ? b1.y : b1.x;
            acc = fma(xa0, xb1, acc);
            acc = fma(-xa1, xb0, acc);
        }
        Bs[tri_index(ne + a, ne + b)] = cmk((oa != ob) ? -acc : acc, 0.0);
    }
}


// B^(s) (packed upper, m x m) from K = Ut [H1 | G2] (n x 2n, rows of Ks with T's stride)
// and the walker rows Ut, for a snapshot with H1 = Qt^T J Qt, G2 = Qt^T J conj(Qt) (its rows
// [H1^T; G2^T] staged in place of Qt, so that K is formed exactly like T).  With
// W1 = K1 Ut^T = T J T^T and W2 = K2 Ut^H = T J conj(T)^T and the empty rows
// R_j = Re T_j, I_j = -Im T_j of the selection,
//     occupied a < b:             W1[a][b]
//     occupied a, empty mode j:   (a, R_j) = (W1 + W2)[a][j] / 2,  (a, I_j) = i (W1 - W2)[a][j] / 2
//     empty modes j1 <= j2 (al = W1, be = W2 at [j1][j2]):
//         (R, R) = Re(al + be)/2, (R, I) = Im(be - al)/2, (I, R) = -Im(al + be)/2,
//         (I, I) = Re(be - al)/2; within one mode only (R_j, I_j) = Im(be)/2.
// Each sum runs over the non-zero columns of walker row b only: column b and [ne, n) for
// an occupied row in reduced form (red), [b, n) in echelon form, [0, ne) and [b, n) for a
// completion row b >= ne.  Three real products per complex term (Gauss's form, with the
// staged sums Ksum = re + im of K1 and re - im of K2, and Uss = re + im of Ut):
//     K1 u:       Re = p1 - p2, Im = p3 - p1 - p2,   p3 = sum (k1r + k1i)(ur + ui)
//     K2 conj(u) = conj(conj(K2) u): Re = q1 + q2, Im = q1 - q2 - q3,
//                 q3 = sum (k2r - k2i)(ur + ui)   (q1 = sum k2r ur, q2 = sum k2i ui).
// The occupied-empty and empty-empty items share their sums' shape, so they run in one loop
// ordered by completion row b (the ne occupied rows a, then the empty modes up to b):
// neighbouring lanes share their loop bounds.
__device__ inline void build_B_from_K(int n, int ne, bool red, const cd *__restrict__ Uts,
                                      const double *__restrict__ Uss, const cd *__restrict__ Ks,
                                      const double *__restrict__ Ksum,
                                      cd *__restrict__ Bs, const uint16_t *__restrict__ tab, int lane,
                                      int nthr) {
    const int d = n - ne, lu = ld_ut(n), lt = ld_t(n), n2 = 2 * n;
    const int c1 = tri_count(ne);
    for (int e = lane; e < c1; e += nthr) {  // occupied x occupied: W1 alone
        int a, b;
        pair_of(tab, e, a, b);
        const cd *kr = Ks + a * lt, *ur = Uts + b * lu;
        const double *ks = Ksum + a * n2, *us = Uss + b * lu;
        double p1 = 0.0, p2 = 0.0, p3 = 0.0;
        if (red) {
            p1 = kr[b].x * ur[b].x;
            p2 = kr[b].y * ur[b].y;
            p3 = ks[b] * us[b];
        }
        for (int k = red ? ne : b; k < n; ++k) {
            const cd kk = kr[k], u = ur[k];
            p1 = fma(kk.x, u.x, p1);
            p2 = fma(kk.y, u.y, p2);
            p3 = fma(ks[k], us[k], p3);
        }
        Bs[tri_index(a, b)] = cmk(p1 - p2, p3 - p1 - p2);
    }
    const int c2 = ne * d + tri_count(d + 1);
    for (int e = lane; e < c2; e += nthr) {
        // completion row b = ne + jj carries ne + jj + 1 items
        int jj = 0, base = 0;
        while (jj + 1 < d && base + ne + jj + 1 <= e) {
            base += ne + jj + 1;
            ++jj;
        }
        const int i = e - base, b = ne + jj;
        const bool occ = i < ne;
        const int a = i;  // K row: occupied row i (i < ne), or that of empty mode i - ne
        const cd *kr = Ks + a * lt, *ur = Uts + b * lu;
        const double *ks = Ksum + a * n2, *us = Uss + b * lu;
        double p1 = 0.0, p2 = 0.0, p3 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
        for (int k = 0; k < ne; ++k) {
            const cd u = ur[k], k1 = kr[k], k2 = kr[n + k];
            p1 = fma(k1.x, u.x, p1);
            p2 = fma(k1.y, u.y, p2);
            p3 = fma(ks[k], us[k], p3);
            q1 = fma(k2.x, u.x, q1);
            q2 = fma(k2.y, u.y, q2);
            q3 = fma(ks[n + k], us[k], q3);
        }
        for (int k = b; k < n; ++k) {
            const cd u = ur[k], k1 = kr[k], k2 = kr[n + k];
            p1 = fma(k1.x, u.x, p1);
            p2 = fma(k1.y, u.y, p2);
            p3 = fma(ks[k], us[k], p3);
            q1 = fma(k2.x, u.x, q1);
            q2 = fma(k2.y, u.y, q2);
            q3 = fma(ks[n + k], us[k], q3);
        }
        const cd w1 = cmk(p1 - p2, p3 - p1 - p2), w2 = cmk(q1 + q2, q1 - q2 - q3);
        if (occ) {
            const cd sp = cadd(w1, w2), dm = csub(w1, w2);
            Bs[tri_index(a, ne + 2 * jj)] = cscale(sp, 0.5);
            Bs[tri_index(a, ne + 2 * jj + 1)] = cmk(-0.5 * dm.y, 0.5 * dm.x);
        } else {
            const int r1 = 2 * (i - ne), r2 = 2 * jj;
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

// Records of node_pfaffians' product trees per warp for NB node matrices per round (vm:
// the entries of the kernel's Gauss-vector buffers, the full matrix or NB complements);
// the ne/2 signed pivots of the shared occupied elimination follow them.
__host__ __device__ inline int pv_records(int vm, int NB, int ne) { return vm / 2 + kMaxNB + NB * (ne / 2); }

// Elimination of the occupied block, shared by every node matrix.  The node matrices
// B + w D differ only in their empty x empty block (D pairs the empty modes), so
// eliminating the ne occupied indices first is the same for all of them:
// pf(B + w D) = pf0 pf(S + w D_ee), S the Schur complement of the occupied block.
// Pivots are taken inside the occupied block (its largest active entry, ties to the
// first pair in packed order); a pivot pair at positions ak < ap of the active list
// contributes (-1)^(ak+ap-1) A_kp, the sign of moving k and p to the front; the ne/2
// signed pivots go to pvo (their product pf0 enters each node's product tree, see
// node_pfaffians).  Works on a copy of B in Ns.  Returns false, with Bs untouched, when a
// pivot is zero or the largest entry of S exceeds 2^8 times the largest entry of B (the
// caller then eliminates each node matrix in full); on success Bs holds S, packed upper
// 2d x 2d.
__device__ inline bool schur_occupied(int m, int ne, cd *__restrict__ Bs, cd *__restrict__ Ns,
                                      cd *__restrict__ Uv, cd *__restrict__ Vv, uint8_t *__restrict__ act0,
                                      uint8_t *__restrict__ act1, const uint16_t *__restrict__ tab,
                                      cd *__restrict__ pvo, int lane) {
    const int T = tri_count(m);
    unsigned kb = 0u;
    for (int e = lane; e < T; e += 32) {
        const cd x = Bs[e];
        Ns[e] = x;
        const unsigned k = pivot_key(x);
        kb = k > kb ? k : kb;
    }
    for (int a = lane; a < m; a += 32) act0[a] = (uint8_t)a;
    kb = __reduce_max_sync(QCS_FULL, kb);
    __syncwarp();
    uint8_t *cur = act0, *nxt = act1;
    for (int s = 0, r = m; s < ne / 2; ++s, r -= 2) {
        const int ro = ne - 2 * s;  // the active occupied indices sit at positions 0 .. ro-1
        unsigned long long bk = 0ull;
        for (int t = lane; t < tri_count(ro); t += 32) {
            int a, b;
            pair_of(tab, t, a, b);
            const unsigned key = pivot_key(Ns[tri_index(cur[a], cur[b])]);
            const unsigned long long c = ((unsigned long long)key << 32) | (unsigned long long)(0xffffffffu - (unsigned)t);
            bk = c > bk ? c : bk;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(QCS_FULL, bk, o);
            bk = ob > bk ? ob : bk;
        }
        if ((bk >> 32) == 0ull) return false;  // the active occupied block is zero
        int ak, ap;
        pair_of(tab, (int)(0xffffffffu - (unsigned)(bk & 0xffffffffull)), ak, ap);
        const int k = cur[ak], p = cur[ap];
        const cd piv = Ns[tri_index(k, p)];
        if (lane == 0) pvo[s] = flip_if(piv, ((ak + ap - 1) & 1) != 0);
        if (r == 2) break;  // no empty modes: the last pivot closes the Pfaffian
        const cd iv = cinv(piv);
        const int rv = r - 2;
        for (int a2 = lane; a2 < rv; a2 += 32) {
            int a = a2;
            if (a >= ak) ++a;
            if (a >= ap) ++a;
            const int i = cur[a];
            const cd aik = skew_get(Ns, i, k);  // A_{i,k}
            const cd aip = skew_get(Ns, i, p);  // A_{i,p}
            Uv[a2] = cmul(aik, iv);
            Vv[a2] = aip;
            nxt[a2] = (uint8_t)i;
        }
        __syncwarp();
        // A_ij -= u_i v_j - v_i u_j with u = A_{.,k}/A_kp, v = A_{.,p}
        const int Tr = tri_count(rv);
        for (int t = lane; t < Tr; t += 32) {
            int a, b;
            pair_of(tab, t, a, b);
            cd *x = Ns + tri_index(nxt[a], nxt[b]);
            cd y = *x;
            cfms(y, Uv[a], Vv[b]);
            cfma(y, Vv[a], Uv[b]);
            *x = y;
        }
        __syncwarp();
        uint8_t *tt = cur;
        cur = nxt;
        nxt = tt;
    }
    // the active list is now the empty indices ne .. m-1 in order
    const int T2 = tri_count(m - ne);
    unsigned ks = 0u;
    for (int t = lane; t < T2; t += 32) {
        int a, b;
        pair_of(tab, t, a, b);
        const unsigned k = pivot_key(Ns[tri_index(ne + a, ne + b)]);
        ks = k > ks ? k : ks;
    }
    ks = __reduce_max_sync(QCS_FULL, ks);
    if (ks > kb + (8u << 20)) return false;  // keys order like |x|; +8 in the exponent field is x 2^8
    for (int t = lane; t < T2; t += 32) {
        int a, b;
        pair_of(tab, t, a, b);
        Bs[t] = Ns[tri_index(ne + a, ne + b)];
    }
    __syncwarp();
    return true;
}

// Pfaffians of nb node matrices B + wnode[v] D held in Ns (packed upper), m x m with
// ne occupied rows first, each times its node weight and the npo factors pvo (the signed
// pivots of a shared occupied elimination, or none): on return pf[v] holds
// gamma[v] prod(pvo) pf(B + wnode[v] D), those factors entering the product tree as more
// records (a tree level costs one complex product whatever its width); m = 0 gives
// gamma[v] prod(pvo).
// The warp is cut into segments of seg lanes (seg = 32 / nb rounded up to a power of
// two); segment v owns node v through each Parlett-Reid step: it finds the pivot of the
// active first row, takes the pivot's reciprocal (every lane of the segment, so no lane
// waits on a divergent branch or a shared-memory round trip) and forms the Gauss
// vectors, after which the rank-2 updates of all nodes are spread over the whole warp.
// The steps run down to four active indices, whose Pfaffian closes the product in
// three terms, a01 a23 - a02 a13 + a03 a12 (two indices: a01).
__device__ inline void node_pfaffians(int m, int ne, const cd *__restrict__ wnode, const cd *__restrict__ gamma,
                                      int nb, const cd *__restrict__ Bs, cd *__restrict__ Ns, cd *__restrict__ Uv,
                                      cd *__restrict__ Vv, cd *__restrict__ pf, uint8_t *__restrict__ act0,
                                      uint8_t *__restrict__ act1, const uint16_t *__restrict__ tab,
                                      cd *__restrict__ pv, int npo, const cd *__restrict__ pvo, int lane) {
    // records per node in pv: the signed pivots of the (m - 4) / 2 steps, the closing
    // Pfaffian (a single record for m = 2 or 4; none for m = 0), the node weight, then
    // the npo factors pvo
    const int S0 = m == 0 ? 0 : (m >= 4 ? m / 2 - 1 : 1), S = S0 + 1 + npo;
    for (int e = lane; e < nb * npo; e += 32) {
        const int v = e / npo, i = e - v * npo;
        pv[v * S + S0 + 1 + i] = pvo[i];
    }
    if (m == 0) {
        if (lane < nb) pv[lane * S] = gamma[lane];
        __syncwarp();
    } else {
        const int d = (m - ne) / 2;
        const int T = tri_count(m);
        for (int e = lane; e < nb * T; e += 32) {
            int v = e / T, t = e - v * T;
            Ns[v * T + t] = Bs[t];
        }
        for (int e = lane; e < nb * m; e += 32) {
            int v = e / m, a = e - v * m;
            act0[v * m + a] = (uint8_t)a;
        }
        __syncwarp();
        for (int e = lane; e < nb * d; e += 32) {
            int v = e / d, i = e - v * d;
            cd *x = Ns + v * T + tri_index(ne + 2 * i, ne + 2 * i + 1);
            *x = cadd(*x, wnode[v]);
        }
        __syncwarp();
        const int seg = nb <= 1 ? 32 : nb <= 2 ? 16 : nb <= 4 ? 8 : 4;
        const int v = lane / seg, sl = lane - v * seg;
        const bool live = v < nb;
        const int vr = live ? v : 0;  // lanes past the last node read node 0 and write nothing
        const cd *__restrict__ Nv = Ns + vr * T;
        uint8_t *cur = act0, *nxt = act1;
        int s = 0;
        for (int r = m; r > 4; r -= 2, ++s) {
            // pivot: largest |A_{k,i}| over the active row of k = cur[0], each lane scanning
            // every seg-th candidate, then a shuffle reduction inside the segment; the key's
            // low bits prefer the first candidate among equal magnitudes
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
            const int a = 0xffff - (int)(bk & 0xffffull);  // 1 .. r - 1 (candidate a = 1 always exists)
            const int p = cur[vr * m + a];
            const cd piv = Nv[tri_index(k, p)];
            if (live && sl == 0) pv[v * S + s] = flip_if(piv, (a - 1) & 1);  // sign (-1)^{a-1} of the Laplace expansion
            // Gauss vectors over the remaining indices (original order kept): u = A_{i,k} / A_{k,p}
            // (A_{i,k} = -A_{k,i}) and v = A_{i,p}; the loads of a lane's first index are
            // issued before the reciprocal, whose dependent FP64 chain they do not wait for
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
                Uv[v * m + sl] = cnegmul(u0, iv);
                Vv[v * m + sl] = v0;
                nxt[v * m + sl] = (uint8_t)i0;
            }
            if (live) {
                for (int a2 = sl + seg; a2 < rv; a2 += seg) {
                    const int aa = a2 + 1 + ((a2 + 1 >= a) ? 1 : 0);
                    const int i = cur[v * m + aa];
                    Uv[v * m + a2] = cnegmul(Nv[tri_index(k, i)], iv);
                    Vv[v * m + a2] = skew_get(Nv, i, p);
                    nxt[v * m + a2] = (uint8_t)i;
                }
            }
            __syncwarp();
            // rank-2 update A_ij -= ut_i v_j - v_i ut_j on the remaining pairs of every node
            const int Tr = tri_count(rv);
            for (int e = lane; e < nb * Tr; e += 32) {
                int w = e / Tr, t = e - w * Tr;
                int ia, ib;
                pair_of(tab, t, ia, ib);
                int i = nxt[w * m + ia], j = nxt[w * m + ib];
                cd *x = Ns + w * T + tri_index(i, j);
                cd y = *x;
                const cd *U_ = Uv + w * m, *V_ = Vv + w * m;
                cfms(y, U_[ia], V_[ib]);
                cfma(y, V_[ia], U_[ib]);
                *x = y;
            }
            __syncwarp();
            uint8_t *t = cur;
            cur = nxt;
            nxt = t;
        }
        // the closing Pfaffian of the last four (or two) active indices, ascending
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
        __syncwarp();
    }
    // pf[v] = prod_s pv[v][s]: pairwise tree over the lanes; each level reads into
    // registers, then stores after a __syncwarp (S <= n + 1 - ne/2 <= 24 with the occupied
    // pivots, S <= m/2 + 1 <= 24 for a full elimination of one node: nb * half <= 96 items)
    for (int len = S; len > 1; len = (len + 1) / 2) {
        const int half = len / 2;
        cd r[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int e = lane + 32 * t;
            if (e < nb * half) {
                const int w = e / half, i = e - w * half;
                r[t] = cmul(pv[w * S + 2 * i], pv[w * S + 2 * i + 1]);
            }
        }
        cd tail = cmk(0.0, 0.0);
        if ((len & 1) && lane < nb) tail = pv[lane * S + len - 1];
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int e = lane + 32 * t;
            if (e < nb * half) {
                const int w = e / half, i = e - w * half;
                pv[w * S + i] = r[t];
            }
        }
        if ((len & 1) && lane < nb) pv[lane * S + half] = tail;
        __syncwarp();
    }
    if (lane < nb) pf[lane] = pv[lane * S];
    __syncwarp();
}

