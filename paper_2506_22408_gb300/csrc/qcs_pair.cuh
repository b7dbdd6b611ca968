// qcs_pair.cuh -- per-pair device building blocks shared by the overlap and
// adjoint kernels: the packed-pair table, the congruence T = Ut Qt^T and the
// selected covariance B^(s) of Eqs. (a_mat), (b_mat).
#pragma once
#include "qcs_common.cuh"

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

// T[j][c] = sum_k Ut[j][k] Qt[c][k]  (n x 2n; entries spread over the lanes)
__device__ inline void build_T(int n, const cd *__restrict__ Uts, const cd *__restrict__ Qs, cd *__restrict__ Ts,
                               int lane) {
    const int n2 = 2 * n, lu = ld_ut(n), lq = ld_qt(n), lt = ld_t(n);
    for (int e = lane; e < n * n2; e += 32) {
        int j = e / n2, c = e - j * n2;
        const cd *ur = Uts + j * lu, *qr = Qs + c * lq;
        cd s = cmk(0.0, 0.0);
        for (int k = 0; k < n; ++k) cfma(s, ur[k], qr[k]);
        Ts[j * lt + c] = s;
    }
}

// Stage a snapshot's rows Qt (2n x n, global) into padded shared rows.
__device__ inline void load_Qt(int n, const cd *__restrict__ Qg, cd *__restrict__ Qs, int lane) {
    const int lq = ld_qt(n);
    for (int e = lane; e < 2 * n * n; e += 32) {
        int c = e / n, k = e - c * n;
        Qs[c * lq + k] = Qg[e];
    }
}

__device__ __forceinline__ void pair_of(const uint16_t *tab, int t, int &a, int &b) {
    unsigned v = tab[t];
    a = v & 0xff;
    b = v >> 8;
}

// B^(s) (packed upper, m x m) from T (n x 2n).
__device__ inline void build_B(int n, int ne, const cd *__restrict__ Ts, cd *__restrict__ Bs,
                               const uint16_t *__restrict__ tab, int lane) {
    const int d = n - ne, n2 = ld_t(n);
    // occupied x occupied: complex x complex
    const int c1 = tri_count(ne);
    for (int e = lane; e < c1; e += 32) {
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
    for (int e = lane; e < c2; e += 32) {
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
        Bs[tri_index(a, ne + r)] = odd ? cneg(acc) : acc;
    }
    // empty x empty: real x real
    const int c3 = tri_count(twod);
    for (int e = lane; e < c3; e += 32) {
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

