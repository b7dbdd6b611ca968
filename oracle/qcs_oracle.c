/*
 * qcs_oracle.c -- plain CPU FP64 oracle for the matchgate-shadow overlap
 * estimator of QC-AFQMC (arXiv 2506.22408), its walker gradient and the
 * AFQMC force bias.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Every step follows the paper's definitions in the paper's order, written as
 * plain dense loops (no blocking, no fusion):
 *
 *   1. C_b        = (+)_j [[0, (-1)^{b_j}], [-(-1)^{b_j}, 0]]        SI "Matrix Definitions", item 2
 *   2. G_p        = Q_p^T C_b Q_p                                     Eq. (b_mat), middle factor
 *   3. Phi = U R  (complete Householder QR), V = U^dagger             SI item 3 (walker as a_tilde^dagger product)
 *   4. M_phi      = 2x2 blocks [[Re V, -Im V], [Im V, Re V]]          SI item 3
 *   5. W          = (+)_{j<=eta} (1/sqrt2)[[1,-i],[1,i]] (+) I         SI item 1 (xi read as eta)
 *   6. B          = W^* M_phi G_p M_phi^T W^dagger                    Eq. (b_mat)
 *   7. (s)        one row per occupied mode (row 2j of the W^* block),
 *                 both rows per empty mode, ascending                  Eq. (a_mat); selection not printed in the paper
 *   8. A(z)       = C_0^(s) + z B^(s)                                 Eq. (a_mat)
 *   9. pf(A(z_k)) by Parlett-Reid elimination with partial pivoting   Sec. "Classical shadows and the evaluation of overlaps" (Wimmer 2012)
 *  10. c_x        by interpolation: the paper's Chebyshev nodes with a least-squares
 *                 Vandermonde fit, or roots of unity with an inverse DFT
 *  11. o_p        = kappa * det R * i^{eta/2} / 2^{n-eta/2} * sum_x c_x C(2n,2x)/C(n,x)
 *                 (estimator equation after the node formula; kappa = 2 restores the
 *                  1/sqrt2 of the (|0>+|Psi_T>)/sqrt2 preparation; det R restores the walker norm)
 *  12. <Psi_T|phi> = (1/P) sum_p o_p                                   same equation
 *  13. gradient   dO/dPhi_kj = O(Phi with column j replaced by e_k): O is linear in
 *                 each column of Phi (the walker is a product of one creation operator
 *                 per column), so this is the exact partial derivative
 *  14. force bias G = Phi g^T / O,  <v_gamma> = i tr(L_gamma G),  xbar = -sqrt(dtau) <v_gamma>
 *                                                                       Eqs. (force_bias), (force_bias_diff)
 *
 * Complex arrays are interleaved (re, im) doubles, i.e. C99 double complex.
 * Matrices are row-major.  Indices in this file are 0-based; the paper's mode j
 * (1-based) is j-1 here and its Majorana pair (2j-1, 2j) is (2(j-1), 2(j-1)+1).
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_MAXN 32

/* Planted-mistake switch for the test-suite's mutation checks: building with
 * -DORC_MUTATION=k plants mistake k (a dropped factor, a wrong row, a sign,
 * a transposed operand, ...) so that a test can confirm the pins catch it.
 * The default build (ORC_MUTATION undefined) contains none of them. */
#ifndef ORC_MUTATION
#define ORC_MUTATION 0
#endif
#define MUT(k) (ORC_MUTATION == (k))
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- helpers */

static double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return floor(r + 0.5);
}

/* ------------------------------------------------------- step 1: C_b (SI) */

void orc_covariance(int n, const uint8_t *b, double *C) {
    int N2 = 2 * n;
    memset(C, 0, sizeof(double) * N2 * N2);
    for (int j = 0; j < n; ++j) {
        double s = (b[j] & 1) ? -1.0 : 1.0; /* (-1)^{b_j} */
        if (MUT(3)) s = -s;
        C[(2 * j) * N2 + 2 * j + 1] = s;
        C[(2 * j + 1) * N2 + 2 * j] = -s;
    }
}

/* ------------------------------------------- step 2: G = Q^T C_b Q (b_mat) */

void orc_snapshot_G(int n, const double *Q, const uint8_t *b, double *G) {
    int N2 = 2 * n;
    double *C = malloc(sizeof(double) * N2 * N2);
    double *CQ = malloc(sizeof(double) * N2 * N2);
    orc_covariance(n, b, C);
    for (int i = 0; i < N2; ++i)
        for (int j = 0; j < N2; ++j) {
            double s = 0.0;
            for (int k = 0; k < N2; ++k) s += C[i * N2 + k] * Q[k * N2 + j];
            CQ[i * N2 + j] = s;
        }
    for (int i = 0; i < N2; ++i)
        for (int j = 0; j < N2; ++j) {
            double s = 0.0;
            for (int k = 0; k < N2; ++k) s += Q[k * N2 + i] * CQ[k * N2 + j];
            G[i * N2 + j] = s;
        }
    if (MUT(5)) /* Q C_b Q^T instead of Q^T C_b Q */
        for (int i = 0; i < N2; ++i)
            for (int j = 0; j < N2; ++j) {
                double s = 0.0;
                for (int k = 0; k < N2; ++k)
                    for (int l = 0; l < N2; ++l) s += Q[i * N2 + k] * C[k * N2 + l] * Q[j * N2 + l];
                G[i * N2 + j] = s;
            }
    free(C);
    free(CQ);
}

/* --------------------------- step 3: complete Householder QR of the walker
 * Phi (n x ne) = U[:, :ne] R with U (n x n) unitary and R (ne x ne) upper
 * triangular.  Textbook complex Householder reflections H = I - 2 v v^H / (v^H v)
 * with alpha = -e^{i arg x0} ||x|| so that H x = alpha e_1; U = H_1 H_2 ... */

void orc_walker_qr(int n, int ne, const cplx *Phi, cplx *U, cplx *R) {
    cplx *A = malloc(sizeof(cplx) * n * ne);
    cplx *v = malloc(sizeof(cplx) * n);
    memcpy(A, Phi, sizeof(cplx) * n * ne);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) U[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int k = 0; k < ne; ++k) {
        double xn2 = 0.0;
        for (int i = k; i < n; ++i) xn2 += creal(A[i * ne + k] * conj(A[i * ne + k]));
        double xn = sqrt(xn2);
        if (xn == 0.0) continue; /* zero column: H = I, R_kk = 0 */
        cplx x0 = A[k * ne + k];
        cplx ph = (cabs(x0) > 0.0) ? x0 / cabs(x0) : 1.0;
        cplx alpha = -ph * xn;
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        for (int i = k; i < n; ++i) v[i] = A[i * ne + k];
        v[k] -= alpha;
        double vn2 = 0.0;
        for (int i = k; i < n; ++i) vn2 += creal(v[i] * conj(v[i]));
        if (vn2 == 0.0) continue;
        /* A <- H A */
        for (int j = 0; j < ne; ++j) {
            cplx s = 0.0;
            for (int i = k; i < n; ++i) s += conj(v[i]) * A[i * ne + j];
            s *= 2.0 / vn2;
            for (int i = k; i < n; ++i) A[i * ne + j] -= v[i] * s;
        }
        /* U <- U H */
        for (int r = 0; r < n; ++r) {
            cplx s = 0.0;
            for (int i = k; i < n; ++i) s += U[r * n + i] * v[i];
            s *= 2.0 / vn2;
            for (int i = k; i < n; ++i) U[r * n + i] -= s * conj(v[i]);
        }
    }
    for (int i = 0; i < ne; ++i)
        for (int j = 0; j < ne; ++j) R[i * ne + j] = (j >= i) ? A[i * ne + j] : 0.0;
    free(A);
    free(v);
}

/* ------------------------------------ step 4: M_phi from V (SI item 3) */

static void walker_M(int n, const cplx *V, double *M) {
    int N2 = 2 * n;
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
            double re = creal(V[j * n + k]), im = cimag(V[j * n + k]);
            M[(2 * j) * N2 + 2 * k] = re;
            M[(2 * j) * N2 + 2 * k + 1] = -im;
            M[(2 * j + 1) * N2 + 2 * k] = im;
            M[(2 * j + 1) * N2 + 2 * k + 1] = re;
        }
}

/* --------------------------------------------- step 5: W (SI item 1) */

static void W_matrix(int n, int ne, cplx *Wm) {
    int N2 = 2 * n;
    const double r = 1.0 / sqrt(2.0);
    for (int i = 0; i < N2 * N2; ++i) Wm[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        int a = 2 * j, b = 2 * j + 1;
        if (j < ne) {
            Wm[a * N2 + a] = r;
            Wm[a * N2 + b] = -I * r;
            Wm[b * N2 + a] = r;
            Wm[b * N2 + b] = I * r;
        } else {
            Wm[a * N2 + a] = 1.0;
            Wm[b * N2 + b] = 1.0;
        }
    }
}

/* ------------------ step 6: B = W^* M G M^T W^dagger (b_mat), full 2n x 2n */

static void B_matrix(int n, int ne, const double *M, const double *G, cplx *B) {
    int N2 = 2 * n;
    double *MG = malloc(sizeof(double) * N2 * N2);
    double *S = malloc(sizeof(double) * N2 * N2);
    cplx *Wm = malloc(sizeof(cplx) * N2 * N2);
    cplx *WS = malloc(sizeof(cplx) * N2 * N2);
    for (int i = 0; i < N2; ++i)
        for (int j = 0; j < N2; ++j) {
            double s = 0.0;
            for (int k = 0; k < N2; ++k) s += M[i * N2 + k] * G[k * N2 + j];
            MG[i * N2 + j] = s;
        }
    for (int i = 0; i < N2; ++i) /* S = (M G) M^T */
        for (int j = 0; j < N2; ++j) {
            double s = 0.0;
            for (int k = 0; k < N2; ++k) s += MG[i * N2 + k] * M[j * N2 + k];
            S[i * N2 + j] = s;
        }
    W_matrix(n, ne, Wm);
    for (int i = 0; i < N2; ++i) /* W^* S */
        for (int j = 0; j < N2; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < N2; ++k) s += conj(Wm[i * N2 + k]) * S[k * N2 + j];
            WS[i * N2 + j] = s;
        }
    for (int i = 0; i < N2; ++i) /* (W^* S) W^dagger,  (W^dagger)_{kj} = conj(W_{jk}) */
        for (int j = 0; j < N2; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < N2; ++k) s += WS[i * N2 + k] * conj(Wm[j * N2 + k]);
            B[i * N2 + j] = s;
        }
    free(MG);
    free(S);
    free(Wm);
    free(WS);
}

/* ------------------------------------------------- step 7: selection (s) */

int orc_selection(int n, int ne, int *idx) {
    int m = 0;
    for (int j = 0; j < n; ++j) {
        if (j < ne) {
            idx[m++] = MUT(2) ? 2 * j : 2 * j + 1; /* the (1, -i)/sqrt2 row of the W^* block */
        } else {
            idx[m++] = 2 * j;
            idx[m++] = 2 * j + 1;
        }
    }
    return m; /* m = 2n - ne */
}

/* ---------------- step 9: Pfaffian by Parlett-Reid with partial pivoting.
 * A (m x m, complex skew-symmetric, row-major) is overwritten.  At each
 * step the pair (k, k+1) is eliminated after bringing the largest |A_ik|,
 * i > k, to row/column k+1 (a symmetric swap flips the sign of pf).  With
 * a = A_{k,k+1}, u_i = A_{i,k}, v_i = A_{i,k+1}, the Schur complement of the
 * 2x2 pivot block is A_ij - (u_i v_j - v_i u_j)/a and
 * pf(A) = a * pf(Schur complement). */

cplx orc_pfaffian_inplace(int m, cplx *A) {
    if (m == 0) return 1.0;
    if (m & 1) return 0.0;
    cplx pf = 1.0;
    for (int k = 0; k < m - 1; k += 2) {
        int p = k + 1;
        double best = cabs(A[(k + 1) * m + k]);
        for (int i = k + 2; i < m; ++i) {
            double a = cabs(A[i * m + k]);
            if (a > best) {
                best = a;
                p = i;
            }
        }
        if (p != k + 1) {
            for (int c = 0; c < m; ++c) { /* swap rows k+1, p */
                cplx t = A[(k + 1) * m + c];
                A[(k + 1) * m + c] = A[p * m + c];
                A[p * m + c] = t;
            }
            for (int r = 0; r < m; ++r) { /* swap columns k+1, p */
                cplx t = A[r * m + k + 1];
                A[r * m + k + 1] = A[r * m + p];
                A[r * m + p] = t;
            }
            if (!MUT(8)) pf = -pf;
        }
        cplx a = A[k * m + k + 1];
        if (a == 0.0) return 0.0;
        pf *= a;
        for (int i = k + 2; i < m; ++i) {
            cplx ui = A[i * m + k], vi = A[i * m + k + 1];
            for (int j = k + 2; j < m; ++j) {
                cplx uj = A[j * m + k], vj = A[j * m + k + 1];
                A[i * m + j] -= (ui * vj - vi * uj) / a;
            }
        }
    }
    return pf;
}

void orc_pfaffian(int m, const cplx *A, cplx *out) {
    cplx *W = malloc(sizeof(cplx) * (m > 0 ? m * m : 1));
    if (m > 0) memcpy(W, A, sizeof(cplx) * m * m);
    *out = orc_pfaffian_inplace(m, W);
    free(W);
}

/* ---------------- step 10: least-squares polynomial fit on real nodes.
 * Solves min || Vd c - y || for Vd_{kx} = z_k^x (N x (deg+1)), y complex,
 * by Householder QR of the real Vandermonde matrix. */

static void vandermonde_lsq(int N, int ncoef, const double *z, const cplx *y, cplx *c) {
    double *Vd = malloc(sizeof(double) * N * ncoef);
    cplx *r = malloc(sizeof(cplx) * N);
    double *v = malloc(sizeof(double) * N);
    for (int k = 0; k < N; ++k) {
        double p = 1.0;
        for (int x = 0; x < ncoef; ++x) {
            Vd[k * ncoef + x] = p;
            p *= z[k];
        }
        r[k] = y[k];
    }
    for (int j = 0; j < ncoef; ++j) {
        double xn2 = 0.0;
        for (int i = j; i < N; ++i) xn2 += Vd[i * ncoef + j] * Vd[i * ncoef + j];
        double xn = sqrt(xn2);
        if (xn == 0.0) continue;
        double alpha = (Vd[j * ncoef + j] > 0) ? -xn : xn;
        for (int i = 0; i < N; ++i) v[i] = 0.0;
        for (int i = j; i < N; ++i) v[i] = Vd[i * ncoef + j];
        v[j] -= alpha;
        double vn2 = 0.0;
        for (int i = j; i < N; ++i) vn2 += v[i] * v[i];
        for (int c2 = j; c2 < ncoef; ++c2) {
            double s = 0.0;
            for (int i = j; i < N; ++i) s += v[i] * Vd[i * ncoef + c2];
            s *= 2.0 / vn2;
            for (int i = j; i < N; ++i) Vd[i * ncoef + c2] -= s * v[i];
        }
        cplx s = 0.0;
        for (int i = j; i < N; ++i) s += v[i] * r[i];
        s *= 2.0 / vn2;
        for (int i = j; i < N; ++i) r[i] -= s * v[i];
    }
    for (int j = ncoef - 1; j >= 0; --j) { /* back substitution R c = Q^T y */
        cplx s = r[j];
        for (int x = j + 1; x < ncoef; ++x) s -= Vd[j * ncoef + x] * c[x];
        c[j] = s / Vd[j * ncoef + j];
    }
    free(Vd);
    free(r);
    free(v);
}

/* ------------------------------------------------------- per-walker state */

typedef struct {
    int n, ne;
    double *M;  /* 2n x 2n */
    cplx detR;
} walker_t;

static void walker_setup(int n, int ne, const cplx *Phi, walker_t *w) {
    cplx *U = malloc(sizeof(cplx) * n * n);
    cplx *R = malloc(sizeof(cplx) * ne * ne);
    cplx *V = malloc(sizeof(cplx) * n * n);
    orc_walker_qr(n, ne, Phi, U, R);
    for (int j = 0; j < n; ++j) /* V = U^dagger */
        for (int k = 0; k < n; ++k) V[j * n + k] = MUT(9) ? U[k * n + j] : conj(U[k * n + j]);
    w->n = n;
    w->ne = ne;
    w->M = malloc(sizeof(double) * 4 * n * n);
    walker_M(n, V, w->M);
    cplx d = 1.0;
    for (int i = 0; i < ne; ++i) d *= R[i * ne + i];
    w->detR = MUT(4) ? d / cabs(d) : d;
    free(U);
    free(R);
    free(V);
}

static void walker_free(walker_t *w) { free(w->M); }

/* Interpolation modes */
#define ORC_INTERP_ROOTS 0     /* z_k = exp(2 pi i k / N), inverse DFT */
#define ORC_INTERP_CHEBYSHEV 1 /* z_k = cos((2k+1) pi / (2N)), least squares */

/* --------------------------- steps 6-11 for one (walker, snapshot) pair.
 * coef: ell+1 polynomial coefficients c_x (may be NULL).
 * nodes: number of interpolation nodes (0 -> default: 2n+1 for roots, n for
 * Chebyshev).  Returns o_p. */

static cplx pair_estimate(const walker_t *w, const double *G, int mode, int nodes, cplx *coef,
                          double *abs_scale) {
    int n = w->n, ne = w->ne, N2 = 2 * n;
    int idx[2 * ORC_MAXN];
    int m = orc_selection(n, ne, idx);
    int ell = n - ne / 2; /* polynomial degree, ell = m/2 */
    cplx *B = malloc(sizeof(cplx) * N2 * N2);
    cplx *Bs = malloc(sizeof(cplx) * m * m);
    double *C0 = malloc(sizeof(double) * N2 * N2);
    double *C0s = malloc(sizeof(double) * m * m);
    cplx *A = malloc(sizeof(cplx) * m * m);
    uint8_t zero_bits[ORC_MAXN];
    memset(zero_bits, 0, sizeof zero_bits);
    B_matrix(n, ne, w->M, G, B);
    orc_covariance(n, zero_bits, C0); /* C_0: vacuum covariance */
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) {
            Bs[a * m + c] = B[idx[a] * N2 + idx[c]];
            C0s[a * m + c] = C0[idx[a] * N2 + idx[c]];
        }
    int N;
    if (mode == ORC_INTERP_CHEBYSHEV) N = nodes > 0 ? nodes : n;
    else N = nodes > 0 ? nodes : 2 * n + 1;
    if (N < ell + 1) N = ell + 1;
    cplx *pfv = malloc(sizeof(cplx) * N);
    double *zr = malloc(sizeof(double) * N);
    cplx *c = malloc(sizeof(cplx) * (N > ell + 1 ? N : ell + 1));
    for (int k = 0; k < N; ++k) {
        cplx z;
        if (mode == ORC_INTERP_CHEBYSHEV) {
            zr[k] = cos((2.0 * k + 1.0) * M_PI / (2.0 * N));
            z = zr[k];
        } else {
            z = cexp(2.0 * M_PI * I * (double)k / (double)N);
        }
        for (int i = 0; i < m * m; ++i) A[i] = C0s[i] + z * Bs[i]; /* Eq. (a_mat) */
        pfv[k] = orc_pfaffian_inplace(m, A);
    }
    if (mode == ORC_INTERP_CHEBYSHEV) {
        vandermonde_lsq(N, ell + 1, zr, pfv, c);
    } else {
        for (int x = 0; x < N; ++x) {
            cplx s = 0.0;
            for (int k = 0; k < N; ++k) s += pfv[k] * cexp(-2.0 * M_PI * I * (double)k * x / (double)N);
            c[x] = s / (double)N;
        }
    }
    /* step 11: o_p = kappa det R i^{eta/2} / 2^{n - eta/2} sum_x c_x C(2n,2x)/C(n,x) */
    cplx sum = 0.0;
    double asum = 0.0;
    for (int x = 0; x <= ell; ++x) {
        double wx = MUT(7) ? binom(n, x) / binom(2 * n, 2 * x) : binom(2 * n, 2 * x) / binom(n, x);
        sum += c[x] * wx;
        asum += cabs(c[x]) * wx;
    }
    cplx ipow = MUT(6) ? 1.0 : cpow(I, ne / 2);
    cplx pref = (MUT(1) ? 1.0 : 2.0) * w->detR * ipow / pow(2.0, n - ne / 2);
    if (coef)
        for (int x = 0; x <= ell; ++x) coef[x] = c[x];
    if (abs_scale) *abs_scale = cabs(pref) * asum;
    free(B);
    free(Bs);
    free(C0);
    free(C0s);
    free(A);
    free(pfv);
    free(zr);
    free(c);
    return pref * sum;
}

/* ---------------------------------------------------- exported per pair */

/* One pair.  Q: 2n x 2n, b: n bytes, Phi: n x ne.  coef: ell+1 (nullable).
 * out[0] = o_p; scale_out (nullable) = |prefactor| * sum_x |c_x| w_x, the
 * magnitude before cancellation, used to state floating-point tolerances. */
void orc_pair(int n, int ne, const double *Q, const uint8_t *b, const cplx *Phi, int mode, int nodes,
              cplx *coef, cplx *out, double *scale_out) {
    int N2 = 2 * n;
    double *G = malloc(sizeof(double) * N2 * N2);
    walker_t w;
    orc_snapshot_G(n, Q, b, G);
    walker_setup(n, ne, Phi, &w);
    *out = pair_estimate(&w, G, mode, nodes, coef, scale_out);
    walker_free(&w);
    free(G);
}

/* The selected matrices of one pair, for structural tests:
 * Bs, C0s: m x m;  detR: 1.  m = 2n - ne. */
void orc_pair_matrices(int n, int ne, const double *Q, const uint8_t *b, const cplx *Phi, cplx *Bs,
                       double *C0s, cplx *detR) {
    int N2 = 2 * n;
    int idx[2 * ORC_MAXN];
    int m = orc_selection(n, ne, idx);
    double *G = malloc(sizeof(double) * N2 * N2);
    cplx *B = malloc(sizeof(cplx) * N2 * N2);
    double *C0 = malloc(sizeof(double) * N2 * N2);
    uint8_t zero_bits[ORC_MAXN];
    memset(zero_bits, 0, sizeof zero_bits);
    walker_t w;
    orc_snapshot_G(n, Q, b, G);
    walker_setup(n, ne, Phi, &w);
    B_matrix(n, ne, w.M, G, B);
    orc_covariance(n, zero_bits, C0);
    for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) {
            Bs[a * m + c] = B[idx[a] * N2 + idx[c]];
            C0s[a * m + c] = C0[idx[a] * N2 + idx[c]];
        }
    *detR = w.detR;
    walker_free(&w);
    free(G);
    free(B);
    free(C0);
}

/* ------------------------------------------------ exported: overlaps
 * Phi: W x n x ne, Q: P x 2n x 2n, b: P x n bytes.
 * overlap: W; per_pair (nullable): W x P o_p; scale (nullable): W x P.
 * threads <= 0: OpenMP default.  Returns the thread count used. */
int orc_overlap(int n, int ne, int64_t W, int64_t P, const cplx *Phi, const double *Q, const uint8_t *b,
                int mode, int nodes, int threads, cplx *overlap, cplx *per_pair, double *scale) {
    int N2 = 2 * n;
    int used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    used = omp_get_max_threads();
#endif
    double *G = malloc(sizeof(double) * (size_t)P * N2 * N2);
    walker_t *wk = malloc(sizeof(walker_t) * (size_t)(W > 0 ? W : 1));
    cplx *op = malloc(sizeof(cplx) * (size_t)(W * P > 0 ? W * P : 1));
    double *sc = malloc(sizeof(double) * (size_t)(W * P > 0 ? W * P : 1));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) orc_snapshot_G(n, Q + p * N2 * N2, b + p * n, G + p * N2 * N2);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w = 0; w < W; ++w) walker_setup(n, ne, Phi + w * n * ne, &wk[w]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < W * P; ++e) {
        int64_t w = e / P, p = e % P;
        op[e] = pair_estimate(&wk[w], G + p * N2 * N2, mode, nodes, NULL, &sc[e]);
    }
    for (int64_t w = 0; w < W; ++w) { /* mean over snapshots, in snapshot order */
        cplx s = 0.0;
        for (int64_t p = 0; p < P; ++p) s += op[w * P + p];
        overlap[w] = (P > 0) ? s / (double)P : 0.0;
    }
    if (per_pair) memcpy(per_pair, op, sizeof(cplx) * (size_t)(W * P));
    if (scale) memcpy(scale, sc, sizeof(double) * (size_t)(W * P));
    for (int64_t w = 0; w < W; ++w) walker_free(&wk[w]);
    free(G);
    free(wk);
    free(op);
    free(sc);
    return used;
}

/* ------------------------------------------ exported: walker gradient
 * grad: W x n x ne, grad[w][k][j] = dO_w / dPhi_w[k][j] (holomorphic).
 * Because O is linear in each column of Phi, the partial derivative with
 * respect to entry (k, j) equals O evaluated with column j replaced by e_k. */
int orc_overlap_grad(int n, int ne, int64_t W, int64_t P, const cplx *Phi, const double *Q,
                     const uint8_t *b, int mode, int nodes, int threads, cplx *overlap, cplx *grad) {
    int N2 = 2 * n;
    int used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    used = omp_get_max_threads();
#endif
    double *G = malloc(sizeof(double) * (size_t)P * N2 * N2);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) orc_snapshot_G(n, Q + p * N2 * N2, b + p * n, G + p * N2 * N2);
    int64_t nvar = (int64_t)n * ne + 1; /* entry 0: the overlap itself */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < W * nvar; ++t) {
        int64_t w = t / nvar, e = t % nvar;
        cplx *Pm = malloc(sizeof(cplx) * n * ne);
        memcpy(Pm, Phi + w * n * ne, sizeof(cplx) * n * ne);
        int k = 0, j = 0;
        if (e > 0) {
            k = (int)((e - 1) / ne);
            j = (int)((e - 1) % ne);
            for (int r = 0; r < n; ++r) Pm[r * ne + j] = (r == k) ? 1.0 : (MUT(11) ? Pm[r * ne + j] : 0.0);
        }
        walker_t wk;
        walker_setup(n, ne, Pm, &wk);
        cplx s = 0.0;
        for (int64_t p = 0; p < P; ++p) s += pair_estimate(&wk, G + p * N2 * N2, mode, nodes, NULL, NULL);
        s = (P > 0) ? s / (double)P : 0.0;
        if (e == 0) overlap[w] = s;
        else grad[w * n * ne + k * ne + j] = s;
        walker_free(&wk);
        free(Pm);
    }
    free(G);
    return used;
}

/* --------------------------------------------- exported: force bias
 * L: nchol x n x n (complex), Phi: W x n x ne, overlap: W, grad: W x n x ne.
 * Green's function G = Phi g^T / O (n x n), <v_gamma> = i tr(L_gamma G),
 * xbar_gamma = -sqrt_dt <v_gamma>;  sqrt_dt == 0 returns <v_gamma>. */
void orc_force_bias(int n, int ne, int64_t W, int nchol, const cplx *L, const cplx *Phi, const cplx *overlap,
                    const cplx *grad, double sqrt_dt, cplx *xbar) {
    cplx *Gf = malloc(sizeof(cplx) * n * n);
    for (int64_t w = 0; w < W; ++w) {
        const cplx *Pw = Phi + w * n * ne, *gw = grad + w * n * ne;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                cplx s = 0.0;
                for (int j = 0; j < ne; ++j) s += Pw[p * ne + j] * gw[q * ne + j];
                Gf[p * n + q] = s / overlap[w];
            }
        for (int g = 0; g < nchol; ++g) {
            const cplx *Lg = L + (size_t)g * n * n;
            cplx tr = 0.0;
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q) tr += Lg[p * n + q] * Gf[MUT(12) ? p * n + q : q * n + p];
            cplx v = I * tr;
            xbar[w * nchol + g] = (sqrt_dt != 0.0) ? -sqrt_dt * v : v;
        }
    }
    free(Gf);
}

/* --------------------------- 15. shadow estimates of Majorana correlators, 1-RDM, particle number
 * Supplementary "Reduced Density Matrices", Eq. (local_fermionic_ob_exp): for rotated
 * Majoranas g~_mu = sum_nu R_{mu nu} g_nu (R in O(2n); identity when R is NULL),
 *   <g~_S> = mean_p C(2n,|S|)/C(n,|S|/2) pf( i (R G_p R^T)|_S ),   G_p = Q_p^T C_b Q_p (step 2),
 * the paper's sum over outcomes read as the mean over the measured snapshots.  For
 * |S| = 2, pf(i X|_S) = i X_{mu nu}; for |S| = 4 it is i^2 (X_01 X_23 - X_02 X_13 + X_03 X_12).
 * The 1-RDM follows Eqs. (1rdm_off_diagonal), (1rdm_diagonal) with the Majoranas of
 * Eq. (majorana_op) at 0-based indices 2p, 2p+1:
 *   a_p^dag a_q = (1/4)(g_2p - i g_2p+1)(g_2q + i g_2q+1)  (p != q),
 *   a_p^dag a_p = (1 + i g_2p g_2p+1) / 2,
 * and the particle number is its trace.  Optional weights w_p give the weighted mean
 * sum_p w_p est_p / sum_p w_p (exact group averages in the tests).
 * Outputs (each may be NULL):
 *   gam2  2n x 2n real, <g~_mu g~_nu> = i gam2[mu][nu] for mu != nu (diagonal 0)
 *   gam4  C(2n,4) real, <g~_mu g~_nu g~_rho g~_sigma> for mu < nu < rho < sigma in
 *         lexicographic order (the estimate of a product of four distinct Majoranas is real)
 *   rdm1  n x n complex, <a_p^dag a_q> in the rotated mode basis
 *   npart particle number */
int orc_shadow_rdm(int n, int64_t P, const double *Q, const uint8_t *b, const double *w, const double *R,
                   double *gam2, double *gam4, cplx *rdm1, double *npart) {
    const int N2 = 2 * n;
    if (n < 1 || n > ORC_MAXN || P < 1) return -1;
    const double K2 = binom(N2, 2) / binom(n, 1), K4 = n >= 2 ? binom(N2, 4) / binom(n, 2) : 0.0;
    const long n4 = N2 >= 4 ? (long)binom(N2, 4) : 0;
    double *G = malloc(sizeof(double) * N2 * N2), *X = malloc(sizeof(double) * N2 * N2);
    double *T = malloc(sizeof(double) * N2 * N2), *acc2 = calloc((size_t)N2 * N2, sizeof(double));
    double *acc4 = gam4 ? calloc((size_t)(n4 > 0 ? n4 : 1), sizeof(double)) : NULL;
    double wsum = 0.0;
    for (int64_t p = 0; p < P; ++p) {
        const double wp = w ? w[p] : 1.0;
        wsum += wp;
        orc_snapshot_G(n, Q + p * N2 * N2, b + p * n, G);
        if (R) { /* X = R G R^T */
            for (int i = 0; i < N2; ++i)
                for (int j = 0; j < N2; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < N2; ++k) s += G[i * N2 + k] * R[j * N2 + k];
                    T[i * N2 + j] = s;
                }
            for (int i = 0; i < N2; ++i)
                for (int j = 0; j < N2; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < N2; ++k) s += R[i * N2 + k] * T[k * N2 + j];
                    X[i * N2 + j] = s;
                }
        } else {
            memcpy(X, G, sizeof(double) * N2 * N2);
        }
        for (int i = 0; i < N2 * N2; ++i) acc2[i] += wp * K2 * X[i];
        if (acc4) {
            long t = 0;
            for (int a = 0; a < N2; ++a)
                for (int bb = a + 1; bb < N2; ++bb)
                    for (int c = bb + 1; c < N2; ++c)
                        for (int d = c + 1; d < N2; ++d, ++t) {
                            double pf4 = X[a * N2 + bb] * X[c * N2 + d] - X[a * N2 + c] * X[bb * N2 + d] +
                                         X[a * N2 + d] * X[bb * N2 + c];
                            acc4[t] += wp * K4 * (-pf4); /* i^2 pf(X|_S) */
                        }
        }
    }
    double *g2 = malloc(sizeof(double) * N2 * N2);
    for (int i = 0; i < N2 * N2; ++i) g2[i] = acc2[i] / wsum;
    for (int i = 0; i < N2; ++i) g2[i * N2 + i] = 0.0;
    if (gam2) memcpy(gam2, g2, sizeof(double) * N2 * N2);
    if (gam4)
        for (long t = 0; t < n4; ++t) gam4[t] = acc4[t] / wsum;
    /* E(mu, nu) = <g_mu g_nu> = i gam2[mu][nu] for mu != nu */
    double np_ = 0.0;
    for (int pp = 0; pp < n; ++pp)
        for (int q = 0; q < n; ++q) {
            cplx d;
            if (pp == q) {
                d = 0.5 * (1.0 - g2[(2 * pp) * N2 + 2 * pp + 1]);
                np_ += creal(d);
            } else {
                cplx e00 = I * g2[(2 * pp) * N2 + 2 * q], e01 = I * g2[(2 * pp) * N2 + 2 * q + 1];
                cplx e10 = I * g2[(2 * pp + 1) * N2 + 2 * q], e11 = I * g2[(2 * pp + 1) * N2 + 2 * q + 1];
                d = 0.25 * (e00 + I * e01 - I * e10 + e11);
                if (MUT(10)) d = 0.25 * (e00 - I * e01 + I * e10 + e11);
            }
            if (rdm1) rdm1[pp * n + q] = d;
        }
    if (npart) *npart = np_;
    free(G);
    free(X);
    free(T);
    free(acc2);
    free(acc4);
    free(g2);
    return 0;
}

/* --------------------------- 16. virtual-correlation-energy walker transform
 * Supplementary "Virtual Correlation Energy Derivation", Eq. (vce_overlap), one spin
 * sector.  Orbitals are ordered core (nc), active (na), virtual; the walker Phi is
 * NB x ne with ne = nc + nea electrons; the trial is the core Slater determinant Xi_c
 * (unit vectors of the core orbitals) times an active state chi times the virtual
 * vacuum.  The virtual rows drop out; with the core block phi_c = Phi[0:nc, :] and the
 * active block phi_a = Phi[nc:nc+na, :],
 *   <Xi_c chi 0_v | phi> = det [ phi_c ; chi^dag phi_a ].
 * The paper takes a unitary V from the SVD of phi_c; any unitary V whose first nc
 * columns span the row space of phi_c serves: from the complete QR phi_c^dag = V [R_c; 0],
 * phi_c V = [R_c^dag, 0], so the determinant is block triangular after right
 * multiplication by V and
 *   <Xi_c chi 0_v | phi> = conj(det R_c) det(chi^dag phi_a V') / det V,
 * V' the last nea columns of V.  Outputs: the active walker act = phi_a V' (na x nea)
 * and factor = conj(det R_c) / det V.  det V by LU with partial pivoting. */

static cplx cdet_lu(int m, const cplx *A) {
    cplx *B = malloc(sizeof(cplx) * (m > 0 ? m * m : 1));
    memcpy(B, A, sizeof(cplx) * m * m);
    cplx d = 1.0;
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int i = k + 1; i < m; ++i)
            if (cabs(B[i * m + k]) > cabs(B[piv * m + k])) piv = i;
        if (B[piv * m + k] == 0.0) {
            free(B);
            return 0.0;
        }
        if (piv != k) {
            for (int j = 0; j < m; ++j) {
                cplx t = B[k * m + j];
                B[k * m + j] = B[piv * m + j];
                B[piv * m + j] = t;
            }
            d = -d;
        }
        d *= B[k * m + k];
        for (int i = k + 1; i < m; ++i) {
            cplx f = B[i * m + k] / B[k * m + k];
            for (int j = k; j < m; ++j) B[i * m + j] -= f * B[k * m + j];
        }
    }
    free(B);
    return d;
}

int orc_vce_transform(int NB, int nc, int na, int nea, const cplx *Phi, cplx *act, cplx *factor) {
    const int ne = nc + nea;
    if (nc < 0 || na < 1 || nea < 0 || nea > na || NB < nc + na) return -1;
    cplx *Ct = malloc(sizeof(cplx) * (ne * (nc > 0 ? nc : 1)));
    cplx *V = malloc(sizeof(cplx) * ne * ne);
    cplx *Rc = malloc(sizeof(cplx) * (nc > 0 ? nc * nc : 1));
    for (int j = 0; j < ne; ++j) /* phi_c^dag: ne x nc */
        for (int i = 0; i < nc; ++i) Ct[j * nc + i] = conj(Phi[i * ne + j]);
    cplx detR = 1.0;
    if (nc > 0) {
        orc_walker_qr(ne, nc, Ct, V, Rc);
        for (int i = 0; i < nc; ++i) detR *= Rc[i * nc + i];
    } else {
        for (int i = 0; i < ne; ++i)
            for (int j = 0; j < ne; ++j) V[i * ne + j] = (i == j) ? 1.0 : 0.0;
    }
    for (int r = 0; r < na; ++r)
        for (int c = 0; c < nea; ++c) {
            cplx s = 0.0;
            for (int k = 0; k < ne; ++k) s += Phi[(nc + r) * ne + k] * V[k * ne + nc + c];
            act[r * nea + c] = s;
        }
    *factor = (MUT(13) ? detR : conj(detR)) / cdet_lu(ne, V);
    free(Ct);
    free(V);
    free(Rc);
    return 0;
}

/* --------------------------- 17. local-energy terms by derivatives of the overlap
 * Eqs. (force_bias_diff), (energy_tb_diff): for a one-body operator
 * Lhat = sum_pq L_pq a_p^dag a_q, e^{lambda Lhat} maps the walker's orbitals Phi to
 * e^{lambda L} Phi (Thouless), so with O the shadow overlap,
 *   <Psi_T| Lhat |phi>      = d/dlambda   O(e^{lambda L} Phi) at 0 = D O[L Phi],
 *   <Psi_T| Lhat Lhat |phi> = d^2/dlambda^2 O(e^{lambda L} Phi) at 0
 *                           = D^2 O[L Phi, L Phi] + D O[L^2 Phi].
 * Each pair term o_p is linear in every column of Phi (step 13), so these derivatives
 * are exact column substitutions:
 *   D o_p[X]     = sum_j o_p(Phi with column j replaced by X_j),
 *   D^2 o_p[X,X] = 2 sum_{j<j'} o_p(Phi with columns j, j' replaced by X_j, X_j').
 * Outputs per walker (each output may be NULL): ov = O, e1 = <Psi_T|hhat|phi>/O (h may be
 * NULL) and e2 = sum_gamma <Psi_T|Lhat_gamma Lhat_gamma|phi>/O, ratios of shadow means
 * (weighted means sum_p w_p o_p / sum_p w_p when wts is given: exact group averages). */
int orc_local_energy(int n, int ne, int64_t W, int64_t P, const cplx *Phi, const double *Q, const uint8_t *b,
                     const double *wts, const cplx *h, int nchol, const cplx *L, int threads, cplx *ov, cplx *e1,
                     cplx *e2) {
    const int N2 = 2 * n;
    int used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    used = omp_get_max_threads();
#endif
    double *G = malloc(sizeof(double) * (size_t)(P > 0 ? P : 1) * N2 * N2);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < P; ++p) orc_snapshot_G(n, Q + p * N2 * N2, b + p * n, G + p * N2 * N2);
    /* variants of one walker: 0 base; per operator (h first when given, then each L_gamma):
       ne single substitutions by columns of X2 (h: X1 = h Phi), then ne(ne-1)/2 pairs by X1 */
    const int nsingle = ne, npair = ne * (ne - 1) / 2;
    const int nop = (h ? 1 : 0) + nchol;
    const int64_t per_op = nsingle + npair;
    const int64_t nvar = 1 + (int64_t)nop * per_op;
    cplx *val = malloc(sizeof(cplx) * (size_t)(W * nvar > 0 ? W * nvar : 1));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < W * nvar; ++t) {
        const int64_t w = t / nvar, v = t % nvar;
        const cplx *Pw = Phi + w * n * ne;
        cplx *Pm = malloc(sizeof(cplx) * n * ne);
        memcpy(Pm, Pw, sizeof(cplx) * n * ne);
        if (v > 0) {
            const int op = (int)((v - 1) / per_op), r = (int)((v - 1) % per_op);
            const int is_h = h && op == 0;
            const cplx *Lo = is_h ? h : L + (size_t)(op - (h ? 1 : 0)) * n * n;
            cplx *X1 = malloc(sizeof(cplx) * n * ne), *X2 = malloc(sizeof(cplx) * n * ne);
            for (int i = 0; i < n; ++i) /* X1 = Lo Phi */
                for (int j = 0; j < ne; ++j) {
                    cplx s = 0.0;
                    for (int k = 0; k < n; ++k) s += Lo[i * n + k] * Pw[k * ne + j];
                    X1[i * ne + j] = s;
                }
            for (int i = 0; i < n; ++i) /* X2 = Lo X1 = Lo^2 Phi */
                for (int j = 0; j < ne; ++j) {
                    cplx s = 0.0;
                    for (int k = 0; k < n; ++k) s += Lo[i * n + k] * X1[k * ne + j];
                    X2[i * ne + j] = s;
                }
            if (r < nsingle) { /* first derivative (h) or the D O[L^2 Phi] term (L_gamma) */
                const cplx *Xs = is_h ? X1 : X2;
                for (int i = 0; i < n; ++i) Pm[i * ne + r] = Xs[i * ne + r];
            } else { /* pair (j, j') of the second-derivative term; h has no such term */
                int q = r - nsingle, j = 0;
                while (q >= ne - 1 - j) {
                    q -= ne - 1 - j;
                    ++j;
                }
                const int j2 = j + 1 + q;
                for (int i = 0; i < n; ++i) {
                    Pm[i * ne + j] = X1[i * ne + j];
                    Pm[i * ne + j2] = X1[i * ne + j2];
                }
            }
            free(X1);
            free(X2);
        }
        const int skip = v > 0 && h && (v - 1) / per_op == 0 && (v - 1) % per_op >= nsingle;
        cplx s = 0.0;
        if (!skip) {
            walker_t wk;
            walker_setup(n, ne, Pm, &wk);
            double ws = 0.0;
            for (int64_t p = 0; p < P; ++p) {
                const double wp = wts ? wts[p] : 1.0;
                s += wp * pair_estimate(&wk, G + p * N2 * N2, ORC_INTERP_ROOTS, 0, NULL, NULL);
                ws += wp;
            }
            walker_free(&wk);
            s = (ws != 0.0) ? s / ws : 0.0;
        }
        val[t] = s;
        free(Pm);
    }
    for (int64_t w = 0; w < W; ++w) {
        const cplx *vw = val + w * nvar;
        const cplx O = vw[0];
        if (ov) ov[w] = O;
        cplx n1 = 0.0, n2 = 0.0;
        for (int op = 0; op < nop; ++op) {
            const cplx *vo = vw + 1 + (int64_t)op * per_op;
            cplx d1 = 0.0, d2 = 0.0;
            for (int r = 0; r < nsingle; ++r) d1 += vo[r];
            for (int r = 0; r < npair; ++r) d2 += vo[nsingle + r];
            if (h && op == 0) n1 = d1;
            else n2 += (MUT(14) ? 1.0 : 2.0) * d2 + d1;
        }
        if (e1) e1[w] = (h && O != 0.0) ? n1 / O : 0.0;
        if (e2) e2[w] = (O != 0.0) ? n2 / O : 0.0;
    }
    free(G);
    free(val);
    return used;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
