"""The tensor-core congruence of the FP64 overlap path, restated on the CPU (no GPU).

The kernel forms B^(s) of Eq. (b_mat) from P = M H M^T, with M the walker's real form
[[A, -B], [B, A]] (Ut = A + iB the walker rows, occupied rows / sqrt2) and
H = N^T J N the snapshot's (N = [C, D], Qt = C + iD its complexified sign-folded rows,
J the canonical skew form on the Majorana index).  Every entry of B^(s) is then a signed
sum of entries of P: for occupied modes the complex row T_j = R_j + i R_{n+j}, for empty
modes the two real rows Re T_j and -Im T_j (R = [Re T; Im T] = M N^T).

The two products run on tensor cores by error-free slicing: every FP64 row is cut into
seven 8-bit integer slices (row scale 2^e, magnitude |x| 2^(56-e) truncated), the slice
products of levels 2..8 are summed exactly (the tensor cores accumulate these integer
sums below 2^24 exactly in FP32), the levels are combined into 64-bit fixed point, Z is
re-sliced by rows of Z^T, and the second product's fixed point is rounded to FP64.

This file restates those steps with Python integers and checks
  * that the assembly of B^(s) from P reproduces the oracle's B^(s) (a wrong sign,
    row order or selection fails here),
  * that the sliced products reproduce M H M^T to the accuracy of an FP64 product
    (about 2^-50 of the row scales), against exact rational arithmetic,
  * that every level sum stays below 2^24, the condition for exact FP32 accumulation.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle.oracle as orc
from paper_2506_22408_gb300 import synth

SLICES = 7
NO_ROW = -100000


def kernel_rows(Q, b, Phi):
    """Walker rows Ut (n x n) and snapshot rows Qt (2n x n) as the walker prep and the
    snapshot build lay them out (from the oracle's complete QR, no echelon rotation)."""
    n, ne = Phi.shape
    U, R = orc.walker_qr(Phi)
    Ut = U.T.copy()
    Ut[:ne] /= math.sqrt(2.0)
    Qt = np.empty((2 * n, n), complex)
    for c in range(2 * n):
        sg = -1.0 if (c & 1) and (b[c >> 1] & 1) else 1.0
        Qt[c] = sg * Q[c, 0::2] - 1j * sg * Q[c, 1::2]
    return Ut, Qt, np.prod(np.diag(R))


def real_forms(Ut, Qt):
    n = Ut.shape[0]
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n], M[:n, n:] = Ut.real, -Ut.imag
    M[n:, :n], M[n:, n:] = Ut.imag, Ut.real
    N = np.concatenate([Qt.real, Qt.imag], axis=1)
    J = np.zeros((2 * n, 2 * n))
    for i in range(n):
        J[2 * i, 2 * i + 1], J[2 * i + 1, 2 * i] = 1.0, -1.0
    return M, N, J


def B_from_P(P, n, ne):
    """The kernel's assembly of B^(s) (m x m) from P = R J R^T."""
    m = 2 * n - ne

    def rows(x):  # selected row x as a list of (row of R, coefficient)
        if x < ne:
            return [(x, 1.0), (n + x, 1j)]
        j = ne + (x - ne) // 2
        return [(j, 1.0)] if (x - ne) % 2 == 0 else [(n + j, -1.0)]

    B = np.zeros((m, m), complex)
    for x in range(m):
        for y in range(m):
            B[x, y] = sum(cx * cy * P[rx, ry] for rx, cx in rows(x) for ry, cy in rows(y))
    return B


# ------------------------------------------------------------------ sliced products

def row_scale(x):
    nz = [math.frexp(v)[1] for v in x if v != 0.0]
    return max(nz) if nz else NO_ROW


def fixed(v, e):
    """|v| 2^(56-e) truncated (v a double with |v| < 2^e)."""
    if v == 0.0:
        return 0
    m, ex = math.frexp(abs(v))
    mant = int(m * 2 ** 53)
    sh = ex - 53 + 56 - e
    return mant << sh if sh >= 0 else mant >> -sh


def slice_rows(X):
    """Row scales e[r] and slices a[i][r][k] (i = 0..6) of the rows of X (32 x 32)."""
    R, K = X.shape
    e = [row_scale(X[r]) for r in range(R)]
    a = np.zeros((SLICES, R, K), np.int64)
    for r in range(R):
        if e[r] == NO_ROW:
            continue
        for k in range(K):
            u = fixed(X[r, k], e[r])
            s = -1 if X[r, k] < 0 else 1
            for i in range(SLICES):
                a[i, r, k] = s * ((u >> (56 - 8 * (i + 1))) & 255)
    return e, a


def levels(a, b):
    """Level sums acc[L-2][r][c] = sum_{i+j=L} sum_k a_i[r][k] b_j[c][k], L = 2..8."""
    acc = np.zeros((SLICES, a.shape[1], b.shape[1]), np.int64)
    for i in range(SLICES):
        for j in range(SLICES):
            L = (i + 1) + (j + 1)
            if L <= SLICES + 1:
                acc[L - 2] += a[i] @ b[j].T
    return acc


def combine(acc):
    """z = sum_{L=2..7} acc_L 2^(8(7-L)) + floor(acc_8 / 2^8) as Python integers."""
    R, C = acc.shape[1:]
    z = [[int(acc[6, r, c]) >> 8 for c in range(C)] for r in range(R)]
    for L in range(2, 8):
        for r in range(R):
            for c in range(C):
                z[r][c] += int(acc[L - 2, r, c]) << (8 * (7 - L))
    return z


def sliced_P(M, H):
    """P = M H M^T as the kernel forms it; returns (P, largest level sum)."""
    e, am = slice_rows(M)
    g, ah = slice_rows(H)
    acc1 = levels(ah, am)                                    # Z[k][b] = (H M^T)[k][b]
    z1 = combine(acc1)
    K = M.shape[0]
    F = [NO_ROW] * K
    ac = np.zeros((SLICES, K, K), np.int64)                  # slices of Z^T, rows b
    for b_ in range(K):
        zs = [z1[k][b_] for k in range(K)]
        tops = [g[k] + abs(z).bit_length() for k, z in enumerate(zs) if z != 0]
        if not tops or e[b_] == NO_ROW:
            continue
        G = max(tops)
        F[b_] = e[b_] + G - 56
        for k, z in enumerate(zs):
            if z == 0:
                continue
            sh = 56 + g[k] - G
            u = abs(z) << sh if sh >= 0 else abs(z) >> -sh
            assert u < 2 ** 56
            s = -1 if z < 0 else 1
            for i in range(SLICES):
                ac[i, b_, k] = s * ((u >> (56 - 8 * (i + 1))) & 255)
    acc2 = levels(ac, am)                                    # [b][a] = (M Z)[a][b]
    z2 = combine(acc2)
    P = np.zeros((K, K))
    for a_ in range(K):
        for b_ in range(K):
            if F[b_] != NO_ROW and e[a_] != NO_ROW:
                P[a_, b_] = math.ldexp(float(z2[b_][a_]), e[a_] + F[b_] - 56)
    top = max(int(np.abs(acc1).max()), int(np.abs(acc2).max()))
    return P, top


def case(seed, n, ne, ensemble="haar"):
    rng = np.random.default_rng(seed)
    Q = (synth.haar_orthogonal(rng, 2 * n, 1) if ensemble == "haar" else synth.signed_permutation(rng, 2 * n, 1))[0]
    b = synth.uniform_bits(rng, n, 1)[0]
    Phi = synth.walkers(rng, n, ne, 1)[0]
    return Q, b, Phi


@pytest.mark.parametrize("n,ne", [(4, 2), (8, 4), (12, 6), (16, 8), (16, 4)])
def test_B_assembled_from_P_matches_the_oracle(n, ne):
    for seed in range(3):
        Q, b, Phi = case(100 + seed, n, ne)
        Ut, Qt, _ = kernel_rows(Q, b, Phi)
        M, N, J = real_forms(Ut, Qt)
        R = M @ N.T
        T = Ut @ Qt.T
        assert np.allclose(R[:n], T.real, atol=1e-14) and np.allclose(R[n:], T.imag, atol=1e-14)
        H = N.T @ J @ N
        assert np.allclose(H, -H.T, atol=1e-14)
        P = M @ H @ M.T
        assert np.allclose(P, R @ J @ R.T, atol=1e-13)
        B = B_from_P(P, n, ne)
        Bo, _, _ = orc.pair_matrices(Q, b, Phi)
        assert np.abs(B - Bo).max() <= 1e-13 * np.abs(Bo).max()


def test_wrong_empty_row_sign_is_caught():
    """A plausible slip in the assembly (Im T_j instead of -Im T_j for the second row
    of an empty mode) fails the comparison with the oracle."""
    n, ne = 8, 4
    Q, b, Phi = case(7, n, ne)
    Ut, Qt, _ = kernel_rows(Q, b, Phi)
    M, N, J = real_forms(Ut, Qt)
    P = M @ (N.T @ J @ N) @ M.T
    B = B_from_P(P, n, ne)
    flip = np.ones(2 * n - ne)
    flip[ne + 1::2] = -1.0
    Bo, _, _ = orc.pair_matrices(Q, b, Phi)
    assert np.abs(B - Bo).max() <= 1e-13 * np.abs(Bo).max()
    assert np.abs(flip[:, None] * B * flip[None, :] - Bo).max() > 1e-3 * np.abs(Bo).max()


def padded(X, K=32):
    Y = np.zeros((K, K))
    Y[: X.shape[0], : X.shape[1]] = X
    return Y


@pytest.mark.parametrize("n,ne,ensemble", [(16, 8, "haar"), (16, 8, "signed"), (12, 6, "haar"), (8, 4, "haar")])
def test_sliced_products_reach_fp64_accuracy(n, ne, ensemble):
    Q, b, Phi = case(300 + n + ne, n, ne, ensemble)
    Ut, Qt, _ = kernel_rows(Q, b, Phi)
    M, N, J = real_forms(Ut, Qt)
    H = N.T @ J @ N
    Mp, Hp = padded(M), padded(H)
    P, top = sliced_P(Mp, Hp)
    assert top < 2 ** 24  # every level sum is exact in FP32
    # exact reference on a sample of entries: rational arithmetic on the FP64 inputs
    K = 2 * n
    Mf = [[Fraction(float(x)) for x in row] for row in M]
    Hf = [[Fraction(float(x)) for x in row] for row in H]
    rng = np.random.default_rng(n)
    absMHM = np.abs(M) @ np.abs(H) @ np.abs(M).T
    worst = 0.0
    for a_, b_ in zip(rng.integers(0, K, 40), rng.integers(0, K, 40)):
        Z = [sum(Hf[k][l] * Mf[b_][l] for l in range(K)) for k in range(K)]
        exact = sum(Mf[a_][k] * Z[k] for k in range(K))
        err = abs(Fraction(float(P[a_, b_])) - exact)
        worst = max(worst, float(err) / absMHM[a_, b_])
    assert worst <= 2.0 ** -48, worst
    assert np.all(P[K:, :] == 0.0) and np.all(P[:, K:] == 0.0)
    # and the resulting B^(s) equals the oracle's to FP64 rounding
    B = B_from_P(P[:K, :K], n, ne)
    Bo, _, _ = orc.pair_matrices(Q, b, Phi)
    assert np.abs(B - Bo).max() <= 1e-13 * np.abs(Bo).max()


def test_level_sums_bound_for_full_slices():
    """The largest possible level sum (all 28 products of levels 2..8 with every slice
    at 255 and equal signs) stays below 2^24: 7 * 32 * 255^2 at level 8."""
    a = np.full((SLICES, 4, 32), 255, np.int64)
    acc = levels(a, a)
    assert acc.max() == 7 * 32 * 255 ** 2 < 2 ** 24
