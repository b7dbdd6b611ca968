"""Host-only checks (numpy, no library) of the identities behind the K-form of the FP64 ALU
overlap kernel above 16 modes and of the gradient kernel.

With T = Ut Qt^T (n x 2n), X the selected rows (occupied T_j, then Re T_j and -Im T_j per
empty mode), J the pairing of the Majorana indices (J[2a][2a+1] = 1) and the snapshot's
rows H1 = Qt^T J Qt, G2 = Qt^T J conj(Qt):
  * B = X J X^T follows from K = Ut [H1 | G2] and the walker rows (W1 = K1 Ut^T,
    W2 = K2 Ut^H, class by class as build_B_from_K writes it);
  * the cotangents Gamma1 = G_X[occ] Qt and Gamma2 = Ht conj(Qt), with G_X = Y X J and
    Ht_i = G_X[ne+2i] - i G_X[ne+2i+1], follow from K and the coefficient rows of Y;
  * Gauss's three-product forms used for K1 u and K2 conj(u) give the complex products.
"""
from __future__ import annotations

import numpy as np
import pytest


def _jmat(n):
    J = np.zeros((2 * n, 2 * n))
    for a in range(n):
        J[2 * a, 2 * a + 1] = 1.0
        J[2 * a + 1, 2 * a] = -1.0
    return J


def _setup(seed, n, ne):
    rng = np.random.default_rng(seed)
    Ut = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    Qt = rng.normal(size=(2 * n, n)) + 1j * rng.normal(size=(2 * n, n))
    d = n - ne
    J = _jmat(n)
    T = Ut @ Qt.T
    X = np.zeros((ne + 2 * d, 2 * n), complex)
    X[:ne] = T[:ne]
    for j in range(d):
        X[ne + 2 * j] = T[ne + j].real
        X[ne + 2 * j + 1] = -T[ne + j].imag
    H1 = Qt.T @ J @ Qt
    G2 = Qt.T @ J @ Qt.conj()
    K = Ut @ np.concatenate([H1.T, G2.T], 0).T  # Ut [H1 | G2], formed like T from the rows Qh
    return Ut, Qt, J, X, K


def _B_from_K(Ut, K, n, ne):
    d, m = n - ne, 2 * n - ne
    K1, K2 = K[:, :n], K[:, n:]
    W1 = K1 @ Ut.T
    W2 = K2 @ Ut.conj().T
    B = np.zeros((m, m), complex)
    for a in range(ne):
        for b in range(a + 1, ne):
            B[a, b] = W1[a, b]
        for jj in range(d):
            j = ne + jj
            B[a, ne + 2 * jj] = (W1[a, j] + W2[a, j]) / 2
            B[a, ne + 2 * jj + 1] = 1j * (W1[a, j] - W2[a, j]) / 2
    for x in range(d):
        for y in range(x, d):
            al, be = W1[ne + x, ne + y], W2[ne + x, ne + y]
            r1, r2 = ne + 2 * x, ne + 2 * y
            if x < y:
                B[r1, r2] = (al + be).real / 2
                B[r1, r2 + 1] = (be - al).imag / 2
                B[r1 + 1, r2] = -(al + be).imag / 2
                B[r1 + 1, r2 + 1] = (be - al).real / 2
            else:
                B[r1, r1 + 1] = be.imag / 2
    return B


@pytest.mark.parametrize("n,ne", [(4, 2), (6, 6), (8, 2), (9, 4), (12, 6)])
def test_B_from_K_is_X_J_Xt(n, ne):
    Ut, Qt, J, X, K = _setup(n * 10 + ne, n, ne)
    B = X @ J @ X.T
    Bk = _B_from_K(Ut, K, n, ne)
    iu = np.triu_indices(2 * n - ne, 1)
    scale = np.abs(B).max()
    assert np.abs(B[iu] - Bk[iu]).max() <= 1e-13 * scale


@pytest.mark.parametrize("n,ne", [(4, 2), (6, 4), (8, 2), (10, 6)])
def test_cotangents_from_K(n, ne):
    Ut, Qt, J, X, K = _setup(7 + n + ne, n, ne)
    d, m = n - ne, 2 * n - ne
    rng = np.random.default_rng(n * ne)
    Y = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    Y = Y - Y.T
    # the definitions: G_X / 2 = Y (X J), Gamma1 = G_X[occ] Qt, Gamma2 = Ht conj(Qt)
    GX = Y @ (X @ J)
    gam1 = GX[:ne] @ Qt
    Ht = np.array([GX[ne + 2 * i] - 1j * GX[ne + 2 * i + 1] for i in range(d)]).reshape(d, 2 * n)
    gam2 = Ht @ Qt.conj()
    want = np.concatenate([gam1, gam2], 0)
    # from K: the coefficient rows y (Y[r] or Yh_i), the empty pairs folded into
    # (y_R + i y_I)/2 on K_j and (y_R - i y_I)/2 on the conjugate of the other half
    got = np.zeros((n, n), complex)
    for r in range(n):
        y = Y[r] if r < ne else Y[ne + 2 * (r - ne)] - 1j * Y[ne + 2 * (r - ne) + 1]
        o1, o2 = (0, n) if r < ne else (n, 0)
        acc = y[:ne] @ K[:ne, o1:o1 + n]
        for j in range(d):
            c = (y[ne + 2 * j] + 1j * y[ne + 2 * j + 1]) / 2
            cp = (y[ne + 2 * j] - 1j * y[ne + 2 * j + 1]) / 2
            acc = acc + c * K[ne + j, o1:o1 + n] + cp * np.conj(K[ne + j, o2:o2 + n])
        got[r] = acc
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_three_product_forms():
    rng = np.random.default_rng(3)
    k1, k2, u = (rng.normal(size=11) + 1j * rng.normal(size=11) for _ in range(3))
    # K1 u: Re = p1 - p2, Im = p3 - p1 - p2 with p3 = sum (k1r + k1i)(ur + ui)
    p1, p2 = (k1.real * u.real).sum(), (k1.imag * u.imag).sum()
    p3 = ((k1.real + k1.imag) * (u.real + u.imag)).sum()
    assert np.isclose(complex(p1 - p2, p3 - p1 - p2), (k1 * u).sum(), rtol=1e-14, atol=0)
    # K2 conj(u) = conj(conj(K2) u): Re = q1 + q2, Im = q1 - q2 - q3, q3 = sum (k2r - k2i)(ur + ui)
    q1, q2 = (k2.real * u.real).sum(), (k2.imag * u.imag).sum()
    q3 = ((k2.real - k2.imag) * (u.real + u.imag)).sum()
    assert np.isclose(complex(q1 + q2, q1 - q2 - q3), (k2 * np.conj(u)).sum(), rtol=1e-14, atol=0)
    # the gradient's form with re - im of u: Im = q3' - q1 + q2, q3' = sum (k2r + k2i)(ur - ui)
    q3b = ((k2.real + k2.imag) * (u.real - u.imag)).sum()
    assert np.isclose(complex(q1 + q2, q3b - q1 + q2), (k2 * np.conj(u)).sum(), rtol=1e-14, atol=0)
