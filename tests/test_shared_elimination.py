"""The overlap kernels' two rearrangements of the per-pair work, checked on the CPU with
matrices from the oracle (no GPU):

* the node matrices B + w D differ only in their empty x empty block, so eliminating the
  occupied block first (pivots restricted to it) gives pf(B + w D) = pf0 pf(S + w D_ee)
  for every node w, S the Schur complement of the occupied block;
* the adjoint's backward pass over those shared steps is affine in the inverse Z of the
  complement, so one pass started from sum_k c_k Z_k (each step's constant scaled by
  sum_k c_k) gives sum_k c_k A_k^{-1};
* the local-energy traces follow from A_k^{-1} = F0 + F Z_k F^T with 2d x 2d work per
  node, and its operator matrices A' need the snapshot only through M^T = Q'^T J X^T,
  formed once per pair;
* the estimator is multilinear and alternating in the occupied orbitals:
  o(Phi W) = det(W) o(Phi) for any ne x ne matrix W, which is what lets the walker prep
  rotate the occupied orbitals to echelon form and fold det W into det R.

The elimination below restates the kernel's steps in numpy (largest entry of the
active occupied block as pivot, the sign (-1)^(ak+ap-1) of moving the pivot pair to
the front, rank-2 update), so that a wrong sign, index or pivot restriction fails here.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle.oracle as orc
from paper_2506_22408_gb300 import synth

GROWTH = 2.0 ** 8  # the kernel's bound on max|S| / max|B| before it falls back


def key(x):
    return max(abs(x.real), abs(x.imag))


def shared_elimination(B, ne):
    """Eliminate the ne occupied indices of the skew matrix B; returns (pf0, S, growth)
    or None when a pivot is zero."""
    A = B.astype(complex).copy()
    act = list(range(A.shape[0]))
    pf0 = 1.0 + 0j
    kb = max(key(x) for x in B[np.triu_indices(B.shape[0], 1)])
    for s in range(ne // 2):
        ro = ne - 2 * s
        kv, ak, ap = max((key(A[act[a], act[b]]), -b * 1000 - a, 0) for b in range(1, ro) for a in range(b))
        if kv == 0:
            return None
        ap, ak = divmod(-ak, 1000)
        k, p = act[ak], act[ap]
        piv = A[k, p]
        pf0 *= piv * (-1) ** (ak + ap - 1)
        rest = [act[x] for x in range(len(act)) if x not in (ak, ap)]
        u = A[rest, k] / piv
        v = A[rest, p]
        A[np.ix_(rest, rest)] -= np.outer(u, v) - np.outer(v, u)
        act = rest
    S = A[np.ix_(act, act)]
    ks = max([key(x) for x in S[np.triu_indices(len(act), 1)]] + [0.0])
    return pf0, S, ks / kb


def node_D(n, ne):
    m, d = 2 * n - ne, n - ne
    D = np.zeros((m, m))
    for i in range(d):
        D[ne + 2 * i, ne + 2 * i + 1], D[ne + 2 * i + 1, ne + 2 * i] = 1.0, -1.0
    return D


@pytest.mark.parametrize("n,ne", [(16, 8), (12, 6), (9, 2), (8, 8), (10, 4)])
def test_shared_occupied_elimination_identity(n, ne):
    rng = np.random.default_rng(100 + n * 7 + ne)
    Q = synth.haar_orthogonal(rng, 2 * n, 12)
    b = synth.uniform_bits(rng, n, 12)
    Phi = synth.walkers(rng, n, ne, 2)
    D = node_D(n, ne)
    nodes = np.exp(-1j * np.array([0.3, 1.4, 2.6]))
    for w in range(2):
        for p in range(12):
            B, _, _ = orc.pair_matrices(Q[p], b[p], Phi[w])
            r = shared_elimination(B, ne)
            assert r is not None
            pf0, S, _ = r
            scale = np.abs(B).max() + 1.0
            m = B.shape[0]
            for z in nodes:
                ref = orc.pfaffian(B + z * D)
                got = pf0 * (orc.pfaffian(S + z * D[ne:, ne:]) if m > ne else 1.0)
                assert abs(got - ref) <= 1e-11 * scale ** (m // 2)


def test_shared_elimination_fallback_is_rare():
    """With the growth bound the kernel uses, the full per-node elimination is the
    exception: under 5 % of Haar pairs at n = 16, eta = 8."""
    n, ne = 16, 8
    rng = np.random.default_rng(5)
    Q = synth.haar_orthogonal(rng, 2 * n, 150)
    b = synth.uniform_bits(rng, n, 150)
    Phi = synth.walkers(rng, n, ne, 2)
    falls = total = 0
    for w in range(2):
        for p in range(150):
            B, _, _ = orc.pair_matrices(Q[p], b[p], Phi[w])
            r = shared_elimination(B, ne)
            total += 1
            falls += r is None or r[2] > GROWTH
    assert falls <= 0.05 * total


def test_occupied_orbitals_alternating():
    """o(Phi W) = det(W) o(Phi): the echelon rotation of the occupied orbitals only
    rescales the overlap by det W."""
    n, ne = 10, 4
    rng = np.random.default_rng(11)
    Q = synth.haar_orthogonal(rng, 2 * n, 40)
    b = synth.uniform_bits(rng, n, 40)
    Phi = synth.walkers(rng, n, ne, 1)[0]
    Wm = rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne))
    refl = np.eye(ne, dtype=complex)
    v = rng.standard_normal(ne) + 1j * rng.standard_normal(ne)
    refl -= 2 * np.outer(v, v.conj()) / np.vdot(v, v)  # a Householder reflection, det -1
    o0, _, sc, _ = orc.overlap(Phi[None], Q, b, per_pair=True)
    for Wx in (Wm, refl):
        o1, _, _, _ = orc.overlap((Phi @ Wx)[None], Q, b, per_pair=True)
        assert abs(o1[0] - np.linalg.det(Wx) * o0[0]) <= 1e-12 * abs(np.linalg.det(Wx)) * sc.mean()
    assert abs(np.linalg.det(refl) + 1) < 1e-12


def backward_block(B, ne, Zc, c):
    """The adjoint's backward pass over the shared occupied steps, restated in numpy:
    forward elimination with the kernel's pivots keeping (k, p, 1/a, active list) per
    step, then from the last step back: new entries -Z g1, -Z g2 and c(-1/a) + g1^T Z g2,
    starting from Zc on the empty indices.  Returns the m x m result."""
    A = B.astype(complex).copy()
    m = A.shape[0]
    act = list(range(m))
    hist = []
    for s in range(ne // 2):
        ro = ne - 2 * s
        best = max((key(A[act[a], act[b]]), -b * 1000 - a) for b in range(1, ro) for a in range(b))
        ap, ak = divmod(-best[1], 1000)
        k, p = act[ak], act[ap]
        piv = A[k, p]
        rest = [act[x] for x in range(len(act)) if x not in (ak, ap)]
        hist.append((k, p, 1.0 / piv, rest, A[np.ix_(rest, [k])].ravel().copy(), A[np.ix_(rest, [p])].ravel().copy()))
        u, v = A[rest, k] / piv, A[rest, p]
        A[np.ix_(rest, rest)] -= np.outer(u, v) - np.outer(v, u)
        act = rest
    Y = np.zeros((m, m), complex)
    Y[np.ix_(act, act)] = Zc
    for k, p, ia, rest, aik, aip in reversed(hist):
        g1 = aip * ia          # v / a, v_i = A_{i,p}
        g2 = -aik * ia         # -u / a, u_i = A_{i,k}
        Z = Y[np.ix_(rest, rest)]
        y1, y2 = Z @ g1, Z @ g2
        Y[rest, k], Y[k, rest] = -y1, y1
        Y[rest, p], Y[p, rest] = -y2, y2
        Y[k, p] = c * (-ia) + g1 @ Z @ g2
        Y[p, k] = -Y[k, p]
    return Y


@pytest.mark.parametrize("n,ne", [(16, 8), (10, 4), (8, 8)])
def test_weighted_backward_pass_gives_weighted_inverse(n, ne):
    """One backward pass over the shared steps, started from sum_k c_k Z_k with the
    constants scaled by sum_k c_k, equals sum_k c_k A_k^{-1} (the adjoint's block form)."""
    rng = np.random.default_rng(200 + n + ne)
    Q = synth.haar_orthogonal(rng, 2 * n, 3)
    b = synth.parity_consistent_bits(rng, Q)  # parity -1 makes B singular when ne = n
    Phi = synth.walkers(rng, n, ne, 1)[0]
    D = node_D(n, ne)
    nodes = np.exp(-1j * np.array([0.3, 1.4, 2.6]))
    cs = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    for p in range(3):
        B, _, _ = orc.pair_matrices(Q[p], b[p], Phi)
        r = shared_elimination(B, ne)
        assert r is not None
        _, S, _ = r
        m = B.shape[0]
        d2 = m - ne
        Zc = sum(c * np.linalg.inv(S + z * D[ne:, ne:]) for c, z in zip(cs, nodes)) if d2 else np.zeros((0, 0))
        got = backward_block(B, ne, Zc, cs.sum())
        ref = sum(c * np.linalg.inv(B + z * D) for c, z in zip(cs, nodes))
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("n,ne", [(16, 8), (12, 4)])
def test_block_form_traces(n, ne):
    """The local-energy kernel's traces from the block form of A_k^{-1}:
    with E = P^-1 B_oe, F = [-E; I], W = A'F, G = F^T W, H = -W_o^T P^-1 W_o,
    tr(A_k^-1 A') = tr(P^-1 A'_oo) + tr(Z_k G) and
    tr((A_k^-1 A')^2) = tr((P^-1 A'_oo)^2) + 2 tr(Z_k H) + tr((Z_k G)^2)."""
    rng = np.random.default_rng(300 + n + ne)
    Q = synth.haar_orthogonal(rng, 2 * n, 2)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 1)[0]
    D = node_D(n, ne)
    B, _, _ = orc.pair_matrices(Q[0], b[0], Phi)
    m = B.shape[0]
    X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Ap = X - X.T
    Pinv = np.linalg.inv(B[:ne, :ne])
    E = Pinv @ B[:ne, ne:]
    S0 = B[ne:, ne:] + B[:ne, ne:].T @ E
    W = -Ap[:, :ne] @ E + Ap[:, ne:]
    G = -E.T @ W[:ne] + W[ne:]
    H = -W[:ne].T @ (Pinv @ W[:ne])
    PA = Pinv @ Ap[:ne, :ne]
    for z in np.exp(-1j * np.array([0.3, 1.4, 2.6])):
        Ai = np.linalg.inv(B + z * D)
        Z = np.linalg.inv(S0 + z * D[ne:, ne:])
        t1, t2 = np.trace(Ai @ Ap), np.trace(Ai @ Ap @ Ai @ Ap)
        b1 = np.trace(PA) + np.trace(Z @ G)
        b2 = np.trace(PA @ PA) + 2 * np.trace(Z @ H) + np.trace(Z @ G @ Z @ G)
        assert abs(b1 - t1) <= 1e-10 * max(1.0, abs(t1))
        assert abs(b2 - t2) <= 1e-10 * max(1.0, abs(t2))


def J_matrix(n):
    J = np.zeros((2 * n, 2 * n))
    for k in range(n):
        J[2 * k, 2 * k + 1], J[2 * k + 1, 2 * k] = 1.0, -1.0
    return J


@pytest.mark.parametrize("n,ne", [(16, 8), (12, 6), (16, 16), (10, 2)])
def test_energy_snapshot_product_once_per_pair(n, ne):
    """The local-energy kernel never forms X' = (K ell) Q'^T: with M^T = Q'^T J X^T, built
    once per pair, X' J X^T = (K ell) M^T and A' = X' J X^T + X J X'^T is (K ell) M^T minus
    its transpose.  Restates the kernel's index formulas (complexified snapshot rows
    Qt[c][k] = Q'[c][2k] - i Q'[c][2k+1], the rows of X for empty modes (Re T_j, -Im T_j))
    and compares with the definition formed by plain matrix products."""
    rng = np.random.default_rng(400 + n + ne)
    m, n2 = 2 * n - ne, 2 * n
    Qp = synth.haar_orthogonal(rng, n2, 1)[0]               # Q' (real)
    Qt = Qp[:, 0::2] - 1j * Qp[:, 1::2]                      # 2n x n
    Ts = rng.standard_normal((n, n2)) + 1j * rng.standard_normal((n, n2))
    X = np.zeros((m, n2), complex)
    X[:ne] = Ts[:ne]
    for r in range(m - ne):
        X[ne + r] = -Ts[ne + r // 2].imag if r & 1 else Ts[ne + r // 2].real
    Ko = rng.standard_normal((m, n2)) + 1j * rng.standard_normal((m, n2))  # K ell
    J = J_matrix(n)
    Xp = Ko @ Qp.T
    ref = Xp @ J @ X.T + X @ J @ Xp.T
    # the kernel's Mt[b][mu] = sum_k Q'[2k][mu] X[b][2k+1] - Q'[2k+1][mu] X[b][2k]
    Mt = np.zeros((m, n2), complex)
    for mu in range(n2):
        kq, odd = mu >> 1, mu & 1
        q0 = -Qt[0::2, kq].imag if odd else Qt[0::2, kq].real      # Q'[2k][mu]
        q1 = -Qt[1::2, kq].imag if odd else Qt[1::2, kq].real      # Q'[2k+1][mu]
        Mt[:, mu] = X[:, 1::2] @ q0 - X[:, 0::2] @ q1
    assert np.all(Mt[ne:].imag == 0)  # real rows for the empty modes
    N = Ko @ Mt.T
    got = N - N.T
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(Mt.T - Qp.T @ J @ X.T).max() <= 1e-12 * np.abs(Mt).max()
