"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against the mathematics or an independent
construction: closed forms, textbook identities, a Fock-space brute force of
the estimator's definition, an exact group average, and exact finite
differences.  ``test_planted_mistakes_are_caught`` rebuilds the oracle with
each planted mistake and confirms that these pins fail for it.
"""
from __future__ import annotations

import itertools
import os
from math import comb

import numpy as np
import pytest

import oracle.oracle as orc
from fock_brute import Fock, channel_weights, pfaffian_by_matchings
from paper_2506_22408_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_skew(rng, m):
    A = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    return A - A.T


# ------------------------------------------------------------- Pfaffian


def test_pfaffian_4x4_closed_form():
    rng = np.random.default_rng(10)
    for _ in range(5):
        A = rand_skew(rng, 4)
        ref = A[0, 1] * A[2, 3] - A[0, 2] * A[1, 3] + A[0, 3] * A[1, 2]
        assert abs(orc.pfaffian(A) - ref) <= 1e-13 * abs(ref)


@pytest.mark.parametrize("m", [2, 4, 6, 8])
def test_pfaffian_perfect_matchings(m):
    rng = np.random.default_rng(11 + m)
    A = rand_skew(rng, m)
    ref = pfaffian_by_matchings(A)
    assert abs(orc.pfaffian(A) - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("m", [2, 6, 12, 24, 36])
def test_pfaffian_squared_is_determinant(m):
    rng = np.random.default_rng(20 + m)
    A = rand_skew(rng, m)
    pf = orc.pfaffian(A)
    sign, logdet = np.linalg.slogdet(A)
    det = sign * np.exp(logdet)
    assert abs(pf * pf - det) <= 1e-10 * abs(det)


def test_pfaffian_block_canonical_and_congruence():
    rng = np.random.default_rng(30)
    m = 10
    a = rng.standard_normal(m // 2) + 1j * rng.standard_normal(m // 2)
    D = np.zeros((m, m), complex)
    for i in range(m // 2):
        D[2 * i, 2 * i + 1] = a[i]
        D[2 * i + 1, 2 * i] = -a[i]
    assert abs(orc.pfaffian(D) - np.prod(a)) <= 1e-13 * abs(np.prod(a))
    X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    A = rand_skew(rng, m)
    lhs = orc.pfaffian(X.T @ A @ X)
    rhs = np.linalg.det(X) * orc.pfaffian(A)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)
    # a permutation congruence of the canonical form: pf = sign(perm) * prod(a)
    perm = rng.permutation(m)
    Pm = np.eye(m)[:, perm]
    sgn = np.linalg.det(Pm)
    assert abs(orc.pfaffian(Pm.T @ D @ Pm) - sgn * np.prod(a)) <= 1e-13 * abs(np.prod(a))


@pytest.mark.parametrize("m", [4, 8, 12])
def test_pfaffian_derivative_equations(m):
    """Eqs. (Pfaffian_der) and (Pfaffian_2nd_der), on which the gradient and local-energy
    kernels are built: for A(t) = A + t A' + t^2 A''/2,
        d pf = (pf/2) tr(A^-1 A'),
        d^2 pf = (pf/2) [tr(A^-1 A'') - tr(A^-1 A' A^-1 A') + tr(A^-1 A')^2 / 2].
    pf(A(t)) is a polynomial of degree <= m in t, so its first two Taylor coefficients
    follow exactly from the oracle's Pfaffian at K > m points of a circle (inverse DFT)."""
    rng = np.random.default_rng(40 + m)
    A, A1, A2 = rand_skew(rng, m), rand_skew(rng, m), rand_skew(rng, m)
    K, r = m + 3, 0.25
    ts = r * np.exp(2j * np.pi * np.arange(K) / K)
    vals = np.array([orc.pfaffian(A + t * A1 + 0.5 * t * t * A2) for t in ts])
    coef = np.array([np.sum(vals * np.exp(-2j * np.pi * np.arange(K) * x / K)) / K / r**x for x in range(3)])
    pf = orc.pfaffian(A)
    Ai = np.linalg.inv(A)
    t1 = np.trace(Ai @ A1)
    d1 = 0.5 * pf * t1
    d2 = 0.5 * pf * (np.trace(Ai @ A2) - np.trace(Ai @ A1 @ Ai @ A1) + 0.5 * t1 * t1)
    assert abs(coef[0] - pf) <= 1e-10 * abs(pf)
    assert abs(coef[1] - d1) <= 1e-9 * abs(pf) * np.abs(t1).max()
    assert abs(2 * coef[2] - d2) <= 1e-8 * abs(d2)
    # a plausible slip in the second-order formula (the squared first-order term left out)
    # is far outside that bound
    assert abs(2 * coef[2] - 0.5 * pf * (np.trace(Ai @ A2) - np.trace(Ai @ A1 @ Ai @ A1))) > 1e-3 * abs(d2)


def test_pfaffian_degenerate():
    rng = np.random.default_rng(31)
    A = rand_skew(rng, 6)
    A[:, 3] = 0
    A[3, :] = 0
    assert orc.pfaffian(A) == 0
    assert orc.pfaffian(np.zeros((0, 0))) == 1
    assert orc.pfaffian(rand_skew(rng, 5)) == 0


# ---------------------------------------------------- walker and snapshot


def test_walker_qr_and_snapshot_invariants():
    rng = np.random.default_rng(40)
    for n, ne in [(4, 2), (8, 4), (16, 8), (24, 12)]:
        Phi = rng.standard_normal((n, ne)) + 1j * rng.standard_normal((n, ne))
        U, R = orc.walker_qr(Phi)
        assert np.abs(U[:, :ne] @ R - Phi).max() < 1e-13 * np.abs(Phi).max() * n
        assert np.abs(U.conj().T @ U - np.eye(n)).max() < 1e-13
        assert np.abs(np.tril(R, -1)).max() == 0
        Q = synth.haar_orthogonal(rng, 2 * n, 1)[0]
        b = synth.uniform_bits(rng, n, 1)[0]
        G = orc.snapshot_G(Q, b)
        # Q^T C_b Q is real skew-symmetric and orthogonal: G^T = -G, G^2 = -I
        assert np.abs(G + G.T).max() < 1e-14
        assert np.abs(G @ G + np.eye(2 * n)).max() < 1e-12
        # Q = I gives back the covariance of |b> (SI item 2: +(-1)^{b_j} upper right)
        G0 = orc.snapshot_G(np.eye(2 * n), b)
        for j in range(n):
            assert G0[2 * j, 2 * j + 1] == (-1.0) ** b[j]


def test_selection_shape():
    for n in range(2, 9):
        for ne in range(2, n + 1, 2):
            idx = orc.selection(n, ne)
            assert len(idx) == 2 * n - ne
            assert list(idx) == sorted(idx)


# --------------------------------------------- estimator vs brute force


def _fock_case(rng, n, ne, det_sign=None, scaled=True):
    Q = synth.haar_orthogonal(rng, 2 * n, 1)[0]
    if det_sign is not None and np.sign(np.linalg.det(Q)) != det_sign:
        Q[:, 0] *= -1
    b = synth.uniform_bits(rng, n, 1)[0]
    Phi = synth.walkers(rng, n, ne, 1)[0]
    if scaled:
        Phi = Phi @ (rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne)))
    return Q, b, Phi


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7])
def test_estimator_matches_fock_bruteforce(n):
    """o_p of the Pfaffian route equals 2 tr(M^{-1}(|phi><0|) rho_{Q,b}) computed in Fock space."""
    rng = np.random.default_rng(100 + n)
    F = Fock(n)
    for ne in range(2, n + 1, 2):
        for trial in range(4 if n <= 5 else 2):
            Q, b, Phi = _fock_case(rng, n, ne, det_sign=(1 if trial % 2 == 0 else -1))
            psi = F.shadow_state(Q, b)
            ob = F.estimator(Phi, psi)
            of, c, scale = orc.pair(Q, b, Phi)
            # parity-forbidden pairs are zero up to rounding on both sides: bound by the walker's norm
            mag = max(scale, abs(np.linalg.det(Phi.conj().T @ Phi)) ** 0.5)
            assert abs(of - ob) <= 1e-10 * mag, (n, ne, trial, of, ob)


@pytest.mark.slow
def test_estimator_matches_fock_bruteforce_n8():
    rng = np.random.default_rng(108)
    F = Fock(8)
    for ne in (4, 6):
        Q, b, Phi = _fock_case(rng, 8, ne, det_sign=1)
        pi = np.sign(np.linalg.det(Q)) * (-1) ** int(b.sum())
        if pi < 0:
            b[0] ^= 1
        of, c, scale = orc.pair(Q, b, Phi)
        ob = F.estimator(Phi, F.shadow_state(Q, b))
        assert abs(of - ob) <= 1e-10 * scale


def test_worked_example_closed_form():
    """n = 2, eta = 2, Phi = I, b = 00, Q a (gamma_2, gamma_3) rotation: o = 3 i sin(theta)
    (derivation in tests/golden/worked_n2_rotation.txt)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "worked_n2_rotation.txt"))
    F = Fock(2)
    for th, re, im in rows:
        c, s = np.cos(th), np.sin(th)
        Q = np.array([[1, 0, 0, 0], [0, c, s, 0], [0, -s, c, 0], [0, 0, 0, 1.0]])
        b = np.zeros(2, np.uint8)
        o, _, _ = orc.pair(Q, b, np.eye(2, dtype=complex))
        assert abs(o - complex(re, im)) < 1e-13
        assert abs(F.estimator(np.eye(2, dtype=complex), F.shadow_state(Q, b)) - complex(re, im)) < 1e-13


# ------------------------------------------- polynomial structure pins


@pytest.mark.parametrize("n,ne", [(4, 2), (6, 4), (8, 4), (12, 6), (16, 8), (16, 4), (20, 10), (24, 12)])
def test_coefficient_structure(n, ne):
    """c_x = 0 for x < ne/2 (D vanishes on occupied rows), c_{n-x} = pi c_x with
    pi = det Q (-1)^{|b|} (parity of the pure Gaussian snapshot state), and
    parity-forbidden pairs are exactly zero because the weights are symmetric."""
    rng = np.random.default_rng(200 + n + ne)
    for trial in range(4):
        Q, b, Phi = _fock_case(rng, n, ne, det_sign=(1 if trial < 2 else -1))
        pi = np.sign(np.linalg.det(Q)) * (-1) ** int(b.sum())
        o, c, scale = orc.pair(Q, b, Phi)
        cmax = np.abs(c).max()
        assert np.abs(c[: ne // 2]).max() <= 1e-13 * cmax
        x = np.arange(ne // 2, n - ne // 2 + 1)
        assert np.abs(c[n - x] - pi * c[x]).max() <= 1e-12 * cmax
        w = np.array([comb(2 * n, 2 * k) / comb(n, k) for k in range(n + 1)])
        assert np.allclose(w, w[::-1])
        if pi < 0:
            assert abs(o) <= 1e-12 * scale


def test_parity_forbidden_is_exactly_zero_in_fock_space():
    rng = np.random.default_rng(300)
    for n, ne in [(3, 2), (4, 2), (4, 4), (5, 4)]:
        F = Fock(n)
        for _ in range(3):
            Q, b, Phi = _fock_case(rng, n, ne)
            pi = np.sign(np.linalg.det(Q)) * (-1) ** int(b.sum())
            if pi > 0:
                b[0] ^= 1
            assert abs(F.estimator(Phi, F.shadow_state(Q, b))) < 1e-12


@pytest.mark.parametrize("n,ne", [(6, 2), (8, 4), (12, 6), (16, 8)])
def test_interpolation_dft_vs_chebyshev(n, ne):
    """Roots-of-unity DFT and the paper's Chebyshev nodes with a least-squares
    Vandermonde fit give the same coefficients."""
    rng = np.random.default_rng(400 + n)
    Q, b, Phi = _fock_case(rng, n, ne, det_sign=1)
    o1, c1, sc = orc.pair(Q, b, Phi, mode=orc.INTERP_ROOTS)
    o2, c2, _ = orc.pair(Q, b, Phi, mode=orc.INTERP_CHEBYSHEV)
    o3, c3, _ = orc.pair(Q, b, Phi, mode=orc.INTERP_ROOTS, nodes=n - ne // 2 + 1)
    cm = np.abs(c1).max()
    assert np.abs(c1 - c3).max() <= 1e-12 * cm
    assert np.abs(c1 - c2).max() <= 1e-8 * cm  # monomial Vandermonde on [-1, 1] loses digits
    assert abs(o1 - o3) <= 1e-11 * sc


def test_walker_scaling_invariance():
    """<Psi_T|phi> for Phi X is det X times that of Phi (the walker is a determinant)."""
    rng = np.random.default_rng(500)
    n, ne = 8, 4
    Q = synth.haar_orthogonal(rng, 2 * n, 16)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 1)
    X = rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne))
    o1, p1, s1, _ = orc.overlap(Phi, Q, b, per_pair=True)
    o2, p2, s2, _ = orc.overlap(Phi @ X, Q, b, per_pair=True)
    d = np.linalg.det(X)
    assert np.abs(p2 - d * p1).max() <= 1e-11 * np.abs(d) * s1.max()


# ------------------------------------------ unbiasedness (exact averages)


def signed_permutation_group(N):
    for perm in itertools.permutations(range(N)):
        for signs in itertools.product((-1.0, 1.0), repeat=N):
            Q = np.zeros((N, N))
            Q[np.arange(N), perm] = signs
            yield Q


def _born_table(F, group, Psi):
    """All (Q, b) with non-zero Born weight p(b|Q) for the group, flattened."""
    n = F.n
    prob = F.born_probabilities(group, Psi)
    bits = np.array([[(x >> j) & 1 for j in range(n)] for x in range(1 << n)], np.uint8)
    g_idx, x_idx = np.nonzero(prob > 1e-15)
    return group[g_idx], bits[x_idx], prob[g_idx, x_idx]


def _random_eta_state(rng, F, ne):
    """A random normalised state with exactly ne particles (not a Slater determinant)."""
    v = np.zeros(F.dim, complex)
    for x in range(F.dim):
        if bin(x).count("1") == ne:
            v[x] = rng.standard_normal() + 1j * rng.standard_normal()
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n", [2, 3])
def test_exact_unbiasedness_signed_permutation_group(n):
    """Averaged over the whole signed-permutation group of O(2n) with Born weights
    p(b|Q) = <Psi|rho_{Q,b}|Psi>, Psi = (|0> + |Psi_T>)/sqrt2, the estimator equals
    <Psi_T|phi> exactly -- this pins the channel weights, kappa and all phases."""
    rng = np.random.default_rng(600 + n)
    ne = 2
    F = Fock(n)
    PsiT = _random_eta_state(rng, F, ne)
    Psi = (F.vac + PsiT) / np.sqrt(2)
    Phi = synth.walkers(rng, n, ne, 1)[0] @ (rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne)))
    exact = np.vdot(PsiT, F.slater(Phi))
    group = np.array(list(signed_permutation_group(2 * n)))
    Qs, bs, ws = _born_table(F, group, Psi)
    _, per, _, _ = orc.overlap(Phi[None], Qs, bs, per_pair=True)
    est = np.sum(ws * per[0]) / len(group)
    assert abs(est - exact) <= 1e-12 * max(1.0, abs(exact)), (est, exact)


def test_channel_eigenvalues_signed_permutations():
    """The measure-and-prepare channel of the signed-permutation ensemble (n = 2)
    scales gamma_S by lambda_{|S|/2} = C(n,k)/C(2n,2k)."""
    n = 2
    F = Fock(n)
    lam = channel_weights(n)
    group = list(signed_permutation_group(2 * n))
    states = {}
    for gi, Q in enumerate(group):
        for x in range(1 << n):
            b = np.array([(x >> j) & 1 for j in range(n)], np.uint8)
            states[(gi, x)] = F.shadow_state(Q, b)
    for S in [(0, 1), (0, 2), (1, 3), (0, 1, 2, 3)]:
        G = np.eye(F.dim, dtype=complex)
        for mu in S:
            G = G @ F.gamma[mu]
        out = np.zeros_like(G)
        for (gi, x), psi in states.items():
            rho = np.outer(psi, psi.conj())
            out += np.trace(G @ rho) * rho
        out /= len(group)
        assert np.abs(out - lam[len(S) // 2] * G).max() < 1e-12


@pytest.mark.slow
def test_haar_born_sampling_converges_to_slater_overlap():
    """Literal shadow protocol at n = 4: Haar Q, b drawn from the Born rule,
    snapshot mean within 4 standard errors of det(Psi_T^dag Phi)."""
    rng = np.random.default_rng(700)
    n, ne, P = 4, 2, 20000
    F = Fock(n)
    Psi_orb = synth.walkers(rng, n, ne, 1)[0]
    Psi_orb /= np.linalg.norm(Psi_orb[:, 0])
    Psi_orb, _ = np.linalg.qr(Psi_orb)
    PsiT = F.slater(Psi_orb)
    PsiT /= np.linalg.norm(PsiT)
    Psi = (F.vac + PsiT) / np.sqrt(2)
    Phi = synth.walkers(rng, n, ne, 1)[0]
    exact = np.linalg.det(Psi_orb.conj().T @ Phi)
    assert abs(np.vdot(PsiT, F.slater(Phi)) - exact) < 1e-12
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    prob = np.clip(F.born_probabilities(Q, Psi), 0.0, None)
    bs = np.zeros((P, n), np.uint8)
    for p in range(P):
        x = rng.choice(1 << n, p=prob[p] / prob[p].sum())
        bs[p] = [(x >> j) & 1 for j in range(n)]
    ov, per, _, _ = orc.overlap(Phi[None], Q, bs, per_pair=True)
    se = np.std(per[0]) / np.sqrt(P)
    assert abs(ov[0] - exact) < 4 * se, (ov[0], exact, se)


# ----------------------------------------------------- gradient pins


def test_gradient_exact_linearity_and_euler():
    rng = np.random.default_rng(800)
    n, ne, P = 6, 4, 24
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 2)
    ov, g, _ = orc.overlap_grad(Phi, Q, b)
    ov2, _, _, _ = orc.overlap(Phi, Q, b)
    assert np.allclose(ov, ov2, rtol=0, atol=1e-13 * np.abs(ov).max())
    for w in range(2):
        # Euler / antisymmetry identity g^T Phi = O I (O is multilinear and alternating in the columns)
        M = g[w].T @ Phi[w]
        assert np.abs(M - ov[w] * np.eye(ne)).max() <= 1e-10 * np.abs(g[w]).max() * np.abs(Phi[w]).max() * n
        # exact t-polynomial of O(Phi + t E) recovered by a DFT on a circle (degree <= ne)
        E = rng.standard_normal((n, ne)) + 1j * rng.standard_normal((n, ne))
        K, r = ne + 1, 0.3
        ts = r * np.exp(2j * np.pi * np.arange(K) / K)
        vals = np.array([orc.overlap((Phi[w] + t * E)[None], Q, b)[0][0] for t in ts])
        c1 = np.sum(vals * np.exp(-2j * np.pi * np.arange(K) / K)) / K / r
        assert abs(c1 - np.sum(g[w] * E)) <= 1e-9 * np.abs(g[w]).sum() * np.abs(E).max()
        # holomorphic: D_{iE} = i D_E (central difference, exact for a polynomial up to O(h^2))
        h = 1e-4
        dE = (orc.overlap((Phi[w] + h * E)[None], Q, b)[0][0] - orc.overlap((Phi[w] - h * E)[None], Q, b)[0][0]) / (2 * h)
        diE = (orc.overlap((Phi[w] + 1j * h * E)[None], Q, b)[0][0]
               - orc.overlap((Phi[w] - 1j * h * E)[None], Q, b)[0][0]) / (2 * h)
        assert abs(diE - 1j * dE) <= 1e-6 * abs(dE)
        assert abs(dE - np.sum(g[w] * E)) <= 1e-6 * abs(dE)


def test_force_bias_exact_for_slater_trial():
    """With the exact signed-permutation group average (n = 3), the shadow overlap
    and gradient are exact, so the force bias equals i tr(L Phi (Psi^dag Phi)^{-1} Psi^dag),
    and, for complex operators without symmetry (so that L and L^T differ), the Fock-space
    mixed estimate i <Psi_T| sum_pq L_pq a_p^dag a_q |phi> / <Psi_T|phi> of Eq. (force_bias)."""
    rng = np.random.default_rng(900)
    n, ne = 3, 2
    F = Fock(n)
    Psi_orb, _ = np.linalg.qr(rng.standard_normal((n, ne)) + 1j * rng.standard_normal((n, ne)))
    PsiT = F.slater(Psi_orb)
    Psi = (F.vac + PsiT) / np.sqrt(2)
    Phi = synth.walkers(rng, n, ne, 1)[0]
    walkers = [Phi]
    for k in range(n):
        for j in range(ne):
            P2 = Phi.copy()
            P2[:, j] = 0
            P2[k, j] = 1
            walkers.append(P2)
    walkers = np.array(walkers)
    group = np.array(list(signed_permutation_group(2 * n)))
    Qs, bs, ws = _born_table(F, group, Psi)
    _, per, _, _ = orc.overlap(walkers, Qs, bs, per_pair=True)
    est = per @ ws / len(group)
    O = est[0]
    g = est[1:].reshape(n, ne)
    S = Psi_orb.conj().T @ Phi
    assert abs(O - np.linalg.det(S)) < 1e-12
    L = synth.cholesky_vectors(rng, n, 5)
    xb = orc.force_bias(L.astype(complex), Phi[None], np.array([O]), g[None], sqrt_dt=0.0)[0]
    Gf = Phi @ np.linalg.inv(S) @ Psi_orb.conj().T
    ref = np.array([1j * np.trace(L[c] @ Gf) for c in range(5)])
    assert np.abs(xb - ref).max() < 1e-11
    xb2 = orc.force_bias(L.astype(complex), Phi[None], np.array([O]), g[None], sqrt_dt=0.1)[0]
    assert np.allclose(xb2, -0.1 * ref, atol=1e-12)
    Lc = rng.standard_normal((3, n, n)) + 1j * rng.standard_normal((3, n, n))
    xc = orc.force_bias(Lc, Phi[None], np.array([O]), g[None], sqrt_dt=0.0)[0]
    phi = F.slater(Phi)
    Ofock = np.vdot(PsiT, phi)
    for c in range(3):
        v = sum(Lc[c, p, q] * (F.a[p].conj().T @ (F.a[q] @ phi)) for p in range(n) for q in range(n))
        assert abs(xc[c] - 1j * np.vdot(PsiT, v) / Ofock) < 1e-11
        assert abs(xc[c] - 1j * np.trace(Lc[c].T @ Gf)) > 1e-3  # the transposed operator differs


# ------------------------------- shadow RDMs (Supplementary "Reduced Density Matrices")


def _rotated_ops(F, R):
    """Rotated Majoranas g~_mu = sum_nu R_{mu nu} g_nu and modes a~_p = (g~_2p + i g~_2p+1)/2."""
    N2 = 2 * F.n
    g = F.gamma if R is None else [sum(R[m, v] * F.gamma[v] for v in range(N2)) for m in range(N2)]
    a = [0.5 * (g[2 * p] + 1j * g[2 * p + 1]) for p in range(F.n)]
    return g, a


def _exact_rdm_quantities(F, Psi, R):
    g, a = _rotated_ops(F, R)
    N2 = 2 * F.n
    E2 = np.array([[np.vdot(Psi, g[m] @ (g[v] @ Psi)) if m != v else 0.0 for v in range(N2)] for m in range(N2)])
    E4 = np.array([np.vdot(Psi, g[i] @ g[j] @ g[k] @ g[l] @ Psi) for i, j, k, l in itertools.combinations(range(N2), 4)])
    D = np.array([[np.vdot(Psi, a[p].conj().T @ (a[q] @ Psi)) for q in range(F.n)] for p in range(F.n)])
    return E2, E4, D


def _rdm_group_check(orc_v, n, rng, rotate) -> float:
    """Largest deviation of the Born-weighted signed-permutation-group average of the
    shadow estimates from the exact expectation values of a random N-particle state."""
    F = Fock(n)
    Psi = _random_eta_state(rng, F, n - 1)
    group = np.array(list(signed_permutation_group(2 * n)))
    Qs, bs, ws = _born_table(F, group, Psi)
    R = synth.haar_orthogonal(rng, 2 * n, 1)[0] if rotate else None
    est = orc_v.shadow_rdm(Qs, bs, w=ws, R=R, deg4=True)
    E2, E4, D = _exact_rdm_quantities(F, Psi, R)
    err = max(np.abs(1j * est["gam2"] - E2).max(), np.abs(est["gam4"] - E4).max(), np.abs(est["rdm1"] - D).max(),
              abs(est["npart"] - np.trace(D).real))
    if not rotate:
        err = max(err, abs(est["npart"] - (n - 1)))
    return err


@pytest.mark.parametrize("n", [2, 3])
@pytest.mark.parametrize("rotate", [False, True])
def test_shadow_rdm_exact_group_average(n, rotate):
    """Averaged over the whole signed-permutation group of O(2n) with Born weights, the
    shadow estimates of <g_S> (|S| = 2, 4), of the 1-RDM and of the particle number equal
    the exact expectation values of the measured (n-1)-particle state, computed with
    Fock-space matrices; with a rotation R the same holds for g~ = R g.  This pins the
    weights C(2n,|S|)/C(n,|S|/2), the Pfaffian signs and the Majorana-to-mode map."""
    rng = np.random.default_rng(700 + 10 * n + rotate)
    assert _rdm_group_check(orc, n, rng, rotate) <= 1e-12


def test_shadow_rdm_single_snapshot_closed_form():
    """One snapshot: gam2 is (2n-1) times the rotated covariance Q^T C_b Q, and a
    product of four distinct Majoranas gets C(2n,4)/C(n,2) times minus the Pfaffian
    of the 4 x 4 block."""
    rng = np.random.default_rng(77)
    n = 4
    Q = synth.haar_orthogonal(rng, 2 * n, 1)
    b = synth.uniform_bits(rng, n, 1)
    G = Q[0].T @ orc.covariance(n, b[0]) @ Q[0]
    est = orc.shadow_rdm(Q, b, deg4=True)
    off = ~np.eye(2 * n, dtype=bool)
    assert np.abs(est["gam2"][off] - (2 * n - 1) * G[off]).max() < 1e-12
    K4 = comb(2 * n, 4) / comb(n, 2)
    for t, (i, j, k, l) in enumerate(itertools.combinations(range(2 * n), 4)):
        blk = G[np.ix_([i, j, k, l], [i, j, k, l])]
        pf = pfaffian_by_matchings(blk)
        assert abs(est["gam4"][t] - K4 * (-pf)) < 1e-11


# ------------------- virtual-correlation-energy transform (Supplementary "VCE Derivation")


def _embed_trial(nc, chi, NB):
    """Full-space orbital matrix of Xi_c (x) chi (x) 0_v: core unit vectors, then chi."""
    na, nea = chi.shape
    Psi = np.zeros((NB, nc + nea), complex)
    Psi[:nc, :nc] = np.eye(nc)
    Psi[nc:nc + na, nc:] = chi
    return Psi


@pytest.mark.parametrize("NB,nc,na,nea", [(14, 3, 6, 2), (20, 0, 8, 4), (12, 5, 4, 0), (30, 10, 8, 4),
                                          (9, 4, 5, 5), (40, 24, 16, 8)])
def test_vce_transform_reproduces_full_space_determinant(NB, nc, na, nea):
    """For Slater trials the full-space overlap is det(Psi^dag Phi); the transform must
    give factor * det(chi^dag act) for every active chi, and the virtual rows must drop out."""
    rng = np.random.default_rng(NB * 100 + nc)
    ne = nc + nea
    Phi = rng.standard_normal((NB, ne)) + 1j * rng.standard_normal((NB, ne))
    act, f = orc.vce_transform(Phi, nc, na, nea)
    for _ in range(3):
        chi = rng.standard_normal((na, nea)) + 1j * rng.standard_normal((na, nea))
        full = np.linalg.det(_embed_trial(nc, chi, NB).conj().T @ Phi)
        got = f * np.linalg.det(chi.conj().T @ act)
        assert abs(got - full) <= 1e-12 * max(1.0, abs(full))
    Phi2 = Phi.copy()
    Phi2[nc + na:] = rng.standard_normal(Phi2[nc + na:].shape)  # virtual rows
    act2, f2 = orc.vce_transform(Phi2, nc, na, nea)
    assert np.allclose(act2, act, rtol=0, atol=1e-14 * np.abs(act).max(initial=1.0)) and abs(f2 - f) <= 1e-14 * abs(f)


def test_vce_transform_multi_determinant_two_spins():
    """Unrestricted walker, multi-determinant active trial sum_i c_i chi_i^a chi_i^b: the
    full-space overlap equals f_a f_b sum_i c_i det(chi_i^a^dag act_a) det(chi_i^b^dag act_b)."""
    rng = np.random.default_rng(17)
    NB, nc, na, nea = 18, 4, 6, 3
    Pa = rng.standard_normal((NB, nc + nea)) + 1j * rng.standard_normal((NB, nc + nea))
    Pb = rng.standard_normal((NB, nc + nea)) + 1j * rng.standard_normal((NB, nc + nea))
    aa, fa = orc.vce_transform(Pa, nc, na, nea)
    ab, fb = orc.vce_transform(Pb, nc, na, nea)
    full = via = 0.0
    for _ in range(4):
        c = rng.standard_normal() + 1j * rng.standard_normal()
        xa = rng.standard_normal((na, nea)) + 1j * rng.standard_normal((na, nea))
        xb = rng.standard_normal((na, nea)) + 1j * rng.standard_normal((na, nea))
        full += c * np.linalg.det(_embed_trial(nc, xa, NB).conj().T @ Pa) * np.linalg.det(
            _embed_trial(nc, xb, NB).conj().T @ Pb)
        via += c * np.linalg.det(xa.conj().T @ aa) * np.linalg.det(xb.conj().T @ ab)
    assert abs(fa * fb * via - full) <= 1e-12 * abs(full)


def test_vce_transform_fock_space_general_active_state():
    """Fock space of NB = 7 modes: trial a^dag_0 .. a^dag_{nc-1} |Psi_act> with a random
    (non-Slater) nea-particle active state; <trial|phi> = factor <Psi_act|act>."""
    rng = np.random.default_rng(23)
    NB, nc, na, nea = 7, 2, 4, 2
    F, Fa = Fock(NB), Fock(na)
    Phi = rng.standard_normal((NB, nc + nea)) + 1j * rng.standard_normal((NB, nc + nea))
    act, f = orc.vce_transform(Phi, nc, na, nea)
    psi_a = _random_eta_state(rng, Fa, nea)
    emb = np.zeros(F.dim, complex)  # active modes nc..nc+na-1 of the full space, rest empty
    for x in range(Fa.dim):
        emb[x << nc] = psi_a[x]
    # Jordan-Wigner signs: the embedding shifts every active mode past nc empty modes
    # (no sign); the core creators act after it
    trial = emb
    for c in reversed(range(nc)):
        trial = F.a[c].conj().T @ trial
    full = np.vdot(trial, F.slater(Phi))
    act_ov = np.vdot(psi_a, Fa.slater(act))
    assert abs(f * act_ov - full) <= 1e-12 * max(1.0, abs(full))


# ----------------------- local-energy terms (Eqs. force_bias_diff, energy_tb_diff)


@pytest.mark.parametrize("n", [2, 3])
def test_local_energy_terms_exact_group_average(n):
    """Averaged over the signed-permutation group with Born weights for
    (|0> + |Psi_T>)/sqrt2, the shadow estimates of <Psi_T|hhat|phi>/<Psi_T|phi> and
    sum_gamma <Psi_T|Lhat_gamma Lhat_gamma|phi>/<Psi_T|phi> equal the Fock-space values
    for a non-Slater Psi_T, a non-orthonormal walker and complex one-body operators."""
    rng = np.random.default_rng(800 + n)
    ne = 2
    F = Fock(n)
    PsiT = _random_eta_state(rng, F, ne)
    Psi = (F.vac + PsiT) / np.sqrt(2)
    Phi = synth.walkers(rng, n, ne, 1)[0] @ (rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne)))
    h = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    L = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    group = np.array(list(signed_permutation_group(2 * n)))
    Qs, bs, ws = _born_table(F, group, Psi)
    ov, e1, e2 = orc.local_energy(Phi[None], Qs, bs, L, h=h, w=ws)
    phi = F.slater(Phi)
    op = lambda M: sum(M[p, q] * F.a[p].conj().T @ F.a[q] for p in range(n) for q in range(n))  # noqa: E731
    O = np.vdot(PsiT, phi)
    ref1 = np.vdot(PsiT, op(h) @ phi) / O
    ref2 = sum(np.vdot(PsiT, op(Lg) @ (op(Lg) @ phi)) for Lg in L) / O
    assert abs(ov[0] - O) <= 1e-12 * max(1.0, abs(O))
    assert abs(e1[0] - ref1) <= 1e-11 * max(1.0, abs(ref1))
    assert abs(e2[0] - ref2) <= 1e-11 * max(1.0, abs(ref2))


def _majorana_form(F, L):
    """ell with [Lhat, g_mu] = sum_a ell[mu][a] g_a for Lhat = sum_pq L_pq a_p^dag a_q, by
    projecting the Fock-space commutator onto the Majoranas (tr(g_a g_b) = 2^n delta_ab)."""
    n = F.n
    Lh = sum(L[p, q] * F.a[p].conj().T @ F.a[q] for p in range(n) for q in range(n))
    ell = np.zeros((2 * n, 2 * n), complex)
    for mu in range(2 * n):
        C = Lh @ F.gamma[mu] - F.gamma[mu] @ Lh
        for a in range(2 * n):
            ell[mu, a] = np.trace(F.gamma[a] @ C) / F.dim
    return ell


def test_operator_moves_the_snapshot_not_the_walker():
    """Reading R19 (how lambda enters A in Eqs. energy_tb_diff, Pfaffian_2nd_der): since
    <0| Lhat = 0, e^{lambda Lhat}|phi><0| = e^{lambda Lhat} (|phi><0|) e^{-lambda Lhat}, so the
    pair estimate of the moved walker e^{lambda L} Phi equals that of Phi against the snapshot
    with covariance R G R^T, R = e^{lambda ell}.  For anti-Hermitian L, R is a rotation and
    that snapshot is Q R^T; checked pair by pair with the oracle.  Also pins the closed form
    of ell that the local-energy kernel's preparation uses, for a general complex L:
    ell[2r][2q] = ell[2r+1][2q+1] = (L_qr - L_rq)/2, ell[2r][2q+1] = -i (L_rq + L_qr)/2,
    ell[2r+1][2q] = i (L_rq + L_qr)/2."""
    from scipy.linalg import expm

    rng = np.random.default_rng(950)
    n, ne = 4, 2
    F = Fock(n)
    Lg = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    ell = _majorana_form(F, Lg)
    cf = np.zeros((2 * n, 2 * n), complex)
    for r in range(n):
        for q in range(n):
            cf[2 * r, 2 * q] = cf[2 * r + 1, 2 * q + 1] = (Lg[q, r] - Lg[r, q]) / 2
            cf[2 * r, 2 * q + 1] = -1j * (Lg[r, q] + Lg[q, r]) / 2
            cf[2 * r + 1, 2 * q] = 1j * (Lg[r, q] + Lg[q, r]) / 2
    assert np.abs(ell - cf).max() < 1e-12
    H = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    L = H - H.conj().T  # anti-Hermitian: e^{lambda Lhat} unitary, ell real
    ell = _majorana_form(F, L)
    assert np.abs(ell.imag).max() < 1e-12
    lam = 0.37
    R = expm(lam * ell.real)
    assert np.abs(R @ R.T - np.eye(2 * n)).max() < 1e-12
    Phi = synth.walkers(rng, n, ne, 1)[0]
    Phi_moved = expm(lam * L) @ Phi
    Q = synth.haar_orthogonal(rng, 2 * n, 6)
    b = synth.parity_consistent_bits(rng, Q)
    for p in range(6):
        o_moved, _, sc = orc.pair(Q[p], b[p], Phi_moved)
        o_snap, _, _ = orc.pair(Q[p] @ R.T, b[p], Phi)
        assert abs(o_moved - o_snap) <= 1e-12 * max(sc, 1.0)
        o_wrong, _, _ = orc.pair(Q[p] @ R, b[p], Phi)  # the other rotation sense does not hold
        assert abs(o_moved - o_wrong) > 1e-6 * max(sc, 1.0)


def test_local_energy_one_body_term_matches_gradient():
    """D O[h Phi] = sum_kj g_kj (h Phi)_kj with the oracle's gradient: two routes through
    the same column substitution agree, and e1 equals tr(h G) with G = Phi g^T / O."""
    rng = np.random.default_rng(81)
    n, ne, P = 6, 4, 30
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 2)
    h = synth.cholesky_vectors(rng, n, 1)[0].astype(complex)
    ov, e1, _ = orc.local_energy(Phi, Q, b, h[None] * 0.0, h=h)
    oo, g, _ = orc.overlap_grad(Phi, Q, b)
    for w in range(2):
        Gf = Phi[w] @ g[w].T / oo[w]
        assert abs(e1[w] - np.trace(h @ Gf)) <= 1e-11 * max(1.0, abs(e1[w]))


# ---------------------------------------------- the pins catch mistakes


def _pin_suite_passes(v) -> bool:
    """A compact re-run of the brute-force, closed-form and Pfaffian pins against oracle variant v."""
    rng = np.random.default_rng(1000)
    A = rand_skew(rng, 6)
    if abs(v.pfaffian(A) - pfaffian_by_matchings(A)) > 1e-10 * abs(pfaffian_by_matchings(A)):
        return False
    for n, ne in [(3, 2), (4, 2), (4, 4)]:
        F = Fock(n)
        for trial in range(3):
            Q, b, Phi = _fock_case(rng, n, ne, det_sign=1)
            pi = np.sign(np.linalg.det(Q)) * (-1) ** int(b.sum())
            if pi < 0:
                b[0] ^= 1
            o, _, sc = v.pair(Q, b, Phi)
            ob = F.estimator(Phi, F.shadow_state(Q, b))
            if abs(o - ob) > 1e-9 * max(abs(ob), 1e-12):
                return False
    if _rdm_group_check(v, 2, rng, rotate=False) > 1e-10:
        return False
    # gradient: the Euler / antisymmetry identity g^T Phi = O I
    n, ne, P = 5, 2, 12
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 1)
    ov, g, _ = v.overlap_grad(Phi, Q, b)
    if np.abs(g[0].T @ Phi[0] - ov[0] * np.eye(ne)).max() > 1e-10 * np.abs(g[0]).max() * np.abs(Phi[0]).max() * n:
        return False
    # VCE: factor * det(chi^dag act) is the full-space determinant
    NB, nc, na, nea = 14, 3, 6, 2
    Phv = rng.standard_normal((NB, nc + nea)) + 1j * rng.standard_normal((NB, nc + nea))
    act, f = v.vce_transform(Phv, nc, na, nea)
    chi = rng.standard_normal((na, nea)) + 1j * rng.standard_normal((na, nea))
    full = np.linalg.det(_embed_trial(nc, chi, NB).conj().T @ Phv)
    if abs(f * np.linalg.det(chi.conj().T @ act) - full) > 1e-12 * max(1.0, abs(full)):
        return False
    # force bias for a Slater trial with its exact overlap and gradient
    # (O = det S, S = Psi^dag Phi, dO/dPhi_kj = sum_i conj(Psi_ki) adj(S)_ji) against the
    # Fock-space mixed estimate of i sum_pq L_pq a_p^dag a_q, L without symmetry
    n, ne = 3, 2
    F = Fock(n)
    Psi, _ = np.linalg.qr(rng.standard_normal((n, ne)) + 1j * rng.standard_normal((n, ne)))
    Phs = synth.walkers(rng, n, ne, 1)[0]
    S = Psi.conj().T @ Phs
    O = np.linalg.det(S)
    g = Psi.conj() @ (O * np.linalg.inv(S)).T
    Lc = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    xb = v.force_bias(Lc, Phs[None], np.array([O]), g[None], sqrt_dt=0.0)[0]
    phi, PsiT = F.slater(Phs), F.slater(Psi)
    for c in range(2):
        vphi = sum(Lc[c, p, q] * (F.a[p].conj().T @ (F.a[q] @ phi)) for p in range(n) for q in range(n))
        ref = 1j * np.vdot(PsiT, vphi) / np.vdot(PsiT, phi)
        if abs(xb[c] - ref) > 1e-10 * max(1.0, abs(ref)):
            return False
    # local energy: exact group average at n = 2 against Fock-space values
    n, ne = 2, 2
    F = Fock(n)
    PsiT = _random_eta_state(rng, F, ne)
    Psi2 = (F.vac + PsiT) / np.sqrt(2)
    Phe = synth.walkers(rng, n, ne, 1)[0]
    L = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    group = np.array(list(signed_permutation_group(2 * n)))
    Qs, bs, ws = _born_table(F, group, Psi2)
    ov, _, e2 = v.local_energy(Phe[None], Qs, bs, L, w=ws)
    phi = F.slater(Phe)
    op = lambda M: sum(M[p, q] * F.a[p].conj().T @ F.a[q] for p in range(n) for q in range(n))  # noqa: E731
    ref2 = sum(np.vdot(PsiT, op(Lg) @ (op(Lg) @ phi)) for Lg in L) / np.vdot(PsiT, phi)
    if abs(e2[0] - ref2) > 1e-10 * max(1.0, abs(ref2)):
        return False
    return True


def test_planted_mistakes_are_caught():
    assert _pin_suite_passes(orc.variant(0))
    for k, what in orc.MUTATIONS.items():
        assert not _pin_suite_passes(orc.variant(k)), f"planted mistake {k} ({what}) went unnoticed"
