"""Node plans of the pair term (host logic; no GPU needed).

The kernels form a pair's term as sum_k gamma_k pf(B + w_k D).  With z_k = 1/w_k,
pf(B + w_k D) = q(z_k) / z_k^d, where q(z) = pf(A(z)) / z^{ne/2} is the
polynomial of degree d = n - ne whose coefficients the paper interpolates (the
o_p formula after Eq. b_mat).  A plan is correct when it reproduces

    L(q) = sum_t C(2n, ne + 2t) / C(n, ne/2 + t) q_t

for every q of its class: palindromic q (parity +1 snapshots) for the default
Gauss plan and for the roots-of-unity plan with the parity shortcut, any q for
QCS_FLAG_ALL_NODES.  The weights below come from math.comb, not from the library.
"""
from __future__ import annotations

from math import comb

import numpy as np
import pytest

from paper_2506_22408_gb300 import qcs

SIZES = [(n, ne) for n in range(2, 25) for ne in range(2, n + 1, 2)]


def weights(n, ne):
    d = n - ne
    return np.array([comb(2 * n, ne + 2 * t) / comb(n, ne // 2 + t) for t in range(d + 1)])


def random_q(rng, d, palindromic):
    q = rng.standard_normal(d + 1) + 1j * rng.standard_normal(d + 1)
    if palindromic:
        q = 0.5 * (q + q[::-1])
    return q


def plan_sum(n, ne, q, nodes=0, flags=0):
    w, g = qcs.node_plan(n, ne, nodes, flags)
    d = n - ne
    z = 1.0 / w
    pf = np.polyval(q[::-1], z) / z**d  # what the kernels evaluate at each node
    return np.sum(g * pf), len(w), w


@pytest.mark.parametrize("n,ne", SIZES)
def test_gauss_plan_is_exact_on_palindromic_polynomials(n, ne):
    rng = np.random.default_rng(100 * n + ne)
    d = n - ne
    wt = weights(n, ne)
    for _ in range(4):
        q = random_q(rng, d, palindromic=True)
        got, nev, w = plan_sum(n, ne, q)
        assert abs(got - np.dot(wt, q)) <= 1e-13 * np.dot(wt, np.abs(q))
    D = d // 2 + 1
    assert nev == (D + 1) // 2                     # ceil(D/2) Pfaffians per pair
    assert np.allclose(np.abs(w), 1.0, atol=1e-15)  # nodes on the unit circle


@pytest.mark.parametrize("n,ne", [(8, 4), (12, 6), (16, 8), (16, 2), (23, 6), (24, 12)])
def test_roots_of_unity_plans(n, ne):
    rng = np.random.default_rng(7 * n + ne)
    d = n - ne
    wt = weights(n, ne)
    q = random_q(rng, d, palindromic=True)
    for nodes, flags in [(0, qcs.QCS_FLAG_DFT_NODES), (d + 1, 0), (d + 4, 0), (min(2 * n + 1, qcs.MAX_NODES), 0)]:
        got, nev, _ = plan_sum(n, ne, q, nodes, flags)
        N = nodes if nodes else d + 1
        assert nev == N // 2 + 1
        assert abs(got - np.dot(wt, q)) <= 1e-13 * np.dot(wt, np.abs(q))
    # every node: exact for any polynomial of degree d
    qg = random_q(rng, d, palindromic=False)
    got, nev, _ = plan_sum(n, ne, qg, 2 * n + 1 if 2 * n + 1 <= qcs.MAX_NODES else 0, qcs.QCS_FLAG_ALL_NODES)
    assert abs(got - np.dot(wt, qg)) <= 1e-13 * np.dot(wt, np.abs(qg))


@pytest.mark.parametrize("n,ne", [(8, 4), (16, 8), (24, 12)])
def test_shortcut_plans_rely_on_the_parity(n, ne):
    """Without the palindromic structure the shortened plans are not exact,
    which is why parity -1 snapshots never reach them (their term is exactly 0)."""
    rng = np.random.default_rng(n)
    d = n - ne
    wt = weights(n, ne)
    q = random_q(rng, d, palindromic=False)
    for flags in (0, qcs.QCS_FLAG_DFT_NODES):
        got, _, _ = plan_sum(n, ne, q, 0, flags)
        assert abs(got - np.dot(wt, q)) > 1e-6 * np.dot(wt, np.abs(q))


def test_plan_arguments_are_checked():
    for args in [(16, 7, 0, 0), (16, 18, 0, 0), (25, 8, 0, 0), (16, 8, 8, 0), (16, 8, 50, 0), (16, 8, -1, 0)]:
        with pytest.raises(qcs.QCSError):
            qcs.node_plan(*args)
