"""Brute-force Fock-space evaluation of the matchgate-shadow overlap estimator.

Test-only, n <= 8.  It shares nothing with the oracle: it builds every object
of the definition explicitly in the 2^n-dimensional Fock space under the
Jordan-Wigner map and never forms a covariance matrix or a Pfaffian.

Definitions used (arXiv 2506.22408):
* Majoranas gamma_{2j-1} = a_j + a_j^dagger, gamma_{2j} = -i (a_j - a_j^dagger)
  (SI "Reduced Density Matrices").
* The walker |phi> = prod_j (sum_k Phi_kj a_k^dagger) |0>, first factor leftmost.
* The snapshot state rho_{Q,b} = U_Q^dagger |b><b| U_Q with
  U_Q^dagger gamma_mu U_Q = sum_nu Q_{mu nu} gamma_nu; since
  |b><b| = prod_j (1 + s_j i gamma_{2j-1} gamma_{2j}) / 2 with s_j = 2 b_j - 1,
  rho_{Q,b} = prod_j (1 + s_j i g_{2j-1} g_{2j}) / 2 with g = Q gamma.
* The matchgate shadow channel scales the Majorana-degree-2k part of an
  operator by lambda_k = C(n,k)/C(2n,2k); its inverse divides by lambda_k
  (the weights C(2N,2x)/C(N,x) of the estimator equation).
* Preparing (|0> + |Psi_T>)/sqrt2 makes 2 tr(M^{-1}(|phi><0|) rho) an unbiased
  estimator of <Psi_T|phi>  (Sec. "Classical shadows and the evaluation of
  overlaps").
"""
from __future__ import annotations

from itertools import combinations
from math import comb

import numpy as np


class Fock:
    """Jordan-Wigner operators on n modes; basis index x = sum_j x_j 2^j."""

    def __init__(self, n: int):
        self.n = n
        self.dim = 1 << n
        dim = self.dim
        self.a = []
        for j in range(n):
            A = np.zeros((dim, dim), complex)
            for x in range(dim):
                if (x >> j) & 1:
                    s = -1.0 if bin(x & ((1 << j) - 1)).count("1") % 2 else 1.0
                    A[x ^ (1 << j), x] = s
            self.a.append(A)
        self.gamma = []
        for A in self.a:
            Ad = A.conj().T
            self.gamma.append(A + Ad)
            self.gamma.append(-1j * (A - Ad))
        # sparse form: (gamma_mu v)[y] = phase[y] * v[perm[y]]
        self.perm, self.phase = [], []
        for G in self.gamma:
            p = np.argmax(np.abs(G), axis=1)
            self.perm.append(p)
            self.phase.append(G[np.arange(dim), p])
        self.vac = np.zeros(dim, complex)
        self.vac[0] = 1.0

    def apply_gamma(self, mu: int, V: np.ndarray) -> np.ndarray:
        """gamma_mu applied to the last axis of V."""
        return self.phase[mu] * V[..., self.perm[mu]]

    def slater(self, Phi: np.ndarray) -> np.ndarray:
        """|phi> = c_1^dag c_2^dag ... c_ne^dag |0>, c_j^dag = sum_k Phi_kj a_k^dag."""
        v = self.vac.copy()
        for j in reversed(range(Phi.shape[1])):
            cd = sum(Phi[k, j] * self.a[k].conj().T for k in range(self.n))
            v = cd @ v
        return v

    def shadow_state(self, Q: np.ndarray, b: np.ndarray) -> np.ndarray:
        """Normalised vector of the rank-one projector rho_{Q,b}."""
        n = self.n
        g = [sum(Q[mu, nu] * self.gamma[nu] for nu in range(2 * n)) for mu in range(2 * n)]
        Pm = np.eye(self.dim, dtype=complex)
        for j in range(n):
            s = 2.0 * float(b[j]) - 1.0
            Pm = Pm @ (0.5 * (np.eye(self.dim) + s * 1j * (g[2 * j] @ g[2 * j + 1])))
        k = int(np.argmax(np.linalg.norm(Pm, axis=0)))
        psi = Pm[:, k]
        return psi / np.linalg.norm(psi)

    def _subset_stack(self, idx, v):
        """gamma_S v for every subset S of idx (ascending product order), with |S|."""
        vecs = [v[None, :]]
        sizes = [np.zeros(1, int)]
        V, Sz = v[None, :], np.zeros(1, int)
        for mu in reversed(idx):  # prepend mu as the smallest element
            V2 = self.apply_gamma(mu, V)
            V = np.concatenate([V, V2], axis=0)
            Sz = np.concatenate([Sz, Sz + 1])
        return V, Sz

    def estimator(self, Phi: np.ndarray, psi: np.ndarray) -> complex:
        """2 tr(M^{-1}(|phi><0|) |psi><psi|) by the Majorana expansion
        (2 / 2^n) sum_{|S| even} <0|gamma_S^dag|phi> <psi|gamma_S|psi> / lambda_{|S|/2}."""
        n = self.n
        phi = self.slater(Phi)
        winv = np.array([comb(2 * n, s) / comb(n, s // 2) if s % 2 == 0 else 0.0 for s in range(2 * n + 1)])
        h = min(4, 2 * n)  # split the 2n Majoranas: low set enumerated in Python, high set stacked
        low, high = list(range(h)), list(range(h, 2 * n))
        V0, Sz = self._subset_stack(high, self.vac)
        Vp, _ = self._subset_stack(high, psi)
        total = 0.0 + 0.0j
        for r in range(h + 1):
            for A in combinations(low, r):
                W0, Wp = V0, Vp
                for mu in reversed(A):
                    W0 = self.apply_gamma(mu, W0)
                    Wp = self.apply_gamma(mu, Wp)
                amp = W0.conj() @ phi  # <0|gamma_S^dag|phi> = (gamma_S|0>)^dag |phi>
                ex = np.einsum("i,si->s", psi.conj(), Wp)  # <psi|gamma_S|psi>
                total += np.sum(winv[Sz + r] * amp * ex)
        return 2.0 * total / self.dim

    def born_probabilities(self, Qs: np.ndarray, Psi: np.ndarray, chunk: int = 2048) -> np.ndarray:
        """p[g, x] = <Psi|rho_{Q_g, b(x)}|Psi> for a batch of Q and every bit string x
        (bit j of x = b_j), from the projector products built in batches."""
        n, dim = self.n, self.dim
        Gm = np.array(self.gamma)  # (2n, dim, dim)
        out = np.zeros((len(Qs), 1 << n))
        eye = np.eye(dim)
        for s0 in range(0, len(Qs), chunk):
            Qc = Qs[s0:s0 + chunk]
            gt = np.einsum("gmn,nab->gmab", Qc, Gm)  # g~_mu = sum_nu Q_{mu nu} gamma_nu
            pairs = np.einsum("gjab,gjbc->gjac", gt[:, 0::2], gt[:, 1::2])  # g~_{2j-1} g~_{2j}
            for x in range(1 << n):
                Pm = np.broadcast_to(eye, (len(Qc), dim, dim)).astype(complex)
                for j in range(n):
                    sj = 2.0 * ((x >> j) & 1) - 1.0
                    Pm = Pm @ (0.5 * (eye + sj * 1j * pairs[:, j]))
                out[s0:s0 + len(Qc), x] = np.real(np.einsum("a,gab,b->g", Psi.conj(), Pm, Psi))
        return out

    def probabilities(self, Q: np.ndarray, Psi: np.ndarray) -> np.ndarray:
        """Born probabilities p(b|Q) = <Psi|rho_{Q,b}|Psi> for all 2^n strings b (bit j of the index = b_j)."""
        n = self.n
        p = np.zeros(1 << n)
        for x in range(1 << n):
            b = np.array([(x >> j) & 1 for j in range(n)], np.uint8)
            psi = self.shadow_state(Q, b)
            p[x] = abs(np.vdot(psi, Psi)) ** 2
        return p


def channel_weights(n: int) -> np.ndarray:
    """lambda_k = C(n,k)/C(2n,2k), k = 0..n."""
    return np.array([comb(n, k) / comb(2 * n, 2 * k) for k in range(n + 1)])


def pfaffian_by_matchings(A: np.ndarray) -> complex:
    """Pfaffian as the signed sum over perfect matchings (O(m!!), m <= 10)."""
    m = A.shape[0]
    if m % 2:
        return 0.0
    if m == 0:
        return 1.0
    total = 0.0 + 0.0j
    for j in range(1, m):
        rest = [i for i in range(1, m) if i != j]
        sub = A[np.ix_(rest, rest)]
        total += (-1) ** (j - 1) * A[0, j] * pfaffian_by_matchings(sub)
    return total
