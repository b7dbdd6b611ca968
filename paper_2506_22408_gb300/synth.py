"""Seeded synthetic inputs for the matchgate-shadow overlap path.

This module only draws random inputs; it contains none of the estimator's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper's own data (quantum-computer shadow records, trial states,
walkers and Cholesky vectors of the (8e,8o) active space) are not available,
so inputs with the same shapes and distributions stand in for them:

* snapshots ``(Q_p, b_p)``: ``Q_p`` Haar-random in O(2n) (Gaussian matrix, QR,
  sign fix of the R diagonal -- Mezzadri's method), or a product of random
  Givens rotations, or a random signed permutation (the ensemble the paper's
  experiment used); ``b_p`` uniform n-bit strings, or uniform over the strings
  whose parity matches det Q (the only outcomes a parity-even state can give);
* walkers ``Phi``: complex Gaussian n x ne matrices, orthonormalised by QR and
  multiplied by a complex scalar with modulus in [0.5, 2] and uniform phase
  (AFQMC walkers are non-orthonormal Slater determinants);
* Cholesky vectors ``L_gamma = (X + X^T)/2`` with X real Gaussian n x n.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def haar_orthogonal(rng: np.random.Generator, N: int, count: int) -> np.ndarray:
    """``count`` Haar-distributed matrices of O(N) (det = +-1)."""
    Z = rng.standard_normal((count, N, N))
    Qm, R = np.linalg.qr(Z)
    d = np.sign(np.diagonal(R, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return np.ascontiguousarray(Qm * d[:, None, :])


def givens_orthogonal(rng: np.random.Generator, N: int, count: int, rotations: int = 120) -> np.ndarray:
    """``count`` products of ``rotations`` plane rotations in random coordinate
    planes of R^N with angles uniform in [0, 2 pi)."""
    Q = np.broadcast_to(np.eye(N), (count, N, N)).copy()
    for _ in range(rotations):
        i = rng.integers(0, N, size=count)
        j = (i + rng.integers(1, N, size=count)) % N
        th = rng.uniform(0.0, 2.0 * np.pi, size=count)
        c, s = np.cos(th), np.sin(th)
        ar = np.arange(count)
        ri, rj = Q[ar, i, :].copy(), Q[ar, j, :].copy()
        Q[ar, i, :] = c[:, None] * ri - s[:, None] * rj
        Q[ar, j, :] = s[:, None] * ri + c[:, None] * rj
    return Q


def signed_permutation(rng: np.random.Generator, N: int, count: int) -> np.ndarray:
    """``count`` uniformly random signed permutation matrices of size N."""
    Q = np.zeros((count, N, N))
    for c in range(count):
        perm = rng.permutation(N)
        sg = rng.choice([-1.0, 1.0], size=N)
        Q[c, np.arange(N), perm] = sg
    return Q


def uniform_bits(rng: np.random.Generator, n: int, count: int) -> np.ndarray:
    return rng.integers(0, 2, size=(count, n), dtype=np.uint8)


def parity_consistent_bits(rng: np.random.Generator, Q: np.ndarray) -> np.ndarray:
    """Uniform bits conditioned on (-1)^{|b|} = det Q."""
    count, N, _ = Q.shape
    n = N // 2
    b = uniform_bits(rng, n, count)
    det = np.sign(np.linalg.det(Q))
    par = np.where(b.sum(axis=1) % 2 == 0, 1.0, -1.0)
    bad = par != det
    b[bad, 0] ^= 1
    return b


def walkers(rng: np.random.Generator, n: int, ne: int, W: int) -> np.ndarray:
    """``W`` non-orthonormal complex n x ne walkers (orthonormal times a scalar)."""
    Z = rng.standard_normal((W, n, ne)) + 1j * rng.standard_normal((W, n, ne))
    Qm, _ = np.linalg.qr(Z)
    mod = rng.uniform(0.5, 2.0, size=W)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=W)
    s = (mod * np.exp(1j * ph))[:, None, None]
    return np.ascontiguousarray(Qm * s)


def cholesky_vectors(rng: np.random.Generator, n: int, nchol: int) -> np.ndarray:
    X = rng.standard_normal((nchol, n, n))
    return np.ascontiguousarray(0.5 * (X + np.transpose(X, (0, 2, 1))))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: n modes, ne electrons, W walkers, P snapshots."""

    name: str
    n: int
    ne: int
    W: int
    P: int
    ensemble: str = "haar"  # haar | givens | signed_perm
    bits: str = "uniform"  # uniform | parity
    nchol: int = 0

    def generate(self, seed: int = 0, W: int | None = None, P: int | None = None):
        """Return dict(Phi, Q, b[, L]) drawn from ``seed``.

        ``W``/``P`` override the counts (a prefix-consistent subset is NOT
        guaranteed; use the same overrides on both sides of a comparison).
        """
        W = self.W if W is None else W
        P = self.P if P is None else P
        rng = np.random.default_rng(seed)
        N = 2 * self.n
        if self.ensemble == "haar":
            Q = haar_orthogonal(rng, N, P)
        elif self.ensemble == "givens":
            Q = givens_orthogonal(rng, N, P)
        elif self.ensemble == "signed_perm":
            Q = signed_permutation(rng, N, P)
        else:
            raise ValueError(self.ensemble)
        b = uniform_bits(rng, self.n, P) if self.bits == "uniform" else parity_consistent_bits(rng, Q)
        Phi = walkers(rng, self.n, self.ne, W)
        out = dict(Phi=Phi, Q=Q, b=b)
        if self.nchol:
            out["L"] = cholesky_vectors(rng, self.n, self.nchol)
        return out


# The five workload shapes of the study (n modes, ne electrons, walkers, snapshots).
PLAIN_SMALL = Workload("plain n=8 ne=4 16x256", 8, 4, 16, 256)
PAPER_SHAPED = Workload("paper-shaped n=16 ne=8 1024x20000", 16, 8, 1024, 20000)
DIFFERENTIATION = Workload("differentiation n=16 ne=8 512x10000 nchol=64", 16, 8, 512, 10000, nchol=64)
PRECISION = Workload("precision n=16 ne=8 2048x50000", 16, 8, 2048, 50000)
BATCH_SYSTEMS = (
    Workload("batch n=8", 8, 4, 1024, 2000),
    Workload("batch n=12", 12, 6, 512, 5000),
    Workload("batch n=16", 16, 8, 256, 10000),
    Workload("batch n=20", 20, 10, 128, 20000),
    Workload("batch n=24", 24, 12, 64, 40000),
)
