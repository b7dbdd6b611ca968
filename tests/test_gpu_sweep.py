"""A sweep over sizes, electron counts, snapshot ensembles, node plans and walker
structures: every per-pair overlap against the oracle in one launch per case, and the
gradient on a subset.  It crosses the kernel paths (one warp per pair with staged rows,
the n = 16 register path in echelon or reduced form, two-warp groups for n > 16, the
shared occupied elimination and its fallback, gathers for signed permutations) with
the inputs that steer them.

Tolerances are those of tests/test_gpu_overlap.py and tests/test_gpu_grad.py, with two
floors for pairs whose value is exactly zero: an absolute one, and 1e-12 of the walker's
largest pair scale for the oracle's own rounding.  Pairs of a parity -1 snapshot are zero
(the library skips them, and they must be exact zeros), and so are pairs whose B matrix
is structurally singular (signed permutations that keep a Majorana pair together, with
every mode occupied); the oracle evaluates them with B singular only up to rounding (two
singular values near 1e-16), which the estimator's weights (about 1e7 at n = ne = 24) lift
to as much as 4e-8, about 1e-15 of the walker's largest pair scale, while the pair's own
scale s_p is of that rounding's size too.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_case(seed, n, ne, ensemble, walkers_kind, W=5, P=40):
    rng = np.random.default_rng(seed)
    if ensemble == "haar":
        Q = synth.haar_orthogonal(rng, 2 * n, P)
    elif ensemble == "givens":
        Q = synth.givens_orthogonal(rng, 2 * n, P, rotations=3 * n)
    else:
        Q = synth.signed_permutation(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    if walkers_kind == "unit":
        eye = np.eye(n, dtype=complex)
        for w in range(W - 1):
            Phi[w] = eye[:, rng.permutation(n)[:ne]] * (0.5 + rng.random(ne))
    elif walkers_kind == "scaled_top":
        for w in range(W):
            Phi[w][: ne // 2] *= 10.0 ** (-rng.integers(0, 4))
    return Q, b, Phi


CASES = []
for n, ne in [(4, 2), (6, 6), (8, 2), (10, 6), (12, 12), (14, 4), (16, 2), (16, 8), (16, 10), (17, 6), (18, 8),
              (20, 2), (20, 14), (22, 6), (24, 12), (24, 20), (24, 24)]:
    for ens in ("haar", "givens", "signed_perm"):
        for kind in ("random", "unit", "scaled_top"):
            CASES.append((n, ne, ens, kind))


@pytest.mark.parametrize("n,ne,ens,kind", CASES[::3] + CASES[1::7])
def test_sweep_overlap(ctx, n, ne, ens, kind):
    seed = 1000 * n + 10 * ne + len(ens) + len(kind)
    Q, b, Phi = make_case(seed, n, ne, ens, kind)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    flags = qcs.QCS_FLAG_DFT_NODES if (n + ne) % 4 == 0 else 0
    ov, pp = qcs.overlap(ctx, s, dev(Phi), per_pair=True, flags=flags)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    # exact zeros: an absolute floor, and the oracle's rounding (1e-12 of the walker's
    # largest pair scale)
    floor = 1e-10 * max(1.0, np.abs(Phi).max()) ** 4 + 1e-12 * sc.max(axis=1, keepdims=True)
    pp = pp.cpu().numpy()
    minus = np.sign(np.linalg.det(Q)) * (-1.0) ** b.astype(np.int64).sum(axis=1) < 0
    assert np.all(pp[:, minus] == 0)  # parity -1: exactly zero
    assert np.all(np.abs(pp - opp) <= TOL * sc + floor), np.max(np.abs(pp - opp) / (sc + 1e-300))
    assert np.all(np.abs(ov.cpu().numpy() - oo) <= TOL * sc.mean(axis=1) + floor[:, 0])


@pytest.mark.parametrize("n,ne,ens,kind", [(16, 8, "haar", "scaled_top"), (20, 14, "givens", "random"),
                                          (10, 6, "haar", "random"), (24, 12, "haar", "random")])
def test_sweep_gradient(ctx, n, ne, ens, kind):
    Q, b, Phi = make_case(77 + n + ne, n, ne, ens, kind, W=3, P=24)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, g = qcs.overlap_grad(ctx, s, dev(Phi))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    g = g.cpu().numpy()
    for w in range(len(Phi)):
        tol = 1e-9 * np.abs(og[w]).max() + 1e-10 * sc[w].mean()
        assert np.abs(g[w] - og[w]).max() <= tol
