"""Signed-permutation snapshots (the ensemble of the paper's experiment): the
snapshot build recognises them, and the pair and gradient kernels form the
congruence by a gather instead of a product.  Parity with the CPU oracle (which
has no such special case) on sets that are all signed permutations and on sets
that mix them with Haar snapshots, so both paths run in one launch.

Tolerances are those of the other GPU tests (per pair 1e-10 of the pair scale,
gradients 1e-9 of the largest entry plus 1e-10 of the mean pair scale).  Signed
permutations make many entries of B exactly zero, so node matrices can need
pivots on exact zeros and pairs can vanish exactly; an absolute floor of 1e-10
times |Phi|^4 (as in the ensemble test) covers pairs whose scale is itself zero.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth
from test_gpu_grad import check_grad

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mixed_set(rng, n, P, frac_sp):
    """P snapshots, a random subset of them signed permutations."""
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    sp = rng.random(P) < frac_sp
    Q[sp] = synth.signed_permutation(rng, 2 * n, int(sp.sum()))
    return Q, sp


@pytest.mark.parametrize("n,ne,W,P,frac", [(16, 8, 6, 120, 1.0), (16, 8, 5, 90, 0.5), (8, 4, 4, 64, 1.0),
                                           (12, 2, 3, 40, 0.7), (24, 12, 2, 16, 1.0), (7, 4, 3, 30, 0.6),
                                           (20, 10, 3, 40, 0.5)])
def test_overlaps_match_oracle(ctx, n, ne, W, P, frac):
    rng = np.random.default_rng(300 + n + ne)
    Q, sp = mixed_set(rng, n, P, frac)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    assert s.signed_perm_count() == int(sp.sum())
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    floor = 1e-10 * np.abs(Phi).max() ** 4
    for kw in (dict(), dict(flags=qcs.QCS_FLAG_ALL_NODES)):
        ov, pp = qcs.overlap(ctx, s, dev(Phi), per_pair=True, **kw)
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        ov, pp = ov.cpu().numpy(), pp.cpu().numpy()
        assert np.all(np.abs(pp - opp) <= TOL * sc + floor)
        assert np.all(np.abs(ov - oo) <= TOL * sc.mean(axis=1) + floor)


@pytest.mark.parametrize("n,ne,W,P,frac", [(16, 8, 3, 40, 1.0), (8, 4, 4, 33, 0.5), (10, 6, 2, 21, 1.0),
                                           (18, 8, 2, 24, 0.5)])
def test_gradient_matches_oracle(ctx, n, ne, W, P, frac):
    rng = np.random.default_rng(400 + n + ne)
    Q, sp = mixed_set(rng, n, P, frac)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, W)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    assert s.signed_perm_count() == int(sp.sum())
    ov, g = qcs.overlap_grad(ctx, s, dev(Phi))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    check_grad(g.cpu().numpy(), og, ov.cpu().numpy(), oo, sc, ov_floor=1e-10 * np.abs(Phi).max() ** 4)


def test_near_permutations_take_the_dense_path(ctx):
    """Only exact signed permutations are recognised: a permutation with one entry
    off by a rounding error, a scaled permutation and a Givens product are not."""
    rng = np.random.default_rng(5)
    n = 8
    Q = synth.signed_permutation(rng, 2 * n, 6)
    Q[1] = Q[1] @ synth.givens_orthogonal(rng, 2 * n, 1, rotations=1)[0]
    r, c = np.nonzero(Q[2])
    Q[2][r[0], c[0]] *= 1.0 + 2.0**-52
    Q[3] *= -1.0  # still a signed permutation
    s = qcs.Snapshots(ctx, dev(Q), dev(synth.uniform_bits(rng, n, 6)))
    assert s.signed_perm_count() == 4
