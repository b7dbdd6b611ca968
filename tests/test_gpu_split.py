"""Split-precision overlaps (QCS_TF32X3): the congruence T = U^T Qt^T on tensor
cores (tcgen05 kind::tf32, three hi/lo passes, FP32 accumulation), B^(s) in
FP32, the Pfaffians in FP64.

Stated bound: per pair |o_split - o_oracle| <= 2e-5 * s_p, with s_p the magnitude
of the pair's terms before cancellation (from the oracle).  Derivation: the
split TF32 products carry a relative error of about 2^-21 (two 11-bit halves of
each operand, FP32 accumulation over 2n = 32 terms), B^(s) adds FP32 rounding of
2n-term sums of |T| ~ 1 entries (~2e-6), and the Pfaffian at each node is a
multilinear form of degree m/2 = 12 in B, which multiplies the relative
perturbation by at most m/2 for a well-conditioned elimination; the node sum
and the weights enter through s_p.  The measured maxima sit well below.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth

pytestmark = pytest.mark.gpu
BOUND = 2e-5


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,ne,W,P", [(16, 8, 13, 91), (16, 4, 6, 40), (12, 6, 7, 45), (8, 4, 9, 61), (10, 4, 5, 23),
                                      (16, 16, 5, 30), (20, 10, 5, 31), (24, 12, 3, 23), (17, 6, 4, 19),
                                      (24, 2, 3, 17), (22, 22, 2, 9)])
def test_split_matches_oracle_within_bound(ctx, n, ne, W, P):
    rng = np.random.default_rng(3000 + 10 * n + ne)
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, pp = qcs.overlap(ctx, s, dev(Phi), per_pair=True, precision=qcs.QCS_TF32X3)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    par = s.parity().cpu().numpy()
    ok = par == 1
    pp = pp.cpu().numpy()
    err = np.abs(pp[:, ok] - opp[:, ok]) / sc[:, ok]
    assert err.max() <= BOUND, err.max()
    assert np.all(pp[:, ~ok] == 0)
    # the split path is not the FP64 path: its error is visible but bounded
    werr = np.abs(ov.cpu().numpy() - oo) / sc.mean(axis=1)
    assert werr.max() <= BOUND


def test_split_agrees_with_fp64_path_and_is_deterministic(ctx):
    wl = synth.Workload("t", 16, 8, 37, 203)
    d = wl.generate(seed=4)
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    Phi = dev(d["Phi"])
    o64, p64 = qcs.overlap(ctx, s, Phi, per_pair=True)
    o1, p1 = qcs.overlap(ctx, s, Phi, per_pair=True, precision=qcs.QCS_TF32X3)
    o2, p2 = qcs.overlap(ctx, s, Phi, per_pair=True, precision=qcs.QCS_TF32X3)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2) and torch.equal(p1, p2)
    scale = p64.abs().mean(dim=1)
    assert ((o1 - o64).abs() / scale).max().item() <= BOUND


def test_split_above_16_modes_uses_the_group_kernel(ctx):
    """16 < n <= 24 runs on the 64-row, K = 48 tiles (two walkers x two snapshots per
    MMA, one 64-thread group per walker): per-pair values are bitwise independent of the
    tile size, as for n <= 16."""
    wl = synth.Workload("t", 20, 10, 5, 37)
    d = wl.generate(seed=9)
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    Phi = dev(d["Phi"])
    o1, p1 = qcs.overlap(ctx, s, Phi, per_pair=True, precision=qcs.QCS_TF32X3)
    o2, p2 = qcs.overlap(ctx, s, Phi, per_pair=True, precision=qcs.QCS_TF32X3,
                         config=qcs.encode_config(tc_subtiles_per_tile=3))
    o64, p64 = qcs.overlap(ctx, s, Phi, per_pair=True)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert torch.equal(p1, p2)
    scale = p64.abs().mean(dim=1)
    assert ((o1 - o64).abs() / scale).max().item() <= BOUND


@pytest.mark.parametrize("subs", [1, 2, 3, 15])
def test_split_tile_sizes_agree(ctx, subs):
    """A tile spans subs sub-chunks of 4 snapshots and each warp sums its walker's pairs
    over the tile in registers: the per-pair values do not depend on the tile size
    (bitwise), the walker sums only through their summation order."""
    wl = synth.Workload("t", 16, 8, 9, 157)
    d = wl.generate(seed=8)
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    Phi = dev(d["Phi"])
    o_ref, p_ref = qcs.overlap(ctx, s, Phi, per_pair=True, precision=qcs.QCS_TF32X3)
    cfg = qcs.encode_config(tc_subtiles_per_tile=subs)
    o, p = qcs.overlap(ctx, s, Phi, per_pair=True, precision=qcs.QCS_TF32X3, config=cfg)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert torch.equal(p, p_ref)
    scale = p_ref.abs().sum(dim=1)
    assert ((o - o_ref).abs() / scale).max().item() <= 1e-14
