"""Parity of the FP64 overlap path with its congruence on tensor cores (through the C ABI).

The tensor-core congruence (the default FP64 path at n = 16, QCS_FLAG_FP64_TC for any
n <= 16) forms P = M H M^T by error-free slicing, so its results carry FP64 rounding:
the tolerances are those of the FP64 ALU path -- per pair 1e-10 of the pair scale s_p
(the magnitude of the estimator's terms before they cancel), per walker 1e-10 of the
mean pair scale and 1e-10 relative to the walker's overlap, parity -1 pairs exactly 0.
The cases span several tiles (32 parity +1 snapshots each, in sub-tiles of four) with
ragged tails, empty and one-snapshot sets, every even ne at n = 16, the node plans,
the snapshot ensembles and walkers with exact zeros; the ALU path (QCS_FLAG_FP64_ALU)
is compared on the same inputs.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth
from parity_checks import check_walkers_relative

pytestmark = pytest.mark.gpu
TOL = 1e-10
TC, ALU = qcs.QCS_FLAG_FP64_TC, qcs.QCS_FLAG_FP64_ALU


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(ctx, data, flags=0, **kw):
    s = qcs.Snapshots(ctx, to_dev(data["Q"]), to_dev(data["b"]))
    ov, pp = qcs.overlap(ctx, s, to_dev(data["Phi"]), per_pair=True, flags=flags, **kw)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    return ov.cpu().numpy(), pp.cpu().numpy(), s.parity().cpu().numpy(), st


def check(ov, pp, par, data, floor=0.0):
    oo, opp, sc, _ = orc.overlap(data["Phi"], data["Q"], data["b"], per_pair=True)
    ok = par == 1
    err = np.abs(pp[:, ok] - opp[:, ok])
    assert np.all(err <= TOL * sc[:, ok] + floor), f"max err/scale {np.max(err / (sc[:, ok] + 1e-300)):.3e}"
    assert np.all(pp[:, ~ok] == 0)
    assert np.all(np.abs(ov - oo) <= TOL * sc.mean(axis=1) + floor)
    if floor == 0.0 and ok.any():
        check_walkers_relative(ov, oo, sc)
    return oo, opp, sc


def make(seed, n, ne, W, P, ensemble="haar"):
    rng = np.random.default_rng(seed)
    if ensemble == "haar":
        Q = synth.haar_orthogonal(rng, 2 * n, P)
    elif ensemble == "givens":
        Q = synth.givens_orthogonal(rng, 2 * n, P)
    else:
        Q = synth.signed_permutation(rng, 2 * n, P)
    return dict(Q=Q, b=synth.uniform_bits(rng, n, P), Phi=synth.walkers(rng, n, ne, W))


@pytest.mark.parametrize("n,ne,W,P", [(16, 8, 13, 91), (16, 8, 3, 7), (16, 8, 5, 200), (16, 2, 4, 23),
                                      (16, 4, 6, 45), (16, 6, 3, 37), (16, 10, 3, 41), (16, 12, 4, 33),
                                      (16, 14, 3, 29), (16, 16, 4, 23), (12, 6, 9, 61), (8, 4, 16, 256),
                                      (10, 4, 7, 45), (5, 2, 6, 33), (2, 2, 3, 17), (14, 8, 4, 70)])
def test_tensor_core_path_matches_oracle(ctx, n, ne, W, P):
    data = make(n * 1000 + ne * 10 + P, n, ne, W, P)
    ov, pp, par, st = run(ctx, data, flags=TC)
    assert st == 0
    check(ov, pp, par, data)


def test_default_at_n16_is_the_tensor_core_path_and_agrees_with_the_alu_path(ctx):
    data = make(5, 16, 8, 9, 150)
    ov_d, pp_d, par, st = run(ctx, data)
    ov_t, pp_t, _, st2 = run(ctx, data, flags=TC)
    ov_a, pp_a, _, st3 = run(ctx, data, flags=ALU)
    assert st == st2 == st3 == 0
    assert np.array_equal(pp_d, pp_t) and np.array_equal(ov_d, ov_t)  # same kernel, same order
    _, _, sc = check(ov_t, pp_t, par, data)
    check(ov_a, pp_a, par, data)
    assert np.all(np.abs(pp_t - pp_a) <= 2 * TOL * sc)


def test_empty_and_single_snapshot_sets(ctx):
    n, ne = 16, 8
    rng = np.random.default_rng(3)
    Phi = synth.walkers(rng, n, ne, 5)
    s = qcs.Snapshots(ctx, torch.zeros((0, 2 * n, 2 * n), dtype=torch.float64, device="cuda"),
                      torch.zeros((0, n), dtype=torch.uint8, device="cuda"))
    ov, _ = qcs.overlap(ctx, s, to_dev(Phi), flags=TC)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0 and np.all(ov.cpu().numpy() == 0)
    Q = synth.haar_orthogonal(rng, 2 * n, 1)
    b = synth.parity_consistent_bits(rng, Q)
    data = dict(Q=Q, b=b, Phi=Phi)
    ov, pp, par, st = run(ctx, data, flags=TC)
    assert st == 0 and par[0] == 1
    check(ov, pp, par, data)


def test_node_plans_on_the_tensor_core_path(ctx):
    data = make(11, 16, 8, 5, 60)
    for kw in (dict(), dict(extra=qcs.QCS_FLAG_DFT_NODES), dict(nodes=33), dict(nodes=12)):
        flags = TC | kw.pop("extra", 0)
        ov, pp, par, st = run(ctx, data, flags=flags, **kw)
        assert st == 0
        check(ov, pp, par, data)


@pytest.mark.parametrize("ensemble", ["givens", "signed_perm"])
def test_snapshot_ensembles_on_the_tensor_core_path(ctx, ensemble):
    data = make(21, 16, 8, 6, 80, ensemble=ensemble)
    ov, pp, par, st = run(ctx, data, flags=TC)
    assert st == 0
    floor = 1e-10 * np.abs(data["Phi"]).max() ** 4 if ensemble == "signed_perm" else 0.0
    check(ov, pp, par, data, floor=floor)


def test_unit_walkers_against_signed_permutations(ctx):
    """Walkers with exact zeros and signed-permutation snapshots: rows of M and H with
    many zero entries, singular occupied blocks and the full-elimination fallback."""
    rng = np.random.default_rng(31)
    n, ne, P = 16, 8, 64
    Q = synth.signed_permutation(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    eye = np.eye(n, dtype=complex)
    R = np.triu(rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne))) + 2 * np.eye(ne)
    Phi = np.stack([eye[:, rng.permutation(n)[:ne]] @ R for _ in range(3)] + [synth.walkers(rng, n, ne, 1)[0]])
    data = dict(Q=Q, b=b, Phi=Phi)
    ov, pp, par, st = run(ctx, data, flags=TC)
    assert st == 0
    check(ov, pp, par, data, floor=1e-10 * np.abs(Phi).max() ** 4)


def test_walker_scales_far_from_one(ctx):
    """Walkers scaled by 1e-30 and 1e+30 (det R spans 1e-240 .. 1e+240): the walker prep
    orthonormalises the rows that are sliced, the magnitude goes into det R, and the
    overlaps keep the oracle's relative accuracy."""
    data = make(41, 16, 8, 4, 50)
    data["Phi"] = data["Phi"] * np.array([1e-30, 1.0, 1e30, 3.0])[:, None, None]
    ov, pp, par, st = run(ctx, data, flags=TC)
    assert st == 0
    check(ov, pp, par, data)


def test_flag_conflicts_and_unsupported_requests(ctx):
    data = make(51, 20, 10, 2, 8)
    s = qcs.Snapshots(ctx, to_dev(data["Q"]), to_dev(data["b"]))
    with pytest.raises(qcs.QCSError) as e:
        qcs.overlap(ctx, s, to_dev(data["Phi"]), flags=TC)
    assert e.value.code == qcs.QCS_ERR_UNSUPPORTED
    d16 = make(52, 16, 8, 2, 8)
    s16 = qcs.Snapshots(ctx, to_dev(d16["Q"]), to_dev(d16["b"]))
    with pytest.raises(qcs.QCSError) as e:
        qcs.overlap(ctx, s16, to_dev(d16["Phi"]), flags=TC | qcs.QCS_FLAG_ALL_NODES)
    assert e.value.code == qcs.QCS_ERR_UNSUPPORTED
    with pytest.raises(qcs.QCSError) as e:
        qcs.overlap(ctx, s16, to_dev(d16["Phi"]), flags=TC | ALU)
    assert e.value.code == qcs.QCS_ERR_ARG


def test_every_node_round_size_agrees(ctx):
    data = make(61, 16, 8, 7, 90)
    ref = None
    for cfg in (1, 2, 3):
        ov, pp, par, st = run(ctx, data, flags=TC, config=cfg)
        assert st == 0
        check(ov, pp, par, data)
        ref = pp if ref is None else ref
        assert np.all(np.abs(pp - ref) <= 1e-13 * np.abs(ref).max())
