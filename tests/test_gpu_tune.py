"""Kernel configurations (qcs_opts.config) and the autotuner, through the C ABI.

Every field of a configuration changes only how the work is laid out: the tile length
of the FP64 ALU pair kernel, the warps per pair for n > 16, the node matrices per round,
the congruence path at n <= 16 and the tile of the tensor-core kernel.  Each choice is
checked against the oracle with the FP64 tolerances (per pair 1e-10 of the pair scale
s_p, per walker 1e-10 of the mean pair scale and 1e-10 relative); the batched launch with
tuned per-system configurations equals qcs_overlap with the same configuration on the
ALU path bit for bit (same tiles, same reduction order), and the autotuner returns a
configuration the kernels run.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth
from parity_checks import check_walkers_relative

pytestmark = pytest.mark.gpu
TOL = 1e-10
ALU = qcs.QCS_FLAG_FP64_ALU


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(seed, n, ne, W, P):
    rng = np.random.default_rng(seed)
    return dict(Q=synth.haar_orthogonal(rng, 2 * n, P), b=synth.uniform_bits(rng, n, P),
                Phi=synth.walkers(rng, n, ne, W))


def run(ctx, d, **kw):
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    ov, pp = qcs.overlap(ctx, s, dev(d["Phi"]), per_pair=True, **kw)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    return ov.cpu().numpy(), pp.cpu().numpy(), s.parity().cpu().numpy()


def check(d, ov, pp, par):
    oo, opp, sc, _ = orc.overlap(d["Phi"], d["Q"], d["b"], per_pair=True)
    ok = par == 1
    assert np.all(np.abs(pp[:, ok] - opp[:, ok]) <= TOL * sc[:, ok])
    assert np.all(pp[:, ~ok] == 0)
    assert np.all(np.abs(ov - oo) <= TOL * sc.mean(axis=1))
    check_walkers_relative(ov, oo, sc)


@pytest.mark.parametrize("fields", [dict(alu_snapshots_per_warp=1), dict(alu_snapshots_per_warp=2),
                                    dict(alu_snapshots_per_warp=8), dict(alu_snapshots_per_warp=15),
                                    dict(alu_snapshots_per_warp=8, node_matrices_per_round=1)])
def test_alu_tiles(ctx, fields):
    d = make(1, 16, 8, 7, 150)
    ov, pp, par = run(ctx, d, flags=ALU, config=qcs.encode_config(**fields))
    check(d, ov, pp, par)


@pytest.mark.parametrize("subs", [1, 2, 4, 15])
def test_tensor_core_tiles(ctx, subs):
    d = make(2, 16, 8, 5, 200)
    ov, pp, par = run(ctx, d, config=qcs.encode_config(path=2, tc_subtiles_per_tile=subs))
    check(d, ov, pp, par)


@pytest.mark.parametrize("n,ne,path", [(12, 6, 1), (12, 6, 2), (16, 8, 1), (16, 8, 2), (8, 4, 2)])
def test_configured_path(ctx, n, ne, path):
    d = make(3 + n, n, ne, 6, 90)
    ov, pp, par = run(ctx, d, config=qcs.encode_config(path=path))
    check(d, ov, pp, par)


@pytest.mark.parametrize("n,ne", [(20, 10), (24, 12), (18, 4)])
@pytest.mark.parametrize("warps", [1, 2])
def test_warps_per_pair_for_large_n(ctx, n, ne, warps):
    d = make(4 + n + ne, n, ne, 5, 40)
    ov, pp, par = run(ctx, d, config=qcs.encode_config(alu_warps_per_pair=warps, alu_snapshots_per_warp=2))
    check(d, ov, pp, par)


def test_batched_with_configured_systems(ctx):
    systems = [(8, 4, 9, 70), (16, 8, 6, 60), (24, 12, 4, 30)]
    cfgs = [qcs.encode_config(alu_snapshots_per_warp=8), qcs.encode_config(node_matrices_per_round=2,
                                                                          alu_snapshots_per_warp=2),
            qcs.encode_config(alu_warps_per_pair=1, alu_snapshots_per_warp=1)]
    ds, args = [], []
    for (n, ne, W, P), cfg in zip(systems, cfgs):
        d = make(5 + n, n, ne, W, P)
        s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
        ctx.set_config(n, ne, cfg)
        ds.append(d)
        args.append((s, dev(d["Phi"])))
    try:
        res = qcs.overlap_batched(ctx, args)
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        for (s, w), r, d, (n, ne, _, _), cfg in zip(args, res, ds, systems, cfgs):
            single, _ = qcs.overlap(ctx, s, w, flags=ALU, config=cfg)
            assert torch.equal(r, single)
            oo, _, sc, _ = orc.overlap(d["Phi"], d["Q"], d["b"], per_pair=True)
            check_walkers_relative(r.cpu().numpy(), oo, sc)
    finally:
        for n, ne, _, _ in systems:
            ctx.set_config(n, ne, 0)


@pytest.mark.parametrize("n,ne", [(24, 12), (8, 4)])
def test_autotuner_returns_a_runnable_configuration(ctx, n, ne):
    best = ctx.autotune(n, ne, save=False)
    f = qcs.decode_config(best)
    assert best > 0
    if n > 16:
        assert f["path"] == "default" and f["tc_subtiles_per_tile"] == 0
    d = make(6 + n, n, ne, 5, 50)
    ov, pp, par = run(ctx, d)  # takes the tuned configuration
    check(d, ov, pp, par)
    ctx.set_config(n, ne, 0)
