"""Parity of the CUDA overlap path (through the C ABI) with the CPU oracle.

Tolerance (plain FP64 path): for every pair |o_gpu - o_oracle| <= 1e-10 * s_p,
where s_p = |prefactor| * sum_x |c_x| C(2n,2x)/C(n,x) is the magnitude of the
estimator's terms before they cancel (returned by the oracle); for a walker
mean, 1e-10 times the mean of s_p and 1e-10 relative to the walker's overlap
(parity_checks.check_walkers_relative).  Parity -1 pairs must be exactly zero.
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


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def to_dev(d):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def run_gpu(ctx, data, per_pair=True, **kw):
    t = to_dev(data)
    snaps = qcs.Snapshots(ctx, t["Q"], t["b"])
    ov, pp = qcs.overlap(ctx, snaps, t["Phi"], per_pair=per_pair, **kw)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    par = snaps.parity().cpu().numpy()
    return ov.cpu().numpy(), (pp.cpu().numpy() if pp is not None else None), par, st


def check_pairs(gpu_pp, orc_pp, scale, parity):
    ok = parity == 1
    err = np.abs(gpu_pp[:, ok] - orc_pp[:, ok])
    assert np.all(err <= TOL * scale[:, ok]), f"max err/scale {np.max(err / scale[:, ok])}"
    assert np.all(gpu_pp[:, ~ok] == 0), "parity -1 pairs must be exactly zero"
    if ok.any():  # the oracle's parity -1 pairs vanish up to rounding of the row's magnitude
        ref = scale[:, ok].max(axis=1, keepdims=True)
        assert np.all(np.abs(orc_pp[:, ~ok]) <= TOL * ref)


def check_walkers(gpu_ov, orc_ov, scale):
    ms = scale.mean(axis=1)
    assert np.all(np.abs(gpu_ov - orc_ov) <= TOL * ms), np.max(np.abs(gpu_ov - orc_ov) / ms)
    check_walkers_relative(gpu_ov, orc_ov, scale)


def test_snapshot_parity_flags(ctx):
    rng = np.random.default_rng(1)
    for n in (2, 5, 8, 16, 24):
        Q = synth.haar_orthogonal(rng, 2 * n, 300)
        b = synth.uniform_bits(rng, n, 300)
        ref = (np.sign(np.linalg.det(Q)) * (-1.0) ** b.sum(axis=1)).astype(np.int8)
        t = to_dev(dict(Q=Q, b=b))
        s = qcs.Snapshots(ctx, t["Q"], t["b"])
        assert np.array_equal(s.parity().cpu().numpy(), ref)


def test_plain_small_config_per_pair(ctx):
    """n = 8, ne = 4, 16 walkers x 256 snapshots (the plain small workload), every pair."""
    data = synth.PLAIN_SMALL.generate(seed=0)
    ov, pp, par, st = run_gpu(ctx, data)
    assert st == 0
    oo, opp, sc, _ = orc.overlap(data["Phi"], data["Q"], data["b"], per_pair=True)
    check_pairs(pp, opp, sc, par)
    check_walkers(ov, oo, sc)


@pytest.mark.parametrize("n,ne,W,P", [(16, 8, 13, 91), (12, 6, 9, 61), (20, 10, 5, 37), (24, 12, 3, 29),
                                      (16, 2, 4, 23), (16, 16, 4, 23), (10, 4, 7, 45), (5, 2, 6, 33)])
def test_sizes_with_ragged_tails(ctx, n, ne, W, P):
    """Several n/ne, walker counts not a multiple of the warps per block and snapshot
    counts not a multiple of the tile chunk."""
    rng = np.random.default_rng(n * 100 + ne)
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    data = dict(Phi=Phi, Q=Q, b=b)
    ov, pp, par, st = run_gpu(ctx, data)
    assert st == 0
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    check_pairs(pp, opp, sc, par)
    check_walkers(ov, oo, sc)


def test_node_options_agree(ctx):
    """Default (Gauss plan, 3 nodes at n=16, ne=8), the minimum roots-of-unity plan
    with parity shortcuts, all nodes with no snapshot skipped, and the literal 2n+1
    roots of unity all give the same overlaps."""
    rng = np.random.default_rng(7)
    n, ne, W, P = 16, 8, 6, 40
    data = dict(Phi=synth.walkers(rng, n, ne, W), Q=synth.haar_orthogonal(rng, 2 * n, P),
                b=synth.uniform_bits(rng, n, P))
    oo, opp, sc, _ = orc.overlap(data["Phi"], data["Q"], data["b"], per_pair=True)
    for kw in (dict(), dict(flags=qcs.QCS_FLAG_DFT_NODES), dict(flags=qcs.QCS_FLAG_ALL_NODES),
               dict(nodes=2 * n + 1), dict(nodes=2 * n + 1, flags=qcs.QCS_FLAG_ALL_NODES), dict(nodes=12)):
        ov, pp, par, st = run_gpu(ctx, data, **kw)
        assert st == 0
        if kw.get("flags", 0) & qcs.QCS_FLAG_ALL_NODES:
            assert np.all(np.abs(pp - opp) <= TOL * sc)
        else:
            check_pairs(pp, opp, sc, par)
        check_walkers(ov, oo, sc)


@pytest.mark.parametrize("ensemble,n,ne", [("givens", 8, 4), ("signed_perm", 8, 4), ("givens", 16, 8),
                                           ("signed_perm", 16, 6)])
def test_other_snapshot_ensembles(ctx, ensemble, n, ne):
    """Givens products and signed permutations (exact zeros and singular node
    matrices occur for the latter)."""
    wl = synth.Workload("t", n, ne, 6, 64, ensemble=ensemble)
    data = wl.generate(seed=3)
    ov, pp, par, st = run_gpu(ctx, data)
    assert st == 0
    oo, opp, sc, _ = orc.overlap(data["Phi"], data["Q"], data["b"], per_pair=True)
    floor = 1e-10 * np.abs(data["Phi"]).max() ** 4
    assert np.all(np.abs(pp - opp) <= TOL * sc + floor)
    assert np.all(np.abs(ov - oo) <= TOL * sc.mean(axis=1) + floor)


def test_degenerate_inputs(ctx):
    rng = np.random.default_rng(9)
    n, ne = 8, 4
    Q = synth.haar_orthogonal(rng, 2 * n, 16)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 3)
    Phi[1][:, 2] = Phi[1][:, 0]  # rank-deficient walker: overlap exactly 0
    Phi[2][:] = 0
    ov, pp, par, st = run_gpu(ctx, dict(Phi=Phi, Q=Q, b=b))
    assert st == 0
    assert np.all(par == 1)
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    assert np.all(np.abs(pp[0] - opp[0]) <= TOL * sc[0])
    assert np.abs(ov[1]) <= 1e-12 * sc[0].mean()
    assert ov[2] == 0
    # zero walkers / all snapshots forbidden
    t = to_dev(dict(Q=Q, b=b))
    snaps = qcs.Snapshots(ctx, t["Q"], t["b"])
    ov0, _ = qcs.overlap(ctx, snaps, torch.zeros((0, n, ne), dtype=torch.complex128, device="cuda"))
    assert ov0.numel() == 0
    b_forb = b.copy()
    b_forb[:, 0] ^= 1
    ovf, ppf, parf, st = run_gpu(ctx, dict(Phi=Phi[:1], Q=Q, b=b_forb))
    assert np.all(parf == -1) and ovf[0] == 0 and np.all(ppf == 0)


@pytest.mark.parametrize("n,ne", [(16, 8), (16, 14), (16, 16), (8, 8), (9, 2), (12, 6)])
def test_structured_walkers(ctx, n, ne):
    """Walkers whose orbital matrix is already in echelon form, is a reversed unit basis
    (zero leading entries), lives on the last modes only, has a zero top-left entry or
    a nearly zero top block: the column reflections that bring the walker rows to
    echelon form meet each of their special cases (nothing to zero, a zero pivot, a
    zero row), and the reduced form [I; X] is taken or refused (zero or tiny top block)."""
    rng = np.random.default_rng(n * 31 + ne)
    Q = synth.haar_orthogonal(rng, 2 * n, 24)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 6)
    eye = np.eye(n, dtype=complex)
    R = np.triu(rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne))) + 2 * np.eye(ne)
    Phi[0] = eye[:, :ne] @ R                        # echelon already
    Phi[1] = eye[:, ne - 1::-1]                     # reversed unit basis
    Phi[2] = eye[:, n - ne:] @ R                    # only the last ne modes
    Phi[3][0, :] = 0                                # zero first row
    Phi[4][:, 0] = 0                                # zero first column: overlap exactly 0
    Phi[4][0, 1] = 0
    Phi[5][:ne] *= 1e-3                             # ill-conditioned top block: echelon, not reduced form
    ov, pp, par, st = run_gpu(ctx, dict(Phi=Phi, Q=Q, b=b))
    assert st == 0
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    live = [0, 1, 2, 5] + ([3] if ne < n else [])  # with ne = n a zero row makes the walker singular
    check_pairs(pp[live], opp[live], sc[live], par)
    check_walkers(ov[live], oo[live], sc[live])
    assert np.all(pp[4] == 0) and ov[4] == 0
    if ne == n:
        assert abs(ov[3]) <= 1e-12 * sc[0].mean()


@pytest.mark.parametrize("n,ne", [(20, 10), (24, 6), (20, 2), (18, 4), (16, 8), (12, 4)])
def test_unit_walkers_signed_permutations(ctx, n, ne):
    """Unit-vector walkers against signed-permutation snapshots: the occupied block of
    the node matrices is often exactly zero or singular, so the shared elimination gives
    way to the full one per node (n > 16 runs on two-warp groups, n = 16 on the
    register path); exact zeros and singular node matrices must still give the oracle's
    pair values."""
    rng = np.random.default_rng(7 * n + ne)
    P = 64
    Q = synth.signed_permutation(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    eye = np.eye(n, dtype=complex)
    R = np.triu(rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne))) + 2 * np.eye(ne)
    Phi = np.stack([eye[:, rng.permutation(n)[:ne]] @ R for _ in range(3)] + [synth.walkers(rng, n, ne, 1)[0]])
    ov, pp, par, st = run_gpu(ctx, dict(Phi=Phi, Q=Q, b=b))
    assert st == 0
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    floor = 1e-10 * np.abs(Phi).max() ** 4
    assert np.all(np.abs(pp - opp) <= TOL * sc + floor)
    assert np.all(np.abs(ov - oo) <= TOL * sc.mean(axis=1) + floor)


def test_argument_errors(ctx):
    n = 6
    Q = torch.from_numpy(synth.haar_orthogonal(np.random.default_rng(0), 2 * n, 4)).cuda()
    b = torch.zeros((4, n), dtype=torch.uint8, device="cuda")
    s = qcs.Snapshots(ctx, Q, b)
    with pytest.raises(qcs.QCSError) as e:
        qcs.overlap(ctx, s, torch.zeros((2, n, 3), dtype=torch.complex128, device="cuda"))
    assert e.value.code == 1
    with pytest.raises(qcs.QCSError):
        qcs.overlap(ctx, s, torch.zeros((2, n, 8), dtype=torch.complex128, device="cuda"))
    with pytest.raises(qcs.QCSError):
        qcs.overlap(ctx, s, torch.zeros((2, n, 2), dtype=torch.complex128, device="cuda"), nodes=2)
    Qbad = torch.zeros((2, 2 * 25, 2 * 25), dtype=torch.float64, device="cuda")
    with pytest.raises(qcs.QCSError):
        qcs.Snapshots(ctx, Qbad, torch.zeros((2, 25), dtype=torch.uint8, device="cuda"))


def test_nonfinite_input_sets_status(ctx):
    rng = np.random.default_rng(11)
    n, ne = 6, 2
    Q = synth.haar_orthogonal(rng, 2 * n, 8)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 2)
    Phi[0, 0, 0] = np.nan
    ov, pp, par, st = run_gpu(ctx, dict(Phi=Phi, Q=Q, b=b))
    assert st & 4


def test_bounded_wait_times_out_and_context_survives(ctx):
    """Failure detection without a fault: a device wait on an mbarrier that nothing
    completes gives up after its iteration limit, raises QCS_ERR_TIMEOUT in the
    status word and returns; the context keeps working afterwards."""
    assert ctx.sync_status() == 0
    for it in (1, 64, 4096):
        assert ctx.selftest_bounded_wait(it) == qcs.QCS_ERR_TIMEOUT
    with pytest.raises(qcs.QCSError):
        ctx.selftest_bounded_wait(0)
    with pytest.raises(qcs.QCSError):
        ctx.selftest_bounded_wait((1 << 20) + 1)
    rng = np.random.default_rng(12)
    n, ne = 6, 2
    Q = synth.haar_orthogonal(rng, 2 * n, 8)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 2)
    ov, pp, par, st = run_gpu(ctx, dict(Phi=Phi, Q=Q, b=b))
    assert st == 0
    oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    check_pairs(pp, opp, sc, par)
    check_walkers(ov, oo, sc)


def test_paper_shaped_full_size_sampled(ctx):
    """n = 16, ne = 8, 1024 walkers x 20000 snapshots as timed by bench.py: sampled
    pairs and three whole walkers are recomputed by the oracle."""
    wl = synth.PAPER_SHAPED
    data = wl.generate(seed=0)
    ov, pp, par, st = run_gpu(ctx, data, per_pair=True)
    assert st == 0
    rng = np.random.default_rng(5)
    ws = rng.integers(0, wl.W, size=160)
    ps = rng.integers(0, wl.P, size=160)
    for w, p in zip(ws, ps):
        o, _, s = orc.pair(data["Q"][p], data["b"][p], data["Phi"][w])
        if par[p] == 1:
            assert abs(pp[w, p] - o) <= TOL * s
        else:
            assert pp[w, p] == 0 and abs(o) <= 1e-10 * s
    sel = np.array([0, 517, wl.W - 1])
    oo, _, sc, _ = orc.overlap(data["Phi"][sel], data["Q"], data["b"], per_pair=True)
    check_walkers(ov[sel], oo, sc)
    # per-walker overlap equals the mean of the per-pair outputs
    assert np.allclose(ov, pp.mean(axis=1), rtol=0, atol=1e-12 * np.abs(pp).mean())


def test_every_kernel_configuration_agrees(ctx):
    """Every node-round size of the pair kernel gives the same overlaps, and the
    autotuner records one of them."""
    rng = np.random.default_rng(13)
    n, ne, W, P = 16, 8, 9, 70
    data = dict(Phi=synth.walkers(rng, n, ne, W), Q=synth.haar_orthogonal(rng, 2 * n, P),
                b=synth.uniform_bits(rng, n, P))
    oo, opp, sc, _ = orc.overlap(data["Phi"], data["Q"], data["b"], per_pair=True)
    for cfg in range(1, 6):
        ov, pp, par, st = run_gpu(ctx, data, config=cfg)
        assert st == 0
        check_pairs(pp, opp, sc, par)
        check_walkers(ov, oo, sc)
    best = ctx.autotune(n, ne, save=False)
    fields = qcs.decode_config(best)
    assert best > 0 and 0 <= fields["node_matrices_per_round"] <= 3 and fields["path"] in ("fp64_alu", "tensor_cores")
    ov, pp, par, st = run_gpu(ctx, data)
    check_pairs(pp, opp, sc, par)
    ctx.set_config(n, ne, 0)  # back to the built-in defaults for the other tests
