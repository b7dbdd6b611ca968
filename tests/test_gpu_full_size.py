"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: sampled outputs the oracle computes one by one, whole walkers where the
oracle finishes in seconds, and properties that hold at any size where it does not.

Tolerances are those of the per-path test files: FP64 pairs 1e-10 of the pair scale
s_p, walker means 1e-10 of the mean pair scale, split precision 2e-5 s_p, local-energy
terms 1e-8 relative, RDM estimates 1e-12 of the channel weight.
"""
from __future__ import annotations

import dataclasses
from math import comb

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_differentiation_full_size(ctx):
    """512 walkers x 10000 snapshots, 64 Cholesky vectors: g^T Phi = O I for every walker,
    sampled walkers' overlaps against the oracle, and the force bias against the oracle's
    formula on the GPU gradient."""
    wl = synth.DIFFERENTIATION
    data = wl.generate(seed=0)
    s = qcs.Snapshots(ctx, dev(data["Q"]), dev(data["b"]))
    Pd = dev(data["Phi"])
    ov, g = qcs.overlap_grad(ctx, s, Pd)
    xb = qcs.force_bias(ctx, dev(data["L"].astype(complex)), Pd, ov, g, sqrt_dt=0.1)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    ov, g, xb = ov.cpu().numpy(), g.cpu().numpy(), xb.cpu().numpy()
    Phi = data["Phi"]
    M = np.einsum("wkj,wkl->wjl", g, Phi)  # g^T Phi
    eye = np.eye(wl.ne)
    for w in range(wl.W):
        assert np.abs(M[w] - ov[w] * eye).max() <= 1e-9 * np.abs(g[w]).max() * np.abs(Phi[w]).max() * wl.n
    sel = np.array([3, 200, wl.W - 1])
    oo, _, sc, _ = orc.overlap(Phi[sel], data["Q"], data["b"], per_pair=True)
    assert np.all(np.abs(ov[sel] - oo) <= 1e-10 * sc.mean(axis=1))
    ref = orc.force_bias(data["L"].astype(complex), Phi[sel], ov[sel], g[sel], sqrt_dt=0.1)
    assert np.abs(xb[sel] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_precision_full_size_sampled(ctx):
    """2048 walkers x 50000 snapshots in QCS_TF32X3: sampled pairs and two whole walkers
    against the oracle within the split path's bound."""
    wl = synth.PRECISION
    data = wl.generate(seed=0)
    s = qcs.Snapshots(ctx, dev(data["Q"]), dev(data["b"]))
    ov, pp = qcs.overlap(ctx, s, dev(data["Phi"]), per_pair=True, precision=qcs.QCS_TF32X3)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    rng = np.random.default_rng(8)
    ws, ps = rng.integers(0, wl.W, 120), rng.integers(0, wl.P, 120)
    got = pp[torch.from_numpy(ws).cuda(), torch.from_numpy(ps).cuda()].cpu().numpy()
    for k, (w, p) in enumerate(zip(ws, ps)):
        o, _, sc = orc.pair(data["Q"][p], data["b"][p], data["Phi"][w])
        assert abs(got[k] - o) <= 2e-5 * sc
    del pp
    sel = np.array([0, wl.W - 1])
    oo, _, sc, _ = orc.overlap(data["Phi"][sel], data["Q"], data["b"], per_pair=True)
    assert np.all(np.abs(ov.cpu().numpy()[sel] - oo) <= 2e-5 * sc.mean(axis=1))


@pytest.mark.parametrize("which", [3, 4])  # the n = 20 and n = 24 systems of the batching workload
def test_precision_large_n_full_size_sampled(ctx, which):
    """QCS_TF32X3 above 16 modes (64-row tiles, K = 48, a 64-thread group per walker) on the
    batching workload's n = 20 (128 x 20000) and n = 24 (64 x 40000) systems: sampled
    pairs against the oracle within the split path's bound, and one whole walker."""
    wl = synth.BATCH_SYSTEMS[which]
    assert wl.n > 16
    data = wl.generate(seed=0)
    s = qcs.Snapshots(ctx, dev(data["Q"]), dev(data["b"]))
    ov, pp = qcs.overlap(ctx, s, dev(data["Phi"]), per_pair=True, precision=qcs.QCS_TF32X3)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    rng = np.random.default_rng(9 + which)
    ws, ps = rng.integers(0, wl.W, 60), rng.integers(0, wl.P, 60)
    got = pp[torch.from_numpy(ws).cuda(), torch.from_numpy(ps).cuda()].cpu().numpy()
    for k, (w, p) in enumerate(zip(ws, ps)):
        o, _, sc = orc.pair(data["Q"][p], data["b"][p], data["Phi"][w])
        assert abs(got[k] - o) <= 2e-5 * sc
    del pp
    sel = np.array([wl.W - 1])
    oo, _, sc, _ = orc.overlap(data["Phi"][sel], data["Q"], data["b"], per_pair=True)
    assert np.all(np.abs(ov.cpu().numpy()[sel] - oo) <= 2e-5 * sc.mean(axis=1))


def test_batch_full_size_sampled(ctx):
    """The five active spaces at full size in one persistent launch: two walkers of each
    system against the oracle."""
    systems, datas = [], []
    for wl in synth.BATCH_SYSTEMS:
        d = wl.generate(seed=0)
        s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
        systems.append((s, dev(d["Phi"])))
        datas.append((wl, d))
    outs = qcs.overlap_batched(ctx, systems)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    for (wl, d), ov in zip(datas, outs):
        sel = np.array([0, wl.W - 1])
        oo, _, sc, _ = orc.overlap(d["Phi"][sel], d["Q"], d["b"], per_pair=True)
        assert np.all(np.abs(ov.cpu().numpy()[sel] - oo) <= 1e-10 * sc.mean(axis=1)), wl.name


def test_signed_permutation_full_size_sampled(ctx):
    """The paper-shaped size with signed-permutation snapshots (gather path): sampled pairs."""
    wl = dataclasses.replace(synth.PAPER_SHAPED, ensemble="signed_perm")
    data = wl.generate(seed=0)
    s = qcs.Snapshots(ctx, dev(data["Q"]), dev(data["b"]))
    assert s.signed_perm_count() == wl.P
    ov, pp = qcs.overlap(ctx, s, dev(data["Phi"]), per_pair=True)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    rng = np.random.default_rng(9)
    ws, ps = rng.integers(0, wl.W, 150), rng.integers(0, wl.P, 150)
    got = pp[torch.from_numpy(ws).cuda(), torch.from_numpy(ps).cuda()].cpu().numpy()
    floor = 1e-10 * np.abs(data["Phi"]).max() ** 4
    for k, (w, p) in enumerate(zip(ws, ps)):
        o, _, sc = orc.pair(data["Q"][p], data["b"][p], data["Phi"][w])
        assert abs(got[k] - o) <= 1e-10 * sc + floor


def test_rdm_full_size(ctx):
    """60000 snapshots at n = 16 (the bench's shadow count): every estimate against the oracle."""
    n, P = 16, 60000
    rng = np.random.default_rng(0)
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    out = qcs.shadow_rdm(ctx, s, deg4=True)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    ref = orc.shadow_rdm(Q, b, deg4=True)
    K2, K4 = comb(2 * n, 2) / n, comb(2 * n, 4) / comb(n, 2)
    assert np.abs(out["gam2"].cpu().numpy() - ref["gam2"]).max() <= 1e-12 * K2
    assert np.abs(out["gam4"].cpu().numpy() - ref["gam4"]).max() <= 1e-12 * K4
    assert np.abs(out["rdm1"].cpu().numpy() - ref["rdm1"]).max() <= 1e-12 * K2
    assert abs(out["npart"].item() - ref["npart"]) <= 1e-12 * K2 * n


def test_local_energy_bench_configuration(ctx):
    """64 walkers x 1000 snapshots with 64 Cholesky vectors (the bench's configuration):
    the one-body term against the adjoint route, the two-body term is additive over a
    split of the Cholesky vectors, and one walker against the oracle on two vectors."""
    n, ne, W, P, nchol = 16, 8, 64, 1000, 64
    rng = np.random.default_rng(0)
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    L = synth.cholesky_vectors(rng, n, nchol).astype(complex)
    h = synth.cholesky_vectors(rng, n, 1)[0].astype(complex)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, e1, e2 = qcs.local_energy(ctx, s, dev(Phi), dev(L), dev(h))
    ovg, g = qcs.overlap_grad(ctx, s, dev(Phi))
    vb = qcs.force_bias(ctx, dev(h[None]), dev(Phi), ovg, g)
    parts = [qcs.local_energy(ctx, s, dev(Phi), dev(L[k:k + 16]))[2] for k in range(0, nchol, 16)]
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    e1, e2 = e1.cpu().numpy(), e2.cpu().numpy()
    assert np.allclose(e1, (-1j * vb[:, 0]).cpu().numpy(), rtol=1e-9, atol=1e-9)
    tot = sum(p.cpu().numpy() for p in parts)
    assert np.all(np.abs(tot - e2) <= 1e-9 * np.maximum(1.0, np.abs(e2)))
    _, _, e2_two = qcs.local_energy(ctx, s, dev(Phi[:1]), dev(L[:2]))
    _, _, o2 = orc.local_energy(Phi[:1], Q, b, L[:2])
    assert abs(e2_two.cpu().numpy()[0] - o2[0]) <= 1e-8 * max(1.0, abs(o2[0]))


def test_vce_bench_configuration(ctx):
    """1024 full-space walkers with 200 orbitals, 20 core, 8 active orbitals and 4 active
    electrons per spin (the bench's configuration): sampled walkers against the oracle
    through the completion-independent product factor * det(chi^dag act)."""
    NB, nc, na, nea, W = 200, 20, 8, 4, 1024
    rng = np.random.default_rng(0)
    Phi = rng.standard_normal((W, NB, nc + nea)) + 1j * rng.standard_normal((W, NB, nc + nea))
    act, f = qcs.vce_transform(ctx, dev(Phi), nc, na, nea)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    act, f = act.cpu().numpy(), f.cpu().numpy()
    for w in (0, 511, W - 1):
        ao, fo = orc.vce_transform(Phi[w], nc, na, nea)
        chi = rng.standard_normal((na, nea)) + 1j * rng.standard_normal((na, nea))
        ref = fo * np.linalg.det(chi.conj().T @ ao)
        assert abs(f[w] * np.linalg.det(chi.conj().T @ act[w]) - ref) <= 1e-12 * abs(ref)
