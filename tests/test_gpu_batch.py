"""Batched overlaps (qcs_overlap_batched): several active spaces in one
persistent launch, equal to the per-system results, and capturable in a
CUDA graph together with a stand-in walker propagation."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth

pytestmark = pytest.mark.gpu

SYSTEMS = [(8, 4, 17, 61), (12, 6, 9, 37), (16, 8, 7, 29), (20, 10, 5, 23), (24, 12, 3, 19)]


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def make_systems(ctx, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for n, ne, W, P in SYSTEMS:
        Q = synth.haar_orthogonal(rng, 2 * n, P)
        b = synth.uniform_bits(rng, n, P)
        Phi = synth.walkers(rng, n, ne, W)
        s = qcs.Snapshots(ctx, torch.from_numpy(Q).cuda(), torch.from_numpy(b).cuda())
        out.append(dict(Q=Q, b=b, Phi=Phi, s=s, walkers=torch.from_numpy(Phi).cuda()))
    return out


def test_batched_equals_per_system(ctx):
    systems = make_systems(ctx)
    res = qcs.overlap_batched(ctx, [(y["s"], y["walkers"]) for y in systems])
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    for y, r in zip(systems, res):
        # the batched launch runs the FP64 ALU pair kernel: same tiles, same reduction order
        single, _ = qcs.overlap(ctx, y["s"], y["walkers"], flags=qcs.QCS_FLAG_FP64_ALU)
        assert torch.equal(r, single)
    y = systems[0]
    oo, _, sc, _ = orc.overlap(y["Phi"], y["Q"], y["b"], per_pair=True)
    assert np.all(np.abs(res[0].cpu().numpy() - oo) <= 1e-10 * sc.mean(axis=1))


def test_batched_in_cuda_graph(ctx):
    """Capture three stand-in AFQMC steps (walkers <- U walkers with a fixed unitary
    per system, then the batched overlaps) in one CUDA graph and replay it."""
    systems = make_systems(ctx, seed=1)
    rng = np.random.default_rng(2)
    Us = []
    for n, ne, W, P in SYSTEMS:
        K = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        K = 0.05 * (K - K.conj().T)
        w, v = np.linalg.eigh(-1j * K)
        Us.append(torch.from_numpy((v * np.exp(1j * w)) @ v.conj().T).cuda())
    walkers0 = [y["walkers"].clone() for y in systems]
    outs = [torch.empty(y["walkers"].shape[0], dtype=torch.complex128, device="cuda") for y in systems]
    pairs = [(y["s"], y["walkers"]) for y in systems]

    def step():
        for y, U in zip(systems, Us):
            y["walkers"].copy_(torch.matmul(U, y["walkers"]))
        qcs.overlap_batched(ctx, pairs, outs=outs)

    # eager reference of three steps
    ref = []
    for _ in range(3):
        step()
        ref.append([o.clone() for o in outs])
    torch.cuda.synchronize()
    for y, w0 in zip(systems, walkers0):
        y["walkers"].copy_(w0)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()  # warm-up on the capture stream: sizes the workspace, loads kernels
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for y, w0 in zip(systems, walkers0):
        y["walkers"].copy_(w0)
    g = torch.cuda.CUDAGraph()
    got = []
    with torch.cuda.graph(g):
        step()
    for y, w0 in zip(systems, walkers0):
        y["walkers"].copy_(w0)
    for i in range(3):
        g.replay()
        torch.cuda.synchronize()
        got.append([o.clone() for o in outs])
    for a, b in zip(ref, got):
        for x, y in zip(a, b):
            assert torch.allclose(x, y, rtol=1e-12, atol=1e-14 * x.abs().max().item())


def test_batched_argument_errors(ctx):
    systems = make_systems(ctx, seed=3)
    with pytest.raises(ValueError):
        qcs.overlap_batched(ctx, [])
    with pytest.raises(ValueError):
        qcs.overlap_batched(ctx, [(systems[0]["s"], systems[1]["walkers"])])
