"""The gradient and local-energy kernels eliminate the occupied block of the node
matrices once per pair and fall back to a full elimination per node when that block
gives a zero pivot (or grows the complement too much).  Signed-permutation snapshots
against unit-vector walkers at n = 6, ne = 2 make the occupied block exactly zero for
many pairs while every node matrix stays invertible; the snapshot set below keeps only
such snapshots (chosen on the CPU with the oracle), so both routes run in one launch and
the results must match the oracle at the tolerances of the gradient and energy tests.
"""
from __future__ import annotations

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


def fallback_case(n=6, ne=2, P=60, seed=7):
    rng = np.random.default_rng(seed)
    m, d = 2 * n - ne, n - ne
    eye = np.eye(n, dtype=complex)
    Phi = np.stack([eye[:, [0, 1]], eye[:, [3, 1]], eye[:, [5, 2]]]) @ np.array([[1.5, 0.4 - 0.2j], [0, 0.8]])
    Phi = np.concatenate([Phi, synth.walkers(rng, n, ne, 1)])
    wn, _ = qcs.node_plan(n, ne)
    D = np.zeros((m, m))
    for i in range(d):
        D[ne + 2 * i, ne + 2 * i + 1], D[ne + 2 * i + 1, ne + 2 * i] = 1.0, -1.0
    Qs, bs, zero_blocks = [], [], 0
    while len(Qs) < P:
        Q = synth.signed_permutation(rng, 2 * n, 1)[0]
        b = synth.parity_consistent_bits(rng, Q[None])[0]
        ok, zb = True, 0
        for w in range(len(Phi)):
            B, _, _ = orc.pair_matrices(Q, b, Phi[w])
            ok &= all(abs(orc.pfaffian(B + z * D)) > 1e-6 for z in wn)
            zb += np.abs(B[:ne, :ne]).max() == 0
        if ok:
            Qs.append(Q)
            bs.append(b)
            zero_blocks += zb
    return np.stack(Qs), np.stack(bs), Phi, zero_blocks


def test_gradient_fallback_route(ctx):
    Q, b, Phi, zero_blocks = fallback_case()
    assert zero_blocks >= 10  # the full elimination runs for these pairs
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, g = qcs.overlap_grad(ctx, s, dev(Phi))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    ov, g = ov.cpu().numpy(), g.cpu().numpy()
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    for w in range(len(Phi)):
        tol = 1e-9 * np.abs(og[w]).max() + 1e-10 * sc[w].mean()
        assert np.abs(g[w] - og[w]).max() <= tol, (w, np.abs(g[w] - og[w]).max(), tol)
        assert abs(ov[w] - oo[w]) <= 1e-10 * sc[w].mean()


def test_local_energy_fallback_route(ctx):
    Q, b, Phi, zero_blocks = fallback_case(seed=8)
    assert zero_blocks >= 10
    rng = np.random.default_rng(3)
    n = Q.shape[1] // 2
    L = rng.standard_normal((2, n, n)) + 0.3j * rng.standard_normal((2, n, n))
    h = synth.cholesky_vectors(rng, n, 1)[0].astype(complex)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, e1, e2 = qcs.local_energy(ctx, s, dev(Phi), dev(L), dev(h))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, o1, o2 = orc.local_energy(Phi, Q, b, L, h=h)
    for got, ref in ((e1, o1), (e2, o2)):
        got = got.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-8 * np.maximum(1.0, np.abs(ref))), (got, ref)
