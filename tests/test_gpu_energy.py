"""Local-energy terms (qcs_local_energy) against the CPU oracle.  The two sides
take different routes: the GPU differentiates the pair Pfaffians with respect to
the selected rows after moving e^{lambda Lhat} onto the snapshot (Eqs.
Pfaffian_der, Pfaffian_2nd_der), the oracle substitutes columns of the walker
(the overlap is linear in each column) and never differentiates a Pfaffian.

Tolerance: e1 and e2 are ratios of shadow means; each numerator term is a sum over
nodes and operators of FP64 traces of O(m^3) products of quantities bounded by the
pair scale, the oracle's columns substitutions sum O(ne^2) overlaps per operator.
Both are accurate to about 1e-12 of the largest term; the test allows 1e-8 relative to
max(1, |value|), far below the O(1) change any formula error (a sign, a factor 2, a
missing term) produces.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def ctx():
    return qcs.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case(seed, n, ne, W, P, nchol, ens="haar", bits="uniform"):
    rng = np.random.default_rng(seed)
    Q = synth.haar_orthogonal(rng, 2 * n, P) if ens == "haar" else synth.signed_permutation(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P) if bits == "uniform" else synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, W)
    L = rng.standard_normal((nchol, n, n)) + 0.3j * rng.standard_normal((nchol, n, n))
    h = synth.cholesky_vectors(rng, n, 1)[0].astype(complex)
    return Q, b, Phi, L, h


@pytest.mark.parametrize("n,ne,W,P,nchol,ens", [(4, 2, 3, 30, 3, "haar"), (6, 4, 2, 25, 2, "haar"),
                                                (8, 4, 2, 20, 3, "haar"), (7, 2, 2, 15, 2, "signed_perm"),
                                                (16, 8, 2, 6, 2, "haar")])
def test_local_energy_matches_oracle(ctx, n, ne, W, P, nchol, ens):
    Q, b, Phi, L, h = case(500 + n + ne, n, ne, W, P, nchol, ens, bits="parity")
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, e1, e2 = qcs.local_energy(ctx, s, dev(Phi), dev(L), dev(h))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, o1, o2 = orc.local_energy(Phi, Q, b, L, h=h)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    assert np.all(np.abs(ov.cpu().numpy() - oo) <= 1e-10 * sc.mean(axis=1))
    for got, ref in ((e1, o1), (e2, o2)):
        got = got.cpu().numpy()
        assert np.all(np.abs(got - ref) <= TOL * np.maximum(1.0, np.abs(ref))), (got, ref)


@pytest.mark.parametrize("n,ne,flags", [(8, 4, qcs.QCS_FLAG_ALL_NODES), (12, 2, qcs.QCS_FLAG_ALL_NODES),
                                         (20, 10, 0)])
def test_node_rounds_and_larger_n(ctx, n, ne, flags):
    """More node matrices than one round holds (all 2n+1 roots of unity: 5 and 11 parity +1
    nodes, two and three rounds that repeat the per-operator work over the snapshot
    product staged once per pair), and n > 16 with the default plan."""
    Q, b, Phi, L, h = case(600 + n + ne, n, ne, 2, 12, 2, bits="parity")
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, e1, e2 = qcs.local_energy(ctx, s, dev(Phi), dev(L), dev(h), flags=flags)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, o1, o2 = orc.local_energy(Phi, Q, b, L, h=h)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    assert np.all(np.abs(ov.cpu().numpy() - oo) <= 1e-10 * sc.mean(axis=1))
    for got, ref in ((e1, o1), (e2, o2)):
        got = got.cpu().numpy()
        assert np.all(np.abs(got - ref) <= TOL * np.maximum(1.0, np.abs(ref))), (got, ref)


def test_one_body_term_matches_gradient_route(ctx):
    """e1 from qcs_local_energy equals tr(h G), G = Phi g^T / O, from the adjoint kernel and
    the force-bias kernel (i tr(L G) with L = h): two GPU routes."""
    Q, b, Phi, L, h = case(71, 16, 8, 3, 200, 1)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, e1, _ = qcs.local_energy(ctx, s, dev(Phi), dev(L), dev(h))
    ovg, g = qcs.overlap_grad(ctx, s, dev(Phi))
    vb = qcs.force_bias(ctx, dev(h[None]), dev(Phi), ovg, g)  # i tr(h G)
    torch.cuda.synchronize()
    ref = (-1j * vb[:, 0]).cpu().numpy()
    assert np.allclose(e1.cpu().numpy(), ref, rtol=1e-9, atol=1e-9)
    assert np.allclose(ov.cpu().numpy(), ovg.cpu().numpy(), rtol=1e-12, atol=0)


def test_without_one_body_operator(ctx):
    Q, b, Phi, L, h = case(72, 6, 2, 2, 12, 2)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, e1, e2 = qcs.local_energy(ctx, s, dev(Phi), dev(L))
    torch.cuda.synchronize()
    assert e1 is None
    _, _, o2 = orc.local_energy(Phi, Q, b, L)
    assert np.all(np.abs(e2.cpu().numpy() - o2) <= TOL * np.maximum(1.0, np.abs(o2)))


def test_one_body_operator_only(ctx):
    """No Cholesky vectors (nchol = 0): the per-snapshot sum over vectors is empty, e2 is
    exactly zero and e1 still matches the oracle."""
    Q, b, Phi, L, h = case(73, 8, 4, 3, 20, 1, bits="parity")
    n = Q.shape[1] // 2
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    L0 = torch.zeros((0, n, n), dtype=torch.complex128, device="cuda")
    ov, e1, e2 = qcs.local_energy(ctx, s, dev(Phi), L0, dev(h))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert np.all(e2.cpu().numpy() == 0)
    _, o1, _ = orc.local_energy(Phi, Q, b, L[:0], h=h)
    got = e1.cpu().numpy()
    assert np.all(np.abs(got - o1) <= TOL * np.maximum(1.0, np.abs(o1)))
