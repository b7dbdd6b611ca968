"""Parity of the CUDA adjoint (qcs_overlap_grad), the force bias and the
autograd wrapper with the CPU oracle, finite differences and exact identities.

Gradient tolerance: the oracle's gradient is exact up to rounding (entry (k, j)
is the overlap of the walker with column j replaced by e_k).  Each gradient entry
is a mean of per-pair terms whose magnitude is bounded by the pair scale s_p
times |A^{-1}| factors; the test bound is 1e-9 times the largest gradient
entry of the walker plus 1e-10 times the mean pair scale, which sits several
orders above FP64 rounding of these sums and far below any formula error
(a wrong sign or factor moves the result by O(1) relative).
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


def gpu_grad(ctx, Phi, Q, b, **kw):
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, g = qcs.overlap_grad(ctx, s, dev(Phi), **kw)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    return ov.cpu().numpy(), g.cpu().numpy(), st, s


def check_grad(g_gpu, g_orc, ov_gpu, ov_orc, sc, ov_floor=0.0):
    for w in range(g_orc.shape[0]):
        tol = 1e-9 * np.abs(g_orc[w]).max() + 1e-10 * sc[w].mean()
        assert np.abs(g_gpu[w] - g_orc[w]).max() <= tol, (w, np.abs(g_gpu[w] - g_orc[w]).max(), tol)
        assert abs(ov_gpu[w] - ov_orc[w]) <= 1e-10 * sc[w].mean() + ov_floor


@pytest.mark.parametrize("n,ne,W,P", [(8, 4, 5, 40), (6, 2, 3, 27), (16, 8, 3, 30), (12, 6, 2, 21),
                                      (10, 10, 2, 17), (24, 12, 1, 9)])
def test_gradient_matches_oracle(ctx, n, ne, W, P):
    rng = np.random.default_rng(1000 + n + ne)
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    ov, g, st, _ = gpu_grad(ctx, Phi, Q, b)
    assert st == 0
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    check_grad(g, og, ov, oo, sc)


@pytest.mark.parametrize("n,ne,ensemble", [(16, 8, "haar"), (16, 8, "signed_perm"), (12, 4, "signed_perm"),
                                           (10, 10, "haar")])
def test_gradient_structured_walkers(ctx, n, ne, ensemble):
    """Walkers in echelon form already, a reversed unit basis and walkers on the last
    modes only, against Haar snapshots and signed permutations: the occupied block of
    the node matrices is then often singular or badly pivoted, so both the block form
    and the full per-node elimination run.  Unit-vector walkers against signed
    permutations make some node matrices exactly singular, where the derivative
    formula (it needs A^{-1}) does not apply: the status word says so, and the
    generic walker's gradient must still be exact."""
    rng = np.random.default_rng(31 * n + ne)
    P = 40
    if ensemble == "haar":
        Q = synth.haar_orthogonal(rng, 2 * n, P)
    else:
        Q = synth.signed_permutation(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, 4)
    eye = np.eye(n, dtype=complex)
    R = np.triu(rng.standard_normal((ne, ne)) + 1j * rng.standard_normal((ne, ne))) + 2 * np.eye(ne)
    Phi[0] = eye[:, :ne] @ R
    Phi[1] = eye[:, ne - 1::-1]
    Phi[2] = eye[:, n - ne:] @ R
    ov, g, st, _ = gpu_grad(ctx, Phi, Q, b)
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    floor = 1e-12 * np.abs(og).max()
    if ensemble == "haar":
        assert st == 0
        check_grad(g, og, ov, oo, sc, ov_floor=floor)
    else:
        assert st in (0, qcs.QCS_ERR_SINGULAR)
        if st == 0:
            check_grad(g, og, ov, oo, sc, ov_floor=floor)
        else:
            check_grad(g[3:], og[3:], ov[3:], oo[3:], sc[3:], ov_floor=floor)
        assert np.all(np.abs(ov - oo) <= 1e-10 * sc.mean(axis=1) + floor)  # overlaps stay exact


def test_gradient_options_and_overlap_agree(ctx):
    rng = np.random.default_rng(5)
    n, ne, W, P = 8, 4, 4, 33
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    for kw in (dict(), dict(flags=qcs.QCS_FLAG_DFT_NODES), dict(flags=qcs.QCS_FLAG_ALL_NODES),
               dict(nodes=2 * n + 1)):
        ov, g, st, s = gpu_grad(ctx, Phi, Q, b, **kw)
        assert st == 0
        check_grad(g, og, ov, oo, sc)
    ov2, _ = qcs.overlap(ctx, s, dev(Phi))
    assert np.allclose(ov2.cpu().numpy(), ov, rtol=0, atol=1e-12 * sc.mean())


def test_gradient_identities_and_finite_differences(ctx):
    """g^T Phi = O I (the overlap is multilinear and alternating in the columns) and
    central finite differences of the GPU overlap along random complex directions."""
    rng = np.random.default_rng(6)
    n, ne, W, P = 16, 8, 2, 64
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    ov, g, st, s = gpu_grad(ctx, Phi, Q, b)
    assert st == 0
    for w in range(W):
        M = g[w].T @ Phi[w]
        assert np.abs(M - ov[w] * np.eye(ne)).max() <= 1e-9 * np.abs(g[w]).max() * np.abs(Phi[w]).max() * n
    E = rng.standard_normal((W, n, ne)) + 1j * rng.standard_normal((W, n, ne))
    h = 1e-5
    for step in (1.0, 1j):
        op, _ = qcs.overlap(ctx, s, dev(Phi + h * step * E))
        om, _ = qcs.overlap(ctx, s, dev(Phi - h * step * E))
        fd = (op - om).cpu().numpy() / (2 * h)
        an = step * np.einsum("wkj,wkj->w", g, E)
        assert np.all(np.abs(fd - an) <= 1e-6 * np.abs(an) + 1e-9 * np.abs(g).max())


def test_gradient_rank_deficient_walker(ctx):
    """adj(R) = det(R) R^{-1} without divisions: the gradient of a walker with two equal
    columns (overlap 0, gradient non-zero) still matches the oracle."""
    rng = np.random.default_rng(7)
    n, ne, P = 8, 4, 24
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, 2)
    Phi[0][:, 3] = Phi[0][:, 1]
    ov, g, st, _ = gpu_grad(ctx, Phi, Q, b)
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    _, _, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
    assert np.abs(og[0]).max() > 1e-3
    # the overlap itself is exactly 0 for walker 0: both sides are rounding noise of the
    # size of its gradient times its entries
    check_grad(g, og, ov, oo, sc, ov_floor=1e-12 * np.abs(og).max() * np.abs(Phi).max())


def test_force_bias(ctx):
    rng = np.random.default_rng(8)
    n, ne, W, P, nchol = 16, 8, 3, 40, 64
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    Phi = synth.walkers(rng, n, ne, W)
    L = synth.cholesky_vectors(rng, n, nchol).astype(np.complex128)
    ov, g, st, _ = gpu_grad(ctx, Phi, Q, b)
    for sdt in (0.0, 0.1):
        xb = qcs.force_bias(ctx, dev(L), dev(Phi), dev(ov), dev(g), sqrt_dt=sdt).cpu().numpy()
        ref = orc.force_bias(L, Phi, ov, g, sqrt_dt=sdt)
        assert np.abs(xb - ref).max() <= 1e-12 * np.abs(ref).max()
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    xo = orc.force_bias(L, Phi, oo, og)
    xg = qcs.force_bias(ctx, dev(L), dev(Phi), dev(ov), dev(g)).cpu().numpy()
    assert np.abs(xg - xo).max() <= 1e-7 * np.abs(xo).max()
    # complex operators without symmetry: L and L^T give different force biases
    Lc = rng.standard_normal((5, n, n)) + 1j * rng.standard_normal((5, n, n))
    xc = qcs.force_bias(ctx, dev(Lc), dev(Phi), dev(ov), dev(g)).cpu().numpy()
    refc = orc.force_bias(Lc, Phi, ov, g)
    assert np.abs(xc - refc).max() <= 1e-12 * np.abs(refc).max()
    refT = orc.force_bias(np.ascontiguousarray(Lc.transpose(0, 2, 1)), Phi, ov, g)
    assert np.abs(refT - refc).max() > 1e-3 * np.abs(refc).max()


def test_autograd_function(ctx):
    rng = np.random.default_rng(9)
    n, ne, W, P = 6, 2, 2, 16
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = dev(synth.walkers(rng, n, ne, W)).requires_grad_(True)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    f = lambda x: qcs.OverlapFn.apply(x, ctx, s)  # noqa: E731
    assert torch.autograd.gradcheck(f, (Phi,), eps=1e-6, atol=1e-7, rtol=1e-6)
    # backward of a real loss follows PyTorch's conjugate-Wirtinger convention:
    # loss = Re(sum out) gives grad = conj(dO/dPhi)
    out = f(Phi)
    out.real.sum().backward()
    _, g = qcs.overlap_grad(ctx, s, Phi.detach())
    assert torch.allclose(Phi.grad, g.conj(), rtol=0, atol=1e-12 * g.abs().max().item())
