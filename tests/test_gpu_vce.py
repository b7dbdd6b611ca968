"""Virtual-correlation-energy walker transform (qcs_vce_transform) against the
CPU oracle and the full-space determinant, and through the active-space shadow
overlap.  (act, factor) is unique only up to a unitary on the active columns
(act W, factor / det W), so the comparisons go through factor * det(chi^dag act),
which is unique, and through the overlap, which is linear in the walker's
determinant.  Tolerances: 1e-12 relative for determinants of O(1) matrices; the
overlap tolerance of the other GPU tests (1e-10 of the mean pair scale)."""
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


def rand_walkers(rng, W, NB, ne):
    return rng.standard_normal((W, NB, ne)) + 1j * rng.standard_normal((W, NB, ne))


@pytest.mark.parametrize("NB,nc,na,nea", [(40, 10, 8, 4), (20, 0, 8, 4), (14, 5, 6, 0), (80, 60, 16, 4),
                                          (9, 4, 5, 5), (30, 1, 24, 12)])
def test_vce_transform_matches_oracle(ctx, NB, nc, na, nea):
    rng = np.random.default_rng(NB + 7 * nc)
    W = 5
    Phi = rand_walkers(rng, W, NB, nc + nea)
    act, f = qcs.vce_transform(ctx, dev(Phi), nc, na, nea)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    act, f = act.cpu().numpy(), f.cpu().numpy()
    for w in range(W):
        ao, fo = orc.vce_transform(Phi[w], nc, na, nea)
        for _ in range(2):
            chi = rng.standard_normal((na, nea)) + 1j * rng.standard_normal((na, nea))
            ref = fo * np.linalg.det(chi.conj().T @ ao)
            got = f[w] * np.linalg.det(chi.conj().T @ act[w])
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


def test_vce_rank_deficient_core_gives_zero_factor(ctx):
    rng = np.random.default_rng(3)
    NB, nc, na, nea = 20, 4, 6, 2
    Phi = rand_walkers(rng, 2, NB, nc + nea)
    Phi[0, :nc, :] = 0.0  # the walker leaves the core empty: no overlap with a full core
    _, f = qcs.vce_transform(ctx, dev(Phi), nc, na, nea)
    torch.cuda.synchronize()
    assert f[0].item() == 0


def test_vce_two_spins_through_shadow_overlap(ctx):
    """Both spin sectors written as the diagonal blocks of one active walker (n = 2 na
    modes, ne = 2 nea); the active-space shadow overlap times the two factors equals the
    oracle's overlap of its own transformed walker times its factors."""
    rng = np.random.default_rng(11)
    NB, nc, na, nea, W, P = 30, 6, 8, 4, 4, 300
    Pa, Pb = rand_walkers(rng, W, NB, nc + nea), rand_walkers(rng, W, NB, nc + nea)
    act = torch.zeros((W, 2 * na, 2 * nea), dtype=torch.complex128, device="cuda")
    _, fa = qcs.vce_transform(ctx, dev(Pa), nc, na, nea, act=act, row0=0, col0=0)
    _, fb = qcs.vce_transform(ctx, dev(Pb), nc, na, nea, act=act, row0=na, col0=nea)
    n = 2 * na
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, _ = qcs.overlap(ctx, s, act)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    got = (ov * fa * fb).cpu().numpy()
    ref_walkers = np.zeros((W, n, 2 * nea), complex)
    fo = np.zeros(W, complex)
    for w in range(W):
        aa, fa_o = orc.vce_transform(Pa[w], nc, na, nea)
        ab, fb_o = orc.vce_transform(Pb[w], nc, na, nea)
        ref_walkers[w, :na, :nea], ref_walkers[w, na:, nea:] = aa, ab
        fo[w] = fa_o * fb_o
    oo, _, sc, _ = orc.overlap(ref_walkers, Q, b, per_pair=True)
    ref = oo * fo
    scale = sc.mean(axis=1) * np.abs(fo)
    assert np.all(np.abs(got - ref) <= 1e-10 * scale + 1e-12 * np.abs(ref))
