"""Shadow estimates of Majorana correlators, the 1-RDM and the particle number
(qcs_shadow_rdm) against the CPU oracle, element by element, on the same
snapshots: plain and rotated Majoranas, Haar and signed-permutation snapshots,
several n including the largest supported.

Tolerances: every estimate is a mean of per-snapshot terms bounded by the channel
weight K_|S| = C(2n,|S|)/C(n,|S|/2) times a small integer (covariance entries of an
orthogonal matrix are at most 1 in magnitude), summed in FP64 in a different order on
the two sides; the bound 1e-12 K_|S| sits well above that rounding and far below any
formula error (a wrong sign, index or weight moves an entry by O(K)).
"""
from __future__ import annotations

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


@pytest.mark.parametrize("n,P,rot,ens", [(3, 50, False, "haar"), (8, 400, True, "haar"), (16, 1000, False, "haar"),
                                         (16, 700, True, "signed_perm"), (11, 300, True, "haar"),
                                         (24, 60, False, "haar")])
def test_rdm_matches_oracle(ctx, n, P, rot, ens):
    rng = np.random.default_rng(900 + n + P)
    Q = synth.haar_orthogonal(rng, 2 * n, P) if ens == "haar" else synth.signed_permutation(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    R = synth.haar_orthogonal(rng, 2 * n, 1)[0] if rot else None
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    out = qcs.shadow_rdm(ctx, s, R=dev(R) if rot else None, deg4=True)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    ref = orc.shadow_rdm(Q, b, R=R, deg4=True)
    K2, K4 = comb(2 * n, 2) / n, comb(2 * n, 4) / comb(n, 2)
    assert np.abs(out["gam2"].cpu().numpy() - ref["gam2"]).max() <= 1e-12 * K2
    assert np.abs(out["gam4"].cpu().numpy() - ref["gam4"]).max() <= 1e-12 * K4
    assert np.abs(out["rdm1"].cpu().numpy() - ref["rdm1"]).max() <= 1e-12 * K2
    assert abs(out["npart"].item() - ref["npart"]) <= 1e-12 * K2 * n


def test_rdm_is_deterministic_and_optional_outputs(ctx):
    rng = np.random.default_rng(31)
    n, P = 16, 3000
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.uniform_bits(rng, n, P)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    a = qcs.shadow_rdm(ctx, s, deg4=True)
    c = qcs.shadow_rdm(ctx, s, deg4=False)  # no four-Majorana estimates: no moment update
    torch.cuda.synchronize()
    assert torch.equal(a["gam2"], c["gam2"]) and torch.equal(a["rdm1"], c["rdm1"])
    a2 = qcs.shadow_rdm(ctx, s, deg4=True)
    torch.cuda.synchronize()
    assert torch.equal(a["gam4"], a2["gam4"])
    # 1-RDM is Hermitian (the estimator's 2-point matrix is real antisymmetric)
    D = a["rdm1"].cpu().numpy()
    assert np.abs(D - D.conj().T).max() <= 1e-13 * np.abs(D).max()
