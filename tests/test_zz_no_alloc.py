"""qcs_overlap_noalloc, the allocation-free overlap entry point.

It exists for callers that cannot let a library allocate device memory when
they need overlaps (hosts whose pool allocator owns all device memory, real-time
loops that must not stall on cudaMalloc); its scratch is a fixed device array
inside the library.  These tests call it through the C ABI twice in a
row, with different sizes, and compare each result with the ordinary entry
point (qcs_build_snapshots + qcs_overlap) within the parity tolerance used by
the other GPU tests (1e-10 times the mean magnitude of the pair terms, taken
from the oracle).  The file is named so that pytest collects it last.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(seed, n, ne, W, P):
    rng = np.random.default_rng(seed)
    return dict(Q=synth.haar_orthogonal(rng, 2 * n, P), b=synth.uniform_bits(rng, n, P),
                Phi=synth.walkers(rng, n, ne, W))


def _reference(data):
    ctx = qcs.Context(0)
    s = qcs.Snapshots(ctx, _dev(data["Q"]), _dev(data["b"]))
    ov, _ = qcs.overlap(ctx, s, _dev(data["Phi"]))
    torch.cuda.synchronize()
    return ov.cpu().numpy()


def test_noalloc_matches_overlap_on_two_calls_in_a_row():
    cases = [_case(21, 16, 8, 40, 600), _case(22, 8, 4, 16, 256)]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for data in cases:
        W = data["Phi"].shape[0]
        out = torch.full((W,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        qcs.overlap_noalloc(_dev(data["Q"]), _dev(data["b"]), _dev(data["Phi"]), out, status)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _reference(data)
        _, _, sc, _ = orc.overlap(data["Phi"], data["Q"], data["b"], per_pair=True)
        assert np.all(np.abs(got - ref) <= TOL * sc.mean(axis=1))
    assert int(status.item()) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n, ne, W, P = 16, 8, 4, 5000  # 5000 snapshots of n = 16 need about 41 MB of scratch
    Q = torch.zeros((P, 2 * n, 2 * n), dtype=torch.float64, device="cuda")
    b = torch.zeros((P, n), dtype=torch.uint8, device="cuda")
    Phi = torch.zeros((W, n, ne), dtype=torch.complex128, device="cuda")
    out = torch.zeros(W, dtype=torch.complex128, device="cuda")
    with pytest.raises(qcs.QCSError) as e:
        qcs.overlap_noalloc(Q, b, Phi, out)
    assert e.value.code == 1
