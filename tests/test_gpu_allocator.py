"""qcs_set_allocator: the library's device memory from the caller's allocator.

With PyTorch's caching allocator behind a context (Context.use_torch_allocator), the
workspace, the buffers of snapshot sets built on the context and the tensor-core slice
records come from torch (the callbacks are counted); results are bit-identical to a
context on cudaMalloc; after one call with the largest sizes, a call captured in a CUDA
graph allocates nothing, and the replayed graph gives the overlaps of the changed
walkers; going back to cudaMalloc returns the workspace to torch.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.oracle as orc
from paper_2506_22408_gb300 import qcs, synth
from parity_checks import check_walkers_relative

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make(seed, n=16, ne=8, W=12, P=100):
    rng = np.random.default_rng(seed)
    return dict(Q=synth.haar_orthogonal(rng, 2 * n, P), b=synth.uniform_bits(rng, n, P),
                Phi=synth.walkers(rng, n, ne, W))


def test_torch_allocator_backs_workspace_and_snapshot_sets():
    d = make(1)
    plain = qcs.Context(0)
    s0 = qcs.Snapshots(plain, dev(d["Q"]), dev(d["b"]))
    ref, _ = qcs.overlap(plain, s0, dev(d["Phi"]))
    ctx = qcs.Context(0)
    ctx.use_torch_allocator()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    n_set = ctx.alloc_calls
    assert n_set == 6  # rows, parity, list, counts, gather codes, tensor-core records (n = 16)
    ov, _ = qcs.overlap(ctx, s, dev(d["Phi"]))
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert ctx.alloc_calls == n_set + 1  # the workspace
    assert torch.cuda.memory_allocated() - before >= ctx.workspace_bytes()
    assert torch.equal(ov, ref)
    s.close()
    assert ctx.free_calls == n_set


def test_no_library_allocation_inside_a_captured_graph():
    d = make(2, W=16, P=160)
    ctx = qcs.Context(0)
    ctx.use_torch_allocator()
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    walkers = dev(d["Phi"])
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        qcs.overlap(ctx, s, walkers)  # warm-up: the workspace grows to this call's size
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    calls = ctx.alloc_calls
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out, _ = qcs.overlap(ctx, s, walkers)
    assert ctx.alloc_calls == calls  # nothing allocated by the library during capture
    rng = np.random.default_rng(3)
    new = synth.walkers(rng, 16, 8, 16)
    walkers.copy_(dev(new))
    g.replay()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    oo, _, sc, _ = orc.overlap(new, d["Q"], d["b"], per_pair=True)
    got = out.cpu().numpy()
    assert np.all(np.abs(got - oo) <= 1e-10 * sc.mean(axis=1))
    check_walkers_relative(got, oo, sc)
    assert ctx.alloc_calls == calls


def test_back_to_cuda_malloc():
    d = make(4, n=12, ne=6)
    ctx = qcs.Context(0)
    ctx.use_torch_allocator()
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    qcs.overlap(ctx, s, dev(d["Phi"]))
    torch.cuda.synchronize()
    a, f = ctx.alloc_calls, ctx.free_calls
    ctx.use_cuda_malloc()  # the workspace goes back to torch
    assert ctx.free_calls == f + 1
    ov, _ = qcs.overlap(ctx, s, dev(d["Phi"]))  # regrows with cudaMalloc
    torch.cuda.synchronize()
    assert ctx.alloc_calls == a and ctx.sync_status() == 0
    oo, _, sc, _ = orc.overlap(d["Phi"], d["Q"], d["b"], per_pair=True)
    assert np.all(np.abs(ov.cpu().numpy() - oo) <= 1e-10 * sc.mean(axis=1))
    s.close()  # the set frees through the allocator it was built with
    # n = 12: no tensor-core records by default, and the one-warp FP64 ALU path forms no
    # rows [H1^T; G2^T]: Qt, parity, list, counts and gather codes
    assert ctx.free_calls == f + 1 + 5


def test_rows_for_K_are_formed_once_per_set():
    """Above 16 modes the FP64 ALU path forms K = U^T [H1 | G2] from rows [H1^T; G2^T] that
    the snapshot set builds on first use, through the set's allocator; later calls reuse
    them, and closing the set frees them."""
    d = make(5, n=20, ne=10, W=8, P=64)
    ctx = qcs.Context(0)
    ctx.use_torch_allocator()
    s = qcs.Snapshots(ctx, dev(d["Q"]), dev(d["b"]))
    n_set = ctx.alloc_calls
    assert n_set == 5  # rows, parity, list, counts, gather codes (no tensor-core records above 16)
    walkers = dev(d["Phi"])
    ov, _ = qcs.overlap(ctx, s, walkers)
    torch.cuda.synchronize()
    assert ctx.alloc_calls == n_set + 2  # the workspace and the rows [H1^T; G2^T]
    ov2, _ = qcs.overlap(ctx, s, walkers)
    torch.cuda.synchronize()
    assert ctx.alloc_calls == n_set + 2 and ctx.sync_status() == 0
    assert torch.equal(ov, ov2)
    oo, _, sc, _ = orc.overlap(d["Phi"], d["Q"], d["b"], per_pair=True)
    got = ov.cpu().numpy()
    assert np.all(np.abs(got - oo) <= 1e-10 * sc.mean(axis=1))
    check_walkers_relative(got, oo, sc)
    f = ctx.free_calls
    s.close()
    assert ctx.free_calls == f + n_set + 1
