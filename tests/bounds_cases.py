"""Small parity cases run in a child process against the library that QCS_LIBRARY
names (the bounds-checked debug build in tests/test_gpu_bounds.py).  Prints one JSON
object: per case the device status word and the error against the oracle."""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle.oracle as orc  # noqa: E402
from paper_2506_22408_gb300 import qcs, synth  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def main():
    ctx = qcs.Context(0)
    out = {"library": qcs.library_path()}
    cases = [("tc", 16, 8, 5, 61, dict(flags=qcs.QCS_FLAG_FP64_TC)),
             ("alu", 16, 8, 5, 61, dict(flags=qcs.QCS_FLAG_FP64_ALU)),
             ("alu_small", 6, 2, 4, 37, {}),
             ("group_n20", 20, 10, 2, 13, {}),
             ("split", 16, 8, 5, 61, dict(precision=qcs.QCS_TF32X3))]
    for name, n, ne, W, P, kw in cases:
        rng = np.random.default_rng(77 + n + ne)
        Q = synth.haar_orthogonal(rng, 2 * n, P)
        b = synth.uniform_bits(rng, n, P)
        Phi = synth.walkers(rng, n, ne, W)
        s = qcs.Snapshots(ctx, dev(Q), dev(b))
        ov, pp = qcs.overlap(ctx, s, dev(Phi), per_pair=True, **kw)
        torch.cuda.synchronize()
        st = ctx.sync_status()
        oo, opp, sc, _ = orc.overlap(Phi, Q, b, per_pair=True)
        err = float((np.abs(pp.cpu().numpy() - opp) / sc).max())
        out[name] = {"status": st, "pair_err_over_scale": err}
    # adjoint and local energy
    n, ne, W, P = 8, 4, 3, 25
    rng = np.random.default_rng(91)
    Q = synth.haar_orthogonal(rng, 2 * n, P)
    b = synth.parity_consistent_bits(rng, Q)
    Phi = synth.walkers(rng, n, ne, W)
    s = qcs.Snapshots(ctx, dev(Q), dev(b))
    ov, g = qcs.overlap_grad(ctx, s, dev(Phi))
    torch.cuda.synchronize()
    st = ctx.sync_status()
    oo, og, _ = orc.overlap_grad(Phi, Q, b)
    out["grad"] = {"status": st, "rel_err": float(np.abs(g.cpu().numpy() - og).max() / np.abs(og).max())}
    L = rng.standard_normal((2, n, n)) + 0.3j * rng.standard_normal((2, n, n))
    h = synth.cholesky_vectors(rng, n, 1)[0].astype(complex)
    ov, e1, e2 = qcs.local_energy(ctx, s, dev(Phi), dev(L), dev(h))
    torch.cuda.synchronize()
    st = ctx.sync_status()
    oo, o1, o2 = orc.local_energy(Phi, Q, b, L, h=h)
    rel = max(float(np.abs(e1.cpu().numpy() - o1).max() / max(1.0, np.abs(o1).max())),
              float(np.abs(e2.cpu().numpy() - o2).max() / max(1.0, np.abs(o2).max())))
    out["energy"] = {"status": st, "rel_err": rel}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
