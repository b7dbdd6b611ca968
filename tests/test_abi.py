"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/qcs.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

from paper_2506_22408_gb300 import _build, qcs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qcs.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qcs_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14
    missing = [nm for nm in names if not hasattr(lib, nm)]
    assert not missing, missing
    assert set(qcs.EXPORTED) == set(names)


def test_flop_accounting_host_only():
    lib = qcs.load()
    f16 = lib.qcs_overlap_flops_per_pair(16, 8, 0, 0)       # Gauss plan: 3 Pfaffians
    f16_dft = lib.qcs_overlap_flops_per_pair(16, 8, 0, 2)   # 5 of 9 roots of unity
    f16_all = lib.qcs_overlap_flops_per_pair(16, 8, 0, 1)   # all 9 roots
    assert 0.9e5 < f16 < f16_dft < f16_all < 3.0e5

    def tri(k):
        return k * (k - 1) // 2

    def step(r):  # one elimination step of an r x r Pfaffian: Gauss vectors + rank-2 update
        return 16 * tri(r - 2) + 6 * (r - 2)

    n, ne = 16, 8
    d, m = n - ne, 2 * n - ne
    # every n: three real products per complex multiply-add over the non-zero walker
    # entries (occupied rows in reduced form), 3 sums per entry of T and re + im of each
    # snapshot entry
    t_3m = 6 * 2 * n * (n * n - ne * (ne - 1) - tri(d)) + 3 * 2 * n * n + 2 * n * n  # reduced form
    # B from T: 2n-term sums per entry (n <= 16, and signed-permutation snapshots)
    b_flops = 16 * n * tri(ne) + 8 * n * ne * 2 * d + 4 * n * tri(2 * d)

    def b_from_k(n, ne):
        # above 16 modes, B from K = U^T [H1 | G2] over the walker rows' non-zero columns, three
        # real products per term: occupied rows in reduced form (1 + d columns, W1 alone),
        # completion row ne + j with ne + j + 1 items of W1 and W2 over n - j columns, halved
        # sums and differences per occupied-empty and empty pair, re + im of K
        d = n - ne
        oo = tri(ne) * (6 * (1 + d) + 3)
        rows = sum((ne + j + 1) * (12 * (n - j) + 6) for j in range(d))
        return oo + rows + 8 * ne * d + 8 * tri(d) + d + 2 * n * n

    shared = sum(step(r) for r in range(m, 2 * d, -2))
    node = sum(step(r) for r in range(2 * d, 2, -2))
    assert f16 == t_3m + b_flops + shared + 3 * node
    assert f16_dft == t_3m + b_flops + shared + 5 * node
    assert lib.qcs_overlap_flops_per_pair_signed_perm(16, 8, 0, 0) == b_flops + shared + 3 * node
    parts = qcs.flops_breakdown(16, 8)
    assert (parts["T"], parts["B"], parts["pfaffian"]) == (t_3m, b_flops, shared + 3 * node)
    # other n: the same form (the one-warp path below 16 modes, two-warp groups above)
    for n, ne in ((12, 6), (20, 10), (24, 4), (24, 12)):
        d = n - ne
        p12 = qcs.flops_breakdown(n, ne)
        assert p12["T"] == 6 * 2 * n * (n * n - ne * (ne - 1) - tri(d)) + 3 * 2 * n * n + 2 * n * n
        bt = 16 * n * tri(ne) + 8 * n * ne * 2 * d + 4 * n * tri(2 * d)
        assert p12["B"] == (b_from_k(n, ne) if n > 16 else bt)
        if n > 16:
            assert p12["B"] < bt
        assert lib.qcs_overlap_flops_per_pair(n, ne, 0, 0) == sum(p12.values())
    assert lib.qcs_overlap_flops_per_pair(16, 7, 0, 0) == 0.0  # odd ne rejected


def test_gradient_flop_accounting_host_only():
    lib = qcs.load()

    def tri(k):
        return k * (k - 1) // 2

    def step(r):  # one elimination step of an r x r Pfaffian
        return 16 * tri(r - 2) + 6 * (r - 2)

    def bstep(rv):  # one backward step of the inverse with rv later indices
        return 16 * rv * rv + 20 * rv

    n, ne, nev = 16, 8, 3  # Gauss plan: 3 nodes
    d, m = n - ne, 2 * n - ne
    macs = 2 * n * (n * n - tri(ne) - tri(d))       # echelon-form walker rows
    t = 6 * macs + 3 * 2 * n * n + 2 * n * n        # three real products per term
    b = 16 * n * tri(ne) + 8 * n * ne * 2 * d + 4 * n * tri(2 * d)
    elim = sum(step(r) for r in range(m, 2 * d, -2)) + nev * sum(step(r) for r in range(2 * d, 2, -2))
    inv = nev * (sum(bstep(rv) for rv in range(2 * d - 2, 0, -2)) + 8 * tri(2 * d))
    inv += sum(bstep(rv) for rv in range(2 * d, m - 1, 2))
    # B from K = Ut [H1 | G2] instead of from T: two n-term complex sums per work item, three
    # real products per term, plus the staged sums of Ut and K
    items = tri(ne) + ne * d + tri(d + 1)
    bk = (12 * n + 6) * items + 8 * ne * d + 8 * tri(d) + d + 3 * n * n + 2 * d * n
    # cotangents from K: coefficient rows and their sums, then n x n entries of m complex
    # multiply-adds with three real products each
    gam = 8 * ne * d + d * (16 * d + 2 * ne) + n * m + 6 * n * n * m + 5 * n * n
    f = lib.qcs_grad_flops_per_pair(16, 8, 0, 0)
    assert f == t + bk + elim + inv + gam
    # signed permutations: T is a gather, B from T, G_X on the occupied rows and Ht = Yh (X J)
    # on the empty modes (Yh = Y[ne+2i] - i Y[ne+2i+1]), each cotangent entry two complex additions
    gx = 2 * d * m + n * 2 * n * (8 * ne + 4 * (m - ne)) + 4 * n * n
    fs = lib.qcs_grad_flops_per_pair_signed_perm(16, 8, 0, 0)
    assert fs == f - t - bk + b - gam + gx
    assert lib.qcs_grad_flops_per_pair(16, 7, 0, 0) == 0.0


def test_host_only_size_checks():
    """The host-only accounting calls accept every size the library supports
    (1 <= n <= QCS_MAX_N, even ne with 2 <= ne <= n) and return 0 otherwise."""
    lib = qcs.load()
    maxn = 24
    calls = [lambda n, ne: lib.qcs_overlap_flops_per_pair(n, ne, 0, 0),
             lambda n, ne: lib.qcs_overlap_flops_per_pair_signed_perm(n, ne, 0, 0),
             lambda n, ne: lib.qcs_grad_flops_per_pair(n, ne, 0, 0),
             lambda n, ne: lib.qcs_grad_flops_per_pair_signed_perm(n, ne, 0, 0),
             lambda n, ne: lib.qcs_local_energy_flops_per_pair(n, ne, 4, 1, 0, 0)]
    for f in calls:
        for n, ne in [(2, 2), (16, 8), (maxn, 2), (maxn, maxn), (maxn, 12)]:
            assert f(n, ne) > 0.0, (n, ne)
        for n, ne in [(maxn + 1, 2), (16, 7), (8, 10), (8, 0)]:
            assert f(n, ne) == 0.0, (n, ne)
    assert lib.qcs_shadow_rdm_flops(16, 1000) > 0.0
    parts = (ctypes.c_double * 3)()
    assert lib.qcs_overlap_flops_breakdown(maxn + 1, 2, 0, 0, parts) == qcs.QCS_ERR_ARG
    assert lib.qcs_overlap_flops_breakdown(16, 8, 0, 0, None) == qcs.QCS_ERR_ARG
    assert lib.qcs_selftest_reciprocal(None, None, None, 0, None) == qcs.QCS_ERR_ARG  # no context: no device work


def test_tensor_core_work_accounting_host_only():
    """The tensor-core congruence's work per non-trivial pair: the FP64 part is the
    Pfaffian eliminations of the ALU count plus two additions per occupied x occupied
    entry of B^(s); the tensor part two sliced products of 28 slice products each."""
    parts = qcs.flops_breakdown(16, 8)
    w = qcs.tc_work_per_pair(16, 8)
    assert w["fp64"] == parts["pfaffian"] + 2 * (8 * 7 // 2)
    assert w["tensor"] == 2 * 28 * 2 * 32 ** 3
    w_dft = qcs.tc_work_per_pair(16, 8, 0, qcs.QCS_FLAG_DFT_NODES)
    assert w_dft["fp64"] == qcs.flops_breakdown(16, 8, 0, qcs.QCS_FLAG_DFT_NODES)["pfaffian"] + 56
    import pytest
    with pytest.raises(qcs.QCSError):
        qcs.tc_work_per_pair(20, 10)  # n > 16 has no tensor-core congruence


def test_config_encoding_round_trip():
    """qcs_opts.config fields (host-side helpers): a plain k is k node matrices per round,
    and every field survives encode -> decode."""
    assert qcs.decode_config(3) == {"node_matrices_per_round": 3, "alu_snapshots_per_warp": 0,
                                    "alu_warps_per_pair": 0, "path": "default", "tc_subtiles_per_tile": 0}
    c = qcs.encode_config(node_matrices_per_round=5, alu_snapshots_per_warp=8, alu_warps_per_pair=1, path=2,
                          tc_subtiles_per_tile=15)
    assert c == 5 | 8 << 4 | 1 << 8 | 2 << 10 | 15 << 12
    f = qcs.decode_config(c)
    assert (f["node_matrices_per_round"], f["alu_snapshots_per_warp"], f["alu_warps_per_pair"], f["path"],
            f["tc_subtiles_per_tile"]) == (5, 8, 1, "tensor_cores", 15)
