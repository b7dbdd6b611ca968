"""Writes qcs_gauss_nodes.h: quadrature rules for the shadow estimator's weighted
coefficient sum, for every n <= 24 and even ne <= n.

What the rules compute.  For a parity +1 snapshot the Pfaffian polynomial
q(z) = pf(A(z)) / z^{ne/2} of degree d = n - ne is palindromic (q_t = q_{d-t}),
and the estimator needs only the linear functional

    L(q) = sum_{t=0..d} w_t q_t,   w_t = C(2n, ne + 2t) / C(n, ne/2 + t)   (o_p formula after Eq. b_mat),

whose weights are symmetric too (w_t = w_{d-t}).  On the unit circle z = e^{i theta},

    q(z) e^{-i d theta / 2} = sum_t q_t cos((t - d/2) theta),

so a rule  L(q) = sum_j beta_j q(z_j) e^{-i d theta_j / 2}  must satisfy
sum_j beta_j cos(u theta_j) = w_{d/2+u} for every u = |t - d/2|, i.e. for
D = floor(d/2) + 1 values of u.

* d even: cos(u theta) = T_u(x), x = cos theta, so the conditions say that the
  rule integrates the Chebyshev polynomials T_0..T_{D-1} to the "Chebyshev
  moments" w_{d/2+u}.  A Gauss rule with k = ceil(D/2) nodes x_j does that
  (it is exact up to degree 2k-1 >= D-1).
* d odd: u = 1/2, 3/2, ..., with phi = theta/2 and s = cos phi,
  cos(u theta) = T_{2u}(s) = s P_u(s^2), so in y = s^2 the conditions become a
  moment problem for polynomials of degree <= D-1 with weights beta_j s_j:
  again a Gauss rule with k = ceil(D/2) nodes y_j; theta_j = 2 arccos(sqrt(y_j)).

When D is odd the rule needs one moment beyond the conditions (order 2k-1);
it takes the next weight of the same formula, w_{d+1} (valid since
ne/2 + d + 1 <= n).  The nodes and weights come from the Golub-Welsch method
(Cholesky of the moment Hankel matrix, eigen-decomposition of the Jacobi
matrix) at 80 significant digits, and every rule is checked on random
palindromic polynomials before it is written.  All rules obtained have real
nodes inside the interval (all z_j on the unit circle) and positive weights.

The kernels evaluate pf(B + wnode_j D) = q(z_j) / z_j^d and sum
gamma_j pf_j, so the table stores wnode_j = e^{-i theta_j} and
gamma_j = beta_j e^{i d theta_j / 2}.

Run:  python gen_gauss_nodes.py   (needs mpmath; writes qcs_gauss_nodes.h beside it)
"""
from __future__ import annotations

import os
import random
from math import comb

import mpmath as mp

mp.mp.dps = 80
MAX_N = 24
MAX_K = 6


def wt(n: int, ne: int, t: int):
    return mp.mpf(comb(2 * n, ne + 2 * t)) / comb(n, ne // 2 + t)


def gauss(mom, k):
    """k-point Gauss rule for monomial moments mom[0..2k] (Golub-Welsch)."""
    H = mp.matrix(k + 1, k + 1)
    for i in range(k + 1):
        for j in range(k + 1):
            H[i, j] = mom[i + j]
    R = mp.cholesky(H).T
    a = [R[j, j + 1] / R[j, j] - (R[j - 1, j] / R[j - 1, j - 1] if j > 0 else 0) for j in range(k)]
    b = [R[j + 1, j + 1] / R[j, j] for j in range(k - 1)]
    J = mp.matrix(k, k)
    for j in range(k):
        J[j, j] = a[j]
        if j + 1 < k:
            J[j, j + 1] = J[j + 1, j] = b[j]
    E, V = mp.eigsy(J)
    return [E[i] for i in range(k)], [mom[0] * V[0, i] ** 2 for i in range(k)]


def rule(n: int, ne: int):
    d = n - ne
    D = d // 2 + 1
    k = (D + 1) // 2
    # moment of order 2k uses weights beyond the conditions only inside the
    # Cholesky's last pivot, which does not enter the Jacobi matrix
    def w_ext(t):
        return wt(n, ne, t) if ne // 2 + t <= n else mp.mpf(0)

    if d % 2 == 0:
        cheb = [w_ext(d // 2 + u) for u in range(2 * k + 1)]
        mom = []
        for p in range(2 * k + 1):  # x^p = 2^{-p} sum_i C(p, i) T_{|p - 2i|}(x)
            mom.append(sum(comb(p, i) * cheb[abs(p - 2 * i)] for i in range(p + 1)) / mp.mpf(2) ** p)
        xs, bs = gauss(mom, k)
        thetas = [mp.acos(x) for x in xs]
        betas = bs
    else:
        def m_odd(j):  # Chebyshev moment of T_j(s), j odd: w at t = (d + j) / 2
            return w_ext((d + j) // 2)

        mom = []
        for p in range(2 * k + 1):  # s^{2p+1} = 2^{-2p} sum_{i<=p} C(2p+1, i) T_{2p+1-2i}(s)
            mom.append(sum(comb(2 * p + 1, i) * m_odd(2 * p + 1 - 2 * i) for i in range(p + 1)) / mp.mpf(4) ** p)
        ys, bs = gauss(mom, k)
        thetas = [2 * mp.acos(mp.sqrt(y)) for y in ys]
        betas = [b / mp.sqrt(y) for b, y in zip(bs, ys)]
    return d, thetas, betas


def check(n, ne, d, thetas, betas):
    assert all(b > 0 for b in betas), (n, ne, "negative weight")
    assert all(0 <= th <= mp.pi for th in thetas), (n, ne, "node off the unit circle")
    rng = random.Random(1000 * n + ne)
    for _ in range(8):
        half = [mp.mpf(rng.uniform(-1, 1)) + 1j * mp.mpf(rng.uniform(-1, 1)) for _ in range(d // 2 + 1)]
        q = [half[min(t, d - t)] for t in range(d + 1)]
        exact = sum(wt(n, ne, t) * q[t] for t in range(d + 1))
        scale = sum(wt(n, ne, t) * abs(q[t]) for t in range(d + 1))
        got = 0
        for th, b in zip(thetas, betas):
            z = mp.expj(th)
            qz = sum(q[t] * z ** t for t in range(d + 1))
            pf = qz / z ** d                               # what the kernels evaluate
            got += b * mp.expj(d * th / 2) * pf            # gamma_j pf_j
        assert abs(got - exact) <= mp.mpf(10) ** -60 * scale, (n, ne, float(abs(got - exact) / scale))


def main():
    rows = []
    for n in range(0, MAX_N + 1):
        for ne in range(0, MAX_N + 1):
            if n < 2 or ne < 2 or ne > n or ne % 2:
                rows.append((0, []))
                continue
            d, thetas, betas = rule(n, ne)
            check(n, ne, d, thetas, betas)
            assert len(thetas) <= MAX_K
            nodes = []
            for th, b in zip(thetas, betas):
                wn = mp.expj(-th)
                g = b * mp.expj(d * th / 2)
                nodes.append((wn.real, wn.imag, g.real, g.imag))
            rows.append((len(nodes), nodes))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qcs_gauss_nodes.h")
    with open(out, "w") as f:
        f.write("// qcs_gauss_nodes.h -- written by gen_gauss_nodes.py (do not edit).\n")
        f.write("// Gauss rules for sum_t w_t q_t over palindromic Pfaffian polynomials q of\n")
        f.write("// degree d = n - ne (weights of the o_p formula), indexed [n][ne]: k nodes, and per node\n")
        f.write("// wnode = e^{-i theta} (multiplier of D) and gamma = beta e^{i d theta / 2}.\n")
        f.write("#pragma once\n\n")
        f.write(f"#define QCS_GAUSS_MAX_N {MAX_N}\n#define QCS_GAUSS_MAX_K {MAX_K}\n\n")
        f.write("struct qcs_gauss_rule {\n    int k;\n    double node[QCS_GAUSS_MAX_K][4];  // wnode re, im, gamma re, im\n};\n\n")
        f.write(f"static const qcs_gauss_rule qcs_gauss_rules[{MAX_N + 1}][{MAX_N + 1}] = {{\n")
        for i, (k, nodes) in enumerate(rows):
            n, ne = divmod(i, MAX_N + 1)
            if ne == 0:
                f.write("  {\n")
            if k == 0:
                f.write("    {0, {}},\n")
            else:
                body = ", ".join("{" + ", ".join(mp.nstr(v, 25, strip_zeros=False, min_fixed=0, max_fixed=0)
                                                 for v in node) + "}" for node in nodes)
                f.write(f"    {{{k}, {{{body}}}}},  // n = {n}, ne = {ne}\n")
            if ne == MAX_N:
                f.write("  },\n")
        f.write("};\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
