// qcs_energy.cu -- local-energy terms of the shadow overlap by Pfaffian derivatives
// (Eqs. force_bias_diff, energy_tb_diff, Pfaffian_der, Pfaffian_2nd_der).
//
// For a one-body operator Lhat = sum_pq L_pq a_p^dag a_q the walker moves as
// Phi -> e^{lambda L} Phi.  Because <0| Lhat = 0, e^{lambda Lhat}|phi><0| is the
// similarity e^{lambda Lhat} (|phi><0|) e^{-lambda Lhat}; the inverse shadow channel
// only rescales Majorana degrees, which such similarities preserve, so the pair
// estimate of the moved walker equals that of the fixed walker against the snapshot
// e^{-lambda Lhat} rho_p e^{lambda Lhat}, whose covariance is R G_p R^T with
// R = e^{lambda ell}, [Lhat, g_mu] = sum_a ell_{mu a} g_a.  In the pair matrices
// B = K G K^T (K: the walker's selected rows, m x 2n) this is K -> K e^{lambda ell}:
//     A'  = X' J X^T + X J X'^T,                 X'  = (K ell) Q'^T,
//     A'' = X'' J X^T + 2 X' J X'^T + X J X''^T,  X'' = (K ell^2) Q'^T,
// with X = K Q'^T the rows the overlap kernels already form from T.  Eq.
// (Pfaffian_2nd_der) then gives per node matrix A_k = B + w_k D
//     d^2 pf = (pf/2) [ tr(A^-1 A'') - tr(A^-1 A' A^-1 A') + tr(A^-1 A')^2 / 2 ],
// and Eq. (Pfaffian_der) d pf = (pf/2) tr(A^-1 A').  The walker prefactor cancels in
//     e1 = sum_p D o_p[hhat] / sum_p o_p,   e2 = sum_gamma sum_p D^2 o_p[Lhat_gamma] / sum_p o_p.
// The node matrices share their occupied block P (ne x ne): with E = P^-1 B_oe,
// F = [-E; I], F0 = [[P^-1, 0], [0, 0]] and Z_k the inverse of the node's 2d x 2d
// complement, A_k^-1 = F0 + F Z_k F^T, so with W = A' F, G = F^T W and
// H = -W_o^T P^-1 W_o the traces need only 2d x 2d work per node:
//     tr(A_k^-1 A') = tr(P^-1 A'_oo) + tr(Z_k G),
//     tr((A_k^-1 A')^2) = tr((P^-1 A'_oo)^2) + 2 tr(Z_k H) + tr((Z_k G)^2).
// P^-1 comes from the backward recursion over the shared steps (qcs_group.cuh) run
// with Z = 0; pairs whose occupied block would grow the complement beyond 2^8 take
// the full inverse per node.  The snapshot enters the operator terms through
// Mt = (Q'^T J X^T)^T, formed once per pair: X' J X^T = (K ell) Mt^T, so A' is
// (K ell) Mt^T minus its transpose and X' itself is never formed.  Per Cholesky vector
// the pair costs O(m^2 n + m^2 d + nodes d^3).  The second-order term's sum_gamma X'_g J X'_g^T is
// K Lambda_p K^T with Lambda_p = sum_gamma ell_gamma G_p ell_gamma^T formed once per
// snapshot (energy_lambda_kernel).
#include "qcs_group.cuh"
#include "qcs_internal.h"

namespace {

struct EnergyArgs {
    int n, ne, m, d, nev, NB, nop, nchol, has_h, all, chunk, nchunks;
    int64_t W, P;
    int group_bytes, tab_bytes;
    int off_Q, off_T, off_B, off_NZ, off_g1, off_g2, off_y1, off_y2, off_pf, off_cf, off_invh, off_int, off_tile,
        off_acth, off_kh, off_ph, off_X1, off_Ap, off_Sacc, off_red, off_acc, off_scr;
    const cd *Ut;
    const cd *Qt;
    const int *idx;
    const int *d_count;
    const cd *Kop;  // W x nop x m x 2n: K ell_o (o < nchol: Cholesky vectors; o = nchol: h)
    const cd *K2;   // W x m x 2n: sum_gamma K ell_gamma^2
    const cd *Kg;   // W x m x 2n: K, the walker's selected rows
    const cd *Lam;  // per parity +1 snapshot (list order): Lambda_p, packed upper 2n x 2n
    cd *partial;    // W x nchunks x 3: (sum o_p, sum first-derivative term, sum second-derivative term)
    unsigned long long *counter;
    unsigned *status;
    cd wnode[QCS_MAX_NODES];
    cd gamma[QCS_MAX_NODES];
};

// Sum of one complex value per thread over the 64 threads of a group, in a fixed
// order (warp shuffles, then the two warp sums in order).  Every thread gets the sum.
__device__ __forceinline__ cd group_sum(cd v, cd *red, int t, int bar) {
    v = warp_csum(v);
    if ((t & 31) == 0) red[t >> 5] = v;
    group_sync(bar);
    const cd s = cadd(red[0], red[1]);
    group_sync(bar);
    return s;
}

// Sacc = sum_gamma X'_g J X'_g^T = K Lambda_p K^T (packed upper, m x m), with Lambda_p
// the snapshot's sum over the Cholesky vectors (energy_lambda_kernel): P = K Lambda
// into the X' region, then Sacc_ab = sum_nu P_a,nu K_b,nu.  K and Lambda_p are read
// from global memory (both stay in L2: one walker's K serves all its tiles).
__device__ inline void build_Sacc(int n, int m, const cd *__restrict__ Kw, const cd *__restrict__ Lp,
                                  cd *__restrict__ Pm, int lx, cd *__restrict__ Sacc, const uint16_t *__restrict__ tab,
                                  int t, int bar) {
    const int n2 = 2 * n, T = tri_count(m);
    for (int e = t; e < m * n2; e += kGroup) {
        const int a = e / n2, nu = e - a * n2;
        const cd *kr = Kw + a * n2;
        cd s = cmk(0.0, 0.0);
        for (int mu = 0; mu < n2; ++mu)
            cfma(s, kr[mu], skew_get0(Lp, mu, nu));  // the diagonal is zero
        Pm[a * lx + nu] = s;
    }
    group_sync(bar);
    for (int u = t; u < T; u += kGroup) {
        int a, b;
        pair_of(tab, u, a, b);
        const cd *pa = Pm + a * lx, *kb = Kw + b * n2;
        cd s = cmk(0.0, 0.0);
        for (int nu = 0; nu < n2; ++nu) cfma(s, pa[nu], kb[nu]);
        Sacc[u] = s;
    }
    group_sync(bar);
}

// Mt[b][mu] = (Q'^T J X^T)[mu][b] = sum_k Q'[2k][mu] X[b][2k+1] - Q'[2k+1][mu] X[b][2k], so that
// X' J X^T = (K ell) Q'^T J X^T = (K ell) Mt^T for every operator: the snapshot enters once
// per pair instead of once per operator.  Q'[c][2k] = Re Qt[c][k], Q'[c][2k+1] = -Im Qt[c][k];
// the rows of X for empty modes are real (Re T_j, -Im T_j), and so are those rows of Mt
// (stored with a zero imaginary part).
__device__ inline void build_Mt(int n, int ne, int m, const cd *__restrict__ Qs, int lq, const cd *__restrict__ Ts,
                                int lt, cd *__restrict__ Mt, int lx, int t) {
    const int n2 = 2 * n;
    for (int e = t; e < m * n2; e += kGroup) {
        const int b = e / n2, mu = e - b * n2, kq = mu >> 1;
        const bool odd = (mu & 1) != 0;
        if (b < ne) {
            const cd *xb = Ts + b * lt;
            cd v = cmk(0.0, 0.0);
            for (int k = 0; k < n; ++k) {
                const cd q0 = Qs[(2 * k) * lq + kq], q1 = Qs[(2 * k + 1) * lq + kq];
                crfma(v, xb[2 * k + 1], odd ? -q0.y : q0.x);
                crfma(v, xb[2 * k], odd ? q1.y : -q1.x);
            }
            Mt[b * lx + mu] = v;
        } else {
            const int r = b - ne;
            const cd *tr = Ts + (ne + (r >> 1)) * lt;
            double v = 0.0;
            for (int k = 0; k < n; ++k) {
                const cd q0 = Qs[(2 * k) * lq + kq], q1 = Qs[(2 * k + 1) * lq + kq];
                const double x1 = (r & 1) ? -tr[2 * k + 1].y : tr[2 * k + 1].x;
                const double x0 = (r & 1) ? -tr[2 * k].y : tr[2 * k].x;
                v = fma(x1, odd ? -q0.y : q0.x, v);
                v = fma(x0, odd ? q1.y : -q1.x, v);
            }
            Mt[b * lx + mu] = cmk(v, 0.0);
        }
    }
}

// A' = N - N^T with N = X' J X^T = Ks Mt^T (Ks: the operator's rows K ell staged in shared
// memory, Mt from build_Mt), plus 2 Sacc on the A'' pass:
//     A'_ab = sum_mu Ks[a][mu] Mt[b][mu] - Ks[b][mu] Mt[a][mu],
// in three uniform loops over the pairs a < b: both occupied, occupied x empty, both
// empty.  The rows of Mt for empty modes are real, so products with them take two real
// multiply-adds instead of four.
__device__ inline void build_Ap(int n, int ne, int m, const cd *__restrict__ Ks, int lx, const cd *__restrict__ Mt,
                                cd *__restrict__ Ap, const cd *__restrict__ Sacc, bool last,
                                const uint16_t *__restrict__ tab, int t) {
    const int n2 = 2 * n, d2 = m - ne, c1 = tri_count(ne), c2 = ne * d2, c3 = tri_count(d2);
    auto finish = [&](int a, int b, cd v) {
        const int e = tri_index(a, b);
        if (last) v = cadd(v, cscale(Sacc[e], 2.0));
        Ap[e] = v;
    };
    for (int u = t; u < c1; u += kGroup) {  // occupied x occupied: complex rows of Mt
        int a, b;
        pair_of(tab, u, a, b);
        const cd *ka = Ks + a * lx, *kb = Ks + b * lx, *ma = Mt + a * lx, *mb = Mt + b * lx;
        cd v = cmk(0.0, 0.0);
        for (int mu = 0; mu < n2; ++mu) {
            cfma(v, ka[mu], mb[mu]);
            cfms(v, kb[mu], ma[mu]);
        }
        finish(a, b, v);
    }
    for (int u = t; u < c2; u += kGroup) {  // occupied a x empty b = ne + r
        const int a = u / d2, r = u - a * d2, b = ne + r;
        const cd *ka = Ks + a * lx, *kb = Ks + b * lx, *ma = Mt + a * lx, *mb = Mt + b * lx;
        cd v = cmk(0.0, 0.0);
        for (int mu = 0; mu < n2; ++mu) {
            crfma(v, ka[mu], mb[mu].x);
            cfms(v, kb[mu], ma[mu]);
        }
        finish(a, b, v);
    }
    for (int u = t; u < c3; u += kGroup) {  // empty x empty: real rows of Mt
        int ra, rb;
        pair_of(tab, u, ra, rb);
        const int a = ne + ra, b = ne + rb;
        const cd *ka = Ks + a * lx, *kb = Ks + b * lx, *ma = Mt + a * lx, *mb = Mt + b * lx;
        cd v = cmk(0.0, 0.0);
        for (int mu = 0; mu < n2; ++mu) {
            crfma(v, ka[mu], mb[mu].x);
            crfma(v, kb[mu], -ma[mu].x);
        }
        finish(a, b, v);
    }
}

// Per pair, before the first operator: Mt into the X' region (free between the node
// rounds and the operator loop), then into the snapshot-row and T regions, which are
// contiguous and no longer needed for this pair.
__device__ inline void stage_Mt(int n, int ne, int m, const cd *__restrict__ Qs, int lq, const cd *__restrict__ Ts,
                                int lt, cd *__restrict__ X1, int lx, cd *__restrict__ Mt, int t, int bar) {
    build_Mt(n, ne, m, Qs, lq, Ts, lt, X1, lx, t);
    group_sync(bar);
    for (int e = t; e < m * lx; e += kGroup) Mt[e] = X1[e];
    group_sync(bar);
}

// The operator's rows K ell (global memory, m x 2n) into the X' region, row stride lx.
__device__ inline void stage_Ko(int n, int m, const cd *__restrict__ Ko, cd *__restrict__ Ks, int lx, int t,
                                int bar) {
    const int n2 = 2 * n;
    for (int e = t; e < m * n2; e += kGroup) {
        const int a = e / n2, c = e - a * n2;
        Ks[a * lx + c] = Ko[e];
    }
    group_sync(bar);
}

__global__ void __launch_bounds__(128, 2) energy_pair_kernel(const __grid_constant__ EnergyArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / kGroup;
    const int t = threadIdx.x - gid * kGroup;
    const int bar = 1 + gid;
    const int n = A.n, n2 = 2 * n, ne = A.ne, m = A.m, T = tri_count(m);
    const int lu = ld_ut(n), lq = ld_qt(n), lt = ld_t(n), lx = n2 + 1;
    // the pair table and the groups' workspaces fit the launch's shared memory
    if (!QCS_IN_BOUNDS(T * (int)sizeof(uint16_t) <= A.tab_bytes &&
                           (size_t)A.tab_bytes + (size_t)(blockDim.x / kGroup) * A.group_bytes <= dyn_smem_bytes(),
                       A.status))
        return;
    uint16_t *tab = reinterpret_cast<uint16_t *>(smem_raw);
    build_pair_table(tab, T);
    __syncthreads();
    unsigned char *wb = smem_raw + A.tab_bytes + (size_t)gid * A.group_bytes;
    // region X1R holds, in turn, the walker rows Ut (until T is built), the backward
    // recursion's vectors (node rounds) and X' (operator loop)
    cd *Uts = reinterpret_cast<cd *>(wb + A.off_X1);
    cd *Qs = reinterpret_cast<cd *>(wb + A.off_Q);
    cd *Ts = reinterpret_cast<cd *>(wb + A.off_T);
    cd *Bs = reinterpret_cast<cd *>(wb + A.off_B);
    cd *Ns = reinterpret_cast<cd *>(wb + A.off_NZ);  // node factors, then their inverses (packed)
    cd *g1v = reinterpret_cast<cd *>(wb + A.off_g1);
    cd *g2v = reinterpret_cast<cd *>(wb + A.off_g2);
    cd *y1v = reinterpret_cast<cd *>(wb + A.off_y1);
    cd *y2v = reinterpret_cast<cd *>(wb + A.off_y2);
    cd *pf = reinterpret_cast<cd *>(wb + A.off_pf);
    cd *cf = reinterpret_cast<cd *>(wb + A.off_cf);
    cd *invh = reinterpret_cast<cd *>(wb + A.off_invh);
    int *pos = reinterpret_cast<int *>(wb + A.off_int);
    long long *slot = reinterpret_cast<long long *>(wb + A.off_tile);
    uint8_t *acth = wb + A.off_acth;
    uint8_t *kh = wb + A.off_kh;
    uint8_t *ph = wb + A.off_ph;
    cd *X1 = reinterpret_cast<cd *>(wb + A.off_X1);     // K ell (or K ell^2) rows, m x (2n+1)
    cd *Mt = Qs;  // from the operator loop on: Mt (m x (2n+1)) over the snapshot-row and T regions
    cd *Ap = reinterpret_cast<cd *>(wb + A.off_Ap);     // A' (packed upper skew)
    cd *Sacc = reinterpret_cast<cd *>(wb + A.off_Sacc); // sum_gamma X'_g J X'_g^T (packed)
    cd *red = reinterpret_cast<cd *>(wb + A.off_red);   // 2 entries
    cd *acc = reinterpret_cast<cd *>(wb + A.off_acc);   // 2 x NB: first / second derivative terms per node
    SharedScratch *scr = reinterpret_cast<SharedScratch *>(wb + A.off_scr);

    const int64_t L = A.all ? A.P : (int64_t)(*A.d_count);
    const int64_t ntiles = A.W * A.nchunks;
    for (;;) {
        if (t == 0) *slot = (long long)atomicAdd(A.counter, 1ull);
        group_sync(bar);
        const int64_t tile = (int64_t)*slot;
        if (tile >= ntiles) break;
        const int ch = (int)(tile / A.W);  // chunk-major order
        const int64_t w = tile - (int64_t)ch * A.W;
        const int64_t p0 = (int64_t)ch * A.chunk;
        const int64_t p1 = p0 + A.chunk < L ? p0 + A.chunk : L;
        if (!QCS_IN_BOUNDS(ch < A.nchunks && L >= 0 && L <= A.P, A.status)) {  // group-uniform
            group_sync(bar);  // every thread has read the slot before it is rewritten
            continue;
        }
        cd So = cmk(0.0, 0.0), S1 = cmk(0.0, 0.0), S2 = cmk(0.0, 0.0);
        if (p0 < L) {
            const cd *Utw = A.Ut + w * n * n;
            const cd *Kw = A.Kop + (size_t)w * A.nop * m * n2;
            const cd *K2w = A.K2 + (size_t)w * m * n2;
            const cd *Kgw = A.Kg + (size_t)w * m * n2;
            for (int64_t pq = p0; pq < p1; ++pq) {
                const int64_t q = A.all ? pq : (int64_t)A.idx[pq];
                if (!QCS_IN_BOUNDS(q >= 0 && q < A.P, A.status)) continue;  // group-uniform
                group_sync(bar);
                load_Qt(n, A.Qt + q * n2 * n, Qs, t, kGroup);
                for (int e = t; e < n * n; e += kGroup) Uts[(e / n) * lu + (e % n)] = Utw[e];
                group_sync(bar);
                build_T(n, Uts, Qs, Ts, t, kGroup);
                group_sync(bar);
                build_B(n, ne, Ts, Bs, tab, t, kGroup);
                group_sync(bar);
                cd Sop = cmk(0.0, 0.0), S1p = cmk(0.0, 0.0), S2p = cmk(0.0, 0.0);
                if (shared_factor(m, ne, Bs, Ns, g1v, g2v, invh, acth, kh, ph, scr, tab, t, bar)) {
                    // Block form: A_k^{-1} = F0 + F Z_k F^T with F0 = [[P^-1, 0], [0, 0]],
                    // F = [-E; I], E = P^-1 B_oe, Z_k = (S0 + w_k D)^{-1} (2d x 2d).  Per
                    // operator, with W = A' F and G = F^T A' F, H = F^T A' F0 A' F = -W_o^T P^-1 W_o:
                    //   tr(A_k^-1 A')       = tr(P^-1 A'_oo) + tr(Z_k G)
                    //   tr((A_k^-1 A')^2)   = tr((P^-1 A'_oo)^2) + 2 tr(Z_k H) + tr((Z_k G)^2)
                    const int d2 = m - ne, Tn = tri_count(d2), To = tri_count(ne);
                    const int zoff = T > A.NB * Tn ? T : A.NB * Tn;
                    cd *Pinv = Ns + zoff;       // P^-1, packed upper (ne x ne)
                    cd *Es = Pinv + To;         // E, ne x 2d
                    cd *Sc = Es + ne * d2;      // S0, packed upper (2d x 2d)
                    const cd pf0 = scr->pf0;
                    for (int e = t; e < Tn; e += kGroup) {
                        int a, b;
                        pair_of(tab, e, a, b);
                        cd *y = Ns + tri_index(ne + a, ne + b);
                        Sc[e] = *y;
                        *y = cmk(0.0, 0.0);
                    }
                    group_sync(bar);
                    // with Z = 0 and unit constant the backward pass gives F0
                    shared_inverse(m, ne, Ns, g1v, g2v, y1v, y2v, invh, acth, kh, ph, cmk(1.0, 0.0), scr, t, bar);
                    for (int e = t; e < To; e += kGroup) Pinv[e] = Ns[e];
                    group_sync(bar);
                    for (int e = t; e < ne * d2; e += kGroup) {
                        const int i = e / d2, j = e - i * d2;
                        cd s = cmk(0.0, 0.0);
                        for (int l = 0; l < ne; ++l)
                            if (l != i) cfma(s, skew_get(Pinv, i, l), Bs[tri_index(l, ne + j)]);
                        Es[e] = s;
                    }
                    group_sync(bar);
                    for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                        const int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                        node_factor(d2, 0, A.wnode + k0, nb, Sc, Ns, g1v, g2v, pf, invh, pos, acth, kh, ph, tab, t,
                                    bar, A.status);
                        node_inverse(d2, nb, Ns, g1v, g2v, y1v, y2v, invh, acth, kh, ph, t, bar);
                        if (t < nb) {
                            cf[t] = cscale(cmul(A.gamma[k0 + t], cmul(pf0, pf[t])), 0.5);
                            acc[t] = cmk(0.0, 0.0);
                            acc[A.NB + t] = cmk(0.0, 0.0);
                        }
                        if (t == 0)
                            for (int v = 0; v < nb; ++v) cfma(Sop, A.gamma[k0 + v], cmul(pf0, pf[v]));
                        group_sync(bar);
                        if (k0 == 0) stage_Mt(n, ne, m, Qs, lq, Ts, lt, X1, lx, Mt, t, bar);
                        for (int o = 0; o <= A.nop; ++o) {
                            const bool is_h = A.has_h && o == A.nchol;
                            const bool last = o == A.nop;
                            const bool second = !is_h && !last;  // a Cholesky vector: second derivative
                            const cd *Ko = last ? K2w : Kw + (size_t)o * m * n2;
                            if (last) build_Sacc(n, m, Kgw, A.Lam + pq * tri_count(n2), X1, lx, Sacc, tab, t, bar);
                            stage_Ko(n, m, Ko, X1, lx, t, bar);
                            build_Ap(n, ne, m, X1, lx, Mt, Ap, Sacc, last, tab, t);
                            group_sync(bar);
                            // X' is consumed: its region holds W, G, V, H
                            cd *Wm = X1, *Gp = X1 + m * d2, *Vm = Gp + Tn, *Hp = Vm + ne * d2;
                            for (int e = t; e < m * d2; e += kGroup) {
                                const int a = e / d2, j = e - a * d2;
                                cd s = (a == ne + j) ? cmk(0.0, 0.0) : skew_get(Ap, a, ne + j);
                                for (int l = 0; l < ne; ++l)
                                    if (l != a) cfms(s, skew_get(Ap, a, l), Es[l * d2 + j]);
                                Wm[e] = s;
                            }
                            group_sync(bar);
                            for (int e = t; e < Tn; e += kGroup) {
                                int i, j;
                                pair_of(tab, e, i, j);
                                cd s = Wm[(ne + i) * d2 + j];
                                for (int l = 0; l < ne; ++l) cfms(s, Es[l * d2 + i], Wm[l * d2 + j]);
                                Gp[e] = s;
                            }
                            if (second)
                                for (int e = t; e < ne * d2; e += kGroup) {
                                    const int i = e / d2, j = e - i * d2;
                                    cd s = cmk(0.0, 0.0);
                                    for (int l = 0; l < ne; ++l)
                                        if (l != i) cfma(s, skew_get(Pinv, i, l), Wm[l * d2 + j]);
                                    Vm[e] = s;
                                }
                            // tr(P^-1 A'_oo) = -2 sum_{a<b} P^-1_ab A'_ab
                            cd tP = cmk(0.0, 0.0);
                            for (int e = t; e < To; e += kGroup) cfma(tP, Pinv[e], Ap[e]);
                            group_sync(bar);
                            tP = cscale(group_sum(tP, red, t, bar), -2.0);
                            cd c0 = cmk(0.0, 0.0);
                            if (second) {
                                for (int e = t; e < Tn; e += kGroup) {
                                    int i, j;
                                    pair_of(tab, e, i, j);
                                    cd s = cmk(0.0, 0.0);
                                    for (int l = 0; l < ne; ++l) cfms(s, Wm[l * d2 + i], Vm[l * d2 + j]);
                                    Hp[e] = s;
                                }
                                // tr((P^-1 A'_oo)^2): one unordered pair {a, b} of occupied indices per item
                                for (int e = t; e < ne * (ne + 1) / 2; e += kGroup) {
                                    int a = 0, r = e;
                                    while (r >= ne - a) {
                                        r -= ne - a;
                                        ++a;
                                    }
                                    const int b = a + r;
                                    cd pab = cmk(0.0, 0.0), pba = cmk(0.0, 0.0);
                                    for (int c = 0; c < ne; ++c) {
                                        if (c != a && c != b) cfma(pab, skew_get(Pinv, a, c), skew_get(Ap, c, b));
                                        if (c != b && c != a) cfma(pba, skew_get(Pinv, b, c), skew_get(Ap, c, a));
                                    }
                                    const cd pr = cmul(pab, pba);
                                    c0 = (a == b) ? cadd(c0, pr) : cadd(c0, cscale(pr, 2.0));
                                }
                                c0 = group_sum(c0, red, t, bar);
                            }
                            // tr((Z G)^2) by three real products per complex multiply-add: re + im
                            // of G and of each node's Z staged in A''s region (A' is consumed)
                            const bool sums = second && (A.NB + 1) * Tn <= 2 * T;
                            double *gsm = reinterpret_cast<double *>(Ap), *zsm = gsm + Tn;
                            if (sums) {
                                for (int e = t; e < Tn; e += kGroup) gsm[e] = Gp[e].x + Gp[e].y;
                                for (int e = t; e < nb * Tn; e += kGroup) zsm[e] = Ns[e].x + Ns[e].y;
                                group_sync(bar);
                            }
                            for (int v = 0; v < nb; ++v) {
                                const cd *Zv = Ns + v * Tn;  // Z_v, packed upper
                                cd zg = cmk(0.0, 0.0), zh = cmk(0.0, 0.0);
                                for (int e = t; e < Tn; e += kGroup) {
                                    cfma(zg, Zv[e], Gp[e]);
                                    if (second) cfma(zh, Zv[e], Hp[e]);
                                }
                                const cd t1 = cadd(tP, cscale(group_sum(zg, red, t, bar), -2.0));
                                if (last) {
                                    if (t == 0) acc[A.NB + v] = cadd(acc[A.NB + v], t1);
                                    continue;
                                }
                                if (is_h) {
                                    if (t == 0) acc[v] = cadd(acc[v], t1);
                                    continue;
                                }
                                // tr((Z G)^2): one unordered pair {a, b} of empty indices per item
                                cd t2 = cscale(zh, -4.0);  // 2 tr(Z H) = -4 sum_{a<b} Z_ab H_ab
                                for (int e = t; e < d2 * (d2 + 1) / 2; e += kGroup) {
                                    int a = 0, r = e;
                                    while (r >= d2 - a) {
                                        r -= d2 - a;
                                        ++a;
                                    }
                                    const int b = a + r;
                                    cd pab = cmk(0.0, 0.0), pba = cmk(0.0, 0.0);
                                    if (sums) {
                                        const double *zs = zsm + v * Tn;
                                        double p1 = 0.0, p2 = 0.0, p3 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
                                        for (int c = 0; c < d2; ++c) {
                                            // Z(a,c) G(c,b) and Z(b,c) G(c,a) from the packed upper
                                            // triangles; c = a or c = b adds nothing (a zero diagonal),
                                            // taken by selects so that no lane branches
                                            const bool skip = c == a || c == b;
                                            const int iz = skip ? 0 : (a < c ? tri_index(a, c) : tri_index(c, a));
                                            const int ig = skip ? 0 : (c < b ? tri_index(c, b) : tri_index(b, c));
                                            const int jz = skip ? 0 : (b < c ? tri_index(b, c) : tri_index(c, b));
                                            const int jg = skip ? 0 : (c < a ? tri_index(c, a) : tri_index(a, c));
                                            const bool s1 = (a > c) != (c > b), s2 = (b > c) != (c > a);
                                            const cd zero = cmk(0.0, 0.0);
                                            const cd z1 = skip ? zero : flip_if(Zv[iz], s1);
                                            const cd z2 = skip ? zero : flip_if(Zv[jz], s2);
                                            const double w1 = skip ? 0.0 : __longlong_as_double(__double_as_longlong(zs[iz]) ^ (s1 ? (long long)0x8000000000000000ull : 0ll));
                                            const double w2 = skip ? 0.0 : __longlong_as_double(__double_as_longlong(zs[jz]) ^ (s2 ? (long long)0x8000000000000000ull : 0ll));
                                            const cd g1 = Gp[ig], g2 = Gp[jg];
                                            p1 = fma(z1.x, g1.x, p1);
                                            p2 = fma(z1.y, g1.y, p2);
                                            p3 = fma(w1, gsm[ig], p3);
                                            q1 = fma(z2.x, g2.x, q1);
                                            q2 = fma(z2.y, g2.y, q2);
                                            q3 = fma(w2, gsm[jg], q3);
                                        }
                                        pab = cmk(p1 - p2, p3 - p1 - p2);
                                        pba = cmk(q1 - q2, q3 - q1 - q2);
                                    } else {
                                        for (int c = 0; c < d2; ++c) {  // zero diagonals: c = a, b add nothing
                                            cfma(pab, skew_get0(Zv, a, c), skew_get0(Gp, c, b));
                                            cfma(pba, skew_get0(Zv, b, c), skew_get0(Gp, c, a));
                                        }
                                    }
                                    const cd pr = cmul(pab, pba);
                                    t2 = (a == b) ? cadd(t2, pr) : cadd(t2, cscale(pr, 2.0));
                                }
                                t2 = cadd(group_sum(t2, red, t, bar), c0);
                                if (t == 0) acc[A.NB + v] = cadd(acc[A.NB + v], csub(cscale(cmul(t1, t1), 0.5), t2));
                            }
                            group_sync(bar);
                        }
                        if (t == 0)
                            for (int v = 0; v < nb; ++v) {
                                cfma(S1p, cf[v], acc[v]);
                                cfma(S2p, cf[v], acc[A.NB + v]);
                            }
                        group_sync(bar);
                    }
                } else {
                    for (int k0 = 0; k0 < A.nev; k0 += A.NB) {
                        const int nb = A.nev - k0 < A.NB ? A.nev - k0 : A.NB;
                        node_factor(m, ne, A.wnode + k0, nb, Bs, Ns, g1v, g2v, pf, invh, pos, acth, kh, ph, tab, t, bar, A.status);
                        node_inverse(m, nb, Ns, g1v, g2v, y1v, y2v, invh, acth, kh, ph, t, bar);
                        if (t < nb) {
                            cf[t] = cscale(cmul(A.gamma[k0 + t], pf[t]), 0.5);
                            acc[t] = cmk(0.0, 0.0);
                            acc[A.NB + t] = cmk(0.0, 0.0);
                        }
                        if (t == 0)
                            for (int v = 0; v < nb; ++v) cfma(Sop, A.gamma[k0 + v], pf[v]);
                        group_sync(bar);
                        if (k0 == 0) stage_Mt(n, ne, m, Qs, lq, Ts, lt, X1, lx, Mt, t, bar);
                        // operators: Cholesky vectors (second derivative), then h (first derivative);
                        // the last pass (o = nop) forms A'' = X'' J X^T + X J X''^T + 2 Sacc
                        for (int o = 0; o <= A.nop; ++o) {
                            const bool is_h = A.has_h && o == A.nchol;
                            const bool last = o == A.nop;
                            const cd *Ko = last ? K2w : Kw + (size_t)o * m * n2;
                            if (last) build_Sacc(n, m, Kgw, A.Lam + pq * tri_count(n2), X1, lx, Sacc, tab, t, bar);
                            stage_Ko(n, m, Ko, X1, lx, t, bar);
                            build_Ap(n, ne, m, X1, lx, Mt, Ap, Sacc, last, tab, t);
                            group_sync(bar);
                            for (int v = 0; v < nb; ++v) {
                                const cd *Zv = Ns + v * T;  // A_v^-1
                                // t1 = tr(A^-1 Ap) = -2 sum_{a<b} Z_ab Ap_ab
                                cd t1 = cmk(0.0, 0.0);
                                for (int e = t; e < T; e += kGroup) cfma(t1, Zv[e], Ap[e]);
                                t1 = cscale(group_sum(t1, red, t, bar), -2.0);
                                if (last) {
                                    if (t == 0) acc[A.NB + v] = cadd(acc[A.NB + v], t1);
                                    continue;
                                }
                                if (is_h) {
                                    if (t == 0) acc[v] = cadd(acc[v], t1);
                                    continue;
                                }
                                // t2 = tr((A^-1 Ap)^2) = sum_{a,b} P_ab P_ba, P = A^-1 Ap: one unordered
                                // pair {a, b} (a <= b) per item, both products formed by the same thread
                                cd t2 = cmk(0.0, 0.0);
                                const int npairs = m * (m + 1) / 2;
                                for (int e = t; e < npairs; e += kGroup) {
                                    int a = 0, r = e;
                                    while (r >= m - a) {
                                        r -= m - a;
                                        ++a;
                                    }
                                    const int b = a + r;
                                    cd pab = cmk(0.0, 0.0), pba = cmk(0.0, 0.0);
                                    for (int c = 0; c < m; ++c) {
                                        cfma(pab, skew_at(Zv, a, c), skew_at(Ap, c, b));
                                        cfma(pba, skew_at(Zv, b, c), skew_at(Ap, c, a));
                                    }
                                    const cd pr = cmul(pab, pba);
                                    t2 = (a == b) ? cadd(t2, pr) : cadd(t2, cscale(pr, 2.0));
                                }
                                t2 = group_sum(t2, red, t, bar);
                                if (t == 0) acc[A.NB + v] = cadd(acc[A.NB + v], csub(cscale(cmul(t1, t1), 0.5), t2));
                            }
                            group_sync(bar);
                        }
                        if (t == 0)
                            for (int v = 0; v < nb; ++v) {
                                cfma(S1p, cf[v], acc[v]);
                                cfma(S2p, cf[v], acc[A.NB + v]);
                            }
                        group_sync(bar);
                    }
                }
                if (t == 0) {
                    if (!cfinite(Sop) || !cfinite(S1p) || !cfinite(S2p)) raise_status(A.status, QCS_ERR_NONFINITE);
                    So = cadd(So, Sop);
                    S1 = cadd(S1, S1p);
                    S2 = cadd(S2, S2p);
                }
            }
        }
        group_sync(bar);
        if (t == 0) {
            cd *out = A.partial + (w * A.nchunks + ch) * 3;
            out[0] = So;
            out[1] = S1;
            out[2] = S2;
        }
    }
}

// Per walker: K (m x 2n) from the rotated rows Ut, and for each operator o the
// Majorana form ell_o of its one-body matrix, [Lhat, g_mu] = sum_a ell_{mu a} g_a:
//   ell[2r][2q] = ell[2r+1][2q+1] = (L_qr - L_rq)/2,
//   ell[2r][2q+1] = -i (L_rq + L_qr)/2,  ell[2r+1][2q] = i (L_rq + L_qr)/2;
// Kop[w][o] = K ell_o and K2[w] = sum_gamma K ell_gamma^2.  One block per walker.
__global__ void energy_prep_kernel(int n, int ne, int64_t W, int nchol, int has_h, const cd *__restrict__ Ut,
                                   const cd *__restrict__ Lg, const cd *__restrict__ h, cd *__restrict__ Kop,
                                   cd *__restrict__ K2, cd *__restrict__ Kg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = 2 * n, m = 2 * n - ne, nop = nchol + has_h;
    cd *K = reinterpret_cast<cd *>(smem_raw);   // m x 2n
    cd *ell = K + m * n2;                       // 2n x 2n
    cd *K1 = ell + n2 * n2;                     // m x 2n (K ell)
    cd *Ka = K1 + m * n2;                       // m x 2n (sum K ell^2)
    for (int64_t w = blockIdx.x; w < W; w += gridDim.x) {
        const cd *U = Ut + w * n * n;
        // Ut~[j][2k] = Ut[j][k], Ut~[j][2k+1] = -i Ut[j][k]; K rows: occupied j -> Ut~_j,
        // empty j -> Re Ut~_j, -Im Ut~_j
        for (int e = threadIdx.x; e < m * n2; e += blockDim.x) {
            const int a = e / n2, c = e - a * n2, k = c >> 1;
            const int j = a < ne ? a : ne + ((a - ne) >> 1);
            const cd u = U[j * n + k];
            const cd ut = (c & 1) ? cmk(u.y, -u.x) : u;
            K[e] = a < ne ? ut : (((a - ne) & 1) ? cmk(-ut.y, 0.0) : cmk(ut.x, 0.0));
            Kg[(size_t)w * m * n2 + e] = K[e];
            Ka[e] = cmk(0.0, 0.0);
        }
        __syncthreads();
        for (int o = 0; o < nop; ++o) {
            const cd *Lo = o < nchol ? Lg + (size_t)o * n * n : h;
            for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
                const int mu = e / n2, a = e - mu * n2, r = mu >> 1, q = a >> 1;
                const cd lrq = Lo[r * n + q], lqr = Lo[q * n + r];
                const cd dif = cscale(csub(lqr, lrq), 0.5), sum = cscale(cadd(lrq, lqr), 0.5);
                cd v;
                if ((mu & 1) == (a & 1)) v = dif;
                else if ((mu & 1) == 0) v = cmk(sum.y, -sum.x);  // -i sum
                else v = cmk(-sum.y, sum.x);                     // i sum
                ell[e] = v;
            }
            __syncthreads();
            cd *Ko = Kop + ((size_t)w * nop + o) * m * n2;
            for (int e = threadIdx.x; e < m * n2; e += blockDim.x) {
                const int a = e / n2, c = e - a * n2;
                cd s = cmk(0.0, 0.0);
                for (int k = 0; k < n2; ++k) cfma(s, K[a * n2 + k], ell[k * n2 + c]);
                K1[e] = s;
                Ko[e] = s;
            }
            __syncthreads();
            if (o < nchol)
                for (int e = threadIdx.x; e < m * n2; e += blockDim.x) {
                    const int a = e / n2, c = e - a * n2;
                    cd s = Ka[e];
                    for (int k = 0; k < n2; ++k) cfma(s, K1[a * n2 + k], ell[k * n2 + c]);
                    Ka[e] = s;
                }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < m * n2; e += blockDim.x) K2[(size_t)w * m * n2 + e] = Ka[e];
        __syncthreads();
    }
}

// Per parity +1 snapshot p (list order): Lambda_p = sum_gamma ell_gamma G_p ell_gamma^T over
// the Cholesky vectors, packed upper (2n x 2n), with G_p = R J R^T and R the snapshot's
// real rows (R[2k][c] = Re Qt[c][k], R[2k+1][c] = -Im Qt[c][k]).  Since every walker's
// X'_gamma = K ell_gamma R, sum_gamma X'_g J X'_g^T = K Lambda_p K^T: the sum over the
// Cholesky vectors is taken once per snapshot instead of once per pair.  One block per
// snapshot; each thread owns up to kLamPer entries of Lambda.
constexpr int kLamThreads = 256, kLamPer = 5;  // 256 x 5 >= tri(2 QCS_MAX_N) = 1128
__global__ void __launch_bounds__(kLamThreads) energy_lambda_kernel(int n, int nchol, int64_t P, int all, const int *__restrict__ idx,
                                     const int *__restrict__ d_count, const cd *__restrict__ Qt,
                                     const cd *__restrict__ Lg, cd *__restrict__ Lam) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n2 = 2 * n, T2 = tri_count(n2);
    double *R = reinterpret_cast<double *>(smem_raw);  // 2n x 2n
    double *G = R + n2 * n2;                           // 2n x 2n
    cd *ell = reinterpret_cast<cd *>(G + n2 * n2);     // 2n x 2n
    cd *M = ell + n2 * n2;                             // ell G
    const int64_t L = all ? P : (int64_t)(*d_count);
    for (int64_t pq = blockIdx.x; pq < L; pq += gridDim.x) {
        const int64_t q = all ? pq : (int64_t)idx[pq];
        for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
            const int mu = e / n2, c = e - mu * n2;
            const cd v = Qt[(q * n2 + c) * n + (mu >> 1)];
            R[e] = (mu & 1) ? -v.y : v.x;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
            const int mu = e / n2, nu = e - mu * n2;
            double g = 0.0;
            for (int j = 0; j < n; ++j) {
                g = fma(R[mu * n2 + 2 * j], R[nu * n2 + 2 * j + 1], g);
                g = fma(-R[mu * n2 + 2 * j + 1], R[nu * n2 + 2 * j], g);
            }
            G[e] = g;
        }
        cd acc[kLamPer];
        int mus[kLamPer], nus[kLamPer];  // the (mu < nu) entries this thread owns
#pragma unroll
        for (int h = 0; h < kLamPer; ++h) {
            acc[h] = cmk(0.0, 0.0);
            const int u = threadIdx.x + h * blockDim.x;
            int nu = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)u)) * 0.5f);
            while (nu * (nu - 1) / 2 > u) --nu;
            while ((nu + 1) * nu / 2 <= u) ++nu;
            nus[h] = nu;
            mus[h] = u - nu * (nu - 1) / 2;
        }
        for (int g = 0; g < nchol; ++g) {
            const cd *Lo = Lg + (size_t)g * n * n;
            __syncthreads();  // G complete; the previous vector's M and ell consumed
            for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
                const int mu = e / n2, a = e - mu * n2, r = mu >> 1, qq = a >> 1;
                const cd lrq = Lo[r * n + qq], lqr = Lo[qq * n + r];
                const cd dif = cscale(csub(lqr, lrq), 0.5), sum = cscale(cadd(lrq, lqr), 0.5);
                cd v;
                if ((mu & 1) == (a & 1)) v = dif;
                else if ((mu & 1) == 0) v = cmk(sum.y, -sum.x);  // -i sum
                else v = cmk(-sum.y, sum.x);                     // i sum
                ell[e] = v;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
                const int mu = e / n2, nu = e - mu * n2;
                cd s = cmk(0.0, 0.0);
                for (int k = 0; k < n2; ++k) crfma(s, ell[mu * n2 + k], G[k * n2 + nu]);
                M[e] = s;
            }
            __syncthreads();
#pragma unroll
            for (int h = 0; h < kLamPer; ++h) {
                if (threadIdx.x + h * blockDim.x < T2) {
                    const cd *mr = M + mus[h] * n2, *lr = ell + nus[h] * n2;
                    cd s = acc[h];
                    for (int k = 0; k < n2; ++k) cfma(s, mr[k], lr[k]);
                    acc[h] = s;
                }
            }
        }
#pragma unroll
        for (int h = 0; h < kLamPer; ++h) {
            const int u = threadIdx.x + h * blockDim.x;
            if (u < T2) Lam[pq * T2 + u] = acc[h];
        }
        __syncthreads();
    }
}

// Per walker: sums of the tile records in order; O = pref sum So / P,
// e1 = sum S1 / sum So, e2 = sum S2 / sum So.
__global__ void energy_reduce_kernel(int64_t W, int64_t P, int nchunks, const cd *__restrict__ partial,
                                     const cd *__restrict__ pref, cd *__restrict__ ov, cd *__restrict__ e1,
                                     cd *__restrict__ e2) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    cd so = cmk(0.0, 0.0), s1 = cmk(0.0, 0.0), s2 = cmk(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) {
        const cd *r = partial + (w * nchunks + c) * 3;
        so = cadd(so, r[0]);
        s1 = cadd(s1, r[1]);
        s2 = cadd(s2, r[2]);
    }
    const double invP = P > 0 ? 1.0 / (double)P : 0.0;
    if (ov) ov[w] = cscale(cmul(pref[w], so), invP);
    const cd iso = cinv(so);
    if (e1) e1[w] = cmul(s1, iso);
    if (e2) e2[w] = cmul(s2, iso);
}

size_t energy_group_layout(EnergyArgs &A) {
    const int n = A.n, m = A.m, T = tri_count(m), NB = A.NB, S = m / 2;
    size_t o = 0;
    A.off_Q = (int)o;
    o = align16(o + (size_t)2 * n * ld_qt(n) * sizeof(cd));
    A.off_T = (int)o;
    o = align16(o + (size_t)n * ld_t(n) * sizeof(cd));
    A.off_B = (int)o;
    o = align16(o + (size_t)T * sizeof(cd));
    A.off_NZ = (int)o;
    // node matrices; in the block form the complements' inverses, then P^-1, E and S0
    const int d2 = m - A.ne, Tn = tri_count(d2), To = tri_count(A.ne);
    size_t nz = (size_t)NB * T;
    const size_t zoff = (size_t)(T > NB * Tn ? T : NB * Tn);
    if (zoff + To + (size_t)A.ne * d2 + Tn > nz) nz = zoff + To + (size_t)A.ne * d2 + Tn;
    o = align16(o + nz * sizeof(cd));
    // shared region: Ut rows, then the recursion vectors, then Mt on its way to the Q and T
    // regions (m (2n+1) <= 2n (n+1) + n (2n+1) entries, contiguous), then each operator's
    // rows K ell (then W, G, V, H)
    size_t r = (size_t)m * (2 * n + 1);
    if ((size_t)n * ld_ut(n) > r) r = (size_t)n * ld_ut(n);
    if ((size_t)4 * NB * m > r) r = (size_t)4 * NB * m;
    if ((size_t)d2 * (m + A.ne) + 2 * (size_t)Tn > r) r = (size_t)d2 * (m + A.ne) + 2 * (size_t)Tn;
    A.off_X1 = (int)o;
    A.off_g1 = (int)o;
    A.off_g2 = (int)(o + (size_t)NB * m * sizeof(cd));
    A.off_y1 = (int)(o + (size_t)2 * NB * m * sizeof(cd));
    A.off_y2 = (int)(o + (size_t)3 * NB * m * sizeof(cd));
    o = align16(o + r * sizeof(cd));
    A.off_pf = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    A.off_cf = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(cd));
    A.off_invh = (int)o;
    o = align16(o + (size_t)NB * S * sizeof(cd));
    A.off_int = (int)o;
    o = align16(o + (size_t)kMaxNBG * sizeof(int));
    A.off_tile = (int)o;
    o = align16(o + sizeof(long long));
    A.off_acth = (int)o;
    o = align16(o + (size_t)NB * (S + 1) * m);
    A.off_kh = (int)o;
    o = align16(o + (size_t)NB * S);
    A.off_ph = (int)o;
    o = align16(o + (size_t)NB * S);
    A.off_Ap = (int)o;
    o = align16(o + (size_t)T * sizeof(cd));
    if (NB >= A.nev) {
        A.off_Sacc = A.off_B;  // one node round: B is dead once copied into the node matrices
    } else {
        A.off_Sacc = (int)o;
        o = align16(o + (size_t)T * sizeof(cd));
    }
    A.off_red = (int)o;
    o = align16(o + (size_t)2 * sizeof(cd));
    A.off_acc = (int)o;
    o = align16(o + (size_t)2 * kMaxNBG * sizeof(cd));
    A.off_scr = (int)o;
    o = align16(o + sizeof(SharedScratch));
    return o;
}

}  // namespace

extern "C" qcs_status qcs_local_energy(qcs_ctx *ctx, const qcs_snapshots *s, int ne, int64_t W,
                                       const double *d_walkers, int nchol, const double *d_L, const double *d_h,
                                       double *d_overlap, double *d_e1, double *d_e2, const qcs_opts *opts,
                                       void *stream) {
    QcsRange range_("qcs_local_energy");
    if (!ctx) return QCS_ERR_ARG;
    if (!s) return qcs_fail(ctx, QCS_ERR_ARG, "null snapshot set");
    const int n = s->n;
    if (n < 2 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1))
        return qcs_fail(ctx, QCS_ERR_ARG, "ne must be even with 2 <= ne <= n");
    if (nchol < 0 || (nchol > 0 && !d_L)) return qcs_fail(ctx, QCS_ERR_ARG, "nchol < 0 or null Cholesky vectors");
    if (W < 0) return qcs_fail(ctx, QCS_ERR_ARG, "W < 0");
    if (W == 0) return QCS_OK;
    if (!d_walkers) return qcs_fail(ctx, QCS_ERR_ARG, "null walkers");
    if (s->device != ctx->device) return qcs_fail(ctx, QCS_ERR_ARG, "snapshot set lives on another device");
    qcs_opts o = {QCS_FP64, 0, 0u, 0};
    if (opts) o = *opts;
    if (o.precision != QCS_FP64) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "local energies are FP64 only");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    qcs_node_plan plan;
    if (qcs_make_node_plan(n, ne, o.nodes, o.flags, &plan) != QCS_OK)
        return qcs_fail(ctx, QCS_ERR_ARG, "nodes must be 0 or in [n-ne+1, QCS_MAX_NODES]");
    const int m = 2 * n - ne, n2 = 2 * n, has_h = d_h ? 1 : 0, nop = nchol + has_h;
    // tiles: about 8 per resident group, one snapshot chunk per tile
    int64_t target = (int64_t)ctx->num_sms * 2 * 8;
    int64_t nch = (target + W - 1) / W;
    if (nch > s->P) nch = s->P;
    if (nch < 1) nch = 1;
    int chunk = (int)((s->P + nch - 1) / nch);
    if (chunk < 1) chunk = 1;
    int nchunks = (int)((s->P + chunk - 1) / chunk);
    if (nchunks < 1) nchunks = 1;
    const size_t b_ut = align16(sizeof(cd) * (size_t)W * n * n);
    const size_t b_pref = align16(sizeof(cd) * (size_t)W);
    const size_t b_kop = align16(sizeof(cd) * (size_t)W * (nop > 0 ? nop : 1) * m * n2);
    const size_t b_k2 = align16(sizeof(cd) * (size_t)W * m * n2);
    const size_t b_kg = align16(sizeof(cd) * (size_t)W * m * n2);
    const size_t b_lam = align16(sizeof(cd) * (size_t)(s->P > 0 ? s->P : 1) * tri_count(n2));
    const size_t b_part = align16(sizeof(cd) * (size_t)W * nchunks * 3);
    void *base = nullptr;
    qcs_status ws = qcs_workspace(ctx, 16 + b_ut + b_pref + b_kop + b_k2 + b_part + b_kg + b_lam, &base, st);
    if (ws != QCS_OK) return ws;
    char *pb = (char *)base;
    unsigned long long *counter = (unsigned long long *)pb;
    cd *Ut = (cd *)(pb + 16);
    cd *pref = (cd *)(pb + 16 + b_ut);
    cd *Kop = (cd *)(pb + 16 + b_ut + b_pref);
    cd *K2 = (cd *)(pb + 16 + b_ut + b_pref + b_kop);
    cd *part = (cd *)(pb + 16 + b_ut + b_pref + b_kop + b_k2);
    cd *Kg = (cd *)(pb + 16 + b_ut + b_pref + b_kop + b_k2 + b_part);
    cd *Lam = (cd *)(pb + 16 + b_ut + b_pref + b_kop + b_k2 + b_part + b_kg);
    qcs_status r = qcs_launch_walker_prep(ctx, n, ne, W, (const cd *)d_walkers, Ut, pref, st);
    if (r != QCS_OK) return r;
    {
        const size_t sm = sizeof(cd) * ((size_t)3 * m * n2 + (size_t)n2 * n2);
        if (qcs_set_smem(ctx, (const void *)energy_prep_kernel, sm) != QCS_OK) return QCS_ERR_CUDA;
        int64_t blocks = W < (int64_t)ctx->num_sms * 4 ? W : (int64_t)ctx->num_sms * 4;
        energy_prep_kernel<<<(unsigned)blocks, 256, sm, st>>>(n, ne, W, nchol, has_h, Ut, (const cd *)d_L,
                                                               (const cd *)d_h, Kop, K2, Kg);
        r = qcs_check_launch(ctx, "energy_prep_kernel");
        if (r != QCS_OK) return r;
    }
    if (s->P > 0) {  // Lambda_p per parity +1 snapshot (zero without Cholesky vectors)
        const size_t sm = (size_t)2 * n2 * n2 * sizeof(double) + (size_t)2 * n2 * n2 * sizeof(cd);
        if (qcs_set_smem(ctx, (const void *)energy_lambda_kernel, sm) != QCS_OK) return QCS_ERR_CUDA;
        int64_t blocks = s->P < (int64_t)ctx->num_sms * 4 ? s->P : (int64_t)ctx->num_sms * 4;
        energy_lambda_kernel<<<(unsigned)blocks, kLamThreads, sm, st>>>(n, nchol, s->P, plan.all, s->idx, s->d_count,
                                                                        s->Qt, (const cd *)d_L, Lam);
        r = qcs_check_launch(ctx, "energy_lambda_kernel");
        if (r != QCS_OK) return r;
    }
    EnergyArgs A;
    memset(&A, 0, sizeof(A));
    A.n = n;
    A.ne = ne;
    A.m = m;
    A.d = n - ne;
    A.nev = plan.nev;
    A.nop = nop;
    A.nchol = nchol;
    A.has_h = has_h;
    A.all = plan.all;
    A.chunk = chunk;
    A.nchunks = nchunks;
    A.W = W;
    A.P = s->P;
    A.tab_bytes = (int)align16((size_t)tri_count(m) * sizeof(uint16_t));
    A.Ut = Ut;
    A.Qt = s->Qt;
    A.idx = s->idx;
    A.d_count = s->d_count;
    A.Kop = Kop;
    A.K2 = K2;
    A.Kg = Kg;
    A.Lam = Lam;
    A.partial = part;
    A.counter = counter;
    A.status = ctx->d_status;
    for (int k = 0; k < plan.nev; ++k) {
        A.wnode[k] = plan.wnode[k];
        A.gamma[k] = plan.gamma[k];
    }
    // node matrices per round: all when they fit, else fewer (rounds then repeat the
    // per-operator work); one or two groups per block
    int NB = plan.nev < kMaxNBG ? plan.nev : kMaxNBG, gpb = 2;
    for (;;) {
        A.NB = NB;
        A.group_bytes = (int)energy_group_layout(A);
        if ((size_t)A.tab_bytes + (size_t)gpb * A.group_bytes <= ctx->smem_optin) break;
        if (gpb == 2) gpb = 1;
        else if (NB > 1) {
            --NB;
            gpb = 2;
        } else {
            return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "local-energy kernel: shared memory too large");
        }
    }
    const size_t smem = (size_t)A.tab_bytes + (size_t)gpb * A.group_bytes;
    if (qcs_set_smem(ctx, (const void *)energy_pair_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, energy_pair_kernel, gpb * kGroup, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t ntiles = W * nchunks;
    int64_t blocks = (int64_t)ctx->num_sms * per_sm;
    const int64_t need = (ntiles + gpb - 1) / gpb;
    if (blocks > need) blocks = need;
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return qcs_fail(ctx, QCS_ERR_CUDA, "energy tile counter reset");
    qcs_prof_begin(ctx, st);
    energy_pair_kernel<<<(unsigned)blocks, gpb * kGroup, smem, st>>>(A);
    qcs_prof_end(ctx, st);
    r = qcs_check_launch(ctx, "energy_pair_kernel");
    if (r != QCS_OK) return r;
    energy_reduce_kernel<<<(unsigned)((W + 127) / 128), 128, 0, st>>>(W, s->P, nchunks, part, pref,
                                                                      (cd *)d_overlap, (cd *)d_e1, (cd *)d_e2);
    return qcs_check_launch(ctx, "energy_reduce_kernel");
}

extern "C" double qcs_local_energy_flops_per_pair(int n, int ne, int nchol, int has_h, int nodes, unsigned flags) {
    qcs_node_plan plan;
    if (n < 2 || n > QCS_MAX_N || ne < 2 || ne > n || (ne & 1) || nchol < 0) return 0.0;
    if (qcs_make_node_plan(n, ne, nodes, flags, &plan) != QCS_OK) return 0.0;
    // the block form (occupied block shared by the nodes), as the kernel runs it
    const int mi = 2 * n - ne, d2i = mi - ne;
    const double m = mi, n2 = 2.0 * n, T = m * (m - 1) / 2, d2 = d2i, Tn = d2 * (d2 - 1) / 2,
                 To = ne * (ne - 1) / 2.0, nev = plan.nev;
    auto bstep = [](int rv) { return 16.0 * rv * rv + 20.0 * rv; };  // one backward step
    double f = qcs_overlap_flops_nev(n, ne, plan.nev, false);        // dense T, B, full eliminations
    f -= (nev - 1.0) * qcs_pf_elim_flops(mi, d2i);                    // ... the occupied steps once
    for (int rv = d2i; rv <= mi - 2; rv += 2) f += bstep(rv);        // F0 = [[P^-1, 0], [0, 0]]
    f += 8.0 * ne * d2 * (ne - 1);                                    // E = P^-1 B_oe
    double inv = 0.0;                                                 // each complement's inverse
    for (int rv = d2i - 2; rv > 0; rv -= 2) inv += bstep(rv);
    f += inv * nev;
    // once per pair: Mt = (Q'^T J X^T)^T, real Q' against complex (occupied) or real
    // (empty) rows of X, n steps of two products per entry
    const double mt = n2 * n * (8.0 * ne + 4.0 * d2);
    // A' = (K ell) Mt^T - its transpose (upper triangle): complex x complex products where
    // the row of Mt is occupied, complex x real where it belongs to an empty mode
    const double c1 = ne * (ne - 1) / 2.0, c2 = ne * d2, c3 = d2 * (d2 - 1) / 2;
    const double aprime = 8.0 * n2 * (2.0 * c1 + c2) + 4.0 * n2 * (c2 + 2.0 * c3);
    const double wg = 8.0 * m * d2 * ne + 8.0 * Tn * ne + 8.0 * To;  // W = A'F, G = F^T W, tr(P^-1 A'_oo)
    const double vh = 8.0 * ne * d2 * (ne - 1) + 8.0 * Tn * ne       // V = P^-1 W_o, H = -W_o^T V
                      + 8.0 * (ne * (ne + 1) / 2.0) * 2.0 * (ne - 1);  // tr((P^-1 A'_oo)^2)
    const double t1 = 8.0 * Tn;                                       // tr(Z_k G) per node
    // tr(Z_k H), tr((Z_k G)^2): three real products per complex multiply-add where the
    // sums of G and of the round's Z_k fit in A''s region (NB as the launcher takes it when
    // the workspace fits), else four
    const int nbr = plan.nev < kMaxNBG ? plan.nev : kMaxNBG;
    const bool sums = (nbr + 1) * Tn <= 2 * T;
    const double items = d2 * (d2 + 1) / 2;
    const double t2 = 8.0 * Tn + (sums ? items * 2.0 * (6.0 * (d2 - 1) + 3.0) : items * 2.0 * 8.0 * (d2 - 1));
    const double npass = nchol + has_h + 1.0;                         // operators and the A'' pass
    f += mt + npass * (aprime + wg + nev * t1);
    f += nchol * (vh + nev * t2);
    // sum_gamma X'_g J X'_g^T = K Lambda_p K^T once per pair (Lambda_p per snapshot, shared by
    // every walker, is the separate energy_lambda_kernel)
    f += (nchol > 0 ? 1.0 : 0.0) * (8.0 * m * n2 * (n2 - 1) + 8.0 * T * n2);
    return f;
}
