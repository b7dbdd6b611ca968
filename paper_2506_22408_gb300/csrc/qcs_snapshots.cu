// qcs_snapshots.cu -- device representation of the shadow snapshots (Q_p, b_p).
//
// Eq. (b_mat) needs G_p = Q_p^T C_b Q_p with C_b the covariance matrix of SI
// "Matrix Definitions" item 2.  Writing C_b = P_b J P_b with
// P_b = diag(1, s_1, 1, s_2, ...), s_j = (-1)^{b_j}, and J = (+)_j [[0,1],[-1,0]],
// gives G_p = Q'^T J Q' with Q' = P_b Q (rows 2j+1 of Q scaled by s_j, 0-based).
// The overlap kernels use the complexified rows
//     Qt[c][k] = Q'[c][2k] - i Q'[c][2k+1],   c < 2n, k < n,
// so that the walker congruence becomes one complex n x n by n x 2n product.
//
// Each snapshot also gets its parity pi_p = det(Q_p) (-1)^{|b_p|} = det(Q'_p): the
// measured state is a pure Gaussian state of that parity, and pairs with
// pi_p = -1 contribute exactly zero to every overlap (the estimator's
// coefficient sequence is palindromic up to pi_p while its weights are
// symmetric).  det(Q_p) = +-1 is obtained from an LU factorisation with
// partial pivoting (only its sign is used).
//
// Snapshots that are signed permutations (every row of Q_p has one nonzero
// entry, exactly +-1: the ensemble of the paper's experiment) also get gather
// codes: row c of Qt then has a single nonzero, a phase 1, i, -1 or -i at column
// k, stored as (k << 2) | phase, and the pair kernels form the congruence by a
// gather instead of a product.
#include "qcs_internal.h"

namespace {

// One warp per snapshot.  Dynamic shared memory: warps * (2n)^2 doubles.
__global__ void snapshot_prepare_kernel(int n, int64_t P, const double *__restrict__ Q, const uint8_t *__restrict__ b,
                                        cd *__restrict__ Qt, int8_t *__restrict__ parity, uint8_t *__restrict__ gth,
                                        int *__restrict__ nsp, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = 2 * n;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    double *A = reinterpret_cast<double *>(smem_raw) + (size_t)warp * N * N;
    for (int64_t p = (int64_t)blockIdx.x * wpb + warp; p < P; p += (int64_t)gridDim.x * wpb) {
        const double *Qp = Q + p * N * N;
        const uint8_t *bp = b + p * n;
        bool bad = false;
        int nb = 0;
        for (int j = lane; j < n; j += 32) nb += (bp[j] & 1);
        for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(QCS_FULL, nb, o);
        for (int e = lane; e < N * N; e += 32) {
            double v = Qp[e];
            bad |= !isfinite(v);
            A[e] = v;
        }
        // complexified, sign-folded rows
        cd *Qtp = Qt + p * N * n;
        for (int e = lane; e < N * n; e += 32) {
            int c = e / n, k = e - c * n;
            double sg = (c & 1) ? ((bp[c >> 1] & 1) ? -1.0 : 1.0) : 1.0;
            double q0 = Qp[c * N + 2 * k], q1 = Qp[c * N + 2 * k + 1];
            Qtp[e] = cmk(sg * q0, -sg * q1);
        }
        bad = __any_sync(QCS_FULL, bad);
        __syncwarp();
        if (gth) {
            // signed permutation?  one lane per row of Q; codes of the rows of Qt
            bool ok = true;
            for (int c = lane; c < N; c += 32) {
                int cnt = 0, col = 0;
                double val = 0.0;
                for (int j = 0; j < N; ++j) {
                    const double v = A[c * N + j];
                    if (v != 0.0) {
                        ++cnt;
                        col = j;
                        val = v;
                    }
                }
                const bool row_ok = cnt == 1 && (val == 1.0 || val == -1.0);
                ok = ok && row_ok;
                // Qt[c][k] = s_c Q[c][2k] - i s_c Q[c][2k+1], s_c the sign folded into row c
                const bool flip = (c & 1) && (bp[c >> 1] & 1);
                const bool pos = (val > 0.0) != flip;
                const int ph = (col & 1) ? (pos ? 3 : 1) : (pos ? 0 : 2);
                gth[p * N + c] = row_ok ? (uint8_t)(((col >> 1) << 2) | ph) : (uint8_t)0xFF;
            }
            ok = __all_sync(QCS_FULL, ok);
            __syncwarp();
            if (lane == 0) {
                if (!ok) gth[p * N] = 0xFF;
                else atomicAdd(nsp, 1);
            }
        }
        // sign of det(Q) by LU with partial pivoting (rows spread over lanes)
        int sign = 1;
        bool singular = false;
        for (int k = 0; k < N && !singular; ++k) {
            double best = -1.0;
            int arg = k;
            for (int i = k + lane; i < N; i += 32) {
                double a = fabs(A[i * N + k]);
                if (a > best) {
                    best = a;
                    arg = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                double ob = __shfl_xor_sync(QCS_FULL, best, o);
                int oa = __shfl_xor_sync(QCS_FULL, arg, o);
                if (ob > best || (ob == best && oa < arg)) {
                    best = ob;
                    arg = oa;
                }
            }
            if (!(best > 0.0)) {
                singular = true;
                break;
            }
            if (arg != k) {
                for (int j = lane; j < N; j += 32) {
                    double t = A[k * N + j];
                    A[k * N + j] = A[arg * N + j];
                    A[arg * N + j] = t;
                }
                sign = -sign;
            }
            __syncwarp();
            double piv = A[k * N + k];
            if (piv < 0) sign = -sign;
            double rp = 1.0 / piv;
            for (int i = k + 1 + lane; i < N; i += 32) {
                double f = A[i * N + k] * rp;
                for (int j = k + 1; j < N; ++j) A[i * N + j] = fma(-f, A[k * N + j], A[i * N + j]);
            }
            __syncwarp();
        }
        if (lane == 0) {
            int8_t pi = 0;
            if (!singular && !bad) pi = (int8_t)(((nb & 1) ? -1 : 1) * sign);
            parity[p] = pi;
            if (bad) raise_status(status, QCS_ERR_NONFINITE);
            else if (singular) raise_status(status, QCS_ERR_SINGULAR);
        }
        __syncwarp();
    }
}

// Stable compaction of the snapshots with parity +1 (single block).
__global__ void snapshot_compact_kernel(int64_t P, const int8_t *__restrict__ parity, int *__restrict__ idx,
                                        int *__restrict__ count) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (int64_t s0 = 0; s0 < P; s0 += blockDim.x) {
        int64_t p = s0 + tid;
        int flag = (p < P && parity[p] == 1) ? 1 : 0;
        unsigned bal = __ballot_sync(QCS_FULL, flag);
        int pre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int w = 0; w < warp; ++w) off += warp_tot[w];
        if (flag) idx[base + off + pre] = (int)p;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < nw; ++w) t += warp_tot[w];
            base += t;
        }
        __syncthreads();
    }
    if (tid == 0) *count = base;
}

// Per dense snapshot (gather code 0xFF, or no codes): Qh = [H1^T; G2^T] (2n x n, Qt's
// layout) with H1 = Qt^T J Qt and G2 = Qt^T J conj(Qt) (n x n; J pairs the Majorana
// indices 2a, 2a + 1 with J[2a][2a+1] = 1).  The FP64 ALU overlap kernel and the gradient
// form K = Ut Qh^T = [Ut H1 | Ut G2] in place of T = Ut Qt^T, from which
//     T_j J T_k^T = (Ut H1 Ut^T)[j][k],   T_j J conj(T_k)^T = (Ut G2 Ut^H)[j][k],
//     T_j J Qt = (Ut H1)[j],              T_j J conj(Qt) = (Ut G2)[j]
// give B^(s) and the gradient's cotangents over n-term sums instead of 2n-term ones.
// One block per snapshot (grid-stride), the snapshot's rows staged in shared memory.
__global__ void hform_kernel(int n, int64_t P, const cd *__restrict__ Qt, const uint8_t *__restrict__ gth,
                             cd *__restrict__ Qh, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cd *Qs = reinterpret_cast<cd *>(smem_raw);  // 2n x n
    const int n2 = 2 * n;
    if (!QCS_IN_BOUNDS((size_t)n2 * n * sizeof(cd) <= dyn_smem_bytes(), status)) return;
    for (int64_t q = blockIdx.x; q < P; q += gridDim.x) {
        if (gth && gth[q * n2] != 0xFF) continue;  // signed permutation: its kernels gather instead
        __syncthreads();
        for (int e = threadIdx.x; e < n2 * n; e += blockDim.x) Qs[e] = Qt[q * n2 * n + e];
        __syncthreads();
        cd *out = Qh + q * n2 * n;
        for (int e = threadIdx.x; e < n2 * n; e += blockDim.x) {
            const int c = e / n, k = e - c * n;
            const bool g2 = c >= n;  // row c of Qh: column c of H1, or column c - n of G2
            const int l = g2 ? c - n : c;
            cd acc = cmk(0.0, 0.0);
            for (int a = 0; a < n; ++a) {
                cd x = Qs[(2 * a + 1) * n + l], y = Qs[(2 * a) * n + l];
                x.y = g2 ? -x.y : x.y;
                y.y = g2 ? -y.y : y.y;
                cfma(acc, Qs[(2 * a) * n + k], x);
                cfms(acc, Qs[(2 * a + 1) * n + k], y);
            }
            out[e] = acc;
        }
    }
}

}  // namespace

qcs_status qcs_launch_snapshot_build(qcs_ctx *ctx, qcs_snapshots *s, const double *d_Q, const uint8_t *d_b,
                                     cudaStream_t st) {
    const int n = s->n;
    const int N = 2 * n;
    if (s->P > 0) {
        const int wpb = 4;
        size_t smem = (size_t)wpb * N * N * sizeof(double);
        if (qcs_set_smem(ctx, (const void *)snapshot_prepare_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
        int64_t blocks = (s->P + wpb - 1) / wpb;
        if (blocks > 4 * ctx->num_sms * 8) blocks = 4 * ctx->num_sms * 8;
        if (cudaMemsetAsync(s->d_count + 1, 0, sizeof(int), st) != cudaSuccess)
            return qcs_fail(ctx, QCS_ERR_CUDA, "snapshot counter reset");
        snapshot_prepare_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(n, s->P, d_Q, d_b, s->Qt, s->parity, s->gth,
                                                                          s->d_count + 1, ctx->d_status);
        if (qcs_check_launch(ctx, "snapshot_prepare_kernel") != QCS_OK) return QCS_ERR_CUDA;
    }
    snapshot_compact_kernel<<<1, 1024, 0, st>>>(s->P, s->parity, s->idx, s->d_count);
    return qcs_check_launch(ctx, "snapshot_compact_kernel");
}

qcs_status qcs_hform_prepare_snapshots(qcs_ctx *ctx, qcs_snapshots *s, cudaStream_t st) {
    if (s->Qh) return QCS_OK;
    const int n = s->n;
    const size_t bytes = sizeof(cd) * (size_t)(s->P > 0 ? s->P : 1) * 2 * n * n;
    if (qcs_dev_alloc(s->alloc, (void **)&s->Qh, bytes, st) != QCS_OK) {
        s->Qh = nullptr;
        return qcs_fail(ctx, QCS_ERR_CUDA, "snapshot rows [H1^T; G2^T]: device allocation failed");
    }
    s->qh_bytes = bytes;
    if (s->P == 0) return QCS_OK;
    const size_t smem = (size_t)2 * n * n * sizeof(cd);
    if (qcs_set_smem(ctx, (const void *)hform_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int64_t blocks = (int64_t)ctx->num_sms * 8;
    if (blocks > s->P) blocks = s->P;
    hform_kernel<<<(unsigned)blocks, 256, smem, st>>>(n, s->P, s->Qt, s->gth, s->Qh, ctx->d_status);
    return qcs_check_launch(ctx, "hform_kernel");
}
