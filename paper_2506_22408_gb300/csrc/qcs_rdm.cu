// qcs_rdm.cu -- shadow estimates of Majorana correlators, the one-particle RDM
// and the particle number (Supplementary "Reduced Density Matrices", Eq.
// local_fermionic_ob_exp): for rotated Majoranas g~ = R g (R in O(2n)),
//     <g~_S> = mean_p C(2n,|S|)/C(n,|S|/2) pf( i (R G_p R^T)|_S ),   G_p = Q_p^T C_b Q_p.
// |S| = 2: pf(i X|_S) = i X_{mu nu}, so <g~_mu g~_nu> = i (2n-1) mean_p X_p,mu nu.
// |S| = 4: pf(i X|_S) = -(X_01 X_23 - X_02 X_13 + X_03 X_12), so the estimates of all
// products of four distinct Majoranas are fixed combinations of the second moments
//     S2[(mu nu), (rho sigma)] = sum_p X_p,mu nu X_p,rho sigma
// of the covariance entries: a symmetric rank-P update (K = P), the FP64 contraction
// that dominates this path.  The 1-RDM follows Eqs. (1rdm_off_diagonal) and
// (1rdm_diagonal): a~_p = (g~_2p + i g~_2p+1)/2.
//
// Kernels: rdm_cov_kernel (warp per snapshot: X_p = (Q' R^T)^T J (Q' R^T) from the
// stored rows Qt, upper triangle to global), rdm_colsum_kernel (deterministic
// column sums), rdm_syrk_kernel (32 x 32 FP64 tiles of S2, split over snapshot
// ranges, upper tiles only), rdm_finalize_kernel (gam2, rdm1, particle number,
// gam4 from the reduced S2).
#include "qcs_internal.h"

namespace {

constexpr int kTile = 32;     // S2 tile edge (small tiles: less work in the lower halves of diagonal tiles)
constexpr int kTThreads = 64; // threads per S2 tile: 8 x 8, each 4 x 4 entries
constexpr int kKStep = 16;    // snapshots staged per step
constexpr int kColRows = 256; // rows per column-sum partial (at least)

// Upper-triangle pair index of (mu, nu), mu < nu < N2, in row-major order.
__host__ __device__ __forceinline__ int pair_rank(int mu, int nu, int N2) {
    return mu * N2 - mu * (mu + 1) / 2 + (nu - mu - 1);
}

__global__ void rdm_cov_kernel(int n, int64_t P, const cd *__restrict__ Qt, const double *__restrict__ R,
                               double *__restrict__ Gu) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N2 = 2 * n, npair = N2 * (N2 - 1) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    double *Qp = reinterpret_cast<double *>(smem_raw) + (size_t)warp * 2 * N2 * N2;  // Q' (N2 x N2)
    double *X = Qp + N2 * N2;                                                       // Q' R^T
    for (int64_t p = (int64_t)blockIdx.x * wpb + warp; p < P; p += (int64_t)gridDim.x * wpb) {
        const cd *q = Qt + p * N2 * n;
        for (int e = lane; e < N2 * n; e += 32) {  // Q'[c][2k] = Re Qt[c][k], Q'[c][2k+1] = -Im Qt[c][k]
            const int c = e / n, k = e - c * n;
            const cd v = q[e];
            Qp[c * N2 + 2 * k] = v.x;
            Qp[c * N2 + 2 * k + 1] = -v.y;
        }
        __syncwarp();
        const double *Y = Qp;
        if (R) {
            for (int e = lane; e < N2 * N2; e += 32) {
                const int c = e / N2, mu = e - c * N2;
                double s = 0.0;
                for (int k = 0; k < N2; ++k) s = fma(Qp[c * N2 + k], R[mu * N2 + k], s);
                X[e] = s;
            }
            __syncwarp();
            Y = X;
        }
        // X_p[mu][nu] = sum_j Y[2j][mu] Y[2j+1][nu] - Y[2j+1][mu] Y[2j][nu]   (Y^T J Y)
        double *out = Gu + p * npair;
        for (int t = lane; t < npair; t += 32) {
            // unrank t -> (mu, nu)
            int mu = 0, rem = t;
            while (rem >= N2 - 1 - mu) {
                rem -= N2 - 1 - mu;
                ++mu;
            }
            const int nu = mu + 1 + rem;
            double s = 0.0;
            for (int j = 0; j < n; ++j) {
                s = fma(Y[(2 * j) * N2 + mu], Y[(2 * j + 1) * N2 + nu], s);
                s = fma(-Y[(2 * j + 1) * N2 + mu], Y[(2 * j) * N2 + nu], s);
            }
            out[t] = s;
        }
        __syncwarp();
    }
}

// part[r][t] = sum of Gu[p][t] over the rows p of block-row r (rows per block-row each).
__global__ void rdm_colsum_kernel(int64_t P, int npair, int64_t rows, const double *__restrict__ Gu,
                                  double *__restrict__ part) {
    const int64_t r = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npair) return;
    const int64_t p0 = r * rows, p1 = p0 + rows < P ? p0 + rows : P;
    double s = 0.0;
    for (int64_t p = p0; p < p1; ++p) s += Gu[p * npair + t];
    part[r * npair + t] = s;
}

// S2 partials: block (ti, tj, ks) with ti <= tj computes the 32 x 32 tile
// sum_{p in range ks} Gu[p][i] Gu[p][j]; each of the 64 threads owns 4 x 4 entries.
__global__ void __launch_bounds__(kTThreads) rdm_syrk_kernel(int64_t P, int npair, int ntile, int64_t krange,
                                                             const double *__restrict__ Gu, double *__restrict__ S2p) {
    __shared__ double As[kKStep][kTile + 1];
    __shared__ double Bs[kKStep][kTile + 1];
    // upper-triangle tile (ti, tj) from the linear block index
    int lin = blockIdx.x, ti = 0;
    while (lin >= ntile - ti) {
        lin -= ntile - ti;
        ++ti;
    }
    const int tj = ti + lin;
    const int64_t ks = blockIdx.y;
    const int64_t p0 = ks * krange, p1 = p0 + krange < P ? p0 + krange : P;
    const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
    const int i0 = ti * kTile, j0 = tj * kTile;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
    for (int64_t pb = p0; pb < p1; pb += kKStep) {
        for (int e = threadIdx.x; e < kKStep * kTile; e += blockDim.x) {
            const int kk = e / kTile, col = e - kk * kTile;
            const int64_t p = pb + kk;
            const bool in = p < p1;
            As[kk][col] = (in && i0 + col < npair) ? Gu[p * npair + i0 + col] : 0.0;
            Bs[kk][col] = (in && j0 + col < npair) ? Gu[p * npair + j0 + col] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKStep; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty + 8 * u];
                bb[u] = Bs[kk][tx + 8 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
        }
        __syncthreads();
    }
    double *out = S2p + (size_t)ks * npair * npair;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + ty + 8 * u, j = j0 + tx + 8 * v;
            if (i < npair && j < npair && i <= j) out[(size_t)i * npair + j] = acc[u][v];
        }
}

__host__ __device__ inline double binom_d(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

// Lexicographic rank of the 4-subset a < b < c < d of {0..N-1}.
__device__ __forceinline__ long long rank4(int a, int b, int c, int d, int N) {
    return (long long)(binom_d(N, 4) + 0.5) - 1 -
           (long long)(binom_d(N - 1 - a, 4) + binom_d(N - 1 - b, 3) + binom_d(N - 1 - c, 2) +
                       binom_d(N - 1 - d, 1) + 0.5);
}

// S2 entry (pair i, pair j) summed over the snapshot ranges (only i <= j is stored).
__device__ __forceinline__ double s2_at(const double *S2p, int nks, int npair, int i, int j) {
    if (i > j) {
        int t = i;
        i = j;
        j = t;
    }
    double s = 0.0;
    for (int k = 0; k < nks; ++k) s += S2p[(size_t)k * npair * npair + (size_t)i * npair + j];
    return s;
}

__global__ void rdm_finalize_kernel(int n, int64_t P, int nrow, const double *__restrict__ part,
                                    const double *__restrict__ S2p, int nks, double *__restrict__ gam2,
                                    double *__restrict__ gam4, cd *__restrict__ rdm1, double *__restrict__ npart) {
    const int N2 = 2 * n, npair = N2 * (N2 - 1) / 2;
    const double invP = 1.0 / (double)P;
    const double K2 = binom_d(N2, 2) / binom_d(n, 1), K4 = n >= 2 ? binom_d(N2, 4) / binom_d(n, 2) : 0.0;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    auto mean_pair = [&](int mu, int nu) {  // K2 mean_p X[mu][nu], antisymmetric, 0 on the diagonal
        if (mu == nu) return 0.0;
        const int lo = mu < nu ? mu : nu, hi = mu < nu ? nu : mu;
        const int t = pair_rank(lo, hi, N2);
        double s = 0.0;
        for (int r = 0; r < nrow; ++r) s += part[(size_t)r * npair + t];
        s *= K2 * invP;
        return mu < nu ? s : -s;
    };
    if (gam2)
        for (int e = tid; e < N2 * N2; e += nthr) gam2[e] = mean_pair(e / N2, e % N2);
    if (rdm1 || npart) {
        // <g_mu g_nu> = i gam2[mu][nu];  a_p^dag a_q = (1/4)(g_2p - i g_2p+1)(g_2q + i g_2q+1)
        for (int e = tid; e < n * n; e += nthr) {
            const int p = e / n, q = e - p * n;
            cd d;
            if (p == q) {
                d = cmk(0.5 * (1.0 - mean_pair(2 * p, 2 * p + 1)), 0.0);
            } else {
                const double g00 = mean_pair(2 * p, 2 * q), g01 = mean_pair(2 * p, 2 * q + 1);
                const double g10 = mean_pair(2 * p + 1, 2 * q), g11 = mean_pair(2 * p + 1, 2 * q + 1);
                // (1/4)(i g00 + i (i g01) - i (i g10) + i g11) = (1/4)(-g01 + g10, g00 + g11)
                d = cmk(0.25 * (g10 - g01), 0.25 * (g00 + g11));
            }
            if (rdm1) rdm1[e] = d;
        }
        if (npart && tid == 0) {
            double s = 0.0;
            for (int p = 0; p < n; ++p) s += 0.5 * (1.0 - mean_pair(2 * p, 2 * p + 1));
            *npart = s;
        }
    }
    if (gam4 && S2p) {
        // one thread per ordered pair of index pairs (mu<nu), (rho<sigma) with nu < rho
        for (long long e = tid; e < (long long)npair * npair; e += nthr) {
            const int t1 = (int)(e / npair), t2 = (int)(e - (long long)t1 * npair);
            int mu = 0, rem = t1;
            while (rem >= N2 - 1 - mu) {
                rem -= N2 - 1 - mu;
                ++mu;
            }
            const int nu = mu + 1 + rem;
            int rho = 0;
            rem = t2;
            while (rem >= N2 - 1 - rho) {
                rem -= N2 - 1 - rho;
                ++rho;
            }
            const int sg = rho + 1 + rem;
            if (nu >= rho) continue;
            const double v = s2_at(S2p, nks, npair, t1, t2) -
                             s2_at(S2p, nks, npair, pair_rank(mu, rho, N2), pair_rank(nu, sg, N2)) +
                             s2_at(S2p, nks, npair, pair_rank(mu, sg, N2), pair_rank(nu, rho, N2));
            gam4[rank4(mu, nu, rho, sg, N2)] = -K4 * v * invP;
        }
    }
}

}  // namespace

extern "C" qcs_status qcs_shadow_rdm(qcs_ctx *ctx, const qcs_snapshots *s, const double *d_R, double *d_gam2,
                                     double *d_gam4, double *d_rdm1, double *d_npart, void *stream) {
    QcsRange range_("qcs_shadow_rdm");
    if (!ctx) return QCS_ERR_ARG;
    if (!s) return qcs_fail(ctx, QCS_ERR_ARG, "null snapshot set");
    if (s->device != ctx->device) return qcs_fail(ctx, QCS_ERR_ARG, "snapshot set lives on another device");
    if (s->P < 1) return qcs_fail(ctx, QCS_ERR_ARG, "the snapshot set is empty");
    const int n = s->n, N2 = 2 * n, npair = N2 * (N2 - 1) / 2;
    if (d_gam4 && n < 2) return qcs_fail(ctx, QCS_ERR_ARG, "four-Majorana estimates need n >= 2");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceGuard g(ctx->device);
    const int64_t P = s->P;
    int64_t rows = kColRows;
    if ((P + rows - 1) / rows > 4096) rows = (P + 4095) / 4096;  // at most 4096 block-rows (grid.y)
    const int nrow = (int)((P + rows - 1) / rows);
    // split the snapshot range of the S2 update so that the grid covers the GPU
    const int ntile = (npair + kTile - 1) / kTile;
    const int nut = ntile * (ntile + 1) / 2;
    int nks = 1;
    if (d_gam4) {
        nks = (int)((16 * (int64_t)ctx->num_sms + nut - 1) / nut);  // 16 blocks of 2 warps per SM
        const int64_t maxks = (P + 4 * kKStep - 1) / (4 * kKStep);
        if (nks > maxks) nks = (int)maxks;
        if (nks < 1) nks = 1;
    }
    const int64_t krange = ((P + nks - 1) / nks + kKStep - 1) / kKStep * kKStep;
    size_t b_gu = align16(sizeof(double) * (size_t)P * npair);
    size_t b_part = align16(sizeof(double) * (size_t)nrow * npair);
    size_t b_s2 = d_gam4 ? align16(sizeof(double) * (size_t)nks * npair * npair) : 0;
    void *base = nullptr;
    qcs_status ws = qcs_workspace(ctx, b_gu + b_part + b_s2, &base, st);
    if (ws != QCS_OK) return ws;
    double *Gu = (double *)base;
    double *part = (double *)((char *)base + b_gu);
    double *S2p = d_gam4 ? (double *)((char *)base + b_gu + b_part) : nullptr;
    {
        const int wpb = 4;
        const size_t smem = (size_t)wpb * 2 * N2 * N2 * sizeof(double);
        if (qcs_set_smem(ctx, (const void *)rdm_cov_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
        int64_t blocks = (P + wpb - 1) / wpb;
        if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
        rdm_cov_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(n, P, s->Qt, d_R, Gu);
        qcs_status r = qcs_check_launch(ctx, "rdm_cov_kernel");
        if (r != QCS_OK) return r;
    }
    rdm_colsum_kernel<<<dim3((unsigned)((npair + 127) / 128), (unsigned)nrow), 128, 0, st>>>(P, npair, rows, Gu,
                                                                                            part);
    qcs_status r = qcs_check_launch(ctx, "rdm_colsum_kernel");
    if (r != QCS_OK) return r;
    if (d_gam4) {
        if (cudaMemsetAsync(S2p, 0, b_s2, st) != cudaSuccess) return qcs_fail(ctx, QCS_ERR_CUDA, "S2 reset");
        qcs_prof_begin(ctx, st);
        rdm_syrk_kernel<<<dim3((unsigned)nut, (unsigned)nks), kTThreads, 0, st>>>(P, npair, ntile, krange, Gu, S2p);
        qcs_prof_end(ctx, st);
        r = qcs_check_launch(ctx, "rdm_syrk_kernel");
        if (r != QCS_OK) return r;
    }
    int64_t fin = d_gam4 ? ((int64_t)npair * npair + 255) / 256 : 4;
    if (fin > (int64_t)ctx->num_sms * 8) fin = (int64_t)ctx->num_sms * 8;
    rdm_finalize_kernel<<<(unsigned)fin, 256, 0, st>>>(n, P, nrow, part, S2p, nks, d_gam2, d_gam4, (cd *)d_rdm1,
                                                       d_npart);
    return qcs_check_launch(ctx, "rdm_finalize_kernel");
}

extern "C" double qcs_shadow_rdm_flops(int n, int64_t P) {
    if (n < 2 || n > QCS_MAX_N || P < 1) return 0.0;
    const double npair = (double)(2 * n) * (2 * n - 1) / 2.0;
    // the symmetric rank-P update of the pair moments (upper triangle incl. diagonal)
    return 2.0 * (double)P * npair * (npair + 1.0) / 2.0;
}
