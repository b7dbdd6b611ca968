// qcs_walker.cu -- per-walker preparation for the overlap kernels.
//
// A walker Phi (n x ne, non-orthonormal) is factored Phi = U[:, :ne] R by
// complex Householder reflections; U (n x n unitary) completes the occupied
// orbitals.  With V = U^dagger the walker is the Slater determinant
// a~_1^dagger ... a~_ne^dagger |0> of SI "Matrix Definitions" item 3 times det R.
//
// Output per walker (U and R optionally, for the gradient):
//   Ut[j][k] = U[k][j] (row j = orbital j), rows j < ne scaled by 1/sqrt2 -- the
//              (1, -i)/sqrt2 row of the W^* block of Eq. (b_mat) selected for an
//              occupied mode contributes conj(V_jk)/sqrt2 = U_kj/sqrt2;
//   pref     = 2 det(R) i^{ne/2} / 2^{n - ne/2}  (prefactor of the estimator;
//              the 2 undoes the 1/sqrt2 of the prepared state (|0>+|Psi_T>)/sqrt2).
//
// Echelon form (echelon = true, for the overlap kernels): the estimator is linear and
// alternating in the occupied orbitals, o_p(U_occ W) = det(W) o_p(U_occ), and does not
// depend on which orthonormal basis completes them.  Column reflections (det -1
// each) therefore bring the top ne x ne block of U_occ and the bottom d x d block of
// the completion to lower-triangular form, det R taking the reflections' sign:
// row j < ne of Ut is then zero in columns k < j, row ne + j' zero in columns
// [ne, ne + j'), ne(ne-1)/2 + d(d-1)/2 exact zeros that the congruence skips.
//
// Reduced form (mode != null): the alternation holds for any invertible W, so the
// occupied orbitals may also be taken as U_occ L^{-1} = [I; X], L the (lower
// triangular) top block, with det R multiplied by det L.  Row j < ne of Ut then has
// one entry 1/sqrt2 at column j and zeros in the other columns k < ne.  A walker
// whose X would exceed 16 in magnitude (an ill-conditioned top block) keeps the
// echelon form; mode[w] records which (1: reduced).
#include "qcs_internal.h"

namespace {

__global__ void walker_prep_kernel(int n, int ne, int64_t W, const cd *__restrict__ Phi, cd *__restrict__ Ut,
                                   cd *__restrict__ pref, cd *__restrict__ Uout, cd *__restrict__ Rout, int echelon,
                                   int *__restrict__ mode, cd *__restrict__ Wout, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const size_t per_warp = (size_t)n * ne + (size_t)n * n + n + (Wout ? (size_t)ne * ne : 0);
    cd *A = reinterpret_cast<cd *>(smem_raw) + warp * per_warp;
    cd *U = A + n * ne;
    cd *v = U + n * n;
    cd *Wr = v + n;  // the occupied columns' rotation W of the echelon form (ne x ne)
    for (int64_t w = (int64_t)blockIdx.x * wpb + warp; w < W; w += (int64_t)gridDim.x * wpb) {
        const cd *Pw = Phi + w * n * ne;
        bool bad = false;
        for (int e = lane; e < n * ne; e += 32) {
            cd x = Pw[e];
            bad |= !cfinite(x);
            A[e] = x;
        }
        for (int e = lane; e < n * n; e += 32) U[e] = cmk((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
        bad = __any_sync(QCS_FULL, bad);
        __syncwarp();
        cd detR = cmk(1.0, 0.0);
        for (int k = 0; k < ne; ++k) {
            cd x = (lane >= k && lane < n) ? A[lane * ne + k] : cmk(0.0, 0.0);
            double xn2 = warp_sum(fma(x.x, x.x, x.y * x.y));
            if (!(xn2 > 0.0)) {  // zero column: R_kk = 0, the determinant vanishes
                detR = cmk(0.0, 0.0);
                continue;
            }
            double xn = sqrt(xn2);
            cd x0 = A[k * ne + k];
            double ax0 = hypot(x0.x, x0.y);
            cd ph = ax0 > 0.0 ? cmk(x0.x / ax0, x0.y / ax0) : cmk(1.0, 0.0);
            cd alpha = cmk(-ph.x * xn, -ph.y * xn);
            cd vi = (lane > k && lane < n) ? x : (lane == k ? csub(x0, alpha) : cmk(0.0, 0.0));
            double vn2 = warp_sum(fma(vi.x, vi.x, vi.y * vi.y));
            double tau = 2.0 / vn2;
            if (lane < n) v[lane] = vi;
            __syncwarp();
            // A <- (I - tau v v^H) A on columns k..ne-1
            for (int j = k; j < ne; ++j) {
                cd a = lane < n ? A[lane * ne + j] : cmk(0.0, 0.0);
                cd s = warp_csum(cmul(cconj(vi), a));
                s = cscale(s, tau);
                if (lane < n) A[lane * ne + j] = csub(a, cmul(vi, s));
            }
            // U <- U (I - tau v v^H): row r = lane
            if (lane < n) {
                cd sr = cmk(0.0, 0.0);
                for (int i = k; i < n; ++i) cfma(sr, U[lane * n + i], v[i]);
                sr = cscale(sr, tau);
                for (int i = k; i < n; ++i) cfms(U[lane * n + i], sr, cconj(v[i]));
            }
            __syncwarp();
            detR = cmul(detR, alpha);
        }
        if (echelon) {
            if (Wout) {  // Wr has room in this warp's slot only when the rotation is requested
                for (int e = lane; e < ne * ne; e += 32) Wr[e] = cmk((e / ne) == (e % ne) ? 1.0 : 0.0, 0.0);
                __syncwarp();
            }
            int nref = 0;  // reflections on the occupied columns (det -1 each)
            for (int blk = 0; blk < 2; ++blk) {
                const int c0 = blk == 0 ? 0 : ne, c1 = blk == 0 ? ne : n;
                for (int r = 0; r + 1 < c1 - c0; ++r) {
                    const int row = c0 + r, cs = c0 + r;  // zero U[row][cs+1 .. c1-1]
                    const cd y = (lane >= cs && lane < c1) ? cconj(U[row * n + lane]) : cmk(0.0, 0.0);
                    const double tail = warp_sum(lane > cs && lane < c1 ? fma(y.x, y.x, y.y * y.y) : 0.0);
                    if (!(tail > 0.0)) continue;  // the row is already in echelon form
                    const cd y0 = cconj(U[row * n + cs]);
                    const double yn = sqrt(tail + fma(y0.x, y0.x, y0.y * y0.y));
                    const double a0 = hypot(y0.x, y0.y);
                    const cd ph = a0 > 0.0 ? cmk(y0.x / a0, y0.y / a0) : cmk(1.0, 0.0);
                    const cd alpha = cmk(-ph.x * yn, -ph.y * yn);
                    const cd vi = (lane == cs) ? csub(y0, alpha) : y;  // v = y - alpha e_cs
                    const double tau = 2.0 / warp_sum(fma(vi.x, vi.x, vi.y * vi.y));
                    if (lane < n) v[lane] = vi;
                    __syncwarp();
                    if (lane < n) {  // U <- U (I - tau v v^H) on columns cs .. c1-1: row = lane
                        cd sr = cmk(0.0, 0.0);
                        for (int c = cs; c < c1; ++c) cfma(sr, U[lane * n + c], v[c]);
                        sr = cscale(sr, tau);
                        for (int c = cs; c < c1; ++c) cfms(U[lane * n + c], sr, cconj(v[c]));
                    }
                    if (Wout && blk == 0 && lane < ne) {  // W <- W (I - tau v v^H), same columns
                        cd sr = cmk(0.0, 0.0);
                        for (int c = cs; c < c1; ++c) cfma(sr, Wr[lane * ne + c], v[c]);
                        sr = cscale(sr, tau);
                        for (int c = cs; c < c1; ++c) cfms(Wr[lane * ne + c], sr, cconj(v[c]));
                    }
                    __syncwarp();
                    if (lane > cs && lane < c1) U[row * n + lane] = cmk(0.0, 0.0);  // exact zeros
                    __syncwarp();
                    if (blk == 0) ++nref;
                }
            }
            if (nref & 1) detR = cneg(detR);  // det R' = conj(det W) det R, det W = (-1)^nref
            if (Wout) {  // det(conj W) W, then det(conj W) itself: adj(W^H R) = adj(R) det(conj W) W
                __syncwarp();
                const double sg = (nref & 1) ? -1.0 : 1.0;
                cd *Wo = Wout + w * ((size_t)ne * ne + 1);
                for (int e = lane; e < ne * ne; e += 32) Wo[e] = cscale(Wr[e], sg);
                if (lane == 0) Wo[ne * ne] = cmk(sg, 0.0);
            }
            if (mode) {
                // X L = U_bot by back substitution over the columns (lane = row of U_bot)
                bool ok = true;
                for (int j = 0; j < ne; ++j) ok &= cmul(U[j * n + j], cconj(U[j * n + j])).x > 0.0;
                cd xr[QCS_MAX_N];
                double xmax = 0.0;
                if (ok && lane >= ne && lane < n) {
                    for (int j = ne - 1; j >= 0; --j) {
                        cd s = U[lane * n + j];
                        for (int l = j + 1; l < ne; ++l) cfms(s, xr[l], U[l * n + j]);
                        const cd x = cmul(s, cinv(U[j * n + j]));
                        xr[j] = x;
                        const double ax = fmax(fabs(x.x), fabs(x.y));
                        xmax = ax > xmax ? ax : xmax;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) xmax = fmax(xmax, __shfl_xor_sync(QCS_FULL, xmax, o));
                const bool red = ok && xmax <= 16.0;
                __syncwarp();
                if (red) {
                    cd dl = cmk(1.0, 0.0);  // det L
                    for (int j = 0; j < ne; ++j) dl = cmul(dl, U[j * n + j]);
                    detR = cmul(detR, dl);
                    if (lane < n)
                        for (int j = 0; j < ne; ++j)
                            U[lane * n + j] = lane < ne ? cmk(lane == j ? 1.0 : 0.0, 0.0) : xr[j];
                }
                __syncwarp();
                if (lane == 0) mode[w] = red ? 1 : 0;
            }
        }
        const double rs2 = 0.70710678118654752440;
        cd *Uw = Ut + w * n * n;
        for (int e = lane; e < n * n; e += 32) {
            int j = e / n, kk = e - j * n;
            cd u = U[kk * n + j];
            Uw[e] = (j < ne) ? cscale(u, rs2) : u;
        }
        if (Uout)
            for (int e = lane; e < n * n; e += 32) Uout[w * n * n + e] = U[e];
        if (Rout)
            for (int e = lane; e < ne * ne; e += 32) {
                int i = e / ne, j = e - i * ne;
                Rout[w * ne * ne + e] = (j >= i) ? A[i * ne + j] : cmk(0.0, 0.0);
            }
        if (lane == 0) {
            cd ip;  // i^{ne/2}
            switch ((ne / 2) & 3) {
                case 0: ip = cmk(1, 0); break;
                case 1: ip = cmk(0, 1); break;
                case 2: ip = cmk(-1, 0); break;
                default: ip = cmk(0, -1); break;
            }
            double sc = 2.0 * ldexp(1.0, -(n - ne / 2));
            pref[w] = cscale(cmul(detR, ip), sc);
            if (bad || !cfinite(detR)) raise_status(status, QCS_ERR_NONFINITE);
        }
        __syncwarp();
    }
}

}  // namespace

qcs_status qcs_launch_walker_prep(qcs_ctx *ctx, int n, int ne, int64_t W, const cd *walkers, cd *Ut, cd *pref,
                                  cudaStream_t st, cd *Uout, cd *Rout, bool echelon, int *mode, cd *Wout) {
    if (W == 0) return QCS_OK;
    const int wpb = 4;
    if (!echelon) Wout = nullptr;
    size_t smem = (size_t)wpb * ((size_t)n * ne + (size_t)n * n + n + (Wout ? (size_t)ne * ne : 0)) * sizeof(cd);
    if (qcs_set_smem(ctx, (const void *)walker_prep_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int64_t blocks = (W + wpb - 1) / wpb;
    if (blocks > (int64_t)ctx->num_sms * 16) blocks = (int64_t)ctx->num_sms * 16;
    walker_prep_kernel<<<(unsigned)blocks, wpb * 32, smem, st>>>(n, ne, W, walkers, Ut, pref, Uout, Rout,
                                                                   echelon ? 1 : 0, echelon ? mode : nullptr,
                                                                   Wout, ctx->d_status);
    return qcs_check_launch(ctx, "walker_prep_kernel");
}
