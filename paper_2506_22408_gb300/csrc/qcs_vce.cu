// qcs_vce.cu -- virtual-correlation-energy walker transform (Eq. vce_overlap,
// Supplementary "Virtual Correlation Energy Derivation"), one spin sector.
//
// Orbitals are ordered core (nc), active (na), virtual; a walker Phi is NB x ne with
// ne = nc + nea.  For a trial Xi_c (x) chi (x) 0_v with every core orbital occupied
// the virtual rows drop out and
//     <Xi_c chi 0_v | phi> = det [ phi_c ; chi^dag phi_a ],
// phi_c = Phi[0:nc, :], phi_a = Phi[nc:nc+na, :].  The paper takes a unitary V from
// an SVD of the core block; any unitary V whose first nc columns span the row space
// of phi_c does the same.  With the complete Householder QR phi_c^dag = V [R_c; 0],
//     <Xi_c chi 0_v | phi> = conj(det R_c) det(chi^dag phi_a V') / det V,
// V' the last nea columns of V: the active walker act = phi_a V' (na x nea) feeds
// the active-space overlap and factor = conj(det R_c) / det V multiplies it.  Each
// reflection H = I - 2 v v^dag / (v^dag v) has det H = -1.
#include "qcs_internal.h"

namespace {

constexpr int kMaxVceNe = 64;  // nc + nea, at most

// One warp per walker.  Shared memory per warp: A (ne x nc), reflectors (ne x nc),
// E (ne x nea), one ne-vector.
__global__ void vce_kernel(int NB, int nc, int na, int nea, int64_t W, const cd *__restrict__ Phi,
                           cd *__restrict__ act, int64_t act_ws, int act_ld, cd *__restrict__ factor,
                           unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ne = nc + nea;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const size_t per = (size_t)2 * ne * (nc > 0 ? nc : 1) + (size_t)ne * (nea > 0 ? nea : 1) + ne;
    cd *A = reinterpret_cast<cd *>(smem_raw) + (size_t)warp * per;
    cd *Vr = A + (size_t)ne * (nc > 0 ? nc : 1);   // reflector k in column k, rows k..ne-1
    cd *E = Vr + (size_t)ne * (nc > 0 ? nc : 1);    // ne x nea, becomes V'
    double *vn2 = reinterpret_cast<double *>(E + (size_t)ne * (nea > 0 ? nea : 1));  // per reflector
    for (int64_t w = (int64_t)blockIdx.x * wpb + warp; w < W; w += (int64_t)gridDim.x * wpb) {
        const cd *P = Phi + w * (int64_t)NB * ne;
        // A = phi_c^dag (ne x nc): A[j][i] = conj(Phi[i][j])
        for (int e = lane; e < ne * nc; e += 32) {
            const int j = e / nc, i = e - j * nc;
            A[e] = cconj(P[i * ne + j]);
        }
        for (int e = lane; e < ne * nea; e += 32) {
            const int r = e / nea, c = e - r * nea;
            E[e] = cmk(r == nc + c ? 1.0 : 0.0, 0.0);
        }
        __syncwarp();
        cd detR = cmk(1.0, 0.0);
        int nref = 0;
        for (int k = 0; k < nc; ++k) {
            double s = 0.0;
            for (int i = k + lane; i < ne; i += 32) {
                const cd x = A[i * nc + k];
                s = fma(x.x, x.x, fma(x.y, x.y, s));
            }
            const double xn = sqrt(warp_sum(s));
            const cd x0 = A[k * nc + k];
            const double a0 = hypot(x0.x, x0.y);
            const cd ph = a0 > 0.0 ? cmk(x0.x / a0, x0.y / a0) : cmk(1.0, 0.0);
            const cd alpha = cmk(-ph.x * xn, -ph.y * xn);
            detR = cmul(detR, alpha);  // R_kk = alpha (0 for a zero column)
            for (int i = lane; i < ne; i += 32) Vr[i * nc + k] = (i < k) ? cmk(0.0, 0.0) : A[i * nc + k];
            __syncwarp();
            if (lane == 0) Vr[k * nc + k] = csub(Vr[k * nc + k], alpha);
            __syncwarp();
            double t = 0.0;
            for (int i = k + lane; i < ne; i += 32) {
                const cd v = Vr[i * nc + k];
                t = fma(v.x, v.x, fma(v.y, v.y, t));
            }
            const double vv = warp_sum(t);
            if (lane == 0) vn2[k] = vv;
            if (xn == 0.0 || vv == 0.0) {
                __syncwarp();
                continue;  // zero column: no reflection (H = I)
            }
            ++nref;
            // A <- H A on columns k..nc-1 (one lane per column)
            for (int j = k + lane; j < nc; j += 32) {
                cd d = cmk(0.0, 0.0);
                for (int i = k; i < ne; ++i) cfma(d, cconj(Vr[i * nc + k]), A[i * nc + j]);
                d = cscale(d, 2.0 / vv);
                for (int i = k; i < ne; ++i) cfms(A[i * nc + j], Vr[i * nc + k], d);
            }
            __syncwarp();
        }
        // V' = H_0 H_1 ... H_{nc-1} E: apply the reflections in reverse order
        for (int k = nc - 1; k >= 0; --k) {
            const double vv = vn2[k];
            if (vv == 0.0) continue;  // zero column: no reflection was applied
            for (int c = lane; c < nea; c += 32) {
                cd d = cmk(0.0, 0.0);
                for (int i = k; i < ne; ++i) cfma(d, cconj(Vr[i * nc + k]), E[i * nea + c]);
                d = cscale(d, 2.0 / vv);
                for (int i = k; i < ne; ++i) cfms(E[i * nea + c], Vr[i * nc + k], d);
            }
            __syncwarp();
        }
        // act = phi_a V'  (na x nea; nothing when nea = 0)
        for (int e = lane; e < na * nea; e += 32) {
            cd *out = act + w * act_ws;
            const int r = e / nea, c = e - r * nea;
            cd s = cmk(0.0, 0.0);
            for (int k = 0; k < ne; ++k) cfma(s, P[(nc + r) * ne + k], E[k * nea + c]);
            out[(int64_t)r * act_ld + c] = s;
            if (!cfinite(s)) raise_status(status, QCS_ERR_NONFINITE);
        }
        if (lane == 0) {
            const cd f = cconj(detR);
            factor[w] = (nref & 1) ? cneg(f) : f;  // det V = (-1)^{reflections}
        }
        __syncwarp();
    }
}

}  // namespace

extern "C" qcs_status qcs_vce_transform(qcs_ctx *ctx, int NB, int nc, int na, int nea, int64_t W,
                                        const double *d_walkers, double *d_act, int64_t act_walker_stride,
                                        int act_row_stride, double *d_factor, void *stream) {
    QcsRange range_("qcs_vce_transform");
    if (!ctx) return QCS_ERR_ARG;
    if (nc < 0 || na < 1 || na > QCS_MAX_N || nea < 0 || nea > na || nc + nea > kMaxVceNe || NB < nc + na)
        return qcs_fail(ctx, QCS_ERR_ARG, "vce: need 0 <= nc, 1 <= na <= QCS_MAX_N, 0 <= nea <= na, "
                                          "nc + nea <= 64, NB >= nc + na");
    if (W < 0) return qcs_fail(ctx, QCS_ERR_ARG, "W < 0");
    if (W == 0) return QCS_OK;
    if (!d_walkers || !d_factor || (nea > 0 && !d_act)) return qcs_fail(ctx, QCS_ERR_ARG, "null pointer");
    if (act_row_stride < nea || act_walker_stride < (int64_t)(na - 1) * act_row_stride + nea)
        return qcs_fail(ctx, QCS_ERR_ARG, "vce: output strides smaller than an na x nea block");
    DeviceGuard g(ctx->device);
    const int ne = nc + nea;
    const size_t per = sizeof(cd) * ((size_t)2 * ne * (nc > 0 ? nc : 1) + (size_t)ne * (nea > 0 ? nea : 1) + ne);
    int wpb = 4;
    while (wpb > 1 && (size_t)wpb * per > ctx->smem_optin) --wpb;
    const size_t smem = (size_t)wpb * per;
    if (smem > ctx->smem_optin) return qcs_fail(ctx, QCS_ERR_UNSUPPORTED, "vce: shared memory too large");
    if (qcs_set_smem(ctx, (const void *)vce_kernel, smem) != QCS_OK) return QCS_ERR_CUDA;
    int64_t blocks = (W + wpb - 1) / wpb;
    if (blocks > (int64_t)ctx->num_sms * 8) blocks = (int64_t)ctx->num_sms * 8;
    vce_kernel<<<(unsigned)blocks, wpb * 32, smem, (cudaStream_t)stream>>>(NB, nc, na, nea, W, (const cd *)d_walkers,
                                                                        (cd *)d_act, act_walker_stride,
                                                                        act_row_stride, (cd *)d_factor,
                                                                        ctx->d_status);
    return qcs_check_launch(ctx, "vce_kernel");
}
