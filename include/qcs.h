/*
 * qcs.h -- C ABI of the GB300 matchgate-shadow overlap library.
 *
 * The library evaluates, on one GPU, the classical post-processing hot path
 * of QC-AFQMC with matchgate shadows (arXiv 2506.22408):
 *
 *   for every walker w (a complex n x ne orbital matrix Phi_w) and every
 *   shadow snapshot p (an orthogonal Q_p in O(2n) and a measured n-bit
 *   string b_p) the estimator o_p(Phi_w) of Sec. "Classical shadows and the
 *   evaluation of overlaps" -- an inverse-channel weighted sum of the
 *   coefficients of the polynomial pf(A(z)), A(z) = C_0^(s) + z B^(s)
 *   (Eqs. a_mat, b_mat) -- and the shadow average
 *   <Psi_T|phi_w> = (1/P) sum_p o_p(Phi_w);
 *
 *   the holomorphic gradient d<Psi_T|phi_w>/dPhi_w through
 *   d pf(A) = pf(A) tr(A^{-1} dA) / 2  (Eq. Pfaffian_der);
 *
 *   the AFQMC force bias xbar_gamma = -sqrt(dtau) <Psi_T|v_gamma|phi>/<Psi_T|phi>
 *   (Eq. force_bias) evaluated as a derivative of the overlap (Eq. force_bias_diff);
 *
 *   the local-energy terms <Psi_T|hhat|phi>/O and sum_gamma <Psi_T|Lhat_gamma^2|phi>/O
 *   by first and second Pfaffian derivatives (Eqs. energy_tb_diff, Pfaffian_2nd_der);
 *
 *   shadow estimates of Majorana correlators, the one-particle RDM and the particle
 *   number (Supplementary "Reduced Density Matrices"), and the virtual-correlation-
 *   energy walker transform (Eq. vce_overlap).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are two consecutive doubles (re, im) (the layout of C99
 *   double complex and of cuDoubleComplex); a "complex array of k entries"
 *   is 2k doubles.
 * - Matrices are row-major.  A walker Phi is n x ne with Phi[k][j] the
 *   coefficient of orbital k in occupied column j; the walker is
 *   |phi> = prod_j (sum_k Phi[k][j] a_k^dagger) |0>, first factor leftmost.
 * - Majoranas are gamma_{2j-1} = a_j + a_j^dagger, gamma_{2j} = -i(a_j - a_j^dagger)
 *   (SI "Reduced Density Matrices"); snapshot p measured |b_p> after the
 *   matchgate circuit U_Q with U_Q^dagger gamma_mu U_Q = sum_nu Q[mu][nu] gamma_nu.
 *   b[j] = 1 means mode j was found occupied.
 * - Every data pointer is a DEVICE pointer owned by the caller unless the
 *   argument says otherwise.  Nothing is freed by the library except its own
 *   handles.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are asynchronous with respect to the host: they enqueue
 *   kernels on `stream` and return.  Argument errors are detected on the host
 *   before anything is enqueued and returned synchronously; numerical
 *   problems found by the kernels (non-finite input, non-finite pivot,
 *   singular matrix where an inverse is needed) are OR-ed into a device
 *   status word read by qcs_sync_status().
 * - Sizes: 1 <= n <= QCS_MAX_N, ne even, 2 <= ne <= n.  An odd ne is
 *   rejected: measurement outcomes are even operators, so the shadow
 *   estimator of an odd-particle overlap is identically zero.
 * - Scratch memory: a context owns one device workspace that grows (with
 *   cudaMalloc, synchronously, or with the caller's allocator set by
 *   qcs_set_allocator) when a call needs more than it holds.  Call each entry
 *   point once with the largest sizes before capturing it in a CUDA graph so
 *   that no allocation happens during capture.  Calls on the same context must
 *   not overlap in time on different streams.
 */
#ifndef QCS_H
#define QCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCS_MAX_N 24
#define QCS_MAX_NODES 49

typedef struct qcs_ctx qcs_ctx;             /* per-device context (workspace, status word) */
typedef struct qcs_snapshots qcs_snapshots; /* device-resident snapshot set */

typedef enum {
    QCS_OK = 0,
    QCS_ERR_ARG = 1,         /* invalid argument (size, null pointer, odd ne, ...) */
    QCS_ERR_CUDA = 2,        /* a CUDA runtime call failed; see qcs_last_error() */
    QCS_ERR_NONFINITE = 4,   /* device: a non-finite input or pivot was met */
    QCS_ERR_SINGULAR = 8,    /* device: A(z_k) singular where its inverse was needed */
    QCS_ERR_TIMEOUT = 16,    /* device: a bounded wait expired */
    QCS_ERR_UNSUPPORTED = 32,/* request outside what the library implements */
    QCS_ERR_BOUNDS = 64      /* device, bounds-checked debug build only (compiled with
                                -DQCS_BOUNDS, libqcs_bounds.so): a kernel found a tile, queue,
                                snapshot or output index, or its shared-memory layout, outside
                                the buffer it addresses; the access was skipped */
} qcs_status;

typedef enum {
    QCS_FP64 = 0,  /* every product and the Pfaffians in FP64 */
    QCS_TF32X3 = 1 /* qcs_overlap only, any n <= QCS_MAX_N: the congruence T = U^T Qt^T on
                      tensor cores (tcgen05 kind::tf32, hi/lo splits, hi*hi + hi*lo + lo*hi
                      accumulated in FP32), B^(s) in FP32; Pfaffians, pivoting and node sums in
                      FP64.  Rows and the contraction are padded to 32 for n <= 16 (tiles of 4
                      walkers x 4 snapshots, a warp per pair) and to 64 x 48 for 16 < n <= 24
                      (2 x 2 tiles, two warps per pair).  The snapshot set gets TF32 operand
                      slabs (8 KB per snapshot for n <= 16, 24 KB above, from the context's
                      allocator) on its first use in this mode. */
} qcs_precision;

/* qcs_opts.flags */
#define QCS_FLAG_ALL_NODES 1u /* roots of unity: evaluate pf(A(z_k)) at every node and skip no
                                 snapshot (disables the parity shortcuts described at qcs_overlap) */
#define QCS_FLAG_DFT_NODES 2u /* roots of unity with the parity shortcuts, also when nodes = 0
                                 (then N = n-ne+1) */
#define QCS_FLAG_FP64_ALU 4u  /* qcs_overlap, QCS_FP64: form the congruence on the FP64 ALU (the
                                 default for n != 16) instead of on tensor cores */
#define QCS_FLAG_FP64_TC 8u   /* qcs_overlap, QCS_FP64: form the congruence on tensor cores at FP64
                                 accuracy (the default for n = 16) for any n <= 16; not with
                                 QCS_FLAG_ALL_NODES (QCS_ERR_UNSUPPORTED) */

/* Node plans (how sum_x c_x C(2n,2x)/C(n,x) is obtained from Pfaffians):
 *  - default (nodes = 0, no node flag): a Gauss rule.  For parity +1 snapshots
 *    q(z) = pf(A(z))/z^{ne/2} is palindromic of degree d = n-ne, the weighted
 *    coefficient sum is a linear functional on a space of dimension
 *    D = floor(d/2)+1, and a Gauss rule with ceil(D/2) nodes on the unit circle
 *    (positive weights) computes it exactly: 3 Pfaffians per pair at n=16, ne=8.
 *  - roots of unity (nodes = N >= n-ne+1, or QCS_FLAG_DFT_NODES): the inverse DFT
 *    of the interpolation step after Eq. (b_mat) on N roots of unity, folded with the weights; with the
 *    parity shortcuts only floor(N/2)+1 nodes are evaluated.
 *  - QCS_FLAG_ALL_NODES: roots of unity, every node, every snapshot.
 * All plans give the same estimator up to rounding. */

typedef struct {
    int precision; /* qcs_precision */
    int nodes;     /* 0 = Gauss plan (or N = n-ne+1 roots with a node flag);
                      N > 0 = N roots of unity, n-ne+1 <= N <= QCS_MAX_NODES */
    unsigned flags;
    int config;    /* kernel configuration: 0 = the context's tuned choice for these sizes
                      (qcs_autotune / qcs_set_config) or the built-in defaults; else the
                      fields below, 0 in a field taking its default:
                        bits 0-3   node matrices per warp round, 1..8 (so a plain k keeps
                                   meaning k matrices per round)
                        bits 4-7   FP64 ALU pair kernel: snapshots per warp in a tile (4)
                        bits 8-9   FP64 ALU pair kernel, n > 16: 1 = one warp per pair,
                                   2 = two warps per pair (2)
                        bits 10-11 FP64 overlaps at n <= 16 without a path flag: 1 = congruence
                                   on the FP64 ALU, 2 = on tensor cores (tensor cores at n = 16)
                        bits 12-15 tensor-core pair kernel: sub-tiles of four snapshots per
                                   tile (8) */
} qcs_opts;

/* ------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  *ctx receives the handle.
 * Errors: QCS_ERR_ARG (ctx NULL), QCS_ERR_CUDA. */
qcs_status qcs_create(qcs_ctx **ctx, int device);

/* Free the context and its workspace (synchronises the device first). */
qcs_status qcs_destroy(qcs_ctx *ctx);

/* Text of the last error raised on this context ("" if none); owned by the context. */
const char *qcs_last_error(const qcs_ctx *ctx);

/* Wait for all work on `stream`, then return (and clear) the OR of the
 * device status bits raised since the last call; QCS_OK if none. */
qcs_status qcs_sync_status(qcs_ctx *ctx, void *stream);

/* Bytes of device workspace currently held by the context. */
size_t qcs_workspace_bytes(const qcs_ctx *ctx);

/* Device allocator callbacks (the ownership convention of the boundary: the library's
 * scratch may come from the caller's allocator, e.g. PyTorch's caching allocator).
 *   alloc_fn(bytes, stream, user) returns a device pointer of at least `bytes` on the
 *     context's device, usable in stream order on `stream` (the stream of the call that
 *     needs it), or NULL on failure (the call then returns QCS_ERR_CUDA);
 *   free_fn(ptr, bytes, stream, user) releases it; the library calls it only after the
 *     device has finished all work that used the memory, with stream = NULL.
 * Once set, the context's workspace, the buffers of snapshot sets built on the context
 * (which remember the allocator they were built with, including those a set forms on its
 * first use by a path: the split-precision slabs, and for the FP64 ALU path above 16 modes
 * and the gradient the rows [H1^T; G2^T]), the tensor-core slice records and the
 * autotuner's sample come from alloc_fn; the context's 4-byte status word and its
 * pinned host mirror, made at qcs_create, do not.  Setting an allocator releases the
 * current workspace (after synchronising the device) so that later growth uses the new
 * one; alloc_fn = free_fn = NULL restores cudaMalloc / cudaFree.  The callbacks run on the
 * calling host thread, inside the library call that needs memory; a call allocates only
 * when the workspace must grow or a set forms a buffer of a path for the first time, so
 * after one call of each path with the largest sizes none does.
 * Errors: QCS_ERR_ARG (ctx NULL, or only one of the two functions given), QCS_ERR_CUDA. */
typedef void *(*qcs_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*qcs_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
qcs_status qcs_set_allocator(qcs_ctx *ctx, qcs_alloc_fn alloc_fn, qcs_free_fn free_fn, void *user);

/* Self-test of the device time-out path (failure detection without a fault).
 * Every device wait of the library (the split-precision kernel's mbarrier waits
 * for its bulk copies and MMAs) is bounded: when the limit runs out the kernel
 * ORs QCS_ERR_TIMEOUT into the status word, drains and returns.  This call
 * launches one block that waits, through the same bounded wait, on an mbarrier
 * whose one expected arrival never happens, polling at most max_iter times;
 * no copy or MMA is issued, so nothing is in flight when it returns.
 * Arguments: max_iter in [1, 2^20]; stream a cudaStream_t (NULL = default).
 * Returns QCS_OK once launched (read QCS_ERR_TIMEOUT with qcs_sync_status),
 * QCS_ERR_ARG for max_iter out of range, QCS_ERR_CUDA if the launch fails. */
qcs_status qcs_selftest_bounded_wait(qcs_ctx *ctx, uint32_t max_iter, void *stream);

/* Self-test of the reciprocal the eliminations use for their pivots (one third-order
 * step r (1 + e + e^2) from a single-precision seed instead of an IEEE division): r[i] = 1/d[i] for
 * n values d[i] >= 0, both device arrays of doubles owned by the caller, through the
 * same device function as the pair kernels.  The result is within 2 ulp of the
 * correctly rounded 1/d; d = 0 gives +inf, as the division does.
 * Errors: QCS_ERR_ARG (ctx NULL, n < 0, null pointers with n > 0), QCS_ERR_CUDA. */
qcs_status qcs_selftest_reciprocal(qcs_ctx *ctx, const double *d, double *r, int64_t n, void *stream);

/* ---------------------------------------------------------- snapshots */

/* Build the device representation of P snapshots (Q_p, b_p).
 *   d_Q : P x 2n x 2n doubles, row-major, each Q_p orthogonal (det +-1)
 *   d_b : P x n bytes, 0 or 1
 * The library computes per snapshot the rotated covariance factor of
 * Eq. (b_mat) -- G_p = Q_p^T C_b Q_p with C_b the covariance matrix of SI
 * item 2 -- in the factorised form Q'_p = P_b Q_p, P_b = diag(1, (-1)^{b_1},
 * 1, (-1)^{b_2}, ...) so that G_p = Q'^T J Q', and the snapshot parity
 * pi_p = det Q_p (-1)^{|b_p|} = det Q'_p.  *out is owned by the library
 * (free with qcs_snapshots_free).  Inputs are only read during the call's
 * kernels; the caller may reuse them once `stream` has passed this call.
 * Some paths add per-set buffers on their first use (the split-precision slabs; for the
 * FP64 ALU path above 16 modes and for the gradient the rows [H1^T; G2^T]), formed on
 * that call's stream: a call on another stream that uses the same set must be ordered
 * after the first call of that path (or that first call made on the same stream).
 * Errors: QCS_ERR_ARG (n out of range, P < 0, null pointers), QCS_ERR_CUDA. */
qcs_status qcs_build_snapshots(qcs_ctx *ctx, int n, int64_t P, const double *d_Q, const uint8_t *d_b,
                               qcs_snapshots **out, void *stream);

qcs_status qcs_snapshots_free(qcs_snapshots *s);

/* Copy the parity pi_p (+1 / -1, one int8 per snapshot, P entries) into the
 * caller's device buffer d_parity. */
qcs_status qcs_snapshots_parity(const qcs_snapshots *s, int8_t *d_parity, void *stream);

/* Number of snapshots of the set that are signed permutations (every row of Q_p
 * has one nonzero entry, exactly +-1: the ensemble of the paper's experiment).
 * For those the pair kernels form the congruence T = U^T Qt^T as a gather with
 * sign flips (no FP64 work), and the gradient's cotangent product likewise.
 * Waits for `stream` (the build must have been issued on it or before it).
 * Errors: QCS_ERR_ARG (null pointers), QCS_ERR_CUDA. */
qcs_status qcs_snapshots_signed_perm_count(const qcs_snapshots *s, int64_t *count, void *stream);

/* Number of snapshots and modes of the set. */
int64_t qcs_snapshots_count(const qcs_snapshots *s);
int qcs_snapshots_modes(const qcs_snapshots *s);

/* ----------------------------------------------------------- overlaps */

/* Shadow overlaps <Psi_T|phi_w> = (1/P) sum_p o_p(Phi_w) for W walkers.
 *   d_walkers : W x n x ne complex (read only)
 *   d_overlap : W complex (written)
 *   d_per_pair: W x P complex (o_p of every pair, row w) or NULL
 *   opts      : NULL = defaults (FP64, Gauss node plan)
 * o_p = 2 det(R_w) i^{ne/2} / 2^{n-ne/2} sum_x c_x C(2n,2x)/C(n,x), where
 * Phi_w = U R (QR), V = U^dagger defines M_phi (SI item 3) and c_x are the
 * coefficients of pf(C_0^(s) + z B^(s)) (Eqs. a_mat, b_mat).  The factor 2
 * undoes the 1/sqrt2 of the prepared state (|0>+|Psi_T>)/sqrt2, and det R
 * restores the norm of a non-orthonormal walker.
 * Parity shortcuts (on unless QCS_FLAG_ALL_NODES): for a pure Gaussian
 * snapshot state of parity pi the coefficients obey c_{n-x} = pi c_x, and the
 * weights obey w_{n-x} = w_x, so pairs with pi = -1 are exactly zero (their
 * per-pair output is written as 0) and pairs with pi = +1 need pf(A(z_k)) at
 * only floor(N/2)+1 of the N roots of unity, or at the ceil(D/2) nodes of the
 * default Gauss plan.
 * Errors: QCS_ERR_ARG, QCS_ERR_CUDA; device bits via qcs_sync_status. */
qcs_status qcs_overlap(qcs_ctx *ctx, const qcs_snapshots *s, int ne, int64_t W, const double *d_walkers,
                       double *d_overlap, double *d_per_pair, const qcs_opts *opts, void *stream);
/* Congruence of the FP64 path.  Every entry of B^(s) is a signed sum of entries of
 * P = M H_p M^T, M the walker's real 2n x 2n form and H_p = N^T J N (N the snapshot's
 * real rows, J the canonical skew form), formed once per snapshot.  At n = 16 by
 * default (any n <= 16 with QCS_FLAG_FP64_TC) the two products Z = H_p M^T and P = M Z
 * run on tensor cores by error-free slicing: each FP64 row is cut into seven 8-bit
 * slices exact in BF16, the 28 slice products of the leading levels accumulate exactly
 * in FP32, and the levels are combined exactly in 64-bit fixed point, so each entry of P
 * carries an error of about 2^-53 times the row scales, like an FP64 product; the
 * Pfaffians stay on the FP64 pipe.  The snapshot set then holds 57,856 bytes per four
 * parity +1 snapshots of slice records (formed by qcs_build_snapshots at n = 16,
 * otherwise on first use), and the context workspace 14,464 bytes per walker. */

/* ---------------------------------------------------- local energy terms */

/* Local-energy terms of the shadow overlap by Pfaffian derivatives (Eqs.
 * force_bias_diff, energy_tb_diff, Pfaffian_der, Pfaffian_2nd_der): for W walkers,
 *   e1[w] = <Psi_T| hhat |phi_w> / <Psi_T|phi_w>,                  hhat = sum_pq h_pq a_p^dag a_q
 *   e2[w] = sum_gamma <Psi_T| Lhat_gamma Lhat_gamma |phi_w> / <Psi_T|phi_w>,
 * with numerators and the overlap as shadow means over the snapshot set.  The
 * one-body moves e^{lambda Lhat} of the walker are carried to the snapshot side
 * (the inverse channel commutes with degree-preserving similarities), so every
 * derivative is a derivative of the pair Pfaffians with respect to the selected
 * rows.  The node matrices share their occupied block, so per pair it is
 * eliminated once and each node keeps only the inverse of its 2d x 2d complement
 * (never stored beyond the pair); each Cholesky vector then costs
 * O(m (2n)^2 + m^2 d + nodes d^3) per pair.  The sum over the vectors of
 * X' J X'^T is taken per snapshot, for all walkers at once.  The Hamiltonian's own
 * factors (e.g. 1/2 on the two-body sum) are the caller's.
 *   d_walkers : W x n x ne complex (device)
 *   d_L       : nchol x n x n complex (device), Lhat_gamma = sum_pq L[gamma][p][q] a_p^dag a_q
 *   d_h       : n x n complex (device) or NULL (then e1 is not computed)
 *   d_overlap, d_e1, d_e2 : W complex each, or NULL
 * Same node options as qcs_overlap; FP64 only.  An exactly singular node matrix
 * raises QCS_ERR_SINGULAR (device status), as in qcs_overlap_grad.
 * Errors: QCS_ERR_ARG, QCS_ERR_UNSUPPORTED (precision, shared memory), QCS_ERR_CUDA. */
qcs_status qcs_local_energy(qcs_ctx *ctx, const qcs_snapshots *s, int ne, int64_t W, const double *d_walkers,
                            int nchol, const double *d_L, const double *d_h, double *d_overlap, double *d_e1,
                            double *d_e2, const qcs_opts *opts, void *stream);

/* Algorithmic FP64 flops of qcs_local_energy per parity +1 pair. */
double qcs_local_energy_flops_per_pair(int n, int ne, int nchol, int has_h, int nodes, unsigned flags);

/* -------------------------------------------- reduced density matrices */

/* Shadow estimates of Majorana correlators, the one-particle reduced density
 * matrix and the particle number from the snapshot set alone (Supplementary
 * "Reduced Density Matrices", Eq. local_fermionic_ob_exp): for rotated Majoranas
 * g~ = R g, <g~_S> = mean_p C(2n,|S|)/C(n,|S|/2) pf(i (R G_p R^T)|_S) with
 * G_p = Q_p^T C_b Q_p; every snapshot of the set counts (parity plays no role).
 *   d_R     : 2n x 2n real orthogonal, row-major (device), or NULL for R = I
 *   d_gam2  : 2n x 2n doubles or NULL: <g~_mu g~_nu> = i gam2[mu][nu] (mu != nu), 0 on the diagonal
 *   d_gam4  : C(2n,4) doubles or NULL: <g~_mu g~_nu g~_rho g~_sigma> (real) for
 *             mu < nu < rho < sigma in lexicographic order, formed from the second
 *             moments of the covariance entries (a rank-P update, FP64)
 *   d_rdm1  : n x n complex or NULL: <a~_p^dagger a~_q>, a~_p = (g~_2p + i g~_2p+1)/2
 *             (Eqs. 1rdm_off_diagonal, 1rdm_diagonal)
 *   d_npart : 1 double or NULL: the particle number, trace of the 1-RDM
 * Outputs are device buffers owned by the caller.  The call uses context workspace
 * (P n (2n-1) doubles for the covariance entries, plus the moment partials).
 * Errors: QCS_ERR_ARG (empty set, set on another device, d_gam4 with n < 2), QCS_ERR_CUDA. */
qcs_status qcs_shadow_rdm(qcs_ctx *ctx, const qcs_snapshots *s, const double *d_R, double *d_gam2, double *d_gam4,
                          double *d_rdm1, double *d_npart, void *stream);

/* Algorithmic FP64 flops of the second-moment update in qcs_shadow_rdm (d_gam4
 * requested) for n modes and P snapshots. */
double qcs_shadow_rdm_flops(int n, int64_t P);

/* ------------------------------------ virtual correlation energy (VCE) */

/* Walker transform of the virtual-correlation-energy technique (Eq. vce_overlap,
 * Supplementary "Virtual Correlation Energy Derivation"), one spin sector.  Orbitals
 * are ordered core (nc), active (na), virtual (NB - nc - na).  For a trial
 * Xi_c (x) chi (x) 0_v with every core orbital occupied,
 *     <Xi_c chi 0_v | phi_w> = factor[w] <chi | act_w>,
 * where act_w = phi_a V' (na x nea) and factor = conj(det R_c) / det V, from the
 * complete Householder QR phi_c^dagger = V [R_c; 0] of the walker's core block
 * (any unitary whose first nc columns span the core block's row space gives the same
 * product; the paper uses an SVD).  The virtual rows are not read.  act feeds
 * qcs_overlap on the active space; the overlap is linear in the walker's determinant,
 * so the full-space overlap is factor times the active one (times the other spin
 * sector's factor for unrestricted walkers).
 *   d_walkers : W x NB x (nc + nea) complex, row-major (device)
 *   d_act     : receives element (r, c) of walker w at
 *               d_act[w * act_walker_stride + r * act_row_stride + c] (complex
 *               elements), so that two spin sectors can be written as the diagonal
 *               blocks of one active walker; other elements are not touched
 *   d_factor  : W complex (device)
 * Limits: 1 <= na <= QCS_MAX_N, 0 <= nea <= na, nc >= 0, nc + nea <= 64, NB >= nc + na.
 * Errors: QCS_ERR_ARG (sizes, strides, null pointers), QCS_ERR_CUDA; a non-finite
 * result raises QCS_ERR_NONFINITE in the status word. */
qcs_status qcs_vce_transform(qcs_ctx *ctx, int NB, int nc, int na, int nea, int64_t W, const double *d_walkers,
                             double *d_act, int64_t act_walker_stride, int act_row_stride, double *d_factor,
                             void *stream);

/* ----------------------------------------------------------- batching */

#define QCS_MAX_SYSTEMS 8

/* One system of a batched call: its snapshot set (which fixes n), electron
 * count, walkers (device, W x n x ne complex) and overlap output (device, W
 * complex). */
typedef struct {
    const qcs_snapshots *snapshots;
    int ne;
    int64_t W;
    const double *d_walkers;
    double *d_overlap;
} qcs_system;

/* Overlaps of up to QCS_MAX_SYSTEMS systems with different active spaces, walker
 * and snapshot counts, with ONE launch of the pair kernel: a persistent grid
 * pulls (system, walker, snapshot-chunk) tiles from a device counter, costliest
 * systems first.  The launch runs the FP64 ALU pair kernel: each system's result
 * equals that of qcs_overlap on it with QCS_FLAG_FP64_ALU (same per-tile arithmetic
 * and reduction order), and that of the default path up to rounding.  opts (NULL = defaults) applies to
 * every system; opts->config = 0 takes each system's tuned configuration (one tuned with
 * QCS_FLAG_FP64_ALU added to the options first, the path this launch runs).
 * The call allocates nothing once the context workspace has grown to the
 * batch's size, so after one warm-up call it can be captured in a CUDA graph.
 * Errors: QCS_ERR_ARG, QCS_ERR_CUDA, QCS_ERR_UNSUPPORTED. */
qcs_status qcs_overlap_batched(qcs_ctx *ctx, int nsys, const qcs_system *systems, const qcs_opts *opts,
                               void *stream);

/* Overlaps and their holomorphic walker gradient
 *   d_grad[w][k][j] = d <Psi_T|phi_w> / d Phi_w[k][j]   (W x n x ne complex).
 * Each pair's contribution is differentiated through
 * d pf(A) = pf(A) tr(A^{-1} dA) / 2 (Eq. Pfaffian_der) with A(z_k)^{-1}
 * recomputed per node (never stored), then chained through the congruence
 * of Eq. (b_mat) and the QR of the walker.  Same options as qcs_overlap
 * (precision must be QCS_FP64).  QCS_ERR_SINGULAR is raised when some
 * A(z_k) is exactly singular (a pivot row of zeros, which structured inputs
 * such as unit-vector walkers with signed-permutation snapshots produce): the
 * formula needs A(z_k)^{-1}, and that node's term is then left out of the
 * gradient (the overlap itself stays exact).  Nearly singular node matrices
 * need no special case.  Context workspace: per walker its rows, QR factors and
 * per-chunk records, and per snapshot of the set 32 n^2 bytes (the rows
 * [H1^T; G2^T], H1 = Qt^T J Qt and G2 = Qt^T J conj(Qt), through which B and the
 * cotangents of a dense snapshot are formed). */
qcs_status qcs_overlap_grad(qcs_ctx *ctx, const qcs_snapshots *s, int ne, int64_t W, const double *d_walkers,
                            double *d_overlap, double *d_grad, const qcs_opts *opts, void *stream);

/* Force bias from overlaps and gradients (Eqs. force_bias, force_bias_diff):
 *   G_w = Phi_w g_w^T / O_w (n x n),  <v_gamma> = i tr(L_gamma G_w),
 *   d_xbar[w][gamma] = -sqrt_dt <v_gamma>   (sqrt_dt == 0: <v_gamma> itself).
 *   d_L: nchol x n x n complex (any complex matrices; real symmetric in AFQMC)
 *   d_walkers, d_overlap, d_grad as returned/used by qcs_overlap_grad.
 * Errors: QCS_ERR_ARG, QCS_ERR_CUDA. */
qcs_status qcs_force_bias(qcs_ctx *ctx, int n, int ne, int64_t W, int nchol, const double *d_L,
                          const double *d_walkers, const double *d_overlap, const double *d_grad, double sqrt_dt,
                          double *d_xbar, void *stream);

/* -------------------------------------------- allocation-free overlaps */

/* Size of the library's fixed device scratch array used by qcs_overlap_noalloc. */
#define QCS_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Shadow overlaps without any device allocation (the paper has no counterpart:
 * this is an embedding convenience).  Meant for callers that cannot let a library
 * allocate device memory when they need overlaps: hosts whose device memory is owned
 * by their own pool allocator and that forbid libraries from allocating behind their
 * back (and plug-ins running inside them), and real-time loops that must not stall on
 * the implicit synchronisation of cudaMalloc.
 * Computes exactly what qcs_build_snapshots followed by qcs_overlap (default
 * options: FP64, Gauss node plan) computes, with every intermediate buffer in a
 * fixed file-scope device array of QCS_NOALLOC_SCRATCH_BYTES (32 MiB) that each
 * GPU loading the library holds until the process exits.  No context is used; the
 * call runs on the current device, and every pointer must be on that device.
 *   d_Q       : P x 2n x 2n doubles (device), d_b : P x n bytes (device)
 *   d_walkers : W x n x ne complex (device), d_overlap : W complex (device, written)
 *   d_status  : caller-owned device word into which numerical status bits are
 *               OR-ed (QCS_ERR_NONFINITE, QCS_ERR_SINGULAR), or NULL
 * The scratch used is 32 n^2 P + 16 n^2 W + 16 W + 64 W ceil(P/16) + 5 P bytes
 * (each term rounded up to 16 bytes, plus 32); a call needing more than
 * QCS_NOALLOC_SCRATCH_BYTES returns QCS_ERR_ARG before enqueuing anything
 * (e.g. n = 16 with 64 walkers: about 8.4 KB per snapshot, so about 3900 snapshots).
 * The first call on a device looks up the array's device address (with that
 * device current).  All calls share the one array and leave their intermediates
 * in it: calls whose work overlaps in time on the GPU (different streams, or
 * different host threads) race and corrupt each other's results; serialise them.
 * Errors: QCS_ERR_ARG (sizes, null pointers, odd ne), QCS_ERR_CUDA. */
qcs_status qcs_overlap_noalloc(int n, int ne, int64_t P, const double *d_Q, const uint8_t *d_b, int64_t W,
                               const double *d_walkers, double *d_overlap, unsigned *d_status, void *stream);

/* ------------------------------------------------------------ tuning */

/* Autotuner of the overlap kernels (no counterpart in the paper).  Times configurations
 * (qcs_opts.config) of qcs_overlap for (n, ne, nodes, flags) on a synthetic sample on the
 * context's device in stages, keeping the best so far: the congruence path (FP64 ALU or
 * tensor cores, n <= 16 and no path flag), then node matrices per warp round
 * (1..min(nodes evaluated, 8)), then the tile (ALU: 2/4/8 snapshots per warp; tensor
 * cores: 2/4/8/15 sub-tiles of four snapshots), then for n > 16 one or two warps per
 * pair.  Records the fastest in the context (calls with config = 0 take it, and so does
 * qcs_overlap_batched for its systems, which keeps the ALU path) and returns it in
 * *config (may be NULL).  Allocates and frees its own sample; synchronises.
 * Errors: QCS_ERR_ARG, QCS_ERR_CUDA. */
qcs_status qcs_autotune(qcs_ctx *ctx, int n, int ne, int nodes, unsigned flags, int *config);

/* Record a configuration for (n, ne, nodes, flags) in the context, e.g. one read
 * from an autotuner cache.  config = 0 clears the entry. */
qcs_status qcs_set_config(qcs_ctx *ctx, int n, int ne, int nodes, unsigned flags, int config);

/* ------------------------------------------------------------ profiling */

/* Measurement hooks (no counterpart in the paper).  While enabled, every
 * launch of a dominant kernel (the pair kernel of qcs_overlap, the adjoint
 * kernel of qcs_overlap_grad) is bracketed by two CUDA events recorded on the
 * launch stream.  qcs_profile_read waits for the recorded events, returns
 * the summed kernel time in milliseconds and the number of launches since the
 * previous read, and clears the record.  Errors: QCS_ERR_ARG, QCS_ERR_CUDA. */
qcs_status qcs_profile_enable(qcs_ctx *ctx, int enable);
qcs_status qcs_profile_read(qcs_ctx *ctx, double *total_ms, int64_t *launches);

/* Sustained FP64 fused multiply-add rate of the context's device in TFLOP/s (no
 * counterpart in the paper; the ceiling that the FP64 kernels' roofline fractions are
 * read against, beside the unit-count peak).  Runs register-only FMA chains, eight
 * independent chains per thread and eight warps per SM, for about 2.5 s (a warm-up
 * that lets the clocks settle under load, then five timed launches); uses context
 * workspace and waits for `stream`.  *tflops: host double (2 flop per FMA).
 * Errors: QCS_ERR_ARG (null pointers), QCS_ERR_CUDA. */
qcs_status qcs_fp64_fma_rate(qcs_ctx *ctx, double *tflops, void *stream);

/* ----------------------------------------------------------- accounting */

/* Algorithmic FP64 flop count per non-trivial (pi = +1) pair of qcs_overlap
 * for (n, ne, nodes), as implemented on the FP64 ALU: the congruence K = U^T Qh^T
 * (Qh the snapshot's rows [H1^T; G2^T], H1 = Qtilde^T J Qtilde, G2 = Qtilde^T J
 * conj(Qtilde), formed once per snapshot set; K costs what T = U^T Qtilde^T would),
 * the selected covariance B^(s) from K and the walker rows (T J T^T = U^T H1 U,
 * T J conj(T)^T = U^T G2 conj(U), sums over the walker rows' non-zero entries
 * only), and the rank-2 Pfaffian updates.  The walker's
 * orbitals are first rotated to echelon form (a reflection of the occupied
 * columns changes det R by its sign, one of the complement changes nothing),
 * which makes ne(ne-1)/2 + d(d-1)/2 entries of U exact zeros that T skips.
 * The occupied orbitals are further taken in reduced form [I; X]
 * (an invertible change of basis, det folded into det R), leaving one non-zero
 * among the first ne entries of each occupied row; walkers whose X would exceed
 * 16 in magnitude (about 3 % of random walkers) keep the echelon form and do
 * ne(ne-1)/2 more products than counted.
 * The node matrices differ only in their empty x empty block, so the occupied
 * block is eliminated once per pair and each node then costs a 2d x 2d
 * Pfaffian; the count is that of this path (pairs whose occupied block would
 * grow the complement more than 2^8-fold, rare, take the full elimination per
 * node instead).  Used by the benchmark's roofline. */
double qcs_overlap_flops_per_pair(int n, int ne, int nodes, unsigned flags);

/* The same count for a pair whose snapshot is a signed permutation (no FP64
 * work in the congruence, B^(s) from the gathered T). */
double qcs_overlap_flops_per_pair_signed_perm(int n, int ne, int nodes, unsigned flags);

/* Host only: the parts of qcs_overlap_flops_per_pair, parts[0] the congruence T,
 * parts[1] the covariance B^(s) (from K), parts[2] the Pfaffian eliminations (the shared
 * occupied steps and the node complements).  At n = 16 the congruence takes three
 * real products per complex multiply-add (counted as executed: 6 flop, plus the
 * sums that form the two results and the snapshot row's re + im); elsewhere four
 * (8 flop).  parts: host array of 3 doubles.  Errors: QCS_ERR_ARG. */
qcs_status qcs_overlap_flops_breakdown(int n, int ne, int nodes, unsigned flags, double *parts);

/* Host only: the work per non-trivial pair of qcs_overlap when the congruence runs on
 * tensor cores (QCS_FP64 at n = 16, or QCS_FLAG_FP64_TC): *fp64 receives the FP64 flops
 * (the assembly of B^(s) from P and the Pfaffian eliminations, as in
 * qcs_overlap_flops_breakdown's parts[2]), *tensor the BF16 tensor-core flops of the two
 * sliced products (28 slice products of 32 x 32 x 32 each).  fp64, tensor: host doubles.
 * Errors: QCS_ERR_ARG (sizes outside n <= 16, nodes out of range, null pointers). */
qcs_status qcs_overlap_tc_work_per_pair(int n, int ne, int nodes, unsigned flags, double *fp64, double *tensor);

/* Host only (no device work): the node plan that (n, ne, nodes, flags) selects.
 * *nev receives the number of Pfaffians evaluated per pair; wnode and gamma
 * (host arrays of 2 * QCS_MAX_NODES doubles, interleaved re/im) receive for each
 * evaluated node the multiplier w_k of D and the weight gamma_k, such that the
 * pair term is sum_k gamma_k pf(B^(s) + w_k C0^(s)) (Eq. a_mat with z = 1/w_k,
 * divided by z^{m/2}).  Errors: QCS_ERR_ARG (sizes or nodes out of range,
 * null pointers). */
qcs_status qcs_node_plan_get(int n, int ne, int nodes, unsigned flags, int *nev, double *wnode, double *gamma);

/* Same for one non-trivial pair of qcs_overlap_grad: the forward pass plus,
 * per evaluated node, the backward assembly of A(z_k)^{-1} from the
 * elimination's Gauss vectors, and the per-pair cotangent products. */
double qcs_grad_flops_per_pair(int n, int ne, int nodes, unsigned flags);

/* The same count for a pair whose snapshot is a signed permutation (no FP64 work
 * in the congruence; 2 of the 2n terms of each cotangent entry). */
double qcs_grad_flops_per_pair_signed_perm(int n, int ne, int nodes, unsigned flags);

#ifdef __cplusplus
}
#endif
#endif /* QCS_H */
