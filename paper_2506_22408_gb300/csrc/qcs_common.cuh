// qcs_common.cuh -- device helpers shared by the GB300 kernels of libqcs.
//
// Complex numbers are double2 (x = re, y = im), the layout of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qcs.h"

typedef double2 cd;

#define QCS_WARP 32
#define QCS_FULL 0xffffffffu

__host__ __device__ __forceinline__ cd cmk(double x, double y) { return make_double2(x, y); }

__device__ __forceinline__ cd cmul(cd a, cd b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cd cadd(cd a, cd b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cd csub(cd a, cd b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cd cneg(cd a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ cd cconj(cd a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ cd cscale(cd a, double s) { return make_double2(a.x * s, a.y * s); }

// acc += a * b
__device__ __forceinline__ void cfma(cd &acc, cd a, cd b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
__device__ __forceinline__ void cfms(cd &acc, cd a, cd b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
// -(a * b), with the negation folded into the FP64 operand modifiers
__device__ __forceinline__ cd cnegmul(cd a, cd b) {
    return make_double2(fma(-a.x, b.x, a.y * b.y), fma(-a.x, b.y, -(a.y * b.x)));
}

// Sign flip of both components by integer XOR on the sign bits (no FP64 work).
__device__ __forceinline__ cd flip_if(cd z, bool f) {
    const long long m = f ? (long long)0x8000000000000000ull : 0ll;
    z.x = __longlong_as_double(__double_as_longlong(z.x) ^ m);
    z.y = __longlong_as_double(__double_as_longlong(z.y) ^ m);
    return z;
}

// acc += a * r  (r real)
__device__ __forceinline__ void crfma(cd &acc, cd a, double r) {
    acc.x = fma(a.x, r, acc.x);
    acc.y = fma(a.y, r, acc.y);
}

// 1/d for d = |a|^2 >= 0 from a single-precision seed r refined by one third-order step:
// with e = 1 - d r, 1/d = r / (1 - e) = r (1 + e + e^2 + e^3 + ...), and the step keeps
// r (1 + e + e^2), i.e. r + r (e + e^2) in two FMAs (the iteration for the reciprocal in
// Markstein, "Computation of elementary functions on the IBM RISC System/6000 processor",
// IBM J. Res. Dev. 34, 1990, carried one term further).  The seed is the hardware's
// approximate FP32 reciprocal of d truncated to 20 mantissa bits, both conversions done on
// the bit patterns, so |e| < 2^-19 and the truncation error e^3 is below 2^-57 relative:
// the result is within one rounding of the last FMA (1 ulp) of 1/d.  Three FP64 FMAs
// against the longer sequence of an IEEE division; exponents outside the FP32 range (and
// zero, infinity, NaN) take the division.
__device__ __forceinline__ double recip_nonneg(double d) {
    const unsigned hi = (unsigned)__double2hiint(d);
    const int E = (int)(hi >> 20) - 1023;  // d >= 0: no sign bit
    if (E < -125 || E > 125) return 1.0 / d;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(((unsigned)(E + 127) << 23) | ((hi & 0xfffffu) << 3))));
    const unsigned rb = __float_as_uint(rf);
    const double r = __hiloint2double((int)(((((rb >> 23) & 0xffu) + 1023u - 127u) << 20) | ((rb & 0x7fffffu) >> 3)),
                                      (int)((rb & 7u) << 29));
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// 1/a for complex a; returns 0 when a == 0.
__device__ __forceinline__ cd cinv(cd a) {
    const double d = fma(a.x, a.x, a.y * a.y);
    if (__double2hiint(d) == 0 && __double2loint(d) == 0) return make_double2(0.0, 0.0);
    const double r = recip_nonneg(d);
    return make_double2(a.x * r, -a.y * r);
}

__device__ __forceinline__ bool cfinite(cd a) { return isfinite(a.x) && isfinite(a.y); }

// Entry (i, j), i != j, of a skew-symmetric matrix stored as its packed strict upper
// triangle: one load, and the sign of the lower triangle flipped on the bit patterns
// (no branch, no FP64 instruction).
__device__ __forceinline__ cd skew_get(const cd *__restrict__ N, int i, int j) {
    const bool lo = i > j;
    const int a = lo ? j : i, b = lo ? i : j;
    return flip_if(N[(b * (b - 1)) / 2 + a], lo);
}

// The same with the diagonal (i == j) read as zero, without a branch: the diagonal
// reads entry 0 and selects zero.
__device__ __forceinline__ cd skew_get0(const cd *__restrict__ N, int i, int j) {
    const bool lo = i > j, diag = i == j;
    const int a = lo ? j : i, b = lo ? i : j;
    const cd x = flip_if(N[diag ? 0 : (b * (b - 1)) / 2 + a], lo);
    return diag ? make_double2(0.0, 0.0) : x;
}

// Pivot magnitude key without floating-point work: the high 32 bits of
// max(|re|, |im|) (sign, exponent and 20 mantissa bits) order magnitudes to a
// relative 2^-20, enough for partial pivoting.  NaN/Inf give the largest keys.
__device__ __forceinline__ unsigned pivot_key(cd a) {
    unsigned hx = (unsigned)__double2hiint(a.x) & 0x7fffffffu;
    unsigned hy = (unsigned)__double2hiint(a.y) & 0x7fffffffu;
    return hx > hy ? hx : hy;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(QCS_FULL, v, o);
    return v;
}
__device__ __forceinline__ cd warp_csum(cd v) {
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    return v;
}

// Packed strict upper triangle: entry (i, j), i < j, at j(j-1)/2 + i.
__host__ __device__ __forceinline__ int tri_index(int i, int j) { return (j * (j - 1)) / 2 + i; }
__host__ __device__ __forceinline__ int tri_count(int m) { return (m * (m - 1)) / 2; }

__device__ __forceinline__ void raise_status(unsigned *status, unsigned bits) {
    if (status) atomicOr(status, bits);
}

// Bounds checks of the debug build (-DQCS_BOUNDS): QCS_IN_BOUNDS(cond, status) is cond,
// and a false cond raises QCS_ERR_BOUNDS in the status word (the caller then skips the
// access; nothing traps).  In the release build the macro is the constant true and
// the checks compile away.
#ifdef QCS_BOUNDS
__device__ __forceinline__ bool qcs_in_bounds(bool ok, unsigned *status) {
    if (!ok) raise_status(status, QCS_ERR_BOUNDS);
    return ok;
}
#define QCS_IN_BOUNDS(cond, status) qcs_in_bounds((cond), (status))
#else
#define QCS_IN_BOUNDS(cond, status) true
#endif

// Dynamic shared memory of the running launch, in bytes.
__device__ __forceinline__ uint32_t dyn_smem_bytes() {
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
