// qcs_ozaki.cuh -- error-free slicing of FP64 operands for tensor-core products.
//
// A real row x (FP64) with row scale 2^e (max |x_k| < 2^e) is written as
//     x_k = 2^e * sum_{i=1..7} a_ik 2^{-8i},   a_ik integers, |a_ik| <= 255,
// i.e. the magnitude |x_k| 2^{56-e} truncated to an integer u_k < 2^56 whose bytes
// (most significant first) are the slices, each carrying the sign of x_k.  Every
// slice is exact in BF16 (8 significant bits).  The product of two sliced rows is
//     sum_k x_k y_k = 2^{e+f} sum_{L=2..14} 2^{-8L} sum_{i+j=L} sum_k a_ik b_jk,
// and each level sum sum_{i+j=L} sum_k a_ik b_jk is an integer of magnitude below
// 7 * 32 * 255^2 < 2^24 for K = 32 terms and at most 7 products per level, so the
// tensor cores accumulate it exactly in FP32 (no rounding anywhere).  Levels
// L = 2..8 are formed; the dropped ones (L >= 9) and the slice truncation bound the
// error by about 2^-53 of sum_k |x_k||y_k| relative to the row scales, the size of
// the rounding error of an FP64 dot product of the same length (Ozaki, Ogita, Oishi
// and Rump's error-free splitting of matrix products, with integer-valued slices).
//
// The level sums are read back as FP32 integers and combined exactly on the integer
// pipe into one 64-bit fixed-point value z = sum_{L=2..7} acc_L 2^{8(7-L)} +
// floor(acc_8 / 2^8), worth z 2^{e+f-56}; |z| < 2^62.  Nothing in this file issues
// an FP64 instruction except the out-of-range branch of fixed_to_f64.
#pragma once
#include <stdint.h>

#include "qcs_common.cuh"

namespace qcs_oz {

constexpr int kSlices = 7;             // 8-bit slices per operand: 56 bits
constexpr int kLevels = kSlices;       // product levels L = 2..8 that are formed
constexpr int kRowsPer = 32;           // padded rows / contraction length of one operand (2n <= 32)
constexpr int kSliceBytes = kRowsPer * kRowsPer * 2;  // one 32 x 32 BF16 slice (K-major core matrices)
constexpr int kNoRow = -100000;        // row scale of an all-zero row

// Byte offset of element (row, k) of a 16-bit K-major operand with 32 columns and no
// swizzle: 8-row x 16-byte core matrices, K-adjacent ones 128 bytes apart (LBO),
// row-adjacent groups of 8 rows 512 bytes apart (SBO).
__host__ __device__ __forceinline__ uint32_t kmajor16(int row, int k) {
    return (uint32_t)((row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// BF16 bit pattern of a signed integer |v| <= 255 (exact): the upper half of the FP32
// bit pattern of v, formed as 1.5 * 2^23 + v minus 1.5 * 2^23 (exact for |v| < 2^22).
__device__ __forceinline__ uint32_t bf16_of_small_int(int v) {
    const float f = __int_as_float(0x4B400000 + v) - 12582912.0f;
    return __float_as_uint(f) >> 16;
}

// Two BF16 patterns in one 32-bit word (lo = first element in memory).
__device__ __forceinline__ uint32_t pack_bf16x2(int lo, int hi) {
    const float flo = __int_as_float(0x4B400000 + lo) - 12582912.0f;
    const float fhi = __int_as_float(0x4B400000 + hi) - 12582912.0f;
    return __byte_perm(__float_as_uint(flo), __float_as_uint(fhi), 0x7632);
}

// Slice i (1..7) of the fixed-point magnitude u < 2^56 with sign s (true = negative).
__device__ __forceinline__ int slice_of(uint64_t u, int i, bool s) {
    const int a = (int)((u >> (56 - 8 * i)) & 255u);
    return s ? -a : a;
}

// Exponent e with |x| < 2^e for a finite nonzero x (the binary exponent of |x| plus one),
// from the bit pattern (no FP64 instruction).  Subnormals are treated as 2^-1022.
__device__ __forceinline__ int row_exp_of(double x) {
    const int hx = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu);
    return (hx == 0 ? 1 : hx) - 1023 + 1;
}

// |x| 2^{56-e} truncated to an integer (|x| < 2^e), from the bit pattern.
__device__ __forceinline__ uint64_t fixed_of(double x, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int hx = (int)((b >> 52) & 0x7ffu);
    if (hx == 0) return 0ull;  // zeros (and subnormals, far below any row scale here)
    const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);  // |x| = m 2^{hx-1075}
    const int sh = hx - 1075 + 56 - e;                             // u = m 2^sh
    if (sh >= 0) return m << (sh < 3 ? sh : 3);  // |x| < 2^e gives sh <= 3 and m 2^sh < 2^56
    return sh <= -64 ? 0ull : m >> (-sh);
}

// Exact integer value of an FP32 that holds an integer of magnitude below 2^24 (the
// level sums are bounded by 7 * 32 * 255^2 < 2^24, so the exponent field is <= 150).
__device__ __forceinline__ long long int_of_f32(float f) {
    const uint32_t b = __float_as_uint(f);
    const int ex = (int)((b >> 23) & 0xffu);
    if (ex < 127) return 0ll;  // zero (a level sum is an integer: |f| < 1 means f = 0)
    const uint32_t m = (b & 0x7fffffu) | 0x800000u;  // |f| = m 2^{ex-150}
    const long long v = (long long)(m >> (150 - (ex < 150 ? ex : 150)));
    return (b >> 31) ? -v : v;
}

// |z| 2^sh as an unsigned fixed-point magnitude (shift left or right; the caller keeps
// the result below 2^56).
__device__ __forceinline__ uint64_t rescale_mag(long long z, int sh) {
    const uint64_t u = z < 0 ? (uint64_t)(-z) : (uint64_t)z;
    if (sh >= 0) return u << (sh < 63 ? sh : 63);
    return sh <= -64 ? 0ull : u >> (-sh);
}

// z = sum_{L=2..7} acc[L-2] 2^{8(7-L)} + floor(acc[6] / 2^8) for the seven level sums
// acc[0..6] (levels 2..8) of one output entry.
__device__ __forceinline__ long long combine_levels(const float (&acc)[kLevels]) {
    long long z = int_of_f32(acc[6]) >> 8;
#pragma unroll
    for (int L = 7; L >= 2; --L) z += int_of_f32(acc[L - 2]) * (1ll << (8 * (7 - L)));
    return z;
}

// Number of significant bits of |z| (0 for z = 0).
__device__ __forceinline__ int bitlen64(long long z) {
    const unsigned long long u = z < 0 ? (unsigned long long)(-z) : (unsigned long long)z;
    return 64 - __clzll((long long)u);
}

// z 2^E as an FP64 (round to nearest on the 11 dropped bits), assembled from the
// bits; the branch for exponents outside the normal range is never taken for the
// magnitudes of this library's matrices.
__device__ __forceinline__ double fixed_to_f64(long long z, int E) {
    if (z == 0) return 0.0;
    const unsigned long long sg = z < 0 ? (1ull << 63) : 0ull;
    const unsigned long long u = z < 0 ? (unsigned long long)(-z) : (unsigned long long)z;
    const int lz = __clzll((long long)u);
    const unsigned long long nrm = u << lz;  // top bit set
    unsigned long long mant = (nrm >> 11) + ((nrm >> 10) & 1ull);
    int ex = 63 - lz + E;
    if (mant >> 53) {
        mant >>= 1;
        ++ex;
    }
    if (ex < -1020 || ex > 1020) return ldexp((double)z, E);
    return __longlong_as_double((long long)(sg | ((unsigned long long)(ex + 1023) << 52) | (mant & ((1ull << 52) - 1))));
}

// Write the seven slices of a 32-entry row (fixed-point magnitudes u[k], signs in the
// bit mask neg) into the K-major slice slabs: slab i (1..7) starts at base + (i-1) *
// slab_stride bytes, the row is `row` of its operand.  Four 16-byte stores per slice.
__device__ __forceinline__ void store_row_slices(unsigned char *base, uint32_t slab_stride, int row,
                                                 const uint64_t (&u)[kRowsPer], uint32_t neg) {
#pragma unroll
    for (int i = 1; i <= kSlices; ++i) {
        unsigned char *slab = base + (size_t)(i - 1) * slab_stride;
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
            uint4 w;
            uint32_t *wp = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = 8 * kb + 2 * t;
                wp[t] = pack_bf16x2(slice_of(u[k], i, (neg >> k) & 1u), slice_of(u[k + 1], i, (neg >> (k + 1)) & 1u));
            }
            *reinterpret_cast<uint4 *>(slab + kmajor16(row, 8 * kb)) = w;
        }
    }
}

}  // namespace qcs_oz
