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
// The level sums are read back as FP32 integers, converted exactly (one F2I each) and
// combined exactly in integer arithmetic into one 64-bit fixed-point value z = sum_{L=2..7} acc_L 2^{8(7-L)} +
// floor(acc_8 / 2^8), worth z 2^{e+f-56}; |z| < 2^62.  Nothing in this file issues
// an FP64 instruction except fixed_to_f64_exact, the path for exponents outside the
// normal range.
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

// Sign factors of the slices of one entry: s = +-1 and -s 2^23.
struct SliceSign {
    float s, m;
};
__device__ __forceinline__ SliceSign slice_sign(bool neg) {
    return neg ? SliceSign{-1.0f, 8388608.0f} : SliceSign{1.0f, -8388608.0f};
}

// Slice i (1..7) of the fixed-point magnitude u < 2^56 with sign s, as an FP32: byte
// 7 - i of u is placed under the exponent of 2^23 (bit pattern 0x4B0000bb, the value
// 2^23 + byte) by one byte permutation, and s (2^23 + byte) - s 2^23 = s byte is exact.
// With i a compile-time constant the word and byte selection fold away.
__device__ __forceinline__ float slice_f32(uint64_t u, int i, SliceSign g) {
    const int byte = 7 - i;
    const uint32_t w = byte >= 4 ? (uint32_t)(u >> 32) : (uint32_t)u;
    const uint32_t bits = __byte_perm(w, 0x4B000000u, (uint32_t)(byte & 3) | 0x7440u);
    return fmaf(__uint_as_float(bits), g.s, g.m);
}

// Two FP32 values that BF16 holds exactly (integers of magnitude <= 255) as one BF16
// pair, lo first in memory (the lower half of the word).
__device__ __forceinline__ uint32_t bf16x2_of(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
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

// |z| 2^sh as an unsigned fixed-point magnitude (shift left or right; the caller keeps
// the result below 2^56).  Selects only, no branch.
__device__ __forceinline__ uint64_t rescale_mag(long long z, int sh) {
    const uint64_t u = z < 0 ? (uint64_t)(-z) : (uint64_t)z;
    const uint64_t l = u << (sh < 63 ? (sh > 0 ? sh : 0) : 63);
    const uint64_t r = sh <= -64 ? 0ull : u >> (sh < 0 ? -sh : 0);
    return sh >= 0 ? l : r;
}

// z = sum_{L=2..7} acc[L-2] 2^{8(7-L)} + floor(acc[6] / 2^8) for the seven level sums
// acc[0..6] (levels 2..8) of one output entry.  Each sum is an integer of magnitude
// below 2^24, so one round-to-nearest conversion gives it exactly; levels 2 and 3
// only touch the upper word ((2^8 acc_2 + acc_3) 2^32, |2^8 acc_2 + acc_3| < 2^30),
// the others enter by widening multiply-adds.
__device__ __forceinline__ long long combine_levels(const float (&acc)[kLevels]) {
    int x[kLevels];
#pragma unroll
    for (int L = 0; L < kLevels; ++L) x[L] = __float2int_rn(acc[L]);
    long long z = (long long)(x[0] * 256 + x[1]) * 4294967296ll;
    z += (long long)x[2] * 16777216ll;
    z += (long long)x[3] * 65536ll;
    z += (long long)x[4] * 256ll;
    z += (long long)x[5];
    z += (long long)(x[6] >> 8);  // arithmetic shift: the floor of acc_8 / 2^8
    return z;
}

// Number of significant bits of |z| (0 for z = 0).
__device__ __forceinline__ int bitlen64(long long z) {
    const unsigned long long u = z < 0 ? (unsigned long long)(-z) : (unsigned long long)z;
    return 64 - __clzll((long long)u);
}

// z 2^E as an FP64 (round to nearest on the 11 dropped bits), assembled from the bits
// with selects only, so that a warp converts its entries without diverging.  The
// exponent of the result must lie in the normal range; range_ok is cleared otherwise
// (zero is always in range), and the caller then takes fixed_to_f64_exact.
__device__ __forceinline__ double fixed_to_f64(long long z, int E, bool &range_ok) {
    const unsigned long long sg = z < 0 ? (1ull << 63) : 0ull;
    const unsigned long long u = z < 0 ? (unsigned long long)(-z) : (unsigned long long)z;
    const int lz = __clzll((long long)u);               // 64 for z = 0
    const unsigned long long nrm = u << (lz & 63);      // top bit set (0 for z = 0)
    // 53 significant bits, rounded on the first dropped bit.  Added to the exponent
    // field (ex + 1022), the leading bit 2^52 of mant raises it to ex + 1023; after a
    // rounding carry mant is 2^53, which gives ex + 1024 with a zero fraction: 2^(ex+1).
    const unsigned long long mant = (nrm >> 11) + ((nrm >> 10) & 1ull);
    const int ex = 63 - lz + E;
    range_ok = range_ok && (u == 0ull || (ex >= -1020 && ex <= 1020));
    const long long bits = (long long)(sg | (((unsigned long long)(ex + 1022) << 52) + mant));
    return u == 0ull ? 0.0 : __longlong_as_double(bits);
}

// The same value for any exponent (subnormal, overflow), by ldexp.
__device__ __forceinline__ double fixed_to_f64_exact(long long z, int E) { return ldexp((double)z, E); }

// Write the seven slices of a 32-entry row (fixed-point magnitudes u[k], signs in the
// bit mask neg) into the K-major slice slabs: slab i (1..7) starts at base + (i-1) *
// slab_stride bytes, the row is `row` of its operand.  Four 16-byte stores per slice.
__device__ __forceinline__ void store_row_slices(unsigned char *base, uint32_t slab_stride, int row,
                                                 const uint64_t (&u)[kRowsPer], uint32_t neg) {
    SliceSign g[kRowsPer];
#pragma unroll
    for (int k = 0; k < kRowsPer; ++k) g[k] = slice_sign((neg >> k) & 1u);
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
                wp[t] = bf16x2_of(slice_f32(u[k], i, g[k]), slice_f32(u[k + 1], i, g[k + 1]));
            }
            *reinterpret_cast<uint4 *>(slab + kmajor16(row, 8 * kb)) = w;
        }
    }
}

}  // namespace qcs_oz
