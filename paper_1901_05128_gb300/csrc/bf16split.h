// Split of an FP64 value into two BF16 values hi + lo (bf16_split) or two TF32
// values (tf32_split, returned as FP32 bit patterns whose 13 low mantissa bits
// are zero) using integer operations only: hi is x rounded to nearest-even with
// 8 (BF16) or 11 (TF32) significant bits and lo is the remainder x - hi rounded
// the same way. On GB300 the FP64 unit is ~60x slower than the integer and FP32
// pipes, so the conversion avoids it entirely. Values whose exponent would fall
// below the normal FP32 range (|x| < 2^-126) give signed zero; values above the
// range give +-Inf; NaN stays NaN. Compiles as plain C (host tests) and as CUDA
// device code.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define BF16SPLIT_FN __host__ __device__ __forceinline__
#else
#define BF16SPLIT_FN static inline
#endif

BF16SPLIT_FN int bf16split_clz64(uint64_t a) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)a);
#else
    return a ? __builtin_clzll(a) : 64;
#endif
}

// Round the magnitude a (> 0) times 2^scale to a BF16 with sign bit s.
// a has at most 63 significant bits.
BF16SPLIT_FN uint16_t bf16split_round(uint64_t a, int scale, uint32_t s) {
    const int nb = 64 - bf16split_clz64(a);            // bit length of a
    int shift = nb - 8;                                 // keep 8 significant bits
    uint64_t q;
    if (shift > 0) {
        q = a >> shift;
        const uint64_t rem = a & ((1ull << shift) - 1ull);
        const uint64_t half = 1ull << (shift - 1);
        if (rem > half || (rem == half && (q & 1ull))) ++q;
        if (q == 256ull) {                              // carried into a new bit
            q = 128ull;
            ++shift;
        }
    } else {
        q = a << (-shift);
    }
    // value = q * 2^(scale + shift), q in [128, 255]; BF16 exponent field = unbiased + 127
    const int e = scale + shift + 7 + 127;
    if (e <= 0) return (uint16_t)(s << 15);             // below the normal range
    if (e >= 255) return (uint16_t)((s << 15) | 0x7f80u);
    return (uint16_t)((s << 15) | ((uint32_t)e << 7) | (uint32_t)(q & 0x7full));
}

BF16SPLIT_FN void bf16_split(double x, uint16_t *hi, uint16_t *lo) {
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    const uint32_t s = (uint32_t)(u >> 63);
    const int ex = (int)((u >> 52) & 0x7ffull);
    const uint64_t frac = u & 0xfffffffffffffull;
    if (ex == 0x7ff) {                                  // Inf / NaN
        *hi = (uint16_t)((s << 15) | 0x7f80u | (frac ? 0x40u : 0u));
        *lo = 0;
        return;
    }
    if (ex == 0) {                                      // zero or FP64 subnormal: far below BF16 range
        *hi = (uint16_t)(s << 15);
        *lo = 0;
        return;
    }
    const uint64_t m = frac | (1ull << 52);             // x = +-m * 2^(ex - 1075)
    const int scale = ex - 1075;
    // hi: 8 significant bits of m, round to nearest even
    uint64_t q = m >> 45;
    const uint64_t rem = m & ((1ull << 45) - 1ull);
    if (rem > (1ull << 44) || (rem == (1ull << 44) && (q & 1ull))) ++q;
    const int64_t res = (int64_t)m - (int64_t)(q << 45); // x - hi in units of 2^scale, |res| <= 2^44
    *hi = bf16split_round(q << 45, scale, s);
    if (((*hi) & 0x7f80u) == 0x7f80u || ((*hi) & 0x7fffu) == 0u || res == 0) {
        *lo = 0;
        return;
    }
    const uint32_t sl = s ^ (res < 0 ? 1u : 0u);
    *lo = bf16split_round((uint64_t)(res < 0 ? -res : res), scale, sl);
}

// Round the magnitude a (> 0, at most 63 significant bits) times 2^scale to nb
// significant bits (nearest, ties to even); FP32 bit pattern with sign bit s.
BF16SPLIT_FN uint32_t split_round_f32(uint64_t a, int scale, uint32_t s, int nb) {
    const int bl = 64 - bf16split_clz64(a);
    int shift = bl - nb;
    uint64_t q;
    if (shift > 0) {
        q = a >> shift;
        const uint64_t rem = a & ((1ull << shift) - 1ull);
        const uint64_t half = 1ull << (shift - 1);
        if (rem > half || (rem == half && (q & 1ull))) ++q;
        if (q == (1ull << nb)) {                        // carried into a new bit
            q >>= 1;
            ++shift;
        }
    } else {
        q = a << (-shift);
    }
    // value = q * 2^(scale + shift), q in [2^(nb-1), 2^nb); FP32 exponent field = unbiased + 127
    const int e = scale + shift + (nb - 1) + 127;
    if (e <= 0) return s << 31;
    if (e >= 255) return (s << 31) | 0x7f800000u;
    return (s << 31) | ((uint32_t)e << 23) | ((uint32_t)(q & ((1ull << (nb - 1)) - 1ull)) << (24 - nb));
}

BF16SPLIT_FN void tf32_split(double x, uint32_t *hi, uint32_t *lo) {
    const int nb = 11;
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    const uint32_t s = (uint32_t)(u >> 63);
    const int ex = (int)((u >> 52) & 0x7ffull);
    const uint64_t frac = u & 0xfffffffffffffull;
    if (ex == 0x7ff) {                                  // Inf / NaN
        *hi = (s << 31) | 0x7f800000u | (frac ? 0x00400000u : 0u);
        *lo = 0;
        return;
    }
    if (ex == 0) {                                      // zero or FP64 subnormal: below the FP32 range
        *hi = s << 31;
        *lo = 0;
        return;
    }
    const uint64_t m = frac | (1ull << 52);             // x = +-m * 2^(ex - 1075)
    const int scale = ex - 1075;
    const int drop = 53 - nb;
    uint64_t q = m >> drop;
    const uint64_t rem = m & ((1ull << drop) - 1ull);
    if (rem > (1ull << (drop - 1)) || (rem == (1ull << (drop - 1)) && (q & 1ull))) ++q;
    const int64_t res = (int64_t)m - (int64_t)(q << drop);   // x - hi in units of 2^scale
    *hi = split_round_f32(q << drop, scale, s, nb);
    if (((*hi) & 0x7f800000u) == 0x7f800000u || ((*hi) & 0x7fffffffu) == 0u || res == 0) {
        *lo = 0;
        return;
    }
    const uint32_t sl = s ^ (res < 0 ? 1u : 0u);
    *lo = split_round_f32((uint64_t)(res < 0 ? -res : res), scale, sl, nb);
}
