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

BF16SPLIT_FN int bf16split_clz32(uint32_t a) {
#if defined(__CUDA_ARCH__)
    return __clz((int)a);
#else
    return a ? __builtin_clz(a) : 32;
#endif
}

// BF16 bits with sign s of the value q * 2^(e - 127 - 7), q in [128, 256] (256 carries into the
// exponent); zero below the normal range, Inf above it.
BF16SPLIT_FN uint16_t bf16split_pack(uint32_t q, int e, uint32_t s) {
    if (q == 256u) {
        q = 128u;
        ++e;
    }
    if (e <= 0) return (uint16_t)(s << 15);
    if (e >= 255) return (uint16_t)((s << 15) | 0x7f80u);
    return (uint16_t)((s << 15) | ((uint32_t)e << 7) | (q & 0x7fu));
}

// The split with 32-bit integer operations only (64-bit integer operations cost several
// instructions each on the GPU). With x = +-m 2^(ex - 1075), m = 2^52 + f:
//   hi = m rounded to its 8 leading bits (nearest, ties to even);
//   res = m - hi (|res| <= 2^44) held as a 45-bit magnitude (mh:ml) and a sign;
//   lo = res rounded to 8 leading bits: normalise (mh:ml) so its leading bit is bit 63, keep
//        the top 8 bits and round on the 56 below.
BF16SPLIT_FN void bf16_split(double x, uint16_t *hi, uint16_t *lo) {
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    const uint32_t hw = (uint32_t)(u >> 32), lw = (uint32_t)u;
    const uint32_t s = hw >> 31;
    const int ex = (int)((hw >> 20) & 0x7ffu);
    const uint32_t fh = hw & 0xfffffu;                  // fraction bits 51..32
    if (ex == 0x7ff) {                                  // Inf / NaN
        *hi = (uint16_t)((s << 15) | 0x7f80u | ((fh | lw) ? 0x40u : 0u));
        *lo = 0;
        return;
    }
    if (ex == 0) {                                      // zero or FP64 subnormal: far below BF16 range
        *hi = (uint16_t)(s << 15);
        *lo = 0;
        return;
    }
    const uint32_t q = 0x80u | (fh >> 13);              // m >> 45: the 8 leading bits
    const uint32_t rh = fh & 0x1fffu;                   // m mod 2^45 = rh * 2^32 + lw
    const uint32_t up = ((rh & 0x1000u) && (((rh & 0xfffu) | lw) != 0u || (q & 1u))) ? 1u : 0u;
    *hi = bf16split_pack(q + up, ex - 896, s);
    uint32_t mh, ml, sl = s;
    if (up) {                                           // res = (m mod 2^45) - 2^45 < 0
        ml = 0u - lw;
        mh = 0x2000u - rh - (lw != 0u ? 1u : 0u);
        sl ^= 1u;
    } else {
        ml = lw;
        mh = rh;
    }
    if (((*hi) & 0x7f80u) == 0x7f80u || ((*hi) & 0x7fffu) == 0u || (mh | ml) == 0u) {
        *lo = 0;
        return;
    }
    const int c = mh ? bf16split_clz32(mh) : 32 + bf16split_clz32(ml);   // leading zeros of mh:ml
    uint32_t top, bot;                                  // (mh:ml) << c
    if (c >= 32) {
        top = ml << (c - 32);
        bot = 0u;
    } else if (c > 0) {
        top = (mh << c) | (ml >> (32 - c));
        bot = ml << c;
    } else {
        top = mh;
        bot = ml;
    }
    const uint32_t q8 = top >> 24;
    const uint32_t up8 = ((top & 0x800000u) && (((top & 0x7fffffu) | bot) != 0u || (q8 & 1u))) ? 1u : 0u;
    *lo = bf16split_pack(q8 + up8, ex - 885 - c, sl);
}

// FP32 bits with sign s of the value q * 2^(e - 127 - 10), q in [1024, 2048] (2048 carries into
// the exponent): a TF32 value (13 low mantissa bits zero); zero below the normal range, Inf above.
BF16SPLIT_FN uint32_t tf32split_pack(uint32_t q, int e, uint32_t s) {
    if (q == 2048u) {
        q = 1024u;
        ++e;
    }
    if (e <= 0) return s << 31;
    if (e >= 255) return (s << 31) | 0x7f800000u;
    return (s << 31) | ((uint32_t)e << 23) | ((q & 0x3ffu) << 13);
}

// The TF32 split (11 significant bits) with 32-bit integer operations, as bf16_split.
BF16SPLIT_FN void tf32_split(double x, uint32_t *hi, uint32_t *lo) {
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    const uint32_t hw = (uint32_t)(u >> 32), lw = (uint32_t)u;
    const uint32_t s = hw >> 31;
    const int ex = (int)((hw >> 20) & 0x7ffu);
    const uint32_t fh = hw & 0xfffffu;
    if (ex == 0x7ff) {                                  // Inf / NaN
        *hi = (s << 31) | 0x7f800000u | ((fh | lw) ? 0x00400000u : 0u);
        *lo = 0;
        return;
    }
    if (ex == 0) {                                      // zero or FP64 subnormal: below the FP32 range
        *hi = s << 31;
        *lo = 0;
        return;
    }
    const uint32_t q = 0x400u | (fh >> 10);             // m >> 42: the 11 leading bits
    const uint32_t rh = fh & 0x3ffu;                    // m mod 2^42 = rh * 2^32 + lw
    const uint32_t up = ((rh & 0x200u) && (((rh & 0x1ffu) | lw) != 0u || (q & 1u))) ? 1u : 0u;
    *hi = tf32split_pack(q + up, ex - 896, s);
    uint32_t mh, ml, sl = s;
    if (up) {                                           // res = (m mod 2^42) - 2^42 < 0
        ml = 0u - lw;
        mh = 0x400u - rh - (lw != 0u ? 1u : 0u);
        sl ^= 1u;
    } else {
        ml = lw;
        mh = rh;
    }
    if (((*hi) & 0x7f800000u) == 0x7f800000u || ((*hi) & 0x7fffffffu) == 0u || (mh | ml) == 0u) {
        *lo = 0;
        return;
    }
    const int c = mh ? bf16split_clz32(mh) : 32 + bf16split_clz32(ml);
    uint32_t top, bot;
    if (c >= 32) {
        top = ml << (c - 32);
        bot = 0u;
    } else if (c > 0) {
        top = (mh << c) | (ml >> (32 - c));
        bot = ml << c;
    } else {
        top = mh;
        bot = ml;
    }
    const uint32_t q11 = top >> 21;
    const uint32_t up11 = ((top & 0x100000u) && (((top & 0xfffffu) | bot) != 0u || (q11 & 1u))) ? 1u : 0u;
    *lo = tf32split_pack(q11 + up11, ex - 885 - c, sl);
}
