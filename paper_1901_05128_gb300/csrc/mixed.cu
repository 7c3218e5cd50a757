// Mixed-precision direct solve (precision forms CQ_BF16X3 and CQ_TF32X3 of the direct scheme).
//
// The direct history h^n = sum_{k=1}^{n-1} d_{n-k} g^k (Eq. 3.8) of all modes is
// computed in time blocks of kMxB steps. For the block starting at n0 the part
// from the levels of earlier blocks, sum_{k=1}^{n0-1} d_{n-k} g^k, is one causal
// Toeplitz contraction on the tensor cores (history_tc.cu: tcgen05, split BF16 or
// TF32 operands, FP32 accumulation), with a separate weight bank per state; the rest,
// from the levels n0 .. n-1 of the block itself, is formed step by step in FP32
// by the kernel that also takes the steps (Eq. 4.1 / Eq. 4.7 in the sine basis).
// A step is evaluated from the FP32 history sums in the two-term form
// x = A l + B e with double-float A and B (lane_step2), or in FP64 when the
// coupling is strong (|a| > 10); the first SBD step uses the double-float form
// (lane_step).
//
// Every mode is pre-scaled by an exact power of two from its G^0, as in the FP32
// fast form, so its values sit near 1 in the FP32 / BF16 range; the contraction
// is linear per mode, so the scaled levels give the scaled history.
//
// Per pair of blocks: one contraction over the earlier pairs' levels for the rows
// of both blocks (two row tiles share each level tile), one short contraction of
// the first block's levels added onto the second block's rows, and one step
// launch per block, which appends the block's levels to the K-major level matrix.
#include "common.cuh"
#include "fp2s_core.cuh"
#include "tc.cuh"

namespace fastcq {

constexpr int kMxB = 128;      // steps per time block (= one tensor-core M tile)
constexpr int kMxSB = 8;       // sub-block / chunk of the in-block sums
constexpr int kMxT = 128;      // threads per CTA: 64 modes x 2 states
constexpr int kMxWOff = 7;                 // weight table: entry i holds d_{i - 7}
constexpr int kMxW = kMxB + 2 * kMxSB;     // entries per state (d_{-7} .. d_{kMxB + 8})

struct MixedLayout {
    char *a_hi[2], *a_lo[2];            // Toeplitz banks of d^1 and d^2
    char *gt_hi, *gt_lo;                // levels (BF16 or TF32 hi / lo), K-major: row s * nmp + mode, column k - 1
    float *acc2b;                       // contraction of two blocks' rows [2 kMxB][2 * nmp]
    float *acc1b;                       // contraction of one block's rows [kMxB][2 * nmp]
    float *carry;                       // g^{n-1}, g^{n-2} at the end of a block: [2][2 * nmp]
    float4 *coef;                       // per lane: A row, B row (double-float), (scaled g^0, exponent)
    int kind, nblk, ntiles;
    int64_t nmp, kpad;
    size_t bytes;
};

static MixedLayout mixed_layout(const Fp2sParams &P, void *base) {
    MixedLayout l{};
    l.kind = P.prec == CQ_TF32X3 ? tc::TC_TF32X3 : tc::TC_BF16X3;
    const int bk = tc::kind_bk(l.kind), es = tc::kind_esize(l.kind);
    l.nmp = (P.nmodes + 3) / 4 * 4;
    l.nblk = (int)((P.N + kMxB - 1) / kMxB);
    const int64_t klev = (int64_t)(l.nblk - 1) * kMxB;          // levels ever contracted
    l.kpad = klev > 0 ? klev : 64;
    l.ntiles = klev > 0 ? (int)(klev / bk) : 1;
    Carve cv(base);
    const size_t bank = (size_t)l.ntiles * tc::BM * bk * es;
    for (int s = 0; s < 2; ++s) {
        l.a_hi[s] = cv.take<char>(bank);
        l.a_lo[s] = cv.take<char>(bank);
    }
    const size_t lev = l.nblk > 1 ? (size_t)2 * l.nmp * l.kpad : 0;
    l.gt_hi = cv.take<char>(lev * es);
    l.gt_lo = cv.take<char>(lev * es);
    l.acc2b = cv.take<float>(l.nblk > 2 ? (size_t)2 * kMxB * 2 * l.nmp : 0);
    l.acc1b = cv.take<float>(l.nblk > 1 ? (size_t)kMxB * 2 * l.nmp : 0);
    l.carry = cv.take<float>((size_t)4 * l.nmp);
    l.coef = cv.take<float4>((size_t)6 * l.nmp);
    l.bytes = cv.bytes();
    return l;
}

size_t mixed_direct_bytes(const Fp2sParams &P) { return mixed_layout(P, nullptr).bytes; }

struct MixedArgs {
    Fp2sParams P;
    int64_t nmp, n0, kpad;
    int solve64, write_levels, kind;
    const double *lam, *g0, *d1, *d2;
    const float *hdf, *acc;             // contraction rows of this block (absent for the first block)
    float *carry;
    float4 *coef;
    char *gt_hi, *gt_lo;
    double *gN;
    int *status;
};

// BF16 hi + lo of an FP32 value: hi = bf16(x), lo = bf16(x - hi) (x - hi is exact in FP32).
__device__ __forceinline__ void split_f32(float x, uint32_t &h, uint32_t &l) {
    const __nv_bfloat16 hb = __float2bfloat16_rn(x);
    const __nv_bfloat16 lb = __float2bfloat16_rn(x - __bfloat162float(hb));
    h = __bfloat16_as_ushort(hb);
    l = __bfloat16_as_ushort(lb);
}

// x (finite) rounded to 11 significant bits, nearest-even: the TF32 value in FP32 bits.
__device__ __forceinline__ uint32_t rn_tf32_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0xfffu + ((u >> 13) & 1u)) & 0xffffe000u;
}

// TF32 hi + lo of an FP32 value (x - hi is exact in FP32).
__device__ __forceinline__ void split_f32_tf32(float x, uint32_t &h, uint32_t &l) {
    h = rn_tf32_bits(x);
    l = rn_tf32_bits(x - __uint_as_float(h));
}

// Steps n0 .. min(n0 + kMxB - 1, N) of 64 modes per CTA. Lanes l < 16 of a warp
// carry state 1 and lanes l + 16 state 2 of the same 16 modes. acc (absent for the
// first block) holds the contribution of the earlier blocks' levels. The block's
// levels stay in shared memory for the in-block sums, four consecutive levels of a
// thread in one 16-byte word (a warp's 16-byte loads cover 512 contiguous bytes).
// Sub-blocks of kMxSB steps first take the earlier in-block levels in 8 x 8
// Toeplitz chunks (15 weights and 8 levels, six 16-byte loads, feed 64 FMAs),
// then their own triangle step by step.
__global__ void __launch_bounds__(kMxT) k_mixed_block(const __grid_constant__ MixedArgs A) {
    extern __shared__ __align__(16) float smx[];
    // levels of the block: level n0 + j of thread t at xs[((j / 4) * kMxT + t) * 4 + j % 4]
    float *xs = smx;
    float *wsm = smx + kMxB * kMxT;           // [2][kMxW]: entry i = d_{i - kMxWOff} of each state
    const Fp2sParams &P = A.P;
    const int tid = threadIdx.x, lane = tid & 31, st = lane >> 4;
    for (int i = tid; i < 2 * kMxW; i += kMxT) {
        const int s = i / kMxW, ii = i % kMxW - kMxWOff;
        wsm[i] = (ii >= 0 && ii <= P.N) ? (float)(s ? A.d2 : A.d1)[ii] : 0.0f;
    }
    __syncthreads();

    const int64_t mode_raw = ((int64_t)blockIdx.x * (kMxT >> 5) + (tid >> 5)) * kFastModesPerWarp + (lane & 15);
    const bool active = mode_raw < P.nmodes;
    const int64_t mode = active ? mode_raw : 0;
    const int64_t col = st * A.nmp + mode;

    // per-lane step coefficients: formed in FP64 by the first block (and by every block
    // when the FP64 step is in use), read back from the table by the others
    LaneStep ls;
    LaneStep2 l2;
    float gz;
    int ex = 0;
    const bool full_setup = A.n0 == 1 || A.solve64;
    if (full_setup) {
        const double gz64 = A.g0[st * P.nmodes + mode];
        const double gmax = fmax(fabs(gz64), fabs(__shfl_xor_sync(0xffffffffu, gz64, 16)));
        if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &ex);
        gz = (float)ldexp(gz64, -ex);
        const bool ok = lane_step_setup(P, A.lam[mode], A.d1[0], A.d2[0], st, ls);
        if (A.n0 == 1 && active && st == 0 && !ok) atomicOr(A.status, ST_SINGULAR);
        lane_step2_setup(P, ls, l2);
        if (A.n0 == 1 && active) {
            A.coef[col] = make_float4(l2.a_hi[0], l2.a_hi[1], l2.a_lo[0], l2.a_lo[1]);
            A.coef[2 * A.nmp + col] = make_float4(l2.b_hi[0], l2.b_hi[1], l2.b_lo[0], l2.b_lo[1]);
            A.coef[4 * A.nmp + col] = make_float4(gz, __int_as_float(ex), 0.0f, 0.0f);
        }
    } else {
        const float4 c0 = A.coef[col], c1 = A.coef[2 * A.nmp + col], c2 = A.coef[4 * A.nmp + col];
        l2.a_hi[0] = c0.x;
        l2.a_hi[1] = c0.y;
        l2.a_lo[0] = c0.z;
        l2.a_lo[1] = c0.w;
        l2.b_hi[0] = c1.x;
        l2.b_hi[1] = c1.y;
        l2.b_lo[0] = c1.z;
        l2.b_lo[1] = c1.w;
        gz = c2.x;
        ex = __float_as_int(c2.y);
    }
    const double *dn = st ? A.d2 : A.d1;
    const float *hd_hi = A.hdf + (size_t)(2 * st) * (P.N + 1), *hd_lo = hd_hi + (P.N + 1);

    float gm1 = gz, gm2 = 0.0f;
    if (A.n0 > 1) {
        gm1 = A.carry[col];
        gm2 = A.carry[2 * A.nmp + col];
    }
    float gm1_o = __shfl_xor_sync(0xffffffffu, gm1, 16), gm2_o = __shfl_xor_sync(0xffffffffu, gm2, 16);
    const float *w = wsm + st * kMxW + kMxWOff;     // w[i] = d_i, i >= -kMxWOff
    float wt[kMxSB];                                 // d_1 .. d_7 of the lane's state
#pragma unroll
    for (int i = 1; i < kMxSB; ++i) wt[i] = w[i];
    float *xc = xs + 4 * tid;
    const float4 *xs4 = reinterpret_cast<const float4 *>(xs) + tid;
    const int64_t ldacc = 2 * A.nmp;
    const int jmax = (int)min((int64_t)kMxB, P.N - A.n0 + 1);      // steps in this block
    float an[kMxSB];                                 // acc rows of the next sub-block (prefetched)
#pragma unroll
    for (int b = 0; b < kMxSB; ++b) an[b] = A.acc ? A.acc[(int64_t)b * ldacc + col] : 0.0f;
    for (int j0 = 0; j0 < jmax; j0 += kMxSB) {
        float a[kMxSB];
#pragma unroll
        for (int b = 0; b < kMxSB; ++b) a[b] = an[b];
        if (A.acc && j0 + kMxSB < jmax) {
#pragma unroll
            for (int b = 0; b < kMxSB; ++b) an[b] = A.acc[(int64_t)(j0 + kMxSB + b) * ldacc + col];
        }
        // earlier in-block levels k in chunks of 8: a[b] += sum_kk d_{j0 + b - kc - kk} x^{n0 + kc + kk};
        // the 15 weights of a chunk are d_{m-7} .. d_{m+7}, m = j0 - kc (four 16-byte loads)
        for (int kc = 0; kc < j0; kc += kMxSB) {
            const float4 *wp = reinterpret_cast<const float4 *>(w + (j0 - kc) - kMxWOff);
            float W[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = wp[q];
                W[4 * q] = v.x;
                W[4 * q + 1] = v.y;
                W[4 * q + 2] = v.z;
                W[4 * q + 3] = v.w;
            }
            const float4 x0 = xs4[(kc / 4) * kMxT], x1 = xs4[(kc / 4 + 1) * kMxT];
            const float X[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int kk = 0; kk < kMxSB; ++kk)
#pragma unroll
                for (int b = 0; b < kMxSB; ++b) a[b] = fmaf(W[b - kk + kMxWOff], X[kk], a[b]);
        }
        // the sub-block's own triangle: each new level is added forward into the later sums
#pragma unroll
        for (int b = 0; b < kMxSB; ++b) {
            const int64_t n = A.n0 + j0 + b;
            if (j0 + b >= jmax) break;
            const float h = a[b];
            float x;
            if (full_setup && (A.solve64 || (P.scheme == CQ_BDF2 && n == 1))) {
                x = lane_step(P, ls, A.solve64, n, h, gm1, gm2, gz, dn, hd_hi, hd_lo);
            } else if (P.scheme == CQ_BE) {
                x = lane_step2(l2, gm1, 0.0f, gm1_o, 0.0f, h, 0.0f, __shfl_xor_sync(0xffffffffu, h, 16), 0.0f);
            } else {
                const df l = two_sum(2.0f * gm1, -0.5f * gm2), lo = two_sum(2.0f * gm1_o, -0.5f * gm2_o);
                // e = h + d_{n-1} g^0 / 2 as a double-float pair
                const df e = df_add(df_mul_f(df{__ldg(hd_hi + n - 1), __ldg(hd_lo + n - 1)}, gz), df{h, 0.0f});
                x = lane_step2(l2, l.hi, l.lo, lo.hi, lo.lo, e.hi, e.lo, __shfl_xor_sync(0xffffffffu, e.hi, 16),
                               __shfl_xor_sync(0xffffffffu, e.lo, 16));
            }
#pragma unroll
            for (int bb = b + 1; bb < kMxSB; ++bb) a[bb] = fmaf(wt[bb - b], x, a[bb]);
            const float x_o = __shfl_xor_sync(0xffffffffu, x, 16);
            xc[((j0 + b) / 4) * 4 * kMxT + (j0 + b) % 4] = x;
            gm2 = gm1;
            gm1 = x;
            gm2_o = gm1_o;
            gm1_o = x_o;
        }
    }
    if (!active) return;
    if (A.write_levels) {
        // level n0 + j goes to column n0 + j - 1 of row col, as 16-byte stores per array
        const int64_t o = col * A.kpad + (A.n0 - 1);
        if (A.kind == tc::TC_TF32X3) {
            uint4 *dh = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(A.gt_hi) + o);
            uint4 *dl = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(A.gt_lo) + o);
            for (int j = 0; j < kMxB; j += 4) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) split_f32_tf32(xc[(j / 4) * 4 * kMxT + i], h[i], l[i]);
                dh[j / 4] = make_uint4(h[0], h[1], h[2], h[3]);
                dl[j / 4] = make_uint4(l[0], l[1], l[2], l[3]);
            }
        } else {
            uint4 *dh = reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(A.gt_hi) + o);
            uint4 *dl = reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(A.gt_lo) + o);
            for (int j = 0; j < kMxB; j += 8) {
                uint32_t h[8], l[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) split_f32(xc[((j + i) / 4) * 4 * kMxT + (j + i) % 4], h[i], l[i]);
                dh[j / 8] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16),
                                       h[6] | (h[7] << 16));
                dl[j / 8] = make_uint4(l[0] | (l[1] << 16), l[2] | (l[3] << 16), l[4] | (l[5] << 16),
                                       l[6] | (l[7] << 16));
            }
        }
        A.carry[col] = gm1;
        A.carry[2 * A.nmp + col] = gm2;
    } else {
        const double out = ldexp((double)gm1, ex);
        A.gN[st * P.nmodes + mode] = out;
        if (!isfinite(out)) atomicOr(A.status, ST_NONFINITE);
    }
}

constexpr size_t kMxSmem = ((size_t)kMxB * kMxT + 2 * kMxW) * sizeof(float);

int mixed_direct_run(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                     const double *d1, const double *d2, const float *hdf, void *region, cudaStream_t s) {
    const MixedLayout l = mixed_layout(P, region);
    int st;
    tc::TcMaps maps;
    if (l.nblk > 1) {
        const double *d[2] = {d1, d2};
        for (int q = 0; q < 2; ++q) {
            if ((st = tc_bank(l.kind, d[q], P.N, tc::kind_bk(l.kind), l.ntiles, l.a_hi[q], l.a_lo[q], s))) return st;
            if ((st = tc_map_bank(l.kind, &maps.a_hi[q], l.a_hi[q], l.ntiles))) return st;
            if ((st = tc_map_bank(l.kind, &maps.a_lo[q], l.a_lo[q], l.ntiles))) return st;
        }
        if ((st = tc_map_levels(l.kind, &maps.b_hi, l.gt_hi, l.kpad, 2 * l.nmp))) return st;
        if ((st = tc_map_levels(l.kind, &maps.b_lo, l.gt_lo, l.kpad, 2 * l.nmp))) return st;
    }
    static unsigned long long attr = 0;
    if ((st = smem_attr_once((const void *)k_mixed_block, (int)kMxSmem, &attr))) return st;
    MixedArgs A;
    A.P = P;
    A.nmp = l.nmp;
    A.kpad = l.kpad;
    A.solve64 = fabs(P.a) > 10.0;
    A.kind = l.kind;
    A.lam = lam;
    A.g0 = g0;
    A.d1 = d1;
    A.d2 = d2;
    A.hdf = hdf;
    A.carry = l.carry;
    A.coef = l.coef;
    A.gt_hi = l.gt_hi;
    A.gt_lo = l.gt_lo;
    A.gN = gN;
    A.status = status;
    const int64_t mpb = (kMxT / 32) * kFastModesPerWarp;
    const unsigned grid = (unsigned)((P.nmodes + mpb - 1) / mpb);
    tc::TcParams T{};
    T.ndof = P.nmodes;
    T.ldh = 2 * l.nmp;
    T.vec2 = 1;                         // ldh and the state offset are multiples of 4 floats
    T.num_i = 1;
    T.delta0 = tc::kind_bk(l.kind);
    T.n_states = 2;
    T.ntile_state = (P.nmodes + tc::BN - 1) / tc::BN;
    T.state_stride = l.nmp;
    // Blocks in pairs (2p, 2p+1). Once both earlier pairs' levels exist, one contraction
    // covers the rows of both blocks over the levels of blocks < 2p (two row tiles per
    // column tile: the level matrix is streamed once for 256 rows); block 2p+1 then adds
    // the levels of block 2p with a short contraction (K = 128) added onto its rows.
    auto contract = [&](int64_t n_lo, int64_t rows, int64_t k_lo, int64_t k_hi, float *out, int add) -> int {
        T.n_lo = n_lo;
        T.add = add;
        T.rows = rows;
        T.num_i = (int)((rows + kMxB - 1) / kMxB);
        T.k_lo = (int)k_lo;
        T.kprime = (int)k_hi;
        int r;
        if ((r = timing_part(s, false))) return r;
        if ((r = tc_contract_f32(l.kind, maps, T, out, status, s))) return r;
        return timing_part(s, true);
    };
    for (int b = 0; b < l.nblk; ++b) {
        const int64_t n0 = 1 + (int64_t)b * kMxB;
        const int64_t left = P.N - n0 + 1;                 // steps from n0 to N
        A.acc = nullptr;
        if (b % 2 == 0) {
            if (b >= 2) {
                if ((st = contract(n0, min((int64_t)2 * kMxB, left), 0, n0 - 1, l.acc2b, 0))) return st;
                A.acc = l.acc2b;
            }
        } else {
            // block 2p+1: its rows of the pair's contraction (rows 128..255), or a fresh buffer
            float *rows = b >= 3 ? l.acc2b + (size_t)kMxB * 2 * l.nmp : l.acc1b;
            if ((st = contract(n0, min((int64_t)kMxB, left), n0 - 1 - kMxB, n0 - 1, rows, b >= 3))) return st;
            A.acc = rows;
        }
        A.n0 = n0;
        A.write_levels = b + 1 < l.nblk;
        k_mixed_block<<<grid, kMxT, kMxSmem, s>>>(A);
        if ((st = launched())) return st;
    }
    return CQ_OK;
}

}  // namespace fastcq
