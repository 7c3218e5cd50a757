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
//
// The gradient (discrete adjoint of the direct scheme) runs on the same machinery.
// The forward solve keeps every level and, in a second level matrix, the increments
// delta^j = x^j - x^{j-1}. The part of dJ/dbeta that pairs with mu^n is
//   hp^n = sum_{k=1}^{n} d'_{n-k} x^k = D'_{n-1} x^0 + sum_{j=1}^{n} D'_{n-j} delta^j,
// d' = d(d_i)/d(beta), D'_i = sum_{l<=i} d'_l. The d'_i sum to about zero (the generating
// function vanishes at zeta = 1), so the left form cancels down to a small fraction of
// its terms, while the D'_i decay and the right form does not cancel: it is the one
// contracted (one full contraction with the weights e_i = D'_{i-1}). The adjoint then
// runs in reversed time (step r = N - m + 1) through the same block / pair structure
// with the transposed 2x2 steps, its levels being mu^m = K lambda^m.
#include "common.cuh"
#include "fp2s_core.cuh"
#include "tc.cuh"
#include "bf16split.h"

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
    float *carry;                       // g^{n-1}, g^{n-2} at the end of a block: [4][2 * nmp] (FP32 parts,
                                        // then the forward solve's double-float remainders)
    float4 *coef;                       // per lane: A row, B row (double-float), (scaled g^0, exponent)
    float *wrem;                        // [2][5]: WeightRem of each state (k_weight_rem)
    // gradient only
    float4 *coef_adj;                   // per lane coefficients of the adjoint steps (as coef)
    float *ht;                          // [N][2 * nmp]: row n - 1 = sum_{j=1}^{n} D'_{n-j} delta^j (scaled levels)
    double *lacc;                       // [3][2 * nmp]: per-lane sums over m of mu^m ht^m, d_{m-1} mu^m, d'_{m-1} mu^m
    float *lbuf;                        // [3][2 * nmp]: lambda^1, mu^1, lambda^2 (scaled)
    float *x1;                          // [2 * nmp]: x^1 (scaled)
    double *rT;                         // [2][nmodes]: dJ/dx^N, the adjoint's terminal condition
    char *dt_hi, *dt_lo;                // increments delta^k of the forward levels, as gt_hi / gt_lo
    double *e[2];                       // [N + 2]: e_0 = 0, e_i = D'_{i-1}
    float *dqf;                         // [2][N + 1]: d' in FP32
    float *cqf;                         // [2][N + 1]: D' in FP32
    char *q_hi[2], *q_lo[2];            // Toeplitz banks of e
    int *tcount;                        // tile counter of the weight-derivative contraction
    int kind, nblk, ntiles, qntiles;
    int64_t nmp, kpad, qdelta0;
    size_t bytes;
};

static MixedLayout mixed_layout(const Fp2sParams &P, void *base, bool grad) {
    MixedLayout l{};
    l.kind = P.prec == CQ_TF32X3 ? tc::TC_TF32X3 : tc::TC_BF16X3;
    const int bk = tc::kind_bk(l.kind), es = tc::kind_esize(l.kind);
    l.nmp = (P.nmodes + 3) / 4 * 4;
    l.nblk = (int)((P.N + kMxB - 1) / kMxB);
    const int64_t klev = (int64_t)(l.nblk - 1) * kMxB;          // levels ever contracted by a solve
    // the gradient keeps every level (N of them) for the weight-derivative contraction
    l.kpad = grad ? (int64_t)l.nblk * kMxB : (klev > 0 ? klev : 64);
    l.ntiles = klev > 0 ? (int)(klev / bk) : 1;
    Carve cv(base);
    const size_t bank = (size_t)l.ntiles * tc::BM * bk * es;
    for (int s = 0; s < 2; ++s) {
        l.a_hi[s] = cv.take<char>(bank);
        l.a_lo[s] = cv.take<char>(bank);
    }
    const size_t lev = (l.nblk > 1 || grad) ? (size_t)2 * l.nmp * l.kpad : 0;
    l.gt_hi = cv.take<char>(lev * es);
    l.gt_lo = cv.take<char>(lev * es);
    l.acc2b = cv.take<float>(l.nblk > 2 ? (size_t)2 * kMxB * 2 * l.nmp : 0);
    l.acc1b = cv.take<float>(l.nblk > 1 ? (size_t)kMxB * 2 * l.nmp : 0);
    l.carry = cv.take<float>((size_t)8 * l.nmp);
    l.coef = cv.take<float4>((size_t)6 * l.nmp);
    l.wrem = cv.take<float>(16);
    if (grad) {
        l.coef_adj = cv.take<float4>((size_t)6 * l.nmp);
        l.ht = cv.take<float>((size_t)P.N * 2 * l.nmp);
        l.lacc = cv.take<double>((size_t)3 * 2 * l.nmp);
        l.lbuf = cv.take<float>((size_t)3 * 2 * l.nmp);
        l.x1 = cv.take<float>((size_t)2 * l.nmp);
        l.rT = cv.take<double>((size_t)2 * P.nmodes);
        l.dt_hi = cv.take<char>(lev * es);
        l.dt_lo = cv.take<char>(lev * es);
        for (int s = 0; s < 2; ++s) l.e[s] = cv.take<double>(P.N + 2);
        l.dqf = cv.take<float>((size_t)2 * (P.N + 1));
        l.cqf = cv.take<float>((size_t)2 * (P.N + 1));
        // rows n' = n + 1 = 2 .. N + 1 over levels 1 .. N: delta = m0 - 1 - kc runs from
        // 1 - kpad (first row tile, last level tile) up to the last row tile's 1 + BM (num_i - 1)
        const int64_t num_i = (P.N + tc::BM - 1) / tc::BM;
        l.qdelta0 = 1 - l.kpad;
        l.qntiles = (int)((1 + tc::BM * (num_i - 1) - l.qdelta0) / bk + 1);
        const size_t qbank = (size_t)l.qntiles * tc::BM * bk * es;
        for (int s = 0; s < 2; ++s) {
            l.q_hi[s] = cv.take<char>(qbank);
            l.q_lo[s] = cv.take<char>(qbank);
        }
        l.tcount = cv.take<int>(1);
    }
    l.bytes = cv.bytes();
    return l;
}

size_t mixed_direct_bytes(const Fp2sParams &P) { return mixed_layout(P, nullptr, false).bytes; }
size_t mixed_grad_bytes(const Fp2sParams &P) { return mixed_layout(P, nullptr, true).bytes; }

struct MixedArgs {
    Fp2sParams P;
    int64_t nmp, n0, kpad;
    int solve64, write_levels, kind;
    const double *lam, *g0, *d1, *d2;   // g0: G^0 (forward) or dJ/dx^N (adjoint), modal
    const float *hdf, *acc;             // contraction rows of this block (absent for the first block)
    float *carry;
    float4 *coef;
    const float *wrem;                  // [2][5] weight remainders (k_weight_rem)
    char *gt_hi, *gt_lo;
    double *gN;
    int *status;
    // gradient: forward extras (x1, increments) and the adjoint's inputs and sums
    float *x1;
    char *dt_hi, *dt_lo;
    const float *ht, *dqf, *cqf;
    const float4 *coef_fwd;
    double *lacc;
    float *lbuf;
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

// Per-lane coefficient table: row A, row B of the two-term step (double-float), the
// lane's scaled initial value and the mode's power-of-two exponent.
__device__ __forceinline__ void coef_store(float4 *coef, int64_t nmp, int64_t col, const LaneStep2 &l2, float z,
                                           int ex) {
    coef[col] = make_float4(l2.a_hi[0], l2.a_hi[1], l2.a_lo[0], l2.a_lo[1]);
    coef[2 * nmp + col] = make_float4(l2.b_hi[0], l2.b_hi[1], l2.b_lo[0], l2.b_lo[1]);
    coef[4 * nmp + col] = make_float4(z, __int_as_float(ex), 0.0f, 0.0f);
}

__device__ __forceinline__ void coef_load(const float4 *coef, int64_t nmp, int64_t col, LaneStep2 &l2, float &z,
                                          int &ex) {
    const float4 c0 = coef[col], c1 = coef[2 * nmp + col], c2 = coef[4 * nmp + col];
    l2.a_hi[0] = c0.x;
    l2.a_hi[1] = c0.y;
    l2.a_lo[0] = c0.z;
    l2.a_lo[1] = c0.w;
    l2.b_hi[0] = c1.x;
    l2.b_hi[1] = c1.y;
    l2.b_lo[0] = c1.z;
    l2.b_lo[1] = c1.w;
    z = c2.x;
    ex = __float_as_int(c2.y);
}

// FP32 remainders of the two largest history weights of a state, d_1 and d_2, for the
// forward step. A weight rounded to FP32 is a fixed relative error that every step
// repeats: d_1 ~ beta tau^-beta, and its rounding alone put ~5e-5 into the 2D 511x511,
// N = 8192 solve. The in-block sums use fl(d_i) (remainder rf), the contraction rows the
// tensor-core operands hi + lo of the kind's split (remainder rb).
struct WeightRem {
    float w1, r1f, r2f, r1b, r2b;
};

__device__ __forceinline__ float split_sum(int kind, double x) {
    if (kind == tc::TC_TF32X3) {
        uint32_t h, l;
        tf32_split(x, &h, &l);
        return __uint_as_float(h) + __uint_as_float(l);
    }
    uint16_t h, l;
    bf16_split(x, &h, &l);
    return __uint_as_float((uint32_t)h << 16) + __uint_as_float((uint32_t)l << 16);
}

// Held in registers through the step loops: otherwise the compiler may recompute the
// remainders from their FP64 sources inside the loop (FP64 work at 1/64 of the FP32 rate).
__device__ __forceinline__ void keep_reg(WeightRem &r) {
    keep_reg(r.w1);
    keep_reg(r.r1f);
    keep_reg(r.r2f);
    keep_reg(r.r1b);
    keep_reg(r.r2b);
}

__device__ __forceinline__ WeightRem weight_rem(int kind, const double *d, int64_t N) {
    const double d1 = N >= 1 ? d[1] : 0.0, d2 = N >= 2 ? d[2] : 0.0;
    WeightRem r;
    r.w1 = (float)d1;
    r.r1f = (float)(d1 - (double)(float)d1);
    r.r2f = (float)(d2 - (double)(float)d2);
    r.r1b = (float)(d1 - (double)split_sum(kind, d1));
    r.r2b = (float)(d2 - (double)split_sum(kind, d2));
    return r;
}

// WeightRem of both states, once per run: wrem[5 s + (w1, r1f, r2f, r1b, r2b)].
__global__ void k_weight_rem(int kind, const double *__restrict__ d1, const double *__restrict__ d2, int64_t N,
                             float *__restrict__ wrem) {
    const int s = threadIdx.x;
    if (s > 1) return;
    const WeightRem r = weight_rem(kind, s ? d2 : d1, N);
    float *o = wrem + 5 * s;
    o[0] = r.w1;
    o[1] = r.r1f;
    o[2] = r.r2f;
    o[3] = r.r1b;
    o[4] = r.r2b;
}

__device__ __forceinline__ WeightRem load_weight_rem(const float *wrem, int s) {
    const float *o = wrem + 5 * s;
    return WeightRem{o[0], o[1], o[2], o[3], o[4]};
}

// The remainder terms of step n (block offset j) of one state: the weight remainders of
// d_1 x^{n-1} and d_2 x^{n-2} (lag i comes from the block's own levels when j >= i, else from
// the contraction) and d_1 times the double-float remainder of x^{n-1}. G^0 is not part of
// the history.
__device__ __forceinline__ float weight_rem_terms(const WeightRem &r, int j, int64_t n, float gm1, float gm1_lo,
                                                  float gm2) {
    float e = 0.0f;
    if (n >= 2) e = fmaf(j >= 1 ? r.r1f : r.r1b, gm1, r.w1 * gm1_lo);
    if (n >= 3) e = fmaf(j >= 2 ? r.r2f : r.r2b, gm2, e);
    return e;
}

// Earlier in-block levels in chunks of 8: a[b] += sum_kk d_{j0 + b - kc - kk} x^{n0 + kc + kk}
// for kc < j0; the 15 weights of a chunk are d_{m-7} .. d_{m+7}, m = j0 - kc (four 16-byte
// loads), the 8 levels two 16-byte loads.
__device__ __forceinline__ void inblock_chunks(float (&a)[kMxSB], const float *w, const float4 *xs4, int j0) {
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
}

// The block's levels of one lane (xc: level j at xc[(j / 4) * 4 * kMxT + j % 4]) as split
// operands, row-contiguous at element offset o of the K-major level matrix; levels j >= jmax
// (past step N) are stored as zeros. 16-byte stores per array.
// With diff set, the increments x_j - x_{j-1} are stored instead (x_{-1} = prev). full: every
// level of the block exists (jmax == kMxB), so no level is tested.
template <bool diff, bool full>
__device__ __forceinline__ void store_levels(int kind, const float *xc, int jmax, char *gt_hi, char *gt_lo, int64_t o,
                                             float prev = 0.0f) {
    // levels j .. j + 3 (j a multiple of 4) in one 16-byte shared-memory load; increments and
    // the zeros past jmax applied in registers
    const float4 *xq = reinterpret_cast<const float4 *>(xc);
    auto quad = [&](int j, float (&v)[4]) {
        const float4 q = xq[(j / 4) * kMxT];
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
        if (diff) {
            const float p0 = prev;
            prev = v[3];
            v[3] -= v[2];
            v[2] -= v[1];
            v[1] -= v[0];
            v[0] -= p0;
        }
        if (!full) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (j + i >= jmax) v[i] = 0.0f;
        }
    };
    if (kind == tc::TC_TF32X3) {
        uint4 *dh = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(gt_hi) + o);
        uint4 *dl = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(gt_lo) + o);
        for (int j = 0; j < kMxB; j += 4) {
            float v[4];
            quad(j, v);
            uint32_t h[4], l[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) split_f32_tf32(v[i], h[i], l[i]);
            dh[j / 4] = make_uint4(h[0], h[1], h[2], h[3]);
            dl[j / 4] = make_uint4(l[0], l[1], l[2], l[3]);
        }
    } else {
        uint4 *dh = reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(gt_hi) + o);
        uint4 *dl = reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(gt_lo) + o);
        for (int j = 0; j < kMxB; j += 8) {
            float v[8];
            quad(j, *reinterpret_cast<float(*)[4]>(v));
            quad(j + 4, *reinterpret_cast<float(*)[4]>(v + 4));
            uint32_t h[8], l[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) split_f32(v[i], h[i], l[i]);
            dh[j / 8] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16),
                                   h[6] | (h[7] << 16));
            dl[j / 8] = make_uint4(l[0] | (l[1] << 16), l[2] | (l[3] << 16), l[4] | (l[5] << 16),
                                   l[6] | (l[7] << 16));
        }
    }
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
        if (A.n0 == 1 && active) coef_store(A.coef, A.nmp, col, l2, gz, ex);
    } else {
        coef_load(A.coef, A.nmp, col, l2, gz, ex);
    }
    keep_reg(l2);
    const double *dn = st ? A.d2 : A.d1;
    const float *hd_hi = A.hdf + (size_t)(2 * st) * (P.N + 1), *hd_lo = hd_hi + (P.N + 1);
    const float *hdo_hi = A.hdf + (size_t)(2 * (1 - st)) * (P.N + 1), *hdo_lo = hdo_hi + (P.N + 1);
    const float gz_o = __shfl_xor_sync(0xffffffffu, gz, 16);      // the partner state's scaled g^0

    // the lane's last two levels as double-float pairs (FP32 part: what the sums and the level
    // matrix see), and the partner state's
    float gm1 = gz, gm2 = 0.0f, gm1_lo = 0.0f, gm2_lo = 0.0f;
    if (A.n0 == 1 && full_setup) gm1_lo = (float)(ldexp(A.g0[st * P.nmodes + mode], -ex) - (double)gz);
    if (A.n0 > 1) {
        gm1 = A.carry[col];
        gm2 = A.carry[2 * A.nmp + col];
        gm1_lo = A.carry[4 * A.nmp + col];
        gm2_lo = A.carry[6 * A.nmp + col];
    }
    const float x_before = gm1;                      // x^{n0 - 1}
    float gm1_o = __shfl_xor_sync(0xffffffffu, gm1, 16), gm2_o = __shfl_xor_sync(0xffffffffu, gm2, 16);
    float gm1_o_lo = __shfl_xor_sync(0xffffffffu, gm1_lo, 16), gm2_o_lo = __shfl_xor_sync(0xffffffffu, gm2_lo, 16);
    WeightRem wr = load_weight_rem(A.wrem, st);
    keep_reg(wr);
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
        inblock_chunks(a, w, xs4, j0);
        float xb[kMxSB] = {};                         // the sub-block's levels, stored as two float4
        // the sub-block's own triangle: each new level is added forward into the later sums
#pragma unroll
        for (int b = 0; b < kMxSB; ++b) {
            const int64_t n = A.n0 + j0 + b;
            if (j0 + b >= jmax) break;
            const float h = a[b];
            const float h_o = __shfl_xor_sync(0xffffffffu, h, 16);
            const float e_lo = weight_rem_terms(wr, j0 + b, n, gm1, gm1_lo, gm2);
            const float e_o_lo = __shfl_xor_sync(0xffffffffu, e_lo, 16);     // the partner state's
            df xd;
            if (full_setup && (A.solve64 || (P.scheme == CQ_BDF2 && n == 1))) {
                xd = lane_step_df(P, ls, A.solve64, n, h, gm1, gm2, gz, dn, hd_hi, hd_lo);
            } else if (P.scheme == CQ_BE) {
                xd = lane_step2_df(l2, gm1, gm1_lo, gm1_o, gm1_o_lo, h, e_lo, h_o, e_o_lo);
            } else {
                df l = two_sum(2.0f * gm1, -0.5f * gm2), lo = two_sum(2.0f * gm1_o, -0.5f * gm2_o);
                l.lo += fmaf(2.0f, gm1_lo, -0.5f * gm2_lo);
                lo.lo += fmaf(2.0f, gm1_o_lo, -0.5f * gm2_o_lo);
                // e = h + d_{n-1} g^0 / 2 (+ the remainder terms) as a double-float pair, for this
                // lane's state and (from the partner's h and g^0, with the same operations) for the
                // partner's
                const df ed = df_mul_f(df{__ldg(hd_hi + n - 1), __ldg(hd_lo + n - 1)}, gz);
                const df edo = df_mul_f(df{__ldg(hdo_hi + n - 1), __ldg(hdo_lo + n - 1)}, gz_o);
                const df e = df_add(ed, df{h, e_lo});
                const df e_o = df_add(edo, df{h_o, e_o_lo});
                xd = lane_step2_df(l2, l.hi, l.lo, lo.hi, lo.lo, e.hi, e.lo, e_o.hi, e_o.lo);
            }
            const float x = xd.hi;
#pragma unroll
            for (int bb = b + 1; bb < kMxSB; ++bb) a[bb] = fmaf(wt[bb - b], x, a[bb]);
            const float x_o = __shfl_xor_sync(0xffffffffu, x, 16);
            const float x_o_lo = __shfl_xor_sync(0xffffffffu, xd.lo, 16);
            xb[b] = x;
            gm2 = gm1;
            gm2_lo = gm1_lo;
            gm1 = x;
            gm1_lo = xd.lo;
            gm2_o = gm1_o;
            gm2_o_lo = gm1_o_lo;
            gm1_o = x_o;
            gm1_o_lo = x_o_lo;
        }
        // 16-byte stores: a warp's 32 lanes write 512 contiguous bytes (no bank conflicts)
        float4 *xw = reinterpret_cast<float4 *>(xs) + (j0 / 4) * kMxT + tid;
        xw[0] = make_float4(xb[0], xb[1], xb[2], xb[3]);
        xw[kMxT] = make_float4(xb[4], xb[5], xb[6], xb[7]);
    }
    if (!active) return;
    if (A.write_levels) {
        // level n0 + j goes to column n0 + j - 1 of row col
        if (jmax == kMxB) store_levels<false, true>(A.kind, xc, jmax, A.gt_hi, A.gt_lo, col * A.kpad + (A.n0 - 1));
        else store_levels<false, false>(A.kind, xc, jmax, A.gt_hi, A.gt_lo, col * A.kpad + (A.n0 - 1));
        if (A.dt_hi)
            store_levels<true, false>(A.kind, xc, jmax, A.dt_hi, A.dt_lo, col * A.kpad + (A.n0 - 1), x_before);
        A.carry[col] = gm1;
        A.carry[2 * A.nmp + col] = gm2;
        A.carry[4 * A.nmp + col] = gm1_lo;
        A.carry[6 * A.nmp + col] = gm2_lo;
    }
    if (A.x1 && A.n0 == 1) A.x1[col] = xc[0];
    if (A.n0 + kMxB > P.N) {                         // the block holding step N
        const double out = ldexp((double)gm1 + (double)gm1_lo, ex);
        A.gN[st * P.nmodes + mode] = out;
        if (!isfinite(out)) atomicOr(A.status, ST_NONFINITE);
    }
}

// Row st of the transposed step inverse (M^T)^{-1} = (M^{-1})^T in the lane's own / other ordering.
__device__ __forceinline__ void adj_rows(const Inv2 &m, int st, double &oo, double &ot) {
    oo = st ? m.i22 : m.i11;
    ot = st ? m.i12 : m.i21;
}

// Two-term adjoint step lambda = A' l + B' e with A' = M'^{-1} / tau, B' = -M'^{-1}.
__device__ __forceinline__ void adj_lane_coef(double oo, double ot, double inv_tau, LaneStep2 &l2) {
    const df x = df_from(oo * inv_tau), y = df_from(ot * inv_tau), u = df_from(-oo), v = df_from(-ot);
    l2.a_hi[0] = x.hi;
    l2.a_lo[0] = x.lo;
    l2.a_hi[1] = y.hi;
    l2.a_lo[1] = y.lo;
    l2.b_hi[0] = u.hi;
    l2.b_lo[0] = u.lo;
    l2.b_hi[1] = v.hi;
    l2.b_lo[1] = v.lo;
}

// Adjoint steps r = n0 .. min(n0 + kMxB - 1, N) (m = N - r + 1) of 64 modes per CTA, in
// the layout of k_mixed_block. Per mode, with K = [[c, -a], [-a, c]] and W_i = diag(d^1_i, d^2_i),
//   (c_m I + e_m W_0 K) lambda^m = l^m / tau - hr^m - [m = N] dJ/dx^N,   mu^m = K lambda^m,
//   hr^m = sum_{n > m} W_{n-m} mu^n  (the reversed-time history of the levels mu),
//   l^m = lambda^{m+1} (BE) or 2 lambda^{m+1} - lambda^{m+2} / 2 (SBD),
// (c_m, e_m) = (1/tau, 1) for BE, (3/(2 tau), 1) for SBD m >= 2 and (1/tau, 2/3) for SBD m = 1,
// i.e. the transposed step matrices of Eq. 4.1 / Eq. 4.7. g0 holds dJ/dx^N, scaled per mode
// by a power of two like G^0 in the forward solve. Per lane and step the sums of dJ/dbeta
// (mu^m hp^m, hp^m = ht^m + D'_{m-1} x^0) and, for SBD, of d_{m-1} mu^m and d'_{m-1} mu^m run in
// FP32 over the block and
// are added to the lane's FP64 totals at its end; lambda^1, mu^1 and lambda^2 are kept.
__global__ void __launch_bounds__(kMxT) k_mixed_adjoint(const __grid_constant__ MixedArgs A) {
    extern __shared__ __align__(16) float smx[];
    float *xs = smx;
    float *wsm = smx + kMxB * kMxT;
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
    const int64_t N = P.N;
    const bool sbd = P.scheme == CQ_BDF2;
    const bool last = A.n0 + kMxB > N;                      // the block holding m = 1

    LaneStep2 l2, l2f;                                       // steps with M'; the SBD step m = 1 (M1')
    double t_oo = 0.0, t_ot = 0.0, t1_oo = 0.0, t1_ot = 0.0;
    float rz;
    int ey = 0;
    if (A.n0 == 1 || A.solve64 || (sbd && last)) {
        const double r64 = A.g0[st * P.nmodes + mode];
        const double rmax = fmax(fabs(r64), fabs(__shfl_xor_sync(0xffffffffu, r64, 16)));
        if (rmax > 0.0 && isfinite(rmax)) frexp(rmax, &ey);
        rz = (float)ldexp(r64, -ey);
        ModeConst mc;
        mode_setup(P, A.lam[mode], A.d1[0], A.d2[0], mc);
        adj_rows(mc.Mn, st, t_oo, t_ot);
        adj_lane_coef(t_oo, t_ot, P.inv_tau, l2);
        l2f = l2;
        if (sbd) {
            adj_rows(mc.M1, st, t1_oo, t1_ot);
            adj_lane_coef(t1_oo, t1_ot, P.inv_tau, l2f);
        }
        if (A.n0 == 1 && active) coef_store(A.coef, A.nmp, col, l2, rz, ey);
    } else {
        coef_load(A.coef, A.nmp, col, l2, rz, ey);
        l2f = l2;
    }
    df dc = df_from(P.a + A.lam[mode]), da = df_from(P.a);
    keep_reg(dc.hi);
    keep_reg(dc.lo);
    keep_reg(da.hi);
    keep_reg(da.lo);
    keep_reg(l2);
    keep_reg(l2f);
    const float *hd_hi = A.hdf + (size_t)(2 * st) * (N + 1);         // d_i / 2 (hi part)
    const float *dq = A.dqf + (size_t)st * (N + 1);                   // d'_i
    const float *cq = A.cqf + (size_t)st * (N + 1);                   // D'_i
    const float x0f = A.coef_fwd[4 * A.nmp + col].x;                  // x^0, scaled like the forward levels

    // lambda^{m+1}, lambda^{m+2} as double-float pairs, and the partner state's
    float gm1 = 0.0f, gm2 = 0.0f, gm1_lo = 0.0f, gm2_lo = 0.0f;
    if (A.n0 > 1) {
        gm1 = A.carry[col];
        gm2 = A.carry[2 * A.nmp + col];
        gm1_lo = A.carry[4 * A.nmp + col];
        gm2_lo = A.carry[6 * A.nmp + col];
    }
    float gm1_o = __shfl_xor_sync(0xffffffffu, gm1, 16), gm2_o = __shfl_xor_sync(0xffffffffu, gm2, 16);
    float gm1_o_lo = __shfl_xor_sync(0xffffffffu, gm1_lo, 16), gm2_o_lo = __shfl_xor_sync(0xffffffffu, gm2_lo, 16);
    // mu^{m+1} (double-float) and mu^{m+2} of the lane's state, the levels of the adjoint's history
    const df mv1 = df_add(df_mul_f(dc, gm1), df_neg(df_mul_f(da, gm1_o)));
    const df mv2 = df_add(df_mul_f(dc, gm2), df_neg(df_mul_f(da, gm2_o)));
    float mu1 = mv1.hi, mu1_lo = mv1.lo, mu2 = mv2.hi + mv2.lo;
    WeightRem wr = load_weight_rem(A.wrem, st);
    keep_reg(wr);
    const float *w = wsm + st * kMxW + kMxWOff;
    float wt[kMxSB];
#pragma unroll
    for (int i = 1; i < kMxSB; ++i) wt[i] = w[i];
    float *xc = xs + 4 * tid;
    const float4 *xs4 = reinterpret_cast<const float4 *>(xs) + tid;
    const int64_t ldacc = 2 * A.nmp;
    const int jmax = (int)min((int64_t)kMxB, N - A.n0 + 1);
    // contraction rows and ht rows (ht row N - r for step r) of the next sub-block, prefetched
    float an[kMxSB], hn[kMxSB];
#pragma unroll
    for (int b = 0; b < kMxSB; ++b) {
        an[b] = A.acc ? A.acc[(int64_t)b * ldacc + col] : 0.0f;
        hn[b] = b < jmax ? A.ht[(N - A.n0 - b) * ldacc + col] : 0.0f;
    }
    float db = 0.0f, sg = 0.0f, sx = 0.0f;
    for (int j0 = 0; j0 < jmax; j0 += kMxSB) {
        float a[kMxSB], hv[kMxSB];
#pragma unroll
        for (int b = 0; b < kMxSB; ++b) {
            a[b] = an[b];
            hv[b] = hn[b];
        }
        if (j0 + kMxSB < jmax) {
#pragma unroll
            for (int b = 0; b < kMxSB; ++b) {
                const int j = j0 + kMxSB + b;
                if (A.acc) an[b] = A.acc[(int64_t)j * ldacc + col];
                hn[b] = j < jmax ? A.ht[(N - A.n0 - j) * ldacc + col] : 0.0f;
            }
        }
        inblock_chunks(a, w, xs4, j0);
        float xb[kMxSB] = {};                         // the sub-block's levels, stored as two float4
#pragma unroll
        for (int b = 0; b < kMxSB; ++b) {
            const int64_t r = A.n0 + j0 + b;
            if (j0 + b >= jmax) break;
            const int64_t m = N - r + 1;
            float h = a[b];
            if (r == 1) h += rz;                             // the terminal term at m = N
            const float h_o = __shfl_xor_sync(0xffffffffu, h, 16);
            // remainders of the history's largest weights (d_1, d_2) and of mu^{m+1}
            const float e_lo = weight_rem_terms(wr, j0 + b, r, mu1, mu1_lo, mu2);
            const float e_o_lo = __shfl_xor_sync(0xffffffffu, e_lo, 16);     // the partner state's
            df ld;
            if (A.solve64) {
                const double l = sbd ? 2.0 * (double)gm1 - 0.5 * (double)gm2 : (double)gm1;
                const double l_o = sbd ? 2.0 * (double)gm1_o - 0.5 * (double)gm2_o : (double)gm1_o;
                const bool f = sbd && m == 1;
                const double bs = l * P.inv_tau - (double)h, bo = l_o * P.inv_tau - (double)h_o;
                ld = df_from((f ? t1_oo : t_oo) * bs + (f ? t1_ot : t_ot) * bo);
            } else if (!sbd) {
                ld = lane_step2_df(l2, gm1, gm1_lo, gm1_o, gm1_o_lo, h, e_lo, h_o, e_o_lo);
            } else {
                df l = two_sum(2.0f * gm1, -0.5f * gm2), lo = two_sum(2.0f * gm1_o, -0.5f * gm2_o);
                l.lo += fmaf(2.0f, gm1_lo, -0.5f * gm2_lo);
                lo.lo += fmaf(2.0f, gm1_o_lo, -0.5f * gm2_o_lo);
                ld = lane_step2_df(m == 1 ? l2f : l2, l.hi, l.lo, lo.hi, lo.lo, h, e_lo, h_o, e_o_lo);
            }
            const float lam = ld.hi;
            const float lam_o = __shfl_xor_sync(0xffffffffu, lam, 16);
            const float lam_o_lo = __shfl_xor_sync(0xffffffffu, ld.lo, 16);
            const df mv = df_add(df_mul_f(dc, lam), df_neg(df_mul_f(da, lam_o)));
            const float mu = mv.hi;
#pragma unroll
            for (int bb = b + 1; bb < kMxSB; ++bb) a[bb] = fmaf(wt[bb - b], mu, a[bb]);
            xb[b] = mu;
            db = fmaf(mu, fmaf(x0f, __ldg(cq + m - 1), hv[b]), db);      // mu^m hp^m
            if (sbd && m >= 2) {
                sg = fmaf(2.0f * __ldg(hd_hi + m - 1), mu, sg);
                sx = fmaf(__ldg(dq + m - 1), mu, sx);
            }
            if (m <= 2 && active) {
                if (m == 1) {
                    A.lbuf[col] = lam;
                    A.lbuf[ldacc + col] = mu;
                } else {
                    A.lbuf[2 * ldacc + col] = lam;
                }
            }
            gm2 = gm1;
            gm2_lo = gm1_lo;
            gm1 = lam;
            gm1_lo = ld.lo;
            gm2_o = gm1_o;
            gm2_o_lo = gm1_o_lo;
            gm1_o = lam_o;
            gm1_o_lo = lam_o_lo;
            mu2 = mu1;
            mu1 = mu;
            mu1_lo = mv.lo;
        }
        float4 *xw = reinterpret_cast<float4 *>(xs) + (j0 / 4) * kMxT + tid;
        xw[0] = make_float4(xb[0], xb[1], xb[2], xb[3]);
        xw[kMxT] = make_float4(xb[4], xb[5], xb[6], xb[7]);
    }
    if (!active) return;
    if (A.write_levels) {
        if (jmax == kMxB) store_levels<false, true>(A.kind, xc, jmax, A.gt_hi, A.gt_lo, col * A.kpad + (A.n0 - 1));
        else store_levels<false, false>(A.kind, xc, jmax, A.gt_hi, A.gt_lo, col * A.kpad + (A.n0 - 1));
        A.carry[col] = gm1;
        A.carry[2 * A.nmp + col] = gm2;
        A.carry[4 * A.nmp + col] = gm1_lo;
        A.carry[6 * A.nmp + col] = gm2_lo;
    }
    const int exf = __float_as_int(A.coef_fwd[4 * A.nmp + col].y);     // the forward levels' exponent
    A.lacc[col] += ldexp((double)db, exf + ey);
    if (sbd) {
        A.lacc[ldacc + col] += ldexp((double)sg, ey);
        A.lacc[2 * ldacc + col] += ldexp((double)sx, ey);
    }
}

struct GradArgs {
    int64_t nmodes, nmp, N;
    int scheme, vjp;
    double wd, inv_tau;
    const double *gN, *tgt, *g0, *d1, *d2, *q1, *q2, *lacc;
    const float *lbuf, *x1;
    const float4 *coef_fwd, *coef_adj;
    double *rT, *gx0, *acc;
};

// dJ/dx^N: h^d (x^N - t) for the misfit, or the given modal gradient (vjp).
__global__ void k_grad_terminal(const GradArgs G) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * G.nmodes) return;
    G.rT[i] = G.vjp ? G.tgt[i] : G.wd * (G.gN[i] - G.tgt[i]);
}

// Per state (block s): D'_i = sum_{l<=i} d'_l (a block-wide scan in FP64), e_0 = 0 and
// e_i = D'_{i-1} (i = 1 .. N + 1), and d', D' in FP32.
__global__ void __launch_bounds__(1024) k_grad_weights(const double *__restrict__ q1, const double *__restrict__ q2,
                                                       int64_t n, double *__restrict__ e1, double *__restrict__ e2,
                                                       float *__restrict__ dqf, float *__restrict__ cqf) {
    __shared__ double part[1024];
    const double *q = blockIdx.x ? q2 : q1;
    double *e = blockIdx.x ? e2 : e1;
    float *df_ = dqf + blockIdx.x * (n + 1), *cf = cqf + blockIdx.x * (n + 1);
    const int t = threadIdx.x, T = blockDim.x;
    const int64_t chunk = (n + 1 + T - 1) / T, lo = t * chunk, hi = min(lo + chunk, n + 1);
    double sum = 0.0;
    for (int64_t i = lo; i < hi; ++i) sum += q[i];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        const double v = t >= off ? part[t - off] : 0.0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    double run = t ? part[t - 1] : 0.0;
    if (t == 0) e[0] = 0.0;
    for (int64_t i = lo; i < hi; ++i) {
        run += q[i];
        e[i + 1] = run;
        df_[i] = (float)q[i];
        cf[i] = (float)run;
    }
}

// Per mode: the modal dJ/dx^0 and the mode's share of J and of dJ/dbeta_s
// (BE:  dJ/dx^0 = -lambda^1 / tau;
//  SBD: dJ/dx^0 = -lambda^1 / tau + W_0 mu^1 / 3 + lambda^2 / (2 tau) + sum_{n>=2} W_{n-1} mu^n / 2,
//       and dJ/dbeta gains mu^1 d'_0 (x^0 - x^1) / 3 + x^0 sum_{n>=2} d'_{n-1} mu^n / 2).
__global__ void __launch_bounds__(256) k_grad_final(const GradArgs G) {
    const int64_t mode = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double J = 0.0, db[2] = {0.0, 0.0};
    if (mode < G.nmodes) {
        const int64_t ld = 2 * G.nmp;
        for (int s = 0; s < 2; ++s) {
            const int64_t col = s * G.nmp + mode, i = s * G.nmodes + mode;
            const int exf = __float_as_int(G.coef_fwd[4 * G.nmp + col].y);
            const int ey = __float_as_int(G.coef_adj[4 * G.nmp + col].y);
            const double l1 = ldexp((double)G.lbuf[col], ey), m1 = ldexp((double)G.lbuf[ld + col], ey);
            const double *d = s ? G.d2 : G.d1, *q = s ? G.q2 : G.q1;
            double g = -l1 * G.inv_tau, b = G.lacc[col];
            if (G.scheme == CQ_BDF2) {
                const double l2 = ldexp((double)G.lbuf[2 * ld + col], ey);
                g += d[0] * m1 / 3.0 + 0.5 * G.inv_tau * l2 + 0.5 * G.lacc[ld + col];
                const double x0 = G.g0[i], x1 = ldexp((double)G.x1[col], exf);
                b += m1 * q[0] * (x0 - x1) / 3.0 + 0.5 * x0 * G.lacc[2 * ld + col];
            }
            G.gx0[i] = g;
            db[s] = b;
            if (!G.vjp) {
                const double e = G.gN[i] - G.tgt[i];
                J += 0.5 * G.wd * e * e;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        J += __shfl_xor_sync(0xffffffffu, J, off);
        db[0] += __shfl_xor_sync(0xffffffffu, db[0], off);
        db[1] += __shfl_xor_sync(0xffffffffu, db[1], off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(G.acc + 0, J);
        atomicAdd(G.acc + 1, db[0]);
        atomicAdd(G.acc + 2, db[1]);
    }
}

constexpr size_t kMxSmem = ((size_t)kMxB * kMxT + 2 * kMxW) * sizeof(float);

// Banks of d^1, d^2 (when some block has earlier blocks' levels) and the level maps.
static int mixed_maps(const MixedLayout &l, const Fp2sParams &P, const double *d1, const double *d2, bool grad,
                      tc::TcMaps &maps, cudaStream_t s) {
    int st;
    if (l.nblk > 1) {
        const double *d[2] = {d1, d2};
        for (int q = 0; q < 2; ++q) {
            if ((st = tc_bank(l.kind, d[q], P.N, tc::kind_bk(l.kind), l.ntiles, l.a_hi[q], l.a_lo[q], s))) return st;
            if ((st = tc_map_bank(l.kind, &maps.a_hi[q], l.a_hi[q], l.ntiles))) return st;
            if ((st = tc_map_bank(l.kind, &maps.a_lo[q], l.a_lo[q], l.ntiles))) return st;
        }
    }
    if (l.nblk > 1 || grad) {
        if ((st = tc_map_levels(l.kind, &maps.b_hi, l.gt_hi, l.kpad, 2 * l.nmp))) return st;
        if ((st = tc_map_levels(l.kind, &maps.b_lo, l.gt_lo, l.kpad, 2 * l.nmp))) return st;
    }
    return CQ_OK;
}

static tc::TcParams mixed_tc_params(const Fp2sParams &P, const MixedLayout &l) {
    tc::TcParams T{};
    T.ndof = P.nmodes;
    T.ldh = 2 * l.nmp;
    T.num_i = 1;
    T.delta0 = tc::kind_bk(l.kind);
    T.n_states = 2;
    T.ntile_state = (P.nmodes + tc::BN - 1) / tc::BN;
    T.state_stride = l.nmp;
    return T;
}

// All blocks of one sweep (the forward solve, or the adjoint with adjoint = true).
// Blocks in pairs (2p, 2p+1). Once both earlier pairs' levels exist, one contraction
// covers the rows of both blocks over the levels of blocks < 2p (two row tiles per
// column tile: the level matrix is streamed once for 256 rows); block 2p+1 then adds
// the levels of block 2p with a short contraction (K = 128) added onto its rows.
static int mixed_sweep(const Fp2sParams &P, const MixedLayout &l, const tc::TcMaps &maps, MixedArgs A, bool adjoint,
                       bool keep_all_levels, int *status, cudaStream_t s) {
    int st;
    static unsigned long long attr[2] = {};
    const void *kern = adjoint ? (const void *)k_mixed_adjoint : (const void *)k_mixed_block;
    if ((st = smem_attr_once(kern, (int)kMxSmem, &attr[adjoint ? 1 : 0]))) return st;
    const int64_t mpb = (kMxT / 32) * kFastModesPerWarp;
    const unsigned grid = (unsigned)((P.nmodes + mpb - 1) / mpb);
    tc::TcParams T = mixed_tc_params(P, l);
    T.max_ctas = device_sms();          // every tile of a launch has the same K: one CTA per SM
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
        A.write_levels = b + 1 < l.nblk || keep_all_levels;
        if (adjoint) k_mixed_adjoint<<<grid, kMxT, kMxSmem, s>>>(A);
        else k_mixed_block<<<grid, kMxT, kMxSmem, s>>>(A);
        if ((st = launched())) return st;
    }
    return CQ_OK;
}

static MixedArgs mixed_args(const Fp2sParams &P, const MixedLayout &l, const double *lam, const double *d1,
                            const double *d2, const float *hdf, int *status) {
    MixedArgs A{};
    A.P = P;
    A.nmp = l.nmp;
    A.kpad = l.kpad;
    A.solve64 = fabs(P.a) > 10.0;
    A.kind = l.kind;
    A.lam = lam;
    A.d1 = d1;
    A.d2 = d2;
    A.hdf = hdf;
    A.carry = l.carry;
    A.coef = l.coef;
    A.wrem = l.wrem;
    A.gt_hi = l.gt_hi;
    A.gt_lo = l.gt_lo;
    A.status = status;
    return A;
}

int mixed_direct_run(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                     const double *d1, const double *d2, const float *hdf, void *region, cudaStream_t s) {
    const MixedLayout l = mixed_layout(P, region, false);
    int st;
    tc::TcMaps maps;
    if ((st = mixed_maps(l, P, d1, d2, false, maps, s))) return st;
    k_weight_rem<<<1, 32, 0, s>>>(l.kind, d1, d2, P.N, l.wrem);
    if ((st = launched())) return st;
    MixedArgs A = mixed_args(P, l, lam, d1, d2, hdf, status);
    A.g0 = g0;
    A.gN = gN;
    return mixed_sweep(P, l, maps, A, false, false, status, s);
}

int mixed_grad_run(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                   const double *d1, const double *d2, const double *q1, const double *q2, const float *hdf,
                   const double *tgt, int vjp, double wd, double *gx0, double *acc, void *region, cudaStream_t s) {
    const MixedLayout l = mixed_layout(P, region, true);
    int st;
    tc::TcMaps maps;
    if ((st = mixed_maps(l, P, d1, d2, true, maps, s))) return st;
    k_weight_rem<<<1, 32, 0, s>>>(l.kind, d1, d2, P.N, l.wrem);
    if ((st = launched())) return st;
    // forward solve, every level kept
    MixedArgs A = mixed_args(P, l, lam, d1, d2, hdf, status);
    A.g0 = g0;
    A.gN = gN;
    A.x1 = l.x1;
    A.dt_hi = l.dt_hi;
    A.dt_lo = l.dt_lo;
    if ((st = mixed_sweep(P, l, maps, A, false, true, status, s))) return st;
    // ht: rows n' = n + 1 = 2 .. N + 1 of the history of the increments with weights e_i = D'_{i-1}
    k_grad_weights<<<2, 1024, 0, s>>>(q1, q2, P.N, l.e[0], l.e[1], l.dqf, l.cqf);
    if ((st = launched())) return st;
    tc::TcMaps qm = maps;
    if ((st = tc_map_levels(l.kind, &qm.b_hi, l.dt_hi, l.kpad, 2 * l.nmp))) return st;
    if ((st = tc_map_levels(l.kind, &qm.b_lo, l.dt_lo, l.kpad, 2 * l.nmp))) return st;
    for (int q = 0; q < 2; ++q) {
        if ((st = tc_bank(l.kind, l.e[q], P.N + 1, l.qdelta0, l.qntiles, l.q_hi[q], l.q_lo[q], s))) return st;
        if ((st = tc_map_bank(l.kind, &qm.a_hi[q], l.q_hi[q], l.qntiles))) return st;
        if ((st = tc_map_bank(l.kind, &qm.a_lo[q], l.q_lo[q], l.qntiles))) return st;
    }
    tc::TcParams T = mixed_tc_params(P, l);
    T.n_lo = 2;
    T.rows = P.N;
    T.num_i = (int)((P.N + tc::BM - 1) / tc::BM);
    T.delta0 = l.qdelta0;
    T.k_lo = 0;
    T.kprime = (int)P.N;
    T.add = 0;
    // a full causal triangle: tiles of unequal K, claimed in order by one CTA per SM
    T.max_ctas = device_sms();
    T.tile_counter = l.tcount;
    if ((st = cuda_status(cudaMemsetAsync(l.tcount, 0, sizeof(int), s)))) return st;
    if ((st = timing_part(s, false))) return st;
    if ((st = tc_contract_f32(l.kind, qm, T, l.ht, status, s))) return st;
    if ((st = timing_part(s, true))) return st;
    // adjoint sweep
    GradArgs G{};
    G.nmodes = P.nmodes;
    G.nmp = l.nmp;
    G.N = P.N;
    G.scheme = P.scheme;
    G.vjp = vjp;
    G.wd = wd;
    G.inv_tau = P.inv_tau;
    G.gN = gN;
    G.tgt = tgt;
    G.g0 = g0;
    G.d1 = d1;
    G.d2 = d2;
    G.q1 = q1;
    G.q2 = q2;
    G.lacc = l.lacc;
    G.lbuf = l.lbuf;
    G.x1 = l.x1;
    G.coef_fwd = l.coef;
    G.coef_adj = l.coef_adj;
    G.rT = l.rT;
    G.gx0 = gx0;
    G.acc = acc;
    k_grad_terminal<<<(unsigned)((2 * P.nmodes + 255) / 256), 256, 0, s>>>(G);
    if ((st = launched())) return st;
    if ((st = cuda_status(cudaMemsetAsync(l.lacc, 0, (size_t)3 * 2 * l.nmp * sizeof(double), s)))) return st;
    if ((st = cuda_status(cudaMemsetAsync(l.lbuf, 0, (size_t)3 * 2 * l.nmp * sizeof(float), s)))) return st;
    MixedArgs B = mixed_args(P, l, lam, d1, d2, hdf, status);
    B.g0 = l.rT;
    B.coef = l.coef_adj;
    B.coef_fwd = l.coef;
    B.ht = l.ht;
    B.dqf = l.dqf;
    B.cqf = l.cqf;
    B.lacc = l.lacc;
    B.lbuf = l.lbuf;
    if ((st = mixed_sweep(P, l, maps, B, true, false, status, s))) return st;
    k_grad_final<<<(unsigned)((P.nmodes + 255) / 256), 256, 0, s>>>(G);
    return launched();
}

}  // namespace fastcq
