// Mixed-precision direct solve (precision form CQ_BF16X3 of the direct scheme).
//
// The direct history h^n = sum_{k=1}^{n-1} d_{n-k} g^k (Eq. 3.8) of all modes is
// computed in time blocks of kMxB steps. For the block starting at n0 the part
// from the levels of earlier blocks, sum_{k=1}^{n0-1} d_{n-k} g^k, is one causal
// Toeplitz contraction on the tensor cores (history_tc.cu: tcgen05, split BF16
// operands, FP32 accumulation), with a separate weight bank per state; the rest,
// from the levels n0 .. n-1 of the block itself, is formed step by step in FP32
// by the kernel that also takes the steps (Eq. 4.1 / Eq. 4.7 in the sine basis),
// evaluated in double-float arithmetic from the FP32 history sums (lane_step).
//
// Every mode is pre-scaled by an exact power of two from its G^0, as in the FP32
// fast form, so its values sit near 1 in the FP32 / BF16 range; the contraction
// is linear per mode, so the scaled levels give the scaled history.
//
// Per block: one contraction launch (blocks after the first) and one step
// launch, which appends the block's levels to the K-major BF16 level matrix.
#include "common.cuh"
#include "fp2s_core.cuh"
#include "tc.cuh"

namespace fastcq {

constexpr int kMxB = 128;      // steps per time block (= one tensor-core M tile)
constexpr int kMxSB = 8;       // register window of the in-block sums
constexpr int kMxT = 128;      // threads per CTA: 64 modes x 2 states
constexpr int kMxW = kMxB + kMxSB;

struct MixedLayout {
    __nv_bfloat16 *a_hi[2], *a_lo[2];   // Toeplitz banks of d^1 and d^2
    __nv_bfloat16 *gt_hi, *gt_lo;       // levels, K-major: row s * nmp + mode, column k - 1
    float *acc;                         // contraction output [kMxB][2 * nmp]
    float *carry;                       // g^{n-1}, g^{n-2} at the end of a block: [2][2 * nmp]
    int nblk, ntiles;
    int64_t nmp, kpad;
    size_t bytes;
};

static MixedLayout mixed_layout(const Fp2sParams &P, void *base) {
    MixedLayout l{};
    l.nmp = (P.nmodes + 3) / 4 * 4;
    l.nblk = (int)((P.N + kMxB - 1) / kMxB);
    const int64_t klev = (int64_t)(l.nblk - 1) * kMxB;          // levels ever contracted
    l.kpad = klev > 0 ? klev : tc::BK;
    l.ntiles = klev > 0 ? (int)(klev / tc::BK) : 1;
    Carve cv(base);
    const size_t bank = (size_t)l.ntiles * tc::BM * tc::BK;
    for (int s = 0; s < 2; ++s) {
        l.a_hi[s] = cv.take<__nv_bfloat16>(bank);
        l.a_lo[s] = cv.take<__nv_bfloat16>(bank);
    }
    const size_t lev = l.nblk > 1 ? (size_t)2 * l.nmp * l.kpad : 0;
    l.gt_hi = cv.take<__nv_bfloat16>(lev);
    l.gt_lo = cv.take<__nv_bfloat16>(lev);
    l.acc = cv.take<float>(l.nblk > 1 ? (size_t)kMxB * 2 * l.nmp : 0);
    l.carry = cv.take<float>((size_t)4 * l.nmp);
    l.bytes = cv.bytes();
    return l;
}

size_t mixed_direct_bytes(const Fp2sParams &P) { return mixed_layout(P, nullptr).bytes; }

struct MixedArgs {
    Fp2sParams P;
    int64_t nmp, n0, kpad;
    int solve64, write_levels;
    const double *lam, *g0, *d1, *d2;
    const float *hdf, *acc;
    float *carry;
    __nv_bfloat16 *gt_hi, *gt_lo;
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

// Steps n0 .. min(n0 + kMxB - 1, N) of 64 modes per CTA. Lanes l < 16 of a warp
// carry state 1 and lanes l + 16 state 2 of the same 16 modes. acc (absent for the
// first block) holds the contribution of the earlier blocks' levels. The block's
// levels stay in shared memory (column tid, conflict-free) for the in-block sums:
// sub-blocks of kMxSB steps first take the earlier in-block levels with a
// shifting register window of weights (one shared-memory load feeds kMxSB FMAs),
// then their own triangle step by step.
__global__ void __launch_bounds__(kMxT) k_mixed_block(const __grid_constant__ MixedArgs A) {
    extern __shared__ __align__(16) float smx[];
    float *xs = smx;                          // [kMxB][kMxT]
    float *wsm = smx + kMxB * kMxT;           // [2][kMxW]: d_i of each state, i < kMxW
    const Fp2sParams &P = A.P;
    const int tid = threadIdx.x, lane = tid & 31, st = lane >> 4;
    for (int i = tid; i < 2 * kMxW; i += kMxT) {
        const int s = i / kMxW, ii = i % kMxW;
        wsm[i] = ii <= P.N ? (float)(s ? A.d2 : A.d1)[ii] : 0.0f;
    }
    __syncthreads();

    const int64_t mode_raw = ((int64_t)blockIdx.x * (kMxT >> 5) + (tid >> 5)) * kFastModesPerWarp + (lane & 15);
    const bool active = mode_raw < P.nmodes;
    const int64_t mode = active ? mode_raw : 0;
    const int64_t col = st * A.nmp + mode;

    const double gz64 = A.g0[st * P.nmodes + mode];
    const double gmax = fmax(fabs(gz64), fabs(__shfl_xor_sync(0xffffffffu, gz64, 16)));
    int ex = 0;
    if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &ex);
    const float gz = (float)ldexp(gz64, -ex);

    LaneStep ls;
    const bool ok = lane_step_setup(P, A.lam[mode], A.d1[0], A.d2[0], st, ls);
    if (A.n0 == 1 && active && st == 0 && !ok) atomicOr(A.status, ST_SINGULAR);
    const double *dn = st ? A.d2 : A.d1;
    const float *hd_hi = A.hdf + (size_t)(2 * st) * (P.N + 1), *hd_lo = hd_hi + (P.N + 1);

    float gm1 = gz, gm2 = 0.0f;
    if (A.n0 > 1) {
        gm1 = A.carry[col];
        gm2 = A.carry[2 * A.nmp + col];
    }
    const float *w = wsm + st * kMxW;
    float *xc = xs + tid;
    const int64_t ldacc = 2 * A.nmp;
    for (int j0 = 0; j0 < kMxB; j0 += kMxSB) {
        if (A.n0 + j0 > P.N) break;
        float a[kMxSB], wv[kMxSB];
#pragma unroll
        for (int b = 0; b < kMxSB; ++b) {
            a[b] = A.acc ? A.acc[(int64_t)(j0 + b) * ldacc + col] : 0.0f;
            wv[b] = w[j0 + b];                      // d_{j0 + b - k} at k = 0
        }
        for (int k = 0; k < j0; ++k) {
            const float x = xc[k * kMxT];
#pragma unroll
            for (int b = 0; b < kMxSB; ++b) a[b] = fmaf(wv[b], x, a[b]);
#pragma unroll
            for (int b = kMxSB - 1; b > 0; --b) wv[b] = wv[b - 1];
            wv[0] = w[j0 - k - 1];
        }
        float lv[kMxSB];
#pragma unroll
        for (int b = 0; b < kMxSB; ++b) {
            const int64_t n = A.n0 + j0 + b;
            if (n > P.N) break;
            float h = a[b];
#pragma unroll
            for (int kk = 0; kk < b; ++kk) h = fmaf(w[b - kk], lv[kk], h);
            const float x = lane_step(P, ls, A.solve64, n, h, gm1, gm2, gz, dn, hd_hi, hd_lo);
            lv[b] = x;
            xc[(j0 + b) * kMxT] = x;
            gm2 = gm1;
            gm1 = x;
        }
    }
    if (!active) return;
    if (A.write_levels) {
        // level n0 + j goes to column n0 + j - 1 of row col; 16 levels = two 16-byte stores per array
        uint4 *dh = reinterpret_cast<uint4 *>(A.gt_hi + col * A.kpad + (A.n0 - 1));
        uint4 *dl = reinterpret_cast<uint4 *>(A.gt_lo + col * A.kpad + (A.n0 - 1));
        for (int j = 0; j < kMxB; j += 8) {
            uint32_t h[8], l[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) split_f32(xc[(j + i) * kMxT], h[i], l[i]);
            dh[j / 8] = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
            dl[j / 8] = make_uint4(l[0] | (l[1] << 16), l[2] | (l[3] << 16), l[4] | (l[5] << 16), l[6] | (l[7] << 16));
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
            if ((st = tc_bank(d[q], P.N, tc::BK, l.ntiles, l.a_hi[q], l.a_lo[q], s))) return st;
            if ((st = tc_map_bank(&maps.a_hi[q], l.a_hi[q], l.ntiles))) return st;
            if ((st = tc_map_bank(&maps.a_lo[q], l.a_lo[q], l.ntiles))) return st;
        }
        if ((st = tc_map_levels(&maps.b_hi, l.gt_hi, l.kpad, 2 * l.nmp))) return st;
        if ((st = tc_map_levels(&maps.b_lo, l.gt_lo, l.kpad, 2 * l.nmp))) return st;
    }
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_mixed_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMxSmem) !=
            cudaSuccess)
            return CQ_ECUDA;
        attr = true;
    }
    MixedArgs A;
    A.P = P;
    A.nmp = l.nmp;
    A.kpad = l.kpad;
    A.solve64 = fabs(P.a) > 10.0;
    A.lam = lam;
    A.g0 = g0;
    A.d1 = d1;
    A.d2 = d2;
    A.hdf = hdf;
    A.carry = l.carry;
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
    T.delta0 = tc::BK;
    T.n_states = 2;
    T.ntile_state = (P.nmodes + tc::BN - 1) / tc::BN;
    T.state_stride = l.nmp;
    for (int b = 0; b < l.nblk; ++b) {
        const int64_t n0 = 1 + (int64_t)b * kMxB;
        if (b > 0) {
            T.n_lo = n0;
            T.rows = min((int64_t)kMxB, P.N - n0 + 1);
            T.kprime = (int)(n0 - 1);
            if ((st = tc_contract_f32(maps, T, l.acc, status, s))) return st;
        }
        A.n0 = n0;
        A.acc = b > 0 ? l.acc : nullptr;
        A.write_levels = b + 1 < l.nblk;
        k_mixed_block<<<grid, kMxT, kMxSmem, s>>>(A);
        if ((st = launched())) return st;
    }
    return CQ_OK;
}

}  // namespace fastcq
