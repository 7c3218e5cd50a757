// Fused direct solve with FP64-class accuracy on the FP32 pipe (CQ_DIRECT with CQ_DF64).
//
// The direct history h^n = sum_{k=1}^{n-1} d_{n-k} g^k (Eq. 3.8, in the schemes of Eqs. 4.1
// and 4.7) costs N^2 / 2 multiply-adds per mode and state; in FP64 each is a DFMA on a pipe
// that runs at 1/64 of the FP32 rate. Here the weights and the stored levels are double-float
// pairs (hi + lo of two FP32 numbers) and each term is a double-float multiply-add of 12 FP32
// operations: Dekker's TwoProduct in its FMA form for the high parts, the two cross terms,
// Knuth's TwoSum into the running high part, the low parts summed unnormalised. The 2x2 step
// (mode_step) stays in FP64. Every mode is scaled by the power of two of its G^0 and the
// factor is applied on output; FP32's exponent range then bounds the growth a mode may show
// over the run (about 2^100, e^70), past which the solve reports CQ_ENONFINITE.
//
// One thread per mode carries both states (one-warp blocks). Time blocks of BT steps: for the
// block starting at n0 the levels 1 .. n0 - 1 are taken BT at a time, with the 2 BT - 1 weights
// that the BT x BT terms of such a group need loaded once (no shifting register window); the
// levels of the next group are copied into shared memory (cp.async) while a group is summed,
// which hides the DRAM latency that otherwise stalled the warps (long-scoreboard stalls 4.5 per
// issued instruction, 47 % issue). The in-block terms follow step by step with the steps. The
// levels are stored as double-float pairs, both states of a mode side by side (16 bytes):
// hist[(k * nmodes + mode) * 2 + s].
#include "fastdf.cuh"

namespace fastcq {

// wz[i] = d_{i - BT} as hi + lo for 1 <= i - BT <= n, else zero; i = 0 .. n + 2 BT.
__global__ void k_pad_df(const double *__restrict__ d, int64_t n, int BT, float2 *__restrict__ wz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n + 2 * BT) return;
    const int64_t idx = i - BT;
    wz[i] = (idx >= 1 && idx <= n) ? df_of(d[idx]) : make_float2(0.0f, 0.0f);
}

// 16-byte asynchronous copy global -> shared through L2 (cp.async.cg: the levels were written
// by plain stores of the same thread, which L2 holds), and its groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int BT>
__global__ void __launch_bounds__(32, 16)
    k_fp2s_direct_df(Fp2sParams P, const double *__restrict__ lam, const double *__restrict__ g0,
                     double *__restrict__ gN, int *__restrict__ status, const double *__restrict__ d1,
                     const double *__restrict__ d2, const float2 *__restrict__ wz1, const float2 *__restrict__ wz2,
                     float2 *__restrict__ hist) {
    const int64_t nm = P.nmodes;
    const int64_t mode = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nm) return;
    // per-mode power-of-two scale from max(|g1^0|, |g2^0|)
    const double gz1r = g0[mode], gz2r = g0[nm + mode];
    const double gmax = fmax(fabs(gz1r), fabs(gz2r));
    int ex = 0;
    if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &ex);
    const double gz1 = ldexp(gz1r, -ex), gz2 = ldexp(gz2r, -ex);
    float4 *h4 = reinterpret_cast<float4 *>(hist);          // level k of the mode at h4[k * nm + mode]
    {
        const float2 a = df_of(gz1), b = df_of(gz2);
        h4[mode] = make_float4(a.x, a.y, b.x, b.y);
    }
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    ModeConst mc;
    if (!mode_setup(P, lam[mode], d10, d20, mc)) atomicOr(status, ST_SINGULAR);
    double gm1_1 = gz1, gm1_2 = gz2, gm2_1 = 0.0, gm2_2 = 0.0;
    const float4 *hb = h4 + mode;
    constexpr int kStages = 3;
    __shared__ float4 sxs[kStages * BT * 32];                // [stage][level j][lane]: both states
    float4 *sx = sxs + (threadIdx.x & 31);
    for (int64_t n0 = 1; n0 <= P.N; n0 += BT) {
        float ah1[BT], al1[BT], ah2[BT], al2[BT];
#pragma unroll
        for (int b = 0; b < BT; ++b) ah1[b] = al1[b] = ah2[b] = al2[b] = 0.0f;
        // levels 1 .. n0 - 1 in groups of BT: level k0 + j enters row b with lag
        // n0 + b - k0 - j = base + (BT - 1 + b - j), base = n0 - k0 - BT + 1 >= 1
        // the groups' levels are staged in shared memory one group ahead of use: the copies of
        // group g + 1 are in flight while group g is summed (three stages: the stage refilled was
        // read two groups earlier)
        const int64_t ngroups = (n0 - 1) / BT;
        auto stage_group = [&](int64_t g) {
            float4 *dst = sx + (int)(g % kStages) * BT * 32;
            const float4 *src = hb + (1 + g * BT) * nm;
#pragma unroll
            for (int j = 0; j < BT; ++j) cp_async16(dst + j * 32, src + j * nm);
        };
        if (ngroups > 0) stage_group(0);
        cp_async_commit();
        for (int64_t g = 0; g < ngroups; ++g) {
            if (g + 1 < ngroups) stage_group(g + 1);
            cp_async_commit();
            cp_async_wait1();                      // group g has landed (own elements only)
            const int64_t k0 = 1 + g * BT;
            const int64_t base = n0 - k0 - BT + 1;
            float2 W1[2 * BT - 1], W2[2 * BT - 1], X1[BT], X2[BT];
#pragma unroll
            for (int t = 0; t < 2 * BT - 1; ++t) {
                W1[t] = __ldg(wz1 + base + t + BT);
                W2[t] = __ldg(wz2 + base + t + BT);
            }
            const float4 *xg = sx + (int)(g % kStages) * BT * 32;
#pragma unroll
            for (int j = 0; j < BT; ++j) {
                const float4 v = xg[j * 32];
                X1[j] = make_float2(v.x, v.y);
                X2[j] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int j = 0; j < BT; ++j)
#pragma unroll
                for (int b = 0; b < BT; ++b) {
                    const float2 w1 = W1[BT - 1 + b - j], w2 = W2[BT - 1 + b - j];
                    acc_prod(w1.x, w1.y, X1[j].x, X1[j].y, ah1[b], al1[b]);
                    acc_prod(w2.x, w2.y, X2[j].x, X2[j].y, ah2[b], al2[b]);
                }
        }
        // the block's own steps
        float2 l1[BT], l2[BT];
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int64_t n = n0 + b;
            if (n > P.N) break;
            float h1 = ah1[b], e1 = al1[b], h2 = ah2[b], e2 = al2[b];
#pragma unroll
            for (int kk = 0; kk < b; ++kk) {
                const float2 w1 = __ldg(wz1 + (b - kk) + BT), w2 = __ldg(wz2 + (b - kk) + BT);
                acc_prod(w1.x, w1.y, l1[kk].x, l1[kk].y, h1, e1);
                acc_prod(w2.x, w2.y, l2[kk].x, l2[kk].y, h2, e2);
            }
            double d1n = 0.0, d2n = 0.0;
            if (P.scheme == CQ_BDF2 && n >= 2) {
                d1n = __ldg(d1 + n - 1);
                d2n = __ldg(d2 + n - 1);
            }
            double x1, x2;
            mode_step(P, mc, n, (double)h1 + (double)e1, (double)h2 + (double)e2, d10, d20, d1n, d2n, gm1_1, gm1_2,
                      gm2_1, gm2_2, gz1, gz2, x1, x2);
            l1[b] = df_of(x1);
            l2[b] = df_of(x2);
            h4[n * nm + mode] = make_float4(l1[b].x, l1[b].y, l2[b].x, l2[b].y);
            gm2_1 = gm1_1;
            gm2_2 = gm1_2;
            gm1_1 = x1;
            gm1_2 = x2;
        }
    }
    const double o1 = ldexp(gm1_1, ex), o2 = ldexp(gm1_2, ex);
    gN[mode] = o1;
    gN[nm + mode] = o2;
    if (!isfinite(o1) || !isfinite(o2)) atomicOr(status, ST_NONFINITE);
}

int direct_df_tables(const Fp2sParams &P, const double *d1, const double *d2, float2 *wz1, float2 *wz2,
                     cudaStream_t s) {
    const unsigned g = (unsigned)((P.N + 2 * kDirDfBT + 256) / 256);
    k_pad_df<<<g, 256, 0, s>>>(d1, P.N, kDirDfBT, wz1);
    k_pad_df<<<g, 256, 0, s>>>(d2, P.N, kDirDfBT, wz2);
    return launched(2);
}

int direct_df_solve(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                    const double *d1, const double *d2, const float2 *wz1, const float2 *wz2, float2 *hist,
                    cudaStream_t s) {
    // one-warp blocks spread the modes evenly over the SMs (every block runs all N steps)
    const unsigned blocks = (unsigned)((P.nmodes + 31) / 32);
    k_fp2s_direct_df<kDirDfBT><<<blocks, 32, 0, s>>>(P, lam, g0, gN, status, d1, d2, wz1, wz2, hist);
    return CQ_OK;
}

}  // namespace fastcq
