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

// wz[i] = d_{i - BT} as hi + lo for 1 <= i - BT <= n, else zero; i = 0 .. len - 1.
__global__ void k_pad_df(const double *__restrict__ d, int64_t n, int BT, int64_t len, float2 *__restrict__ wz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
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

// ---------------------------------------------------------------------------
// Adjoint of the direct scheme in double-float (the gradient of fp2s_gradient / fp2s_vjp
// with CQ_DF64): the same backward sweep as the FP64 adjoint (transposed 2x2 steps in FP64,
// run from m = N down to 1), with the two reversed-time histories
//   hr^m = sum_{n > m} d_{n-m} mu^n   and   hq^m = sum_{n >= m} d'_{n-m} mu^n
// summed in double-float from the stored mu^n (pairs, both states side by side, future levels
// staged in shared memory with cp.async as in the forward kernel). Everything that scales with
// the adjoint variables is scaled by the power of two of the terminal condition; the forward
// levels carry the forward's scale; both are undone in the per-mode sums at the end.
// mu[(n * nm + mode)] (float4) for n = 1 .. N + BT, the levels past N zero (the caller clears
// them); wa/qa: d and d' padded (k_pad_df with length N + 4 BT).
// ---------------------------------------------------------------------------
template <int BT>
__global__ void __launch_bounds__(32, 16)
    k_adjoint_direct_df(Fp2sParams P, double wd, const double *__restrict__ lam, const double *__restrict__ g0,
                        const double *__restrict__ d1, const double *__restrict__ d2,
                        const double *__restrict__ q1, const double *__restrict__ q2,
                        const float2 *__restrict__ wa1, const float2 *__restrict__ wa2,
                        const float2 *__restrict__ qa1, const float2 *__restrict__ qa2,
                        const float2 *__restrict__ hist, const double *__restrict__ gN,
                        const double *__restrict__ tgt, int vjp, float2 *__restrict__ mu,
                        double *__restrict__ gx0, double *__restrict__ acc) {
    const int64_t nm = P.nmodes;
    const int64_t mode_raw = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = mode_raw < nm;
    const int64_t mode = active ? mode_raw : 0;
    const int64_t N = P.N;
    const double a = P.a, c = a + lam[mode], it = P.inv_tau;
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    Inv2 Mn, M1;
    bool ok;
    {
        const double c0 = (P.scheme == CQ_BE) ? it : 1.5 * it;
        ok = invert2(c0 + d10 * c, -d10 * a, -d20 * a, c0 + d20 * c, Mn);
        if (P.scheme == CQ_BDF2)
            ok &= invert2(it + (2.0 / 3.0) * d10 * c, -(2.0 / 3.0) * d10 * a, -(2.0 / 3.0) * d20 * a,
                          it + (2.0 / 3.0) * d20 * c, M1);
    }
    // the forward's scale of this mode (as in k_fp2s_direct_df)
    int exf = 0;
    {
        const double gmax = fmax(fabs(g0[mode]), fabs(g0[nm + mode]));
        if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &exf);
    }
    const float4 *h4 = reinterpret_cast<const float4 *>(hist);
    float4 *m4 = reinterpret_cast<float4 *>(mu);
    // terminal condition dJ/dx^N in true units, then scaled by the power of two of its size
    const double xN1 = gN[mode], xN2 = gN[nm + mode];
    const double e1 = xN1 - tgt[mode], e2 = xN2 - tgt[nm + mode];
    const double r1t = vjp ? tgt[mode] : wd * e1, r2t = vjp ? tgt[nm + mode] : wd * e2;
    double Jpart = (active && !vjp) ? 0.5 * wd * (e1 * e1 + e2 * e2) : 0.0;
    int ey = 0;
    {
        const double rmax = fmax(fabs(r1t), fabs(r2t));
        if (rmax > 0.0 && isfinite(rmax)) frexp(rmax, &ey);
    }
    const double r1 = ldexp(r1t, -ey), r2 = ldexp(r2t, -ey);
    double lp1_1 = 0.0, lp1_2 = 0.0, lp2_1 = 0.0, lp2_2 = 0.0;      // lambda^{m+1}, lambda^{m+2}
    double db1 = 0.0, db2 = 0.0, sg1 = 0.0, sg2 = 0.0, sx1 = 0.0, sx2 = 0.0;
    double lam1_1 = 0.0, lam1_2 = 0.0, lam2_1 = 0.0, lam2_2 = 0.0, mu1_1 = 0.0, mu1_2 = 0.0;
    const float4 *mb = m4 + mode;
    constexpr int kStages = 3;
    __shared__ float4 sxs[kStages * BT * 32];
    float4 *sx = sxs + (threadIdx.x & 31);
    // idle lanes (past the last mode) skip the sweep: they take part in the warp sums only
    for (int64_t mhi = active ? N : 0; mhi >= 1; mhi -= BT) {
        float ar1[BT], er1[BT], ar2[BT], er2[BT], aq1[BT], eq1[BT], aq2[BT], eq2[BT];
#pragma unroll
        for (int b = 0; b < BT; ++b) ar1[b] = er1[b] = ar2[b] = er2[b] = aq1[b] = eq1[b] = aq2[b] = eq2[b] = 0.0f;
        // future levels n = mhi + 1 .. N in groups of BT (the last one padded with zero levels):
        // level n1 + j enters row b (m = mhi - b) with lag n1 - mhi + j + b
        const int64_t ngroups = (N - mhi + BT - 1) / BT;
        auto stage_group = [&](int64_t g) {
            float4 *dst = sx + (int)(g % kStages) * BT * 32;
            const float4 *src = mb + (mhi + 1 + g * BT) * nm;
#pragma unroll
            for (int j = 0; j < BT; ++j) cp_async16(dst + j * 32, src + j * nm);
        };
        if (ngroups > 0) stage_group(0);
        cp_async_commit();
        for (int64_t g = 0; g < ngroups; ++g) {
            if (g + 1 < ngroups) stage_group(g + 1);
            cp_async_commit();
            cp_async_wait1();
            const int64_t base = 1 + g * BT + BT;                 // padded index of lag 1 + g BT
            float2 W1[2 * BT - 1], W2[2 * BT - 1], Q1[2 * BT - 1], Q2[2 * BT - 1], X1[BT], X2[BT];
#pragma unroll
            for (int t = 0; t < 2 * BT - 1; ++t) {
                W1[t] = __ldg(wa1 + base + t);
                W2[t] = __ldg(wa2 + base + t);
                Q1[t] = __ldg(qa1 + base + t);
                Q2[t] = __ldg(qa2 + base + t);
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
                    acc_prod(W1[j + b].x, W1[j + b].y, X1[j].x, X1[j].y, ar1[b], er1[b]);
                    acc_prod(W2[j + b].x, W2[j + b].y, X2[j].x, X2[j].y, ar2[b], er2[b]);
                    acc_prod(Q1[j + b].x, Q1[j + b].y, X1[j].x, X1[j].y, aq1[b], eq1[b]);
                    acc_prod(Q2[j + b].x, Q2[j + b].y, X2[j].x, X2[j].y, aq2[b], eq2[b]);
                }
        }
        float2 u1[BT], u2[BT];
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int64_t m = mhi - b;
            if (m < 1) break;
            float h1 = ar1[b], f1 = er1[b], h2 = ar2[b], f2 = er2[b];
            float k1 = aq1[b], z1 = eq1[b], k2 = aq2[b], z2 = eq2[b];
#pragma unroll
            for (int bb = 0; bb < b; ++bb) {
                const float2 w1 = __ldg(wa1 + (b - bb) + BT), w2 = __ldg(wa2 + (b - bb) + BT);
                const float2 v1 = __ldg(qa1 + (b - bb) + BT), v2 = __ldg(qa2 + (b - bb) + BT);
                acc_prod(w1.x, w1.y, u1[bb].x, u1[bb].y, h1, f1);
                acc_prod(w2.x, w2.y, u2[bb].x, u2[bb].y, h2, f2);
                acc_prod(v1.x, v1.y, u1[bb].x, u1[bb].y, k1, z1);
                acc_prod(v2.x, v2.y, u2[bb].x, u2[bb].y, k2, z2);
            }
            double b1 = -((double)h1 + (double)f1), b2 = -((double)h2 + (double)f2);
            if (m == N) {
                b1 -= r1;
                b2 -= r2;
            }
            const bool first = (P.scheme == CQ_BDF2 && m == 1);
            if (P.scheme == CQ_BE) {
                if (m < N) {
                    b1 += lp1_1 * it;
                    b2 += lp1_2 * it;
                }
            } else {
                if (m + 1 <= N) {
                    b1 += 2.0 * it * lp1_1;
                    b2 += 2.0 * it * lp1_2;
                }
                if (m + 2 <= N) {
                    b1 -= 0.5 * it * lp2_1;
                    b2 -= 0.5 * it * lp2_2;
                }
            }
            const double i11 = first ? M1.i11 : Mn.i11, i12 = first ? M1.i12 : Mn.i12;
            const double i21 = first ? M1.i21 : Mn.i21, i22 = first ? M1.i22 : Mn.i22;
            const double l1 = i11 * b1 + i12 * b2;
            const double l2 = i21 * b1 + i22 * b2;
            const double v1 = c * l1 - a * l2, v2 = -a * l1 + c * l2;
            u1[b] = df_of(v1);
            u2[b] = df_of(v2);
            m4[m * nm + mode] = make_float4(u1[b].x, u1[b].y, u2[b].x, u2[b].y);
            // hq^m: the d' history plus the n = m term d'_0 mu^m, against the forward level x^m
            const double hq1 = fma(__ldg(q1), v1, (double)k1 + (double)z1);
            const double hq2 = fma(__ldg(q2), v2, (double)k2 + (double)z2);
            const float4 xm = h4[m * nm + mode];
            db1 = fma((double)xm.x + (double)xm.y, hq1, db1);
            db2 = fma((double)xm.z + (double)xm.w, hq2, db2);
            if (m >= 2) {
                sg1 = fma(__ldg(d1 + m - 1), v1, sg1);
                sg2 = fma(__ldg(d2 + m - 1), v2, sg2);
                sx1 = fma(__ldg(q1 + m - 1), v1, sx1);
                sx2 = fma(__ldg(q2 + m - 1), v2, sx2);
            }
            if (m == 1) {
                lam1_1 = l1;
                lam1_2 = l2;
                mu1_1 = v1;
                mu1_2 = v2;
            } else if (m == 2) {
                lam2_1 = l1;
                lam2_2 = l2;
            }
            lp2_1 = lp1_1;
            lp2_2 = lp1_2;
            lp1_1 = l1;
            lp1_2 = l2;
        }
    }
    const float4 x0 = h4[mode];
    const double x01 = (double)x0.x + (double)x0.y, x02 = (double)x0.z + (double)x0.w;
    double g1, g2;
    if (P.scheme == CQ_BE) {
        g1 = -lam1_1 * it;
        g2 = -lam1_2 * it;
    } else {
        g1 = -lam1_1 * it + d10 * mu1_1 / 3.0 + 0.5 * it * lam2_1 + 0.5 * sg1;
        g2 = -lam1_2 * it + d20 * mu1_2 / 3.0 + 0.5 * it * lam2_2 + 0.5 * sg2;
        const float4 xx = h4[nm + mode];
        const double x11 = (double)xx.x + (double)xx.y, x12 = (double)xx.z + (double)xx.w;
        db1 += mu1_1 * __ldg(q1) * (x01 - x11) / 3.0 + 0.5 * x01 * sx1;
        db2 += mu1_2 * __ldg(q2) * (x02 - x12) / 3.0 + 0.5 * x02 * sx2;
    }
    if (active) {
        gx0[mode] = ldexp(g1, ey);
        gx0[nm + mode] = ldexp(g2, ey);
        db1 = ldexp(db1, exf + ey);
        db2 = ldexp(db2, exf + ey);
    } else {
        db1 = db2 = 0.0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Jpart += __shfl_xor_sync(0xffffffffu, Jpart, off);
        db1 += __shfl_xor_sync(0xffffffffu, db1, off);
        db2 += __shfl_xor_sync(0xffffffffu, db2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + 0, Jpart);
        atomicAdd(acc + 1, db1);
        atomicAdd(acc + 2, db2);
    }
    if (active && !ok) atomicAdd(acc + 3, 1.0);
}

int direct_df_grad_tables(int64_t N, const double *d1, const double *d2, const double *q1, const double *q2,
                          float2 *wa1, float2 *wa2, float2 *qa1, float2 *qa2, cudaStream_t s) {
    const int64_t len = N + 4 * kAdjDfBT;
    const unsigned g = (unsigned)((len + 255) / 256);
    k_pad_df<<<g, 256, 0, s>>>(d1, N, kAdjDfBT, len, wa1);
    k_pad_df<<<g, 256, 0, s>>>(d2, N, kAdjDfBT, len, wa2);
    k_pad_df<<<g, 256, 0, s>>>(q1, N, kAdjDfBT, len, qa1);
    k_pad_df<<<g, 256, 0, s>>>(q2, N, kAdjDfBT, len, qa2);
    return launched(4);
}

int direct_df_gradient_slice(const Fp2sParams &P, double wd, const double *lam, const double *g0, double *gN,
                             int *status, const double *d1, const double *d2, const double *q1, const double *q2,
                             const float2 *wz1, const float2 *wz2, const float2 *wa1, const float2 *wa2,
                             const float2 *qa1, const float2 *qa2, float2 *hist, const double *tgt, int vjp,
                             float2 *mu, double *gx0, double *acc, cudaStream_t s) {
    const unsigned blocks = (unsigned)((P.nmodes + 31) / 32);
    // the zero levels N + 1 .. N + BT that pad the adjoint's last group of future levels
    if (cudaMemsetAsync(mu + (size_t)(P.N + 1) * P.nmodes * 2, 0, (size_t)kAdjDfBT * P.nmodes * 2 * sizeof(float2),
                        s) != cudaSuccess)
        return CQ_ECUDA;
    k_fp2s_direct_df<kDirDfBT><<<blocks, 32, 0, s>>>(P, lam, g0, gN, status, d1, d2, wz1, wz2, hist);
    k_adjoint_direct_df<kAdjDfBT><<<blocks, 32, 0, s>>>(P, wd, lam, g0, d1, d2, q1, q2, wa1, wa2, qa1, qa2, hist, gN,
                                                        tgt, vjp, mu, gx0, acc);
    return launched(2);
}

int direct_df_tables(const Fp2sParams &P, const double *d1, const double *d2, float2 *wz1, float2 *wz2,
                     cudaStream_t s) {
    const unsigned g = (unsigned)((P.N + 2 * kDirDfBT + 256) / 256);
    k_pad_df<<<g, 256, 0, s>>>(d1, P.N, kDirDfBT, P.N + 2 * kDirDfBT + 1, wz1);
    k_pad_df<<<g, 256, 0, s>>>(d2, P.N, kDirDfBT, P.N + 2 * kDirDfBT + 1, wz2);
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
