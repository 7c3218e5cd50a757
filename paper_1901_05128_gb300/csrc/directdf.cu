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
// issued instruction, 47 % issue). The in-block terms follow step by step with the steps. The two
// states of a mode share every level index and weight lag, so their terms run as one packed
// two-wide double-float multiply-add (acc_prod2: Blackwell's FADD2 / FMUL2 / FFMA2, component k
// = state k + 1), which halves the issued instructions. Levels and weights are stored with the
// two states' high parts side by side and then their low parts (16 bytes):
// hist[k * nmodes + mode] = (x1_hi, x2_hi, x1_lo, x2_lo), wz[i] = (d1_hi, d2_hi, d1_lo, d2_lo).
#include "fastdf.cuh"

namespace fastcq {

// wz[i] = d_{i - BT} of both states as (d1_hi, d2_hi, d1_lo, d2_lo) for 1 <= i - BT <= n, else
// zero; i = 0 .. len - 1.
__global__ void k_pad_df(const double *__restrict__ d1, const double *__restrict__ d2, int64_t n, int BT, int64_t len,
                         float4 *__restrict__ wz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const int64_t idx = i - BT;
    if (idx >= 1 && idx <= n) {
        const float2 a = df_of(d1[idx]), b = df_of(d2[idx]);
        wz[i] = make_float4(a.x, b.x, a.y, b.y);
    } else {
        wz[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

// 16-byte asynchronous copy global -> shared through L2 (cp.async.cg: the levels were written
// by plain stores of the same thread, which L2 holds), and its groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ float2 lo_half(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 hi_half(float4 v) { return make_float2(v.x, v.y); }

template <int BT>
__global__ void __launch_bounds__(32, 16)
    k_fp2s_direct_df(Fp2sParams P, const double *__restrict__ lam, const double *__restrict__ g0,
                     double *__restrict__ gN, int *__restrict__ status, const double *__restrict__ d1,
                     const double *__restrict__ d2, const float4 *__restrict__ wz, float4 *__restrict__ h4) {
    const int64_t nm = P.nmodes;
    const int64_t mode = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nm) return;
    // per-mode power-of-two scale from max(|g1^0|, |g2^0|)
    const double gz1r = g0[mode], gz2r = g0[nm + mode];
    const double gmax = fmax(fabs(gz1r), fabs(gz2r));
    int ex = 0;
    if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &ex);
    const double gz1 = ldexp(gz1r, -ex), gz2 = ldexp(gz2r, -ex);
    {
        const float2 a = df_of(gz1), b = df_of(gz2);
        h4[mode] = make_float4(a.x, b.x, a.y, b.y);        // level k of the mode at h4[k * nm + mode]
    }
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    ModeConst mc;
    if (!mode_setup(P, lam[mode], d10, d20, mc)) atomicOr(status, ST_SINGULAR);
    double gm1_1 = gz1, gm1_2 = gz2, gm2_1 = 0.0, gm2_2 = 0.0;
    const float4 *hb = h4 + mode;
    constexpr int kStages = 3;
    __shared__ float4 sxs[kStages * BT * 32];                // [stage][level j][lane]
    float4 *sx = sxs + (threadIdx.x & 31);
    for (int64_t n0 = 1; n0 <= P.N; n0 += BT) {
        float2 ah[BT], al[BT];                               // row b: (state 1, state 2) hi / lo
#pragma unroll
        for (int b = 0; b < BT; ++b) ah[b] = al[b] = make_float2(0.0f, 0.0f);
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
            float4 W[2 * BT - 1], X[BT];
#pragma unroll
            for (int t = 0; t < 2 * BT - 1; ++t) W[t] = __ldg(wz + base + t + BT);
            const float4 *xg = sx + (int)(g % kStages) * BT * 32;
#pragma unroll
            for (int j = 0; j < BT; ++j) X[j] = xg[j * 32];
#pragma unroll
            for (int j = 0; j < BT; ++j)
#pragma unroll
                for (int b = 0; b < BT; ++b) {
                    const float4 w = W[BT - 1 + b - j];
                    acc_prod2(hi_half(w), lo_half(w), hi_half(X[j]), lo_half(X[j]), ah[b], al[b]);
                }
        }
        // the block's own steps
        float2 lh[BT], ll[BT];                               // the block's levels, (state 1, state 2)
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int64_t n = n0 + b;
            if (n > P.N) break;
            float2 h = ah[b], e = al[b];
#pragma unroll
            for (int kk = 0; kk < b; ++kk) {
                const float4 w = __ldg(wz + (b - kk) + BT);
                acc_prod2(hi_half(w), lo_half(w), lh[kk], ll[kk], h, e);
            }
            double d1n = 0.0, d2n = 0.0;
            if (P.scheme == CQ_BDF2 && n >= 2) {
                d1n = __ldg(d1 + n - 1);
                d2n = __ldg(d2 + n - 1);
            }
            double x1, x2;
            mode_step(P, mc, n, (double)h.x + (double)e.x, (double)h.y + (double)e.y, d10, d20, d1n, d2n, gm1_1,
                      gm1_2, gm2_1, gm2_2, gz1, gz2, x1, x2);
            const float2 a = df_of(x1), c = df_of(x2);
            lh[b] = make_float2(a.x, c.x);
            ll[b] = make_float2(a.y, c.y);
            h4[n * nm + mode] = make_float4(a.x, c.x, a.y, c.y);
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
// staged in shared memory with cp.async as in the forward kernel), both states of a mode in one
// packed two-wide multiply-add per term and weight sequence. Everything that scales with the
// adjoint variables is scaled by the power of two of the terminal condition; the forward levels
// carry the forward's scale; both are undone in the per-mode sums at the end.
// mu[n * nm + mode] = (mu1_hi, mu2_hi, mu1_lo, mu2_lo) for n = 1 .. N + BT, the levels past N zero
// (the caller clears them); wa / qa: d and d' of both states padded (k_pad_df, length N + 4 BT).
// ---------------------------------------------------------------------------
template <int BT>
__global__ void __launch_bounds__(32, 16)
    k_adjoint_direct_df(Fp2sParams P, double wd, const double *__restrict__ lam, const double *__restrict__ g0,
                        const double *__restrict__ d1, const double *__restrict__ d2,
                        const double *__restrict__ q1, const double *__restrict__ q2,
                        const float4 *__restrict__ wa, const float4 *__restrict__ qa,
                        const float4 *__restrict__ h4, const double *__restrict__ gN,
                        const double *__restrict__ tgt, int vjp, float4 *__restrict__ m4,
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
        // row b: the d-history (ar, er) and the d'-history (aq, eq) of (state 1, state 2)
        float2 ar[BT], er[BT], aq[BT], eq[BT];
#pragma unroll
        for (int b = 0; b < BT; ++b) ar[b] = er[b] = aq[b] = eq[b] = make_float2(0.0f, 0.0f);
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
            float4 W[2 * BT - 1], Q[2 * BT - 1], X[BT];
#pragma unroll
            for (int t = 0; t < 2 * BT - 1; ++t) {
                W[t] = __ldg(wa + base + t);
                Q[t] = __ldg(qa + base + t);
            }
            const float4 *xg = sx + (int)(g % kStages) * BT * 32;
#pragma unroll
            for (int j = 0; j < BT; ++j) X[j] = xg[j * 32];
#pragma unroll
            for (int j = 0; j < BT; ++j)
#pragma unroll
                for (int b = 0; b < BT; ++b) {
                    acc_prod2(hi_half(W[j + b]), lo_half(W[j + b]), hi_half(X[j]), lo_half(X[j]), ar[b], er[b]);
                    acc_prod2(hi_half(Q[j + b]), lo_half(Q[j + b]), hi_half(X[j]), lo_half(X[j]), aq[b], eq[b]);
                }
        }
        float2 uh[BT], ul[BT];                               // the block's adjoint levels mu, hi / lo
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int64_t m = mhi - b;
            if (m < 1) break;
            float2 h = ar[b], f = er[b], k = aq[b], z = eq[b];
#pragma unroll
            for (int bb = 0; bb < b; ++bb) {
                const float4 w = __ldg(wa + (b - bb) + BT), v = __ldg(qa + (b - bb) + BT);
                acc_prod2(hi_half(w), lo_half(w), uh[bb], ul[bb], h, f);
                acc_prod2(hi_half(v), lo_half(v), uh[bb], ul[bb], k, z);
            }
            double b1 = -((double)h.x + (double)f.x), b2 = -((double)h.y + (double)f.y);
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
            const float2 p1 = df_of(v1), p2 = df_of(v2);
            uh[b] = make_float2(p1.x, p2.x);
            ul[b] = make_float2(p1.y, p2.y);
            m4[m * nm + mode] = make_float4(p1.x, p2.x, p1.y, p2.y);
            // hq^m: the d' history plus the n = m term d'_0 mu^m, against the forward level x^m
            const double hq1 = fma(__ldg(q1), v1, (double)k.x + (double)z.x);
            const double hq2 = fma(__ldg(q2), v2, (double)k.y + (double)z.y);
            const float4 xm = h4[m * nm + mode];
            db1 = fma((double)xm.x + (double)xm.z, hq1, db1);
            db2 = fma((double)xm.y + (double)xm.w, hq2, db2);
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
    const double x01 = (double)x0.x + (double)x0.z, x02 = (double)x0.y + (double)x0.w;
    double g1, g2;
    if (P.scheme == CQ_BE) {
        g1 = -lam1_1 * it;
        g2 = -lam1_2 * it;
    } else {
        g1 = -lam1_1 * it + d10 * mu1_1 / 3.0 + 0.5 * it * lam2_1 + 0.5 * sg1;
        g2 = -lam1_2 * it + d20 * mu1_2 / 3.0 + 0.5 * it * lam2_2 + 0.5 * sg2;
        const float4 xx = h4[nm + mode];
        const double x11 = (double)xx.x + (double)xx.z, x12 = (double)xx.y + (double)xx.w;
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
                          float4 *wa, float4 *qa, cudaStream_t s) {
    const int64_t len = N + 4 * kAdjDfBT;
    const unsigned g = (unsigned)((len + 255) / 256);
    k_pad_df<<<g, 256, 0, s>>>(d1, d2, N, kAdjDfBT, len, wa);
    k_pad_df<<<g, 256, 0, s>>>(q1, q2, N, kAdjDfBT, len, qa);
    return launched(2);
}

int direct_df_gradient_slice(const Fp2sParams &P, double wd, const double *lam, const double *g0, double *gN,
                             int *status, const double *d1, const double *d2, const double *q1, const double *q2,
                             const float4 *wz, const float4 *wa, const float4 *qa, float4 *hist,
                             const double *tgt, int vjp, float4 *mu, double *gx0, double *acc, cudaStream_t s) {
    const unsigned blocks = (unsigned)((P.nmodes + 31) / 32);
    // the zero levels N + 1 .. N + BT that pad the adjoint's last group of future levels
    if (cudaMemsetAsync(mu + (size_t)(P.N + 1) * P.nmodes, 0, (size_t)kAdjDfBT * P.nmodes * sizeof(float4), s) !=
        cudaSuccess)
        return CQ_ECUDA;
    k_fp2s_direct_df<kDirDfBT><<<blocks, 32, 0, s>>>(P, lam, g0, gN, status, d1, d2, wz, hist);
    k_adjoint_direct_df<kAdjDfBT><<<blocks, 32, 0, s>>>(P, wd, lam, g0, d1, d2, q1, q2, wa, qa, hist, gN, tgt, vjp,
                                                        mu, gx0, acc);
    return launched(2);
}

int direct_df_tables(const Fp2sParams &P, const double *d1, const double *d2, float4 *wz, cudaStream_t s) {
    const unsigned g = (unsigned)((P.N + 2 * kDirDfBT + 256) / 256);
    k_pad_df<<<g, 256, 0, s>>>(d1, d2, P.N, kDirDfBT, P.N + 2 * kDirDfBT + 1, wz);
    return launched();
}

int direct_df_solve(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                    const double *d1, const double *d2, const float4 *wz, float4 *hist, cudaStream_t s) {
    // one-warp blocks spread the modes evenly over the SMs (every block runs all N steps)
    const unsigned blocks = (unsigned)((P.nmodes + 31) / 32);
    k_fp2s_direct_df<kDirDfBT><<<blocks, 32, 0, s>>>(P, lam, g0, gN, status, d1, d2, wz, hist);
    return CQ_OK;
}

}  // namespace fastcq
