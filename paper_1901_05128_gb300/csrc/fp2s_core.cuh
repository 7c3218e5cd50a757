// Per-mode algebra of the two-state schemes, shared by the single-problem
// kernels (fp2s.cu) and the batched persistent kernel (batch.cu).
#pragma once

#include "common.cuh"

namespace fastcq {

struct Fp2sParams {
    double a, tau, inv_tau;
    int64_t N, nmodes;
    int scheme, form, np, L;     // np Gauss-Jacobi points per state, L exact window (2 for BE)
    int prec;                    // CQ_F64; CQ_F32 or CQ_DF64 (fast form); CQ_BF16X3 or CQ_TF32X3 (direct)
};

// ---------------------------------------------------------------------------
// per-mode step algebra
// ---------------------------------------------------------------------------
struct Inv2 {
    double i11, i12, i21, i22;
};

__device__ __forceinline__ bool invert2(double A11, double A12, double A21, double A22, Inv2 &m) {
    const double det = A11 * A22 - A12 * A21;
    const double sc = fmax(fabs(A11 * A22), fabs(A12 * A21));
    const double id = 1.0 / det;
    m.i11 = A22 * id;
    m.i12 = -A12 * id;
    m.i21 = -A21 * id;
    m.i22 = A11 * id;
    return fabs(det) > 1e-14 * sc;
}

struct ModeConst {
    double c;                // a + lambda
    Inv2 Mn;                 // n >= 2 (BE: n >= 1)
    Inv2 M1;                 // SBD n = 1
};

__device__ __forceinline__ bool mode_setup(const Fp2sParams &P, double lam, double d10, double d20, ModeConst &mc) {
    const double c = P.a + lam;
    mc.c = c;
    const double lead = (P.scheme == CQ_BE) ? P.inv_tau : 1.5 * P.inv_tau;
    bool ok = invert2(lead + c * d10, -P.a * d20, -P.a * d10, lead + c * d20, mc.Mn);
    if (P.scheme == CQ_BDF2)
        ok &= invert2(P.inv_tau + (2.0 / 3.0) * c * d10, -(2.0 / 3.0) * P.a * d20, -(2.0 / 3.0) * P.a * d10,
                      P.inv_tau + (2.0 / 3.0) * c * d20, mc.M1);
    return ok;
}

// One time step of one mode given its histories h1, h2. gm1 = g^{n-1}, gm2 = g^{n-2}, gz = g^0.
__device__ __forceinline__ void mode_step(const Fp2sParams &P, const ModeConst &mc, int64_t n, double h1, double h2,
                                 double d10, double d20, double d1n, double d2n, double gm1_1, double gm1_2,
                                 double gm2_1, double gm2_2, double gz1, double gz2, double &x1, double &x2) {
    const double a = P.a, c = mc.c;
    double b1, b2;
    const Inv2 *M = &mc.Mn;
    if (P.scheme == CQ_BE) {
        b1 = gm1_1 * P.inv_tau - c * h1 + a * h2;
        b2 = gm1_2 * P.inv_tau - c * h2 + a * h1;
    } else if (n == 1) {
        b1 = gz1 * P.inv_tau - c * d10 * gz1 * (1.0 / 3.0) + a * d20 * gz2 * (1.0 / 3.0);
        b2 = gz2 * P.inv_tau - c * d20 * gz2 * (1.0 / 3.0) + a * d10 * gz1 * (1.0 / 3.0);
        M = &mc.M1;
    } else {
        const double e1 = fma(0.5 * d1n, gz1, h1);
        const double e2 = fma(0.5 * d2n, gz2, h2);
        b1 = (2.0 * gm1_1 - 0.5 * gm2_1) * P.inv_tau - c * e1 + a * e2;
        b2 = (2.0 * gm1_2 - 0.5 * gm2_2) * P.inv_tau - c * e2 + a * e1;
    }
    x1 = M->i11 * b1 + M->i12 * b2;
    x2 = M->i21 * b1 + M->i22 * b2;
}

// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (Dekker 1971, "A floating-point technique for extending the
// available precision"; Knuth's TwoSum). Products use the FMA form of
// Dekker's TwoProduct. About 44 significant bits, computed on the FP32 pipe.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_from(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ df df_fast_norm(float s, float e) {       // |s| >= |e|
    const float t = s + e;
    return {t, e - (t - s)};
}

__device__ __forceinline__ df two_sum(float a, float b) {       // exact: a + b = hi + lo
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return df_fast_norm(s, e + (a.lo + b.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return df_fast_norm(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    const float p = a.hi * b;
    const float e = fmaf(a.hi, b, -p);
    return df_fast_norm(p, fmaf(a.lo, b, e));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df df_shfl_xor16(df a) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, 16), __shfl_xor_sync(0xffffffffu, a.lo, 16)};
}

// Per-lane constants of the FP32-precision step: a lane carries state st of one
// mode (its partner lane, lane ^ 16, the other state). The step matrices are
// formed in FP64 and kept as double-float values.
struct LaneStep {
    double c, mn_oo, mn_ot, m1_oo, m1_ot, d_s0;
    df da, dc, dinv_tau, dmn_oo, dmn_ot, dm1_oo, dm1_ot, dd_s0_3;
};

__device__ __forceinline__ bool lane_step_setup(const Fp2sParams &P, double lam, double d10, double d20, int st,
                                                LaneStep &ls) {
    ModeConst mc;
    const bool ok = mode_setup(P, lam, d10, d20, mc);
    ls.c = mc.c;
    ls.d_s0 = st ? d20 : d10;
    ls.mn_oo = st ? mc.Mn.i22 : mc.Mn.i11;
    ls.mn_ot = st ? mc.Mn.i21 : mc.Mn.i12;
    ls.m1_oo = st ? mc.M1.i22 : mc.M1.i11;
    ls.m1_ot = st ? mc.M1.i21 : mc.M1.i12;
    ls.da = df_from(P.a);
    ls.dc = df_from(mc.c);
    ls.dinv_tau = df_from(P.inv_tau);
    ls.dmn_oo = df_from(ls.mn_oo);
    ls.dmn_ot = df_from(ls.mn_ot);
    ls.dm1_oo = df_from(ls.m1_oo);
    ls.dm1_ot = df_from(ls.m1_ot);
    ls.dd_s0_3 = df_from(ls.d_s0 * (1.0 / 3.0));
    return ok;
}

// One step of the lane's state from its FP32 history sum h (both lanes of a mode
// call it together: the states are exchanged with shuffles). gm1, gm2 = g^{n-1},
// g^{n-2} and gz = g^0 of the lane's state. dn: FP64 weights of the state;
// hd_hi/hd_lo: d_i / 2 of the state as double-float. The right-hand side and the
// 2x2 solve run in double-float arithmetic (FP32 pipe): FP32-rounded step
// coefficients would perturb the per-step amplification by ~1e-7, which compounds
// over the steps. solve64 selects FP64 instead (strong coupling, |a| > 10).
__device__ __forceinline__ df lane_step_df(const Fp2sParams &P, const LaneStep &ls, int solve64, int64_t n, float h,
                                           float gm1, float gm2, float gz, const double *__restrict__ dn,
                                           const float *__restrict__ hd_hi, const float *__restrict__ hd_lo) {
    if (solve64) {
        double e, lead, m_oo = ls.mn_oo, m_ot = ls.mn_ot;
        if (P.scheme == CQ_BE) {
            e = h;
            lead = (double)gm1 * P.inv_tau;
        } else if (n == 1) {
            e = ls.d_s0 * (double)gz * (1.0 / 3.0);
            lead = (double)gz * P.inv_tau;
            m_oo = ls.m1_oo;
            m_ot = ls.m1_ot;
        } else {
            e = fma(0.5 * __ldg(dn + n - 1), (double)gz, (double)h);
            lead = (2.0 * (double)gm1 - 0.5 * (double)gm2) * P.inv_tau;
        }
        const double e_o = __shfl_xor_sync(0xffffffffu, e, 16);
        const double b = lead - ls.c * e + P.a * e_o;
        const double b_o = __shfl_xor_sync(0xffffffffu, b, 16);
        return df_from(m_oo * b + m_ot * b_o);
    }
    df e, lead;
    df m_oo = ls.dmn_oo, m_ot = ls.dmn_ot;
    if (P.scheme == CQ_BE) {
        e = {h, 0.0f};
        lead = df_mul_f(ls.dinv_tau, gm1);
    } else if (n == 1) {
        e = df_mul_f(ls.dd_s0_3, gz);
        lead = df_mul_f(ls.dinv_tau, gz);
        m_oo = ls.dm1_oo;
        m_ot = ls.dm1_ot;
    } else {
        e = df_add(df_mul_f(df{__ldg(hd_hi + n - 1), __ldg(hd_lo + n - 1)}, gz), df{h, 0.0f});
        const df lin = df_add(df{2.0f * gm1, 0.0f}, df{-0.5f * gm2, 0.0f});
        lead = df_mul(ls.dinv_tau, lin);
    }
    const df e_o = df_shfl_xor16(e);
    const df b = df_add(df_add(lead, df_neg(df_mul(ls.dc, e))), df_mul(ls.da, e_o));
    const df b_o = df_shfl_xor16(b);
    return df_add(df_mul(m_oo, b), df_mul(m_ot, b_o));
}
// The same step rounded to one FP32 value.
__device__ __forceinline__ float lane_step(const Fp2sParams &P, const LaneStep &ls, int solve64, int64_t n, float h,
                                           float gm1, float gm2, float gz, const double *__restrict__ dn,
                                           const float *__restrict__ hd_hi, const float *__restrict__ hd_lo) {
    return lane_step_df(P, ls, solve64, n, h, gm1, gm2, gz, dn, hd_hi, hd_lo).hi;
}

// Two-term form of the FP32-precision step, for steps with the common matrix M
// (BE n >= 1; SBD n >= 2): with A = M^{-1} / tau and B = -M^{-1} K,
//     x^n = A l + B e,   l = g^{n-1} (BE) or 2 g^{n-1} - g^{n-2} / 2 (SBD),
//                        e = h (BE) or h + d_{n-1} g^0 / 2 (SBD).
// A and B are kept as double-float values and the four products are summed with
// error-free transformations: for slowly varying modes x^n differs from the terms
// by far less than their size, so FP32-rounded coefficients would act like a
// perturbed operator whose effect compounds over the steps.
struct LaneStep2 {
    float a_hi[2], a_lo[2];   // row s of A: [own state, other state]
    float b_hi[2], b_lo[2];   // row s of B
};

__device__ __forceinline__ void lane_step2_setup(const Fp2sParams &P, const LaneStep &ls, LaneStep2 &l2) {
    // row st of M^{-1}: (m_oo, m_ot) in the lane's own/other ordering; K = [[c, -a], [-a, c]]
    // is symmetric with equal diagonal, so row st of M^{-1} K is (m_oo c - m_ot a, -m_oo a + m_ot c)
    const double a_oo = ls.mn_oo * P.inv_tau, a_ot = ls.mn_ot * P.inv_tau;
    const double b_oo = -(ls.mn_oo * ls.c - ls.mn_ot * P.a), b_ot = -(-ls.mn_oo * P.a + ls.mn_ot * ls.c);
    const df x = df_from(a_oo), y = df_from(a_ot), u = df_from(b_oo), v = df_from(b_ot);
    l2.a_hi[0] = x.hi;
    l2.a_lo[0] = x.lo;
    l2.a_hi[1] = y.hi;
    l2.a_lo[1] = y.lo;
    l2.b_hi[0] = u.hi;
    l2.b_lo[0] = u.lo;
    l2.b_hi[1] = v.hi;
    l2.b_lo[1] = v.lo;
}

// x = A l + B e for the lane's state: (l, l_lo) and (l_o, l_o_lo) the double-float l
// of the lane's and the other state, (e, e_lo) and (e_o, e_o_lo) the history terms.
// The result as a normalised double-float pair (hi = its FP32 rounding).
__device__ __forceinline__ df lane_step2_df(const LaneStep2 &c, float l, float l_lo, float l_o, float l_o_lo, float e,
                                            float e_lo, float e_o, float e_o_lo) {
    const float p1 = c.a_hi[0] * l;
    float r = fmaf(c.a_hi[0], l, -p1);
    r = fmaf(c.a_hi[0], l_lo, fmaf(c.a_lo[0], l, r));
    const float p2 = c.a_hi[1] * l_o;
    r += fmaf(c.a_hi[1], l_o_lo, fmaf(c.a_lo[1], l_o, fmaf(c.a_hi[1], l_o, -p2)));
    const float p3 = c.b_hi[0] * e;
    r += fmaf(c.b_hi[0], e_lo, fmaf(c.b_lo[0], e, fmaf(c.b_hi[0], e, -p3)));
    const float p4 = c.b_hi[1] * e_o;
    r += fmaf(c.b_hi[1], e_o_lo, fmaf(c.b_lo[1], e_o, fmaf(c.b_hi[1], e_o, -p4)));
    const df s12 = two_sum(p1, p2), s34 = two_sum(p3, p4);
    const df s = two_sum(s12.hi, s34.hi);
    return df_fast_norm(s.hi, s.lo + ((s12.lo + s34.lo) + r));
}
__device__ __forceinline__ float lane_step2(const LaneStep2 &c, float l, float l_lo, float l_o, float l_o_lo, float e,
                                            float e_lo, float e_o, float e_o_lo) {
    return lane_step2_df(c, l, l_lo, l_o, l_o_lo, e, e_lo, e_o, e_o_lo).hi;
}

// Opaque register barrier: the value is kept as computed. Step coefficients formed in
// FP64 before a step loop pass through it; otherwise the compiler may recompute them
// inside the loop to save registers, which puts FP64 work (1/64 of the FP32 rate on
// this GPU) into every step.
__device__ __forceinline__ void keep_reg(float &v) { asm volatile("" : "+f"(v)); }
__device__ __forceinline__ void keep_reg(LaneStep2 &c) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        keep_reg(c.a_hi[i]);
        keep_reg(c.a_lo[i]);
        keep_reg(c.b_hi[i]);
        keep_reg(c.b_lo[i]);
    }
}

constexpr int kFastModesPerWarp = 16;     // a warp carries 16 modes x 2 states

// Fast solve in double-float (CQ_DF64, fastdf.cu): node bound for np points per state (0: more
// than it supports), its tables (from the FP64 tables r, c and the weights; kDfTabFloats floats)
// and the solve over all N steps.
constexpr int kDfTabFloats = 8 * 128 + 4 * kMaxNs;
int df_np_bound(int np);
int fast_df_tables(const Fp2sParams &P, const double *tab1, const double *tab2, const double *d1, const double *d2,
                   float *out, cudaStream_t s);
int fast_df_solve(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                  const double *d1, const double *d2, const float *dftab, cudaStream_t s);

// Direct solve in double-float (CQ_DIRECT with CQ_DF64, directdf.cu): time block, the padded
// double-float weights of both states (wz: n + 2 kDirDfBT + 1 entries (d1_hi, d2_hi, d1_lo,
// d2_lo)) and the solve over all N steps (hist: (N + 1) x nmodes entries (x1_hi, x2_hi, x1_lo,
// x2_lo)).
constexpr int kDirDfBT = 8;
int direct_df_tables(const Fp2sParams &P, const double *d1, const double *d2, float4 *wz, cudaStream_t s);
int direct_df_solve(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                    const double *d1, const double *d2, const float4 *wz, float4 *hist, cudaStream_t s);
// Its gradient (the discrete adjoint in double-float): time block of the adjoint, the padded
// weights d and d' of both states (wa, qa: N + 4 kAdjDfBT entries each, laid out as wz), and one
// slice of modes: forward solve with every level kept (hist), then the adjoint sweep (mu:
// (N + 1 + kAdjDfBT) x nmodes entries, laid out as hist), adding J, dJ/dbeta_1, dJ/dbeta_2 and a
// singular-step count to acc[0..3].
constexpr int kAdjDfBT = 4;
int direct_df_grad_tables(int64_t N, const double *d1, const double *d2, const double *q1, const double *q2,
                          float4 *wa, float4 *qa, cudaStream_t s);
int direct_df_gradient_slice(const Fp2sParams &P, double wd, const double *lam, const double *g0, double *gN,
                             int *status, const double *d1, const double *d2, const double *q1, const double *q2,
                             const float4 *wz, const float4 *wa, const float4 *qa, float4 *hist,
                             const double *tgt, int vjp, float4 *mu, double *gx0, double *acc, cudaStream_t s);

// Gradient of the fast form in FP64 (fastgrad.cu): der = (c'_j, c_j r'_j) of one state's tables
// tab = (r, c) at beta (tmp: 8 np doubles, gj_scratch: the table builder's 2 np), and the backward
// sweep over one slice of modes from the forward levels hist ((N + 1) x 2 x nmodes), adding J,
// dJ/dbeta_1, dJ/dbeta_2 and a singular-step count to acc[0..3] and writing dJ/dx^0 (modal) to gx0.
int fast_grad_tables(int scheme, double beta, double tau, int np1, int np2, int L, const double *tab,
                     double *gj_scratch, double *tmp, double *der, cudaStream_t s);
int fast_adjoint_slice(const Fp2sParams &P, double wd, const double *lam, const double *d1, const double *d2,
                       const double *q1, const double *q2, const double *tab1, const double *tab2,
                       const double *der1, const double *der2, const double *hist, const double *tgt, int vjp,
                       double *gx0, double *acc, cudaStream_t s);

// Mixed-precision direct solve (mixed.cu): workspace bytes of its own region, and
// the run over all N steps (weights, spectrum and the modal G^0 already in place;
// hdf: d_i / 2 of both states as double-float, [4][N + 1]).
size_t mixed_direct_bytes(const Fp2sParams &P);
int mixed_direct_run(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                     const double *d1, const double *d2, const float *hdf, void *region, cudaStream_t s);
// Its gradient (discrete adjoint): the forward solve with every level kept, the
// weight-derivative contraction and the reversed-time adjoint sweep. q1, q2: d(d_i)/d(beta);
// tgt: the modal target (misfit) or dL/dx^N (vjp); writes the modal dJ/dx^0 to gx0 and
// adds J, dJ/dbeta_1, dJ/dbeta_2 to acc[0..2].
size_t mixed_grad_bytes(const Fp2sParams &P);
int mixed_grad_run(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                   const double *d1, const double *d2, const double *q1, const double *q2, const float *hdf,
                   const double *tgt, int vjp, double wd, double *gx0, double *acc, void *region, cudaStream_t s);

}  // namespace fastcq
