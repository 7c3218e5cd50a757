// Per-mode algebra of the two-state schemes, shared by the single-problem
// kernels (fp2s.cu) and the batched persistent kernel (batch.cu).
#pragma once

#include "common.cuh"

namespace fastcq {

struct Fp2sParams {
    double a, tau, inv_tau;
    int64_t N, nmodes;
    int scheme, form, np, L;     // np Gauss-Jacobi points per state, L exact window (2 for BE)
    int prec;                    // CQ_F64 or CQ_F32 (fast form only)
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

constexpr int kFastModesPerWarp = 16;     // a warp carries 16 modes x 2 states

}  // namespace fastcq
