// The double-float backward sweep of the fast-form gradient (fastgrad.cu; fp2s_gradient /
// fp2s_vjp with CQ_FAST and CQ_DF64, np1 + np2 <= 128): its tables (kAdjDfTabFloats floats:
// ranked node pairs of (r or 1 - r, c, c', c r') and the window d, d' as hi + lo pairs), and the
// sweep over one slice of modes from the forward levels hist ((N + 1) x 2 x nmodes), adding
// J, dJ/dbeta_1, dJ/dbeta_2 and a singular-step count to acc[0..3] and writing dJ/dx^0 to gx0.
#pragma once

#include "fp2s_core.cuh"

namespace fastcq {

constexpr int kAdjDfTabFloats = 16 * 128 + 8 * kMaxNs;
int fast_adjoint_df_tables(const Fp2sParams &P, const double *tab1, const double *tab2, const double *der1,
                           const double *der2, const double *d1, const double *d2, const double *q1,
                           const double *q2, float *out, cudaStream_t s);
// The double-float fast solve (fastdf.cu) with every level stored in true units:
// hist[(n * 2 + s) * nmodes + mode], n = 0 .. N (the forward sweep of this gradient).
int fast_df_solve_hist(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                       const double *d1, const double *d2, const float *dftab, double *hist, cudaStream_t s);
int fast_adjoint_df_slice(const Fp2sParams &P, double wd, const double *lam, const double *d1, const double *d2,
                          const double *q1, const double *q2, const float *adtab, const double *hist,
                          const double *tgt, int vjp, double *gx0, double *acc, cudaStream_t s);

}  // namespace fastcq
