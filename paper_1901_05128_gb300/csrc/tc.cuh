// Interface of the tcgen05 BF16x3 causal contraction (history_tc.cu) for its
// users inside the library: the direct history entry point and the mixed
// precision direct solve.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace fastcq {
namespace tc {

constexpr int BM = 128;                     // steps per tile (UMMA M)
constexpr int BN = 256;                     // DOFs per tile (UMMA N)
constexpr int BK = 64;                      // levels per stage (one 128-byte swizzle row of BF16)

// Output rows are steps m in [n_lo, n_lo + rows); row m, column j of state s is
//   sum over levels k = 1 .. kprime of  d^s_{m-k} * G[s * state_stride + j][k - 1]
// (terms with m - k < 1 are absent), j < ndof, written to H[(m - n_lo) * ldh + s * state_stride + j].
struct TcParams {
    int64_t ndof, n_lo, rows, ldh;
    int vec2;                  // output rows 16-byte aligned: vector stores
    int num_i;                 // tiles along the steps
    int64_t delta0;            // delta of bank tile 0
    int kprime;                // levels 1 .. kprime contribute
    int n_states;              // 1, or 2 (two weight sequences on two halves of the DOFs)
    int64_t ntile_state;       // DOF tiles per state
    int64_t state_stride;      // levels rows and output columns of state s start at s * state_stride
};

// Tensor maps of one contraction: per state the Toeplitz bank (hi, lo); the levels (hi, lo).
struct TcMaps {
    CUtensorMap a_hi[2], a_lo[2], b_hi, b_lo;
};

}  // namespace tc

// Bank of Toeplitz tiles of the weights d_1..d_nw (index 0 and > nw read as 0):
// tile t, row r, column c = d_{delta0 + 64 t + r - c}, split into BF16 hi + lo.
int tc_bank(const double *d, int64_t nw, int64_t delta0, int ntiles, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
            cudaStream_t s);
// Tensor map of a bank of ntiles tiles.
int tc_map_bank(CUtensorMap *m, const __nv_bfloat16 *bank, int ntiles);
// Tensor map of K-major levels [rows][kpad] (kpad a multiple of 64).
int tc_map_levels(CUtensorMap *m, const __nv_bfloat16 *levels, int64_t kpad, int64_t rows);
// Launch the contraction with FP32 output (timeouts recorded in *status).
int tc_contract_f32(const tc::TcMaps &maps, const tc::TcParams &P, float *H, int *status, cudaStream_t s);

}  // namespace fastcq
