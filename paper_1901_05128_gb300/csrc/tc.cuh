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

// Operand forms: BF16 hi + lo (kind::f16) or TF32 hi + lo (kind::tf32, FP32 containers
// with the 13 low mantissa bits zero). A stage holds one 128-byte swizzle row per
// operand row: 64 BF16 or 32 TF32 levels.
enum : int { TC_BF16X3 = 0, TC_TF32X3 = 1 };
__host__ __device__ constexpr int kind_bk(int kind) { return kind == TC_TF32X3 ? 32 : 64; }
__host__ __device__ constexpr int kind_esize(int kind) { return kind == TC_TF32X3 ? 4 : 2; }
constexpr int BK = 64;                      // BF16 levels per stage (kind_bk(TC_BF16X3))

// Output rows are steps m in [n_lo, n_lo + rows); row m, column j of state s is
//   sum over levels k = k_lo + 1 .. kprime of  d^s_{m-k} * G[s * state_stride + j][k - 1]
// (terms with m - k < 1 are absent), j < ndof, written to H[(m - n_lo) * ldh + s * state_stride + j].
// k_lo is a multiple of 64.
struct TcParams {
    int64_t ndof, n_lo, rows, ldh;
    int num_i;                 // tiles along the steps
    int64_t delta0;            // delta of bank tile 0
    int kprime;                // levels k_lo + 1 .. kprime contribute
    int k_lo;
    int add;                   // FP32 output only: add to what H holds instead of overwriting
    int n_states;              // 1, or 2 (two weight sequences on two halves of the DOFs)
    int64_t ntile_state;       // DOF tiles per state
    int64_t state_stride;      // levels rows and output columns of state s start at s * state_stride
    int64_t max_ctas;          // 0: one CTA per output tile; else at most this many CTAs, each taking
                               // every max_ctas-th tile (for launches whose tiles have equal K)
    int *tile_counter;         // with max_ctas: a zeroed counter from which the CTAs claim tiles in
                               // order instead (tiles of unequal K); nullptr: the fixed order above
    int test_stall;            // failure-path test: each CTA withholds its first operand load
    unsigned long long wait_ns;  // limit of each wait between the CTA's roles; 0: the default (2 s)
};

// Tensor maps of one contraction: per state the Toeplitz bank (hi, lo); the levels (hi, lo).
struct TcMaps {
    CUtensorMap a_hi[2], a_lo[2], b_hi, b_lo;
};

}  // namespace tc

// Bank of Toeplitz tiles of the weights d_1..d_nw (index 0 and > nw read as 0):
// tile t, row r, column c = d_{delta0 + BK t + r - c} (BK = kind_bk(kind)), split into
// hi + lo of the kind's element type (128 x BK elements per tile).
int tc_bank(int kind, const double *d, int64_t nw, int64_t delta0, int ntiles, void *hi, void *lo, cudaStream_t s);
// Tensor map of a bank of ntiles tiles.
int tc_map_bank(int kind, CUtensorMap *m, const void *bank, int ntiles);
// Tensor map of K-major levels [rows][kpad] (kpad a multiple of 64).
int tc_map_levels(int kind, CUtensorMap *m, const void *levels, int64_t kpad, int64_t rows);
// Launch the contraction with FP32 output (timeouts recorded in *status).
int tc_contract_f32(int kind, const tc::TcMaps &maps, const tc::TcParams &P, float *H, int *status, cudaStream_t s);

}  // namespace fastcq
