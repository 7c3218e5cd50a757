// Fused fast solve with FP64-class accuracy on the FP32 pipe (precision form CQ_DF64).
//
// The fast history (recurrences after Eq. 3.10 for BE, after Eq. 3.18 for SBD;
// Remarks 4.1 and 4.7) dominates the fast solve: per mode-state and step, every
// Gauss-Jacobi node j updates Y_j = r_j Y_j + G^{n-L} and adds c_j Y_j to h^n. In
// FP64 that is two DFMAs per node, and on GB300 the FP64 pipe runs at 1/64 of the
// FP32 rate. Here each Y_j, each table entry and the history sum are double-float
// values (an unevaluated sum hi + lo of two FP32 numbers: Dekker's TwoProduct in
// its FMA form and Knuth's TwoSum), so the node work runs on the FP32 pipe at about
// 27 FP32 operations per node instead of 2 DFMAs (128 FP64-pipe cycles per warp).
// The 2x2 step of Eq. 4.1 / 4.7 stays in FP64 (a few DFMAs per step).
//
// Two points keep the error at the level of the FP64 form:
//  * The ratios of the slow nodes are held as u_j = 1 - r_j and the update is
//    Y = Y - u_j Y + G. A ratio near 1 held as hi + lo is off by up to ~2^-49 in
//    absolute terms, i.e. by 2^-49 / u_j relative to u_j, and the geometric sum
//    repeats that error every step over ~1/u_j steps; in the u form the error is
//    relative to u_j itself. The nodes are ranked by r on the device and the top
//    quarter of the slots take this form.
//  * All error-free transformations use the non-contracting intrinsics
//    (__fadd_rn, __fmul_rn, __fmaf_rn): a product fused into a later addition by
//    the compiler would break them.
//
// Each mode is pre-scaled by an exact power of two (from its G^0) and rescaled by
// another power of two whenever its level leaves [2^-40, 2^40], so that the FP32
// exponent range is never reached; the exponent is carried in an integer and
// applied on output. Layout and lane roles as the FP64 kernel: lane l < 16 of a warp
// carries state 1 and lane l + 16 state 2 of the same mode; the node states of a
// lane live in registers (the top 80 slots: 160 registers; for NP > 80, a compile-time bound
// of at most 128, the fastest-decaying NP - 80 slots in shared memory, column tid), the last L
// levels in a per-lane ring in shared memory. Measured on the 2D 255 x 255 grid
// (80 points, N = 4096): holding half of the node states in shared memory to fit three
// warps per scheduler was slower (80 against 58 ms), as was a loop body with the node
// part and the window behind branches (76 ms): the FP64 step is a long dependency chain
// that needs the node work of the next step in the same basic block to hide it.
#include <algorithm>

#include "fastdf.cuh"
#include "fastgrad.cuh"

namespace fastcq {

// ---------------------------------------------------------------------------
// Tables of one problem: one block of 256 threads.
// ---------------------------------------------------------------------------
__global__ void k_df_tables(int NP, int np, int L, int64_t N, const double *__restrict__ tab1,
                            const double *__restrict__ tab2, const double *__restrict__ d1,
                            const double *__restrict__ d2, float *__restrict__ out) {
    df_tables_fill(NP, np, L, N, tab1, tab2, d1, d2, out, threadIdx.x, blockDim.x);
}

// One problem: 16 modes per warp, every block runs all N steps of its 64 modes (HIST: every level
// also stored, for the fast-form gradient).
template <int NP, bool BE, int WL, bool HIST>
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks)
    k_fp2s_fast_df(Fp2sParams P, const double *__restrict__ lam, const double *__restrict__ g0,
                   double *__restrict__ gN, int *__restrict__ status, const double *__restrict__ d1,
                   const double *__restrict__ d2, const float *__restrict__ dftab, double *__restrict__ hist) {
    constexpr int KS = df_smem_slots(NP);
    extern __shared__ __align__(16) float smd[];
    const int L = P.L, T = blockDim.x, tid = threadIdx.x;
    float2 *R = reinterpret_cast<float2 *>(smd + df_table_floats(NP));      // [L][T]
    float2 *Ys = R + (size_t)L * T;                                          // [KS][T]
    for (int e = tid; e < df_table_floats(NP); e += T) smd[e] = dftab[e];
    for (int j = 0; j < L; ++j) R[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
    for (int j = 0; j < KS; ++j) Ys[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
    __syncthreads();
    const int64_t mode_raw = ((int64_t)blockIdx.x * (T >> 5) + (tid >> 5)) * kFastModesPerWarp + (tid & 15);
    df_solve_lane<NP, BE, WL, HIST>(P, lam, g0, gN, status, d1, d2, reinterpret_cast<const float4 *>(smd),
                                    reinterpret_cast<const float2 *>(smd + 8 * NP), R, Ys, T, tid, mode_raw,
                                    P.nmodes, hist);
}

static size_t df_smem_bytes(int NP, int L) {
    return (size_t)df_table_floats(NP) * sizeof(float) + (size_t)(L + df_smem_slots(NP)) * kDfThreads * sizeof(float2);
}

int df_np_bound(int np) { return df_np_class(np); }

int fast_df_tables(const Fp2sParams &P, const double *tab1, const double *tab2, const double *d1, const double *d2,
                   float *out, cudaStream_t s) {
    const int NP = df_np_bound(P.np);
    if (NP == 0 || df_table_floats(NP) > kDfTabFloats) return CQ_EUNSUPPORTED;
    k_df_tables<<<1, 256, 0, s>>>(NP, P.np, P.L, P.N, tab1, tab2, d1, d2, out);
    return launched();
}

// Every warp runs all N steps of its 16 modes, so a launch takes ceil(blocks / (SMs x CTAs per
// SM)) equal rounds. The number of resident CTAs per SM is chosen (by padding the dynamic shared
// memory, at most the register limit) to make the last round as full as possible: e.g. 1355
// blocks of 96 threads would take 3 rounds of 456 blocks at 3 CTAs per SM (99 % full) against
// 3 rounds of 608 at 4 (74 %). The rounds' fullness is weighed against the issue rate, modelled
// as saturating at two warps per scheduler.
template <int NP, bool BE, int WL, bool HIST>
static int launch_df_kernel(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                            const double *d1, const double *d2, const float *dftab, double *hist, cudaStream_t s) {
    auto kern = k_fp2s_fast_df<NP, BE, WL, HIST>;
    const int64_t mpb = (int64_t)(kDfThreads / 32) * kFastModesPerWarp;
    const int64_t blocks = (P.nmodes + mpb - 1) / mpb;
    const size_t base = df_smem_bytes(NP, P.L);
    int dev = 0, sm_smem = 0, reserved = 0, max_block = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return CQ_ECUDA;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_block) != cudaSuccess)
        return CQ_ECUDA;
    int fit = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, kDfThreads, base) != cudaSuccess || fit < 1)
        return CQ_EUNSUPPORTED;
    // score = fullness of the rounds x issue rate, modelled as saturating at two warps per
    // scheduler (eight per SM)
    const int64_t sms = device_sms();
    int best = fit;
    double best_score = -1.0;
    for (int c = fit; c >= 1; --c) {
        const int64_t round = sms * c, rounds = (blocks + round - 1) / round;
        const double eff = (double)blocks / (double)(rounds * round);
        const double rate = std::min(1.0, (double)(c * kDfThreads / 32) / 8.0);
        if (eff * rate > best_score + 0.02) {
            best_score = eff * rate;
            best = c;
        }
    }
    size_t smem = base;
    if (best < fit) {                            // pad so that exactly `best` CTAs fit per SM
        const size_t pad = (size_t)sm_smem / best - (size_t)reserved;
        smem = std::min<size_t>(std::max(base, pad / 128 * 128), (size_t)max_block);
    }
    kern<<<(unsigned)blocks, kDfThreads, smem, s>>>(P, lam, g0, gN, status, d1, d2, dftab, hist);
    return CQ_OK;
}

template <int NP, bool HIST>
static int launch_df(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                     const double *d1, const double *d2, const float *dftab, double *hist, cudaStream_t s) {
    if (P.scheme == CQ_BE) return launch_df_kernel<NP, true, 2, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
    if (P.L <= 17) return launch_df_kernel<NP, false, 17, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
    return launch_df_kernel<NP, false, kMaxNs, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
}

template <bool HIST>
static int fast_df_run(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                       const double *d1, const double *d2, const float *dftab, double *hist, cudaStream_t s) {
    switch (df_np_bound(P.np)) {
        case 16: return launch_df<16, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        case 32: return launch_df<32, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        case 48: return launch_df<48, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        case 64: return launch_df<64, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        case 80: return launch_df<80, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        case 96: return launch_df<96, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        case 112: return launch_df<112, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        case 128: return launch_df<128, HIST>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
        default: return CQ_EUNSUPPORTED;
    }
}

int fast_df_solve(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                  const double *d1, const double *d2, const float *dftab, cudaStream_t s) {
    return fast_df_run<false>(P, lam, g0, gN, status, d1, d2, dftab, nullptr, s);
}

int fast_df_solve_hist(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                       const double *d1, const double *d2, const float *dftab, double *hist, cudaStream_t s) {
    return fast_df_run<true>(P, lam, g0, gN, status, d1, d2, dftab, hist, s);
}

}  // namespace fastcq
