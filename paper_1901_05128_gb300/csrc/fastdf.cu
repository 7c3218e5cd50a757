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

#include "common.cuh"
#include "fp2s_core.cuh"

namespace fastcq {

constexpr int kDfThreads = 128;       // four warps per CTA
constexpr int kDfMinBlocks = 2;       // two CTAs per SM: two warps per scheduler, up to 255 registers

// Slots of the u form (the slowest-decaying nodes): the top quarter.
__host__ __device__ constexpr int df_u_slots(int NP) { return NP / 4; }

// Node slots held in registers (the top ones: the slowest nodes, u form included); the bottom
// NP - kDfRegSlots slots (fast-decaying, r form) live in shared memory, column tid.
constexpr int kDfRegSlots = 80;
__host__ __device__ constexpr int df_smem_slots(int NP) { return NP > kDfRegSlots ? NP - kDfRegSlots : 0; }

// Floats of the kernel's table: [NP][2] float4 (a_hi, a_lo, c_hi, c_lo) with a = r or
// a = 1 - r, then [kMaxNs][2] float2 window weights d_i.
__host__ __device__ constexpr int df_table_floats(int NP) { return 8 * NP + 4 * kMaxNs; }

// ---- double-float operations (no contraction into FMAs) --------------------
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void tsum(float a, float b, float &s, float &e) {
    s = fadd(a, b);
    const float bb = fsub(s, a);
    e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
}

// Low part of (ah + al)(yh + yl) - fl(ah yh): the exact product error of the high
// parts plus the two cross terms (Dekker's TwoProduct with an FMA).
__device__ __forceinline__ float prod_lo(float ah, float al, float yh, float yl, float ph) {
    float pe = ffma(ah, yh, -ph);
    pe = ffma(ah, yl, pe);
    return ffma(al, yh, pe);
}

// Y <- r Y + G with r = ah + al.
__device__ __forceinline__ void node_r(float ah, float al, float gh, float gl, float &yh, float &yl) {
    const float ph = fmul(ah, yh);
    const float pe = prod_lo(ah, al, yh, yl, ph);
    float s, e;
    tsum(ph, gh, s, e);
    const float t = fadd(e, fadd(pe, gl));
    const float nh = fadd(s, t);
    yl = fsub(t, fsub(nh, s));
    yh = nh;
}

// Y <- Y - u Y + G with u = 1 - r = uh + ul.
__device__ __forceinline__ void node_u(float uh, float ul, float gh, float gl, float &yh, float &yl) {
    const float ph = fmul(uh, yh);
    const float pe = prod_lo(uh, ul, yh, yl, ph);
    float s1, e1, s2, e2;
    tsum(yh, -ph, s1, e1);
    tsum(s1, gh, s2, e2);
    const float t = fadd(fadd(e1, e2), fadd(fsub(yl, pe), gl));
    const float nh = fadd(s2, t);
    yl = fsub(t, fsub(nh, s2));
    yh = nh;
}

// (sh, sl) += (ch + cl)(yh + yl); sl collects the low parts unnormalised.
__device__ __forceinline__ void acc_prod(float ch, float cl, float yh, float yl, float &sh, float &sl) {
    const float p = fmul(ch, yh);
    const float pe = prod_lo(ch, cl, yh, yl, p);
    float s, e;
    tsum(sh, p, s, e);
    sh = s;
    sl = fadd(sl, fadd(e, pe));
}

// FP64 value -> hi + lo.
__device__ __forceinline__ float2 df_of(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// ---------------------------------------------------------------------------
// Tables: per state the np nodes are ranked by r (ascending, ties by index) and put in
// the top np of the NP slots; slot t of state s is word 2 t + s: (a_hi, a_lo, c_hi, c_lo)
// with a = r_j, or a = 1 - r_j in the top df_u_slots(NP) slots; unused slots are zero
// (Y = G, no contribution). Then the window weights d_i, i < L, as (hi, lo) in word 2 i + s.
// One block of 256 threads.
// ---------------------------------------------------------------------------
__global__ void k_df_tables(int NP, int np, int L, int64_t N, const double *__restrict__ tab1,
                            const double *__restrict__ tab2,
                            const double *__restrict__ d1, const double *__restrict__ d2, float *__restrict__ out) {
    const int tid = threadIdx.x, KU = df_u_slots(NP);
    for (int i = tid; i < df_table_floats(NP); i += blockDim.x) out[i] = 0.0f;
    __syncthreads();
    float4 *tab = reinterpret_cast<float4 *>(out);
    float2 *wdf = reinterpret_cast<float2 *>(out + 8 * NP);
    for (int e = tid; e < 2 * np; e += blockDim.x) {
        const int st = e / np, j = e - st * np;
        const double *tq = st ? tab2 : tab1;
        const double r = tq[j];
        int rank = 0;
        for (int k = 0; k < np; ++k) {
            const double rk = tq[k];
            rank += (rk < r || (rk == r && k < j)) ? 1 : 0;
        }
        const int t = NP - np + rank;
        const float2 a = df_of(t >= NP - KU ? 1.0 - r : r), c = df_of(tq[np + j]);
        tab[2 * t + st] = make_float4(a.x, a.y, c.x, c.y);
    }
    for (int e = tid; e < 2 * L; e += blockDim.x) {
        const int st = e & 1, i = e >> 1;
        wdf[e] = i <= N ? df_of((st ? d2 : d1)[i]) : make_float2(0.0f, 0.0f);   // d has N + 1 entries
    }
}

// ---------------------------------------------------------------------------
// The solve. Software-pipelined as the FP32 form: the node part of step n + 1 needs
// G^{n+1-L} (L >= 2: written at step n - 1 or earlier) and not G^n, so it runs in the
// iteration of step n, beside the window and the FP64 step of step n. The loop body is
// branch-free up to the rare rescale, so that the compiler can interleave the latency-bound
// FP64 step with the node work: the node part runs from the first step (it reads ring slots
// that are still zero until level 1 exists), and the window is unrolled to WL - 1 terms
// (WL >= L, a compile-time bound) whose weights beyond d_{L-1} are zero.
// ---------------------------------------------------------------------------
template <int NP, bool BE, int WL>
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks)
    k_fp2s_fast_df(Fp2sParams P, const double *__restrict__ lam, const double *__restrict__ g0,
                   double *__restrict__ gN, int *__restrict__ status, const double *__restrict__ d1,
                   const double *__restrict__ d2, const float *__restrict__ dftab) {
    constexpr int KR = NP - df_u_slots(NP);       // slots of the r form
    constexpr int KS = df_smem_slots(NP);         // slots in shared memory (all of the r form)
    static_assert(KS <= KR, "shared-memory slots take the r form");
    extern __shared__ __align__(16) float smd[];
    const int L = P.L, T = blockDim.x, tid = threadIdx.x;
    const float4 *tab = reinterpret_cast<const float4 *>(smd);
    const float2 *wdf = reinterpret_cast<const float2 *>(smd + 8 * NP);
    float2 *R = reinterpret_cast<float2 *>(smd + df_table_floats(NP));      // [L][T]
    float2 *Ys = R + (size_t)L * T;                                          // [KS][T]
    for (int e = tid; e < df_table_floats(NP); e += T) smd[e] = dftab[e];
    for (int j = 0; j < L; ++j) R[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
    for (int j = 0; j < KS; ++j) Ys[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
    __syncthreads();

    const int lane = tid & 31, st = lane >> 4;
    const int64_t mode_raw = ((int64_t)blockIdx.x * (T >> 5) + (tid >> 5)) * kFastModesPerWarp + (lane & 15);
    const bool active = mode_raw < P.nmodes;
    const int64_t mode = active ? mode_raw : 0;
    const float4 *tb = tab + st;
    const float2 *ws = wdf + st;
    float2 *Rc = R + tid, *Yc = Ys + tid;
    const double *dn = st ? d2 : d1;

    // per-mode power-of-two scale from max(|g1^0|, |g2^0|)
    const double gz64 = g0[st * P.nmodes + mode];
    const double gmax = fmax(fabs(gz64), fabs(__shfl_xor_sync(0xffffffffu, gz64, 16)));
    int ex = 0;
    if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &ex);
    double gz = ldexp(gz64, -ex);

    const double d_s0 = dn[0], d_o0 = (st ? d1 : d2)[0];
    ModeConst mc;
    const bool ok = mode_setup(P, lam[mode], st ? d_o0 : d_s0, st ? d_s0 : d_o0, mc);
    if (active && st == 0 && !ok) atomicOr(status, ST_SINGULAR);
    const double mn_oo = st ? mc.Mn.i22 : mc.Mn.i11, mn_ot = st ? mc.Mn.i21 : mc.Mn.i12;
    const double a = P.a, c = mc.c, inv_tau = P.inv_tau;

    float yh[NP - KS], yl[NP - KS];              // slot j >= KS in register j - KS
#pragma unroll
    for (int j = 0; j < NP - KS; ++j) yh[j] = yl[j] = 0.0f;
    double gm1 = gz, gm2 = 0.0;
    const int64_t N = P.N;
    int slot = 1 % L;                            // n % L
    int64_t n = 1;
    if (!BE && N >= 1) {
        // the first SBD step (Eq. 4.7, n = 1: its own matrix, no history)
        const double m1_oo = st ? mc.M1.i22 : mc.M1.i11, m1_ot = st ? mc.M1.i21 : mc.M1.i12;
        const double e = d_s0 * gz * (1.0 / 3.0);
        const double e_o = __shfl_xor_sync(0xffffffffu, e, 16);
        const double b = gz * inv_tau - c * e + a * e_o;
        const double b_o = __shfl_xor_sync(0xffffffffu, b, 16);
        const double x = m1_oo * b + m1_ot * b_o;
        Rc[(size_t)slot * T] = df_of(x);
        gm2 = gm1;
        gm1 = x;
        slot = (slot + 1 == L) ? 0 : slot + 1;
        n = 2;
    }
    // node part of the current step (two double-float partial sums): zero while n <= L
    float ch0 = 0.0f, cl0 = 0.0f, ch1 = 0.0f, cl1 = 0.0f;
    for (; n <= N; ++n) {
        // node part of step n + 1, from level n + 1 - L (slot (n + 1) % L; zero before level 1)
        const int next = (slot + 1 == L) ? 0 : slot + 1;
        float nh0 = 0.0f, nl0 = 0.0f, nh1 = 0.0f, nl1 = 0.0f;
        const float2 g = Rc[(size_t)next * T];
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            const float4 t = tb[2 * j];
            float2 y = Yc[(size_t)j * T];
            node_r(t.x, t.y, g.x, g.y, y.x, y.y);
            Yc[(size_t)j * T] = y;
            if (j & 1) acc_prod(t.z, t.w, y.x, y.y, nh1, nl1);
            else acc_prod(t.z, t.w, y.x, y.y, nh0, nl0);
        }
#pragma unroll
        for (int j = KS; j < NP; ++j) {
            const float4 t = tb[2 * j];
            float &ya = yh[j - KS], &yb = yl[j - KS];
            if (j < KR) node_r(t.x, t.y, g.x, g.y, ya, yb);
            else node_u(t.x, t.y, g.x, g.y, ya, yb);
            if (j & 1) acc_prod(t.z, t.w, ya, yb, nh1, nl1);
            else acc_prod(t.z, t.w, ya, yb, nh0, nl0);
        }
        // exact window of step n: d_i x^{n-i}, i = 1 .. L - 1 (levels before 1 are zero slots;
        // terms i >= L have zero weights)
        int sl = slot;
#pragma unroll
        for (int i = 1; i < WL; ++i) {
            sl = (sl == 0) ? L - 1 : sl - 1;
            const float2 w = ws[2 * i], x = Rc[(size_t)sl * T];
            if (i & 1) acc_prod(w.x, w.y, x.x, x.y, ch1, cl1);
            else acc_prod(w.x, w.y, x.x, x.y, ch0, cl0);
        }
        float hs, he;
        tsum(ch0, ch1, hs, he);
        const double h = (double)hs + (double)fadd(he, fadd(cl0, cl1));
        // the 2x2 step in FP64 (Eq. 4.1 / 4.7)
        double e, lead;
        if (BE) {
            e = h;
            lead = gm1 * inv_tau;
        } else {
            e = fma(0.5 * __ldg(dn + n - 1), gz, h);
            lead = (2.0 * gm1 - 0.5 * gm2) * inv_tau;
        }
        const double e_o = __shfl_xor_sync(0xffffffffu, e, 16);
        const double b = lead - c * e + a * e_o;
        const double b_o = __shfl_xor_sync(0xffffffffu, b, 16);
        double x = mn_oo * b + mn_ot * b_o;
        float2 xd = df_of(x);
        // keep the mode's values inside [2^-40, 2^40]: both lanes of the mode see the same
        // magnitude and rescale together by an exact power of two
        const float am = fmaxf(fabsf(xd.x), fabsf(__shfl_xor_sync(0xffffffffu, xd.x, 16)));
        if (am > 0x1p40f || (am < 0x1p-40f && am > 0.0f)) {
            int k;
            frexpf(am, &k);
            k = max(-120, min(120, k));
            const float f = ldexpf(1.0f, -k);
            const double fd = ldexp(1.0, -k);
#pragma unroll
            for (int j = 0; j < NP - KS; ++j) {
                yh[j] *= f;
                yl[j] *= f;
            }
            for (int j = 0; j < KS; ++j) {
                const float2 v = Yc[(size_t)j * T];
                Yc[(size_t)j * T] = make_float2(v.x * f, v.y * f);
            }
            for (int j = 0; j < L; ++j) {
                const float2 v = Rc[(size_t)j * T];
                Rc[(size_t)j * T] = make_float2(v.x * f, v.y * f);
            }
            nh0 *= f;
            nl0 *= f;
            nh1 *= f;
            nl1 *= f;
            x *= fd;
            gm1 *= fd;
            gm2 *= fd;
            gz *= fd;
            xd = make_float2(xd.x * f, xd.y * f);
            ex += k;
        }
        Rc[(size_t)slot * T] = xd;
        gm2 = gm1;
        gm1 = x;
        ch0 = nh0;
        cl0 = nl0;
        ch1 = nh1;
        cl1 = nl1;
        slot = next;
    }
    if (active) {
        const double out = ldexp(gm1, ex);
        gN[st * P.nmodes + mode] = out;
        if (!isfinite(out)) atomicOr(status, ST_NONFINITE);
    }
}

static size_t df_smem_bytes(int NP, int L) {
    return (size_t)df_table_floats(NP) * sizeof(float) + (size_t)(L + df_smem_slots(NP)) * kDfThreads * sizeof(float2);
}

int df_np_bound(int np) {
    for (int b : {16, 32, 48, 64, 80, 96, 112, 128})
        if (np <= b) return b;
    return 0;
}

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
template <int NP, bool BE, int WL>
static int launch_df_kernel(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                            const double *d1, const double *d2, const float *dftab, cudaStream_t s) {
    auto kern = k_fp2s_fast_df<NP, BE, WL>;
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
    kern<<<(unsigned)blocks, kDfThreads, smem, s>>>(P, lam, g0, gN, status, d1, d2, dftab);
    return CQ_OK;
}

template <int NP>
static int launch_df(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                     const double *d1, const double *d2, const float *dftab, cudaStream_t s) {
    if (P.scheme == CQ_BE) return launch_df_kernel<NP, true, 2>(P, lam, g0, gN, status, d1, d2, dftab, s);
    if (P.L <= 17) return launch_df_kernel<NP, false, 17>(P, lam, g0, gN, status, d1, d2, dftab, s);
    return launch_df_kernel<NP, false, kMaxNs>(P, lam, g0, gN, status, d1, d2, dftab, s);
}

int fast_df_solve(const Fp2sParams &P, const double *lam, const double *g0, double *gN, int *status,
                  const double *d1, const double *d2, const float *dftab, cudaStream_t s) {
    switch (df_np_bound(P.np)) {
        case 16: return launch_df<16>(P, lam, g0, gN, status, d1, d2, dftab, s);
        case 32: return launch_df<32>(P, lam, g0, gN, status, d1, d2, dftab, s);
        case 48: return launch_df<48>(P, lam, g0, gN, status, d1, d2, dftab, s);
        case 64: return launch_df<64>(P, lam, g0, gN, status, d1, d2, dftab, s);
        case 80: return launch_df<80>(P, lam, g0, gN, status, d1, d2, dftab, s);
        case 96: return launch_df<96>(P, lam, g0, gN, status, d1, d2, dftab, s);
        case 112: return launch_df<112>(P, lam, g0, gN, status, d1, d2, dftab, s);
        case 128: return launch_df<128>(P, lam, g0, gN, status, d1, d2, dftab, s);
        default: return CQ_EUNSUPPORTED;
    }
}

}  // namespace fastcq
