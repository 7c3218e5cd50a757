// Fast solve in double-float arithmetic (precision form CQ_DF64): constants, the
// double-float operations, the table builder and the per-lane solve, shared by the
// single-problem kernel (fastdf.cu) and the batched persistent kernel (batch.cu).
#pragma once

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

// Compile-time node bound for np points per state (0: more than 128).
__host__ __device__ inline int df_np_class(int np) {
    return np <= 16 ? 16 : np <= 32 ? 32 : np <= 48 ? 48 : np <= 64 ? 64 : np <= 80 ? 80 : np <= 96 ? 96
                          : np <= 112 ? 112 : np <= 128 ? 128 : 0;
}

// Floats of the kernel's table: per pair of node slots (2p, 2p + 1) and state two float4
// words, (a_hi, a_hi', a_lo, a_lo') and (c_hi, c_hi', c_lo, c_lo') (primes: slot 2p + 1) with
// a = r or a = 1 - r, then [kMaxNs][2] float2 window weights d_i.
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

// ---- the same operations on two independent values at once -----------------
// Blackwell's packed two-wide FP32 instructions (FADD2 / FMUL2 / FFMA2) round each component
// as the scalar instruction does, and halve the instructions issued. Component k of every
// argument belongs to the k-th of two independent double-float computations.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ void tsum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = fadd2(a, b);
    const float2 bb = fsub2(s, a);
    e = fadd2(fsub2(a, fsub2(s, bb)), fsub2(b, bb));
}

__device__ __forceinline__ float2 prod_lo2(float2 ah, float2 al, float2 yh, float2 yl, float2 ph) {
    float2 pe = ffma2(ah, yh, neg2(ph));
    pe = ffma2(ah, yl, pe);
    return ffma2(al, yh, pe);
}

// node_r / node_u / acc_prod on a pair of nodes
__device__ __forceinline__ void node_r2(float2 ah, float2 al, float2 gh, float2 gl, float2 &yh, float2 &yl) {
    const float2 ph = fmul2(ah, yh);
    const float2 pe = prod_lo2(ah, al, yh, yl, ph);
    float2 s, e;
    tsum2(ph, gh, s, e);
    const float2 t = fadd2(e, fadd2(pe, gl));
    const float2 nh = fadd2(s, t);
    yl = fsub2(t, fsub2(nh, s));
    yh = nh;
}

__device__ __forceinline__ void node_u2(float2 uh, float2 ul, float2 gh, float2 gl, float2 &yh, float2 &yl) {
    const float2 ph = fmul2(uh, yh);
    const float2 pe = prod_lo2(uh, ul, yh, yl, ph);
    float2 s1, e1, s2, e2;
    tsum2(yh, neg2(ph), s1, e1);
    tsum2(s1, gh, s2, e2);
    const float2 t = fadd2(fadd2(e1, e2), fadd2(fsub2(yl, pe), gl));
    const float2 nh = fadd2(s2, t);
    yl = fsub2(t, fsub2(nh, s2));
    yh = nh;
}

__device__ __forceinline__ void acc_prod2(float2 ch, float2 cl, float2 yh, float2 yl, float2 &sh, float2 &sl) {
    const float2 p = fmul2(ch, yh);
    const float2 pe = prod_lo2(ch, cl, yh, yl, p);
    float2 s, e;
    tsum2(sh, p, s, e);
    sh = s;
    sl = fadd2(sl, fadd2(e, pe));
}

// ---------------------------------------------------------------------------
// Tables: per state the np nodes are ranked by r (ascending, ties by index) and put in
// the top np of the NP slots; slot t = 2 p + e of state s is component e of the pairs in
// words 4 p + 2 s (a_hi, a_lo) and 4 p + 2 s + 1 (c_hi, c_lo), with a = r_j, or a = 1 - r_j in
// the top df_u_slots(NP) slots; unused slots are zero (Y = G, no contribution). Then the window weights d_i, i < L, as (hi, lo) in word 2 i + s.
// Called by every thread of a block (tid, nthr); out is global or shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_tables_fill(int NP, int np, int L, int64_t N, const double *__restrict__ tab1,
                                               const double *__restrict__ tab2, const double *__restrict__ d1,
                                               const double *__restrict__ d2, float *__restrict__ out, int tid,
                                               int nthr) {
    const int KU = df_u_slots(NP);
    for (int i = tid; i < df_table_floats(NP); i += nthr) out[i] = 0.0f;
    __syncthreads();
    float4 *tab = reinterpret_cast<float4 *>(out);
    float2 *wdf = reinterpret_cast<float2 *>(out + 8 * NP);
    for (int e = tid; e < 2 * np; e += nthr) {
        const int st = e / np, j = e - st * np;
        const double *tq = st ? tab2 : tab1;
        const double r = tq[j];
        int rank = 0;
        for (int k = 0; k < np; ++k) {
            const double rk = tq[k];
            rank += (rk < r || (rk == r && k < j)) ? 1 : 0;
        }
        const int t = NP - np + rank, p = t >> 1, el = t & 1;
        const float2 a = df_of(t >= NP - KU ? 1.0 - r : r), c = df_of(tq[np + j]);
        float *wa = reinterpret_cast<float *>(tab + 4 * p + 2 * st), *wc = wa + 4;
        wa[el] = a.x;
        wa[2 + el] = a.y;
        wc[el] = c.x;
        wc[2 + el] = c.y;
    }
    for (int e = tid; e < 2 * L; e += nthr) {
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
// Per lane: state st = (lane >> 4) of mode mode_raw (its partner state on lane ^ 16), over all
// P.N steps; lanes with mode_raw >= mode_end take part in the shuffles on mode 0 and write
// nothing. Shared memory (the caller fills the tables and zeroes R and Ys first): tab [NP / 2][2][2]
// float4, wdf [kMaxNs][2] float2, R [L][T] float2 and Ys [df_smem_slots(NP) / 2][T] float4 (the
// pair (yh, yh', yl, yl') of slots 2p, 2p + 1), column tid. Node slots are updated in pairs with
// the packed operations (node_r2 / node_u2 / acc_prod2); component 0 of the partial sums collects
// the even slots and component 1 the odd ones. With HIST every level is also stored in true
// units (the forward sweep of the fast-form gradient): hist[(n * 2 + s) * nmodes + mode], n = 0 .. N.
template <int NP, bool BE, int WL, bool HIST = false>
__device__ __forceinline__ void df_solve_lane(const Fp2sParams &P, const double *__restrict__ lam,
                                              const double *__restrict__ g0, double *__restrict__ gN,
                                              int *__restrict__ status, const double *__restrict__ d1,
                                              const double *__restrict__ d2, const float4 *tab, const float2 *wdf,
                                              float2 *R, float2 *Ys, int T, int tid, int64_t mode_raw,
                                              int64_t mode_end, double *__restrict__ hist = nullptr) {
    constexpr int KR = NP - df_u_slots(NP);       // slots of the r form
    constexpr int KS = df_smem_slots(NP);         // slots in shared memory (all of the r form)
    static_assert(KS <= KR, "shared-memory slots take the r form");
    static_assert(NP % 2 == 0 && KR % 2 == 0 && KS % 2 == 0, "every slot class holds whole pairs");
    const int L = P.L;
    const int lane = tid & 31, st = lane >> 4;
    const bool active = mode_raw < mode_end;
    const int64_t mode = active ? mode_raw : 0;
    const float4 *tb = tab + 2 * st;              // pair p: tb[4 p] (a), tb[4 p + 1] (c)
    const float2 *ws = wdf + st;
    float2 *Rc = R + tid;
    float4 *Yc = reinterpret_cast<float4 *>(Ys) + tid;
    const double *dn = st ? d2 : d1;

    // per-mode power-of-two scale from max(|g1^0|, |g2^0|)
    const double gz64 = g0[st * P.nmodes + mode];
    const double gmax = fmax(fabs(gz64), fabs(__shfl_xor_sync(0xffffffffu, gz64, 16)));
    int ex = 0;
    if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &ex);
    double gz = ldexp(gz64, -ex);
    if (HIST && active) hist[st * P.nmodes + mode] = gz64;

    const double d_s0 = dn[0], d_o0 = (st ? d1 : d2)[0];
    ModeConst mc;
    const bool ok = mode_setup(P, lam[mode], st ? d_o0 : d_s0, st ? d_s0 : d_o0, mc);
    if (active && st == 0 && !ok) atomicOr(status, ST_SINGULAR);
    const double mn_oo = st ? mc.Mn.i22 : mc.Mn.i11, mn_ot = st ? mc.Mn.i21 : mc.Mn.i12;
    const double a = P.a, c = mc.c, inv_tau = P.inv_tau;

    constexpr int PS = KS / 2;                    // pairs in shared memory
    float2 yh[NP / 2 - PS], yl[NP / 2 - PS];      // pair p >= PS in register p - PS
#pragma unroll
    for (int j = 0; j < NP / 2 - PS; ++j) yh[j] = yl[j] = make_float2(0.0f, 0.0f);
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
        if (HIST && active) hist[(2 + st) * P.nmodes + mode] = ldexp(x, ex);
        gm2 = gm1;
        gm1 = x;
        slot = (slot + 1 == L) ? 0 : slot + 1;
        n = 2;
    }
    // node part of the current step (double-float partial sums of the even / odd slots in
    // components 0 / 1): zero while n <= L
    float2 ch = make_float2(0.0f, 0.0f), cl = make_float2(0.0f, 0.0f);
    for (; n <= N; ++n) {
        // node part of step n + 1, from level n + 1 - L (slot (n + 1) % L; zero before level 1)
        const int next = (slot + 1 == L) ? 0 : slot + 1;
        float2 nh = make_float2(0.0f, 0.0f), nl = make_float2(0.0f, 0.0f);
        const float2 g = Rc[(size_t)next * T];
        const float2 gh = make_float2(g.x, g.x), gl = make_float2(g.y, g.y);
#pragma unroll
        for (int p = 0; p < PS; ++p) {
            const float4 a = tb[4 * p], c = tb[4 * p + 1];
            const float4 y = Yc[(size_t)p * T];
            float2 ya = make_float2(y.x, y.y), yb = make_float2(y.z, y.w);
            node_r2(make_float2(a.x, a.y), make_float2(a.z, a.w), gh, gl, ya, yb);
            Yc[(size_t)p * T] = make_float4(ya.x, ya.y, yb.x, yb.y);
            acc_prod2(make_float2(c.x, c.y), make_float2(c.z, c.w), ya, yb, nh, nl);
        }
#pragma unroll
        for (int p = PS; p < NP / 2; ++p) {
            const float4 a = tb[4 * p], c = tb[4 * p + 1];
            float2 &ya = yh[p - PS], &yb = yl[p - PS];
            if (2 * p < KR) node_r2(make_float2(a.x, a.y), make_float2(a.z, a.w), gh, gl, ya, yb);
            else node_u2(make_float2(a.x, a.y), make_float2(a.z, a.w), gh, gl, ya, yb);
            acc_prod2(make_float2(c.x, c.y), make_float2(c.z, c.w), ya, yb, nh, nl);
        }
        // exact window of step n: d_i x^{n-i}, i = 1 .. L - 1 (levels before 1 are zero slots;
        // terms i >= L have zero weights)
        int sl = slot;
#pragma unroll
        for (int i = 1; i < WL; ++i) {
            sl = (sl == 0) ? L - 1 : sl - 1;
            const float2 w = ws[2 * i], x = Rc[(size_t)sl * T];
            if (i & 1) acc_prod(w.x, w.y, x.x, x.y, ch.y, cl.y);
            else acc_prod(w.x, w.y, x.x, x.y, ch.x, cl.x);
        }
        float hs, he;
        tsum(ch.x, ch.y, hs, he);
        const double h = (double)hs + (double)fadd(he, fadd(cl.x, cl.y));
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
            for (int j = 0; j < NP / 2 - PS; ++j) {
                yh[j] = make_float2(yh[j].x * f, yh[j].y * f);
                yl[j] = make_float2(yl[j].x * f, yl[j].y * f);
            }
            for (int p = 0; p < PS; ++p) {
                const float4 v = Yc[(size_t)p * T];
                Yc[(size_t)p * T] = make_float4(v.x * f, v.y * f, v.z * f, v.w * f);
            }
            for (int j = 0; j < L; ++j) {
                const float2 v = Rc[(size_t)j * T];
                Rc[(size_t)j * T] = make_float2(v.x * f, v.y * f);
            }
            nh = make_float2(nh.x * f, nh.y * f);
            nl = make_float2(nl.x * f, nl.y * f);
            x *= fd;
            gm1 *= fd;
            gm2 *= fd;
            gz *= fd;
            xd = make_float2(xd.x * f, xd.y * f);
            ex += k;
        }
        Rc[(size_t)slot * T] = xd;
        if (HIST && active) hist[(n * 2 + st) * P.nmodes + mode] = ldexp(x, ex);
        gm2 = gm1;
        gm1 = x;
        ch = nh;
        cl = nl;
        slot = next;
    }
    if (active) {
        const double out = ldexp(gm1, ex);
        gN[st * P.nmodes + mode] = out;
        if (!isfinite(out)) atomicOr(status, ST_NONFINITE);
    }
}

}  // namespace fastcq
