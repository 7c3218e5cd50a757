// Gradient of the fast form (fp2s_gradient / fp2s_vjp with CQ_FAST, FP64 or CQ_DF64): the
// discrete adjoint of the fast scheme.
//
// The fast history (recurrences after Eq. 3.10 and Eq. 3.18) is the direct history of
// Eq. 3.8 with the weights
//     dt_i = d_i                          for i < L (the exact window),
//     dt_i = sum_j c_j r_j^(i - L)        for i >= L (the geometric history parts),
// so its adjoint is the adjoint of the direct scheme with these weights: per mode, the
// transposed 2x2 steps of Eq. 4.1 / Eq. 4.7 run backward from m = N, the adjoint levels
// mu^m = K lambda^m (K = [[a + lam_k, -a], [-a, a + lam_k]]) feed the reversed-time history
//     hr^m = sum_{n > m} dt_{n-m} mu^n,
// and dJ/dbeta of a state is sum_m x^m hq^m with hq^m = sum_{n >= m} dt'_{n-m} mu^n (dt' the
// derivative of the weights in beta), plus the terms of the first SBD step and of the
// 1/2 d_{n-1} G^0 correction (exact weights, as in the direct adjoint).
// The geometric parts give backward recurrences of O(Np) work per step:
//     V_j^m = r_j V_j^{m+1} + mu^{m+L},   sum_{n >= m + L} r_j^(n-m-L) mu^n = V_j^m,
//     W_j^m = r_j W_j^{m+1} + V_j^{m+1},  sum_{n >= m + L} (n-m-L) r_j^(n-m-L-1) mu^n = W_j^m,
// so that hr^m = window + sum_j c_j V_j^m and, with dt'_i = c'_j r_j^(i-L) + c_j (i-L)
// r_j^(i-L-1) r'_j, hq^m = d'_0 mu^m + window' + sum_j (c'_j V_j^m + c_j r'_j W_j^m).
// The derivatives r'_j, c'_j of the Gauss-Jacobi based tables in beta are taken by
// Richardson-extrapolated central differences of the same table construction (four extra
// builds per state), which is accurate to ~1e-10 relative; the weights d_i and their
// derivatives d'_i are exact (the product / Cauchy forms).
//
// One lane per mode and state as in the fused fast solve (lanes l < 16: state 1, l + 16: state
// 2 of the same mode); a lane keeps V_j, W_j and the last L adjoint levels in shared memory
// (column tid) and reads its forward levels x^m from the history the forward sweep stored (the
// FP64 fused fast solve, or for CQ_DF64 the double-float one, with every level kept).
#include "common.cuh"
#include "fastdf.cuh"
#include "fastgrad.cuh"
#include "fp2s_core.cuh"

namespace fastcq {

// der = (c'_j, c_j r'_j), j < np, from the tables t[k] = (r[np], c[np]) built at beta + delta,
// beta - delta, beta + delta / 2, beta - delta / 2 (k = 0 .. 3) and tab = (r, c) at beta:
// D(h) = (f(beta + h) - f(beta - h)) / (2 h), f' = (4 D(delta / 2) - D(delta)) / 3.
__global__ void k_fast_table_derivs(int np, double delta, const double *__restrict__ t, const double *__restrict__ tab,
                                    double *__restrict__ der) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    auto deriv = [&](int off) {
        const double dh = (t[off + j] - t[2 * np + off + j]) / (2.0 * delta);
        const double dh2 = (t[4 * np + off + j] - t[6 * np + off + j]) / delta;
        return (4.0 * dh2 - dh) / 3.0;
    };
    der[j] = deriv(np);
    der[np + j] = tab[np + j] * deriv(0);
}

int fast_grad_tables(int scheme, double beta, double tau, int np1, int np2, int L, const double *tab,
                     double *gj_scratch, double *tmp, double *der, cudaStream_t s) {
    const int np = scheme == CQ_BE ? np1 : np1 + np2;
    const double delta = fmin(2e-3, 0.25 * fmin(beta, 1.0 - beta));
    const double b4[4] = {beta + delta, beta - delta, beta + 0.5 * delta, beta - 0.5 * delta};
    int st;
    for (int k = 0; k < 4; ++k) {
        double *r = tmp + (size_t)2 * np * k;
        if ((st = build_fast_coeffs(scheme, b4[k], tau, np1, np2, L, gj_scratch, r, r + np, s))) return st;
    }
    k_fast_table_derivs<<<(np + 127) / 128, 128, 0, s>>>(np, delta, tmp, tab, der);
    return launched();
}

constexpr int kAdjFastMaxT = 64;

// Shared memory: tables interleaved by state (word 2 j + s): r, c, c', c r' ([NP][2] each, zero
// past np), the window weights d_i and d'_i (i < L, [kMaxNs][2] each), then per lane V [NP][T],
// W [NP][T] and the adjoint levels mu^n at slot n % L ([L][T]). NP is a compile-time bound of np
// (the node loop unrolls fully, so the compiler issues the state loads well ahead of their use);
// the zero-padded slots contribute nothing.
static size_t adj_fast_smem(int NP, int L, int T) {
    return ((size_t)8 * NP + 4 * kMaxNs + (size_t)(2 * NP + L) * T) * sizeof(double);
}

static int adj_np_class(int np) {
    for (int b : {16, 32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256})
        if (np <= b) return b;
    return 0;
}

template <int NP>
__global__ void __launch_bounds__(kAdjFastMaxT) k_adjoint_fast(
    Fp2sParams P, double wd, const double *__restrict__ lam, const double *__restrict__ d1,
    const double *__restrict__ d2, const double *__restrict__ q1, const double *__restrict__ q2,
    const double *__restrict__ tab1, const double *__restrict__ tab2, const double *__restrict__ der1,
    const double *__restrict__ der2, const double *__restrict__ hist, const double *__restrict__ tgt, int vjp,
    double *__restrict__ gx0, double *__restrict__ acc) {
    extern __shared__ double sm[];
    const int np = P.np, L = P.L, T = blockDim.x, tid = threadIdx.x;
    double *rt = sm, *ct = rt + 2 * NP, *cpt = ct + 2 * NP, *crt = cpt + 2 * NP;
    double *wt = crt + 2 * NP, *qt = wt + 2 * kMaxNs;
    double *V = qt + 2 * kMaxNs, *W = V + (size_t)NP * T, *Rm = W + (size_t)NP * T;
    for (int i = tid; i < NP; i += T) {
        const bool in = i < np;
        rt[2 * i] = in ? tab1[i] : 0.0;
        rt[2 * i + 1] = in ? tab2[i] : 0.0;
        ct[2 * i] = in ? tab1[np + i] : 0.0;
        ct[2 * i + 1] = in ? tab2[np + i] : 0.0;
        cpt[2 * i] = in ? der1[i] : 0.0;
        cpt[2 * i + 1] = in ? der2[i] : 0.0;
        crt[2 * i] = in ? der1[np + i] : 0.0;
        crt[2 * i + 1] = in ? der2[np + i] : 0.0;
    }
    for (int i = tid; i < L; i += T) {                   // d and d' have N + 1 entries
        const bool in = i <= P.N;
        wt[2 * i] = in ? d1[i] : 0.0;
        wt[2 * i + 1] = in ? d2[i] : 0.0;
        qt[2 * i] = in ? q1[i] : 0.0;
        qt[2 * i + 1] = in ? q2[i] : 0.0;
    }
    for (int j = 0; j < NP; ++j) V[(size_t)j * T + tid] = W[(size_t)j * T + tid] = 0.0;
    for (int j = 0; j < L; ++j) Rm[(size_t)j * T + tid] = 0.0;
    __syncthreads();

    const int lane = tid & 31, st = lane >> 4;
    const int64_t nm = P.nmodes, N = P.N;
    const int64_t mode_raw = ((int64_t)blockIdx.x * (T >> 5) + (tid >> 5)) * kFastModesPerWarp + (lane & 15);
    const bool active = mode_raw < nm;
    const int64_t mode = active ? mode_raw : 0;           // idle lanes take part in the shuffles
    const double a = P.a, c = a + lam[mode], it = P.inv_tau;
    const double d10 = wt[0], d20 = wt[1];
    // transposed step matrices and their inverses; the lane's own row, ordered (own, other)
    Inv2 Mn{}, M1{};
    bool ok;
    {
        const double c0 = (P.scheme == CQ_BE) ? it : 1.5 * it;
        ok = invert2(c0 + d10 * c, -d10 * a, -d20 * a, c0 + d20 * c, Mn);
        if (P.scheme == CQ_BDF2)
            ok &= invert2(it + (2.0 / 3.0) * d10 * c, -(2.0 / 3.0) * d10 * a, -(2.0 / 3.0) * d20 * a,
                          it + (2.0 / 3.0) * d20 * c, M1);
    }
    const double mn_oo = st ? Mn.i22 : Mn.i11, mn_ot = st ? Mn.i21 : Mn.i12;
    const double m1_oo = st ? M1.i22 : M1.i11, m1_ot = st ? M1.i21 : M1.i12;
    // terminal condition dJ/dx^N of the lane's state
    const double xN = hist[(N * 2 + st) * nm + mode];
    const double e = xN - tgt[st * nm + mode];
    const double rT = vjp ? tgt[st * nm + mode] : wd * e;
    double Jpart = (active && !vjp) ? 0.5 * wd * e * e : 0.0;
    const double *rs = rt + st, *cs = ct + st, *cps = cpt + st, *crs = crt + st, *ws = wt + st, *qs = qt + st;
    const double *dn = st ? d2 : d1, *qn = st ? q2 : q1;
    const double dq0 = qs[0];
    double *Vc = V + tid, *Wc = W + tid, *Rc = Rm + tid;
    double lp1 = 0.0, lp2 = 0.0, db = 0.0, sg = 0.0, sx = 0.0, lam1 = 0.0, lam2 = 0.0, mu1 = 0.0;
    int slot = (int)(N % L);                                // slot of level m
    for (int64_t m = N; m >= 1; --m) {
        const double in = Rc[(size_t)slot * T];            // mu^{m+L} (zero past N)
        double h0 = 0.0, h1 = 0.0, k0 = 0.0, k1 = 0.0;
#pragma unroll
        for (int j = 0; j < NP; j += 2) {
            const double ra = rs[2 * j], rb = rs[2 * j + 2];
            const double va = Vc[(size_t)j * T], vb = Vc[(size_t)(j + 1) * T];
            const double wa = fma(ra, Wc[(size_t)j * T], va), wb = fma(rb, Wc[(size_t)(j + 1) * T], vb);
            const double na = fma(ra, va, in), nb = fma(rb, vb, in);
            Wc[(size_t)j * T] = wa;
            Wc[(size_t)(j + 1) * T] = wb;
            Vc[(size_t)j * T] = na;
            Vc[(size_t)(j + 1) * T] = nb;
            h0 = fma(cs[2 * j], na, h0);
            h1 = fma(cs[2 * j + 2], nb, h1);
            k0 = fma(cps[2 * j], na, fma(crs[2 * j], wa, k0));
            k1 = fma(cps[2 * j + 2], nb, fma(crs[2 * j + 2], wb, k1));
        }
        // exact window: mu^{m+i}, i = 1 .. L - 1, at slot (m + i) % L
        int sl = slot;
        for (int i = 1; i < L; ++i) {
            sl = (sl + 1 == L) ? 0 : sl + 1;
            const double u = Rc[(size_t)sl * T];
            h1 = fma(ws[2 * i], u, h1);
            k1 = fma(qs[2 * i], u, k1);
        }
        double b = -(h0 + h1);
        if (m == N) b -= rT;
        const bool first = (P.scheme == CQ_BDF2 && m == 1);
        if (P.scheme == CQ_BE) {
            if (m < N) b += lp1 * it;
        } else {
            if (m + 1 <= N) b += 2.0 * it * lp1;
            if (m + 2 <= N) b -= 0.5 * it * lp2;
        }
        const double b_o = __shfl_xor_sync(0xffffffffu, b, 16);
        const double l = first ? fma(m1_oo, b, m1_ot * b_o) : fma(mn_oo, b, mn_ot * b_o);
        const double l_o = __shfl_xor_sync(0xffffffffu, l, 16);
        const double v = c * l - a * l_o;                  // mu^m of the lane's state
        Rc[(size_t)slot * T] = v;
        // hq^m (with the n = m term d'_0 mu^m) against the forward level x^m
        const double hq = fma(dq0, v, k0 + k1);
        db = fma(hist[(m * 2 + st) * nm + mode], hq, db);
        if (m >= 2) {
            sg = fma(__ldg(dn + m - 1), v, sg);
            sx = fma(__ldg(qn + m - 1), v, sx);
        }
        if (m == 1) {
            lam1 = l;
            mu1 = v;
        } else if (m == 2) {
            lam2 = l;
        }
        lp2 = lp1;
        lp1 = l;
        slot = (slot == 0) ? L - 1 : slot - 1;
    }
    const double x0 = hist[st * nm + mode];
    double g;
    if (P.scheme == CQ_BE) {
        g = -lam1 * it;
    } else {
        g = -lam1 * it + (st ? d20 : d10) * mu1 / 3.0 + 0.5 * it * lam2 + 0.5 * sg;
        const double x1 = hist[(2 + st) * nm + mode];
        db += mu1 * dq0 * (x0 - x1) / 3.0 + 0.5 * x0 * sx;
    }
    if (active) gx0[st * nm + mode] = g;
    else db = 0.0;
    // J over the whole warp; dJ/dbeta per state over each half-warp
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) Jpart += __shfl_xor_sync(0xffffffffu, Jpart, off);
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) db += __shfl_xor_sync(0xffffffffu, db, off);
    if (lane == 0) {
        atomicAdd(acc + 0, Jpart);
        atomicAdd(acc + 1, db);
    } else if (lane == 16) {
        atomicAdd(acc + 2, db);
    }
    if (active && st == 0 && !ok) atomicAdd(acc + 3, 1.0);
}

int fast_adjoint_slice(const Fp2sParams &P, double wd, const double *lam, const double *d1, const double *d2,
                       const double *q1, const double *q2, const double *tab1, const double *tab2,
                       const double *der1, const double *der2, const double *hist, const double *tgt, int vjp,
                       double *gx0, double *acc, cudaStream_t s) {
    const int NP = adj_np_class(P.np);
    if (NP == 0) return CQ_EUNSUPPORTED;
    int T = kAdjFastMaxT;
    while (T > 32 && adj_fast_smem(NP, P.L, T) > 227 * 1024) T /= 2;
    const size_t smem = adj_fast_smem(NP, P.L, T);
    if (smem > 227 * 1024) return CQ_EUNSUPPORTED;
    const int64_t mpb = (int64_t)(T / 32) * kFastModesPerWarp;
    const unsigned blocks = (unsigned)((P.nmodes + mpb - 1) / mpb);
    int st = CQ_OK;
    auto run = [&](auto kern, unsigned long long *attr) {
        if ((st = smem_attr_once((const void *)kern, 227 * 1024, attr))) return;
        kern<<<blocks, T, smem, s>>>(P, wd, lam, d1, d2, q1, q2, tab1, tab2, der1, der2, hist, tgt, vjp, gx0, acc);
        st = launched();
    };
#define CQ_ADJ_FAST(NPV)                        \
    case NPV: {                                 \
        static unsigned long long attr = 0;     \
        run(k_adjoint_fast<NPV>, &attr);        \
        break;                                  \
    }
    switch (NP) {
        CQ_ADJ_FAST(16)
        CQ_ADJ_FAST(32)
        CQ_ADJ_FAST(48)
        CQ_ADJ_FAST(64)
        CQ_ADJ_FAST(80)
        CQ_ADJ_FAST(96)
        CQ_ADJ_FAST(112)
        CQ_ADJ_FAST(128)
        CQ_ADJ_FAST(160)
        CQ_ADJ_FAST(192)
        CQ_ADJ_FAST(224)
        CQ_ADJ_FAST(256)
        default: return CQ_EUNSUPPORTED;
    }
#undef CQ_ADJ_FAST
    return st;
}

// ---------------------------------------------------------------------------
// The backward sweep in double-float (fp2s_gradient / fp2s_vjp with CQ_FAST and CQ_DF64): the
// same recurrences with V_j, W_j, the tables (r or u = 1 - r, c, c', c r') and the adjoint
// levels as hi + lo FP32 pairs, node slots updated two at a time with the packed two-wide
// operations of the double-float fast solve (node_r2 / node_u2 / acc_prod2), the transposed
// 2x2 steps and every per-mode sum in FP64. As in the forward double-float solve the nodes are
// ranked by r and the slowest quarter takes the u form (a ratio near 1 held as hi + lo loses
// 2^-49 / (1 - r) relative to 1 - r, and the geometric sums repeat that error); the adjoint
// variables are scaled by the power of two of the mode's terminal condition. The forward sweep
// is the double-float fast solve, which stores its levels in true units (FP64).
// ---------------------------------------------------------------------------

// Per state s and node pair p (slots 2p, 2p + 1) four float4 words at (p * 2 + s) * 4 + k:
// k = 0: (a_hi, a_hi', a_lo, a_lo') with a = r or a = 1 - r in the top df_u_slots(NP) slots;
// k = 1, 2, 3: c, c' and c r' in the same layout; then the window weights d_i and d'_i (i < L,
// zero past N) as (hi, lo) pairs at wdf[(i * 2 + s) * 2 + {0: d, 1: d'}].
__host__ __device__ constexpr int adj_df_table_floats(int NP) { return 16 * NP + 4 * 2 * kMaxNs; }

__global__ void k_adj_df_tables(int NP, int np, int L, int64_t N, const double *__restrict__ tab1,
                                const double *__restrict__ tab2, const double *__restrict__ der1,
                                const double *__restrict__ der2, const double *__restrict__ d1,
                                const double *__restrict__ d2, const double *__restrict__ q1,
                                const double *__restrict__ q2, float *__restrict__ out) {
    const int tid = threadIdx.x, nthr = blockDim.x, KU = df_u_slots(NP);
    for (int i = tid; i < adj_df_table_floats(NP); i += nthr) out[i] = 0.0f;
    __syncthreads();
    for (int e = tid; e < 2 * np; e += nthr) {
        const int st = e / np, j = e - st * np;
        const double *tq = st ? tab2 : tab1, *dq = st ? der2 : der1;
        const double r = tq[j];
        int rank = 0;
        for (int k = 0; k < np; ++k) rank += (tq[k] < r || (tq[k] == r && k < j)) ? 1 : 0;
        const int t = NP - np + rank, p = t >> 1, el = t & 1;
        const double v[4] = {t >= NP - KU ? 1.0 - r : r, tq[np + j], dq[j], dq[np + j]};
        for (int k = 0; k < 4; ++k) {
            const float2 h = df_of(v[k]);
            float *w = out + ((size_t)(p * 2 + st) * 4 + k) * 4;
            w[el] = h.x;
            w[2 + el] = h.y;
        }
    }
    float2 *wdf = reinterpret_cast<float2 *>(out + 16 * NP);
    for (int e = tid; e < 2 * L; e += nthr) {
        const int st = e & 1, i = e >> 1;
        const bool in = i <= N;
        wdf[e * 2] = in ? df_of((st ? d2 : d1)[i]) : make_float2(0.0f, 0.0f);
        wdf[e * 2 + 1] = in ? df_of((st ? q2 : q1)[i]) : make_float2(0.0f, 0.0f);
    }
}

// Shared memory: the table, then per lane V and W ([NP / 2][T] float4: (hi, hi', lo, lo') of the
// pair) and the adjoint levels mu^n as (hi, lo) at slot n % L ([L][T] float2).
static size_t adj_df_smem(int NP, int L, int T) {
    return (size_t)adj_df_table_floats(NP) * sizeof(float) + (size_t)NP * T * 16 + (size_t)L * T * 8;
}

template <int NP>
__global__ void __launch_bounds__(kAdjFastMaxT) k_adjoint_fast_df(
    Fp2sParams P, double wd, const double *__restrict__ lam, const double *__restrict__ d1,
    const double *__restrict__ d2, const double *__restrict__ q1, const double *__restrict__ q2,
    const float *__restrict__ adtab, const double *__restrict__ hist, const double *__restrict__ tgt, int vjp,
    double *__restrict__ gx0, double *__restrict__ acc) {
    constexpr int KR = NP - df_u_slots(NP);         // slots of the r form
    static_assert(KR % 2 == 0, "slot classes hold whole pairs");
    extern __shared__ __align__(16) float sa[];
    const int L = P.L, T = blockDim.x, tid = threadIdx.x;
    for (int e = tid; e < adj_df_table_floats(NP); e += T) sa[e] = adtab[e];
    float4 *V = reinterpret_cast<float4 *>(sa + adj_df_table_floats(NP));
    float4 *W = V + (size_t)(NP / 2) * T;
    float2 *Rm = reinterpret_cast<float2 *>(W + (size_t)(NP / 2) * T);
    for (int p = 0; p < NP / 2; ++p) V[(size_t)p * T + tid] = W[(size_t)p * T + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < L; ++j) Rm[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
    __syncthreads();

    const int lane = tid & 31, st = lane >> 4;
    const int64_t nm = P.nmodes, N = P.N;
    const int64_t mode_raw = ((int64_t)blockIdx.x * (T >> 5) + (tid >> 5)) * kFastModesPerWarp + (lane & 15);
    const bool active = mode_raw < nm;
    const int64_t mode = active ? mode_raw : 0;           // idle lanes take part in the shuffles
    const double a = P.a, c = a + lam[mode], it = P.inv_tau;
    const double d10 = d1[0], d20 = d2[0];
    Inv2 Mn{}, M1{};
    bool ok;
    {
        const double c0 = (P.scheme == CQ_BE) ? it : 1.5 * it;
        ok = invert2(c0 + d10 * c, -d10 * a, -d20 * a, c0 + d20 * c, Mn);
        if (P.scheme == CQ_BDF2)
            ok &= invert2(it + (2.0 / 3.0) * d10 * c, -(2.0 / 3.0) * d10 * a, -(2.0 / 3.0) * d20 * a,
                          it + (2.0 / 3.0) * d20 * c, M1);
    }
    const double mn_oo = st ? Mn.i22 : Mn.i11, mn_ot = st ? Mn.i21 : Mn.i12;
    const double m1_oo = st ? M1.i22 : M1.i11, m1_ot = st ? M1.i21 : M1.i12;
    // terminal condition, scaled by the power of two of the mode's larger state
    const double xN = hist[(N * 2 + st) * nm + mode];
    const double e = xN - tgt[st * nm + mode];
    const double rT = vjp ? tgt[st * nm + mode] : wd * e;
    double Jpart = (active && !vjp) ? 0.5 * wd * e * e : 0.0;
    int ey = 0;
    {
        const double rmax = fmax(fabs(rT), fabs(__shfl_xor_sync(0xffffffffu, rT, 16)));
        if (rmax > 0.0 && isfinite(rmax)) frexp(rmax, &ey);
    }
    const double rs = ldexp(rT, -ey);
    const float4 *tb = reinterpret_cast<const float4 *>(sa) + st * 4;       // pair p: tb[p * 8 + k]
    const float2 *wdf = reinterpret_cast<const float2 *>(sa + 16 * NP) + st * 2;  // i: wdf[i * 4 + {0, 1}]
    const double *dn = st ? d2 : d1, *qn = st ? q2 : q1;
    const double dq0 = qn[0];
    float4 *Vc = V + tid, *Wc = W + tid;
    float2 *Rc = Rm + tid;
    double lp1 = 0.0, lp2 = 0.0, db = 0.0, sg = 0.0, sx = 0.0, lam1 = 0.0, lam2 = 0.0, mu1 = 0.0;
    int slot = (int)(N % L);
    for (int64_t m = N; m >= 1; --m) {
        const float2 in = Rc[(size_t)slot * T];             // mu^{m+L}
        const float2 gh = make_float2(in.x, in.x), gl = make_float2(in.y, in.y);
        float2 hh = make_float2(0.f, 0.f), hl = hh, kh = hh, kl = hh;
#pragma unroll
        for (int p = 0; p < NP / 2; ++p) {
            const float4 A = tb[p * 8], Cc = tb[p * 8 + 1], Cp = tb[p * 8 + 2], Cr = tb[p * 8 + 3];
            const float4 v4 = Vc[(size_t)p * T], w4 = Wc[(size_t)p * T];
            float2 vh = make_float2(v4.x, v4.y), vl = make_float2(v4.z, v4.w);
            float2 wh = make_float2(w4.x, w4.y), wl = make_float2(w4.z, w4.w);
            const float2 ah = make_float2(A.x, A.y), al = make_float2(A.z, A.w);
            // W <- a W + V (with V^{m+1}), then V <- a V + mu^{m+L}
            if (2 * p < KR) {
                node_r2(ah, al, vh, vl, wh, wl);
                node_r2(ah, al, gh, gl, vh, vl);
            } else {
                node_u2(ah, al, vh, vl, wh, wl);
                node_u2(ah, al, gh, gl, vh, vl);
            }
            Vc[(size_t)p * T] = make_float4(vh.x, vh.y, vl.x, vl.y);
            Wc[(size_t)p * T] = make_float4(wh.x, wh.y, wl.x, wl.y);
            acc_prod2(make_float2(Cc.x, Cc.y), make_float2(Cc.z, Cc.w), vh, vl, hh, hl);
            acc_prod2(make_float2(Cp.x, Cp.y), make_float2(Cp.z, Cp.w), vh, vl, kh, kl);
            acc_prod2(make_float2(Cr.x, Cr.y), make_float2(Cr.z, Cr.w), wh, wl, kh, kl);
        }
        // exact window of d and d': mu^{m+i} at slot (m + i) % L
        float wh_ = 0.f, wl_ = 0.f, qh_ = 0.f, ql_ = 0.f;
        int sl = slot;
        for (int i = 1; i < L; ++i) {
            sl = (sl + 1 == L) ? 0 : sl + 1;
            const float2 u = Rc[(size_t)sl * T], dw = wdf[i * 4], dqw = wdf[i * 4 + 1];
            acc_prod(dw.x, dw.y, u.x, u.y, wh_, wl_);
            acc_prod(dqw.x, dqw.y, u.x, u.y, qh_, ql_);
        }
        float hs, he, ks, ke;
        tsum(hh.x, hh.y, hs, he);
        tsum(kh.x, kh.y, ks, ke);
        const double hr = ((double)hs + (double)fadd(he, fadd(hl.x, hl.y))) + ((double)wh_ + (double)wl_);
        const double hq0 = ((double)ks + (double)fadd(ke, fadd(kl.x, kl.y))) + ((double)qh_ + (double)ql_);
        double b = -hr;
        if (m == N) b -= rs;
        const bool first = (P.scheme == CQ_BDF2 && m == 1);
        if (P.scheme == CQ_BE) {
            if (m < N) b += lp1 * it;
        } else {
            if (m + 1 <= N) b += 2.0 * it * lp1;
            if (m + 2 <= N) b -= 0.5 * it * lp2;
        }
        const double b_o = __shfl_xor_sync(0xffffffffu, b, 16);
        const double l = first ? fma(m1_oo, b, m1_ot * b_o) : fma(mn_oo, b, mn_ot * b_o);
        const double l_o = __shfl_xor_sync(0xffffffffu, l, 16);
        const double v = c * l - a * l_o;
        Rc[(size_t)slot * T] = df_of(v);
        const double hq = fma(dq0, v, hq0);
        db = fma(hist[(m * 2 + st) * nm + mode], hq, db);
        if (m >= 2) {
            sg = fma(__ldg(dn + m - 1), v, sg);
            sx = fma(__ldg(qn + m - 1), v, sx);
        }
        if (m == 1) {
            lam1 = l;
            mu1 = v;
        } else if (m == 2) {
            lam2 = l;
        }
        lp2 = lp1;
        lp1 = l;
        slot = (slot == 0) ? L - 1 : slot - 1;
    }
    const double x0 = hist[st * nm + mode];
    double g;
    if (P.scheme == CQ_BE) {
        g = -lam1 * it;
    } else {
        g = -lam1 * it + (st ? d20 : d10) * mu1 / 3.0 + 0.5 * it * lam2 + 0.5 * sg;
        const double x1 = hist[(2 + st) * nm + mode];
        db += mu1 * dq0 * (x0 - x1) / 3.0 + 0.5 * x0 * sx;
    }
    if (active) {
        gx0[st * nm + mode] = ldexp(g, ey);
        db = ldexp(db, ey);
    } else {
        db = 0.0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) Jpart += __shfl_xor_sync(0xffffffffu, Jpart, off);
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) db += __shfl_xor_sync(0xffffffffu, db, off);
    if (lane == 0) {
        atomicAdd(acc + 0, Jpart);
        atomicAdd(acc + 1, db);
    } else if (lane == 16) {
        atomicAdd(acc + 2, db);
    }
    if (active && st == 0 && !ok) atomicAdd(acc + 3, 1.0);
}

int fast_adjoint_df_tables(const Fp2sParams &P, const double *tab1, const double *tab2, const double *der1,
                           const double *der2, const double *d1, const double *d2, const double *q1,
                           const double *q2, float *out, cudaStream_t s) {
    const int NP = df_np_class(P.np);
    if (NP == 0 || adj_df_table_floats(NP) > kAdjDfTabFloats) return CQ_EUNSUPPORTED;
    k_adj_df_tables<<<1, 256, 0, s>>>(NP, P.np, P.L, P.N, tab1, tab2, der1, der2, d1, d2, q1, q2, out);
    return launched();
}

int fast_adjoint_df_slice(const Fp2sParams &P, double wd, const double *lam, const double *d1, const double *d2,
                          const double *q1, const double *q2, const float *adtab, const double *hist,
                          const double *tgt, int vjp, double *gx0, double *acc, cudaStream_t s) {
    const int NP = df_np_class(P.np);
    if (NP == 0) return CQ_EUNSUPPORTED;
    int T = kAdjFastMaxT;
    while (T > 32 && adj_df_smem(NP, P.L, T) > 227 * 1024) T /= 2;
    const size_t smem = adj_df_smem(NP, P.L, T);
    if (smem > 227 * 1024) return CQ_EUNSUPPORTED;
    const int64_t mpb = (int64_t)(T / 32) * kFastModesPerWarp;
    const unsigned blocks = (unsigned)((P.nmodes + mpb - 1) / mpb);
    int st = CQ_OK;
    auto run = [&](auto kern, unsigned long long *attr) {
        if ((st = smem_attr_once((const void *)kern, 227 * 1024, attr))) return;
        kern<<<blocks, T, smem, s>>>(P, wd, lam, d1, d2, q1, q2, adtab, hist, tgt, vjp, gx0, acc);
        st = launched();
    };
#define CQ_ADJ_DF(NPV)                          \
    case NPV: {                                 \
        static unsigned long long attr = 0;     \
        run(k_adjoint_fast_df<NPV>, &attr);     \
        break;                                  \
    }
    switch (NP) {
        CQ_ADJ_DF(16)
        CQ_ADJ_DF(32)
        CQ_ADJ_DF(48)
        CQ_ADJ_DF(64)
        CQ_ADJ_DF(80)
        CQ_ADJ_DF(96)
        CQ_ADJ_DF(112)
        CQ_ADJ_DF(128)
        default: return CQ_EUNSUPPORTED;
    }
#undef CQ_ADJ_DF
    return st;
}

}  // namespace fastcq
