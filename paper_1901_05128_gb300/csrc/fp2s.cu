// Two-state fractional Fokker-Planck schemes (Eqs. 4.1, 4.3, 4.7, 4.8) in the
// sine basis of the Dirichlet finite-difference Laplacian. Every mode k
// (eigenvalue lambda_k) is an independent pair (g1, g2); with c = a + lambda_k:
//
//   BE, n >= 1:       [1/tau + c d1_0, -a d2_0; -a d1_0, 1/tau + c d2_0] g^n
//                       = g^{n-1}/tau - c h_s + a h_o          (per state s, other o)
//   SBD, n = 1:       [1/tau + 2/3 c d1_0, -2/3 a d2_0; ...] g^1
//                       = g^0/tau - 1/3 c d_s0 g_s^0 + 1/3 a d_o0 g_o^0
//   SBD, n >= 2:      [3/(2tau) + c d1_0, -a d2_0; ...] g^n
//                       = (2 g^{n-1} - g^{n-2}/2)/tau - c e_s + a e_o,  e = h + d_{n-1} g^0 / 2
//
// h is the direct history sum_{i=1}^{n-1} d_i g^{n-i} or the fast one
// (geometric history parts). The step matrix is the same for every n >= 2
// (BE: n >= 1), so its inverse is formed once per mode.
//
// fp2s_solve runs all N steps of a mode inside one thread of one persistent
// kernel: modes never interact, so there is no grid-wide synchronisation.
#include "common.cuh"
#include "fastgrad.cuh"
#include "fp2s_core.cuh"

namespace fastcq {

constexpr int kDirBT = 8;        // time block of the fused direct kernel
constexpr int kF32TabFloats = 1024;   // FP32 fast form: node tables (<= 4*128 + 8*8 + 2 floats)

struct Fp2sLayout {
    int *status;
    double *d1, *d2, *dz1, *dz2;
    double *tab1, *tab2, *scr1, *scr2;
    double *lam, *S, *tmp, *g0, *gN;
    float *hdf;                   // FP32 fast form: 0.5*d_i of both states as double-float, [4][N+1]
    float *ftab;                  // FP32 fast form: node tables in the fused kernel's order (k_f32_tables)
    double *hist;                 // direct: (N+1) x 2 x nmodes
    float4 *wz, *hist2;           // direct, CQ_DF64: padded double-float weights; levels [N+1][nmodes]
    double *Y, *ring, *glast;     // step API, fast: 2 x np x nm, 2 x L x nm; both: 2 levels x 2 x nm
    void *mixed;                  // direct, CQ_BF16X3 / CQ_TF32X3: region of the mixed-precision solve
    double *wscr;                 // N > kMaxWeights: scratch of the weight builder
    size_t bytes;
};

// hist_modes: modes of the FP64 level history (all modes unless a gradient runs in slices); the
// direct FP64 solve keeps it, and so does the fast FP64 form inside a gradient (grad).
// lam_modes: eigenvalues computed (all modes of the grid when the solve covers a range of them).
static Fp2sLayout fp2s_layout(const fp2s_problem_t *p, const Fp2sParams &P, void *ws, bool stepper,
                              bool grad = false, int64_t hist_modes = -1, int64_t lam_modes = -1) {
    Carve cv(ws);
    Fp2sLayout l{};
    const int64_t nm = P.nmodes;
    l.status = cv.take<int>(64);
    l.d1 = cv.take<double>(P.N + 1);
    l.d2 = cv.take<double>(P.N + 1);
    if (P.N > kMaxWeights) l.wscr = cv.take<double>(P.N + 1);
    if (P.form == CQ_DIRECT && P.prec == CQ_F64) {
        l.dz1 = cv.take<double>(P.N + 2 * kDirBT + 1);
        l.dz2 = cv.take<double>(P.N + 2 * kDirBT + 1);
    } else if (P.form == CQ_FAST) {
        l.tab1 = cv.take<double>(2 * P.np);
        l.tab2 = cv.take<double>(2 * P.np);
        l.scr1 = cv.take<double>(2 * P.np);
        l.scr2 = cv.take<double>(2 * P.np);
    }
    l.lam = cv.take<double>(lam_modes < 0 ? nm : lam_modes);
    l.S = cv.take<double>((size_t)p->M * p->M);
    l.tmp = cv.take<double>(2 * nm);
    l.g0 = cv.take<double>(2 * nm);
    l.gN = cv.take<double>(2 * nm);
    if (((P.form == CQ_DIRECT || grad) && P.prec == CQ_F64) || (grad && P.form == CQ_FAST && P.prec == CQ_DF64))
        l.hist = cv.take<double>((size_t)(P.N + 1) * 2 * (hist_modes < 0 ? nm : hist_modes));
    if (P.form == CQ_DIRECT && P.prec == CQ_DF64) {
        l.wz = cv.take<float4>(P.N + 2 * kDirDfBT + 1);
        l.hist2 = cv.take<float4>((size_t)(P.N + 1) * (hist_modes < 0 ? nm : hist_modes));
    }
    if (P.prec != CQ_F64 && P.prec != CQ_DF64) l.hdf = cv.take<float>((size_t)4 * (P.N + 1));
    if (P.form == CQ_FAST && P.prec == CQ_F32) l.ftab = cv.take<float>(kF32TabFloats);
    if (P.form == CQ_FAST && P.prec == CQ_DF64) l.ftab = cv.take<float>(kDfTabFloats);
    if (P.form == CQ_DIRECT && (P.prec == CQ_BF16X3 || P.prec == CQ_TF32X3)) {
        Fp2sParams Pm = P;                 // a gradient may run over slices of hist_modes modes
        if (grad && hist_modes >= 0) Pm.nmodes = hist_modes;
        l.mixed = cv.take<char>(grad ? mixed_grad_bytes(Pm) : mixed_direct_bytes(Pm));
    }
    if (stepper) {
        if (P.form == CQ_FAST) {
            l.Y = cv.take<double>((size_t)2 * P.np * nm);
            l.ring = cv.take<double>((size_t)2 * P.L * nm);
        }
        l.glast = cv.take<double>((size_t)4 * nm);
    }
    l.bytes = cv.bytes();
    return l;
}

static int derive(const fp2s_problem_t *p, Fp2sParams &P, int &np1, int &np2) {
    if (!p) return CQ_EINVAL;
    if (!(p->alpha1 > 0.0 && p->alpha1 < 1.0 && p->alpha2 > 0.0 && p->alpha2 < 1.0)) return CQ_EINVAL;
    if (!(p->m >= 0.0 && p->m < 1.0) || p->m == 0.5) return CQ_EINVAL;
    if (!(p->T > 0.0) || p->N < 1 || p->N > kMaxSolveSteps) return CQ_EINVAL;
    if (p->dim < 1 || p->dim > 3) return CQ_EINVAL;
    if (p->M < 1 || p->M > (p->dim == 1 ? (1 << 16) : p->dim == 2 ? 4096 : 1024)) return CQ_EINVAL;
    if (p->scheme != CQ_BE && p->scheme != CQ_BDF2) return CQ_EINVAL;
    if (p->form != CQ_DIRECT && p->form != CQ_FAST) return CQ_EINVAL;
    if (p->prec != CQ_F64 && p->prec != CQ_DF64 && !(p->prec == CQ_F32 && p->form == CQ_FAST) &&
        !((p->prec == CQ_BF16X3 || p->prec == CQ_TF32X3) && p->form == CQ_DIRECT))
        return CQ_EUNSUPPORTED;
    P.prec = p->prec;
    P.a = (1.0 - p->m) / (2.0 * p->m - 1.0);
    P.tau = p->T / (double)p->N;
    P.inv_tau = 1.0 / P.tau;
    P.N = p->N;
    P.nmodes = (p->dim == 1) ? p->M : (p->dim == 2) ? (int64_t)p->M * p->M : (int64_t)p->M * p->M * p->M;
    P.scheme = p->scheme;
    P.form = p->form;
    np1 = p->fast.np1;
    np2 = (p->scheme == CQ_BE) ? 0 : p->fast.np2;
    P.L = (p->scheme == CQ_BE) ? 2 : p->fast.ns;
    P.np = np1 + np2;
    if (p->form == CQ_FAST) {
        if (np1 < 1 || np2 < 0 || P.np > kMaxNp) return CQ_EINVAL;
        if (p->scheme == CQ_BDF2 && (np2 < 1 || P.L < 3 || P.L > kMaxNs)) return CQ_EINVAL;
        if (P.prec == CQ_DF64 && df_np_bound(P.np) == 0) return CQ_EUNSUPPORTED;
    }
    return CQ_OK;
}

// ---------------------------------------------------------------------------
// Fused fast solve. Each mode is carried by two lanes of one warp for all N
// steps: lane l < 16 holds state 1 and lane l + 16 state 2 of the same mode,
// so a warp advances 16 modes. A lane owns the history-part states
// Y[j][tid] and the last L levels R[slot][tid] (level k in slot k % L) of its
// state in shared memory (column tid: conflict-free); the two lanes of a mode
// swap e = h (+ G^0 correction) and the right-hand side b with one shuffle
// each to finish the 2x2 step. Tables are interleaved by state (word 2j + s)
// so the two half-warps read different banks. Four partial sums break the
// dependency chain of h = sum_j c_j Y_j. With HIST (the forward sweep of the fast-form
// gradient) every level is also stored: hist[(n * 2 + s) * nmodes + mode], n = 0 .. N.
// ---------------------------------------------------------------------------
template <bool HIST>
__global__ void __launch_bounds__(1024) k_fp2s_fast(Fp2sParams P, const double *__restrict__ lam,
                                                    const double *__restrict__ g0, double *__restrict__ gN,
                                                    int *__restrict__ status, const double *__restrict__ d1,
                                                    const double *__restrict__ d2, const double *__restrict__ tab1,
                                                    const double *__restrict__ tab2, double *__restrict__ hist) {
    extern __shared__ double sm[];
    const int np = P.np, L = P.L, T = blockDim.x, tid = threadIdx.x;
    double *rt = sm;                          // rt[2j + s] = r_j of state s
    double *ct = rt + 2 * np;                 // ct[2j + s] = c_j of state s
    double *wt = ct + 2 * np;                 // wt[2i + s] = d_i of state s, i < L
    double *Y = wt + 2 * kMaxNs;              // [np][T]
    double *R = Y + (size_t)np * T;           // [L][T]
    for (int i = tid; i < np; i += T) {
        rt[2 * i] = tab1[i];
        rt[2 * i + 1] = tab2[i];
        ct[2 * i] = tab1[np + i];
        ct[2 * i + 1] = tab2[np + i];
    }
    for (int i = tid; i < L; i += T) {
        wt[2 * i] = d1[i];
        wt[2 * i + 1] = d2[i];
    }
    for (int j = 0; j < np; ++j) Y[(size_t)j * T + tid] = 0.0;
    for (int j = 0; j < L; ++j) R[(size_t)j * T + tid] = 0.0;
    __syncthreads();

    const int lane = tid & 31, st = lane >> 4;            // st: 0 = state 1, 1 = state 2
    const int64_t mode_raw = ((int64_t)blockIdx.x * (T >> 5) + (tid >> 5)) * kFastModesPerWarp + (lane & 15);
    const bool active = mode_raw < P.nmodes;
    const int64_t mode = active ? mode_raw : 0;           // idle lanes still take part in the shuffles
    const double *rs = rt + st, *cs = ct + st, *ws = wt + st;
    const double *dn = st ? d2 : d1;
    double *Yc = Y + tid, *Rc = R + tid;

    const double gz = g0[st * P.nmodes + mode];
    if (HIST && active) hist[st * P.nmodes + mode] = gz;
    const double d_s0 = ws[0], d_o0 = wt[1 - st];
    ModeConst mc;
    const bool ok = mode_setup(P, lam[mode], st ? d_o0 : d_s0, st ? d_s0 : d_o0, mc);
    if (active && st == 0 && !ok) atomicOr(status, ST_SINGULAR);
    // own row of the inverse step matrices, ordered (own, other)
    const double mn_oo = st ? mc.Mn.i22 : mc.Mn.i11, mn_ot = st ? mc.Mn.i21 : mc.Mn.i12;
    const double m1_oo = st ? mc.M1.i22 : mc.M1.i11, m1_ot = st ? mc.M1.i21 : mc.M1.i12;
    const double a = P.a, c = mc.c;
    double gm1 = gz, gm2 = 0.0;
    int slot = 0;                                           // n % L
    for (int64_t n = 1; n <= P.N; ++n) {
        slot = (slot + 1 == L) ? 0 : slot + 1;
        double h0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0;
        if (n - L >= 1) {
            const double in = Rc[(size_t)slot * T];
            int j = 0;
            for (; j + 4 <= np; j += 4) {
                const double y0 = fma(rs[2 * j], Yc[(size_t)j * T], in);
                const double y1 = fma(rs[2 * j + 2], Yc[(size_t)(j + 1) * T], in);
                const double y2 = fma(rs[2 * j + 4], Yc[(size_t)(j + 2) * T], in);
                const double y3 = fma(rs[2 * j + 6], Yc[(size_t)(j + 3) * T], in);
                Yc[(size_t)j * T] = y0;
                Yc[(size_t)(j + 1) * T] = y1;
                Yc[(size_t)(j + 2) * T] = y2;
                Yc[(size_t)(j + 3) * T] = y3;
                h0 = fma(cs[2 * j], y0, h0);
                h1 = fma(cs[2 * j + 2], y1, h1);
                h2 = fma(cs[2 * j + 4], y2, h2);
                h3 = fma(cs[2 * j + 6], y3, h3);
            }
            for (; j < np; ++j) {
                const double y = fma(rs[2 * j], Yc[(size_t)j * T], in);
                Yc[(size_t)j * T] = y;
                h0 = fma(cs[2 * j], y, h0);
            }
        }
        const int imax = (int)min((int64_t)(L - 1), n - 1);
        int sl = slot;
        for (int i = 1; i <= imax; ++i) {
            sl = (sl == 0) ? L - 1 : sl - 1;                // slot of level n - i
            if (i & 1) h1 = fma(ws[2 * i], Rc[(size_t)sl * T], h1);
            else h2 = fma(ws[2 * i], Rc[(size_t)sl * T], h2);
        }
        const double h = (h0 + h1) + (h2 + h3);
        double e, lead, m_oo = mn_oo, m_ot = mn_ot;
        if (P.scheme == CQ_BE) {
            e = h;
            lead = gm1 * P.inv_tau;
        } else if (n == 1) {
            e = d_s0 * gz * (1.0 / 3.0);
            lead = gz * P.inv_tau;
            m_oo = m1_oo;
            m_ot = m1_ot;
        } else {
            e = fma(0.5 * __ldg(dn + n - 1), gz, h);
            lead = (2.0 * gm1 - 0.5 * gm2) * P.inv_tau;
        }
        const double e_o = __shfl_xor_sync(0xffffffffu, e, 16);
        const double b = lead - c * e + a * e_o;
        const double b_o = __shfl_xor_sync(0xffffffffu, b, 16);
        const double x = m_oo * b + m_ot * b_o;
        Rc[(size_t)slot * T] = x;
        if (HIST && active) hist[(n * 2 + st) * P.nmodes + mode] = x;
        gm2 = gm1;
        gm1 = x;
    }
    if (active) {
        gN[st * P.nmodes + mode] = gm1;
        if (!isfinite(gm1)) atomicOr(status, ST_NONFINITE);
    }
}

// ---------------------------------------------------------------------------
// Fused fast solve for problems with few modes (1D grids, small 2D grids): one
// warp per mode, lanes l < 16 state 1 and l + 16 state 2 as above, and the
// history nodes of a state split over its 16 lanes (node j on lane j % 16), so
// a lane keeps only its NPL states Y_j and table entries in registers. The
// partial sums meet through xor shuffles inside the half-warp; every lane then
// takes the step itself and lane 0 of each half stores the new level into the
// warp's ring of the last L levels in shared memory.
// ---------------------------------------------------------------------------
template <int NPL>
__global__ void __launch_bounds__(32) k_fp2s_fast_split(Fp2sParams P, const double *__restrict__ lam,
                                                        const double *__restrict__ g0, double *__restrict__ gN,
                                                        int *__restrict__ status, const double *__restrict__ d1,
                                                        const double *__restrict__ d2,
                                                        const double *__restrict__ tab1,
                                                        const double *__restrict__ tab2) {
    __shared__ double ring[2][kMaxNs];
    const int lane = threadIdx.x, st = lane >> 4, sub = lane & 15;
    const int64_t mode = blockIdx.x;
    const int np = P.np, L = P.L;
    const double *tab = st ? tab2 : tab1;
    double Y[NPL], r[NPL], c[NPL];
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
        const int j = sub + 16 * q;
        r[q] = j < np ? tab[j] : 0.0;
        c[q] = j < np ? tab[np + j] : 0.0;
        Y[q] = 0.0;
    }
    for (int i = lane; i < 2 * kMaxNs; i += 32) ring[i / kMaxNs][i % kMaxNs] = 0.0;
    __syncwarp();
    double *rs = ring[st];
    const double *dn = st ? d2 : d1;

    const double gz = g0[st * P.nmodes + mode];
    const double d_s0 = __ldg(dn), d_o0 = __ldg(st ? d1 : d2);
    ModeConst mc;
    const bool ok = mode_setup(P, lam[mode], st ? d_o0 : d_s0, st ? d_s0 : d_o0, mc);
    if (lane == 0 && !ok) atomicOr(status, ST_SINGULAR);
    const double mn_oo = st ? mc.Mn.i22 : mc.Mn.i11, mn_ot = st ? mc.Mn.i21 : mc.Mn.i12;
    const double m1_oo = st ? mc.M1.i22 : mc.M1.i11, m1_ot = st ? mc.M1.i21 : mc.M1.i12;
    const double a = P.a, cc = mc.c;
    double gm1 = gz, gm2 = 0.0;
    int slot = 0;
    for (int64_t n = 1; n <= P.N; ++n) {
        slot = (slot + 1 == L) ? 0 : slot + 1;
        double ha = 0.0, hb = 0.0;
        if (n - L >= 1) {
            const double in = rs[slot];
#pragma unroll
            for (int q = 0; q < NPL; q += 2) {
                Y[q] = fma(r[q], Y[q], in);
                ha = fma(c[q], Y[q], ha);
                if (q + 1 < NPL) {
                    Y[q + 1] = fma(r[q + 1], Y[q + 1], in);
                    hb = fma(c[q + 1], Y[q + 1], hb);
                }
            }
        }
        const int imax = (int)min((int64_t)(L - 1), n - 1);
        for (int i = 1 + sub; i <= imax; i += 16) {         // this lane's terms of the exact window
            const int sl = (slot - i + L) % L;                // slot of level n - i
            ha = fma(__ldg(dn + i), rs[sl], ha);
        }
        double h = ha + hb;
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) h += __shfl_xor_sync(0xffffffffu, h, off);
        double e, lead, m_oo = mn_oo, m_ot = mn_ot;
        if (P.scheme == CQ_BE) {
            e = h;
            lead = gm1 * P.inv_tau;
        } else if (n == 1) {
            e = d_s0 * gz * (1.0 / 3.0);
            lead = gz * P.inv_tau;
            m_oo = m1_oo;
            m_ot = m1_ot;
        } else {
            e = fma(0.5 * __ldg(dn + n - 1), gz, h);
            lead = (2.0 * gm1 - 0.5 * gm2) * P.inv_tau;
        }
        const double e_o = __shfl_xor_sync(0xffffffffu, e, 16);
        const double b = lead - cc * e + a * e_o;
        const double b_o = __shfl_xor_sync(0xffffffffu, b, 16);
        const double x = m_oo * b + m_ot * b_o;
        __syncwarp();                                         // every lane has read the slot's old level
        if (sub == 0) rs[slot] = x;
        __syncwarp();
        gm2 = gm1;
        gm1 = x;
    }
    if (sub == 0) {
        gN[st * P.nmodes + mode] = gm1;
        if (!isfinite(gm1)) atomicOr(status, ST_NONFINITE);
    }
}

// Modes below which the fast solve gives each mode a whole warp (fewer than four
// warps per SM with 16 modes per warp).
static bool fast_use_split(int64_t nmodes) { return nmodes < (int64_t)152 * 4 * kFastModesPerWarp; }

static int launch_fast_split(const Fp2sParams &P, const Fp2sLayout &l, cudaStream_t s) {
    const int npl = (P.np + 15) / 16;
    const unsigned grid = (unsigned)P.nmodes;
#define CQ_FAST_SPLIT(NPLV) \
    k_fp2s_fast_split<NPLV><<<grid, 32, 0, s>>>(P, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.tab1, l.tab2)
    if (npl <= 2) CQ_FAST_SPLIT(2);
    else if (npl <= 4) CQ_FAST_SPLIT(4);
    else if (npl <= 8) CQ_FAST_SPLIT(8);
    else if (npl <= 16) CQ_FAST_SPLIT(16);
    else return CQ_EUNSUPPORTED;
#undef CQ_FAST_SPLIT
    return CQ_OK;
}

static size_t fast_smem_bytes(int np, int L, int T) {
    return ((size_t)4 * np + 2 * kMaxNs + (size_t)(np + L) * T) * sizeof(double);
}

static int num_sms() { return device_sms(); }

// Warps per block: the largest that fits shared memory among those whose grid
// fills whole waves best (one block per SM).
static int fast_block_threads(int np, int L, int64_t nmodes) {
    const size_t limit = 227 * 1024;
    const int sms = num_sms();
    int best = 0;
    double best_eff = -1.0;
    for (int wb = 32; wb >= 1; --wb) {
        if (fast_smem_bytes(np, L, 32 * wb) > limit) continue;
        const int64_t blocks = (nmodes + (int64_t)kFastModesPerWarp * wb - 1) / ((int64_t)kFastModesPerWarp * wb);
        const int64_t waves = (blocks + sms - 1) / sms;
        const double eff = (double)nmodes / (double)(waves * sms * kFastModesPerWarp * wb);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = wb;
        }
    }
    return best * 32;
}

// ---------------------------------------------------------------------------
// Fused fast solve, FP32 precision form. Each lane carries one state of TWO
// modes over HALF of the history-part nodes: lanes l = 16 s + 8 h + q hold state s
// of the modes 2p, 2p + 1 of pair p = 8 w + q (w the warp) over the nodes of half h.
// One 16-byte table word (r_j, c_j r_j, r_{j+1}, c_{j+1} r_{j+1}) then feeds both
// modes (eight FMAs), and the four (half, state) words a load touches are adjacent.
// The history sum is taken from the states before their update,
//     h^n = sum_j c_j Y_j^n = sum_j (c_j r_j) Y_j^{n-1} + C G^{n-L},  C = sum_j c_j,
// so the FMAs of a node do not wait on each other. Per step the two halves add their
// partial sums with one shuffle per mode, lane h takes the 2x2 step of mode 2p + h with
// its partner state (lane ^ 16), and the two new levels are exchanged with one shuffle;
// the exact window (L - 1 terms) is split between the halves by parity. Each lane keeps
// its own ring of the last L levels of its two modes (float2) in shared memory. The
// states Y_j live in FP32 registers (NP is a compile-time bound; the tables are
// zero-padded up to it). Weights, quadrature coefficients and the per-mode step
// matrices are computed in FP64; the step is evaluated from the FP32 history sums in
// the two-term form x = A l + B e with double-float A and B (lane_step2), or in FP64
// when the coupling is strong (|a| > 10, i.e. m within ~0.045 of 1/2); the first SBD
// step uses the double-float form. Every mode is pre-scaled by an exact power of two
// (from its G^0) so that its values sit near 1 in FP32 range; the factor is undone on
// output.
// ---------------------------------------------------------------------------
constexpr int kF32Threads = 128;

// Node pairs per lane (NQ = NP / 4) of the FP32 fast form whose ratios r_j are kept as
// double-float (r = fl(r) + r_lo): the top quarter of the slots, which hold the slowest
// decaying nodes. A ratio near 1 rounded to FP32 changes 1 - r by up to 2^-25 / (1 - r)
// relatively, and the geometric sum carries that error over ~1 / (1 - r) steps: with 128
// points at tau = 1/8192 the slowest nodes have 1 - r ~ 2e-4, and the rounded ratios alone
// put ~5e-5 into the solution. Faster nodes (1 - r > ~0.15) lose < 2e-7 this way.
__host__ __device__ constexpr int f32_df_pairs(int NP) { return NP / 16 > 0 ? NP / 16 : 1; }

// FP32 tables of the fused FP32 fast solve, in the order the kernel reads them
// (ftab: [4 NP] float4-packed words, then [8 KD] floats, then 2 floats):
//   per state s the np nodes are ranked by r (ascending, ties by index) and placed in the
//   top np of the NP slots; slot t = 4 kk + 2 hf + e of state s sits in word 4 kk + 2 hf + s,
//   which holds (r_t0, r_t1, c r_t0, c r_t1) for its two slots e = 0, 1 (so that each pair
//   feeds one packed two-wide FMA); the bottom NP - np slots are zero. The top 4 KD slots
//   also get r - fl(r) in the float2 word 4 (kk - (NQ - KD)) + 2 hf + s, component e.
//   The last two floats are C_s = sum_j c_j.
// One block of 256 threads (2 np <= 256).
__global__ void k_f32_tables(int NP, int KD, int np, const double *__restrict__ tab1, const double *__restrict__ tab2,
                             float *__restrict__ out) {
    const int NQ = NP / 4, tid = threadIdx.x;
    float *tab = out, *tlo = out + 4 * NP, *csum = tlo + 8 * KD;
    for (int i = tid; i < 4 * NP + 8 * KD; i += blockDim.x) out[i] = 0.0f;
    __syncthreads();
    for (int e = tid; e < 2 * np; e += blockDim.x) {
        const int st = e / np, j = e - st * np;
        const double *tq = st ? tab2 : tab1;
        const double r = tq[j];
        int rank = 0;
        for (int k = 0; k < np; ++k) {
            const double rk = tq[k];
            rank += (rk < r || (rk == r && k < j)) ? 1 : 0;
        }
        const int t = NP - np + rank, kk = t >> 2, hf = (t >> 1) & 1, el = t & 1;
        const float rf = (float)r;
        float *w = tab + 4 * (4 * kk + 2 * hf + st);
        w[el] = rf;
        w[2 + el] = (float)(tq[np + j] * r);
        if (kk >= NQ - KD) tlo[2 * (4 * (kk - (NQ - KD)) + 2 * hf + st) + el] = (float)(r - (double)rf);
    }
    if (tid < 2) {
        const double *tq = tid ? tab2 : tab1;
        double c = 0.0;
        for (int j = 0; j < np; ++j) c += tq[np + j];
        csum[tid] = (float)c;
    }
}

// ---------------------------------------------------------------------------
// Fused fast solve, FP32 precision form. Each lane carries one state of TWO
// modes over HALF of the history-part nodes: lanes l = 16 s + 8 h + q hold state s
// of the modes 2p, 2p + 1 of pair p = 8 w + q (w the warp) over the node slots
// 4 kk + 2 h, 4 kk + 2 h + 1 (kk < NP / 4), so both halves hold nodes of similar r at
// the same kk. One 16-byte table word (r_j, r_{j+1}, c_j r_j, c_{j+1} r_{j+1}) then feeds
// both modes (eight FMAs, issued as four packed two-wide FMAs: Blackwell's FFMA2 halves the
// instructions of the node work, which bounds this kernel by issue rather than by the FMA
// pipe), and the four (half, state) words a load touches are adjacent.
// The history sum is taken from the states before their update,
//     h^n = sum_j c_j Y_j^n = sum_j (c_j r_j) Y_j^{n-1} + C G^{n-L},  C = sum_j c_j,
// so the FMAs of a node do not wait on each other. The slowest quarter of the nodes
// (the top slots) update with a double-float ratio, Y = fl(r) Y + (r_lo Y + G): one more
// FMA per node. Per step the two halves add their partial sums with one shuffle per mode,
// lane h takes the 2x2 step of mode 2p + h with its partner state (lane ^ 16), and the two
// new levels are exchanged with one shuffle; the exact window (L - 1 terms) is split between
// the halves by parity. Each lane keeps its own ring of the last L levels of its two modes
// (float2) in shared memory. The states Y_j live in FP32 registers (NP is a compile-time
// bound; the tables are zero-padded up to it). Weights, quadrature coefficients and the
// per-mode step matrices are computed in FP64; the step is evaluated from the FP32 history
// sums in the two-term form x = A l + B e with double-float A and B (lane_step2_df), or in
// FP64 when the coupling is strong (|a| > 10, i.e. m within ~0.045 of 1/2); the first SBD
// step uses the double-float form. The lane's own level is carried between steps as a
// double-float pair: its low part enters l and, through d_1 x_lo^{n-1}, e (the term of the
// window with the largest weight); the ring, the node inputs and the other window terms
// use the FP32 part. Every mode is pre-scaled by an exact power of two (from its G^0) so
// that its values sit near 1 in FP32 range; the factor is undone on output.
// ---------------------------------------------------------------------------

// The FP64 / first-SBD step of the FP32 form, out of line (it runs on rare steps only).
__device__ __noinline__ df lane_step_rare(const Fp2sParams P, const LaneStep ls, int solve64, int64_t n, float h,
                                          float gm1, float gm2, float gz, const double *dn, const float *hd_hi,
                                          const float *hd_lo) {
    return lane_step_df(P, ls, solve64, n, h, gm1, gm2, gz, dn, hd_hi, hd_lo);
}

// Node part of one step (two modes, this lane's half of the nodes): the partial history
// sums sum_j (c_j r_j) Y_j^{n-1} + C G^{n-L} into hA / hB, then Y_j^n = r_j Y_j^{n-1} + G^{n-L}
// (the last KD node pairs with the double-float ratio fl(r_j) + r_lo_j from tl). YA[kk] holds the
// states of the node pair kk of mode A; every FMA is a packed two-wide one over such a pair
// (each component rounded as a scalar FMA). Partial sum q of a mode: pair parity q >> 1, pair
// element q & 1.
template <int NQ, int KD>
__device__ __forceinline__ void f32_node_part(const float4 *tb, const float2 *tl, float cs, float2 in,
                                              float2 (&YA)[NQ], float2 (&YB)[NQ], float (&hA)[4],
                                              float (&hB)[4]) {
    float2 pA[2] = {make_float2(cs * in.x, 0.0f), make_float2(0.0f, 0.0f)};
    float2 pB[2] = {make_float2(cs * in.y, 0.0f), make_float2(0.0f, 0.0f)};
    const float2 gA = make_float2(in.x, in.x), gB = make_float2(in.y, in.y);
#pragma unroll
    for (int kk = 0; kk < NQ; ++kk) {
        const float4 t = tb[4 * kk];
        const float2 r = make_float2(t.x, t.y), cr = make_float2(t.z, t.w);
        const int c = kk & 1;
        pA[c] = __ffma2_rn(cr, YA[kk], pA[c]);
        pB[c] = __ffma2_rn(cr, YB[kk], pB[c]);
        if (kk >= NQ - KD) {
            const float2 lo = tl[4 * (kk - (NQ - KD))];
            YA[kk] = __ffma2_rn(r, YA[kk], __ffma2_rn(lo, YA[kk], gA));
            YB[kk] = __ffma2_rn(r, YB[kk], __ffma2_rn(lo, YB[kk], gB));
        } else {
            YA[kk] = __ffma2_rn(r, YA[kk], gA);
            YB[kk] = __ffma2_rn(r, YB[kk], gB);
        }
    }
    hA[0] = pA[0].x;
    hA[1] = pA[0].y;
    hA[2] = pA[1].x;
    hA[3] = pA[1].y;
    hB[0] = pB[0].x;
    hB[1] = pB[0].y;
    hB[2] = pB[1].x;
    hB[3] = pB[1].y;
}

// Exact window d_i x^{n-i}, i = 1 .. min(L - 1, n - 1), of both modes into hA[3] / hB[3]: odd i
// on half 0, even i on half 1 (same trip count on both halves; the last term of half 1 may be
// absent). slot holds x^{n-L} .. and receives x^n. With LO, the same terms with the FP32
// remainders of the weights (d_i - fl(d_i), wsl) go into wlA / wlB.
template <bool LO>
__device__ __forceinline__ void f32_window(const float2 *Rc, const float *ws, const float *wsl, int T, int L, int slot,
                                           int n, int hf, float (&hA)[4], float (&hB)[4], float &wlA, float &wlB) {
    const int imax = min(L - 1, n - 1);
    for (int q = 0; 2 * q < imax; ++q) {
        const int i = 2 * q + 1 + hf;
        int sl = slot - i;
        if (sl < 0) sl += L;
        const bool on = i <= imax;
        const float2 v = Rc[(on ? sl : slot) * T];
        const float w = on ? ws[2 * i] : 0.0f;
        hA[3] = fmaf(w, v.x, hA[3]);
        hB[3] = fmaf(w, v.y, hB[3]);
        if (LO) {
            const float wl = on ? wsl[2 * i] : 0.0f;
            wlA = fmaf(wl, v.x, wlA);
            wlB = fmaf(wl, v.y, wlB);
        }
    }
}

// The same window unrolled to a compile-time bound WL >= L, with no branch: terms i >= L have
// zero weight, and levels before level 1 sit in ring slots that are still zero. In the
// pipelined loop this keeps the node part, the window and the step in one basic block, so
// the compiler can interleave the step's dependency chain with the node work.
template <bool LO, int WL>
__device__ __forceinline__ void f32_window_u(const float2 *Rc, const float *ws, const float *wsl, int T, int L,
                                             int slot, int hf, float (&hA)[4], float (&hB)[4], float &wlA,
                                             float &wlB) {
#pragma unroll
    for (int q = 0; 2 * q < WL - 1; ++q) {
        const int i = 2 * q + 1 + hf;
        const bool on = i < L;
        int sl = slot - i;
        if (sl < 0) sl += L;
        const float2 v = Rc[(on ? sl : slot) * T];
        const float w = on ? ws[2 * i] : 0.0f;
        hA[3] = fmaf(w, v.x, hA[3]);
        hB[3] = fmaf(w, v.y, hB[3]);
        if (LO) {
            const float wl = on ? wsl[2 * i] : 0.0f;
            wlA = fmaf(wl, v.x, wlA);
            wlB = fmaf(wl, v.y, wlB);
        }
    }
}

template <int NP, bool BE, int WL>
__global__ void __launch_bounds__(kF32Threads) k_fp2s_fast_f32(Fp2sParams P, int solve64,
                                                               const double *__restrict__ lam,
                                                               const double *__restrict__ g0,
                                                               double *__restrict__ gN, int *__restrict__ status,
                                                               const double *__restrict__ d1,
                                                               const double *__restrict__ d2,
                                                               const float *__restrict__ ftab,
                                                               const float *__restrict__ hdf) {
    constexpr int NQ = NP / 4;               // node pairs per lane
    constexpr int KD = f32_df_pairs(NP);   // trailing node pairs with double-float ratios
    extern __shared__ __align__(16) float smf[];
    const int L = P.L, T = blockDim.x, tid = threadIdx.x;
    float4 *tab4 = reinterpret_cast<float4 *>(smf);                    // [NQ][half][state]
    float2 *tlo = reinterpret_cast<float2 *>(smf + 4 * NP);            // [KD][half][state]
    float *csum = smf + 4 * NP + 8 * KD;                                // C of each state
    float *wt = csum + 2;                                               // wt[2i + s] = fl(d_i) of state s, i < L
    float *wlo = wt + 2 * kMaxNs;                                       // wlo[2i + s] = d_i - fl(d_i)
    float2 *R = reinterpret_cast<float2 *>(wlo + 2 * kMaxNs);          // [L][T]
    for (int e = tid; e < 4 * NP + 8 * KD + 2; e += T) smf[e] = ftab[e];
    for (int i = tid; i < L; i += T) {
        const float a = (float)d1[i], b = (float)d2[i];
        wt[2 * i] = a;
        wt[2 * i + 1] = b;
        wlo[2 * i] = (float)(d1[i] - (double)a);
        wlo[2 * i + 1] = (float)(d2[i] - (double)b);
    }
    for (int j = 0; j < L; ++j) R[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
    __syncthreads();

    const int lane = tid & 31, st = lane >> 4, hf = (lane >> 3) & 1;
    const int64_t pair = ((int64_t)blockIdx.x * (T >> 5) + (tid >> 5)) * 8 + (lane & 7);
    const int64_t mode_raw = 2 * pair + hf;                             // the mode this lane steps
    const bool active = mode_raw < P.nmodes;
    const int64_t mode = active ? mode_raw : 0;
    const float4 *tb = tab4 + (2 * hf + st);
    const float2 *tl = tlo + (2 * hf + st);
    const float *ws = wt + st, *wsl = wlo + st;
    float cs = hf ? 0.0f : csum[st];         // C G^{n-L} enters the sums of half 0 only
    keep_reg(cs);
    // d_1 of the own / other state as double-float (the BE window is d_1 x^{n-1} alone)
    float w1 = wt[2 + st], w1_lo = wlo[2 + st], w1_o = wt[3 - st], w1_o_lo = wlo[3 - st];
    keep_reg(w1);
    keep_reg(w1_lo);
    keep_reg(w1_o);
    keep_reg(w1_o_lo);
    const double *dn = st ? d2 : d1;
    const float *hd_hi = hdf + (size_t)(2 * st) * (P.N + 1), *hd_lo = hd_hi + (P.N + 1);
    float2 *Rc = R + tid;

    // per-mode power-of-two scale from max(|g1^0|, |g2^0|)
    const double gz64 = g0[st * P.nmodes + mode];
    const double gmax = fmax(fabs(gz64), fabs(__shfl_xor_sync(0xffffffffu, gz64, 16)));
    int ex = 0;
    if (gmax > 0.0 && isfinite(gmax)) frexp(gmax, &ex);
    const df gzd = df_from(ldexp(gz64, -ex));
    const float gz = gzd.hi;

    LaneStep ls;
    const bool ok = lane_step_setup(P, lam[mode], d1[0], d2[0], st, ls);
    if (active && st == 0 && !ok) atomicOr(status, ST_SINGULAR);
    LaneStep2 l2;
    lane_step2_setup(P, ls, l2);
    keep_reg(l2);

    float2 YA[NQ], YB[NQ];                   // the two modes' states over this lane's node pairs
#pragma unroll
    for (int j = 0; j < NQ; ++j) YA[j] = YB[j] = make_float2(0.0f, 0.0f);
    // own (and partner state's) last two levels as double-float pairs
    float gm1 = gz, gm1_lo = gzd.lo, gm2 = 0.0f, gm2_lo = 0.0f;
    float gm1_o = __shfl_xor_sync(0xffffffffu, gz, 16), gm1_o_lo = __shfl_xor_sync(0xffffffffu, gzd.lo, 16);
    float gm2_o = 0.0f, gm2_o_lo = 0.0f;
    const int N = (int)P.N;
    float hA[4] = {}, hB[4] = {};            // node part of the current step
    // the new level x^n of the lane's mode: both halves' levels into the ring, shift the history
    auto finish = [&](df x, int slot) {
        const float x_o = __shfl_xor_sync(0xffffffffu, x.hi, 16);    // partner state, same mode
        const float x_o_lo = __shfl_xor_sync(0xffffffffu, x.lo, 16);
        const float x_p = __shfl_xor_sync(0xffffffffu, x.hi, 8);     // same state, other mode of the pair
        Rc[slot * T] = hf ? make_float2(x_p, x.hi) : make_float2(x.hi, x_p);
        gm2 = gm1;
        gm2_lo = gm1_lo;
        gm1 = x.hi;
        gm1_lo = x.lo;
        gm2_o = gm1_o;
        gm2_o_lo = gm1_o_lo;
        gm1_o = x_o;
        gm1_o_lo = x_o_lo;
    };
    auto combine = [&]() -> float {
        float sA = (hA[0] + hA[1]) + (hA[2] + hA[3]);
        float sB = (hB[0] + hB[1]) + (hB[2] + hB[3]);
        sA += __shfl_xor_sync(0xffffffffu, sA, 8);                   // both halves: same sums
        sB += __shfl_xor_sync(0xffffffffu, sB, 8);
        return hf ? sB : sA;
    };
    if (solve64) {
        // strong coupling: every step in FP64 (not pipelined)
        int slot = 0;
        for (int n = 1; n <= N; ++n) {
            slot = (slot + 1 == L) ? 0 : slot + 1;
            float wlA = 0.0f, wlB = 0.0f;
            f32_node_part<NQ, KD>(tb, tl, cs, Rc[slot * T], YA, YB, hA, hB);
            f32_window<false>(Rc, ws, wsl, T, L, slot, n, hf, hA, hB, wlA, wlB);
            const float h = combine();
            finish(lane_step_rare(P, ls, 1, n, h, gm1, gm2, gz, dn, hd_hi, hd_lo), slot);
        }
    } else {
        // Software-pipelined: the node part of step n + 1 needs G^{n+1-L} (L >= 2: written at
        // step n - 1 or earlier) and not x^n, so it sits in the same iteration as the window and
        // 2x2 step of step n and the two chains interleave.
        int n = 1, slot = 1 % L;
#pragma unroll
        for (int q = 0; q < 4; ++q) hA[q] = hB[q] = 0.0f;           // node part of step 1 (no input yet)
        if (!BE) {                           // the first SBD step (its own matrix), out of line
            finish(lane_step_rare(P, ls, 0, 1, combine(), gm1, gm2, gz, dn, hd_hi, hd_lo), slot);
            n = 2;
            slot = (slot + 1 == L) ? 0 : slot + 1;
        }
        for (; n <= N; ++n) {
            const int next = (slot + 1 == L) ? 0 : slot + 1;
            float nA[4], nB[4];
            f32_node_part<NQ, KD>(tb, tl, cs, Rc[next * T], YA, YB, nA, nB);  // step n + 1
            float wlA = 0.0f, wlB = 0.0f;
            f32_window_u<!BE, WL>(Rc, ws, wsl, T, L, slot, hf, hA, hB, wlA, wlB);  // step n
            const float h = combine();
            // The window took fl(d_i) fl(x^{n-i}); the FP32 remainders of the weights (a weight
            // rounded to FP32 is a fixed relative error of up to 2^-25 that every step repeats,
            // and d_1 is of size beta tau^-beta) and of the own level x^{n-1} go into e_lo.
            // G^0 is not part of the history: nothing at n = 1.
            df x;
            if (BE) {
                const float e_lo = n > 1 ? fmaf(w1_lo, gm1, w1 * gm1_lo) : 0.0f;
                const float e_o_lo = n > 1 ? fmaf(w1_o_lo, gm1_o, w1_o * gm1_o_lo) : 0.0f;
                x = lane_step2_df(l2, gm1, gm1_lo, gm1_o, gm1_o_lo, h, e_lo, __shfl_xor_sync(0xffffffffu, h, 16),
                                  e_o_lo);
            } else {
                // window remainders of the own mode: this half's terms plus the other half's
                const float wl = (hf ? wlB : wlA) + __shfl_xor_sync(0xffffffffu, hf ? wlA : wlB, 8);
                const float e_lo = fmaf(w1, gm1_lo, wl);
                df l = two_sum(2.0f * gm1, -0.5f * gm2), lo = two_sum(2.0f * gm1_o, -0.5f * gm2_o);
                l.lo += fmaf(2.0f, gm1_lo, -0.5f * gm2_lo);
                lo.lo += fmaf(2.0f, gm1_o_lo, -0.5f * gm2_o_lo);
                // e = h + d_{n-1} g^0 / 2 (+ the low parts) as a double-float pair
                const df e = df_add(df_mul(df{__ldg(hd_hi + n - 1), __ldg(hd_lo + n - 1)}, gzd), df{h, e_lo});
                x = lane_step2_df(l2, l.hi, l.lo, lo.hi, lo.lo, e.hi, e.lo, __shfl_xor_sync(0xffffffffu, e.hi, 16),
                                  __shfl_xor_sync(0xffffffffu, e.lo, 16));
            }
            finish(x, slot);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                hA[q] = nA[q];
                hB[q] = nB[q];
            }
            slot = next;
        }
    }
    if (active) {
        const double out = ldexp((double)gm1 + (double)gm1_lo, ex);
        gN[st * P.nmodes + mode] = out;
        if (!isfinite(out)) atomicOr(status, ST_NONFINITE);
    }
}

static size_t f32_smem_bytes(int NP, int L, int T) {
    return ((size_t)4 * NP + 8 * f32_df_pairs(NP) + 2 + 4 * kMaxNs) * sizeof(float) + (size_t)L * T * sizeof(float2);
}

template <int NP>
static void launch_f32(const Fp2sParams &P, int solve64, const Fp2sLayout &l, cudaStream_t s) {
    const int T = kF32Threads;
    const int64_t mpb = (int64_t)(T / 32) * kFastModesPerWarp;
    const unsigned blocks = (unsigned)((P.nmodes + mpb - 1) / mpb);
    const size_t smem = f32_smem_bytes(NP, P.L, T);
#define CQ_F32_LAUNCH(BEV, WLV)                                                                              \
    k_fp2s_fast_f32<NP, BEV, WLV><<<blocks, T, smem, s>>>(P, solve64, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, \
                                                          l.ftab, l.hdf)
    if (P.scheme == CQ_BE) CQ_F32_LAUNCH(true, 2);
    else if (P.L <= 17) CQ_F32_LAUNCH(false, 17);
    else CQ_F32_LAUNCH(false, kMaxNs);
#undef CQ_F32_LAUNCH
}

// The compile-time node bound NP of the FP32 fast kernel for np points per state (0: too many).
static int f32_np_bound(int np) {
    for (int b : {16, 32, 48, 64, 80, 96, 128})
        if (np <= b) return b;
    return 0;
}

// hdf[(2s)(N+1) + i], hdf[(2s+1)(N+1) + i] = hi, lo of d^s_i / 2
__global__ void k_half_weights_df(const double *__restrict__ d1, const double *__restrict__ d2, int64_t n,
                                  float *__restrict__ hdf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const double a = 0.5 * d1[i], b = 0.5 * d2[i];
    const float ah = (float)a, bh = (float)b;
    hdf[i] = ah;
    hdf[(n + 1) + i] = (float)(a - (double)ah);
    hdf[2 * (n + 1) + i] = bh;
    hdf[3 * (n + 1) + i] = (float)(b - (double)bh);
}

static int fp2s_fast_f32(const Fp2sParams &P, const Fp2sLayout &l, cudaStream_t s) {
    const int solve64 = fabs(P.a) > 10.0;
    switch (f32_np_bound(P.np)) {
        case 16: launch_f32<16>(P, solve64, l, s); break;
        case 32: launch_f32<32>(P, solve64, l, s); break;
        case 48: launch_f32<48>(P, solve64, l, s); break;
        case 64: launch_f32<64>(P, solve64, l, s); break;
        case 80: launch_f32<80>(P, solve64, l, s); break;
        case 96: launch_f32<96>(P, solve64, l, s); break;
        case 128: launch_f32<128>(P, solve64, l, s); break;
        default: return CQ_EUNSUPPORTED;
    }
    return CQ_OK;
}

// ---------------------------------------------------------------------------
// Fused direct solve: one thread per mode, time blocks of kDirBT steps. For a
// block starting at n0 the contribution of the levels 1..n0-1 is accumulated
// with a shifting register window of weights (one level load feeds 2*kDirBT
// FMAs); the in-block terms follow step by step together with the solves.
// hist[(k*2 + s)*nmodes + mode] holds level k of state s.
// ---------------------------------------------------------------------------
template <int BT>
__global__ void __launch_bounds__(32, 16) k_fp2s_direct(Fp2sParams P, const double *__restrict__ lam,
                                                     const double *__restrict__ g0, double *__restrict__ gN,
                                                     int *__restrict__ status, const double *__restrict__ d1,
                                                     const double *__restrict__ d2,
                                                     const double *__restrict__ dz1,
                                                     const double *__restrict__ dz2, double *__restrict__ hist) {
    const int64_t nm = P.nmodes;
    const int64_t mode = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nm) return;
    const double gz1 = g0[mode], gz2 = g0[nm + mode];
    hist[mode] = gz1;
    hist[nm + mode] = gz2;
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    ModeConst mc;
    if (!mode_setup(P, lam[mode], d10, d20, mc)) atomicOr(status, ST_SINGULAR);
    double gm1_1 = gz1, gm1_2 = gz2, gm2_1 = 0.0, gm2_2 = 0.0;
    for (int64_t n0 = 1; n0 <= P.N; n0 += BT) {
        double a1[BT], a2[BT], w1[BT], w2[BT], l1[BT] = {}, l2[BT] = {};
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            a1[b] = 0.0;
            a2[b] = 0.0;
            w1[b] = __ldg(dz1 + (n0 + b - 1) + BT);
            w2[b] = __ldg(dz2 + (n0 + b - 1) + BT);
        }
        const double *hp = hist + 2 * nm + mode;          // level 1
        for (int64_t k = 1; k < n0; ++k, hp += 2 * nm) {
            const double x1 = hp[0], x2 = hp[nm];
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                a1[b] = fma(w1[b], x1, a1[b]);
                a2[b] = fma(w2[b], x2, a2[b]);
            }
#pragma unroll
            for (int b = BT - 1; b > 0; --b) {
                w1[b] = w1[b - 1];
                w2[b] = w2[b - 1];
            }
            w1[0] = __ldg(dz1 + (n0 - k - 1) + BT);
            w2[0] = __ldg(dz2 + (n0 - k - 1) + BT);
        }
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int64_t n = n0 + b;
            if (n > P.N) break;
            double h1 = a1[b], h2 = a2[b];
#pragma unroll
            for (int kk = 0; kk < b; ++kk) {
                h1 = fma(__ldg(d1 + (b - kk)), l1[kk], h1);
                h2 = fma(__ldg(d2 + (b - kk)), l2[kk], h2);
            }
            double d1n = 0.0, d2n = 0.0;
            if (P.scheme == CQ_BDF2 && n >= 2) {
                d1n = __ldg(d1 + n - 1);
                d2n = __ldg(d2 + n - 1);
            }
            double x1, x2;
            mode_step(P, mc, n, h1, h2, d10, d20, d1n, d2n, gm1_1, gm1_2, gm2_1, gm2_2, gz1, gz2, x1, x2);
            l1[b] = x1;
            l2[b] = x2;
            hist[(n * 2) * nm + mode] = x1;
            hist[(n * 2 + 1) * nm + mode] = x2;
            gm2_1 = gm1_1;
            gm2_2 = gm1_2;
            gm1_1 = x1;
            gm1_2 = x2;
        }
    }
    gN[mode] = gm1_1;
    gN[nm + mode] = gm1_2;
    if (!isfinite(gm1_1) || !isfinite(gm1_2)) atomicOr(status, ST_NONFINITE);
}

// ---------------------------------------------------------------------------
// Fused direct solve for problems with few modes (1D grids, small 2D grids):
// LP lanes of a warp share one mode. Each lane takes every LP-th history level
// of the block's sums (consecutive lanes read consecutive levels: coalesced
// 16-byte loads from the mode-major history histm[mode][k][state]); the LP
// partial sums are combined with xor shuffles inside the lane group, and every
// lane of the group then takes the block's steps itself (one lane stores).
// The FP64 pipe bounds the kernel, so the per-level weight loads (from L1) and
// the shuffles cost little next to the FMAs they feed.
// ---------------------------------------------------------------------------
template <int LP, int BT>
__global__ void __launch_bounds__(256) k_fp2s_direct_split(Fp2sParams P, const double *__restrict__ lam,
                                                           const double *__restrict__ g0, double *__restrict__ gN,
                                                           int *__restrict__ status, const double *__restrict__ d1,
                                                           const double *__restrict__ d2, double *__restrict__ histm) {
    const int64_t nm = P.nmodes;
    const int lane = threadIdx.x & 31, sl = lane % LP;
    const int64_t mode_raw = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / LP) + lane / LP;
    const bool active = mode_raw < nm;
    const int64_t mode = active ? mode_raw : 0;
    double *hm = histm + (size_t)mode * 2 * (P.N + 1);          // level k of state s at hm[2k + s]
    const double gz1 = g0[mode], gz2 = g0[nm + mode];
    if (active && sl == 0) {
        hm[0] = gz1;
        hm[1] = gz2;
    }
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    ModeConst mc;
    if (!mode_setup(P, lam[mode], d10, d20, mc) && active && sl == 0) atomicOr(status, ST_SINGULAR);
    double gm1_1 = gz1, gm1_2 = gz2, gm2_1 = 0.0, gm2_2 = 0.0;
    for (int64_t n0 = 1; n0 <= P.N; n0 += BT) {
        double a1[BT], a2[BT], l1[BT] = {}, l2[BT] = {};
#pragma unroll
        for (int b = 0; b < BT; ++b) a1[b] = a2[b] = 0.0;
        for (int64_t k = 1 + sl; k < n0; k += LP) {
            const double2 x = *reinterpret_cast<const double2 *>(hm + 2 * k);
            const int64_t i0 = n0 - k;                     // weight index of the block's first step
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                if (i0 + b <= P.N) {
                    a1[b] = fma(__ldg(d1 + i0 + b), x.x, a1[b]);
                    a2[b] = fma(__ldg(d2 + i0 + b), x.y, a2[b]);
                }
            }
        }
#pragma unroll
        for (int off = LP / 2; off > 0; off >>= 1) {
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                a1[b] += __shfl_xor_sync(0xffffffffu, a1[b], off);
                a2[b] += __shfl_xor_sync(0xffffffffu, a2[b], off);
            }
        }
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int64_t n = n0 + b;
            if (n > P.N) break;
            double h1 = a1[b], h2 = a2[b];
#pragma unroll
            for (int kk = 0; kk < b; ++kk) {
                h1 = fma(__ldg(d1 + (b - kk)), l1[kk], h1);
                h2 = fma(__ldg(d2 + (b - kk)), l2[kk], h2);
            }
            double d1n = 0.0, d2n = 0.0;
            if (P.scheme == CQ_BDF2 && n >= 2) {
                d1n = __ldg(d1 + n - 1);
                d2n = __ldg(d2 + n - 1);
            }
            double x1, x2;
            mode_step(P, mc, n, h1, h2, d10, d20, d1n, d2n, gm1_1, gm1_2, gm2_1, gm2_2, gz1, gz2, x1, x2);
            l1[b] = x1;
            l2[b] = x2;
            if (active && sl == 0) *reinterpret_cast<double2 *>(hm + 2 * n) = make_double2(x1, x2);
            gm2_1 = gm1_1;
            gm2_2 = gm1_2;
            gm1_1 = x1;
            gm1_2 = x2;
        }
        __syncwarp();                                      // the stored levels are read by the group next block
    }
    if (active && sl == 0) {
        gN[mode] = gm1_1;
        gN[nm + mode] = gm1_2;
        if (!isfinite(gm1_1) || !isfinite(gm1_2)) atomicOr(status, ST_NONFINITE);
    }
}

// Lanes per mode of the direct solve: one lane per mode (the register-window kernel)
// once that gives 8 warps per SM, else enough lanes per mode for about 16 warps per SM.
static int direct_lanes_per_mode(int64_t nmodes) {
    if (nmodes >= (int64_t)152 * 8 * 32) return 1;
    int lp = 1;
    while (lp < 32 && nmodes * lp < (int64_t)152 * 16 * 32) lp *= 2;
    return lp;
}

// One-warp blocks: a warp or two per SM already keeps its FP64 pipe busy (16 independent
// FMA chains per lane), so small grids are spread over every SM rather than packed.
template <int LP>
static void launch_direct_split(const Fp2sParams &P, const Fp2sLayout &l, cudaStream_t s) {
    const int64_t mpw = 32 / LP;
    const unsigned blocks = (unsigned)((P.nmodes + mpw - 1) / mpw);
    k_fp2s_direct_split<LP, kDirBT><<<blocks, 32, 0, s>>>(P, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.hist);
}

__global__ void k_pad(const double *__restrict__ d, int64_t n, int BT, double *__restrict__ dz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n + 2 * BT) return;
    const int64_t idx = i - BT;
    dz[i] = (idx >= 1 && idx <= n) ? d[idx] : 0.0;
}

// ---------------------------------------------------------------------------
// Step API kernels (state in the workspace, one launch per time step).
// glast[(lvl*2 + s)*nm + mode]: lvl 0 = g^{n-1}, lvl 1 = g^{n-2}.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fp2s_step_fast(Fp2sParams P, int64_t n, const double *__restrict__ lam,
                                                        const double *__restrict__ g0, double *__restrict__ gout,
                                                        int *__restrict__ status, const double *__restrict__ d1,
                                                        const double *__restrict__ d2,
                                                        const double *__restrict__ tab1,
                                                        const double *__restrict__ tab2, double *__restrict__ Y,
                                                        double *__restrict__ ring, double *__restrict__ glast) {
    const int64_t nm = P.nmodes;
    const int64_t mode = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nm) return;
    const int np = P.np, L = P.L;
    double *Y1 = Y + mode, *Y2 = Y + (size_t)np * nm + mode;
    double *R1 = ring + mode, *R2 = ring + (size_t)L * nm + mode;
    const int slot = (int)(n % L);
    double h1 = 0.0, h2 = 0.0;
    if (n - L >= 1) {
        const double in1 = R1[(size_t)slot * nm], in2 = R2[(size_t)slot * nm];
        for (int j = 0; j < np; ++j) {
            const double y1 = fma(__ldg(tab1 + j), Y1[(size_t)j * nm], in1);
            const double y2 = fma(__ldg(tab2 + j), Y2[(size_t)j * nm], in2);
            Y1[(size_t)j * nm] = y1;
            Y2[(size_t)j * nm] = y2;
            h1 = fma(__ldg(tab1 + np + j), y1, h1);
            h2 = fma(__ldg(tab2 + np + j), y2, h2);
        }
    }
    const int imax = (int)min((int64_t)(L - 1), n - 1);
    for (int i = 1; i <= imax; ++i) {
        const int sl = (int)((n - i) % L);
        h1 = fma(__ldg(d1 + i), R1[(size_t)sl * nm], h1);
        h2 = fma(__ldg(d2 + i), R2[(size_t)sl * nm], h2);
    }
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    ModeConst mc;
    if (!mode_setup(P, lam[mode], d10, d20, mc)) atomicOr(status, ST_SINGULAR);
    const double gz1 = g0[mode], gz2 = g0[nm + mode];
    const double gm1_1 = glast[mode], gm1_2 = glast[nm + mode];
    const double gm2_1 = glast[2 * nm + mode], gm2_2 = glast[3 * nm + mode];
    double d1n = 0.0, d2n = 0.0;
    if (P.scheme == CQ_BDF2 && n >= 2) {
        d1n = __ldg(d1 + n - 1);
        d2n = __ldg(d2 + n - 1);
    }
    double x1, x2;
    mode_step(P, mc, n, h1, h2, d10, d20, d1n, d2n, gm1_1, gm1_2, gm2_1, gm2_2, gz1, gz2, x1, x2);
    R1[(size_t)slot * nm] = x1;
    R2[(size_t)slot * nm] = x2;
    glast[2 * nm + mode] = gm1_1;
    glast[3 * nm + mode] = gm1_2;
    glast[mode] = x1;
    glast[nm + mode] = x2;
    gout[mode] = x1;
    gout[nm + mode] = x2;
    if (!isfinite(x1) || !isfinite(x2)) atomicOr(status, ST_NONFINITE);
}

__global__ void __launch_bounds__(256) k_fp2s_step_direct(Fp2sParams P, int64_t n, const double *__restrict__ lam,
                                                          const double *__restrict__ g0, double *__restrict__ gout,
                                                          int *__restrict__ status,
                                                          const double *__restrict__ d1,
                                                          const double *__restrict__ d2, double *__restrict__ hist,
                                                          double *__restrict__ glast) {
    const int64_t nm = P.nmodes;
    const int64_t mode = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode >= nm) return;
    double h1 = 0.0, h2 = 0.0;
    for (int64_t i = 1; i <= n - 1; ++i) {
        const double *lv = hist + ((n - i) * 2) * nm + mode;
        h1 = fma(__ldg(d1 + i), lv[0], h1);
        h2 = fma(__ldg(d2 + i), lv[nm], h2);
    }
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    ModeConst mc;
    if (!mode_setup(P, lam[mode], d10, d20, mc)) atomicOr(status, ST_SINGULAR);
    const double gz1 = g0[mode], gz2 = g0[nm + mode];
    const double gm1_1 = glast[mode], gm1_2 = glast[nm + mode];
    const double gm2_1 = glast[2 * nm + mode], gm2_2 = glast[3 * nm + mode];
    double d1n = 0.0, d2n = 0.0;
    if (P.scheme == CQ_BDF2 && n >= 2) {
        d1n = __ldg(d1 + n - 1);
        d2n = __ldg(d2 + n - 1);
    }
    double x1, x2;
    mode_step(P, mc, n, h1, h2, d10, d20, d1n, d2n, gm1_1, gm1_2, gm2_1, gm2_2, gz1, gz2, x1, x2);
    hist[(n * 2) * nm + mode] = x1;
    hist[(n * 2 + 1) * nm + mode] = x2;
    glast[2 * nm + mode] = gm1_1;
    glast[3 * nm + mode] = gm1_2;
    glast[mode] = x1;
    glast[nm + mode] = x2;
    gout[mode] = x1;
    gout[nm + mode] = x2;
    if (!isfinite(x1) || !isfinite(x2)) atomicOr(status, ST_NONFINITE);
}

__global__ void k_copy_levels(const double *__restrict__ g0, int64_t nm, double *__restrict__ hist,
                              double *__restrict__ glast) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * nm) return;
    if (hist) hist[i] = g0[i];
    if (glast) {
        glast[i] = g0[i];
        glast[2 * nm + i] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int status_from_bits(int bits) {
    if (bits & ST_TIMEOUT) return CQ_ETIMEOUT;
    if (bits & ST_SINGULAR) return CQ_ESINGULAR;
    if (bits & ST_NONFINITE) return CQ_ENONFINITE;
    return CQ_OK;
}

// The status word of one call (a buffer per call, so that calls from several host threads
// do not share it).
static int read_status(const int *status_dev, cudaStream_t s) {
    int host = 0;
    if (cudaMemcpyAsync(&host, status_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CQ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CQ_ECUDA;
    return status_from_bits(host);
}

// Status word, weights and the fast-form tables of a solve.
static int setup_tables(const fp2s_problem_t *p, const Fp2sParams &P, int np1, int np2, const Fp2sLayout &l,
                        cudaStream_t s) {
    int st;
    const double b1 = 1.0 - p->alpha1, b2 = 1.0 - p->alpha2;
    if ((st = cuda_status(cudaMemsetAsync(l.status, 0, 64 * sizeof(int), s)))) return st;
    if ((st = launch_weights(P.scheme, b1, P.tau, P.N, l.d1, s, l.wscr))) return st;
    if ((st = launch_weights(P.scheme, b2, P.tau, P.N, l.d2, s, l.wscr))) return st;
    if (P.prec != CQ_F64 && P.prec != CQ_DF64) {
        k_half_weights_df<<<(unsigned)((P.N + 256) / 256), 256, 0, s>>>(l.d1, l.d2, P.N, l.hdf);
        if ((st = launched())) return st;
    }
    if (P.form == CQ_DIRECT && P.prec == CQ_DF64) {
        if ((st = direct_df_tables(P, l.d1, l.d2, l.wz, s))) return st;
    } else if (P.form == CQ_DIRECT && P.prec == CQ_F64) {
        const unsigned g = (unsigned)((P.N + 2 * kDirBT + 256) / 256);
        k_pad<<<g, 256, 0, s>>>(l.d1, P.N, kDirBT, l.dz1);
        k_pad<<<g, 256, 0, s>>>(l.d2, P.N, kDirBT, l.dz2);
        if ((st = launched(2))) return st;
    } else if (P.form == CQ_FAST) {
        if ((st = build_fast_coeffs(P.scheme, b1, P.tau, np1, np2, P.L, l.scr1, l.tab1, l.tab1 + P.np, s))) return st;
        if ((st = build_fast_coeffs(P.scheme, b2, P.tau, np1, np2, P.L, l.scr2, l.tab2, l.tab2 + P.np, s))) return st;
        if (P.prec == CQ_F32) {
            const int NP = f32_np_bound(P.np);
            if (NP == 0) return CQ_EUNSUPPORTED;
            k_f32_tables<<<1, 256, 0, s>>>(NP, f32_df_pairs(NP), P.np, l.tab1, l.tab2, l.ftab);
            if ((st = launched())) return st;
        } else if (P.prec == CQ_DF64) {
            if ((st = fast_df_tables(P, l.tab1, l.tab2, l.d1, l.d2, l.ftab, s))) return st;
        }
    }
    return CQ_OK;
}

// Common set-up of fp2s_solve and fp2s_init: status, weights, tables, spectrum, DST of G0.
static int setup(const fp2s_problem_t *p, const Fp2sParams &P, int np1, int np2, const Fp2sLayout &l,
                 const double *G0, cudaStream_t s) {
    int st;
    if ((st = setup_tables(p, P, np1, np2, l, s))) return st;
    if ((st = launch_mode_eigenvalues(p->M, p->dim, l.lam, s))) return st;
    if ((st = launch_dst_matrix(p->M, l.S, s))) return st;
    return launch_dst_field(p->M, p->dim, l.S, G0, l.g0, l.tmp, s);
}

// The single-launch solve kernels (fast FP64, fast FP32, direct FP64).
static int solve_kernel(const Fp2sParams &P, const Fp2sLayout &l, cudaStream_t s) {
    if (P.form == CQ_FAST && P.prec == CQ_F32) return fp2s_fast_f32(P, l, s);
    if (P.form == CQ_FAST && P.prec == CQ_DF64)
        return fast_df_solve(P, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.ftab, s);
    if (P.form == CQ_DIRECT && P.prec == CQ_DF64)
        return direct_df_solve(P, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.wz, l.hist2, s);
    if (P.form == CQ_FAST && fast_use_split(P.nmodes)) return launch_fast_split(P, l, s);
    if (P.form == CQ_FAST) {
        const int T = fast_block_threads(P.np, P.L, P.nmodes);
        if (T == 0) return CQ_EUNSUPPORTED;
        const size_t smem = fast_smem_bytes(P.np, P.L, T);
        if (cudaFuncSetAttribute(k_fp2s_fast<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return CQ_ECUDA;
        const int64_t mpb = (int64_t)(T / 32) * kFastModesPerWarp;
        const unsigned blocks = (unsigned)((P.nmodes + mpb - 1) / mpb);
        k_fp2s_fast<false><<<blocks, T, smem, s>>>(P, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.tab1, l.tab2,
                                                    nullptr);
    } else if (const int lp = direct_lanes_per_mode(P.nmodes); lp > 1) {
        switch (lp) {
            case 2: launch_direct_split<2>(P, l, s); break;
            case 4: launch_direct_split<4>(P, l, s); break;
            case 8: launch_direct_split<8>(P, l, s); break;
            case 16: launch_direct_split<16>(P, l, s); break;
            default: launch_direct_split<32>(P, l, s); break;
        }
    } else {
        // one-warp blocks: every block runs all N steps, so small blocks spread the
        // modes evenly over the SMs (at most one warp of imbalance per SM)
        const unsigned blocks = (unsigned)((P.nmodes + 31) / 32);
        k_fp2s_direct<kDirBT><<<blocks, 32, 0, s>>>(P, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.dz1, l.dz2,
                                                    l.hist);
    }
    return CQ_OK;
}

}  // namespace fastcq

using namespace fastcq;

// The time loop of a solve on the modal G^0 in l.g0, writing the modal G^N to l.gN: the
// fused kernel, or the block / contraction launches of the mixed-precision direct solve.
static int run_modes(const Fp2sParams &P, const Fp2sLayout &l, cudaStream_t s) {
    int st;
    if ((st = timing_begin(s))) return st;
    if (P.form == CQ_DIRECT && (P.prec == CQ_BF16X3 || P.prec == CQ_TF32X3)) {
        // counts its own launches
        if ((st = mixed_direct_run(P, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.hdf, l.mixed, s))) return st;
    } else {
        if ((st = solve_kernel(P, l, s))) return st;
        if ((st = launched())) return st;
    }
    return timing_end(s);
}

extern "C" int fp2s_solve(const fp2s_problem_t *p, const double *G0_dev, double *GN_dev, void *ws_dev,
                          size_t *ws_bytes, void *stream) {
    Fp2sParams P;
    int np1 = 0, np2 = 0;
    int st = derive(p, P, np1, np2);
    if (st) return st;
    if (!ws_bytes) return CQ_EINVAL;
    Fp2sLayout l = fp2s_layout(p, P, ws_dev, false);
    if (!ws_dev) { *ws_bytes = l.bytes; return CQ_OK; }
    if (*ws_bytes < l.bytes) return CQ_ENOMEM;
    if (!G0_dev || !GN_dev || ((uintptr_t)ws_dev & 255)) return CQ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = setup(p, P, np1, np2, l, G0_dev, s))) return st;
    if ((st = run_modes(P, l, s))) return st;
    if ((st = launch_dst_field(p->M, p->dim, l.S, l.gN, GN_dev, l.tmp, s))) return st;
    if (p->flags & FP2S_ASYNC) return CQ_OK;
    return read_status(l.status, s);
}

extern "C" int fp2s_solve_modes(const fp2s_problem_t *p, int64_t mode_lo, int64_t mode_hi, const double *g0_dev,
                                double *gN_dev, void *ws_dev, size_t *ws_bytes, void *stream) {
    Fp2sParams P;
    int np1 = 0, np2 = 0;
    int st = derive(p, P, np1, np2);
    if (st) return st;
    if (!ws_bytes) return CQ_EINVAL;
    const int64_t all = P.nmodes;
    if (mode_lo < 0 || mode_hi > all || mode_lo >= mode_hi) return CQ_EINVAL;
    P.nmodes = mode_hi - mode_lo;
    Fp2sLayout l = fp2s_layout(p, P, ws_dev, false, false, -1, all);
    if (!ws_dev) { *ws_bytes = l.bytes; return CQ_OK; }
    if (*ws_bytes < l.bytes) return CQ_ENOMEM;
    if (!g0_dev || !gN_dev || ((uintptr_t)ws_dev & 255)) return CQ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = setup_tables(p, P, np1, np2, l, s))) return st;
    if ((st = launch_mode_eigenvalues(p->M, p->dim, l.lam, s))) return st;
    // the kernels see the range as a problem of its own: its spectrum, modal G^0 and G^N
    Fp2sLayout lr = l;
    lr.lam = l.lam + mode_lo;
    lr.g0 = const_cast<double *>(g0_dev);
    lr.gN = gN_dev;
    if ((st = run_modes(P, lr, s))) return st;
    if (p->flags & FP2S_ASYNC) return CQ_OK;
    return read_status(l.status, s);
}

extern "C" int fp2s_init(const fp2s_problem_t *p, const double *G0_dev, void *ws_dev, size_t *ws_bytes,
                         void *stream) {
    Fp2sParams P;
    int np1 = 0, np2 = 0;
    int st = derive(p, P, np1, np2);
    if (st) return st;
    if (P.prec != CQ_F64) return CQ_EUNSUPPORTED;
    if (!ws_bytes) return CQ_EINVAL;
    Fp2sLayout l = fp2s_layout(p, P, ws_dev, true);
    if (!ws_dev) { *ws_bytes = l.bytes; return CQ_OK; }
    if (*ws_bytes < l.bytes) return CQ_ENOMEM;
    if (!G0_dev || ((uintptr_t)ws_dev & 255)) return CQ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = setup(p, P, np1, np2, l, G0_dev, s))) return st;
    if (P.form == CQ_FAST) {
        if ((st = cuda_status(cudaMemsetAsync(l.Y, 0, (size_t)2 * P.np * P.nmodes * sizeof(double), s)))) return st;
        if ((st = cuda_status(cudaMemsetAsync(l.ring, 0, (size_t)2 * P.L * P.nmodes * sizeof(double), s)))) return st;
    }
    const unsigned g = (unsigned)((2 * P.nmodes + 255) / 256);
    k_copy_levels<<<g, 256, 0, s>>>(l.g0, P.nmodes, l.hist, l.glast);
    if ((st = launched())) return st;
    return cuda_status(cudaMemcpyAsync(l.gN, l.g0, 2 * P.nmodes * sizeof(double), cudaMemcpyDeviceToDevice, s));
}

extern "C" int fp2s_step(const fp2s_problem_t *p, int64_t n, void *ws_dev, size_t ws_bytes, double *G_out_dev,
                         void *stream) {
    Fp2sParams P;
    int np1 = 0, np2 = 0;
    int st = derive(p, P, np1, np2);
    if (st) return st;
    if (P.prec != CQ_F64) return CQ_EUNSUPPORTED;
    if (!ws_dev || n < 1 || n > P.N) return CQ_EINVAL;
    Fp2sLayout l = fp2s_layout(p, P, ws_dev, true);
    if (ws_bytes < l.bytes) return CQ_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((P.nmodes + 255) / 256);
    if (P.form == CQ_FAST)
        k_fp2s_step_fast<<<blocks, 256, 0, s>>>(P, n, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.tab1, l.tab2, l.Y,
                                                l.ring, l.glast);
    else
        k_fp2s_step_direct<<<blocks, 256, 0, s>>>(P, n, l.lam, l.g0, l.gN, l.status, l.d1, l.d2, l.hist, l.glast);
    if ((st = launched())) return st;
    if (G_out_dev) return launch_dst_field(p->M, p->dim, l.S, l.gN, G_out_dev, l.tmp, s);
    return CQ_OK;
}

extern "C" int fp2s_modal(const fp2s_problem_t *p, const void *ws_dev, size_t ws_bytes, double *g_dev,
                          void *stream) {
    Fp2sParams P;
    int np1 = 0, np2 = 0;
    int st = derive(p, P, np1, np2);
    if (st) return st;
    if (!ws_dev || !g_dev) return CQ_EINVAL;
    Fp2sLayout l = fp2s_layout(p, P, const_cast<void *>(ws_dev), true);
    if (ws_bytes < l.bytes) return CQ_ENOMEM;
    return cuda_status(cudaMemcpyAsync(g_dev, l.gN, 2 * P.nmodes * sizeof(double), cudaMemcpyDeviceToDevice,
                                       (cudaStream_t)stream));
}

extern "C" int fp2s_status(const fp2s_problem_t *p, const void *ws_dev, size_t ws_bytes, void *stream) {
    Fp2sParams P;
    int np1 = 0, np2 = 0;
    int st = derive(p, P, np1, np2);
    if (st) return st;
    if (!ws_dev) return CQ_EINVAL;
    Fp2sLayout l = fp2s_layout(p, P, const_cast<void *>(ws_dev), false);
    (void)ws_bytes;
    return read_status(l.status, (cudaStream_t)stream);
}

// ===========================================================================
// Gradient of J = 1/2 h^dim sum (G^N - Gt)^2 through the direct schemes
// (discrete adjoint). Per mode, with K = [[c, -a], [-a, c]], W_i = diag(d1_i, d2_i),
// mu^n = K lambda^n, the adjoint runs backwards from m = N:
//   BE:  (I/tau + W_0 K) lambda^m = -[m=N] r + [m<N] lambda^{m+1}/tau - sum_{n>m} W_{n-m} mu^n
//   SBD: (c_m I + e_m W_0 K) lambda^m = -[m=N] r - sum_{n>m} W_{n-m} mu^n
//                                       + (2/tau) lambda^{m+1} - lambda^{m+2}/(2 tau)
//        ((c_1, e_1) = (1/tau, 2/3), (c_m, e_m) = (3/(2tau), 1) for m >= 2),
// r = h^dim (x^N - t). The sum over n > m is the CQ convolution run backwards in
// time with the same weights. dJ/dbeta_s = sum_m x_s^m sum_{n>=m} d'_{n-m} mu_s^n
// (+ the SBD first-step and G^0 terms), dJ/dx^0 from lambda^1, lambda^2 and
// sum_{n>=2} d_{n-1} mu^n. One backward sweep per mode (one thread), in blocks of
// BT steps: one pass over the future mu^n feeds both running sums through two
// shifting register windows of weights (d and d').
// ===========================================================================

// d(d_i)/d(beta), i = 0..n: with g_i the coefficients of (1-zeta)^beta,
// g'_i = g_i S_i, S_i = -sum_{k=1}^{i} 1/(k-1-beta) (a block-wide sum scan), and
//   BE:   d_i = tau^-beta g_i                          -> d'_i = tau^-beta (g'_i - ln(tau) g_i)
//   BDF2: d_i = tau^-beta 1.5^beta sum_k g_{i-k} g_k 3^-k
//         -> d'_i = tau^-beta 1.5^beta [ (ln 1.5 - ln tau) c_i + sum_k (g'_{i-k} g_k + g_{i-k} g'_k) 3^-k ].
__global__ void __launch_bounds__(1024) k_dweights(int scheme, double beta, double tau, int n,
                                                   double *__restrict__ out) {
    extern __shared__ double smd[];
    double *g = smd, *gp = smd + (n + 1);
    __shared__ double part[1024], psum[1024];
    __shared__ double bk[65], bpk[65];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (n + 1 + T - 1) / T;
    const int lo = t * chunk, hi = min(lo + chunk, n + 1);
    double p = 1.0, q = 0.0;
    for (int i = max(lo, 1); i < hi; ++i) {
        p *= (i - 1.0 - beta) / i;
        q -= 1.0 / (i - 1.0 - beta);
    }
    part[t] = p;
    psum[t] = q;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        const double x = (t >= off) ? part[t - off] : 1.0;
        const double y = (t >= off) ? psum[t - off] : 0.0;
        __syncthreads();
        part[t] *= x;
        psum[t] += y;
        __syncthreads();
    }
    double v = (t == 0) ? 1.0 : part[t - 1];
    double S = (t == 0) ? 0.0 : psum[t - 1];
    for (int i = lo; i < hi; ++i) {
        if (i >= 1) {
            v *= (i - 1.0 - beta) / i;
            S -= 1.0 / (i - 1.0 - beta);
        }
        g[i] = v;
        gp[i] = v * S;
    }
    __syncthreads();
    const double tb = pow(tau, -beta), lt = log(tau);
    if (scheme == CQ_BE) {
        for (int i = t; i <= n; i += T) out[i] = tb * (gp[i] - lt * g[i]);
        return;
    }
    if (t <= 64 && t <= n) {
        const double s3 = pow(3.0, (double)t);
        bk[t] = g[t] / s3;
        bpk[t] = gp[t] / s3;
    }
    __syncthreads();
    const double C = pow(1.5, beta), l15 = log(1.5);
    for (int i = t; i <= n; i += T) {
        const int kmax = min(i, 64);
        double c = 0.0, cp = 0.0;
        for (int k = kmax; k >= 0; --k) {
            c = fma(g[i - k], bk[k], c);
            cp = fma(gp[i - k], bk[k], fma(g[i - k], bpk[k], cp));
        }
        out[i] = tb * C * ((l15 - lt) * c + cp);
    }
}

constexpr int kAdjBT = 4;

template <int BT>
__global__ void __launch_bounds__(32, 12) k_adjoint_direct(
    Fp2sParams P, double wd, const double *__restrict__ lam, const double *__restrict__ d1,
    const double *__restrict__ d2, const double *__restrict__ dz1, const double *__restrict__ dz2,
    const double *__restrict__ q1, const double *__restrict__ q2, const double *__restrict__ qz1,
    const double *__restrict__ qz2, const double *__restrict__ hist, const double *__restrict__ tgt, int vjp,
    double *__restrict__ mu, double *__restrict__ gx0, double *__restrict__ acc) {
    const int64_t nm = P.nmodes;
    const int64_t mode_raw = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = mode_raw < nm;
    const int64_t mode = active ? mode_raw : 0;
    const int64_t N = P.N;
    const double a = P.a, c = a + lam[mode], it = P.inv_tau;
    const double d10 = __ldg(d1), d20 = __ldg(d2);
    // transposed step matrices c0 I + e0 W_0 K and their inverses
    Inv2 Mn, M1;
    bool ok;
    {
        const double c0 = (P.scheme == CQ_BE) ? it : 1.5 * it;
        ok = invert2(c0 + d10 * c, -d10 * a, -d20 * a, c0 + d20 * c, Mn);
        if (P.scheme == CQ_BDF2)
            ok &= invert2(it + (2.0 / 3.0) * d10 * c, -(2.0 / 3.0) * d10 * a, -(2.0 / 3.0) * d20 * a,
                          it + (2.0 / 3.0) * d20 * c, M1);
    }
    const double xN1 = hist[(N * 2) * nm + mode], xN2 = hist[(N * 2 + 1) * nm + mode];
    // terminal condition dJ/dx^N: the misfit's wd (x^N - t), or (vjp) the given modal gradient
    const double e1 = xN1 - tgt[mode], e2 = xN2 - tgt[nm + mode];
    const double r1 = vjp ? tgt[mode] : wd * e1, r2 = vjp ? tgt[nm + mode] : wd * e2;
    double Jpart = (active && !vjp) ? 0.5 * wd * (e1 * e1 + e2 * e2) : 0.0;
    double lp1_1 = 0.0, lp1_2 = 0.0, lp2_1 = 0.0, lp2_2 = 0.0;      // lambda^{m+1}, lambda^{m+2}
    double db1 = 0.0, db2 = 0.0, sg1 = 0.0, sg2 = 0.0, sx1 = 0.0, sx2 = 0.0;
    double lam1_1 = 0.0, lam1_2 = 0.0, lam2_1 = 0.0, lam2_2 = 0.0, mu1_1 = 0.0, mu1_2 = 0.0;
    // idle lanes (past the last mode) skip the sweep: they take part in the warp sums only
    for (int64_t mhi = active ? N : 0; mhi >= 1; mhi -= BT) {
        double ar1[BT], ar2[BT], aq1[BT], aq2[BT], w1[BT], w2[BT], wq1[BT], wq2[BT], u1[BT] = {}, u2[BT] = {};
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            ar1[b] = ar2[b] = aq1[b] = aq2[b] = 0.0;
            w1[b] = __ldg(dz1 + 1 + b + BT);
            w2[b] = __ldg(dz2 + 1 + b + BT);
            wq1[b] = __ldg(qz1 + 1 + b + BT);
            wq2[b] = __ldg(qz2 + 1 + b + BT);
        }
        const double *mp = mu + ((mhi + 1) * 2) * nm + mode;
        for (int64_t n = mhi + 1; n <= N; ++n, mp += 2 * nm) {
            const double v1 = mp[0], v2 = mp[nm];
#pragma unroll
            for (int b = 0; b < BT; ++b) {
                ar1[b] = fma(w1[b], v1, ar1[b]);
                ar2[b] = fma(w2[b], v2, ar2[b]);
                aq1[b] = fma(wq1[b], v1, aq1[b]);
                aq2[b] = fma(wq2[b], v2, aq2[b]);
            }
#pragma unroll
            for (int b = 0; b < BT - 1; ++b) {
                w1[b] = w1[b + 1];
                w2[b] = w2[b + 1];
                wq1[b] = wq1[b + 1];
                wq2[b] = wq2[b + 1];
            }
            const int64_t top = (n + 1 - mhi + BT - 1) + BT;
            w1[BT - 1] = __ldg(dz1 + top);
            w2[BT - 1] = __ldg(dz2 + top);
            wq1[BT - 1] = __ldg(qz1 + top);
            wq2[BT - 1] = __ldg(qz2 + top);
        }
#pragma unroll
        for (int b = 0; b < BT; ++b) {
            const int64_t m = mhi - b;
            if (m < 1) break;
            double h1 = ar1[b], h2 = ar2[b], hq1 = aq1[b], hq2 = aq2[b];
#pragma unroll
            for (int bb = 0; bb < b; ++bb) {
                h1 = fma(__ldg(dz1 + (b - bb) + BT), u1[bb], h1);
                h2 = fma(__ldg(dz2 + (b - bb) + BT), u2[bb], h2);
                hq1 = fma(__ldg(qz1 + (b - bb) + BT), u1[bb], hq1);
                hq2 = fma(__ldg(qz2 + (b - bb) + BT), u2[bb], hq2);
            }
            double b1 = -h1, b2 = -h2;
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
            u1[b] = v1;
            u2[b] = v2;
            mu[(m * 2) * nm + mode] = v1;
            mu[(m * 2 + 1) * nm + mode] = v2;
            hq1 = fma(__ldg(q1), v1, hq1);                      // n = m term, d'_0
            hq2 = fma(__ldg(q2), v2, hq2);
            db1 = fma(hist[(m * 2) * nm + mode], hq1, db1);
            db2 = fma(hist[(m * 2 + 1) * nm + mode], hq2, db2);
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
    const double x01 = hist[mode], x02 = hist[nm + mode];
    double g1, g2;
    if (P.scheme == CQ_BE) {
        g1 = -lam1_1 * it;
        g2 = -lam1_2 * it;
    } else {
        g1 = -lam1_1 * it + d10 * mu1_1 / 3.0 + 0.5 * it * lam2_1 + 0.5 * sg1;
        g2 = -lam1_2 * it + d20 * mu1_2 / 3.0 + 0.5 * it * lam2_2 + 0.5 * sg2;
        const double x11 = hist[2 * nm + mode], x12 = hist[3 * nm + mode];
        db1 += mu1_1 * __ldg(q1) * (x01 - x11) / 3.0 + 0.5 * x01 * sx1;
        db2 += mu1_2 * __ldg(q2) * (x02 - x12) / 3.0 + 0.5 * x02 * sx2;
    }
    if (active) {
        gx0[mode] = g1;
        gx0[nm + mode] = g2;
    } else {
        db1 = db2 = 0.0;
    }
    // warp sums, one atomic per warp and quantity
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

struct GradLayout {
    double *tgt, *mu, *gx0, *q1, *q2, *qz1, *qz2, *dza1, *dza2, *acc;
    double *fder1, *fder2, *ftmp;        // fast form: (c', c r') of each state's tables; their builds
    float *adtab;                        // fast form, CQ_DF64: tables of the double-float backward sweep
    float4 *wa, *qa;                     // CQ_DF64: d and d' of both states padded for the double-float adjoint
    double *cg0, *ctgt, *cgx0, *cgN;     // compact [2][ns] copies of a slice (sliced runs only)
    size_t bytes;
};

// ns: modes per slice (the forward history and the adjoint variables hold ns modes).
static GradLayout grad_layout(const Fp2sParams &P, const Fp2sLayout &base, void *ws, int64_t ns) {
    GradLayout g{};
    Carve cv(ws);
    cv.off = base.bytes;
    const int64_t nm = P.nmodes;
    g.acc = cv.take<double>(8);
    g.tgt = cv.take<double>(2 * nm);
    g.gx0 = cv.take<double>(2 * nm);
    g.q1 = cv.take<double>(P.N + 1);
    g.q2 = cv.take<double>(P.N + 1);
    if (P.form == CQ_FAST) {             // the fast adjoint keeps its levels on chip: no mu
        g.fder1 = cv.take<double>(2 * P.np);
        g.fder2 = cv.take<double>(2 * P.np);
        g.ftmp = cv.take<double>(8 * P.np);
        if (P.prec == CQ_DF64) g.adtab = cv.take<float>(kAdjDfTabFloats);
        if (ns < nm) {
            g.cg0 = cv.take<double>(2 * ns);
            g.ctgt = cv.take<double>(2 * ns);
            g.cgx0 = cv.take<double>(2 * ns);
            g.cgN = cv.take<double>(2 * ns);
        }
        g.bytes = cv.bytes();
        return g;
    }
    g.qz1 = cv.take<double>(P.N + 2 * kAdjBT + 1);
    g.qz2 = cv.take<double>(P.N + 2 * kAdjBT + 1);
    g.dza1 = cv.take<double>(P.N + 2 * kAdjBT + 1);
    g.dza2 = cv.take<double>(P.N + 2 * kAdjBT + 1);
    const bool df = P.prec == CQ_DF64;
    if (df) {
        g.wa = cv.take<float4>(P.N + 4 * kAdjDfBT);
        g.qa = cv.take<float4>(P.N + 4 * kAdjDfBT);
    }
    // FP64: [N + 1][2][ns] doubles; CQ_DF64: [N + 1 + kAdjDfBT][ns] float4 (zero levels past N)
    g.mu = cv.take<double>((size_t)(P.N + 1 + (df ? kAdjDfBT : 0)) * 2 * ns);
    if (ns < nm) {
        g.cg0 = cv.take<double>(2 * ns);
        g.ctgt = cv.take<double>(2 * ns);
        g.cgx0 = cv.take<double>(2 * ns);
        g.cgN = cv.take<double>(2 * ns);
    }
    g.bytes = cv.bytes();
    return g;
}

static size_t grad64_bytes(const fp2s_problem_t *p, const Fp2sParams &P, int64_t ns) {
    const Fp2sLayout l = fp2s_layout(p, P, nullptr, false, true, ns);
    return grad_layout(P, l, nullptr, ns).bytes;
}

constexpr int64_t kGradSliceQuantum = 32;    // modes per warp of the forward and adjoint kernels

// Modes per slice of the FP64 gradient for a workspace of `cap` bytes: all modes when the
// whole problem fits, else the largest multiple of 32 that fits (0: nothing fits).
static int64_t grad64_slice(const fp2s_problem_t *p, const Fp2sParams &P, size_t cap) {
    if (grad64_bytes(p, P, P.nmodes) <= cap) return P.nmodes;
    int64_t lo = 0, hi = (P.nmodes - 1) / kGradSliceQuantum;           // in units of 32 modes
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (grad64_bytes(p, P, mid * kGradSliceQuantum) <= cap) lo = mid;
        else hi = mid - 1;
    }
    return lo * kGradSliceQuantum;
}

// [2][cnt] <-> rows s * nm + m0 .. + cnt of a [2][nm] array.
static int copy_slice(double *dst, int64_t ldd, const double *src, int64_t lds, int64_t cnt, cudaStream_t s) {
    for (int st = 0; st < 2; ++st) {
        if (cudaMemcpyAsync(dst + st * ldd, src + st * lds, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            return CQ_ECUDA;
    }
    return CQ_OK;
}

static int weight_derivatives(const Fp2sParams &P, const fp2s_problem_t *p, double *q1, double *q2,
                              cudaStream_t s) {
    static unsigned long long attr = 0;
    int st;
    if ((st = smem_attr_once((const void *)k_dweights, (int)(2 * 13001 * sizeof(double)), &attr))) return st;
    const size_t dsm = (size_t)2 * (P.N + 1) * sizeof(double);
    k_dweights<<<1, 1024, dsm, s>>>(P.scheme, 1.0 - p->alpha1, P.tau, (int)P.N, q1);
    k_dweights<<<1, 1024, dsm, s>>>(P.scheme, 1.0 - p->alpha2, P.tau, (int)P.N, q2);
    return launched(2);
}

static double grid_weight(const fp2s_problem_t *p) {
    const double h = 1.0 / (p->M + 1);
    return (p->dim == 1) ? h : (p->dim == 2) ? h * h : h * h * h;
}

// Gradient through the mixed-precision direct solve (mixed.cu): same outputs as the
// FP64 gradient, computed from FP32 levels and tensor-core histories. The mixed region
// holds the split levels and histories of ns modes: all modes, or (when the workspace is
// capped) a slice, the slices running one after the other with compact [2][ns] copies of
// their modal G^0, target and dJ/dx^0.
struct MixedGradLayout {
    Fp2sLayout l;
    double *acc, *tgt, *gx0, *q1, *q2;
    double *cg0, *ctgt, *cgx0, *cgN;
    size_t bytes;
};

static MixedGradLayout mixed_grad_layout(const fp2s_problem_t *p, const Fp2sParams &P, void *ws, int64_t ns) {
    MixedGradLayout g{};
    g.l = fp2s_layout(p, P, ws, false, true, ns);
    Carve cv(ws);
    cv.off = g.l.bytes;
    g.acc = cv.take<double>(8);
    g.tgt = cv.take<double>(2 * P.nmodes);
    g.gx0 = cv.take<double>(2 * P.nmodes);
    g.q1 = cv.take<double>(P.N + 1);
    g.q2 = cv.take<double>(P.N + 1);
    if (ns < P.nmodes) {
        g.cg0 = cv.take<double>(2 * ns);
        g.ctgt = cv.take<double>(2 * ns);
        g.cgx0 = cv.take<double>(2 * ns);
        g.cgN = cv.take<double>(2 * ns);
    }
    g.bytes = cv.bytes();
    return g;
}

constexpr int64_t kMixedSliceQuantum = 64;   // modes per CTA of the mixed block kernels

// Modes per slice of the mixed gradient within `cap` bytes (all modes when they fit; 0: none fits).
static int64_t mixed_grad_slice(const fp2s_problem_t *p, const Fp2sParams &P, size_t cap) {
    if (mixed_grad_layout(p, P, nullptr, P.nmodes).bytes <= cap) return P.nmodes;
    int64_t lo = 0, hi = (P.nmodes - 1) / kMixedSliceQuantum;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (mixed_grad_layout(p, P, nullptr, mid * kMixedSliceQuantum).bytes <= cap) lo = mid;
        else hi = mid - 1;
    }
    return lo * kMixedSliceQuantum;
}

static int gradient_mixed(const fp2s_problem_t *p, const Fp2sParams &P, int np1, int np2, const double *G0_dev,
                          const double *Gt_dev, int vjp, double *J_host, double *dJdG0_dev, double *dJdalpha_host,
                          void *ws_dev, size_t *ws_bytes, cudaStream_t s) {
    if (!ws_dev) {
        if (*ws_bytes == 0) { *ws_bytes = mixed_grad_layout(p, P, nullptr, P.nmodes).bytes; return CQ_OK; }
        const int64_t ns = mixed_grad_slice(p, P, *ws_bytes);
        if (ns == 0) return CQ_ENOMEM;
        *ws_bytes = mixed_grad_layout(p, P, nullptr, ns).bytes;
        return CQ_OK;
    }
    const int64_t ns = mixed_grad_slice(p, P, *ws_bytes);
    if (ns == 0) return CQ_ENOMEM;
    const MixedGradLayout g = mixed_grad_layout(p, P, ws_dev, ns);
    const Fp2sLayout &l = g.l;
    if (!G0_dev || !Gt_dev || (!vjp && !J_host) || !dJdG0_dev || !dJdalpha_host || ((uintptr_t)ws_dev & 255))
        return CQ_EINVAL;
    int st;
    if ((st = setup(p, P, np1, np2, l, G0_dev, s))) return st;
    if ((st = timing_begin(s))) return st;
    if ((st = launch_dst_field(p->M, p->dim, l.S, Gt_dev, g.tgt, l.tmp, s))) return st;
    if ((st = weight_derivatives(P, p, g.q1, g.q2, s))) return st;
    if ((st = cuda_status(cudaMemsetAsync(g.acc, 0, 8 * sizeof(double), s)))) return st;
    const int64_t nm = P.nmodes;
    for (int64_t m0 = 0; m0 < nm; m0 += ns) {
        const int64_t cnt = min(ns, nm - m0);
        Fp2sParams Ps = P;
        Ps.nmodes = cnt;
        const double *g0 = l.g0, *tgt = g.tgt;
        double *gN = l.gN, *gx0 = g.gx0;
        if (ns < nm) {
            if ((st = copy_slice(g.cg0, cnt, l.g0 + m0, nm, cnt, s))) return st;
            if ((st = copy_slice(g.ctgt, cnt, g.tgt + m0, nm, cnt, s))) return st;
            g0 = g.cg0;
            tgt = g.ctgt;
            gN = g.cgN;
            gx0 = g.cgx0;
        }
        if ((st = mixed_grad_run(Ps, l.lam + m0, g0, gN, l.status, l.d1, l.d2, g.q1, g.q2, l.hdf, tgt, vjp,
                                 grid_weight(p), gx0, g.acc, l.mixed, s)))
            return st;
        if (ns < nm && (st = copy_slice(g.gx0 + m0, nm, g.cgx0, cnt, cnt, s))) return st;
    }
    if ((st = timing_end(s))) return st;
    if ((st = launch_dst_field(p->M, p->dim, l.S, g.gx0, dJdG0_dev, l.tmp, s))) return st;
    double host[4];
    if (cudaMemcpyAsync(host, g.acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CQ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CQ_ECUDA;
    if (J_host) *J_host = host[0];
    dJdalpha_host[0] = -host[1];
    dJdalpha_host[1] = -host[2];
    if ((st = read_status(l.status, s))) return st;
    if (!isfinite(host[0]) || !isfinite(host[1]) || !isfinite(host[2])) return CQ_ENONFINITE;
    return CQ_OK;
}

// Forward direct solve (history kept), then the adjoint sweep. vjp = 0: terminal condition
// from the misfit against Gt; vjp = 1: Gt holds dL/dG^N and J is not formed.
static int gradient_impl(const fp2s_problem_t *p, const double *G0_dev, const double *Gt_dev, int vjp,
                         double *J_host, double *dJdG0_dev, double *dJdalpha_host, void *ws_dev, size_t *ws_bytes,
                         void *stream) {
    Fp2sParams P;
    int np1 = 0, np2 = 0;
    int st = derive(p, P, np1, np2);
    if (st) return st;
    if (!ws_bytes) return CQ_EINVAL;
    const bool mixed = P.prec == CQ_BF16X3 || P.prec == CQ_TF32X3;
    const bool fast = P.form == CQ_FAST;
    if (fast ? (P.prec != CQ_F64 && P.prec != CQ_DF64) : !(P.prec == CQ_F64 || P.prec == CQ_DF64 || mixed))
        return CQ_EUNSUPPORTED;
    if (P.N > 13000) return CQ_EUNSUPPORTED;            // shared-memory bound of the weight derivatives
    if (mixed)
        return gradient_mixed(p, P, np1, np2, G0_dev, Gt_dev, vjp, J_host, dJdG0_dev, dJdalpha_host, ws_dev,
                              ws_bytes, (cudaStream_t)stream);
    // The forward history and the adjoint variables take (N + 1) x 2 x modes each. Modes are
    // independent, so a workspace that cannot hold them for all modes runs the forward and
    // adjoint sweeps over slices of modes; a nonzero *ws_bytes in a size query is such a cap.
    if (!ws_dev) {
        if (*ws_bytes == 0) { *ws_bytes = grad64_bytes(p, P, P.nmodes); return CQ_OK; }
        const int64_t ns = grad64_slice(p, P, *ws_bytes);
        if (ns == 0) return CQ_ENOMEM;
        *ws_bytes = grad64_bytes(p, P, ns);
        return CQ_OK;
    }
    const int64_t ns = grad64_slice(p, P, *ws_bytes);
    if (ns == 0) return CQ_ENOMEM;
    Fp2sLayout l = fp2s_layout(p, P, ws_dev, false, true, ns);
    GradLayout gl = grad_layout(P, l, ws_dev, ns);
    if (!G0_dev || !Gt_dev || (!vjp && !J_host) || !dJdG0_dev || !dJdalpha_host || ((uintptr_t)ws_dev & 255))
        return CQ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = setup(p, P, np1, np2, l, G0_dev, s))) return st;
    if ((st = timing_begin(s))) return st;
    if ((st = launch_dst_field(p->M, p->dim, l.S, Gt_dev, gl.tgt, l.tmp, s))) return st;
    if ((st = weight_derivatives(P, p, gl.q1, gl.q2, s))) return st;
    const bool df = P.prec == CQ_DF64;
    if (df && !fast && (st = direct_df_grad_tables(P.N, l.d1, l.d2, gl.q1, gl.q2, gl.wa, gl.qa, s)))
        return st;
    double *dzA1 = gl.dza1, *dzA2 = gl.dza2;
    if (fast) {
        // derivatives of the fast tables in beta (the tables at beta are in place)
        if ((st = fast_grad_tables(P.scheme, 1.0 - p->alpha1, P.tau, np1, np2, P.L, l.tab1, l.scr1, gl.ftmp,
                                   gl.fder1, s)))
            return st;
        if ((st = fast_grad_tables(P.scheme, 1.0 - p->alpha2, P.tau, np1, np2, P.L, l.tab2, l.scr1, gl.ftmp,
                                   gl.fder2, s)))
            return st;
        if (df && (st = fast_adjoint_df_tables(P, l.tab1, l.tab2, gl.fder1, gl.fder2, l.d1, l.d2, gl.q1, gl.q2,
                                               gl.adtab, s)))
            return st;
    } else {
        const unsigned pg = (unsigned)((P.N + 2 * kAdjBT + 256) / 256);
        k_pad<<<pg, 256, 0, s>>>(gl.q1, P.N, kAdjBT, gl.qz1);
        k_pad<<<pg, 256, 0, s>>>(gl.q2, P.N, kAdjBT, gl.qz2);
        if ((st = launched(2))) return st;
        // the adjoint needs the weights padded for its own block size
        k_pad<<<pg, 256, 0, s>>>(l.d1, P.N, kAdjBT, dzA1);
        k_pad<<<pg, 256, 0, s>>>(l.d2, P.N, kAdjBT, dzA2);
        if ((st = launched(2))) return st;
    }
    if ((st = cuda_status(cudaMemsetAsync(gl.acc, 0, 8 * sizeof(double), s)))) return st;
    const double wd = grid_weight(p);
    const int64_t nm = P.nmodes;
    for (int64_t m0 = 0; m0 < nm; m0 += ns) {
        const int64_t cnt = min(ns, nm - m0);
        Fp2sParams Ps = P;
        Ps.nmodes = cnt;
        const double *g0 = l.g0, *tgt = gl.tgt;
        double *gN = l.gN, *gx0 = gl.gx0;
        if (ns < nm) {                      // compact [2][cnt] copies of the slice
            if ((st = copy_slice(gl.cg0, cnt, l.g0 + m0, nm, cnt, s))) return st;
            if ((st = copy_slice(gl.ctgt, cnt, gl.tgt + m0, nm, cnt, s))) return st;
            g0 = gl.cg0;
            tgt = gl.ctgt;
            gN = gl.cgN;
            gx0 = gl.cgx0;
        }
        if (fast) {
            // forward fast solve keeping every level (double-float for CQ_DF64), then the backward
            // sweep of the fast adjoint
            if (df) {
                if ((st = fast_df_solve_hist(Ps, l.lam + m0, g0, gN, l.status, l.d1, l.d2, l.ftab, l.hist, s)))
                    return st;
                if ((st = launched())) return st;
            } else {
                const int T = fast_block_threads(P.np, P.L, cnt);
                if (T == 0) return CQ_EUNSUPPORTED;
                const size_t smem = fast_smem_bytes(P.np, P.L, T);
                if (cudaFuncSetAttribute(k_fp2s_fast<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem) != cudaSuccess)
                    return CQ_ECUDA;
                const int64_t mpb = (int64_t)(T / 32) * kFastModesPerWarp;
                k_fp2s_fast<true><<<(unsigned)((cnt + mpb - 1) / mpb), T, smem, s>>>(
                    Ps, l.lam + m0, g0, gN, l.status, l.d1, l.d2, l.tab1, l.tab2, l.hist);
                if ((st = launched())) return st;
            }
            st = df ? fast_adjoint_df_slice(Ps, wd, l.lam + m0, l.d1, l.d2, gl.q1, gl.q2, gl.adtab, l.hist, tgt, vjp,
                                            gx0, gl.acc, s)
                    : fast_adjoint_slice(Ps, wd, l.lam + m0, l.d1, l.d2, gl.q1, gl.q2, l.tab1, l.tab2, gl.fder1,
                                         gl.fder2, l.hist, tgt, vjp, gx0, gl.acc, s);
            if (st) return st;
            if (ns < nm && (st = copy_slice(gl.gx0 + m0, nm, gl.cgx0, cnt, cnt, s))) return st;
            continue;
        }
        if (df) {
            if ((st = direct_df_gradient_slice(Ps, wd, l.lam + m0, g0, gN, l.status, l.d1, l.d2, gl.q1, gl.q2, l.wz,
                                               gl.wa, gl.qa, l.hist2, tgt, vjp, reinterpret_cast<float4 *>(gl.mu),
                                               gx0, gl.acc, s)))
                return st;
            if (ns < nm && (st = copy_slice(gl.gx0 + m0, nm, gl.cgx0, cnt, cnt, s))) return st;
            continue;
        }
        const unsigned fblocks = (unsigned)((cnt + 31) / 32);
        k_fp2s_direct<kDirBT><<<fblocks, 32, 0, s>>>(Ps, l.lam + m0, g0, gN, l.status, l.d1, l.d2, l.dz1, l.dz2,
                                                     l.hist);
        k_adjoint_direct<kAdjBT><<<fblocks, 32, 0, s>>>(Ps, wd, l.lam + m0, l.d1, l.d2, dzA1, dzA2, gl.q1, gl.q2,
                                                        gl.qz1, gl.qz2, l.hist, tgt, vjp, gl.mu, gx0, gl.acc);
        if ((st = launched(2))) return st;
        if (ns < nm && (st = copy_slice(gl.gx0 + m0, nm, gl.cgx0, cnt, cnt, s))) return st;
    }
    if ((st = timing_end(s))) return st;
    if ((st = launch_dst_field(p->M, p->dim, l.S, gl.gx0, dJdG0_dev, l.tmp, s))) return st;
    double host[4];
    if (cudaMemcpyAsync(host, gl.acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CQ_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CQ_ECUDA;
    if (J_host) *J_host = host[0];
    dJdalpha_host[0] = -host[1];
    dJdalpha_host[1] = -host[2];
    if (host[3] != 0.0) return CQ_ESINGULAR;
    if ((st = read_status(l.status, s))) return st;
    if (!isfinite(host[0]) || !isfinite(host[1]) || !isfinite(host[2])) return CQ_ENONFINITE;
    return CQ_OK;
}

extern "C" int fp2s_gradient(const fp2s_problem_t *p, const double *G0_dev, const double *Gt_dev, double *J_host,
                             double *dJdG0_dev, double *dJdalpha_host, void *ws_dev, size_t *ws_bytes,
                             void *stream) {
    return gradient_impl(p, G0_dev, Gt_dev, 0, J_host, dJdG0_dev, dJdalpha_host, ws_dev, ws_bytes, stream);
}

extern "C" int fp2s_vjp(const fp2s_problem_t *p, const double *G0_dev, const double *dGN_dev, double *dG0_dev,
                        double *dalpha_host, void *ws_dev, size_t *ws_bytes, void *stream) {
    return gradient_impl(p, G0_dev, dGN_dev, 1, nullptr, dG0_dev, dalpha_host, ws_dev, ws_bytes, stream);
}
