// Batched solves: many independent two-state problems (uneven alpha, m, grid,
// N, scheme) advanced by one persistent launch of the fused fast FP64 kernel.
//
// fp2s_batch_plan validates the problems, lays out one workspace with every
// instance's tables (CQ weights, Gauss-Jacobi rules, fast coefficients,
// sine-mode eigenvalues, DST-I matrix), builds them with batched kernels (one
// launch per kind of table for the whole batch), cuts every instance into work
// units of 16 x WB modes, orders the units by decreasing cost (longest
// processing time first) and, when asked, autotunes the launch shape: every
// block width WB whose shared memory fits, each with the full occupancy and with
// half of it (resident CTAs per SM), and each node-loop width (2, 4 or 8 partial
// sums), timed on a shortened run (median of three) and the fastest kept.
// fp2s_solve_batched then only transforms G0, runs the persistent kernel (its
// CTAs take units from an atomic counter: no CTA ever waits for another) and
// transforms back: five launches and one memset, with no host synchronisation,
// so the call can be captured in a CUDA graph.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "fastdf.cuh"
#include "fp2s_core.cuh"
#include "table_kernels.cuh"

namespace fastcq {

// Instances of one batch: the per-instance set-up and transform kernels put the instance
// on the grid's y axis.
constexpr int kMaxBatch = 65535;

struct InstDesc {
    double a, tau, inv_tau, beta1, beta2;
    int64_t N, nmodes;
    int scheme, np, np1, np2, L, M, dim, pad;
    int64_t o_w, o_tab, o_scr, o_lam, o_S, o_modal, o_field;
};

struct Unit {
    int inst;
    int first_mode;
};

struct BatchLayout {
    int *status, *counter;
    InstDesc *desc;
    Unit *units;
    double *W, *tab, *scr, *lam, *S, *modal;
    float *dftab;                        // double-float batches: [instance][kDfTabFloats]
    size_t bytes;
};

struct BatchSizes {
    int64_t w = 0, tab = 0, scr = 0, lam = 0, S = 0, modal = 0, field = 0, dftab = 0;
    int maxnp = 1, maxL = 2, maxM = 1;
    int64_t maxN = 1, max_nmodes = 1;
};

enum { R_STATUS, R_COUNTER, R_DESC, R_UNITS, R_W, R_TAB, R_SCR, R_LAM, R_S, R_MODAL, R_DFTAB, R_END };

static BatchLayout batch_layout(void *ws, int n_inst, int64_t n_units, const BatchSizes &z, int64_t *off) {
    Carve cv(ws);
    BatchLayout l{};
    auto mark = [&](int r) { if (off) off[r] = (int64_t)align_up(cv.off); };
    mark(R_STATUS);
    l.status = cv.take<int>(64);
    mark(R_COUNTER);
    l.counter = cv.take<int>(64);
    mark(R_DESC);
    l.desc = cv.take<InstDesc>(n_inst);
    mark(R_UNITS);
    l.units = cv.take<Unit>(n_units);
    mark(R_W);
    l.W = cv.take<double>(z.w);
    mark(R_TAB);
    l.tab = cv.take<double>(z.tab);
    mark(R_SCR);
    l.scr = cv.take<double>(z.scr);
    mark(R_LAM);
    l.lam = cv.take<double>(z.lam);
    mark(R_S);
    l.S = cv.take<double>(z.S);
    mark(R_MODAL);
    l.modal = cv.take<double>(z.modal);
    mark(R_DFTAB);
    l.dftab = cv.take<float>(z.dftab);
    l.bytes = cv.bytes();
    if (off) off[R_END] = (int64_t)l.bytes;
    return l;
}

static BatchLayout layout_from_plan(const fp2s_batch_t *plan, void *ws) {
    char *b = static_cast<char *>(ws);
    BatchLayout l{};
    l.status = reinterpret_cast<int *>(b + plan->off[R_STATUS]);
    l.counter = reinterpret_cast<int *>(b + plan->off[R_COUNTER]);
    l.desc = reinterpret_cast<InstDesc *>(b + plan->off[R_DESC]);
    l.units = reinterpret_cast<Unit *>(b + plan->off[R_UNITS]);
    l.W = reinterpret_cast<double *>(b + plan->off[R_W]);
    l.tab = reinterpret_cast<double *>(b + plan->off[R_TAB]);
    l.scr = reinterpret_cast<double *>(b + plan->off[R_SCR]);
    l.lam = reinterpret_cast<double *>(b + plan->off[R_LAM]);
    l.S = reinterpret_cast<double *>(b + plan->off[R_S]);
    l.modal = reinterpret_cast<double *>(b + plan->off[R_MODAL]);
    l.dftab = reinterpret_cast<float *>(b + plan->off[R_DFTAB]);
    l.bytes = (size_t)plan->off[R_END];
    return l;
}

// ---------------------------------------------------------------------------
// batched set-up kernels (blockIdx.x = instance unless stated)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWThreads) k_b_weights(const InstDesc *__restrict__ D, double *__restrict__ W) {
    extern __shared__ double g[];
    const InstDesc d = D[blockIdx.x];
    const int s = blockIdx.y;
    const double beta = s ? d.beta2 : d.beta1;
    weights_block(d.scheme, beta, pow(d.tau, -beta), (int)d.N, W + d.o_w + s * (d.N + 1), g);
}

// grid (instance, 4 = state x family, node blocks of kGJThreads)
__global__ void __launch_bounds__(kGJThreads) k_b_gauss_jacobi(const InstDesc *__restrict__ D, double *__restrict__ scr) {
    const InstDesc d = D[blockIdx.x];
    const int s = blockIdx.y >> 1, fam = blockIdx.y & 1;
    const int n = fam ? d.np2 : d.np1;
    const int j0 = blockIdx.z * kGJThreads;
    if (n == 0 || j0 >= n) return;
    const double beta = s ? d.beta2 : d.beta1;
    const double b = (d.scheme == CQ_BE) ? 1.0 - beta : 2.0 - 2.0 * beta;
    double *base = scr + d.o_scr + (int64_t)s * 2 * d.np + (fam ? 2 * d.np1 : 0);
    gauss_jacobi_block(n, beta, b, j0, base, base + n);
}

// grid (instance, state), block 256
__global__ void k_b_coeffs(const InstDesc *__restrict__ D, const double *__restrict__ scr, double *__restrict__ tab) {
    const InstDesc d = D[blockIdx.x];
    const int s = blockIdx.y;
    const double beta = s ? d.beta2 : d.beta1;
    const double *base = scr + d.o_scr + (int64_t)s * 2 * d.np;
    double *r = tab + d.o_tab + (int64_t)s * 2 * d.np, *c = r + d.np;
    for (int j = threadIdx.x; j < d.np; j += blockDim.x) {
        const bool fam1 = j < d.np1;
        const double sj = fam1 ? base[j] : base[2 * d.np1 + (j - d.np1)];
        const double lj = fam1 ? base[d.np1 + j] : base[2 * d.np1 + d.np2 + (j - d.np1)];
        fast_coeff_point(d.scheme, beta, d.tau, d.np1, d.L, j, sj, lj, r + j, c + j);
    }
}

// grid (element blocks, instance): eigenvalues (nmodes) and DST matrix (M*M)
__global__ void k_b_spectrum(const InstDesc *__restrict__ D, double *__restrict__ lam, double *__restrict__ S) {
    const InstDesc d = D[blockIdx.y];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int M = d.M;
    const double q = 2.0 * (M + 1), f = 4.0 * (double)(M + 1) * (double)(M + 1);
    if (i < d.nmodes) {
        if (d.dim == 1) {
            const double sv = sinpi((double)(i + 1) / q);
            lam[d.o_lam + i] = f * sv * sv;
        } else {
            const double sy = sinpi((double)(i / M + 1) / q), sx = sinpi((double)(i % M + 1) / q);
            lam[d.o_lam + i] = f * sy * sy + f * sx * sx;
        }
    }
    if (i < (int64_t)M * M) {
        const int64_t j = i / M + 1, k = i % M + 1;
        S[d.o_S + i] = sqrt(2.0 / (M + 1)) * sinpi((double)((j * k) % (2 * (int64_t)(M + 1))) / (double)(M + 1));
    }
}

// One pass of the sine transform of every instance. Regions: 0 = packed physical
// field (in / out argument), 1 = modal g0, 2 = modal gN, 3 = modal scratch.
// 1D: out = S in in one pass (pass 1, src -> dst). 2D (dof = iy*M + ix):
// pass 1 along y (src -> scratch), pass 2 along x (scratch -> dst).
__device__ __forceinline__ double *region(double *field, double *modal, const InstDesc &d, int which) {
    if (which == 0) return field + d.o_field;
    return modal + d.o_modal + (int64_t)(which - 1) * 2 * d.nmodes;
}

__global__ void k_b_dst_pass(const InstDesc *__restrict__ D, const double *__restrict__ S, const double *field_in,
                             double *field_out, double *modal, int pass, int src, int dst) {
    const InstDesc d = D[blockIdx.y];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * d.nmodes) return;
    if (d.dim == 1 && pass == 2) return;
    const int M = d.M;
    const double *Sm = S + d.o_S;
    const double *in = (pass == 1) ? region(const_cast<double *>(field_in), modal, d, src) : region(nullptr, modal, d, 3);
    double *out = (pass == 1 && d.dim == 2) ? region(nullptr, modal, d, 3) : region(field_out, modal, d, dst);
    const int64_t s = e / d.nmodes, r = e % d.nmodes;
    const double *ins = in + s * d.nmodes;
    double acc = 0.0;
    if (d.dim == 1) {
        for (int j = 0; j < M; ++j) acc = fma(Sm[(int64_t)r * M + j], ins[j], acc);
    } else if (pass == 1) {                                 // along y: out[y][x] = sum_j S[y][j] in[j][x]
        const int64_t y = r / M, x = r % M;
        for (int j = 0; j < M; ++j) acc = fma(Sm[y * M + j], ins[(int64_t)j * M + x], acc);
    } else {                                                // along x: out[y][x] = sum_j in[y][j] S[j][x]
        const int64_t y = r / M, x = r % M;
        for (int j = 0; j < M; ++j) acc = fma(ins[y * M + j], Sm[(int64_t)j * M + x], acc);
    }
    out[s * d.nmodes + r] = acc;
}

// ---------------------------------------------------------------------------
// persistent fast solve over work units (same per-mode arithmetic as k_fp2s_fast)
// ---------------------------------------------------------------------------
// NU: partial sums of the node loop (nodes processed NU at a time; a tuning knob).
template <int NU>
__global__ void __launch_bounds__(1024) k_b_fast(const InstDesc *__restrict__ D, const Unit *__restrict__ U,
                                                 int n_units, int *__restrict__ counter, int maxnp, int maxL,
                                                 int64_t step_cap, const double *__restrict__ W,
                                                 const double *__restrict__ tab, const double *__restrict__ lamp,
                                                 double *__restrict__ modal, int *__restrict__ status) {
    extern __shared__ double sm[];
    __shared__ int s_unit;
    const int T = blockDim.x, tid = threadIdx.x;
    double *rt = sm, *ct = rt + 2 * maxnp, *wt = ct + 2 * maxnp;
    double *Y = wt + 2 * kMaxNs;              // [maxnp][T]
    double *R = Y + (size_t)maxnp * T;        // [maxL][T]
    const int lane = tid & 31, st = lane >> 4;
    const int modes_per_unit = (T >> 5) * kFastModesPerWarp;
    for (;;) {
        if (tid == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= n_units) break;
        const Unit un = U[u];
        const InstDesc d = D[un.inst];
        const int np = d.np, L = d.L;
        const double *t1 = tab + d.o_tab, *t2 = t1 + 2 * np;
        const double *d1 = W + d.o_w, *d2 = d1 + d.N + 1;
        for (int i = tid; i < np; i += T) {
            rt[2 * i] = t1[i];
            rt[2 * i + 1] = t2[i];
            ct[2 * i] = t1[np + i];
            ct[2 * i + 1] = t2[np + i];
        }
        for (int i = tid; i < L; i += T) {
            wt[2 * i] = d1[i];
            wt[2 * i + 1] = d2[i];
        }
        for (int j = 0; j < np; ++j) Y[(size_t)j * T + tid] = 0.0;
        for (int j = 0; j < L; ++j) R[(size_t)j * T + tid] = 0.0;
        __syncthreads();

        Fp2sParams P;
        P.a = d.a;
        P.tau = d.tau;
        P.inv_tau = d.inv_tau;
        P.N = d.N < step_cap ? d.N : step_cap;
        P.nmodes = d.nmodes;
        P.scheme = d.scheme;
        P.form = CQ_FAST;
        P.np = np;
        P.L = L;
        P.prec = CQ_F64;
        const int64_t mode_raw = (int64_t)un.first_mode + (tid >> 5) * kFastModesPerWarp + (lane & 15);
        const bool active = mode_raw < d.nmodes && mode_raw < (int64_t)un.first_mode + modes_per_unit;
        const int64_t mode = active ? mode_raw : un.first_mode;
        const double *rs = rt + st, *cs = ct + st, *ws = wt + st;
        const double *dn = st ? d2 : d1;
        double *Yc = Y + tid, *Rc = R + tid;
        const double *g0 = modal + d.o_modal;
        double *gN = modal + d.o_modal + 2 * d.nmodes;
        const double gz = g0[st * d.nmodes + mode];
        const double d_s0 = ws[0], d_o0 = wt[1 - st];
        ModeConst mc;
        const bool ok = mode_setup(P, lamp[d.o_lam + mode], st ? d_o0 : d_s0, st ? d_s0 : d_o0, mc);
        if (active && st == 0 && !ok) atomicOr(status, ST_SINGULAR);
        const double mn_oo = st ? mc.Mn.i22 : mc.Mn.i11, mn_ot = st ? mc.Mn.i21 : mc.Mn.i12;
        const double m1_oo = st ? mc.M1.i22 : mc.M1.i11, m1_ot = st ? mc.M1.i21 : mc.M1.i12;
        const double a = P.a, c = mc.c;
        double gm1 = gz, gm2 = 0.0;
        int slot = 0;
        for (int64_t n = 1; n <= P.N; ++n) {
            slot = (slot + 1 == L) ? 0 : slot + 1;
            double hp[NU];
#pragma unroll
            for (int u = 0; u < NU; ++u) hp[u] = 0.0;
            if (n - L >= 1) {
                const double in = Rc[(size_t)slot * T];
                int j = 0;
                for (; j + NU <= np; j += NU) {
                    double y[NU];
#pragma unroll
                    for (int u = 0; u < NU; ++u) y[u] = fma(rs[2 * (j + u)], Yc[(size_t)(j + u) * T], in);
#pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        Yc[(size_t)(j + u) * T] = y[u];
                        hp[u] = fma(cs[2 * (j + u)], y[u], hp[u]);
                    }
                }
                for (; j < np; ++j) {
                    const double y = fma(rs[2 * j], Yc[(size_t)j * T], in);
                    Yc[(size_t)j * T] = y;
                    hp[0] = fma(cs[2 * j], y, hp[0]);
                }
            }
            const int imax = (int)min((int64_t)(L - 1), n - 1);
            int sl = slot;
            for (int i = 1; i <= imax; ++i) {
                sl = (sl == 0) ? L - 1 : sl - 1;
                if (i & 1) hp[1] = fma(ws[2 * i], Rc[(size_t)sl * T], hp[1]);
                else hp[NU > 2 ? 2 : 0] = fma(ws[2 * i], Rc[(size_t)sl * T], hp[NU > 2 ? 2 : 0]);
            }
            double h = 0.0;
#pragma unroll
            for (int w = 1; w < NU; w *= 2)
#pragma unroll
                for (int u = 0; u + w < NU; u += 2 * w) hp[u] += hp[u + w];
            h = hp[0];
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
            gm2 = gm1;
            gm1 = x;
        }
        if (active) {
            gN[st * d.nmodes + mode] = gm1;
            if (!isfinite(gm1)) atomicOr(status, ST_NONFINITE);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Double-float batches (every instance CQ_DF64): the per-lane solve of the single-problem
// double-float kernel (fastdf.cuh) over work units of 64 modes, taken from the same atomic
// counter. Tables per instance in double-float (ranked nodes, u form for the slowest quarter)
// are built once by the plan; a unit copies its instance's table into shared memory and
// dispatches on its node class and scheme.
// ---------------------------------------------------------------------------
__global__ void k_b_df_tables(const InstDesc *__restrict__ D, const double *__restrict__ W,
                              const double *__restrict__ tab, float *__restrict__ dftab) {
    const InstDesc d = D[blockIdx.x];
    const double *t1 = tab + d.o_tab, *t2 = t1 + 2 * d.np, *d1 = W + d.o_w, *d2 = d1 + d.N + 1;
    df_tables_fill(df_np_class(d.np), d.np, d.L, d.N, t1, t2, d1, d2, dftab + (size_t)blockIdx.x * kDfTabFloats,
                   threadIdx.x, blockDim.x);
}

template <int WL>
__global__ void __launch_bounds__(kDfThreads, kDfMinBlocks)
    k_b_df(const InstDesc *__restrict__ D, const Unit *__restrict__ U, int n_units, int *__restrict__ counter,
           int maxL, int maxKS, int64_t step_cap, const double *__restrict__ W, const float *__restrict__ dftab,
           const double *__restrict__ lamp, double *__restrict__ modal, int *__restrict__ status) {
    extern __shared__ __align__(16) float smd[];
    __shared__ int s_unit;
    const int T = blockDim.x, tid = threadIdx.x;
    float2 *R = reinterpret_cast<float2 *>(smd + kDfTabFloats);      // [maxL][T]
    float2 *Ys = R + (size_t)maxL * T;                                // [maxKS][T]
    const int modes_per_unit = (T >> 5) * kFastModesPerWarp;
    for (;;) {
        if (tid == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= n_units) break;
        const Unit un = U[u];
        const InstDesc d = D[un.inst];
        const int NP = df_np_class(d.np);
        const float *src = dftab + (size_t)un.inst * kDfTabFloats;
        for (int e = tid; e < df_table_floats(NP); e += T) smd[e] = src[e];
        for (int j = 0; j < d.L; ++j) R[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
        for (int j = 0; j < df_smem_slots(NP); ++j) Ys[(size_t)j * T + tid] = make_float2(0.0f, 0.0f);
        __syncthreads();
        Fp2sParams P;
        P.a = d.a;
        P.tau = d.tau;
        P.inv_tau = d.inv_tau;
        P.N = d.N < step_cap ? d.N : step_cap;
        P.nmodes = d.nmodes;
        P.scheme = d.scheme;
        P.form = CQ_FAST;
        P.np = d.np;
        P.L = d.L;
        P.prec = CQ_DF64;
        const double *lam = lamp + d.o_lam, *d1 = W + d.o_w, *d2 = d1 + d.N + 1;
        const double *g0 = modal + d.o_modal;
        double *gN = modal + d.o_modal + 2 * d.nmodes;
        const int64_t mode_raw = (int64_t)un.first_mode + (tid >> 5) * kFastModesPerWarp + (tid & 15);
        const int64_t mode_end = min(d.nmodes, (int64_t)un.first_mode + modes_per_unit);
        const float4 *tb = reinterpret_cast<const float4 *>(smd);
        const float2 *wd = reinterpret_cast<const float2 *>(smd + 8 * NP);
#define CQ_B_DF(NPV)                                                                                            \
    case NPV:                                                                                                   \
        if (d.scheme == CQ_BE)                                                                                  \
            df_solve_lane<NPV, true, 2>(P, lam, g0, gN, status, d1, d2, tb, wd, R, Ys, T, tid, mode_raw, mode_end); \
        else                                                                                                    \
            df_solve_lane<NPV, false, WL>(P, lam, g0, gN, status, d1, d2, tb, wd, R, Ys, T, tid, mode_raw, mode_end); \
        break;
        switch (NP) {
            CQ_B_DF(16)
            CQ_B_DF(32)
            CQ_B_DF(48)
            CQ_B_DF(64)
            CQ_B_DF(80)
            CQ_B_DF(96)
            CQ_B_DF(112)
            CQ_B_DF(128)
            default: break;
        }
#undef CQ_B_DF
        __syncthreads();
    }
}

static size_t bdf_smem(int maxL, int maxKS) {
    return (size_t)kDfTabFloats * sizeof(float) + (size_t)(maxL + maxKS) * kDfThreads * sizeof(float2);
}

static size_t bfast_smem(int maxnp, int maxL, int T) {
    return ((size_t)4 * maxnp + 2 * kMaxNs + (size_t)(maxnp + maxL) * T) * sizeof(double);
}

static int validate(const fp2s_problem_t &p, InstDesc &d) {
    if (!(p.alpha1 > 0.0 && p.alpha1 < 1.0 && p.alpha2 > 0.0 && p.alpha2 < 1.0)) return CQ_EINVAL;
    if (!(p.m >= 0.0 && p.m < 1.0) || p.m == 0.5) return CQ_EINVAL;
    if (!(p.T > 0.0) || p.N < 1 || p.N > kMaxWeights) return CQ_EINVAL;
    if (p.dim != 1 && p.dim != 2) return CQ_EINVAL;
    if (p.M < 1 || p.M > (p.dim == 1 ? (1 << 16) : 4096)) return CQ_EINVAL;
    if (p.scheme != CQ_BE && p.scheme != CQ_BDF2) return CQ_EINVAL;
    if (p.form != CQ_FAST || (p.prec != CQ_F64 && p.prec != CQ_DF64)) return CQ_EUNSUPPORTED;
    const int np1 = p.fast.np1, np2 = (p.scheme == CQ_BE) ? 0 : p.fast.np2;
    const int L = (p.scheme == CQ_BE) ? 2 : p.fast.ns;
    if (np1 < 1 || np2 < 0 || np1 + np2 > kMaxNp) return CQ_EINVAL;
    if (p.scheme == CQ_BDF2 && (np2 < 1 || L < 3 || L > kMaxNs)) return CQ_EINVAL;
    if (p.prec == CQ_DF64 && df_np_class(np1 + np2) == 0) return CQ_EUNSUPPORTED;
    d = InstDesc{};
    d.a = (1.0 - p.m) / (2.0 * p.m - 1.0);
    d.tau = p.T / (double)p.N;
    d.inv_tau = 1.0 / d.tau;
    d.beta1 = 1.0 - p.alpha1;
    d.beta2 = 1.0 - p.alpha2;
    d.N = p.N;
    d.nmodes = (p.dim == 1) ? p.M : (int64_t)p.M * p.M;
    d.scheme = p.scheme;
    d.np1 = np1;
    d.np2 = np2;
    d.np = np1 + np2;
    d.L = L;
    d.M = p.M;
    d.dim = p.dim;
    return CQ_OK;
}

static void make_units(const std::vector<InstDesc> &descs, int wb, std::vector<Unit> &units) {
    const int mpu = wb * kFastModesPerWarp;
    std::vector<std::pair<double, Unit>> tmp;
    for (int i = 0; i < (int)descs.size(); ++i) {
        const InstDesc &d = descs[i];
        for (int64_t m0 = 0; m0 < d.nmodes; m0 += mpu) {
            const int64_t cnt = std::min<int64_t>(mpu, d.nmodes - m0);
            const double cost = (double)d.N * (double)(d.np + d.L + 8) * (double)((cnt + 15) / 16);
            tmp.push_back({cost, Unit{i, (int)m0}});
        }
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const std::pair<double, Unit> &x, const std::pair<double, Unit> &y) {
        return x.first > y.first;
    });
    units.clear();
    for (auto &t : tmp) units.push_back(t.second);
}

static int num_sms_b() { return device_sms(); }

// The persistent kernel for a node-loop width (2, 4 or 8 partial sums; 0 = the default 4).
using BFastKernel = void (*)(const InstDesc *, const Unit *, int, int *, int, int, int64_t, const double *,
                             const double *, const double *, double *, int *);
static BFastKernel bfast_kernel(int node_unroll) {
    if (node_unroll == 2) return k_b_fast<2>;
    if (node_unroll == 8) return k_b_fast<8>;
    return k_b_fast<4>;
}

// Resident CTAs per SM of the persistent kernel for a block width (0 when it does not fit).
static int occupancy(int max_np, int max_L, int wb, int node_unroll) {
    const int T = 32 * wb;
    const size_t smem = bfast_smem(max_np, max_L, T);
    const BFastKernel k = bfast_kernel(node_unroll);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, smem) != cudaSuccess) return 0;
    return per_sm;
}

// Double-float batch: one persistent launch with every CTA that fits per SM.
static int launch_df_batch(const fp2s_batch_t *plan, const BatchLayout &l, int64_t step_cap, cudaStream_t s) {
    const int maxKS = df_smem_slots(df_np_class(plan->max_np));
    const size_t smem = bdf_smem(plan->max_L, maxKS);
    auto kern = plan->max_L <= 17 ? k_b_df<17> : k_b_df<kMaxNs>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return CQ_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDfThreads, smem) != cudaSuccess || per_sm < 1)
        return CQ_EUNSUPPORTED;
    const int blocks = (int)std::min<int64_t>((int64_t)num_sms_b() * per_sm, plan->n_units);
    int st = cuda_status(cudaMemsetAsync(l.counter, 0, sizeof(int), s));
    if (st) return st;
    kern<<<blocks, kDfThreads, smem, s>>>(l.desc, l.units, plan->n_units, l.counter, plan->max_L, maxKS, step_cap,
                                          l.W, l.dftab, l.lam, l.modal, l.status);
    return launched();
}

// One persistent launch: plan->ctas_per_sm CTAs per SM (0: as many as fit), never more than units.
static int launch_main(const fp2s_batch_t *plan, const BatchLayout &l, int64_t step_cap, cudaStream_t s) {
    if (plan->flags & 2) return launch_df_batch(plan, l, step_cap, s);
    const int T = 32 * plan->warps_per_block;
    const size_t smem = bfast_smem(plan->max_np, plan->max_L, T);
    const int fit = occupancy(plan->max_np, plan->max_L, plan->warps_per_block, plan->node_unroll);
    if (fit < 1) return CQ_EUNSUPPORTED;
    const int per_sm = plan->ctas_per_sm > 0 ? std::min(plan->ctas_per_sm, fit) : fit;
    const int64_t want = (int64_t)num_sms_b() * per_sm;
    const int blocks = (int)std::min<int64_t>(want, plan->n_units);
    int st = cuda_status(cudaMemsetAsync(l.counter, 0, sizeof(int), s));
    if (st) return st;
    bfast_kernel(plan->node_unroll)<<<blocks, T, smem, s>>>(l.desc, l.units, plan->n_units, l.counter, plan->max_np,
                                                           plan->max_L, step_cap, l.W, l.tab, l.lam, l.modal,
                                                           l.status);
    return launched();
}

// CUDA events of the autotuner, destroyed on every path out of it.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok() {
        return cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    }
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

static int transform(const fp2s_batch_t *plan, const BatchLayout &l, const double *field_in, double *field_out, int src,
                     int dst, cudaStream_t s) {
    const unsigned gx = (unsigned)((2 * plan->max_modes + 255) / 256);
    const dim3 grid(gx, (unsigned)plan->n_inst);
    k_b_dst_pass<<<grid, 256, 0, s>>>(l.desc, l.S, field_in, field_out, l.modal, 1, src, dst);
    k_b_dst_pass<<<grid, 256, 0, s>>>(l.desc, l.S, field_in, field_out, l.modal, 2, src, dst);
    return launched(2);
}

static BatchSizes sizes_of(const std::vector<InstDesc> &descs) {
    BatchSizes z;
    for (const InstDesc &d : descs) {
        z.w += 2 * (d.N + 1);
        z.tab += 4 * d.np;
        z.scr += 4 * d.np;
        z.lam += d.nmodes;
        z.S += (int64_t)d.M * d.M;
        z.modal += 6 * d.nmodes;
        z.field += 2 * d.nmodes;
        z.maxnp = std::max(z.maxnp, d.np);
        z.maxL = std::max(z.maxL, d.L);
        z.maxM = std::max(z.maxM, d.M);
        z.maxN = std::max(z.maxN, d.N);
        z.max_nmodes = std::max(z.max_nmodes, d.nmodes);
    }
    return z;
}

}  // namespace fastcq

using namespace fastcq;

extern "C" int fp2s_batch_plan(const fp2s_problem_t *probs, int32_t n, int32_t tune, fp2s_batch_t *plan,
                               void *ws_dev, size_t *ws_bytes, void *stream) {
    if (!probs || n < 1 || !plan || !ws_bytes) return CQ_EINVAL;
    if (n > kMaxBatch) return CQ_EUNSUPPORTED;
    std::vector<InstDesc> descs(n);
    for (int i = 0; i < n; ++i) {
        const int st = validate(probs[i], descs[i]);
        if (st) return st;
        if (probs[i].prec != probs[0].prec) return CQ_EUNSUPPORTED;      // one precision per batch
    }
    const bool df = probs[0].prec == CQ_DF64;
    // offsets
    int64_t ow = 0, otab = 0, oscr = 0, olam = 0, oS = 0, omod = 0, ofield = 0;
    for (InstDesc &d : descs) {
        d.o_w = ow;
        ow += 2 * (d.N + 1);
        d.o_tab = otab;
        otab += 4 * d.np;
        d.o_scr = oscr;
        oscr += 4 * d.np;
        d.o_lam = olam;
        olam += d.nmodes;
        d.o_S = oS;
        oS += (int64_t)d.M * d.M;
        d.o_modal = omod;
        omod += 6 * d.nmodes;
        d.o_field = ofield;
        ofield += 2 * d.nmodes;
    }
    BatchSizes z = sizes_of(descs);
    if (df) z.dftab = (int64_t)n * kDfTabFloats;
    // block widths that fit shared memory; the largest is the default (double-float batches:
    // the fixed width of their kernel)
    std::vector<int> cands;
    if (df) cands.push_back(kDfThreads / 32);
    else
        for (int wb = 16; wb >= 1; --wb)
            if (bfast_smem(z.maxnp, z.maxL, 32 * wb) <= 227 * 1024) cands.push_back(wb);
    if (cands.empty()) return CQ_EUNSUPPORTED;
    // the unit list is largest for the smallest width: size the workspace for it
    std::vector<Unit> units_max;
    make_units(descs, cands.back(), units_max);
    int64_t off[R_END + 1];
    BatchLayout l = batch_layout(ws_dev, n, (int64_t)units_max.size(), z, off);
    if (!ws_dev) { *ws_bytes = l.bytes; return CQ_OK; }
    if (*ws_bytes < l.bytes || ((uintptr_t)ws_dev & 255)) return CQ_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    plan->n_inst = n;
    plan->max_np = z.maxnp;
    plan->max_L = z.maxL;
    plan->max_N = (int32_t)z.maxN;
    plan->max_M = z.maxM;
    plan->max_modes = z.max_nmodes;
    plan->field_elems = z.field;
    plan->ws_bytes = (int64_t)l.bytes;
    plan->flags = df ? 2 : 0;
    for (int r = 0; r <= R_END; ++r) plan->off[r] = off[r];
    int st;
    if ((st = cuda_status(cudaMemcpyAsync(l.desc, descs.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice, s))))
        return st;
    if ((st = cuda_status(cudaMemsetAsync(l.status, 0, 64 * sizeof(int), s)))) return st;
    if ((st = cuda_status(cudaMemsetAsync(l.modal, 0, z.modal * sizeof(double), s)))) return st;
    // tables for the whole batch
    static unsigned long long attr = 0;
    if ((st = smem_attr_once((const void *)k_b_weights, (int)((kMaxWeights + 1) * sizeof(double)), &attr)))
        return st;
    k_b_weights<<<dim3(n, 2), kWThreads, (z.maxN + 1) * sizeof(double), s>>>(l.desc, l.W);
    k_b_gauss_jacobi<<<dim3(n, 4, (kMaxNp + kGJThreads - 1) / kGJThreads), kGJThreads, 0, s>>>(l.desc, l.scr);
    k_b_coeffs<<<dim3(n, 2), 256, 0, s>>>(l.desc, l.scr, l.tab);
    const int64_t spec = std::max<int64_t>(z.max_nmodes, (int64_t)z.maxM * z.maxM);
    k_b_spectrum<<<dim3((unsigned)((spec + 255) / 256), n), 256, 0, s>>>(l.desc, l.lam, l.S);
    if ((st = launched(4))) return st;
    if (df) {
        k_b_df_tables<<<n, 256, 0, s>>>(l.desc, l.W, l.tab, l.dftab);
        if ((st = launched())) return st;
    }
    // launch shape: the widest block with full occupancy and 4 partial sums by default, or the
    // fastest candidate (block width x resident CTAs per SM x node-loop width) on a shortened
    // run, median of three timings each
    int best = cands.front(), best_cps = 0, best_nu = 4;
    plan->tuned_candidates = 0;
    plan->node_unroll = 4;
    if (df) {
        best_nu = 0;                         // the double-float kernel has no tuned knob
    } else if (tune) {
        EventPair ev;
        if (!ev.ok()) return CQ_ECUDA;
        float best_ms = 1e30f;
        const int64_t cap = std::min<int64_t>(z.maxN, 96);
        for (int wb : cands) {
            if (wb < 2) continue;
            std::vector<Unit> units;
            make_units(descs, wb, units);
            plan->warps_per_block = wb;
            plan->n_units = (int32_t)units.size();
            if ((st = cuda_status(cudaMemcpyAsync(l.units, units.data(), units.size() * sizeof(Unit),
                                                  cudaMemcpyHostToDevice, s))))
                return st;
            for (int nu : {4, 2, 8}) {
                const int fit = occupancy(z.maxnp, z.maxL, wb, nu);
                if (fit < 1) continue;
                plan->node_unroll = nu;
                for (int cps : {fit, fit / 2}) {
                    if (cps < 1 || (cps == fit / 2 && fit / 2 == fit)) continue;
                    plan->ctas_per_sm = cps;
                    if ((st = launch_main(plan, l, cap, s))) return st;        // warm-up
                    float t[3];
                    for (float &ti : t) {
                        cudaEventRecord(ev.a, s);
                        if ((st = launch_main(plan, l, cap, s))) return st;
                        cudaEventRecord(ev.b, s);
                        if (cudaEventSynchronize(ev.b) != cudaSuccess) return CQ_ECUDA;
                        if (cudaEventElapsedTime(&ti, ev.a, ev.b) != cudaSuccess) return CQ_ECUDA;
                    }
                    std::sort(t, t + 3);
                    ++plan->tuned_candidates;
                    if (t[1] < best_ms * 0.98f) {
                        best_ms = t[1];
                        best = wb;
                        best_cps = cps == fit ? 0 : cps;
                        best_nu = nu;
                    }
                }
            }
        }
        plan->flags |= 1;
    }
    plan->node_unroll = best_nu;
    plan->ctas_per_sm = best_cps;
    std::vector<Unit> units;
    make_units(descs, best, units);
    plan->warps_per_block = best;
    plan->n_units = (int32_t)units.size();
    if ((st = cuda_status(cudaMemcpyAsync(l.units, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice,
                                          s))))
        return st;
    if ((st = cuda_status(cudaMemsetAsync(l.status, 0, 64 * sizeof(int), s)))) return st;
    return cudaStreamSynchronize(s) == cudaSuccess ? CQ_OK : CQ_ECUDA;   // host vectors go out of scope
}

extern "C" int fp2s_solve_batched(const fp2s_batch_t *plan, const double *G0_dev, double *GN_dev, void *ws_dev,
                                  void *stream) {
    if (!plan || !G0_dev || !GN_dev || !ws_dev || plan->n_inst < 1 || plan->n_units < 1 || plan->warps_per_block < 1)
        return CQ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const BatchLayout l = layout_from_plan(plan, ws_dev);
    int st;
    if ((st = transform(plan, l, G0_dev, nullptr, 0, 1, s))) return st;          // G0 -> modal g0
    if ((st = timing_begin(s))) return st;
    if ((st = launch_main(plan, l, INT64_MAX, s))) return st;
    if ((st = timing_end(s))) return st;
    return transform(plan, l, nullptr, GN_dev, 2, 0, s);                           // modal gN -> GN
}

extern "C" int fp2s_batch_status(const fp2s_batch_t *plan, const void *ws_dev, void *stream) {
    if (!plan || !ws_dev) return CQ_EINVAL;
    const BatchLayout l = layout_from_plan(plan, const_cast<void *>(ws_dev));
    int h = 0;
    if (cudaMemcpyAsync(&h, l.status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
        return CQ_ECUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CQ_ECUDA;
    if (h & ST_SINGULAR) return CQ_ESINGULAR;
    if (h & ST_NONFINITE) return CQ_ENONFINITE;
    return CQ_OK;
}
