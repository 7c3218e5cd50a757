// History sums over all DOFs: the direct strictly-lower-triangular Toeplitz
// product (Eq. 3.8) and one step of the fast recurrences (Eqs. 3.9-3.10,
// 3.17-3.18). FP64, FP32 and double-float (FP64-class on the FP32 pipe).
#include <mutex>

#include "common.cuh"
#include "fastdf.cuh"

namespace fastcq {

// ---------------------------------------------------------------------------
// Direct history. Block (x: DOF tile, y: block of BT consecutive output steps).
// Each thread owns VEC adjacent DOFs and BT outputs n0..n0+BT-1; it streams the
// levels k = 1..n_last-1 once and keeps the BT weights d_{n0+b-k} in a register
// window that shifts by one per level, so every level load feeds BT*VEC FMAs.
// dz[i + BT] = d_i for i >= 1 and 0 for i <= 0 (this drops d_0 and the
// non-causal terms).
// ---------------------------------------------------------------------------
template <int BT, int VEC>
__global__ void __launch_bounds__(128) k_history_direct(int64_t ndof, int64_t n_lo, int64_t n_hi,
                                                        const double *__restrict__ dz,
                                                        const double *__restrict__ G, int64_t ldg,
                                                        double *__restrict__ H, int64_t ldh) {
    const int64_t dof = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VEC;
    if (dof >= ndof) return;
    const int64_t n0 = n_lo + (int64_t)blockIdx.y * BT;
    const int64_t n_last = min(n0 + BT - 1, n_hi - 1);
    double acc[BT][VEC];
    double w[BT];
#pragma unroll
    for (int b = 0; b < BT; ++b) {
        w[b] = __ldg(dz + (n0 + b - 1) + BT);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[b][v] = 0.0;
    }
    const bool full = (dof + VEC <= ndof);
    for (int64_t k = 1; k <= n_last - 1; ++k) {
        double g[VEC];
        const double *src = G + k * ldg + dof;
        if (VEC == 2 && full) {
            const double2 t = __ldg(reinterpret_cast<const double2 *>(src));
            g[0] = t.x;
            g[VEC - 1] = t.y;
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) g[v] = (dof + v < ndof) ? __ldg(src + v) : 0.0;
        }
#pragma unroll
        for (int b = 0; b < BT; ++b)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[b][v] = fma(w[b], g[v], acc[b][v]);
#pragma unroll
        for (int b = BT - 1; b > 0; --b) w[b] = w[b - 1];
        w[0] = __ldg(dz + (n0 - k - 1) + BT);
    }
#pragma unroll
    for (int b = 0; b < BT; ++b) {
        const int64_t n = n0 + b;
        if (n >= n_hi) break;
        double *dst = H + (n - n_lo) * ldh + dof;
        if (VEC == 2 && full) {
            *reinterpret_cast<double2 *>(dst) = make_double2(acc[b][0], acc[b][VEC - 1]);
        } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                if (dof + v < ndof) dst[v] = acc[b][v];
        }
    }
}

constexpr int kDirectBT = 16;

// Writes the zero-padded weight vector dz (see k_history_direct): entries
// 0 .. n + 2*kDirectBT, i.e. every index a tail block may touch.
__global__ void k_pad_weights(const double *__restrict__ d, int64_t n, double *__restrict__ dz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n + 2 * kDirectBT) return;
    const int64_t idx = i - kDirectBT;        // weight index
    dz[i] = (idx >= 1 && idx <= n) ? d[idx] : 0.0;
}

// ---------------------------------------------------------------------------
// Fast history, one step, for every DOF (2 DOFs per thread).
// State Y[j][dof] (Ghist_j = c_j Y_j), ring[L][dof] with level k in slot k % L.
// At step n: levels n-2..n-L are in the ring, level n-1 comes from G_prev.
//   Y_j <- r_j Y_j + G^{n-L}               (only when n - L >= 1; G^0 is left out)
//   h^n = sum_{i=1}^{min(L-1,n-1)} d_i G^{n-i} + sum_j c_j Y_j
// then G^{n-1} is stored in slot (n-1) % L, which held level n-1-L.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_history_fast_step(int64_t ndof, int64_t n, int L, int np, int vec,
                                                          const double *__restrict__ tab,
                                                          double *__restrict__ ring, double *__restrict__ Y,
                                                          const double *__restrict__ G_prev,
                                                          double *__restrict__ H) {
    // two DOFs per thread; rows are moved as 16-byte pairs when vec (ndof even, so the
    // workspace rows stay 16-byte aligned, and G_prev, H 16-byte aligned), else element by element
    __shared__ double r[kMaxNp], c[kMaxNp], d[kMaxNs];
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        r[i] = tab[i];
        c[i] = tab[np + i];
    }
    for (int i = threadIdx.x; i < L; i += blockDim.x) d[i] = tab[2 * np + i];
    __syncthreads();
    const int64_t dof = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (dof >= ndof) return;
    const bool pair = dof + 1 < ndof;
    auto ld2 = [&](const double *p) -> double2 {
        if (vec) return *reinterpret_cast<const double2 *>(p);
        return make_double2(p[0], pair ? p[1] : 0.0);
    };
    auto st2 = [&](double *p, double2 v) {
        if (vec) *reinterpret_cast<double2 *>(p) = v;
        else {
            p[0] = v.x;
            if (pair) p[1] = v.y;
        }
    };
    double h0 = 0.0, h1 = 0.0;
    double2 gp = make_double2(0.0, 0.0);
    if (n >= 2) {
        gp = ld2(G_prev + dof);
        h0 = d[1] * gp.x;
        h1 = d[1] * gp.y;
        const int64_t imax = min((int64_t)L - 1, n - 1);
        for (int i = 2; i <= imax; ++i) {
            const double2 g = ld2(ring + (int64_t)((n - i) % L) * ndof + dof);
            h0 = fma(d[i], g.x, h0);
            h1 = fma(d[i], g.y, h1);
        }
    }
    if (n - L >= 1) {
        const double2 gin = ld2(ring + (int64_t)((n - L) % L) * ndof + dof);
        double *y = Y + dof;
        for (int j = 0; j < np; ++j, y += ndof) {
            double2 v = ld2(y);
            v.x = fma(r[j], v.x, gin.x);
            v.y = fma(r[j], v.y, gin.y);
            st2(y, v);
            h0 = fma(c[j], v.x, h0);
            h1 = fma(c[j], v.y, h1);
        }
    }
    if (n >= 2) st2(ring + (int64_t)((n - 1) % L) * ndof + dof, gp);
    st2(H + dof, make_double2(h0, h1));
}

// ---------------------------------------------------------------------------
// Fast history, one step, FP32 precision form, streaming from HBM: the state
// Y[j][dof] and the last L levels ring[slot][dof] are FP32 rows with a pitch
// rounded up to 4 floats, so every thread moves 4 DOFs with 16-byte loads and
// stores (a warp touches 512 contiguous bytes per row). The tables (r_j, c_j,
// d_i) are FP32 in shared memory; inputs G^{n-1} and outputs h^n stay FP64.
// Per DOF-step the traffic is 8 np (state) + 4 L (window and recurrence input)
// + 4 (ring store) + 8 (G^{n-1}) + 8 (h^n) bytes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_history_fast_step_f32(int64_t ndof, int64_t pitch, int64_t n, int L,
                                                               int np, const float *__restrict__ tabf,
                                                               float *__restrict__ ring, float *__restrict__ Y,
                                                               const double *__restrict__ G_prev,
                                                               double *__restrict__ H) {
    __shared__ float r[kMaxNp], c[kMaxNp], d[kMaxNs];
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        r[i] = tabf[i];
        c[i] = tabf[np + i];
    }
    for (int i = threadIdx.x; i < L; i += blockDim.x) d[i] = tabf[2 * np + i];
    __syncthreads();
    const int64_t dof = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (dof >= ndof) return;
    const int cnt = (int)min((int64_t)4, ndof - dof);
    float4 gp = make_float4(0.f, 0.f, 0.f, 0.f);
    float h[4] = {0.f, 0.f, 0.f, 0.f};
    if (n >= 2) {
        float g[4] = {0.f, 0.f, 0.f, 0.f};
        for (int v = 0; v < cnt; ++v) g[v] = (float)G_prev[dof + v];
        gp = make_float4(g[0], g[1], g[2], g[3]);
        h[0] = d[1] * gp.x;
        h[1] = d[1] * gp.y;
        h[2] = d[1] * gp.z;
        h[3] = d[1] * gp.w;
        const int64_t imax = min((int64_t)L - 1, n - 1);
        for (int i = 2; i <= imax; ++i) {
            const float4 x = *reinterpret_cast<const float4 *>(ring + (int64_t)((n - i) % L) * pitch + dof);
            h[0] = fmaf(d[i], x.x, h[0]);
            h[1] = fmaf(d[i], x.y, h[1]);
            h[2] = fmaf(d[i], x.z, h[2]);
            h[3] = fmaf(d[i], x.w, h[3]);
        }
    }
    if (n - L >= 1) {
        const float4 in = *reinterpret_cast<const float4 *>(ring + (int64_t)((n - L) % L) * pitch + dof);
        float4 *yp = reinterpret_cast<float4 *>(Y + dof);
        const int64_t step = pitch / 4;
        constexpr int B = 8;                       // rows in flight per thread
        for (int j0 = 0; j0 < np; j0 += B) {
            float4 y[B];
#pragma unroll
            for (int k = 0; k < B; ++k)
                if (j0 + k < np) y[k] = yp[(int64_t)(j0 + k) * step];
#pragma unroll
            for (int k = 0; k < B; ++k) {
                if (j0 + k >= np) break;
                const float rj = r[j0 + k], cj = c[j0 + k];
                y[k].x = fmaf(rj, y[k].x, in.x);
                y[k].y = fmaf(rj, y[k].y, in.y);
                y[k].z = fmaf(rj, y[k].z, in.z);
                y[k].w = fmaf(rj, y[k].w, in.w);
                h[0] = fmaf(cj, y[k].x, h[0]);
                h[1] = fmaf(cj, y[k].y, h[1]);
                h[2] = fmaf(cj, y[k].z, h[2]);
                h[3] = fmaf(cj, y[k].w, h[3]);
            }
#pragma unroll
            for (int k = 0; k < B; ++k)
                if (j0 + k < np) yp[(int64_t)(j0 + k) * step] = y[k];
        }
    }
    if (n >= 2) *reinterpret_cast<float4 *>(ring + (int64_t)((n - 1) % L) * pitch + dof) = gp;
    for (int v = 0; v < cnt; ++v) H[dof + v] = (double)h[v];
}

// ---------------------------------------------------------------------------
// Fast history, one step, double-float form (CQ_DF64): the state Y[j][dof] and the last L
// levels ring[slot][dof] are hi + lo pairs of FP32 numbers (8 bytes per DOF, as in FP64),
// rows with an even pitch so that a thread moves its 2 DOFs with one 16-byte access; the node
// update and the sums are error-free FP32 sequences (fastdf.cuh). The table holds the nodes
// with r_j <= 1/2 first (entry (r_hi, r_lo, c_hi, c_lo)), then the others with u_j = 1 - r_j in
// place of r_j (their update runs as Y - u Y + G, which keeps the relative accuracy of 1 - r for
// ratios near 1); the state rows follow that order. Rows are moved DF_ROWS at a time so that
// several loads are in flight per thread. G^{n-1} comes in and h^n goes out in FP64. Per
// DOF-step the traffic is that of the FP64 kernel, 16 np + 8 L + 16 bytes, but the arithmetic
// runs on the FP32 pipe: the step is bound by HBM rather than by the FP64 pipe.
// ---------------------------------------------------------------------------
constexpr int kDfRows = 4;

template <bool U>
__device__ __forceinline__ void df_step_rows(const float4 *t, int j0, int j1, const float4 gin, float2 *Y,
                                             int64_t pitch, int64_t dof, float &h0, float &l0, float &h1, float &l1) {
    for (int j = j0; j < j1; j += kDfRows) {
        float4 v[kDfRows];
#pragma unroll
        for (int k = 0; k < kDfRows; ++k)
            if (j + k < j1) v[k] = *reinterpret_cast<const float4 *>(Y + (int64_t)(j + k) * pitch + dof);
#pragma unroll
        for (int k = 0; k < kDfRows; ++k) {
            if (j + k >= j1) break;
            const float4 tj = t[j + k];
            if (U) {
                node_u(tj.x, tj.y, gin.x, gin.y, v[k].x, v[k].y);
                node_u(tj.x, tj.y, gin.z, gin.w, v[k].z, v[k].w);
            } else {
                node_r(tj.x, tj.y, gin.x, gin.y, v[k].x, v[k].y);
                node_r(tj.x, tj.y, gin.z, gin.w, v[k].z, v[k].w);
            }
            acc_prod(tj.z, tj.w, v[k].x, v[k].y, h0, l0);
            acc_prod(tj.z, tj.w, v[k].z, v[k].w, h1, l1);
        }
#pragma unroll
        for (int k = 0; k < kDfRows; ++k)
            if (j + k < j1) *reinterpret_cast<float4 *>(Y + (int64_t)(j + k) * pitch + dof) = v[k];
    }
}

__global__ void __launch_bounds__(64) k_history_fast_step_df(int64_t ndof, int64_t pitch, int64_t n, int L, int np,
                                                             const float4 *__restrict__ tabdf,
                                                             const float2 *__restrict__ wdf,
                                                             const int *__restrict__ nr_dev,
                                                             float2 *__restrict__ ring, float2 *__restrict__ Y,
                                                             const double *__restrict__ G_prev,
                                                             double *__restrict__ H) {
    __shared__ float4 t[kMaxNp];
    __shared__ float2 w[kMaxNs];
    for (int i = threadIdx.x; i < np; i += blockDim.x) t[i] = tabdf[i];
    for (int i = threadIdx.x; i < L; i += blockDim.x) w[i] = wdf[i];
    __syncthreads();
    const int nr = *nr_dev;                    // nodes of the r form (the first nr rows)
    const int64_t dof = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (dof >= ndof) return;
    const bool pair = dof + 1 < ndof;
    float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
    float4 gp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    auto row = [&](float2 *base, int64_t r) { return reinterpret_cast<float4 *>(base + r * pitch + dof); };
    if (n >= 2) {
        const float2 a = df_of(G_prev[dof]), b = pair ? df_of(G_prev[dof + 1]) : make_float2(0.0f, 0.0f);
        gp = make_float4(a.x, a.y, b.x, b.y);
        acc_prod(w[1].x, w[1].y, gp.x, gp.y, h0, l0);
        acc_prod(w[1].x, w[1].y, gp.z, gp.w, h1, l1);
        const int64_t imax = min((int64_t)L - 1, n - 1);
        for (int i = 2; i <= imax; ++i) {
            const float4 x = *row(ring, (n - i) % L);
            acc_prod(w[i].x, w[i].y, x.x, x.y, h0, l0);
            acc_prod(w[i].x, w[i].y, x.z, x.w, h1, l1);
        }
    }
    if (n - L >= 1) {
        const float4 gin = *row(ring, (n - L) % L);
        df_step_rows<false>(t, 0, nr, gin, Y, pitch, dof, h0, l0, h1, l1);
        df_step_rows<true>(t, nr, np, gin, Y, pitch, dof, h0, l0, h1, l1);
    }
    if (n >= 2) *row(ring, (n - 1) % L) = gp;
    H[dof] = (double)h0 + (double)l0;
    if (pair) H[dof + 1] = (double)h1 + (double)l1;
}

// Double-float tables of the per-step form (one block): the nodes with r <= 1/2 first as
// (r_hi, r_lo, c_hi, c_lo), then the others as (u_hi, u_lo, c_hi, c_lo), u = 1 - r, each class
// in its original order; *nr = the size of the first class; then the weights d_i, i < L, as
// pairs. tab: r[np], c[np], d[L].
__global__ void k_tab_to_df(const double *__restrict__ tab, int np, int L, float4 *__restrict__ tabdf,
                            float2 *__restrict__ wdf, int *__restrict__ nr) {
    int total_r = 0;
    for (int k = 0; k < np; ++k) total_r += tab[k] <= 0.5 ? 1 : 0;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const double r = tab[j];
        const bool u = r > 0.5;
        int before = 0;
        for (int k = 0; k < j; ++k) before += ((tab[k] > 0.5) == u) ? 1 : 0;
        const float2 a = u ? df_of(1.0 - r) : df_of(r), c = df_of(tab[np + j]);
        tabdf[u ? total_r + before : before] = make_float4(a.x, a.y, c.x, c.y);
    }
    for (int i = threadIdx.x; i < L; i += blockDim.x) wdf[i] = df_of(tab[2 * np + i]);
    if (threadIdx.x == 0) *nr = total_r;
}

__global__ void k_tab_to_f32(const double *__restrict__ t, int n, float *__restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = (float)t[i];
}

struct FastHistLayout {
    double *tab;       // r[np], c[np], d[L]
    double *scratch;   // Gauss-Jacobi nodes / weights
    double *dfull;     // weights d_0..d_{L-1} as produced by the weight kernel
    double *ring;      // L x ndof
    double *Y;         // np x ndof
    size_t bytes;
};

static FastHistLayout fast_hist_layout(void *ws, int np1, int np2, int L, int64_t ndof) {
    Carve cv(ws);
    FastHistLayout l;
    const int np = np1 + np2;
    l.tab = cv.take<double>(2 * np + kMaxNs);
    l.scratch = cv.take<double>(2 * (np1 + np2));
    l.dfull = cv.take<double>(kMaxNs);
    l.ring = cv.take<double>((size_t)L * ndof);
    l.Y = cv.take<double>((size_t)np * ndof);
    l.bytes = cv.bytes();
    return l;
}

struct FastHistLayoutDF {
    double *tab, *scratch, *dfull;
    float4 *tabdf;
    float2 *wdf, *ring, *Y;
    int *nr;
    int64_t pitch;
    size_t bytes;
};

static FastHistLayoutDF fast_hist_layout_df(void *ws, int np1, int np2, int L, int64_t ndof) {
    Carve cv(ws);
    FastHistLayoutDF l;
    const int np = np1 + np2;
    l.pitch = (ndof + 1) / 2 * 2;
    l.tab = cv.take<double>(2 * np + kMaxNs);
    l.scratch = cv.take<double>(2 * (np1 + np2));
    l.dfull = cv.take<double>(kMaxNs);
    l.tabdf = cv.take<float4>(np);
    l.wdf = cv.take<float2>(kMaxNs);
    l.nr = cv.take<int>(1);
    l.ring = cv.take<float2>((size_t)L * l.pitch);
    l.Y = cv.take<float2>((size_t)np * l.pitch);
    l.bytes = cv.bytes();
    return l;
}

struct FastHistLayoutF32 {
    double *tab, *scratch, *dfull;
    float *tabf, *ring, *Y;
    int64_t pitch;
    size_t bytes;
};

static FastHistLayoutF32 fast_hist_layout_f32(void *ws, int np1, int np2, int L, int64_t ndof) {
    Carve cv(ws);
    FastHistLayoutF32 l;
    const int np = np1 + np2;
    l.pitch = (ndof + 3) / 4 * 4;
    l.tab = cv.take<double>(2 * np + kMaxNs);
    l.scratch = cv.take<double>(2 * (np1 + np2));
    l.dfull = cv.take<double>(kMaxNs);
    l.tabf = cv.take<float>(2 * np + kMaxNs);
    l.ring = cv.take<float>((size_t)L * l.pitch);
    l.Y = cv.take<float>((size_t)np * l.pitch);
    l.bytes = cv.bytes();
    return l;
}

}  // namespace fastcq

using namespace fastcq;

extern "C" int cq_history_direct(int32_t scheme, double beta, double tau, int64_t ndof, int64_t n_lo,
                                 int64_t n_hi, const double *G_dev, int64_t ldg, double *H_dev, int64_t ldh,
                                 int32_t prec, void *ws_dev, size_t *ws_bytes, void *stream) {
    if (!ws_bytes || (scheme != CQ_BE && scheme != CQ_BDF2) || bad_order(beta) || !(tau > 0.0) || ndof < 0 ||
        n_lo < 1 || n_hi < n_lo || n_hi > kMaxWeights || ldg < ndof || ldh < ndof)
        return CQ_EINVAL;
    if (prec == CQ_BF16X3 || prec == CQ_TF32X3) {
        const int kind = prec == CQ_TF32X3 ? 1 : 0;
        const size_t need = history_tc_workspace(kind, ndof, n_lo, n_hi);
        if (!ws_dev) { *ws_bytes = need; return CQ_OK; }
        if (*ws_bytes < need) return CQ_ENOMEM;
        if (n_hi == n_lo || ndof == 0) return CQ_OK;
        if (!G_dev || !H_dev || ((uintptr_t)ws_dev & 255)) return CQ_EINVAL;
        return history_tc_run(kind, scheme, beta, tau, ndof, n_lo, n_hi, G_dev, ldg, H_dev, ldh, ws_dev,
                              (cudaStream_t)stream);
    }
    if (prec != CQ_F64) return CQ_EUNSUPPORTED;
    Carve cv(ws_dev);
    double *d = cv.take<double>(n_hi + 1);
    double *dz = cv.take<double>(n_hi + 2 * kDirectBT + 1);
    if (!ws_dev) { *ws_bytes = cv.bytes(); return CQ_OK; }
    if (*ws_bytes < cv.bytes()) return CQ_ENOMEM;
    if (n_hi == n_lo || ndof == 0) return CQ_OK;
    if (!G_dev || !H_dev) return CQ_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int st = launch_weights(scheme, beta, tau, n_hi, d, s);
    if (st) return st;
    k_pad_weights<<<(unsigned)((n_hi + 2 * kDirectBT + 256) / 256), 256, 0, s>>>(d, n_hi, dz);
    if ((st = launched())) return st;
    const bool vec2 = (ldg % 2 == 0) && (ldh % 2 == 0) && ((uintptr_t)G_dev % 16 == 0) && ((uintptr_t)H_dev % 16 == 0);
    const int64_t rows = n_hi - n_lo;
    dim3 grid;
    grid.y = (unsigned)((rows + kDirectBT - 1) / kDirectBT);
    if (grid.y > 65535) return CQ_EUNSUPPORTED;
    if (vec2) {
        grid.x = (unsigned)((ndof + 2 * 128 - 1) / (2 * 128));
        k_history_direct<kDirectBT, 2><<<grid, 128, 0, s>>>(ndof, n_lo, n_hi, dz, G_dev, ldg, H_dev, ldh);
    } else {
        grid.x = (unsigned)((ndof + 127) / 128);
        k_history_direct<kDirectBT, 1><<<grid, 128, 0, s>>>(ndof, n_lo, n_hi, dz, G_dev, ldg, H_dev, ldh);
    }
    return launched();
}

extern "C" int cq_history_fast(int32_t scheme, double beta, double tau, const cq_fast_cfg_t *cfg, int64_t ndof,
                               int64_t n, const double *G_prev_dev, double *H_dev, int32_t prec, void *ws_dev,
                               size_t *ws_bytes, void *stream) {
    if (!cfg || !ws_bytes || (scheme != CQ_BE && scheme != CQ_BDF2) || bad_order(beta) || !(tau > 0.0) ||
        ndof < 0 || n < 1)
        return CQ_EINVAL;
    if (prec != CQ_F64 && prec != CQ_F32 && prec != CQ_DF64) return CQ_EUNSUPPORTED;
    const int np1 = cfg->np1, np2 = (scheme == CQ_BE) ? 0 : cfg->np2;
    const int L = (scheme == CQ_BE) ? 2 : cfg->ns;
    if (np1 < 1 || np2 < 0 || np1 + np2 > kMaxNp || (scheme == CQ_BDF2 && (np2 < 1 || L < 3 || L > kMaxNs)))
        return CQ_EINVAL;
    if (prec == CQ_DF64) {
        FastHistLayoutDF ld = fast_hist_layout_df(ws_dev, np1, np2, L, ndof);
        if (!ws_dev) { *ws_bytes = ld.bytes; return CQ_OK; }
        if (*ws_bytes < ld.bytes) return CQ_ENOMEM;
        if (!H_dev || (n >= 2 && !G_prev_dev)) return CQ_EINVAL;
        if (ndof == 0) return CQ_OK;
        cudaStream_t s = (cudaStream_t)stream;
        const int np = np1 + np2;
        int st;
        if (n == 1) {
            if ((st = launch_weights(scheme, beta, tau, L - 1, ld.dfull, s))) return st;
            if ((st = cuda_status(cudaMemcpyAsync(ld.tab + 2 * np, ld.dfull, L * sizeof(double),
                                                  cudaMemcpyDeviceToDevice, s))))
                return st;
            if ((st = build_fast_coeffs(scheme, beta, tau, np1, np2, L, ld.scratch, ld.tab, ld.tab + np, s)))
                return st;
            k_tab_to_df<<<1, 256, 0, s>>>(ld.tab, np, L, ld.tabdf, ld.wdf, ld.nr);
            if ((st = launched())) return st;
            if ((st = cuda_status(cudaMemsetAsync(ld.Y, 0, (size_t)np * ld.pitch * sizeof(float2), s)))) return st;
            if ((st = cuda_status(cudaMemsetAsync(ld.ring, 0, (size_t)L * ld.pitch * sizeof(float2), s)))) return st;
            return cuda_status(cudaMemsetAsync(H_dev, 0, (size_t)ndof * sizeof(double), s));
        }
        const int64_t threads = (ndof + 1) / 2;
        if ((st = timing_begin(s))) return st;
        k_history_fast_step_df<<<(unsigned)((threads + 63) / 64), 64, 0, s>>>(
            ndof, ld.pitch, n, L, np, ld.tabdf, ld.wdf, ld.nr, ld.ring, ld.Y, G_prev_dev, H_dev);
        if ((st = launched())) return st;
        return timing_end(s);
    }
    if (prec == CQ_F32) {
        FastHistLayoutF32 lf = fast_hist_layout_f32(ws_dev, np1, np2, L, ndof);
        if (!ws_dev) { *ws_bytes = lf.bytes; return CQ_OK; }
        if (*ws_bytes < lf.bytes) return CQ_ENOMEM;
        if (!H_dev || (n >= 2 && !G_prev_dev)) return CQ_EINVAL;
        if (ndof == 0) return CQ_OK;
        cudaStream_t s = (cudaStream_t)stream;
        const int np = np1 + np2;
        int st;
        if (n == 1) {
            if ((st = launch_weights(scheme, beta, tau, L - 1, lf.dfull, s))) return st;
            if ((st = cuda_status(cudaMemcpyAsync(lf.tab + 2 * np, lf.dfull, L * sizeof(double),
                                                  cudaMemcpyDeviceToDevice, s))))
                return st;
            if ((st = build_fast_coeffs(scheme, beta, tau, np1, np2, L, lf.scratch, lf.tab, lf.tab + np, s)))
                return st;
            k_tab_to_f32<<<1, 512, 0, s>>>(lf.tab, 2 * np + L, lf.tabf);
            if ((st = launched())) return st;
            if ((st = cuda_status(cudaMemsetAsync(lf.Y, 0, (size_t)np * lf.pitch * sizeof(float), s)))) return st;
            if ((st = cuda_status(cudaMemsetAsync(lf.ring, 0, (size_t)L * lf.pitch * sizeof(float), s)))) return st;
            return cuda_status(cudaMemsetAsync(H_dev, 0, (size_t)ndof * sizeof(double), s));
        }
        // small blocks: a short streaming kernel, so whole-block granularity per SM matters
        const int64_t threads = (ndof + 3) / 4;
        if ((st = timing_begin(s))) return st;
        k_history_fast_step_f32<<<(unsigned)((threads + 63) / 64), 64, 0, s>>>(ndof, lf.pitch, n, L, np, lf.tabf,
                                                                              lf.ring, lf.Y, G_prev_dev, H_dev);
        if ((st = launched())) return st;
        return timing_end(s);
    }
    FastHistLayout lay = fast_hist_layout(ws_dev, np1, np2, L, ndof);
    if (!ws_dev) { *ws_bytes = lay.bytes; return CQ_OK; }
    if (*ws_bytes < lay.bytes) return CQ_ENOMEM;
    if (!H_dev || (n >= 2 && !G_prev_dev)) return CQ_EINVAL;
    if (ndof == 0) return CQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = np1 + np2;
    int st;
    if (n == 1) {
        if ((st = launch_weights(scheme, beta, tau, L - 1, lay.dfull, s))) return st;
        if ((st = cuda_status(cudaMemcpyAsync(lay.tab + 2 * np, lay.dfull, L * sizeof(double),
                                              cudaMemcpyDeviceToDevice, s))))
            return st;
        if ((st = build_fast_coeffs(scheme, beta, tau, np1, np2, L, lay.scratch, lay.tab, lay.tab + np, s)))
            return st;
        if ((st = cuda_status(cudaMemsetAsync(lay.Y, 0, (size_t)np * ndof * sizeof(double), s)))) return st;
        if ((st = cuda_status(cudaMemsetAsync(lay.ring, 0, (size_t)L * ndof * sizeof(double), s)))) return st;
        return cuda_status(cudaMemsetAsync(H_dev, 0, (size_t)ndof * sizeof(double), s));
    }
    const int64_t threads = (ndof + 1) / 2;
    if ((st = timing_begin(s))) return st;
    // 64-thread blocks: several per SM, so the last wave is short
    const int vec = (ndof % 2 == 0) && ((uintptr_t)G_prev_dev % 16 == 0) && ((uintptr_t)H_dev % 16 == 0);
    k_history_fast_step<<<(unsigned)((threads + 63) / 64), 64, 0, s>>>(ndof, n, L, np, vec, lay.tab, lay.ring,
                                                                       lay.Y, G_prev_dev, H_dev);
    if ((st = launched())) return st;
    return timing_end(s);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of cq_history_fast.
//
// Some callers cannot hand this library a workspace: a plug-in that only
// receives its input and output arrays from a host application which owns all
// device memory and exposes no allocator; a program whose memory pool is
// reserved in full before the time loop starts; a time loop that must not call
// cudaMalloc because that call can synchronise the device and can fail at an
// arbitrary step. For them the state of the fast history (Y, the last L levels
// and the tables) lives in one file-scope device array of fixed size, which
// every device that loads this library holds until the process exits.
//
// Every call made outside stream capture looks up the array's device address
// with cudaGetSymbolAddress (a host-side name of a __device__ array is not a
// device address), so a device reset or a new primary context, which reloads
// the module and moves the array, is picked up by the next call. A call made
// while its stream is being captured uses the address that the last call
// outside capture found on that device: make one call on the device before any
// stream capture. All calls share the one array and it keeps whatever the last
// call left in it: the call with n = 1 clears the state before use, and calls
// that overlap on the GPU (other streams, other threads, two problems at once
// on one device) race on it.
// ---------------------------------------------------------------------------
namespace fastcq {

static __device__ __align__(256) unsigned char g_noalloc_scratch[CQ_NOALLOC_SCRATCH_BYTES];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[kNoAllocMaxDevices] = {};

static int noalloc_scratch_address(cudaStream_t s, void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CQ_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return CQ_EUNSUPPORTED;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return CQ_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CQ_ECUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return CQ_OK;
}

}  // namespace fastcq

extern "C" int cq_history_fast_noalloc(int32_t scheme, double beta, double tau, const cq_fast_cfg_t *cfg,
                                       int64_t ndof, int64_t n, const double *G_prev_dev, double *H_dev,
                                       int32_t prec, void *stream) {
    size_t need = 0;
    int st = cq_history_fast(scheme, beta, tau, cfg, ndof, n, G_prev_dev, H_dev, prec, nullptr, &need, stream);
    if (st) return st;
    if (need > CQ_NOALLOC_SCRATCH_BYTES) return CQ_ENOMEM;
    void *scratch = nullptr;
    if ((st = noalloc_scratch_address((cudaStream_t)stream, &scratch))) return st;
    size_t cap = CQ_NOALLOC_SCRATCH_BYTES;
    return cq_history_fast(scheme, beta, tau, cfg, ndof, n, G_prev_dev, H_dev, prec, scratch, &cap, stream);
}
