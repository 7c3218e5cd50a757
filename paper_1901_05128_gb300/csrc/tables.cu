// Table builders: CQ weights, Gauss-Jacobi rules, fast-form coefficients,
// sine-mode eigenvalues, the DST-I matrix and the small FP64 GEMM that applies it.
// All run on the GPU in FP64 (FP32 only for the bracketing bisection of the
// Gauss-Jacobi nodes, which is followed by FP64 Newton steps).
#include "common.cuh"
#include "table_kernels.cuh"

namespace fastcq {

// ---------------------------------------------------------------------------
// CQ weights (Sec. 3, Eqs. 3.4 and 3.12).
// g_i = coefficients of (1 - zeta)^beta: g_0 = 1, g_i = g_{i-1} (i - 1 - beta)/i.
// One block: each thread forms the product of the factors of its chunk, an
// exclusive multiplicative block scan supplies the prefix, and each thread
// then writes its chunk. BE: d_i = tau^-beta g_i.
// BDF2: 3/2 - 2 zeta + zeta^2/2 = (3/2)(1 - zeta)(1 - zeta/3), so
//   d_i = tau^-beta (3/2)^beta sum_k g_{i-k} g_k 3^-k;
// terms with k > 64 are below 3^-64 relative and are left out.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWThreads) k_weights(int scheme, double beta, double scale, int n,
                                                       double *__restrict__ out, double *__restrict__ gscr) {
    extern __shared__ double gsm[];               // g[0..n] in shared memory, or in gscr (longer runs)
    weights_block(scheme, beta, scale, n, out, gscr ? gscr : gsm);
}

int launch_weights(int scheme, double beta, double tau, int64_t n, double *out, cudaStream_t s, double *scratch) {
    if (n < 0 || n > (scratch ? kMaxSolveSteps : kMaxWeights)) return CQ_EINVAL;
    const bool global = n > kMaxWeights;
    size_t smem = global ? 0 : (size_t)(n + 1) * sizeof(double);
    static unsigned long long attr = 0;
    int st;
    if ((st = smem_attr_once((const void *)k_weights, (int)((kMaxWeights + 1) * sizeof(double)), &attr))) return st;
    k_weights<<<1, kWThreads, smem, s>>>(scheme, beta, pow(tau, -beta), (int)n, out, global ? scratch : nullptr);
    return launched();
}

// ---------------------------------------------------------------------------
// Gauss-Jacobi rule for (1-s)^a (1+s)^b on [-1,1].
// Jacobi matrix of the monic Jacobi polynomials (three-term recurrence):
//   alpha_0 = (b-a)/(a+b+2), alpha_k = (b^2-a^2)/((2k+a+b)(2k+a+b+2)),
//   beta_k  = 4k(k+a)(k+b)(k+a+b)/((2k+a+b)^2 (2k+a+b+1)(2k+a+b-1)).
// Each thread owns one node: FP32 Sturm-count bisection brackets the j-th
// eigenvalue, FP64 Newton on the monic P_n (recurrence and its derivative)
// converges it, and the weight is the Christoffel number
//   lambda_j = 1 / sum_{k<n} phat_k(s_j)^2
// with phat_k orthonormal (phat_0 = mu0^-1/2, mu0 = int (1-s)^a (1+s)^b ds).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGJThreads) k_gauss_jacobi(int n, double a, double b,
                                                             double *__restrict__ nodes,
                                                             double *__restrict__ wts) {
    gauss_jacobi_block(n, a, b, blockIdx.x * blockDim.x, nodes, wts);
}

int launch_gauss_jacobi(int n, double a, double b, double *nodes, double *wts, cudaStream_t s) {
    if (n < 1 || n > kMaxNp || !(a > -1.0) || !(b > -1.0)) return CQ_EINVAL;
    k_gauss_jacobi<<<(n + kGJThreads - 1) / kGJThreads, kGJThreads, 0, s>>>(n, a, b, nodes, wts);
    return launched();
}

// ---------------------------------------------------------------------------
// Fast-form coefficients (Eqs. 3.6-3.7 for BE; Eqs. 3.14-3.16 with the real
// parts of Remark 3.2 for BDF2). K = 1/(tau^beta Gamma(1-beta) Gamma(beta)).
//   BE:    r = (s+1)/2,       c = w = -K lambda / 4
//   fam 1: r = (s+1)/(s+5),   c = w1 (s+5)^-4 r^(Ns-3),  w1 = -2^(2+2beta) cos(pi beta) K lambda1
//   fam 2: r = (s+1)/2,       c = w2 Re((1+3s)^beta) r^(Ns-3),  w2 = -2^(-beta-3) K lambda2
// The history part of a point is c * Y with Y <- r Y + G(t_{n-L}).
// ---------------------------------------------------------------------------
__global__ void k_fast_coeffs(int scheme, double beta, double tau, int np1, int np2, int ns,
                              const double *__restrict__ s1, const double *__restrict__ l1,
                              const double *__restrict__ s2, const double *__restrict__ l2,
                              double *__restrict__ r, double *__restrict__ c) {
    const int np = (scheme == CQ_BE) ? np1 : np1 + np2;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const bool fam1 = (scheme == CQ_BE) || j < np1;
    const double s = fam1 ? s1[j] : s2[j - np1];
    const double l = fam1 ? l1[j] : l2[j - np1];
    fast_coeff_point(scheme, beta, tau, np1, ns, j, s, l, r + j, c + j);
}

int launch_fast_coeffs(int scheme, double beta, double tau, int np1, int np2, int ns,
                       const double *nodes1, const double *w1, const double *nodes2, const double *w2,
                       double *r_out, double *c_out, cudaStream_t s) {
    const int np = (scheme == CQ_BE) ? np1 : np1 + np2;
    k_fast_coeffs<<<(np + 127) / 128, 128, 0, s>>>(scheme, beta, tau, np1, np2, ns, nodes1, w1, nodes2, w2,
                                                    r_out, c_out);
    return launched();
}

size_t fast_coeff_scratch_bytes(int np1, int np2) {
    return align_up((size_t)2 * (np1 + np2) * sizeof(double));
}

int build_fast_coeffs(int scheme, double beta, double tau, int np1, int np2, int ns, double *scratch,
                      double *r_out, double *c_out, cudaStream_t s) {
    double *n1 = scratch, *w1 = scratch + np1;
    double *n2 = scratch + 2 * np1, *w2 = n2 + np2;
    int st;
    if (scheme == CQ_BE) {
        if ((st = launch_gauss_jacobi(np1, beta, 1.0 - beta, n1, w1, s))) return st;
    } else {
        if ((st = launch_gauss_jacobi(np1, beta, 2.0 - 2.0 * beta, n1, w1, s))) return st;
        if ((st = launch_gauss_jacobi(np2, beta, 2.0 - 2.0 * beta, n2, w2, s))) return st;
    }
    return launch_fast_coeffs(scheme, beta, tau, np1, np2, ns, n1, w1, n2, w2, r_out, c_out, s);
}

// ---------------------------------------------------------------------------
// Spatial operator: lambda_k = 4 (M+1)^2 sin^2(k pi / (2(M+1))), summed over the
// axes in 2D / 3D with mode = ky*M + kx / (kz*M + ky)*M + kx; DST-I
// S_{jk} = sqrt(2/(M+1)) sin(j k pi/(M+1))
// with the angle reduced exactly in integers before sinpi.
// ---------------------------------------------------------------------------
static int64_t field_size(int M, int dim) {
    return dim == 1 ? (int64_t)M : dim == 2 ? (int64_t)M * M : (int64_t)M * M * M;
}

__global__ void k_mode_eigenvalues(int M, int dim, int64_t total, double *__restrict__ lam) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const double q = 2.0 * (M + 1);
    const double f = 4.0 * (double)(M + 1) * (double)(M + 1);
    // mode = (kz * M + ky) * M + kx: one sine factor per axis
    int64_t r = i;
    double acc = 0.0;
    for (int ax = 0; ax < dim; ++ax) {
        const int k = (int)(r % M);
        r /= M;
        const double sv = sinpi((double)(k + 1) / q);
        acc += f * sv * sv;
    }
    lam[i] = acc;
}

int launch_mode_eigenvalues(int M, int dim, double *lam, cudaStream_t s) {
    const int64_t total = field_size(M, dim);
    k_mode_eigenvalues<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(M, dim, total, lam);
    return launched();
}

__global__ void k_dst_matrix(int M, double *__restrict__ S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * M) return;
    const int64_t j = i / M + 1, k = i % M + 1;
    const int64_t per = 2 * (int64_t)(M + 1);
    const int64_t r = (j * k) % per;
    S[i] = sqrt(2.0 / (M + 1)) * sinpi((double)r / (double)(M + 1));
}

int launch_dst_matrix(int M, double *S, cudaStream_t s) {
    const int64_t total = (int64_t)M * M;
    k_dst_matrix<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(M, S);
    return launched();
}

// ---------------------------------------------------------------------------
// Small FP64 GEMM C = A B (M x M, row-major with row strides lda, ldb, ldc),
// batched over blockIdx.z. 64x64 tile per block, 16x16 threads with 4x4
// register tiles, K step 16.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dgemm_square(int M, const double *__restrict__ A, int64_t sA, int64_t lda,
                                                      const double *__restrict__ B, int64_t sB, int64_t ldb,
                                                      double *__restrict__ C, int64_t sC, int64_t ldc) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    A += blockIdx.z * sA;
    B += blockIdx.z * sB;
    C += blockIdx.z * sC;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * 64, col0 = blockIdx.x * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < M; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e & 15, rr = e >> 4;          // A tile: rows row0.., cols k0..
            const int r = row0 + rr, k = k0 + kk;
            As[kk][rr] = (r < M && k < M) ? A[(int64_t)r * lda + k] : 0.0;
            const int cc = e & 63, kb = e >> 6;          // B tile: rows k0.., cols col0..
            const int kb2 = k0 + kb, c = col0 + cc;
            Bs[kb][cc] = (kb2 < M && c < M) ? B[(int64_t)kb2 * ldb + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i) b[i] = Bs[kk][tx + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(a[i], b[jj], acc[i][jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * jj;
            if (r < M && c < M) C[(int64_t)r * ldc + c] = acc[i][jj];
        }
}

static int dgemm_strided(int M, int batch, const double *A, int64_t sA, int64_t lda, const double *B, int64_t sB,
                         int64_t ldb, double *C, int64_t sC, int64_t ldc, cudaStream_t s) {
    if (batch < 1 || batch > 65535) return CQ_EUNSUPPORTED;
    dim3 grid((M + 63) / 64, (M + 63) / 64, batch);
    k_dgemm_square<<<grid, 256, 0, s>>>(M, A, sA, lda, B, sB, ldb, C, sC, ldc);
    return launched();
}

int launch_dgemm_square(int M, int batch, const double *A, int64_t sA, const double *B, int64_t sB, double *C,
                        int64_t sC, cudaStream_t s) {
    return dgemm_strided(M, batch, A, sA, M, B, sB, M, C, sC, M, s);
}

// 1D: out[s][k] = sum_j S[k][j] in[s][j]
__global__ void k_dst_1d(int M, const double *__restrict__ S, const double *__restrict__ in,
                         double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int st = blockIdx.y;
    if (k >= M) return;
    double acc = 0.0;
    for (int j = 0; j < M; ++j) acc = fma(S[(int64_t)k * M + j], in[(int64_t)st * M + j], acc);
    out[(int64_t)st * M + k] = acc;
}

int launch_dst_field(int M, int dim, const double *S, const double *in, double *out, double *tmp, cudaStream_t s) {
    if (dim == 1) {
        k_dst_1d<<<dim3((M + 127) / 128, 2), 128, 0, s>>>(M, S, in, out);
        return launched();
    }
    const int64_t mm = (int64_t)M * M;
    if (dim == 2) {
        int st = launch_dgemm_square(M, 2, S, 0, in, mm, tmp, mm, s);      // S F
        if (st) return st;
        return launch_dgemm_square(M, 2, tmp, mm, S, 0, out, mm, s);       // (S F) S
    }
    // 3D, F[z][y][x] per state: along x (F[z] S, batched over z), along y (S F[z]), then along z:
    // for each y the z-x plane (row stride M^2) is multiplied by S from the left
    const int64_t m3 = mm * M;
    int st;
    if ((st = dgemm_strided(M, 2 * M, in, mm, M, S, 0, M, out, mm, M, s))) return st;
    if ((st = dgemm_strided(M, 2 * M, S, 0, M, out, mm, M, tmp, mm, M, s))) return st;
    for (int q = 0; q < 2; ++q)
        if ((st = dgemm_strided(M, M, S, 0, M, tmp + q * m3, M, mm, out + q * m3, M, mm, s))) return st;
    return CQ_OK;
}

}  // namespace fastcq

using namespace fastcq;

extern "C" int cq_weights(int32_t scheme, double beta, double tau, int64_t n, double *w_dev, void *stream) {
    if ((scheme != CQ_BE && scheme != CQ_BDF2) || bad_order(beta) || !(tau > 0.0) || n < 0 ||
        n > kMaxWeights || !w_dev)
        return CQ_EINVAL;
    return launch_weights(scheme, beta, tau, n, w_dev, (cudaStream_t)stream);
}

extern "C" int cq_gauss_jacobi(int32_t n, double a, double b, double *nodes_dev, double *weights_dev,
                               void *stream) {
    if (!nodes_dev || !weights_dev) return CQ_EINVAL;
    return launch_gauss_jacobi(n, a, b, nodes_dev, weights_dev, (cudaStream_t)stream);
}

extern "C" int cq_fast_coeffs(int32_t scheme, double beta, double tau, const cq_fast_cfg_t *cfg,
                              double *coef_dev, void *ws_dev, size_t *ws_bytes, void *stream) {
    if (!cfg || !ws_bytes || (scheme != CQ_BE && scheme != CQ_BDF2) || bad_order(beta) || !(tau > 0.0))
        return CQ_EINVAL;
    const int np1 = cfg->np1, np2 = (scheme == CQ_BE) ? 0 : cfg->np2, ns = cfg->ns;
    if (np1 < 1 || np2 < 0 || np1 + np2 > kMaxNp || (scheme == CQ_BDF2 && (np2 < 1 || ns < 3 || ns > kMaxNs)))
        return CQ_EINVAL;
    const size_t need = fast_coeff_scratch_bytes(np1, np2);
    if (!ws_dev) { *ws_bytes = need; return CQ_OK; }
    if (*ws_bytes < need) return CQ_ENOMEM;
    if (!coef_dev) return CQ_EINVAL;
    const int np = np1 + np2;
    return build_fast_coeffs(scheme, beta, tau, np1, np2, ns, (double *)ws_dev, coef_dev, coef_dev + np,
                             (cudaStream_t)stream);
}
