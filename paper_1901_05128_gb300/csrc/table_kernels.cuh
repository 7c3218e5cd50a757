// Device bodies of the table builders (CQ weights, Gauss-Jacobi rules,
// fast-form coefficients), shared by the single-problem kernels (tables.cu)
// and the batched set-up kernels (batch.cu).
#pragma once

#include "common.cuh"

namespace fastcq {

constexpr int kWThreads = 1024;
constexpr int kCauchyTerms = 64;

// Block-wide body (blockDim.x == kWThreads); g: n+1 doubles of shared memory.
__device__ __forceinline__ void weights_block(int scheme, double beta, double scale, int n, double *__restrict__ out,
                              double *__restrict__ g) {
    __shared__ double part[kWThreads];
    __shared__ double bk[kCauchyTerms + 1];
    const int t = threadIdx.x;
    const int T = blockDim.x;
    const int chunk = (n + 1 + T - 1) / T;
    const int lo = t * chunk;
    const int hi = min(lo + chunk, n + 1);
    double p = 1.0;
    for (int i = max(lo, 1); i < hi; ++i) p *= (i - 1.0 - beta) / i;
    part[t] = p;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        double x = (t >= off) ? part[t - off] : 1.0;
        __syncthreads();
        part[t] *= x;
        __syncthreads();
    }
    double v = (t == 0) ? 1.0 : part[t - 1];
    for (int i = lo; i < hi; ++i) {
        if (i >= 1) v *= (i - 1.0 - beta) / i;
        g[i] = v;
    }
    __syncthreads();
    if (scheme == CQ_BE) {
        for (int i = t; i <= n; i += T) out[i] = g[i] * scale;
        return;
    }
    if (t <= kCauchyTerms && t <= n) {
        bk[t] = g[t] / pow(3.0, (double)t);
    }
    __syncthreads();
    const double c0 = pow(1.5, beta) * scale;
    for (int i = t; i <= n; i += T) {
        const int kmax = min(i, kCauchyTerms);
        double acc = 0.0;
        for (int k = kmax; k >= 0; --k) acc = fma(g[i - k], bk[k], acc);
        out[i] = acc * c0;
    }
}

constexpr int kGJThreads = 64;

// Block body: node j = j0 + threadIdx.x (j0 = first node of this block).
__device__ __forceinline__ void gauss_jacobi_block(int n, double a, double b, int j0, double *__restrict__ nodes,
                                   double *__restrict__ wts) {
    __shared__ double al[kMaxNp], be[kMaxNp], sq[kMaxNp];
    __shared__ float fal[kMaxNp], fbe[kMaxNp];
    const double ab = a + b;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double dk = (k == 0) ? (b - a) / (ab + 2.0) : (b * b - a * a) / ((2.0 * k + ab) * (2.0 * k + ab + 2.0));
        al[k] = dk;
        fal[k] = (float)dk;
        double o2 = 0.0;
        if (k >= 1) {
            const double c = 2.0 * k + ab;
            o2 = 4.0 * k * (k + a) * (k + b) * (k + ab) / (c * c * (c + 1.0) * (c - 1.0));
        }
        be[k] = o2;
        sq[k] = sqrt(o2);
        fbe[k] = (float)o2;
    }
    __syncthreads();
    const int j = j0 + threadIdx.x;
    if (j >= n) return;
    float lo = -1.0f, hi = 1.0f;
    for (int it = 0; it < 26; ++it) {
        const float mid = 0.5f * (lo + hi);
        float q = fal[0] - mid;
        int cnt = (q < 0.0f);
        for (int k = 1; k < n; ++k) {
            if (q == 0.0f) q = 1e-30f;
            q = (fal[k] - mid) - fbe[k] / q;
            cnt += (q < 0.0f);
        }
        if (cnt > j) hi = mid; else lo = mid;
    }
    double x = 0.5 * ((double)lo + (double)hi);
    for (int it = 0; it < 6; ++it) {
        double p0 = 1.0, p1 = x - al[0], d0 = 0.0, d1 = 1.0;
        for (int k = 1; k < n; ++k) {
            const double u = x - al[k];
            const double p2 = u * p1 - be[k] * p0;
            const double d2 = p1 + u * d1 - be[k] * d0;
            p0 = p1; p1 = p2; d0 = d1; d1 = d2;
        }
        x -= p1 / d1;
    }
    const double mu0 = exp2(ab + 1.0) * tgamma(a + 1.0) * tgamma(b + 1.0) / tgamma(ab + 2.0);
    double pm = 0.0, pk = 1.0 / sqrt(mu0), sum = pk * pk;
    for (int k = 0; k + 1 < n; ++k) {
        const double pn = ((x - al[k]) * pk - sq[k] * pm) / sq[k + 1];
        pm = pk;
        pk = pn;
        sum = fma(pk, pk, sum);
    }
    nodes[j] = x;
    wts[j] = 1.0 / sum;
}

// Fast-form (r_j, c_j) of point j from its Gauss-Jacobi node s and weight l
// (see k_fast_coeffs in tables.cu for the formulas).
__device__ __forceinline__ void fast_coeff_point(int scheme, double beta, double tau, int np1, int ns, int j, double s,
                                                 double l, double *r, double *c) {
    const double K = 1.0 / (pow(tau, beta) * tgamma(1.0 - beta) * tgamma(beta));
    if (scheme == CQ_BE) {
        *r = 0.5 * (s + 1.0);
        *c = -0.25 * K * l;
    } else if (j < np1) {
        const double rr = (s + 1.0) / (s + 5.0);
        const double w = -exp2(2.0 + 2.0 * beta) * cospi(beta) * K * l;
        const double s5 = s + 5.0;
        *r = rr;
        *c = w / (s5 * s5 * s5 * s5) * pow(rr, (double)(ns - 3));
    } else {
        const double rr = 0.5 * (s + 1.0);
        const double w = -exp2(-beta - 3.0) * K * l;
        const double u = 1.0 + 3.0 * s;
        const double re = (u >= 0.0) ? pow(u, beta) : pow(-u, beta) * cospi(beta);
        *r = rr;
        *c = w * re * pow(rr, (double)(ns - 3));
    }
}

}  // namespace fastcq
