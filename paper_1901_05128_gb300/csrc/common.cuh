// Shared helpers of the fastcq CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <math.h>

#include "../../include/fastcq.h"

namespace fastcq {

// Kernels launched by this library since load (reported by cq_launch_count).
void count_launches(int64_t k);
// Events around a call's main kernel when timing is enabled (cq_timing_enable).
int timing_begin(cudaStream_t s);
int timing_end(cudaStream_t s);
// Events around one sub-launch of the timed region (end = false before it, true after);
// cq_timing_part(1) sums them. At most kMaxTimedParts sub-launches per call are timed.
constexpr int kMaxTimedParts = 512;
int timing_part(cudaStream_t s, bool end);

// Status bits written by kernels into a workspace status word.
enum : int { ST_NONFINITE = 1, ST_SINGULAR = 2, ST_TIMEOUT = 4 };

constexpr int kMaxNp = 256;      // Gauss-Jacobi points per state (np1 + np2)
constexpr int kMaxNs = 32;       // exact window of the fast BDF2 form
constexpr int64_t kMaxWeights = 24000;       // weights built in shared memory (and per-call limit of the history APIs)
constexpr int64_t kMaxSolveSteps = 1 << 20;  // fp2s_solve: longer weight tables go through a global scratch

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Bump allocator over a caller workspace: offsets are computed identically for
// the size query (base == nullptr) and the real call.
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base(static_cast<char *>(b)) {}
    template <class T> T *take(size_t count) {
        off = align_up(off);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t bytes() const { return align_up(off); }
};

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? CQ_OK : CQ_ECUDA; }

// Launch check: counts one launch and converts a launch error into CQ_ECUDA.
inline int launched(int64_t k = 1) {
    count_launches(k);
    return cuda_status(cudaGetLastError());
}

inline bool bad_order(double beta) { return !(beta > 0.0 && beta < 1.0); }

// Device-wide settings are per device: a kernel's dynamic shared-memory limit is set once
// per device (bit d of *done marks device d; devices beyond 63 set it on every call).
int smem_attr_once(const void *func, int bytes, unsigned long long *done);
// Multiprocessor count of the current device.
int device_sms();

// ---- table builders (tables.cu), all enqueue on `s` -------------------------
// weights d_i, i = 0..n, of scheme into out (device). Single block. n <= kMaxWeights, or
// n <= kMaxSolveSteps with scratch (n + 1 doubles of device memory).
int launch_weights(int scheme, double beta, double tau, int64_t n, double *out, cudaStream_t s,
                   double *scratch = nullptr);
// Gauss-Jacobi nodes / weights.
int launch_gauss_jacobi(int n, double a, double b, double *nodes, double *wts, cudaStream_t s);
// Fast-form (r_j, c_j) from Gauss-Jacobi rules already in nodes1/w1 (and nodes2/w2).
int launch_fast_coeffs(int scheme, double beta, double tau, int np1, int np2, int ns,
                       const double *nodes1, const double *w1, const double *nodes2, const double *w2,
                       double *r_out, double *c_out, cudaStream_t s);
// Full fast-coefficient pipeline with scratch from a Carve (2 rules).
size_t fast_coeff_scratch_bytes(int np1, int np2);
int build_fast_coeffs(int scheme, double beta, double tau, int np1, int np2, int ns,
                      double *scratch, double *r_out, double *c_out, cudaStream_t s);
// Sine-mode eigenvalues of the FD Laplacian (dim 1, 2 or 3), M^dim values.
int launch_mode_eigenvalues(int M, int dim, double *lam, cudaStream_t s);
// Orthonormal DST-I matrix S (M x M, row-major).
int launch_dst_matrix(int M, double *S, cudaStream_t s);
// C[batch] = A[batch] * B[batch] for M x M row-major matrices (FP64), batch strides in elements.
int launch_dgemm_square(int M, int batch, const double *A, int64_t sA, const double *B, int64_t sB,
                        double *C, int64_t sC, cudaStream_t s);
// Sine transform of a two-state field along every axis (1D: out[s] = S in[s]; 2D: S in[s] S;
// 3D: along x, y, z); tmp: 2*M^dim doubles (2D, 3D); in and out must differ.
int launch_dst_field(int M, int dim, const double *S, const double *in, double *out, double *tmp,
                     cudaStream_t s);

// Tensor-core (tcgen05, BF16x3 or TF32x3: kind 0 / 1) direct history (history_tc.cu).
size_t history_tc_workspace(int kind, int64_t ndof, int64_t n_lo, int64_t n_hi);
int history_tc_run(int kind, int scheme, double beta, double tau, int64_t ndof, int64_t n_lo, int64_t n_hi,
                   const double *G, int64_t ldg, double *H, int64_t ldh, void *ws, cudaStream_t s);

}  // namespace fastcq
