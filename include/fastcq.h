/*
 * fastcq — convolution-quadrature (CQ) history sums of the Riemann-Liouville
 * derivative and the two-state fractional Fokker-Planck schemes of
 * Sun, Nie & Deng, "Fast algorithms for convolution quadrature of
 * Riemann-Liouville fractional derivative" (arXiv 1901.05128), on NVIDIA
 * GB300 (sm_103a).
 *
 * C ABI. Every pointer named *_dev is CUDA device memory owned by the caller;
 * *_host is host memory owned by the caller. The library never allocates
 * device memory at call time (cq_history_fast_noalloc uses one fixed array
 * that exists from load): entry points that need scratch take a caller workspace
 * (ws_dev, ws_bytes). Passing ws_dev == NULL turns such a call into a size
 * query: *ws_bytes receives the required size and nothing runs. Workspaces
 * must be 256-byte aligned (cudaMalloc / torch allocations are).
 *
 * Unless stated otherwise a call only enqueues work on `stream` (a
 * cudaStream_t; NULL = legacy default stream) and returns at once; argument
 * errors are reported before anything is enqueued. Return values are CQ_OK
 * or a negative CQ_E* status; cq_strerror() turns one into text. No entry
 * point aborts, traps or exits.
 *
 * Host threads: calls on different workspaces may run from several threads
 * at once. Process-wide exceptions: the timing functions (cq_timing_*) and the
 * test switch cq_test_expire_waits keep one state for the whole process, and
 * every cq_history_fast_noalloc call uses the same device array (calls whose
 * work overlaps on the GPU race).
 *
 * Notation (paper's): beta = 1 - alpha is the CQ order used for a state,
 * tau = T/N the step, G^n the level at t_n, d_i the CQ weights,
 * a = (1-m)/(2m-1) the coupling, A = -Laplacian (Dirichlet).
 */
#ifndef FASTCQ_H
#define FASTCQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CQ_OK            0
#define CQ_EINVAL       -1   /* invalid argument (range, size, pointer, order of calls) */
#define CQ_ENOMEM       -2   /* caller workspace smaller than required */
#define CQ_ECUDA        -3   /* a CUDA runtime call failed (launch, copy, sync) */
#define CQ_ESINGULAR    -4   /* a 2x2 step matrix is singular to working precision */
#define CQ_ENONFINITE   -5   /* the result contains Inf or NaN */
#define CQ_ETIMEOUT     -6   /* a bounded device wait gave up */
#define CQ_EUNSUPPORTED -7   /* valid request outside what this build implements */

/* ---- enumerations ------------------------------------------------------ */
#define CQ_BE      1   /* backward Euler generating function (1 - zeta)/tau */
#define CQ_BDF2    2   /* second-order backward difference ((1-zeta) + (1-zeta)^2/2)/tau */
#define CQ_DIRECT  0   /* plain O(N^2) history (Eq. 3.8 / 4.1 / 4.7) */
#define CQ_FAST    1   /* fast O(N Np) history (Eqs. 3.9-3.10, 3.17-3.18) */
#define CQ_F64     0   /* FP64 end to end */
#define CQ_F32     1   /* precision form of the fast solve: FP32 history state and sums, FP64 tables
                        * and per-mode matrices, double-float (FP64 when |a| > 10) 2x2 step */
#define CQ_BF16X3  2   /* precision form of the direct history on tensor cores: operands split into
                        * BF16 hi + lo, hi*hi + hi*lo + lo*hi accumulated in FP32 */
#define CQ_TF32X3  3   /* the same with TF32 hi + lo (11 significant bits each; half the BF16
                        * tensor rate, twice the operand bytes, ~2^6 times smaller split error) */
#define CQ_DF64    4   /* FP64-class form of the solves: history state (fast form) or stored levels
                        * (direct form), weights, tables and sums as double-float pairs (hi + lo of
                        * two FP32 numbers) on the FP32 pipe, the 2x2 step in FP64
                        * (fast: np1 + np2 <= 128) */

/* Fast-form sizes. BE (Eqs. 3.6-3.10): np1 = Np Gauss-Jacobi points, np2
 * ignored, ns ignored (the exact window of BE is d_1 alone).
 * BDF2 (Eqs. 3.14-3.18): np1 = N_{p,1}, np2 = N_{p,2} points of the two
 * families, ns = N_s >= 3 exact weights d_0..d_{Ns-1} (Remark 3.3).
 * Limits: 1 <= np1 + np2 <= 256, ns <= 32. */
typedef struct { int32_t np1, np2, ns; } cq_fast_cfg_t;

/* ---- library information ----------------------------------------------- */
const char *cq_strerror(int status);
/* Number of CUDA kernels this library has launched since it was loaded. */
int64_t cq_launch_count(void);
/* When enabled (on != 0), fp2s_solve, fp2s_solve_batched, fp2s_gradient,
 * cq_history_fast (n >= 2) and the tensor-core cq_history_direct record CUDA
 * events around their main kernel on the caller's stream;
 * cq_timing_last() returns that kernel's duration in milliseconds for the most
 * recent such call (it synchronises on the closing event). */
int cq_timing_enable(int on);
int cq_timing_last(double *ms_main_kernel);
/* Parts of the most recent timed call: part 0 = the same as cq_timing_last;
 * part 1 = summed duration of the tensor-core contraction launches of the
 * mixed-precision direct solve (fp2s_solve, CQ_DIRECT with CQ_BF16X3 or
 * CQ_TF32X3) or of the mixed-precision gradient (0 for other calls).
 * Synchronises on the recorded events.
 * CQ_EINVAL for another part, a NULL pointer or no timed call yet. */
int cq_timing_part(int part, double *ms);
/* Test switch for the failure path of the tensor-core kernels (on != 0: on;
 * process-wide; enqueued work is not affected). While on, every tensor-core
 * launch (cq_history_direct with CQ_BF16X3 / CQ_TF32X3, the mixed-precision
 * solve and gradient) withholds the first operand load of each CTA and bounds
 * the waits between the CTA's producer, MMA and epilogue roles by 10 ms
 * instead of 2 s. The MMA thread's wait for that load then expires: the kernel
 * records the timeout, writes NaN to its tiles, drains its loads and frees its
 * tensor memory; the mixed-precision fp2s_solve, fp2s_gradient and fp2s_vjp
 * return CQ_ETIMEOUT and cq_history_direct leaves NaN in the outputs it could
 * not form. The device
 * stays usable. For tests only; off when the library loads. Always CQ_OK. */
int cq_test_expire_waits(int on);

/* ---- CQ weights (Sec. 3, Eqs. 3.4 and 3.12) ---------------------------- */
/* w_dev[i] = d^beta_{s,i}, i = 0..n: the Taylor coefficients of delta(zeta)^beta
 * with delta = (1-zeta)/tau (CQ_BE, Eq. 3.4) or ((1-zeta)+(1-zeta)^2/2)/tau
 * (CQ_BDF2, Eq. 3.12). 0 < beta < 1, tau > 0, 0 <= n <= 24000.
 * Output: n+1 doubles in device memory. */
int cq_weights(int32_t scheme, double beta, double tau, int64_t n, double *w_dev, void *stream);

/* ---- Gauss-Jacobi rule (used by Eqs. 3.6 and 3.14) --------------------- */
/* Nodes s_j (ascending) and weights lambda_j, j = 0..n-1, of the n-point
 * Gauss rule for int_{-1}^{1} (1-s)^a (1+s)^b f(s) ds. 1 <= n <= 256,
 * a, b > -1. Outputs: n doubles each, device memory. */
int cq_gauss_jacobi(int32_t n, double a, double b, double *nodes_dev, double *weights_dev, void *stream);

/* ---- fast-form coefficients (Eqs. 3.6-3.7, 3.14-3.16, Remark 3.2) ------ */
/* For each Gauss-Jacobi point j (BE: j < np1; BDF2: the np1 points of family 1
 * then the np2 points of family 2) the ratio r_j of its geometric sequence and
 * the coefficient c_j such that the history part of the paper satisfies
 *   Ghist_j(t_n) = c_j * Y_j(t_n),   Y_j(t_n) = r_j * Y_j(t_{n-1}) + G(t_{n-L}),
 * with L = 2 for BE (c_j = w_j) and L = Ns for BDF2
 * (c_j = w1_j (s+5)^-4 r1_j^(Ns-3), resp. w2_j Re((1+3s)^beta) r2_j^(Ns-3)).
 * coef_dev: 2*np doubles, [r_0..r_{np-1}, c_0..c_{np-1}], np = np1 (BE) or
 * np1+np2 (BDF2). ws_dev: scratch of *ws_bytes (size query when NULL). */
int cq_fast_coeffs(int32_t scheme, double beta, double tau, const cq_fast_cfg_t *cfg,
                   double *coef_dev, void *ws_dev, size_t *ws_bytes, void *stream);

/* ---- direct history (Eq. 3.8; Eqs. 4.1 and 4.7 leave G^0 out) --------- */
/* For every n in [n_lo, n_hi) and every DOF:
 *     H_dev[(n - n_lo) * ldh + dof] = sum_{i=1}^{n-1} d_i G_dev[(n - i) * ldg + dof]
 * i.e. the strictly lower-triangular Toeplitz product of the CQ weights with
 * the levels G^1..G^{n-1} (row t of G_dev holds G^t; row 0 is never read).
 * 1 <= n_lo <= n_hi, ndof >= 0, ldg, ldh >= ndof. The weights are computed
 * into the workspace. prec: CQ_F64 (FP64 FMAs), CQ_BF16X3 or CQ_TF32X3
 * (tcgen05 tensor cores; G and the Toeplitz tiles are split and staged in the
 * workspace, which then holds about 4 (BF16) or 8 (TF32) * ndof * n_hi bytes;
 * n_hi + 128 <= 24000; the tensor cores' FP32 accumulation, which rounds toward
 * zero, runs in chunks of 128 (BF16) or 32 (TF32) levels that are summed with
 * round-to-nearest; magnitudes below 2^-126 in the FP32 accumulator are returned
 * as zero). On a device fault or an expired internal wait the tensor-core paths
 * write NaN to the affected outputs. */
int cq_history_direct(int32_t scheme, double beta, double tau, int64_t ndof,
                      int64_t n_lo, int64_t n_hi, const double *G_dev, int64_t ldg,
                      double *H_dev, int64_t ldh, int32_t prec,
                      void *ws_dev, size_t *ws_bytes, void *stream);

/* The operand split of the tensor-core forms, as cq_history_direct applies it
 * to the levels and weights (exposed so that it can be checked against exact
 * rounding): for i < n,
 *     hi = x_dev[i] rounded to nearest-even with 8 (CQ_BF16X3) or 11
 *          (CQ_TF32X3) significant bits, lo = (x_dev[i] - hi) rounded the same way,
 * written as BF16 bit patterns (uint16_t, prec CQ_BF16X3) or FP32 bit patterns
 * with the 13 low mantissa bits zero (uint32_t, CQ_TF32X3) to hi_dev[i] and
 * lo_dev[i]. Parts below the normal FP32 range (2^-126) are signed zeros,
 * parts above it +-Inf (lo = 0 then); NaN stays NaN. n >= 0; n = 0 does
 * nothing. CQ_EUNSUPPORTED for other precisions. */
int cq_split(int32_t prec, const double *x_dev, int64_t n, void *hi_dev, void *lo_dev, void *stream);

/* ---- fast history, one step (Eqs. 3.9-3.10 / 3.17-3.18, Remarks 4.1, 4.7) */
/* Forms h^n = sum_{i=1}^{min(L-1, n-1)} d_i G^{n-i} + sum_j Ghist_j(t_n) for all
 * DOFs, L = 2 (BE) or Ns (BDF2), advancing the history parts from t_{n-1} to t_n.
 * Must be called with n = 1, 2, 3, ... in order on the same workspace; the call
 * with n = 1 (re)initialises the workspace (tables, zero state) and writes
 * h^1 = 0. G_prev_dev = G^{n-1} (ndof doubles; ignored for n = 1, may be NULL).
 * H_dev = h^n (ndof doubles). The workspace holds the Ghist state
 * (np x ndof), the last L levels and the tables; its size depends on
 * (scheme, cfg, ndof, prec) only. prec: CQ_F64, CQ_F32 (state, levels and
 * sums in FP32, streamed with 16-byte accesses; tables computed in FP64), or
 * CQ_DF64 (state, levels, tables and sums as double-float pairs on the FP32
 * pipe, 8 bytes per value as in FP64; the FP64 error bar at HBM-bound speed).
 * CQ_F32 and CQ_DF64 hold every value in FP32's exponent range and, unlike the
 * solves, apply no scaling of their own: levels or states of magnitude below
 * about 2^-126 lose their low bits (down to zero below 2^-149), and above
 * about 2^127 become infinite. The history is linear in G, so a caller whose
 * levels lie outside that range scales them by a power of two (exact) and
 * scales h^n back. */
int cq_history_fast(int32_t scheme, double beta, double tau, const cq_fast_cfg_t *cfg,
                    int64_t ndof, int64_t n, const double *G_prev_dev, double *H_dev,
                    int32_t prec, void *ws_dev, size_t *ws_bytes, void *stream);

/* ---- allocation-free fast history (no counterpart in the paper) --------- */
/* Same computation, arguments and call order as cq_history_fast, but with no
 * workspace argument. It is meant for callers that cannot allocate device
 * memory: a plug-in that is handed only its input and output arrays by a host
 * application which owns all device memory; a program whose memory pool is
 * fully reserved before its time loop; a loop that must not call cudaMalloc,
 * which can synchronise the device and can fail at an arbitrary step.
 * The state lives in one library-owned device array of
 * CQ_NOALLOC_SCRATCH_BYTES (16 MiB) that every device loading the library
 * keeps until the process exits. A request whose state does not fit
 * ((np + L) * ndof doubles plus small tables; e.g. ndof <= ~21,600 for
 * np = 80, L = 17) returns CQ_ENOMEM before any work is enqueued.
 * Each call made outside stream capture looks up the array's device address on
 * the current device, so a device reset or a new primary context (which moves
 * the array) is picked up by the next call; a call made while `stream` is being
 * captured reuses the address the last call outside capture found on that
 * device: make one call on the device before any stream capture. Every call shares
 * the array, which keeps the last call's contents: the n = 1 call clears the
 * state, and calls that overlap on the GPU (several problems or streams at
 * once on one device) race on it. It calls no allocating routine. */
#define CQ_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int cq_history_fast_noalloc(int32_t scheme, double beta, double tau, const cq_fast_cfg_t *cfg,
                            int64_t ndof, int64_t n, const double *G_prev_dev, double *H_dev,
                            int32_t prec, void *stream);

/* ---- two-state fractional Fokker-Planck system (Eqs. 1.1-1.3, 2.1) ----- */
/* Problem on (0,1)^dim, dim in {1,2,3}, with M interior points per axis of the
 * centred finite-difference Laplacian (h = 1/(M+1); M <= 65536, 4096, 1024 for
 * dim 1, 2, 3); DOFs of one state are ordered dof = ix (1D), iy*M + ix (2D),
 * (iz*M + iy)*M + ix (3D), and a two-state field is [2][M^dim] doubles.
 * 0 < alpha1, alpha2 < 1; 0 <= m < 1, m != 1/2; T > 0; 1 <= N <= 2^20
 * (N <= 24000 in the batch API, N <= 13000 for gradients).
 * flags bit 0 (FP2S_ASYNC): fp2s_solve does not synchronise and does not
 * report device status (CQ_ENONFINITE); use fp2s_status() later. */
#define FP2S_ASYNC 1
typedef struct {
    double alpha1, alpha2, m, T;
    int64_t N;
    int32_t dim, M;
    int32_t scheme;        /* CQ_BE or CQ_BDF2 */
    int32_t form;          /* CQ_DIRECT or CQ_FAST */
    cq_fast_cfg_t fast;    /* used when form == CQ_FAST */
    int32_t prec;          /* CQ_F64; in fp2s_solve also CQ_F32 with form == CQ_FAST (np1 + np2 <= 128),
                              CQ_DF64 with either form (fast: np1 + np2 <= 128)
                              and CQ_BF16X3 or CQ_TF32X3 with form == CQ_DIRECT (mixed-precision
                              direct solve); fp2s_gradient / fp2s_vjp take CQ_F64 and CQ_DF64
                              with either form (fast, CQ_DF64: np1 + np2 <= 128), and CQ_BF16X3
                              and CQ_TF32X3 with form == CQ_DIRECT */
    int32_t flags;
} fp2s_problem_t;

/* Whole solve, fused: G0_dev (physical [2][M^dim]) -> GN_dev (physical
 * [2][M^dim], the level t_N of the BE scheme Eq. 4.1 / fast BE Eq. 4.3 /
 * SBD Eq. 4.7 / fast SBD Eq. 4.8). Every sine mode is advanced through all N
 * steps by one persistent kernel (FP64, CQ_F32). The mixed-precision direct
 * solve (CQ_DIRECT with CQ_BF16X3 or CQ_TF32X3) runs in blocks of 128 steps:
 * the history from earlier blocks is a tcgen05 contraction of split BF16 or
 * TF32 operands (FP32 accumulation per chunk, chunks summed with
 * round-to-nearest), the in-block part and the steps run in FP32 /
 * double-float (FP64 when |a| > 10), with the FP32 remainders of d_1 and d_2
 * and of the previous level carried into the step; its workspace holds the
 * levels as hi + lo (about 4 (BF16) or 8 (TF32) bytes per DOF-step). Relative
 * errors against the FP64 scheme are of order 1e-6 (TF32x3) to 3e-6 (BF16x3)
 * on 2D 511x511, N = 8192. CQ_F32 (fast form): of order 1e-6 on the same grid.
 * Synchronises `stream` at the end to read the device status unless
 * flags & FP2S_ASYNC. */
int fp2s_solve(const fp2s_problem_t *p, const double *G0_dev, double *GN_dev,
               void *ws_dev, size_t *ws_bytes, void *stream);

/* The same schemes on the sine coefficients of a contiguous range of modes
 * [mode_lo, mode_hi) of the grid (mode = ix-fastest index of the sine indices,
 * like dof), with no transform: g0_dev holds [2][mode_hi - mode_lo] doubles, the
 * coefficients of G^0 in the orthonormal DST-I basis of every axis (state 1 then
 * state 2), and gN_dev receives those of G^N. In the sine basis of the Dirichlet
 * Laplacian every mode is an independent 2x2 system (Eq. 2.1 with A diagonal), so a
 * range is solved exactly as in fp2s_solve, mode by mode; ranges of one grid can be
 * solved in separate calls (or on separate devices) and concatenated. The result for
 * a mode equals fp2s_solve's before its inverse transform, bit for bit when both
 * calls take the same kernel (the few-mode kernels serve problems with fewer than
 * 9,728 (fast) or 38,912 (direct) modes). Same forms, precisions, flags, status and
 * synchronisation as fp2s_solve; 0 <= mode_lo < mode_hi <= M^dim, else CQ_EINVAL.
 * The workspace size depends on the range length (size query when ws_dev == NULL). */
int fp2s_solve_modes(const fp2s_problem_t *p, int64_t mode_lo, int64_t mode_hi, const double *g0_dev,
                     double *gN_dev, void *ws_dev, size_t *ws_bytes, void *stream);

/* Step-by-step use of the same schemes: fp2s_init transforms G0 and sets up
 * the tables and state in the workspace; fp2s_step(n) advances from t_{n-1}
 * to t_n (n = 1..N in order) and, when G_out_dev != NULL, writes the physical
 * level G^n ([2][M^dim]). */
int fp2s_init(const fp2s_problem_t *p, const double *G0_dev, void *ws_dev, size_t *ws_bytes,
              void *stream);
int fp2s_step(const fp2s_problem_t *p, int64_t n, void *ws_dev, size_t ws_bytes,
              double *G_out_dev, void *stream);
/* Modal levels: g_dev receives the sine coefficients [2][M^dim] of the latest
 * level computed by fp2s_step. */
int fp2s_modal(const fp2s_problem_t *p, const void *ws_dev, size_t ws_bytes, double *g_dev,
               void *stream);
/* Gradient of the final-time misfit J = 1/2 h^dim sum_{s,dof} (G_s^N - Gt_s)^2
 * through the scheme of p (N <= 13000): the discrete adjoint of Eq. 4.1 / Eq. 4.7,
 * i.e. the transposed 2x2 steps run backwards in time with the CQ convolution
 * reversed in time (same weights), and the beta-derivatives of the weights for
 * dJ/dalpha_i = -dJ/dbeta_i.
 * form == CQ_DIRECT, prec == CQ_F64: FP64 throughout; the workspace holds the
 * forward history and the adjoint variables, two [N+1][2][M^dim] FP64 arrays.
 * form == CQ_DIRECT, prec == CQ_DF64: the same sweeps with double-float weights,
 * stored levels and histories (FP64 steps); FP64-class results.
 * form == CQ_FAST, prec == CQ_F64: the adjoint of the fast scheme (recurrences after
 * Eqs. 3.10 / 3.18), which is the direct scheme with the quadrature weights for lags
 * i >= L: the reversed-time history and the weight-derivative history both run as
 * backward geometric recurrences per quadrature node (O(N (np1 + np2)) per mode);
 * the derivatives of the quadrature tables in beta are Richardson-extrapolated
 * central differences of the same table construction (accurate to ~1e-10). The
 * workspace holds the forward levels ([N+1][2][M^dim] FP64) only.
 * form == CQ_FAST, prec == CQ_DF64: the same with the backward recurrences in
 * double-float (the forward sweep and the per-mode sums in FP64); FP64-class
 * results. Sine modes are
 * independent, so a smaller workspace is accepted: the forward and adjoint
 * sweeps then run over slices of modes (the largest multiple of 32 modes whose
 * two arrays fit), with the same results up to the summation order of J and
 * dJ/dalpha. Size query (ws_dev == NULL): *ws_bytes == 0 on input returns the
 * unsliced size; a nonzero *ws_bytes is taken as a cap and the size of the
 * largest slicing within it is returned (CQ_ENOMEM when one 32-mode slice does
 * not fit). The same rule picks the slice size from *ws_bytes at run time.
 * prec == CQ_BF16X3 / CQ_TF32X3: forward and adjoint sweeps of the
 * mixed-precision direct solve (FP32 levels, tensor-core histories), with the
 * weight-derivative history as one more contraction; the workspace holds the
 * split levels and increments (2 x 2 x N x 2 x modes operands) and an FP32
 * [N][2][modes] history. With a smaller workspace the sweeps run over slices of
 * modes (multiples of 64) by the same size-query rule as in FP64. Relative
 * errors of order 1e-5 against the FP64 form.
 * Inputs G0_dev, Gt_dev: physical [2][M^dim]. Outputs: *J_host; dJdG0_dev
 * [2][M^dim] (gradient with respect to the nodal values of G^0); dJdalpha_host[2].
 * Synchronises `stream`. CQ_EUNSUPPORTED for other forms and precisions. */
int fp2s_gradient(const fp2s_problem_t *p, const double *G0_dev, const double *Gt_dev, double *J_host,
                  double *dJdG0_dev, double *dJdalpha_host, void *ws_dev, size_t *ws_bytes, void *stream);
/* Vector-Jacobian product of the solve G^N = fp2s_solve(G^0; alpha1, alpha2):
 * the backward pass for an arbitrary upstream gradient dL/dG^N (physical
 * [2][M^dim], device). Same adjoint sweep as fp2s_gradient with the terminal
 * condition dL/dx^N = S dL/dG^N (S the orthonormal DST-I) instead of the misfit's.
 * Outputs: dG0_dev [2][M^dim] = dL/dG^0 (device); dalpha_host[2] = dL/dalpha_i.
 * Same restrictions, workspace size and errors as fp2s_gradient; synchronises
 * `stream`. */
int fp2s_vjp(const fp2s_problem_t *p, const double *G0_dev, const double *dGN_dev, double *dG0_dev,
             double *dalpha_host, void *ws_dev, size_t *ws_bytes, void *stream);
/* ---- batches: many independent problems in one persistent launch ------- */
/* Plan of a batch (host memory, filled by fp2s_batch_plan; treat as opaque
 * apart from the documented fields). */
typedef struct {
    int32_t n_inst, n_units;        /* problems; work units of 16 * warps_per_block modes */
    int32_t warps_per_block;        /* block width of the persistent kernel (autotuned or default) */
    int32_t max_np, max_L, max_N, max_M, flags;   /* flags bit 0: launch shape chosen by the autotuner;
                                                     bit 1: double-float batch (CQ_DF64) */
    int32_t ctas_per_sm;            /* resident CTAs per SM of the persistent launch (0: as many as fit) */
    int32_t tuned_candidates;       /* launch shapes the autotuner timed (0 without tuning) */
    int32_t node_unroll;            /* partial sums of the node loop: 2, 4 or 8 (autotuned or 4; 0 for CQ_DF64) */
    int64_t max_modes, field_elems; /* field_elems: doubles of a packed [instance][2][M^dim] field */
    int64_t ws_bytes;
    int64_t off[16];                /* workspace regions (internal) */
} fp2s_batch_t;

/* Plans and prepares a batch of n problems (each with form == CQ_FAST,
 * dim 1 or 2; any mix of dim, M, N, scheme, alpha, m and fast sizes; one precision
 * for the whole batch: CQ_F64, or CQ_DF64 with np1 + np2 <= 128, else
 * CQ_EUNSUPPORTED): builds every instance's tables in the workspace with batched
 * kernels and orders the work units by decreasing cost. 1 <= n <= 65535 (more:
 * CQ_EUNSUPPORTED; split such a set into several batches). A CQ_DF64 batch runs the
 * double-float kernel of fp2s_solve over units of 64 modes (flags bit 1 set,
 * warps_per_block 4, no tuning). For CQ_F64, tune != 0 autotunes the launch shape:
 * every block width whose shared memory fits (2..16 warps), each with all and
 * with half of the CTAs per SM that fit and with 2, 4 or 8 partial sums in the
 * node loop, is timed on a shortened run (96 steps, median of three) and the
 * fastest is kept (warps_per_block, ctas_per_sm, node_unroll).
 * Size query when ws_dev == NULL. Synchronises `stream`; the plan and the
 * workspace stay valid for any number of fp2s_solve_batched calls. */
int fp2s_batch_plan(const fp2s_problem_t *probs, int32_t n, int32_t tune, fp2s_batch_t *plan, void *ws_dev,
                    size_t *ws_bytes, void *stream);
/* Solves every planned problem: G0_dev / GN_dev are packed fields, instance i
 * occupying [2][M_i^dim] doubles in plan order. Enqueues five kernels and one
 * memset on `stream` and does not synchronise (it can be captured in a CUDA
 * graph); read the device status with fp2s_batch_status. Calls that overlap on
 * the GPU must use different workspaces. */
int fp2s_solve_batched(const fp2s_batch_t *plan, const double *G0_dev, double *GN_dev, void *ws_dev, void *stream);
int fp2s_batch_status(const fp2s_batch_t *plan, const void *ws_dev, void *stream);

/* Device status of the last fp2s_* work on this workspace (synchronises the stream). */
int fp2s_status(const fp2s_problem_t *p, const void *ws_dev, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FASTCQ_H */
