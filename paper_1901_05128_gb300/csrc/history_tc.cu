// Direct history on the 5th-generation tensor cores (tcgen05), split BF16
// ("BF16x3", kind::f16) or split TF32 ("TF32x3", kind::tf32) operands with FP32
// accumulation in tensor memory.
//
// The direct history of Eq. 3.8 over a range of steps is the product of a
// strictly lower-triangular Toeplitz matrix with the matrix of levels:
//     H[n][dof] = sum_{k=1}^{n-1} d_{n-k} G[k][dof],   n in [n_lo, n_hi).
// With k' = k - 1 (levels 1.. only) this is a GEMM with M = steps, N = DOFs,
// K = levels:  A[m][k'] = d_{m-1-k'} (0 unless m-1-k' >= 1),  B[dof][k'] = G[k'+1][dof].
// Each operand x is split as x = hi + lo with hi = rn(x), lo = rn(x - hi) to 8
// (BF16) or 11 (TF32) significant bits (round to nearest even, computed with
// integer operations: bf16split.h); the product is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term, <= 2^-16 resp. 2^-22
// relative, is dropped; the split itself leaves <= 2^-16 resp. 2^-22 of x).
// Both forms use the same shared-memory tiles: a 128-byte swizzle row holds 64
// BF16 or 32 TF32 levels, and one MMA instruction consumes 32 bytes of K.
//
// A 128 x 64 tile of A at rows m0.. and columns k0'.. depends only on
// delta = m0 - 1 - k0', so the distinct tiles are precomputed once per call
// into a small bank (L2-resident) and streamed by TMA like any operand. G is
// split and transposed once into K-major BF16 arrays.
//
// Kernel: one CTA per SM over 128 x 256 output tiles; warp 0 issues TMA loads into a
// two-stage shared-memory ring, warp 1 issues tcgen05.mma (one thread) into two
// 128 x 256 FP32 accumulators in tensor memory, one chunk of levels at a time
// (128 BF16 levels, 32 TF32 levels), alternating; warps 2-9 read each finished chunk
// back with tcgen05.ld and add it to FP32 running sums (round to nearest) while the
// next chunk is being formed, then store FP64 (or FP32) results. The tensor cores'
// own accumulation rounds toward zero: every MMA instruction that adds to an
// accumulator of size |S| loses up to ulp(S) toward zero, and on a history whose
// terms share a sign these losses are a bias that a time-stepping scheme repeats
// at every step. Chunking keeps it to one chunk's worth, and within a stage the
// small products (hi*lo, lo*hi, 2^-8 resp. 2^-11 of the result) are issued before
// the hi*hi products, while the accumulator is still small: per TF32 chunk only
// the four hi*hi instructions truncate a value of the chunk's full size (instead
// of all twelve, or 48 in a 128-level chunk). Every mbarrier wait
// is bounded by a global-timer deadline; on expiry the kernel records
// ST_TIMEOUT, writes NaN to its tile, drains what it started and frees its
// tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include "bf16split.h"
#include "common.cuh"
#include "tc.cuh"

namespace fastcq {
namespace tc {

constexpr int STAGES = 2;
constexpr int ROW_BYTES = 128;              // one swizzle row of K per operand row and stage
constexpr int A_BYTES = BM * ROW_BYTES;     // 16 KiB
constexpr int B_BYTES = BN * ROW_BYTES;     // 32 KiB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int EPI_WARPS = 8;                // two warps per TMEM lane quarter, one per column half
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int TMEM_COLS = 512;              // two 128 x 256 FP32 accumulators
// levels accumulated per tensor-memory pass (see the truncation note above)
__host__ __device__ constexpr int chunk_levels(int kind) { return kind == TC_TF32X3 ? 32 : 128; }
constexpr int STG_FLOATS = 32 * 33;          // per epilogue warp: a 32 x 32 block, padded rows
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 256 + (size_t)EPI_WARPS * STG_FLOATS * 4;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s per wait
constexpr int TQ = 4;                       // tile ring entries (claimed tiles in flight in a CTA)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of the phase with the given parity. Gives up
// after limit_ns, or at once when any CTA has already recorded a timeout (so a
// failure ends the whole grid quickly instead of every CTA waiting in turn).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns,
                                          const int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
        if (*(const volatile int *)status & ST_TIMEOUT) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptors: FP32 accumulator (bits 4-5), A and B format (bits 7-9, 10-12:
// BF16 = 1 under kind::f16, TF32 = 2 under kind::tf32), both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc(int fmt) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    if constexpr (KIND == TC_TF32X3) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc(2)), "r"(accumulate));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc(1)), "r"(accumulate));
    }
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// FP32 -> FP64 by bit manipulation on the integer pipe (on GB300 the FP64 unit
// that would otherwise convert is ~60x slower than FP32). FP32 subnormals
// (|x| < 2^-126) become signed zero; Inf / NaN are kept.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint64_t man = (uint64_t)(u & 0x7fffffu) << 29;
    uint64_t bits;
    if (e == 0u) bits = sign;
    else if (e == 0xffu) bits = sign | (0x7ffull << 52) | man;
    else bits = sign | ((uint64_t)(e + 896u) << 52) | man;
    return __longlong_as_double((long long)bits);
}

// One output element. Add mode (FP32 output only): a reduction without return value; each
// element receives exactly one addition per launch, so the sum is that of a load-add-store,
// without holding the old value or waiting for it.
__device__ __forceinline__ void store1(float *dst, float v, int add) {
    if (add) atomicAdd(dst, v);
    else *dst = v;
}
__device__ __forceinline__ void store1(double *dst, float v, int) { *dst = f32_to_f64_bits(v); }

// Geometry of output tile b (tiles of one column tile are consecutive, longest K first).
struct TileGeom {
    int state, num_k, nchunks;
    int64_t m0, n0, brow;
};

template <int KIND>
__device__ __forceinline__ TileGeom tile_geom(const TcParams &P, int64_t b) {
    constexpr int BKK = kind_bk(KIND);
    constexpr int CHUNK = chunk_levels(KIND) / BKK;
    TileGeom g;
    const int64_t ntile = b / P.num_i;
    g.state = (int)(ntile / P.ntile_state);
    const int nt = (int)(ntile % P.ntile_state);
    const int it = P.num_i - 1 - (int)(b % P.num_i);
    g.m0 = P.n_lo + (int64_t)it * BM;                      // first step of the tile
    g.n0 = (int64_t)nt * BN;                               // first DOF of the tile (within its state)
    g.brow = (int64_t)g.state * P.state_stride + g.n0;     // first row of the levels operand
    const int64_t m_last = min(g.m0 + BM - 1, P.n_lo + P.rows - 1);
    // levels k' < m_last - 1 contribute (k = k' + 1 <= m_last - 1)
    const int64_t k_end = min((int64_t)P.kprime, m_last - 1);
    g.num_k = k_end > P.k_lo ? (int)((k_end - P.k_lo + BKK - 1) / BKK) : 0;
    g.nchunks = (g.num_k + CHUNK - 1) / CHUNK;
    return g;
}

// A CTA takes the output tiles blockIdx.x, blockIdx.x + gridDim.x, ...: one tile when the
// grid has a CTA per tile, several when the host launches fewer CTAs (tiles of equal K:
// one CTA per SM, the next tile's loads and MMAs overlapping the previous tile's epilogue).
// With a tile counter (tiles of unequal K) the CTA's first tile is blockIdx.x and the
// producer thread claims each further one from the counter, so a CTA that finishes early
// takes the next tile in order; it hands the tile numbers to the MMA thread and the
// epilogue warps through a ring of TQ entries in shared memory. Stages and accumulator
// chunks are counted across the CTA's tiles, so the mbarrier phases run on without a
// reset between tiles.
template <typename OutT, int KIND>
__global__ void __launch_bounds__(THREADS, 1) k_history_tc(const __grid_constant__ TcMaps maps, TcParams P,
                                                          OutT *__restrict__ H, int *__restrict__ status) {
    constexpr int BKK = kind_bk(KIND);                          // levels per stage
    constexpr int CHUNK = chunk_levels(KIND) / BKK;             // stages per accumulator chunk
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;            // accumulator buffer b holds a finished chunk
    uint64_t *tempty = tfull + 2;                // accumulator buffer b has been read back
    uint64_t *drain = tempty + 2;                // every MMA this CTA issued has completed
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drain + 1);
    int *abort_flag = reinterpret_cast<int *>(tmem_holder + 1);   // [0]: abort, [1]: always 0
    uint64_t *tq_full = drain + 3;               // ring entry holds a claimed tile number
    uint64_t *tq_empty = tq_full + TQ;           // ring entry read by the MMA thread and every epilogue warp
    int64_t *tq = reinterpret_cast<int64_t *>(tq_empty + TQ);
    const bool dyn = P.tile_counter != nullptr;
    const unsigned long long wlim = P.wait_ns ? P.wait_ns : WAIT_NS;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total = P.ntile_state * P.n_states * P.num_i;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&tfull[q], 1);
            mbar_init(&tempty[q], 32 * EPI_WARPS);
        }
        mbar_init(drain, 1);
        for (int i = 0; i < TQ; ++i) {
            mbar_init(&tq_full[i], 1);
            mbar_init(&tq_empty[i], 1 + EPI_WARPS);
        }
        abort_flag[0] = (*(const volatile int *)status & ST_TIMEOUT) ? 1 : 0;   // an earlier CTA gave up
        abort_flag[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    const bool aborted = *(volatile int *)abort_flag != 0;
    if (warp == 0 && lane == 0 && !aborted) {
        // ---------------- TMA producer
        int64_t armed[STAGES];
        for (int i = 0; i < STAGES; ++i) armed[i] = -1;
        int64_t gks = 0;                                  // stages issued by this CTA so far
        bool stop = false;
        for (int64_t t = 0; !stop; ++t) {
            int64_t b = blockIdx.x + t * gridDim.x;
            if (dyn) {
                const int slot = (int)(t % TQ);
                if (!mbar_wait(&tq_empty[slot], ((uint32_t)(t / TQ) & 1u) ^ 1u, wlim, status)) {
                    atomicOr(status, ST_TIMEOUT);
                    *(volatile int *)abort_flag = 1;
                    break;
                }
                b = t == 0 ? (int64_t)blockIdx.x : (int64_t)gridDim.x + atomicAdd(P.tile_counter, 1);
                *(volatile int64_t *)&tq[slot] = b;
                mbar_arrive(&tq_full[slot]);                  // b >= total tells the others to finish
            }
            if (b >= total) break;
            const TileGeom g = tile_geom<KIND>(P, b);
            const CUtensorMap *tA_hi = &maps.a_hi[g.state], *tA_lo = &maps.a_lo[g.state];
            for (int ks = 0; ks < g.num_k; ++ks, ++gks) {
                const int s = (int)(gks % STAGES);
                const uint32_t ph = (uint32_t)(gks / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, wlim, status)) {
                    atomicOr(status, ST_TIMEOUT);
                    *(volatile int *)abort_flag = 1;
                    stop = true;
                    break;
                }
                if (*(volatile int *)abort_flag) {
                    stop = true;
                    break;
                }
                if (P.test_stall && gks == 0) continue;           // never armed: the MMA thread's wait expires
                unsigned char *st = smem + s * STAGE_BYTES;
                const int kc = P.k_lo + ks * BKK;                 // first level column of the stage
                const int64_t delta = g.m0 - 1 - (int64_t)kc;
                const int arow = (int)((delta - P.delta0) / BKK) * BM;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(st, tA_hi, &full[s], 0, arow);
                tma_load_2d(st + A_BYTES, tA_lo, &full[s], 0, arow);
                tma_load_2d(st + 2 * A_BYTES, &maps.b_hi, &full[s], kc, (int)g.brow);
                tma_load_2d(st + 2 * A_BYTES + B_BYTES, &maps.b_lo, &full[s], kc, (int)g.brow);
                armed[s] = gks;
            }
        }
        if (*(volatile int *)abort_flag) {
            // drain the loads this thread started before the CTA releases its shared memory
            for (int i = 0; i < STAGES; ++i)
                if (armed[i] >= 0) (void)mbar_wait(&full[i], (uint32_t)(armed[i] / STAGES) & 1u, WAIT_NS, abort_flag + 1);
        }
    } else if (warp == 1 && lane == 0 && !aborted) {
        // ---------------- MMA issuer: chunk c (counted over the CTA's tiles) of CHUNK stages goes
        // to accumulator buffer c & 1, starting from zero, once the epilogue has read back that
        // buffer's previous chunk
        int64_t gks = 0, gc = 0;
        bool stop = false;
        for (int64_t t = 0; !stop; ++t) {
            int64_t b = blockIdx.x + t * gridDim.x;
            if (dyn) {
                const int slot = (int)(t % TQ);
                if (!mbar_wait(&tq_full[slot], (uint32_t)(t / TQ) & 1u, wlim, status)) {
                    atomicOr(status, ST_TIMEOUT);
                    *(volatile int *)abort_flag = 1;
                    break;
                }
                b = *(volatile int64_t *)&tq[slot];
                mbar_arrive(&tq_empty[slot]);
            }
            if (b >= total) break;
            const TileGeom g = tile_geom<KIND>(P, b);
            for (int ks = 0; ks < g.num_k; ++ks, ++gks) {
                const int s = (int)(gks % STAGES);
                const uint32_t ph = (uint32_t)(gks / STAGES) & 1u;
                const int64_t c = gc + ks / CHUNK;
                const int buf = (int)(c & 1);
                if (ks % CHUNK == 0) {
                    if (!mbar_wait(&tempty[buf], ((uint32_t)(c >> 1) & 1u) ^ 1u, wlim, status) ||
                        *(volatile int *)abort_flag) {
                        atomicOr(status, ST_TIMEOUT);
                        *(volatile int *)abort_flag = 1;
                        stop = true;
                        break;
                    }
                }
                if (!mbar_wait(&full[s], ph, wlim, status) || *(volatile int *)abort_flag) {
                    atomicOr(status, ST_TIMEOUT);
                    *(volatile int *)abort_flag = 1;
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t a_hi = sa, a_lo = sa + A_BYTES, b_hi = sa + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
                const uint32_t acc = tmem + (uint32_t)(buf * BN);
                // one MMA: 32 bytes along K (16 BF16 or 8 TF32); the small products of the
                // stage first, the first of a chunk starting the accumulator from zero
#pragma unroll
                for (int kk = 0; kk < ROW_BYTES / 32; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint32_t acc0 = (ks % CHUNK > 0 || kk > 0) ? 1u : 0u;
                    umma<KIND>(acc, sdesc(a_hi + off), sdesc(b_lo + off), acc0);
                    umma<KIND>(acc, sdesc(a_lo + off), sdesc(b_hi + off), 1u);
                }
#pragma unroll
                for (int kk = 0; kk < ROW_BYTES / 32; ++kk) {
                    const uint32_t off = kk * 32;
                    umma<KIND>(acc, sdesc(a_hi + off), sdesc(b_hi + off), 1u);
                }
                umma_commit(&empty[s]);                       // stage reusable once these MMAs are done
                if (ks % CHUNK == CHUNK - 1 || ks == g.num_k - 1) umma_commit(&tfull[buf]);
            }
            gc += g.nchunks;
        }
        umma_commit(drain);                               // everything issued above has completed
    } else if (warp >= 2) {
        // ---------------- epilogue: each chunk is read back from tensor memory and added to
        // FP32 running sums with round-to-nearest (the tensor-core accumulation within a chunk
        // rounds toward zero; summing chunks here keeps that bias to one chunk's worth)
        const int q = warp & 3;                           // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;                 // columns [128 half, 128 half + 128)
        float *stg = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES + 256) + (warp - 2) * STG_FLOATS;
        bool have = !aborted;
        int64_t gc = 0;
        for (int64_t t = 0;; ++t) {
            int64_t b = blockIdx.x + t * gridDim.x;
            if (dyn) {
                // lane 0 takes the tile number from the ring and passes it to the warp
                const int slot = (int)(t % TQ);
                int ok = 0;
                long long bb = 0;
                if (lane == 0 && have) {
                    ok = mbar_wait(&tq_full[slot], (uint32_t)(t / TQ) & 1u, wlim, status) ? 1 : 0;
                    if (ok) {
                        bb = *(volatile int64_t *)&tq[slot];
                        mbar_arrive(&tq_empty[slot]);
                    } else {
                        atomicOr(status, ST_TIMEOUT);
                        *(volatile int *)abort_flag = 1;
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
                b = __shfl_sync(0xffffffffu, bb, 0);
            }
            if (b >= total) break;
            const TileGeom g = tile_geom<KIND>(P, b);
            float accr[BN / 2];
#pragma unroll
            for (int i = 0; i < BN / 2; ++i) accr[i] = 0.0f;
            for (int c = 0; c < g.nchunks; ++c) {
                const int64_t cc = gc + c;
                const int buf = (int)(cc & 1);
                if (have) {
                    have = mbar_wait(&tfull[buf], (uint32_t)(cc >> 1) & 1u, wlim, status);
                    if (!have) {
                        atomicOr(status, ST_TIMEOUT);
                        *(volatile int *)abort_flag = 1;
                    }
                }
                if (have) {
                    tc_fence_after();
                    const uint32_t base =
                        tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + half * (BN / 2));
#pragma unroll
                    for (int j = 0; j < BN / 2; j += 16) {
                        float v[16];
                        tmem_ld16(base + (uint32_t)j, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) accr[j + i] += v[i];
                    }
                    tc_fence_before();
                }
                mbar_arrive(&tempty[buf]);
            }
            gc += g.nchunks;
            // the warp's 32 rows x 128 columns, in 32 x 32 blocks transposed through shared
            // memory so that each store instruction writes 32 consecutive columns of one row
            const int64_t row0 = g.m0 + q * 32;
            OutT *hbase = H + (row0 - P.n_lo) * P.ldh + (int64_t)g.state * P.state_stride;
            const float nanf_ = __int_as_float(0x7fc00000);
#pragma unroll
            for (int j = 0; j < BN / 2; j += 32) {
#pragma unroll
                for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = have ? accr[j + i] : nanf_;
                __syncwarp();
                const int64_t col = g.n0 + half * (BN / 2) + j + lane;
                const int rmax = (int)min((int64_t)32, P.n_lo + P.rows - row0);
                if (col < P.ndof) {
#pragma unroll 8
                    for (int r = 0; r < 32; ++r)
                        if (r < rmax) store1(hbase + (int64_t)r * P.ldh + col, stg[r * 33 + lane], P.add);
                }
                __syncwarp();
            }
            if (!have) break;                             // this tile holds NaN; the grid is draining
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        // nothing may still write tensor memory when it is freed
        if (!aborted && lane == 0) (void)mbar_wait(drain, 0, WAIT_NS, abort_flag + 1);
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Fast form of the split for FP64 exponents in [949, 1149] (2^-74 <= |x| < 2^127), bit-identical
// to the integer-only split of bf16split.h, which serves every other value:
//   t  = x rounded to odd at 24 significant bits, an FP32 bit pattern assembled from the FP64
//        fields (truncate, then set the last bit when any dropped bit is set);
//   hi = t rounded to nearest-even at 8 (BF16) or 11 (TF32) bits, which equals x rounded so
//        directly (rounding to odd with at least two extra bits, then to nearest, rounds once);
//   r  = x - hi, exact in FP64 (|r| <= 2^-8 |x| and both are multiples of x's last bit), so one
//        FP64 subtraction; lo = r rounded the same way (r is 0 or at least 2^-126 here).
__device__ __forceinline__ uint32_t ro24_bits(uint32_t hw, uint32_t lw) {
    // (hw:lw) << 3 keeps the exponent's low 9 bits; rebiasing by 896 modulo 2^32 is exact for
    // biased exponents 897 .. 1150
    const uint32_t t = __funnelshift_l(lw, hw, 3) - (896u << 23);
    return t | (hw & 0x80000000u) | ((lw & 0x1fffffffu) != 0u ? 1u : 0u);
}
__device__ __forceinline__ uint32_t rn_bf16_of_f32bits(uint32_t u) { return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16; }
__device__ __forceinline__ uint32_t rn_tf32_of_f32bits(uint32_t u) {
    return (u + 0xfffu + ((u >> 13) & 1u)) & 0xffffe000u;
}
__device__ __forceinline__ bool split_fast_range(uint32_t hw) {
    const uint32_t ex = (hw >> 20) & 0x7ffu;
    return ex >= 949u && ex <= 1149u;
}
__device__ __forceinline__ uint32_t dhi(double x) { return (uint32_t)((unsigned long long)__double_as_longlong(x) >> 32); }
__device__ __forceinline__ uint32_t dlo(double x) { return (uint32_t)__double_as_longlong(x); }

// Element of a hi / lo pair: BF16 bits or TF32 (FP32 bits with 13 low zero bits).
template <int KIND> struct Elem;
template <> struct Elem<TC_BF16X3> {
    using T = uint16_t;
    __device__ static void split(double v, T &h, T &l) {
        const uint32_t hw = dhi(v), lw = dlo(v);
        if (!split_fast_range(hw)) {
            bf16_split(v, &h, &l);
            return;
        }
        const uint32_t h16 = rn_bf16_of_f32bits(ro24_bits(hw, lw));
        const uint32_t hh = (((h16 & 0x7fffu) << 13) + (896u << 20)) | ((h16 & 0x8000u) << 16);
        const double r = __dsub_rn(v, __hiloint2double((int)hh, 0));
        const uint32_t rw = dhi(r), rl = dlo(r);
        h = (T)h16;
        l = ((rw & 0x7fffffffu) | rl) ? (T)rn_bf16_of_f32bits(ro24_bits(rw, rl)) : (T)0;
    }
};
template <> struct Elem<TC_TF32X3> {
    using T = uint32_t;
    __device__ static void split(double v, T &h, T &l) {
        const uint32_t hw = dhi(v), lw = dlo(v);
        if (!split_fast_range(hw)) {
            tf32_split(v, &h, &l);
            return;
        }
        const uint32_t h32 = rn_tf32_of_f32bits(ro24_bits(hw, lw));
        const uint32_t hh = (((h32 & 0x7fffffffu) >> 3) + (896u << 20)) | (h32 & 0x80000000u);
        const double r = __dsub_rn(v, __hiloint2double((int)hh, 0));
        const uint32_t rw = dhi(r), rl = dlo(r);
        h = h32;
        l = ((rw & 0x7fffffffu) | rl) ? rn_tf32_of_f32bits(ro24_bits(rw, rl)) : 0u;
    }
};

// Bank of Toeplitz tiles: tile t, row r, column c holds d_{delta0 + BK t + r - c} when
// that index lies in [1, nw], else 0; split into hi + lo.
template <int KIND>
__global__ void k_toeplitz_bank(const double *__restrict__ d, int64_t nw, int64_t delta0, int ntiles,
                                typename Elem<KIND>::T *__restrict__ hi, typename Elem<KIND>::T *__restrict__ lo) {
    constexpr int BKK = kind_bk(KIND);
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ntiles * BM * BKK) return;
    const int c = (int)(e % BKK);
    const int64_t rr = e / BKK;                  // t * BM + r
    const int r = (int)(rr % BM);
    const int64_t t = rr / BM;
    const int64_t q = delta0 + BKK * t + r - c;
    const double v = (q >= 1 && q <= nw) ? d[q] : 0.0;
    typename Elem<KIND>::T h, l;
    Elem<KIND>::split(v, h, l);
    hi[e] = h;
    lo[e] = l;
}

// Gt[dof][k'] = split(G[k' + 1][dof]) for k' < kprime, 0 for kprime <= k' < kpad.
// Tile of 64 levels (blockIdx.x) x 32 DOFs (blockIdx.y, and every gridDim.y-th after it when
// there are more DOF tiles than grid rows): coalesced FP64 row reads, then every thread writes
// a pair of elements (a warp stores 128 or 256 contiguous bytes per array). One CTA per tile in
// launch order keeps the CTAs in flight on neighbouring tiles (a persistent version whose
// CTAs loop over tiles was slower on large inputs: they drift apart in memory).
template <int KIND>
__global__ void __launch_bounds__(256) k_split_transpose(const double *__restrict__ G, int64_t ldg, int64_t ndof,
                                                         int kprime, int kpad, typename Elem<KIND>::T *__restrict__ hi,
                                                         typename Elem<KIND>::T *__restrict__ lo) {
    using T = typename Elem<KIND>::T;
    __shared__ double tile[32][65];                 // [dof][level]
    const int k0 = blockIdx.x * 64;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int64_t d0 = (int64_t)blockIdx.y * 32; d0 < ndof; d0 += (int64_t)gridDim.y * 32) {
        for (int j = ty; j < 64; j += 8) {
            const int k = k0 + j;
            const int64_t dof = d0 + tx;
            tile[tx][j] = (k < kprime && dof < ndof) ? G[(int64_t)(k + 1) * ldg + dof] : 0.0;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int64_t dof = d0 + r;
            if (dof >= ndof) break;
            T h0, l0, h1, l1;
            Elem<KIND>::split(tile[r][2 * tx], h0, l0);
            Elem<KIND>::split(tile[r][2 * tx + 1], h1, l1);
            const int64_t o = dof * kpad + k0 + 2 * tx;
            if constexpr (KIND == TC_TF32X3) {
                *reinterpret_cast<uint2 *>(hi + o) = make_uint2(h0, h1);
                *reinterpret_cast<uint2 *>(lo + o) = make_uint2(l0, l1);
            } else {
                *reinterpret_cast<uint32_t *>(hi + o) = (uint32_t)h0 | ((uint32_t)h1 << 16);
                *reinterpret_cast<uint32_t *>(lo + o) = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
        }
        __syncthreads();                            // the tile is refilled for the next DOF tile
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2D tensor [rows][cols] of the kind's elements (cols contiguous, pitch in elements),
// box {128 bytes of columns, box_rows}, 128-byte swizzle.
static int make_map(int kind, CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t pitch,
                    uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return CQ_ECUDA;
    const int es = kind_esize(kind);
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {pitch * (uint64_t)es};
    const cuuint32_t box[2] = {(cuuint32_t)kind_bk(kind), box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = kind == TC_TF32X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUresult r = fn(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CQ_OK : CQ_ECUDA;
}

struct TcLayout {
    int *status;
    double *d;
    char *a_hi, *a_lo, *g_hi, *g_lo;
    int ntiles, kpad;
    int64_t delta0;
    size_t bytes;
};

static TcLayout tc_layout(int kind, void *ws, int64_t ndof, int64_t n_lo, int64_t n_hi) {
    TcLayout l{};
    const int bk = kind_bk(kind), es = kind_esize(kind);
    const int64_t kprime = n_hi - 2 > 0 ? n_hi - 2 : 0;
    l.kpad = (int)(((kprime + 63) / 64) * 64);      // multiple of the split tile (64 levels)
    if (l.kpad == 0) l.kpad = 64;
    const int64_t rows = n_hi - n_lo;
    const int64_t num_i = (rows + BM - 1) / BM;
    // delta = m0 - 1 - bk j over tiles i (m0 = n_lo + 128 i) and K-steps j; smallest at i = 0, largest j
    const int64_t jmax0 = l.kpad / bk;
    l.delta0 = n_lo - 1 - bk * jmax0;
    const int64_t dmax = n_lo - 1 + BM * (num_i > 0 ? num_i - 1 : 0);
    l.ntiles = (int)((dmax - l.delta0) / bk + 1);
    Carve cv(ws);
    l.status = cv.take<int>(64);
    l.d = cv.take<double>(n_hi + BM + 2);
    l.a_hi = cv.take<char>((size_t)l.ntiles * BM * bk * es);
    l.a_lo = cv.take<char>((size_t)l.ntiles * BM * bk * es);
    l.g_hi = cv.take<char>((size_t)ndof * l.kpad * es);
    l.g_lo = cv.take<char>((size_t)ndof * l.kpad * es);
    l.bytes = cv.bytes();
    return l;
}

static int tc_attr() {
    static unsigned long long done[4] = {};
    const int sm = (int)SMEM_BYTES;
    int st;
    if ((st = smem_attr_once((const void *)k_history_tc<double, TC_BF16X3>, sm, &done[0])) ||
        (st = smem_attr_once((const void *)k_history_tc<float, TC_BF16X3>, sm, &done[1])) ||
        (st = smem_attr_once((const void *)k_history_tc<double, TC_TF32X3>, sm, &done[2])) ||
        (st = smem_attr_once((const void *)k_history_tc<float, TC_TF32X3>, sm, &done[3])))
        return st;
    return CQ_OK;
}

template <int KIND>
static void launch_bank(const double *d, int64_t nw, int64_t delta0, int ntiles, void *hi, void *lo, cudaStream_t s) {
    using T = typename Elem<KIND>::T;
    const int64_t elems = (int64_t)ntiles * BM * kind_bk(KIND);
    k_toeplitz_bank<KIND><<<(unsigned)((elems + 255) / 256), 256, 0, s>>>(d, nw, delta0, ntiles,
                                                                           static_cast<T *>(hi), static_cast<T *>(lo));
}

}  // namespace tc

// Failure-path test switch (cq_test_expire_waits): launches withhold their first operand load
// and wait at most 10 ms, so the bounded waits expire and the error path runs.
static int g_test_expire = 0;
static void apply_test_switch(tc::TcParams &P) {
    if (g_test_expire) {
        P.test_stall = 1;
        P.wait_ns = 10000000ull;
    }
}

size_t history_tc_workspace(int kind, int64_t ndof, int64_t n_lo, int64_t n_hi) {
    return tc::tc_layout(kind, nullptr, ndof, n_lo, n_hi).bytes;
}

int history_tc_run(int kind, int scheme, double beta, double tau, int64_t ndof, int64_t n_lo, int64_t n_hi,
                   const double *G, int64_t ldg, double *H, int64_t ldh, void *ws, cudaStream_t s) {
    using namespace tc;
    TcLayout l = tc_layout(kind, ws, ndof, n_lo, n_hi);
    const int64_t nw = n_hi + BM;
    if (nw > kMaxWeights) return CQ_EUNSUPPORTED;
    if (ndof > ((int64_t)1 << 31) - BN) return CQ_EUNSUPPORTED;
    int st;
    if ((st = cuda_status(cudaMemsetAsync(l.status, 0, 64 * sizeof(int), s)))) return st;
    if ((st = launch_weights(scheme, beta, tau, nw, l.d, s))) return st;
    if ((st = tc_bank(kind, l.d, n_hi, l.delta0, l.ntiles, l.a_hi, l.a_lo, s))) return st;
    const int kprime = (int)(n_hi - 2 > 0 ? n_hi - 2 : 0);
    const int64_t ndt = (ndof + 31) / 32;
    const dim3 tg((unsigned)(l.kpad / 64), (unsigned)min(ndt, (int64_t)65535));
    if (kind == TC_TF32X3)
        k_split_transpose<TC_TF32X3><<<tg, dim3(32, 8), 0, s>>>(G, ldg, ndof, kprime, l.kpad,
                                                                 reinterpret_cast<uint32_t *>(l.g_hi),
                                                                 reinterpret_cast<uint32_t *>(l.g_lo));
    else
        k_split_transpose<TC_BF16X3><<<tg, dim3(32, 8), 0, s>>>(G, ldg, ndof, kprime, l.kpad,
                                                                 reinterpret_cast<uint16_t *>(l.g_hi),
                                                                 reinterpret_cast<uint16_t *>(l.g_lo));
    if ((st = launched())) return st;
    TcMaps maps;
    if ((st = tc_map_bank(kind, &maps.a_hi[0], l.a_hi, l.ntiles))) return st;
    if ((st = tc_map_bank(kind, &maps.a_lo[0], l.a_lo, l.ntiles))) return st;
    maps.a_hi[1] = maps.a_hi[0];
    maps.a_lo[1] = maps.a_lo[0];
    if ((st = tc_map_levels(kind, &maps.b_hi, l.g_hi, l.kpad, ndof))) return st;
    if ((st = tc_map_levels(kind, &maps.b_lo, l.g_lo, l.kpad, ndof))) return st;
    TcParams P{};
    P.ndof = ndof;
    P.n_lo = n_lo;
    P.rows = n_hi - n_lo;
    P.ldh = ldh;
    P.num_i = (int)((P.rows + BM - 1) / BM);
    P.delta0 = l.delta0;
    P.kprime = kprime;
    P.k_lo = 0;
    P.add = 0;
    const int64_t num_n = (ndof + BN - 1) / BN;
    P.n_states = 1;
    P.ntile_state = num_n;
    P.state_stride = 0;
    const int64_t tiles = num_n * P.num_i;
    if (tiles > 0x7fffffffLL - 65536) return CQ_EUNSUPPORTED;
    // one CTA per SM; tiles have unequal K (a causal triangle), so they are claimed in order
    // from a counter (zeroed with the status words above)
    P.max_ctas = device_sms();
    P.tile_counter = l.status + 32;
    apply_test_switch(P);
    const int64_t blocks = min(tiles, P.max_ctas);
    if ((st = tc_attr())) return st;
    if ((st = timing_begin(s))) return st;
    if (kind == TC_TF32X3)
        k_history_tc<double, TC_TF32X3><<<(unsigned)blocks, THREADS, SMEM_BYTES, s>>>(maps, P, H, l.status);
    else
        k_history_tc<double, TC_BF16X3><<<(unsigned)blocks, THREADS, SMEM_BYTES, s>>>(maps, P, H, l.status);
    if ((st = launched())) return st;
    return timing_end(s);
}

namespace tc {
template <int KIND>
__global__ void k_split(const double *__restrict__ x, int64_t n, typename Elem<KIND>::T *__restrict__ hi,
                        typename Elem<KIND>::T *__restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    typename Elem<KIND>::T h, l;
    Elem<KIND>::split(x[i], h, l);
    hi[i] = h;
    lo[i] = l;
}
}  // namespace tc

int tc_bank(int kind, const double *d, int64_t nw, int64_t delta0, int ntiles, void *hi, void *lo, cudaStream_t s) {
    using namespace tc;
    if (ntiles <= 0) return CQ_EINVAL;
    if (kind == TC_TF32X3) launch_bank<TC_TF32X3>(d, nw, delta0, ntiles, hi, lo, s);
    else launch_bank<TC_BF16X3>(d, nw, delta0, ntiles, hi, lo, s);
    return launched();
}

int tc_map_bank(int kind, CUtensorMap *m, const void *bank, int ntiles) {
    using namespace tc;
    const int bk = kind_bk(kind);
    return make_map(kind, m, bank, bk, (uint64_t)ntiles * BM, bk, BM);
}

int tc_map_levels(int kind, CUtensorMap *m, const void *levels, int64_t kpad, int64_t rows) {
    using namespace tc;
    if (kpad % 64) return CQ_EINVAL;
    return make_map(kind, m, levels, (uint64_t)kpad, (uint64_t)rows, (uint64_t)kpad, BN);
}

int tc_contract_f32(int kind, const tc::TcMaps &maps, const tc::TcParams &Pin, float *H, int *status,
                    cudaStream_t s) {
    using namespace tc;
    TcParams P = Pin;
    apply_test_switch(P);
    const int64_t tiles = P.ntile_state * P.n_states * P.num_i;
    if (tiles <= 0 || tiles > 0x7fffffffLL - 65536) return CQ_EUNSUPPORTED;
    if (P.tile_counter && P.max_ctas <= 0) return CQ_EINVAL;
    const int64_t blocks = P.max_ctas > 0 ? min(tiles, P.max_ctas) : tiles;
    int st;
    if ((st = tc_attr())) return st;
    if (kind == TC_TF32X3)
        k_history_tc<float, TC_TF32X3><<<(unsigned)blocks, THREADS, SMEM_BYTES, s>>>(maps, P, H, status);
    else
        k_history_tc<float, TC_BF16X3><<<(unsigned)blocks, THREADS, SMEM_BYTES, s>>>(maps, P, H, status);
    return launched();
}

}  // namespace fastcq

extern "C" int cq_split(int32_t prec, const double *x_dev, int64_t n, void *hi_dev, void *lo_dev, void *stream) {
    using namespace fastcq;
    if (n < 0) return CQ_EINVAL;
    if (prec != CQ_BF16X3 && prec != CQ_TF32X3) return CQ_EUNSUPPORTED;
    if (n == 0) return CQ_OK;
    if (!x_dev || !hi_dev || !lo_dev) return CQ_EINVAL;
    if (n > (int64_t)0x7fffffff * 256) return CQ_EUNSUPPORTED;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == CQ_TF32X3)
        tc::k_split<tc::TC_TF32X3><<<blocks, 256, 0, s>>>(x_dev, n, static_cast<uint32_t *>(hi_dev),
                                                         static_cast<uint32_t *>(lo_dev));
    else
        tc::k_split<tc::TC_BF16X3><<<blocks, 256, 0, s>>>(x_dev, n, static_cast<uint16_t *>(hi_dev),
                                                         static_cast<uint16_t *>(lo_dev));
    return launched();
}

extern "C" int cq_test_expire_waits(int on) {
    fastcq::g_test_expire = on != 0;
    return CQ_OK;
}
