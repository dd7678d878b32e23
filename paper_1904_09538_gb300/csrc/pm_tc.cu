// BF16-in / FP32-accumulate tensor-core matmul on the 5th-generation tensor
// cores (tcgen05): C[M x N] = A[M x K] * Bt[N x K]^T, A and Bt row-major
// (both K-major, the usual tensor-core "TN" layout), C row-major FP32.
//
// One CTA of 128 threads computes a 128 x 256 tile of C:
//   warp 0 lane 0: TMA producer -- per 64-wide k tile, one 128x64 tile of A
//       and one 256x64 tile of Bt (128-byte swizzle) into a shared-memory
//       ring of STAGES stages, completion tracked by "full" mbarriers;
//   warp 1 lane 0: MMA issuer -- four tcgen05.mma (M=128, N=256, K=16) per k
//       tile accumulating in tensor memory; tcgen05.commit releases the
//       stage ("empty" mbarrier) and finally signals the accumulator;
//   warp 2: allocates / frees 256 TMEM columns;
//   all four warps: epilogue -- tcgen05.ld of their 32 TMEM lanes (= rows),
//       16-byte stores to C.
// Two pipeline shapes: 4 stages with one CTA per SM, or 2 stages with two
// CTAs per SM (2 x 256 TMEM columns), where one CTA's epilogue overlaps the
// other's main loop.  CTAs are numbered in groups of 16 tile rows sharing a
// sweep over the tile columns, so that concurrently resident CTAs reuse the
// same A and Bt tiles from L2.
// Every mbarrier wait is bounded; on timeout the kernel sets an error word
// (read by the host after synchronising), stops issuing work, drains its own
// copies (bounded), frees its TMEM and returns.
#include <algorithm>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "pm_internal.h"
#include "pm_tma.cuh"

namespace pm {

static __device__ int g_tc_timeout;   // set to 1 by any CTA whose bounded wait ran out

namespace {

constexpr int TM = 128, TN = 256, TK = 64, GROUP_M = 16;
constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 1ll << 26;  // polls of a try_wait before giving up

// bounded wait on this kernel's error word
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    return mbar_wait_bounded(bar, parity, &g_tc_timeout, WAIT_LIMIT);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;            // start address, bits 0-13
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for this layout), bits 16-29
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset, bits 32-45
    d |= (uint64_t)1 << 46;                  // version, bits 46-47
    d |= (uint64_t)2 << 61;                  // layout: 128-byte swizzle, bits 61-63
    return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major,
// N = 256, M = 128.
constexpr uint32_t IDESC = (1u << 4)            // D format FP32
                         | (1u << 7)            // A format BF16
                         | (1u << 10)           // B format BF16
                         | ((uint32_t)(TN >> 3) << 17)
                         | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

template <int STAGES>
struct __align__(8) TcShared {
    uint64_t full[STAGES], empty[STAGES], accum;
    uint32_t tmem_base;
    int issued;   // k tiles whose copies the producer issued
};

template <int STAGES>
constexpr size_t tc_smem() { return (size_t)STAGES * STAGE_BYTES + sizeof(TcShared<STAGES>) + 2048; }

template <int STAGES, int MINB>
__global__ void __launch_bounds__(128, MINB) k_mm_tc(const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ CUtensorMap tmB, float *__restrict__ C,
                                                     int M, int N, int K) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned ring of stages, then the barriers
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared<STAGES> *S = (TcShared<STAGES> *)(base + STAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // CTA -> tile: groups of GROUP_M tile rows, column-major inside a group
    const int ntm = M / TM, ntn = N / TN, per_group = GROUP_M * ntn;
    const int t = blockIdx.x, grp = t / per_group, first = grp * GROUP_M;
    const int gsz = min(ntm - first, GROUP_M), r = t - grp * per_group;
    const int m0 = (first + r % gsz) * TM, n0 = (r / gsz) * TN;
    const int KT = K / TK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&S->full[s], 1);
            mbar_init(&S->empty[s], 1);
        }
        mbar_init(&S->accum, 1);
        S->issued = 0;
        mbar_init_fence();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer
            for (int kt = 0; kt < KT; kt++) {
                const int s = kt % STAGES, r = kt / STAGES;
                if (r > 0 && !mbar_wait(&S->empty[s], (uint32_t)((r - 1) & 1))) break;
                unsigned char *st = base + s * STAGE_BYTES;
                mbar_expect_tx(&S->full[s], STAGE_BYTES);
                tma_load_2d(st, &tmA, &S->full[s], kt * TK, m0);
                tma_load_2d(st + A_BYTES, &tmB, &S->full[s], kt * TK, n0);
                S->issued = kt + 1;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            for (int kt = 0; kt < KT; kt++) {
                const int s = kt % STAGES, r = kt / STAGES;
                if (!mbar_wait(&S->full[s], (uint32_t)(r & 1))) break;
                tc_fence_after();
                unsigned char *st = base + s * STAGE_BYTES;
                const uint64_t ad = smem_desc(st), bd = smem_desc(st + A_BYTES);
#pragma unroll
                for (int kk = 0; kk < TK / 16; kk++)   // 16-element k slices: +32 bytes in the start address
                    mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, (kt > 0 || kk > 0) ? 1u : 0u);
                mma_commit(&S->empty[s]);
            }
            mma_commit(&S->accum);
        }
        __syncwarp();
    }

    // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31
    const bool ok = mbar_wait(&S->accum, 0);
    __syncwarp();
    tc_fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        float *crow = C + (size_t)row * N + n0;
#pragma unroll 1
        for (int c = 0; c < TN / 32; c++) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                  "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                  "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float4 *dst = reinterpret_cast<float4 *>(crow + c * 32);
#pragma unroll
            for (int q = 0; q < 8; q++)
                dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                     __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && (!ok || *(volatile int *)&g_tc_timeout)) {
        // drain: every stage's last issued copy must have landed before the
        // shared memory goes away (bounded waits; the error word is set)
        const int issued = S->issued;
        for (int s = 0; s < STAGES && s < issued; s++) {
            const int last = s + ((issued - 1 - s) / STAGES) * STAGES;
            const uint32_t a = smem_u32(&S->full[s]);
            for (long long i = 0; i < WAIT_LIMIT; i++) {
                uint32_t done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(done)
                    : "r"(a), "r"((uint32_t)((last / STAGES) & 1))
                    : "memory");
                if (done) break;
            }
        }
    }
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------- persistent
// One CTA of 192 threads per SM walks the tiles t = blockIdx.x, +gridDim.x,
// ... (same CTA -> tile numbering as above): warp 0 lane 0 produces into a
// 4-stage ring that runs on across tiles, warp 1 lane 0 issues the MMAs into
// one of two TMEM accumulators (2 x 256 columns), and warps 2-5 drain the
// other accumulator (warp w reads TMEM lanes 32 (w mod 4) ...), so a tile's
// epilogue overlaps the next tile's main loop.  Accumulator b is handed over
// by tfull[b] (MMA commit) and returned by tempty[b] (one arrival per
// epilogue warp).  The tile <-> logical work-group correspondence is the
// same bijection as above, so the counts of the logical decomposition hold;
// only the CTA schedule differs.
constexpr int PST = 4;
struct __align__(8) TcPersist {
    uint64_t full[PST], empty[PST], tfull[2], tempty[2], done;
    uint32_t tmem_base;
    int issued;
};
constexpr size_t kPersistSmem = (size_t)PST * STAGE_BYTES + sizeof(TcPersist) + 2048;

__device__ __forceinline__ void tile_origin(int t, int ntm, int ntn, int &m0, int &n0) {
    const int per_group = GROUP_M * ntn, grp = t / per_group, first = grp * GROUP_M;
    const int gsz = min(ntm - first, GROUP_M), r = t - grp * per_group;
    m0 = (first + r % gsz) * TM;
    n0 = (r / gsz) * TN;
}

__global__ void __launch_bounds__(192, 1) k_mm_tc_persist(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB,
                                                          float *__restrict__ C, int M, int N, int K) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcPersist *S = (TcPersist *)(base + PST * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntm = M / TM, ntn = N / TN, tiles = ntm * ntn, KT = K / TK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < PST; s++) {
            mbar_init(&S->full[s], 1);
            mbar_init(&S->empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&S->tfull[b], 1);
            mbar_init(&S->tempty[b], 4);
        }
        mbar_init(&S->done, 1);
        S->issued = 0;
        mbar_init_fence();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(2 * TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                int m0, n0;
                tile_origin(t, ntm, ntn, m0, n0);
                for (int kt = 0; kt < KT; kt++, it++) {
                    const int s = it % PST, r = it / PST;
                    if (r > 0 && !mbar_wait(&S->empty[s], (uint32_t)((r - 1) & 1))) { ok = false; break; }
                    unsigned char *st = base + s * STAGE_BYTES;
                    mbar_expect_tx(&S->full[s], STAGE_BYTES);
                    tma_load_2d(st, &tmA, &S->full[s], kt * TK, m0);
                    tma_load_2d(st + A_BYTES, &tmB, &S->full[s], kt * TK, n0);
                    S->issued = it + 1;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, lt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, lt++) {
                const int b = lt & 1, u = lt >> 1;
                if (u > 0 && !mbar_wait(&S->tempty[b], (uint32_t)((u - 1) & 1))) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * TMEM_COLS);
                for (int kt = 0; kt < KT; kt++, it++) {
                    const int s = it % PST, r = it / PST;
                    if (!mbar_wait(&S->full[s], (uint32_t)(r & 1))) { ok = false; break; }
                    tc_fence_after();
                    unsigned char *st = base + s * STAGE_BYTES;
                    const uint64_t ad = smem_desc(st), bd = smem_desc(st + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TK / 16; kk++)
                        mma_bf16(d, ad + 2 * kk, bd + 2 * kk, (kt > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&S->empty[s]);
                }
                if (ok) mma_commit(&S->tfull[b]);
            }
            mma_commit(&S->done);   // arrives once every MMA this thread issued has completed
        }
        __syncwarp();
    } else {
        const int q = warp & 3;   // TMEM lane quarter this warp may read
        int lt = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, lt++) {
            const int b = lt & 1, u = lt >> 1;
            const bool got = mbar_wait(&S->tfull[b], (uint32_t)(u & 1));
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            int m0, n0;
            tile_origin(t, ntm, ntn, m0, n0);
            float *crow = C + (size_t)(m0 + q * 32 + lane) * N + n0;
#pragma unroll 1
            for (int c = 0; c < TN / 32; c++) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TMEM_COLS + c * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                      "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float4 *dst = reinterpret_cast<float4 *>(crow + c * 32);
#pragma unroll
                for (int k = 0; k < 8; k++)
                    dst[k] = make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                                         __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S->tempty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int *)&g_tc_timeout) {
        // drain: every stage's last issued copy must land before the shared memory goes away
        const int issued = S->issued;
        for (int s = 0; s < PST && s < issued; s++) {
            const int last = s + ((issued - 1 - s) / PST) * PST;
            for (long long i = 0; i < WAIT_LIMIT; i++)
                if (mbar_try(&S->full[s], (uint32_t)((last / PST) & 1))) break;
        }
    }
    __syncthreads();
    if (warp == 1) {
        mbar_wait(&S->done, 0);   // no MMA may still write the accumulators being released
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------- 256 x 256 tiles
// One CTA of 256 threads per 256 x 256 tile of C (one CTA per SM): per
// 64-wide k tile one 256x64 box of A and one 256x64 box of Bt (64 KB per
// stage, 3 stages) and eight MMAs -- the two 128-row halves of the A box
// against the same Bt box, four k slices each -- into two accumulators of
// 256 TMEM columns.  Per flop this moves two thirds of the operand bytes of
// the 128 x 256 tile.  Epilogue: warps w and w + 4 drain TMEM lanes
// 32 (w mod 4) ... of accumulator 0 and 1, i.e. work-item t stores row t.
constexpr int WM = 256, W_STAGES = 3, GROUP_W = 8;
constexpr int WA_BYTES = WM * TK * 2, W_STAGE_BYTES = WA_BYTES + B_BYTES;
struct __align__(8) TcWide {
    uint64_t full[W_STAGES], empty[W_STAGES], accum;
    uint32_t tmem_base;
    int issued;
};
constexpr size_t kWideSmem = (size_t)W_STAGES * W_STAGE_BYTES + sizeof(TcWide) + 2048;
static_assert(kWideSmem <= 227 * 1024, "wide tile ring exceeds shared memory");
static_assert(2 * kWideSmem > 228 * 1024, "one wide CTA per SM: the 512 TMEM columns are not shared");

__global__ void __launch_bounds__(256, 1) k_mm_tc_w(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, float *__restrict__ C,
                                                    int M, int N, int K) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcWide *S = (TcWide *)(base + W_STAGES * W_STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // CTA -> tile: groups of GROUP_W tile rows, column-major inside a group
    const int ntm = M / WM, ntn = N / TN, per_group = GROUP_W * ntn;
    const int t = blockIdx.x, grp = t / per_group, first = grp * GROUP_W;
    const int gsz = min(ntm - first, GROUP_W), r = t - grp * per_group;
    const int m0 = (first + r % gsz) * WM, n0 = (r / gsz) * TN;
    const int KT = K / TK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < W_STAGES; s++) {
            mbar_init(&S->full[s], 1);
            mbar_init(&S->empty[s], 1);
        }
        mbar_init(&S->accum, 1);
        S->issued = 0;
        mbar_init_fence();
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(2 * TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            for (int kt = 0; kt < KT; kt++) {
                const int s = kt % W_STAGES, r = kt / W_STAGES;
                if (r > 0 && !mbar_wait(&S->empty[s], (uint32_t)((r - 1) & 1))) break;
                unsigned char *st = base + s * W_STAGE_BYTES;
                mbar_expect_tx(&S->full[s], W_STAGE_BYTES);
                tma_load_2d(st, &tmA, &S->full[s], kt * TK, m0);
                tma_load_2d(st + WA_BYTES, &tmB, &S->full[s], kt * TK, n0);
                S->issued = kt + 1;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kt = 0; kt < KT; kt++) {
                const int s = kt % W_STAGES, r = kt / W_STAGES;
                if (!mbar_wait(&S->full[s], (uint32_t)(r & 1))) break;
                tc_fence_after();
                unsigned char *st = base + s * W_STAGE_BYTES;
                // rows 128..255 of the A box start 128 rows x 128 bytes in
                const uint64_t a0 = smem_desc(st), a1 = smem_desc(st + WA_BYTES / 2), bd = smem_desc(st + WA_BYTES);
#pragma unroll
                for (int kk = 0; kk < TK / 16; kk++) {
                    const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                    mma_bf16(tmem, a0 + 2 * kk, bd + 2 * kk, acc);
                    mma_bf16(tmem + (uint32_t)TMEM_COLS, a1 + 2 * kk, bd + 2 * kk, acc);
                }
                mma_commit(&S->empty[s]);
            }
            mma_commit(&S->accum);
        }
        __syncwarp();
    }

    const bool ok = mbar_wait(&S->accum, 0);
    __syncwarp();
    tc_fence_after();
    if (ok) {
        const int h = warp >> 2, q = warp & 3;
        float *crow = C + (size_t)(m0 + h * 128 + q * 32 + lane) * N + n0;
#pragma unroll 1
        for (int c = 0; c < TN / 32; c++) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * TMEM_COLS + c * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                  "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
                  "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float4 *dst = reinterpret_cast<float4 *>(crow + c * 32);
#pragma unroll
            for (int k = 0; k < 8; k++)
                dst[k] = make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                                     __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && (!ok || *(volatile int *)&g_tc_timeout)) {
        // drain: every stage's last issued copy must land before the shared memory goes away
        const int issued = S->issued;
        for (int s = 0; s < W_STAGES && s < issued; s++) {
            const int last = s + ((issued - 1 - s) / W_STAGES) * W_STAGES;
            for (long long i = 0; i < WAIT_LIMIT; i++)
                if (mbar_try(&S->full[s], (uint32_t)((last / W_STAGES) & 1))) break;
        }
    }
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static pm_status get_encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    if (!g_encode) return fail(PM_ECUDA, "mm_tc: cuTensorMapEncodeTiled is not available");
    return PM_OK;
}

pm_status tensor_map_2d(CUtensorMap *map, int bf16, const void *ptr, uint64_t cols, uint64_t rows, uint64_t row_bytes,
                        uint32_t box_cols, uint32_t box_rows, int swizzle128) {
    pm_status s = get_encoder();
    if (s) return s;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    auto encode = [&] {
        return g_encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    };
    CUresult r = encode();
    if (r == CUDA_ERROR_INVALID_CONTEXT) {
        // no context current on this thread yet (e.g. a resource query
        // before any other CUDA call): make the runtime's one current
        PM_CUDA_TRY(cudaFree(nullptr));
        r = encode();
    }
    if (r != CUDA_SUCCESS) return fail(PM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PM_OK;
}

template <int STAGES, int MINB>
pm_status launch_tc_t(const CUtensorMap &ta, const CUtensorMap &tb, float *c, int n, cudaStream_t st) {
    constexpr size_t smem = tc_smem<STAGES>();
    static_assert(MINB * (smem + 1024) <= 228 * 1024, "resident CTAs exceed shared memory");
    static_assert(MINB * 256 <= 512, "resident CTAs exceed tensor memory");
    auto fn = k_mm_tc<STAGES, MINB>;
    PM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    launch_k(fn, (unsigned)((n / TN) * (n / TM)), 128, smem, st, ta, tb, c, n, n, n);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status launch_tc(const KP &kp, void *const *b, void *stream) {
    const int n = (int)kp.i(0), pipe = (int)kp.i(1);
    for (int a = 0; a < 3; a++)
        if ((uintptr_t)b[a] % 16) return fail(PM_EINVAL, "mm_tc: buffer %d must be 16-byte aligned", a);
    pm_status s;
    CUtensorMap ta, tb;
    if (kp.def->variant == 1) {
        if ((s = tensor_map_2d(&ta, 1, b[0], n, n, (uint64_t)n * 2, TK, WM, 1))) return s;
        if ((s = tensor_map_2d(&tb, 1, b[1], n, n, (uint64_t)n * 2, TK, TN, 1))) return s;
        PM_CUDA_TRY(cudaFuncSetAttribute(k_mm_tc_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWideSmem));
        launch_k(k_mm_tc_w, (unsigned)((n / TN) * (n / WM)), 256, kWideSmem, (cudaStream_t)stream, ta, tb,
                 (float *)b[2], n, n, n);
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }
    if ((s = tensor_map_2d(&ta, 1, b[0], n, n, (uint64_t)n * 2, TK, TM, 1))) return s;
    if ((s = tensor_map_2d(&tb, 1, b[1], n, n, (uint64_t)n * 2, TK, TN, 1))) return s;
    if (pipe == 0) return launch_tc_t<4, 1>(ta, tb, (float *)b[2], n, (cudaStream_t)stream);
    if (pipe == 1) return launch_tc_t<2, 2>(ta, tb, (float *)b[2], n, (cudaStream_t)stream);
    // persistent: one CTA per SM (at most one per tile)
    int dev = 0, sms = 0;
    PM_CUDA_TRY(cudaGetDevice(&dev));
    PM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int tiles = (n / TN) * (n / TM);
    PM_CUDA_TRY(cudaFuncSetAttribute(k_mm_tc_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPersistSmem));
    launch_k(k_mm_tc_persist, (unsigned)std::min(tiles, sms), 192, kPersistSmem, (cudaStream_t)stream, ta, tb,
             (float *)b[2], n, n, n);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

// After a synchronisation: PM_ETIMEOUT if any CTA's bounded wait ran out
// since the last check (the word is cleared).
pm_status tc_check_timeout() {
    int v = 0, z = 0;
    PM_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof v));
    if (v) {
        PM_CUDA_TRY(cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof z));
        return fail(PM_ETIMEOUT, "mm_tc: a bounded wait gave up (pipeline stalled)");
    }
    return PM_OK;
}

}  // namespace pm
