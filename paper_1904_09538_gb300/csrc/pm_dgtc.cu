// DG derivative on the 5th-generation tensor cores ("dg_tc"):
//   res[m, k, i] = sum_j D[m, i, j] u[k, j]      (Section "DG")
// as one product per 128-element tile: C (128 x NR) = U (128 x Np) Ds^T,
// Ds the operator rows stacked over the CTA's m (MS = 3 for Np <= 40, and
// for Np <= 64 when the u operand is in shared memory; else one m per CTA),
// on tcgen05.mma kind::tf32 with FP32 accumulation in TMEM.
//
// FP32 accuracy from TF32 operands: every operand value x is split into a
// head x_h (x rounded to nearest at TF32's 10 mantissa bits, low 13 bits
// zero, so the tensor core reads it exactly) and the remainder
// x_l = x - x_h (exact in FP32, |x_l| <= 2^-11 |x|).  Three passes
// accumulate U_h Ds_h + U_h Ds_l + U_l Ds_h; the dropped U_l Ds_l is below
// 2^-22 |U||Ds| per term and the remainders' own TF32 rounding below 2^-21,
// so each product term carries a relative error of a few 2^-22.
//
// Shared-memory operand layout: K-major, 128-byte swizzle (16-byte chunk c
// of row r at r * 128 + ((c ^ (r & 7)) << 4) within 1024-byte-aligned atoms
// of 8 rows), 32 columns (j) per atom: Np needs KA = ceil(Np / 32) atoms and
// the MMA runs KS = ceil(Np / 8) steps of K = 8, i.e. atom a is read up to
// chunk CN(a) = 2 min(4, KS - 4a).  Operator rows: row n = mm * NP8 + i
// (NP8 = Np rounded up to 8, so each m's accumulator columns start on a
// multiple of 8), zero for i >= Np and for the padding rows up to NR.
//
// Persistent CTAs of 320 threads (352 with A = 1) on a grid (G, P), G = 3 / MS m-groups:
// CTA (g, p) serves m-group g and the tiles t = p, p + P, ... (the G CTAs of
// one p are adjacent in launch order, so a u tile comes from HBM once):
//   all threads, once: stage Ds_h and Ds_l from D (thread i = operator row i
//       of each of the CTA's m, its row's chunks in turn);
//   warp 8 lane 0: TMA producer (Np % 4 == 0: one 128 x 32 box of u per
//       (tile, atom), 128-byte swizzle, zero fill beyond Np and Nel) into a
//       ring of raw atoms; warp 8 also allocates and frees the TMEM;
//   warps 4-7: converters -- thread r = element row r of the tile: its
//       chunks of each atom (from the staged atom; when Np % 4 != 0 from
//       the tile's rows staged by one bulk copy (A = 1) or from global
//       memory (A = 0), guarded) split into head and remainder;
//   warp 9 lane 0: MMA issuer -- per atom 3 MMAs per k step into one of two
//       TMEM accumulators; commits free the operand stage and hand over the
//       accumulator.  With A = 1 warps 9 and 10 issue, each the tiles of one
//       accumulator (alternate tiles): an MMA instruction leaves its thread
//       only about when the tensor core takes it up, so every wait, commit and
//       address step of a single issuer leaves the tensor pipe idle, and the
//       second issuer's MMAs fill those gaps;
//   warps 0-3: epilogue -- warp w reads TMEM lanes 32w.. (its 32 elements),
//       writes each m's 128 x Np block row-major into one of OB staging
//       buffers, and one thread stores it with one bulk copy (contiguous in
//       res), so the HBM writes are whole lines.
// Two forms (parameter A):
//   A = 0: the u operand in shared memory -- ST stages of 32 KB (head,
//       remainder); the TMA writes the raw atom into the head half and the
//       converters split it in place; the MMA (both operands from shared
//       memory) frees the stage.  TMEM: two accumulators of NR columns.
//   A = 1: the u operand in tensor memory -- the converters write head and
//       remainder of their row with tcgen05.st into one of SA = 4 TMEM
//       operand stages (64 columns at 256 + 64 s), the MMA reads A from TMEM
//       and only the operator atoms from shared memory (half the shared
//       bytes per MMA); raw atoms (4 stages of 16 KB) are freed by the
//       converters.  TMEM: all 512 columns (accumulators at 0 and 128), one
//       CTA per SM.
// Every mbarrier wait is bounded: on expiry the kernel sets an error word,
// the roles stop, the producer drains its copies in flight, the MMA issuers'
// last commits are awaited (bounded) before the TMEM is freed.  The epilogue
// warps agree on every accumulator hand-over through a reducing named
// barrier, so none of them waits at a named barrier that the others left.
#include <algorithm>
#include <cstring>
#include <cuda.h>
#include <cuda_runtime.h>

#include "pm_internal.h"
#include "pm_tma.cuh"

namespace pm {

static __device__ int g_dgc_timeout;

namespace {

constexpr long long DGC_WAIT = 1ll << 26;
constexpr int ATOM = 128 * 128;   // 128 rows x 32 FP32 columns
constexpr int SA = 4;             // TMEM operand stages (A = 1)
constexpr int kGB300SMs = 152;    // default persistent grid: resident CTAs of one GB300

__host__ __device__ constexpr DgcShape dgc_shape0(int np) {
    return np <= 20 ? DgcShape{3, 2, 2, 2} : np <= 40 ? DgcShape{3, 1, 3, 2} : np <= 64 ? DgcShape{1, 1, 4, 2}
                                                                                      : DgcShape{1, 1, 3, 1};
}
__host__ __device__ constexpr int pow2_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

template <int NP, bool TS>
struct Dgc {
    // the shared-memory form holds the three m's operator rows for Np <= 64
    // (N = 3 NP8 <= 176), the tensor-memory form (accumulators 128 columns
    // apart) only for Np <= 40
    static constexpr DgcShape S = (!TS && NP > 40 && NP <= 64) ? DgcShape{3, 1, 2, 2} : dgc_shape0(NP);
    static constexpr int MS = S.ms, G = 3 / S.ms;
    static constexpr int R = TS ? 1 : S.r;                          // CTAs per SM
    // A = 1 with Np % 4 != 0: whole u tiles (row-major, one bulk copy each)
    static constexpr bool BULK = TS && NP % 4 != 0;
    static constexpr int RAWB = (128 * NP * 4 + 1023) / 1024 * 1024;
    static constexpr int ST = TS ? (NP % 4 == 0 ? 4 : 2) : S.st;    // shared-memory stages
    static constexpr int SBYTES = TS ? (BULK ? RAWB : ATOM) : 2 * ATOM;   // bytes per shared-memory stage
    static constexpr int OB = TS ? 2 : S.ob;
    // MMA issuers: two in the tensor-memory form (alternate tiles).  Sound
    // because an issuer's wait for atom x on operand slot x % SA always finds
    // the slot's previous use (atom x - SA) converted: the converters work in
    // atom order and the issuer has consumed atom x - 1 of its tile, or for a
    // tile's first atom the last atom x - KA - 1 of its previous tile, both
    // >= x - SA for KA <= 3.  The shared-memory form keeps one issuer: with as
    // many stages as atoms per tile (ST = KA at Np = 56 and 84) a parity wait
    // could not tell the awaited phase from the one two uses back.
    static constexpr int NI = TS ? 2 : 1;
    static constexpr int THREADS = 320 + 32 * (NI - 1);
    static constexpr int NP8 = (NP + 7) / 8 * 8;
    static constexpr int NR = (MS * NP8 + 15) / 16 * 16;            // MMA N
    static constexpr int KA = (NP + 31) / 32;
    static constexpr int KS = (NP + 7) / 8;
    static constexpr int TCOLS = TS ? 512 : pow2_cols(2 * NR);
    static constexpr int ACC = TS ? 128 : TCOLS / 2;                // column of accumulator 1
    static constexpr int BBYTES = KA * NR * 128;                    // one operator copy (head or remainder)
    static constexpr int OBYTES = 128 * NP * 4;
    static constexpr int RING = ST * SBYTES;
    static constexpr int BAR_OFF = RING + 2 * BBYTES + OB * OBYTES;
    static constexpr size_t NEED = (size_t)BAR_OFF + 256 + 1024;
    // A = 1 holds all 512 TMEM columns: at least 116 KB keeps it at one CTA per SM
    static constexpr size_t SMEM = (TS && NEED < 116 * 1024) ? 116 * 1024 : NEED;
    static constexpr uint32_t IDESC = (1u << 4)                         // D format FP32
                                    | (2u << 7) | (2u << 10)            // A, B format TF32
                                    | ((uint32_t)(NR >> 3) << 17)       // N
                                    | ((uint32_t)(128 >> 4) << 24);     // M = 128
    static_assert(NR >= 16 && NR <= 256 && NR % 16 == 0, "MMA N out of range");
    static_assert(NI == 1 || KA + 1 <= SA, "two issuers need a free operand slot beyond a tile's atoms");
    static_assert(NR <= ACC, "accumulators overlap");
    static_assert(ST >= 1 && ST <= 4, "ring depth");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(R * (SMEM + 1024) <= 228 * 1024, "resident CTAs exceed shared memory");
    static_assert(R * TCOLS <= 512, "resident CTAs exceed tensor memory");
};

struct __align__(8) DgcBars {
    uint64_t full[4], empty[4], ready[4], free_[4], tfull[2], tempty[2], done;
    uint32_t tmem_base;
    int issued;
};
static_assert(sizeof(DgcBars) <= 256, "barrier block");

__device__ __forceinline__ bool dgc_wait(uint64_t *bar, uint32_t parity) {
    return mbar_wait_bounded(bar, parity, &g_dgc_timeout, DGC_WAIT);
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// K-major, 128-byte swizzle, 8-row groups 1024 bytes apart, version 1
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// both operands from shared memory
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// A from tensor memory, B from shared memory
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}"
        ::"r"(d), "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit_to(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

__device__ __forceinline__ float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts4(uint32_t a, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
__device__ __forceinline__ float lds1(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts1(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// head: x rounded to nearest (ties away from zero) at TF32's precision
__device__ __forceinline__ float tf32_head(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split4(float4 v, float4 &h, float4 &l) {
    h = make_float4(tf32_head(v.x), tf32_head(v.y), tf32_head(v.z), tf32_head(v.w));
    l = make_float4(__fsub_rn(v.x, h.x), __fsub_rn(v.y, h.y), __fsub_rn(v.z, h.z), __fsub_rn(v.w, h.w));
}
// physical byte offset of logical 16-byte chunk c of row r in a swizzled atom
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
// named barrier over n threads that also ANDs a predicate across them
__device__ __forceinline__ bool bar_and(int id, int n, bool p) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred o, %2, %3, q;\n selp.u32 %0, 1, 0, o;\n}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void bulk_store(void *gdst, uint32_t ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"((uint64_t)gdst), "r"(ssrc),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int NP, bool TMA_U, bool TS>
__global__ void __launch_bounds__(Dgc<NP, TS>::THREADS, (Dgc<NP, TS>::R))
    k_dg_tc(const __grid_constant__ CUtensorMap tmU, const float *__restrict__ D, const float *__restrict__ u,
            float *__restrict__ res, int Nel) {
    using C = Dgc<NP, TS>;
    constexpr int MS = C::MS, ST = C::ST, OB = C::OB, NP8 = C::NP8, NR = C::NR, KA = C::KA, KS = C::KS;
    constexpr bool BULK = C::BULK;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t sraw = smem_u32(smem_raw);
    const uint32_t sbase = (sraw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (sbase - sraw);   // generic pointer to the same byte (TMA destinations)
    const uint32_t s_bh = sbase + C::RING, s_bl = s_bh + C::BBYTES, s_out = s_bl + C::BBYTES;
    DgcBars *S = reinterpret_cast<DgcBars *>(gbase + C::BAR_OFF);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x, p = blockIdx.y, P = gridDim.y;
    const int T = (Nel + 127) / 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 4; s++) {
            mbar_init(&S->full[s], 1);
            mbar_init(&S->empty[s], TS ? 4 : 1);   // A = 1: freed by the converter warps
            mbar_init(&S->ready[s], 4);
            mbar_init(&S->free_[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&S->tfull[b], 1);
            mbar_init(&S->tempty[b], 4);
        }
        mbar_init(&S->done, C::NI);   // each issuer's last commit
        S->issued = 0;
        mbar_init_fence();
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(C::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_before();
    }
    // operator rows: thread i stages row mm * NP8 + i of each of the CTA's m,
    // then the padding rows MS * NP8 .. NR - 1 (zero)
    if (threadIdx.x < NP8) {
        const int i = threadIdx.x;
        for (int mm = 0; mm < MS; mm++) {
            const int n = mm * NP8 + i, m = MS == 3 ? mm : g;
            const float *drow = D + (m * NP + i) * NP;
            for (int ac = 0; ac < 8 * KA; ac++) {
                const int j0 = 4 * ac;
                float4 v;
                v.x = (i < NP && j0 < NP) ? __ldg(drow + j0) : 0.0f;
                v.y = (i < NP && j0 + 1 < NP) ? __ldg(drow + j0 + 1) : 0.0f;
                v.z = (i < NP && j0 + 2 < NP) ? __ldg(drow + j0 + 2) : 0.0f;
                v.w = (i < NP && j0 + 3 < NP) ? __ldg(drow + j0 + 3) : 0.0f;
                float4 h, l;
                split4(v, h, l);
                const uint32_t off = (uint32_t)((ac >> 3) * NR * 128) + swz(n, ac & 7);
                sts4(s_bh + off, h);
                sts4(s_bl + off, l);
            }
        }
    }
    if ((int)threadIdx.x < NR - MS * NP8) {
        const int n = MS * NP8 + threadIdx.x;
        for (int ac = 0; ac < 8 * KA; ac++) {
            const uint32_t off = (uint32_t)((ac >> 3) * NR * 128) + swz(n, ac & 7);
            sts4(s_bh + off, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
            sts4(s_bl + off, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
        }
    }
    fence_async_smem();
    __syncthreads();
    tc_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == 8) {
        if (BULK && lane == 0) {
            // one bulk copy of the tile's rows (contiguous in u) per tile
            int it = 0;
            for (int t = p; t < T; t += P, it++) {
                const int s = it % ST, r = it / ST;
                if (r > 0 && !dgc_wait(&S->empty[s], (uint32_t)((r - 1) & 1))) break;
                const uint32_t bytes = (uint32_t)min(128LL, (long long)Nel - 128LL * t) * NP * 4u;
                mbar_expect_tx(&S->full[s], bytes);
                bulk_load(gbase + s * C::SBYTES, u + 128LL * t * NP, bytes, &S->full[s]);
                S->issued = it + 1;
            }
        } else if (TMA_U && lane == 0) {
            int it = 0;
            bool ok = true;
            for (int t = p; t < T && ok; t += P)
                for (int a = 0; a < KA; a++, it++) {
                    const int s = it % ST, r = it / ST;
                    if (r > 0 && !dgc_wait(&S->empty[s], (uint32_t)((r - 1) & 1))) { ok = false; break; }
                    mbar_expect_tx(&S->full[s], ATOM);
                    tma_load_2d(gbase + s * C::SBYTES, &tmU, &S->full[s], 32 * a, 128 * t);
                    S->issued = it + 1;
                }
        }
        __syncwarp();
    } else if (warp == 9 || warp == 10) {
        if (lane == 0) {
            // issuer ki serves the CTA's tiles lt = ki, ki + NI, ... (NI = 2:
            // always accumulator ki)
            const int ki = warp - 9;
            int lt = ki;
            bool ok = true;
            for (int t = p + ki * P; t < T && ok; t += C::NI * P, lt += C::NI) {
                const int b = lt & 1, uu = lt >> 1;
                int it = lt * KA;
                if (uu > 0 && !dgc_wait(&S->tempty[b], (uint32_t)((uu - 1) & 1))) break;
                tc_after();
                const uint32_t d = tmem + (uint32_t)(b * C::ACC);
                // unrolled: every atom's k steps and operand offsets are
                // compile-time, so the MMAs issue back to back
#pragma unroll
                for (int a = 0; a < KA; a++, it++) {
                    const int s = TS ? it % SA : it % ST, r = TS ? it / SA : it / ST;
                    if (!dgc_wait(&S->ready[s], (uint32_t)(r & 1))) { ok = false; break; }
                    tc_after();
                    const uint64_t bh = sw128_desc(s_bh + a * NR * 128), bl = sw128_desc(s_bl + a * NR * 128);
                    if (TS) {
                        const uint32_t ah = tmem + (uint32_t)(256 + 64 * s), al = ah + 32;
#pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            if (4 * a + kk >= KS) break;
                            mma_ts(d, ah + 8 * kk, bh + 2 * kk, C::IDESC, (a > 0 || kk > 0) ? 1u : 0u);
                            mma_ts(d, ah + 8 * kk, bl + 2 * kk, C::IDESC, 1u);
                            mma_ts(d, al + 8 * kk, bh + 2 * kk, C::IDESC, 1u);
                        }
                        mma_commit_to(&S->free_[s]);
                    } else {
                        const uint32_t hs = sbase + s * C::SBYTES;
                        const uint64_t ah = sw128_desc(hs), al = sw128_desc(hs + ATOM);
#pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            if (4 * a + kk >= KS) break;
                            mma_ss(d, ah + 2 * kk, bh + 2 * kk, C::IDESC, (a > 0 || kk > 0) ? 1u : 0u);
                            mma_ss(d, ah + 2 * kk, bl + 2 * kk, C::IDESC, 1u);
                            mma_ss(d, al + 2 * kk, bh + 2 * kk, C::IDESC, 1u);
                        }
                        mma_commit_to(&S->empty[s]);
                    }
                }
                if (ok) mma_commit_to(&S->tfull[b]);
            }
            mma_commit_to(&S->done);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // converters: thread r = element row r of the tile (TMEM lane r)
        const int q = warp - 4, r = 32 * q + lane;
        int it = 0, itile = 0;
        for (int t = p; t < T; t += P, itile++) {
            bool ok = true;
            const long long k = 128LL * t + r;
            const uint32_t raw = sbase + (uint32_t)((itile % ST) * C::SBYTES);   // BULK: the tile's rows
            if (BULK) {
                const bool got = dgc_wait(&S->full[itile % ST], (uint32_t)((itile / ST) & 1));
                if (!__all_sync(0xffffffffu, got)) break;
            }
#pragma unroll
            for (int a = 0; a < KA; a++, it++) {
                const int CN = 2 * min(4, KS - 4 * a);   // chunks of this atom the MMA reads
                const int s = it % ST, rs = it / ST;
                const uint32_t hs = sbase + s * C::SBYTES;
                bool got = true;
                if (TMA_U) got = dgc_wait(&S->full[s], (uint32_t)(rs & 1));
                else if (!TS && rs > 0) got = dgc_wait(&S->empty[s], (uint32_t)((rs - 1) & 1));
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                float4 h[8], l[8];
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    if (c >= CN) break;
                    float4 v;
                    if (TMA_U) {
                        v = lds4(hs + swz(r, c));
                    } else if (BULK) {
                        const int j0 = 32 * a + 4 * c;
                        const uint32_t src = raw + (uint32_t)((r * NP + j0) * 4);
                        const bool in = k < Nel;
                        v.x = (in && j0 < NP) ? lds1(src) : 0.0f;
                        v.y = (in && j0 + 1 < NP) ? lds1(src + 4) : 0.0f;
                        v.z = (in && j0 + 2 < NP) ? lds1(src + 8) : 0.0f;
                        v.w = (in && j0 + 3 < NP) ? lds1(src + 12) : 0.0f;
                    } else {
                        const int j0 = 32 * a + 4 * c;
                        const float *src = u + k * NP + j0;
                        const bool in = k < Nel;
                        v.x = (in && j0 < NP) ? __ldg(src) : 0.0f;
                        v.y = (in && j0 + 1 < NP) ? __ldg(src + 1) : 0.0f;
                        v.z = (in && j0 + 2 < NP) ? __ldg(src + 2) : 0.0f;
                        v.w = (in && j0 + 3 < NP) ? __ldg(src + 3) : 0.0f;
                    }
                    split4(v, h[c], l[c]);
                    if (!TS) {
                        sts4(hs + swz(r, c), h[c]);
                        sts4(hs + ATOM + swz(r, c), l[c]);
                    }
                }
                if (TS) {
                    if (TMA_U) {
                        // this lane's shared reads of the raw atom are ordered
                        // before the TMA engine's next write into the stage
                        // (async proxy): a release on the barrier alone orders
                        // them only against generic accesses
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&S->empty[s]);   // the raw atom is consumed
                    }
                    const int sa = it % SA, ra = it / SA;
                    const bool fr = ra == 0 || dgc_wait(&S->free_[sa], (uint32_t)((ra - 1) & 1));
                    if (!__all_sync(0xffffffffu, fr)) { ok = false; break; }
                    tc_after();
                    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(256 + 64 * sa);
#pragma unroll
                    for (int c8 = 0; c8 < 4; c8++) {
                        if (2 * c8 >= CN) break;
                        const float hv[8] = {h[2 * c8].x, h[2 * c8].y, h[2 * c8].z, h[2 * c8].w,
                                             h[2 * c8 + 1].x, h[2 * c8 + 1].y, h[2 * c8 + 1].z, h[2 * c8 + 1].w};
                        const float lv[8] = {l[2 * c8].x, l[2 * c8].y, l[2 * c8].z, l[2 * c8].w,
                                             l[2 * c8 + 1].x, l[2 * c8 + 1].y, l[2 * c8 + 1].z, l[2 * c8 + 1].w};
                        tmem_st8(ta + 8 * c8, hv);
                        tmem_st8(ta + 32 + 8 * c8, lv);
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    tc_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S->ready[sa]);
                } else {
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S->ready[s]);
                }
            }
            if (BULK) {
                fence_async_smem();   // the staged rows' reads before the next bulk copy into them
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->empty[itile % ST]);   // the raw tile is consumed
            }
            if (!ok) break;
        }
    } else {
        // epilogue: warp w drains TMEM lanes 32w .. 32w + 31 (elements)
        const int row = 32 * warp + lane;
        int lt = 0, nout = 0;
        for (int t = p; t < T; t += P, lt++) {
            const int b = lt & 1, uu = lt >> 1;
            const bool got = dgc_wait(&S->tfull[b], (uint32_t)(uu & 1));
            if (!bar_and(1, 128, got)) break;
            tc_after();
            const long long k0 = 128LL * t;
            const int rows = (int)min(128LL, (long long)Nel - k0);
#pragma unroll 1
            for (int mm = 0; mm < MS; mm++, nout++) {
                const int m = MS == 3 ? mm : g, buf = nout % OB;
                if (nout >= OB && threadIdx.x == 0) bulk_wait_read<OB - 1>();
                bar_sync(2, 128);
                uint32_t v[NP8];
                const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * C::ACC + mm * NP8);
#pragma unroll
                for (int c = 0; c < NP8 / 8; c++)
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                                 : "=r"(v[8 * c]), "=r"(v[8 * c + 1]), "=r"(v[8 * c + 2]), "=r"(v[8 * c + 3]),
                                   "=r"(v[8 * c + 4]), "=r"(v[8 * c + 5]), "=r"(v[8 * c + 6]), "=r"(v[8 * c + 7])
                                 : "r"(ta + (uint32_t)(8 * c)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const uint32_t orow = s_out + (uint32_t)(buf * C::OBYTES + row * NP * 4);
                if (NP % 4 == 0) {
#pragma unroll
                    for (int i = 0; i < NP; i += 4)
                        sts4(orow + 4 * i, make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]),
                                                       __uint_as_float(v[i + 2]), __uint_as_float(v[i + 3])));
                } else {
#pragma unroll
                    for (int i = 0; i < NP; i++) sts1(orow + 4 * i, __uint_as_float(v[i]));
                }
                fence_async_smem();
                bar_sync(2, 128);
                if (threadIdx.x == 0) {
                    bulk_store(res + ((long long)m * Nel + k0) * NP, s_out + (uint32_t)(buf * C::OBYTES),
                               (uint32_t)rows * NP * 4u);
                    bulk_commit();
                }
            }
            tc_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S->tempty[b]);
        }
        if (threadIdx.x == 0) bulk_wait_all();
    }
    tc_before();
    __syncthreads();
    if ((TMA_U || BULK) && threadIdx.x == 256 && *(volatile int *)&g_dgc_timeout) {
        // drain: every stage's last issued copy lands before the shared memory goes away
        const int issued = S->issued;
        for (int s = 0; s < ST && s < issued; s++) {
            const int last = s + ((issued - 1 - s) / ST) * ST;
            mbar_drain(&S->full[s], (uint32_t)((last / ST) & 1), DGC_WAIT);
        }
    }
    __syncthreads();
    if (warp == 8) {
        // no MMA may still write the accumulators being released
        if (lane == 0) mbar_drain(&S->done, 0, DGC_WAIT);
        __syncwarp();
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS) : "memory");
    }
}

template <int NP, bool TS>
pm_status launch_dgc_t(void *const *b, int Nel, int P, cudaStream_t st) {
    using C = Dgc<NP, TS>;
    CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    if constexpr (NP % 4 == 0) {
        // u rows are 16-byte multiples: TMA boxes of 128 rows x 32 columns
        pm_status s = tensor_map_2d(&tm, 0, b[1], (uint64_t)NP, (uint64_t)Nel, (uint64_t)NP * 4, 32, 128, 1);
        if (s != PM_OK) return s;
    }
    auto fn = k_dg_tc<NP, NP % 4 == 0, TS>;
    PM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    launch_k(fn, dim3((unsigned)C::G, (unsigned)P), dim3(C::THREADS), C::SMEM, st, tm, (const float *)b[0],
             (const float *)b[1], (float *)b[2], Nel);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

template <int NP>
pm_status launch_dgc_np(void *const *b, int Nel, int P, int A, cudaStream_t st) {
    return A ? launch_dgc_t<NP, true>(b, Nel, P, st) : launch_dgc_t<NP, false>(b, Nel, P, st);
}

}  // namespace

DgcShape dgc_geometry(int Np, int A) {
    if (!A && Np > 40 && Np <= 64) return DgcShape{3, 1, 2, 2};
    DgcShape s = dgc_shape0(Np);
    if (A) s.r = 1;
    return s;
}

// the faster form per node count (timed on GB300): tensor memory for
// 20 < Np <= 40 and Np > 64, shared memory (three m per CTA up to Np = 64)
int dgc_resolve_a(int Np, int A) { return A < 0 ? (((Np > 20 && Np <= 40) || Np > 64) ? 1 : 0) : A; }

int dgc_resolve_p(int Np, int64_t Nel, int A, int P) {
    if (P > 0) return P;
    const int T = (int)((Nel + 127) / 128);
    const DgcShape s = dgc_geometry(Np, dgc_resolve_a(Np, A));
    return std::min(T, kGB300SMs * s.r / (3 / s.ms));
}

pm_status launch_dgc(const KP &kp, void *const *b, void *stream) {
    const int Np = (int)kp.i(0), Nel = (int)kp.i(1);
    const int A = dgc_resolve_a(Np, (int)kp.i(3)), P = dgc_resolve_p(Np, Nel, A, (int)kp.i(2));
    for (int a = 0; a < 3; a++)
        if ((uintptr_t)b[a] % 16) return fail(PM_EINVAL, "dg_tc: buffer %d must be 16-byte aligned", a);
    cudaStream_t st = (cudaStream_t)stream;
    switch (Np) {   // the node counts of tetrahedral elements of order 1..6
    case 4: return launch_dgc_np<4>(b, Nel, P, A, st);
    case 10: return launch_dgc_np<10>(b, Nel, P, A, st);
    case 20: return launch_dgc_np<20>(b, Nel, P, A, st);
    case 35: return launch_dgc_np<35>(b, Nel, P, A, st);
    case 56: return launch_dgc_np<56>(b, Nel, P, A, st);
    case 84: return launch_dgc_np<84>(b, Nel, P, A, st);
    default: return fail(PM_EINVAL, "dg_tc: Np must be 4, 10, 20, 35, 56 or 84");
    }
}

pm_status dgc_check_timeout() {
    int v = 0, z = 0;
    PM_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_dgc_timeout, sizeof v));
    if (v) {
        PM_CUDA_TRY(cudaMemcpyToSymbol(g_dgc_timeout, &z, sizeof z));
        return fail(PM_ETIMEOUT, "dg_tc: a bounded wait gave up");
    }
    return PM_OK;
}

}  // namespace pm
