// Autotuning spaces: the register-tiled SIMT fp32 matmul family (24 tile
// shapes).  Loop nest (the one pm_counts counts), work-group (BN/8) x (BM/8),
// every work-item owns 8 rows (8 lid1 + i) x 2 column vectors (lid0 and
// L0 + lid0, L0 = BN/8) of C:
//   per k tile of width BK:
//     barrier;
//     A tile, rows lid1 + L1 r (r < 8), vector columns lid0 + L0 q (< BK/4),
//       one 16-byte load each, stored transposed (k-major, rows padded to
//       BM + 4 floats) as four floats, the row's quad of four XOR-ed with
//       the k chunk (bits 0-2) so that a warp's transposed stores are
//       conflict-free (the counts give the logical position k, row);
//     B tile, rows lid1 + L1 r (< BK), vector columns lid0 + L0 q (q < 2),
//       one 16-byte load and one 16-byte shared store each;
//     barrier;
//     for kk < BK: two 16-byte shared loads of A (8 rows), two of B
//       (vectors lid0 and L0 + lid0 of row kk, so the 16-byte words of
//       consecutive threads are adjacent and the loads are bank-conflict
//       free), 64 fused multiply-adds;
//   16 vector stores of C.
// The shared-memory tiles take (BM + 4 + BN) * BK * 4 bytes (up to 129 KiB).
//
// Stencil tile family "fd_block" (12 shapes BX x BY, V = 4 or 8 outputs per
// work-item): the five-point stencil on an input with a padded row pitch
// P = n + 4 (16-byte multiple, as TMA requires), one BY x BX output tile per
// work-group of (BX/V) x BY work-items.  Work-item (0, 0) copies the
// (BY + 2) x (BX + 4) input box into shared memory with one TMA load
// (mbarrier completion, bounded wait); after a barrier every work-item reads
// V + 2 centre-row and 2V north/south values, computes V consecutive outputs
// (3 adds, 1 multiply, 1 multiply-add each) and stores them as V/4 16-byte
// vectors.  V = 8 halves the threads per tile, so twice as many tiles (and
// TMA copies in flight) fit on an SM.
#include <cuda.h>
#include <cuda_runtime.h>

#include "pm_internal.h"
#include "pm_tma.cuh"

namespace pm {
namespace {

template <int BM, int BN, int BK>
__global__ void __launch_bounds__((BM / 8) * (BN / 8)) k_mm_simt(const float4 *__restrict__ A4, const float4 *__restrict__ B4,
                                                              float4 *__restrict__ C4, int n) {
    constexpr int L0 = BN / 8, L1 = BM / 8, KC = BK / 4, NC = BN / 4;
    constexpr int QA = (KC + L0 - 1) / L0, RB = (BK + L1 - 1) / L1;
    constexpr int BMP = BM + 4;       // padded row (16-byte aligned rows of the transposed tile)
    extern __shared__ __align__(16) float smem[];
    float *As = smem;                 // [BK][BMP]
    float *Bs = smem + BK * BMP;      // [BK][BN]
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const size_t n4 = (size_t)n / 4;
    const size_t arow0 = (size_t)BM * blockIdx.y;
    // acc[i][h] = C(row i, columns 2h and 2h + 1): two fused multiply-adds per
    // paired instruction (FFMA2), each the same single-rounded FMA as before
    float2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int h = 0; h < 4; h++) acc[i][h] = make_float2(0.0f, 0.0f);
    const int K = n / BK;
    for (int kt = 0; kt < K; kt++) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const int row = l1 + L1 * r;
#pragma unroll
            for (int q = 0; q < QA; q++) {
                const int c = l0 + L0 * q;
                if (c < KC) {
                    const float4 v = A4[n4 * (arow0 + row) + (size_t)KC * kt + c];
                    // row quad XOR-swizzled by the k chunk: a warp's transposed
                    // stores (k rows 4c + e, c over the lanes) fall in distinct banks
                    const int pr = (((row >> 2) ^ (c & 7)) << 2) | (row & 3);
                    As[(4 * c + 0) * BMP + pr] = v.x;
                    As[(4 * c + 1) * BMP + pr] = v.y;
                    As[(4 * c + 2) * BMP + pr] = v.z;
                    As[(4 * c + 3) * BMP + pr] = v.w;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RB; r++) {
            const int row = l1 + L1 * r;
            if (row < BK) {
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const int c = l0 + L0 * q;
                    reinterpret_cast<float4 *>(Bs)[row * NC + c] =
                        B4[n4 * ((size_t)BK * kt + row) + (size_t)NC * blockIdx.x + c];
                }
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; kk++) {
            const int sw = (kk >> 2) & 7;   // the swizzle of k row kk
            const float4 a0 = reinterpret_cast<const float4 *>(As)[kk * (BMP / 4) + ((2 * l1) ^ sw)];
            const float4 a1 = reinterpret_cast<const float4 *>(As)[kk * (BMP / 4) + ((2 * l1 + 1) ^ sw)];
            // vectors lid0 and L0 + lid0: consecutive threads read consecutive 16-byte words
            const float4 b0 = reinterpret_cast<const float4 *>(Bs)[kk * NC + l0];
            const float4 b1 = reinterpret_cast<const float4 *>(Bs)[kk * NC + L0 + l0];
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                                 make_float2(b1.z, b1.w)};
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const float2 ai = make_float2(a[i], a[i]);
#pragma unroll
                for (int h = 0; h < 4; h++) acc[i][h] = __ffma2_rn(ai, b[h], acc[i][h]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const size_t row = arow0 + 8 * l1 + i;
#pragma unroll
        for (int h = 0; h < 2; h++)
            C4[n4 * row + (size_t)NC * blockIdx.x + l0 + L0 * h] =
                make_float4(acc[i][2 * h].x, acc[i][2 * h].y, acc[i][2 * h + 1].x, acc[i][2 * h + 1].y);
    }
}

template <int BM, int BN, int BK>
pm_status launch_simt_t(void *const *b, int n, cudaStream_t st) {
    constexpr size_t smem = (size_t)(BM + 4 + BN) * BK * sizeof(float);
    auto fn = k_mm_simt<BM, BN, BK>;
    PM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(n / BN, n / BM), blk(BN / 8, BM / 8);
    launch_k(fn, grid, blk, smem, st, (const float4 *)b[0], (const float4 *)b[1], (float4 *)b[2], n);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

template <int BM, int BN>
pm_status launch_simt_bk(int BK, void *const *b, int n, cudaStream_t st) {
    return BK == 32 ? launch_simt_t<BM, BN, 32>(b, n, st) : launch_simt_t<BM, BN, 64>(b, n, st);
}

template <int BM>
pm_status launch_simt_bn(int BN, int BK, void *const *b, int n, cudaStream_t st) {
    switch (BN) {
    case 64: return launch_simt_bk<BM, 64>(BK, b, n, st);
    case 128: return launch_simt_bk<BM, 128>(BK, b, n, st);
    default: return launch_simt_bk<BM, 256>(BK, b, n, st);
    }
}

// ---------------------------------------------------------------- stencil tile family
static __device__ int g_fdb_timeout;

template <int BX, int BY, int V>
__global__ void __launch_bounds__((BX / V) * BY) k_fd_block(const __grid_constant__ CUtensorMap tmU,
                                                         float *__restrict__ res, int n, float c0, float c1) {
    constexpr int TW = BX + 4, TH = BY + 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // align by an offset into the shared array itself: a pointer that went
    // through an integer would lose the shared address space, and every
    // access through it would become a generic load or store
    const unsigned pad = (128u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u;
    float *T = reinterpret_cast<float *>(smem_raw + pad);
    uint64_t *bar = reinterpret_cast<uint64_t *>(T + TW * TH + 2);   // 8-byte aligned (TW * TH even)
    const int lx = threadIdx.x, ly = threadIdx.y;
    const bool leader = lx == 0 && ly == 0;
    if (leader) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (leader) {
        mbar_expect_tx(bar, (uint32_t)(TW * TH * sizeof(float)));
        tma_load_2d(T, &tmU, bar, BX * blockIdx.x, BY * blockIdx.y);
    }
    bool ok = mbar_wait_bounded(bar, 0, &g_fdb_timeout, 1ll << 26);
    if (!ok && leader) mbar_drain(bar, 0, 1ll << 26);   // drain our own copy
    if (!ok) return;
    const float *r0 = T + ly * TW + V * lx;       // north row
    const float *r1 = r0 + TW;                    // centre row
    const float *r2 = r1 + TW;                    // south row
    float m[V + 2], o[V];
#pragma unroll
    for (int q = 0; q < V + 2; q++) m[q] = r1[q];
#pragma unroll
    for (int q = 1; q <= V; q++)
        o[q - 1] = __fmaf_rn(c0, m[q], __fmul_rn(c1, __fadd_rn(__fadd_rn(__fadd_rn(r0[q], r2[q]), m[q - 1]), m[q + 1])));
    const size_t row = (size_t)BY * blockIdx.y + ly;
    float4 *dst = reinterpret_cast<float4 *>(res) + row * (n / 4) + (size_t)(BX / 4) * blockIdx.x + (V / 4) * lx;
#pragma unroll
    for (int h = 0; h < V / 4; h++) dst[h] = make_float4(o[4 * h], o[4 * h + 1], o[4 * h + 2], o[4 * h + 3]);
}

template <int BX, int BY, int V>
pm_status launch_fdb_t(void *const *b, int n, float c0, float c1, cudaStream_t st) {
    constexpr int TW = BX + 4, TH = BY + 2;
    const size_t smem = 128 + (size_t)TW * TH * sizeof(float) + 32;
    CUtensorMap tm;
    const uint64_t P = (uint64_t)n + 4;
    pm_status s = tensor_map_2d(&tm, 0, b[0], P, (uint64_t)n + 2, P * sizeof(float), TW, TH, 0);
    if (s) return s;
    dim3 grid(n / BX, n / BY), blk(BX / V, BY);
    launch_k(k_fd_block<BX, BY, V>, grid, blk, smem, st, tm, (float *)b[1], n, c0, c1);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

template <int BX, int V>
pm_status launch_fdb_by(int BY, void *const *b, int n, float c0, float c1, cudaStream_t st) {
    switch (BY) {
    case 4: return launch_fdb_t<BX, 4, V>(b, n, c0, c1, st);
    case 8: return launch_fdb_t<BX, 8, V>(b, n, c0, c1, st);
    case 16: return launch_fdb_t<BX, 16, V>(b, n, c0, c1, st);
    default: return launch_fdb_t<BX, 32, V>(b, n, c0, c1, st);
    }
}

template <int V>
pm_status launch_fdb_v(int BX, int BY, void *const *b, int n, float c0, float c1, cudaStream_t st) {
    switch (BX) {
    case 32: return launch_fdb_by<32, V>(BY, b, n, c0, c1, st);
    case 64: return launch_fdb_by<64, V>(BY, b, n, c0, c1, st);
    default: return launch_fdb_by<128, V>(BY, b, n, c0, c1, st);
    }
}

// ---------------------------------------------------------------- DG tile
// res[m, k, i] = sum_j D[m, i, j] u[k, j] for one m (blockIdx.x < 3) and
// 128 elements k (blockIdx.y) per CTA, as one product C (128 x NPP) =
// U (128 x 2Q) Dt^T.  NB = ceil(Np / 16) columns per thread over
// XL = ceil(Np / NB) x-lanes (XL x 16 threads), so the rows of Dt are padded
// only to NPP = XL NB (exact for Np = 20, 56, 84); j runs in Q = ceil(Np / 2)
// pairs.  Operands are read as 8-byte pairs: on GB300 a warp-wide 8-byte
// shared load that only a few addresses feed (the u rows: 2-4 per warp)
// costs about a quarter of a 16-byte one, and the XL distinct Dt rows of a
// warp fall in distinct bank pairs (row pitch PD % 32 == 2).  Thread (x, y)
// accumulates rows y + 16 a (a < 8) and columns x + XL b (b < NB) in
// registers.  The three CTAs of a tile are adjacent in launch order, so the
// tile is read from HBM once.  The u tile (contiguous, rows x Np floats)
// arrives by one bulk copy on the TMA engine while the threads stage D with
// 8-byte loads and stores; when Np is odd the rows are then re-laid out with
// pitch 2Q behind a second barrier.  The mbarrier wait is bounded (error
// word; a thread that gives up still passes the second barrier and stores
// nothing).
static __device__ int g_dgt_timeout;

__host__ __device__ constexpr int dgt_pd(int Q) { return 2 * Q + ((34 - (2 * Q) % 32) % 32); }
__host__ __device__ constexpr int dgt_xl(int Np, int NB) { return (Np + NB - 1) / NB; }

size_t dgt_smem(int Np) {
    const int Q = (Np + 1) / 2, NB = (Np + 15) / 16, NPP = dgt_xl(Np, NB) * NB;
    return (size_t)128 * 2 * Q * 4 + (Np % 2 ? (size_t)128 * Np * 4 : 0) + (size_t)NPP * dgt_pd(Q) * 4 + 8;
}

// NPC: Np fixed at compile time (the paper's sizes), 0 = taken from the
// argument.  Six CTAs per SM for Np = 20 (64 registers, no spills; measured
// 4 % faster than five at 68 registers at 2^20 elements, which was 7 % faster
// than the unconstrained 72)
template <int NB, int NPC>
__global__ void __launch_bounds__(NPC ? 16 * dgt_xl(NPC, NB) : 256, (NPC && NB <= 2) ? 6 : (NB <= 3 ? 3 : 2))
    k_dg_tile(const float *__restrict__ D, const float *__restrict__ u, float *__restrict__ res, int np_arg, int Nel) {
    constexpr int QBM = NB / 2 + 2;   // bound on ceil(Q / XL)
    const int Np = NPC ? NPC : np_arg;
    const int XL = dgt_xl(Np, NB), NPP = XL * NB, Q = (Np + 1) / 2, PD = dgt_pd(Q), P2 = PD / 2;
    const int QB = (Q + XL - 1) / XL, RB = (NPP + 15) / 16;
    const bool even = (Np & 1) == 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Us = reinterpret_cast<float *>(smem_raw);   // 16-byte aligned; stays a shared-space pointer
    float *R = Us + 128 * 2 * Q;                       // raw rows (odd Np only)
    float *Dt = R + (even ? 0 : 128 * Np);
    uint64_t *bar = reinterpret_cast<uint64_t *>(Dt + NPP * PD);
    const int x = threadIdx.x, y = threadIdx.y, m = blockIdx.x;
    const bool leader = x == 0 && y == 0;
    const long long k0 = 128LL * blockIdx.y;
    const int rows = (int)min(128LL, (long long)Nel - k0);
    if (leader) {
        mbar_init(bar, 1);
        mbar_init_fence();
        const uint32_t bytes = (uint32_t)rows * (uint32_t)Np * 4u;
        mbar_expect_tx(bar, bytes);
        bulk_load(even ? Us : R, u + k0 * Np, bytes, bar);
    }
    // D staging: all of a thread's loads in flight before its stores
    {
        float2 dv[NB][QBM];
#pragma unroll
        for (int ib = 0; ib < NB; ib++)
#pragma unroll
            for (int qb = 0; qb < QBM; qb++) {
                const int i = y + 16 * ib, q = x + XL * qb;
                float2 d = make_float2(0.0f, 0.0f);
                if (ib < RB && qb < QB && q < Q && i < Np) {
                    const float *src = D + (m * Np + i) * Np + 2 * q;
                    if (even) {
                        d = __ldg(reinterpret_cast<const float2 *>(src));
                    } else {
                        d.x = __ldg(src);
                        if (2 * q + 1 < Np) d.y = __ldg(src + 1);
                    }
                }
                dv[ib][qb] = d;
            }
#pragma unroll
        for (int ib = 0; ib < NB; ib++)
#pragma unroll
            for (int qb = 0; qb < QBM; qb++) {
                const int i = y + 16 * ib, q = x + XL * qb;
                if (ib < RB && qb < QB && q < Q && i < NPP) reinterpret_cast<float2 *>(Dt + i * PD)[q] = dv[ib][qb];
            }
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(bar, 0, &g_dgt_timeout, 1ll << 26);
    if (!ok && leader) mbar_drain(bar, 0, 1ll << 26);   // drain our own copy
    if (!even) {
        if (ok)
#pragma unroll
            for (int rb = 0; rb < 8; rb++)
                for (int qb = 0; qb < QB; qb++) {
                    const int r = y + 16 * rb, q = x + XL * qb;
                    if (q >= Q) continue;
                    const float *src = R + r * Np + 2 * q;
                    const float2 t = make_float2(src[0], 2 * q + 1 < Np ? src[1] : 0.0f);
                    reinterpret_cast<float2 *>(Us + r * 2 * Q)[q] = t;
                }
        __syncthreads();
    }
    if (!ok) return;
    // acc[a][b] = (sum over even j, sum over odd j): one paired FMA (FFMA2)
    // per loaded pair of u and D values, combined by one add at the end
    float2 acc[8][NB];
#pragma unroll
    for (int a = 0; a < 8; a++)
#pragma unroll
        for (int b = 0; b < NB; b++) acc[a][b] = make_float2(0.0f, 0.0f);
    const float2 *U2 = reinterpret_cast<const float2 *>(Us) + y * Q;
    const float2 *D2 = reinterpret_cast<const float2 *>(Dt) + x * P2;
#pragma unroll((NPC && NB < 6) ? 2 : 1)
    for (int q = 0; q < Q; q++) {
        float2 av[8];
#pragma unroll
        for (int a = 0; a < 8; a++) av[a] = U2[16 * a * Q + q];
#pragma unroll
        for (int b = 0; b < NB; b++) {
            const float2 bv = D2[XL * b * P2 + q];
#pragma unroll
            for (int a = 0; a < 8; a++) acc[a][b] = __ffma2_rn(av[a], bv, acc[a][b]);
        }
    }
    float *out = res + (long long)m * Nel * Np;
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const int i = x + XL * b;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            const float r = __fadd_rn(acc[a][b].x, acc[a][b].y);
            const long long k = k0 + y + 16 * a;
            if (i < Np && k < Nel) out[k * Np + i] = r;
        }
    }
}

template <int NB, int NPC>
pm_status launch_dgt_t(void *const *b, int Np, int Nel, cudaStream_t st) {
    const size_t smem = dgt_smem(Np);
    auto fn = k_dg_tile<NB, NPC>;
    PM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    launch_k(fn, dim3(3, (unsigned)((Nel + 127) / 128)), dim3((unsigned)dgt_xl(Np, NB), 16), smem, st,
             (const float *)b[0], (const float *)b[1], (float *)b[2], Np, Nel);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

// Test of the bounded-wait path: one thread waits on an mbarrier whose
// phase nothing completes (no arrival, no copy), through the dg_tile kernel's
// wait and error word.
__global__ void k_wait_nothing(long long polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        mbar_wait_bounded(&bar, 0, &g_dgt_timeout, polls);
    }
}

}  // namespace

pm_status dgt_check_timeout() {
    int v = 0, z = 0;
    PM_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_dgt_timeout, sizeof v));
    if (v) {
        PM_CUDA_TRY(cudaMemcpyToSymbol(g_dgt_timeout, &z, sizeof z));
        return fail(PM_ETIMEOUT, "dg_tile: a bounded wait gave up");
    }
    return PM_OK;
}

pm_status fdb_check_timeout() {
    int v = 0, z = 0;
    PM_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_fdb_timeout, sizeof v));
    if (v) {
        PM_CUDA_TRY(cudaMemcpyToSymbol(g_fdb_timeout, &z, sizeof z));
        return fail(PM_ETIMEOUT, "fd_block: a bounded wait gave up");
    }
    return PM_OK;
}

pm_status launch_tiles(const KP &kp, void *const *b, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (kp.def->fam == FAM_DGT) {
        const int Np = (int)kp.i(0), Nel = (int)kp.i(1);
        for (int a = 0; a < 2; a++)
            if ((uintptr_t)b[a] % 16) return fail(PM_EINVAL, "dg_tile: buffer %d must be 16-byte aligned", a);
        switch (Np) {   // the paper's node counts, specialised
        case 20: return launch_dgt_t<2, 20>(b, Np, Nel, st);
        case 35: return launch_dgt_t<3, 35>(b, Np, Nel, st);
        case 56: return launch_dgt_t<4, 56>(b, Np, Nel, st);
        case 84: return launch_dgt_t<6, 84>(b, Np, Nel, st);
        default: break;
        }
        switch ((Np + 15) / 16) {
        case 1: return launch_dgt_t<1, 0>(b, Np, Nel, st);
        case 2: return launch_dgt_t<2, 0>(b, Np, Nel, st);
        case 3: return launch_dgt_t<3, 0>(b, Np, Nel, st);
        case 4: return launch_dgt_t<4, 0>(b, Np, Nel, st);
        case 5: return launch_dgt_t<5, 0>(b, Np, Nel, st);
        default: return launch_dgt_t<6, 0>(b, Np, Nel, st);
        }
    }
    if (kp.def->fam == FAM_FDB) {
        const int n = (int)kp.i(0), BX = (int)kp.i(1), BY = (int)kp.i(2), V = (int)kp.i(5);
        const float c0 = (float)kp.v[3], c1 = (float)kp.v[4];
        for (int a = 0; a < 2; a++)
            if ((uintptr_t)b[a] % 16) return fail(PM_EINVAL, "fd_block: buffer %d must be 16-byte aligned", a);
        if (V == 8) return launch_fdb_v<8>(BX, BY, b, n, c0, c1, st);
        return launch_fdb_v<4>(BX, BY, b, n, c0, c1, st);
    }
    if (kp.def->fam != FAM_SIMT) return fail(PM_EINVAL, "not a tile-family kernel");
    const int n = (int)kp.i(0), BM = (int)kp.i(1), BN = (int)kp.i(2), BK = (int)kp.i(3);
    for (int a = 0; a < 3; a++)
        if ((uintptr_t)b[a] % 16) return fail(PM_EINVAL, "mm_simt: buffer %d must be 16-byte aligned", a);
    switch (BM) {
    case 64: return launch_simt_bn<64>(BN, BK, b, n, st);
    case 96: return launch_simt_bn<96>(BN, BK, b, n, st);
    case 128: return launch_simt_bn<128>(BN, BK, b, n, st);
    default: return launch_simt_bn<256>(BN, BK, b, n, st);
    }
}

}  // namespace pm

extern "C" pm_status pm_test_bounded_wait(int64_t polls, void *stream) {
    using namespace pm;
    if (polls < 1 || polls > (1 << 20)) return fail(PM_EINVAL, "pm_test_bounded_wait: polls must be 1..2^20");
    cudaStream_t st = (cudaStream_t)stream;
    k_wait_nothing<<<1, 32, 0, st>>>((long long)polls);
    PM_CUDA_TRY(cudaGetLastError());
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    return dgt_check_timeout();
}
