// Autotuning spaces: the register-tiled SIMT fp32 matmul family (24 tile
// shapes).  Loop nest (the one pm_counts counts), work-group (BN/8) x (BM/8),
// every work-item owns an 8 x 8 block of C:
//   per k tile of width BK:
//     barrier;
//     A tile, rows lid1 + L1 r (r < 8), vector columns lid0 + L0 q (< BK/4),
//       one 16-byte load each, stored transposed (k-major) as four floats;
//     B tile, rows lid1 + L1 r (< BK), vector columns lid0 + L0 q (q < 2),
//       one 16-byte load and one 16-byte shared store each;
//     barrier;
//     for kk < BK: two 16-byte shared loads of A (8 rows), two of B (8
//       columns), 64 fused multiply-adds;
//   16 vector stores of C.
// The shared-memory tiles take (BM + BN) * BK * 4 bytes (up to 128 KiB).
#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pm {
namespace {

template <int BM, int BN, int BK>
__global__ void __launch_bounds__((BM / 8) * (BN / 8)) k_mm_simt(const float4 *__restrict__ A4, const float4 *__restrict__ B4,
                                                              float4 *__restrict__ C4, int n) {
    constexpr int L0 = BN / 8, L1 = BM / 8, KC = BK / 4, NC = BN / 4;
    constexpr int QA = (KC + L0 - 1) / L0, RB = (BK + L1 - 1) / L1;
    extern __shared__ __align__(16) float smem[];
    float *As = smem;                 // [BK][BM]
    float *Bs = smem + BK * BM;       // [BK][BN]
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const size_t n4 = (size_t)n / 4;
    const size_t arow0 = (size_t)BM * blockIdx.y;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.0f;
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
                    As[(4 * c + 0) * BM + row] = v.x;
                    As[(4 * c + 1) * BM + row] = v.y;
                    As[(4 * c + 2) * BM + row] = v.z;
                    As[(4 * c + 3) * BM + row] = v.w;
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
            const float4 a0 = reinterpret_cast<const float4 *>(As)[kk * (BM / 4) + 2 * l1];
            const float4 a1 = reinterpret_cast<const float4 *>(As)[kk * (BM / 4) + 2 * l1 + 1];
            const float4 b0 = reinterpret_cast<const float4 *>(Bs)[kk * NC + 2 * l0];
            const float4 b1 = reinterpret_cast<const float4 *>(Bs)[kk * NC + 2 * l0 + 1];
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const size_t row = arow0 + 8 * l1 + i;
#pragma unroll
        for (int h = 0; h < 2; h++)
            C4[n4 * row + (size_t)NC * blockIdx.x + 2 * l0 + h] =
                make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
    }
}

template <int BM, int BN, int BK>
pm_status launch_simt_t(void *const *b, int n, cudaStream_t st) {
    constexpr size_t smem = (size_t)(BM + BN) * BK * sizeof(float);
    auto fn = k_mm_simt<BM, BN, BK>;
    PM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(n / BN, n / BM), blk(BN / 8, BM / 8);
    fn<<<grid, blk, smem, st>>>((const float4 *)b[0], (const float4 *)b[1], (float4 *)b[2], n);
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

}  // namespace

pm_status launch_tiles(const KP &kp, void *const *b, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
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
