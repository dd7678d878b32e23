// Modeled computations of Section "Results" and their work-removed
// (global-memory-only) twins of Algorithm 3.  Each kernel executes exactly
// the loop domain pm_counts describes (one CUDA thread per work-item, one CTA
// per work-group), so its features are exact.
//
//   matmul (Section "Matrix Multiplication"): C = A B, fp32, 16x16
//     work-groups, gid0 -> column tile, gid1 -> row tile.
//       PF:   per 16-wide k tile: barrier, stage a 16x16 tile of A and of B in
//             shared memory, barrier, 16 multiply-adds from shared memory.
//       noPF: n multiply-adds straight from global memory.
//   DG (Section "DG"): res[m,k,i] = sum_j D[m,i,j] u[k,j], m < 3,
//     k = L0 gid0 + lid0, i = L1 gid1 + lid1, guard i < Np.
//       noPF: j loop over global memory.
//       dmPF: j split by L0; per (m, j tile) the L1 x L0 tile of D is staged
//             in shared memory between two barriers.
//       uPF (square work-groups): j split by L1; per j tile the L0 x L1
//             tile of u is staged in shared memory (work-item (lid0, lid1)
//             fetches u[L0 gid0 + lid1, L1 jo + lid0], lid0 along j), loops
//             j tile -> j -> m with three accumulators.
//       dmPF-T: dmPF on the transposed layouts uT[j, k] and resT[m, i, k],
//             so lid0 (k) has stride 1 in both.
//   stencil (Section "Finite Differences"):
//     res[i,j] = c0 u[i+1,j+1] + c1 (u[i,j+1] + u[i+2,j+1] + u[i+1,j] + u[i+1,j+2]).
//       tile:   16x16 work-group stages a 16x16 tile (origin 14 gid) in shared
//               memory; the 14x14 interior computes.
//       tile18: 18x18 work-group stages an 18x18 tile (origin 16 gid); the
//               16x16 interior computes.
//       direct: 16x16 work-group, one output per work-item, 5 global loads.
//   Twins keep the loop nest and the kept global accesses, replace arithmetic
//   by tgt = tgt + load, keep the stores (writing tgt), and otherwise write tgt
//   to tgt_dest[(L1 gid1 + lid1) * (L0 G0) + L0 gid0 + lid0].
#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pm {
namespace {

// ---------------------------------------------------------------- matmul
__global__ void __launch_bounds__(256) k_mm_pf(const float *__restrict__ a, const float *__restrict__ b,
                                               float *__restrict__ c, int n) {
    __shared__ float at[16][16];
    __shared__ float bt[16][16];
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const size_t row = 16 * (size_t)blockIdx.y + l1, col = 16 * (size_t)blockIdx.x + l0;
    const float *arow = a + (size_t)n * row + l0;
    const float *bcol = b + (size_t)n * l1 + col;
    float acc = 0.0f;
    for (int ko = 0; ko < n / 16; ko++) {
        __syncthreads();
        at[l1][l0] = arow[16 * ko];
        bt[l1][l0] = bcol[(size_t)n * 16 * ko];
        __syncthreads();
#pragma unroll
        for (int ki = 0; ki < 16; ki++) acc = __fmaf_rn(at[l1][ki], bt[ki][l0], acc);
    }
    c[(size_t)n * row + col] = acc;
}

__global__ void __launch_bounds__(256) k_mm_nopf(const float *__restrict__ a, const float *__restrict__ b,
                                                 float *__restrict__ c, int n) {
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const size_t row = 16 * (size_t)blockIdx.y + l1, col = 16 * (size_t)blockIdx.x + l0;
    const float *arow = a + (size_t)n * row;
    const float *bcol = b + col;
    float acc = 0.0f;
#pragma unroll 8
    for (int k = 0; k < n; k++) acc = __fmaf_rn(arow[k], bcol[(size_t)n * k], acc);
    c[(size_t)n * row + col] = acc;
}

// variant: 2 PF-a, 3 PF-b, 4 noPF-a, 5 noPF-b
template <int V>
__global__ void __launch_bounds__(256) k_mm_twin(const float *__restrict__ x, float *__restrict__ dest, int n) {
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const size_t g0 = blockIdx.x, g1 = blockIdx.y;
    const size_t row = 16 * g1 + l1, col = 16 * g0 + l0;
    float t = 0.0f;
    if (V == 2)
        for (int ko = 0; ko < n / 16; ko++) t = __fadd_rn(t, x[(size_t)n * row + 16 * ko + l0]);
    if (V == 3)
        for (int ko = 0; ko < n / 16; ko++) t = __fadd_rn(t, x[(size_t)n * (16 * ko + l1) + col]);
    if (V == 4)
        for (int k = 0; k < n; k++) t = __fadd_rn(t, x[(size_t)n * row + k]);
    if (V == 5)
        for (int k = 0; k < n; k++) t = __fadd_rn(t, x[(size_t)n * k + col]);
    dest[(size_t)n * row + col] = t;
}

pm_status launch_mm(const KP &kp, void *const *b, cudaStream_t st) {
    int n = (int)kp.i(0);
    dim3 grid(n / 16, n / 16), blk(16, 16);
    switch (kp.def->variant) {
    case 0: launch_k(k_mm_pf, grid, blk, 0, st, (const float *)b[0], (const float *)b[1], (float *)b[2], n); break;
    case 1: launch_k(k_mm_nopf, grid, blk, 0, st, (const float *)b[0], (const float *)b[1], (float *)b[2], n); break;
    case 2: launch_k(k_mm_twin<2>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n); break;
    case 3: launch_k(k_mm_twin<3>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n); break;
    case 4: launch_k(k_mm_twin<4>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n); break;
    default: launch_k(k_mm_twin<5>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n); break;
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

// ---------------------------------------------------------------- DG
template <int L0, int L1>
__global__ void __launch_bounds__(L0 *L1) k_dg_nopf(const float *__restrict__ D, const float *__restrict__ u,
                                                    float *__restrict__ res, int Np, int Nel) {
    const int k = L0 * blockIdx.x + threadIdx.x, i = L1 * blockIdx.y + threadIdx.y;
    if (i >= Np) return;
    const float *uk = u + (size_t)Np * k;
    for (int m = 0; m < 3; m++) {
        const float *Dm = D + (size_t)Np * Np * m + (size_t)Np * i;
        float acc = 0.0f;
        for (int j = 0; j < Np; j++) acc = __fmaf_rn(Dm[j], uk[j], acc);
        res[(size_t)Nel * Np * m + (size_t)Np * k + i] = acc;
    }
}

template <int L0, int L1>
__global__ void __launch_bounds__(L0 *L1) k_dg_dmpf(const float *__restrict__ D, const float *__restrict__ u,
                                                    float *__restrict__ res, int Np, int Nel) {
    __shared__ float Dt[L1 * L0];
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int k = L0 * blockIdx.x + l0, i = L1 * blockIdx.y + l1;
    const int nj = (Np + L0 - 1) / L0;
    const float *uk = u + (size_t)Np * k;
    for (int m = 0; m < 3; m++) {
        float acc = 0.0f;
        for (int jo = 0; jo < nj; jo++) {
            __syncthreads();
            if (i < Np && L0 * jo + l0 < Np) Dt[L0 * l1 + l0] = D[(size_t)Np * Np * m + (size_t)Np * i + L0 * jo + l0];
            __syncthreads();
            if (i < Np) {
                const int jn = min(L0, Np - L0 * jo);
                if (jn == L0) {
#pragma unroll
                    for (int ji = 0; ji < L0; ji++) acc = __fmaf_rn(Dt[L0 * l1 + ji], uk[L0 * jo + ji], acc);
                } else {
                    for (int ji = 0; ji < jn; ji++) acc = __fmaf_rn(Dt[L0 * l1 + ji], uk[L0 * jo + ji], acc);
                }
            }
        }
        if (i < Np) res[(size_t)Nel * Np * m + (size_t)Np * k + i] = acc;
    }
}

template <int L>
__global__ void __launch_bounds__(L *L) k_dg_upf(const float *__restrict__ D, const float *__restrict__ u,
                                                float *__restrict__ res, int Np, int Nel) {
    __shared__ float uf[L][L + 1];   // uf[k_in][j_in]
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int k = L * blockIdx.x + l0, i = L * blockIdx.y + l1;
    const int nj = (Np + L - 1) / L;
    const size_t NN = (size_t)Np * Np;
    const float *urow = u + (size_t)Np * (L * blockIdx.x + l1);
    const float *Di = D + (size_t)Np * i;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    for (int jo = 0; jo < nj; jo++) {
        __syncthreads();
        if (L * jo + l0 < Np) uf[l1][l0] = urow[L * jo + l0];
        __syncthreads();
        if (i < Np) {
            const int jn = min(L, Np - L * jo);
            for (int ji = 0; ji < jn; ji++) {
                const float x = uf[l0][ji];
                const int j = L * jo + ji;
                a0 = __fmaf_rn(Di[j], x, a0);
                a1 = __fmaf_rn(Di[NN + j], x, a1);
                a2 = __fmaf_rn(Di[2 * NN + j], x, a2);
            }
        }
    }
    if (i < Np) {
        const size_t o = (size_t)Np * k + i, M = (size_t)Nel * Np;
        res[o] = a0;
        res[M + o] = a1;
        res[2 * M + o] = a2;
    }
}

template <int L0, int L1>
__global__ void __launch_bounds__(L0 *L1) k_dg_dmpft(const float *__restrict__ D, const float *__restrict__ uT,
                                                     float *__restrict__ resT, int Np, int Nel) {
    __shared__ float Dt[L1 * L0];
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int k = L0 * blockIdx.x + l0, i = L1 * blockIdx.y + l1;
    const int nj = (Np + L0 - 1) / L0;
    const float *uk = uT + k;
    for (int m = 0; m < 3; m++) {
        float acc = 0.0f;
        for (int jo = 0; jo < nj; jo++) {
            __syncthreads();
            if (i < Np && L0 * jo + l0 < Np) Dt[L0 * l1 + l0] = D[(size_t)Np * Np * m + (size_t)Np * i + L0 * jo + l0];
            __syncthreads();
            if (i < Np) {
                const int jn = min(L0, Np - L0 * jo);
                const float *uj = uk + (size_t)Nel * L0 * jo;
                if (jn == L0) {
#pragma unroll
                    for (int ji = 0; ji < L0; ji++) acc = __fmaf_rn(Dt[L0 * l1 + ji], uj[(size_t)Nel * ji], acc);
                } else {
                    for (int ji = 0; ji < jn; ji++) acc = __fmaf_rn(Dt[L0 * l1 + ji], uj[(size_t)Nel * ji], acc);
                }
            }
        }
        if (i < Np) resT[(size_t)Nel * Np * m + (size_t)Nel * i + k] = acc;
    }
}

// variant: 2 noPF-u, 3 noPF-dm, 4 dmPF-u, 5 dmPF-dm, 6 res, 9 uPF-u,
// 10 dmPF-T-u (reads uT), 11 dmPF-T-res (writes resT)
template <int L0, int L1, int V>
__global__ void __launch_bounds__(L0 *L1) k_dg_twin(const float *__restrict__ D, const float *__restrict__ u,
                                                    float *__restrict__ out, int Np, int Nel) {
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int k = L0 * blockIdx.x + l0, i = L1 * blockIdx.y + l1;
    const int nj = (Np + L0 - 1) / L0;
    float t = 0.0f;
    if (V == 6) {
        if (i < Np)
            for (int m = 0; m < 3; m++) out[(size_t)Nel * Np * m + (size_t)Np * k + i] = t;
        return;
    }
    if (V == 11) {
        if (i < Np)
            for (int m = 0; m < 3; m++) out[(size_t)Nel * Np * m + (size_t)Nel * i + k] = t;
        return;
    }
    if (V == 9) {   // every work-item fetches, whatever its row
        const float *urow = u + (size_t)Np * (L0 * blockIdx.x + l1);
        const int njl = (Np + L1 - 1) / L1;
        for (int jo = 0; jo < njl; jo++)
            if (L1 * jo + l0 < Np) t = __fadd_rn(t, urow[L1 * jo + l0]);
    }

    if (V == 2) {
        if (i < Np)
            for (int m = 0; m < 3; m++)
                for (int j = 0; j < Np; j++) t = __fadd_rn(t, u[(size_t)Np * k + j]);
    }
    if (V == 4 || V == 10) {
        // the parent's j loop shape (full tiles unrolled) keeps its memory-level parallelism
        const float *uk = V == 4 ? u + (size_t)Np * k : u + k;
        const size_t js = V == 4 ? 1 : (size_t)Nel;
        if (i < Np)
            for (int m = 0; m < 3; m++)
                for (int jo = 0; jo < nj; jo++) {
                    const int jn = min(L0, Np - L0 * jo);
                    const float *uj = uk + js * L0 * jo;
                    if (jn == L0) {
#pragma unroll
                        for (int ji = 0; ji < L0; ji++) t = __fadd_rn(t, uj[js * ji]);
                    } else {
                        for (int ji = 0; ji < jn; ji++) t = __fadd_rn(t, uj[js * ji]);
                    }
                }
    }
    if (V == 3) {
        if (i < Np)
            for (int m = 0; m < 3; m++)
                for (int j = 0; j < Np; j++) t = __fadd_rn(t, D[(size_t)Np * Np * m + (size_t)Np * i + j]);
    }
    if (V == 5) {
        for (int m = 0; m < 3; m++)
            for (int jo = 0; jo < nj; jo++)
                if (i < Np && L0 * jo + l0 < Np)
                    t = __fadd_rn(t, D[(size_t)Np * Np * m + (size_t)Np * i + L0 * jo + l0]);
    }
    out[(size_t)Nel * i + k] = t;
}

template <int L0, int L1>
pm_status launch_dg_t(int var, void *const *b, int Np, int Nel, cudaStream_t st) {
    dim3 grid(Nel / L0, (Np + L1 - 1) / L1), blk(L0, L1);
    const float *D = nullptr, *u = nullptr;
    float *o = nullptr;
    switch (var) {
    case 0: launch_k(k_dg_nopf<L0, L1>, grid, blk, 0, st, (const float *)b[0], (const float *)b[1], (float *)b[2], Np, Nel); break;
    case 1: launch_k(k_dg_dmpf<L0, L1>, grid, blk, 0, st, (const float *)b[0], (const float *)b[1], (float *)b[2], Np, Nel); break;
    case 2: case 4:
        u = (const float *)b[0]; o = (float *)b[1];
        if (var == 2) launch_k(k_dg_twin<L0, L1, 2>, grid, blk, 0, st, D, u, o, Np, Nel);
        else launch_k(k_dg_twin<L0, L1, 4>, grid, blk, 0, st, D, u, o, Np, Nel);
        break;
    case 3: case 5:
        D = (const float *)b[0]; o = (float *)b[1];
        if (var == 3) launch_k(k_dg_twin<L0, L1, 3>, grid, blk, 0, st, D, u, o, Np, Nel);
        else launch_k(k_dg_twin<L0, L1, 5>, grid, blk, 0, st, D, u, o, Np, Nel);
        break;
    case 6:
        launch_k(k_dg_twin<L0, L1, 6>, grid, blk, 0, st, D, u, (float *)b[0], Np, Nel);
        break;
    case 7:
        if constexpr (L0 == L1)
            launch_k(k_dg_upf<L0>, grid, blk, 0, st, (const float *)b[0], (const float *)b[1], (float *)b[2], Np, Nel);
        else
            return fail(PM_EINVAL, "dg_upf needs a square work-group");
        break;
    case 8: launch_k(k_dg_dmpft<L0, L1>, grid, blk, 0, st, (const float *)b[0], (const float *)b[1], (float *)b[2], Np, Nel); break;
    case 9: case 10:
        u = (const float *)b[0]; o = (float *)b[1];
        if (var == 9) launch_k(k_dg_twin<L0, L1, 9>, grid, blk, 0, st, D, u, o, Np, Nel);
        else launch_k(k_dg_twin<L0, L1, 10>, grid, blk, 0, st, D, u, o, Np, Nel);
        break;
    default:
        launch_k(k_dg_twin<L0, L1, 11>, grid, blk, 0, st, D, u, (float *)b[0], Np, Nel);
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status launch_dg(const KP &kp, void *const *b, cudaStream_t st) {
    int Np = (int)kp.i(0), Nel = (int)kp.i(1), L0 = (int)kp.i(2);
    return L0 == 16 ? launch_dg_t<16, 16>(kp.def->variant, b, Np, Nel, st)
                    : launch_dg_t<32, 8>(kp.def->variant, b, Np, Nel, st);
}

// ---------------------------------------------------------------- stencil
__device__ __forceinline__ float fd_combine(float c0, float c1, float C, float N, float S, float Wv, float E) {
    // 3 adds, 1 mul, 1 multiply-add
    const float s = __fadd_rn(__fadd_rn(__fadd_rn(N, S), Wv), E);
    return __fmaf_rn(c0, C, __fmul_rn(c1, s));
}

// T x T work-group, tile origin (T - 2) gid, interior (T - 2) x (T - 2)
template <int T>
__global__ void __launch_bounds__(T *T) k_fd_tile(const float *__restrict__ u, float *__restrict__ res, int n,
                                                 float c0, float c1) {
    __shared__ float t[T][T];
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int W = n + 2;
    const int r = (T - 2) * blockIdx.y + l1, q = (T - 2) * blockIdx.x + l0;
    if (r < W && q < W) t[l1][l0] = u[(size_t)W * r + q];
    __syncthreads();
    if (l0 >= 1 && l0 <= T - 2 && l1 >= 1 && l1 <= T - 2 && r - 1 < n && q - 1 < n)
        res[(size_t)n * (r - 1) + (q - 1)] =
            fd_combine(c0, c1, t[l1][l0], t[l1 - 1][l0], t[l1 + 1][l0], t[l1][l0 - 1], t[l1][l0 + 1]);
}

__global__ void __launch_bounds__(256) k_fd_direct(const float *__restrict__ u, float *__restrict__ res, int n,
                                                   float c0, float c1) {
    const int i = 16 * blockIdx.y + threadIdx.y, j = 16 * blockIdx.x + threadIdx.x;
    if (i >= n || j >= n) return;
    const size_t W = (size_t)n + 2;
    const float *p = u + W * i + j;
    res[(size_t)n * i + j] = fd_combine(c0, c1, p[W + 1], p[1], p[2 * W + 1], p[W], p[W + 2]);
}

// variant 2 tile-u, 3 tile-res, 4 direct-u, 5 direct-res; T the work-group
// width of the tile variants (16 or 18)
template <int V, int T>
__global__ void __launch_bounds__(T *T) k_fd_twin(const float *__restrict__ u, float *__restrict__ out, int n) {
    const int l0 = threadIdx.x, l1 = threadIdx.y;
    const int W = n + 2;
    float t = 0.0f;
    if (V == 2 || V == 3) {
        const int r = (T - 2) * blockIdx.y + l1, q = (T - 2) * blockIdx.x + l0;
        if (V == 2) {
            if (r < W && q < W) t = __fadd_rn(t, u[(size_t)W * r + q]);
            out[(size_t)T * gridDim.x * (T * blockIdx.y + l1) + T * blockIdx.x + l0] = t;
        } else if (l0 >= 1 && l0 <= T - 2 && l1 >= 1 && l1 <= T - 2 && r - 1 < n && q - 1 < n) {
            out[(size_t)n * (r - 1) + (q - 1)] = t;
        }
    } else {
        const int i = 16 * blockIdx.y + l1, j = 16 * blockIdx.x + l0;
        const bool in = i < n && j < n;
        if (V == 4) {
            if (in) {
                const float *p = u + (size_t)W * i + j;
                t = __fadd_rn(t, p[(size_t)W + 1]);
                t = __fadd_rn(t, p[1]);
                t = __fadd_rn(t, p[2 * (size_t)W + 1]);
                t = __fadd_rn(t, p[(size_t)W]);
                t = __fadd_rn(t, p[(size_t)W + 2]);
            }
            out[(size_t)16 * gridDim.x * i + j] = t;
        } else if (in) {
            out[(size_t)n * i + j] = t;
        }
    }
}

pm_status launch_fd(const KP &kp, void *const *b, cudaStream_t st) {
    int n = (int)kp.i(0);
    float c0 = (float)kp.v[1], c1 = (float)kp.v[2];
    int var = kp.def->variant;
    int G = (var == 0 || var == 2 || var == 3) ? (n + 13) / 14 : (n + 15) / 16;
    const int T = var >= 6 ? 18 : 16;
    dim3 grid(G, G), blk(T, T);
    switch (var) {
    case 0: launch_k(k_fd_tile<16>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n, c0, c1); break;
    case 1: launch_k(k_fd_direct, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n, c0, c1); break;
    case 2: launch_k(k_fd_twin<2, 16>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n); break;
    case 3: launch_k(k_fd_twin<3, 16>, grid, blk, 0, st, nullptr, (float *)b[0], n); break;
    case 4: launch_k(k_fd_twin<4, 16>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n); break;
    case 5: launch_k(k_fd_twin<5, 16>, grid, blk, 0, st, nullptr, (float *)b[0], n); break;
    case 6: launch_k(k_fd_tile<18>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n, c0, c1); break;
    case 7: launch_k(k_fd_twin<2, 18>, grid, blk, 0, st, (const float *)b[0], (float *)b[1], n); break;
    default: launch_k(k_fd_twin<3, 18>, grid, blk, 0, st, nullptr, (float *)b[0], n); break;
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

}  // namespace

pm_status launch_modeled(const KP &kp, void *const *b, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (kp.def->fam) {
    case FAM_MM: return launch_mm(kp, b, st);
    case FAM_DG: return launch_dg(kp, b, st);
    case FAM_FD: return launch_fd(kp, b, st);
    default: return fail(PM_EINVAL, "not a modeled kernel");
    }
}

}  // namespace pm
