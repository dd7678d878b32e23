// Calibration-suite measurement kernels (Section "Measurement Kernel Design"):
// global-memory stream, arithmetic loop, local-memory shuffle, local barrier,
// local/global overlap (Section "Modeling Operation Overlap") and empty.
//
// Each kernel executes exactly the loop domain that pm_counts describes: one
// CUDA thread per work-item, one CTA per work-group; large logical 2-D grids
// are flattened onto gridDim.x (gid0 = blockIdx.x mod G0, gid1 = blockIdx.x /
// G0, the same issue order as a 2-D grid).
#include <cuda_runtime.h>

#include "pm_internal.h"

namespace pm {
namespace {

// ---------------------------------------------------------------- stream
// out[idx] = in0[idx] + in1[idx] + ... (left to right), element type T (a
// scalar or a 16-byte vector added lane by lane).
template <typename T> struct VAdd;
template <> struct VAdd<float> { __device__ static float f(float a, float b) { return __fadd_rn(a, b); } };
template <> struct VAdd<double> { __device__ static double f(double a, double b) { return __dadd_rn(a, b); } };
template <> struct VAdd<float4> {
    __device__ static float4 f(float4 a, float4 b) {
        return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
    }
};
template <> struct VAdd<double2> {
    __device__ static double2 f(double2 a, double2 b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
};

// shape 0: 256 work-items, idx = s*lid0 + gid0 + 256*s*gid1, grid (s, M/(256 s)).
// shape 1: 16x16 work-items, idx = lid0 + W*lid1 + 16*gid0 + 16*W*gid1, grid (W/16, M/(16 W)).
template <typename T, int L, int SHAPE>
__global__ void __launch_bounds__(256) k_stream(const T *__restrict__ in0, const T *__restrict__ in1,
                                                const T *__restrict__ in2, const T *__restrict__ in3,
                                                T *__restrict__ out, int log2s_or_W, int G0) {
    unsigned g0, g1;
    size_t idx;
    if (SHAPE == 0) {
        const int ls = log2s_or_W;
        g0 = blockIdx.x & ((1u << ls) - 1u);
        g1 = blockIdx.x >> ls;
        idx = ((size_t)threadIdx.x << ls) + g0 + ((size_t)g1 << (8 + ls));
    } else {
        const size_t W = (size_t)log2s_or_W;
        g0 = blockIdx.x % (unsigned)G0;
        g1 = blockIdx.x / (unsigned)G0;
        idx = threadIdx.x + W * threadIdx.y + 16 * (size_t)g0 + 16 * W * g1;
    }
    // read-only (non-coherent) loads: 5 % faster at unit stride, equal at larger strides
    T v = __ldg(in0 + idx);
    if (L > 1) v = VAdd<T>::f(v, __ldg(in1 + idx));
    if (L > 2) v = VAdd<T>::f(v, __ldg(in2 + idx));
    if (L > 3) v = VAdd<T>::f(v, __ldg(in3 + idx));
    out[idx] = v;
}

template <typename T, int SHAPE>
pm_status launch_stream_t(int L, void *const *b, int arg, int G0, unsigned grid, cudaStream_t st) {
    const T *i0 = (const T *)b[0];
    const T *i1 = L > 1 ? (const T *)b[1] : nullptr;
    const T *i2 = L > 2 ? (const T *)b[2] : nullptr;
    const T *i3 = L > 3 ? (const T *)b[3] : nullptr;
    T *o = (T *)b[L];
    dim3 blk = SHAPE == 0 ? dim3(256) : dim3(16, 16);
    switch (L) {
    case 1: launch_k(k_stream<T, 1, SHAPE>, grid, blk, 0, st, i0, i1, i2, i3, o, arg, G0); break;
    case 2: launch_k(k_stream<T, 2, SHAPE>, grid, blk, 0, st, i0, i1, i2, i3, o, arg, G0); break;
    case 3: launch_k(k_stream<T, 3, SHAPE>, grid, blk, 0, st, i0, i1, i2, i3, o, arg, G0); break;
    default: launch_k(k_stream<T, 4, SHAPE>, grid, blk, 0, st, i0, i1, i2, i3, o, arg, G0); break;
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status launch_stream(const KP &kp, void *const *b, cudaStream_t st) {
    int dt = (int)kp.i(0), vec = (int)kp.i(1), L = (int)kp.i(4), shape = (int)kp.i(5);
    int64_t N = kp.i(2), s = kp.i(3), W = kp.i(6);
    int64_t w = vec ? (dt == 0 ? 4 : 2) : 1, M = N / w;
    int64_t nblk = M / 256;
    if (nblk > 0x7fffffffLL) return fail(PM_EINVAL, "stream: too many work-groups");
    unsigned grid = (unsigned)nblk;
    int arg, G0;
    if (shape == 0) {
        int ls = 0;
        while ((1LL << ls) < s) ls++;
        arg = ls;
        G0 = (int)s;
    } else {
        arg = (int)W;
        G0 = (int)(W / 16);
    }
    for (int a = 0; a <= L; a++)
        if (((uintptr_t)b[a]) % (vec ? 16 : (dt ? 8 : 4)))
            return fail(PM_EINVAL, "stream: buffer %d is not aligned to its element size", a);
#define PM_STREAM_CASE(T)                                                       \
    return shape == 0 ? launch_stream_t<T, 0>(L, b, arg, G0, grid, st)          \
                      : launch_stream_t<T, 1>(L, b, arg, G0, grid, st)
    if (dt == 0 && !vec) PM_STREAM_CASE(float);
    if (dt == 0 && vec) PM_STREAM_CASE(float4);
    if (dt == 1 && !vec) PM_STREAM_CASE(double);
    PM_STREAM_CASE(double2);
#undef PM_STREAM_CASE
}

// ---------------------------------------------------------------- arithmetic
// 32 private variables, x_t = u + t/32; F/32 rounds of x_t <- op(x_t) (each
// variable depends only on itself, 32 statements back); out = x_0 + ... + x_31.
// add: x + 2^-13; mul: x * (1 - 2^-12); madd: x * (1 - 2^-10) + 2^-10.
template <typename T> struct Ar;
template <> struct Ar<float> {
    __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Ar<double> {
    __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

template <typename T, int OP>
__global__ void __launch_bounds__(256) k_fma(const T *__restrict__ seed, T *__restrict__ out, int rounds) {
    const size_t gt = (size_t)blockIdx.x * 256 + threadIdx.x;
    const T u = seed[gt];
    T x[32];
#pragma unroll
    for (int t = 0; t < 32; t++) x[t] = Ar<T>::add(u, (T)t * (T)0.03125);
    const T ca = (T)0.0001220703125, ma = (T)0.999755859375, fa = (T)0.9990234375, fb = (T)0.0009765625;
#pragma unroll 2
    for (int r = 0; r < rounds; r++) {
#pragma unroll
        for (int t = 0; t < 32; t++) {
            if (OP == 0) x[t] = Ar<T>::add(x[t], ca);
            else if (OP == 1) x[t] = Ar<T>::mul(x[t], ma);
            else x[t] = Ar<T>::fma(x[t], fa, fb);
        }
    }
    T s = x[0];
#pragma unroll
    for (int t = 1; t < 32; t++) s = Ar<T>::add(s, x[t]);
    out[gt] = s;
}

template <typename T>
pm_status launch_fma_t(int op, const void *seed, void *out, int rounds, unsigned G, cudaStream_t st) {
    if (op == 0) launch_k(k_fma<T, 0>, G, 256, 0, st, (const T *)seed, (T *)out, rounds);
    else if (op == 1) launch_k(k_fma<T, 1>, G, 256, 0, st, (const T *)seed, (T *)out, rounds);
    else launch_k(k_fma<T, 2>, G, 256, 0, st, (const T *)seed, (T *)out, rounds);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

// ---------------------------------------------------------------- local memory
// Each work-item stores its element at slot lid0, passes a barrier, then moves
// it to slot 256+lid0 and back R/4 times (volatile: every access is issued),
// with a barrier per iteration when SYNC; finally writes slot lid0 out.
template <int SYNC>
__global__ void __launch_bounds__(256) k_smem(const float *__restrict__ in, float *__restrict__ out, int iters) {
    __shared__ float sm[512];
    volatile float *s = sm;
    const int l0 = threadIdx.x;
    const size_t gt = (size_t)blockIdx.x * 256 + l0;
    s[l0] = in[gt];
    __syncthreads();
    for (int r = 0; r < iters; r++) {
        s[256 + l0] = s[l0];
        s[l0] = s[256 + l0];
        if (SYNC) __syncthreads();
    }
    out[gt] = s[l0];
}

// 2-D variant: T x T work-group, local index a = T lid1 + lid0, slots a and
// T^2 + a; one barrier after the initial store.
template <int T>
__global__ void __launch_bounds__(T *T) k_smem2d(const float *__restrict__ in, float *__restrict__ out, int iters) {
    __shared__ float sm[2 * T * T];
    volatile float *s = sm;
    const int a = T * threadIdx.y + threadIdx.x;
    const size_t gt = (size_t)blockIdx.x * (T * T) + a;
    s[a] = in[gt];
    __syncthreads();
    for (int r = 0; r < iters; r++) {
        s[T * T + a] = s[a];
        s[a] = s[T * T + a];
    }
    out[gt] = s[a];
}

__global__ void __launch_bounds__(256) k_barrier(const float *__restrict__ in, float *__restrict__ out, int B) {
    const size_t gt = (size_t)blockIdx.x * 256 + threadIdx.x;
    const float v = in[gt];
    for (int b = 0; b < B; b++) __syncthreads();
    out[gt] = v;
}

// One global load, m local store/load pairs, one global store.
__global__ void __launch_bounds__(256) k_overlap(const float *__restrict__ in, float *__restrict__ out, int m) {
    __shared__ float sm[256];
    volatile float *s = sm;
    const int l0 = threadIdx.x;
    const size_t gt = (size_t)blockIdx.x * 256 + l0;
    float v = in[gt];
    for (int i = 0; i < m; i++) {
        s[l0] = v;
        v = s[l0];
    }
    out[gt] = v;
}

__global__ void __launch_bounds__(256) k_empty() {}

}  // namespace

pm_status launch_suite(const KP &kp, void *const *b, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    switch (kp.def->fam) {
    case FAM_STREAM: return launch_stream(kp, b, st);
    case FAM_FMA: {
        int dt = (int)kp.i(0), op = (int)kp.i(1);
        int rounds = (int)(kp.i(2) / 32);
        unsigned G = (unsigned)kp.i(3);
        return dt == 0 ? launch_fma_t<float>(op, b[0], b[1], rounds, G, st)
                       : launch_fma_t<double>(op, b[0], b[1], rounds, G, st);
    }
    case FAM_SMEM: {
        int iters = (int)(kp.i(0) / 4);
        unsigned G = (unsigned)kp.i(2);
        if (kp.i(1)) launch_k(k_smem<1>, G, 256, 0, st, (const float *)b[0], (float *)b[1], iters);
        else launch_k(k_smem<0>, G, 256, 0, st, (const float *)b[0], (float *)b[1], iters);
        break;
    }
    case FAM_SMEM2D: {
        int iters = (int)(kp.i(0) / 4);
        unsigned G = (unsigned)kp.i(2);
        if (kp.i(1) == 16) launch_k(k_smem2d<16>, G, dim3(16, 16), 0, st, (const float *)b[0], (float *)b[1], iters);
        else launch_k(k_smem2d<18>, G, dim3(18, 18), 0, st, (const float *)b[0], (float *)b[1], iters);
        break;
    }
    case FAM_BARRIER:
        launch_k(k_barrier, (unsigned)kp.i(1), 256, 0, st, (const float *)b[0], (float *)b[1], (int)kp.i(0));
        break;
    case FAM_OVERLAP:
        launch_k(k_overlap, (unsigned)(kp.i(1) / 256), 256, 0, st, (const float *)b[0], (float *)b[1], (int)kp.i(0));
        break;
    case FAM_EMPTY:
        launch_k(k_empty, (unsigned)kp.i(0), 256, 0, st);
        break;
    default:
        return fail(PM_EINVAL, "not a suite kernel");
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

}  // namespace pm
