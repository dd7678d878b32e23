// Per-model differentiation and the plain Levenberg-Marquardt calibration
// (Section "Computing Model Parameters": minimise the relative residual
// 1 - g(p; f_k)/t_k over the parameters with the model's derivatives, by
// Levenberg-Marquardt).
//
// * pm_residual / pm_residual_vjp / pm_jacobian: the residual of one model
//   on l rows, its vector-Jacobian product and its Jacobian, by reverse-mode
//   differentiation of the model program (the paper differentiates the model
//   symbolically).  They back the PyTorch autograd.Function.
// * pm_lm_init / pm_lm_step / pm_lm_update / pm_lm_report: the per-iteration
//   arithmetic of a host-driven LM loop over one model -- the damped step
//   solve and the accept / reject / damping update -- with the loop's state
//   in a caller-owned device buffer, so the caller's loop (autograd.py
//   lm_fit) only sequences calls and reads one status word per trial.
//
// Precision: per row the model program runs in float-float arithmetic on the
// FP32 pipes from FP64 features and outputs (split into hi + lo pairs as they
// are read).  The vector-Jacobian product, which fixes the solution (the LM
// stops where J^T r = 0), takes the float-float reverse sweep; the Jacobian,
// which only steers the step, the FP32 sweep over the high parts.  The LM
// solve (Cholesky of the damped, unit-diagonal normal matrix), the SSR and
// the damping update run in FP64 on one CTA: m <= 16 parameters.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cuda_runtime.h>

#include "pm_df.cuh"
#include "pm_eval.cuh"
#include "pm_internal.h"
#include "pm_model.h"

namespace pm {
namespace {

constexpr int MP = kMaxParamsFit;
constexpr int NA = MP * (MP + 1) / 2;
constexpr double EPS_DF = 1e-13;   // relative accuracy of a float-float residual (conservative)
constexpr double kStepTiny = 1e-9; // a negligible step below the SSR's noise floor (scaled coordinates)
constexpr int kMaxBelow = 4;       // at most this many unverifiable steps in a row
constexpr int kMaxRetries = 16;    // rejected trials per iteration
constexpr int kRunning = 1;

// State of one LM loop (device memory, PM_LM_STATE_BYTES bytes owned by the
// caller).  Scaled coordinates q = p / s, s = |p0| (1 where p0 = 0).
struct LMState {
    double q[MP], s[MP], dq[MP], dmax[MP], b[MP];
    double A[NA];               // J^T J in the scaled coordinates (upper triangle, row-major)
    double lambda, ssr, pred, noise, ftol, xtol;
    int m, max_iter, iterations, retries, nbelow, status, accepted, have_sys;
};
static_assert(sizeof(LMState) <= PM_LM_STATE_BYTES, "LM state larger than PM_LM_STATE_BYTES");

__device__ __forceinline__ df split_d(double x) {
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}

// The model program, its constants and the parameters in shared memory.
struct Prog {
    Ins code[kMaxIns];
    df cst[kMaxIns];
    df p[MP];
};

__device__ void load_prog(Prog &P, const Ins *code, int n, const double *p, int m) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const Ins in = code[k];
        P.code[k] = in;
        P.cst[k] = split_d(in.c);
    }
    if ((int)threadIdx.x < m) P.p[threadIdx.x] = split_d(p[threadIdx.x]);
    __syncthreads();
}

// r_k = 1 - g(p; X_k) / t_k in float-float, stored as FP64
__global__ void __launch_bounds__(128) k_resid(const Ins *__restrict__ code, int n, int m, int nf,
                                               const double *__restrict__ X, const double *__restrict__ t, size_t l,
                                               const double *__restrict__ p, double *__restrict__ r) {
    __shared__ Prog P;
    load_prog(P, code, n, p, m);
    df v[kMaxIns];
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < l; row += (size_t)gridDim.x * blockDim.x) {
        const df g = forward_df(P.code, P.cst, n, X + row * nf, P.p, v);
        const df rr = df_sub(df{1.0f, 0.0f}, df_div(g, split_d(t[row])));
        r[row] = (double)rr.hi + (double)rr.lo;
    }
}

// pbar_i += sum_k rbar_k dr_k/dp_i = -sum_k g_i(k) rbar_k / t_k, float-float
// products and compensated sums per thread, per-warp float-float sums in a
// fixed order, one FP64 atomic per parameter and CTA
__global__ void __launch_bounds__(256) k_vjp(const Ins *__restrict__ code, int n, int m, int nf,
                                             const double *__restrict__ X, const double *__restrict__ t, size_t l,
                                             const double *__restrict__ p, const double *__restrict__ rbar,
                                             double *__restrict__ pbar) {
    __shared__ Prog P;
    __shared__ df red[MP][8];
    load_prog(P, code, n, p, m);
    df v[kMaxIns], adj[kMaxIns], g[MP];
    CAcc acc[MP];
    for (int i = 0; i < MP; i++) acc[i].init();
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < l; row += (size_t)gridDim.x * blockDim.x) {
        forward_df(P.code, P.cst, n, X + row * nf, P.p, v);
        reverse_dd(P.code, n, v, adj, g, m);
        const df w = df_div(split_d(rbar[row]), split_d(t[row]));
        for (int i = 0; i < m; i++) {
            const df x = df_mul(g[i], w);
            acc[i].add(-x.hi, -x.lo);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = 0; i < m; i++) {
        const df x = warp_sum(acc[i].sum());
        if (lane == 0) red[i][warp] = x;
    }
    __syncthreads();
    if ((int)threadIdx.x < m) {
        df x = red[threadIdx.x][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) x = df_add(x, red[threadIdx.x][w]);
        atomicAdd(&pbar[threadIdx.x], (double)x.hi + (double)x.lo);
    }
}

// J[k, i] = dr_k/dp_i = -g_i(k) / t_k, FP32 (reverse sweep over the high
// parts of the float-float forward values)
__global__ void __launch_bounds__(256) k_jacobian(const Ins *__restrict__ code, int n, int m, int nf,
                                                  const double *__restrict__ X, const double *__restrict__ t, size_t l,
                                                  const double *__restrict__ p, float *__restrict__ J) {
    __shared__ Prog P;
    load_prog(P, code, n, p, m);
    df v[kMaxIns];
    float adj[kMaxIns], g[MP];
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < l; row += (size_t)gridDim.x * blockDim.x) {
        forward_df(P.code, P.cst, n, X + row * nf, P.p, v);
        reverse_df(P.code, n, v, adj, g, m);
        const float tk = (float)t[row];
        for (int i = 0; i < m; i++) J[row * m + i] = __fdiv_rn(-g[i], tk);
    }
}

// Sum over the CTA (blockDim.x a multiple of 32, at most 1024) in a fixed
// order; every thread receives the result.
__device__ double block_sum(double x, double *sh) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[warp] = x;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += sh[w];
    return s;
}

__device__ __forceinline__ int tri(int m, int i, int j) { return i * m - i * (i - 1) / 2 + (j - i); }

// One CTA.  At a new point (have_sys == 0): the SSR from r, A = S J^T J S
// (exact FP32 products, compensated sums) and b = S (J^T r) from the
// caller's vector-Jacobian product, dmax updated.  Then thread 0 solves
// (Ahat + diag(lam)) y = -bhat with Ahat the unit-diagonal scaling of A on
// the parameters whose diagonal is not zero, lam_i = lambda max(dmax_i /
// A_ii, 1) (the damping lambda dmax_i on A's diagonal), by Cholesky in FP64;
// a non-positive pivot multiplies lambda by 10 and tries again (at most
// kMaxRetries times).  dq = y / sqrt(diag A), pred = -y.bhat + sum lam_i
// y_i^2 (the predicted SSR decrease), p_try = (q + dq) s.
__global__ void __launch_bounds__(256) k_lm_step(LMState *__restrict__ S, const double *__restrict__ r,
                                                 const double *__restrict__ b, const float *__restrict__ J, size_t l,
                                                 double *__restrict__ p_try) {
    __shared__ double sh[32];
    __shared__ int run, have;
    const int m = S->m, tid = threadIdx.x;
    if (tid == 0) {
        run = S->status == kRunning;
        have = S->have_sys;
    }
    __syncthreads();
    if (!run) {
        if (tid < m) p_try[tid] = S->q[tid] * S->s[tid];
        return;
    }
    if (!have) {
        double x = 0.0;
        for (size_t k = tid; k < l; k += blockDim.x) x = fma(r[k], r[k], x);
        const double ssr = block_sum(x, sh);
        const int na = m * (m + 1) / 2;
        for (int e = tid; e < na; e += blockDim.x) {
            int i = 0, rem = e;
            while (rem >= m - i) { rem -= m - i; i++; }
            const int j = i + rem;
            CAcc a;
            a.init();
            for (size_t k = 0; k < l; k++) a.add_prod(J[k * m + i], J[k * m + j]);
            S->A[e] = a.value() * S->s[i] * S->s[j];
        }
        if (tid < m) S->b[tid] = b[tid] * S->s[tid];
        __syncthreads();
        if (tid == 0) {
            S->ssr = ssr;
            S->noise = 4.0 * EPS_DF * sqrt((double)l * ssr) + (double)l * EPS_DF * EPS_DF;
            for (int i = 0; i < m; i++) S->dmax[i] = fmax(S->dmax[i], S->A[tri(m, i, i)]);
            S->have_sys = 1;
        }
        __syncthreads();
    }
    if (tid == 0) {
        double M[MP][MP], rhs[MP], dinv[MP], lam[MP], y[MP];
        int idx[MP], n = 0;
        for (int i = 0; i < m; i++)
            if (S->A[tri(m, i, i)] > 0.0) idx[n++] = i;
        bool ok = false;
        for (int tr = 0; tr < kMaxRetries && !ok; tr++) {
            const double lambda = S->lambda;
            for (int a = 0; a < n; a++) {
                const int i = idx[a];
                const double aii = S->A[tri(m, i, i)];
                dinv[a] = 1.0 / sqrt(aii);
                lam[a] = lambda * fmax(S->dmax[i] / aii, 1.0);
            }
            for (int a = 0; a < n; a++) {
                for (int c = 0; c <= a; c++) {
                    const int i = idx[a], j = idx[c];
                    M[a][c] = S->A[i <= j ? tri(m, i, j) : tri(m, j, i)] * dinv[a] * dinv[c];
                }
                M[a][a] += lam[a];
                rhs[a] = -S->b[idx[a]] * dinv[a];
            }
            ok = true;
            for (int k = 0; k < n && ok; k++) {
                double d = M[k][k];
                for (int c = 0; c < k; c++) d -= M[k][c] * M[k][c];
                if (!(d > 1e-10)) { ok = false; break; }
                M[k][k] = sqrt(d);
                for (int a = k + 1; a < n; a++) {
                    double x = M[a][k];
                    for (int c = 0; c < k; c++) x -= M[a][c] * M[k][c];
                    M[a][k] = x / M[k][k];
                }
            }
            if (!ok) {
                S->lambda = lambda * 10.0;
                continue;
            }
            for (int a = 0; a < n; a++) {
                double x = rhs[a];
                for (int c = 0; c < a; c++) x -= M[a][c] * y[c];
                y[a] = x / M[a][a];
            }
            for (int a = n - 1; a >= 0; a--) {
                double x = y[a];
                for (int c = a + 1; c < n; c++) x -= M[c][a] * y[c];
                y[a] = x / M[a][a];
            }
            double pred = 0.0;
            for (int i = 0; i < m; i++) S->dq[i] = 0.0;
            for (int a = 0; a < n; a++) {
                S->dq[idx[a]] = y[a] * dinv[a];
                pred += lam[a] * y[a] * y[a] - y[a] * (S->b[idx[a]] * dinv[a]);
            }
            S->pred = pred;
        }
        if (!ok) {
            // no positive definite damped system: keep the current point
            for (int i = 0; i < m; i++) S->dq[i] = 0.0;
            S->pred = 0.0;
            S->status = PM_OK;
        }
    }
    __syncthreads();
    if (tid < m) p_try[tid] = (S->q[tid] + S->dq[tid]) * S->s[tid];
}

// One CTA.  SSR at the trial point; accept when it is finite and not above
// the current SSR, or when the predicted decrease is below the SSR's noise
// floor (the step then comes from the gradient alone).  Accepted: q += dq, p
// written, lambda / 10 (not below 1e-12), the system to be re-assembled at
// the new point; the loop ends when the step is negligible (xtol), when
// steps below the noise floor have become negligible (kStepTiny) or
// kMaxBelow of them came in a row, or when a measurable decrease fell below
// ftol relative.  Rejected: lambda x 10; after kMaxRetries rejections in one
// iteration no decrease is possible above the noise floor and the loop ends
// at the current point.  flags = {status, accepted}.
__global__ void __launch_bounds__(256) k_lm_update(LMState *__restrict__ S, const double *__restrict__ r_try, size_t l,
                                                   double *__restrict__ p, int *__restrict__ flags) {
    __shared__ double sh[32];
    double x = 0.0;
    for (size_t k = threadIdx.x; k < l; k += blockDim.x) x = fma(r_try[k], r_try[k], x);
    const double sn = block_sum(x, sh);
    if (threadIdx.x != 0) return;
    const int m = S->m;
    int accepted = 0;
    if (S->status == kRunning) {
        if (isfinite(sn) && (sn <= S->ssr || S->pred <= S->noise)) {
            accepted = 1;
            double dn = 0.0, qn = 0.0, da = 0.0, qa = 0.0;
            for (int i = 0; i < m; i++) {
                S->q[i] += S->dq[i];
                p[i] = S->q[i] * S->s[i];
                dn += S->dq[i] * S->dq[i];
                qn += S->q[i] * S->q[i];
                da = fmax(da, fabs(S->dq[i]));
                qa = fmax(qa, fabs(S->q[i]));
            }
            const bool below = S->pred <= S->noise;
            S->nbelow = below ? S->nbelow + 1 : 0;
            const bool stop = sqrt(dn) <= S->xtol * (sqrt(qn) + S->xtol) ||
                              (below && (da <= kStepTiny * fmax(qa, 1.0) || S->nbelow >= kMaxBelow)) ||
                              (!below && (S->ssr - sn) <= S->ftol * S->ssr);
            S->ssr = sn;
            S->lambda = fmax(S->lambda * 0.1, 1e-12);
            S->iterations++;
            S->retries = 0;
            S->have_sys = 0;
            if (stop) S->status = PM_OK;
            else if (S->iterations >= S->max_iter) S->status = PM_ENOTCONV;
        } else {
            S->lambda *= 10.0;
            if (++S->retries >= kMaxRetries) S->status = PM_OK;
        }
    }
    S->accepted = accepted;
    flags[0] = S->status;
    flags[1] = accepted;
}

pm_status ensure_device_code(const pm_model *m) {
    int dev = 0;
    PM_CUDA_TRY(cudaGetDevice(&dev));
    pm_model *mm = const_cast<pm_model *>(m);
    if (mm->d_code && mm->d_device == dev) return PM_OK;
    if (mm->d_code) {
        cudaFree(mm->d_code);
        mm->d_code = nullptr;
    }
    PM_ALLOC_TRY(cudaMalloc(&mm->d_code, m->code.size() * sizeof(Ins)));
    PM_CUDA_TRY(cudaMemcpy(mm->d_code, m->code.data(), m->code.size() * sizeof(Ins), cudaMemcpyHostToDevice));
    mm->d_device = dev;
    return PM_OK;
}

unsigned grid_for(size_t l, unsigned per, unsigned cap) { return (unsigned)std::min<size_t>((l + per - 1) / per, cap); }

}  // namespace
}  // namespace pm

extern "C" {

pm_status pm_residual(const pm_model *m, const double *X, const double *t, size_t l, const double *p, double *r,
                      void *stream) {
    using namespace pm;
    if (!m || !t || !p || !r || (!X && !m->features.empty())) return fail(PM_EINVAL, "pm_residual: NULL argument");
    if (l == 0) return PM_OK;
    pm_status s = ensure_device_code(m);
    if (s) return s;
    k_resid<<<grid_for(l, 128, 1216), 128, 0, (cudaStream_t)stream>>>(m->d_code, (int)m->code.size(),
                                                                      (int)m->params.size(), (int)m->features.size(),
                                                                      X, t, l, p, r);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_residual_vjp(const pm_model *m, const double *X, const double *t, size_t l, const double *p,
                          const double *rbar, double *pbar, void *stream) {
    using namespace pm;
    if (!m || !t || !p || !rbar || !pbar || (!X && !m->features.empty()))
        return fail(PM_EINVAL, "pm_residual_vjp: NULL argument");
    pm_status s = ensure_device_code(m);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    PM_CUDA_TRY(cudaMemsetAsync(pbar, 0, m->params.size() * 8, st));
    if (l == 0) return PM_OK;
    k_vjp<<<grid_for(l, 256, 304), 256, 0, st>>>(m->d_code, (int)m->code.size(), (int)m->params.size(),
                                                  (int)m->features.size(), X, t, l, p, rbar, pbar);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_jacobian(const pm_model *m, const double *X, const double *t, size_t l, const double *p, float *J,
                      void *stream) {
    using namespace pm;
    if (!m || !t || !p || !J || (!X && !m->features.empty())) return fail(PM_EINVAL, "pm_jacobian: NULL argument");
    if (l == 0) return PM_OK;
    pm_status s = ensure_device_code(m);
    if (s) return s;
    k_jacobian<<<grid_for(l, 256, 1216), 256, 0, (cudaStream_t)stream>>>(m->d_code, (int)m->code.size(),
                                                                        (int)m->params.size(),
                                                                        (int)m->features.size(), X, t, l, p, J);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_lm_init(const pm_model *m, const double *p0, const pm_fit_opts *opts, void *state, double *p,
                     void *stream) {
    using namespace pm;
    if (!m || !p0 || !state || !p) return fail(PM_EINVAL, "pm_lm_init: NULL argument");
    const int np = (int)m->params.size();
    LMState h;
    memset(&h, 0, sizeof(h));
    h.m = np;
    h.max_iter = opts ? opts->max_iter : 200;
    h.ftol = opts ? opts->ftol : 1e-15;
    h.xtol = opts ? opts->xtol : 1e-12;
    if (h.max_iter < 0 || !(h.ftol >= 0.0) || !(h.xtol >= 0.0))
        return fail(PM_EINVAL, "pm_lm_init: max_iter, ftol and xtol must be >= 0");
    for (int i = 0; i < np; i++) {
        if (!std::isfinite(p0[i])) return fail(PM_EINVAL, "pm_lm_init: start point %d is not finite", i);
        h.s[i] = p0[i] != 0.0 ? fabs(p0[i]) : 1.0;
        h.q[i] = p0[i] / h.s[i];
    }
    h.lambda = 1e-3;
    h.status = h.max_iter > 0 ? kRunning : PM_ENOTCONV;
    pm_status s = ensure_device_code(m);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // pageable sources: each copy returns once its source has been staged
    PM_CUDA_TRY(cudaMemcpyAsync(state, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    PM_CUDA_TRY(cudaMemcpyAsync(p, p0, np * sizeof(double), cudaMemcpyHostToDevice, st));
    return PM_OK;
}

pm_status pm_lm_step(void *state, const double *r, const double *b, const float *J, size_t l, double *p_try,
                     void *stream) {
    using namespace pm;
    if (!state || !r || !b || !J || !p_try || l == 0) return fail(PM_EINVAL, "pm_lm_step: bad argument");
    k_lm_step<<<1, 256, 0, (cudaStream_t)stream>>>((LMState *)state, r, b, J, l, p_try);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_lm_update(void *state, const double *r_try, size_t l, double *p, int32_t *flags, void *stream) {
    using namespace pm;
    if (!state || !r_try || !p || !flags || l == 0) return fail(PM_EINVAL, "pm_lm_update: bad argument");
    k_lm_update<<<1, 256, 0, (cudaStream_t)stream>>>((LMState *)state, r_try, l, p, flags);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_lm_report(const void *state, pm_fit_report *report, void *stream) {
    using namespace pm;
    if (!state || !report) return fail(PM_EINVAL, "pm_lm_report: NULL argument");
    LMState h;
    cudaStream_t st = (cudaStream_t)stream;
    PM_CUDA_TRY(cudaMemcpyAsync(&h, state, sizeof(h), cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    report->status = h.status == kRunning ? PM_ENOTCONV : h.status;
    report->iterations = h.iterations;
    report->rank = h.m;
    report->linear = 0;
    report->residual = sqrt(h.ssr);
    report->lambda = h.lambda;
    report->cond = NAN;
    return PM_OK;
}

}  // extern "C"
