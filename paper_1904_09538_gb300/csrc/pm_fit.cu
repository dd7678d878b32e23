// Calibration and prediction (Section "Computing Model Parameters",
// Section "Predicting Cost", Eq. overlap_differentiable / Eq. tanh).
//
// Residual r_k = 1 - g(p; f_k)/t_k (relative error, the paper's
// scale_features_by_output); Jacobian by reverse-mode differentiation of the
// model's SSA program (the paper differentiates the model symbolically).
//
// Precision: everything per row runs on the FP32 pipes.  The Jacobian is
// plain FP32 (it only steers the iteration); the residual, which fixes the
// solution, is evaluated in float-float arithmetic (pairs of FP32 with
// error-free TwoSum / TwoProd transformations) from float-float copies of the
// features and outputs; J^T J, J^T r and the SSR are accumulated with exact
// FP32 products (TwoProd) and compensated FP32 sums.  FP64 is used only for
// the m x m normal-equation solve (Cholesky, or a Jacobi eigen-decomposition
// for rank-deficient linear designs) and the Levenberg-Marquardt damping
// update.
//
// Batched path: one CTA per model in one persistent kernel launch; a plan
// captures [H2D copies -> FP64->FP32 conversion -> fit kernel -> D2H copies]
// in a CUDA graph.  Every loop is bounded (max_iter, 16 damping retries, 12
// Jacobi sweeps); no kernel waits on another.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cuda_runtime.h>
#include <mutex>
#include <new>
#include <vector>

#include "pm_df.cuh"
#include "pm_eval.cuh"
#include "pm_internal.h"
#include "pm_model.h"

pm_model::~pm_model() {
    if (d_code) cudaFree(d_code);
}

namespace pm {
namespace {

constexpr int MP = kMaxParamsFit;               // max parameters
constexpr int NENT = MP * (MP + 1) / 2 + MP + 1; // A (upper), b, ssr
constexpr double EPS_DF = 1e-13;  // relative accuracy of a float-float residual (conservative)
// End of the iteration below the SSR's noise floor: a step of at most
// kStepTiny (max |dq_i| over max(max |q_i|, 1), scaled coordinates), or
// kMaxBelow such steps in a row
constexpr double kStepTiny = 1e-9;
constexpr int kMaxBelow = 4;

struct FitJob {
    const Ins *code;
    const Ins *start_code;
    int n_code, n_start;
    int m, nf, l;
    int linear, use_p0;
    unsigned start_mask;
    const float2 *X;  // l x nf, (hi, lo) float-float
    const float2 *t;  // l, (hi, lo)
    double *p;        // m, in/out
    double *rep;      // 8 per job
};

struct FitCfg {
    int max_iter;
    double ftol, xtol;
};

// ---------------------------------------------------------------- per-CTA state
template <int T>
struct Smem {
    Ins code[kMaxIns];
    df cst[kMaxIns];   // constants of `code` in float-float
    float J[T * (MP + 1)];
    float Jl[T * (MP + 1)];   // low parts of J (direct linear solves only)
    float r[T], rl[T];
    double acc[NENT];
    df accf[NENT];    // the same entries in float-float (the fast solve reads these)
    double q[MP], s[MP], dq[MP], qt[MP];
    double dmax[MP];   // largest diag(J^T J) seen by the LM so far (its damping scale)
    df pd[MP];
    float sf[MP];      // S.s in FP32 (the Jacobian's column scales), set with the parameters
    df sdf[MP];        // S.s in float-float
    double M[MP][MP + 1], V[MP][MP + 1], rhs[MP], y[MP];
    int idx[MP];
    df Mf[MP][MP + 1], rhsf[MP], dinvf[MP];
    df redf[T / 32];
    float redc[T / 32][MP + 1];   // per-warp column sums of the start design (and of t)
    double sbig;                  // start point: max |p| of its linear fit
    unsigned zmask;               // start point: parameters whose column is zero at the origin
    df part[T];       // per row-group partial sums of the assembled entries
    double ssr, pred, lambda, med[2], noise, cond;
    int stop, below, nbelow;
    int nact, ok, rankdef, rank;
};

template <int T>
__device__ void load_code(Smem<T> &S, const Ins *code, int n) {
    for (int k = threadIdx.x; k < n; k += T) {
        const Ins in = code[k];
        S.code[k] = in;
        const float h = (float)in.c;
        S.cst[k] = df{h, (float)(in.c - (double)h)};
    }
    __syncthreads();
}

// p = s * q -> float-float copy for evaluation
template <int T>
__device__ void set_params(Smem<T> &S, const double *q, int m) {
    if (threadIdx.x < m) {
        const double p = S.s[threadIdx.x] * q[threadIdx.x];
        S.sf[threadIdx.x] = (float)S.s[threadIdx.x];
        const float sh = (float)S.s[threadIdx.x];
        S.sdf[threadIdx.x] = df{sh, (float)(S.s[threadIdx.x] - (double)sh)};
        const float h = (float)p;
        S.pd[threadIdx.x] = df{h, (float)(p - (double)h)};
    }
    __syncthreads();
}

// r_k = 1 - g_k / t_k in float-float
__device__ __forceinline__ df resid_df(df g, float2 t) { return df_sub(df{1.0f, 0.0f}, df_div(g, df{t.x, t.y})); }

// Entry e of the assembled system over rows k = k0, k0 + step, ... < rows of
// the staged block: A_ij (e < nA, row-major upper triangle), b_i, or the SSR.
// EXACT: J carries low parts (S.Jl) and the products include the cross
// terms hi lo + lo hi.
template <int T, bool EXACT>
__device__ __forceinline__ void add_entry(const Smem<T> &S, CAcc &a, int e, int m, int nA, int k0, int step,
                                          int rows) {
    if (e < nA) {
        int i = 0, rem = e;
        while (rem >= m - i) { rem -= m - i; i++; }
        const int j = i + rem;
        for (int k = k0; k < rows; k += step) {
            if (EXACT) {
                const float hi = S.J[k * (MP + 1) + i], hj = S.J[k * (MP + 1) + j];
                float p, er;
                two_prod(hi, hj, p, er);
                er = __fmaf_rn(hi, S.Jl[k * (MP + 1) + j], er);
                a.add(p, __fmaf_rn(S.Jl[k * (MP + 1) + i], hj, er));
            } else {
                a.add_prod(S.J[k * (MP + 1) + i], S.J[k * (MP + 1) + j]);
            }
        }
    } else if (e < nA + m) {
        const int i = e - nA;
        for (int k = k0; k < rows; k += step) {
            const float ji = S.J[k * (MP + 1) + i];
            float p, er;
            two_prod(ji, S.r[k], p, er);
            er = __fmaf_rn(ji, S.rl[k], er);
            if (EXACT) er = __fmaf_rn(S.Jl[k * (MP + 1) + i], S.r[k], er);
            a.add(p, er);
        }
    } else {
        for (int k = k0; k < rows; k += step) {
            float p, er;
            two_prod(S.r[k], S.r[k], p, er);
            a.add(p, __fmaf_rn(2.0f * S.r[k], S.rl[k], er));
        }
    }
}

// Assemble over all rows of the job: A = J^T J (upper, if want_A), b = J^T r,
// ssr = r^T r, with J_ki = -(dg_k/dp_i) s_i / t_k (scaled coordinates q).
// Parameters outside `mask` get a zero column.  With nE entries and
// 2 nE <= T, each entry is summed by G = T / nE threads over interleaved
// rows (compensated FP32 sums, one per thread across all row blocks), and
// the G partial sums are added in FP64 in a fixed order; otherwise each
// thread sums whole entries.
template <int T, bool EXACT = false>
__device__ void assemble(Smem<T> &S, const FitJob &jb, int n, unsigned mask, bool want_A) {
    const int m = jb.m, tid = threadIdx.x;
    const int nA = m * (m + 1) / 2, nE = nA + m + 1;
    const int G = 2 * nE <= T ? T / nE : 1;
    const int ge = tid % nE, gg = tid / nE;   // grouped mode: entry, row group
    CAcc acc[3];
    for (int u = 0; u < 3; u++) acc[u].init();
    df v[kMaxIns];
    float adj[kMaxIns], g[MP];
    for (int base = 0; base < jb.l; base += T) {
        const int row = base + tid;
        df rr = df{0.0f, 0.0f};
        if (row < jb.l) {
            const float2 *frow = jb.X + (size_t)row * jb.nf;
            const float2 tk = jb.t[row];
            const df gk = forward_df(S.code, S.cst, n, frow, S.pd, v);
            rr = resid_df(gk, tk);
            if (EXACT) {
                df adjd[kMaxIns], gd[MP];
                reverse_dd(S.code, n, v, adjd, gd, m);
                const df tdf = df{tk.x, tk.y};
                for (int i = 0; i < m; i++) {
                    const df jv = ((mask >> i) & 1u) ? df_neg(df_div(df_mul(gd[i], S.sdf[i]), tdf)) : df{0.0f, 0.0f};
                    S.J[tid * (MP + 1) + i] = jv.hi;
                    S.Jl[tid * (MP + 1) + i] = jv.lo;
                }
            } else {
                reverse_df(S.code, n, v, adj, g, m);
                const float rt = __frcp_rn(tk.x);
                for (int i = 0; i < m; i++)
                    S.J[tid * (MP + 1) + i] = ((mask >> i) & 1u) ? -g[i] * S.sf[i] * rt : 0.0f;
            }
        } else {
            for (int i = 0; i < m; i++) {
                S.J[tid * (MP + 1) + i] = 0.0f;
                if (EXACT) S.Jl[tid * (MP + 1) + i] = 0.0f;
            }
        }
        S.r[tid] = rr.hi;
        S.rl[tid] = rr.lo;
        __syncthreads();
        const int rows = min(T, jb.l - base);
        if (G > 1) {
            if (gg < G && (want_A || ge >= nA)) add_entry<T, EXACT>(S, acc[0], ge, m, nA, gg, G, rows);
        } else {
            for (int u = 0; u < 3; u++) {
                const int e = tid + u * T;
                if (e >= nE) break;
                if (e < nA && !want_A) continue;
                add_entry<T, EXACT>(S, acc[u], e, m, nA, 0, 1, rows);
            }
        }
        __syncthreads();
    }
    if (G > 1) {
        if (gg < G) S.part[gg * nE + ge] = acc[0].sum();
        __syncthreads();
        if (tid < nE && (want_A || tid >= nA)) {
            df x = S.part[tid];
            for (int g2 = 1; g2 < G; g2++) x = df_add(x, S.part[g2 * nE + tid]);
            S.accf[tid] = x;
            S.acc[tid] = (double)x.hi + (double)x.lo;
        }
    } else {
        for (int u = 0; u < 3; u++) {
            const int e = tid + u * T;
            if (e < nE && (want_A || e >= nA)) {
                S.accf[e] = acc[u].sum();
                S.acc[e] = (double)S.accf[e].hi + (double)S.accf[e].lo;
            }
        }
    }
    __syncthreads();
    if (tid == 0) S.ssr = S.acc[nE - 1];
    __syncthreads();
}

// SSR only, at parameters S.pd (float-float residuals, exact squares).
template <int T>
__device__ double ssr_pass(Smem<T> &S, const FitJob &jb, int n) {
    CAcc a;
    a.init();
    df v[kMaxIns];
    for (int row = threadIdx.x; row < jb.l; row += T) {
        const df gk = forward_df(S.code, S.cst, n, jb.X + (size_t)row * jb.nf, S.pd, v);
        const df rr = resid_df(gk, jb.t[row]);
        float p, er;
        two_prod(rr.hi, rr.hi, p, er);
        a.add(p, __fmaf_rn(2.0f * rr.hi, rr.lo, er));
    }
    df x = warp_sum(a.sum());
    if ((threadIdx.x & 31) == 0) S.redf[threadIdx.x >> 5] = x;
    __syncthreads();
    df tot = S.redf[0];
    for (int w = 1; w < T / 32; w++) tot = df_add(tot, S.redf[w]);
    __syncthreads();
    return (double)tot.hi + (double)tot.lo;
}

__device__ __forceinline__ double A_at(const double *acc, int m, int i, int j) {
    if (i > j) { const int t = i; i = j; j = t; }
    return acc[i * m - i * (i - 1) / 2 + (j - i)];
}

__device__ __forceinline__ df A_atf(const df *acc, int m, int i, int j) {
    if (i > j) { const int t = i; i = j; j = t; }
    return acc[i * m - i * (i - 1) / 2 + (j - i)];
}

// Warp 0: solve (A + lambda E) dq = -b on the active set, E = diag(dmax)
// (the largest diag A seen by the LM, Moré's scaling; unused at lambda = 0),
// as (Ahat + lambda E / diag A) y = -bhat with Ahat the unit-diagonal scaling
// of A and dq = y / sqrt(diag A).  Float-float arithmetic on the FP32 pipes
// (GB300's FP64 pipe retires about two lanes per clock per SM; the LM step
// is refined by the iteration itself).  S.ok = 0 when a pivot is not
// positive (relative 1e-10).  Also S.pred = predicted SSR decrease
// -(2 dq.b + dq^T A dq), evaluated as -dq.b + lambda dq^T E dq.
template <int T>
__device__ void solve_chol(Smem<T> &S, int m, double lambda) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, n = S.nact;
        const df *acc = S.accf;
        const int nA = m * (m + 1) / 2;
        df dinv = df{0.0f, 0.0f};
        if (lane < n) dinv = df_div(df{1.0f, 0.0f}, df_sqrt(A_atf(acc, m, S.idx[lane], S.idx[lane])));
        // damping lambda * dmax_i on the diagonal of A (Moré's scaling: the
        // largest diagonal entry met so far), lambda * dmax_i / A_ii once the
        // rows are scaled to a unit diagonal
        double lam_d = 0.0;
        if (lane < n && lambda != 0.0) {
            const int gi = S.idx[lane];
            lam_d = lambda * fmax(S.dmax[gi] / A_at(S.acc, m, gi, gi), 1.0);
        }
        const float lh = (float)lam_d;
        const df lam = df{lh, (float)(lam_d - (double)lh)};
        if (lane < MP) S.dinvf[lane] = dinv;
        if (lane == 0) S.ok = 1;
        __syncwarp();
        if (lane < n) {
            const int gi = S.idx[lane];
            for (int c = 0; c < n; c++) {
                df x = df_mul(df_mul(A_atf(acc, m, gi, S.idx[c]), dinv), S.dinvf[c]);
                if (c == lane) x = df_add(x, lam);
                S.Mf[lane][c] = x;
            }
            S.rhsf[lane] = df_neg(df_mul(acc[nA + gi], dinv));
        }
        __syncwarp();
        // Cholesky, lower factor in place
        for (int k = 0; k < n; k++) {
            const df d = S.Mf[k][k];
            if (lane == 0 && !(d.hi > 1e-10f)) S.ok = 0;
            const df piv = df_sqrt(d.hi > 1e-30f ? d : df{1e-30f, 0.0f});
            if (lane > k && lane < n) S.Mf[lane][k] = df_div(S.Mf[lane][k], piv);
            __syncwarp();
            if (lane == k) S.Mf[k][k] = piv;
            if (lane > k && lane < n) {
                const df lk = S.Mf[lane][k];
                for (int j = k + 1; j <= lane; j++) S.Mf[lane][j] = df_sub(S.Mf[lane][j], df_mul(lk, S.Mf[j][k]));
            }
            __syncwarp();
        }
        // forward: L z = rhs
        for (int k = 0; k < n; k++) {
            if (lane == k) S.rhsf[k] = df_div(S.rhsf[k], S.Mf[k][k]);
            __syncwarp();
            if (lane > k && lane < n) S.rhsf[lane] = df_sub(S.rhsf[lane], df_mul(S.Mf[lane][k], S.rhsf[k]));
            __syncwarp();
        }
        // backward: L^T y = z
        for (int k = n - 1; k >= 0; k--) {
            if (lane == k) S.rhsf[k] = df_div(S.rhsf[k], S.Mf[k][k]);
            __syncwarp();
            if (lane < k) S.rhsf[lane] = df_sub(S.rhsf[lane], df_mul(S.Mf[k][lane], S.rhsf[k]));
            __syncwarp();
        }
        // dq in every parameter slot (zero outside the active set)
        df dql = df{0.0f, 0.0f};
        int gl = -1;
        if (lane < n) {
            gl = S.idx[lane];
            dql = df_mul(S.rhsf[lane], dinv);
        }
        __syncwarp();
        if (lane < m) S.dq[lane] = 0.0;
        __syncwarp();
        if (gl >= 0) S.dq[gl] = (double)dql.hi + (double)dql.lo;
        // predicted decrease -(2 dq.b + dq^T A dq).  With (A + lambda E) dq = -b
        // (E = diag dmax) it equals -dq.b + lambda dq^T E dq, in the scaled
        // coordinates -y.bhat + sum_i lam_i y_i^2 (lam_i the damping on row i
        // above): non-negative terms, free of the cancellation the first form
        // suffers near convergence.
        df t = df{0.0f, 0.0f};
        if (lane < n) {
            const df y = S.rhsf[lane];
            const df bh = df_mul(acc[nA + gl], dinv);
            t = df_sub(df_mul(lam, df_mul(y, y)), df_mul(y, bh));
        }
        t = warp_sum(t);
        if (lane == 0) S.pred = (double)t.hi + (double)t.lo;
    }
    __syncthreads();
}

// Warp 0: cyclic Jacobi eigen-decomposition of Ahat (unit diagonal) on the
// active set -> S.V (columns = eigenvectors), S.y (eigenvalues), S.rank.
template <int T>
__device__ void eigen(Smem<T> &S, int m) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, n = S.nact;
        if (lane < n) {
            const int gi = S.idx[lane];
            const double di = sqrt(A_at(S.acc, m, gi, gi));
            for (int c = 0; c < n; c++) {
                const int gj = S.idx[c];
                S.M[lane][c] = A_at(S.acc, m, gi, gj) / (di * sqrt(A_at(S.acc, m, gj, gj)));
                S.V[lane][c] = lane == c ? 1.0 : 0.0;
            }
        }
        __syncwarp();
        for (int sweep = 0; sweep < 12; sweep++) {
            double off = 0.0;
            for (int i = 0; i < n; i++)
                for (int j = i + 1; j < n; j++) off += S.M[i][j] * S.M[i][j];
            if (off < 1e-30) break;
            for (int p = 0; p < n; p++)
                for (int qq = p + 1; qq < n; qq++) {
                    const double apq = S.M[p][qq];
                    if (fabs(apq) < 1e-300) continue;
                    const double theta = (S.M[qq][qq] - S.M[p][p]) / (2.0 * apq);
                    const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                    __syncwarp();
                    if (lane < n) {
                        const double akp = S.M[lane][p], akq = S.M[lane][qq];
                        S.M[lane][p] = c * akp - s * akq;
                        S.M[lane][qq] = s * akp + c * akq;
                    }
                    __syncwarp();
                    if (lane < n) {
                        const double apk = S.M[p][lane], aqk = S.M[qq][lane];
                        S.M[p][lane] = c * apk - s * aqk;
                        S.M[qq][lane] = s * apk + c * aqk;
                        const double vkp = S.V[lane][p], vkq = S.V[lane][qq];
                        S.V[lane][p] = c * vkp - s * vkq;
                        S.V[lane][qq] = s * vkp + c * vkq;
                    }
                    __syncwarp();
                }
        }
        if (lane == 0) {
            double emax = 0.0;
            for (int i = 0; i < n; i++) emax = fmax(emax, S.M[i][i]);
            int r = 0;
            // singular value threshold 1e-5 relative (FP32 data): eigenvalue 1e-10
            for (int i = 0; i < n; i++) {
                S.y[i] = S.M[i][i] > 1e-10 * emax ? S.M[i][i] : 0.0;
                r += S.y[i] > 0.0;
            }
            S.rank = r;
        }
    }
    __syncthreads();
}

// Warp 0: dq = -D^-1/2 V diag(1/e) V^T D^-1/2 b (truncated pseudo-inverse).
template <int T>
__device__ void solve_pinv(Smem<T> &S, int m) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, n = S.nact, nA = m * (m + 1) / 2;
        if (lane < n) {
            const int gi = S.idx[lane];
            S.rhs[lane] = -S.acc[nA + gi] / sqrt(A_at(S.acc, m, gi, gi));
        }
        __syncwarp();
        double w = 0.0;
        if (lane < n && S.y[lane] > 0.0) {
            for (int k = 0; k < n; k++) w += S.V[k][lane] * S.rhs[k];
            w /= S.y[lane];
        }
        __syncwarp();
        if (lane < n) S.qt[lane] = w;  // temporary: coefficients in the eigenbasis
        __syncwarp();
        if (lane < m) S.dq[lane] = 0.0;
        __syncwarp();
        if (lane < n) {
            double z = 0.0;
            for (int k = 0; k < n; k++) z += S.V[lane][k] * S.qt[k];
            const int gi = S.idx[lane];
            S.dq[gi] = z / sqrt(A_at(S.acc, m, gi, gi));
        }
    }
    __syncthreads();
}

template <int T>
__device__ void set_active(Smem<T> &S, int m, unsigned mask) {
    if (threadIdx.x == 0) {
        int n = 0;
        for (int i = 0; i < m; i++)
            if ((mask >> i) & 1u) {
                if (A_at(S.acc, m, i, i) > 0.0) S.idx[n++] = i;
            }
        S.nact = n;
    }
    __syncthreads();
}

// Condition estimate of the unit-diagonal normal matrix at the current
// assembly (lambda = 0): (max / min Cholesky pivot)^2, or the eigenvalue
// ratio when the factorisation fails (+inf if rank-deficient).  Overwrites
// the last step (S.dq, S.pred).
template <int T>
__device__ void cond_estimate(Smem<T> &S, int m) {
    solve_chol(S, m, 0.0);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, n = S.nact;
        float mx = 0.0f, mn = 3.0e38f;
        if (lane < n) {
            mx = S.Mf[lane][lane].hi;
            mn = mx;
        }
        for (int o = 16; o; o >>= 1) {
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        }
        if (lane == 0) {
            const double r = (double)mx / (double)mn;
            S.cond = n == 0 ? 1.0 : (S.ok ? r * r : -1.0);
        }
    }
    __syncthreads();
    if (S.cond < 0.0) {
        eigen(S, m);
        if (threadIdx.x == 0) {
            double emax = 0.0, emin = INFINITY;
            for (int i = 0; i < S.nact; i++)
                if (S.y[i] > 0.0) {
                    emax = fmax(emax, S.y[i]);
                    emin = fmin(emin, S.y[i]);
                }
            S.cond = S.rank < S.nact ? INFINITY : emax / emin;
        }
        __syncthreads();
    }
}

// Linear least squares on `code` for the parameters in mask; S.s must be set.
// Result (scaled) in S.q; S.rank, S.rankdef set.
template <int T>
__device__ void linear_fit(Smem<T> &S, const FitJob &jb, int n, unsigned mask) {
    const int m = jb.m;
    if (threadIdx.x < m) S.q[threadIdx.x] = 0.0;
    __syncthreads();
    set_params(S, S.q, m);
    assemble<T, true>(S, jb, n, mask, true);
    set_active(S, m, mask);
    solve_chol(S, m, 0.0);
    const bool pinv = !S.ok;
    if (pinv) eigen(S, m);
    if (threadIdx.x == 0) {
        S.rankdef = pinv && S.rank < S.nact;
        if (!pinv) S.rank = S.nact;
    }
    __syncthreads();
    for (int it = 0; it < 3; it++) {  // solve, then iterative refinement (b at the new q)
        if (it > 0) {
            set_params(S, S.q, m);
            assemble<T, true>(S, jb, n, mask, false);
            if (pinv) solve_pinv(S, m);
            else {
                // A unchanged (linear): reuse the factorisation by re-solving
                solve_chol(S, m, 0.0);
            }
        } else if (pinv) {
            solve_pinv(S, m);
        }
        if (threadIdx.x < m) S.q[threadIdx.x] += S.dq[threadIdx.x];
        __syncthreads();
    }
    set_params(S, S.q, m);
    const double ssr = ssr_pass(S, jb, n);
    if (threadIdx.x == 0) S.ssr = ssr;
    __syncthreads();
}

// Start-point column sums: S.redc[w][i] (i < m) = sum of |d g_start / d p_i|
// at the point `at` over warp w's rows, S.redc[w][m] = sum of t over them
// (the start code is loaded and S.s = 1).  Used to replace a non-positive
// start coefficient by 1e-3 * sum t / sum |h_i|.
template <int T>
__device__ void start_column_sums(Smem<T> &S, const FitJob &jb, int n, const double *at) {
    const int m = jb.m, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    set_params(S, at, m);
    float cs[MP], ts = 0.0f;
#pragma unroll
    for (int i = 0; i < MP; i++) cs[i] = 0.0f;
    df v[kMaxIns];
    float adj[kMaxIns], g[MP];
    for (int row = tid; row < jb.l; row += T) {
        forward_df(S.code, S.cst, n, jb.X + (size_t)row * jb.nf, S.pd, v);
        reverse_df(S.code, n, v, adj, g, m);
#pragma unroll
        for (int i = 0; i < MP; i++)
            if (i < m) cs[i] += fabsf(g[i]);
        ts += jb.t[row].x;
    }
#pragma unroll
    for (int i = 0; i < MP; i++) {
        if (i >= m) break;
        float x = cs[i];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) S.redc[warp][i] = x;
    }
    for (int o = 16; o; o >>= 1) ts += __shfl_xor_sync(0xffffffffu, ts, o);
    if (lane == 0) S.redc[warp][m] = ts;
    __syncthreads();
}

template <int T>
__global__ void __launch_bounds__(T) k_fit(const FitJob *__restrict__ jobs, FitCfg cfg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<T> &S = *reinterpret_cast<Smem<T> *>(smem_raw);
    const FitJob jb = jobs[blockIdx.x];
    const int m = jb.m, tid = threadIdx.x;
    const unsigned all = m >= 32 ? 0xffffffffu : ((1u << m) - 1u);
    int status = PM_OK, iters = 0;

    if (jb.linear) {
        if (tid < m) S.s[tid] = 1.0;
        __syncthreads();
        load_code(S, jb.code, jb.n_code);
        linear_fit(S, jb, jb.n_code, all);
        if (tid < m) jb.p[tid] = S.q[tid] * S.s[tid];
        set_active(S, m, all);
        cond_estimate(S, m);
        if (tid == 0) {
            jb.rep[0] = S.rankdef ? PM_ERANK : PM_OK;
            jb.rep[1] = 1;
            jb.rep[2] = S.rank;
            jb.rep[3] = 1;
            jb.rep[4] = sqrt(S.ssr);
            jb.rep[5] = 0.0;
            jb.rep[6] = S.cond;
        }
        return;
    }

    // ---- start point
    if (!jb.use_p0) {
        if (tid < m) S.s[tid] = 1.0;
        __syncthreads();
        load_code(S, jb.start_code, jb.n_start);
        linear_fit(S, jb, jb.n_start, jb.start_mask);
        // median of t (rank selection; ties handled by rank ranges)
        const int k1 = (jb.l - 1) / 2, k2 = jb.l / 2;
        for (int i = tid; i < jb.l; i += T) {
            const float x = jb.t[i].x;
            int lt = 0, eq = 0;
            for (int j = 0; j < jb.l; j++) {
                const float y = jb.t[j].x;
                lt += y < x;
                eq += y == x;
            }
            if (lt <= k1 && k1 < lt + eq) S.med[0] = x;
            if (lt <= k2 && k2 < lt + eq) S.med[1] = x;
        }
        __syncthreads();
        // a non-positive start coefficient: its term set to carry about 0.1 %
        // of the outputs, 1e-3 * sum t / sum |h_i| (h_i its column at the
        // origin); a column that vanishes there (a parameter that only
        // multiplies others): the same rule on its column at the point
        // reached so far, 1e-3 * max |p| if that vanishes too
        bool clamp = false;
        for (int i = 0; i < m; i++) clamp |= ((jb.start_mask >> i) & 1u) && !(S.q[i] > 0.0);
        if (clamp) {
            if (tid < m) S.qt[tid] = 0.0;
            __syncthreads();
            start_column_sums(S, jb, jb.n_start, S.qt);
        }
        if (tid == 0) {
            double big = 0.0;
            for (int i = 0; i < m; i++)
                if ((jb.start_mask >> i) & 1u) big = fmax(big, fabs(S.q[i]));
            big = fmax(big, 1e-300);
            double tsum = 0.0;
            if (clamp)
                for (int w = 0; w < T / 32; w++) tsum += (double)S.redc[w][m];
            const double pe = 10.0 / (0.5 * (S.med[0] + S.med[1]));
            unsigned zm = 0u;
            for (int i = 0; i < m; i++) {
                if ((jb.start_mask >> i) & 1u) {
                    if (S.q[i] > 0.0) continue;
                    double cs = 0.0;
                    for (int w = 0; w < T / 32; w++) cs += (double)S.redc[w][i];
                    if (cs > 0.0) {
                        S.q[i] = 1e-3 * tsum / cs;
                    } else {
                        S.q[i] = 0.0;
                        zm |= 1u << i;
                    }
                } else {
                    S.q[i] = pe;
                }
            }
            S.zmask = zm;
            S.sbig = big;
        }
        __syncthreads();
        if (S.zmask) {
            start_column_sums(S, jb, jb.n_start, S.q);
            if (tid == 0) {
                double tsum = 0.0;
                for (int w = 0; w < T / 32; w++) tsum += (double)S.redc[w][m];
                for (int i = 0; i < m; i++) {
                    if (!((S.zmask >> i) & 1u)) continue;
                    double cs = 0.0;
                    for (int w = 0; w < T / 32; w++) cs += (double)S.redc[w][i];
                    S.q[i] = cs > 0.0 ? 1e-3 * tsum / cs : 1e-3 * S.sbig;
                }
            }
            __syncthreads();
        }
    } else {
        if (tid < m) S.q[tid] = jb.p[tid];
        __syncthreads();
    }

    // ---- Levenberg-Marquardt in scaled coordinates q = p / s, s = |p0|
    if (tid < m) {
        const double p0 = S.q[tid];
        S.s[tid] = p0 != 0.0 ? fabs(p0) : 1.0;
        S.q[tid] = p0 / S.s[tid];
    }
    if (tid == 0) {
        S.lambda = 1e-3;
        S.nbelow = 0;
        S.below = 0;
    }
    __syncthreads();
    load_code(S, jb.code, jb.n_code);
    set_params(S, S.q, m);
    assemble(S, jb, jb.n_code, all, true);
    set_active(S, m, all);
    if (tid < m) S.dmax[tid] = A_at(S.acc, m, tid, tid);
    __syncthreads();
    bool converged = false;
    for (int it = 0; it < cfg.max_iter; it++) {
        bool accepted = false;
        const double ssr_old = S.ssr;
        // noise floor of an SSR built from float-float residuals (one thread:
        // FP64 work on every warp costs the whole CTA)
        if (tid == 0) S.noise = 4.0 * EPS_DF * sqrt((double)jb.l * ssr_old) + (double)jb.l * EPS_DF * EPS_DF;
        __syncthreads();
        const double noise = S.noise;
        for (int tr = 0; tr < 16; tr++) {
            solve_chol(S, m, S.lambda);
            if (!S.ok) {
                if (tid == 0) S.lambda *= 10.0;
                __syncthreads();
                continue;
            }
            if (tid < m) S.qt[tid] = S.q[tid] + S.dq[tid];
            __syncthreads();
            // a predicted decrease below the noise floor is accepted whatever
            // the SSR says, so its SSR pass is skipped (the assembly at the
            // new point computes the SSR; a non-finite one is undone there)
            if (S.pred <= noise) {
                accepted = true;
                break;
            }
            set_params(S, S.qt, m);
            const double sn = ssr_pass(S, jb, jb.n_code);
            if (isfinite(sn) && sn <= ssr_old) {
                accepted = true;
                break;
            }
            if (tid == 0) S.lambda *= 10.0;
            __syncthreads();
        }
        if (!accepted) {
            converged = true;  // no decrease possible above the noise floor
            break;
        }
        if (tid == 0) {
            double dn = 0.0, qn = 0.0, da = 0.0, qa = 0.0;
            for (int i = 0; i < m; i++) {
                dn += S.dq[i] * S.dq[i];
                qn += S.qt[i] * S.qt[i];
                da = fmax(da, fabs(S.dq[i]));
                qa = fmax(qa, fabs(S.qt[i]));
            }
            // a step whose predicted gain is below the SSR's noise floor cannot
            // be verified by the SSR, but its direction comes from the gradient,
            // which stays accurate there: such steps continue until they are
            // negligible (kStepTiny in the scaled coordinates) or kMaxBelow of
            // them have been taken in a row
            S.below = S.pred <= noise;
            S.nbelow = S.below ? S.nbelow + 1 : 0;
            S.stop = sqrt(dn) <= cfg.xtol * (sqrt(qn) + cfg.xtol) ||
                     (S.below && (da <= kStepTiny * fmax(qa, 1.0) || S.nbelow >= kMaxBelow));
        }
        __syncthreads();
        if (tid < m) S.q[tid] = S.qt[tid];
        if (tid == 0) S.lambda = fmax(S.lambda * 0.1, 1e-12);
        __syncthreads();
        iters++;
        set_params(S, S.q, m);
        assemble(S, jb, jb.n_code, all, true);
        if (!isfinite(S.ssr)) {
            // an unverified step that left the model's domain: back to the
            // previous point, which ends the fit
            if (tid < m) S.q[tid] -= S.dq[tid];
            __syncthreads();
            set_params(S, S.q, m);
            assemble(S, jb, jb.n_code, all, true);
            if (tid == 0) S.stop = 1;
            iters--;
        }
        set_active(S, m, all);
        if (tid < m) S.dmax[tid] = fmax(S.dmax[tid], A_at(S.acc, m, tid, tid));
        // the relative-decrease test only where the decrease is measurable
        if (tid == 0) S.stop = S.stop || (!S.below && (ssr_old - S.ssr) <= cfg.ftol * ssr_old);
        __syncthreads();
        if (S.stop) {
            converged = true;
            break;
        }
    }
    if (!converged) status = PM_ENOTCONV;
    if (tid < m) jb.p[tid] = S.q[tid] * S.s[tid];
    cond_estimate(S, m);
    if (tid == 0) {
        jb.rep[0] = status;
        jb.rep[1] = iters;
        jb.rep[2] = S.nact;
        jb.rep[3] = 0;
        jb.rep[4] = sqrt(S.ssr);
        jb.rep[5] = S.lambda;
        jb.rep[6] = S.cond;
    }
}

// FP64 -> float-float (hi, lo) split of the uploaded features and outputs
__global__ void k_split(const double *__restrict__ a, float2 *__restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double x = a[i];
        const float h = (float)x;
        b[i] = make_float2(h, (float)(x - (double)h));
    }
}

__global__ void k_predict(const Ins *__restrict__ code, int n, int nf, const double *__restrict__ X, size_t l,
                          const double *__restrict__ p, double *__restrict__ out, int m) {
    __shared__ double pd[MP];
    __shared__ Ins cs[kMaxIns];
    for (int k = threadIdx.x; k < n; k += blockDim.x) cs[k] = code[k];
    if (threadIdx.x < m) pd[threadIdx.x] = p[threadIdx.x];
    __syncthreads();
    double v[kMaxIns];
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < l; row += (size_t)gridDim.x * blockDim.x)
        out[row] = forward<double, double>(cs, n, X + row * nf, pd, v);
}

template <int T>
size_t smem_bytes() { return sizeof(Smem<T>); }

template <int T>
pm_status launch_fit_t(const FitJob *jobs, int njobs, FitCfg cfg, cudaStream_t st) {
    const size_t sb = smem_bytes<T>();
    PM_CUDA_TRY(cudaFuncSetAttribute(k_fit<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    k_fit<T><<<njobs, T, sb, st>>>(jobs, cfg);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status launch_fit(int threads, const FitJob *jobs, int njobs, FitCfg cfg, cudaStream_t st) {
    switch (threads) {
    case 64: return launch_fit_t<64>(jobs, njobs, cfg, st);
    case 256: return launch_fit_t<256>(jobs, njobs, cfg, st);
    case 512: return launch_fit_t<512>(jobs, njobs, cfg, st);
    default: return launch_fit_t<128>(jobs, njobs, cfg, st);
    }
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace
}  // namespace pm

using namespace pm;

struct pm_fit_plan {
    std::vector<const pm_model *> models;
    std::vector<size_t> rows, xoff, poff;
    size_t nx = 0, nt = 0, np = 0;
    int threads = 128;
    FitCfg cfg{};
    int use_p0 = 0;
    // device
    double *dX64 = nullptr, *dt64 = nullptr, *dp = nullptr, *drep = nullptr;
    float2 *dX32 = nullptr, *dt32 = nullptr;
    Ins *dcode = nullptr;
    FitJob *djobs = nullptr;
    // pinned host staging
    double *hX = nullptr, *ht = nullptr, *hp = nullptr, *hrep = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~pm_fit_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        cudaFree(dX64); cudaFree(dt64); cudaFree(dp); cudaFree(drep);
        cudaFree(dX32); cudaFree(dt32); cudaFree(dcode); cudaFree(djobs);
        cudaFreeHost(hX); cudaFreeHost(ht); cudaFreeHost(hp); cudaFreeHost(hrep);
    }
};

namespace pm {
namespace {

pm_status plan_build(pm_fit_plan *P) {
    const size_t K = P->models.size();
    std::vector<Ins> code;
    std::vector<size_t> coff(K), soff(K);
    for (size_t k = 0; k < K; k++) {
        coff[k] = code.size();
        code.insert(code.end(), P->models[k]->code.begin(), P->models[k]->code.end());
        soff[k] = code.size();
        code.insert(code.end(), P->models[k]->start_code.begin(), P->models[k]->start_code.end());
    }
    PM_ALLOC_TRY(cudaMalloc(&P->dX64, std::max<size_t>(P->nx, 1) * 8));
    PM_ALLOC_TRY(cudaMalloc(&P->dX32, std::max<size_t>(P->nx, 1) * 8));
    PM_ALLOC_TRY(cudaMalloc(&P->dt64, P->nt * 8));
    PM_ALLOC_TRY(cudaMalloc(&P->dt32, P->nt * 8));
    PM_ALLOC_TRY(cudaMalloc(&P->dp, P->np * 8));
    PM_ALLOC_TRY(cudaMalloc(&P->drep, K * 8 * 8));
    PM_ALLOC_TRY(cudaMalloc(&P->dcode, code.size() * sizeof(Ins)));
    PM_ALLOC_TRY(cudaMalloc(&P->djobs, K * sizeof(FitJob)));
    PM_ALLOC_TRY(cudaMallocHost(&P->hX, std::max<size_t>(P->nx, 1) * 8));
    PM_ALLOC_TRY(cudaMallocHost(&P->ht, P->nt * 8));
    PM_ALLOC_TRY(cudaMallocHost(&P->hp, P->np * 8));
    PM_ALLOC_TRY(cudaMallocHost(&P->hrep, K * 8 * 8));
    std::vector<FitJob> jobs(K);
    size_t toff = 0;
    for (size_t k = 0; k < K; k++) {
        const pm_model *md = P->models[k];
        FitJob &j = jobs[k];
        j.code = P->dcode + coff[k];
        j.start_code = P->dcode + soff[k];
        j.n_code = (int)md->code.size();
        j.n_start = (int)md->start_code.size();
        j.m = (int)md->params.size();
        j.nf = (int)md->features.size();
        j.l = (int)P->rows[k];
        j.linear = md->linear;
        j.use_p0 = P->use_p0;
        j.start_mask = md->start_mask;
        j.X = P->dX32 + P->xoff[k];
        j.t = P->dt32 + toff;
        j.p = P->dp + P->poff[k];
        j.rep = P->drep + 8 * k;
        toff += P->rows[k];
    }
    PM_CUDA_TRY(cudaMemcpy(P->dcode, code.data(), code.size() * sizeof(Ins), cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(P->djobs, jobs.data(), K * sizeof(FitJob), cudaMemcpyHostToDevice));
    // capture the per-run work into a graph
    PM_CUDA_TRY(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
    PM_CUDA_TRY(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
    pm_status s = PM_OK;
    cudaError_t e = cudaSuccess;
    if (P->nx) e = cudaMemcpyAsync(P->dX64, P->hX, P->nx * 8, cudaMemcpyHostToDevice, P->cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->dt64, P->ht, P->nt * 8, cudaMemcpyHostToDevice, P->cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->dp, P->hp, P->np * 8, cudaMemcpyHostToDevice, P->cap);
    if (e == cudaSuccess && P->nx) {
        k_split<<<152, 256, 0, P->cap>>>(P->dX64, P->dX32, P->nx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_split<<<152, 256, 0, P->cap>>>(P->dt64, P->dt32, P->nt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) s = launch_fit(P->threads, P->djobs, (int)K, P->cfg, P->cap);
    if (e == cudaSuccess && s == PM_OK) e = cudaMemcpyAsync(P->hp, P->dp, P->np * 8, cudaMemcpyDeviceToHost, P->cap);
    if (e == cudaSuccess && s == PM_OK)
        e = cudaMemcpyAsync(P->hrep, P->drep, K * 64, cudaMemcpyDeviceToHost, P->cap);
    cudaError_t e2 = cudaStreamEndCapture(P->cap, &P->graph);
    if (s) return s;
    if (e != cudaSuccess) return fail(PM_ECUDA, "fit plan capture: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(PM_ECUDA, "fit plan capture: %s", cudaGetErrorString(e2));
    PM_CUDA_TRY(cudaGraphInstantiate(&P->exec, P->graph, 0));
    return PM_OK;
}

pm_status check_opts(const pm_fit_opts *o, FitCfg &cfg, int &use_p0) {
    cfg.max_iter = 200;
    cfg.ftol = 1e-15;
    cfg.xtol = 1e-12;
    use_p0 = 0;
    if (o) {
        if (o->max_iter < 0 || o->max_iter > 100000) return fail(PM_EINVAL, "fit: max_iter must be 0..100000");
        if (!(o->ftol >= 0) || !(o->xtol >= 0)) return fail(PM_EINVAL, "fit: ftol and xtol must be >= 0");
        cfg.max_iter = o->max_iter;
        cfg.ftol = o->ftol;
        cfg.xtol = o->xtol;
        use_p0 = o->use_p0 ? 1 : 0;
    }
    return PM_OK;
}

}  // namespace
}  // namespace pm

extern "C" {

pm_status pm_fit_plan_create(const pm_model *const *models, size_t nmodels, const size_t *rows,
                             const pm_fit_opts *opts, int32_t threads, pm_fit_plan **plan) {
    if (!models || !rows || !plan || nmodels == 0) return fail(PM_EINVAL, "pm_fit_plan_create: bad argument");
    if (nmodels > 65535) return fail(PM_EINVAL, "pm_fit_plan_create: at most 65535 models");
    if (threads != 0 && threads != 64 && threads != 128 && threads != 256 && threads != 512)
        return fail(PM_EINVAL, "pm_fit_plan_create: threads must be 0, 64, 128, 256 or 512");
    pm_fit_plan *P = new (std::nothrow) pm_fit_plan();
    if (!P) return fail(PM_ENOMEM, "pm_fit_plan_create: out of memory");
    pm_status s = check_opts(opts, P->cfg, P->use_p0);
    if (s) { delete P; return s; }
    P->threads = threads ? threads : 128;
    for (size_t k = 0; k < nmodels; k++) {
        const pm_model *m = models[k];
        if (!m) { delete P; return fail(PM_EINVAL, "pm_fit_plan_create: model %zu is NULL", k); }
        if (rows[k] < 1 || rows[k] > (1u << 24)) {
            delete P;
            return fail(PM_EINVAL, "pm_fit_plan_create: model %zu needs 1..2^24 rows", k);
        }
        P->models.push_back(m);
        P->rows.push_back(rows[k]);
        P->xoff.push_back(P->nx);
        P->poff.push_back(P->np);
        P->nx += rows[k] * m->features.size();
        P->nt += rows[k];
        P->np += m->params.size();
    }
    s = plan_build(P);
    if (s) { delete P; return s; }
    *plan = P;
    return PM_OK;
}

void pm_fit_plan_destroy(pm_fit_plan *plan) { delete plan; }

pm_status pm_fit_plan_run(pm_fit_plan *P, const double *X, const double *t, double *p_inout, pm_fit_report *reports,
                          void *stream) {
    if (!P || !t || !p_inout || (P->nx && !X)) return fail(PM_EINVAL, "pm_fit_plan_run: NULL argument");
    // validate while copying into the pinned staging buffers (one pass)
    for (size_t k = 0, o = 0; k < P->models.size(); k++)
        for (size_t r = 0; r < P->rows[k]; r++, o++) {
            const double v = t[o];
            if (!finite_pos(v)) return fail(PM_EINVAL, "fit: model %zu row %zu: output must be finite and > 0", k, r);
            P->ht[o] = v;
        }
    bool bad = false;
    for (size_t i = 0; i < P->nx; i++) {
        const double v = X[i];
        bad |= !std::isfinite(v);
        P->hX[i] = v;
    }
    if (bad)
        for (size_t i = 0; i < P->nx; i++)
            if (!std::isfinite(X[i])) return fail(PM_EINVAL, "fit: feature value %zu is not finite", i);
    if (P->use_p0)
        for (size_t i = 0; i < P->np; i++)
            if (!std::isfinite(p_inout[i])) return fail(PM_EINVAL, "fit: start point %zu is not finite", i);
    memcpy(P->hp, p_inout, P->np * 8);
    cudaStream_t st = (cudaStream_t)stream;
    PM_CUDA_TRY(cudaGraphLaunch(P->exec, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    memcpy(p_inout, P->hp, P->np * 8);
    if (reports)
        for (size_t k = 0; k < P->models.size(); k++) {
            const double *r = P->hrep + 8 * k;
            reports[k].status = (int32_t)r[0];
            reports[k].iterations = (int32_t)r[1];
            reports[k].rank = (int32_t)r[2];
            reports[k].linear = (int32_t)r[3];
            reports[k].residual = r[4];
            reports[k].lambda = r[5];
            reports[k].cond = r[6];
        }
    return PM_OK;
}

pm_status pm_fit_batched(const pm_model *const *models, size_t nmodels, const double *X, const double *t,
                         const size_t *rows, const pm_fit_opts *opts, double *p_inout, pm_fit_report *reports,
                         void *stream) {
    pm_fit_plan *P = nullptr;
    pm_status s = pm_fit_plan_create(models, nmodels, rows, opts, 0, &P);
    if (s) return s;
    s = pm_fit_plan_run(P, X, t, p_inout, reports, stream);
    pm_fit_plan_destroy(P);
    return s;
}

pm_status pm_fit(const pm_model *m, const double *X, const double *t, size_t l, const pm_fit_opts *opts,
                 double *p_inout, pm_fit_report *report) {
    if (!m || !t || !p_inout) return fail(PM_EINVAL, "pm_fit: NULL argument");
    pm_fit_report rep{};
    pm_status s = pm_fit_batched(&m, 1, X, t, &l, opts, p_inout, &rep, nullptr);
    if (s) return s;
    if (report) *report = rep;
    if (rep.status == PM_ERANK) return fail(PM_ERANK, "pm_fit: rank-deficient design (rank %d of %zu)", rep.rank,
                                            m->params.size());
    if (rep.status == PM_ENOTCONV) return fail(PM_ENOTCONV, "pm_fit: no convergence in %d iterations", rep.iterations);
    return (pm_status)rep.status;
}

pm_status pm_predict(const pm_model *m, const double *p, const double *X, size_t l, double *t_out) {
    if (!m || !p || !t_out || (l && !X && !m->features.empty())) return fail(PM_EINVAL, "pm_predict: NULL argument");
    if (l == 0) return PM_OK;
    const size_t nf = m->features.size(), np = m->params.size();
    pm_status s = retain_staging_pool();
    if (s) return s;
    // stream-ordered staging from the device's memory pool (kept reserved):
    // no cudaMalloc / cudaFree per call, which would synchronise the device
    // and slow the host-to-device copies issued after it
    cudaStream_t st = 0;
    double *dX = nullptr, *dp = nullptr, *dout = nullptr;
    Ins *dc = nullptr;
    auto alloc = [&](void **q, size_t b) { return !alloc_fault_injected() && cudaMallocAsync(q, b, st) == cudaSuccess; };
    if (!alloc((void **)&dX, std::max<size_t>(l * nf, 1) * 8) || !alloc((void **)&dp, np * 8) ||
        !alloc((void **)&dout, l * 8) || !alloc((void **)&dc, m->code.size() * sizeof(Ins)))
        s = fail(PM_ENOMEM, "pm_predict: device allocation failed");
    if (!s && nf && cudaMemcpyAsync(dX, X, l * nf * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        s = fail(PM_ECUDA, "pm_predict: copy failed");
    if (!s && cudaMemcpyAsync(dp, p, np * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        s = fail(PM_ECUDA, "pm_predict: copy failed");
    if (!s && cudaMemcpyAsync(dc, m->code.data(), m->code.size() * sizeof(Ins), cudaMemcpyHostToDevice, st) != cudaSuccess)
        s = fail(PM_ECUDA, "pm_predict: copy failed");
    if (!s) {
        const unsigned blocks = (unsigned)std::min<size_t>((l + 127) / 128, 1216);
        k_predict<<<blocks, 128, 0, st>>>(dc, (int)m->code.size(), (int)nf, dX, l, dp, dout, (int)np);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(t_out, dout, l * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = fail(PM_ECUDA, "pm_predict: %s", cudaGetErrorString(e));
    }
    for (void *q : {(void *)dX, (void *)dp, (void *)dout, (void *)dc})
        if (q) cudaFreeAsync(q, st);
    cudaStreamSynchronize(st);
    return s;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free batched fit
// Scratch for pm_fit_batched_noalloc: one file-scope device array, present on
// every GPU that loads this library until the process exits.  Host code must
// not hand the symbol itself to a kernel (on the host it names a host-side
// shadow); it looks up the device address once per device with
// cudaGetSymbolAddress and passes that.
namespace pm {
namespace {

static __device__ __align__(256) unsigned char g_fit_scratch[PM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr size_t kNoallocMaxModels = 256;
static void *g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Host image of the scratch's first region (job table, then every model's
// program and start program), built here and uploaded with one copy.  Static
// storage: the call allocates no host memory either.  A model's start program
// is never longer than its program (kMaxIns instructions).
constexpr size_t kStageBytes = align256(kNoallocMaxModels * sizeof(FitJob)) + kNoallocMaxModels * 2 * kMaxIns * sizeof(Ins);
static __align__(256) unsigned char g_host_stage[kStageBytes];

// Device address of g_fit_scratch on the current device, looked up on the
// first call per device (with that device current) and cached.
pm_status scratch_address(void **out) {
    int dev = 0;
    PM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(PM_EINVAL, "noalloc fit: device ordinal %d unsupported", dev);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fit_scratch);
        if (e != cudaSuccess || !p)
            return fail(PM_ECUDA, "noalloc fit: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PM_OK;
}

}  // namespace
}  // namespace pm

extern "C" pm_status pm_fit_batched_noalloc(const pm_model *const *models, size_t nmodels, const double *X,
                                            const double *t, const size_t *rows, const pm_fit_opts *opts,
                                            double *p_inout, pm_fit_report *reports, void *stream) {
    using namespace pm;
    if (!models || !rows || !t || !p_inout || nmodels == 0) return fail(PM_EINVAL, "pm_fit_batched_noalloc: bad argument");
    if (nmodels > kNoallocMaxModels)
        return fail(PM_EINVAL, "pm_fit_batched_noalloc: at most %zu models per call", kNoallocMaxModels);
    FitCfg cfg;
    int use_p0 = 0;
    pm_status s = check_opts(opts, cfg, use_p0);
    if (s) return s;
    // layout of the scratch: jobs | code | X (FP64) | X (hi, lo) | t (FP64) | t (hi, lo) | p | reports
    size_t nx = 0, nt = 0, np = 0, ncode = 0;
    for (size_t k = 0; k < nmodels; k++) {
        const pm_model *m = models[k];
        if (!m) return fail(PM_EINVAL, "pm_fit_batched_noalloc: model %zu is NULL", k);
        if (rows[k] < 1 || rows[k] > (1u << 24)) return fail(PM_EINVAL, "pm_fit_batched_noalloc: model %zu needs 1..2^24 rows", k);
        nx += rows[k] * m->features.size();
        nt += rows[k];
        np += m->params.size();
        ncode += m->code.size() + m->start_code.size();
    }
    if (nx && !X) return fail(PM_EINVAL, "pm_fit_batched_noalloc: X is NULL");
    const size_t o_jobs = 0, o_code = align256(o_jobs + nmodels * sizeof(FitJob));
    const size_t o_x64 = align256(o_code + ncode * sizeof(Ins)), o_x2 = align256(o_x64 + nx * 8);
    const size_t o_t64 = align256(o_x2 + nx * 8), o_t2 = align256(o_t64 + nt * 8);
    const size_t o_p = align256(o_t2 + nt * 8), o_rep = align256(o_p + np * 8);
    const size_t need = align256(o_rep + nmodels * 64);
    if (need > (size_t)PM_NOALLOC_SCRATCH_BYTES)
        return fail(PM_EINVAL, "pm_fit_batched_noalloc: request needs %zu bytes of scratch, the limit is %zu",
                    need, (size_t)PM_NOALLOC_SCRATCH_BYTES);
    if (o_code + ncode * sizeof(Ins) > kStageBytes)
        return fail(PM_EINVAL, "pm_fit_batched_noalloc: model programs exceed the staging area");
    for (size_t k = 0, o = 0; k < nmodels; k++)
        for (size_t r = 0; r < rows[k]; r++, o++)
            if (!finite_pos(t[o])) return fail(PM_EINVAL, "fit: model %zu row %zu: output must be finite and > 0", k, r);
    for (size_t i = 0; i < nx; i++)
        if (!std::isfinite(X[i])) return fail(PM_EINVAL, "fit: feature value %zu is not finite", i);
    if (use_p0)
        for (size_t i = 0; i < np; i++)
            if (!std::isfinite(p_inout[i])) return fail(PM_EINVAL, "fit: start point %zu is not finite", i);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    void *base = nullptr;
    if ((s = scratch_address(&base))) return s;
    unsigned char *B = (unsigned char *)base;
    cudaStream_t st = (cudaStream_t)stream;
    // job table and programs: built in the host image of [0, o_x64), one upload
    FitJob *jobs = (FitJob *)(g_host_stage + o_jobs);
    Ins *hcode = (Ins *)(g_host_stage + o_code);
    size_t co = 0, xo = 0, to = 0, po = 0;
    for (size_t k = 0; k < nmodels; k++) {
        const pm_model *md = models[k];
        FitJob &j = jobs[k];
        memcpy(hcode + co, md->code.data(), md->code.size() * sizeof(Ins));
        memcpy(hcode + co + md->code.size(), md->start_code.data(), md->start_code.size() * sizeof(Ins));
        Ins *code = (Ins *)(B + o_code) + co;
        j.code = code;
        j.start_code = code + md->code.size();
        j.n_code = (int)md->code.size();
        j.n_start = (int)md->start_code.size();
        j.m = (int)md->params.size();
        j.nf = (int)md->features.size();
        j.l = (int)rows[k];
        j.linear = md->linear;
        j.use_p0 = use_p0;
        j.start_mask = md->start_mask;
        j.X = (const float2 *)(B + o_x2) + xo;
        j.t = (const float2 *)(B + o_t2) + to;
        j.p = (double *)(B + o_p) + po;
        j.rep = (double *)(B + o_rep) + 8 * k;
        co += md->code.size() + md->start_code.size();
        xo += rows[k] * md->features.size();
        to += rows[k];
        po += md->params.size();
    }
    // pageable-source copies return once the source has been staged, so the
    // host image may be rebuilt by the next call as soon as this one returns
    PM_CUDA_TRY(cudaMemcpyAsync(B + o_jobs, g_host_stage, o_code + ncode * sizeof(Ins), cudaMemcpyHostToDevice, st));
    if (nx) PM_CUDA_TRY(cudaMemcpyAsync(B + o_x64, X, nx * 8, cudaMemcpyHostToDevice, st));
    PM_CUDA_TRY(cudaMemcpyAsync(B + o_t64, t, nt * 8, cudaMemcpyHostToDevice, st));
    PM_CUDA_TRY(cudaMemcpyAsync(B + o_p, p_inout, np * 8, cudaMemcpyHostToDevice, st));
    if (nx) k_split<<<152, 256, 0, st>>>((const double *)(B + o_x64), (float2 *)(B + o_x2), nx);
    k_split<<<152, 256, 0, st>>>((const double *)(B + o_t64), (float2 *)(B + o_t2), nt);
    PM_CUDA_TRY(cudaGetLastError());
    if ((s = launch_fit(128, (const FitJob *)(B + o_jobs), (int)nmodels, cfg, st))) return s;
    PM_CUDA_TRY(cudaMemcpyAsync(p_inout, B + o_p, np * 8, cudaMemcpyDeviceToHost, st));
    double rep_host[kNoallocMaxModels * 8];
    PM_CUDA_TRY(cudaMemcpyAsync(rep_host, B + o_rep, nmodels * 64, cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    if (reports)
        for (size_t k = 0; k < nmodels; k++) {
            const double *r = rep_host + 8 * k;
            reports[k].status = (int32_t)r[0];
            reports[k].iterations = (int32_t)r[1];
            reports[k].rank = (int32_t)r[2];
            reports[k].linear = (int32_t)r[3];
            reports[k].residual = r[4];
            reports[k].lambda = r[5];
            reports[k].cond = r[6];
        }
    return PM_OK;
}
