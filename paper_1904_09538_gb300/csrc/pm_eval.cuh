// Evaluation and reverse-mode differentiation of a model's SSA program
// (Section "Modeling Kernel Execution Time": a model is an expression over
// features f_* and parameters p_*; Section "Computing Model Parameters": its
// derivatives with respect to the parameters).  Shared by the batched fit
// (pm_fit.cu) and the per-model differentiation entry points
// (pm_autograd.cu).
#pragma once
#include <cuda_runtime.h>

#include "pm_df.cuh"
#include "pm_model.h"

namespace pm {
namespace {

__device__ __forceinline__ float fn32(int op, float x) {
    switch (op) {
    case OP_TANH: return tanhf(x);
    case OP_EXP: return expf(x);
    case OP_LOG: return logf(x);
    default: return sqrtf(x);
    }
}
__device__ __forceinline__ double fn64(int op, double x) {
    switch (op) {
    case OP_TANH: return tanh(x);
    case OP_EXP: return exp(x);
    case OP_LOG: return log(x);
    default: return sqrt(x);
    }
}

// Forward sweep over the SSA program; v[k] receives every value.
template <typename T, typename F>
__device__ T forward(const Ins *code, int n, const F *frow, const T *par, T *v) {
    for (int k = 0; k < n; k++) {
        const Ins in = code[k];
        T x;
        switch (in.op) {
        case OP_FEAT: x = (T)frow[in.arg]; break;
        case OP_PAR: x = par[in.arg]; break;
        case OP_CONST: x = (T)in.c; break;
        case OP_ADD: x = v[in.a] + v[in.b]; break;
        case OP_SUB: x = v[in.a] - v[in.b]; break;
        case OP_MUL: x = v[in.a] * v[in.b]; break;
        case OP_DIV: x = v[in.a] / v[in.b]; break;
        case OP_NEG: x = -v[in.a]; break;
        default:
            if (sizeof(T) == 4) x = (T)fn32(in.op, (float)v[in.a]);
            else x = (T)fn64(in.op, (double)v[in.a]);
        }
        v[k] = x;
    }
    return v[n - 1];
}

// A feature value as float-float: stored as a (hi, lo) pair, or as FP64
// (split on the fly).
__device__ __forceinline__ df feat_df(const float2 *row, int i) {
    const float2 f = row[i];
    return df{f.x, f.y};
}
__device__ __forceinline__ df feat_df(const double *row, int i) {
    const double x = row[i];
    const float h = (float)x;
    return df{h, (float)(x - (double)h)};
}

// Forward sweep in float-float; cst[k] holds instruction k's constant as a
// float-float value (converted once per program load, not per row).
template <typename R>
__device__ df forward_df(const Ins *code, const df *cst, int n, const R *frow, const df *par, df *v) {
    for (int k = 0; k < n; k++) {
        const Ins in = code[k];
        df x;
        switch (in.op) {
        case OP_FEAT: x = feat_df(frow, in.arg); break;
        case OP_PAR: x = par[in.arg]; break;
        case OP_CONST: x = cst[k]; break;
        case OP_ADD: x = df_add(v[in.a], v[in.b]); break;
        case OP_SUB: x = df_sub(v[in.a], v[in.b]); break;
        case OP_MUL: x = df_mul(v[in.a], v[in.b]); break;
        case OP_DIV: x = df_div(v[in.a], v[in.b]); break;
        case OP_NEG: x = df_neg(v[in.a]); break;
        case OP_TANH: x = df_tanh(v[in.a]); break;
        case OP_EXP: x = df_exp(v[in.a]); break;
        case OP_LOG: x = df_log(v[in.a]); break;
        default: x = df_sqrt(v[in.a]);
        }
        v[k] = x;
    }
    return v[n - 1];
}

// d tanh(x) / dx = 1 - tanh(x)^2 = 4 e / (1 + e)^2 with e = exp(-2|x|): from the
// argument, without the cancellation of 1 - t*t when |t| is near 1 (at x = -8
// the FP32 value of t leaves 1 - t*t about 13 % off, enough to misdirect an
// LM step along the saturated column)
__device__ __forceinline__ float sech2f(float x) {
    const float e = expf(-2.0f * fabsf(x));
    const float d = 1.0f + e;
    return 4.0f * e / (d * d);
}

// Reverse sweep over the high parts of float-float forward values.
__device__ void reverse_df(const Ins *code, int n, const df *vd, float *adj, float *g, int m) {
    for (int k = 0; k < n; k++) adj[k] = 0.0f;
    for (int i = 0; i < m; i++) g[i] = 0.0f;
    adj[n - 1] = 1.0f;
    for (int k = n - 1; k >= 0; k--) {
        const float a = adj[k];
        if (a == 0.0f) continue;
        const Ins in = code[k];
        switch (in.op) {
        case OP_PAR: g[in.arg] += a; break;
        case OP_ADD: adj[in.a] += a; adj[in.b] += a; break;
        case OP_SUB: adj[in.a] += a; adj[in.b] -= a; break;
        case OP_MUL: adj[in.a] += a * vd[in.b].hi; adj[in.b] += a * vd[in.a].hi; break;
        case OP_DIV: adj[in.a] += a / vd[in.b].hi; adj[in.b] -= a * vd[k].hi / vd[in.b].hi; break;
        case OP_NEG: adj[in.a] -= a; break;
        case OP_TANH: adj[in.a] += a * sech2f(vd[in.a].hi); break;
        case OP_EXP: adj[in.a] += a * vd[k].hi; break;
        case OP_LOG: adj[in.a] += a / vd[in.a].hi; break;
        case OP_SQRT: adj[in.a] += a * 0.5f / vd[k].hi; break;
        default: break;
        }
    }
}

// Reverse sweep in float-float (adjoints and derivatives as hi + lo): the
// exact Jacobian of a linear model's direct solve.
__device__ void reverse_dd(const Ins *code, int n, const df *vd, df *adj, df *g, int m) {
    for (int k = 0; k < n; k++) adj[k] = df{0.0f, 0.0f};
    for (int i = 0; i < m; i++) g[i] = df{0.0f, 0.0f};
    adj[n - 1] = df{1.0f, 0.0f};
    for (int k = n - 1; k >= 0; k--) {
        const df a = adj[k];
        if (a.hi == 0.0f && a.lo == 0.0f) continue;
        const Ins in = code[k];
        switch (in.op) {
        case OP_PAR: g[in.arg] = df_add(g[in.arg], a); break;
        case OP_ADD: adj[in.a] = df_add(adj[in.a], a); adj[in.b] = df_add(adj[in.b], a); break;
        case OP_SUB: adj[in.a] = df_add(adj[in.a], a); adj[in.b] = df_sub(adj[in.b], a); break;
        case OP_MUL:
            adj[in.a] = df_add(adj[in.a], df_mul(a, vd[in.b]));
            adj[in.b] = df_add(adj[in.b], df_mul(a, vd[in.a]));
            break;
        case OP_DIV:
            adj[in.a] = df_add(adj[in.a], df_div(a, vd[in.b]));
            adj[in.b] = df_sub(adj[in.b], df_div(df_mul(a, vd[k]), vd[in.b]));
            break;
        case OP_NEG: adj[in.a] = df_sub(adj[in.a], a); break;
        case OP_TANH: adj[in.a] = df_add(adj[in.a], df_mul(a, df_sub(df{1.0f, 0.0f}, df_mul(vd[k], vd[k])))); break;
        case OP_EXP: adj[in.a] = df_add(adj[in.a], df_mul(a, vd[k])); break;
        case OP_LOG: adj[in.a] = df_add(adj[in.a], df_div(a, vd[in.a])); break;
        case OP_SQRT: adj[in.a] = df_add(adj[in.a], df_div(df_mulf(a, 0.5f), vd[k])); break;
        default: break;
        }
    }
}

}  // namespace
}  // namespace pm
