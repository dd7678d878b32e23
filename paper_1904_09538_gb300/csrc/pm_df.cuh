// Float-float ("double-float") arithmetic on the FP32 pipes: a value is an
// unevaluated sum hi + lo of two floats (about 48 significant bits).  Built
// from the error-free transformations TwoSum (Knuth) and TwoProd (via fused
// multiply-add), in the style of Dekker's and Bailey's double-double
// arithmetic.  Every operation uses explicitly rounded FP32 intrinsics so the
// compiler cannot re-associate or contract them.
#pragma once
#include <cuda_runtime.h>

namespace pm {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df dfv(float h, float l = 0.0f) { return df{h, l}; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// |a| >= |b|
__device__ __forceinline__ void quick_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_add(df x, df y) {
    float s, e, t, f;
    two_sum(x.hi, y.hi, s, e);
    two_sum(x.lo, y.lo, t, f);
    e = __fadd_rn(e, t);
    quick_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    quick_two_sum(s, e, s, e);
    return df{s, e};
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y) {
    float p, e;
    two_prod(x.hi, y.hi, p, e);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    quick_two_sum(p, e, p, e);
    return df{p, e};
}
__device__ __forceinline__ df df_mulf(df x, float b) {
    float p, e;
    two_prod(x.hi, b, p, e);
    e = __fmaf_rn(x.lo, b, e);
    quick_two_sum(p, e, p, e);
    return df{p, e};
}
// Long division with three quotient digits.  Each digit only needs to be
// close (the exact remainder r = x - y q carries its error into the next
// one), so they come from one reciprocal of y.hi (approximate, a few ulp):
// after q1 the remainder is ~2^-22 |x|, after q2 ~2^-44, and q3 brings the
// result to float-float accuracy.
__device__ __forceinline__ df df_div(df x, df y) {
    const float ry = __fdividef(1.0f, y.hi);
    const float q1 = __fmul_rn(x.hi, ry);
    df r = df_sub(x, df_mulf(y, q1));
    const float q2 = __fmul_rn(r.hi, ry);
    r = df_sub(r, df_mulf(y, q2));
    const float q3 = __fmul_rn(r.hi, ry);
    float s, e;
    quick_two_sum(q1, q2, s, e);
    return df_add(df{s, e}, df{q3, 0.0f});
}
__device__ __forceinline__ df df_sqrt(df x) {
    if (!(x.hi > 0.0f)) return df{sqrtf(x.hi), 0.0f};
    const float s = sqrtf(x.hi);
    // one Newton step: s + (x - s^2) / (2 s)
    const df r = df_sub(x, df_mul(df{s, 0.0f}, df{s, 0.0f}));
    const float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
    float a, b;
    quick_two_sum(s, c, a, b);
    return df{a, b};
}

// e^x - 1 for x in float-float: x = k ln2 + r, |r| <= ln2/2; e^(r/16) - 1 by
// its Taylor series (degree 8: remainder below 2^-60 for |r/16| <= 0.022),
// then s <- 2 s + s^2 four times gives e^r - 1, then 2^k (1 + s) - 1.
__device__ __forceinline__ df df_expm1(df x) {
    const df LN2 = df{0.693147182464599609375f, -1.9046542999577797e-09f};
    if (x.hi > 88.0f) return df{__int_as_float(0x7f800000), 0.0f};
    if (x.hi < -88.0f) return df{-1.0f, 0.0f};
    const float k = rintf(__fmul_rn(x.hi, 1.44269502162933349609375f));
    df r = df_sub(x, df_mulf(LN2, k));
    r = df{__fmul_rn(r.hi, 0.0625f), __fmul_rn(r.lo, 0.0625f)};
    // Horner on r: sum_{k<8} r^k / (k+1)!, the coefficients as float-float
    // constants (hi + lo of 1/(k+1)! to 2^-49 relative)
    df p = df{0x1.a01a02p-16f, -0x1.7f97fap-42f};                        // 1/8!
    p = df_add(df_mul(p, r), df{0x1.a01a02p-13f, -0x1.7f97fap-39f});       // 1/7!
    p = df_add(df_mul(p, r), df{0x1.6c16c2p-10f, -0x1.27d27ep-35f});       // 1/6!
    p = df_add(df_mul(p, r), df{0x1.111112p-7f, -0x1.dddddep-32f});        // 1/5!
    p = df_add(df_mul(p, r), df{0x1.555556p-5f, -0x1.555556p-30f});        // 1/4!
    p = df_add(df_mul(p, r), df{0x1.555556p-3f, -0x1.555556p-28f});        // 1/3!
    p = df_add(df_mul(p, r), df{0.5f, 0.0f});                              // 1/2!
    p = df_add(df_mul(p, r), df{1.0f, 0.0f});                              // 1/1!
    df s = df_mul(p, r);  // e^(r/16) - 1
    for (int i = 0; i < 4; i++) s = df_add(df_mulf(s, 2.0f), df_mul(s, s));
    if (k == 0.0f) return s;
    const int ki = (int)k;
    df e = df_add(s, df{1.0f, 0.0f});
    e = df{ldexpf(e.hi, ki), ldexpf(e.lo, ki)};
    return df_sub(e, df{1.0f, 0.0f});
}
__device__ __forceinline__ df df_exp(df x) {
    if (x.hi < -88.0f) return df{0.0f, 0.0f};
    return df_add(df_expm1(x), df{1.0f, 0.0f});
}
// tanh(y) = s / (s + 2), s = e^(2y) - 1, for y >= 0 (odd extension)
__device__ __forceinline__ df df_tanh(df x) {
    const bool neg = x.hi < 0.0f;
    df y = neg ? df_neg(x) : x;
    df t;
    if (y.hi > 40.0f) t = df{1.0f, 0.0f};
    else {
        const df s = df_expm1(df_mulf(y, 2.0f));
        t = df_div(s, df_add(s, df{2.0f, 0.0f}));
    }
    return neg ? df_neg(t) : t;
}
// log by one Newton step from the FP32 logarithm: y1 = y0 + x e^-y0 - 1
__device__ __forceinline__ df df_log(df x) {
    const float y0 = logf(x.hi);
    if (!isfinite(y0)) return df{y0, 0.0f};
    const df d = df_sub(df_mul(x, df_exp(df{-y0, 0.0f})), df{1.0f, 0.0f});
    return df_add(df{y0, 0.0f}, d);
}

// Compensated accumulator of float-float terms (hi + lo), error-free TwoSum
// of the high parts with the rounding errors collected separately.
struct CAcc {
    float s, c;
    __device__ void init() { s = 0.0f; c = 0.0f; }
    __device__ void add(float hi, float lo) {
        float t, e;
        two_sum(s, hi, t, e);
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, lo));
    }
    // a * b exactly (TwoProd) into the sum
    __device__ void add_prod(float a, float b) {
        float p, e;
        two_prod(a, b, p, e);
        add(p, e);
    }
    __device__ double value() const { return (double)s + (double)c; }
    // the sum as a float-float value (no FP64 arithmetic)
    __device__ df sum() const {
        float h, l;
        two_sum(s, c, h, l);
        return df{h, l};
    }
};

// Sum of a float-float value over the 32 lanes of a warp (butterfly; every
// lane receives the same result, df_add being symmetric in its operands).
__device__ __forceinline__ df warp_sum(df x) {
    for (int o = 16; o; o >>= 1) {
        const df y = df{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
        x = df_add(x, y);
    }
    return x;
}

}  // namespace pm
