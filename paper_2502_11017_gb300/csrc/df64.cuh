// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32 numbers
// (|l| <= ulp(h)/2), about 48 significant bits. Built from error-free
// transformations (Knuth's TwoSum, FMA-based TwoProduct; Dekker 1971; the
// formulations of Joldes, Muller and Popescu, "Tight and rigorous error bounds for
// basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017), so it
// runs on the FP32 pipes. On GB300 these are ~64x the FP64 throughput and have
// ~1/15 of its dependent latency. All operations use the _rn intrinsics, which
// the compiler never contracts or reassociates.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace curk {

struct df64 {
    float h, l;
};

__device__ __forceinline__ df64 df_make(float h, float l = 0.f) { return df64{h, l}; }

// s + e = a + b exactly
__device__ __forceinline__ df64 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df64{s, e};
}
// s + e = a + b exactly, given |a| >= |b|
__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df64{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// p + e = a * b exactly
__device__ __forceinline__ df64 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return df64{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
    const df64 s = two_sum(a.h, b.h);
    const df64 t = two_sum(a.l, b.l);
    df64 v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ df64 df_neg(df64 a) { return df64{-a.h, -a.l}; }
__device__ __forceinline__ df64 df_sub(df64 a, df64 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
    df64 p = two_prod(a.h, b.h);
    float t = __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h));
    return fast_two_sum(p.h, __fadd_rn(p.l, t));
}
// double-float times float
__device__ __forceinline__ df64 df_mul_f(df64 a, float b) {
    df64 p = two_prod(a.h, b);
    return fast_two_sum(p.h, __fmaf_rn(a.l, b, p.l));
}
__device__ __forceinline__ df64 df_div(df64 a, df64 b) {
    const float q1 = __fdiv_rn(a.h, b.h);
    const df64 r = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.h, b.h);
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ float df_abs_h(df64 a) { return fabsf(a.h); }
__device__ __forceinline__ double df_to_d(df64 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ df64 df_from_d(double x) {
    const float h = (float)x;
    return df64{h, (float)(x - (double)h)};
}

// Running product of magnitudes as (mantissa in [1, 2), integer exponent), so that
// log|prod| = log(mantissa) + exponent * ln 2 needs a single logarithm at the end.
struct LogAcc {
    df64 mant;
    int expo;
    __device__ __forceinline__ void init() { mant = df64{1.f, 0.f}; expo = 0; }
    __device__ __forceinline__ void mul(df64 v) {
        v = v.h < 0.f ? df_neg(v) : v;
        int e;
        const float fh = frexpf(v.h, &e);        // v.h = fh * 2^e, fh in [0.5, 1)
        const float sc = ldexpf(1.f, 1 - e);     // exact power of two
        mant = df_mul(mant, df64{__fmul_rn(v.h, sc), __fmul_rn(v.l, sc)});
        expo += e - 1;
        int e2;
        const float m2 = frexpf(mant.h, &e2);
        (void)m2;
        const float s2 = ldexpf(1.f, 1 - e2);
        mant = df64{__fmul_rn(mant.h, s2), __fmul_rn(mant.l, s2)};
        expo += e2 - 1;
    }
    __device__ __forceinline__ double log_value() const {
        return log(df_to_d(mant)) + (double)expo * 0.6931471805599453;
    }
};

}  // namespace curk
