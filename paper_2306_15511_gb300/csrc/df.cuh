// Double-FP32 ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi) / 2, about 48 significant bits.  On GB300
// the FP32 pipe issues 64 times as many operations per clock as the FP64
// pipe, so a multiply-add in this arithmetic (about twelve FP32 operations)
// runs several times faster than a native FP64 one while its rounding error
// (~2^-47 relative per operation) stays far below the 1e-10 the FP64
// transforms are held to.  The exponent range is FP32's: the Legendre values
// start at 2^-80 (FP64 start-state threshold) and the data are O(1e-3 ..
// 1e4), so every hi and lo stays normal.
//
// Error-free transformations (restated from the literature):
//   two_sum      s + e = a + b exactly          (Knuth, TAOCP vol. 2, 4.2.2)
//   fast_two_sum s + e = a + b for |a| >= |b|   (Dekker 1971)
//   two_prod     p + e = a * b exactly, via FMA (Dekker 1971 with a fused
//                multiply-add in place of his splitting)
#pragma once
#include <cuda_runtime.h>

// host and device: the kernels use these on the GPU, and a CPU test checks
// the error-free transformations and error bounds exactly on the host
#define SHTG_DF_FN __host__ __device__ __forceinline__

namespace shtg {

struct __align__(8) df {
    float hi, lo;
};
struct __align__(16) dfc {   // complex
    df re, im;
};

SHTG_DF_FN df df_make(float h, float l) {
    df r;
    r.hi = h;
    r.lo = l;
    return r;
}
SHTG_DF_FN df df_zero() { return df_make(0.f, 0.f); }

SHTG_DF_FN float two_sum(float a, float b, float &e) {
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}
SHTG_DF_FN float fast_two_sum(float a, float b, float &e) {
    const float s = a + b;
    e = b - (s - a);
    return s;
}
SHTG_DF_FN float two_prod(float a, float b, float &e) {
    const float p = a * b;
    e = fmaf(a, b, -p);
    return p;
}

// nearest df of a double (three FP64-pipe operations: used only when data
// are staged, never per multiply-add)
SHTG_DF_FN df df_from(double x) {
#ifdef __CUDA_ARCH__
    const float h = __double2float_rn(x);
    return df_make(h, __double2float_rn(x - (double)h));
#else
    const float h = (float)x;   // round to nearest, the host default
    return df_make(h, (float)(x - (double)h));
#endif
}
SHTG_DF_FN double df_to(df a) { return (double)a.hi + (double)a.lo; }

SHTG_DF_FN df df_neg(df a) { return df_make(-a.hi, -a.lo); }

// a + b: error below 2^-47 (|a| + |b|)
SHTG_DF_FN df df_add(df a, df b) {
    float e;
    const float s = two_sum(a.hi, b.hi, e);
    e += a.lo + b.lo;
    float l;
    const float h = fast_two_sum(s, e, l);
    return df_make(h, l);
}
SHTG_DF_FN df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b: error below 2^-46 |a b|
SHTG_DF_FN df df_mul(df a, df b) {
    float e;
    const float p = two_prod(a.hi, b.hi, e);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float l;
    const float h = fast_two_sum(p, e, l);
    return df_make(h, l);
}

// Running sum of products, not renormalised per term: hi collects the
// leading products through two_sum, lo the rounding errors and the
// lower-order product terms.  lo grows by one error term per product, so
// the sum is renormalised (df_acc_norm) every few dozen terms.
struct dfacc {
    float hi, lo;
};
SHTG_DF_FN void df_acc_zero(dfacc &s) { s.hi = s.lo = 0.f; }
// s += a * b
SHTG_DF_FN void df_fma(dfacc &s, df a, df b) {
    float e;
    const float p = two_prod(a.hi, b.hi, e);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float e2;
    s.hi = two_sum(s.hi, p, e2);
    s.lo += e2 + e;
}
// (two_sum: after cancellation hi may be smaller than lo)
SHTG_DF_FN void df_acc_norm(dfacc &s) {
    float l;
    s.hi = two_sum(s.hi, s.lo, l);
    s.lo = l;
}
SHTG_DF_FN double df_acc_to(const dfacc &s) { return (double)s.hi + (double)s.lo; }

}  // namespace shtg
