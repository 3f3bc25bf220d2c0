// Double-float arithmetic: a real number held as the unevaluated sum hi + lo of
// two FP32 values with |lo| <= ulp(hi) / 2, about 48 significant bits.  GB300
// issues FP32 at 64 times its FP64 rate, so kernels whose FP64 work sits on a
// latency-bound critical path (the Householder tridiagonalisation) run it here.
//
// Building blocks, each exact in round-to-nearest FP32:
//   - TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the rounding error e,
//     a + b = s + e;
//   - FastTwoSum (Dekker 1971), for |a| >= |b|: the same with three operations;
//   - TwoProduct by one fused multiply-add: p = fl(a b), e = fma(a, b, -p),
//     a b = p + e.
// Sums and products of double-floats are Dekker's add2/mul2 with the low-order
// terms summed in FP32 and one renormalisation; their relative error is a few
// units of 2^-48 (add: relative to |x| + |y|).  Division and square root take
// one Newton correction on the FP32 quotient or root.  Every operation goes
// through the _rn intrinsics on the device (the compiler may not fuse or
// reassociate them); the host versions are plain FP32 expressions and must be
// compiled without contraction (-ffp-contract=off).
#pragma once
#include <math.h>
#include <string.h>

#ifdef __CUDACC__
#define DF_FN __host__ __device__ __forceinline__
#else
#define DF_FN inline
#endif

namespace rsdft {
namespace dfl {

DF_FN float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
DF_FN float fsub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
DF_FN float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
DF_FN float ffma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
DF_FN float fdiv(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdiv_rn(a, b);
#else
    return a / b;
#endif
}
DF_FN float fsqrt(float a) {
#ifdef __CUDA_ARCH__
    return __fsqrt_rn(a);
#else
    return sqrtf(a);
#endif
}

// FP32 bit patterns (exponent tests and exact powers of two)
DF_FN int fbits(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_int(x);
#else
    int b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}
DF_FN float ffrombits(int b) {
#ifdef __CUDA_ARCH__
    return __int_as_float(b);
#else
    float x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}
DF_FN int fexp(float x) { return ((fbits(x) >> 23) & 0xff) - 127; }   // unbiased exponent

struct df {
    float h, l;
};

// complex double-float
struct cdf {
    df re, im;
};

DF_FN df mk(float h) { return df{h, 0.0f}; }

DF_FN df two_sum(float a, float b) {
    const float s = fadd(a, b);
    const float bb = fsub(s, a);
    const float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
    return df{s, e};
}

// requires |a| >= |b| (or a == 0)
DF_FN df fast_two_sum(float a, float b) {
    const float s = fadd(a, b);
    return df{s, fsub(b, fsub(s, a))};
}

DF_FN df two_prod(float a, float b) {
    const float p = fmul(a, b);
    return df{p, ffma(a, b, -p)};
}

DF_FN df neg(df x) { return df{-x.h, -x.l}; }

DF_FN df add(df x, df y) {
    const df s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, fadd(s.l, fadd(x.l, y.l)));
}

DF_FN df sub(df x, df y) { return add(x, neg(y)); }

DF_FN df mul(df x, df y) {
    const df p = two_prod(x.h, y.h);
    return fast_two_sum(p.h, ffma(x.h, y.l, ffma(x.l, y.h, p.l)));
}

DF_FN df mul_f(df x, float c) {   // c exact in FP32 (a power of two, a small integer)
    const df p = two_prod(x.h, c);
    return fast_two_sum(p.h, ffma(x.l, c, p.l));
}

DF_FN df sqr(df x) {
    const df p = two_prod(x.h, x.h);
    return fast_two_sum(p.h, ffma(fadd(x.h, x.h), x.l, p.l));
}

// x / y, y != 0
DF_FN df div(df x, df y) {
    const float q1 = fdiv(x.h, y.h);
    const df r = sub(x, mul(y, mk(q1)));
    const float q2 = fdiv(r.h, y.h);
    return fast_two_sum(q1, q2);
}

// sqrt(x), x >= 0 (0 for x <= 0)
DF_FN df sqrt(df x) {
    if (!(x.h > 0.0f)) return df{0.0f, 0.0f};
    const float s = fsqrt(x.h);
    const df r = sub(x, two_prod(s, s));
    return fast_two_sum(s, fdiv(r.h, fadd(s, s)));
}

// conversions at the FP64 boundary (FP64 operations: used once per value)
DF_FN df from_double(double v) {
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
}
DF_FN double to_double(df x) { return (double)x.h + (double)x.l; }

// ---- complex -----------------------------------------------------------------------
DF_FN cdf cadd(cdf a, cdf b) { return cdf{add(a.re, b.re), add(a.im, b.im)}; }
DF_FN cdf csub(cdf a, cdf b) { return cdf{sub(a.re, b.re), sub(a.im, b.im)}; }
DF_FN cdf cconj(cdf a) { return cdf{a.re, neg(a.im)}; }
DF_FN cdf cneg(cdf a) { return cdf{neg(a.re), neg(a.im)}; }

// a b
DF_FN cdf cmul(cdf a, cdf b) {
    return cdf{sub(mul(a.re, b.re), mul(a.im, b.im)), add(mul(a.re, b.im), mul(a.im, b.re))};
}
// conj(a) b
DF_FN cdf cmulc(cdf a, cdf b) {
    return cdf{add(mul(a.re, b.re), mul(a.im, b.im)), sub(mul(a.re, b.im), mul(a.im, b.re))};
}
DF_FN cdf cscale(cdf a, df s) { return cdf{mul(a.re, s), mul(a.im, s)}; }
DF_FN df cabs2(cdf a) { return add(sqr(a.re), sqr(a.im)); }

}  // namespace dfl
}  // namespace rsdft
