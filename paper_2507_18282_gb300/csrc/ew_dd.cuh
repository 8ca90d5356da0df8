// ew_dd.cuh -- double-FP32 arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
//
// Why: on this part FP64 arithmetic runs at a small fraction of the FP32 rate,
// so the FP64 filter applications of the mixed-precision eigen-solver are
// bound by the FP64 units; the same wave-solve in pairs of FP32 numbers costs
// 11 FP32 operations per addition, 7 per product and 15 per multiply-add, on
// the full-rate FP32 pipes.
//
// The building blocks are the error-free transformations:
//   two_sum(a, b):  s = fl(a + b) and the exact error e, a + b = s + e
//                   (Knuth's branch-free form, six additions)
//   fast_two_sum:   the same when |a| >= |b| (three additions)
//   two_prod(a, b): p = fl(a b) and e = fma(a, b, -p), a b = p + e
// and the pair operations built on them: addition adds the trailing parts to
// the error of the leading sum and renormalises (error bounded relative to the
// operands), multiplication adds the cross products to the error of the
// leading product.  Every rounding is explicit (_rn
// intrinsics on the device), so no compiler contraction or reassociation can
// change a result.
#pragma once

#include <cuda_runtime.h>

namespace ew {

#if defined(__CUDA_ARCH__)
#define EW_DD_ADD(a, b) __fadd_rn((a), (b))
#define EW_DD_SUB(a, b) __fsub_rn((a), (b))
#define EW_DD_MUL(a, b) __fmul_rn((a), (b))
#define EW_DD_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#define EW_DD_ADD(a, b) ((float)((a) + (b)))
#define EW_DD_SUB(a, b) ((float)((a) - (b)))
#define EW_DD_MUL(a, b) ((float)((a) * (b)))
#define EW_DD_FMA(a, b, c) fmaf((a), (b), (c))
#endif

struct dd {
    float hi, lo;
    __host__ __device__ dd() : hi(0.f), lo(0.f) {}
    __host__ __device__ dd(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ dd(float h, float l) : hi(h), lo(l) {}
    // nearest pair to a double (exact when the double has at most 48 significant bits)
    __host__ __device__ explicit dd(double v) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = EW_DD_ADD(a, b);
    const float bb = EW_DD_SUB(s, a);
    e = EW_DD_ADD(EW_DD_SUB(a, EW_DD_SUB(s, bb)), EW_DD_SUB(b, bb));
}
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = EW_DD_ADD(a, b);
    e = EW_DD_SUB(b, EW_DD_SUB(s, a));
}
__host__ __device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = EW_DD_MUL(a, b);
    e = EW_DD_FMA(a, b, -p);
}

// addition: the error of the leading sum, plus the trailing parts, renormalised;
// the error is bounded by a few 2^-48 (|x| + |y|) -- relative to the operands,
// not to the sum, which is what the stencil sums need: their cancelling terms
// are products that already carry errors of that size
__host__ __device__ __forceinline__ dd dd_add(dd x, dd y) {
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    e = EW_DD_ADD(e, EW_DD_ADD(x.lo, y.lo));
    fast_two_sum(s, e, s, e);
    return dd(s, e);
}
__host__ __device__ __forceinline__ dd dd_neg(dd x) { return dd(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ dd dd_mul(dd x, dd y) {
    float p, e;
    two_prod(x.hi, y.hi, p, e);
    e = EW_DD_FMA(x.hi, y.lo, e);
    e = EW_DD_FMA(x.lo, y.hi, e);
    fast_two_sum(p, e, p, e);
    return dd(p, e);
}
// a x + y: the product's error term joins the addition's, one renormalisation
// (15 FP32 operations; error bounded relative to |a x| + |y|)
__host__ __device__ __forceinline__ dd dd_fma(dd a, dd x, dd y) {
    float p, e, s, t;
    two_prod(a.hi, x.hi, p, e);
    e = EW_DD_FMA(a.hi, x.lo, e);
    e = EW_DD_FMA(a.lo, x.hi, e);
    two_sum(p, y.hi, s, t);
    t = EW_DD_ADD(t, EW_DD_ADD(e, y.lo));
    fast_two_sum(s, t, s, t);
    return dd(s, t);
}

__host__ __device__ __forceinline__ dd operator+(dd a, dd b) { return dd_add(a, b); }
__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__host__ __device__ __forceinline__ dd operator*(dd a, dd b) { return dd_mul(a, b); }
__host__ __device__ __forceinline__ dd operator-(dd a) { return dd_neg(a); }
__host__ __device__ __forceinline__ dd& operator+=(dd& a, dd b) {
    a = dd_add(a, b);
    return a;
}

// two values, for the column-pair arithmetic of the blocked 2D kernels
struct __align__(16) dd2 {
    dd x, y;
};

// significant bits of the stored coefficient grid (make_stencil)
template <typename T>
struct MantBits;
template <>
struct MantBits<float> {
    static constexpr int value = 24;
};
template <>
struct MantBits<double> {
    static constexpr int value = 53;
};
template <>
struct MantBits<dd> {
    static constexpr int value = 48;
};

}  // namespace ew
