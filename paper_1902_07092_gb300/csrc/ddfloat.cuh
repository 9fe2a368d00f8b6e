// Double-float arithmetic on the FP32 pipe: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
// On GB300 the FP32 pipe issues 64 times the FP64 rate, so FP64-accurate
// transforms whose cost is FP64 issue run faster in this form.
//
// Error-free transformations used (published methods):
//   two-sum (Knuth, TAOCP vol. 2, 4.2.2):   s = a + b,  e = (a - (s - bb)) + (b - bb),
//                                           bb = s - a;  a + b = s + e exactly;
//   fast two-sum (Dekker 1971), |a| >= |b|: s = a + b,  e = b - (s - a);
//   two-product with a fused multiply-add:  p = a b,  e = fma(a, b, -p).
// Sums use one two-sum of the leading parts plus the trailing parts ("sloppy"
// addition): its error is bounded relative to |a| + |b|, which is the bound the
// error analysis of an FFT needs.  Products add the cross terms hi*lo to the
// two-product's error before the final renormalisation.
// Range: that of float (|x| < 3.4e38; below ~1e-38 the trailing part loses bits).
// The primitives use the _rn intrinsics, which the compiler never contracts
// into fused multiply-adds: the transformations rely on each operation being
// rounded on its own.
#pragma once
#include <cuda_runtime.h>

namespace pz {

struct __align__(8) ddf {
    float hi, lo;
};
struct __align__(16) ddc {
    ddf x, y;
};

__device__ __forceinline__ ddf dd_renorm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return ddf{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ddf operator+(ddf a, ddf b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return dd_renorm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ddf operator-(ddf a) { return ddf{-a.hi, -a.lo}; }
__device__ __forceinline__ ddf operator-(ddf a, ddf b) { return a + (-b); }
__device__ __forceinline__ ddf operator*(ddf a, ddf b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return dd_renorm(p, e);
}
// multiplication by an exact power of two (or any float whose products are exact)
__device__ __forceinline__ ddf dd_scale2(ddf a, float s) { return ddf{__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)}; }

__device__ __forceinline__ ddf fmat(ddf a, ddf b, ddf c) { return a * b + c; }

// conversions: the nearest float and the float nearest the remainder
__device__ __forceinline__ ddf dd_from(double v) {
    const float h = __double2float_rn(v);
    return ddf{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double dd_to(ddf a) { return (double)a.hi + (double)a.lo; }

// complex double-float
__device__ __forceinline__ ddc cadd(ddc a, ddc b) { return ddc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ ddc csub(ddc a, ddc b) { return ddc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ ddc cscale(ddc a, ddf s) { return ddc{a.x * s, a.y * s}; }
__device__ __forceinline__ ddc cmul(ddc a, ddc b) { return ddc{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ ddc cfma(ddc w, ddc b, ddc a) { return cadd(a, cmul(w, b)); }  // a + w b
__device__ __forceinline__ ddc creflect(ddc a, ddc s) {                                 // 2a - s
    return ddc{dd_scale2(a.x, 2.f) - s.x, dd_scale2(a.y, 2.f) - s.y};
}
__device__ __forceinline__ ddc dd_from(double2 v) { return ddc{dd_from(v.x), dd_from(v.y)}; }
__device__ __forceinline__ double2 dd_to(ddc a) { return make_double2(dd_to(a.x), dd_to(a.y)); }

}  // namespace pz
