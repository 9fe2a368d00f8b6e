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

// The same conversions taken apart on the IEEE 754 fields with integer and FP32
// instructions.  On GB300 a conversion between float and double issues on the
// FP64 unit (2 per clock per SM), which made the conversions of a transform's
// inputs and outputs cost as much as a quarter of its time.
//
// v = (-1)^s 1.f 2^e (52 fraction bits f) splits into h = the first 24
// significant bits (truncated) and the remainder r 2^(e-52), r = the low 29 bits
// of f, rounded to a float; one fast two-sum renormalises (|h| >= |r 2^(e-52)|).
// The pair holds v to 2^-48 relative.  |v| below float's normal range gives a
// signed zero, |v| above it (and inf, NaN) a signed infinity.
__device__ __forceinline__ ddf dd_from_bits(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const unsigned sign = hw & 0x80000000u;
    const int E = (int)((hw >> 20) & 0x7ffu) - 896;  // biased float exponent of 2^e
    if (E <= 0) return ddf{__uint_as_float(sign), 0.f};
    if (E >= 255) return ddf{__uint_as_float(sign | 0x7f800000u), 0.f};
    const float h = __uint_as_float(sign | ((unsigned)E << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    // r = 64 (r >> 6) + (r & 63), both parts exact floats by the 2^23 offset
    const unsigned r = lw & 0x1fffffffu;
    const float r1 = __fsub_rn(__uint_as_float(0x4b000000u | (r >> 6)), 8388608.f);
    const float r0 = __fsub_rn(__uint_as_float(0x4b000000u | (r & 63u)), 8388608.f);
    const float rf = __fmul_rn(__fmaf_rn(r1, 64.f, r0), 2.220446049250313e-16f);  // r 2^-52
    const float l = __fmul_rn(rf, __uint_as_float((unsigned)E << 23));          // times 2^e
    return dd_renorm(h, __uint_as_float(__float_as_uint(l) ^ sign));
}
__device__ __forceinline__ ddc dd_from_bits(double2 v) { return ddc{dd_from_bits(v.x), dd_from_bits(v.y)}; }

// a float as the double of the same value (exact); subnormal floats give zero
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu, sign = b & 0x80000000u;
    const unsigned ed = (e == 0xffu) ? 0x7ffu : e + 896u;
    const unsigned hw = (e == 0u) ? sign : sign | (ed << 20) | ((b & 0x7fffffu) >> 3);
    const unsigned lw = (e == 0u) ? 0u : b << 29;
    return __hiloint2double((int)hw, (int)lw);
}
// the float nearest v (ties away from zero), by an integer rounding of the
// fraction; below float's normal range a signed zero, above it a signed infinity
__device__ __forceinline__ float f32_from_bits(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const unsigned sign = hw & 0x80000000u;
    const int E = (int)((hw >> 20) & 0x7ffu) - 896;
    if (E <= 0) return __uint_as_float(sign);
    if (E >= 255) return __uint_as_float(sign | 0x7f800000u);
    // exponent and leading 23 fraction bits (mod 2^32), plus the rounding bit;
    // a carry out of the fraction steps the exponent, as rounding does
    unsigned t = ((hw << 3) | (lw >> 29)) - (896u << 23);
    t = (t & 0x7fffffffu) + ((lw >> 28) & 1u);
    return __uint_as_float(sign | min(t, 0x7f800000u));
}

// hi + lo rounded to double: one FP64 add
__device__ __forceinline__ double dd_to_bits(ddf a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }
__device__ __forceinline__ double2 dd_to_bits(ddc a) { return make_double2(dd_to_bits(a.x), dd_to_bits(a.y)); }

// hi + lo as a double with integer instructions only.  hi widened to double
// leaves 29 zero fraction bits below its 24; a renormalised lo (|lo| <= ulp(hi)/2,
// exponent at least 24 below hi's) is lo's significand shifted into them
// (truncated past the double's last place), added to the bit pattern when the
// signs agree and subtracted otherwise, at twice the shift when hi is a power of
// two (the difference then lies in the binade below).  Within one unit in the
// last place of the double nearest hi + lo; a subnormal lo counts as zero.
__device__ __forceinline__ double dd_compose(ddf a) {
    const unsigned hb = __float_as_uint(a.hi), lb = __float_as_uint(a.lo);
    const unsigned eh = (hb >> 23) & 0xffu, el = (lb >> 23) & 0xffu;
    if (eh == 0u || eh == 0xffu || el == 0u) return f2d_bits(a.hi);
    const int sh = 29 - (int)(eh - el);
    if (sh > 5) return dd_to_bits(a);  // not a renormalised pair
    const unsigned ml = (lb & 0x7fffffu) | 0x800000u;
    const unsigned L = (sh >= 0) ? (ml << sh) : ((sh > -24) ? (ml >> -sh) : 0u);
    unsigned long long H =
        ((unsigned long long)(((eh + 896u) << 20) | ((hb & 0x7fffffu) >> 3)) << 32) | (unsigned long long)(hb << 29);
    if ((hb ^ lb) & 0x80000000u)
        H -= ((hb & 0x7fffffu) == 0u) ? 2ull * L : (unsigned long long)L;
    else
        H |= L;
    return __longlong_as_double((long long)(H | ((unsigned long long)(hb & 0x80000000u) << 32)));
}
__device__ __forceinline__ double2 dd_compose(ddc a) { return make_double2(dd_compose(a.x), dd_compose(a.y)); }

// a double-float times a float (two-product of the leading parts plus lo b)
__device__ __forceinline__ ddf dd_mulf(ddf a, float b) {
    const float p = __fmul_rn(a.hi, b);
    return dd_renorm(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
// i t a for a complex double-float a and a float t
__device__ __forceinline__ ddc cmul_if(ddc a, float t) { return ddc{-dd_mulf(a.y, t), dd_mulf(a.x, t)}; }

}  // namespace pz
