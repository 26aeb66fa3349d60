// dfloat.cuh -- double-float arithmetic on the FP32 pipe: a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// The compensated precision (MRSIM_FP32_KAHAN) runs the forward kernels with this type in place
// of double: every product and sum is formed with error-free transformations (two-sum, and the
// FMA form of two-product), so the rounding error of each step is carried instead of dropped and
// the state does not drift through long sequences.  Sums use the "sloppy" form (one two-sum of the
// leading parts, the trailing parts added, one renormalisation), whose error is a few units of
// 2^-48 of the operands' magnitude; the magnetisation and its coefficients are O(M0), so that is
// an absolute error of ~1e-14 M0 per operation.  GB300 runs float64 at 1/64 of the float32 rate;
// a double-float product costs ~7 float32 operations and a sum ~10.
#pragma once
#include <cuda_runtime.h>

namespace mrsim {
namespace dev {

struct alignas(8) dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // exact split of a double into its leading float and the rounded remainder
    __host__ __device__ dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ dfl(int i) : hi((float)i), lo(0.0f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = a + b;
    return dfl(s, b - (s - a));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return df_fast_two_sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) {
    a = a + b;
    return a;
}

// the element-wise operations the kernels are written in (packed.cuh has the float and double
// versions)
// a·b + c in one step: the product's FMA residual and cross terms join the small part of the
// two-sum with c (15 float32 operations against 17 for a product and a sum)
__device__ __forceinline__ dfl vfma(dfl a, dfl b, dfl c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = p + c.hi;
    const float bb = s - p;
    const float t = (p - (s - bb)) + (c.hi - bb);
    return df_fast_two_sum(s, t + (e + c.lo));
}
__device__ __forceinline__ dfl vmul(dfl a, dfl b) { return a * b; }
__device__ __forceinline__ dfl vadd(dfl a, dfl b) { return a + b; }
__device__ __forceinline__ dfl vsub(dfl a, dfl b) { return a - b; }
__device__ __forceinline__ dfl vneg(dfl a) { return -a; }
__device__ __forceinline__ dfl hsum(dfl a) { return a; }
__device__ __forceinline__ dfl lane_of(dfl a, int) { return a; }
__device__ __forceinline__ void splat(dfl &o, dfl x) { o = x; }
__device__ __forceinline__ void set_lanes(dfl &o, const dfl (&x)[1]) { o = x[0]; }

// a·b + c·d in one step: both products exactly as (leading product, FMA residual plus cross
// terms), one two-sum of the two leading products, the small parts added, one renormalisation.
// 19 float32 operations where a product followed by a multiply-add takes 24; the same error
// bound (a few units of 2^-48 of |a·b| + |c·d|).
__device__ __forceinline__ dfl vdot2(dfl a, dfl b, dfl c, dfl d) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float q = c.hi * d.hi;
    float f = fmaf(c.hi, d.hi, -q);
    f = fmaf(c.hi, d.lo, f);
    f = fmaf(c.lo, d.hi, f);
    const float s = p + q;
    const float bb = s - p;
    const float t = (p - (s - bb)) + (q - bb);
    return df_fast_two_sum(s, t + (e + f));
}

// a·b + c·d + e·f in one step: three exact products, two two-sums, one renormalisation (31
// float32 operations against 41 for three products and two sums)
__device__ __forceinline__ dfl vdot3(dfl a, dfl b, dfl c, dfl d, dfl e, dfl f) {
    const float p1 = a.hi * b.hi;
    float r1 = fmaf(a.hi, b.hi, -p1);
    r1 = fmaf(a.hi, b.lo, r1);
    r1 = fmaf(a.lo, b.hi, r1);
    const float p2 = c.hi * d.hi;
    float r2 = fmaf(c.hi, d.hi, -p2);
    r2 = fmaf(c.hi, d.lo, r2);
    r2 = fmaf(c.lo, d.hi, r2);
    const float p3 = e.hi * f.hi;
    float r3 = fmaf(e.hi, f.hi, -p3);
    r3 = fmaf(e.hi, f.lo, r3);
    r3 = fmaf(e.lo, f.hi, r3);
    const float s1 = p1 + p2;
    const float b1 = s1 - p1;
    const float t1 = (p1 - (s1 - b1)) + (p2 - b1);
    const float s2 = s1 + p3;
    const float b2 = s2 - s1;
    const float t2 = (s1 - (s2 - b2)) + (p3 - b2);
    return df_fast_two_sum(s2, (t1 + t2) + ((r1 + r2) + r3));
}

// warp exchange of a value (float, double or double-float)
__device__ __forceinline__ float shfl_x(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double shfl_x(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ dfl shfl_x(dfl v, int off) {
    return dfl(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}

// value types whose kernels take the float64 program and layouts: double, and double-float
template <typename R>
struct is_wide {
    static constexpr bool value = false;
};
template <>
struct is_wide<double> {
    static constexpr bool value = true;
};
template <>
struct is_wide<dfl> {
    static constexpr bool value = true;
};

}  // namespace dev
}  // namespace mrsim
