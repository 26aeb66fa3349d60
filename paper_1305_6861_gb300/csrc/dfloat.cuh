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
__device__ __forceinline__ dfl vfma(dfl a, dfl b, dfl c) { return a * b + c; }
__device__ __forceinline__ dfl vmul(dfl a, dfl b) { return a * b; }
__device__ __forceinline__ dfl vadd(dfl a, dfl b) { return a + b; }
__device__ __forceinline__ dfl vsub(dfl a, dfl b) { return a - b; }
__device__ __forceinline__ dfl vneg(dfl a) { return -a; }
__device__ __forceinline__ dfl hsum(dfl a) { return a; }
__device__ __forceinline__ dfl lane_of(dfl a, int) { return a; }
__device__ __forceinline__ void splat(dfl &o, dfl x) { o = x; }
__device__ __forceinline__ void set_lanes(dfl &o, const dfl (&x)[1]) { o = x[0]; }

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
