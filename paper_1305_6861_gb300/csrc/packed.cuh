// packed.cuh -- float32 pairs in 64-bit registers (f32x2 arithmetic) and the matching scalar
// overloads, shared by the forward and the K-t kernels.
#pragma once
#include <cuda_runtime.h>

namespace mrsim {
namespace dev {

// ---- packed float32 pairs -------------------------------------------------------------------
// sm_100-class SMs execute two float32 lanes per instruction (fma/mul/add/sub .rn.f32x2 on a
// 64-bit register pair).  A thread with K >= 2 float32 spins keeps each quantity as K/2 pairs,
// which halves the instructions issued for rotations, relaxations and spin sums; every lane is
// rounded exactly like the scalar operation.
struct f2 {
    unsigned long long r;
};
__device__ __forceinline__ f2 pk2(float a, float b) {
    f2 o;
    asm("mov.b64 %0, {%1, %2};" : "=l"(o.r) : "f"(a), "f"(b));
    return o;
}
__device__ __forceinline__ void unpk2(f2 a, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.r));
}
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}
__device__ __forceinline__ f2 vmul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ f2 vadd(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ f2 vsub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
// sign flip of both lanes on the integer pipe (the FMA pipe is the bound)
__device__ __forceinline__ f2 vneg(f2 a) {
    f2 o;
    asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(o.r) : "l"(a.r));
    return o;
}
__device__ __forceinline__ float hsum(f2 a) {
    float x, y;
    unpk2(a, x, y);
    return x + y;
}
__device__ __forceinline__ float lane_of(f2 a, int h) {
    float x, y;
    unpk2(a, x, y);
    return h ? y : x;
}
__device__ __forceinline__ void splat(f2 &o, float x) { o = pk2(x, x); }
__device__ __forceinline__ void set_lanes(f2 &o, const float (&x)[2]) { o = pk2(x[0], x[1]); }

// a·b + c·d with c·d formed first (the rounding order of every rotation in the kernels)
__device__ __forceinline__ f2 vdot2(f2 a, f2 b, f2 c, f2 d) { return vfma(a, b, vmul(c, d)); }

// the same operations on one scalar lane (float64, and float32 with one spin per thread)
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
template <typename T>
__device__ __forceinline__ T vmul(T a, T b) { return a * b; }
template <typename T>
__device__ __forceinline__ T vadd(T a, T b) { return a + b; }
template <typename T>
__device__ __forceinline__ T vsub(T a, T b) { return a - b; }
template <typename T>
__device__ __forceinline__ T vneg(T a) { return -a; }
template <typename T>
__device__ __forceinline__ T hsum(T a) { return a; }
template <typename T>
__device__ __forceinline__ T lane_of(T a, int) { return a; }
template <typename T>
__device__ __forceinline__ void splat(T &o, T x) { o = x; }
template <typename T>
__device__ __forceinline__ void set_lanes(T &o, const T (&x)[1]) { o = x[0]; }
__device__ __forceinline__ float vdot2(float a, float b, float c, float d) { return vfma(a, b, vmul(c, d)); }
__device__ __forceinline__ double vdot2(double a, double b, double c, double d) { return vfma(a, b, vmul(c, d)); }

}  // namespace dev
}  // namespace mrsim
