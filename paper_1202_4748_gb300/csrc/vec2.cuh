// Arithmetic on one lattice site (float, double) or on two sites in lockstep
// (float2, issued as the paired FP32 instructions of sm_100 and later: one
// instruction updates both lanes).  Every operation is rounded once and never
// contracted into a fused multiply-add behind the caller's back, so each lane
// of the paired form gives exactly the bits of the scalar float form; the
// step kernels that run one site per thread and those that run two therefore
// produce identical trajectories.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbf {

template <class V>
struct VT;
template <>
struct VT<float> {
    using S = float;
    static constexpr int W = 1;
};
template <>
struct VT<double> {
    using S = double;
    static constexpr int W = 1;
};
template <>
struct VT<float2> {
    using S = float;
    static constexpr int W = 2;
};

// Paired FP32 operations as inline PTX with explicit rounding.  The code
// generator fuses a paired multiply whose result feeds a paired add into one
// fused multiply-add even when both carry .rn (it never does so for the
// scalar forms), which would round differently from the scalar form.  The
// paired multiply is therefore issued as a fused multiply-add with a zero
// addend that the compiler cannot see is zero (a constant-memory word): it
// rounds exactly like a multiply (a product of exactly -0 comes out as +0,
// which no later operation tells apart), and a fused multiply-add is never
// merged with the add that follows it.
__device__ __forceinline__ unsigned long long f2bits(float2 v) {
    unsigned long long u;
    __builtin_memcpy(&u, &v, 8);
    return u;
}
__device__ __forceinline__ float2 bits2f(unsigned long long u) {
    float2 v;
    __builtin_memcpy(&v, &u, 8);
    return v;
}
static __constant__ unsigned long long vec2_zero = 0ull;   // (+0, +0), opaque to the compiler

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bits2f(d);
}

__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)));
    return bits2f(d);
}

__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)), "l"(vec2_zero));
    return bits2f(d);
}

// a * b + c, rounded once
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)), "l"(f2bits(c)));
    return bits2f(d);
}

// broadcast of a scalar to every lane
template <class V>
__device__ __forceinline__ V vbc(typename VT<V>::S s);
template <>
__device__ __forceinline__ float vbc<float>(float s) { return s; }
template <>
__device__ __forceinline__ double vbc<double>(double s) { return s; }
template <>
__device__ __forceinline__ float2 vbc<float2>(float s) { return make_float2(s, s); }

// compile-time constant in the lane precision
template <class V>
__device__ __forceinline__ V vk(double c) {
    return vbc<V>(typename VT<V>::S(c));
}

// lane access
__device__ __forceinline__ float lane(float v, int) { return v; }
__device__ __forceinline__ double lane(double v, int) { return v; }
__device__ __forceinline__ float lane(float2 v, int k) { return k ? v.y : v.x; }
__device__ __forceinline__ void set_lane(float& v, int, float s) { v = s; }
__device__ __forceinline__ void set_lane(double& v, int, double s) { v = s; }
__device__ __forceinline__ void set_lane(float2& v, int k, float s) {
    if (k) v.y = s;
    else v.x = s;
}

// per-lane application of a scalar function
template <class F>
__device__ __forceinline__ float vmap(float a, F&& f) { return f(a); }
template <class F>
__device__ __forceinline__ double vmap(double a, F&& f) { return f(a); }
template <class F>
__device__ __forceinline__ float2 vmap(float2 a, F&& f) { return make_float2(f(a.x), f(a.y)); }

}  // namespace lbf
