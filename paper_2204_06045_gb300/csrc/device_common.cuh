// Device helpers shared by the forward kernels (kernels.cu) and the reverse
// sweep (backward.cu): complex types and arithmetic, operand pairs, and the
// parallel bit extract that maps an output index to an operand index.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.hpp"

namespace qt {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename R>
struct CT;
template <>
struct CT<float> {
    using c = float2;
};
template <>
struct CT<double> {
    using c = double2;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <typename C>
struct Pair {
    C v0, v1;
};

// Element layout of every tensor (gate tables, results, cotangents): entries
// 2k and 2k+1 form a pair -- the x = 0 and x = 1 entries of the summed
// variable of the bucket that reads the tensor -- stored planar as
// (Re[2k], Re[2k+1], Im[2k], Im[2k+1]). A pair starts at the byte where an
// interleaved pair would (element 2k of a complex array), so pair addresses
// are plain `base + 2k`; only single entries sit apart within their pair.
// Every tensor starts at an even element offset.
__device__ __forceinline__ Pair<float2> unpack_pair(float4 v) {
    return {make_float2(v.x, v.z), make_float2(v.y, v.w)};
}
__device__ __forceinline__ float4 pack_pair(float2 a, float2 b) { return make_float4(a.x, b.x, a.y, b.y); }
__device__ __forceinline__ Pair<double2> unpack_pair(double2 re, double2 im) {
    return {make_double2(re.x, im.x), make_double2(re.y, im.y)};
}

// Entry e of a tensor whose first element is `base` (read, write, atomic add).
template <typename C>
__device__ __forceinline__ auto elem_scalar(C* base, uint64_t e) {
    using R = decltype(base->x);
    return reinterpret_cast<R*>(base + (e & ~1ull)) + (e & 1u);  // its real part; the imaginary part is 2 further
}
template <typename C>
__device__ __forceinline__ auto elem_scalar(const C* base, uint64_t e) {
    using R = decltype(base->x);
    return reinterpret_cast<const R*>(base + (e & ~1ull)) + (e & 1u);
}
template <typename C>
__device__ __forceinline__ C elem_ld(const C* base, uint64_t e) {
    const auto p = elem_scalar(base, e);
    C v;
    v.x = p[0];
    v.y = p[2];
    return v;
}
template <typename C>
__device__ __forceinline__ C elem_ldg(const C* base, uint64_t e) {  // read-only path
    const auto p = elem_scalar(base, e);
    C v;
    v.x = __ldg(p);
    v.y = __ldg(p + 2);
    return v;
}
template <typename C>
__device__ __forceinline__ C elem_ldcg(const C* base, uint64_t e) {  // at L2 (written by another SM)
    const auto p = elem_scalar(base, e);
    C v;
    v.x = __ldcg(p);
    v.y = __ldcg(p + 2);
    return v;
}
template <typename C>
__device__ __forceinline__ void elem_st(C* base, uint64_t e, C v) {
    const auto p = elem_scalar(base, e);
    p[0] = v.x;
    p[2] = v.y;
}
template <typename C>
__device__ __forceinline__ void elem_atomic_add(C* base, uint64_t e, C v) {
    const auto p = elem_scalar(base, e);
    atomicAdd(p, v.x);
    atomicAdd(p + 2, v.y);
}

// Bits of x selected by m, packed to the low end (parallel bit extract).
__device__ __forceinline__ uint32_t pext_u32(uint32_t x, uint32_t m) {
    uint32_t r = 0, t = x & m;
    while (t) {
        uint32_t low = t & (0u - t);
        r |= 1u << __popc(m & (low - 1u));
        t ^= low;
    }
    return r;
}

// Packed FP32 pairs (f32x2): two floats in one 64-bit register, operated on
// by one instruction (sm_100 and later). A planar complex64 entry pair loads
// as two of them: the real parts (x = 0, 1) and the imaginary parts.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_neg(f32x2 a) { return a ^ 0x8000000080000000ull; }  // both signs, exact
__device__ __forceinline__ float x2_lo(f32x2 a) { return __uint_as_float((uint32_t)a); }
__device__ __forceinline__ float x2_hi(f32x2 a) { return __uint_as_float((uint32_t)(a >> 32)); }
__device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
    return (f32x2)__float_as_uint(lo) | ((f32x2)__float_as_uint(hi) << 32);
}

}  // namespace
}  // namespace qt
