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

}  // namespace
}  // namespace qt
