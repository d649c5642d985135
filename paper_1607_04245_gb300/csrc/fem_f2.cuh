// fem_f2.cuh -- packed pairs of float32 values (two cells in one 64-bit register).
//
// sm_100-family GPUs execute add / sub / mul / fma on .f32x2 operands as one
// instruction, so the float32 cell arithmetic of two cells runs at half the issue cost.
// The kernels process cells in pairs: every float32 quantity of the per-cell algebra
// (Jacobian, adjugate, field gradient, quadrature sums, element vector) is an f2 whose
// two lanes belong to two different cells. Every operation rounds to nearest.
//
// The rounded product of a packed multiply is NOT reliably kept as such: bitwise checks
// on sm_103a found the result of mul.rn.f32x2, when consumed by later packed adds, to
// differ from the scalar correctly rounded product in longer dependent sequences (and
// to agree in short ones), as if the multiply had been fused into its consumer. An
// error-free transformation needs the rounded product itself, so TwoProduct takes it
// from mul_rn_exact below: two scalar __fmul_rn, which are never contracted.
#pragma once

#include <stdint.h>

namespace fem {

struct f2 {
    unsigned long long v;
};

__device__ __forceinline__ f2 f2_make(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ f2 f2_splat(float a) { return f2_make(a, a); }

__device__ __forceinline__ float f2_x(f2 a) { return __uint_as_float(static_cast<uint32_t>(a.v)); }

__device__ __forceinline__ float f2_y(f2 a) { return __uint_as_float(static_cast<uint32_t>(a.v >> 32)); }

__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

// the correctly rounded product per lane, for error-free transformations (see above)
__device__ __forceinline__ f2 mul_rn_exact(f2 a, f2 b) {
    return f2_make(__fmul_rn(f2_x(a), f2_x(b)), __fmul_rn(f2_y(a), f2_y(b)));
}

__device__ __forceinline__ f2 operator-(f2 a) {
    // flip both sign bits (exact)
    f2 r;
    r.v = a.v ^ 0x8000000080000000ull;
    return r;
}

__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

}  // namespace fem
