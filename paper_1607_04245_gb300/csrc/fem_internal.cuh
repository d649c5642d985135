// fem_internal.cuh -- shared pieces of libfem's CUDA translation units.
//
// Kernel design (GB300, sm_103a): one thread owns CPT consecutive cells, so every
// cell-indexed array (connectivity rows, coefficient rows, output rows) is read and
// written with coalesced 128-bit accesses; the per-vertex arrays (coordinates, nodal
// values) are gathered through L1/L2. There is no shared memory and no cross-thread
// reduction: for P1 the field gradient is constant on a cell, so the quadrature phase
// and the basis phase of Sec. 3 collapse into register arithmetic per cell.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fem.h"

namespace fem {

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
fem_status fail(fem_status st, const char *fmt, ...);
fem_status check_launch(const char *what);

// ------------------------------------------------------------------ launch parameters

// Quadrature weights travel by value in the kernel parameter block (no constant-memory
// copy, nothing to synchronise, safe under stream capture).
struct QuadW {
    double wd[FEM_MAX_QPTS];
    float wf[FEM_MAX_QPTS];
    int nq;
};

fem_status load_quadrature(int dim, int n_q, const double *qpts, const double *qw, QuadW &out);
fem_status check_common(int dim, int64_t n_cells, int64_t n_verts, const double *coords, const int32_t *conn);
int sm_count();  // multiprocessors of the current device (cached)
float mixed_tau();

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

constexpr int kBlock = 256;

// ------------------------------------------------------------------ device helpers

// Clamp a vertex id into [0, n): malformed input cannot read out of bounds.
__device__ __forceinline__ uint32_t clamp_vid(int32_t v, uint32_t n) {
    return min(static_cast<uint32_t>(v), n - 1u);
}

// Split a float64 value, given as its two 32-bit words, into float32 hi + lo with
// hi = x truncated to 24 significant bits and lo ~ x - hi (the next 23 bits), using
// integer operations only (the float64 pipe of GB300 is narrow). Exactness: hi is
// exact; lo carries the remainder to 2^-47 relative. Inputs with |x| < 2^-126 come out
// as (0 or a float32 subnormal, ~0): an absolute error below 2^-126. Inputs with
// |x| >= 2^128 produce a non-finite hi, which the mixed kernels route to float64.
//
// Returned: hi, and lo_u = lo * 2^23 (unscaled; callers multiply the difference of two
// lo_u values by 2^-23, folding the scale into one multiply per Jacobian entry).
__device__ __forceinline__ void split_f64(uint32_t lo_w, uint32_t hi_w, float &hi, float &lo_u) {
    // clamp the biased exponent into [896, 1151] = float32's [0, 255] after rebiasing
    uint32_t mag = min(max(hi_w & 0x7fffffffu, 0x38000000u), 0x47ffffffu);
    uint32_t hb = __funnelshift_l(lo_w, mag - 0x38000000u, 3); // rebias 1023 -> 127, 52 -> 23 bits
    hb |= hi_w & 0x80000000u;
    hi = __uint_as_float(hb);
    uint32_t base = hb & 0xff800000u;                          // sign and exponent of hi
    float f1 = __uint_as_float(base | ((lo_w >> 6) & 0x007fffffu));
    lo_u = f1 - __uint_as_float(base);                         // (next 23 bits) * ulp(hi) * 2^23
}

// Round a float64 (as words) to float32 with integer ops (the FP32 ablation form):
// nearest rounding of the truncated mantissa (ties away from zero).
__device__ __forceinline__ float round_f64_to_f32(uint32_t lo_w, uint32_t hi_w) {
    uint32_t mag = min(max(hi_w & 0x7fffffffu, 0x38000000u), 0x47efffffu);
    uint32_t hb = __funnelshift_l(lo_w, mag - 0x38000000u, 3);
    hb += (lo_w >> 28) & 1u;  // carry propagates into the exponent
    return __uint_as_float(hb | (hi_w & 0x80000000u));
}

// Error-free transformations (Knuth's TwoSum; TwoProduct via FMA), used for the
// compensated quadrature sum of Ogita, Rump and Oishi's Dot2 algorithm.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);  // never contracted into a later add: p must be the rounded product
    e = fmaf(a, b, -p);
}

// Streaming (read-once / write-once) accesses: keep them out of L1, evict first from L2.
__device__ __forceinline__ int4 ld_stream(const int4 *p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2 *p) { return __ldcs(p); }
__device__ __forceinline__ int ld_stream(const int *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }

template <class T>
__device__ __forceinline__ T ld_gather(const T *p) { return __ldg(p); }

// Grid size: enough CTAs to cover the work, capped at a whole number of waves of the
// device's SMs (the kernels are grid-stride loops).
int grid_for(int64_t n_threads, int block, const void *kernel);
fem_status staged_grid(const void *kernel, int block, size_t smem, int64_t n_tiles, int &grid);

}  // namespace fem
