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
inline bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

constexpr int kBlock = 256;

// ------------------------------------------------------------------ device helpers

// ------------------------------------------------------------------ device error word
//
// One word per device (fem_core.cu) collects error bits from the kernels; launchers pass
// its device address (device_error_word()) as a kernel argument, and fem_device_error()
// reads and clears it. FEM_DEVERR_TIMEOUT: a staged kernel gave up a bounded wait.
// FEM_DEVERR_BADMESH: a kernel met a vertex id outside [0, V) (it was clamped, the
// result is meaningless) or a cell with det J = 0 or a non-finite det J.
enum : unsigned { FEM_DEVERR_TIMEOUT = 1u, FEM_DEVERR_BADMESH = 2u };
unsigned *device_error_word();
// Kernels launched by the calling host thread report into `w` instead (per-request error
// words of the serving launch); nullptr restores the device-wide word.
void set_error_word_override(unsigned *w);

__device__ __forceinline__ void record_device_error(unsigned *err, unsigned bits) {
    // the read first: after the first report, further threads find the bit set and skip
    // the atomic (a badly broken mesh would otherwise send one atomic per cell)
    if ((*reinterpret_cast<volatile unsigned *>(err) & bits) != bits) atomicOr(err, bits);
}

// ------------------------------------------------------------------ overlapped launches
//
// Programmatic dependent launch (sm_90 and later): a kernel launched with programmatic
// stream serialisation may be scheduled onto the SMs while the kernel before it on the
// stream is still draining. pdl_wait() holds the calling thread until that kernel has
// completed and its writes are visible, so a kernel that calls it before touching global
// memory keeps plain stream order for its data; without the launch attribute it returns
// at once. pdl_trigger() allows the next such kernel to be scheduled as this one's CTAs
// exit (it changes nothing about what that kernel sees: it waits in turn).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch k with programmatic stream serialisation, except while `s` is being captured
// into a graph (there the launch is plain, so graph bodies keep full dependencies). The
// kernel must call pdl_wait() before its first global memory access.
template <class... KArgs, class... Args>
cudaError_t launch_overlapped(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    bool plain = cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    if (plain) cudaGetLastError();  // a refused query only selects the plain launch
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = plain ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Clamp a vertex id into [0, n): malformed input cannot read out of bounds.
__device__ __forceinline__ uint32_t clamp_vid(int32_t v, uint32_t n) {
    return min(static_cast<uint32_t>(v), n - 1u);
}

// The same, also folding the id (as unsigned: a negative id counts as too large) into the
// running maximum vmax of the calling thread; vmax >= n at the end means a bad id.
__device__ __forceinline__ uint32_t clamp_vid(int32_t v, uint32_t n, uint32_t &vmax) {
    vmax = max(vmax, static_cast<uint32_t>(v));
    return min(static_cast<uint32_t>(v), n - 1u);
}

// det J = 0 or not finite (checked on the bits: integer operations only)
__device__ __forceinline__ bool det_bad(double d) {
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(d)) & 0x7fffffffu;
    const uint32_t lo = static_cast<uint32_t>(__double2loint(d));
    return (hi | lo) == 0u || hi >= 0x7ff00000u;
}
__device__ __forceinline__ bool det_bad(float d) {
    const uint32_t b = __float_as_uint(d) & 0x7fffffffu;
    return b == 0u || b >= 0x7f800000u;
}

// A cell whose vertex ids repeat (its det J vanishes in exact arithmetic; computed with FMA
// contraction it may come out as a rounding residue instead of an exact zero)
template <int NB>
__device__ __forceinline__ bool ids_repeat(const uint32_t (&v)[NB]) {
    bool r = false;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int j = i + 1; j < NB; ++j) r |= v[i] == v[j];
    return r;
}

// End of a thread's cells: report a bad id (vmax >= n) or a degenerate cell.
__device__ __forceinline__ void report_mesh(unsigned *err, uint32_t vmax, uint32_t n, bool bad_det) {
    if ((vmax >= n || bad_det) && err) record_device_error(err, FEM_DEVERR_BADMESH);
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
// One wave: as many CTAs as are resident on the device at once, at most one per `block`
// threads of work (for grid-stride kernels whose CTAs stay until the work runs out).
int resident_grid(const void *kernel, int block, int64_t n_threads);
fem_status staged_grid(const void *kernel, int block, size_t smem, int64_t n_tiles, int &grid);

}  // namespace fem
