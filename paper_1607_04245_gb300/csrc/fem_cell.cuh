// fem_cell.cuh -- per-cell device arithmetic shared by the integration kernels.
//
// Geometry of a P1 simplex (reference vertices 0, e_1, ..., e_d):
//   columns of the Jacobian   e_j = x_j - x_0                  (j = 1..d)
//   adjugate rows             n_j = det(J) * (row j of J^{-1})
//       2D: n_1 = (e_2y, -e_2x), n_2 = (-e_1y, e_1x)
//       3D: n_1 = e_2 x e_3, n_2 = e_3 x e_1, n_3 = e_1 x e_2
//   determinant               det J = e_1 . n_1
// so the physical basis gradients are G_j = J^{-T} grad_ref phi_j = n_j / det J for
// j >= 1 and G_0 = -(G_1 + ... + G_d). All kernels work with n_j and det J and divide
// once per cell.
#pragma once

#include <cfloat>
#include <type_traits>

#include "fem_f2.cuh"
#include "fem_internal.cuh"

namespace fem {

template <int P>
using val_t = typename std::conditional<P == FEM_FP64, double, float>::type;

// ------------------------------------------------------------------ row access (cell-indexed arrays)

template <int CPT>
__device__ __forceinline__ void load_row(const int32_t *p, int32_t (&v)[CPT]) {
    if constexpr (CPT == 4) {
        int4 t = ld_stream(reinterpret_cast<const int4 *>(p));
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else if constexpr (CPT == 2) {
        int2 t = __ldcs(reinterpret_cast<const int2 *>(p));
        v[0] = t.x, v[1] = t.y;
    } else {
#pragma unroll
        for (int i = 0; i < CPT; ++i) v[i] = ld_stream(p + i);
    }
}

template <int CPT>
__device__ __forceinline__ void load_row(const float *p, float (&v)[CPT]) {
    if constexpr (CPT == 4) {
        float4 t = ld_stream(reinterpret_cast<const float4 *>(p));
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else if constexpr (CPT == 2) {
        float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
        v[0] = t.x, v[1] = t.y;
    } else {
#pragma unroll
        for (int i = 0; i < CPT; ++i) v[i] = ld_stream(p + i);
    }
}

template <int CPT>
__device__ __forceinline__ void load_row(const double *p, double (&v)[CPT]) {
    if constexpr (CPT == 4) {
        double2 a = ld_stream(reinterpret_cast<const double2 *>(p));
        double2 b = ld_stream(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    } else if constexpr (CPT == 2) {
        double2 a = ld_stream(reinterpret_cast<const double2 *>(p));
        v[0] = a.x, v[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < CPT; ++i) v[i] = ld_stream(p + i);
    }
}

template <int CPT>
__device__ __forceinline__ void store_row(float *p, const float (&v)[CPT]) {
    if constexpr (CPT == 4) {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
    } else if constexpr (CPT == 2) {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
    } else {
#pragma unroll
        for (int i = 0; i < CPT; ++i) __stcs(p + i, v[i]);
    }
}

template <int CPT>
__device__ __forceinline__ void store_row(double *p, const double (&v)[CPT]) {
    if constexpr (CPT == 4) {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
        __stcs(reinterpret_cast<double2 *>(p) + 1, make_double2(v[2], v[3]));
    } else if constexpr (CPT == 2) {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    } else {
#pragma unroll
        for (int i = 0; i < CPT; ++i) __stcs(p + i, v[i]);
    }
}

// ------------------------------------------------------------------ generic arithmetic
// The cell algebra below is written once for double, float and f2 (two cells per value).

// (both overloads are declared here: an unqualified fma() inside namespace fem must never
// resolve a double call to the float version)
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }

// a*b - c*d
__device__ __forceinline__ double diffprod(double a, double b, double c, double d) { return fma(a, b, -(c * d)); }
__device__ __forceinline__ float diffprod(float a, float b, float c, float d) { return fmaf(a, b, -(c * d)); }
__device__ __forceinline__ f2 diffprod(f2 a, f2 b, f2 c, f2 d) { return a * b - c * d; }

// num / |den| in float64. The IEEE division is about a dozen float64 instructions and the
// float64 forms are bound by the float64 pipe, so: |den| = m 2^e with m in [1, 2) (integer
// operations on the exponent field); a float32 reciprocal of m, truncated to 23 bits, as the
// seed (relative error below 2^-22); two Newton-Raphson steps y <- y + y (1 - m y) in
// float64, each squaring the relative error, so the second ends at the float64 rounding
// level; the exponent put back and one product -- five float64 instructions, a result
// within about two units in the last place of the correctly rounded quotient. |den|
// outside [2^-1000, 2^1001) (zero, subnormal, infinite, NaN or extreme) takes the IEEE
// division.
__device__ __forceinline__ double quot_abs(double num, double den) {
    const uint32_t hw = static_cast<uint32_t>(__double2hiint(den)) & 0x7fffffffu;
    const uint32_t lw = static_cast<uint32_t>(__double2loint(den));
    const int ef = static_cast<int>(hw >> 20);  // biased exponent of |den|
    if (ef < 23 || ef > 2023) return num / fabs(den);
    const double m = __hiloint2double(static_cast<int>((hw & 0x000fffffu) | 0x3ff00000u), static_cast<int>(lw));
    const float yf = __frcp_rn(__uint_as_float(0x3f800000u | ((hw & 0x000fffffu) << 3) | (lw >> 29)));
    // yf in [0.5, 1]: widen it to float64 exactly with integer operations
    const uint32_t fb = __float_as_uint(yf);
    double y = __hiloint2double(static_cast<int>(((((fb >> 23) & 0xffu) + 896u) << 20) | ((fb & 0x7fffffu) >> 3)),
                                static_cast<int>(fb << 29));
    y = fma(y, fma(-m, y, 1.0), y);
    y = fma(y, fma(-m, y, 1.0), y);
    // 1 / |den| = y 2^-(ef - 1023): y's exponent field stays inside [22, 2023]
    const uint32_t yh = static_cast<uint32_t>(__double2hiint(y)) - (static_cast<uint32_t>(ef - 1023) << 20);
    return num * __hiloint2double(static_cast<int>(yh), __double2loint(y));
}
// float32: the fast reciprocal (the mixed form's tolerance is far above its error)
__device__ __forceinline__ float quot_abs(float num, float den) { return __fdividef(num, fabsf(den)); }
__device__ __forceinline__ f2 quot_abs(f2 num, f2 den) {
    return f2_make(__fdividef(f2_x(num), fabsf(f2_x(den))), __fdividef(f2_y(num), fabsf(f2_y(den))));
}

__device__ __forceinline__ double neg(double x) { return -x; }
__device__ __forceinline__ float neg(float x) { return -x; }
__device__ __forceinline__ f2 neg(f2 x) { return f2{0ull} - x; }

template <class T> __device__ __forceinline__ T zero();
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ float zero<float>() { return 0.0f; }
template <> __device__ __forceinline__ f2 zero<f2>() { return f2{0ull}; }

// ------------------------------------------------------------------ geometry

template <int DIM, class T>
__device__ __forceinline__ T adjugate_rows(const T (&e)[DIM][DIM], T (&n)[DIM][DIM]) {
    if constexpr (DIM == 2) {
        n[0][0] = e[1][1], n[0][1] = -e[1][0];
        n[1][0] = -e[0][1], n[1][1] = e[0][0];
        return diffprod(e[0][0], e[1][1], e[0][1], e[1][0]);
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T *a = e[(j + 1) % 3], *b = e[(j + 2) % 3];
            n[j][0] = diffprod(a[1], b[2], a[2], b[1]);
            n[j][1] = diffprod(a[2], b[0], a[0], b[2]);
            n[j][2] = diffprod(a[0], b[1], a[1], b[0]);
        }
        return fma(e[0][2], n[0][2], fma(e[0][1], n[0][1], e[0][0] * n[0][0]));
    }
}

template <int DIM, class T>
__device__ __forceinline__ T dotv(const T *a, const T *b) {
    T s = a[0] * b[0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) s = fma(a[i], b[i], s);
    return s;
}

// Gather the float64 coordinates of a cell's vertices: x[b][k] = X[k][v[b]].
template <int DIM>
__device__ __forceinline__ void gather_coords(const double *const (&X)[DIM], const uint32_t (&v)[DIM + 1],
                                              double (&x)[DIM + 1][DIM]) {
#pragma unroll
    for (int b = 0; b <= DIM; ++b)
#pragma unroll
        for (int k = 0; k < DIM; ++k) x[b][k] = ld_gather(X[k] + v[b]);
}

// Float64 Jacobian columns e_j = x_j - x_0.
template <int DIM>
__device__ __forceinline__ void columns_f64(const double (&x)[DIM + 1][DIM], double (&e)[DIM][DIM]) {
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int k = 0; k < DIM; ++k) e[j][k] = x[j + 1][k] - x[0][k];
}

// Float32 Jacobian columns from float64 coordinates split into (hi, lo) pairs:
// e_jk = (hi_jk - hi_0k) + (lo_jk - lo_0k); exact up to float32 rounding of the result.
template <int DIM>
__device__ __forceinline__ void columns_mixed(const double (&x)[DIM + 1][DIM], float (&e)[DIM][DIM]) {
    float hi[DIM + 1][DIM], lo[DIM + 1][DIM];
#pragma unroll
    for (int b = 0; b <= DIM; ++b)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
            split_f64(static_cast<uint32_t>(__double2loint(x[b][k])), static_cast<uint32_t>(__double2hiint(x[b][k])),
                      hi[b][k], lo[b][k]);
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int k = 0; k < DIM; ++k) e[j][k] = fmaf(lo[j + 1][k] - lo[0][k], 0x1p-23f, hi[j + 1][k] - hi[0][k]);
}

// The same for two cells at once (lane x: cell xa, lane y: cell xb).
template <int DIM>
__device__ __forceinline__ void columns_mixed2(const double (&xa)[DIM + 1][DIM], const double (&xb)[DIM + 1][DIM],
                                               f2 (&e)[DIM][DIM]) {
    f2 hi[DIM + 1][DIM], lo[DIM + 1][DIM];
#pragma unroll
    for (int b = 0; b <= DIM; ++b)
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            float ha, la, hb, lb;
            split_f64(static_cast<uint32_t>(__double2loint(xa[b][k])), static_cast<uint32_t>(__double2hiint(xa[b][k])),
                      ha, la);
            split_f64(static_cast<uint32_t>(__double2loint(xb[b][k])), static_cast<uint32_t>(__double2hiint(xb[b][k])),
                      hb, lb);
            hi[b][k] = f2_make(ha, hb);
            lo[b][k] = f2_make(la, lb);
        }
    const f2 scale = f2_splat(0x1p-23f);
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int k = 0; k < DIM; ++k) e[j][k] = fma(lo[j + 1][k] - lo[0][k], scale, hi[j + 1][k] - hi[0][k]);
}

// Float32 Jacobian columns from coordinates rounded to float32 (FP32 ablation).
template <int DIM>
__device__ __forceinline__ void columns_f32(const double (&x)[DIM + 1][DIM], float (&e)[DIM][DIM]) {
    float xf[DIM + 1][DIM];
#pragma unroll
    for (int b = 0; b <= DIM; ++b)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
            xf[b][k] = round_f64_to_f32(static_cast<uint32_t>(__double2loint(x[b][k])),
                                        static_cast<uint32_t>(__double2hiint(x[b][k])));
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int k = 0; k < DIM; ++k) e[j][k] = xf[j + 1][k] - xf[0][k];
}

// The same for two cells at once.
template <int DIM>
__device__ __forceinline__ void columns_f32_2(const double (&xa)[DIM + 1][DIM], const double (&xb)[DIM + 1][DIM],
                                              f2 (&e)[DIM][DIM]) {
    f2 xf[DIM + 1][DIM];
#pragma unroll
    for (int b = 0; b <= DIM; ++b)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
            xf[b][k] = f2_make(round_f64_to_f32(static_cast<uint32_t>(__double2loint(xa[b][k])),
                                                static_cast<uint32_t>(__double2hiint(xa[b][k]))),
                               round_f64_to_f32(static_cast<uint32_t>(__double2loint(xb[b][k])),
                                                static_cast<uint32_t>(__double2hiint(xb[b][k]))));
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int k = 0; k < DIM; ++k) e[j][k] = xf[j + 1][k] - xf[0][k];
}

// Shape test of the mixed form: det^2 >= tau^2 prod_j |e_j|^2 (Hadamard ratio >= tau),
// with det^2 inside float32's normal range; failing cells take the float64 path.
template <int DIM>
__device__ __forceinline__ bool shape_ok(const float (&e)[DIM][DIM], float det, float tau2) {
    float p = dotv<DIM>(e[0], e[0]);
#pragma unroll
    for (int j = 1; j < DIM; ++j) p *= dotv<DIM>(e[j], e[j]);
    float d2 = det * det;
    return d2 >= fmaxf(tau2 * p, FLT_MIN) && d2 <= FLT_MAX;
}

// The shape test for two cells: (ok of lane x, ok of lane y).
template <int DIM>
__device__ __forceinline__ void shape_ok2(const f2 (&e)[DIM][DIM], f2 det, float tau2, bool &oka, bool &okb) {
    f2 p = dotv<DIM>(e[0], e[0]);
#pragma unroll
    for (int j = 1; j < DIM; ++j) p = p * dotv<DIM>(e[j], e[j]);
    const f2 d2 = det * det;
    const f2 lim = p * f2_splat(tau2);
    const float da = f2_x(d2), db = f2_y(d2);
    oka = da >= fmaxf(f2_x(lim), FLT_MIN) && da <= FLT_MAX;
    okb = db >= fmaxf(f2_y(lim), FLT_MIN) && db <= FLT_MAX;
}

// ------------------------------------------------------------------ quadrature sums

// sum_q w_q c_q, plain (FMA chain) -- float64 form and float32 ablation
template <class T>
struct PlainSum {
    T s;
    __device__ __forceinline__ void first(T w, T c) { s = w * c; }
    __device__ __forceinline__ void add(T w, T c) { s = fma(w, c, s); }
    __device__ __forceinline__ T value() const { return s; }
    __device__ __forceinline__ double value_f64() const { return static_cast<double>(s); }
};

// sum_q w_q c_q compensated: Dot2 (Ogita, Rump, Oishi 2005) with TwoProduct and TwoSum;
// the result is as accurate as if computed in twice the working precision.
struct Dot2Sum {
    float s, c;
    __device__ __forceinline__ void first(float w, float x) { two_prod(w, x, s, c); }
    __device__ __forceinline__ void add(float w, float x) {
        float p, pe, se;
        two_prod(w, x, p, pe);
        two_sum(s, p, s, se);
        c += pe + se;
    }
    __device__ __forceinline__ float value() const { return s + c; }
    __device__ __forceinline__ double value_f64() const { return static_cast<double>(s) + static_cast<double>(c); }
};

// Dot2 for two cells at once. The compensation is kept negated (m = -c): TwoProduct's
// error term then comes out of one FMA, m_p = fma(-w, x, p) = p - w x exactly, with p
// the correctly rounded product (mul_rn_exact), and no negation is needed anywhere.
struct Dot2Sum2 {
    f2 s, m;
    __device__ __forceinline__ void first(float w, f2 x) {
        s = mul_rn_exact(f2_splat(w), x);
        m = fma(f2_splat(-w), x, s);
    }
    __device__ __forceinline__ void add(float w, f2 x) {
        const f2 p = mul_rn_exact(f2_splat(w), x);
        const f2 mp = fma(f2_splat(-w), x, p);
        const f2 t = s + p;
        const f2 bb = t - s;
        const f2 se = (s - (t - bb)) + (p - bb);
        s = t;
        m = m + (mp - se);
    }
    __device__ __forceinline__ f2 value() const { return s - m; }
    __device__ __forceinline__ double value_f64_x() const { return double(f2_x(s)) - double(f2_x(m)); }
    __device__ __forceinline__ double value_f64_y() const { return double(f2_y(s)) - double(f2_y(m)); }
};

// sum_q w_q c_q in plain f32x2 (FP32 ablation)
struct PlainSum2 {
    f2 s;
    __device__ __forceinline__ void first(float w, f2 x) { s = f2_splat(w) * x; }
    __device__ __forceinline__ void add(float w, f2 x) { s = fma(f2_splat(w), x, s); }
    __device__ __forceinline__ f2 value() const { return s; }
    __device__ __forceinline__ double value_f64_x() const { return double(f2_x(s)); }
    __device__ __forceinline__ double value_f64_y() const { return double(f2_y(s)); }
};

// fixed-order sum of a vertex's list entries (the nodal gather E^T): plain in float64,
// compensated (TwoSum) in float32
template <class T>
struct NodeSum {
    T s = T(0);
    __device__ __forceinline__ void add(T x) { s += x; }
    __device__ __forceinline__ T value() const { return s; }
};

template <>
struct NodeSum<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        float t, e;
        two_sum(s, x, t, e);
        s = t;
        c += e;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

// list entries whose loads a gather keeps in flight at once
constexpr int kGatherBatch = 8;

template <int P>
using qsum_t = typename std::conditional<P == FEM_FP64, PlainSum<double>,
                                         typename std::conditional<P == FEM_FP32_MIXED, Dot2Sum, PlainSum<float>>::type>::type;

}  // namespace fem
