// fem_pointwise.cu -- element vectors of Eq. 2 for pointwise functions given by the caller
// as CUDA source strings, compiled at run time.
//
// Sec. 5 of the paper builds its kernel source from run-time parameters and hands it to
// the OpenCL just-in-time compiler, with the user's f0 and f1 inlined into it; this file
// does the same with NVRTC for the GPU the call runs on. The generated kernel evaluates
// the bracket of Eq. 2 one cell per thread, the pointwise functions at every quadrature point
// (the user's physics may be nonlinear in u and depend on x; the built-in kernels collapse
// the point loop further, which only a linear f1 allows):
//
//     r_{e,b,k} = sum_q w_q |det J| [ phi_b(xi_q) f0_k(q) + sum_i G_{b,i} f1_{k,i}(q) ]
//
// with, at every quadrature point, u_k(q) = sum_b phi_b(xi_q) u_{b,k} and x(q) =
// sum_b phi_b(xi_q) x_b, and (constant on a P1 cell) grad u_{k,i} = sum_b u_{b,k} G_{b,i},
// G_b = J^{-T} grad_ref phi_b = n_b / det J from the adjugate rows n_b.
//
// NVRTC is opened at run time (dlopen), so the library loads and every other entry point
// works where it is absent; the compiled modules are loaded with the runtime's library
// API (cudaLibraryLoadData) and cached per (device, precision, sizes, sources).
#include <dlfcn.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fem_internal.cuh"

namespace fem {

// ------------------------------------------------------------------ the kernel source
//
// Prepended at generation: FEM_DIM, FEM_NCOMP, FEM_NCOEF, FEM_NQ, FEM_MIXED, FEM_HAS_F0,
// FEM_HAS_F1, the value type T, and the user's functions fem_f0 / fem_f1. The argument
// block PwArgs has the same layout as the host-side struct below.
static const char *kKernelSource = R"FEMSRC(
#define NB (FEM_DIM + 1)
typedef unsigned int u32;
typedef long long i64;

struct PwArgs {
    const double *X0, *X1, *X2;
    const int *conn;
    const void *u;
    const void *coef;
    void *out;
    i64 C;
    u32 V;
    float tau2;
    u32 *err;
    double w[32];
    double phi[32][4];
    float wf[32];       // the same tables rounded to float32 (the mixed form reads these: a
    float phif[32][4];  // float64 -> float32 conversion per point would run on the float64 pipe)
};

#if FEM_MIXED
#define FEM_W(q) a.wf[q]
#define FEM_PHI(q, b) a.phif[q][b]
#else
#define FEM_W(q) a.w[q]
#define FEM_PHI(q, b) a.phi[q][b]
#endif

__device__ __forceinline__ void record_err(u32 *err) {
    if ((*(volatile u32 *)err & 2u) == 0u) atomicOr(err, 2u);
}

// det J = 0 or not finite
__device__ __forceinline__ bool det_bad64(double d) {
    const u32 hi = (u32)__double2hiint(d) & 0x7fffffffu, lo = (u32)__double2loint(d);
    return (hi | lo) == 0u || hi >= 0x7ff00000u;
}

// adjugate rows n[j] (det J times row j of J^{-1}) of the columns e[j], and det J
template <class R>
__device__ __forceinline__ R adjugate(const R (&e)[FEM_DIM][FEM_DIM], R (&n)[FEM_DIM][FEM_DIM]) {
#if FEM_DIM == 2
    n[0][0] = e[1][1]; n[0][1] = -e[1][0];
    n[1][0] = -e[0][1]; n[1][1] = e[0][0];
    return e[0][0] * e[1][1] - e[0][1] * e[1][0];
#else
    for (int j = 0; j < 3; ++j) {
        const R *a = e[(j + 1) % 3], *b = e[(j + 2) % 3];
        n[j][0] = a[1] * b[2] - a[2] * b[1];
        n[j][1] = a[2] * b[0] - a[0] * b[2];
        n[j][2] = a[0] * b[1] - a[1] * b[0];
    }
    return e[0][0] * n[0][0] + e[0][1] * n[0][1] + e[0][2] * n[0][2];
#endif
}

#if FEM_MIXED
// float64 -> float32 (hi, lo * 2^23) with integer operations: hi is x truncated to 24
// significant bits, lo the next 23 bits, so that differences of nearby coordinates come
// out exact to float32 rounding; exponents outside float32's range are clamped (a cell
// with such coordinates fails the shape test and is recomputed in float64)
__device__ __forceinline__ void split64(double x, float &hi, float &lo_u) {
    const u32 lo_w = (u32)__double2loint(x), hi_w = (u32)__double2hiint(x);
    const u32 mag = min(max(hi_w & 0x7fffffffu, 0x38000000u), 0x47ffffffu);
    u32 hb = __funnelshift_l(lo_w, mag - 0x38000000u, 3);
    hb |= hi_w & 0x80000000u;
    hi = __uint_as_float(hb);
    const u32 base = hb & 0xff800000u;
    lo_u = __uint_as_float(base | ((lo_w >> 6) & 0x007fffffu)) - __uint_as_float(base);
}
#endif

extern "C" __global__ void __launch_bounds__(256) fem_pointwise_kernel(const PwArgs a) {
    // launched overlapped with the kernel before it on the stream (outside graph capture):
    // its writes are visible from here on
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const i64 C = a.C;
    const T *u = (const T *)a.u;
    const T *coef = (const T *)a.coef;
    T *out = (T *)a.out;
    const double *X[3] = {a.X0, a.X1, a.X2};
    u32 vmax = 0;
    bool bad = false;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < C; e += (i64)gridDim.x * blockDim.x) {
        u32 v[NB];
        for (int b = 0; b < NB; ++b) {
            const int id = __ldcs(a.conn + b * C + e);
            vmax = max(vmax, (u32)id);
            v[b] = min((u32)id, a.V - 1u);
        }
        double xs[NB][FEM_DIM];
        for (int b = 0; b < NB; ++b)
            for (int i = 0; i < FEM_DIM; ++i) xs[b][i] = X[i][v[b]];
        // geometry: physical basis gradients G[b] and |det J|
        T G[NB][FEM_DIM], adet;
        T x0[FEM_DIM], ec[FEM_DIM][FEM_DIM];  // x_0 and the columns, for x(q)
#if FEM_MIXED
        {
            float hi[NB][FEM_DIM], lo[NB][FEM_DIM];
            for (int b = 0; b < NB; ++b)
                for (int i = 0; i < FEM_DIM; ++i) split64(xs[b][i], hi[b][i], lo[b][i]);
            for (int j = 0; j < FEM_DIM; ++j)
                for (int i = 0; i < FEM_DIM; ++i)
                    ec[j][i] = fmaf(lo[j + 1][i] - lo[0][i], 0x1p-23f, hi[j + 1][i] - hi[0][i]);
            for (int i = 0; i < FEM_DIM; ++i) x0[i] = fmaf(lo[0][i], 0x1p-23f, hi[0][i]);
            float n[FEM_DIM][FEM_DIM];
            const float det = adjugate<float>(ec, n);
            float p = 1.0f;
            for (int j = 0; j < FEM_DIM; ++j) {
                float s = 0.0f;
                for (int i = 0; i < FEM_DIM; ++i) s = fmaf(ec[j][i], ec[j][i], s);
                p *= s;
            }
            const float d2 = det * det;
            if (d2 >= fmaxf(a.tau2 * p, 1.17549435e-38f) && d2 <= 3.40282347e38f) {
                const float y = 1.0f / det;
                for (int j = 0; j < FEM_DIM; ++j)
                    for (int i = 0; i < FEM_DIM; ++i) G[j + 1][i] = n[j][i] * y;
                adet = fabsf(det);
            } else {
                // badly shaped (or out-of-range) cell: the geometry in float64
                double e64[FEM_DIM][FEM_DIM], n64[FEM_DIM][FEM_DIM];
                for (int j = 0; j < FEM_DIM; ++j)
                    for (int i = 0; i < FEM_DIM; ++i) e64[j][i] = xs[j + 1][i] - xs[0][i];
                const double det64 = adjugate<double>(e64, n64);
                bool rep = false;
                for (int b = 0; b < NB; ++b)
                    for (int c = b + 1; c < NB; ++c) rep |= v[b] == v[c];
                bad |= det_bad64(det64) | rep;
                for (int j = 0; j < FEM_DIM; ++j)
                    for (int i = 0; i < FEM_DIM; ++i) G[j + 1][i] = (float)(n64[j][i] / det64);
                adet = (float)fabs(det64);
            }
        }
#else
        {
            double n[FEM_DIM][FEM_DIM];
            for (int j = 0; j < FEM_DIM; ++j)
                for (int i = 0; i < FEM_DIM; ++i) ec[j][i] = xs[j + 1][i] - xs[0][i];
            for (int i = 0; i < FEM_DIM; ++i) x0[i] = xs[0][i];
            const double det = adjugate<double>(ec, n);
            bool rep = false;
            for (int b = 0; b < NB; ++b)
                for (int c = b + 1; c < NB; ++c) rep |= v[b] == v[c];
            bad |= det_bad64(det) | rep;
            const double y = 1.0 / det;
            for (int j = 0; j < FEM_DIM; ++j)
                for (int i = 0; i < FEM_DIM; ++i) G[j + 1][i] = n[j][i] * y;
            adet = fabs(det);
        }
#endif
        for (int i = 0; i < FEM_DIM; ++i) {
            T s = G[1][i];
            for (int j = 2; j <= FEM_DIM; ++j) s += G[j][i];
            G[0][i] = -s;
        }
        // nodal values and the (cell-constant) gradient
        T ub[NB][FEM_NCOMP], gu[FEM_NCOMP * FEM_DIM];
        for (int b = 0; b < NB; ++b)
            for (int k = 0; k < FEM_NCOMP; ++k) ub[b][k] = u[(i64)k * a.V + v[b]];
        for (int k = 0; k < FEM_NCOMP; ++k)
            for (int i = 0; i < FEM_DIM; ++i) {
                T s = ub[0][k] * G[0][i];
                for (int b = 1; b < NB; ++b) s += ub[b][k] * G[b][i];
                gu[k * FEM_DIM + i] = s;
            }
        // For P1 the basis gradients G_b do not depend on the point, so the f1 part of the
        // quadrature sum is G_b . (sum_q w_q f1(q)): the point loop accumulates F1 = sum_q
        // w_q f1(q) and F0_b = sum_q w_q phi_b(q) f0(q), and the basis phase runs once.
        T F1[FEM_NCOMP * FEM_DIM], F0[NB][FEM_NCOMP];
        for (int k = 0; k < FEM_NCOMP * FEM_DIM; ++k) F1[k] = (T)0;
        for (int b = 0; b < NB; ++b)
            for (int k = 0; k < FEM_NCOMP; ++k) F0[b][k] = (T)0;
        for (int q = 0; q < FEM_NQ; ++q) {
            T ph[NB], uq[FEM_NCOMP], xq[FEM_DIM], aq[FEM_NCOEF > 0 ? FEM_NCOEF : 1];
            for (int b = 0; b < NB; ++b) ph[b] = (T)FEM_PHI(q, b);
            for (int k = 0; k < FEM_NCOMP; ++k) {
                T s = ph[0] * ub[0][k];
                for (int b = 1; b < NB; ++b) s += ph[b] * ub[b][k];
                uq[k] = s;
            }
            // x(q) = x_0 + sum_j phi_j(q) (x_j - x_0)
            for (int i = 0; i < FEM_DIM; ++i) {
                T s = x0[i];
                for (int j = 0; j < FEM_DIM; ++j) s += ph[j + 1] * ec[j][i];
                xq[i] = s;
            }
            for (int c = 0; c < FEM_NCOEF; ++c) aq[c] = __ldcs(coef + ((i64)c * FEM_NQ + q) * C + e);
            const T wq = (T)FEM_W(q);
#if FEM_HAS_F0
            T f0[FEM_NCOMP];
            for (int k = 0; k < FEM_NCOMP; ++k) f0[k] = (T)0;
            fem_f0(uq, gu, aq, xq, f0);
            for (int b = 0; b < NB; ++b)
                for (int k = 0; k < FEM_NCOMP; ++k) F0[b][k] += (wq * ph[b]) * f0[k];
#endif
#if FEM_HAS_F1
            T f1[FEM_NCOMP * FEM_DIM];
            for (int k = 0; k < FEM_NCOMP * FEM_DIM; ++k) f1[k] = (T)0;
            fem_f1(uq, gu, aq, xq, f1);
            for (int k = 0; k < FEM_NCOMP * FEM_DIM; ++k) F1[k] += wq * f1[k];
#endif
        }
        // basis phase: r_{b,k} = |det J| (F0_{b,k} + G_b . F1_k)
        for (int b = 0; b < NB; ++b)
            for (int k = 0; k < FEM_NCOMP; ++k) {
                T s = F0[b][k];
                for (int i = 0; i < FEM_DIM; ++i) s += G[b][i] * F1[k * FEM_DIM + i];
                __stcs(out + (i64)(b * FEM_NCOMP + k) * C + e, adet * s);
            }
    }
    if (vmax >= a.V || bad) record_err(a.err);
}
)FEMSRC";

// host mirror of the kernel's argument block
struct PwArgs {
    const double *X0, *X1, *X2;
    const int32_t *conn;
    const void *u;
    const void *coef;
    void *out;
    int64_t C;
    uint32_t V;
    float tau2;
    unsigned *err;
    double w[32];
    double phi[32][4];
    float wf[32];
    float phif[32][4];
};
static_assert(FEM_MAX_QPTS == 32, "the generated argument block holds 32 quadrature points");

// ------------------------------------------------------------------ NVRTC, opened at run time

typedef int nvrtcResult_t;
struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult_t (*create)(void **, const char *, const char *, int, const char *const *, const char *const *);
    nvrtcResult_t (*compile)(void *, int, const char *const *);
    nvrtcResult_t (*log_size)(void *, size_t *);
    nvrtcResult_t (*log)(void *, char *);
    nvrtcResult_t (*cubin_size)(void *, size_t *);
    nvrtcResult_t (*cubin)(void *, char *);
    nvrtcResult_t (*destroy)(void **);
    const char *(*errstr)(nvrtcResult_t);
};

static Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            n.why = "NVRTC (libnvrtc.so) not found";
            return;
        }
        bool all = true;
        auto sym = [&](const char *s) {
            void *p = dlsym(h, s);
            all = all && p;
            return p;
        };
        n.create = reinterpret_cast<decltype(n.create)>(sym("nvrtcCreateProgram"));
        n.compile = reinterpret_cast<decltype(n.compile)>(sym("nvrtcCompileProgram"));
        n.log_size = reinterpret_cast<decltype(n.log_size)>(sym("nvrtcGetProgramLogSize"));
        n.log = reinterpret_cast<decltype(n.log)>(sym("nvrtcGetProgramLog"));
        n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(sym("nvrtcGetCUBINSize"));
        n.cubin = reinterpret_cast<decltype(n.cubin)>(sym("nvrtcGetCUBIN"));
        n.destroy = reinterpret_cast<decltype(n.destroy)>(sym("nvrtcDestroyProgram"));
        n.errstr = reinterpret_cast<decltype(n.errstr)>(sym("nvrtcGetErrorString"));
        if (!all) {
            n.why = "NVRTC lacks an expected entry point";
            return;
        }
        n.ok = true;
    });
    return n;
}

// ------------------------------------------------------------------ module cache

struct PwModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    int grid_per_sm = 1;
};

static std::mutex g_pw_mu;
static std::map<std::string, PwModule> g_pw_cache;

static std::string generate(int dim, int n_comp, int n_coef, int n_q, bool mixed, const char *f0, const char *f1) {
    std::string s;
    char head[512];
    snprintf(head, sizeof(head),
             "#define FEM_DIM %d\n#define FEM_NCOMP %d\n#define FEM_NCOEF %d\n#define FEM_NQ %d\n"
             "#define FEM_MIXED %d\n#define FEM_HAS_F0 %d\n#define FEM_HAS_F1 %d\ntypedef %s T;\n",
             dim, n_comp, n_coef, n_q, mixed ? 1 : 0, f0 ? 1 : 0, f1 ? 1 : 0, mixed ? "float" : "double");
    s += head;
    s += "#define DIM FEM_DIM\n#define NCOMP FEM_NCOMP\n#define NCOEF FEM_NCOEF\n";
    const char *sig = "(const T *__restrict__ u, const T *__restrict__ grad_u, const T *__restrict__ a, "
                      "const T *__restrict__ x, T *__restrict__ ";
    if (f0) {
        s += std::string("__device__ __forceinline__ void fem_f0") + sig + "f0) {\n#line 1 \"f0\"\n";
        s += f0;
        s += "\n}\n";
    }
    if (f1) {
        s += std::string("__device__ __forceinline__ void fem_f1") + sig + "f1) {\n#line 1 \"f1\"\n";
        s += f1;
        s += "\n}\n";
    }
    s += "#line 1 \"fem_pointwise_kernel\"\n";
    s += kKernelSource;
    return s;
}

static fem_status get_module(int dev, int dim, int n_comp, int n_coef, int n_q, bool mixed, const char *f0,
                             const char *f1, PwModule &out) {
    std::string key = std::to_string(dev) + "|" + std::to_string(dim) + "|" + std::to_string(n_comp) + "|" +
                      std::to_string(n_coef) + "|" + std::to_string(n_q) + "|" + (mixed ? "m" : "d") + "|" +
                      (f0 ? "1" : "0") + (f1 ? "1" : "0") + "|" + std::to_string(f0 ? strlen(f0) : 0) + "|" +
                      (f0 ? f0 : "") + "|" + (f1 ? f1 : "");
    std::lock_guard<std::mutex> lk(g_pw_mu);
    auto it = g_pw_cache.find(key);
    if (it != g_pw_cache.end()) {
        out = it->second;
        return FEM_OK;
    }
    Nvrtc &nv = nvrtc();
    if (!nv.ok) return fail(FEM_ERR_UNSUPPORTED, "fem_integrate_pointwise: %s", nv.why.c_str());
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(FEM_ERR_CUDA, "fem_integrate_pointwise: cannot query the device");
    }
    const std::string src = generate(dim, n_comp, n_coef, n_q, mixed, f0, f1);
    void *prog = nullptr;
    nvrtcResult_t r = nv.create(&prog, src.c_str(), "fem_pointwise.cu", 0, nullptr, nullptr);
    if (r != 0) return fail(FEM_ERR_CUDA, "nvrtcCreateProgram: %s", nv.errstr(r));
    char arch[64];
    snprintf(arch, sizeof(arch), "--gpu-architecture=sm_%d%d", major, minor);
    const char *opts[] = {arch, "-std=c++17", "--fmad=true"};
    r = nv.compile(prog, 3, opts);
    if (r != 0) {
        size_t n = 0;
        nv.log_size(prog, &n);
        std::vector<char> log(n + 1, '\0');
        if (n) nv.log(prog, log.data());
        nv.destroy(&prog);
        return fail(FEM_ERR_ARG, "fem_integrate_pointwise: the physics source does not compile (%s):\n%.400s",
                    nv.errstr(r), log.data());
    }
    size_t nbin = 0;
    nv.cubin_size(prog, &nbin);
    std::vector<char> bin(nbin);
    if (nbin) nv.cubin(prog, bin.data());
    nv.destroy(&prog);
    PwModule m;
    cudaError_t e = cudaLibraryLoadData(&m.lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&m.kernel, m.lib, "fem_pointwise_kernel");
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m.grid_per_sm, reinterpret_cast<const void *>(m.kernel),
                                                          256, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (m.lib) cudaLibraryUnload(m.lib);
        return fail(FEM_ERR_CUDA, "fem_integrate_pointwise: loading the compiled kernel: %s", cudaGetErrorString(e));
    }
    if (m.grid_per_sm < 1) m.grid_per_sm = 1;
    g_pw_cache.emplace(key, m);
    out = m;
    return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" fem_status fem_integrate_pointwise(const char *f0_src, const char *f1_src, int dim, int n_comp,
                                              int n_coef, int64_t n_cells, int64_t n_verts, const double *coords,
                                              const int32_t *conn, const void *u, const void *coef, int n_q,
                                              const double *qpts, const double *qw, void *elem_out,
                                              fem_precision prec, fem_stream stream) {
    fem_status st = check_common(dim, n_cells, n_verts, coords, conn);
    if (st != FEM_OK) return st;
    if (prec != FEM_FP64 && prec != FEM_FP32_MIXED)
        return fail(FEM_ERR_ARG, "fem_integrate_pointwise: precision %d (FEM_FP64 or FEM_FP32_MIXED)", int(prec));
    if (n_comp < 1 || n_comp > 3) return fail(FEM_ERR_ARG, "n_comp = %d outside [1, 3]", n_comp);
    if (n_coef < 0 || n_coef > FEM_POINTWISE_MAX_COEF)
        return fail(FEM_ERR_ARG, "n_coef = %d outside [0, %d]", n_coef, FEM_POINTWISE_MAX_COEF);
    if (!f0_src && !f1_src) return fail(FEM_ERR_ARG, "neither f0 nor f1 given");
    if (int64_t(n_comp) * n_verts >= (int64_t(1) << 31) || int64_t(n_coef) * n_q * n_cells >= (int64_t(1) << 40))
        return fail(FEM_ERR_SHAPE, "too many values");
    QuadW w;
    if ((st = load_quadrature(dim, n_q, qpts, qw, w)) != FEM_OK) return st;
    if (!qpts) return fail(FEM_ERR_ARG, "qpts is required: u(x_q), x_q and the f0 term use phi_b(xi_q)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(FEM_ERR_CUDA, "cudaGetDevice failed");
    PwModule m;
    if ((st = get_module(dev, dim, n_comp, n_coef, n_q, prec == FEM_FP32_MIXED, f0_src, f1_src, m)) != FEM_OK)
        return st;
    if (n_cells == 0) return FEM_OK;  // compiled and cached, nothing to integrate
    if (!u || !elem_out || (n_coef > 0 && !coef)) return fail(FEM_ERR_ARG, "u, coef or elem_out is NULL");
    PwArgs a;
    a.X0 = coords;
    a.X1 = coords + (dim > 1 ? n_verts : 0);
    a.X2 = coords + (dim > 2 ? 2 * n_verts : 0);
    a.conn = conn;
    a.u = u;
    a.coef = coef;
    a.out = elem_out;
    a.C = n_cells;
    a.V = static_cast<uint32_t>(n_verts);
    const float tau = mixed_tau();
    a.tau2 = tau * tau;
    if (!(a.err = device_error_word())) return fail(FEM_ERR_CUDA, "device error word unavailable");
    for (int q = 0; q < 32; ++q) {
        a.w[q] = q < n_q ? qw[q] : 0.0;
        for (int b = 0; b < 4; ++b) a.phi[q][b] = 0.0;
        if (q < n_q) {
            double s = 0.0;
            for (int k = 0; k < dim; ++k) s += qpts[q * dim + k];
            a.phi[q][0] = 1.0 - s;
            for (int b = 1; b <= dim; ++b) a.phi[q][b] = qpts[q * dim + b - 1];
        }
        a.wf[q] = static_cast<float>(a.w[q]);
        for (int b = 0; b < 4; ++b) a.phif[q][b] = static_cast<float>(a.phi[q][b]);
    }
    const int64_t need = (n_cells + 255) / 256, cap = int64_t(m.grid_per_sm) * sm_count();
    const unsigned grid = static_cast<unsigned>(need < cap ? need : cap);
    void *params[] = {&a};
    // overlapped with the previous kernel's tail, as the built-in kernels are (the kernel
    // waits for it first), except while the stream is being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool refused = cudaStreamIsCapturing(stream, &cs) != cudaSuccess;
    if (refused) cudaGetLastError();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    cfg.attrs = at;
    cfg.numAttrs = (refused || cs != cudaStreamCaptureStatusNone) ? 0 : 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, reinterpret_cast<const void *>(m.kernel), params);
    if (e != cudaSuccess) return fail(FEM_ERR_CUDA, "fem_integrate_pointwise launch: %s", cudaGetErrorString(e));
    return FEM_OK;
}
