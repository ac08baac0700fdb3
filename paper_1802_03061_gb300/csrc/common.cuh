// Shared device/host utilities of the RTE operator library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "ff.cuh"

#define RTE_MAX_L 64                     // largest angular truncation |k| <= L
#define RTE_MAX_L_DIRECT 8               // largest L of the direct (compile-time) mode mix
#define RTE_MAX_CH (2 * RTE_MAX_L + 1)   // real channels of a J-symmetric field
#define RTE_MAX_STAGES 16

// ----------------------------------------------------------------------------
// complex helpers, templated on the real type (float or double)
// ----------------------------------------------------------------------------
template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using T = float2; };
template <> struct cplx_of<double> { using T = double2; };

// Programmatic dependent launch (PDL).  A kernel launched with launch_pdl may
// start while its predecessor in the stream is still running: it first does
// work that reads nothing the predecessor writes (plan constants, data of
// earlier kernels), then pdl_wait() -- which returns once the predecessor has
// completed and its writes are visible (at once for an ordinary launch) --
// and only then pdl_trigger(), which lets its own successor start.  Since a
// kernel triggers only after its wait, every kernel before the predecessor
// has completed when a successor starts.  Launches into a stream that is
// being captured into a graph stay ordinary: inside the solve graphs the
// programmatic edges measured slower (c2 1.335 against 1.324 ms per solve,
// unpreconditioned 2.130 against 2.083 ms), while back-to-back applications in
// a stream gain (the FP32 K application at 256^2, L = 8: 40.8 -> 35.0 us).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

#ifndef RTE_PDL_ATTR
#define RTE_PDL_ATTR 1
#endif
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = RTE_PDL_ATTR;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    cfg.attrs = at;
    cfg.numAttrs = (RTE_PDL_ATTR && cs == cudaStreamCaptureStatusNone) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

template <typename T> struct real_of;
template <> struct real_of<float2> { using R = float; };
template <> struct real_of<double2> { using R = double; };
template <> struct real_of<ffc> { using R = ff; };

template <typename T> __host__ __device__ __forceinline__ T mk(typename real_of<T>::R x, typename real_of<T>::R y) {
    T r; r.x = x; r.y = y; return r;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ T cconj(T a) { return mk<T>(a.x, -a.y); }
// multiply by DIR * i (DIR = +1 or -1)
template <int DIR, typename T> __device__ __forceinline__ T cmul_i(T a) {
    return DIR > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}
template <typename T> __device__ __forceinline__ T cscale(T a, typename real_of<T>::R s) {
    return mk<T>(a.x * s, a.y * s);
}

// storage conversions between field storage and compute types
template <typename T, typename TF> __device__ __forceinline__ T to_c(TF v) { return v; }
template <> __device__ __forceinline__ ffc to_c<ffc, double2>(double2 v) { return to_ffc(v); }
template <typename TF, typename T> __device__ __forceinline__ TF to_f(T v) { return v; }
template <> __device__ __forceinline__ double2 to_f<double2, ffc>(ffc v) { return to_double2(v); }

// storage conversions for kernel spectra (double2 / float2 / bf16x2 / ffc)
__device__ __forceinline__ ffc ld_spec(const ffc* p, long i, ffc) { return p[i]; }
__device__ __forceinline__ double2 ld_spec(const double2* p, long i, double2) { return p[i]; }
__device__ __forceinline__ float2 ld_spec(const double2* p, long i, float2) {
    double2 v = p[i]; return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ float2 ld_spec(const float2* p, long i, float2) { return p[i]; }
__device__ __forceinline__ double2 ld_spec(const float2* p, long i, double2) {
    float2 v = p[i]; return make_double2(v.x, v.y);
}
__device__ __forceinline__ float2 ld_spec(const __nv_bfloat162* p, long i, float2) {
    return __bfloat1622float2(p[i]);
}
__device__ __forceinline__ double2 ld_spec(const __nv_bfloat162* p, long i, double2) {
    float2 v = __bfloat1622float2(p[i]); return make_double2(v.x, v.y);
}

// ----------------------------------------------------------------------------
// FFT schedule: Q = product of radices in {2,3,4,8}
// ----------------------------------------------------------------------------
struct FftSched {
    int Q;
    int ns;
    int radix[RTE_MAX_STAGES];
};

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on the device (Newton iteration on P_N)
// ---------------------------------------------------------------------------
__device__ inline void gl_node(int N, int i, double* x, double* w) {
    double z = cos(M_PI * (i + 0.75) / (N + 0.5));
    double pp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= N; ++j) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = N * (z * p1 - p2) / (z * z - 1.0);
        double z1 = z;
        z = z1 - p1 / pp;
        if (fabs(z - z1) < 1e-15) break;
    }
    // final derivative at the converged node
    double p1 = 1.0, p2 = 0.0;
    for (int j = 1; j <= N; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
    }
    pp = N * (z * p1 - p2) / (z * z - 1.0);
    *x = z;
    *w = 2.0 / ((1.0 - z * z) * pp * pp);
}

__device__ __forceinline__ double radial_factor(double mu, double R) {
    // int_0^R exp(-mu r) dr
    return mu > 0.0 ? -expm1(-mu * R) / mu : R;
}

// ----------------------------------------------------------------------------
// error plumbing
// ----------------------------------------------------------------------------
#define RTE_CUDA_TRY(expr)                                       \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return rte_cuda_fail(_e, #expr);  \
    } while (0)
