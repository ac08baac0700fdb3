// The spherical-harmonic (anisotropic 3D) operator's handle and what its two
// translation units share: aniso3d.cu (spectra, general-Q Stockham passes,
// solve, C ABI) and aniso3d_warp.cu (the warp-register FFT passes for
// Q = 64, 128, 256, all M channels of a pass in one launch).
#pragma once
#include "ff.cuh"
#include "internal.h"

#define RTE_ANISO_MAX_L 4
#define RTE_ANISO_MAX_M ((RTE_ANISO_MAX_L + 1) * (RTE_ANISO_MAX_L + 1))

// degree l of channel a = l^2 + l + m
__host__ __device__ constexpr int chan_l(int a) {
    int l = 0;
    while ((l + 1) * (l + 1) <= a) ++l;
    return l;
}

// parities of Y_{l,m} under x -> -x, y -> -y, z -> -z (+1 even, -1 odd)
__host__ __device__ constexpr int sh_px(int a) {
    const int l = chan_l(a), m = a - l * l - l, am = m < 0 ? -m : m;
    const int sm = (am & 1) ? -1 : 1;
    return m >= 0 ? sm : -sm;
}
__host__ __device__ constexpr int sh_py(int a) {
    const int l = chan_l(a), m = a - l * l - l;
    return m >= 0 ? 1 : -1;
}
__host__ __device__ constexpr int sh_pz(int a) {
    const int l = chan_l(a), m = a - l * l - l, am = m < 0 ? -m : m;
    return ((l + am) & 1) ? -1 : 1;
}

// Channel pairs: the unordered pairs a <= b numbered row by row; W_ab = W_ba,
// so (a, b) and (b, a) share one spectrum.  pair_info = pair index |
// imaginary spectrum << 16 | odd in y << 17 | odd in z << 18 (W_ab has the
// product parities of Y_a and Y_b; odd total parity: imaginary spectrum).
__host__ __device__ constexpr int pair_index(int a, int b, int M) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo * M - lo * (lo - 1) / 2 + (hi - lo);
}
__host__ __device__ constexpr int pair_info(int a, int b, int M) {
    const int px = sh_px(a) * sh_px(b), py = sh_py(a) * sh_py(b), pz = sh_pz(a) * sh_pz(b);
    const int imag = (px * py * pz) < 0 ? 1 : 0;
    return pair_index(a, b, M) | (imag << 16) | ((py < 0) << 17) | ((pz < 0) << 18);
}
// the channels (a <= b) of pair P
__host__ __device__ constexpr int pair_first(int P, int M) {
    int a = 0;
    while (P >= M - a) {
        P -= M - a;
        ++a;
    }
    return a;
}
__host__ __device__ constexpr int pair_second(int P, int M) {
    int a = 0;
    while (P >= M - a) {
        P -= M - a;
        ++a;
    }
    return a + P;
}

struct rte_aniso3d_s {
    int n = 0, L = 0, M = 0, Q = 0, H = 0, np = 0, Bz64 = 0, Bz32 = 0;
    int RQ = 0;              // Q / 32 on the warp path (Q = 64, 128, 256), 0 on the Stockham path
    int Bw16 = 0, Bw8 = 0;   // warp path: Z lines per block for 16-byte and 8-byte complex types
    double h = 0.0, mu_t = 0.0, mu_s = 0.0, ms_pre = 0.0;
    double sig[RTE_ANISO_MAX_L + 1] = {};
    double Dh[RTE_ANISO_MAX_M * RTE_ANISO_MAX_M] = {};
    FftSched sc;
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    ffc* twff = nullptr;    // warp path: float-float twiddles
    double* S64 = nullptr;  // [np][H][H][H], xi_z fastest
    float* S32 = nullptr;
    ff* Sff = nullptr;      // warp path: float-float copy of S64
    double* wz = nullptr;   // [M] input weights mu_s sigma_hat_{l_b}
    int* pinfo = nullptr;   // [M][M]: pair index | imaginary << 16 | odd in y << 17 | odd in z << 18
    void* T1 = nullptr;     // Stockham: one n*H*n slab; warp path: M slabs (16-byte complex)
    void* T2 = nullptr;     // M*H*Q*n complex (16-byte)
    // solve: device GMRES in a CUDA graph (the plan's solver on this operator)
    double* u = nullptr;    // [M][n^3] solution
    double* f = nullptr;    // [n^3] source
    double* b64 = nullptr;
    double* r64 = nullptr;
    double* x64 = nullptr;  // FP64 mode: inner solution
    double* part64 = nullptr;
    float* r32 = nullptr;
    float* d32 = nullptr;
    void* ref = nullptr;    // device refinement state
    void* ref_host = nullptr;  // pinned staging, 2 x its size
    KrylovWs k64, k32;
    void* graph[3] = {nullptr, nullptr, nullptr};  // instantiated solve graphs by precision
    int graph_m[3] = {0, 0, 0};
    SolveGraphInfo ginfo[3];
};

// warp path (aniso3d_warp.cu): out_a = ca x_a + cb (K v)_a + cc z_a with the
// input channels v_b = w_b x_b (+ xf in channel 0 when xf is given), w_b =
// wz[b]; rhs = 1: one input channel x = f of weight 1 and out_a = cb (K~^{a0} f)_a.
// T1 and T2 are the handle's scratch.
template <typename T, typename R, typename TS>
cudaError_t aniso_run_warp(rte_aniso3d op, const R* x, R* out, int rhs, double ca, double cb, const R* zv, double cc,
                           const double* xf, const TS* S, const T* tw, cudaStream_t s);
// lines per block of the warp Z pass for an element size (0: one line does not fit)
int aniso_warp_lines(int RQ, int M, int elem_bytes);
// sets the warp kernels' shared-memory limits (once; before any graph capture)
cudaError_t aniso_warp_prepare(int RQ);
