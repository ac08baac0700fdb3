// 3D isotropic operator passes: y = a*x + b*(K x) + c*z  (or b*(K~ f)).
//
// Sec. 2.3.1 with d = 3: kappa(r) = exp(-mu_t|r|)/(4 pi |r|^2) is a
// convolution on the zero-padded Q^3 grid, so K x = mu_s * iFFT(S * FFT(x)),
// with the real, even spectrum S stored as its octant [H][H][H].  Passes:
//   X  : two real rows packed into one complex FFT along x, split into the
//        half spectra xi_x = 0..Q/2              -> T1[z][xi_x][y]
//   Y  : FFT along y (zero padded), per (z, xi_x) -> T2[xi_x][xi_y][z]
//   Z  : FFT along z, multiply by S, inverse FFT, keep z < n (in place)
//   Y' : inverse FFT along y, keep y < n           -> T1[z][xi_x][y]
//   X' : Hermitian completion of two rows, inverse complex FFT, keep x < n,
//        epilogue.
// Each intermediate is laid out so that the next pass reads contiguous lines.
#include <type_traits>

#include "fft.cuh"
#include "internal.h"
#include "wfft.cuh"

#include "op3d_passes.cuh"

#include "op3d_warp.cuh"

template <int RQ, typename T, typename R, typename TS>
static cudaError_t op3d_run_warp(int n, int H, const R* x, R* out, double w, double a, double b, double c,
                                 const R* z, T* T1, T* T2, const TS* S, const T* tw, cudaStream_t s,
                                 const double* xf) {
    constexpr int Q = 32 * RQ;
    static bool once = false;
    cudaError_t e;
    using W = wfft_shape<RQ>;
    const size_t smx = (size_t)(Q + 8 * (Q + 34)) * sizeof(T);
    const size_t smy = (size_t)(Q + (Q * 17 > 16 * W::SCRATCH ? Q * 17 : 16 * W::SCRATCH)) * sizeof(T);
    const size_t smz = (size_t)(Q + 8 * W::SCRATCH) * sizeof(T);
    if (!once) {
        if ((e = cudaFuncSetAttribute(k3w_x_fwd<RQ, T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k3w_x_inv<RQ, T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k3w_y_fwd<RQ, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k3w_y_inv<RQ, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k3w_z_mix<RQ, T, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smz)) != cudaSuccess)
            return e;
        once = true;
    }
    const unsigned gy = (unsigned)((n + 15) / 16);
    const double* nowz = nullptr;
    if ((e = launch_pdl(k3w_x_fwd<RQ, T, R>, dim3(gy, n), dim3(256), smx, s, x, T1, tw, n, H, w, xf, nowz)) !=
        cudaSuccess)
        return e;
    if ((e = launch_pdl(k3w_y_fwd<RQ, T>, dim3(gy, H), dim3(512), smy, s, (const T*)T1, T2, tw, n, H)) != cudaSuccess)
        return e;
    const long nlines = (long)H * Q;
    if ((e = launch_pdl(k3w_z_mix<RQ, T, TS>, dim3((unsigned)((nlines + 7) / 8)), dim3(256), smz, s, T2, S, tw, n, H,
                        nlines)) != cudaSuccess)
        return e;
    if ((e = launch_pdl(k3w_y_inv<RQ, T>, dim3(gy, H), dim3(512), smy, s, (const T*)T2, T1, tw, n, H)) != cudaSuccess)
        return e;
    if ((e = launch_pdl(k3w_x_inv<RQ, T, R>, dim3(gy, n), dim3(256), smx, s, (const T*)T1, x, z, out, tw, n, H, a, b,
                        c)) != cudaSuccess)
        return e;
    rte_count_launches(5);
    return cudaSuccess;
}

template <typename K> static cudaError_t allow(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, RTE_SMEM_OPTIN);
}

template <typename T> static int lines_per_block(int Q) {
    int b = 65536 / (2 * Q * (int)sizeof(T));
    if (b > 16) b = 16;
    if (b < 2) b = 2;
    return b & ~1;
}

template <typename T, typename R, typename TS>
static cudaError_t op3d_run(rte_plan p, const R* x, R* out, double w, double a, double b, double c, const R* z,
                            T* T1, T* T2, const TS* S, const T* tw, cudaStream_t s, const double* xf = nullptr) {
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow(k3_x_fwd<T, R>)) != cudaSuccess) return e;
        if ((e = allow(k3_y_fwd<T>)) != cudaSuccess) return e;
        if ((e = allow(k3_z_mix<T, TS>)) != cudaSuccess) return e;
        if ((e = allow(k3_y_inv<T>)) != cudaSuccess) return e;
        if ((e = allow(k3_x_inv<T, R>)) != cudaSuccess) return e;
        once = true;
    }
    if constexpr (!std::is_same<T, double2>::value) {
        // FP32 and float-float: warp-register passes when Q = 32 * 2^j
        switch (p->Q) {
            case 64: return op3d_run_warp<2>(p->n, p->H, x, out, w, a, b, c, z, T1, T2, S, tw, s, xf);
            case 128: return op3d_run_warp<4>(p->n, p->H, x, out, w, a, b, c, z, T1, T2, S, tw, s, xf);
            case 256: return op3d_run_warp<8>(p->n, p->H, x, out, w, a, b, c, z, T1, T2, S, tw, s, xf);
            case 512: return op3d_run_warp<16>(p->n, p->H, x, out, w, a, b, c, z, T1, T2, S, tw, s, xf);
            default: break;
        }
    }
    P3 pp;
    pp.n = p->n;
    pp.Q = p->Q;
    pp.H = p->H;
    pp.sc = p->sched;
    const int n = p->n, Q = p->Q, H = p->H;
    pp.B = lines_per_block<T>(Q);
    const int B = pp.B;
    const size_t smx = (size_t)(Q + 2 * (B / 2) * Q) * sizeof(T);
    const size_t smy = (size_t)(Q + 2 * B * Q) * sizeof(T);
    k3_x_fwd<T, R><<<dim3((n + B - 1) / B, n), 256, smx, s>>>(x, T1, tw, pp, w, xf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k3_y_fwd<T><<<dim3((n + B - 1) / B, H), 256, smy, s>>>(T1, T2, tw, pp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long nlines = (long)H * Q;
    k3_z_mix<T, TS><<<(unsigned)((nlines + B - 1) / B), 256, smy, s>>>(T2, S, tw, pp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k3_y_inv<T><<<dim3((n + B - 1) / B, H), 256, smy, s>>>(T2, T1, tw, pp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k3_x_inv<T, R><<<dim3((n + B - 1) / B, n), 256, smx, s>>>(T1, x, z, out, tw, pp, a, b, c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    rte_count_launches(5);
    return cudaSuccess;
}

rte_status op3d_apply64(rte_plan p, MixKind kind, const double* x, double* out, double a, double b, double c,
                        const double* z, cudaStream_t s) {
    const double w = kind == MIX_RHS ? 1.0 : p->mu_s;
    cudaError_t e = op3d_run<double2, double, double>(p, x, out, w, kind == MIX_RHS ? 0.0 : a, b, c, z,
                                                      (double2*)p->T64, (double2*)p->U64, p->S3_64, p->tw64, s,
                                                      kind == MIX_KF ? p->f_dev : nullptr);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op3d_apply64");
    return RTE_OK;
}

rte_status op3d_apply32(rte_plan p, const float* x, float* out, float a, float b, float c, const float* z,
                        cudaStream_t s) {
    cudaError_t e = op3d_run<float2, float, float>(p, x, out, p->mu_s, a, b, c, z, (float2*)p->T32, (float2*)p->U32,
                                                   p->S3_32, p->tw32, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op3d_apply32");
    return RTE_OK;
}

rte_status op3d_apply_ff(rte_plan p, MixKind kind, const double* x, double* out, double a, double b, double c,
                         const double* z, cudaStream_t s) {
    // MIX_KF: K x + K~ f = K~ (mu_s x + f), the plan's source f
    const double w = kind == MIX_RHS ? 1.0 : p->mu_s;
    cudaError_t e = op3d_run<ffc, double, ff>(p, x, out, w, kind == MIX_RHS ? 0.0 : a, b, c, z, (ffc*)p->T64,
                                             (ffc*)p->U64, p->S3ff, p->twff, s, kind == MIX_KF ? p->f_dev : nullptr);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op3d_apply_ff");
    return RTE_OK;
}

__global__ void k_narrow(const double* __restrict__ src, float* __restrict__ dst, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// b = K~ f in FP32; f32 (n^3 floats) receives the source rounded to FP32
rte_status op3d_rhs32(rte_plan p, float* f32, float* out, cudaStream_t s) {
    k_narrow<<<1024, 256, 0, s>>>(p->f_dev, f32, p->ncell);
    rte_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = op3d_run<float2, float, float>(p, f32, out, 1.0, 0.0, 1.0, 0.0, nullptr, (float2*)p->T32, (float2*)p->U32,
                                           p->S3_32, p->tw32, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op3d_rhs32");
    return RTE_OK;
}

// the periodic preconditioner's 3D application out = M x (precond.cu): the
// same passes with the inverse spectrum and unit input weight
cudaError_t op3d_run_pc32(rte_plan p, const float* x, float* out, cudaStream_t s) {
    return op3d_run<float2, float, float>(p, x, out, 1.0, 0.0, 1.0, 0.0, nullptr, (float2*)p->T32, (float2*)p->U32,
                                          p->S3p, p->tw32, s);
}
