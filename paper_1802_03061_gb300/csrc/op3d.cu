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

template <typename RO, typename RR> __device__ __forceinline__ RO out_cast(RR v) { return static_cast<RO>(v); }

template <int RQ, typename T, typename RI>
__global__ void __launch_bounds__(256) k3w_x_fwd(const RI* __restrict__ x, T* __restrict__ T1,
                                                 const T* __restrict__ tw, int n, int H, double w,
                                                 const double* __restrict__ xf) {
    constexpr int Q = 32 * RQ, LS = Q + 34;  // a line also holds the warp's FFT scratch (Q + 32)
    using RR = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Z = twl + Q;
    const int z = blockIdx.y, y0 = blockIdx.x * 16;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    __syncthreads();
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RR ww = (RR)w;
    const int ya = y0 + 2 * wp, yb = ya + 1;
    T v[RQ];
#pragma unroll
    for (int r = 0; r < RQ; ++r) {
        const int e = lane + 32 * r;
        RR a = (RR)0, b = (RR)0;
        if (e < n) {
            if (ya < n) a = ww * (RR)x[((long)z * n + ya) * n + e];
            if (yb < n) b = ww * (RR)x[((long)z * n + yb) * n + e];
            if (xf) {  // the source joins unweighted: K x + K~ f in one application
                if (ya < n) a = a + (RR)xf[((long)z * n + ya) * n + e];
                if (yb < n) b = b + (RR)xf[((long)z * n + yb) * n + e];
            }
        }
        v[r] = mk<T>(a, b);
    }
    warp_fft_fwd<RQ>(v, twl, Z + wp * LS);
#pragma unroll
    for (int j = 0; j < RQ; ++j) Z[wp * LS + swz16(wfreq<RQ>(j, lane))] = v[j];
    __syncthreads();
    for (int idx = threadIdx.x; idx < H * 16; idx += blockDim.x) {
        const int r = idx & 15, xi = idx >> 4;
        const int y = y0 + r;
        if (y >= n) continue;
        const int line = r >> 1;
        const T Zp = Z[line * LS + swz16(xi)];
        const T Zm = Z[line * LS + swz16(xi == 0 ? 0 : Q - xi)];
        T o;
        if ((r & 1) == 0) o = mk<T>((RR)0.5 * (Zp.x + Zm.x), (RR)0.5 * (Zp.y - Zm.y));
        else o = mk<T>((RR)0.5 * (Zp.y + Zm.y), (RR)-0.5 * (Zp.x - Zm.x));
        T1[((long)z * H + xi) * n + y] = o;
    }
}

template <int RQ, typename T>
__global__ void __launch_bounds__(512) k3w_y_fwd(const T* __restrict__ T1, T* __restrict__ T2,
                                                 const T* __restrict__ tw, int n, int H) {
    constexpr int Q = 32 * RQ, ZS = 17;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Y = twl + Q;  // [s][ZS] tile; before it is written, the 16 warps' FFT scratch
    const int kx = blockIdx.y, z0 = blockIdx.x * 16;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    __syncthreads();
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = z0 + wp;
    T v[RQ];
#pragma unroll
    for (int r = 0; r < RQ; ++r) {
        const int y = lane + 32 * r;
        v[r] = (z < n && y < n) ? T1[((long)z * H + kx) * n + y] : mk<T>(0, 0);
    }
    warp_fft_fwd<RQ>(v, twl, Y + wp * wfft_shape<RQ>::SCRATCH);
    __syncthreads();  // every warp is done with its scratch
#pragma unroll
    for (int k1 = 0; k1 < RQ; ++k1) Y[(k1 * 32 + lane) * ZS + wp] = v[k1];
    __syncthreads();
    const int nz = min(16, n - z0);
    for (int idx = threadIdx.x; idx < Q * 16; idx += blockDim.x) {
        const int zl = idx & 15, sl = idx >> 4;
        if (zl < nz) T2[((long)kx * Q + sl) * n + z0 + zl] = Y[sl * ZS + zl];
    }
}

template <int RQ, typename T, typename TS>
__global__ void __launch_bounds__(256) k3w_z_mix(T* __restrict__ T2, const TS* __restrict__ S,
                                                 const T* __restrict__ tw, int n, int H, long nlines) {
    constexpr int Q = 32 * RQ;
    using RR = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* scr = twl + Q + warp * wfft_shape<RQ>::SCRATCH;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    __syncthreads();
    const long line = (long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (line >= nlines) return;
    T v[RQ];
#pragma unroll
    for (int r = 0; r < RQ; ++r) {
        const int z = lane + 32 * r;
        v[r] = z < n ? T2[line * n + z] : mk<T>(0, 0);
    }
    warp_fft_fwd<RQ>(v, twl, scr);
    const int kx = (int)(line / Q), sl = (int)(line % Q);
    const int ky = wfreq<RQ>(sl >> 5, sl & 31);  // slot -> frequency
    const TS* Srow = S + ((long)kx * H + fold(ky, Q)) * H;
#pragma unroll
    for (int j = 0; j < RQ; ++j) {
        const RR sv = (RR)Srow[fold(wfreq<RQ>(j, lane), Q)];
        v[j] = mk<T>(v[j].x * sv, v[j].y * sv);
    }
    warp_fft_inv<RQ>(v, twl, scr);
#pragma unroll
    for (int r = 0; r < RQ; ++r) {
        const int z = lane + 32 * r;
        if (z < n) T2[line * n + z] = v[r];
    }
}

template <int RQ, typename T>
__global__ void __launch_bounds__(512) k3w_y_inv(const T* __restrict__ T2, T* __restrict__ T1,
                                                 const T* __restrict__ tw, int n, int H) {
    constexpr int Q = 32 * RQ, ZS = 17;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Y = twl + Q;  // [s][ZS] tile, then the 16 warps' FFT scratch
    const int kx = blockIdx.y, z0 = blockIdx.x * 16;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    const int nz = min(16, n - z0);
    for (int idx = threadIdx.x; idx < Q * 16; idx += blockDim.x) {
        const int zl = idx & 15, sl = idx >> 4;
        Y[sl * ZS + zl] = zl < nz ? T2[((long)kx * Q + sl) * n + z0 + zl] : mk<T>(0, 0);
    }
    __syncthreads();
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T v[RQ];
#pragma unroll
    for (int k1 = 0; k1 < RQ; ++k1) v[k1] = Y[(k1 * 32 + lane) * ZS + wp];
    __syncthreads();  // the tile is read; its space becomes the warps' FFT scratch
    warp_fft_inv<RQ>(v, twl, Y + wp * wfft_shape<RQ>::SCRATCH);
    const int z = z0 + wp;
    if (z >= n) return;
#pragma unroll
    for (int r = 0; r < RQ; ++r) {
        const int y = lane + 32 * r;
        if (y < n) T1[((long)z * H + kx) * n + y] = v[r];
    }
}

template <int RQ, typename T, typename RI>
__global__ void __launch_bounds__(256) k3w_x_inv(const T* __restrict__ T1, const RI* __restrict__ x,
                                                 const RI* __restrict__ zv, RI* __restrict__ out,
                                                 const T* __restrict__ tw, int n, int H, double a, double b,
                                                 double c) {
    constexpr int Q = 32 * RQ, LS = Q + 34;
    using RR = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Z = twl + Q;
    const int z = blockIdx.y, y0 = blockIdx.x * 16;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    for (int idx = threadIdx.x; idx < H * 8; idx += blockDim.x) {
        const int li = idx & 7, xi = idx >> 3;
        const int ya = y0 + 2 * li, yb = ya + 1;
        T Fv = mk<T>(0, 0), Gv = mk<T>(0, 0);
        if (ya < n) Fv = T1[((long)z * H + xi) * n + ya];
        if (yb < n) Gv = T1[((long)z * H + xi) * n + yb];
        Z[li * LS + swz16(xi)] = mk<T>(Fv.x - Gv.y, Fv.y + Gv.x);
        if (xi > 0 && xi < Q - xi) Z[li * LS + swz16(Q - xi)] = mk<T>(Fv.x + Gv.y, Gv.x - Fv.y);
    }
    __syncthreads();
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T v[RQ];
#pragma unroll
    for (int j = 0; j < RQ; ++j) v[j] = Z[wp * LS + swz16(wfreq<RQ>(j, lane))];
    __syncwarp();
    warp_fft_inv<RQ>(v, twl, Z + wp * LS);
    const RR ra = (RR)a, rb = (RR)b, rc = (RR)c;
    const int ya = y0 + 2 * wp, yb = ya + 1;
#pragma unroll
    for (int r = 0; r < RQ; ++r) {
        const int e = lane + 32 * r;
        if (e >= n) continue;
        if (ya < n) {
            const long o = ((long)z * n + ya) * n + e;
            RR q = rb * v[r].x;
            if (x) q = q + ra * (RR)x[o];
            if (zv) q = q + rc * (RR)zv[o];
            out[o] = out_cast<RI>(q);
        }
        if (yb < n) {
            const long o = ((long)z * n + yb) * n + e;
            RR q = rb * v[r].y;
            if (x) q = q + ra * (RR)x[o];
            if (zv) q = q + rc * (RR)zv[o];
            out[o] = out_cast<RI>(q);
        }
    }
}

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
    k3w_x_fwd<RQ, T, R><<<dim3(gy, n), 256, smx, s>>>(x, T1, tw, n, H, w, xf);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k3w_y_fwd<RQ, T><<<dim3(gy, H), 512, smy, s>>>(T1, T2, tw, n, H);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long nlines = (long)H * Q;
    k3w_z_mix<RQ, T, TS><<<(unsigned)((nlines + 7) / 8), 256, smz, s>>>(T2, S, tw, n, H, nlines);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k3w_y_inv<RQ, T><<<dim3(gy, H), 512, smy, s>>>(T2, T1, tw, n, H);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k3w_x_inv<RQ, T, R><<<dim3(gy, n), 256, smx, s>>>(T1, x, z, out, tw, n, H, a, b, c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
