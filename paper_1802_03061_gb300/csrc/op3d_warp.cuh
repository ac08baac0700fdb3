// 3D warp-register FFT passes (Q = 32 RQ): x (two real rows packed into one
// complex FFT, split into the half spectra), y, the isotropic z pass with the
// spectrum product, and the inverse y and x passes with the epilogue.  Shared
// by the isotropic operator (op3d.cu, one field) and the spherical-harmonic
// operator (aniso3d.cu, M channels in one launch: blockIdx.z is the channel,
// each channel's input, output and intermediates at fixed strides; wz, when
// given, holds each channel's input weight).
#pragma once
#include "fft.cuh"
#include "internal.h"
#include "op3d_passes.cuh"  // fold, RTE_SMEM_OPTIN
#include "wfft.cuh"

template <typename RO, typename RR> __device__ __forceinline__ RO out_cast(RR v) { return static_cast<RO>(v); }

template <int RQ, typename T, typename RI>
__global__ void __launch_bounds__(256) k3w_x_fwd(const RI* __restrict__ x, T* __restrict__ T1,
                                                 const T* __restrict__ tw, int n, int H, double w,
                                                 const double* __restrict__ xf,
                                                 const double* __restrict__ wz = nullptr) {
    constexpr int Q = 32 * RQ, LS = Q + 34;  // a line also holds the warp's FFT scratch (Q + 32)
    using RR = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Z = twl + Q;
    const int z = blockIdx.y, y0 = blockIdx.x * 16, ch = blockIdx.z;
    x += (long)ch * n * n * n;
    T1 += (long)ch * n * H * n;
    if (wz) w = wz[ch];
    if (ch > 0) xf = nullptr;  // the source joins channel 0 only
    stage_twiddles<Q, 256>(twl, tw);
    pdl_wait();  // x may be the predecessor's output
    pdl_trigger();
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
    __syncthreads();  // the twiddles are staged (the loads above overlap the barrier)
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
    const int kx = blockIdx.y, z0 = blockIdx.x * 16, ch = blockIdx.z;
    T1 += (long)ch * n * H * n;
    T2 += (long)ch * H * Q * n;
    stage_twiddles<Q, 512>(twl, tw);
    pdl_wait();  // T1: the x pass's output
    pdl_trigger();
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
    stage_twiddles<Q, 256>(twl, tw);
    pdl_wait();  // T2: the y pass's output
    pdl_trigger();
    const long line = (long)blockIdx.x * (blockDim.x >> 5) + warp;
    T v[RQ];
#pragma unroll
    for (int r = 0; r < RQ; ++r) {
        const int z = lane + 32 * r;
        v[r] = (line < nlines && z < n) ? T2[line * n + z] : mk<T>(0, 0);
    }
    __syncthreads();  // the twiddles are staged (the loads above overlap the barrier)
    if (line >= nlines) return;
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
    const int kx = blockIdx.y, z0 = blockIdx.x * 16, ch = blockIdx.z;
    T1 += (long)ch * n * H * n;
    T2 += (long)ch * H * Q * n;
    stage_twiddles<Q, 512>(twl, tw);
    pdl_wait();  // T2: the z pass's output
    pdl_trigger();
    const int nz = min(16, n - z0);
    // Q * 16 / 512 = RQ elements per thread, in groups of four whose loads
    // are all issued before their writes to the tile
    constexpr int IT = Q * 16 / 512, GR = IT < 4 ? IT : 4;
#pragma unroll
    for (int g0 = 0; g0 < IT; g0 += GR) {
        T vv[GR];
#pragma unroll
        for (int g = 0; g < GR; ++g) {
            const int idx = threadIdx.x + (g0 + g) * 512;
            const int zl = idx & 15, sl = idx >> 4;
            vv[g] = zl < nz ? T2[((long)kx * Q + sl) * n + z0 + zl] : mk<T>(0, 0);
        }
#pragma unroll
        for (int g = 0; g < GR; ++g) {
            const int idx = threadIdx.x + (g0 + g) * 512;
            Y[(idx >> 4) * ZS + (idx & 15)] = vv[g];
        }
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
    const int z = blockIdx.y, y0 = blockIdx.x * 16, ch = blockIdx.z;
    {
        const long N3 = (long)n * n * n;
        T1 += (long)ch * n * H * n;
        if (x) x += ch * N3;
        if (zv) zv += ch * N3;
        out += ch * N3;
    }
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ya = y0 + 2 * wp, yb = ya + 1;
    // the epilogue's x values, loaded before the transform so that their
    // latency overlaps it: n <= Q/2, so only registers r < RQ/2 hold x < n
    constexpr int RH = RQ / 2;
    RI pxa[RH], pxb[RH];
#pragma unroll
    for (int r = 0; r < RH; ++r) {
        const int e = lane + 32 * r;
        pxa[r] = (x && e < n && ya < n) ? x[((long)z * n + ya) * n + e] : (RI)0;
        pxb[r] = (x && e < n && yb < n) ? x[((long)z * n + yb) * n + e] : (RI)0;
    }
    stage_twiddles<Q, 256>(twl, tw);
    pdl_wait();  // T1: the y' pass's output
    pdl_trigger();
    {
        // H = Q/2 + 1 is fixed by RQ: every load of this thread is issued
        // before its first write to Z, so their latencies overlap
        constexpr int HH = Q / 2 + 1, IT = (HH * 8 + 255) / 256;
        T F[IT], G[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int idx = threadIdx.x + it * 256;
            const int li = idx & 7, xi = idx >> 3;
            const int la = y0 + 2 * li, lb = la + 1;
            T Fv = mk<T>(0, 0), Gv = mk<T>(0, 0);
            if (idx < HH * 8) {
                if (la < n) Fv = T1[((long)z * H + xi) * n + la];
                if (lb < n) Gv = T1[((long)z * H + xi) * n + lb];
            }
            F[it] = Fv;
            G[it] = Gv;
        }
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int idx = threadIdx.x + it * 256;
            if (idx >= HH * 8) continue;
            const int li = idx & 7, xi = idx >> 3;
            const T Fv = F[it], Gv = G[it];
            Z[li * LS + swz16(xi)] = mk<T>(Fv.x - Gv.y, Fv.y + Gv.x);
            if (xi > 0 && xi < Q - xi) Z[li * LS + swz16(Q - xi)] = mk<T>(Fv.x + Gv.y, Gv.x - Fv.y);
        }
    }
    __syncthreads();
    T v[RQ];
#pragma unroll
    for (int j = 0; j < RQ; ++j) v[j] = Z[wp * LS + swz16(wfreq<RQ>(j, lane))];
    __syncwarp();
    warp_fft_inv<RQ>(v, twl, Z + wp * LS);
    const RR ra = (RR)a, rb = (RR)b, rc = (RR)c;
#pragma unroll
    for (int r = 0; r < RH; ++r) {
        const int e = lane + 32 * r;
        if (e >= n) continue;
        if (ya < n) {
            const long o = ((long)z * n + ya) * n + e;
            RR q = rb * v[r].x;
            if (x) q = q + ra * (RR)pxa[r];
            if (zv) q = q + rc * (RR)zv[o];
            out[o] = out_cast<RI>(q);
        }
        if (yb < n) {
            const long o = ((long)z * n + yb) * n + e;
            RR q = rb * v[r].y;
            if (x) q = q + ra * (RR)pxb[r];
            if (zv) q = q + rc * (RR)zv[o];
            out[o] = out_cast<RI>(q);
        }
    }
}

