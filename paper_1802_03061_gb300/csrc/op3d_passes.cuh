// The five 3D passes in general-Q Stockham form (any Q = 2^a 3^b), shared by
// the isotropic operator and the spherical-harmonic (anisotropic) one.
//   X  : two real rows packed into one complex FFT along x, split into the
//        half spectra xi_x = 0..Q/2              -> T1[z][xi_x][y]
//   Y  : FFT along y (zero padded), per (z, xi_x) -> T2[xi_x][xi_y][z]
//   Z  : FFT along z, multiply by S, inverse FFT, keep z < n (in place)
//   Y' : inverse FFT along y, keep y < n           -> T1[z][xi_x][y]
//   X' : Hermitian completion of two rows, inverse complex FFT, keep x < n,
//        epilogue.
#pragma once
#include "fft.cuh"
#include "internal.h"

#ifndef RTE_SMEM_OPTIN
#define RTE_SMEM_OPTIN 232448
#endif

struct P3 {
    int n, Q, H, B;  // B: lines (rows / z values / columns) per block
    FftSched sc;
};

__device__ __forceinline__ int fold(int a, int Q) { return a <= Q / 2 ? a : Q - a; }

// X: in real [n][n][n] (x fastest); grid (ceil(n/B), n), B even
template <typename T, typename R>
__global__ void __launch_bounds__(256) k3_x_fwd(const R* __restrict__ x, T* __restrict__ T1, const T* __restrict__ tw,
                                                P3 p, double w, const double* __restrict__ xf) {
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, B = p.B;
    const int z = blockIdx.y, y0 = blockIdx.x * B, nl = B / 2;
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)nl * Q;
    load_twiddles(twl, tw, Q);
    using RR = typename real_of<T>::R;
    const RR ww = (RR)w;
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int li = idx / Q, e = idx - li * Q;
        const int ya = y0 + 2 * li, yb = ya + 1;
        RR a = 0, b = 0;
        if (e < n) {
            if (ya < n) a = ww * (RR)x[((long)z * n + ya) * n + e];
            if (yb < n) b = ww * (RR)x[((long)z * n + yb) * n + e];
            if (xf) {  // the source joins unweighted: K x + K~ f in one application
                if (ya < n) a = a + (RR)xf[((long)z * n + ya) * n + e];
                if (yb < n) b = b + (RR)xf[((long)z * n + yb) * n + e];
            }
        }
        buf[idx] = mk<T>(a, b);
    }
    __syncthreads();
    T* res = fft_lines<-1>(buf, tmp, nl, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < H * B; idx += blockDim.x) {
        const int r = idx % B, xi = idx / B;
        const int y = y0 + r;
        if (y >= n) continue;
        const int line = r >> 1;
        const T Z = res[line * Q + xi];
        const T Zm = res[line * Q + (xi == 0 ? 0 : Q - xi)];
        T v;
        if ((r & 1) == 0) v = mk<T>((RR)0.5 * (Z.x + Zm.x), (RR)0.5 * (Z.y - Zm.y));
        else v = mk<T>((RR)0.5 * (Z.y + Zm.y), (RR)-0.5 * (Z.x - Zm.x));
        T1[((long)z * H + xi) * n + y] = v;
    }
}

// Y: T1[z][xi_x][y] -> T2[xi_x][xi_y][z]; grid (ceil(n/B), H): B consecutive z
template <typename T>
__global__ void __launch_bounds__(256) k3_y_fwd(const T* __restrict__ T1, T* __restrict__ T2, const T* __restrict__ tw,
                                                P3 p) {
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, B = p.B;
    const int kx = blockIdx.y, z0 = blockIdx.x * B;
    const int nl = min(B, n - z0);
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)B * Q;
    load_twiddles(twl, tw, Q);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int li = idx / Q, e = idx - li * Q;
        buf[idx] = e < n ? T1[((long)(z0 + li) * H + kx) * n + e] : mk<T>(0, 0);
    }
    __syncthreads();
    T* res = fft_lines<-1>(buf, tmp, nl, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int li = idx % nl, ky = idx / nl;
        T2[((long)kx * Q + ky) * n + z0 + li] = res[li * Q + ky];
    }
}

// Z: per (xi_x, xi_y) line along z: FFT, * S, iFFT, keep z < n; grid ceil(H*Q/B)
template <typename T, typename TS>
__global__ void __launch_bounds__(256) k3_z_mix(T* __restrict__ T2, const TS* __restrict__ S, const T* __restrict__ tw,
                                                P3 p) {
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    using RR = typename real_of<T>::R;
    const int n = p.n, Q = p.Q, H = p.H, B = p.B;
    const long l0 = (long)blockIdx.x * B;
    const long nlines = (long)H * Q;
    const int nl = (int)min((long)B, nlines - l0);
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)B * Q;
    load_twiddles(twl, tw, Q);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int li = idx / Q, e = idx - li * Q;
        buf[idx] = e < n ? T2[(l0 + li) * n + e] : mk<T>(0, 0);
    }
    __syncthreads();
    T* res = fft_lines<-1>(buf, tmp, nl, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int li = idx / Q, kz = idx - li * Q;
        const long l = l0 + li;
        const int kx = (int)(l / Q), ky = (int)(l % Q);
        const RR s = (RR)S[((long)kx * H + fold(ky, Q)) * H + fold(kz, Q)];
        res[idx] = cscale(res[idx], s);
    }
    __syncthreads();
    T* other = (res == buf) ? tmp : buf;
    T* res2 = fft_lines<1>(res, other, nl, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int li = idx / n, e = idx - li * n;
        T2[(l0 + li) * n + e] = res2[li * Q + e];
    }
}

// Y': T2[xi_x][xi_y][z] -> T1[z][xi_x][y], y < n; grid (ceil(n/B), H)
template <typename T>
__global__ void __launch_bounds__(256) k3_y_inv(const T* __restrict__ T2, T* __restrict__ T1, const T* __restrict__ tw,
                                                P3 p) {
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, B = p.B;
    const int kx = blockIdx.y, z0 = blockIdx.x * B;
    const int nl = min(B, n - z0);
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)B * Q;
    load_twiddles(twl, tw, Q);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int li = idx % nl, ky = idx / nl;
        buf[li * Q + ky] = T2[((long)kx * Q + ky) * n + z0 + li];
    }
    __syncthreads();
    T* res = fft_lines<1>(buf, tmp, nl, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int li = idx / n, e = idx - li * n;
        T1[((long)(z0 + li) * H + kx) * n + e] = res[li * Q + e];
    }
}

// X': T1[z][xi_x][y] -> out[z][y][x] = a*x + b*v + c*zv; grid (ceil(n/B), n)
template <typename T, typename R>
__global__ void __launch_bounds__(256) k3_x_inv(const T* __restrict__ T1, const R* __restrict__ x,
                                                const R* __restrict__ zv, R* __restrict__ out, const T* __restrict__ tw,
                                                P3 p, double a, double b, double c) {
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, B = p.B;
    const int z = blockIdx.y, y0 = blockIdx.x * B, nl = B / 2;
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)nl * Q;
    load_twiddles(twl, tw, Q);
    for (int idx = threadIdx.x; idx < H * nl; idx += blockDim.x) {
        const int li = idx % nl, xi = idx / nl;
        const int ya = y0 + 2 * li, yb = ya + 1;
        T Fv = mk<T>(0, 0), Gv = mk<T>(0, 0);
        if (ya < n) Fv = T1[((long)z * H + xi) * n + ya];
        if (yb < n) Gv = T1[((long)z * H + xi) * n + yb];
        buf[li * Q + xi] = mk<T>(Fv.x - Gv.y, Fv.y + Gv.x);
        if (xi > 0 && xi < Q - xi) buf[li * Q + (Q - xi)] = mk<T>(Fv.x + Gv.y, Gv.x - Fv.y);
    }
    __syncthreads();
    T* res = fft_lines<1>(buf, tmp, nl, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int li = idx / n, e = idx - li * n;
        const T v = res[li * Q + e];
        const int ya = y0 + 2 * li, yb = ya + 1;
        if (ya < n) {
            const long o = ((long)z * n + ya) * n + e;
            double r = b * (double)v.x;
            if (x) r += a * (double)x[o];
            if (zv) r += c * (double)zv[o];
            out[o] = (R)r;
        }
        if (yb < n) {
            const long o = ((long)z * n + yb) * n + e;
            double r = b * (double)v.y;
            if (x) r += a * (double)x[o];
            if (zv) r += c * (double)zv[o];
            out[o] = (R)r;
        }
    }
}

// ---------------------------------------------------------------------------
// The same five passes with the warp-register FFT (Q = 32 RQ, FP32 or
// float-float compute), one warp per line:
//   X  : 8 warps per block = 16 rows of one z plane (packed pairs), split
//        through a swizzled shared line buffer     -> T1[z][xi_x][y]
//   Y  : 16 warps per block = 16 consecutive z of one xi_x; the spectrum is
//        written in the FFT's slot order s = j*32 + lane (xi_y =
//        wfreq<RQ>(j, lane)) through a shared [s][z] tile -> T2[xi_x][s][z]
//   Z  : per (xi_x, s) line: FFT, * S, iFFT in registers (in place)
//   Y' : reads the slot order back into the inverse  -> T1[z][xi_x][y]
//   X' : Hermitian rebuild, inverse FFT, epilogue in the compute type.
// ---------------------------------------------------------------------------
