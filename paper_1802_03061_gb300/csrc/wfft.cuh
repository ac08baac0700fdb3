// Warp-register FFT of length Q = 32 R (R = 2, 4, 8, 16): one warp per line,
// no shared memory traffic and no block barriers inside the transform.
//
// Lane l, register r holds x[l + 32 r] (coalesced loads).  With
// k = k1 + R k2:   X[k] = sum_l W32^{l k2} W_Q^{l k1} (sum_r x[l + 32 r] W_R^{r k1})
// so the forward transform is an R-point DFT in registers, a twiddle
// W_Q^{l k1}, and a 32-point decimation-in-frequency DFT across the lanes
// (butterflies with __shfl_xor_sync).  The result sits at lane l, register
// k1 as X[k1 + R brev5(l)].  The inverse takes exactly that layout: a
// 32-point decimation-in-time DFT across lanes (the mirror of the forward),
// the conjugate twiddle, then the R-point inverse DFT in registers, and
// returns x in the natural (l + 32 r) layout -- so a fused
// FFT -> pointwise -> inverse FFT moves no data between its halves.
#pragma once
#include "fft.cuh"

__device__ __forceinline__ int brev5(int l) { return __brev(l) >> 27; }

// bank swizzle of a line of Q (a multiple of 16) complex values in shared
// memory: xi -> xi ^ ((xi >> 4) & 15) stays inside its aligned group of 16,
// so it is a bijection; the 32 lanes of a warp that store one register
// (frequencies k1 + R brev5(lane), equal low bits) land on 16 distinct bank
// pairs instead of one
__device__ __forceinline__ int swz16(int xi) { return xi ^ ((xi >> 4) & 15); }

template <int DIR, typename T> __device__ __forceinline__ void dft16(T* v) {
    // 16 = 4 x 4: inner DFT4 over n1 of x[4 n1 + n2], twiddle W16^{n2 k1}, outer DFT4 over n2
    using Rr = typename real_of<T>::R;
    T t[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        T a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
        bfly4<DIR>(a);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) t[n2][k1] = a[k1];
    }
    // twiddles W16^{n2 k1} = exp(DIR 2 pi i n2 k1 / 16)
    const Rr c1 = (Rr)0.92387953251128675613, s1 = (Rr)0.38268343236508977173;  // cos, sin(pi/8)
    const Rr r2 = (Rr)0.70710678118654752440;
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) {
            const int e = (n2 * k1) & 15;  // angle e * pi / 8
            Rr c, s;
            switch (e) {
                case 1: c = c1; s = s1; break;
                case 2: c = r2; s = r2; break;
                case 3: c = s1; s = c1; break;
                case 4: c = 0; s = 1; break;
                case 6: c = -r2; s = r2; break;
                case 9: c = -c1; s = -s1; break;
                default: c = 1; s = 0; break;
            }
            const T w = mk<T>(c, DIR * s);
            t[n2][k1] = cmul(t[n2][k1], w);
        }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        T a[4] = {t[0][k1], t[1][k1], t[2][k1], t[3][k1]};
        bfly4<DIR>(a);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = a[k2];
    }
}

// exchange a complex value with lane ^ m
__device__ __forceinline__ float2 shfl_xor_c(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ double2 shfl_xor_c(double2 v, int m) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ ffc shfl_xor_c(ffc v, int m) {
    ffc r;
    r.x = ff(__shfl_xor_sync(0xffffffffu, v.x.hi, m), __shfl_xor_sync(0xffffffffu, v.x.lo, m));
    r.y = ff(__shfl_xor_sync(0xffffffffu, v.y.hi, m), __shfl_xor_sync(0xffffffffu, v.y.lo, m));
    return r;
}
template <typename T> __device__ __forceinline__ T cneg(T a) { return mk<T>(-a.x, -a.y); }

template <int R, int DIR, typename T> __device__ __forceinline__ void dft_regs(T* v) {
    if (R == 2) bfly2<DIR>(v);
    if (R == 4) bfly4<DIR>(v);
    if (R == 8) bfly8<DIR>(v);
    if (R == 16) dft16<DIR>(v);
}

// one decimation-in-frequency lane stage of span h: lower lane a + b, upper
// lane (a - b) w, written branch-free as (+-own + partner) * w with w = 1 on
// the lower lane (exact)
template <int R, typename T> __device__ __forceinline__ void lane_stage_fwd(T* v, const T* tw, int h, int lane) {
    constexpr int Q = 32 * R;
    const bool upper = lane & h;
    const T tw1 = twid<-1>(tw, (lane & (h - 1)) * (Q / (2 * h)));
    const T w = upper ? tw1 : mk<T>(1, 0);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
        const T pv = shfl_xor_c(v[k1], h);
        const T own = upper ? cneg(v[k1]) : v[k1];
        v[k1] = cmul(cadd(own, pv), w);
    }
}
// one decimation-in-time lane stage: lower lane a + w b, upper lane a - w b
// (a on the lower, b on the upper lane): one product per lane
template <int R, typename T> __device__ __forceinline__ void lane_stage_inv(T* v, const T* tw, int h, int lane) {
    constexpr int Q = 32 * R;
    const bool upper = lane & h;
    const T w = twid<1>(tw, (lane & (h - 1)) * (Q / (2 * h)));
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
        const T pv = shfl_xor_c(v[k1], h);
        const T a = upper ? pv : v[k1];
        const T m = cmul(upper ? v[k1] : pv, w);
        v[k1] = cadd(a, upper ? cneg(m) : m);
    }
}
// wide types (float-float) keep the five lane stages rolled: unrolled, the
// transform outgrows the instruction cache
template <typename T> struct roll_lane_stages { static constexpr bool value = sizeof(T) > 8; };

// forward: v[r] = x[lane + 32 r]  ->  v[k1] = X[k1 + R brev5(lane)]
// tw: table exp(-2 pi i t / Q), Q = 32 R
template <int R, typename T> __device__ __forceinline__ void warp_fft_fwd(T* v, const T* tw) {
    constexpr int Q = 32 * R;
    const int lane = threadIdx.x & 31;
    dft_regs<R, -1>(v);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], twid<-1>(tw, lane * k1));
    if constexpr (roll_lane_stages<T>::value) {
#pragma unroll 1
        for (int h = 16; h >= 1; h >>= 1) lane_stage_fwd<R>(v, tw, h, lane);
    } else {
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) lane_stage_fwd<R>(v, tw, h, lane);
    }
    (void)Q;
}

// inverse (unnormalised): v[k1] = X[k1 + R brev5(lane)]  ->  v[r] = Q x[lane + 32 r]
template <int R, typename T> __device__ __forceinline__ void warp_fft_inv(T* v, const T* tw) {
    const int lane = threadIdx.x & 31;
    if constexpr (roll_lane_stages<T>::value) {
#pragma unroll 1
        for (int h = 1; h <= 16; h <<= 1) lane_stage_inv<R>(v, tw, h, lane);
    } else {
#pragma unroll
        for (int h = 1; h <= 16; h <<= 1) lane_stage_inv<R>(v, tw, h, lane);
    }
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) v[k1] = cmul(v[k1], twid<1>(tw, lane * k1));
    dft_regs<R, 1>(v);
}
