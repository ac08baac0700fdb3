// Warp FFT of length Q = 32 R (R = 2, 4, 8, 16): one warp per line, the data
// in registers, one transpose through a per-warp shared scratch.
//
// Lane l, register r holds x[l + 32 r] (coalesced loads).  With
// xi = k1 + R kappa (k1 < R, kappa < 32) and n = l + 32 r,
//   X[xi] = sum_l W32^{l kappa} [ W_Q^{l k1} sum_r x[l + 32 r] W_R^{r k1} ],
// i.e. an R-point DFT in registers and a twiddle (step 1), then 32-point DFTs
// over l, one per k1 (step 2).  Step 2 does not run over five cross-lane
// stages: the R x 32 block is transposed through shared memory so that the
// P = 32/R lanes L = P k1 + b (b < P) share the DFT of k1, lane b holding the
// inputs l = P m + b (m < R).  Splitting kappa = kappa' + R c (kappa' < R,
// c < P),
//   X[k1 + R (kappa' + R c)] = sum_b W_P^{b c} W32^{b kappa'} DFT_R[m](Y[P m + b])[kappa'],
// so each lane does a second R-point DFT in registers and a twiddle, and the
// P lanes finish with log2(P) decimation-in-frequency radix-2 stages
// (__shfl_xor_sync).  Lane L = P k1 + b, register j then holds
// X[k1 + R (j + R brev(b))] (brev over log2 P bits; wfreq below).  The
// inverse mirrors every step and returns x in the natural (l + 32 r) layout,
// so a fused FFT -> pointwise -> inverse FFT needs no reordering.  Counted in
// instructions this is about half of a transform with five lane stages.
#pragma once
#include "fft.cuh"

// the Q-entry twiddle table into shared memory by a block of NT threads: the
// trip count is a compile-time constant, so a thread's loads are all issued
// before its stores (a loop over blockDim.x waits for each load in turn)
template <int Q, int NT, typename T>
__device__ __forceinline__ void stage_twiddles(T* __restrict__ sm, const T* __restrict__ g) {
    constexpr int IT = (Q + NT - 1) / NT;
    T t[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int i = threadIdx.x + it * NT;
        if (i < Q) t[it] = g[i];
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int i = threadIdx.x + it * NT;
        if (i < Q) sm[i] = t[it];
    }
}

// bank swizzle of a line of Q (a multiple of 16) complex values in shared
// memory: xi -> xi ^ ((xi >> 4) & 15) stays inside its aligned group of 16,
// so it is a bijection; it spreads the frequencies that the 32 lanes of a
// warp hold in one register (which differ mostly in their high bits) over
// the banks
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

template <int R> struct wfft_shape {
    static constexpr int Q = 32 * R;
    static constexpr int P = 32 / R;                            // lanes per 32-point DFT in step 2
    static constexpr int LP = R == 16 ? 1 : R == 8 ? 2 : R == 4 ? 3 : 4;  // log2 P
    static constexpr int ST = 32 + P;                           // scratch row stride (bank spread)
    static constexpr int SCRATCH = R * ST;                      // scratch elements per warp (Q + 32)
};

// frequency held by register j of lane L = P g + b after the forward
// transform.  R >= P (R = 8, 16): register j = P t + c holds
// X[g + R (kappa' + R c)] with kappa' = b + P t (the P-point DFTs of the last
// step run in registers after a transpose); R < P: register j holds
// X[g + R (j + R brev(b))] (the last step runs as lane stages).
__host__ __device__ __forceinline__ int wfreq_map(int R, int j, int lane) {
    const int P = 32 / R;
    const int LP = R == 16 ? 1 : R == 8 ? 2 : R == 4 ? 3 : 4;
    const int g = lane >> LP, b = lane & (P - 1);
    if (R >= P) {
        const int t = j / P, c = j % P;
        return g + R * ((b + P * t) + R * c);
    }
    int c = 0;
    for (int i = 0; i < LP; ++i) c |= ((b >> i) & 1) << (LP - 1 - i);
    return g + R * (j + R * c);
}
template <int R> __device__ __forceinline__ int wfreq(int j, int lane) { return wfreq_map(R, j, lane); }
// the same with R known at run time (plan-time permutations)
__device__ __forceinline__ int wfreq_rt(int R, int j, int lane) { return wfreq_map(R, j, lane); }

// frequency of slot sl of a spectrum held as two warp FFTs of length QW =
// Q / 2 (residues r = xi mod 2): slot r * QW + s holds xi = 2 wfreq_QW(s) + r
__device__ __forceinline__ int slot_freq_res(int sl, int QW) {
    const int r = sl / QW, s = sl % QW;
    return 2 * wfreq_rt(QW / 32, s >> 5, s & 31) + r;
}
// frequency of slot sl (= j * 32 + lane) of the column passes' spectra.
// Q <= 512: the warp FFT's own order.  Q = 1024 runs as two 512-point warp
// FFTs (residues, see k_col_warp2).
__device__ __forceinline__ int slot_freq(int sl, int Q) {
    if (Q <= 512) return wfreq_rt(Q / 32, sl >> 5, sl & 31);
    return slot_freq_res(sl, 512);
}
// the same for the float-float column passes, which run Q = 512 as two
// 256-point residues as well (a one-warp 512-point float-float line needs
// too many registers)
__device__ __forceinline__ int slot_freq_ff(int sl, int Q) {
    if (Q < 512) return wfreq_rt(Q / 32, sl >> 5, sl & 31);
    return slot_freq_res(sl, Q / 2);
}

// P-point DFT (P = 2, 4) in registers
template <int P, int DIR, typename T> __device__ __forceinline__ void dft_small(T* u) {
    if constexpr (P == 2) bfly2<DIR>(u);
    if constexpr (P == 4) bfly4<DIR>(u);
}

// last step for R >= P: lane L = P g + b holds Y[g][b][kappa'] in v[kappa'];
// the P-point DFTs over b (one per kappa') are gathered by a transpose in the
// warp's scratch (lane rows of R + 1: conflict-free 8-byte accesses), lane
// (g, b') computing those of kappa' = b' + P t; v[P t + c] = output c.  The
// scratch needs 32 (R + 1) = R (32 + P) elements, the same as step 1's.
template <int R, int DIR, typename T> __device__ __forceinline__ void warp_last_regs(T* v, T* S, int lane) {
    using W = wfft_shape<R>;
    constexpr int P = W::P, RS = R + 1;
    const int g = lane >> W::LP, b = lane & (P - 1);
#pragma unroll
    for (int j = 0; j < R; ++j) S[lane * RS + j] = v[j];
    __syncwarp();
#pragma unroll
    for (int t = 0; t < R / P; ++t) {
        T u[P];
#pragma unroll
        for (int bb = 0; bb < P; ++bb) u[bb] = S[(g * P + bb) * RS + b + P * t];
        dft_small<P, DIR>(u);
#pragma unroll
        for (int c = 0; c < P; ++c) v[P * t + c] = u[c];
    }
    __syncwarp();
}
// its inverse: v[P t + c] -> lane (g, b) holds P Y[g][b][kappa'] in v[kappa']
template <int R, typename T> __device__ __forceinline__ void warp_first_regs_inv(T* v, T* S, int lane) {
    using W = wfft_shape<R>;
    constexpr int P = W::P, RS = R + 1;
    const int g = lane >> W::LP, b = lane & (P - 1);
#pragma unroll
    for (int t = 0; t < R / P; ++t) {
        T u[P];
#pragma unroll
        for (int c = 0; c < P; ++c) u[c] = v[P * t + c];
        dft_small<P, 1>(u);
#pragma unroll
        for (int bb = 0; bb < P; ++bb) S[(g * P + bb) * RS + b + P * t] = u[bb];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = S[lane * RS + j];
    __syncwarp();
}

// twiddle multiply v[k] *= W^k (DIR = -1) or conj(W)^k (DIR = +1),
// W = exp(-2 pi i base / Q), k = 1..R-1 (base = lane in step 1, b R in step 2;
// base (R - 1) < Q either way).  FP32 with R <= 8 reads W, W^2, W^4
// from the table and forms W^3, W^5, W^6, W^7 as products of two of them (one
// rounding each, next to the FFT's own log2 Q roundings): the 3D passes issue
// from shared memory (transposes and twiddle reads), so fewer reads pay more
// than the extra multiplies.  R = 16 (the register-heavy 2D passes) and the
// float-float types read every power from the table, each just before use.
template <int R, int DIR, typename T> __device__ __forceinline__ void lane_twiddle_mul(T* v, const T* tw, int base) {
    if constexpr (sizeof(T) == 8 && R <= 8) {
        T W[R];
#pragma unroll
        for (int k = 1; k < R; k <<= 1) W[k] = tw[base * k];
#pragma unroll
        for (int k = 3; k < R; ++k) {
            if ((k & (k - 1)) == 0) continue;
            const int hb = k >= 4 ? 4 : 2;  // highest power of two in k (k < 8)
            W[k] = cmul(W[hb], W[k - hb]);
        }
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmul(v[k], DIR < 0 ? W[k] : cconj(W[k]));
    } else {
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmul(v[k], twid<DIR>(tw, base * k));
    }
}

// forward: v[r] = x[lane + 32 r]  ->  v[j] = X[wfreq<R>(j, lane)]
// tw: table exp(-2 pi i t / Q); S: this warp's scratch (wfft_shape<R>::SCRATCH
// elements of shared memory), free again when the call returns
template <int R, typename T> __device__ __forceinline__ void warp_fft_fwd(T* v, const T* tw, T* S) {
    using W = wfft_shape<R>;
    const int lane = threadIdx.x & 31;
    dft_regs<R, -1>(v);
    lane_twiddle_mul<R, -1>(v, tw, lane);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) S[k1 * W::ST + lane] = v[k1];
    __syncwarp();
    const int g = lane >> W::LP, b = lane & (W::P - 1);
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = S[g * W::ST + W::P * m + b];
    __syncwarp();
    dft_regs<R, -1>(v);
    lane_twiddle_mul<R, -1>(v, tw, b * R);
    if constexpr (R >= W::P) {
        warp_last_regs<R, -1>(v, S, lane);
    } else {
#pragma unroll
        for (int h = W::P / 2; h >= 1; h >>= 1) lane_stage_fwd<R>(v, tw, h, lane);
    }
}

// inverse (unnormalised): v[j] = X[wfreq<R>(j, lane)]  ->  v[r] = Q x[lane + 32 r]
// (S must be free on entry: the caller synchronises the warp after its own
// last use of it)
template <int R, typename T> __device__ __forceinline__ void warp_fft_inv(T* v, const T* tw, T* S) {
    using W = wfft_shape<R>;
    const int lane = threadIdx.x & 31;
    if constexpr (R >= W::P) {
        warp_first_regs_inv<R>(v, S, lane);
    } else {
#pragma unroll
        for (int h = 1; h <= W::P / 2; h <<= 1) lane_stage_inv<R>(v, tw, h, lane);
    }
    const int g = lane >> W::LP, b = lane & (W::P - 1);
    lane_twiddle_mul<R, 1>(v, tw, b * R);
    dft_regs<R, 1>(v);
#pragma unroll
    for (int m = 0; m < R; ++m) S[g * W::ST + W::P * m + b] = v[m];
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) v[k1] = S[k1 * W::ST + lane];
    __syncwarp();
    lane_twiddle_mul<R, 1>(v, tw, lane);
    dft_regs<R, 1>(v);
}
