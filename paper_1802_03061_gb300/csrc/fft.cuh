// Shared-memory Stockham FFT (mixed radix 2/3/4/8), used by every pass kernel.
//
// A block transforms `nl` lines of length Q that sit in shared memory (line
// stride `ld` elements).  Each stage of radix R with Ns = product of the
// earlier radices maps butterfly j (0 <= j < Q/R) as
//     inputs   a[j + r Q/R],                      r = 0..R-1
//     twiddle  w^(r * (j mod Ns) * Q/(Ns R)),    w = exp(DIR 2 pi i / Q)
//     outputs  b[(j / Ns) Ns R + (j mod Ns) + r Ns]
// (the self-sorting Stockham autosort form), ping-ponging between two
// buffers.  Output is in natural order; no normalisation is applied.
// DIR = -1 is the forward transform exp(-2 pi i k x / Q), DIR = +1 the inverse.
#pragma once
#include "common.cuh"

template <int DIR, typename T> __device__ __forceinline__ T twid(const T* tw, int t) {
    T w = tw[t];                       // table holds exp(-2 pi i t / Q)
    return DIR < 0 ? w : cconj(w);
}

template <int DIR, typename T> __device__ __forceinline__ void bfly2(T* v) {
    T a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int DIR, typename T> __device__ __forceinline__ void bfly3(T* v) {
    using R = typename real_of<T>::R;
    const R c = (R)-0.5;
    const R s = (R)(DIR * 0.86602540378443864676372317075294);  // DIR * sin(2 pi / 3)
    T a0 = v[0], a1 = v[1], a2 = v[2];
    T sum = cadd(a1, a2), dif = csub(a1, a2);
    T t = mk<T>(a0.x + c * sum.x, a0.y + c * sum.y);
    T rot = mk<T>(-s * dif.y, s * dif.x);  // i * s * dif
    v[0] = cadd(a0, sum);
    v[1] = cadd(t, rot);
    v[2] = csub(t, rot);
}

template <int DIR, typename T> __device__ __forceinline__ void bfly4(T* v) {
    T s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    T s13 = cadd(v[1], v[3]), d13 = cmul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}

template <int DIR, typename T> __device__ __forceinline__ void bfly8(T* v) {
    using R = typename real_of<T>::R;
    const R r2 = (R)0.70710678118654752440084436210485;
    T e[4] = {v[0], v[2], v[4], v[6]};
    T o[4] = {v[1], v[3], v[5], v[7]};
    bfly4<DIR>(e);
    bfly4<DIR>(o);
    // o[k] *= w8^k, w8 = exp(DIR 2 pi i / 8) = (1 + DIR i)/sqrt2
    T o1 = mk<T>(r2 * (o[1].x - DIR * o[1].y), r2 * (o[1].y + DIR * o[1].x));
    T o2 = cmul_i<DIR>(o[2]);
    T o3 = mk<T>(r2 * (-o[3].x - DIR * o[3].y), r2 * (-o[3].y + DIR * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

// radix-8 butterfly whose inputs 4..7 are zero (zero-padded line, first stage)
template <int DIR, typename T> __device__ __forceinline__ void bfly8_half(T* v) {
    using R = typename real_of<T>::R;
    const R r2 = (R)0.70710678118654752440084436210485;
    // even part DFT4(v0, v2, 0, 0), odd part DFT4(v1, v3, 0, 0)
    const T e0 = cadd(v[0], v[2]), e2 = csub(v[0], v[2]);
    const T w2 = cmul_i<DIR>(v[2]);
    const T e1 = cadd(v[0], w2), e3 = csub(v[0], w2);
    const T o0 = cadd(v[1], v[3]), o2s = csub(v[1], v[3]);
    const T w3 = cmul_i<DIR>(v[3]);
    const T o1s = cadd(v[1], w3), o3s = csub(v[1], w3);
    const T o1 = mk<T>(r2 * (o1s.x - DIR * o1s.y), r2 * (o1s.y + DIR * o1s.x));
    const T o2 = cmul_i<DIR>(o2s);
    const T o3 = mk<T>(r2 * (-o3s.x - DIR * o3s.y), r2 * (-o3s.y + DIR * o3s.x));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

// First stage (Ns = 1) of a radix-8 schedule on lines whose entries at
// index >= Q/2 are zero (zero padding, n <= Q/2): inputs r = 4..7 are zero.
template <int DIR, typename T>
__device__ __forceinline__ void fft_stage8_first_half(const T* __restrict__ in, T* __restrict__ out, int nl, int ld,
                                                      int Q) {
    const int per = Q / 8;
    const int tot = nl * per;
    const bool p2 = (Q & (Q - 1)) == 0;
    const int lper = p2 ? __ffs(per) - 1 : 0;
    for (int job = threadIdx.x; job < tot; job += blockDim.x) {
        int line, j;
        if (p2) { line = job >> lper; j = job & (per - 1); }
        else { line = job / per; j = job - line * per; }
        const T* a = in + (long)line * ld;
        T* b = out + (long)line * ld;
        T v[8];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = a[j + r * per];
        bfly8_half<DIR>(v);
        const int d = j * 8;
#pragma unroll
        for (int r = 0; r < 8; ++r) b[d + r] = v[r];
    }
}

template <int R, int DIR, typename T>
__device__ __forceinline__ void fft_stage(const T* __restrict__ in, T* __restrict__ out, int nl, int ld,
                                          int Q, int Ns, const T* __restrict__ tw) {
    const int per = Q / R;
    const int tot = nl * per;
    const int step = Q / (Ns * R);
    // power-of-two lengths: index arithmetic by shifts and masks
    const bool p2 = (Q & (Q - 1)) == 0;
    const int lper = p2 ? __ffs(per) - 1 : 0;
    const int lns = p2 ? __ffs(Ns) - 1 : 0;
    for (int job = threadIdx.x; job < tot; job += blockDim.x) {
        int line, j, k, jq;
        if (p2) {
            line = job >> lper;
            j = job & (per - 1);
            k = j & (Ns - 1);
            jq = j >> lns;
        } else {
            line = job / per;
            j = job - line * per;
            jq = j / Ns;
            k = j - jq * Ns;
        }
        const T* a = in + (long)line * ld;
        T* b = out + (long)line * ld;
        T v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = a[j + r * per];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twid<DIR>(tw, r * k * step));
        }
        if (R == 2) bfly2<DIR>(v);
        if (R == 3) bfly3<DIR>(v);
        if (R == 4) bfly4<DIR>(v);
        if (R == 8) bfly8<DIR>(v);
        const int d = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) b[d + r * Ns] = v[r];
    }
}

// Runs all stages; returns the buffer (buf or tmp) that holds the result.
// Ends with a __syncthreads(); the caller must have synchronised before.
// half_zero: the entries at index >= Q/2 of every line are zero (prunes
// the first radix-8 stage).
template <int DIR, typename T>
__device__ T* fft_lines(T* buf, T* tmp, int nl, int ld, const FftSched& s, const T* tw, bool half_zero = false) {
    T* in = buf;
    T* out = tmp;
    int Ns = 1;
    for (int st = 0; st < s.ns; ++st) {
        const int R = s.radix[st];
        if (st == 0 && R == 8 && half_zero) fft_stage8_first_half<DIR>(in, out, nl, ld, s.Q);
        else if (R == 8) fft_stage<8, DIR>(in, out, nl, ld, s.Q, Ns, tw);
        else if (R == 4) fft_stage<4, DIR>(in, out, nl, ld, s.Q, Ns, tw);
        else if (R == 3) fft_stage<3, DIR>(in, out, nl, ld, s.Q, Ns, tw);
        else fft_stage<2, DIR>(in, out, nl, ld, s.Q, Ns, tw);
        __syncthreads();
        T* t = in; in = out; out = t;
        Ns *= R;
    }
    return in;
}

// Load the Q-entry twiddle table into shared memory.
template <typename T>
__device__ __forceinline__ void load_twiddles(T* sm, const T* __restrict__ g, int Q) {
    for (int i = threadIdx.x; i < Q; i += blockDim.x) sm[i] = g[i];
}
