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
template <int DIR, typename T>
__device__ T* fft_lines(T* buf, T* tmp, int nl, int ld, const FftSched& s, const T* tw) {
    T* in = buf;
    T* out = tmp;
    int Ns = 1;
    for (int st = 0; st < s.ns; ++st) {
        const int R = s.radix[st];
        if (R == 8) fft_stage<8, DIR>(in, out, nl, ld, s.Q, Ns, tw);
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
