// 2D operator passes: y = a*x + b*(K x) + c*z  (or b*(K~ g) for the RHS).
//
// The field u has modes k = 0..L with u_{-k} = conj(u_k); its 2L+1 real
// channels are Re u_0, Re u_k, Im u_k.  K is a translation-invariant
// convolution on the real channels (Sec. 3.3.1: per (k,k') the kernel only
// depends on x - y), so the passes are
//   1. row pass    : weight by mu_s sigma_hat_k, zero-pad each row to Q,
//                    complex FFT along x of u_k (k >= 1) or of two packed rows
//                    of u_0, split into the half spectra (xi_x = 0..Q/2) of
//                    the real channels; write T[c][xi_x][y] (y contiguous).
//   2. column pass : per xi_x: FFT along y of every channel (zero padded),
//                    per frequency the (2L+1)x(2L+1) mode mix with the
//                    spectra S_m, m = 0..2L (Sec. 3.3.1 remark: the kernel
//                    depends only on k - k'), inverse FFT, keep y < n.
//   3. inverse row : rebuild the full x spectrum of u_k = Re + i Im from the
//                    two half spectra, inverse FFT, keep x < n, epilogue.
//
// Mode mix.  With P_m = (S_m + S_{-m})/2, M_m = (S_m - S_{-m})/2 and
// S_{-m}(xi) = (-1)^m conj(S_m(xi)) (kappa real and even), the spectra of the
// real output channels are, for k = 0..L (A = spectrum of Re w, B of Im w,
// w_k = mu_s sigma_hat_k u_k):
//   Re v_k : P_k A_0 + sum_{k'=1..L} (P_{k-k'} + P_{k+k'}) A_k' + i (M_{k-k'} - M_{k+k'}) B_k'
//   Im v_k : -i M_k A_0 + sum_{k'} -i (M_{k-k'} + M_{k+k'}) A_k' + (P_{k-k'} - P_{k+k'}) B_k'
// For even m, P_m = Re S_m and M_m = i Im S_m; for odd m, P_m = i Im S_m and
// M_m = Re S_m; P_{-m} = P_m, M_{-m} = -M_m.  Every coefficient is therefore
// purely real or purely imaginary, known at compile time for fixed (k, k').
#pragma once
#include "fft.cuh"
#include "internal.h"
#include "wfft.cuh"

// channel index of Re u_k / Im u_k
__host__ __device__ __forceinline__ int chA(int k) { return k == 0 ? 0 : 2 * k - 1; }
__host__ __device__ __forceinline__ int chB(int k) { return 2 * k; }

struct RowParams {
    int n, Q, H, L, RB;
    FftSched sc;
    double wk[RTE_MAX_L + 1];  // per-mode input weight
};

// ---------------------------------------------------------------------------
// 1. forward row pass
//    x: [L+1][n][n] complex (may be null when f is given), f: real [n][n]
//    source that replaces the mode-0 input (RHS).  out: T [nch][H][n].
//    grid (ceil(n/RB), nmodes_in), block 256.
// ---------------------------------------------------------------------------
template <typename T, typename TF>
__global__ void __launch_bounds__(256) k_row_fwd(const TF* __restrict__ x, const double* __restrict__ f,
                                                 T* __restrict__ out, const T* __restrict__ tw, RowParams p) {
    using R = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, RB = p.RB;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * RB;
    const int nl = (k == 0) ? RB / 2 : RB;
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)RB * Q;
    load_twiddles(twl, tw, Q);
    const R w = (R)p.wk[k];
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int li = idx / Q, e = idx - li * Q;
        T v = mk<T>(0, 0);
        if (e < n) {
            if (k == 0) {
                const int ya = y0 + 2 * li, yb = ya + 1;
                R a = 0, b = 0;
                if (x) {
                    if (ya < n) a = w * (R)x[(long)ya * n + e].x;
                    if (yb < n) b = w * (R)x[(long)yb * n + e].x;
                }
                if (f) {  // the source joins unweighted (MIX_RHS: w = 1, no x)
                    if (ya < n) a = a + (R)f[(long)ya * n + e];
                    if (yb < n) b = b + (R)f[(long)yb * n + e];
                }
                v = mk<T>(a, b);
            } else {
                const int y = y0 + li;
                if (y < n) {
                    T u = to_c<T>(x[((long)k * n + y) * n + e]);
                    v = mk<T>(w * u.x, w * u.y);
                }
            }
        }
        buf[idx] = v;
    }
    __syncthreads();
    T* res = fft_lines<-1>(buf, tmp, nl, Q, p.sc, twl, 2 * n <= Q);
    // split Z = F + i G (F, G real rows) into their half spectra:
    //   F(xi) = (Z(xi) + conj Z(-xi))/2,  G(xi) = (Z(xi) - conj Z(-xi))/(2i)
    const int rows = (k == 0) ? RB : RB;
    for (int idx = threadIdx.x; idx < H * rows; idx += blockDim.x) {
        const int r = idx % rows, xi = idx / rows;
        const int y = y0 + r;
        if (y >= n) continue;
        int line, which, ch;
        if (k == 0) { line = r >> 1; which = r & 1; ch = 0; }
        else { line = r; which = -1; ch = -1; }
        const T Z = res[line * Q + xi];
        const T Zm = res[line * Q + (xi == 0 ? 0 : Q - xi)];
        const T Fv = mk<T>((R)0.5 * (Z.x + Zm.x), (R)0.5 * (Z.y - Zm.y));
        const T Gv = mk<T>((R)0.5 * (Z.y + Zm.y), (R)-0.5 * (Z.x - Zm.x));
        if (k == 0) {
            out[((long)ch * H + xi) * n + y] = which == 0 ? Fv : Gv;
        } else {
            out[((long)chA(k) * H + xi) * n + y] = Fv;
            out[((long)chB(k) * H + xi) * n + y] = Gv;
        }
    }
}

// ---------------------------------------------------------------------------
// 3. inverse row pass + epilogue  out = a*x + b*v + c*z
//    in: T [nch][H][n] (column-pass output), grid (ceil(n/RB), L+1)
// ---------------------------------------------------------------------------
template <typename T, typename TF>
__global__ void __launch_bounds__(256) k_row_inv(const T* __restrict__ in, const TF* __restrict__ x,
                                                 const TF* __restrict__ z, TF* __restrict__ out,
                                                 const T* __restrict__ tw, RowParams p,
                                                 typename real_of<T>::R a, typename real_of<T>::R b,
                                                 typename real_of<T>::R c) {
    using R = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, RB = p.RB;
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * RB;
    const int nl = (k == 0) ? RB / 2 : RB;
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)RB * Q;
    load_twiddles(twl, tw, Q);
    // Z(xi) = F(xi) + i G(xi); Z(Q-xi) = conj F(xi) + i conj G(xi)
    for (int idx = threadIdx.x; idx < H * nl; idx += blockDim.x) {
        const int li = idx % nl, xi = idx / nl;
        T Fv = mk<T>(0, 0), Gv = mk<T>(0, 0);
        if (k == 0) {
            const int ya = y0 + 2 * li, yb = ya + 1;
            if (ya < n) Fv = in[((long)0 * H + xi) * n + ya];
            if (yb < n) Gv = in[((long)0 * H + xi) * n + yb];
        } else {
            const int y = y0 + li;
            if (y < n) {
                Fv = in[((long)chA(k) * H + xi) * n + y];
                Gv = in[((long)chB(k) * H + xi) * n + y];
            }
        }
        buf[li * Q + xi] = mk<T>(Fv.x - Gv.y, Fv.y + Gv.x);
        if (xi > 0 && xi < Q - xi) buf[li * Q + (Q - xi)] = mk<T>(Fv.x + Gv.y, Gv.x - Fv.y);
    }
    __syncthreads();
    T* res = fft_lines<1>(buf, tmp, nl, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < nl * n; idx += blockDim.x) {
        const int li = idx / n, e = idx - li * n;
        const T v = res[li * Q + e];
        if (k == 0) {
            const int ya = y0 + 2 * li, yb = ya + 1;
            if (ya < n) {
                const long o = (long)ya * n + e;
                T r = mk<T>(b * v.x, (R)0);
                if (x) { const T xv = to_c<T>(x[o]); r.x += a * xv.x; r.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); r.x += c * zv.x; r.y += c * zv.y; }
                out[o] = to_f<TF>(r);
            }
            if (yb < n) {
                const long o = (long)yb * n + e;
                T r = mk<T>(b * v.y, (R)0);
                if (x) { const T xv = to_c<T>(x[o]); r.x += a * xv.x; r.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); r.x += c * zv.x; r.y += c * zv.y; }
                out[o] = to_f<TF>(r);
            }
        } else {
            const int y = y0 + li;
            if (y < n) {
                const long o = ((long)k * n + y) * n + e;
                T r = mk<T>(b * v.x, b * v.y);
                if (x) { const T xv = to_c<T>(x[o]); r.x += a * xv.x; r.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); r.x += c * zv.x; r.y += c * zv.y; }
                out[o] = to_f<TF>(r);
            }
        }
    }
}

// The inverse warp row passes' first step: the half spectra of the block's 8
// lines (mode k, rows from y0) into the line buffer Z as full spectra,
// Z(xi) = F(xi) + i G(xi), Z(Q - xi) = conj F(xi) + i conj G(xi).  H = Q/2 + 1
// is fixed by R, so each thread's trip count is a compile-time constant: all
// of its loads are issued before the first write to Z and their latencies
// overlap (a loop with a run-time bound waited for each load in turn).
// Block of 256 threads; line stride LS = Q + 34.
template <int R, typename T>
__device__ __forceinline__ void rebuild_lines(const T* __restrict__ in, T* __restrict__ Z, int k, int y0, int n,
                                              int H) {
    constexpr int Q = 32 * R, LS = Q + 34, HH = Q / 2 + 1, NT = 256;
    constexpr int IT = (HH * 8 + NT - 1) / NT;
    T F[IT], G[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int idx = threadIdx.x + it * NT;
        const int li = idx & 7, xi = idx >> 3;
        T Fv = mk<T>(0, 0), Gv = mk<T>(0, 0);
        if (idx < HH * 8) {
            if (k == 0) {
                const int ya = y0 + 2 * li, yb = ya + 1;
                if (ya < n) Fv = in[(long)xi * n + ya];
                if (yb < n) Gv = in[(long)xi * n + yb];
            } else {
                const int y = y0 + li;
                if (y < n) {
                    Fv = in[((long)chA(k) * H + xi) * n + y];
                    Gv = in[((long)chB(k) * H + xi) * n + y];
                }
            }
        }
        F[it] = Fv;
        G[it] = Gv;
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
        const int idx = threadIdx.x + it * NT;
        if (idx >= HH * 8) continue;
        const int li = idx & 7, xi = idx >> 3;
        const T Fv = F[it], Gv = G[it];
        Z[li * LS + swz16(xi)] = mk<T>(Fv.x - Gv.y, Fv.y + Gv.x);
        if (xi > 0 && xi < Q - xi) Z[li * LS + swz16(Q - xi)] = mk<T>(Fv.x + Gv.y, Gv.x - Fv.y);
    }
}

// ---------------------------------------------------------------------------
// 1w/3w. row passes with the warp FFT (Q = 32 R; FP32 or float-float compute
// T, field storage TF): one warp per line (a row of u_k, or two packed rows
// of u_0), 8 lines per block.  The transform stays in registers; shared
// memory holds each warp's FFT scratch and then the spectra of the block's
// lines (swizzled) for the half-spectrum split / rebuild, which keep the same
// y-contiguous global layout as the generic passes.
// grid (ceil(n / 8), modes), block 256; rows per block 8 (k >= 1) or 16 (k = 0)
// ---------------------------------------------------------------------------
template <int R, typename T, typename TF>
__global__ void __launch_bounds__(256) k_row_fwd_warp(const TF* __restrict__ x, const double* __restrict__ f,
                                                      T* __restrict__ out, const T* __restrict__ tw, RowParams p) {
    using RR = typename real_of<T>::R;
    constexpr int Q = 32 * R;
    // line stride: holds the FFT scratch (Q + 32), consecutive lines 2 bank pairs apart
    constexpr int LS = Q + 34;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Z = twl + Q;
    const int n = p.n, H = p.H;
    const int k = blockIdx.y;
    const int rows = k == 0 ? 16 : 8;
    const int y0 = blockIdx.x * rows;
    if (y0 >= n) return;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    pdl_wait();  // x may be the predecessor's output
    pdl_trigger();
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RR wt = (RR)p.wk[k];
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = lane + 32 * r;
        T val = mk<T>(0, 0);
        if (e < n) {
            if (k == 0) {
                const int ya = y0 + 2 * w, yb = ya + 1;
                RR a = (RR)0, b = (RR)0;
                if (x) {
                    if (ya < n) a = wt * to_c<T>(x[(long)ya * n + e]).x;
                    if (yb < n) b = wt * to_c<T>(x[(long)yb * n + e]).x;
                }
                if (f) {  // the source joins unweighted (MIX_RHS: no x)
                    if (ya < n) a = a + (RR)f[(long)ya * n + e];
                    if (yb < n) b = b + (RR)f[(long)yb * n + e];
                }
                val = mk<T>(a, b);
            } else {
                const int y = y0 + w;
                if (y < n) {
                    const T u = to_c<T>(x[((long)k * n + y) * n + e]);
                    val = mk<T>(wt * u.x, wt * u.y);
                }
            }
        }
        v[r] = val;
    }
    warp_fft_fwd<R>(v, twl, Z + w * LS);  // the line doubles as the FFT scratch
#pragma unroll
    for (int j = 0; j < R; ++j) Z[w * LS + swz16(wfreq<R>(j, lane))] = v[j];
    __syncthreads();
    // split Z = F + i G into the half spectra (as in k_row_fwd)
    for (int idx = threadIdx.x; idx < H * rows; idx += blockDim.x) {
        const int r = idx % rows, xi = idx / rows;
        const int y = y0 + r;
        if (y >= n) continue;
        const int line = k == 0 ? r >> 1 : r;
        const T Zp = Z[line * LS + swz16(xi)];
        const T Zm = Z[line * LS + swz16(xi == 0 ? 0 : Q - xi)];
        const T Fv = mk<T>((RR)0.5 * (Zp.x + Zm.x), (RR)0.5 * (Zp.y - Zm.y));
        const T Gv = mk<T>((RR)0.5 * (Zp.y + Zm.y), (RR)-0.5 * (Zp.x - Zm.x));
        if (k == 0) {
            out[(long)xi * n + y] = (r & 1) ? Gv : Fv;
        } else {
            out[((long)chA(k) * H + xi) * n + y] = Fv;
            out[((long)chB(k) * H + xi) * n + y] = Gv;
        }
    }
}

template <int R, typename T, typename TF>
__global__ void __launch_bounds__(256, 2) k_row_inv_warp(const T* __restrict__ in, const TF* __restrict__ x,
                                                      const TF* __restrict__ z, TF* __restrict__ out,
                                                      const T* __restrict__ tw, RowParams p,
                                                      typename real_of<T>::R a, typename real_of<T>::R b,
                                                      typename real_of<T>::R c) {
    using RR = typename real_of<T>::R;
    constexpr int Q = 32 * R;
    constexpr int LS = Q + 34;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Z = twl + Q;
    const int n = p.n, H = p.H;
    const int k = blockIdx.y;
    const int rows = k == 0 ? 16 : 8;
    const int y0 = blockIdx.x * rows;
    if (y0 >= n) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the epilogue's x values (mode 0: rows ya, yb; mode k: row y), loaded
    // before the transform so that their latency overlaps it: n <= Q/2, so
    // only registers r < R/2 hold x < n
    constexpr int RH = R / 2;
    TF px0[RH], px1[RH];
    {
        const int ya = k == 0 ? y0 + 2 * w : y0 + w, yb = ya + 1;
        const long ra = k == 0 ? (long)ya * n : ((long)k * n + ya) * n, rb = (long)yb * n;
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int e = lane + 32 * r;
            px0[r] = (x && e < n && ya < n) ? x[ra + e] : TF{};
            px1[r] = (x && k == 0 && e < n && yb < n) ? x[rb + e] : TF{};
        }
    }
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    pdl_wait();  // in: the column pass's output
    pdl_trigger();
    rebuild_lines<R, T>(in, Z, k, y0, n, H);
    __syncthreads();
    T v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = Z[w * LS + swz16(wfreq<R>(j, lane))];
    __syncwarp();
    warp_fft_inv<R>(v, twl, Z + w * LS);
#pragma unroll
    for (int r = 0; r < RH; ++r) {
        const int e = lane + 32 * r;
        if (e >= n) continue;
        if (k == 0) {
            const int ya = y0 + 2 * w, yb = ya + 1;
            if (ya < n) {
                const long o = (long)ya * n + e;
                T q = mk<T>(b * v[r].x, (RR)0);
                if (x) { const T xv = to_c<T>(px0[r]); q.x += a * xv.x; q.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); q.x += c * zv.x; q.y += c * zv.y; }
                out[o] = to_f<TF>(q);
            }
            if (yb < n) {
                const long o = (long)yb * n + e;
                T q = mk<T>(b * v[r].y, (RR)0);
                if (x) { const T xv = to_c<T>(px1[r]); q.x += a * xv.x; q.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); q.x += c * zv.x; q.y += c * zv.y; }
                out[o] = to_f<TF>(q);
            }
        } else {
            const int y = y0 + w;
            if (y < n) {
                const long o = ((long)k * n + y) * n + e;
                T q = mk<T>(b * v[r].x, b * v[r].y);
                if (x) { const T xv = to_c<T>(px0[r]); q.x += a * xv.x; q.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); q.x += c * zv.x; q.y += c * zv.y; }
                out[o] = to_f<TF>(q);
            }
        }
    }
}

// Row passes as two warp FFTs of half the length (residues r = xi mod 2, n <=
// Q/2 nonzero inputs, as k_col_warp2): FP32 at Q = 1024 (R = 16, both
// passes) and the float-float forward pass at Q = 512 (R = 8, where a
// one-warp 512-point float-float line needs too many registers).  The line buffer Z holds the Q-point spectrum
// (swizzled) for the half-spectrum split / rebuild, and each warp has a
// separate FFT scratch.  tw: the plan's Q-point table (compute type T, field
// storage TF).
// grid (ceil(n / 8), modes), block 256; rows per block 8 (k >= 1) or 16 (k = 0)
// input register r of the two-residue forward row pass (weighted field of
// mode k, the source joining mode 0 unweighted, two packed rows for k = 0)
template <typename T, typename TF>
__device__ __forceinline__ T row2_input(const TF* __restrict__ x, const double* __restrict__ f, int k, int y0,
                                        int w, int e, int n, typename real_of<T>::R wt) {
    using RR = typename real_of<T>::R;
    T val = mk<T>(0, 0);
    if (e < n) {
        if (k == 0) {
            const int ya = y0 + 2 * w, yb = ya + 1;
            RR a = (RR)0, b = (RR)0;
            if (x) {
                if (ya < n) a = wt * to_c<T>(x[(long)ya * n + e]).x;
                if (yb < n) b = wt * to_c<T>(x[(long)yb * n + e]).x;
            }
            if (f) {
                if (ya < n) a = a + (RR)f[(long)ya * n + e];
                if (yb < n) b = b + (RR)f[(long)yb * n + e];
            }
            val = mk<T>(a, b);
        } else {
            const int y = y0 + w;
            if (y < n) {
                const T uu = to_c<T>(x[((long)k * n + y) * n + e]);
                val = mk<T>(wt * uu.x, wt * uu.y);
            }
        }
    }
    return val;
}

template <int R, typename T, typename TF>
__global__ void __launch_bounds__(256) k_row_fwd_warp2(const TF* __restrict__ x, const double* __restrict__ f,
                                                       T* __restrict__ out, const T* __restrict__ tw,
                                                       RowParams p) {
    using RR = typename real_of<T>::R;
    constexpr int QW = 32 * R, Q = 2 * QW, LS = Q + 2;
    constexpr int SC = wfft_shape<R>::SCRATCH;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);  // exp(-2 pi i t / QW)
    T* Z = twl + QW;                       // [8][LS]
    T* scr = Z + 8 * LS;                   // [8][SC]
    const int n = p.n, H = p.H;
    const int k = blockIdx.y;
    const int rows = k == 0 ? 16 : 8;
    const int y0 = blockIdx.x * rows;
    if (y0 >= n) return;
    for (int i = threadIdx.x; i < QW; i += blockDim.x) twl[i] = tw[2 * i];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RR wt = (RR)p.wk[k];
    // FP32 (R = 16) loads its inputs again for the second residue (cache hits)
    // rather than holding them across the first transform: 128 registers
    // instead of 154, two blocks per SM.  Float-float keeps them (reloading
    // its FP64 fields measured slower: 28.8 -> 35.0 us at Q = 512).
    constexpr bool RELOAD = sizeof(T) == 8;
    T u[RELOAD ? 1 : R];
    if constexpr (!RELOAD) {
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = row2_input<T>(x, f, k, y0, w, lane + 32 * r, n, wt);
    }
    for (int rs = 0; rs < 2; ++rs) {
        T v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = lane + 32 * r;
            T val;
            if constexpr (RELOAD) val = row2_input<T>(x, f, k, y0, w, e, n, wt);
            else val = u[r];
            v[r] = (rs && e < n) ? cmul(val, tw[e]) : val;
        }
        warp_fft_fwd<R>(v, twl, scr + w * SC);
#pragma unroll
        for (int j = 0; j < R; ++j) Z[w * LS + swz16(2 * wfreq<R>(j, lane) + rs)] = v[j];
        __syncwarp();
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < H * rows; idx += blockDim.x) {
        const int r = idx % rows, xi = idx / rows;
        const int y = y0 + r;
        if (y >= n) continue;
        const int line = k == 0 ? r >> 1 : r;
        const T Zp = Z[line * LS + swz16(xi)];
        const T Zm = Z[line * LS + swz16(xi == 0 ? 0 : Q - xi)];
        const T Fv = mk<T>((RR)0.5 * (Zp.x + Zm.x), (RR)0.5 * (Zp.y - Zm.y));
        const T Gv = mk<T>((RR)0.5 * (Zp.y + Zm.y), (RR)-0.5 * (Zp.x - Zm.x));
        if (k == 0) {
            out[(long)xi * n + y] = (r & 1) ? Gv : Fv;
        } else {
            out[((long)chA(k) * H + xi) * n + y] = Fv;
            out[((long)chB(k) * H + xi) * n + y] = Gv;
        }
    }
}

template <int R, typename T, typename TF>
__global__ void __launch_bounds__(256) k_row_inv_warp2(const T* __restrict__ in, const TF* __restrict__ x,
                                                       const TF* __restrict__ z, TF* __restrict__ out,
                                                       const T* __restrict__ tw, RowParams p,
                                                       typename real_of<T>::R a, typename real_of<T>::R b,
                                                       typename real_of<T>::R c) {
    using RR = typename real_of<T>::R;
    constexpr int QW = 32 * R, Q = 2 * QW, LS = Q + 2;
    constexpr int SC = wfft_shape<R>::SCRATCH;
    extern __shared__ unsigned char smraw[];
    T* twl = reinterpret_cast<T*>(smraw);
    T* Z = twl + QW;
    T* scr = Z + 8 * LS;
    const int n = p.n, H = p.H;
    const int k = blockIdx.y;
    const int rows = k == 0 ? 16 : 8;
    const int y0 = blockIdx.x * rows;
    if (y0 >= n) return;
    for (int i = threadIdx.x; i < QW; i += blockDim.x) twl[i] = tw[2 * i];
    // the half spectra in groups of four elements per thread whose loads are
    // all issued before their writes to Z (H = Q/2 + 1 is fixed by R)
    constexpr int HH = Q / 2 + 1, NT = 256, IT = (HH * 8 + NT - 1) / NT, CH = 4;
#pragma unroll 1
    for (int i0 = 0; i0 < IT; i0 += CH) {
        T F[CH], G[CH];
#pragma unroll
        for (int g = 0; g < CH; ++g) {
            const int idx = threadIdx.x + (i0 + g) * NT;
            const int li = idx & 7, xi = idx >> 3;
            T Fv = mk<T>(0, 0), Gv = mk<T>(0, 0);
            if (idx < HH * 8) {
                if (k == 0) {
                    const int ya = y0 + 2 * li, yb = ya + 1;
                    if (ya < n) Fv = in[(long)xi * n + ya];
                    if (yb < n) Gv = in[(long)xi * n + yb];
                } else {
                    const int y = y0 + li;
                    if (y < n) {
                        Fv = in[((long)chA(k) * H + xi) * n + y];
                        Gv = in[((long)chB(k) * H + xi) * n + y];
                    }
                }
            }
            F[g] = Fv;
            G[g] = Gv;
        }
#pragma unroll
        for (int g = 0; g < CH; ++g) {
            const int idx = threadIdx.x + (i0 + g) * NT;
            if (idx >= HH * 8) continue;
            const int li = idx & 7, xi = idx >> 3;
            const T Fv = F[g], Gv = G[g];
            Z[li * LS + swz16(xi)] = mk<T>(Fv.x - Gv.y, Fv.y + Gv.x);
            if (xi > 0 && xi < Q - xi) Z[li * LS + swz16(Q - xi)] = mk<T>(Fv.x + Gv.y, Gv.x - Fv.y);
        }
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T acc[R];
    for (int rs = 0; rs < 2; ++rs) {
        T v[R];
#pragma unroll
        for (int j = 0; j < R; ++j) v[j] = Z[w * LS + swz16(2 * wfreq<R>(j, lane) + rs)];
        warp_fft_inv<R>(v, twl, scr + w * SC);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = lane + 32 * r;
            if (rs == 0) acc[r] = v[r];
            else if (e < n) acc[r] = cadd(acc[r], cmul(v[r], cconj(tw[e])));
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = lane + 32 * r;
        if (e >= n) continue;
        if (k == 0) {
            const int ya = y0 + 2 * w, yb = ya + 1;
            if (ya < n) {
                const long o = (long)ya * n + e;
                T q = mk<T>(b * acc[r].x, (RR)0);
                if (x) { const T xv = to_c<T>(x[o]); q.x += a * xv.x; q.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); q.x += c * zv.x; q.y += c * zv.y; }
                out[o] = to_f<TF>(q);
            }
            if (yb < n) {
                const long o = (long)yb * n + e;
                T q = mk<T>(b * acc[r].y, (RR)0);
                if (x) { const T xv = to_c<T>(x[o]); q.x += a * xv.x; q.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); q.x += c * zv.x; q.y += c * zv.y; }
                out[o] = to_f<TF>(q);
            }
        } else {
            const int y = y0 + w;
            if (y < n) {
                const long o = ((long)k * n + y) * n + e;
                T q = mk<T>(b * acc[r].x, b * acc[r].y);
                if (x) { const T xv = to_c<T>(x[o]); q.x += a * xv.x; q.y += a * xv.y; }
                if (z) { const T zv = to_c<T>(z[o]); q.x += c * zv.x; q.y += c * zv.y; }
                out[o] = to_f<TF>(q);
            }
        }
    }
}

// The preconditioned inner step applies M and then K to M's output.  The
// inverse row pass of M and the forward row pass of K touch the same rows of
// the same mode k and nothing else, so one kernel does both (FP32): rebuild
// the row spectra from the column pass's half spectra, inverse warp FFT,
// out = x + v (M's output, also K's input and the identity term of A later),
// then out weighted by mu_s sigma_hat_k, forward warp FFT, and the half
// spectra back into Tb (in place: a block reads and writes only its rows).
// grid (ceil(n / 8), L+1), block 256; rows per block 8 (k >= 1) or 16 (k = 0)
template <int R>
__global__ void __launch_bounds__(256) k_row_invfwd_warp(float2* __restrict__ Tb, const float2* __restrict__ x,
                                                         float2* __restrict__ out, const float2* __restrict__ tw,
                                                         RowParams p) {
    constexpr int Q = 32 * R;
    constexpr int LS = Q + 34;
    extern __shared__ unsigned char smraw[];
    float2* twl = reinterpret_cast<float2*>(smraw);
    float2* Z = twl + Q;
    const int n = p.n, H = p.H;
    const int k = blockIdx.y;
    const int rows = k == 0 ? 16 : 8;
    const int y0 = blockIdx.x * rows;
    if (y0 >= n) return;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    pdl_wait();  // Tb: the column pass's output
    pdl_trigger();
    // M: Z(xi) = F(xi) + i G(xi); Z(Q-xi) = conj F(xi) + i conj G(xi)
    rebuild_lines<R, float2>(Tb, Z, k, y0, n, H);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = Z[w * LS + swz16(wfreq<R>(j, lane))];
    __syncwarp();
    warp_fft_inv<R>(v, twl, Z + w * LS);
    // out = x + v, and K's weighted input in v (zero beyond the n cells)
    const float wt = (float)p.wk[k];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = lane + 32 * r;
        float2 nv = make_float2(0.f, 0.f);
        if (e < n) {
            if (k == 0) {
                const int ya = y0 + 2 * w, yb = ya + 1;
                float qa = 0.f, qb = 0.f;
                if (ya < n) {
                    const long o = (long)ya * n + e;
                    const float2 xv = x[o];
                    const float2 q = make_float2(v[r].x + xv.x, xv.y);
                    out[o] = q;
                    qa = q.x;
                }
                if (yb < n) {
                    const long o = (long)yb * n + e;
                    const float2 xv = x[o];
                    const float2 q = make_float2(v[r].y + xv.x, xv.y);
                    out[o] = q;
                    qb = q.x;
                }
                nv = make_float2(wt * qa, wt * qb);
            } else {
                const int y = y0 + w;
                if (y < n) {
                    const long o = ((long)k * n + y) * n + e;
                    const float2 xv = x[o];
                    const float2 q = make_float2(v[r].x + xv.x, v[r].y + xv.y);
                    out[o] = q;
                    nv = make_float2(wt * q.x, wt * q.y);
                }
            }
        }
        v[r] = nv;
    }
    __syncwarp();
    // K: forward warp FFT of the weighted row(s), half spectra back into Tb
    warp_fft_fwd<R>(v, twl, Z + w * LS);
#pragma unroll
    for (int j = 0; j < R; ++j) Z[w * LS + swz16(wfreq<R>(j, lane))] = v[j];
    __syncthreads();
    for (int idx = threadIdx.x; idx < H * rows; idx += blockDim.x) {
        const int r = idx % rows, xi = idx / rows;
        const int y = y0 + r;
        if (y >= n) continue;
        const int line = k == 0 ? r >> 1 : r;
        const float2 Zp = Z[line * LS + swz16(xi)];
        const float2 Zm = Z[line * LS + swz16(xi == 0 ? 0 : Q - xi)];
        const float2 Fv = make_float2(0.5f * (Zp.x + Zm.x), 0.5f * (Zp.y - Zm.y));
        const float2 Gv = make_float2(0.5f * (Zp.y + Zm.y), -0.5f * (Zp.x - Zm.x));
        if (k == 0) {
            Tb[(long)xi * n + y] = (r & 1) ? Gv : Fv;
        } else {
            Tb[((long)chA(k) * H + xi) * n + y] = Fv;
            Tb[((long)chB(k) * H + xi) * n + y] = Gv;
        }
    }
}

// ---------------------------------------------------------------------------
// 2. mode mix at one frequency: X[c] (in) -> X[c] (out), tagged coefficients
// ---------------------------------------------------------------------------
// acc += s * v  (im == false)   or   acc += (i s) * v  (im == true)
template <typename T>
__device__ __forceinline__ void tmac(T& acc, typename real_of<T>::R s, bool im, T v) {
    if (im) { acc.x -= s * v.y; acc.y += s * v.x; }
    else { acc.x += s * v.x; acc.y += s * v.y; }
}

// in / outv: T* or any indexable that yields T / T& (a strided view of
// global or shared memory)
// sr / si: the real / imaginary parts of S_m, m = 0..2L, as arrays or any
// indexable yielding R.  Only the outputs k with k % kmod == kres are formed
// (several threads may share one frequency).
template <int L, typename T, typename SR, typename SI, typename I, typename O>
__device__ __forceinline__ void mode_mix(const SR& sr, const SI& si, I&& in, O&& outv, int kmod = 1, int kres = 0) {
    using R = typename real_of<T>::R;
    // P(m): value, imag flag ; M(m): value, imag flag (m may be negative)
#define PV(m) ((((m) < 0 ? -(m) : (m)) & 1) ? si[(m) < 0 ? -(m) : (m)] : sr[(m) < 0 ? -(m) : (m)])
#define PI_(m) ((((m) < 0 ? -(m) : (m)) & 1) != 0)
#define MV_(m) ((((m) < 0 ? -(m) : (m)) & 1) ? sr[(m) < 0 ? -(m) : (m)] : si[(m) < 0 ? -(m) : (m)])
#define MV(m) ((m) < 0 ? -MV_(m) : MV_(m))
#define MI_(m) ((((m) < 0 ? -(m) : (m)) & 1) == 0)
#pragma unroll
    for (int k = 0; k <= L; ++k) {
        if (k % kmod != kres) continue;
        T Ra = mk<T>(0, 0), Ia = mk<T>(0, 0);
        const T A0 = in[0];
        tmac(Ra, PV(k), PI_(k), A0);
        // -i * M(k):  M imag (k even): -i * i m = m (real) ; M real (k odd): -i m (imag, -m)
        if (MI_(k)) tmac(Ia, MV(k), false, A0);
        else tmac(Ia, -MV(k), true, A0);
#pragma unroll
        for (int kp = 1; kp <= L; ++kp) {
            const T A = in[chA(kp)], B = in[chB(kp)];
            const int d = k - kp, s = k + kp;
            // (P_d + P_s) A   (P_d, P_s share parity)
            tmac(Ra, PV(d) + PV(s), PI_(d), A);
            // i (M_d - M_s) B
            {
                const R vm = MV(d) - MV(s);
                if (MI_(d)) tmac(Ra, -vm, false, B);  // i * (i vm) = -vm
                else tmac(Ra, vm, true, B);
            }
            // -i (M_d + M_s) A
            {
                const R vm = MV(d) + MV(s);
                if (MI_(d)) tmac(Ia, vm, false, A);   // -i * (i vm) = vm
                else tmac(Ia, -vm, true, A);
            }
            // (P_d - P_s) B
            tmac(Ia, PV(d) - PV(s), PI_(d), B);
        }
        outv[chA(k)] = Ra;
        if (k > 0) outv[chB(k)] = Ia;
    }
#undef PV
#undef PI_
#undef MV
#undef MV_
#undef MI_
}

// the mode mix when only A_0 is nonzero (right-hand side K~ g):
//   Re v_k = P_k A_0,  Im v_k = -i M_k A_0
template <int L, typename T, typename O>
__device__ __forceinline__ void mode_mix_rhs(const typename real_of<T>::R* sr, const typename real_of<T>::R* si,
                                             T A0, O&& outv) {
#pragma unroll
    for (int k = 0; k <= L; ++k) {
        T Ra = mk<T>(0, 0), Ia = mk<T>(0, 0);
        if (k & 1) {
            tmac(Ra, si[k], true, A0);   // P_k = i Im S_k
            tmac(Ia, -sr[k], true, A0);  // -i M_k, M_k = Re S_k
        } else {
            tmac(Ra, sr[k], false, A0);  // P_k = Re S_k
            tmac(Ia, si[k], false, A0);  // -i M_k = -i (i Im S_k) = Im S_k
        }
        outv[chA(k)] = Ra;
        if (k > 0) outv[chB(k)] = Ia;
    }
}

// a view of channel c at base[c * stride]
template <typename T> struct Strided {
    T* base;
    long stride;
    __device__ __forceinline__ T& operator[](int c) const { return base[c * stride]; }
};

struct ColParams {
    int n, Q, H, L, nin, G;   // nin: input channels (nch for K, 1 for the RHS)
    FftSched sc;
};

// load S_m(xi_x, xi_y), m = 0..2L, into (sr, si)
template <int L, typename T, typename TS>
__device__ __forceinline__ void load_spec(const TS* __restrict__ S, int kx, int ky, int Q,
                                          typename real_of<T>::R* sr, typename real_of<T>::R* si) {
#pragma unroll
    for (int m = 0; m <= 2 * L; ++m) {
        const T v = ld_spec(S, ((long)kx * (2 * L + 1) + m) * Q + ky, T());
        sr[m] = v.x;
        si[m] = v.y;
    }
}

// channels [c0, c0+cnt) of X (line stride Q) through an FFT, result left in X
template <int DIR, typename T>
__device__ void fft_channels(T* X, T* tmp, int c0, int cnt, int G, const FftSched& sc, const T* twl,
                             bool half_zero = false) {
    const int Q = sc.Q;
    for (int g0 = c0; g0 < c0 + cnt; g0 += G) {
        const int nl = min(G, c0 + cnt - g0);
        T* res = fft_lines<DIR>(X + (long)g0 * Q, tmp, nl, Q, sc, twl, half_zero);
        if (res != X + (long)g0 * Q) {
            for (int i = threadIdx.x; i < nl * Q; i += blockDim.x) X[(long)g0 * Q + i] = res[i];
            __syncthreads();
        }
    }
}

// fused column pass, one block per xi_x; T is updated in place
template <int L, typename T, typename TS>
__global__ void __launch_bounds__(256) k_col_fused(T* __restrict__ Tb, const TS* __restrict__ S,
                                                   const T* __restrict__ tw, ColParams p) {
    constexpr int NCH = 2 * L + 1;
    using R = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H;
    const int kx = blockIdx.x;
    T* twl = sm;
    T* X = sm + Q;
    T* tmp = X + (long)NCH * Q;
    load_twiddles(twl, tw, Q);
    for (int idx = threadIdx.x; idx < p.nin * Q; idx += blockDim.x) {
        const int c = idx / Q, e = idx - c * Q;
        X[idx] = e < n ? Tb[((long)c * H + kx) * n + e] : mk<T>(0, 0);
    }
    __syncthreads();
    fft_channels<-1>(X, tmp, 0, p.nin, p.G, p.sc, twl, 2 * n <= Q);
    if (p.nin == 1) {
        // right-hand side: only the mode-0 channel is nonzero
        for (int ky = threadIdx.x; ky < Q; ky += blockDim.x) {
            R sr[2 * L + 1], si[2 * L + 1];
            load_spec<L, T>(S, kx, ky, Q, sr, si);
            T o[NCH];
            mode_mix_rhs<L, T>(sr, si, X[ky], o);
#pragma unroll
            for (int c = 0; c < NCH; ++c) X[(long)c * Q + ky] = o[c];
        }
    } else {
        for (int ky = threadIdx.x; ky < Q; ky += blockDim.x) {
            R sr[2 * L + 1], si[2 * L + 1];
            load_spec<L, T>(S, kx, ky, Q, sr, si);
            T in[NCH], o[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c) in[c] = X[(long)c * Q + ky];
            mode_mix<L, T>(sr, si, in, o);
#pragma unroll
            for (int c = 0; c < NCH; ++c) X[(long)c * Q + ky] = o[c];
        }
    }
    __syncthreads();
    fft_channels<1>(X, tmp, 0, NCH, p.G, p.sc, twl);
    for (int idx = threadIdx.x; idx < NCH * n; idx += blockDim.x) {
        const int c = idx / n, e = idx - c * n;
        Tb[((long)c * H + kx) * n + e] = X[(long)c * Q + e];
    }
}

// split column pass (when all channels of a column do not fit in shared
// memory): per xi_x FFT channel groups between Tb [nch][H][n] and the full
// column spectra Ts [nch][H][Q]; the mix runs pointwise on Ts.
template <typename T>
__global__ void __launch_bounds__(256) k_col_fft_split(T* __restrict__ Tb, T* __restrict__ Ts,
                                                       const T* __restrict__ tw, ColParams p, int fwd,
                                                       int nchan) {
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, G = p.G;
    const int kx = blockIdx.x;
    T* twl = sm;
    T* X = sm + Q;
    T* tmp = X + (long)G * Q;
    load_twiddles(twl, tw, Q);
    for (int c0 = 0; c0 < nchan; c0 += G) {
        const int nl = min(G, nchan - c0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
            const int c = c0 + idx / Q, e = idx % Q;
            T v;
            if (fwd) v = e < n ? Tb[((long)c * H + kx) * n + e] : mk<T>(0, 0);
            else v = Ts[((long)c * H + kx) * Q + e];
            X[idx] = v;
        }
        __syncthreads();
        T* res = fwd ? fft_lines<-1>(X, tmp, nl, Q, p.sc, twl) : fft_lines<1>(X, tmp, nl, Q, p.sc, twl);
        for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
            const int c = c0 + idx / Q, e = idx % Q;
            if (fwd) Ts[((long)c * H + kx) * Q + e] = res[idx];
            else if (e < n) Tb[((long)c * H + kx) * n + e] = res[idx];
        }
    }
}

// ---------------------------------------------------------------------------
// Mode coupling by FFTs along the mode axis (large L).  The kernel of the pair
// (k, k') depends only on k - k' (Sec. 3.3.1 remark), so per frequency xi
//   V_k = sum_{k'=-L..L} S_{k-k'} W_k',   k = -L..L,
// is a linear convolution in the mode index.  With the inputs W_k' placed at
// k' mod P and S_m at m mod P (m = -2L..2L), a circular convolution of length
// P >= 4L+1 gives exactly these V_k (all needed differences k - k' are
// distinct mod P): V = iDFT_P(DFT_P(S) DFT_P(W)), with DFT_P(S)/P precomputed
// per frequency (Sm).  The complex modes come from the real channels' column
// spectra A_k (Re w_k), B_k (Im w_k): W_{+-k} = A_k +- i B_k, and the real
// output channels are Re v_k: (V_k + V_-k)/2, Im v_k: (V_k - V_-k)/(2i).
// Cost per frequency O(P log P) against (2L+1)^2 for the direct mix.
// One block handles MF_LINES consecutive frequencies id = xi_x Q + xi_y of Ts
// ([nch][H][Q], channel stride H Q), in place.
// ---------------------------------------------------------------------------
#define MF_LINES 16

struct ModeFftParams {
    int L, P, nin;   // nin: input channels (nch, or 1 for the right-hand side)
    long nfreq;      // H * Q
    FftSched sc;     // schedule of length P
};

template <typename T> __device__ __forceinline__ T half_c(T v) { return cscale(v, (typename real_of<T>::R)0.5); }

template <typename T, typename TS>
__global__ void __launch_bounds__(256) k_mix_modefft(T* __restrict__ Ts, const TS* __restrict__ Sm,
                                                     const T* __restrict__ twm, ModeFftParams p) {
    extern __shared__ unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int P = p.P, L = p.L;
    T* twl = sm;
    T* buf = sm + P;
    T* tmp = buf + MF_LINES * P;
    load_twiddles(twl, twm, P);
    const long f0 = (long)blockIdx.x * MF_LINES;
    const long rem = p.nfreq - f0;
    const int nf = rem < MF_LINES ? (int)rem : MF_LINES;
    const long cs = p.nfreq;
    for (int i = threadIdx.x; i < MF_LINES * P; i += blockDim.x) buf[i] = mk<T>(0, 0);
    __syncthreads();
    // gather W_{+-k} of each frequency (consecutive threads: consecutive frequencies)
    const int kin = p.nin > 1 ? L : 0;
    for (int i = threadIdx.x; i < (kin + 1) * MF_LINES; i += blockDim.x) {
        const int k = i / MF_LINES, f = i - k * MF_LINES;
        if (f >= nf) continue;
        T* line = buf + f * P;
        const long id = f0 + f;
        if (k == 0) {
            line[0] = Ts[id];
        } else {
            const T A = Ts[chA(k) * cs + id], B = Ts[chB(k) * cs + id];
            line[k] = mk<T>(A.x - B.y, A.y + B.x);      // A + i B
            line[P - k] = mk<T>(A.x + B.y, A.y - B.x);  // A - i B
        }
    }
    __syncthreads();
    T* r = fft_lines<-1>(buf, tmp, MF_LINES, P, p.sc, twl);
    for (int i = threadIdx.x; i < nf * P; i += blockDim.x) r[i] = cmul(r[i], ld_spec(Sm, f0 * P + i, T()));
    __syncthreads();
    T* o = fft_lines<1>(r, r == buf ? tmp : buf, MF_LINES, P, p.sc, twl);
    for (int i = threadIdx.x; i < (L + 1) * MF_LINES; i += blockDim.x) {
        const int k = i / MF_LINES, f = i - k * MF_LINES;
        if (f >= nf) continue;
        const T* line = o + f * P;
        const long id = f0 + f;
        if (k == 0) {
            Ts[id] = line[0];
        } else {
            const T vp = line[k], vm = line[P - k];
            Ts[chA(k) * cs + id] = half_c(cadd(vp, vm));
            const T d = half_c(csub(vp, vm));
            Ts[chB(k) * cs + id] = mk<T>(d.y, -d.x);     // -i (V_k - V_-k)/2
        }
    }
}

// float-float mode mix.  The (2L+1)-channel state of a frequency (inputs and
// spectra, 544 bytes at L = 8) does not fit in registers with useful
// occupancy, so a block stages 32 frequencies in shared memory and its four
// warps share them: warp g forms the outputs k = g (mod 4) for the 32
// frequencies of its lanes, reading every operand afresh from shared memory
// (volatile loads, so the compiler keeps no copies in registers).  The loops
// over k and k' stay rolled (unrolled, the float-float code outgrows the
// instruction cache); the coefficient parities are still compile-time: all
// outputs of a warp share the parity of k, and k' steps by two.
__device__ __forceinline__ ff lds_ff(const ff* p) {
    ff r;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.volatile.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.hi), "=f"(r.lo) : "r"(a));
    return r;
}
__device__ __forceinline__ ffc lds_ffc(const ffc* p) {
    ffc r;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x.hi), "=f"(r.x.lo), "=f"(r.y.hi), "=f"(r.y.lo)
                 : "r"(a));
    return r;
}
// acc += s v (IM = false) or acc += (i s) v (IM = true)
template <bool IM> __device__ __forceinline__ void tmac_ff(ffc& acc, ff s, ffc v) {
    if (IM) { acc.x -= s * v.y; acc.y += s * v.x; }
    else { acc.x += s * v.x; acc.y += s * v.y; }
}
// the k' term of output k; ODD = parity of k - k' (= parity of k + k')
template <bool ODD>
__device__ __forceinline__ void mix_term_ff(ffc& Ra, ffc& Ia, int k, int kp, const ffc* in, const ff* sr,
                                            const ff* si) {
    const ffc A = lds_ffc(in + 32 * chA(kp)), B = lds_ffc(in + 32 * chB(kp));
    const int d = k - kp, ad = d < 0 ? -d : d, sm = k + kp;
    const ff* Pt = ODD ? si : sr;
    const ff* Mt = ODD ? sr : si;
    const ff pd = lds_ff(Pt + 32 * ad), ps = lds_ff(Pt + 32 * sm);
    ff md = lds_ff(Mt + 32 * ad);
    if (d < 0) md = -md;
    const ff ms = lds_ff(Mt + 32 * sm);
    tmac_ff<ODD>(Ra, pd + ps, A);                  // (P_d + P_s) A
    const ff vm1 = md - ms;                        // i (M_d - M_s) B
    tmac_ff<ODD>(Ra, ODD ? vm1 : -vm1, B);
    const ff vm2 = md + ms;                        // -i (M_d + M_s) A
    tmac_ff<ODD>(Ia, ODD ? -vm2 : vm2, A);
    tmac_ff<ODD>(Ia, pd - ps, B);                  // (P_d - P_s) B
}
// outputs k = k0, k0 + 4, ... (all of parity KODD)
template <int L, bool KODD>
__device__ __forceinline__ void mix_outputs_ff(int k0, const ffc* in, const ff* sr, const ff* si, ffc* out,
                                               long cs) {
#pragma unroll 1
    for (int k = k0; k <= L; k += 4) {
        ffc Ra = mk<ffc>(0, 0), Ia = mk<ffc>(0, 0);
        const ffc A0 = lds_ffc(in);
        tmac_ff<KODD>(Ra, lds_ff((KODD ? si : sr) + 32 * k), A0);   // P_k A_0
        const ff mk_ = lds_ff((KODD ? sr : si) + 32 * k);            // -i M_k A_0
        tmac_ff<KODD>(Ia, KODD ? -mk_ : mk_, A0);
#pragma unroll 1
        for (int kp = 1; kp <= L; kp += 2) {
            mix_term_ff<!KODD>(Ra, Ia, k, kp, in, sr, si);           // k' odd
            if (kp + 1 <= L) mix_term_ff<KODD>(Ra, Ia, k, kp + 1, in, sr, si);
        }
        out[(long)chA(k) * cs] = Ra;
        if (k > 0) out[(long)chB(k) * cs] = Ia;
    }
}

// grid ceil(H Q / 32), block 128
template <int L>
__global__ void __launch_bounds__(128) k_mix_ff(ffc* __restrict__ Ts, const ffc* __restrict__ S, ColParams p) {
    constexpr int NCH = 2 * L + 1;
    __shared__ ffc xin[NCH * 32];  // [c][lane]
    __shared__ ff sre[NCH * 32];   // [m][lane] Re S_m
    __shared__ ff sim[NCH * 32];   // [m][lane] Im S_m
    const int Q = p.Q, H = p.H;
    const long tot = (long)H * Q, cs = (long)H * Q;
    const long base = (long)blockIdx.x * 32;
    for (int i = threadIdx.x; i < 2 * NCH * 32; i += blockDim.x) {
        const int row = i >> 5;
        const long idx = base + (i & 31);
        ffc v = mk<ffc>(0, 0);
        if (idx < tot) {
            const int kx = (int)(idx / Q), ky = (int)(idx % Q);
            if (row < NCH) {
                if (row < p.nin) v = Ts[(long)row * cs + (long)kx * Q + ky];
            } else {
                v = S[((long)kx * NCH + (row - NCH)) * Q + ky];
            }
        }
        if (row < NCH) {
            xin[i] = v;
        } else {
            sre[i - NCH * 32] = v.x;
            sim[i - NCH * 32] = v.y;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long idx = base + lane;
    if (idx >= tot) return;
    const int kx = (int)(idx / Q), ky = (int)(idx % Q);
    ffc* out = Ts + (long)kx * Q + ky;
    // P_m = Re S_m (m even) / i Im S_m (m odd); M_m = i Im S_m (even) / Re S_m (odd);
    // P_{-m} = P_m, M_{-m} = -M_m (the same formulas as mode_mix); warp g
    // forms k = g, g + 4, ..., all of the parity of g
    if (warp & 1) mix_outputs_ff<L, true>(warp, xin + lane, sre + lane, sim + lane, out, cs);
    else mix_outputs_ff<L, false>(warp, xin + lane, sre + lane, sim + lane, out, cs);
}

template <int L, typename T, typename TS>
__global__ void k_mix_pointwise(T* __restrict__ Ts, const TS* __restrict__ S, ColParams p) {
    constexpr int NCH = 2 * L + 1;
    using R = typename real_of<T>::R;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Q = p.Q, H = p.H;
    if (idx >= (long)H * Q) return;
    const int kx = (int)(idx / Q), ky = (int)(idx % Q);
    R sr[2 * L + 1], si[2 * L + 1];
    load_spec<L, T>(S, kx, ky, Q, sr, si);
    T in[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) in[c] = c < p.nin ? Ts[((long)c * H + kx) * Q + ky] : mk<T>(0, 0);
    // every input is in registers: the outputs go straight back in place
    mode_mix<L, T>(sr, si, in, Strided<T>{Ts + (long)kx * Q + ky, (long)H * Q});
}

// ---------------------------------------------------------------------------
// column pass with the warp-register FFT (FP32, Q = 32 R, R = 2..16): one
// block per xi_x, each warp transforms whole channel columns.  Spectra of
// all channels meet in shared memory in the slot layout s = k1 * 32 + lane
// (frequency xi_y = wfreq<R>(k1, lane)), the same layout the plan stores the
// permuted spectra Sp[xi_x][m][s] in; the inverse starts from that layout.
// ---------------------------------------------------------------------------
template <int L, int R, typename TS>
__global__ void __launch_bounds__(256) k_col_warp(float2* __restrict__ Tb, const TS* __restrict__ Sp,
                                                     const float2* __restrict__ tw, int n, int H, int nin) {
    constexpr int NCH = 2 * L + 1;
    constexpr int Q = 32 * R;
    // channel c occupies QS = Q + 32 slots: its spectrum in slot order, and
    // while its column is being transformed, the warp's FFT scratch; the
    // twiddles are read from global memory (L1-resident).  (Three blocks per
    // SM would need <= 85 registers: the mix then spills and runs slower.)
    constexpr int QS = wfft_shape<R>::SCRATCH;
    extern __shared__ unsigned char smraw[];
    float2* X = reinterpret_cast<float2*>(smraw);  // [NCH][QS]
    const int kx = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    pdl_wait();  // Tb: the row pass's output
    pdl_trigger();
    for (int c = warp; c < nin; c += nw) {
        float2 v[R];
        const float2* col = Tb + ((long)c * H + kx) * n;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = lane + 32 * r;
            v[r] = y < n ? col[y] : make_float2(0.f, 0.f);
        }
        float2* Xc = X + (long)c * QS;
        warp_fft_fwd<R>(v, tw, Xc);
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) Xc[k1 * 32 + lane] = v[k1];
    }
    __syncthreads();
    for (int sl = threadIdx.x; sl < Q; sl += blockDim.x) {
        float sr[2 * L + 1], si[2 * L + 1];
#pragma unroll
        for (int m = 0; m <= 2 * L; ++m) {
            const float2 v = ld_spec(Sp, ((long)kx * (2 * L + 1) + m) * Q + sl, float2());
            sr[m] = v.x;
            si[m] = v.y;
        }
        // every input of this slot is read before any output is written
        if (nin == 1) {
            mode_mix_rhs<L, float2>(sr, si, X[sl], Strided<float2>{X + sl, QS});
        } else {
            float2 in[NCH];
#pragma unroll
            for (int c = 0; c < NCH; ++c) in[c] = X[(long)c * QS + sl];
            mode_mix<L, float2>(sr, si, in, Strided<float2>{X + sl, QS});
        }
    }
    __syncthreads();
    for (int c = warp; c < NCH; c += nw) {
        float2 v[R];
        float2* Xc = X + (long)c * QS;
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) v[k1] = Xc[k1 * 32 + lane];
        __syncwarp();
        warp_fft_inv<R>(v, tw, Xc);
        float2* col = Tb + ((long)c * H + kx) * n;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = lane + 32 * r;
            if (y < n) col[y] = v[r];
        }
    }
}

// Column FFTs of the float-float passes with the warp-register FFT: one
// warp per line (channel c, frequency xi_x; line = c * H + xi_x), so the
// kernels hold no channel group in shared memory and keep many warps per SM.
// The forward leaves the spectrum in the slot order (s = k1 * 32 + lane) in
// Ts [line][Q]; the pointwise mode mix then runs on the slot-ordered spectra
// Sp, and the inverse starts from that order.
// dynamic shared memory: the twiddle table (Q) and 8 warps' FFT scratch
template <int R>
__global__ void __launch_bounds__(256) k_colw_fwd(const ffc* __restrict__ Tb, ffc* __restrict__ Ts,
                                                  const ffc* __restrict__ tw, int n, int nlines) {
    constexpr int Q = 32 * R;
    extern __shared__ unsigned char smraw[];
    ffc* twl = reinterpret_cast<ffc*>(smraw);
    ffc* scr = twl + Q + (threadIdx.x >> 5) * wfft_shape<R>::SCRATCH;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    __syncthreads();
    const int line = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (line >= nlines) return;
    const int lane = threadIdx.x & 31;
    const ffc* col = Tb + (long)line * n;
    ffc v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = lane + 32 * r;
        v[r] = y < n ? col[y] : mk<ffc>(0, 0);
    }
    warp_fft_fwd<R>(v, twl, scr);
    ffc* o = Ts + (long)line * Q;
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) o[k1 * 32 + lane] = v[k1];
}

template <int R>
__global__ void __launch_bounds__(256) k_colw_inv(ffc* __restrict__ Tb, const ffc* __restrict__ Ts,
                                                  const ffc* __restrict__ tw, int n, int nlines) {
    constexpr int Q = 32 * R;
    extern __shared__ unsigned char smraw[];
    ffc* twl = reinterpret_cast<ffc*>(smraw);
    ffc* scr = twl + Q + (threadIdx.x >> 5) * wfft_shape<R>::SCRATCH;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    __syncthreads();
    const int line = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (line >= nlines) return;
    const int lane = threadIdx.x & 31;
    const ffc* in = Ts + (long)line * Q;
    ffc v[R];
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) v[k1] = in[k1 * 32 + lane];
    warp_fft_inv<R>(v, twl, scr);
    ffc* col = Tb + (long)line * n;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = lane + 32 * r;
        if (y < n) col[y] = v[r];
    }
}

// ---------------------------------------------------------------------------
// Q = 1024 as two 512-point warp FFTs.  The inputs have n <= Q/2 = 512
// nonzero entries, so the padded transform splits by the residue r = xi mod 2:
//   X[2k + r] = FFT_512( x[j] W_1024^{j r} )[k],
// and the cropped inverse recombines y[j] = z_0[j] + W_1024^{-j} z_1[j] with
// z_r = IFFT_512( X[2 . + r] ) (both unnormalised).  The spectra are stored
// by slot_freq (slot r * 512 + s holds xi = 2 wfreq_512(s) + r).  tw is the
// plan's table exp(-2 pi i t / 1024); the 512-point table is its even half.
// ---------------------------------------------------------------------------

// FP32 column pass (as k_col_warp, R = 16): a block runs the two residues one
// after the other; residue 0's inverse goes to Tz, residue 1 adds its part and
// writes Tb (whose input residue 1 has read by then).
template <int L, typename TS>
__global__ void __launch_bounds__(256, 2) k_col_warp2(float2* __restrict__ Tb, float2* __restrict__ Tz,
                                                      const TS* __restrict__ Sp, const float2* __restrict__ tw,
                                                      int n, int H, int nin) {
    constexpr int NCH = 2 * L + 1;
    constexpr int R = 16, QW = 512, Q = 1024;
    constexpr int QS = wfft_shape<R>::SCRATCH;
    extern __shared__ unsigned char smraw[];
    float2* twl = reinterpret_cast<float2*>(smraw);  // exp(-2 pi i t / 512)
    float2* X = twl + QW;                            // [NCH][QS]
    const int kx = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < QW; i += blockDim.x) twl[i] = tw[2 * i];
    __syncthreads();
    for (int r = 0; r < 2; ++r) {
        for (int c = warp; c < nin; c += nw) {
            float2 v[R];
            const float2* col = Tb + ((long)c * H + kx) * n;
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
                const int y = lane + 32 * rr;
                float2 a = make_float2(0.f, 0.f);
                if (y < n) {
                    a = col[y];
                    if (r) a = cmul(a, tw[y]);
                }
                v[rr] = a;
            }
            float2* Xc = X + (long)c * QS;
            warp_fft_fwd<R>(v, twl, Xc);
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) Xc[k1 * 32 + lane] = v[k1];
        }
        __syncthreads();
        for (int sl = threadIdx.x; sl < QW; sl += blockDim.x) {
            float sr[2 * L + 1], si[2 * L + 1];
#pragma unroll
            for (int m = 0; m <= 2 * L; ++m) {
                const float2 v = ld_spec(Sp, ((long)kx * (2 * L + 1) + m) * Q + r * QW + sl, float2());
                sr[m] = v.x;
                si[m] = v.y;
            }
            if (nin == 1) {
                mode_mix_rhs<L, float2>(sr, si, X[sl], Strided<float2>{X + sl, QS});
            } else {
                float2 in[NCH];
#pragma unroll
                for (int c = 0; c < NCH; ++c) in[c] = X[(long)c * QS + sl];
                mode_mix<L, float2>(sr, si, in, Strided<float2>{X + sl, QS});
            }
        }
        __syncthreads();
        for (int c = warp; c < NCH; c += nw) {
            float2 v[R];
            float2* Xc = X + (long)c * QS;
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) v[k1] = Xc[k1 * 32 + lane];
            __syncwarp();
            warp_fft_inv<R>(v, twl, Xc);
            float2* col = Tb + ((long)c * H + kx) * n;
            float2* zc = Tz + ((long)c * H + kx) * n;
#pragma unroll
            for (int rr = 0; rr < R; ++rr) {
                const int y = lane + 32 * rr;
                if (y < n) {
                    if (r == 0) zc[y] = v[rr];
                    else col[y] = cadd(zc[y], cmul(v[rr], cconj(tw[y])));
                }
            }
        }
        __syncthreads();  // residue 1 reuses X
    }
}

// float-float column FFTs for Q = 1024 (as k_colw_fwd / k_colw_inv, one warp
// per line): the forward writes both residues' spectra into the line of Ts,
// the inverse adds the two residues' parts into Tb
template <int R>  // 16: Q = 1024
__global__ void __launch_bounds__(256) k_colw_fwd2(const ffc* __restrict__ Tb, ffc* __restrict__ Ts,
                                                   const ffc* __restrict__ tw, int n, int nlines) {
    constexpr int QW = 32 * R, Q = 2 * QW;
    extern __shared__ unsigned char smraw[];
    ffc* twl = reinterpret_cast<ffc*>(smraw);
    ffc* scr = twl + QW + (threadIdx.x >> 5) * wfft_shape<R>::SCRATCH;
    for (int i = threadIdx.x; i < QW; i += blockDim.x) twl[i] = tw[2 * i];
    __syncthreads();
    const int line = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (line >= nlines) return;
    const int lane = threadIdx.x & 31;
    const ffc* col = Tb + (long)line * n;
    for (int r = 0; r < 2; ++r) {
        ffc v[R];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
            const int y = lane + 32 * rr;
            ffc a = mk<ffc>(0, 0);
            if (y < n) {
                a = col[y];
                if (r) a = cmul(a, tw[y]);
            }
            v[rr] = a;
        }
        warp_fft_fwd<R>(v, twl, scr);
        ffc* o = Ts + (long)line * Q + r * QW;
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) o[k1 * 32 + lane] = v[k1];
    }
}

template <int R>  // 16: Q = 1024
__global__ void __launch_bounds__(256) k_colw_inv2(ffc* __restrict__ Tb, const ffc* __restrict__ Ts,
                                                   const ffc* __restrict__ tw, int n, int nlines) {
    constexpr int QW = 32 * R, Q = 2 * QW;
    extern __shared__ unsigned char smraw[];
    ffc* twl = reinterpret_cast<ffc*>(smraw);
    ffc* scr = twl + QW + (threadIdx.x >> 5) * wfft_shape<R>::SCRATCH;
    for (int i = threadIdx.x; i < QW; i += blockDim.x) twl[i] = tw[2 * i];
    __syncthreads();
    const int line = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (line >= nlines) return;
    const int lane = threadIdx.x & 31;
    ffc* col = Tb + (long)line * n;
    for (int r = 0; r < 2; ++r) {
        ffc v[R];
        const ffc* in = Ts + (long)line * Q + r * QW;
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) v[k1] = in[k1 * 32 + lane];
        warp_fft_inv<R>(v, twl, scr);
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
            const int y = lane + 32 * rr;
            if (y < n) {
                if (r == 0) col[y] = v[rr];
                else col[y] = cadd(col[y], cmul(v[rr], cconj(tw[y])));
            }
        }
    }
}

// Sp[xi_x][m][sl] = S[xi_x][m][slot_freq(sl, Q)]
template <typename TS>
__global__ void k_permute_spec(const TS* __restrict__ S, TS* __restrict__ Sp, long rows, int Q) {
    const long tot = rows * Q;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
        const long row = i / Q;
        const int sl = (int)(i % Q);
        Sp[i] = S[row * Q + slot_freq(sl, Q)];
    }
}
