// Host launchers of the 2D passes, instantiated per precision in op2d_64.cu
// and op2d_32.cu.
#pragma once
#include <type_traits>

#include "op2d.cuh"

#define RTE_SMEM_OPTIN 232448   // 227 KB dynamic shared memory per block on sm_103a

template <typename K> static cudaError_t allow_smem(K kern) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, RTE_SMEM_OPTIN);
}

template <typename T> static int rows_per_block(int Q) {
    int rb = 65536 / (2 * Q * (int)sizeof(T));
    if (rb > 16) rb = 16;
    if (rb < 2) rb = 2;
    return rb & ~1;
}

template <typename T> static size_t row_smem(int Q, int RB) { return (size_t)(Q + 2 * RB * Q) * sizeof(T); }

// Column pass choice: fused (all channels resident) when it fits.
template <typename T> static bool col_fits(int nch, int Q) {
    return (size_t)(Q + nch * Q + Q) * sizeof(T) <= 200 * 1024;
}
// FFT group size of the fused column pass: as many channels per FFT sweep as
// still let two blocks share an SM (about 110 KB each), else one block
template <typename T> static int col_group(int nch, int Q) {
    long left2 = 110L * 1024 / (long)sizeof(T) - (long)Q - (long)nch * Q;
    int G = (int)(left2 / Q);
    if (G >= 4 || G >= nch) return G > nch ? nch : G;
    long left = 200L * 1024 / (long)sizeof(T) - (long)Q - (long)nch * Q;
    G = (int)(left / Q);
    if (G > nch) G = nch;
    if (G < 1) G = 1;
    return G;
}
template <typename T> static int split_group(int nch, int Q) {
    long G = (200L * 1024 / (long)sizeof(T) / Q - 1) / 2;
    if (G > nch) G = nch;
    if (G < 1) G = 1;
    return (int)G;
}

// float-float mode mix, instantiated in op2d_ff_mix_{a,b,c}.cu
cudaError_t launch_mix_ff(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s);
cudaError_t launch_mix_ff_a(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s);
cudaError_t launch_mix_ff_b(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s);
cudaError_t launch_mix_ff_c(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s);
inline cudaError_t launch_mix_ff(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s) {
    return L <= 5 ? launch_mix_ff_a(L, Ts, S, cp, s) : (L <= 7 ? launch_mix_ff_b(L, Ts, S, cp, s)
                                                                : launch_mix_ff_c(L, Ts, S, cp, s));
}

// split-only instantiations for float-float: the fused kernel would inline
// the float-float mode mix into every FFT stage variant (slow to compile)
template <typename T> struct allow_fused { static constexpr bool value = true; };
template <> struct allow_fused<ffc> { static constexpr bool value = false; };

template <int L, typename T, typename TS>
static cudaError_t launch_col(T* Tb, T* Ts, const TS* S, const T* tw, ColParams cp, bool split, cudaStream_t s) {
    constexpr int NCH = 2 * L + 1;
    const int Q = cp.Q;
    cudaError_t e;
    (void)split;
    if constexpr (allow_fused<T>::value) if (!split) {
        static bool once = false;
        if (!once) { e = allow_smem(k_col_fused<L, T, TS>); if (e != cudaSuccess) return e; once = true; }
        cp.G = col_group<T>(NCH, Q);
        const size_t smem = (size_t)(Q + NCH * Q + cp.G * Q) * sizeof(T);
        k_col_fused<L, T, TS><<<cp.H, 256, smem, s>>>(Tb, S, tw, cp);
        return cudaGetLastError();
    }
    static bool once2 = false;
    if (!once2) { e = allow_smem(k_col_fft_split<T>); if (e != cudaSuccess) return e; once2 = true; }
    cp.G = split_group<T>(NCH, Q);
    const size_t smem = (size_t)(Q + 2 * cp.G * Q) * sizeof(T);
    k_col_fft_split<T><<<cp.H, 256, smem, s>>>(Tb, Ts, tw, cp, 1, cp.nin);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if constexpr (allow_fused<T>::value) {
        const long tot = (long)cp.H * Q;
        k_mix_pointwise<L, T, TS><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Ts, S, cp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        if ((e = launch_mix_ff(L, (ffc*)Ts, (const ffc*)S, cp, s)) != cudaSuccess) return e;
    }
    k_col_fft_split<T><<<cp.H, 256, smem, s>>>(Tb, Ts, tw, cp, 0, NCH);
    return cudaGetLastError();
}

template <int L, int R, typename TS>
static cudaError_t launch_col_warp(float2* Tb, const TS* Sp, const float2* tw, const ColParams& cp, cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) { e = allow_smem(k_col_warp<L, R, TS>); if (e != cudaSuccess) return e; once = true; }
    const size_t smem = (size_t)(2 * L + 1) * wfft_shape<R>::SCRATCH * sizeof(float2);
    return launch_pdl(k_col_warp<L, R, TS>, dim3(cp.H), dim3(256), smem, s, Tb, Sp, tw, cp.n, cp.H, cp.nin);
}

// Q = 1024: two 512-point residues per block (k_col_warp2), Tz holds the first
template <int L, typename TS>
static cudaError_t launch_col_warp2(float2* Tb, float2* Tz, const TS* Sp, const float2* tw, const ColParams& cp,
                                   cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) { e = allow_smem(k_col_warp2<L, TS>); if (e != cudaSuccess) return e; once = true; }
    const size_t smem = (size_t)(512 + (2 * L + 1) * wfft_shape<16>::SCRATCH) * sizeof(float2);
    k_col_warp2<L, TS><<<cp.H, 256, smem, s>>>(Tb, Tz, Sp, tw, cp.n, cp.H, cp.nin);
    return cudaGetLastError();
}

template <int L, typename TS>
static cudaError_t launch_col_warp_q(float2* Tb, float2* Tz, const TS* Sp, const float2* tw, const ColParams& cp,
                                     cudaStream_t s) {
    switch (cp.Q) {
        case 64: return launch_col_warp<L, 2>(Tb, Sp, tw, cp, s);
        case 128: return launch_col_warp<L, 4>(Tb, Sp, tw, cp, s);
        case 256: return launch_col_warp<L, 8>(Tb, Sp, tw, cp, s);
        case 512: return launch_col_warp<L, 16>(Tb, Sp, tw, cp, s);
        case 1024: return Tz ? launch_col_warp2<L>(Tb, Tz, Sp, tw, cp, s) : cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

template <typename TS>
static cudaError_t dispatch_col_warp(int L, float2* Tb, float2* Tz, const TS* Sp, const float2* tw,
                                     const ColParams& cp, cudaStream_t s) {
    switch (L) {
        case 0: return launch_col_warp_q<0>(Tb, Tz, Sp, tw, cp, s);
        case 1: return launch_col_warp_q<1>(Tb, Tz, Sp, tw, cp, s);
        case 2: return launch_col_warp_q<2>(Tb, Tz, Sp, tw, cp, s);
        case 3: return launch_col_warp_q<3>(Tb, Tz, Sp, tw, cp, s);
        case 4: return launch_col_warp_q<4>(Tb, Tz, Sp, tw, cp, s);
        case 5: return launch_col_warp_q<5>(Tb, Tz, Sp, tw, cp, s);
        case 6: return launch_col_warp_q<6>(Tb, Tz, Sp, tw, cp, s);
        case 7: return launch_col_warp_q<7>(Tb, Tz, Sp, tw, cp, s);
        case 8: return launch_col_warp_q<8>(Tb, Tz, Sp, tw, cp, s);
    }
    return cudaErrorInvalidValue;
}

// the warp-register column passes (FP32, float-float, preconditioner) take
// Q in {64, 128, 256, 512} and Q = 1024 as two 512-point residues; the warp
// row passes take Q <= 512
static inline bool col_warp_ok(int Q) { return Q == 64 || Q == 128 || Q == 256 || Q == 512 || Q == 1024; }
static inline bool row_warp_ok(int Q) { return Q == 64 || Q == 128 || Q == 256 || Q == 512 || Q == 1024; }
// shared memory of the two-residue row kernels (Q = 64 R): QW-point
// twiddles, 8 lines of Q + 2, 8 warp FFT scratches
template <typename T, int R> static inline size_t row_warp2_smem() {
    return (size_t)(32 * R + 8 * (64 * R + 2) + 8 * wfft_shape<R>::SCRATCH) * sizeof(T);
}
// float-float forward row pass at Q = 512 as two 256-point residues
static inline bool row_ff2_ok(int Q) { return Q == 512; }

template <typename T, typename TS>
static cudaError_t dispatch_col(int L, T* Tb, T* Ts, const TS* S, const T* tw, ColParams cp, bool split,
                                cudaStream_t s) {
    switch (L) {
        case 0: return launch_col<0>(Tb, Ts, S, tw, cp, split, s);
        case 1: return launch_col<1>(Tb, Ts, S, tw, cp, split, s);
        case 2: return launch_col<2>(Tb, Ts, S, tw, cp, split, s);
        case 3: return launch_col<3>(Tb, Ts, S, tw, cp, split, s);
        case 4: return launch_col<4>(Tb, Ts, S, tw, cp, split, s);
        case 5: return launch_col<5>(Tb, Ts, S, tw, cp, split, s);
        case 6: return launch_col<6>(Tb, Ts, S, tw, cp, split, s);
        case 7: return launch_col<7>(Tb, Ts, S, tw, cp, split, s);
        case 8: return launch_col<8>(Tb, Ts, S, tw, cp, split, s);
    }
    return cudaErrorInvalidValue;
}

// float-float column pass with the warp-register FFT: forward FFT of the
// input channels' lines, pointwise mode mix on the slot-ordered spectra
// (slot_freq_ff: Q = 512 and 1024 as two half-length residues), inverse FFT
// of all channels' lines (3 launches)
static cudaError_t colw_ff(int L, ffc* Tb, ffc* Ts, const ffc* Sp, const ffc* tw, const ColParams& cp,
                           cudaStream_t s) {
    const int lin = cp.nin * cp.H, lout = (2 * L + 1) * cp.H;
    const unsigned gin = (unsigned)((lin + 7) / 8), gout = (unsigned)((lout + 7) / 8);
    // twiddles + 8 FFT scratches (Q = 512, 1024: those of the half-length residues)
    const int QW = cp.Q >= 512 ? cp.Q / 2 : cp.Q;
    const size_t sm = (size_t)(QW + 8 * (QW + 32)) * sizeof(ffc);
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_colw_fwd<2>)) != cudaSuccess || (e = allow_smem(k_colw_fwd<4>)) != cudaSuccess ||
            (e = allow_smem(k_colw_fwd<8>)) != cudaSuccess ||
            (e = allow_smem(k_colw_inv<2>)) != cudaSuccess || (e = allow_smem(k_colw_inv<4>)) != cudaSuccess ||
            (e = allow_smem(k_colw_inv<8>)) != cudaSuccess ||
            (e = allow_smem(k_colw_fwd2<8>)) != cudaSuccess || (e = allow_smem(k_colw_inv2<8>)) != cudaSuccess ||
            (e = allow_smem(k_colw_fwd2<16>)) != cudaSuccess || (e = allow_smem(k_colw_inv2<16>)) != cudaSuccess)
            return e;
        once = true;
    }
    switch (cp.Q) {
        case 64: k_colw_fwd<2><<<gin, 256, sm, s>>>(Tb, Ts, tw, cp.n, lin); break;
        case 128: k_colw_fwd<4><<<gin, 256, sm, s>>>(Tb, Ts, tw, cp.n, lin); break;
        case 256: k_colw_fwd<8><<<gin, 256, sm, s>>>(Tb, Ts, tw, cp.n, lin); break;
        case 512: k_colw_fwd2<8><<<gin, 256, sm, s>>>(Tb, Ts, tw, cp.n, lin); break;
        case 1024: k_colw_fwd2<16><<<gin, 256, sm, s>>>(Tb, Ts, tw, cp.n, lin); break;
        default: return cudaErrorInvalidValue;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_mix_ff(L, Ts, Sp, cp, s)) != cudaSuccess) return e;
    switch (cp.Q) {
        case 64: k_colw_inv<2><<<gout, 256, sm, s>>>(Tb, Ts, tw, cp.n, lout); break;
        case 128: k_colw_inv<4><<<gout, 256, sm, s>>>(Tb, Ts, tw, cp.n, lout); break;
        case 256: k_colw_inv<8><<<gout, 256, sm, s>>>(Tb, Ts, tw, cp.n, lout); break;
        case 512: k_colw_inv2<8><<<gout, 256, sm, s>>>(Tb, Ts, tw, cp.n, lout); break;
        case 1024: k_colw_inv2<16><<<gout, 256, sm, s>>>(Tb, Ts, tw, cp.n, lout); break;
    }
    return cudaGetLastError();
}

// warp row passes (Q in {64, 128, 256, 512}) for FP32 fields and compute.  The
// kernels also instantiate for float-float on FP64 fields, but there the
// shared-memory passes are faster: the warp forward needs 194 registers per
// thread, and the warp inverse (128 registers) measured 43.2 us against 38.5 us
// at 256^2, L = 8, Q = 512.
template <typename T, typename TF> struct row_warp_types { static constexpr bool value = false; };
template <> struct row_warp_types<float2, float2> { static constexpr bool value = true; };
template <typename T> static inline size_t row_warp_smem(int Q) { return (size_t)(Q + 8 * (Q + 34)) * sizeof(T); }

template <typename T, typename TF>
static cudaError_t row_fwd_warp(int Q, dim3 grid, const TF* x, const double* f, T* out, const T* tw,
                                const RowParams& rp, cudaStream_t s) {
    const size_t sm = row_warp_smem<T>(Q);
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_row_fwd_warp<2, T, TF>)) != cudaSuccess ||
            (e = allow_smem(k_row_fwd_warp<4, T, TF>)) != cudaSuccess ||
            (e = allow_smem(k_row_fwd_warp<8, T, TF>)) != cudaSuccess ||
            (e = allow_smem(k_row_fwd_warp<16, T, TF>)) != cudaSuccess)
            return e;
        once = true;
    }
    e = cudaSuccess;
    switch (Q) {
        case 64: e = launch_pdl(k_row_fwd_warp<2, T, TF>, grid, dim3(256), sm, s, x, f, out, tw, rp); break;
        case 128: e = launch_pdl(k_row_fwd_warp<4, T, TF>, grid, dim3(256), sm, s, x, f, out, tw, rp); break;
        case 256: e = launch_pdl(k_row_fwd_warp<8, T, TF>, grid, dim3(256), sm, s, x, f, out, tw, rp); break;
        case 512: e = launch_pdl(k_row_fwd_warp<16, T, TF>, grid, dim3(256), sm, s, x, f, out, tw, rp); break;
        case 1024:
            if constexpr (std::is_same<T, float2>::value && std::is_same<TF, float2>::value) {
                static bool once2 = false;
                if (!once2) {
                    if ((e = allow_smem(k_row_fwd_warp2<16, float2, float2>)) != cudaSuccess) return e;
                    once2 = true;
                }
                k_row_fwd_warp2<16, float2, float2><<<grid, 256, row_warp2_smem<float2, 16>(), s>>>(x, f, out, tw, rp);
                break;
            }
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// M's inverse row pass fused with K's forward row pass (k_row_invfwd_warp)
static cudaError_t row_invfwd_warp(int Q, dim3 grid, float2* Tb, const float2* x, float2* out, const float2* tw,
                                   const RowParams& rp, cudaStream_t s) {
    const size_t sm = row_warp_smem<float2>(Q);
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_row_invfwd_warp<2>)) != cudaSuccess || (e = allow_smem(k_row_invfwd_warp<4>)) != cudaSuccess ||
            (e = allow_smem(k_row_invfwd_warp<8>)) != cudaSuccess || (e = allow_smem(k_row_invfwd_warp<16>)) != cudaSuccess)
            return e;
        once = true;
    }
    e = cudaSuccess;
    switch (Q) {
        case 64: e = launch_pdl(k_row_invfwd_warp<2>, grid, dim3(256), sm, s, Tb, x, out, tw, rp); break;
        case 128: e = launch_pdl(k_row_invfwd_warp<4>, grid, dim3(256), sm, s, Tb, x, out, tw, rp); break;
        case 256: e = launch_pdl(k_row_invfwd_warp<8>, grid, dim3(256), sm, s, Tb, x, out, tw, rp); break;
        case 512: e = launch_pdl(k_row_invfwd_warp<16>, grid, dim3(256), sm, s, Tb, x, out, tw, rp); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T, typename TF>
static cudaError_t row_inv_warp(int Q, dim3 grid, const T* in, const TF* x, const TF* z, TF* out, const T* tw,
                                const RowParams& rp, typename real_of<T>::R a, typename real_of<T>::R b,
                                typename real_of<T>::R c, cudaStream_t s) {
    const size_t sm = row_warp_smem<T>(Q);
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_row_inv_warp<2, T, TF>)) != cudaSuccess ||
            (e = allow_smem(k_row_inv_warp<4, T, TF>)) != cudaSuccess ||
            (e = allow_smem(k_row_inv_warp<8, T, TF>)) != cudaSuccess ||
            (e = allow_smem(k_row_inv_warp<16, T, TF>)) != cudaSuccess)
            return e;
        once = true;
    }
    e = cudaSuccess;
    switch (Q) {
        case 64: e = launch_pdl(k_row_inv_warp<2, T, TF>, grid, dim3(256), sm, s, in, x, z, out, tw, rp, a, b, c); break;
        case 128: e = launch_pdl(k_row_inv_warp<4, T, TF>, grid, dim3(256), sm, s, in, x, z, out, tw, rp, a, b, c); break;
        case 256: e = launch_pdl(k_row_inv_warp<8, T, TF>, grid, dim3(256), sm, s, in, x, z, out, tw, rp, a, b, c); break;
        case 512: e = launch_pdl(k_row_inv_warp<16, T, TF>, grid, dim3(256), sm, s, in, x, z, out, tw, rp, a, b, c); break;
        case 1024:
            if constexpr (std::is_same<T, float2>::value && std::is_same<TF, float2>::value) {
                static bool once2 = false;
                if (!once2) {
                    if ((e = allow_smem(k_row_inv_warp2<16, float2, float2>)) != cudaSuccess) return e;
                    once2 = true;
                }
                k_row_inv_warp2<16, float2, float2><<<grid, 256, row_warp2_smem<float2, 16>(), s>>>(in, x, z, out, tw, rp, a, b, c);
                break;
            }
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// float-float forward row pass at Q = 512 as two 256-point residues (R = 8).
// The inverse stays on the shared-memory pass: as two residues (107
// registers, its epilogue's x loads after the transforms) it measured 41.1 us
// against 38.9 us at 256^2, L = 8; the forward 28.6 against 35.3 us.
template <typename T, typename TF>
static cudaError_t row_fwd_res(dim3 grid, const TF* x, const double* f, T* out, const T* tw, const RowParams& rp,
                               cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_row_fwd_warp2<8, T, TF>)) != cudaSuccess) return e;
        once = true;
    }
    k_row_fwd_warp2<8, T, TF><<<grid, 256, row_warp2_smem<T, 8>(), s>>>(x, f, out, tw, rp);
    return cudaGetLastError();
}

// the mode-axis FFT spectra and twiddles of a plan for compute type T
static inline const float2* modefft_spec(const rte_plan p, float2*) { return p->Sm32; }
static inline const double2* modefft_spec(const rte_plan p, double2*) { return p->Sm64; }
static inline const ffc* modefft_spec(const rte_plan p, ffc*) { return p->Smff; }
static inline const float2* modefft_tw(const rte_plan p, float2*) { return p->twm32; }
static inline const double2* modefft_tw(const rte_plan p, double2*) { return p->twm64; }
static inline const ffc* modefft_tw(const rte_plan p, ffc*) { return p->twmff; }

// column pass with the mode-axis FFT coupling (p->mix_fft): column FFTs of
// the input channels into Ts, k_mix_modefft in place, inverse column FFTs of
// all channels back into Tb (3 launches)
template <typename T>
static cudaError_t col_modefft(rte_plan p, T* Tb, T* Ts, const T* tw, ColParams cp, cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_col_fft_split<T>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_mix_modefft<T, T>)) != cudaSuccess) return e;
        once = true;
    }
    cp.G = split_group<T>(p->nch, cp.Q);
    const size_t smem = (size_t)(cp.Q + 2 * cp.G * cp.Q) * sizeof(T);
    k_col_fft_split<T><<<cp.H, 256, smem, s>>>(Tb, Ts, tw, cp, 1, cp.nin);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ModeFftParams mp;
    mp.L = p->L;
    mp.P = p->Pm;
    mp.nin = cp.nin;
    mp.nfreq = (long)cp.H * cp.Q;
    mp.sc = p->sched_m;
    const size_t smm = (size_t)(p->Pm + 2 * MF_LINES * p->Pm) * sizeof(T);
    k_mix_modefft<T, T><<<(unsigned)((mp.nfreq + MF_LINES - 1) / MF_LINES), 256, smm, s>>>(
        Ts, modefft_spec(p, (T*)nullptr), modefft_tw(p, (T*)nullptr), mp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_col_fft_split<T><<<cp.H, 256, smem, s>>>(Tb, Ts, tw, cp, 0, p->nch);
    return cudaGetLastError();
}

// out = a*x + b*(Op x) + c*z ; Op = K (MIX_K), K~ on the source f (MIX_RHS),
// or K x + K~ f (MIX_KF)
// stage: -1 all three passes; 0 row pass; 1 column pass; 2 inverse row pass
template <typename T, typename TS, typename TF = T>
static cudaError_t op2d_run(rte_plan p, MixKind kind, const TF* x, const double* f, TF* out, double a, double b,
                            double c, const TF* z, T* Tb, T* Ts, const TS* S, const T* tw, bool split,
                            cudaStream_t s, int stage = -1, const TS* Sp = nullptr) {
    using R = typename real_of<T>::R;
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_row_fwd<T, TF>)) != cudaSuccess) return e;
        if ((e = allow_smem(k_row_inv<T, TF>)) != cudaSuccess) return e;
        once = true;
    }
    RowParams rp;
    rp.n = p->n; rp.Q = p->Q; rp.H = p->H; rp.L = p->L;
    rp.RB = rows_per_block<T>(p->Q);
    // small grids: fewer rows per block until the row passes have a block per
    // SM (the row FFTs, and the row pairs of mode 0, are the same for any even RB)
    while (rp.RB > 2 && (long)((p->n + rp.RB - 1) / rp.RB) * (p->L + 1) < p->nsm) rp.RB = (rp.RB / 2) & ~1;
    if (rp.RB < 2) rp.RB = 2;
    if (p->rb_force >= 2 && p->rb_force <= 16 && row_smem<T>(p->Q, p->rb_force & ~1) <= 200 * 1024)
        rp.RB = p->rb_force & ~1;
    rp.sc = p->sched;
    for (int k = 0; k <= RTE_MAX_L; ++k) rp.wk[k] = 0.0;
    const bool use_x = kind != MIX_RHS, use_f = kind != MIX_K;
    if (use_x) {
        for (int k = 0; k <= p->L; ++k) rp.wk[k] = p->mu_s * p->sigma_hat[k];
    } else {
        rp.wk[0] = 1.0;
    }
    const int nmod_in = use_x ? p->L + 1 : 1;
    const size_t smr = row_smem<T>(p->Q, rp.RB);
    bool row_warp = false, row_res = false;
    if constexpr (row_warp_types<T, TF>::value) row_warp = row_warp_ok(p->Q) && p->rb_force < 2;
    constexpr bool ffrows = std::is_same<T, ffc>::value && std::is_same<TF, double2>::value;
    if constexpr (ffrows) row_res = row_ff2_ok(p->Q) && p->rb_force < 2;
    if (stage < 0 || stage == 0) {
        if (row_warp) {
            if constexpr (row_warp_types<T, TF>::value) {
                const dim3 grid((p->n + 7) / 8, nmod_in);
                if ((e = row_fwd_warp<T, TF>(p->Q, grid, use_x ? x : nullptr, use_f ? f : nullptr,
                                             Tb, tw, rp, s)) != cudaSuccess)
                    return e;
            }
        } else if (row_res) {
            if constexpr (ffrows) {
                const dim3 grid((p->n + 7) / 8, nmod_in);
                if ((e = row_fwd_res<T, TF>(grid, use_x ? x : nullptr, use_f ? f : nullptr, Tb, tw, rp, s)) !=
                    cudaSuccess)
                    return e;
            }
        } else {
            const dim3 grid((p->n + rp.RB - 1) / rp.RB, nmod_in);
            k_row_fwd<T, TF><<<grid, 256, smr, s>>>(use_x ? x : nullptr, use_f ? f : nullptr, Tb, tw,
                                                    rp);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        rte_count_launches(1);
    }
    if (stage < 0 || stage == 1) {
        ColParams cp;
        cp.n = p->n; cp.Q = p->Q; cp.H = p->H; cp.L = p->L;
        cp.nin = use_x ? p->nch : 1;
        cp.G = 1;
        cp.sc = p->sched;
        int launches = split ? 3 : 1;
        bool warp_path = false;
        if (p->mix_fft) {
            if ((e = col_modefft<T>(p, Tb, Ts, tw, cp, s)) != cudaSuccess) return e;
            rte_count_launches(3);
            warp_path = true;  // handled: skip the direct-mix paths below
            launches = 0;
        }
        if constexpr (sizeof(T) == sizeof(float2)) {
            if (!warp_path && Sp && col_warp_ok(p->Q)) {
                if ((e = dispatch_col_warp<TS>(p->L, (float2*)Tb, p->Tz32, Sp, (const float2*)tw, cp, s)) != cudaSuccess)
                    return e;
                warp_path = true;
                launches = 1;
            }
        }
        if constexpr (!allow_fused<T>::value) {
            if (!warp_path && Sp && col_warp_ok(p->Q)) {
                if ((e = colw_ff(p->L, Tb, Ts, Sp, tw, cp, s)) != cudaSuccess) return e;
                warp_path = true;
                launches = 3;
            }
        }
        if (!warp_path && (e = dispatch_col<T, TS>(p->L, Tb, Ts, S, tw, cp, split, s)) != cudaSuccess) return e;
        rte_count_launches(launches);
    }
    if (stage < 0 || stage == 2) {
        if (row_warp) {
            if constexpr (row_warp_types<T, TF>::value) {
                const dim3 grid2((p->n + 7) / 8, p->L + 1);
                if ((e = row_inv_warp<T, TF>(p->Q, grid2, Tb, use_x ? x : nullptr, z, out, tw, rp, (R)a,
                                             (R)b, (R)c, s)) != cudaSuccess)
                    return e;
            }
        } else {
            const dim3 grid2((p->n + rp.RB - 1) / rp.RB, p->L + 1);
            k_row_inv<T, TF><<<grid2, 256, smr, s>>>(Tb, use_x ? x : nullptr, z, out, tw, rp, (R)a, (R)b,
                                                     (R)c);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        rte_count_launches(1);
    }
    return cudaSuccess;
}

// average duration of each pass over `reps` back-to-back launches (CUDA
// events on stream s); ms[0..2] = row, column, inverse row
template <typename T, typename TS, typename TF = T>
static cudaError_t op2d_time(rte_plan p, const TF* x, TF* out, T* Tb, T* Ts, const TS* S, const T* tw, bool split,
                             int reps, double* ms, cudaStream_t s, const TS* Sp = nullptr) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaSuccess;
    for (int st = 0; st < 3 && e == cudaSuccess; ++st) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = op2d_run<T, TS, TF>(p, MIX_K, x, nullptr, out, 1.0, -1.0, 0.0, nullptr, Tb, Ts, S, tw, split, s, st, Sp);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[st] = t / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}
