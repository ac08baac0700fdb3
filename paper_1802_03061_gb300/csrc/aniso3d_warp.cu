// Warp-register FFT passes of the spherical-harmonic operator (Sec. 3.1.2 with
// the FFT application of Sec. 2.3.1) for Q = 64, 128, 256: the isotropic 3D
// warp passes (op3d_warp.cuh) with the channel as the grid's z index, so one
// launch transforms all M channels of a pass, and a Z pass that mixes the
// channels.  Per application five launches: X and Y over the input channels,
// the Z mix, Y' and X' over the output channels.
//
// Z mix, per block of B (xi_x, xi_y) lines: each warp FFTs one (channel, line)
// along z in registers and leaves the spectrum in shared memory in the warp
// FFT's slot order; then one thread per (line, slot) forms
// out_a = sum_b S_ab in_b at that frequency; then each warp transforms one
// output (channel, line) back and keeps z < n.  S_ab(xi) = +-s_p(xi_x, |xi_y|,
// |xi_z|) (times i for the imaginary pairs), p the pair's stored octant.
#include <utility>

#include "aniso3d.cuh"
#include "op3d_warp.cuh"

template <typename RR> __device__ __forceinline__ RR cneg(RR v, bool c) { return c ? -v : v; }

// acc += S x with S = s (real pair) or i s (imaginary pair)
template <bool IM, typename T, typename RR> __device__ __forceinline__ void madd(T& acc, RR s, const T& x) {
    if constexpr (IM) {
        acc.x -= s * x.y;
        acc.y += s * x.x;
    } else {
        acc.x += s * x.x;
        acc.y += s * x.y;
    }
}

// pair P = (a, b), a <= b, with its flags known at compile time: one load of
// its spectrum, out_a += S_ab x_b and out_b += S_ab x_a
template <int P, int M, typename T, typename TS>
__device__ __forceinline__ void mix_pair(T* acc, const T* xin, const TS* __restrict__ S, long H3, long so, bool fy,
                                         bool fz, int Min) {
    using RR = typename real_of<T>::R;
    constexpr int a = pair_first(P, M), b = pair_second(P, M);
    constexpr int info = pair_info(a, b, M);
    static_assert((info & 0xffff) == P, "pair numbering");
    constexpr bool IM = (info >> 16) & 1;
    RR s = (RR)S[P * H3 + so];
    if constexpr ((info >> 17) & 1) s = cneg(s, fy);
    if constexpr ((info >> 18) & 1) s = cneg(s, fz);
    if (b < Min) madd<IM>(acc[a], s, xin[b]);
    if constexpr (a != b) {
        if (a < Min) madd<IM>(acc[b], s, xin[a]);
    }
}

template <int M, typename T, typename TS, int... Ps>
__device__ __forceinline__ void mix_all(std::integer_sequence<int, Ps...>, T* acc, const T* xin,
                                        const TS* __restrict__ S, long H3, long so, bool fy, bool fz, int Min) {
    (mix_pair<Ps, M, T, TS>(acc, xin, S, H3, so, fy, fz, Min), ...);
}

// Any M (L = 3, 4): B consecutive (xi_x, xi_y) lines per block, the pair
// table read from pinfo.  Min = 1 (the right-hand side: channel 0 only) or M.
template <int RQ, typename T, typename TS>
__global__ void __launch_bounds__(256) k3wa_z_mix(T* __restrict__ T2, long chs, int Min, int Mout,
                                                  const TS* __restrict__ S, long H3, const int* __restrict__ pinfo,
                                                  int M, const T* __restrict__ tw, int n, int H, int B, int bufl) {
    constexpr int Q = 32 * RQ, SCR = wfft_shape<RQ>::SCRATCH;
    using RR = typename real_of<T>::R;
    extern __shared__ unsigned char smraw[];
    __shared__ int pis[RTE_ANISO_MAX_M * RTE_ANISO_MAX_M];
    T* twl = reinterpret_cast<T*>(smraw);
    T* bin = twl + Q;      // [Min][nb][Q] input spectra; the inverse FFTs' scratch afterwards
    T* bout = bin + bufl;  // [Mout][nb][Q] mixed spectra; the forward FFTs' scratch before
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long nlines = (long)H * Q, l0 = (long)blockIdx.x * B;
    const int nb = (int)min((long)B, nlines - l0);
    for (int i = threadIdx.x; i < Q; i += blockDim.x) twl[i] = tw[i];
    for (int i = threadIdx.x; i < M * M; i += blockDim.x) pis[i] = pinfo[i];
    pdl_wait();  // T2: the y pass's output
    pdl_trigger();
    __syncthreads();
    for (int it = warp; it < Min * nb; it += 8) {
        const int c = it / nb, lb = it - c * nb;
        const T* src = T2 + c * chs + (l0 + lb) * n;
        T v[RQ];
#pragma unroll
        for (int r = 0; r < RQ; ++r) {
            const int z = lane + 32 * r;
            v[r] = z < n ? src[z] : mk<T>(0, 0);
        }
        warp_fft_fwd<RQ>(v, twl, bout + warp * SCR);
        T* dst = bin + (c * nb + lb) * Q;
#pragma unroll
        for (int j = 0; j < RQ; ++j) dst[j * 32 + lane] = v[j];
        __syncwarp();
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * Q; idx += blockDim.x) {
        const int lb = idx / Q, sl = idx - lb * Q;
        const int kz = wfreq<RQ>(sl >> 5, sl & 31);
        const long line = l0 + lb;
        const int kx = (int)(line / Q), sy = (int)(line % Q);
        const int ky = wfreq<RQ>(sy >> 5, sy & 31);
        const long so = ((long)kx * H + fold(ky, Q)) * H + fold(kz, Q);
        const bool ny = ky > Q / 2, nz = kz > Q / 2;
        for (int a = 0; a < Mout; ++a) {
            RR ar = 0, ai = 0;
            for (int b = 0; b < Min; ++b) {
                const int info = pis[a * M + b];
                RR s = (RR)S[(long)(info & 0xffff) * H3 + so];
                if (((info >> 17) & 1) && ny) s = -s;
                if (((info >> 18) & 1) && nz) s = -s;
                const T xv = bin[(b * nb + lb) * Q + sl];
                if ((info >> 16) & 1) {  // i s x
                    ar -= s * xv.y;
                    ai += s * xv.x;
                } else {
                    ar += s * xv.x;
                    ai += s * xv.y;
                }
            }
            bout[(a * nb + lb) * Q + sl] = mk<T>(ar, ai);
        }
    }
    __syncthreads();
    for (int it = warp; it < Mout * nb; it += 8) {
        const int a = it / nb, lb = it - a * nb;
        const T* src = bout + (a * nb + lb) * Q;
        T v[RQ];
#pragma unroll
        for (int j = 0; j < RQ; ++j) v[j] = src[j * 32 + lane];
        warp_fft_inv<RQ>(v, twl, bin + warp * SCR);
        T* dst = T2 + a * chs + (l0 + lb) * n;
#pragma unroll
        for (int r = 0; r < RQ; ++r) {
            const int z = lane + 32 * r;
            if (z < n) dst[z] = v[r];
        }
        __syncwarp();
    }
}

// 4- or 8-byte asynchronous global -> shared copy
template <int BYTES> __device__ __forceinline__ void cp_async_ca(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
                 "n"(BYTES)
                 : "memory");
}

// L = LT <= 2 (M <= 9): one block per (xi_x, |xi_y|), i.e. the line xi_y and
// its mirror Q - xi_y, which read the same octant row of every pair spectrum.
// The block copies those rows (M(M+1)/2 x H values) into shared memory while
// its warps transform the input channels of both lines; the mix then reads
// the spectra from shared memory with the pair flags known at compile time.
// max(M, 8) warps: two FFT rounds per phase and one mix item per thread at M = 9.
template <int LT> __host__ __device__ constexpr int zpair_warps() { return (LT + 1) * (LT + 1) > 8 ? (LT + 1) * (LT + 1) : 8; }

template <int RQ, typename T, typename TS, int LT>
__global__ void __launch_bounds__(32 * zpair_warps<LT>())
    k3wa_z_pair(T* __restrict__ T2, long chs, int Min, const TS* __restrict__ S, long H3, const T* __restrict__ tw,
                int n, int H, int bufl) {
    constexpr int Q = 32 * RQ, SCR = wfft_shape<RQ>::SCRATCH;
    constexpr int M = (LT + 1) * (LT + 1), NP = M * (M + 1) / 2, NW = zpair_warps<LT>();
    extern __shared__ unsigned char smraw[];
    __shared__ int slot_of[Q];
    T* twl = reinterpret_cast<T*>(smraw);
    T* bin = twl + Q;      // [Min][nb][Q]; the inverse FFTs' scratch afterwards
    T* bout = bin + bufl;  // [M][nb][Q]; the forward FFTs' scratch before
    TS* Ss = reinterpret_cast<TS*>(bout + bufl);  // [NP][H]: the pairs' rows at (xi_x, |xi_y|)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kx = blockIdx.x / H, k = blockIdx.x - kx * H;
    const int nb = (k == 0 || 2 * k == Q) ? 1 : 2;  // line 0: xi_y = k; line 1: xi_y = Q - k
    {
        const TS* src = S + ((long)kx * H + k) * H;
        for (int p = warp; p < NP; p += NW)
            for (int e = lane; e < H; e += 32) cp_async_ca<sizeof(TS)>(Ss + p * H + e, src + (long)p * H3 + e);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        twl[i] = tw[i];
        slot_of[wfreq<RQ>(i >> 5, i & 31)] = i;
    }
    pdl_wait();  // T2: the y pass's output (the spectra are plan constants)
    pdl_trigger();
    __syncthreads();
    for (int it = warp; it < Min * nb; it += NW) {
        const int c = it / nb, lb = it - c * nb;
        const long line = (long)kx * Q + slot_of[lb ? Q - k : k];
        const T* src = T2 + c * chs + line * n;
        T v[RQ];
#pragma unroll
        for (int r = 0; r < RQ; ++r) {
            const int z = lane + 32 * r;
            v[r] = z < n ? src[z] : mk<T>(0, 0);
        }
        warp_fft_fwd<RQ>(v, twl, bout + warp * SCR);
        T* dst = bin + (c * nb + lb) * Q;
#pragma unroll
        for (int j = 0; j < RQ; ++j) dst[j * 32 + lane] = v[j];
        __syncwarp();
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * Q; idx += blockDim.x) {
        const int lb = idx / Q, sl = idx - lb * Q;
        const int kz = wfreq<RQ>(sl >> 5, sl & 31);
        T xin[M], acc[M];
#pragma unroll
        for (int b = 0; b < M; ++b) {
            xin[b] = b < Min ? bin[(b * nb + lb) * Q + sl] : mk<T>(0, 0);
            acc[b] = mk<T>(0, 0);
        }
        mix_all<M, T, TS>(std::make_integer_sequence<int, NP>{}, acc, xin, Ss, H, fold(kz, Q), lb == 1, kz > Q / 2,
                          Min);
#pragma unroll
        for (int a = 0; a < M; ++a) bout[(a * nb + lb) * Q + sl] = acc[a];
    }
    __syncthreads();
    for (int it = warp; it < M * nb; it += NW) {
        const int a = it / nb, lb = it - a * nb;
        const T* src = bout + (a * nb + lb) * Q;
        T v[RQ];
#pragma unroll
        for (int j = 0; j < RQ; ++j) v[j] = src[j * 32 + lane];
        warp_fft_inv<RQ>(v, twl, bin + warp * SCR);
        const long line = (long)kx * Q + slot_of[lb ? Q - k : k];
        T* dst = T2 + a * chs + line * n;
#pragma unroll
        for (int r = 0; r < RQ; ++r) {
            const int z = lane + 32 * r;
            if (z < n) dst[z] = v[r];
        }
        __syncwarp();
    }
}

// elements of one Z buffer for B lines: M B Q, at least the eight warps' FFT scratch
static long zbuf_elems(int RQ, int M, int B) {
    const long scr = 8L * RQ * (32 + 32 / RQ);
    const long need = (long)M * B * 32 * RQ;
    return need > scr ? need : scr;
}
static size_t zsmem(int RQ, int M, int B, int elem) {
    return (size_t)(32L * RQ + 2 * zbuf_elems(RQ, M, B)) * elem;
}

// dynamic shared memory a Z block may take: the opt-in limit less the static
// pair table and a margin
static const size_t kWarpZCap = (size_t)RTE_SMEM_OPTIN - RTE_ANISO_MAX_M * RTE_ANISO_MAX_M * sizeof(int) - 1024;

// paired-line kernel (L <= 2): each Z buffer holds two lines of M channels and
// at least the block's FFT scratch; then the spectra rows
static long zpair_buf(int RQ, int M) {
    const int nw = M > 8 ? M : 8;
    const long scr = (long)nw * RQ * (32 + 32 / RQ);
    const long need = (long)M * 2 * 32 * RQ;
    return need > scr ? need : scr;
}
static size_t zpair_smem(int RQ, int M, int H, int elem, int selem) {
    return (size_t)(32L * RQ + 2 * zpair_buf(RQ, M)) * elem + (size_t)M * (M + 1) / 2 * H * selem;
}

// lines per block of the generic Z kernel (L >= 3): the largest B <= 4 within
// 64 KB (three or more blocks per SM), else B = 1 if it fits at all; for
// L <= 2 (the paired-line kernel) 2 if it fits
int aniso_warp_lines(int RQ, int M, int elem_bytes) {
    if (M <= 9) {
        const int H = 16 * RQ + 1;
        return zpair_smem(RQ, M, H, elem_bytes, elem_bytes / 2) <= kWarpZCap ? 2 : 0;
    }
    for (int B = 4; B >= 1; --B)
        if (zsmem(RQ, M, B, elem_bytes) <= 64 * 1024) return B;
    return zsmem(RQ, M, 1, elem_bytes) <= kWarpZCap ? 1 : 0;
}

template <int RQ, typename T, typename R, typename TS> static cudaError_t prepare_one() {
    constexpr int Q = 32 * RQ;
    using W = wfft_shape<RQ>;
    const int smx = (int)((Q + 8 * (Q + 34)) * sizeof(T));
    const int smy = (int)((Q + (Q * 17 > 16 * W::SCRATCH ? Q * 17 : 16 * W::SCRATCH)) * sizeof(T));
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k3w_x_fwd<RQ, T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smx)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k3w_x_inv<RQ, T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smx)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k3w_y_fwd<RQ, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smy)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k3w_y_inv<RQ, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smy)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k3wa_z_mix<RQ, T, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kWarpZCap)) != cudaSuccess)
        return e;
    for (auto k : {k3wa_z_pair<RQ, T, TS, 0>, k3wa_z_pair<RQ, T, TS, 1>, k3wa_z_pair<RQ, T, TS, 2>})
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpZCap)) != cudaSuccess)
            return e;
    return cudaSuccess;
}

template <int RQ> static cudaError_t prepare_rq() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e;
    if ((e = prepare_one<RQ, float2, float, float>()) != cudaSuccess) return e;
    if ((e = prepare_one<RQ, double2, double, double>()) != cudaSuccess) return e;
    if ((e = prepare_one<RQ, ffc, double, ff>()) != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

cudaError_t aniso_warp_prepare(int RQ) {
    switch (RQ) {
        case 2: return prepare_rq<2>();
        case 4: return prepare_rq<4>();
        case 8: return prepare_rq<8>();
        default: return cudaErrorInvalidValue;
    }
}

template <int RQ, typename T, typename R, typename TS>
static cudaError_t run_rq(rte_aniso3d op, const R* x, R* out, int rhs, double ca, double cb, const R* zv, double cc,
                          const double* xf, const TS* S, const T* tw, cudaStream_t s) {
    constexpr int Q = 32 * RQ;
    using W = wfft_shape<RQ>;
    const int n = op->n, H = op->H, M = op->M;
    const size_t smx = (size_t)(Q + 8 * (Q + 34)) * sizeof(T);
    const size_t smy = (size_t)(Q + (Q * 17 > 16 * W::SCRATCH ? Q * 17 : 16 * W::SCRATCH)) * sizeof(T);
    const int B = sizeof(T) == 8 ? op->Bw8 : op->Bw16;
    const long bufl = zbuf_elems(RQ, M, B);
    const size_t smz = zsmem(RQ, M, B, (int)sizeof(T));
    T* T1 = (T*)op->T1;
    T* T2 = (T*)op->T2;
    const long chs = (long)H * Q * n;
    const int Min = rhs ? 1 : M;
    const unsigned gy = (unsigned)((n + 15) / 16);
    cudaError_t e;
    const double* xf0 = rhs ? nullptr : xf;
    const double* wz0 = rhs ? nullptr : op->wz;
    if ((e = launch_pdl(k3w_x_fwd<RQ, T, R>, dim3(gy, n, Min), dim3(256), smx, s, x, T1, tw, n, H, 1.0, xf0, wz0)) !=
        cudaSuccess)
        return e;
    if ((e = launch_pdl(k3w_y_fwd<RQ, T>, dim3(gy, H, Min), dim3(512), smy, s, (const T*)T1, T2, tw, n, H)) !=
        cudaSuccess)
        return e;
    const long nlines = (long)H * Q;
    if (op->L <= 2) {
        const long bp = zpair_buf(RQ, M);
        const size_t smp = zpair_smem(RQ, M, H, (int)sizeof(T), (int)sizeof(TS));
        const unsigned grid = (unsigned)H * H;
        const long H3 = (long)H * H * H;
        if (op->L == 0)
            e = launch_pdl(k3wa_z_pair<RQ, T, TS, 0>, dim3(grid), dim3(32 * zpair_warps<0>()), smp, s, T2, chs, Min,
                           S, H3, tw, n, H, (int)bp);
        else if (op->L == 1)
            e = launch_pdl(k3wa_z_pair<RQ, T, TS, 1>, dim3(grid), dim3(32 * zpair_warps<1>()), smp, s, T2, chs, Min,
                           S, H3, tw, n, H, (int)bp);
        else
            e = launch_pdl(k3wa_z_pair<RQ, T, TS, 2>, dim3(grid), dim3(32 * zpair_warps<2>()), smp, s, T2, chs, Min,
                           S, H3, tw, n, H, (int)bp);
    } else {
        e = launch_pdl(k3wa_z_mix<RQ, T, TS>, dim3((unsigned)((nlines + B - 1) / B)), dim3(256), smz, s, T2, chs, Min,
                       M, S, (long)H * H * H, (const int*)op->pinfo, M, tw, n, H, B, (int)bufl);
    }
    if (e != cudaSuccess) return e;
    if ((e = launch_pdl(k3w_y_inv<RQ, T>, dim3(gy, H, M), dim3(512), smy, s, (const T*)T2, T1, tw, n, H)) !=
        cudaSuccess)
        return e;
    const R* xe = (rhs || ca == 0.0) ? nullptr : x;
    if ((e = launch_pdl(k3w_x_inv<RQ, T, R>, dim3(gy, n, M), dim3(256), smx, s, (const T*)T1, xe, zv, out, tw, n, H,
                        ca, cb, cc)) != cudaSuccess)
        return e;
    rte_count_launches(5);
    return cudaSuccess;
}

template <typename T, typename R, typename TS>
cudaError_t aniso_run_warp(rte_aniso3d op, const R* x, R* out, int rhs, double ca, double cb, const R* zv, double cc,
                           const double* xf, const TS* S, const T* tw, cudaStream_t s) {
    switch (op->RQ) {
        case 2: return run_rq<2, T, R, TS>(op, x, out, rhs, ca, cb, zv, cc, xf, S, tw, s);
        case 4: return run_rq<4, T, R, TS>(op, x, out, rhs, ca, cb, zv, cc, xf, S, tw, s);
        case 8: return run_rq<8, T, R, TS>(op, x, out, rhs, ca, cb, zv, cc, xf, S, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t aniso_run_warp<float2, float, float>(rte_aniso3d, const float*, float*, int, double, double,
                                                          const float*, double, const double*, const float*,
                                                          const float2*, cudaStream_t);
template cudaError_t aniso_run_warp<double2, double, double>(rte_aniso3d, const double*, double*, int, double, double,
                                                             const double*, double, const double*, const double*,
                                                             const double2*, cudaStream_t);
template cudaError_t aniso_run_warp<ffc, double, ff>(rte_aniso3d, const double*, double*, int, double, double,
                                                     const double*, double, const double*, const ff*, const ffc*,
                                                     cudaStream_t);
