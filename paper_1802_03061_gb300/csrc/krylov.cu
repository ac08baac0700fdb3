// Device GMRES (Saad & Schultz) for (I - K) u = b, plus the mixed-precision
// iterative refinement driver.
//
// The paper solves step T.2 (Sec. 3.3.1) -- and S.2 for L = 0 (Sec. 2.3.1) --
// with GMRES/MINRES on the FFT matvec.  Here the Krylov vectors are the real
// channels of J-symmetric fields (u_{-k} = conj(u_k)), with the inner
// product of the full complex vector over modes -L..L:
//   <u, v> = sum_{mode 0} u v + 2 sum_{modes k>=1} Re(conj(u_k) v_k),
// so residual norms equal those of the paper's NM-dimensional system.
//
// Arnoldi: classical Gram-Schmidt, once (FP32 inner solves) or twice (FP64),
// as a single-pass multi-dot over the basis and a fused multi-axpy + norm.
// The Hessenberg matrix, Givens rotations and residual estimate live in
// device memory (FP64) and are updated by one warp.
//
// The whole solve is one CUDA graph with device-side control: T.1, then a
// conditional WHILE over refinement steps, inside it a WHILE over GMRES
// restart cycles, inside that a WHILE over Arnoldi steps (an IF node
// recomputes the residual for a restart).  Small one-thread kernels decide
// the loop conditions from FP64 state in device memory, so the host only
// launches the graph and reads the statistics at the end.
//
// The graph is built on a KrylovOp (internal.h): the operator as callbacks
// that enqueue its kernels, and the work vectors.  The plan supplies one for
// its J-symmetric channels (with the periodic preconditioner and MINRES as
// options); the spherical-harmonic operator (aniso3d.cu) supplies one for its
// real moments, where every element weighs 1.
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "internal.h"

#define GM_MMAX 128
#define TILE 2048   // elements per block in the vector kernels (256 threads x 8)

struct GmresDev {
    int j;       // Arnoldi index (number of finished columns after the step)
    int its;     // iterations in this solve
    int stop;    // 1: end of cycle
    int conv;    // 1: estimated residual <= target
    int m;       // restart length
    int maxit;
    int cgs2;    // 1: re-orthogonalise
    int cycle;   // restart cycles done in this inner solve
    double tol;     // relative tolerance (set by the host before each solve)
    double target;  // absolute residual target tol * ||rhs||
    double beta;
    double res;     // |g_{j}|, the residual estimate
    double nrm;     // last norm result
    double bnorm;   // ||rhs||
    double vscale;  // FP32 steps: the newest basis vector V_j is stored unscaled; V_j * vscale is unit
    unsigned int cnt1, cnt2, cnt3;  // finished-block counters of the fused FP32 kernels (reset by the last block)
    // MINRES (symmetric L = 0 inner solves): step number and the Lanczos / QR recurrence scalars
    int mr_it;
    double mr_beta1, mr_beta, mr_oldb, mr_alfa, mr_dbar, mr_epsln, mr_oldeps, mr_delta, mr_gamma, mr_phi,
        mr_phibar, mr_cs, mr_sn;
    double cs[GM_MMAX], sn[GM_MMAX], g[GM_MMAX + 1];
    double Hc[(GM_MMAX + 1) * GM_MMAX];  // H[i + j*(m+1)]
    double hA[GM_MMAX + 1], hB[GM_MMAX + 1], y[GM_MMAX];
};

// --------------------------------------------------------------------------
// vector kernels (T = float or double storage)
// element e has weight 1 when e < nw1 (mode 0), else 2
//
// FP64 is about 1/64 of the FP32 rate on this GPU, so for FP32 vectors the
// inner products keep double-precision accuracy with error-free
// transformations on the FP32 units: a*b = p + e exactly (p = fl(a*b),
// e = fma(a, b, -p)) and s + t = sum + err exactly (Knuth's TwoSum), giving
// (hi, lo) pairs with about 48 significant bits.  The _rn intrinsics keep the
// compiler from contracting the transformations into FMAs.
// --------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// (hi, lo) += (bh, bl)
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
    float s, e;
    two_sum(hi, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}
// (hi, lo) += a * b
__device__ __forceinline__ void ff_fma(float& hi, float& lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    ff_add(hi, lo, p, pe);
}
__device__ __forceinline__ void ff_warp_sum(float& hi, float& lo) {
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_down_sync(0xffffffffu, hi, o);
        const float bl = __shfl_down_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, bh, bl);
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_mdot(const T* __restrict__ V, long nr, const T* __restrict__ w,
                                              const int* __restrict__ cnt_src, int cnt_add, long nw1,
                                              double* __restrict__ part) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    __shared__ double red[GM_MMAX + 1][8];
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if constexpr (sizeof(T) == sizeof(float)) {
        float wv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            wv[q] = e < nr ? (float)w[e] * (e < nw1 ? 1.f : 2.f) : 0.f;
        }
        for (int i = 0; i < count; ++i) {
            const T* v = V + (long)i * nr;
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long e = base + 256 * q;
                if (e < nr) ff_fma(hi, lo, (float)v[e], wv[q]);
            }
            ff_warp_sum(hi, lo);
            if (lane == 0) red[i][wid] = (double)hi + (double)lo;
        }
    } else {
        double wv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            wv[q] = e < nr ? (double)w[e] * (e < nw1 ? 1.0 : 2.0) : 0.0;
        }
        for (int i = 0; i < count; ++i) {
            const T* v = V + (long)i * nr;
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long e = base + 256 * q;
                if (e < nr) s += (double)v[e] * wv[q];
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) red[i][wid] = s;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[i][q];
        part[(long)i * gridDim.x + blockIdx.x] = t;
    }
}

// out[i] = sum_b part[i][b] (fixed order), i < count; one block per i
__global__ void k_reduce(const double* __restrict__ part, int nblk, const int* __restrict__ cnt_src, int cnt_add,
                         double* __restrict__ out, int do_sqrt) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    const int i = blockIdx.x;
    if (i >= count) return;
    __shared__ double red[256];
    double t = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) t += part[(long)i * nblk + b];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = do_sqrt ? sqrt(red[0]) : red[0];
}

// w += sgn * sum_{i<count} coef[i] V_i ; optionally partial ||w||^2 per block
template <typename T>
__global__ void __launch_bounds__(256) k_maxpy(const T* __restrict__ V, long nr, T* __restrict__ w,
                                               const double* __restrict__ coef, const int* __restrict__ cnt_src,
                                               int cnt_add, double sgn, long nw1, double* __restrict__ part) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    __shared__ double c[GM_MMAX + 1];
    __shared__ double red[8];
    for (int i = threadIdx.x; i < count; i += blockDim.x) c[i] = sgn * coef[i];
    __syncthreads();
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    double sqd = 0.0;
    if constexpr (sizeof(T) == sizeof(float)) {
        // the result is stored in FP32: FP32 arithmetic, compensated norm
        float acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.f;
        for (int i = 0; i < count; ++i) {
            const T* v = V + (long)i * nr;
            const float ci = (float)c[i];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long e = base + 256 * q;
                if (e < nr) acc[q] = fmaf(ci, (float)v[e], acc[q]);
            }
        }
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            if (e < nr) {
                const float nv = (float)w[e] + acc[q];
                w[e] = (T)nv;
                if (part) ff_fma(hi, lo, nv, nv * (e < nw1 ? 1.f : 2.f));
            }
        }
        if (part) {
            ff_warp_sum(hi, lo);
            sqd = (double)hi + (double)lo;
        }
    } else {
        double acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.0;
        for (int i = 0; i < count; ++i) {
            const T* v = V + (long)i * nr;
            const double ci = c[i];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const long e = base + 256 * q;
                if (e < nr) acc[q] += ci * (double)v[e];
            }
        }
        double sq = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            if (e < nr) {
                const T nv = (T)((double)w[e] + acc[q]);
                w[e] = nv;
                sq += (double)nv * (double)nv * (e < nw1 ? 1.0 : 2.0);
            }
        }
        if (part)
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
        sqd = sq;
    }
    if (part) {
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sqd;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += red[q];
            part[blockIdx.x] = t;
        }
    }
}

// w = rhs - w
template <typename T>
__global__ void k_rsub(const T* __restrict__ rhs, T* __restrict__ w, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        w[e] = rhs[e] - w[e];
}

// u += d (FP64)
__global__ void k_add64(double* __restrict__ u, const double* __restrict__ d, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        u[e] += d[e];
}

// dst = src * (1 / *s)  (0 if *s == 0)
template <typename T, typename U>
__global__ void k_scale_inv(const T* __restrict__ src, U* __restrict__ dst, long nr, const double* __restrict__ s) {
    const double inv = (*s != 0.0) ? 1.0 / *s : 0.0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = (U)((double)src[e] * inv);
}

// u += (*a) * d
template <typename T>
__global__ void k_axpy_scaled(double* __restrict__ u, const T* __restrict__ d, long nr, const double* __restrict__ a) {
    const double s = *a;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        u[e] += s * (double)d[e];
}

// V_{j+off} = w / nrm and the matvec input slot gets the same vector
template <typename T>
__global__ void k_scale_basis(const T* __restrict__ w, T* __restrict__ V, T* __restrict__ vin, long nr,
                              const GmresDev* __restrict__ st, int off) {
    const int slot = st->j + off;
    const double nrm = st->nrm;
    const T inv = (T)(nrm > 0.0 ? 1.0 / nrm : 0.0);  // in the storage precision
    T* dst = V + (long)slot * nr;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x) {
        const T v = w[e] * inv;
        dst[e] = v;
        vin[e] = v;
    }
}

// start of a cycle: the residual norm is in st->nrm
__global__ void k_cycle_init(GmresDev* st, cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0) return;
    const double nrm = st->nrm;
    if (st->cycle == 0) {
        st->bnorm = nrm;
        st->target = st->tol * nrm;
    }
    st->j = 0;
    st->stop = 0;
    st->conv = 0;
    st->vscale = 1.0;  // V_0 is written normalised
    st->beta = nrm;
    st->res = nrm;
    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
    st->g[0] = nrm;
    bool skip = false;
    if (!isfinite(nrm)) { st->stop = 1; skip = true; }
    else if (!(nrm > st->target)) { st->stop = 1; st->conv = 1; skip = true; }
    if (st->its >= st->maxit) { st->stop = 1; skip = true; }
    cudaGraphSetConditional(loop, skip ? 0u : 1u);
}

// One Givens update of column j from col[0..j] (Hessenberg column, FP64) and
// h_{j+1} = hn; one thread.  Updates the residual estimate and the loop
// condition.
__device__ void givens_update(GmresDev* st, double* col, double hn, cudaGraphConditionalHandle loop) {
    const int j = st->j, m = st->m, ld = m + 1;
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double c = st->cs[i], sn = st->sn[i];
        const double t = c * col[i] + sn * col[i + 1];
        col[i + 1] = -sn * col[i] + c * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], b = col[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    st->cs[j] = c;
    st->sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    double* Hc = st->Hc + (long)j * ld;
    for (int i = 0; i <= j + 1; ++i) Hc[i] = col[i];
    const double gj = st->g[j];
    st->g[j + 1] = -s * gj;
    st->g[j] = c * gj;
    st->res = fabs(st->g[j + 1]);
    st->its += 1;
    st->j = j + 1;
    int stop = 0;
    if (st->res <= st->target) { stop = 1; st->conv = 1; }
    if (!(hn > 1e-300) || !isfinite(st->res)) stop = 1;  // breakdown or non-finite
    if (j + 1 >= m || st->its >= st->maxit) stop = 1;
    st->stop = stop;
    cudaGraphSetConditional(loop, stop ? 0u : 1u);
}

// Givens step of the FP64 path: column h = hA (+ hB), h_{j+1} = st->nrm
__global__ void k_givens(GmresDev* st, cudaGraphConditionalHandle loop) {
    __shared__ double col[GM_MMAX + 2];
    const int j = st->j;
    const int two = st->cgs2;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = st->hA[i] + (two ? st->hB[i] : 0.0);
    __syncwarp();
    if (threadIdx.x != 0) return;
    givens_update(st, col, st->nrm, loop);
}

// --------------------------------------------------------------------------
// FP64 Arnoldi step (CGS2) for short vectors (nr <= CGS64_SHORT): three
// kernels and the basis scaling after the matvec instead of nine.  Block b
// owns the elements [b chunk, (b+1) chunk), so the FP64 work spreads over
// ceil(nr / 256) SMs (FP64 runs at 1/64 of the FP32 rate: one block doing a
// 64^2 step alone took twice as long as the nine kernels); the last block to
// finish sums the per-block partials in a fixed order (deterministic).
//   PASS 0: h_A = <V_i, w>, i <= j
//   PASS 1: w -= V h_A, then h_B = <V_i, w>
//   PASS 2: w -= V h_B, ||w||, and the Givens update with h_A + h_B
// --------------------------------------------------------------------------
#define CGS64_SHORT 65536
template <int PASS>
__global__ void __launch_bounds__(256) k_cgs64(const double* __restrict__ V, long nr, double* __restrict__ w,
                                               GmresDev* __restrict__ st, long nw1, double* __restrict__ part,
                                               long chunk, cudaGraphConditionalHandle loop) {
    const int j = st->j, count = j + 1;
    const int nb = gridDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ double c[GM_MMAX + 1];
    __shared__ double red[GM_MMAX + 1][8];
    __shared__ double col[GM_MMAX + 2];
    __shared__ bool last;
    const long e0 = (long)blockIdx.x * chunk, e1 = e0 + chunk < nr ? e0 + chunk : nr;
    if (PASS > 0) {
        for (int i = threadIdx.x; i < count; i += blockDim.x) c[i] = PASS == 1 ? st->hA[i] : st->hB[i];
        __syncthreads();
        for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            double acc = 0.0;
            for (int i = 0; i < count; ++i) acc += c[i] * V[(long)i * nr + e];
            w[e] -= acc;
        }
    }
    const int ncol = PASS < 2 ? count : 1;
    for (int i = 0; i < ncol; ++i) {
        double sacc = 0.0;
        for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const double we = w[e] * (e < nw1 ? 1.0 : 2.0);
            sacc += (PASS < 2 ? V[(long)i * nr + e] : w[e]) * we;
        }
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_down_sync(0xffffffffu, sacc, o);
        if (lane == 0) red[i][wid] = sacc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncol; i += blockDim.x) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[i][q];
        part[(long)i * nb + blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    unsigned int* cnt = PASS == 0 ? &st->cnt1 : PASS == 1 ? &st->cnt2 : &st->cnt3;
    if (threadIdx.x == 0) last = atomicAdd(cnt, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (PASS < 2) {
        double* h = PASS == 0 ? st->hA : st->hB;
        for (int i = wid; i < count; i += 8) {
            double t = 0.0;
            for (int b = lane; b < nb; b += 32) t += __ldcg(part + (long)i * nb + b);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) h[i] = t;
        }
        if (threadIdx.x == 0) *cnt = 0u;
        return;
    }
    if (wid != 0) return;
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += __ldcg(part + b);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    for (int i = lane; i < count; i += 32) col[i] = st->hA[i] + st->hB[i];
    __syncwarp();
    if (lane == 0) {
        *cnt = 0u;
        const double nrm = sqrt(t);
        st->nrm = nrm;
        givens_update(st, col, nrm, loop);
    }
}

// --------------------------------------------------------------------------
// fused FP32 Arnoldi step (CGS1): two kernels after the matvec instead of six.
// V_j arrives unscaled (the previous step stored w without dividing by its
// norm); with s = vscale, A V_j = s * w_raw.
//  k_step_dot : V_j <- s V_j (in place, once), h_i = <V_i, s w_raw>, i <= j;
//               the last block to finish sums the per-block partials in a
//               fixed order (deterministic) into hA.
//  k_step_upd : w = s w_raw - sum_i h_i V_i, stored unscaled as V_{j+1} and as
//               the next matvec input, partial ||w||^2; the last block forms
//               the norm, vscale = 1/||w||, and the Givens update.
// "Last block" = the block whose atomic increment of the finished counter
// returns gridDim.x - 1 after a __threadfence(); nothing waits.
// --------------------------------------------------------------------------
// Vectorised forms for nr % 4 == 0 (every basis vector then starts on a
// 16-byte boundary): thread t of a block owns elements [4t, 4t+4) and
// [1024 + 4t, 1024 + 4t + 4) of the block's TILE, read as float4, and the
// loop over basis vectors is unrolled by four, so each thread keeps eight
// 16-byte loads in flight -- enough bytes in flight per SM for the loop to
// run at HBM speed rather than at load latency.
__device__ __forceinline__ float4 f4scale(float4 a, float s) {
    return make_float4(__fmul_rn(a.x, s), __fmul_rn(a.y, s), __fmul_rn(a.z, s), __fmul_rn(a.w, s));
}
__device__ __forceinline__ void ff_fma4(float& hi, float& lo, float4 a, const float* b) {
    ff_fma(hi, lo, a.x, b[0]);
    ff_fma(hi, lo, a.y, b[1]);
    ff_fma(hi, lo, a.z, b[2]);
    ff_fma(hi, lo, a.w, b[3]);
}

__global__ void __launch_bounds__(256) k_step_dot4(float* __restrict__ V, long nr, const float* __restrict__ w,
                                                   GmresDev* __restrict__ st, long nw1, double* __restrict__ part) {
    pdl_wait();  // w: the operator's output
    pdl_trigger();
    const int j = st->j, count = j + 1;
    const float s = (float)st->vscale;
    const bool rescale = s != 1.f;
    const int nb = gridDim.x;
    __shared__ double red[GM_MMAX + 1][8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long e0 = (long)blockIdx.x * TILE + 4 * threadIdx.x, e1 = e0 + 1024;
    const bool in0 = e0 < nr, in1 = e1 < nr;
    float wv[8];
    {
        const float4 a = in0 ? *reinterpret_cast<const float4*>(w + e0) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = in1 ? *reinterpret_cast<const float4*>(w + e1) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float av[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = (q < 4 ? e0 : e1) + (q & 3);
            wv[q] = __fmul_rn(s, av[q]) * (e < nw1 ? 1.f : 2.f);
        }
    }
    for (int i0 = 0; i0 < count; i0 += 4) {
        float4 va[4], vb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k;
            const float* v = V + (long)i * nr;
            va[k] = (i < count && in0) ? *reinterpret_cast<const float4*>(v + e0) : make_float4(0.f, 0.f, 0.f, 0.f);
            vb[k] = (i < count && in1) ? *reinterpret_cast<const float4*>(v + e1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k;
            if (i == j && rescale) {
                float* v = V + (long)i * nr;
                va[k] = f4scale(va[k], s);
                vb[k] = f4scale(vb[k], s);
                if (in0) *reinterpret_cast<float4*>(v + e0) = va[k];
                if (in1) *reinterpret_cast<float4*>(v + e1) = vb[k];
            }
            hi[k] = 0.f;
            lo[k] = 0.f;
            ff_fma4(hi[k], lo[k], va[k], wv);
            ff_fma4(hi[k], lo[k], vb[k], wv + 4);
        }
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float bh = __shfl_down_sync(0xffffffffu, hi[k], o);
                const float bl = __shfl_down_sync(0xffffffffu, lo[k], o);
                ff_add(hi[k], lo[k], bh, bl);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i0 + k < count) red[i0 + k][wid] = (double)hi[k] + (double)lo[k];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[i][q];
        part[(long)i * nb + blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->cnt1, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = wid; i < count; i += 8) {
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(part + (long)i * nb + b);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) st->hA[i] = t;
    }
    if (threadIdx.x == 0) st->cnt1 = 0u;
}

__global__ void __launch_bounds__(256) k_step_upd4(const float* __restrict__ V, long nr, const float* __restrict__ w,
                                                   float* __restrict__ vin, GmresDev* __restrict__ st, long nw1,
                                                   double* __restrict__ part, cudaGraphConditionalHandle loop,
                                                   const float* __restrict__ zsrc, float* __restrict__ Z) {
    pdl_wait();  // hA: the multi-dot's result
    pdl_trigger();
    const int j = st->j, count = j + 1;
    const float s = (float)st->vscale;
    const int nb = gridDim.x;
    __shared__ double c[GM_MMAX + 1];
    __shared__ double red[256];
    __shared__ bool last;
    for (int i = threadIdx.x; i < count; i += blockDim.x) c[i] = -st->hA[i];
    __syncthreads();
    const long e0 = (long)blockIdx.x * TILE + 4 * threadIdx.x, e1 = e0 + 1024;
    const bool in0 = e0 < nr, in1 = e1 < nr;
    float4 a0 = in0 ? f4scale(*reinterpret_cast<const float4*>(w + e0), s) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a1 = in1 ? f4scale(*reinterpret_cast<const float4*>(w + e1), s) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i0 = 0; i0 < count; i0 += 4) {
        float4 va[4], vb[4];
        float ck[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = i0 + k;
            const float* v = V + (long)i * nr;
            const bool ok = i < count;
            ck[k] = ok ? (float)c[i] : 0.f;
            va[k] = (ok && in0) ? *reinterpret_cast<const float4*>(v + e0) : make_float4(0.f, 0.f, 0.f, 0.f);
            vb[k] = (ok && in1) ? *reinterpret_cast<const float4*>(v + e1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a0.x = fmaf(ck[k], va[k].x, a0.x); a0.y = fmaf(ck[k], va[k].y, a0.y);
            a0.z = fmaf(ck[k], va[k].z, a0.z); a0.w = fmaf(ck[k], va[k].w, a0.w);
            a1.x = fmaf(ck[k], vb[k].x, a1.x); a1.y = fmaf(ck[k], vb[k].y, a1.y);
            a1.z = fmaf(ck[k], vb[k].z, a1.z); a1.w = fmaf(ck[k], vb[k].w, a1.w);
        }
    }
    float* vn = const_cast<float*>(V) + (long)(j + 1) * nr;
    float hi = 0.f, lo = 0.f;
    if (Z) {  // z_j = M v_j (see k_step_upd)
        float* zj = Z + (long)j * nr;
        if (in0) *reinterpret_cast<float4*>(zj + e0) = f4scale(*reinterpret_cast<const float4*>(zsrc + e0), s);
        if (in1) *reinterpret_cast<float4*>(zj + e1) = f4scale(*reinterpret_cast<const float4*>(zsrc + e1), s);
    }
    if (in0) {
        *reinterpret_cast<float4*>(vn + e0) = a0;
        *reinterpret_cast<float4*>(vin + e0) = a0;
        const float av[4] = {a0.x, a0.y, a0.z, a0.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) ff_fma(hi, lo, av[q], av[q] * (e0 + q < nw1 ? 1.f : 2.f));
    }
    if (in1) {
        *reinterpret_cast<float4*>(vn + e1) = a1;
        *reinterpret_cast<float4*>(vin + e1) = a1;
        const float bv[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) ff_fma(hi, lo, bv[q], bv[q] * (e1 + q < nw1 ? 1.f : 2.f));
    }
    ff_warp_sum(hi, lo);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)hi + (double)lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q];
        part[blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->cnt2, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(part + b);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double nrm = sqrt(red[0]);
    st->nrm = nrm;
    st->vscale = nrm > 0.0 ? 1.0 / nrm : 0.0;
    st->cnt2 = 0u;
    for (int i = 0; i <= j; ++i) c[i] = st->hA[i];
    givens_update(st, c, nrm, loop);
}

__global__ void __launch_bounds__(256) k_step_dot(float* __restrict__ V, long nr, const float* __restrict__ w,
                                                  GmresDev* __restrict__ st, long nw1, double* __restrict__ part) {
    pdl_wait();  // w: the operator's output
    pdl_trigger();
    const int j = st->j, count = j + 1;
    const float s = (float)st->vscale;
    const bool rescale = s != 1.f;
    const int nb = gridDim.x;
    __shared__ double red[GM_MMAX + 1][8];
    __shared__ bool last;
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float wv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        wv[q] = e < nr ? __fmul_rn(s, w[e]) * (e < nw1 ? 1.f : 2.f) : 0.f;
    }
    for (int i = 0; i < count; ++i) {
        float* v = V + (long)i * nr;
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            if (e < nr) {
                float vv = v[e];
                if (i == j && rescale) {
                    vv = __fmul_rn(vv, s);
                    v[e] = vv;
                }
                ff_fma(hi, lo, vv, wv[q]);
            }
        }
        ff_warp_sum(hi, lo);
        if (lane == 0) red[i][wid] = (double)hi + (double)lo;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[i][q];
        part[(long)i * nb + blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->cnt1, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = wid; i < count; i += 8) {
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(part + (long)i * nb + b);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) st->hA[i] = t;
    }
    if (threadIdx.x == 0) st->cnt1 = 0u;
}

// zsrc / Z (right-preconditioned steps): zsrc = M applied to this step's
// unscaled input, stored scaled as z_j = M v_j in Z[j] for the cycle end
__global__ void __launch_bounds__(256) k_step_upd(const float* __restrict__ V, long nr, const float* __restrict__ w,
                                                  float* __restrict__ vin, GmresDev* __restrict__ st, long nw1,
                                                  double* __restrict__ part, cudaGraphConditionalHandle loop,
                                                  const float* __restrict__ zsrc, float* __restrict__ Z) {
    pdl_wait();  // hA: the multi-dot's result
    pdl_trigger();
    const int j = st->j, count = j + 1;
    const float s = (float)st->vscale;
    const int nb = gridDim.x;
    __shared__ double c[GM_MMAX + 1];
    __shared__ double red[256];
    __shared__ bool last;
    for (int i = threadIdx.x; i < count; i += blockDim.x) c[i] = -st->hA[i];
    __syncthreads();
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        acc[q] = e < nr ? __fmul_rn(s, w[e]) : 0.f;
    }
    for (int i = 0; i < count; ++i) {
        const float* v = V + (long)i * nr;
        const float ci = (float)c[i];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            if (e < nr) acc[q] = fmaf(ci, v[e], acc[q]);
        }
    }
    float* vn = const_cast<float*>(V) + (long)(j + 1) * nr;
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        if (e < nr) {
            const float nv = acc[q];
            vn[e] = nv;
            vin[e] = nv;
            ff_fma(hi, lo, nv, nv * (e < nw1 ? 1.f : 2.f));
            if (Z) Z[(long)j * nr + e] = s * zsrc[e];
        }
    }
    ff_warp_sum(hi, lo);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)hi + (double)lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q];
        part[blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->cnt2, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(part + b);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double nrm = sqrt(red[0]);
    st->nrm = nrm;
    st->vscale = nrm > 0.0 ? 1.0 / nrm : 0.0;
    st->cnt2 = 0u;
    for (int i = 0; i <= j; ++i) c[i] = st->hA[i];  // reuse shared storage for the column
    givens_update(st, c, nrm, loop);
}

// back substitution H(0:k,0:k) y = g(0:k), k = st->j
__global__ void k_solve_tri(GmresDev* st) {
    if (threadIdx.x != 0) return;
    const int k = st->j, ld = st->m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double t = st->g[i];
        for (int q = i + 1; q < k; ++q) t -= st->Hc[i + (long)q * ld] * st->y[q];
        const double d = st->Hc[i + (long)i * ld];
        st->y[i] = d != 0.0 ? t / d : 0.0;
    }
}


// --------------------------------------------------------------------------
// refinement / solve control (one thread each)
// --------------------------------------------------------------------------
struct RefDev {
    int outer, max_outer, its, maxit;
    int use_guess, mixed, cycles, restarts;
    int status, pad0, pad1, pad2;
    double tol, inner_tol, bnorm, rnorm, relres;
};

__global__ void k_copy_vec(const double* __restrict__ src, double* __restrict__ dst, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

template <typename T>
__global__ void k_copy_T(const T* __restrict__ src, T* __restrict__ dst, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// FP32 -> FP64 copy
__global__ void k_widen(const float* __restrict__ src, double* __restrict__ dst, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = (double)src[e];
}

template <typename T>
__global__ void k_zero_T(T* __restrict__ dst, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = (T)0;
}

__global__ void k_zero_unless_guess(double* __restrict__ u, long nr, const RefDev* __restrict__ ref) {
    if (ref->use_guess) return;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        u[e] = 0.0;
}

// after ||b||: start values; the guess branch runs only with a guess
__global__ void k_ref_start(RefDev* ref, cudaGraphConditionalHandle c_guess) {
    if (threadIdx.x != 0) return;
    const double b = ref->bnorm;
    ref->rnorm = b;
    ref->relres = b > 0.0 ? 1.0 : 0.0;
    ref->outer = 0;
    ref->its = 0;
    ref->cycles = 0;
    ref->restarts = 0;
    ref->status = isfinite(b) ? 0 : 7;
    cudaGraphSetConditional(c_guess, (ref->use_guess && b > 0.0 && isfinite(b)) ? 1u : 0u);
}

__global__ void k_ref_relres(RefDev* ref) {
    if (threadIdx.x != 0) return;
    ref->relres = ref->bnorm > 0.0 ? ref->rnorm / ref->bnorm : 0.0;
}

// a guess whose residual is not below ||b|| (or not finite) is replaced by
// the zero start: u = 0, r = b
__global__ void k_guess_fallback(double* __restrict__ u, double* __restrict__ r, const double* __restrict__ b, long nr,
                                 const RefDev* __restrict__ ref) {
    if (ref->rnorm < ref->bnorm) return;  // false for NaN as well: fall back
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x) {
        u[e] = 0.0;
        r[e] = b[e];
    }
}
__global__ void k_guess_fallback_state(RefDev* ref) {
    if (threadIdx.x != 0) return;
    if (!(ref->rnorm < ref->bnorm)) {
        ref->rnorm = ref->bnorm;
        ref->relres = ref->bnorm > 0.0 ? 1.0 : 0.0;
        ref->pad0 = 1;  // guess rejected
    }
}

__global__ void k_ref_gate(RefDev* ref, cudaGraphConditionalHandle c_outer) {
    if (threadIdx.x != 0) return;
    const bool fin = isfinite(ref->relres) && isfinite(ref->bnorm);
    if (!fin) ref->status = 7;
    const bool go = fin && ref->bnorm > 0.0 && ref->relres > ref->tol && ref->its < ref->maxit;
    cudaGraphSetConditional(c_outer, go ? 1u : 0u);
}

// inner GMRES start: tolerance relative to its right-hand side
__global__ void k_gm_start(GmresDev* st, const RefDev* ref, int m, int cgs2, cudaGraphConditionalHandle c_cycle) {
    if (threadIdx.x != 0) return;
    st->m = m;
    st->cgs2 = cgs2;
    st->its = 0;
    st->cycle = 0;
    const int left = ref->maxit - ref->its;
    st->maxit = left < 1 ? 1 : left;
    double tin;
    if (ref->mixed) {
        // the inner solve need not go beyond what the outer target needs
        tin = ref->inner_tol;
        const double need = ref->relres > 0.0 ? 0.5 * ref->tol / ref->relres : 1.0;
        if (need > tin) tin = need;
    } else {
        tin = ref->rnorm > 0.0 ? 0.5 * ref->tol * ref->bnorm / ref->rnorm : 1.0;
    }
    st->tol = tin;
    cudaGraphSetConditional(c_cycle, 1u);
}

__global__ void k_cycle_end(GmresDev* st, RefDev* ref, cudaGraphConditionalHandle c_cycle,
                            cudaGraphConditionalHandle c_restart) {
    if (threadIdx.x != 0) return;
    st->cycle += 1;
    ref->cycles += 1;
    const bool cont = !st->conv && st->its < st->maxit && st->j > 0 && isfinite(st->res);
    if (cont) ref->restarts += 1;
    cudaGraphSetConditional(c_cycle, cont ? 1u : 0u);
    cudaGraphSetConditional(c_restart, cont ? 1u : 0u);
}

__global__ void k_ref_after(RefDev* ref, const GmresDev* st) {
    if (threadIdx.x != 0) return;
    ref->its += st->its;
    ref->outer += 1;
}

__global__ void k_ref_check(RefDev* ref, cudaGraphConditionalHandle c_outer) {
    if (threadIdx.x != 0) return;
    ref->relres = ref->bnorm > 0.0 ? ref->rnorm / ref->bnorm : 0.0;
    const bool fin = isfinite(ref->relres);
    if (!fin) ref->status = 7;
    const bool go = fin && ref->relres > ref->tol && ref->outer < ref->max_outer && ref->its < ref->maxit;
    cudaGraphSetConditional(c_outer, go ? 1u : 0u);
}
// --------------------------------------------------------------------------
// host side: graph construction
// --------------------------------------------------------------------------
static int grid_for(long nr) {
    long g = (nr + 255) / 256;
    return (int)(g < 1216 ? (g < 1 ? 1 : g) : 1216);
}
static int tiles(long nr) { return (int)((nr + TILE - 1) / TILE); }

long krylov_tiles(long nr) { return tiles(nr); }
// columns of the per-block partial sums: one per TILE, or one per 256
// elements for the short FP64 step (k_cgs64)
static long part_cols(long nr) {
    const long a = tiles(nr), b = (nr + 255) / 256;
    return (nr <= CGS64_SHORT && b > a) ? b : a;
}

static rte_status apply_A_T(const KrylovOp& o, const double* x, double* y, cudaStream_t s) {
    return o.A64(o.ctx, x, y, s);
}
static rte_status apply_A_T(const KrylovOp& o, const float* x, float* y, cudaStream_t s) {
    return o.A32(o.ctx, x, y, s);
}

// weighted norm of v into *out (device)
template <typename T>
static rte_status dev_norm(const T* v, long nr, long nw1, double* part, double* out, cudaStream_t s) {
    const int nb = tiles(nr);
    k_mdot<T><<<nb, 256, 0, s>>>(v, nr, v, nullptr, 1, nw1, part);
    RTE_CUDA_TRY(cudaGetLastError());
    k_reduce<<<1, 256, 0, s>>>(part, nb, nullptr, 1, out, 1);
    RTE_CUDA_TRY(cudaGetLastError());
    rte_count_launches(2);
    return RTE_OK;
}

template <typename T> struct Gm {
    const KrylovOp* op;
    T* V;
    T* w;
    T* vin;
    T* Z = nullptr;  // right-preconditioned: z_j = M v_j, j = 0..m
    GmresDev* st;
    double* part;
    long nr, nw1;
    int m;
};

template <typename T>
static rte_status gm_setup(Gm<T>& G, const KrylovOp& o, KrylovWs& ws, int m, cudaStream_t s, bool pc) {
    G.op = &o;
    G.nr = o.nr;
    G.nw1 = o.nw1;
    G.m = m;
    if (ws.m != m || !ws.V) {
        krylov_free_ws(ws);
        if (rte_dev_malloc(&ws.V, (size_t)(m + 2) * o.nr * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return RTE_ENOMEM; }
        if (rte_dev_malloc(&ws.w, (size_t)o.nr * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return RTE_ENOMEM; }
        if (rte_dev_malloc((void**)&ws.part, (size_t)(GM_MMAX + 1) * part_cols(o.nr) * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return RTE_ENOMEM;
        }
        if (rte_dev_malloc((void**)&ws.st, sizeof(GmresDev)) != cudaSuccess) { cudaGetLastError(); return RTE_ENOMEM; }
        RTE_CUDA_TRY(cudaMemsetAsync(ws.st, 0, sizeof(GmresDev), s));
        ws.m = m;
    }
    if (pc && !ws.Z && rte_dev_malloc(&ws.Z, (size_t)(m + 1) * o.nr * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return RTE_ENOMEM;
    }
    G.V = (T*)ws.V;
    G.Z = (T*)ws.Z;
    G.vin = G.V + (long)(m + 1) * o.nr;  // slot m+1 is the matvec input
    G.w = (T*)ws.w;
    G.st = (GmresDev*)ws.st;
    G.part = ws.part;
    return RTE_OK;
}

// --------------------------------------------------------------------------
// MINRES (Paige & Saunders) for the inner solves of symmetric operators: for
// L = 0 the Nystrom matrix is symmetric (Sec. 2.3.1, Eq. iso_discretization),
// and the paper solves that case with MINRES.  Lanczos three-term recurrence
// with unnormalised vectors r1, r2 (rotating through three buffers B[0..2]
// by the step number), QR of the tridiagonal matrix by one Givens rotation
// per step, search directions w rotating through W[0..2], so a step streams
// a fixed number of vectors instead of the whole Arnoldi basis.  Step it
// (1-based), with v = vin the normalised Lanczos vector and y = A v:
//   alpha = v.(y - (beta/oldb) r1)            (k_mr_dot; r1 term from it = 2)
//   y' = y - (beta/oldb) r1 - (alpha/beta) r2, beta' = |y'|     (k_mr_upd)
//   delta = cs dbar + sn alpha,  gbar = sn dbar - cs alpha,
//   eps = sn beta',  dbar = -cs beta',  gamma = |(gbar, beta')|,
//   cs = gbar/gamma, sn = beta'/gamma, phi = cs phibar, phibar = sn phibar
//   w = (v - oldeps w1 - delta w2)/gamma, x += phi w, v = y'/beta'  (k_mr_sol)
// |phibar| is the residual norm of the inner system.  Dots in EFT
// arithmetic, scalars FP64; the "last block" reductions are those of the
// fused GMRES step (deterministic, nothing waits).
// --------------------------------------------------------------------------
__global__ void k_mr_start(GmresDev* st, const RefDev* ref, cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0) return;
    const int left = ref->maxit - ref->its;
    st->maxit = left < 1 ? 1 : left;
    st->its = 0;
    double tin = ref->inner_tol;  // as k_gm_start (mixed mode)
    const double need = ref->relres > 0.0 ? 0.5 * ref->tol / ref->relres : 1.0;
    if (need > tin) tin = need;
    st->tol = tin;
    const double b1 = st->nrm;
    st->mr_it = 1;
    st->mr_beta1 = b1;
    st->mr_beta = b1;
    st->mr_oldb = 0.0;
    st->mr_dbar = 0.0;
    st->mr_epsln = 0.0;
    st->mr_phibar = b1;
    st->mr_cs = -1.0;
    st->mr_sn = 0.0;
    st->target = tin * b1;
    st->res = b1;
    st->conv = !(b1 > st->target) ? 1 : 0;
    const bool go = isfinite(b1) && b1 > st->target;
    cudaGraphSetConditional(loop, go ? 1u : 0u);
}

// B[2] = rhs, vin = rhs / beta1, W[0..2] = 0, x = 0
__global__ void k_mr_init(const float* __restrict__ rhs, float* __restrict__ B, float* __restrict__ W,
                          float* __restrict__ vin, float* __restrict__ x, long nr, const GmresDev* __restrict__ st) {
    const double b1 = st->mr_beta1;
    const float inv = b1 > 0.0 ? (float)(1.0 / b1) : 0.f;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x) {
        const float r = rhs[e];
        B[2 * nr + e] = r;
        vin[e] = r * inv;
        W[e] = 0.f;
        W[nr + e] = 0.f;
        W[2 * nr + e] = 0.f;
        x[e] = 0.f;
    }
}

__global__ void __launch_bounds__(256) k_mr_dot(const float* __restrict__ v, const float* __restrict__ y,
                                                const float* __restrict__ B, GmresDev* __restrict__ st, long nr,
                                                long nw1, double* __restrict__ part) {
    const int it = st->mr_it;
    const float* r1 = B + (long)(it % 3) * nr;
    const bool two = it >= 2;
    const int nb = gridDim.x;
    __shared__ double red[2][8];
    __shared__ bool last;
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float ha = 0.f, la = 0.f, hc = 0.f, lc = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        if (e < nr) {
            const float vv = v[e] * (e < nw1 ? 1.f : 2.f);
            ff_fma(ha, la, vv, y[e]);
            if (two) ff_fma(hc, lc, vv, r1[e]);
        }
    }
    ff_warp_sum(ha, la);
    ff_warp_sum(hc, lc);
    if (lane == 0) {
        red[0][wid] = (double)ha + (double)la;
        red[1][wid] = (double)hc + (double)lc;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[threadIdx.x][q];
        part[(long)threadIdx.x * nb + blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->cnt1, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (wid < 2) {
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(part + (long)wid * nb + b);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[wid][0] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double c = two ? st->mr_beta / st->mr_oldb : 0.0;
        st->mr_alfa = red[0][0] - c * red[1][0];
        st->cnt1 = 0u;
    }
}

__global__ void __launch_bounds__(256) k_mr_upd(const float* __restrict__ y, float* __restrict__ B,
                                                GmresDev* __restrict__ st, long nr, long nw1,
                                                double* __restrict__ part, cudaGraphConditionalHandle loop) {
    const int it = st->mr_it;
    const float* r1 = B + (long)(it % 3) * nr;
    const float* r2 = B + (long)((it + 1) % 3) * nr;
    float* out = B + (long)((it + 2) % 3) * nr;
    const double beta = st->mr_beta;
    const float c1 = it >= 2 ? (float)(beta / st->mr_oldb) : 0.f;
    const float c2 = (float)(st->mr_alfa / beta);
    const int nb = gridDim.x;
    __shared__ double red[256];
    __shared__ bool last;
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        if (e < nr) {
            const float nv = fmaf(-c2, r2[e], fmaf(-c1, r1[e], y[e]));
            out[e] = nv;
            ff_fma(hi, lo, nv, nv * (e < nw1 ? 1.f : 2.f));
        }
    }
    ff_warp_sum(hi, lo);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)hi + (double)lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q];
        part[blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->cnt2, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(part + b);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double bnew = sqrt(red[0]);
    const double alfa = st->mr_alfa, cs = st->mr_cs, sn = st->mr_sn, dbar = st->mr_dbar;
    st->mr_oldb = beta;
    st->mr_beta = bnew;
    st->mr_oldeps = st->mr_epsln;
    st->mr_delta = cs * dbar + sn * alfa;
    const double gbar = sn * dbar - cs * alfa;
    st->mr_epsln = sn * bnew;
    st->mr_dbar = -cs * bnew;
    double gamma = hypot(gbar, bnew);
    if (!(gamma > 1e-300)) gamma = 1e-300;
    const double cn = gbar / gamma, snn = bnew / gamma;
    st->mr_cs = cn;
    st->mr_sn = snn;
    st->mr_gamma = gamma;
    st->mr_phi = cn * st->mr_phibar;
    st->mr_phibar = snn * st->mr_phibar;
    st->res = fabs(st->mr_phibar);
    st->its += 1;
    st->cnt2 = 0u;
    int stop = 0;
    if (st->res <= st->target) { stop = 1; st->conv = 1; }
    if (!(bnew > 1e-300) || !isfinite(st->res)) stop = 1;  // invariant subspace reached, or non-finite
    if (st->its >= st->maxit) stop = 1;
    st->stop = stop;
    cudaGraphSetConditional(loop, stop ? 0u : 1u);
}

__global__ void __launch_bounds__(256) k_mr_sol(float* __restrict__ vin, const float* __restrict__ B,
                                                float* __restrict__ W, float* __restrict__ x,
                                                GmresDev* __restrict__ st, long nr) {
    const int it = st->mr_it;
    const float* w1 = W + (long)(it % 3) * nr;
    const float* w2 = W + (long)((it + 1) % 3) * nr;
    float* wn = W + (long)((it + 2) % 3) * nr;
    const float* yn = B + (long)((it + 2) % 3) * nr;
    const float ig = (float)(1.0 / st->mr_gamma);
    const float oe = (float)st->mr_oldeps, dl = (float)st->mr_delta, ph = (float)st->mr_phi;
    const double bn = st->mr_beta;
    const float ib = bn > 1e-300 ? (float)(1.0 / bn) : 0.f;
    const int nb = gridDim.x;
    __shared__ bool last;
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        if (e < nr) {
            const float wv = (vin[e] - oe * w1[e] - dl * w2[e]) * ig;
            wn[e] = wv;
            x[e] = fmaf(ph, wv, x[e]);
            vin[e] = yn[e] * ib;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->cnt3, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (last && threadIdx.x == 0) {
        st->mr_it = it + 1;
        st->cnt3 = 0u;
    }
}

__global__ void k_mr_after(RefDev* ref, const GmresDev* st) {
    if (threadIdx.x != 0) return;
    ref->its += st->its;
    ref->outer += 1;
    ref->cycles += 1;
}

// one Arnoldi step (graph body)
template <typename T>
static rte_status arnoldi_body(Gm<T>& G, bool cgs2, bool pc, cudaGraphConditionalHandle loop, cudaStream_t s) {
    const long nr = G.nr;
    const int nb = tiles(nr), gr = grid_for(nr);
    rte_status e;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (pc) {  // right preconditioning: w = A (M v), M v kept in pv1
            e = G.op->pcA32(G.op->ctx, (const float*)G.vin, G.op->pv1, (float*)G.w, s);
        } else {
            e = apply_A_T(*G.op, G.vin, G.w, s);
        }
    } else {
        e = apply_A_T(*G.op, G.vin, G.w, s);
    }
    if (e != RTE_OK) return e;
    const int* jp = &G.st->j;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (!cgs2) {
            const float* zs = pc ? G.op->pv1 : nullptr;
            float* Zs = pc ? (float*)G.Z : nullptr;
            if (nr % 4 == 0) {
                RTE_CUDA_TRY(launch_pdl(k_step_dot4, dim3(nb), dim3(256), 0, s, (float*)G.V, nr,
                                        (const float*)G.w, G.st, G.nw1, G.part));
                RTE_CUDA_TRY(launch_pdl(k_step_upd4, dim3(nb), dim3(256), 0, s, (const float*)G.V, nr,
                                        (const float*)G.w, (float*)G.vin, G.st, G.nw1, G.part, loop, zs, Zs));
            } else {
                RTE_CUDA_TRY(launch_pdl(k_step_dot, dim3(nb), dim3(256), 0, s, (float*)G.V, nr, (const float*)G.w,
                                        G.st, G.nw1, G.part));
                RTE_CUDA_TRY(launch_pdl(k_step_upd, dim3(nb), dim3(256), 0, s, (const float*)G.V, nr,
                                        (const float*)G.w, (float*)G.vin, G.st, G.nw1, G.part, loop, zs, Zs));
            }
            rte_count_launches(2);
            return RTE_OK;
        }
    }
    if constexpr (sizeof(T) == sizeof(double)) {
        if (cgs2 && nr <= CGS64_SHORT) {
            const long chunk = 256;
            const unsigned nbs = (unsigned)((nr + chunk - 1) / chunk);
            double* V = (double*)G.V;
            double* w = (double*)G.w;
            k_cgs64<0><<<nbs, 256, 0, s>>>(V, nr, w, G.st, G.nw1, G.part, chunk, loop);
            k_cgs64<1><<<nbs, 256, 0, s>>>(V, nr, w, G.st, G.nw1, G.part, chunk, loop);
            k_cgs64<2><<<nbs, 256, 0, s>>>(V, nr, w, G.st, G.nw1, G.part, chunk, loop);
            // after the Givens update st->j is the new basis index
            k_scale_basis<double><<<gr, 256, 0, s>>>(w, V, (double*)G.vin, nr, G.st, 0);
            rte_count_launches(4);
            RTE_CUDA_TRY(cudaGetLastError());
            return RTE_OK;
        }
    }
    k_mdot<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, jp, 1, G.nw1, G.part);
    k_reduce<<<G.m + 1, 256, 0, s>>>(G.part, nb, jp, 1, G.st->hA, 0);
    rte_count_launches(2);
    if (cgs2) {
        k_maxpy<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, G.st->hA, jp, 1, -1.0, G.nw1, nullptr);
        k_mdot<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, jp, 1, G.nw1, G.part);
        k_reduce<<<G.m + 1, 256, 0, s>>>(G.part, nb, jp, 1, G.st->hB, 0);
        k_maxpy<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, G.st->hB, jp, 1, -1.0, G.nw1, G.part);
        rte_count_launches(4);
    } else {
        k_maxpy<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, G.st->hA, jp, 1, -1.0, G.nw1, G.part);
        rte_count_launches(1);
    }
    k_reduce<<<1, 256, 0, s>>>(G.part, nb, nullptr, 1, &G.st->nrm, 1);
    k_scale_basis<T><<<gr, 256, 0, s>>>(G.w, G.V, G.vin, nr, G.st, 1);
    k_givens<<<1, 32, 0, s>>>(G.st, loop);
    rte_count_launches(3);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// Stream-capture helper that appends to a graph after one dependency node
// and reports the new sink (the capture frontier).
struct Seg {
    cudaStream_t cs;
    cudaGraph_t g;
    cudaGraphNode_t dep;
    long long k0;
};

static rte_status seg_begin(Seg& S, cudaStream_t cs, cudaGraph_t g, cudaGraphNode_t dep) {
    S.cs = cs;
    S.g = g;
    S.dep = dep;
    S.k0 = rte_kernel_launches();
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, g, dep ? &S.dep : nullptr, nullptr, dep ? 1 : 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return rte_cuda_fail(e, "begin capture");
    return RTE_OK;
}

// ends the capture; *sink = last node (unchanged if nothing was captured);
// *kernels = kernels captured in this segment
static rte_status seg_end(Seg& S, cudaGraphNode_t* sink, long long* kernels) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(S.cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
    cudaGraphNode_t last = (e == cudaSuccess && nd == 1) ? deps[0] : S.dep;
    cudaGraph_t gg = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(S.cs, &gg);
    if (e != cudaSuccess) return rte_cuda_fail(e, "capture info");
    if (e2 != cudaSuccess) return rte_cuda_fail(e2, "end capture");
    if (nd > 1) return rte_cuda_fail(cudaErrorInvalidValue, "capture frontier has several nodes");
    *sink = last;
    if (kernels) *kernels += rte_kernel_launches() - S.k0;
    return RTE_OK;
}

static rte_status add_cond(cudaGraph_t g, cudaGraphNode_t* dep, cudaGraphConditionalHandle h,
                           cudaGraphConditionalNodeType type, cudaGraph_t* body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddNode(&node, g, *dep ? dep : nullptr, nullptr, *dep ? 1 : 0, &cp);
    if (e != cudaSuccess) return rte_cuda_fail(e, "add conditional node");
    *body = cp.conditional.phGraph_out[0];
    *dep = node;
    return RTE_OK;
}

#define SEG(graph, dep, cnt, ...)                                                     \
    do {                                                                              \
        Seg S_;                                                                       \
        rte_status e_ = seg_begin(S_, cs, graph, dep);                                \
        if (e_ != RTE_OK) return e_;                                                  \
        rte_status b_ = [&]() -> rte_status { __VA_ARGS__ return RTE_OK; }();         \
        rte_status f_ = seg_end(S_, &dep, cnt);                                       \
        if (b_ != RTE_OK) return b_;                                                  \
        if (f_ != RTE_OK) return f_;                                                  \
    } while (0)

#define TRYS(x)                        \
    do {                               \
        rte_status t_ = (x);           \
        if (t_ != RTE_OK) return t_;   \
    } while (0)

// Append the whole solve of plan p (precision T: double = plain FP64 GMRES,
// float = FP32 inner GMRES + FP64 refinement) to graph g after *dep.
// Inputs/outputs are the plan's own f_dev / u_dev; options are read from
// the plan's device RefDev at run time.
template <typename T>
static rte_status build_solve(const KrylovOp& o, KrylovWs& ws, int m, bool minres, bool pc, cudaGraph_t g,
                              cudaGraphNode_t* dep_io,
                              cudaStream_t cs, SolveGraphInfo* info) {
    const bool mixed = sizeof(T) == sizeof(float);
    const bool use_mr = mixed && minres && m >= 5;  // MINRES buffers: basis slots 0..5
    const bool use_pc = mixed && pc && !use_mr && o.pcA32;  // preconditioned inner GMRES
    const bool cgs2 = !mixed;
    Gm<T> G;
    TRYS(gm_setup<T>(G, o, ws, m, cs, use_pc));
    RTE_CUDA_TRY(cudaStreamSynchronize(cs));
    const long nr = o.nr;
    const int gr = grid_for(nr), nb = tiles(nr);
    const long nw1 = G.nw1;
    RefDev* ref = (RefDev*)o.ref;
    T* rhs = mixed ? (T*)o.r32 : (T*)o.r64;
    T* x = mixed ? (T*)o.d32 : (T*)o.x64;
    cudaGraphConditionalHandle c_guess = 0, c_outer = 0, c_cycle = 0, c_loop = 0, c_restart = 0;
    // every handle must belong to a conditional node of the graph: the
    // restart-cycle handles exist only with GMRES inner solves
    RTE_CUDA_TRY(cudaGraphConditionalHandleCreate(&c_guess, g, 0, cudaGraphCondAssignDefault));
    RTE_CUDA_TRY(cudaGraphConditionalHandleCreate(&c_outer, g, 0, cudaGraphCondAssignDefault));
    RTE_CUDA_TRY(cudaGraphConditionalHandleCreate(&c_loop, g, 0, cudaGraphCondAssignDefault));
    if (!use_mr) {
        RTE_CUDA_TRY(cudaGraphConditionalHandleCreate(&c_cycle, g, 0, cudaGraphCondAssignDefault));
        RTE_CUDA_TRY(cudaGraphConditionalHandleCreate(&c_restart, g, 0, cudaGraphCondAssignDefault));
    }
    cudaGraphNode_t dep = *dep_io;
    *info = SolveGraphInfo();
    // T.1 and start values
    // FP64-accurate applications: float-float on the FP32 units in the mixed
    // mode, native FP64 in the plain FP64 mode.  The mixed mode forms b = K~ f
    // in FP32 only (it is the first inner right-hand side and sets ||b||) and
    // every residual as r = K~ (mu_s sigma_hat u + f) - u: one FP64-accurate
    // application that equals b - (I - K) u with the exact b.
    auto residual = [&]() -> rte_status { return o.resid(o.ctx, mixed ? 1 : 0, cs); };
    SEG(g, dep, &info->k_fixed, {
        TRYS(o.rhs(o.ctx, mixed ? 1 : 0, cs));
        TRYS(dev_norm<double>(o.b64, nr, nw1, o.part64, &ref->bnorm, cs));
        k_ref_start<<<1, 32, 0, cs>>>(ref, c_guess);
        k_zero_unless_guess<<<gr, 256, 0, cs>>>(o.u, nr, ref);
        k_copy_vec<<<gr, 256, 0, cs>>>(o.b64, o.r64, nr);
        rte_count_launches(3);
    });
    // residual of a guess
    {
        cudaGraph_t body;
        TRYS(add_cond(g, &dep, c_guess, cudaGraphCondTypeIf, &body));
        cudaGraphNode_t d = nullptr;
        SEG(body, d, &info->k_guess, {
            TRYS(residual());
            TRYS(dev_norm<double>(o.r64, nr, nw1, o.part64, &ref->rnorm, cs));
            k_guess_fallback<<<gr, 256, 0, cs>>>(o.u, o.r64, o.b64, nr, ref);
            k_guess_fallback_state<<<1, 32, 0, cs>>>(ref);
            k_ref_relres<<<1, 32, 0, cs>>>(ref);
            rte_count_launches(3);
        });
    }
    SEG(g, dep, &info->k_fixed, {
        k_ref_gate<<<1, 32, 0, cs>>>(ref, c_outer);
        rte_count_launches(1);
    });
    // refinement loop
    cudaGraph_t outer_body;
    TRYS(add_cond(g, &dep, c_outer, cudaGraphCondTypeWhile, &outer_body));
    if constexpr (sizeof(T) == sizeof(float)) {
        if (use_mr) {
            // inner solve: MINRES on the FP32 operator
            cudaGraphNode_t d = nullptr;
            float* B = (float*)G.V;
            float* W = B + 3 * nr;
            SEG(outer_body, d, &info->k_outer, {
                k_scale_inv<double, float><<<gr, 256, 0, cs>>>(o.r64, o.r32, nr, &ref->rnorm);
                rte_count_launches(1);
            });
            SEG(outer_body, d, &info->k_cycle, {
                TRYS(dev_norm<float>((const float*)rhs, nr, nw1, G.part, &G.st->nrm, cs));
                k_mr_start<<<1, 32, 0, cs>>>(G.st, ref, c_loop);
                k_mr_init<<<gr, 256, 0, cs>>>((const float*)rhs, B, W, (float*)G.vin, (float*)x, nr, G.st);
                rte_count_launches(2);
            });
            cudaGraph_t loop_body;
            TRYS(add_cond(outer_body, &d, c_loop, cudaGraphCondTypeWhile, &loop_body));
            {
                cudaGraphNode_t dl = nullptr;
                SEG(loop_body, dl, &info->k_step, {
                    TRYS(apply_A_T(o, (const float*)G.vin, (float*)G.w, cs));
                    k_mr_dot<<<nb, 256, 0, cs>>>((const float*)G.vin, (const float*)G.w, B, G.st, nr, nw1, G.part);
                    k_mr_upd<<<nb, 256, 0, cs>>>((const float*)G.w, B, G.st, nr, nw1, G.part, c_loop);
                    k_mr_sol<<<nb, 256, 0, cs>>>((float*)G.vin, B, W, (float*)x, G.st, nr);
                    rte_count_launches(3);
                });
            }
            SEG(outer_body, d, &info->k_outer, {
                k_axpy_scaled<float><<<gr, 256, 0, cs>>>(o.u, (const float*)x, nr, &ref->rnorm);
                k_mr_after<<<1, 32, 0, cs>>>(ref, G.st);
                rte_count_launches(2);
                TRYS(residual());
                TRYS(dev_norm<double>(o.r64, nr, nw1, o.part64, &ref->rnorm, cs));
                k_ref_check<<<1, 32, 0, cs>>>(ref, c_outer);
                rte_count_launches(1);
            });
            *dep_io = dep;
            return RTE_OK;
        }
    }
    {
        cudaGraphNode_t d = nullptr;
        SEG(outer_body, d, &info->k_outer, {
            if (mixed) {
                k_scale_inv<double, float><<<gr, 256, 0, cs>>>(o.r64, o.r32, nr, &ref->rnorm);
                rte_count_launches(1);
            }
            k_zero_T<T><<<gr, 256, 0, cs>>>(x, nr);
            k_copy_T<T><<<gr, 256, 0, cs>>>(rhs, G.w, nr);
            k_gm_start<<<1, 32, 0, cs>>>(G.st, ref, m, cgs2 ? 1 : 0, c_cycle);
            rte_count_launches(3);
        });
        cudaGraph_t cycle_body;
        TRYS(add_cond(outer_body, &d, c_cycle, cudaGraphCondTypeWhile, &cycle_body));
        {
            cudaGraphNode_t dc = nullptr;
            SEG(cycle_body, dc, &info->k_cycle, {
                TRYS(dev_norm<T>(G.w, nr, nw1, G.part, &G.st->nrm, cs));
                k_cycle_init<<<1, 32, 0, cs>>>(G.st, c_loop);
                k_scale_basis<T><<<gr, 256, 0, cs>>>(G.w, G.V, G.vin, nr, G.st, 0);
                rte_count_launches(2);
            });
            cudaGraph_t loop_body;
            TRYS(add_cond(cycle_body, &dc, c_loop, cudaGraphCondTypeWhile, &loop_body));
            {
                cudaGraphNode_t dl = nullptr;
                SEG(loop_body, dl, &info->k_step, { TRYS(arnoldi_body<T>(G, cgs2, use_pc, c_loop, cs)); });
            }
            SEG(cycle_body, dc, &info->k_cycle, {
                k_solve_tri<<<1, 32, 0, cs>>>(G.st);
                if (use_pc) {
                    // x += M (V y) = Z y: the steps stored z_j = M v_j
                    k_maxpy<T><<<nb, 256, 0, cs>>>((const T*)G.Z, nr, x, G.st->y, &G.st->j, 0, 1.0, nw1, nullptr);
                    rte_count_launches(1);
                } else {
                    k_maxpy<T><<<nb, 256, 0, cs>>>(G.V, nr, x, G.st->y, &G.st->j, 0, 1.0, nw1, nullptr);
                    rte_count_launches(1);
                }
                k_cycle_end<<<1, 32, 0, cs>>>(G.st, ref, c_cycle, c_restart);
                rte_count_launches(2);
            });
            cudaGraph_t restart_body;
            TRYS(add_cond(cycle_body, &dc, c_restart, cudaGraphCondTypeIf, &restart_body));
            {
                cudaGraphNode_t dr = nullptr;
                SEG(restart_body, dr, &info->k_restart, {
                    TRYS(apply_A_T(o, x, G.w, cs));
                    k_rsub<T><<<gr, 256, 0, cs>>>(rhs, G.w, nr);
                    rte_count_launches(1);
                });
            }
        }
        SEG(outer_body, d, &info->k_outer, {
            if (mixed) {
                k_axpy_scaled<float><<<gr, 256, 0, cs>>>(o.u, (const float*)x, nr, &ref->rnorm);
            } else {
                k_add64<<<gr, 256, 0, cs>>>(o.u, (const double*)x, nr);
            }
            k_ref_after<<<1, 32, 0, cs>>>(ref, G.st);
            rte_count_launches(2);
            TRYS(residual());
            TRYS(dev_norm<double>(o.r64, nr, nw1, o.part64, &ref->rnorm, cs));
            k_ref_check<<<1, 32, 0, cs>>>(ref, c_outer);
            rte_count_launches(1);
        });
    }
    *dep_io = dep;
    return RTE_OK;
}

// captured, not executed: take the capture-time counts back out
struct CountGuard {
    long long c0;
    CountGuard() : c0(rte_kernel_launches()) {}
    ~CountGuard() { rte_count_launches(-(rte_kernel_launches() - c0)); }
};

// MINRES inner solves: requested, symmetric operator (L = 0), mixed mode
bool solve_uses_minres(const rte_plan p, const rte_opts* o) {
    return o->prec != RTE_PREC_FP64 && p->L == 0 && o->inner_solver == RTE_INNER_MINRES && o->restart >= 5;
}

// periodic preconditioner for the FP32 inner GMRES: requested, mixed mode,
// GMRES inner solves, and a plan shape the preconditioner supports
bool solve_uses_precond(const rte_plan p, const rte_opts* o) {
    return o->prec != RTE_PREC_FP64 && o->precond != 0 && !solve_uses_minres(p, o) && plan_precond_supported(p);
}

// the plan as a KrylovOp: its own f_dev / u_dev and work vectors
static rte_status plan_A32(void* c, const float* x, float* y, cudaStream_t s) {
    return plan_apply32((rte_plan)c, x, y, 1.0f, -1.0f, 0.0f, nullptr, s);
}
static rte_status plan_A64(void* c, const double* x, double* y, cudaStream_t s) {
    return plan_apply64((rte_plan)c, MIX_K, x, y, 1.0, -1.0, 0.0, nullptr, s);
}
static rte_status plan_pcA(void* c, const float* x, float* z, float* y, cudaStream_t s) {
    return plan_apply_pcA32((rte_plan)c, x, z, y, s);
}
// mixed: b = K~ f in FP32 (the first inner right-hand side; it sets ||b||),
// widened; FP64: one native FP64 application
static rte_status plan_rhs(void* c, int mixed, cudaStream_t s) {
    rte_plan p = (rte_plan)c;
    if (!mixed) return plan_apply64(p, MIX_RHS, p->f_dev, p->b64, 0.0, 1.0, 0.0, nullptr, s);
    TRYS(plan_rhs32(p, (float*)p->r32, s));
    k_widen<<<grid_for(p->nr), 256, 0, s>>>((const float*)p->r32, p->b64, p->nr);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}
// FP64-accurate residuals: float-float on the FP32 units in the mixed mode,
// r = K~ (mu_s sigma_hat u + f) - u in one application (equal to
// b - (I - K) u with the exact b); native FP64 in the FP64 mode
static rte_status plan_resid(void* c, int mixed, cudaStream_t s) {
    rte_plan p = (rte_plan)c;
    if (mixed) return plan_apply64e(p, MIX_KF, p->u_dev, p->r64, -1.0, 1.0, 0.0, nullptr, s);
    return plan_apply64(p, MIX_K, p->u_dev, p->r64, -1.0, 1.0, 1.0, p->b64, s);
}

static KrylovOp plan_krylov_op(rte_plan p) {
    KrylovOp o;
    o.ctx = p;
    o.nr = p->nr;
    o.nw1 = p->dim == 2 ? 2L * p->n * p->n : p->nr;
    o.u = p->u_dev;
    o.b64 = p->b64;
    o.r64 = p->r64;
    o.x64 = (double*)p->x64;
    o.part64 = p->part64;
    o.r32 = (float*)p->r32;
    o.d32 = (float*)p->d32;
    o.pv1 = p->pv1;
    o.ref = p->ref;
    o.A32 = plan_A32;
    o.A64 = plan_A64;
    o.pcA32 = plan_pcA;
    o.rhs = plan_rhs;
    o.resid = plan_resid;
    return o;
}

rte_status solve_graph_append(rte_plan p, int prec, int m, bool minres, bool pc, cudaGraph_t g,
                              cudaGraphNode_t* dep, cudaStream_t cs, SolveGraphInfo* info) {
    CountGuard guard;
    const rte_prec saved = p->opts.prec;
    p->opts.prec = (rte_prec)prec;  // selects the inner spectra precision at capture
    const KrylovOp o = plan_krylov_op(p);
    rte_status st = prec == RTE_PREC_FP64 ? build_solve<double>(o, p->k64, m, false, false, g, dep, cs, info)
                                          : build_solve<float>(o, p->k32, m, minres, pc, g, dep, cs, info);
    p->opts.prec = saved;
    return st;
}

rte_status krylov_op_graph(const KrylovOp& o, KrylovWs& ws, int prec, int m, cudaStream_t s, void** exec,
                           SolveGraphInfo* info) {
    *exec = nullptr;
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    cudaGraph_t g = nullptr;
    RTE_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return rte_cuda_fail(e, "krylov_op_graph");
    }
    cudaGraphNode_t dep = nullptr;
    rte_status st;
    {
        CountGuard guard;
        *info = SolveGraphInfo();
        st = prec == RTE_PREC_FP64 ? build_solve<double>(o, ws, m, false, false, g, &dep, cs, info)
                                   : build_solve<float>(o, ws, m, false, false, g, &dep, cs, info);
    }
    cudaStreamDestroy(cs);
    if (st == RTE_OK) {
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) st = rte_cuda_fail(e, "instantiate solve graph");
        else *exec = ex;
    }
    cudaGraphDestroy(g);
    return st;
}

static rte_status get_solve_graph(rte_plan p, int prec, int m, bool minres, bool pc, cudaStream_t s,
                                  cudaGraphExec_t* out) {
    SolveGraph& sg = p->graphs[prec];
    if (sg.exec && sg.m == m && sg.minres == minres && sg.pc == pc) {
        *out = (cudaGraphExec_t)sg.exec;
        return RTE_OK;
    }
    if (sg.exec) cudaGraphExecDestroy((cudaGraphExec_t)sg.exec);
    sg.exec = nullptr;
    // workspace allocations happen here, before the capture
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    cudaGraph_t g = nullptr;
    RTE_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaStream_t cs;
    RTE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraphNode_t dep = nullptr;
    rte_status st = pc ? plan_precond_build(p, s) : RTE_OK;  // allocates: before the capture
    if (st == RTE_OK) st = solve_graph_append(p, prec, m, minres, pc, g, &dep, cs, &sg.info);
    cudaStreamDestroy(cs);
    if (st == RTE_OK) {
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) st = rte_cuda_fail(e, "instantiate solve graph");
        else { sg.exec = ex; sg.m = m; sg.minres = minres; sg.pc = pc; *out = ex; }
    }
    cudaGraphDestroy(g);
    return st;
}

// options into the device RefDev (from the plan's pinned staging area)
rte_status solve_set_options(rte_plan p, const rte_opts* o, cudaStream_t s) {
    RefDev* h = (RefDev*)(p->hst + 32);
    memset(h, 0, sizeof(RefDev));
    h->max_outer = o->prec == RTE_PREC_FP64 ? 4 : 40;
    h->maxit = o->maxit;
    h->use_guess = o->use_guess ? 1 : 0;
    h->mixed = o->prec != RTE_PREC_FP64;
    h->tol = o->tol;
    h->inner_tol = o->inner_tol;
    RTE_CUDA_TRY(cudaMemcpyAsync(p->ref, h, sizeof(RefDev), cudaMemcpyHostToDevice, s));
    return RTE_OK;
}

static rte_status collect_core(const SolveGraphInfo& gi, int prec, const RefDev* hr, double rho, double ms_pre,
                               rte_stats* stats, double ms) {
    rte_count_launches(gi.k_fixed + (hr->use_guess ? gi.k_guess : 0) + (long long)hr->outer * gi.k_outer +
                       (long long)hr->cycles * gi.k_cycle + (long long)hr->its * gi.k_step +
                       (long long)hr->restarts * gi.k_restart);
    if (stats) {
        const double cond = rho < 1.0 ? (1.0 + rho) / (1.0 - rho) : INFINITY;
        stats->iters = hr->its;
        stats->outer = prec == RTE_PREC_FP64 ? 0 : hr->outer;
        stats->relres_true = hr->relres;
        stats->converged = hr->relres <= hr->tol ? 1 : 0;
        stats->ms_total = ms;
        stats->ms_pre = ms_pre;
        stats->est_err_bound = cond * hr->relres;
    }
    if (hr->status == 7 || !isfinite(hr->relres)) return RTE_ENAN;
    if (!(hr->relres <= hr->tol)) return RTE_ENOCONV;
    return RTE_OK;
}

rte_status solve_collect(rte_plan p, int prec, const RefDev* hr, rte_stats* stats, double ms) {
    const double rho = p->mu_t > 0 ? p->mu_s / p->mu_t : 0.0;
    return collect_core(p->graphs[prec].info, prec, hr, rho, p->ms_pre, stats, ms);
}

rte_status krylov_op_run(const KrylovOp& op, void* exec, const SolveGraphInfo& info, const rte_opts* o, void* hst,
                         double rho, double ms_pre, rte_stats* stats, cudaStream_t s) {
    RefDev* h = (RefDev*)hst;
    RefDev* hr = h + 1;
    fill_ref_template(h, o);
    cudaEvent_t ev0, ev1;
    RTE_CUDA_TRY(cudaEventCreate(&ev0));
    cudaError_t e = cudaEventCreate(&ev1);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev0);
        return rte_cuda_fail(e, "krylov_op_run");
    }
    e = cudaMemcpyAsync(op.ref, h, sizeof(RefDev), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch((cudaGraphExec_t)exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr, op.ref, sizeof(RefDev), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (e != cudaSuccess) return rte_cuda_fail(e, "krylov_op_run");
    return collect_core(info, (int)o->prec, hr, rho, ms_pre, stats, ms);
}

size_t refdev_size() { return sizeof(RefDev); }

// Solve for the plan's f_dev into u_dev (both plan-owned), one graph launch.
rte_status krylov_solve(rte_plan p, const rte_opts* o, rte_stats* stats, cudaStream_t s, void* u_out,
                        cudaMemcpyKind kind) {
    cudaGraphExec_t ex = nullptr;
    const int prec = (int)o->prec;
    // the FP64 workspace is only needed by the FP64 mode
    rte_status st = get_solve_graph(p, prec, o->restart, solve_uses_minres(p, o), solve_uses_precond(p, o), s, &ex);
    if (st != RTE_OK) return st;
    for (int i = 0; i < 2; ++i)
        if (!p->ev[i]) RTE_CUDA_TRY(cudaEventCreate((cudaEvent_t*)&p->ev[i]));
    cudaEvent_t ev0 = (cudaEvent_t)p->ev[0], ev1 = (cudaEvent_t)p->ev[1];
    st = solve_set_options(p, o, s);
    if (st != RTE_OK) return st;
    RTE_CUDA_TRY(cudaEventRecord(ev0, s));
    RTE_CUDA_TRY(cudaGraphLaunch(ex, s));
    RTE_CUDA_TRY(cudaEventRecord(ev1, s));
    RefDev* hr = (RefDev*)(p->hst + 16);
    RTE_CUDA_TRY(cudaMemcpyAsync(hr, p->ref, sizeof(RefDev), cudaMemcpyDeviceToHost, s));
    if (u_out) RTE_CUDA_TRY(cudaMemcpyAsync(u_out, p->u_dev, p->nr * sizeof(double), kind, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    return solve_collect(p, prec, hr, stats, ms);
}

void krylov_free_ws(KrylovWs& ws) {
    if (ws.V) rte_dev_free(ws.V);
    if (ws.w) rte_dev_free(ws.w);
    if (ws.part) rte_dev_free(ws.part);
    if (ws.st) rte_dev_free(ws.st);
    if (ws.Z) rte_dev_free(ws.Z);
    ws = KrylovWs();
}

rte_status krylov_free(rte_plan p) {
    for (int i = 0; i < 2; ++i)
        if (p->ev[i]) {
            cudaEventDestroy((cudaEvent_t)p->ev[i]);
            p->ev[i] = nullptr;
        }
    for (int i = 0; i < 3; ++i) {
        if (p->graphs[i].exec) cudaGraphExecDestroy((cudaGraphExec_t)p->graphs[i].exec);
        p->graphs[i] = SolveGraph();
    }
    krylov_free_ws(p->k64);
    krylov_free_ws(p->k32);
    return RTE_OK;
}

// --------------------------------------------------------------------------
// batch support: options from a device template, state out to a packed array
// --------------------------------------------------------------------------
__global__ void k_ref_load(RefDev* ref, const RefDev* __restrict__ tmpl) {
    if (threadIdx.x == 0) *ref = *tmpl;
}
__global__ void k_ref_store(const RefDev* __restrict__ ref, RefDev* __restrict__ dst) {
    if (threadIdx.x == 0) *dst = *ref;
}

void launch_ref_load(rte_plan p, const void* tmpl, cudaStream_t s) {
    k_ref_load<<<1, 32, 0, s>>>((RefDev*)p->ref, (const RefDev*)tmpl);
    rte_count_launches(1);
}
void launch_ref_store(rte_plan p, void* dst, cudaStream_t s) {
    k_ref_store<<<1, 32, 0, s>>>((const RefDev*)p->ref, (RefDev*)dst);
    rte_count_launches(1);
}
void launch_copy(const double* src, double* dst, long n, cudaStream_t s) {
    k_copy_vec<<<grid_for(n), 256, 0, s>>>(src, dst, n);
    rte_count_launches(1);
}
// host image of the options template (same fields solve_set_options writes)
void fill_ref_template(void* host, const rte_opts* o) {
    RefDev* h = (RefDev*)host;
    memset(h, 0, sizeof(RefDev));
    h->max_outer = o->prec == RTE_PREC_FP64 ? 4 : 40;
    h->maxit = o->maxit;
    h->use_guess = 0;
    h->mixed = o->prec != RTE_PREC_FP64;
    h->tol = o->tol;
    h->inner_tol = o->inner_tol;
}
