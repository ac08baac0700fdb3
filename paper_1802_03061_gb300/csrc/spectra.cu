// Plan-time work: FFT schedules, twiddle tables, singular-cell weights,
// kernel sampling on the periodic zero-padded grid and the kernel spectra.
//
// Sec. 2.3.1: kappa is extended periodically from [-1,1]^d and the field is
// zero padded, so the Nystrom matrix becomes circulant; its "Fourier modes"
// are precomputed once.  Sec. 3.3.1: for the mode-coupled kernels the same is
// done per angular difference m = k - k'.
#include <math.h>
#include <stdio.h>

#include "fft.cuh"
#include "internal.h"

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
static bool smooth23(int q) {
    while (q % 2 == 0) q /= 2;
    while (q % 3 == 0) q /= 3;
    return q == 1;
}

int choose_Q(int n) {
    // smallest even 2^a 3^b with Q >= 2n - 1 (offsets -(n-1)..(n-1) must not wrap)
    int q = 2 * n - 1;
    if (q < 2) q = 2;
    while (q % 2 || !smooth23(q)) ++q;
    return q;
}

// mode-axis FFT length: the smallest 2^a 3^b >= 4L + 1 (at least 2); every
// difference k - k' in -2L..2L then has its own residue mod P
int choose_P(int L) {
    int q = 4 * L + 1;
    if (q < 2) q = 2;
    while (!smooth23(q)) ++q;
    return q;
}

void make_sched(FftSched* s, int Q) {
    s->Q = Q;
    s->ns = 0;
    int q = Q, twos = 0;
    while (q % 2 == 0) { q /= 2; ++twos; }
    int threes = 0;
    while (q % 3 == 0) { q /= 3; ++threes; }
    // powers of two: as many radix-8 stages as possible, then one 4 or 2
    while (twos >= 3) { s->radix[s->ns++] = 8; twos -= 3; }
    if (twos == 2) s->radix[s->ns++] = 4;
    if (twos == 1) s->radix[s->ns++] = 2;
    for (int i = 0; i < threes; ++i) s->radix[s->ns++] = 3;
}

// ---------------------------------------------------------------------------
// twiddles: tw[t] = exp(-2 pi i t / Q)
// ---------------------------------------------------------------------------
__global__ void k_twiddles(double2* tw64, float2* tw32, int Q) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Q) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)Q, &s, &c);
    tw64[t] = make_double2(c, -s);
    tw32[t] = make_float2((float)c, (float)-s);
}

// 2D singular-cell weights (Sec. 2.3, diagonal of Eq. iso_discretization):
// D_m = int_cell kappa(r) e^{i m theta} dr
//     = (1/2pi) int_0^{2pi} cos(m phi) (1 - e^{-mu R(phi)})/mu dphi,
// R(phi) = (h/2)/max(|cos|,|sin|).  Eight smooth pieces between the corner
// directions, 64-point Gauss-Legendre on each.  One block of 64 threads.
__global__ void k_cell_weights_2d(double mu, double h, int mmax, double* D) {
    __shared__ double acc[64];
    const int i = threadIdx.x;
    double x, w;
    gl_node(64, i, &x, &w);
    const double a = 0.5 * h;
    double c1[8], cm1[8], cm2[8], rad[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const double phi = q * (M_PI / 4) + (x + 1.0) * (M_PI / 8);
        double s, c;
        sincos(phi, &s, &c);
        const double R = a / fmax(fabs(c), fabs(s));
        rad[q] = radial_factor(mu, R) * w * (M_PI / 8);
        c1[q] = c;
        cm2[q] = 1.0;
        cm1[q] = c;
    }
    // cos(m phi) by the Chebyshev recurrence c_m = 2 cos(phi) c_{m-1} - c_{m-2};
    // one block reduction per m (mmax up to 2 RTE_MAX_L)
    for (int m = 0; m <= mmax; ++m) {
        double part = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            double cur;
            if (m == 0) cur = 1.0;
            else if (m == 1) cur = c1[q];
            else {
                cur = 2.0 * c1[q] * cm1[q] - cm2[q];
                cm2[q] = cm1[q];
                cm1[q] = cur;
            }
            part += cur * rad[q];
        }
        acc[i] = part;
        __syncthreads();
        if (i == 0) {
            double t = 0.0;
            for (int j = 0; j < 64; ++j) t += acc[j];
            D[m] = t / (2.0 * M_PI);
        }
        __syncthreads();
    }
}

// 3D singular-cell weight: D = (1/4pi) int_{S^2} (1-e^{-mu R})/mu dOmega,
// written over the six faces: for the face z = a the solid angle element is
// a dx dy / rho^3 and R = rho = sqrt(x^2+y^2+a^2).  The face integrand is
// analytic (rho >= a); 4 quadrants x 64^2 Gauss-Legendre.  One block of 64.
__global__ void k_cell_weight_3d(double mu, double h, double* D) {
    __shared__ double xs[64], ws[64], acc[64];
    const int i = threadIdx.x;
    double x, w;
    gl_node(64, i, &x, &w);
    const double a = 0.5 * h;
    xs[i] = 0.5 * a * (x + 1.0);  // nodes on [0, a]
    ws[i] = 0.5 * a * w;
    __syncthreads();
    double t = 0.0;
    for (int j = 0; j < 64; ++j) {
        const double r2 = xs[i] * xs[i] + xs[j] * xs[j] + a * a;
        const double rho = sqrt(r2);
        t += ws[i] * ws[j] * radial_factor(mu, rho) * a / (r2 * rho);
    }
    acc[i] = t;
    __syncthreads();
    if (i == 0) {
        double s = 0.0;
        for (int j = 0; j < 64; ++j) s += acc[j];
        D[0] = 6.0 * 4.0 * s / (4.0 * M_PI);
    }
}

// ---------------------------------------------------------------------------
// kernel sampling: g_m[o] on the Q^2 periodic grid (Sec. 2.3.1 / 3.3.1)
//   g_m(o) = h^2 kappa(o h) exp(-i m theta(o)),  0 < |o|, all |o_i| <= n-1
//   g_m(0) = D_m,   zero elsewhere (padding)
// stored G[m][oy][ox] complex
// ---------------------------------------------------------------------------
__global__ void k_sample_2d(double2* G, int n, int Q, int mmax, double h, double mu, const double* D) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long P = (long)Q * Q;
    if (idx >= P) return;
    const int ox = (int)(idx % Q), oy = (int)(idx / Q);
    const int sx = ox < Q / 2 ? ox : ox - Q;
    const int sy = oy < Q / 2 ? oy : oy - Q;
    if (abs(sx) >= n || abs(sy) >= n) {
        for (int m = 0; m <= mmax; ++m) G[m * P + idx] = make_double2(0.0, 0.0);
        return;
    }
    if (sx == 0 && sy == 0) {
        for (int m = 0; m <= mmax; ++m) G[m * P + idx] = make_double2(D[m], 0.0);
        return;
    }
    const double rx = sx * h, ry = sy * h;
    const double r = sqrt(rx * rx + ry * ry);
    const double k = h * h * exp(-mu * r) / (2.0 * M_PI * r);
    // e^{-i theta} = (rx - i ry)/r, raised to the m-th power by recurrence
    const double ex = rx / r, ey = -ry / r;
    double cr = 1.0, ci = 0.0;
    for (int m = 0; m <= mmax; ++m) {
        G[m * P + idx] = make_double2(k * cr, k * ci);
        const double nr = cr * ex - ci * ey;
        ci = cr * ey + ci * ex;
        cr = nr;
    }
}

// 3D: real g on the Q^3 grid stored as complex G[oz][oy][ox]
__global__ void k_sample_3d(double2* G, int n, int Q, double h, double mu, const double* D) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long P = (long)Q * Q * Q;
    if (idx >= P) return;
    const int ox = (int)(idx % Q), oy = (int)((idx / Q) % Q), oz = (int)(idx / ((long)Q * Q));
    const int sx = ox < Q / 2 ? ox : ox - Q;
    const int sy = oy < Q / 2 ? oy : oy - Q;
    const int sz = oz < Q / 2 ? oz : oz - Q;
    double v = 0.0;
    if (abs(sx) < n && abs(sy) < n && abs(sz) < n) {
        if (sx == 0 && sy == 0 && sz == 0) {
            v = D[0];
        } else {
            const double r = h * sqrt((double)sx * sx + (double)sy * sy + (double)sz * sz);
            v = h * h * h * exp(-mu * r) / (4.0 * M_PI * r * r);
        }
    }
    G[idx] = make_double2(v, 0.0);
}

// ---------------------------------------------------------------------------
// generic batched line FFT (plan time, FP64, forward): line l -> base offset
// (l % nA) * sA + (l / nA) * sB, element stride sE.  LPB lines per block.
// ---------------------------------------------------------------------------
__global__ void k_fft_lines64(double2* data, FftSched sc, const double2* tw, long nlines, long nA,
                              long sA, long sB, long sE, int LPB) {
    extern __shared__ double2 sm[];
    const int Q = sc.Q;
    double2* twl = sm;
    double2* buf = sm + Q;
    double2* tmp = buf + (long)LPB * Q;
    load_twiddles(twl, tw, Q);
    const long l0 = (long)blockIdx.x * LPB;
    const int nl = (int)min((long)LPB, nlines - l0);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        int li, e;
        if (sE == 1) { li = idx / Q; e = idx % Q; }
        else { li = idx % nl; e = idx / nl; }
        const long l = l0 + li;
        const long off = (l % nA) * sA + (l / nA) * sB + e * sE;
        buf[li * Q + e] = data[off];
    }
    __syncthreads();
    double2* res = fft_lines<-1>(buf, tmp, nl, Q, sc, twl);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        int li, e;
        if (sE == 1) { li = idx / Q; e = idx % Q; }
        else { li = idx % nl; e = idx / nl; }
        const long l = l0 + li;
        const long off = (l % nA) * sA + (l / nA) * sB + e * sE;
        data[off] = res[li * Q + e];
    }
}

rte_status fft_lines_host(double2* data, const FftSched& sc, const double2* tw, long nlines,
                                 long nA, long sA, long sB, long sE, cudaStream_t s) {
    const int Q = sc.Q;
    int LPB = 4096 / Q;
    if (LPB < 1) LPB = 1;
    if (LPB > 16) LPB = 16;
    const size_t smem = (size_t)(2 * LPB + 1) * Q * sizeof(double2);
    RTE_CUDA_TRY(cudaFuncSetAttribute(k_fft_lines64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long nblk = (nlines + LPB - 1) / LPB;
    k_fft_lines64<<<(unsigned)nblk, 256, smem, s>>>(data, sc, tw, nlines, nA, sA, sB, sE, LPB);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// S[xi_x][m][xi_y] = G[m][xi_y][xi_x] / Q^2 for xi_x < H, with FP32 and BF16 copies
__global__ void k_extract_2d(const double2* G, int Q, int H, int nm, double2* S64, float2* S32,
                             __nv_bfloat162* S16) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long tot = (long)H * nm * Q;
    if (idx >= tot) return;
    const int ky = (int)(idx % Q);
    const int m = (int)((idx / Q) % nm);
    const int kx = (int)(idx / ((long)Q * nm));
    const double sc = 1.0 / ((double)Q * (double)Q);
    double2 v = G[((long)m * Q + ky) * Q + kx];
    v.x *= sc;
    v.y *= sc;
    S64[idx] = v;
    S32[idx] = make_float2((float)v.x, (float)v.y);
    if (S16) S16[idx] = __floats2bfloat162_rn((float)v.x, (float)v.y);  // no BF16 copy for mode-FFT plans
}

// octant of the real even 3D spectrum: S3[kx][ky][kz] = Re G[kz][ky][kx] / Q^3
__global__ void k_extract_3d(const double2* G, int Q, int H, double* S64, float* S32) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long tot = (long)H * H * H;
    if (idx >= tot) return;
    const int kz = (int)(idx % H), ky = (int)((idx / H) % H), kx = (int)(idx / ((long)H * H));
    const double sc = 1.0 / ((double)Q * Q * Q);
    const double v = G[((long)kz * Q + ky) * Q + kx].x * sc;
    S64[idx] = v;
    S32[idx] = (float)v;
}

rte_status plan_build_spectra(rte_plan p, cudaStream_t s) {
    const int Q = p->Q, H = p->H;
    k_twiddles<<<(Q + 255) / 256, 256, 0, s>>>(p->tw64, p->tw32, Q);
    RTE_CUDA_TRY(cudaGetLastError());
    if (p->dim == 2) {
        const int nm = 2 * p->L + 1;
        k_cell_weights_2d<<<1, 64, 0, s>>>(p->mu_t, p->h, 2 * p->L, p->Dm);
        RTE_CUDA_TRY(cudaGetLastError());
        const long P = (long)Q * Q;
        double2* G = nullptr;
        RTE_CUDA_TRY(rte_dev_malloc_async((void**)&G, (size_t)nm * P * sizeof(double2), s));
        k_sample_2d<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(G, p->n, Q, 2 * p->L, p->h, p->mu_t, p->Dm);
        RTE_CUDA_TRY(cudaGetLastError());
        // rows (x direction): lines = (m, oy), contiguous
        rte_status st = fft_lines_host(G, p->sched, p->tw64, (long)nm * Q, (long)nm * Q, Q, 0, 1, s);
        if (st != RTE_OK) return st;
        // columns (y direction): line = (ox, m): offset ox + m*P, stride Q
        st = fft_lines_host(G, p->sched, p->tw64, (long)nm * Q, Q, 1, P, Q, s);
        if (st != RTE_OK) return st;
        const long tot = (long)H * nm * Q;
        k_extract_2d<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, Q, H, nm, p->S64, p->S32, p->S16);
        RTE_CUDA_TRY(cudaGetLastError());
        RTE_CUDA_TRY(rte_dev_free_async(G, s));
    } else {
        k_cell_weight_3d<<<1, 64, 0, s>>>(p->mu_t, p->h, p->Dm);
        RTE_CUDA_TRY(cudaGetLastError());
        const long P = (long)Q * Q * Q;
        double2* G = nullptr;
        RTE_CUDA_TRY(rte_dev_malloc_async((void**)&G, (size_t)P * sizeof(double2), s));
        k_sample_3d<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(G, p->n, Q, p->h, p->mu_t, p->Dm);
        RTE_CUDA_TRY(cudaGetLastError());
        const long Q2 = (long)Q * Q;
        // x lines: (oy, oz) -> offset line*Q
        rte_status st = fft_lines_host(G, p->sched, p->tw64, Q2, Q2, Q, 0, 1, s);
        if (st != RTE_OK) return st;
        // y lines: (ox, oz) -> ox + oz*Q^2, stride Q
        st = fft_lines_host(G, p->sched, p->tw64, Q2, Q, 1, Q2, Q, s);
        if (st != RTE_OK) return st;
        // z lines: (ox, oy) -> ox + oy*Q, stride Q^2
        st = fft_lines_host(G, p->sched, p->tw64, Q2, Q2, 1, 0, Q2, s);
        if (st != RTE_OK) return st;
        const long tot = (long)H * H * H;
        k_extract_3d<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, Q, H, p->S3_64, p->S3_32);
        RTE_CUDA_TRY(cudaGetLastError());
        RTE_CUDA_TRY(rte_dev_free_async(G, s));
    }
    return RTE_OK;
}

// ---------------------------------------------------------------------------
// Mode-axis DFTs of the spectra (plans that couple the modes by FFTs along the
// mode axis): per frequency id = xi_x Q + xi_y the line s[m mod P] = S_m(xi),
// m = -2L..2L, with S_{-m} = (-1)^m conj(S_m) (the kernel is real and even),
// forward DFT of length P, scaled by 1/P; FP64 into Sm64, rounded copies in
// Sm32 and float-float in Smff.  16 frequencies per block.
// ---------------------------------------------------------------------------
#define MFS_LINES 16
__global__ void __launch_bounds__(256) k_modefft_spectra(const double2* __restrict__ S64, int H, int Q, int L, int P,
                                                         FftSched sc, const double2* __restrict__ twm,
                                                         double2* __restrict__ Sm64, float2* __restrict__ Sm32,
                                                         ffc* __restrict__ Smff) {
    extern __shared__ unsigned char smraw[];
    double2* sm = reinterpret_cast<double2*>(smraw);
    double2* twl = sm;
    double2* buf = sm + P;
    double2* tmp = buf + MFS_LINES * P;
    load_twiddles(twl, twm, P);
    const long nfreq = (long)H * Q;
    const long f0 = (long)blockIdx.x * MFS_LINES;
    const long rem = nfreq - f0;
    const int nf = rem < MFS_LINES ? (int)rem : MFS_LINES;
    const int nm = 2 * L + 1;
    for (int i = threadIdx.x; i < MFS_LINES * P; i += blockDim.x) buf[i] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int i = threadIdx.x; i < nm * MFS_LINES; i += blockDim.x) {
        const int m = i / MFS_LINES, f = i - m * MFS_LINES;
        if (f >= nf) continue;
        const long id = f0 + f;
        const long kx = id / Q, ky = id - kx * Q;
        const double2 v = S64[(kx * nm + m) * Q + ky];
        double2* line = buf + f * P;
        line[m] = v;
        if (m > 0) line[P - m] = (m & 1) ? make_double2(-v.x, v.y) : make_double2(v.x, -v.y);
    }
    __syncthreads();
    double2* r = fft_lines<-1>(buf, tmp, MFS_LINES, P, sc, twl);
    const double inv = 1.0 / P;
    for (int i = threadIdx.x; i < nf * P; i += blockDim.x) {
        const double2 v = make_double2(r[i].x * inv, r[i].y * inv);
        Sm64[f0 * P + i] = v;
        Sm32[f0 * P + i] = make_float2((float)v.x, (float)v.y);
        Smff[f0 * P + i] = to_ffc(v);
    }
}

__global__ void k_twiddles_ff(const double2* __restrict__ tw64, ffc* __restrict__ twff, int P) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < P) twff[t] = to_ffc(tw64[t]);
}

rte_status plan_build_modefft(rte_plan p, cudaStream_t s) {
    if (!p->mix_fft) return RTE_OK;
    const int P = p->Pm;
    k_twiddles<<<(P + 255) / 256, 256, 0, s>>>(p->twm64, p->twm32, P);
    k_twiddles_ff<<<(P + 255) / 256, 256, 0, s>>>(p->twm64, p->twmff, P);
    RTE_CUDA_TRY(cudaGetLastError());
    const size_t smem = (size_t)(P + 2 * MFS_LINES * P) * sizeof(double2);
    static bool once = false;
    if (!once) {
        RTE_CUDA_TRY(cudaFuncSetAttribute(k_modefft_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448));
        once = true;
    }
    const long nfreq = (long)p->H * p->Q;
    k_modefft_spectra<<<(unsigned)((nfreq + MFS_LINES - 1) / MFS_LINES), 256, smem, s>>>(
        p->S64, p->H, p->Q, p->L, P, p->sched_m, p->twm64, p->Sm64, p->Sm32, p->Smff);
    rte_count_launches(3);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}
