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
    __shared__ double acc[64][RTE_MAX_CH * 2 + 1];
    const int i = threadIdx.x;
    double x, w;
    gl_node(64, i, &x, &w);
    double part[2 * RTE_MAX_CH + 1];
    for (int m = 0; m <= mmax; ++m) part[m] = 0.0;
    const double a = 0.5 * h;
    for (int q = 0; q < 8; ++q) {
        const double phi = q * (M_PI / 4) + (x + 1.0) * (M_PI / 8);
        double s, c;
        sincos(phi, &s, &c);
        const double R = a / fmax(fabs(c), fabs(s));
        const double rad = radial_factor(mu, R) * w * (M_PI / 8);
        // cos(m phi) by the Chebyshev recurrence c_m = 2 cos(phi) c_{m-1} - c_{m-2}
        double cm2 = 1.0, cm1 = c;
        part[0] += rad;
        if (mmax >= 1) part[1] += c * rad;
        for (int m = 2; m <= mmax; ++m) {
            const double cm = 2.0 * c * cm1 - cm2;
            part[m] += cm * rad;
            cm2 = cm1;
            cm1 = cm;
        }
    }
    for (int m = 0; m <= mmax; ++m) acc[i][m] = part[m];
    __syncthreads();
    if (i <= mmax) {
        double t = 0.0;
        for (int j = 0; j < 64; ++j) t += acc[j][i];
        D[i] = t / (2.0 * M_PI);
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
    S16[idx] = __floats2bfloat162_rn((float)v.x, (float)v.y);
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
