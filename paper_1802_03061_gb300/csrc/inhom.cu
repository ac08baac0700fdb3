// Inhomogeneous medium, isotropic scattering, 2D: the Nystrom matrix of
// Sec. 2.3 (Eq. iso_discretization) applied directly, O(N^2), on the GPU.
//
//   K~_ij = h^2 E(x_i, x_j) / (2 pi |x_i - x_j|)          (i != j)
//   E(x, y) = exp(-|x - y| int_0^1 mu_t(x - s (x - y)) ds)  (5-point Gauss-Legendre)
//   K~_ii = (2h/pi) ln(1 + sqrt 2) + int_cell (E(x_i, y) - 1)/(2 pi |x_i - y|) dy
//           (the smooth part by the 15 x 15 tensor Gauss-Legendre rule)
//
// mu_t between samples: bilinear interpolation of the cell-centred values,
// the sample index clamped to the grid.  Points are handled in index units:
// cell (i1, i2) has its centre at ((i1 + 1/2) h, (i2 + 1/2) h), so a point
// c_i + s (c_j - c_i) sits at continuous sample index (i1 + s (j1 - i1),
// i2 + s (j2 - i2)).  The homogeneous FFT method does not apply here (the
// kernel is not translation invariant).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "internal.h"

static constexpr double kPi = 3.14159265358979323846;

struct rte_inhom_s {
    int n = 0;
    double h = 0.0;
    double* mu64 = nullptr;   // [n][n] mu_t samples
    float* mu32 = nullptr;
    double* diag64 = nullptr;  // K~_ii
    float* diag32 = nullptr;
    double s5[5], w5[5];       // 5-point Gauss-Legendre on [0, 1]
};

// q-point Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on the
// Legendre polynomial P_q (three-term recurrence; P_q' from
// (x^2 - 1) P_q' = q (x P_q - P_{q-1})), started at the Chebyshev-like guess
// cos(pi (k - 1/4) / (q + 1/2)).
static void gauss_legendre(int q, double* x, double* w) {
    for (int k = 0; k < q; ++k) {
        double z = cos(kPi * (k + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= q; ++j) {
                const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= q; ++j) {
            const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1.0);
        x[k] = z;
        w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct Gl5 {
    double s[5], w[5];
};

// mu_t at continuous sample index (u, v) (u along x): bilinear, clamped
template <typename T>
__device__ __forceinline__ T mu_bilinear(const T* __restrict__ mu, int n, T u, T v) {
    if (n == 1) return mu[0];
    int i0 = (int)floor(u), j0 = (int)floor(v);
    i0 = i0 < 0 ? 0 : (i0 > n - 2 ? n - 2 : i0);
    j0 = j0 < 0 ? 0 : (j0 > n - 2 ? n - 2 : j0);
    T t = u - (T)i0, s = v - (T)j0;
    t = t < (T)0 ? (T)0 : (t > (T)1 ? (T)1 : t);
    s = s < (T)0 ? (T)0 : (s > (T)1 ? (T)1 : s);
    const T* m = mu + (long)j0 * n + i0;
    return ((T)1 - s) * (((T)1 - t) * m[0] + t * m[1]) + s * (((T)1 - t) * m[n] + t * m[n + 1]);
}

// the integral of mu_t along the unit-parameter segment from (u0, v0) to
// (u0 + du, v0 + dv), in sample-index units, by 5-point Gauss-Legendre
template <typename T>
__device__ __forceinline__ T line_mean(const T* __restrict__ mu, int n, T u0, T v0, T du, T dv, const Gl5& g) {
    T acc = (T)0;
#pragma unroll
    for (int q = 0; q < 5; ++q) acc += (T)g.w[q] * mu_bilinear(mu, n, u0 + (T)g.s[q] * du, v0 + (T)g.s[q] * dv);
    return acc;
}

// K~_ii, one thread per cell, FP64: closed-form mean of 1/(2 pi r) + the
// 15 x 15 tensor rule on the smooth part (limit -mu_t(x_i)/(2 pi) at r = 0)
struct Gl15 {
    double x[15], w[15];
};
__global__ void k_inhom_diag(const double* __restrict__ mu, double* __restrict__ d64, float* __restrict__ d32, int n,
                             double h, Gl5 g5, Gl15 g15) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * n) return;
    const double u0 = (double)(i % n), v0 = (double)(i / n);
    const double mu0 = mu_bilinear(mu, n, u0, v0);
    double total = 0.0;
    for (int a = 0; a < 15; ++a)
        for (int b = 0; b < 15; ++b) {
            const double du = 0.5 * g15.x[a], dv = 0.5 * g15.x[b];  // half a cell in index units
            const double r = h * sqrt(du * du + dv * dv);
            double gv;
            if (r == 0.0) {
                gv = -mu0 / (2.0 * kPi);
            } else {
                const double tau = r * line_mean(mu, n, u0, v0, du, dv, g5);
                gv = expm1(-tau) / (2.0 * kPi * r);
            }
            total += g15.w[a] * g15.w[b] * gv;
        }
    const double v = (2.0 * h / kPi) * log1p(sqrt(2.0)) + 0.25 * h * h * total;
    d64[i] = v;
    d32[i] = (float)v;
}

// mu_t at a point of a segment between two cell centres: its sample index
// (u, v) lies in [0, n-1]^2, so only the upper cell needs a clamp (n >= 2)
template <typename T>
__device__ __forceinline__ T mu_seg(const T* __restrict__ mu, int n, T u, T v) {
    const int i0 = min((int)u, n - 2), j0 = min((int)v, n - 2);
    const T t = u - (T)i0, s = v - (T)j0;
    const T* m = mu + (long)j0 * n + i0;
    return ((T)1 - s) * (((T)1 - t) * m[0] + t * m[1]) + s * (((T)1 - t) * m[n] + t * m[n + 1]);
}

// y_i = sum_{j != i} h^2 E_ij / (2 pi r_ij) x_j + K~_ii x_i.  A block owns 32
// consecutive outputs (the lanes) and splits the sources over its 8 warps;
// each warp sums its slice with compensated (Kahan) accumulation, the 8
// partial sums per output meet in shared memory.  mu_t staged in shared
// memory when small (<= 48 KB), else read through L1.
template <typename T>
__global__ void __launch_bounds__(256) k_inhom_apply(const T* __restrict__ mu_g, const T* __restrict__ diag,
                                                     const T* __restrict__ x, T* __restrict__ y, int n, T h,
                                                     int mu_smem, Gl5 g5) {
    extern __shared__ unsigned char smraw[];
    __shared__ T part[8][32], pcomp[8][32];
    const int N = n * n;
    const T* mu = mu_g;
    if (mu_smem) {
        T* ms = reinterpret_cast<T*>(smraw);
        for (int k = threadIdx.x; k < N; k += blockDim.x) ms[k] = mu_g[k];
        __syncthreads();
        mu = ms;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const bool live = i < N;
    const int ii = live ? i : 0;
    const int i1 = ii % n, i2 = ii / n;
    const int per = (N + 7) / 8, j0 = warp * per, j1 = min(N, j0 + per);
    T acc = (T)0, comp = (T)0;
    if (n > 1) {
        int c1 = j0 % n, c2 = j0 / n;  // the source cell of j, stepped along with j
        for (int j = j0; j < j1; ++j, ++c1) {
            if (c1 == n) {
                c1 = 0;
                ++c2;
            }
            if (j == ii) continue;
            const T du = (T)(c1 - i1), dv = (T)(c2 - i2);
            const T r = h * sqrt(du * du + dv * dv);
            T mean = (T)0;
#pragma unroll
            for (int q = 0; q < 5; ++q)
                mean += (T)g5.w[q] * mu_seg(mu, n, (T)i1 + (T)g5.s[q] * du, (T)i2 + (T)g5.s[q] * dv);
            const T term = exp(-r * mean) / r * x[j];
            const T yk = term - comp;
            const T t2 = acc + yk;
            comp = (t2 - acc) - yk;
            acc = t2;
        }
    }
    part[warp][lane] = acc;
    pcomp[warp][lane] = comp;
    __syncthreads();
    if (warp == 0 && live) {
        T sum = (T)0, c = (T)0;
        for (int w = 0; w < 8; ++w) {
            const T yk = (part[w][lane] - pcomp[w][lane]) - c;
            const T t2 = sum + yk;
            c = (t2 - sum) - yk;
            sum = t2;
        }
        y[i] = h * h / (T)(2.0 * kPi) * sum + diag[i] * x[i];
    }
}

// FP32, using the symmetry K~_ij = K~_ji (E(x, y) = E(y, x)): each unordered
// pair's optical depth is computed once.  y starts as diag(K~) x (k_inhom_diag_x);
// a block owns the 32 rows i0..i0+31 (its lanes) and the 256 columns
// j0..j0+255 (32 per warp) and takes the pairs with j > i: row i gains
// K~_ij x_j, column j gains K~_ij x_i.  Row sums meet over the warps in shared
// memory, column sums over the lanes by shuffles; both reach y by one atomic
// add per block and row or per warp and column (the summation order is not
// fixed, unlike k_inhom_apply).  Blocks wholly below the diagonal return.
__global__ void k_inhom_diag_x(const float* __restrict__ diag, const float* __restrict__ x, float* __restrict__ y,
                               int N) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) y[i] = diag[i] * x[i];
}

__global__ void __launch_bounds__(256) k_inhom_apply_sym(const float* __restrict__ mu_g, const float* __restrict__ x,
                                                         float* __restrict__ y, int n, float h, int mu_smem, Gl5 g5) {
    extern __shared__ unsigned char smraw[];
    __shared__ float part[8][32];
    const int N = n * n;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 256;
    if (j0 + 255 <= i0) return;  // no pair j > i in this block (uniform)
    const float* mu = mu_g;
    if (mu_smem) {
        float* ms = reinterpret_cast<float*>(smraw);
        for (int k = threadIdx.x; k < N; k += blockDim.x) ms[k] = mu_g[k];
        __syncthreads();
        mu = ms;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = i0 + lane;
    const bool live = i < N;
    const int ii = live ? i : 0;
    const int i1 = ii % n, i2 = ii / n;
    const float xi = live ? x[ii] : 0.f;
    const float scale = h * h / (float)(2.0 * kPi);
    float acc = 0.f, comp = 0.f;
    const int jb = j0 + warp * 32;
    // the source cell (j1, j2) of j, stepped along with j (no division per pair)
    int j1 = jb % n, j2 = jb / n;
    for (int jj = 0; jj < 32; ++jj, ++j1) {
        const int j = jb + jj;
        if (j >= N) break;  // uniform over the warp
        if (j1 == n) {
            j1 = 0;
            ++j2;
        }
        float e = 0.f;
        if (live && j > i) {
            const float du = (float)(j1 - i1), dv = (float)(j2 - i2);
            const float r = h * sqrtf(du * du + dv * dv);
            float mean = 0.f;
#pragma unroll
            for (int q = 0; q < 5; ++q)
                mean += (float)g5.w[q] * mu_seg(mu, n, (float)i1 + (float)g5.s[q] * du, (float)i2 + (float)g5.s[q] * dv);
            e = expf(-r * mean) / r;
        }
        // row i: + e x_j (compensated); column j: + sum over the lanes of e x_i
        const float term = e * x[j];
        const float yk = term - comp;
        const float t2 = acc + yk;
        comp = (t2 - acc) - yk;
        acc = t2;
        float cs = e * xi;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
        if (lane == 0 && cs != 0.f) atomicAdd(&y[j], scale * cs);
    }
    part[warp][lane] = acc - comp;
    __syncthreads();
    if (warp == 0 && live) {
        float sum = 0.f;
        for (int w = 0; w < 8; ++w) sum += part[w][lane];
        if (sum != 0.f) atomicAdd(&y[i], scale * sum);
    }
}

static size_t inhom_smem(int n, size_t el) {
    const size_t b = (size_t)n * n * el;
    return b <= 48 * 1024 ? b : 0;
}

extern "C" rte_status rte_inhom_destroy(rte_inhom op) {
    if (!op) return RTE_OK;
    if (op->mu64) rte_dev_free(op->mu64);
    if (op->mu32) rte_dev_free(op->mu32);
    if (op->diag64) rte_dev_free(op->diag64);
    if (op->diag32) rte_dev_free(op->diag32);
    delete op;
    return RTE_OK;
}

extern "C" rte_status rte_inhom_create(rte_inhom* out, int n, double h, const double* mu_t_host, void* stream) {
    if (!out) return RTE_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 4096 || !(h > 0.0) || !mu_t_host) return RTE_EINVAL;
    const long N = (long)n * n;
    for (long k = 0; k < N; ++k)
        if (!(mu_t_host[k] >= 0.0) || !isfinite(mu_t_host[k])) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_inhom op = new rte_inhom_s();
    op->n = n;
    op->h = h;
    double x5[5], w5[5];
    gauss_legendre(5, x5, w5);
    Gl5 g5;
    for (int q = 0; q < 5; ++q) {
        g5.s[q] = op->s5[q] = 0.5 * (x5[q] + 1.0);
        g5.w[q] = op->w5[q] = 0.5 * w5[q];
    }
    Gl15 g15;
    gauss_legendre(15, g15.x, g15.w);
    std::vector<float> m32(N);
    for (long k = 0; k < N; ++k) m32[k] = (float)mu_t_host[k];
    if (rte_dev_malloc((void**)&op->mu64, N * sizeof(double)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->mu32, N * sizeof(float)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->diag64, N * sizeof(double)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->diag32, N * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        rte_inhom_destroy(op);
        return rte_fail(RTE_ENOMEM, "rte_inhom_create");
    }
    cudaError_t e = cudaMemcpyAsync(op->mu64, mu_t_host, N * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(op->mu32, m32.data(), N * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_inhom_diag<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(op->mu64, op->diag64, op->diag32, n, h, g5, g15);
        rte_count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // m32 is a host temporary
    if (e != cudaSuccess) {
        rte_inhom_destroy(op);
        return rte_cuda_fail(e, "rte_inhom_create");
    }
    *out = op;
    return RTE_OK;
}

template <typename T>
static rte_status inhom_apply(rte_inhom op, const T* mu, const T* diag, const T* x, T* y, cudaStream_t s) {
    const int N = op->n * op->n;
    Gl5 g5;
    for (int q = 0; q < 5; ++q) {
        g5.s[q] = op->s5[q];
        g5.w[q] = op->w5[q];
    }
    const size_t sm = inhom_smem(op->n, sizeof(T));
    static bool once = false;
    if (!once) {
        cudaError_t e = cudaFuncSetAttribute(k_inhom_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
        if (e != cudaSuccess) return rte_cuda_fail(e, "rte_inhom_apply");
        once = true;
    }
    k_inhom_apply<T><<<(unsigned)((N + 31) / 32), 256, sm, s>>>(mu, diag, x, y, op->n, (T)op->h, sm ? 1 : 0, g5);
    rte_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_inhom_apply");
    return RTE_OK;
}

extern "C" rte_status rte_inhom_apply32(rte_inhom op, const float* x_dev, float* y_dev, void* stream) {
    if (!op || !x_dev || !y_dev || x_dev == y_dev) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = op->n, N = n * n;
    Gl5 g5;
    for (int q = 0; q < 5; ++q) {
        g5.s[q] = op->s5[q];
        g5.w[q] = op->w5[q];
    }
    const size_t sm = inhom_smem(n, sizeof(float));
    static bool once = false;
    if (!once) {
        cudaError_t e = cudaFuncSetAttribute(k_inhom_apply_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
        if (e != cudaSuccess) return rte_cuda_fail(e, "rte_inhom_apply32");
        once = true;
    }
    k_inhom_diag_x<<<(unsigned)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096), 256, 0, s>>>(op->diag32, x_dev, y_dev, N);
    const dim3 grid((unsigned)((N + 255) / 256), (unsigned)((N + 31) / 32));
    k_inhom_apply_sym<<<grid, 256, sm, s>>>(op->mu32, x_dev, y_dev, n, (float)op->h, sm ? 1 : 0, g5);
    rte_count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_inhom_apply32");
    return RTE_OK;
}

extern "C" rte_status rte_inhom_apply64(rte_inhom op, const double* x_dev, double* y_dev, void* stream) {
    if (!op || !x_dev || !y_dev || x_dev == y_dev) return RTE_EINVAL;
    return inhom_apply<double>(op, op->mu64, op->diag64, x_dev, y_dev, (cudaStream_t)stream);
}

extern "C" rte_status rte_inhom_diag(rte_inhom op, double* diag_host) {
    if (!op || !diag_host) return RTE_EINVAL;
    const long N = (long)op->n * op->n;
    RTE_CUDA_TRY(cudaMemcpy(diag_host, op->diag64, N * sizeof(double), cudaMemcpyDeviceToHost));
    return RTE_OK;
}
