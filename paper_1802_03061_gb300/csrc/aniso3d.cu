// 3D anisotropic scattering in real spherical harmonics (Sec. 3.1.2).
//
// With a real orthonormal basis Y_a, a = l^2 + l + m (|m| <= l <= L), the
// angular moments u_a = (4 pi)^{-1/2} int Phi Y_a dv solve M = (L+1)^2
// coupled Fredholm equations of the second kind,
//   u_a = sum_b K~^{ab} (mu_s sigma_hat_{l_b} u_b) + K~^{a0} f,
//   K~^{ab}_{ij} = h^3 exp(-mu_t r)/(4 pi r^2) W_ab(v_ij)   (i != j),
//   K~^{ab}_{ii} = D_ab = int_cell exp(-mu_t r)/(4 pi r^2) W_ab(y/r) dy,
//   W_ab(v) = 4 pi Y_a(v) Y_b(v),   v_ij = (x_i - x_j)/|x_i - x_j|,
// sigma_hat_l the Legendre moments of the phase function (sigma_hat_0 = 1).
// L = 0 is the isotropic equation.  Every K~^{ab} is a convolution, applied
// with FFTs on the zero-padded Q^3 grid (Sec. 2.3.1): the input channels
// take the X and Y passes, one Z pass transforms all M channels of a
// (xi_x, xi_y) line, mixes them with the M x M spectra at each xi_z and
// transforms back, and the output channels take the Y' and X' passes.  For
// Q = 64, 128, 256 the warp-register passes of aniso3d_warp.cu run each pass
// over all channels in one launch; otherwise the general-Q Stockham passes
// below run channel by channel.  The solve (T.1, T.2) is the plan's device
// solve graph (krylov.cu) built on this operator.
//
// Each W_ab has a definite parity in x, y and z (Y_a does), so its spectrum
// is real (even total parity) or imaginary (odd) with the same parities; it is
// stored as the octant xi in [0, Q/2]^3 of its real or imaginary part, and
// W_ab = W_ba gives (L+1)^2 ((L+1)^2 + 1)/2 distinct spectra.
#include <math.h>
#include <string.h>

#include <vector>

#include "aniso3d.cuh"
#include "op3d_passes.cuh"

// Real orthonormal spherical harmonics of degree <= L at the unit vector
// (x, y, z), no Condon-Shortley phase:
//   Y_{l,0} = N_l0 P_l(z),  Y_{l,+-m} = sqrt2 N_lm Q_l^m(z) {Re, Im}(x + i y)^m,
// N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), Q_l^m = P_l^m / (1-z^2)^{m/2}
// (a polynomial) by the three-term recurrence in l from Q_m^m = (2m-1)!!.
__device__ void sh_real(int L, double x, double y, double z, double* Y) {
    double cr = 1.0, ci = 0.0;  // (x + i y)^m
    double qmm = 1.0;           // (2m - 1)!!
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            qmm *= (double)(2 * m - 1);
            const double nr = cr * x - ci * y;
            ci = cr * y + ci * x;
            cr = nr;
        }
        double q1 = 0.0, q2 = 0.0;
        for (int l = m; l <= L; ++l) {
            double q;
            if (l == m) q = qmm;
            else if (l == m + 1) q = z * (double)(2 * m + 1) * qmm;
            else q = ((double)(2 * l - 1) * z * q1 - (double)(l + m - 1) * q2) / (double)(l - m);
            q2 = q1;
            q1 = q;
            double ratio = 1.0;  // (l - m)! / (l + m)!
            for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
            const double N = sqrt((double)(2 * l + 1) / (4.0 * M_PI) * ratio);
            if (m == 0) {
                Y[l * l + l] = N * q;
            } else {
                Y[l * l + l + m] = M_SQRT2 * N * q * cr;
                Y[l * l + l - m] = M_SQRT2 * N * q * ci;
            }
        }
    }
}

// The channel-pair table (pair_info for every ordered pair, row-major);
// pimag[pair] = the imaginary flag.
static void aniso_pair_table(int M, int* pinfo, int* pimag) {
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
            const int info = pair_info(a, b, M);
            pinfo[a * M + b] = info;
            pimag[info & 0xffff] = (info >> 16) & 1;
        }
}

// D_ab over the six faces of the cell: on the face of the point p = (.., +-a, ..)
// the solid-angle element is a dx dy / |p|^3 and the ray reaches |p|, so
// D_ab = sum_faces int Y_a(p/|p|) Y_b(p/|p|) (1 - e^{-mu |p|})/mu a/|p|^3 dx dy
// (W_ab/(4 pi) = Y_a Y_b); each face as four quadrants of 64^2 Gauss-Legendre
// points.  Block (a, b) with a <= b; 256 threads.
__global__ void __launch_bounds__(256) k_aniso_cell_weights(int L, int M, double mu, double h, double* D) {
    __shared__ double xs[64], ws[64], red[256];
    const double ha = 0.5 * h;
    if (threadIdx.x < 64) {
        double x, w;
        gl_node(64, threadIdx.x, &x, &w);
        xs[threadIdx.x] = 0.5 * ha * (x + 1.0);
        ws[threadIdx.x] = 0.5 * ha * w;
    }
    __syncthreads();
    const int a = blockIdx.x / M, b = blockIdx.x % M;
    if (b < a) return;  // uniform over the block
    const int la = chan_l(a), lb = chan_l(b);
    const int Lq = la > lb ? la : lb;
    double Y[RTE_ANISO_MAX_M];
    double acc = 0.0;
    for (int k = threadIdx.x; k < 6 * 4 * 64 * 64; k += blockDim.x) {
        const int j = k & 63, i = (k >> 6) & 63, quad = (k >> 12) & 3, face = k >> 14;
        const int axis = face >> 1;
        const double sgn = (face & 1) ? -1.0 : 1.0;
        const double u = ((quad & 1) ? -1.0 : 1.0) * xs[i];
        const double v = ((quad & 2) ? -1.0 : 1.0) * xs[j];
        double p[3];
        p[axis] = sgn * ha;
        p[(axis + 1) % 3] = u;
        p[(axis + 2) % 3] = v;
        const double rho = sqrt(u * u + v * v + ha * ha);
        const double wgt = ws[i] * ws[j] * radial_factor(mu, rho) * ha / (rho * rho * rho);
        sh_real(Lq, p[0] / rho, p[1] / rho, p[2] / rho, Y);
        acc += wgt * Y[a] * Y[b];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        D[a * M + b] = red[0];
        D[b * M + a] = red[0];
    }
}

// g_ab on the periodic Q^3 grid, stored complex G[oz][oy][ox]:
// h^3 exp(-mu r)/(4 pi r^2) W_ab(o/|o|) for 0 < |o_k| <= n-1, D_ab at o = 0
__global__ void k_aniso_sample(double2* G, int n, int Q, double h, double mu, int Lq, int a, int b, double Dab) {
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
            v = Dab;
        } else {
            const double d = sqrt((double)sx * sx + (double)sy * sy + (double)sz * sz);
            const double r = h * d;
            double Y[RTE_ANISO_MAX_M];
            sh_real(Lq, sx / d, sy / d, sz / d, Y);
            v = h * h * h * exp(-mu * r) / (r * r) * Y[a] * Y[b];  // (1/4pi) * 4 pi Y_a Y_b
        }
    }
    G[idx] = make_double2(v, 0.0);
}

// octant of the real (or imaginary) part: S[kx][ky][kz] = {Re, Im} G[kz][ky][kx] / Q^3
__global__ void k_aniso_extract(const double2* G, int Q, int H, int imag, double* S64, float* S32) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long tot = (long)H * H * H;
    if (idx >= tot) return;
    const int kz = (int)(idx % H), ky = (int)((idx / H) % H), kx = (int)(idx / ((long)H * H));
    const double2 g = G[((long)kz * Q + ky) * Q + kx];
    const double v = (imag ? g.y : g.x) / ((double)Q * Q * Q);
    S64[idx] = v;
    S32[idx] = (float)v;
}

// Z pass over all channels of B (xi_x, xi_y) lines: FFT along z of the Min
// input channels, out_a = sum_b S_ab in_b at every xi_z, inverse FFT of the
// Mout output channels, keep z < n.  T2 holds channel c at c * chs
// (layout [xi_x][xi_y][z] per channel); grid ceil(H*Q/B).
template <typename T, typename TS>
__global__ void __launch_bounds__(256) k3a_z_mix(T* __restrict__ T2, long chs, int Min, int Mout,
                                                 const TS* __restrict__ S, long H3, const int* __restrict__ pinfo,
                                                 int M, const T* __restrict__ tw, P3 p) {
    extern __shared__ unsigned char smraw[];
    __shared__ int pis[RTE_ANISO_MAX_M * RTE_ANISO_MAX_M];
    T* sm = reinterpret_cast<T*>(smraw);
    using RR = typename real_of<T>::R;
    const int n = p.n, Q = p.Q, H = p.H, B = p.B;
    const long l0 = (long)blockIdx.x * B;
    const long nlines = (long)H * Q;
    const int nb = (int)min((long)B, nlines - l0);
    const int Mx = Min > Mout ? Min : Mout;
    T* twl = sm;
    T* buf = sm + Q;
    T* tmp = buf + (long)Mx * B * Q;
    load_twiddles(twl, tw, Q);
    for (int i = threadIdx.x; i < M * M; i += blockDim.x) pis[i] = pinfo[i];
    for (int idx = threadIdx.x; idx < Min * nb * Q; idx += blockDim.x) {
        const int row = idx / Q, e = idx - row * Q;
        const int c = row / nb, lb = row - c * nb;
        buf[idx] = e < n ? T2[c * chs + (l0 + lb) * n + e] : mk<T>(0, 0);
    }
    __syncthreads();
    T* res = fft_lines<-1>(buf, tmp, Min * nb, Q, p.sc, twl);
    T* other = (res == buf) ? tmp : buf;
    for (int idx = threadIdx.x; idx < nb * Q; idx += blockDim.x) {
        const int lb = idx / Q, kz = idx - lb * Q;
        const long l = l0 + lb;
        const int kx = (int)(l / Q), ky = (int)(l % Q);
        const long so = ((long)kx * H + fold(ky, Q)) * H + fold(kz, Q);
        const bool ny = ky > Q / 2, nz = kz > Q / 2;
        for (int a = 0; a < Mout; ++a) {
            RR ar = 0, ai = 0;
            for (int b = 0; b < Min; ++b) {
                const int info = pis[a * M + b];
                RR s = (RR)S[(long)(info & 0xffff) * H3 + so];
                if (((info >> 17) & 1) && ny) s = -s;
                if (((info >> 18) & 1) && nz) s = -s;
                const T xv = res[(b * nb + lb) * Q + kz];
                if ((info >> 16) & 1) {  // i s x
                    ar -= s * xv.y;
                    ai += s * xv.x;
                } else {
                    ar += s * xv.x;
                    ai += s * xv.y;
                }
            }
            other[(a * nb + lb) * Q + kz] = mk<T>(ar, ai);
        }
    }
    __syncthreads();
    T* res2 = fft_lines<1>(other, res, Mout * nb, Q, p.sc, twl);
    for (int idx = threadIdx.x; idx < Mout * nb * n; idx += blockDim.x) {
        const int row = idx / n, e = idx - row * n;
        const int a = row / nb, lb = row - a * nb;
        T2[a * chs + (l0 + lb) * n + e] = res2[row * Q + e];
    }
}

template <typename T> static int aniso_lines_per_block(int Q) {
    int b = 65536 / (2 * Q * (int)sizeof(T));
    if (b > 16) b = 16;
    if (b < 2) b = 2;
    return b & ~1;
}

template <typename T> static size_t zmix_smem(int Q, int M, int B) {
    return (size_t)(Q + 2 * (long)M * B * Q) * sizeof(T);
}

// dynamic shared memory a Z block may take: the opt-in limit less the static
// pair table (and a margin)
static const size_t kZmixCap = (size_t)RTE_SMEM_OPTIN - RTE_ANISO_MAX_M * RTE_ANISO_MAX_M * sizeof(int) - 1024;

// lines per Z block: the largest B <= 8 whose buffers stay within 48 KB, so that
// at least four blocks share an SM (the pass is latency-bound: one 140 KB block
// per SM kept 8 warps active and reached 3 % of the DRAM bandwidth); B = 1 when
// even one line needs more, if it fits at all (0: it does not)
template <typename T> static int zmix_lines(int Q, int M) {
    for (int B = 8; B >= 1; --B)
        if (zmix_smem<T>(Q, M, B) <= 48 * 1024) return B;
    return zmix_smem<T>(Q, M, 1) <= kZmixCap ? 1 : 0;
}

template <typename K> static cudaError_t allow_big(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, RTE_SMEM_OPTIN);
}

template <typename T, typename R, typename TS> static cudaError_t stockham_prepare() {
    static bool once = false;
    if (once) return cudaSuccess;
    cudaError_t e;
    if ((e = allow_big(k3_x_fwd<T, R>)) != cudaSuccess) return e;
    if ((e = allow_big(k3_y_fwd<T>)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k3a_z_mix<T, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kZmixCap)) !=
        cudaSuccess)
        return e;
    if ((e = allow_big(k3_y_inv<T>)) != cudaSuccess) return e;
    if ((e = allow_big(k3_x_inv<T, R>)) != cudaSuccess) return e;
    once = true;
    return cudaSuccess;
}

// out_a = ca * x_a + cb * (K v)_a + cc * z_a  (rhs = 0; x has M channels,
//         v_b = mu_s sigma_hat_{l_b} x_b, plus xf in channel 0 when xf is given), or
// out_a = cb * (K~^{a0} f)_a                  (rhs = 1; x = f, one channel).
// Stockham passes channel by channel (any Q = 2^a 3^b).
template <typename T, typename R, typename TS>
static cudaError_t aniso_run(rte_aniso3d op, const R* x, R* out, int rhs, double ca, double cb, const R* zv, double cc,
                             const double* xf, const TS* S, const T* tw, int Bz, cudaStream_t s) {
    cudaError_t e;
    if ((e = stockham_prepare<T, R, TS>()) != cudaSuccess) return e;
    const int n = op->n, Q = op->Q, H = op->H, M = op->M;
    P3 pp;
    pp.n = n;
    pp.Q = Q;
    pp.H = H;
    pp.sc = op->sc;
    pp.B = aniso_lines_per_block<T>(Q);
    const int B = pp.B;
    const size_t smx = (size_t)(Q + 2 * (B / 2) * Q) * sizeof(T);
    const size_t smy = (size_t)(Q + 2 * B * Q) * sizeof(T);
    T* T1 = (T*)op->T1;
    T* T2 = (T*)op->T2;
    const long N = (long)n * n * n, chs = (long)H * Q * n;
    const int Min = rhs ? 1 : M;
    long launches = 0;
    for (int b = 0; b < Min; ++b) {
        const double w = rhs ? 1.0 : op->mu_s * op->sig[chan_l(b)];
        k3_x_fwd<T, R><<<dim3((n + B - 1) / B, n), 256, smx, s>>>(x + b * N, T1, tw, pp, w,
                                                                    (!rhs && b == 0) ? xf : nullptr);
        k3_y_fwd<T><<<dim3((n + B - 1) / B, H), 256, smy, s>>>(T1, T2 + b * chs, tw, pp);
        launches += 2;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    P3 pz = pp;
    pz.B = Bz;
    const long nlines = (long)H * Q;
    k3a_z_mix<T, TS><<<(unsigned)((nlines + Bz - 1) / Bz), 256, zmix_smem<T>(Q, M, Bz), s>>>(
        T2, chs, Min, M, S, (long)H * H * H, op->pinfo, M, tw, pz);
    ++launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int a = 0; a < M; ++a) {
        k3_y_inv<T><<<dim3((n + B - 1) / B, H), 256, smy, s>>>(T2 + a * chs, T1, tw, pp);
        k3_x_inv<T, R><<<dim3((n + B - 1) / B, n), 256, smx, s>>>(T1, (rhs || ca == 0.0) ? nullptr : x + a * N,
                                                                    zv ? zv + a * N : nullptr, out + a * N, tw, pp,
                                                                    ca, cb, cc);
        launches += 2;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    rte_count_launches(launches);
    return cudaSuccess;
}

// FP64: native FP64 passes
static rte_status aniso_apply64(rte_aniso3d op, const double* x, double* y, int rhs, double ca, double cb,
                                const double* zv, double cc, const double* xf, cudaStream_t s) {
    cudaError_t e = op->RQ ? aniso_run_warp<double2, double, double>(op, x, y, rhs, ca, cb, zv, cc, xf, op->S64,
                                                                     op->tw64, s)
                           : aniso_run<double2, double, double>(op, x, y, rhs, ca, cb, zv, cc, xf, op->S64, op->tw64,
                                                                op->Bz64, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d apply");
    return RTE_OK;
}
// FP64-accurate on the FP32 units: float-float warp passes (native FP64 on the
// Stockham path)
static rte_status aniso_apply64e(rte_aniso3d op, const double* x, double* y, int rhs, double ca, double cb,
                                 const double* zv, double cc, const double* xf, cudaStream_t s) {
    if (!op->RQ) return aniso_apply64(op, x, y, rhs, ca, cb, zv, cc, xf, s);
    cudaError_t e = aniso_run_warp<ffc, double, ff>(op, x, y, rhs, ca, cb, zv, cc, xf, op->Sff, op->twff, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d apply64e");
    return RTE_OK;
}
static rte_status aniso_apply32(rte_aniso3d op, const float* x, float* y, double ca, double cb, cudaStream_t s) {
    cudaError_t e = op->RQ ? aniso_run_warp<float2, float, float>(op, x, y, 0, ca, cb, nullptr, 0.0, nullptr,
                                                                  op->S32, op->tw32, s)
                           : aniso_run<float2, float, float>(op, x, y, 0, ca, cb, nullptr, 0.0, nullptr, op->S32,
                                                             op->tw32, op->Bz32, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d apply32");
    return RTE_OK;
}

// the solve's operator callbacks (captured into the solve graph)
static rte_status an_A32(void* c, const float* x, float* y, cudaStream_t s) {
    return aniso_apply32((rte_aniso3d)c, x, y, 1.0, -1.0, s);
}
static rte_status an_A64(void* c, const double* x, double* y, cudaStream_t s) {
    return aniso_apply64((rte_aniso3d)c, x, y, 0, 1.0, -1.0, nullptr, 0.0, nullptr, s);
}
__global__ void k_aniso_narrow(const double* __restrict__ src, float* __restrict__ dst, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}
__global__ void k_aniso_widen(const float* __restrict__ src, double* __restrict__ dst, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// b = K~^{.0} f (T.1).  FP64 mode: native FP64.  Mixed: in FP32 (the source
// narrowed into d32, b formed in r32 and widened): b only seeds the first
// inner right-hand side and ||b||, since every residual is the fused exact form
// below
static rte_status an_rhs(void* c, int mixed, cudaStream_t s) {
    rte_aniso3d op = (rte_aniso3d)c;
    if (!mixed) return aniso_apply64(op, op->f, op->b64, 1, 0.0, 1.0, nullptr, 0.0, nullptr, s);
    const long N3 = (long)op->n * op->n * op->n, len = op->M * N3;
    k_aniso_narrow<<<1024, 256, 0, s>>>(op->f, op->d32, N3);
    rte_count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = op->RQ ? aniso_run_warp<float2, float, float>(op, op->d32, op->r32, 1, 0.0, 1.0, nullptr, 0.0, nullptr,
                                                          op->S32, op->tw32, s)
                   : aniso_run<float2, float, float>(op, op->d32, op->r32, 1, 0.0, 1.0, nullptr, 0.0, nullptr,
                                                     op->S32, op->tw32, op->Bz32, s);
    if (e == cudaSuccess) {
        k_aniso_widen<<<1024, 256, 0, s>>>(op->r32, op->b64, len);
        rte_count_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d rhs32");
    return RTE_OK;
}
// r = b - (I - K) u.  Mixed: r = K~ (mu_s sigma_hat u + f) - u in one
// float-float application (the source joins channel 0's input), equal to it
// with the exact b; FP64: r = K u - u + b in native FP64.
static rte_status an_resid(void* c, int mixed, cudaStream_t s) {
    rte_aniso3d op = (rte_aniso3d)c;
    if (mixed) return aniso_apply64e(op, op->u, op->r64, 0, -1.0, 1.0, nullptr, 0.0, op->f, s);
    return aniso_apply64(op, op->u, op->r64, 0, -1.0, 1.0, op->b64, 1.0, nullptr, s);
}

static KrylovOp aniso_krylov_op(rte_aniso3d op) {
    KrylovOp o;
    o.ctx = op;
    o.nr = (long)op->M * op->n * op->n * op->n;
    o.nw1 = o.nr;  // real moments: the plain Euclidean inner product
    o.u = op->u;
    o.b64 = op->b64;
    o.r64 = op->r64;
    o.x64 = op->x64;
    o.part64 = op->part64;
    o.r32 = op->r32;
    o.d32 = op->d32;
    o.ref = op->ref;
    o.A32 = an_A32;
    o.A64 = an_A64;
    o.rhs = an_rhs;
    o.resid = an_resid;
    return o;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" rte_status rte_aniso3d_destroy(rte_aniso3d op) {
    if (!op) return RTE_OK;
    for (int i = 0; i < 3; ++i)
        if (op->graph[i]) cudaGraphExecDestroy((cudaGraphExec_t)op->graph[i]);
    krylov_free_ws(op->k64);
    krylov_free_ws(op->k32);
    void* ptrs[] = {op->tw64, op->tw32, op->twff, op->S64, op->S32, op->Sff, op->wz,    op->pinfo, op->T1,  op->T2,
                    op->u,    op->f,    op->b64,  op->r64, op->x64, op->part64, op->r32, op->d32,  op->ref};
    for (void* q : ptrs)
        if (q) rte_dev_free(q);
    if (op->ref_host) rte_host_free(op->ref_host);
    delete op;
    return RTE_OK;
}

// float-float copies of the FP64 spectra and twiddles
__global__ void k_aniso_split(const double* __restrict__ src, ff* __restrict__ dst, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = ff(src[i]);
}
__global__ void k_aniso_split2(const double2* __restrict__ src, ffc* __restrict__ dst, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = to_ffc(src[i]);
}

// Q: the warp FFT's power of two (64, 128, 256) for 17 <= n <= 128, else the
// smallest even 2^a 3^b >= 2n - 1 with the Stockham passes
static int aniso_choose_Q(int n, int* RQ) {
    *RQ = 0;
    if (n >= 17 && n <= 128) {
        int q = 64;
        while (q < 2 * n - 1) q *= 2;
        *RQ = q / 32;
        return q;
    }
    return choose_Q(n);
}

extern "C" rte_status rte_aniso3d_create(rte_aniso3d* out, int n, double h, double mu_t, double mu_s, int L,
                                         const double* sigma_hat, void* stream) {
    if (!out) return RTE_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 1024 || !(h > 0) || !isfinite(h)) return RTE_EINVAL;
    if (!(mu_t >= 0) || !(mu_s >= 0) || !(mu_s <= mu_t) || !isfinite(mu_t)) return RTE_EINVAL;
    if (L < 0 || L > RTE_ANISO_MAX_L || !sigma_hat) return RTE_EINVAL;
    if (fabs(sigma_hat[0] - 1.0) > 1e-12) return RTE_EINVAL;
    for (int l = 1; l <= L; ++l)
        if (!(fabs(sigma_hat[l]) <= 1.0)) return RTE_EINVAL;
    const int M = (L + 1) * (L + 1);
    int RQ = 0;
    const int Q = aniso_choose_Q(n, &RQ), H = Q / 2 + 1;
    int Bz64 = 0, Bz32 = 0, Bw16 = 0, Bw8 = 0;
    if (RQ) {
        Bw16 = aniso_warp_lines(RQ, M, 16);
        Bw8 = aniso_warp_lines(RQ, M, 8);
        if (Bw16 == 0 || Bw8 == 0)
            return rte_fail(RTE_EUNSUPPORTED, "rte_aniso3d_create: M x Q too large for one Z block");
    } else {
        Bz64 = zmix_lines<double2>(Q, M);
        Bz32 = zmix_lines<float2>(Q, M);
        if (Bz64 == 0 || Bz32 == 0)
            return rte_fail(RTE_EUNSUPPORTED, "rte_aniso3d_create: M x Q too large for one Z block");
    }
    cudaStream_t s = (cudaStream_t)stream;
    {
        // kernel attributes are set here, before any solve graph is captured
        cudaError_t ep = RQ ? aniso_warp_prepare(RQ) : stockham_prepare<double2, double, double>();
        if (ep == cudaSuccess && !RQ) ep = stockham_prepare<float2, float, float>();
        if (ep != cudaSuccess) return rte_cuda_fail(ep, "rte_aniso3d_create");
    }
    rte_aniso3d op = new rte_aniso3d_s();
    op->n = n;
    op->L = L;
    op->M = M;
    op->Q = Q;
    op->H = H;
    op->RQ = RQ;
    op->np = M * (M + 1) / 2;
    op->Bz64 = Bz64;
    op->Bz32 = Bz32;
    op->Bw16 = Bw16;
    op->Bw8 = Bw8;
    op->h = h;
    op->mu_t = mu_t;
    op->mu_s = mu_s;
    for (int l = 0; l <= L; ++l) op->sig[l] = sigma_hat[l];
    make_sched(&op->sc, Q);
    const long H3 = (long)H * H * H, P = (long)Q * Q * Q;
    // pair table
    std::vector<int> pinfo(M * M);
    std::vector<int> pimag(op->np);
    aniso_pair_table(M, pinfo.data(), pimag.data());
    cudaError_t e = cudaSuccess;
    double2* G = nullptr;
    double* Dd = nullptr;
    const size_t t1slabs = RQ ? (size_t)M : 1;
    if (rte_dev_malloc((void**)&op->tw64, Q * sizeof(double2)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->tw32, Q * sizeof(float2)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->S64, op->np * H3 * sizeof(double)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->S32, op->np * H3 * sizeof(float)) != cudaSuccess ||
        (RQ && rte_dev_malloc((void**)&op->twff, Q * sizeof(ffc)) != cudaSuccess) ||
        (RQ && rte_dev_malloc((void**)&op->Sff, op->np * H3 * sizeof(ff)) != cudaSuccess) ||
        rte_dev_malloc((void**)&op->wz, M * sizeof(double)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->pinfo, M * M * sizeof(int)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->T1, t1slabs * n * H * n * sizeof(double2)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->T2, (size_t)M * H * Q * n * sizeof(double2)) != cudaSuccess ||
        rte_dev_malloc((void**)&G, (size_t)P * sizeof(double2)) != cudaSuccess ||
        rte_dev_malloc((void**)&Dd, M * M * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        if (G) rte_dev_free(G);
        if (Dd) rte_dev_free(Dd);
        rte_aniso3d_destroy(op);
        return rte_fail(RTE_ENOMEM, "rte_aniso3d_create");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    e = cudaMemcpyAsync(op->pinfo, pinfo.data(), M * M * sizeof(int), cudaMemcpyHostToDevice, s);
    double wz[RTE_ANISO_MAX_M];
    for (int b = 0; b < M; ++b) wz[b] = mu_s * op->sig[chan_l(b)];
    if (e == cudaSuccess) e = cudaMemcpyAsync(op->wz, wz, M * sizeof(double), cudaMemcpyHostToDevice, s);
    long launches = 0;
    if (e == cudaSuccess) {
        k_twiddles<<<(Q + 255) / 256, 256, 0, s>>>(op->tw64, op->tw32, Q);
        k_aniso_cell_weights<<<M * M, 256, 0, s>>>(L, M, mu_t, h, Dd);
        launches += 2;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(op->Dh, Dd, M * M * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const long Q2 = (long)Q * Q;
    for (int a = 0; a < M && e == cudaSuccess; ++a)
        for (int b = a; b < M && e == cudaSuccess; ++b) {
            const int pidx = pinfo[a * M + b] & 0xffff;
            const int la = chan_l(a), lb = chan_l(b);
            k_aniso_sample<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(G, n, Q, h, mu_t, la > lb ? la : lb, a, b,
                                                                       op->Dh[a * M + b]);
            ++launches;
            e = cudaGetLastError();
            rte_status st = RTE_OK;
            if (e == cudaSuccess) st = fft_lines_host(G, op->sc, op->tw64, Q2, Q2, Q, 0, 1, s);
            if (e == cudaSuccess && st == RTE_OK) st = fft_lines_host(G, op->sc, op->tw64, Q2, Q, 1, Q2, Q, s);
            if (e == cudaSuccess && st == RTE_OK) st = fft_lines_host(G, op->sc, op->tw64, Q2, Q2, 1, 0, Q2, s);
            launches += 3;
            if (st != RTE_OK) e = cudaErrorUnknown;
            if (e == cudaSuccess) {
                k_aniso_extract<<<(unsigned)((H3 + 255) / 256), 256, 0, s>>>(G, Q, H, pimag[pidx], op->S64 + pidx * H3,
                                                                             op->S32 + pidx * H3);
                ++launches;
                e = cudaGetLastError();
            }
        }
    if (e == cudaSuccess && RQ) {
        k_aniso_split<<<1024, 256, 0, s>>>(op->S64, op->Sff, op->np * H3);
        k_aniso_split2<<<(Q + 255) / 256, 256, 0, s>>>(op->tw64, op->twff, Q);
        launches += 2;
        e = cudaGetLastError();
    }
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rte_dev_free(G);
    rte_dev_free(Dd);
    rte_count_launches(launches);
    if (e != cudaSuccess) {
        rte_aniso3d_destroy(op);
        return rte_cuda_fail(e, "rte_aniso3d_create");
    }
    op->ms_pre = ms;
    *out = op;
    return RTE_OK;
}

extern "C" rte_status rte_aniso3d_pair_table(int L, int* out_host) {
    if (L < 0 || L > RTE_ANISO_MAX_L || !out_host) return RTE_EINVAL;
    const int M = (L + 1) * (L + 1);
    std::vector<int> pimag(M * (M + 1) / 2);
    aniso_pair_table(M, out_host, pimag.data());
    return RTE_OK;
}

extern "C" rte_status rte_aniso3d_info(rte_aniso3d op, int* M, int* Q) {
    if (!op) return RTE_EINVAL;
    if (M) *M = op->M;
    if (Q) *Q = op->Q;
    return RTE_OK;
}

extern "C" rte_status rte_aniso3d_cell_weights(rte_aniso3d op, double* out_host) {
    if (!op || !out_host) return RTE_EINVAL;
    memcpy(out_host, op->Dh, (size_t)op->M * op->M * sizeof(double));
    return RTE_OK;
}

extern "C" rte_status rte_aniso3d_apply_K(rte_aniso3d op, const double* x_dev, double* y_dev, void* stream) {
    if (!op || !x_dev || !y_dev || x_dev == y_dev) return RTE_EINVAL;
    return aniso_apply64(op, x_dev, y_dev, 0, 0.0, 1.0, nullptr, 0.0, nullptr, (cudaStream_t)stream);
}

extern "C" rte_status rte_aniso3d_apply_K64e(rte_aniso3d op, const double* x_dev, double* y_dev, void* stream) {
    if (!op || !x_dev || !y_dev || x_dev == y_dev) return RTE_EINVAL;
    return aniso_apply64e(op, x_dev, y_dev, 0, 0.0, 1.0, nullptr, 0.0, nullptr, (cudaStream_t)stream);
}

extern "C" rte_status rte_aniso3d_apply_K32(rte_aniso3d op, const float* x_dev, float* y_dev, void* stream) {
    if (!op || !x_dev || !y_dev || x_dev == y_dev) return RTE_EINVAL;
    return aniso_apply32(op, x_dev, y_dev, 0.0, 1.0, (cudaStream_t)stream);
}

extern "C" rte_status rte_aniso3d_rhs(rte_aniso3d op, const double* f_dev, double* b_dev, void* stream) {
    if (!op || !f_dev || !b_dev) return RTE_EINVAL;
    return aniso_apply64(op, f_dev, b_dev, 1, 0.0, 1.0, nullptr, 0.0, nullptr, (cudaStream_t)stream);
}

// the solve's vectors, each allocated once (a failed allocation is retried
// by the next call)
static rte_status aniso_solve_buffers(rte_aniso3d op, bool mixed) {
    const long N3 = (long)op->n * op->n * op->n, len = op->M * N3;
    struct {
        void** p;
        size_t bytes;
        bool need;
    } bufs[] = {
        {(void**)&op->u, len * sizeof(double), true},
        {(void**)&op->f, N3 * sizeof(double), true},
        {(void**)&op->b64, len * sizeof(double), true},
        {(void**)&op->r64, len * sizeof(double), true},
        {(void**)&op->part64, (size_t)krylov_tiles(len) * sizeof(double), true},
        {(void**)&op->ref, refdev_size(), true},
        {(void**)&op->x64, len * sizeof(double), !mixed},
        {(void**)&op->r32, len * sizeof(float), mixed},
        {(void**)&op->d32, len * sizeof(float), mixed},
    };
    for (auto& b : bufs)
        if (b.need && !*b.p && rte_dev_malloc(b.p, b.bytes) != cudaSuccess) {
            cudaGetLastError();
            return rte_fail(RTE_ENOMEM, "rte_aniso3d_solve");
        }
    if (!op->ref_host && rte_host_malloc(&op->ref_host, 2 * refdev_size()) != cudaSuccess) {
        cudaGetLastError();
        return rte_fail(RTE_ENOMEM, "rte_aniso3d_solve");
    }
    return RTE_OK;
}

// T.1 then T.2 on the device: the plan's solve graph (restarted GMRES with
// device-side control, FP64 or FP32 inner solves with float-float residuals)
// on this operator; f and u are copied into and out of the handle's vectors.
extern "C" rte_status rte_aniso3d_solve(rte_aniso3d op, const double* f_dev, double* u_dev, double tol, int restart,
                                        int maxit, int prec, rte_stats* stats, void* stream) {
    if (!op || !f_dev || !u_dev || !(tol > 0) || restart < 1 || restart > 128 || maxit < 1)
        return RTE_EINVAL;
    if (prec != RTE_PREC_FP64 && prec != RTE_PREC_MIXED_FP32) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const bool mixed = prec == RTE_PREC_MIXED_FP32;
    const long N3 = (long)op->n * op->n * op->n, len = op->M * N3;
    rte_status st = aniso_solve_buffers(op, mixed);
    if (st != RTE_OK) return st;
    const KrylovOp o = aniso_krylov_op(op);
    if (!op->graph[prec] || op->graph_m[prec] != restart) {
        if (op->graph[prec]) cudaGraphExecDestroy((cudaGraphExec_t)op->graph[prec]);
        op->graph[prec] = nullptr;
        st = krylov_op_graph(o, mixed ? op->k32 : op->k64, prec, restart, s, &op->graph[prec], &op->ginfo[prec]);
        if (st != RTE_OK) return st;
        op->graph_m[prec] = restart;
    }
    RTE_CUDA_TRY(cudaMemcpyAsync(op->f, f_dev, N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rte_opts ro;
    memset(&ro, 0, sizeof(ro));
    ro.prec = (rte_prec)prec;
    ro.tol = tol;
    ro.restart = restart;
    ro.maxit = maxit;
    ro.inner_tol = 1e-4;
    const double rho = op->mu_t > 0 ? op->mu_s / op->mu_t : 0.0;
    st = krylov_op_run(o, op->graph[prec], op->ginfo[prec], &ro, op->ref_host, rho, op->ms_pre, stats, s);
    if (st == RTE_OK || st == RTE_ENOCONV) {
        cudaError_t e = cudaMemcpyAsync(u_dev, op->u, len * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d_solve");
    }
    return st;
}
