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
// take the X and Y passes one by one, one Z pass transforms all M channels of
// a (xi_x, xi_y) line, mixes them with the M x M spectra at each xi_z and
// transforms back, and the output channels take the Y' and X' passes.
//
// Each W_ab has a definite parity in x, y and z (Y_a does), so its spectrum
// is real (even total parity) or imaginary (odd) with the same parities; it is
// stored as the octant xi in [0, Q/2]^3 of its real or imaginary part, and
// W_ab = W_ba gives (L+1)^2 ((L+1)^2 + 1)/2 distinct spectra.
#include <math.h>
#include <string.h>

#include <vector>

#include "internal.h"
#include "op3d_passes.cuh"

#define RTE_ANISO_MAX_L 4
#define RTE_ANISO_MAX_M ((RTE_ANISO_MAX_L + 1) * (RTE_ANISO_MAX_L + 1))

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

__host__ __device__ inline int chan_l(int a) {
    int l = 0;
    while ((l + 1) * (l + 1) <= a) ++l;
    return l;
}

// parities of Y_{l,m} under x -> -x, y -> -y, z -> -z (+1 even, -1 odd)
static void sh_parity(int a, int* px, int* py, int* pz) {
    const int l = chan_l(a), m = a - l * l - l, am = m < 0 ? -m : m;
    const int sm = (am & 1) ? -1 : 1;
    *px = m >= 0 ? sm : -sm;
    *py = m >= 0 ? 1 : -1;
    *pz = ((l + am) & 1) ? -1 : 1;
}

// The channel-pair table: for a, b < M, pair index (a <= b numbered row by row)
// | imaginary spectrum << 16 | odd in y << 17 | odd in z << 18, symmetric in
// (a, b); pimag[pair] = the imaginary flag.
static void aniso_pair_table(int M, int* pinfo, int* pimag) {
    int pidx = 0;
    for (int a = 0; a < M; ++a)
        for (int b = a; b < M; ++b) {
            int ax, ay, az, bx, by, bz;
            sh_parity(a, &ax, &ay, &az);
            sh_parity(b, &bx, &by, &bz);
            const int px = ax * bx, py = ay * by, pz = az * bz;
            const int imag = (px * py * pz) < 0 ? 1 : 0;
            const int info = pidx | (imag << 16) | ((py < 0) << 17) | ((pz < 0) << 18);
            pinfo[a * M + b] = pinfo[b * M + a] = info;
            pimag[pidx] = imag;
            ++pidx;
        }
}

struct rte_aniso3d_s {
    int n = 0, L = 0, M = 0, Q = 0, H = 0, np = 0, Bz64 = 0, Bz32 = 0;
    double h = 0.0, mu_t = 0.0, mu_s = 0.0, ms_pre = 0.0;
    double sig[RTE_ANISO_MAX_L + 1] = {};
    double Dh[RTE_ANISO_MAX_M * RTE_ANISO_MAX_M] = {};
    FftSched sc;
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    double* S64 = nullptr;  // [np][H][H][H], xi_z fastest
    float* S32 = nullptr;
    int* pinfo = nullptr;   // [M][M]: pair index | imaginary << 16 | odd in y << 17 | odd in z << 18
    void* T1 = nullptr;     // n*H*n complex doubles
    void* T2 = nullptr;     // M*H*Q*n complex doubles
    // FP64 GMRES workspace
    int gm = 0;
    double* V = nullptr;     // (gm + 1) x len
    double* bvec = nullptr;  // len
    double* r = nullptr;     // len
    double* part = nullptr;  // (gm + 1) x nblk partial sums
    double* hd = nullptr;    // gm + 1 coefficients
    // FP32 inner solves of the mixed refinement
    float* V32 = nullptr;  // (gm + 1) x len
    float* r32 = nullptr;
    float* x32 = nullptr;
    float* b32 = nullptr;
};

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

// out_a = ca * x_a + cb * (K x)_a  (rhs = 0; x has M channels), or
// out_a = cb * (K~^{a0} f)_a       (rhs = 1; x = f, one channel).
template <typename T, typename R, typename TS>
static cudaError_t aniso_run(rte_aniso3d op, const R* x, R* out, int rhs, double ca, double cb, const TS* S,
                             const T* tw, int Bz, cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_big(k3_x_fwd<T, R>)) != cudaSuccess) return e;
        if ((e = allow_big(k3_y_fwd<T>)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k3a_z_mix<T, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kZmixCap)) !=
            cudaSuccess)
            return e;
        if ((e = allow_big(k3_y_inv<T>)) != cudaSuccess) return e;
        if ((e = allow_big(k3_x_inv<T, R>)) != cudaSuccess) return e;
        once = true;
    }
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
        k3_x_fwd<T, R><<<dim3((n + B - 1) / B, n), 256, smx, s>>>(x + b * N, T1, tw, pp, w, nullptr);
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
                                                                    nullptr, out + a * N, tw, pp, ca, cb, 0.0);
        launches += 2;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    rte_count_launches(launches);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Restarted GMRES on (I - K) u = b (Sec. 3.3, T.2): classical Gram-Schmidt
// applied twice, inner products accumulated in FP64, the small Hessenberg
// problem on the host.  T = double (the FP64 solve) or float (the inner solves
// of the mixed refinement, whose residuals are FP64 applications).
// ---------------------------------------------------------------------------
#define ANISO_NBLK 304  // 2 x 152 SMs

// part[i * nblk + blk] = sum over the block's chunk of V_i . w
template <typename T>
__global__ void __launch_bounds__(256) k_aniso_dots(const T* __restrict__ V, long len, const T* __restrict__ w,
                                                    double* __restrict__ part) {
    __shared__ double red[256];
    const int i = blockIdx.y;
    const T* v = V + (long)i * len;
    double acc = 0.0;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (long)gridDim.x * blockDim.x)
        acc += (double)v[t] * (double)w[t];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long)i * gridDim.x + blockIdx.x] = red[0];
}

// out[i] = sum of the nblk partial sums of row i (fixed order)
__global__ void k_aniso_sum(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) acc += part[(long)blockIdx.x * nblk + t];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// w += sgn * sum_{i < k} c_i V_i
template <typename T>
__global__ void k_aniso_comb(T* __restrict__ w, const T* __restrict__ V, long len, int k, const double* __restrict__ c,
                             double sgn) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc += c[i] * (double)V[(long)i * len + t];
        w[t] = (T)((double)w[t] + sgn * acc);
    }
}

// dst = alpha * src  (or dst = b - dst when b != null)
template <typename T>
__global__ void k_aniso_scale(T* dst, const T* src, const T* b, long len, double alpha) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (long)gridDim.x * blockDim.x)
        dst[t] = b ? (T)((double)b[t] - (double)dst[t]) : (T)(alpha * (double)src[t]);
}

// r32 = (float)(alpha * r)  /  u += alpha * (double)d32
__global__ void k_aniso_narrow(float* __restrict__ dst, const double* __restrict__ src, long len, double alpha) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (long)gridDim.x * blockDim.x)
        dst[t] = (float)(alpha * src[t]);
}
__global__ void k_aniso_widen_add(double* __restrict__ u, const float* __restrict__ d, long len, double alpha) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (long)gridDim.x * blockDim.x)
        u[t] += alpha * (double)d[t];
}

template <typename T>
static cudaError_t aniso_dots(rte_aniso3d op, const T* V, int k, const T* w, long len, double* h_host,
                              cudaStream_t s) {
    k_aniso_dots<T><<<dim3(ANISO_NBLK, k), 256, 0, s>>>(V, len, w, op->part);
    k_aniso_sum<<<k, 256, 0, s>>>(op->part, ANISO_NBLK, op->hd);
    rte_count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(h_host, op->hd, k * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// (I - K) x  in the vector's precision (ca = 1, cb = -1), or K~^{.0} f (rhs)
static rte_status aniso_apply(rte_aniso3d op, const double* x, double* y, int rhs, double ca, double cb,
                              cudaStream_t s) {
    cudaError_t e = aniso_run<double2, double, double>(op, x, y, rhs, ca, cb, op->S64, op->tw64, op->Bz64, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d apply");
    return RTE_OK;
}
static rte_status aniso_apply(rte_aniso3d op, const float* x, float* y, int rhs, double ca, double cb,
                              cudaStream_t s) {
    cudaError_t e = aniso_run<float2, float, float>(op, x, y, rhs, ca, cb, op->S32, op->tw32, op->Bz32, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d apply32");
    return RTE_OK;
}
static rte_status aniso_apply64(rte_aniso3d op, const double* x, double* y, int rhs, double ca, double cb,
                                cudaStream_t s) {
    return aniso_apply(op, x, y, rhs, ca, cb, s);
}

// GMRES(m) from x = 0 on (I - K) x = rhs until ||rhs - (I - K) x|| <= tol ||rhs||
// (residuals in T) or maxit iterations; V holds m + 1 vectors, r one.
template <typename T>
static rte_status aniso_gmres(rte_aniso3d op, const T* rhs, T* x, T* V, T* r, long len, double tol, int m, int maxit,
                              int* iters_out, int* cycles_out, double* relres_out, cudaStream_t s) {
    const unsigned gb = ANISO_NBLK;
    std::vector<double> Hm((m + 1) * m), cs(m), sn(m), g(m + 1), hcol(m + 1), h2(m + 1), y(m);
    cudaError_t e = cudaSuccess;
    rte_status st = RTE_OK;
    double bn = 0.0;
    if ((e = aniso_dots<T>(op, rhs, 1, rhs, len, &bn, s)) != cudaSuccess) return rte_cuda_fail(e, "aniso_gmres");
    bn = sqrt(bn);
    if ((e = cudaMemsetAsync(x, 0, len * sizeof(T), s)) != cudaSuccess) return rte_cuda_fail(e, "aniso_gmres");
    k_aniso_scale<T><<<gb, 256, 0, s>>>(r, rhs, (const T*)nullptr, len, 1.0);
    rte_count_launches(1);
    double beta = bn, relres = bn > 0 ? 1.0 : 0.0;
    int iters = 0, cycles = 0;
    bool conv = !(bn > 0);
    while (!conv && iters < maxit) {
        ++cycles;
        k_aniso_scale<T><<<gb, 256, 0, s>>>(V, r, (const T*)nullptr, len, 1.0 / beta);
        rte_count_launches(1);
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int j = 0;
        for (; j < m && iters < maxit; ++j) {
            T* w = V + (long)(j + 1) * len;
            if ((st = aniso_apply(op, V + (long)j * len, w, 0, 1.0, -1.0, s)) != RTE_OK) return st;
            // two passes of classical Gram-Schmidt
            for (int pass = 0; pass < 2; ++pass) {
                double* hp = pass ? h2.data() : hcol.data();
                if ((e = aniso_dots<T>(op, V, j + 1, w, len, hp, s)) != cudaSuccess) break;
                if ((e = cudaMemcpyAsync(op->hd, hp, (j + 1) * sizeof(double), cudaMemcpyHostToDevice, s)) !=
                    cudaSuccess)
                    break;
                k_aniso_comb<T><<<gb, 256, 0, s>>>(w, V, len, j + 1, op->hd, -1.0);
                rte_count_launches(1);
            }
            if (e != cudaSuccess) break;
            for (int i = 0; i <= j; ++i) hcol[i] += h2[i];
            double hn = 0.0;
            if ((e = aniso_dots<T>(op, w, 1, w, len, &hn, s)) != cudaSuccess) break;
            hn = sqrt(hn);
            hcol[j + 1] = hn;
            if (hn > 0) {
                k_aniso_scale<T><<<gb, 256, 0, s>>>(w, w, (const T*)nullptr, len, 1.0 / hn);
                rte_count_launches(1);
            }
            for (int i = 0; i < j; ++i) {  // previous Givens rotations
                const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = t;
            }
            const double den = hypot(hcol[j], hcol[j + 1]);
            cs[j] = den > 0 ? hcol[j] / den : 1.0;
            sn[j] = den > 0 ? hcol[j + 1] / den : 0.0;
            hcol[j] = den;
            hcol[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) Hm[i * m + j] = hcol[i];
            ++iters;
            if (fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
                ++j;
                break;
            }
        }
        if (e != cudaSuccess) break;
        for (int i = j - 1; i >= 0; --i) {  // R y = g
            double t = g[i];
            for (int k = i + 1; k < j; ++k) t -= Hm[i * m + k] * y[k];
            y[i] = Hm[i * m + i] != 0.0 ? t / Hm[i * m + i] : 0.0;
        }
        if (j > 0) {
            if ((e = cudaMemcpyAsync(op->hd, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
                break;
            k_aniso_comb<T><<<gb, 256, 0, s>>>(x, V, len, j, op->hd, 1.0);
            rte_count_launches(1);
        }
        // residual r = rhs - (I - K) x in T
        if ((st = aniso_apply(op, x, r, 0, 1.0, -1.0, s)) != RTE_OK) return st;
        k_aniso_scale<T><<<gb, 256, 0, s>>>(r, (const T*)nullptr, rhs, len, 0.0);
        rte_count_launches(1);
        double rn = 0.0;
        if ((e = aniso_dots<T>(op, r, 1, r, len, &rn, s)) != cudaSuccess) break;
        beta = sqrt(rn);
        relres = beta / bn;
        conv = relres <= tol;
        if (!(beta > 0)) break;
    }
    if (e != cudaSuccess) return rte_cuda_fail(e, "aniso_gmres");
    *iters_out += iters;
    *cycles_out += cycles;
    *relres_out = relres;
    return RTE_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" rte_status rte_aniso3d_destroy(rte_aniso3d op) {
    if (!op) return RTE_OK;
    void* ptrs[] = {op->tw64, op->tw32, op->S64, op->S32,  op->pinfo, op->T1,  op->T2,  op->V,
                    op->bvec, op->r,    op->part, op->hd, op->V32,   op->r32, op->x32, op->b32};
    for (void* q : ptrs)
        if (q) rte_dev_free(q);
    delete op;
    return RTE_OK;
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
    const int Q = choose_Q(n), H = Q / 2 + 1;
    const int Bz64 = zmix_lines<double2>(Q, M), Bz32 = zmix_lines<float2>(Q, M);
    if (Bz64 == 0 || Bz32 == 0) return rte_fail(RTE_EUNSUPPORTED, "rte_aniso3d_create: M x Q too large for one Z block");
    cudaStream_t s = (cudaStream_t)stream;
    rte_aniso3d op = new rte_aniso3d_s();
    op->n = n;
    op->L = L;
    op->M = M;
    op->Q = Q;
    op->H = H;
    op->np = M * (M + 1) / 2;
    op->Bz64 = Bz64;
    op->Bz32 = Bz32;
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
    if (rte_dev_malloc((void**)&op->tw64, Q * sizeof(double2)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->tw32, Q * sizeof(float2)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->S64, op->np * H3 * sizeof(double)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->S32, op->np * H3 * sizeof(float)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->pinfo, M * M * sizeof(int)) != cudaSuccess ||
        rte_dev_malloc((void**)&op->T1, (size_t)n * H * n * sizeof(double2)) != cudaSuccess ||
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
    return aniso_apply64(op, x_dev, y_dev, 0, 0.0, 1.0, (cudaStream_t)stream);
}

extern "C" rte_status rte_aniso3d_apply_K32(rte_aniso3d op, const float* x_dev, float* y_dev, void* stream) {
    if (!op || !x_dev || !y_dev || x_dev == y_dev) return RTE_EINVAL;
    cudaError_t e = aniso_run<float2, float, float>(op, x_dev, y_dev, 0, 0.0, 1.0, op->S32, op->tw32, op->Bz32,
                                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d_apply_K32");
    return RTE_OK;
}

extern "C" rte_status rte_aniso3d_rhs(rte_aniso3d op, const double* f_dev, double* b_dev, void* stream) {
    if (!op || !f_dev || !b_dev) return RTE_EINVAL;
    return aniso_apply64(op, f_dev, b_dev, 1, 0.0, 1.0, (cudaStream_t)stream);
}

extern "C" rte_status rte_aniso3d_solve(rte_aniso3d op, const double* f_dev, double* u_dev, double tol, int restart,
                                        int maxit, int prec, rte_stats* stats, void* stream) {
    if (!op || !f_dev || !u_dev || !(tol > 0) || restart < 1 || restart > 200 || maxit < 1) return RTE_EINVAL;
    if (prec != RTE_PREC_FP64 && prec != RTE_PREC_MIXED_FP32) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const long len = (long)op->M * op->n * op->n * op->n;
    const bool mixed = prec == RTE_PREC_MIXED_FP32;
    if (op->gm != restart || (mixed && !op->V32)) {
        for (void** q : {(void**)&op->V, (void**)&op->bvec, (void**)&op->r, (void**)&op->part, (void**)&op->hd,
                         (void**)&op->V32, (void**)&op->r32, (void**)&op->x32, (void**)&op->b32})
            if (*q) {
                rte_dev_free(*q);
                *q = nullptr;
            }
        op->gm = 0;
        bool ok = rte_dev_malloc((void**)&op->bvec, len * sizeof(double)) == cudaSuccess &&
                  rte_dev_malloc((void**)&op->r, len * sizeof(double)) == cudaSuccess &&
                  rte_dev_malloc((void**)&op->part, (size_t)(restart + 1) * ANISO_NBLK * sizeof(double)) == cudaSuccess &&
                  rte_dev_malloc((void**)&op->hd, (restart + 1) * sizeof(double)) == cudaSuccess;
        if (ok && !mixed) ok = rte_dev_malloc((void**)&op->V, (size_t)(restart + 1) * len * sizeof(double)) == cudaSuccess;
        if (ok && mixed)
            ok = rte_dev_malloc((void**)&op->V32, (size_t)(restart + 1) * len * sizeof(float)) == cudaSuccess &&
                 rte_dev_malloc((void**)&op->r32, len * sizeof(float)) == cudaSuccess &&
                 rte_dev_malloc((void**)&op->x32, len * sizeof(float)) == cudaSuccess &&
                 rte_dev_malloc((void**)&op->b32, len * sizeof(float)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return rte_fail(RTE_ENOMEM, "rte_aniso3d_solve");
        }
        op->gm = restart;
    }
    if (!mixed && !op->V) {
        if (rte_dev_malloc((void**)&op->V, (size_t)(restart + 1) * len * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return rte_fail(RTE_ENOMEM, "rte_aniso3d_solve");
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    int iters = 0, cycles = 0, outer = 0;
    double relres = 1.0;
    rte_status st = aniso_apply(op, f_dev, op->bvec, 1, 0.0, 1.0, s);  // b = K~^{.0} f (T.1)
    cudaError_t e = cudaSuccess;
    if (st == RTE_OK && !mixed) {
        st = aniso_gmres<double>(op, op->bvec, u_dev, op->V, op->r, len, tol, restart, maxit, &iters, &outer, &relres,
                                 s);
    } else if (st == RTE_OK) {
        // T.2 refined: FP32 GMRES on (I - K) d = r/||r|| to max(1e-4, tol/(2 relres)),
        // u += ||r|| d, every residual r = b - (I - K) u an FP64 application
        const unsigned gb = ANISO_NBLK;
        double bn = 0.0;
        e = aniso_dots<double>(op, op->bvec, 1, op->bvec, len, &bn, s);
        bn = sqrt(bn);
        if (e == cudaSuccess) e = cudaMemsetAsync(u_dev, 0, len * sizeof(double), s);
        if (e == cudaSuccess) {
            k_aniso_scale<double><<<gb, 256, 0, s>>>(op->r, op->bvec, (const double*)nullptr, len, 1.0);
            rte_count_launches(1);
        }
        double rn = bn;
        relres = bn > 0 ? 1.0 : 0.0;
        while (st == RTE_OK && e == cudaSuccess && relres > tol && iters < maxit && outer < 50) {
            ++outer;
            k_aniso_narrow<<<gb, 256, 0, s>>>(op->b32, op->r, len, 1.0 / rn);
            rte_count_launches(1);
            double itol = fmax(1e-4, 0.5 * tol / relres);
            if (itol > 0.5) itol = 0.5;
            double rr32 = 0.0;
            st = aniso_gmres<float>(op, op->b32, op->x32, op->V32, op->r32, len, itol, restart, maxit - iters, &iters,
                                    &cycles, &rr32, s);
            if (st != RTE_OK) break;
            k_aniso_widen_add<<<gb, 256, 0, s>>>(u_dev, op->x32, len, rn);
            rte_count_launches(1);
            if ((st = aniso_apply(op, u_dev, op->r, 0, 1.0, -1.0, s)) != RTE_OK) break;
            k_aniso_scale<double><<<gb, 256, 0, s>>>(op->r, (const double*)nullptr, op->bvec, len, 0.0);
            rte_count_launches(1);
            double r2 = 0.0;
            if ((e = aniso_dots<double>(op, op->r, 1, op->r, len, &r2, s)) != cudaSuccess) break;
            rn = sqrt(r2);
            relres = bn > 0 ? rn / bn : 0.0;
            if (!(rn > 0)) break;
        }
    }
    cudaEventRecord(e1, s);
    cudaError_t e2 = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RTE_OK) return st;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_aniso3d_solve");
    const bool conv = relres <= tol;
    if (stats) {
        const double rr = op->mu_t > 0 ? op->mu_s / op->mu_t : 1.0;
        stats->iters = iters;
        stats->outer = outer;
        stats->converged = conv ? 1 : 0;
        stats->relres_true = relres;
        stats->ms_total = ms;
        stats->ms_pre = op->ms_pre;
        stats->est_err_bound = rr < 1 ? (1 + rr) / (1 - rr) * relres : INFINITY;
    }
    if (!isfinite(relres)) return rte_fail(RTE_ENOCONV, "rte_aniso3d_solve: non-finite residual");
    return conv ? RTE_OK : RTE_ENOCONV;
}
