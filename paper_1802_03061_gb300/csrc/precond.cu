// Periodic (circulant) preconditioner for the FP32 inner solves.
//
// The operator K is a convolution cropped to the n^d cells (Sec. 2.3.1,
// 3.3.1): K x = crop(C pad(x)), where C is the convolution with the same kernel
// samples on the Q^d periodic grid.  C is diagonal in Fourier space -- a scalar
// per frequency for d = 3 (L = 0), a (2L+1) x (2L+1) matrix T(xi) on the real
// channels for d = 2 -- so (I - C)^{-1} is exact and cheap on the periodic
// grid, and M = crop (I - C)^{-1} pad approximates (I - K)^{-1} everywhere
// except near the boundary of the square / cube.  GMRES on A M (right
// preconditioning: the inner solves still measure the true residual) then
// needs a few iterations instead of tens.  Not in the paper (which runs
// GMRES / MINRES without a preconditioner); the answer is the same to the
// solve's tolerance.
//
// 2D, block lower triangular in the modes: with "low" the channels of the
// modes |k| <= lmax (nl = 2 lmax + 1 of them), the stored matrix is
// P = T[:, low] (I - T_ll)^{-1} and M x = x + crop P pad(x_low).  For
// lmax = L this is crop (I - T)^{-1} pad (P = (I - T)^{-1} - I); for smaller
// lmax the higher modes keep their coupling to the inverted block and drop
// T_lh and T_hh, which carry mu_s sigma_hat_k of the high modes only.
//
// T(xi) has entries that are purely real or purely imaginary, imaginary
// exactly when the modes of the two channels differ in parity (see the mode
// mix in op2d.cuh), and so has P: one real number per entry.  Mirroring
// xi_y -> -xi_y reverses the angle of every kernel sample, which maps mode k
// to -k; on the real channels (A_k, B_k) = ((u_k + u_-k)/2, (u_k - u_-k)/2i)
// that is A -> A, B -> -B, so P(xi_x, -xi_y) = S P(xi_x, xi_y) S with
// S = diag(+1 on A, -1 on B).  Only xi_y in [0, Q/2] is stored, in BF16 (the
// preconditioner only has to be close, not exact), as Pp[xi_x][c][c'][xi_y]
// (c < 2L+1, c' < nl) with rows of pc_row(Q) = Q/2 + 8 entries, scaled by
// 1/Q^2 for the unnormalised transforms of the passes.
#include "op2d_launch.cuh"

__host__ __device__ __forceinline__ int ch_mode(int c) { return (c + 1) >> 1; }
__host__ __device__ __forceinline__ bool ch_isB(int c) { return c > 0 && !(c & 1); }
// table row length (xi_y = 0..Q/2, padded to 16 bytes)
__host__ __device__ __forceinline__ int pc_row(int Q) { return Q / 2 + 8; }

// slot (j * 32 + lane) of the warp FFT that holds frequency xi: the inverse
// of wfreq<R>
template <int R> __device__ __forceinline__ int wslot(int xi) {
    using W = wfft_shape<R>;
    const int g = xi % R, kap = (xi / R) % R, c = xi / (R * R);
    if constexpr (R >= W::P) {
        // register P t + c of lane P g + b holds kappa' = b + P t
        return (W::P * (kap / W::P) + c) * 32 + ((g << W::LP) | (kap % W::P));
    } else {
        const int b = (int)(__brev((unsigned)c) >> (32 - W::LP));
        return kap * 32 + ((g << W::LP) | b);
    }
}

// 3D: S3p = (1/Q^3) / (1 - mu_s Q^3 S3)  (S3 already holds FFT(g) / Q^3)
__global__ void k_build_pc3d(const double* __restrict__ S3, float* __restrict__ S3p, long tot, double mu_s,
                             double Q3) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x)
        S3p[i] = (float)((1.0 / Q3) / (1.0 - mu_s * Q3 * S3[i]));
}

// 2D: one thread per (xi_x, xi_y), xi_y = 0..Q/2.  T[c][c'] = Q^2 *
// mix(S(xi))[c][c'] * w(c') with w = mu_s sigma_hat_{k(c')} (the row pass's
// input weights).  With the first nl channels (modes |k| <= lmax) as the
// inverted block, the stored matrix is P = T[:, <nl] (I - T_ll)^{-1}
// (Gauss-Jordan with partial pivoting in complex FP64), so that
// M x = x + crop P pad(x_<nl): for nl = 2L+1 this is (I - T)^{-1} exactly
// (P = (I - T)^{-1} - I); for fewer channels the higher modes keep their
// coupling to the inverted block and drop the weak rest.
template <int L>
__global__ void k_build_pc2d(const double2* __restrict__ S64, __nv_bfloat16* __restrict__ Pp, int H, int Q,
                             RowParams rp, double Q2, int nl) {
    constexpr int NCH = 2 * L + 1;
    const int QH = Q / 2 + 1, QR = pc_row(Q);
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)H * QH) return;
    const int kx = (int)(idx / QH), ky = (int)(idx % QH);
    double sr[2 * L + 1], si[2 * L + 1];
#pragma unroll
    for (int m = 0; m <= 2 * L; ++m) {
        const double2 v = S64[((long)kx * NCH + m) * Q + ky];
        sr[m] = v.x;
        si[m] = v.y;
    }
    double2 T[NCH][NCH];  // columns < nl used
    for (int cp = 0; cp < nl; ++cp) {
        double2 in[NCH], o[NCH];
        for (int c = 0; c < NCH; ++c) in[c] = make_double2(c == cp ? 1.0 : 0.0, 0.0);
        mode_mix<L, double2>(sr, si, in, o);
        const double w = rp.wk[ch_mode(cp)] * Q2;
        for (int c = 0; c < NCH; ++c) T[c][cp] = make_double2(w * o[c].x, w * o[c].y);
    }
    double2 A[NCH][NCH], Inv[NCH][NCH];  // I - T_ll, then (I - T_ll)^{-1} (nl x nl)
    for (int r = 0; r < nl; ++r)
        for (int c = 0; c < nl; ++c) {
            A[r][c] = make_double2((r == c ? 1.0 : 0.0) - T[r][c].x, -T[r][c].y);
            Inv[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
        }
    for (int col = 0; col < nl; ++col) {
        int piv = col;
        double best = hypot(A[col][col].x, A[col][col].y);
        for (int r = col + 1; r < nl; ++r) {
            const double a = hypot(A[r][col].x, A[r][col].y);
            if (a > best) { best = a; piv = r; }
        }
        if (piv != col) {
            for (int c = 0; c < nl; ++c) {
                double2 t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t;
                t = Inv[col][c]; Inv[col][c] = Inv[piv][c]; Inv[piv][c] = t;
            }
        }
        const double2 d = A[col][col];
        const double dd = d.x * d.x + d.y * d.y;
        const double2 inv = make_double2(d.x / dd, -d.y / dd);
        for (int c = 0; c < nl; ++c) {
            A[col][c] = cmul(A[col][c], inv);
            Inv[col][c] = cmul(Inv[col][c], inv);
        }
        for (int r = 0; r < nl; ++r) {
            if (r == col) continue;
            const double2 f = A[r][col];
            for (int c = 0; c < nl; ++c) {
                A[r][c] = csub(A[r][c], cmul(f, A[col][c]));
                Inv[r][c] = csub(Inv[r][c], cmul(f, Inv[col][c]));
            }
        }
    }
    for (int c = 0; c < NCH; ++c)
        for (int cq = 0; cq < nl; ++cq) {
            double2 v = make_double2(0.0, 0.0);
            for (int cp = 0; cp < nl; ++cp) v = cadd(v, cmul(T[c][cp], Inv[cp][cq]));
            const bool im = ((ch_mode(c) ^ ch_mode(cq)) & 1) != 0;
            Pp[(((long)kx * NCH + c) * nl + cq) * QR + ky] = __float2bfloat16_rn((float)((im ? v.y : v.x) / Q2));
        }
}

// y[c] = sum_{c' < nl} P[c][c'] x[c'] for one frequency (or the mirror pair
// (xi, Q - xi), the mirror with S P S), every output channel c < 2L+1.  The
// loop over the inverted inputs c' has a run-time bound; for each c' the
// 2L+1 coefficients P[.][c'] are independent loads.  An entry is i v when the
// channel modes differ in parity and its mirror sign flips when exactly one
// of c, c' is a B channel; c' enters both only through (parity, B) -- uniform
// over the block -- so a switch on them keeps every tag a compile-time constant.
template <int L, bool PAIR, int PC, bool BC>
__device__ __forceinline__ void pc_mix_term(float2* ra, float2* rb, float2 a, float2 b, const __nv_bfloat16* Pcp,
                                            long cstride) {
    constexpr int NCH = 2 * L + 1;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const float v = __bfloat162float(Pcp[c * cstride]);
        const bool im = ((ch_mode(c) & 1) ^ PC) != 0;
        if (im) {
            ra[c].x -= v * a.y;
            ra[c].y += v * a.x;
        } else {
            ra[c].x += v * a.x;
            ra[c].y += v * a.y;
        }
        if (PAIR) {
            const float w = ch_isB(c) != BC ? -v : v;
            if (im) {
                rb[c].x -= w * b.y;
                rb[c].y += w * b.x;
            } else {
                rb[c].x += w * b.x;
                rb[c].y += w * b.y;
            }
        }
    }
}

template <int L, bool PAIR>
__device__ __forceinline__ void pc_mix(float2* X, int QS, int s1, int s2, const __nv_bfloat16* P, int QR, int nl) {
    constexpr int NCH = 2 * L + 1;
    float2 ra[NCH], rb[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        ra[c] = make_float2(0.f, 0.f);
        rb[c] = make_float2(0.f, 0.f);
    }
    const long cstride = (long)nl * QR;  // P[c][c'] at P + c * nl * QR + c' * QR
    for (int cp = 0; cp < nl; ++cp) {
        const float2 a = X[cp * QS + s1];
        const float2 b = PAIR ? X[cp * QS + s2] : make_float2(0.f, 0.f);
        const __nv_bfloat16* Pcp = P + (long)cp * QR;
        const int pc = ch_mode(cp) & 1;
        const bool bc = ch_isB(cp);
        if (pc == 0 && !bc) pc_mix_term<L, PAIR, 0, false>(ra, rb, a, b, Pcp, cstride);
        else if (pc == 0) pc_mix_term<L, PAIR, 0, true>(ra, rb, a, b, Pcp, cstride);
        else if (!bc) pc_mix_term<L, PAIR, 1, false>(ra, rb, a, b, Pcp, cstride);
        else pc_mix_term<L, PAIR, 1, true>(ra, rb, a, b, Pcp, cstride);
    }
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        X[c * QS + s1] = ra[c];
        if (PAIR) X[c * QS + s2] = rb[c];
    }
}

template <int L>
__device__ __forceinline__ void pc_mix_one(float2* X, int QS, int sl, const __nv_bfloat16* P, int QR, int nl) {
    pc_mix<L, false>(X, QS, sl, sl, P, QR, nl);
}
template <int L>
__device__ __forceinline__ void pc_mix_pair(float2* X, int QS, int s1, int s2, const __nv_bfloat16* P, int QR,
                                            int nl) {
    pc_mix<L, true>(X, QS, s1, s2, P, QR, nl);
}

// 16-byte global -> shared copy that bypasses the registers (cp.async), and
// its group bookkeeping
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// one mix step of the staged column pass: the inverted input channel cp with
// its coefficients P[.][cp][.] in shared memory (rows of QR entries)
template <int L, int PC, bool BC>
__device__ __forceinline__ void pc_stage_term(float2* ra, float2* rb, float2 a, float2 b,
                                              const __nv_bfloat16* __restrict__ buf, int QR, int t, int t2,
                                              bool mirror) {
    constexpr int NCH = 2 * L + 1;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const float v = __bfloat162float(buf[c * QR + t]);
        float w = __bfloat162float(buf[c * QR + t2]);
        if (mirror && ch_isB(c) != BC) w = -w;
        const bool im = ((ch_mode(c) & 1) ^ PC) != 0;
        if (im) {
            ra[c].x -= v * a.y;
            ra[c].y += v * a.x;
            rb[c].x -= w * b.y;
            rb[c].y += w * b.x;
        } else {
            ra[c].x += v * a.x;
            ra[c].y += v * a.y;
            rb[c].x += w * b.x;
            rb[c].y += w * b.y;
        }
    }
}

// column pass of the preconditioner (Q = 32 R <= 512): FFT_y of the nl
// inverted channels, per frequency pair (xi, Q - xi) the tagged product with
// P, inverse FFT_y of every channel (as k_col_warp).  The table slice of one
// inverted channel (17 rows of Q/2 + 8 BF16) is copied into shared memory by
// cp.async, two stages ahead: the first two while the forward FFTs run, the
// next one while a stage is being used.  Thread t < Q/2 takes the pair
// (t, Q - t); thread 0 takes xi = 0 and xi = Q/2, each its own mirror.
template <int L, int R>
__global__ void __launch_bounds__(256, 2) k_col_warp_pc(float2* __restrict__ Tb, const __nv_bfloat16* __restrict__ Pp,
                                                     const float2* __restrict__ tw, int n, int H, int nl) {
    constexpr int NCH = 2 * L + 1;
    constexpr int Q = 32 * R;
    constexpr int QR = Q / 2 + 8;
    constexpr int QS = wfft_shape<R>::SCRATCH;
    constexpr int CPR = QR * 2 / 16;  // 16-byte chunks per table row
    extern __shared__ unsigned char smraw[];
    float2* X = reinterpret_cast<float2*>(smraw);  // [NCH][QS]
    __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(X + NCH * QS);  // [2][NCH][QR]
    const int kx = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const __nv_bfloat16* Pk = Pp + (long)kx * NCH * nl * QR;
    auto issue = [&](int cp) {
        __nv_bfloat16* dst = stage + (cp & 1) * NCH * QR;
        for (int q = threadIdx.x; q < NCH * CPR; q += blockDim.x) {
            const int c = q / CPR, k = q - c * CPR;
            cp_async16(reinterpret_cast<char*>(dst + c * QR) + 16 * k,
                       reinterpret_cast<const char*>(Pk + ((long)c * nl + cp) * QR) + 16 * k);
        }
    };
    issue(0);
    cp_async_commit();
    if (nl > 1) issue(1);
    cp_async_commit();
    pdl_wait();  // Tb: the row pass's output (the table is a plan constant)
    pdl_trigger();
    for (int c = warp; c < nl; c += nw) {
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
    const int t = threadIdx.x;
    const bool act = t < Q / 2;
    const int s1 = wslot<R>(act ? t : 0), s2 = wslot<R>(t == 0 ? Q / 2 : (act ? Q - t : 0));
    const int t2 = t == 0 ? Q / 2 : t;  // table column of the second frequency
    float2 ra[NCH], rb[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        ra[c] = make_float2(0.f, 0.f);
        rb[c] = make_float2(0.f, 0.f);
    }
    for (int cp = 0; cp < nl; ++cp) {
        cp_async_wait1();  // this thread's copies of stage cp have landed
        __syncthreads();   // everyone's (and, for cp = 0, the forward FFTs)
        if (act) {
            const __nv_bfloat16* buf = stage + (cp & 1) * NCH * QR;
            const float2 a = X[cp * QS + s1], b = X[cp * QS + s2];
            const int pcp = ch_mode(cp) & 1;
            const bool bc = ch_isB(cp), mirror = t != 0;
            if (pcp == 0 && !bc) pc_stage_term<L, 0, false>(ra, rb, a, b, buf, QR, t, t2, mirror);
            else if (pcp == 0) pc_stage_term<L, 0, true>(ra, rb, a, b, buf, QR, t, t2, mirror);
            else if (!bc) pc_stage_term<L, 1, false>(ra, rb, a, b, buf, QR, t, t2, mirror);
            else pc_stage_term<L, 1, true>(ra, rb, a, b, buf, QR, t, t2, mirror);
        }
        __syncthreads();  // stage cp & 1 is free again
        if (cp + 2 < nl) issue(cp + 2);
        cp_async_commit();
    }
    if (act) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            X[c * QS + s1] = ra[c];
            X[c * QS + s2] = rb[c];
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

// Q = 1024 as two 512-point residues r = xi mod 2 (as k_col_warp2): the
// mirror Q - xi of a frequency of residue r has residue r too (Q - 2k =
// 2(512 - k), Q - 2k - 1 = 2(511 - k) + 1), so the pairs stay within a residue:
// r = 0 pairs k with 512 - k (k = 0 and 256 alone), r = 1 pairs k with 511 - k.
template <int L>
__global__ void __launch_bounds__(256, 2) k_col_warp_pc2(float2* __restrict__ Tb, float2* __restrict__ Tz,
                                                         const __nv_bfloat16* __restrict__ Pp,
                                                         const float2* __restrict__ tw, int n, int H, int nl) {
    constexpr int NCH = 2 * L + 1;
    constexpr int R = 16, QW = 512, Q = 1024;
    constexpr int QR = Q / 2 + 8;
    constexpr int QS = wfft_shape<R>::SCRATCH;
    constexpr int CPR = QR * 2 / 16;
    extern __shared__ unsigned char smraw[];
    float2* twl = reinterpret_cast<float2*>(smraw);  // exp(-2 pi i t / 512)
    float2* X = twl + QW;                            // [NCH][QS]
    __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(X + NCH * QS);  // [2][NCH][QR]
    const int kx = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const __nv_bfloat16* Pk = Pp + (long)kx * NCH * nl * QR;
    // stage g = r * nl + cp holds the table rows of the inverted channel cp
    auto issue = [&](int g) {
        const int cp = g % nl;
        __nv_bfloat16* dst = stage + (g & 1) * NCH * QR;
        for (int q = threadIdx.x; q < NCH * CPR; q += blockDim.x) {
            const int c = q / CPR, k = q - c * CPR;
            cp_async16(reinterpret_cast<char*>(dst + c * QR) + 16 * k,
                       reinterpret_cast<const char*>(Pk + ((long)c * nl + cp) * QR) + 16 * k);
        }
    };
    const int ng = 2 * nl;
    issue(0);
    cp_async_commit();
    issue(1);
    cp_async_commit();
    for (int i = threadIdx.x; i < QW; i += blockDim.x) twl[i] = tw[2 * i];
    __syncthreads();
    const int t = threadIdx.x;
    const bool act = t < QW / 2;
    for (int r = 0; r < 2; ++r) {
        for (int c = warp; c < nl; c += nw) {
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
        // residue 0: thread 0 takes xi = 0 and Q/2 (own mirrors, columns 0 and
        // 512), thread t pairs k = t with 512 - t (column 2t); residue 1: k = t
        // with 511 - t (column 2t + 1)
        const int tt = act ? t : 0;
        const bool single = r == 0 && t == 0;
        const int s1 = wslot<R>(tt);
        const int s2 = wslot<R>(single ? QW / 2 : (r == 0 ? QW - tt : QW - 1 - tt));
        const int col1 = 2 * tt + r, col2 = single ? QW : col1;
        float2 ra[NCH], rb[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            ra[c] = make_float2(0.f, 0.f);
            rb[c] = make_float2(0.f, 0.f);
        }
        for (int cp = 0; cp < nl; ++cp) {
            const int g = r * nl + cp;
            cp_async_wait1();
            __syncthreads();
            if (act) {
                const __nv_bfloat16* buf = stage + (g & 1) * NCH * QR;
                const float2 a = X[cp * QS + s1], b = X[cp * QS + s2];
                const int pcp = ch_mode(cp) & 1;
                const bool bc = ch_isB(cp), mirror = !single;
                if (pcp == 0 && !bc) pc_stage_term<L, 0, false>(ra, rb, a, b, buf, QR, col1, col2, mirror);
                else if (pcp == 0) pc_stage_term<L, 0, true>(ra, rb, a, b, buf, QR, col1, col2, mirror);
                else if (!bc) pc_stage_term<L, 1, false>(ra, rb, a, b, buf, QR, col1, col2, mirror);
                else pc_stage_term<L, 1, true>(ra, rb, a, b, buf, QR, col1, col2, mirror);
            }
            __syncthreads();
            if (g + 2 < ng) issue(g + 2);
            cp_async_commit();
        }
        if (act) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                X[c * QS + s1] = ra[c];
                X[c * QS + s2] = rb[c];
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

template <int L>
static cudaError_t launch_col_pc2(float2* Tb, float2* Tz, const __nv_bfloat16* Pp, const float2* tw, int n, int H,
                                  int nl, cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_col_warp_pc2<L>)) != cudaSuccess) return e;
        once = true;
    }
    const size_t smem = (size_t)(512 + (2 * L + 1) * wfft_shape<16>::SCRATCH) * sizeof(float2) +
                        (size_t)2 * (2 * L + 1) * (1024 / 2 + 8) * sizeof(__nv_bfloat16);
    k_col_warp_pc2<L><<<H, 256, smem, s>>>(Tb, Tz, Pp, tw, n, H, nl);
    return cudaGetLastError();
}

// the same pass with the shared-memory (Stockham, radix 2/3/4/8) FFT for the
// other Q: every channel column of one xi_x resident in natural frequency
// order, FFT groups of G columns (as k_col_fused)
template <int L>
__global__ void __launch_bounds__(256) k_col_pc_fused(float2* __restrict__ Tb, const __nv_bfloat16* __restrict__ Pp,
                                                      const float2* __restrict__ tw, ColParams p, int nl) {
    constexpr int NCH = 2 * L + 1;
    extern __shared__ unsigned char smraw[];
    float2* sm = reinterpret_cast<float2*>(smraw);
    const int n = p.n, Q = p.Q, H = p.H, QR = pc_row(Q);
    const int kx = blockIdx.x;
    float2* twl = sm;
    float2* X = sm + Q;
    float2* tmp = X + (long)NCH * Q;
    load_twiddles(twl, tw, Q);
    for (int idx = threadIdx.x; idx < nl * Q; idx += blockDim.x) {
        const int c = idx / Q, e = idx - c * Q;
        X[idx] = e < n ? Tb[((long)c * H + kx) * n + e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_channels<-1>(X, tmp, 0, nl, p.G, p.sc, twl, 2 * n <= Q);
    const __nv_bfloat16* Pk = Pp + (long)kx * NCH * nl * QR;
    for (int t = threadIdx.x; t < Q / 2; t += blockDim.x) {
        if (t == 0) {
            pc_mix_one<L>(X, Q, 0, Pk, QR, nl);
            pc_mix_one<L>(X, Q, Q / 2, Pk + Q / 2, QR, nl);
        } else {
            pc_mix_pair<L>(X, Q, t, Q - t, Pk + t, QR, nl);
        }
    }
    __syncthreads();
    fft_channels<1>(X, tmp, 0, NCH, p.G, p.sc, twl);
    for (int idx = threadIdx.x; idx < NCH * n; idx += blockDim.x) {
        const int c = idx / n, e = idx - c * n;
        Tb[((long)c * H + kx) * n + e] = X[(long)c * Q + e];
    }
}

// shared memory of k_col_pc_fused: twiddles, the NCH columns, G FFT scratch lines
static size_t pc_fused_smem(int nch, int Q, int G) { return (size_t)(Q + nch * Q + G * Q) * sizeof(float2); }

template <int L>
static cudaError_t launch_col_pc_fused(rte_plan p, float2* Tb, cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_col_pc_fused<L>)) != cudaSuccess) return e;
        once = true;
    }
    ColParams cp;
    cp.n = p->n; cp.Q = p->Q; cp.H = p->H; cp.L = L; cp.nin = 2 * L + 1;
    cp.sc = p->sched;
    cp.G = col_group<float2>(2 * L + 1, p->Q);
    k_col_pc_fused<L><<<p->H, 256, pc_fused_smem(2 * L + 1, p->Q, cp.G), s>>>(Tb, p->Pp, p->tw32, cp, p->pc_nl);
    return cudaGetLastError();
}

template <int L, int R>
static cudaError_t launch_col_pc(float2* Tb, const __nv_bfloat16* Pp, const float2* tw, int n, int H, int nl,
                                 cudaStream_t s) {
    static bool once = false;
    cudaError_t e;
    if (!once) {
        if ((e = allow_smem(k_col_warp_pc<L, R>)) != cudaSuccess) return e;
        once = true;
    }
    // the columns' spectra and two staged table slices (2 x (2L+1) rows of Q/2 + 8 BF16)
    const int Q = 32 * R;
    const size_t smem = (size_t)(2 * L + 1) * wfft_shape<R>::SCRATCH * sizeof(float2) +
                        (size_t)2 * (2 * L + 1) * (Q / 2 + 8) * sizeof(__nv_bfloat16);
    return launch_pdl(k_col_warp_pc<L, R>, dim3(H), dim3(256), smem, s, Tb, Pp, tw, n, H, nl);
}

template <int L>
static cudaError_t launch_col_pc_q(int Q, float2* Tb, float2* Tz, const __nv_bfloat16* Pp, const float2* tw, int n,
                                   int H, int nl, cudaStream_t s) {
    switch (Q) {
        case 1024: return Tz ? launch_col_pc2<L>(Tb, Tz, Pp, tw, n, H, nl, s) : cudaErrorInvalidValue;
        case 64: return launch_col_pc<L, 2>(Tb, Pp, tw, n, H, nl, s);
        case 128: return launch_col_pc<L, 4>(Tb, Pp, tw, n, H, nl, s);
        case 256: return launch_col_pc<L, 8>(Tb, Pp, tw, n, H, nl, s);
        case 512: return launch_col_pc<L, 16>(Tb, Pp, tw, n, H, nl, s);
    }
    return cudaErrorInvalidValue;
}

template <int L>
static cudaError_t build_pc2d(rte_plan p, const RowParams& rp, cudaStream_t s) {
    const long tot = (long)p->H * (p->Q / 2 + 1);
    k_build_pc2d<L><<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(p->S64, p->Pp, p->H, p->Q, rp,
                                                                  (double)p->Q * p->Q, p->pc_nl);
    return cudaGetLastError();
}

static RowParams pc_rowparams(rte_plan p, bool unit) {
    RowParams rp;
    rp.n = p->n; rp.Q = p->Q; rp.H = p->H; rp.L = p->L;
    rp.RB = 8;
    rp.sc = p->sched;
    for (int k = 0; k <= RTE_MAX_L; ++k) rp.wk[k] = 0.0;
    for (int k = 0; k <= p->L; ++k) rp.wk[k] = unit ? 1.0 : p->mu_s * p->sigma_hat[k];
    return rp;
}

// 3D: every Q.  2D: the warp column pass (Q = 64..512, 32 * 2^j), else the
// shared-memory pass while its columns fit in shared memory (Q <= 1024 at L = 8)
bool plan_precond_supported(const rte_plan p) {
    if (p->dim == 2 && p->mix_fft) return false;  // built on the direct-mix passes (L <= 8)
    if (p->dim == 3 || col_warp_ok(p->Q)) return true;
    return pc_fused_smem(p->nch, p->Q, col_group<float2>(p->nch, p->Q)) <= 200 * 1024;
}

// builds the preconditioner data once per plan (allocates; call outside any capture)
// modes the 2D preconditioner inverts: rte_opts.precond_lmax, else the
// smallest lmax with (mu_s/mu_t) max_{k > lmax} |sigma_hat_k| <= 0.03 (the
// coupling left out of the inverted block stays small)
static int pc_lmax(const rte_plan p) {
    const int L = p->L, req = p->opts.precond_lmax;
    if (req > 0) return req < L ? req : L;
    const double rho = p->mu_t > 0.0 ? p->mu_s / p->mu_t : 0.0;
    for (int l = 0; l < L; ++l) {
        double m = 0.0;
        for (int k = l + 1; k <= L; ++k) m = fmax(m, fabs(p->sigma_hat[k]));
        if (rho * m <= 0.03) return l;
    }
    return L;
}

rte_status plan_precond_build(rte_plan p, cudaStream_t s) {
    if (p->pc_ready) return RTE_OK;
    if (!plan_precond_supported(p)) return RTE_EUNSUPPORTED;
    cudaError_t e = cudaSuccess;
    if (!p->pv1 && rte_dev_malloc((void**)&p->pv1, p->nr * sizeof(float)) != cudaSuccess) return rte_fail(RTE_ENOMEM, "precond buffer");
    if (!p->pv2 && rte_dev_malloc((void**)&p->pv2, p->nr * sizeof(float)) != cudaSuccess) return rte_fail(RTE_ENOMEM, "precond buffer");
    if (p->dim == 3) {
        const long tot = (long)p->H * p->H * p->H;
        if (rte_dev_malloc((void**)&p->S3p, tot * sizeof(float)) != cudaSuccess) return rte_fail(RTE_ENOMEM, "precond spectrum");
        const double Q3 = (double)p->Q * p->Q * p->Q;
        k_build_pc3d<<<1024, 256, 0, s>>>(p->S3_64, p->S3p, tot, p->mu_s, Q3);
        e = cudaGetLastError();
    } else {
        p->pc_nl = 2 * pc_lmax(p) + 1;
        const long tot = (long)p->H * pc_row(p->Q) * p->nch * p->pc_nl;
        if (rte_dev_malloc((void**)&p->Pp, tot * sizeof(__nv_bfloat16)) != cudaSuccess) return rte_fail(RTE_ENOMEM, "precond matrices");
        if ((e = cudaMemsetAsync(p->Pp, 0, tot * sizeof(__nv_bfloat16), s)) != cudaSuccess)
            return rte_cuda_fail(e, "plan_precond_build");
        const RowParams rp = pc_rowparams(p, false);
        switch (p->L) {
            case 0: e = build_pc2d<0>(p, rp, s); break;
            case 1: e = build_pc2d<1>(p, rp, s); break;
            case 2: e = build_pc2d<2>(p, rp, s); break;
            case 3: e = build_pc2d<3>(p, rp, s); break;
            case 4: e = build_pc2d<4>(p, rp, s); break;
            case 5: e = build_pc2d<5>(p, rp, s); break;
            case 6: e = build_pc2d<6>(p, rp, s); break;
            case 7: e = build_pc2d<7>(p, rp, s); break;
            case 8: e = build_pc2d<8>(p, rp, s); break;
        }
    }
    rte_count_launches(1);
    if (e != cudaSuccess) return rte_cuda_fail(e, "plan_precond_build");
    p->pc_ready = true;
    return RTE_OK;
}

// one pass of the 2D application: 0 row, 1 column (mix with Pp), 2 inverse row;
// warp-register passes for Q = 32 * 2^j (64..512), shared-memory ones otherwise
static cudaError_t pc2d_pass(rte_plan p, int st, const float* x, float* out, cudaStream_t s) {
    RowParams rp = pc_rowparams(p, true);
    float2* Tb = (float2*)p->T32;
    const bool warp = col_warp_ok(p->Q);
    if (st == 0 || st == 2) {
        // forward: the inverted modes 0..lmax; inverse: every mode, out = x + v
        const int lmax = (p->pc_nl - 1) / 2;
        if (row_warp_ok(p->Q)) {
            const dim3 grid((p->n + 7) / 8, st == 0 ? lmax + 1 : p->L + 1);
            if (st == 0) return row_fwd_warp<float2, float2>(p->Q, grid, (const float2*)x, nullptr, Tb, p->tw32, rp, s);
            return row_inv_warp<float2, float2>(p->Q, grid, Tb, (const float2*)x, nullptr, (float2*)out, p->tw32, rp,
                                                1.f, 1.f, 0.f, s);
        }
        static bool once = false;
        cudaError_t e;
        if (!once) {
            if ((e = allow_smem(k_row_fwd<float2, float2>)) != cudaSuccess) return e;
            if ((e = allow_smem(k_row_inv<float2, float2>)) != cudaSuccess) return e;
            once = true;
        }
        rp.RB = rows_per_block<float2>(p->Q);
        const dim3 grid((p->n + rp.RB - 1) / rp.RB, st == 0 ? lmax + 1 : p->L + 1);
        const size_t smr = row_smem<float2>(p->Q, rp.RB);
        if (st == 0) k_row_fwd<float2, float2><<<grid, 256, smr, s>>>((const float2*)x, nullptr, Tb, p->tw32, rp);
        else k_row_inv<float2, float2><<<grid, 256, smr, s>>>(Tb, (const float2*)x, nullptr, (float2*)out, p->tw32, rp,
                                                              1.f, 1.f, 0.f);
        return cudaGetLastError();
    }
    if (!warp) {
        switch (p->L) {
            case 0: return launch_col_pc_fused<0>(p, Tb, s);
            case 1: return launch_col_pc_fused<1>(p, Tb, s);
            case 2: return launch_col_pc_fused<2>(p, Tb, s);
            case 3: return launch_col_pc_fused<3>(p, Tb, s);
            case 4: return launch_col_pc_fused<4>(p, Tb, s);
            case 5: return launch_col_pc_fused<5>(p, Tb, s);
            case 6: return launch_col_pc_fused<6>(p, Tb, s);
            case 7: return launch_col_pc_fused<7>(p, Tb, s);
            case 8: return launch_col_pc_fused<8>(p, Tb, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (p->L) {
        case 0: return launch_col_pc_q<0>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 1: return launch_col_pc_q<1>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 2: return launch_col_pc_q<2>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 3: return launch_col_pc_q<3>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 4: return launch_col_pc_q<4>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 5: return launch_col_pc_q<5>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 6: return launch_col_pc_q<6>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 7: return launch_col_pc_q<7>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
        case 8: return launch_col_pc_q<8>(p->Q, Tb, p->Tz32, p->Pp, p->tw32, p->n, p->H, p->pc_nl, s);
    }
    return cudaErrorInvalidValue;
}

// out = M x (FP32 fields, the plan's FP32 layout); the plan's pass buffers
rte_status plan_apply_pc32(rte_plan p, const float* x, float* out, cudaStream_t s) {
    if (!p->pc_ready) return RTE_EINVAL;
    cudaError_t e = cudaSuccess;
    if (p->dim == 3) {
        e = op3d_run_pc32(p, x, out, s);
    } else {
        for (int st = 0; st < 3 && e == cudaSuccess; ++st) e = pc2d_pass(p, st, x, out, s);
        rte_count_launches(3);
    }
    if (e != cudaSuccess) return rte_cuda_fail(e, "plan_apply_pc32");
    return RTE_OK;
}

// one preconditioned inner step: pv = M v, w = A pv = pv - K pv.  With the
// warp row passes (2D, Q <= 512) M's inverse row pass and K's forward row
// pass run as one kernel (k_row_invfwd_warp); otherwise M and A one after
// the other.
rte_status plan_apply_pcA32(rte_plan p, const float* v, float* pv, float* w, cudaStream_t s) {
    if (!p->pc_ready) return RTE_EINVAL;
    if (p->dim == 2 && row_warp_ok(p->Q) && p->Q <= 512 && p->rb_force < 2) {
        cudaError_t e = pc2d_pass(p, 0, v, pv, s);
        if (e == cudaSuccess) e = pc2d_pass(p, 1, v, pv, s);
        if (e == cudaSuccess) {
            RowParams rp = pc_rowparams(p, false);  // K's input weights mu_s sigma_hat_k
            const dim3 grid((p->n + 7) / 8, p->L + 1);
            e = row_invfwd_warp(p->Q, grid, (float2*)p->T32, (const float2*)v, (float2*)pv, p->tw32, rp, s);
        }
        rte_count_launches(3);
        if (e != cudaSuccess) return rte_cuda_fail(e, "plan_apply_pcA32");
        rte_status st = op2d_apply32_stage(p, pv, w, 1.0f, -1.0f, 0.0f, 1, s);
        if (st == RTE_OK) st = op2d_apply32_stage(p, pv, w, 1.0f, -1.0f, 0.0f, 2, s);
        return st;
    }
    rte_status st = plan_apply_pc32(p, v, pv, s);
    if (st == RTE_OK) st = plan_apply32(p, pv, w, 1.0f, -1.0f, 0.0f, nullptr, s);
    return st;
}

// average ms of each 2D pass over reps back-to-back launches (plan scratch)
rte_status plan_time_pc(rte_plan p, int reps, double* ms, cudaStream_t s) {
    if (p->dim != 2) return RTE_EUNSUPPORTED;
    rte_status st0 = plan_precond_build(p, s);
    if (st0 != RTE_OK) return st0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return rte_fail(RTE_ECUDA, "plan_time_pc");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return rte_fail(RTE_ECUDA, "plan_time_pc");
    }
    cudaError_t e = cudaSuccess;
    for (int st = 0; st < 3 && e == cudaSuccess; ++st) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = pc2d_pass(p, st, p->pv1, p->pv2, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms[st] = t / reps;
    }
    rte_count_launches(3L * reps);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return rte_cuda_fail(e, "plan_time_pc");
    return RTE_OK;
}
