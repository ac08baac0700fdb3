// Learned initial guess for the GMRES solve (task extension; the paper has
// no counterpart): a small 3x3 convolutional network, NHWC BF16 activations,
// FP32 accumulation on the BF16 tensor cores, trained on the GPU by its own
// forward / data-gradient / weight-gradient kernels and Adam.  All three
// convolution products run on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in TMEM): k_conv_tc (forward and data gradient, K-major
// operands) and k_conv_wgrad_tc (weight gradient, M/N-major operands).
//
// Layer l: Y = act(conv3x3(X, W_l) + bias_l), same padding (zeros outside the
// image), channel counts padded to multiples of 16.  Weights W_l[tap][cin][cout]
// (tap = 3*(dy+1) + (dx+1)); a master FP32 copy is updated by Adam, the BF16
// copy feeds the kernels.
//
// Implicit GEMM: rows = output pixels (a run of 128 along x in one image row),
// columns = output channels, reduction = 9 taps x input channels.  The
// data gradient is the same product with the taps mirrored and W transposed;
// the weight gradient reduces over pixels: dW[tap][ci][co] = sum_p
// X[p + d(tap)][ci] dY[p][co], written as per-block partial sums and reduced
// in a fixed order.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "internal.h"
#include "tc05.cuh"

typedef __nv_bfloat16 bf16;

#define CNN_TILE 128       // pixels per block (along x)



// ---------------------------------------------------------------------------
// forward / data-gradient convolution on tcgen05 tensor cores
//   out[p][n] = sum_tap sum_c X[p + s d(tap)][c] Wk[tap][n][c]
//   s = +1 (forward, Wk[tap][co][ci]: the weights transposed) or -1 (data
//   gradient dX[q] = sum_tap dY[q - d(tap)] W[tap]^T, Wk = W[tap][ci][co])
// One CTA: a run of 128 output pixels along x (the MMA's M = 128 rows, one
// TMEM lane each) by all NOUT output channels (N), reduced over the 9 taps x
// CX input channels (K, 16 per MMA).  The three input rows y-1, y, y+1 over
// pixels x0-1 .. x0+128 (zeros outside the image) are staged once, per row
// and 16-byte channel chunk as a run of 130 pixels of 16 bytes: in that
// layout the operand of tap (dy, dx) is the same core-matrix view started
// dx + 1 pixels (16 bytes) further in row dy + 1 (core matrices of 8
// consecutive pixels: row-group stride 128 bytes, K-chunk stride 130 x 16),
// so all 9 taps read one staged tile.  The tap's weights (N x CX, K-major
// core matrices) are double-buffered: while one thread issues a tap's MMAs,
// the CTA stages the next tap's weights; an mbarrier signalled by
// tcgen05.commit frees a buffer.  Epilogue: tcgen05.ld of the FP32
// accumulators, bias, ReLU, BF16 (or FP32) NHWC store.  (Staging all 9
// taps' weights up front instead measured 1.7x slower: the larger shared
// memory leaves one CTA per SM, so loads and MMAs no longer overlap.)
// X: [B][H][Wd][CX] bf16; out: [B][H][Wd][NOUT]; grid (ceil(Wd/128), H, B), 128 threads.
// ---------------------------------------------------------------------------
#define CONV_TC_PX 130   // staged pixels per row: 128 + the two halo pixels
template <int CX, int NOUT> struct ConvTc {
    static constexpr int KC = CX / 8;                          // 16-byte channel chunks
    static constexpr int IN_BYTES = 3 * KC * CONV_TC_PX * 16;  // the three staged input rows
    static constexpr int W_BYTES = NOUT * CX * 2;              // one tap's weights
    static constexpr int NCOLS = NOUT < 32 ? 32 : NOUT;        // TMEM columns (a power of two >= 32)
    // at most 512 / NCOLS CTAs may hold TMEM on an SM at once: pad the shared
    // memory so that no more are resident (228 KB per SM)
    static constexpr int PAD = 233472 / (512 / NCOLS + 1) + 1;
    static constexpr int NEED = IN_BYTES + 2 * W_BYTES + 1024;  // + alignment slack
    static constexpr int SMEM = NEED > PAD ? NEED : PAD;
};
#define CONV_TC_POLLS (1L << 20)  // polls before an mbarrier wait gives up (error flag) instead of hanging

template <int CX, int NOUT>
__device__ __forceinline__ void conv_tc_stage_w(uint8_t* Wb, const bf16* __restrict__ Wk, int tap, int tid) {
    constexpr int KC = CX / 8;
    const bf16* wt = Wk + (long)tap * NOUT * CX;
    for (int c = tid; c < NOUT * KC; c += 128) {
        const int nr = c / KC, kc = c - nr * KC;
        cp_async16(Wb + ((nr >> 3) * KC + kc) * 128 + (nr & 7) * 16, wt + (long)nr * CX + kc * 8, 16);
    }
    cp_async_wait_all();
}

template <int CX, int NOUT>
__global__ void __launch_bounds__(128) k_conv_tc(const bf16* __restrict__ X, const bf16* __restrict__ Wk, int flip,
                                                 const float* __restrict__ bias, int relu, bf16* __restrict__ Ybf,
                                                 float* __restrict__ Yf, int H, int Wd, int* __restrict__ err) {
    using C = ConvTc<CX, NOUT>;
    constexpr int KC = C::KC;
    constexpr uint32_t LBO = CONV_TC_PX * 16;  // next 16-byte channel chunk of a staged row
    extern __shared__ uint8_t smraw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tslot;
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    uint8_t* In = sbase;                 // [3 rows][KC][130 pixels][16 bytes]
    uint8_t* Wbuf = sbase + C::IN_BYTES;  // 2 x [N/8][KC][8][16 bytes]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * 128, y = blockIdx.y, b = blockIdx.z;
    if (warp == 0) tc_alloc(&tslot, C::NCOLS);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    // the input rows (consecutive threads: consecutive 16-byte chunks of a pixel, then pixels)
    // (asynchronous 16-byte copies, zero-filled outside the image: all of a
    // thread's copies are in flight at once)
    for (int c = tid; c < 3 * CONV_TC_PX * KC; c += 128) {
        const int kc = c % KC, px = (c / KC) % CONV_TC_PX, r = c / (KC * CONV_TC_PX);
        const int yy = y + r - 1, xx = x0 + px - 1;
        const bool in = yy >= 0 && yy < H && xx >= 0 && xx < Wd;
        const bf16* src = in ? X + (((long)b * H + yy) * Wd + xx) * CX + kc * 8 : X;
        cp_async16(In + ((r * KC + kc) * CONV_TC_PX + px) * 16, src, in ? 16u : 0u);
    }
    conv_tc_stage_w<CX, NOUT>(Wbuf, Wk, 0, tid);  // waits for all of this thread's copies
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, NOUT);
    const int sgn = flip ? -1 : 1;
    const uint32_t in0 = smem_u32(In), w0 = smem_u32(Wbuf);
    bool ok = true;
    for (int tap = 0; tap < 9; ++tap) {
        const int st = tap & 1;
        if (tid == 0) {
            tc_fence_after();
            const int dy = sgn * (tap / 3 - 1), dx = sgn * (tap % 3 - 1);
            // output pixel m reads staged pixel m + dx + 1 of staged row dy + 1
            const uint32_t a0 = in0 + (uint32_t)(((dy + 1) * KC) * CONV_TC_PX + dx + 1) * 16;
            const uint32_t b0 = w0 + st * C::W_BYTES;
#pragma unroll
            for (int ks = 0; ks < CX / 16; ++ks) {
                // K = 16 = two 16-byte channel chunks per step
                const uint64_t ad = tc_desc_kmajor(a0 + ks * 2 * LBO, LBO, 128);
                const uint64_t bd = tc_desc_kmajor(b0 + ks * 256, 128, KC * 128);
                tc_mma_bf16(tmem, ad, bd, IDESC, (tap | ks) ? 1u : 0u);
            }
            tc_commit(&mbar[st]);
        }
        if (tap + 1 < 9) {
            // the next tap's weights go to the other buffer, last read by the
            // MMAs of tap - 1: one thread waits for their commit, the barrier
            // passes the outcome to all (uniform control flow)
            if (tap >= 1) {
                int bad = 0;
                if (tid == 0) bad = !mbar_wait(&mbar[st ^ 1], ((tap - 1) >> 1) & 1, CONV_TC_POLLS);
                if (__syncthreads_or(bad)) {
                    ok = false;
                    break;
                }
            }
            fence_async_smem();
            conv_tc_stage_w<CX, NOUT>(Wbuf + (st ^ 1) * C::W_BYTES, Wk, tap + 1, tid);
            fence_async_smem();
            __syncthreads();
        }
    }
    // the last commit (tap 8: buffer 0, fifth phase, parity 0) covers every
    // MMA; buffer 1's fourth arrival (tap 7, parity 1) is waited for too so
    // that no arrival is pending when the CTA exits
    {
        int bad = 0;
        if (tid == 0) bad = !mbar_wait(&mbar[0], 0, CONV_TC_POLLS) || !mbar_wait(&mbar[1], 1, CONV_TC_POLLS);
        if (__syncthreads_or(bad)) ok = false;
    }
    tc_fence_after();
    float acc[NOUT];
#pragma unroll
    for (int c0 = 0; c0 < NOUT; c0 += 16) tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc + c0);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, C::NCOLS);
    if (!ok) {
        if (lane == 0) atomicExch(err, 1);
        return;
    }
    const int px = x0 + warp * 32 + lane;
    if (px >= Wd) return;
    const long o = (((long)b * H + y) * Wd + px) * NOUT;
#pragma unroll
    for (int n = 0; n < NOUT; ++n) {
        float v = acc[n];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
        acc[n] = v;
    }
    if (Yf) {
#pragma unroll
        for (int n = 0; n < NOUT; n += 4)
            *reinterpret_cast<float4*>(Yf + o + n) = make_float4(acc[n], acc[n + 1], acc[n + 2], acc[n + 3]);
    } else {
#pragma unroll
        for (int n = 0; n < NOUT; n += 8) {
            __nv_bfloat162 h[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(acc[n + 2 * q], acc[n + 2 * q + 1]);
            *reinterpret_cast<uint4*>(Ybf + o + n) = *reinterpret_cast<const uint4*>(h);
        }
    }
}

// ---------------------------------------------------------------------------
// weight gradient on tcgen05: dW[tap][ci][co] = sum_p X[p + d(tap)][ci] dY[p][co]
// GEMM with M = (tap row, ci), N = co, K = pixels.  Both operands are
// M/N-major in their natural NHWC order (for a pixel, the channels are
// contiguous), staged like the forward's input tile: per channel chunk a run
// of pixels at a 16-byte stride.  RST = 128 / CI consecutive staged input rows
// form one M = 128 operand (the row stride of the staged tile is KC x 130 x 16
// bytes = KC x the chunk stride, so M blocks run on through the next row); G
// such groups cover the rows y - 1, y, y + 1 (staged rows beyond y + 1 are
// zeros and their results are dropped); the three x shifts dx are three start
// addresses.  So one CTA holds 3 G accumulators of 128 x CO in TMEM and, for
// each 128-pixel tile of its share, issues 3 G x 8 MMAs (K = 16 pixels each),
// with the next tile's staging (cp.async) overlapping them (two stages, an
// mbarrier per stage signalled by tcgen05.commit).  Partial sums per CTA go to
// part[cta][tap][ci][co] (reduced in a fixed order by k_reduce_parts).
// grid: CTAs over the B x H x ceil(W/128) tiles, 128 threads.
// ---------------------------------------------------------------------------
template <int CI, int CO> struct WgTc {
    static constexpr int KCI = CI / 8, KCO = CO / 8;
    static constexpr int RST = 128 / CI;             // staged rows per M = 128 group
    static constexpr int G = (3 + RST - 1) / RST;    // groups covering dy = -1, 0, 1
    static constexpr int S = G * RST;                // staged input rows
    static constexpr int X_BYTES = S * KCI * CONV_TC_PX * 16;
    static constexpr int Y_BYTES = KCO * 128 * 16;
    static constexpr int STAGE = X_BYTES + Y_BYTES;
    static constexpr int NACC = 3 * G;
    static constexpr int NCOLS = NACC * CO <= 32 ? 32 : NACC * CO <= 64 ? 64 : NACC * CO <= 128 ? 128
                                 : NACC * CO <= 256 ? 256 : 512;
    static constexpr int PAD = 233472 / (512 / NCOLS + 1) + 1;  // no more resident CTAs than TMEM allows
    static constexpr int NEED = 2 * STAGE + 1024;
    static constexpr int SMEM = NEED > PAD ? NEED : PAD;
};

template <int CI, int CO>
__global__ void __launch_bounds__(128) k_conv_wgrad_tc(const bf16* __restrict__ X, const bf16* __restrict__ dY,
                                                       float* __restrict__ part, int B, int H, int Wd,
                                                       int* __restrict__ err) {
    using C = WgTc<CI, CO>;
    constexpr int KCI = C::KCI, KCO = C::KCO;
    extern __shared__ uint8_t smraw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tslot;
    uint8_t* sbase = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int xt_n = (Wd + 127) / 128;
    const long ntiles = (long)B * H * xt_n;
    if (warp == 0) tc_alloc(&tslot, C::NCOLS);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    constexpr uint32_t IDESC = tc_idesc_bf16(128, CO, true);
    bool ok = true;
    int i = 0;  // local tile count
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int st = i & 1;
        uint8_t* Xs = sbase + st * C::STAGE;
        uint8_t* Ys = Xs + C::X_BYTES;
        if (i >= 2) {
            int bad = 0;
            if (tid == 0) bad = !mbar_wait(&mbar[st], ((i - 2) >> 1) & 1, CONV_TC_POLLS);
            if (__syncthreads_or(bad)) {
                ok = false;
                break;
            }
        }
        fence_async_smem();
        const int xt = (int)(t % xt_n);
        const long by = t / xt_n;
        const int y = (int)(by % H), b = (int)(by / H);
        const int x0 = xt * 128;
        // input rows y - 1 .. y - 1 + S - 1 (those past y + 1 are not needed: zeros)
        for (int c = tid; c < C::S * CONV_TC_PX * KCI; c += 128) {
            const int kc = c % KCI, px = (c / KCI) % CONV_TC_PX, r = c / (KCI * CONV_TC_PX);
            const int yy = y + r - 1, xx = x0 + px - 1;
            const bool in = r < 3 && yy >= 0 && yy < H && xx >= 0 && xx < Wd;
            const bf16* src = in ? X + (((long)b * H + yy) * Wd + xx) * CI + kc * 8 : X;
            cp_async16(Xs + ((r * KCI + kc) * CONV_TC_PX + px) * 16, src, in ? 16u : 0u);
        }
        // output-gradient row y, pixels x0 .. x0 + 127
        for (int c = tid; c < 128 * KCO; c += 128) {
            const int kc = c % KCO, px = c / KCO;
            const int xx = x0 + px;
            const bool in = xx < Wd;
            const bf16* src = in ? dY + (((long)b * H + y) * Wd + xx) * CO + kc * 8 : dY;
            cp_async16(Ys + (kc * 128 + px) * 16, src, in ? 16u : 0u);
        }
        cp_async_wait_all();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t xa = smem_u32(Xs), ya = smem_u32(Ys);
#pragma unroll
            for (int g = 0; g < C::G; ++g)
#pragma unroll
                for (int dxi = 0; dxi < 3; ++dxi) {
                    const uint32_t acc = tmem + (uint32_t)((g * 3 + dxi) * CO);
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        // A: M blocks = channel chunks (then the next staged row) at 130 x 16 bytes,
                        // K blocks = 8 pixels at 128 bytes; staged pixel p + dx + 1 for pixel p
                        const uint64_t ad = tc_desc_kmajor(
                            xa + (uint32_t)((g * C::RST * KCI) * CONV_TC_PX + 16 * ks + dxi) * 16, 128,
                            CONV_TC_PX * 16);
                        // B: N blocks = channel chunks at 128 x 16 bytes, K blocks at 128 bytes
                        const uint64_t bd = tc_desc_kmajor(ya + (uint32_t)(16 * ks) * 16, 128, 128 * 16);
                        tc_mma_bf16(acc, ad, bd, IDESC, (i > 0 || ks > 0) ? 1u : 0u);
                    }
                }
            tc_commit(&mbar[st]);
        }
    }
    // wait for the last tile's commit (it covers every MMA) and for the other
    // stage's last arrival, so that none is pending at exit
    if (i > 0) {
        int bad = 0;
        if (tid == 0) {
            const int il = i - 1;
            bad = !mbar_wait(&mbar[il & 1], (il >> 1) & 1, CONV_TC_POLLS);
            if (!bad && il >= 1) bad = !mbar_wait(&mbar[(il - 1) & 1], ((il - 1) >> 1) & 1, CONV_TC_POLLS);
        }
        if (__syncthreads_or(bad)) ok = false;
    }
    tc_fence_after();
    // epilogue: TMEM lane m = 32 warp + lane is row (r_local = m / CI, ci = m % CI)
    const int m = warp * 32 + lane;
    const int rl = m / CI, ci = m % CI;
    for (int g = 0; g < C::G; ++g) {
        const int dy = g * C::RST + rl - 1;
        for (int dxi = 0; dxi < 3; ++dxi) {
            float v[CO];
#pragma unroll
            for (int c0 = 0; c0 < CO; c0 += 16)
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((g * 3 + dxi) * CO + c0), v + c0);
            if (ok && i > 0 && dy >= -1 && dy <= 1) {
                const int tap = (dy + 1) * 3 + dxi;
                float* dst = part + (((long)blockIdx.x * 9 + tap) * CI + ci) * CO;
#pragma unroll
                for (int co = 0; co < CO; co += 4) *reinterpret_cast<float4*>(dst + co) = make_float4(v[co], v[co + 1], v[co + 2], v[co + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, C::NCOLS);
    if (!ok && lane == 0) atomicExch(err, 1);
}

// dW[i] = sum_b part[b][i] (fixed order), i < 9*CI*CO
__global__ void k_reduce_parts(const float* __restrict__ part, int nblk, long per, float* __restrict__ dW) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += (long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += part[(long)b * per + i];
        dW[i] = s;
    }
}

// bias gradient: db[c] = sum_p dY[p][c]; one block per channel
__global__ void k_bias_grad(const bf16* __restrict__ dY, long P, int C, float* __restrict__ db) {
    const int c = blockIdx.x;
    __shared__ float red[256];
    float s = 0.f;
    for (long p = threadIdx.x; p < P; p += blockDim.x) s += __bfloat162float(dY[p * C + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] = red[0];
}

// dY *= (Y > 0)
__global__ void k_relu_bwd(bf16* __restrict__ dY, const bf16* __restrict__ Y, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(Y[i]) > 0.f)) dY[i] = __float2bfloat16(0.f);
}

// mean squared error over the first `used` of C channels; dOut = d loss / d out (bf16)
__global__ void k_mse(const float* __restrict__ out, const bf16* __restrict__ tgt, long P, int C, int used,
                      bf16* __restrict__ dOut, float* __restrict__ loss_part) {
    __shared__ float red[256];
    const double inv = 1.0 / ((double)P * used);
    float s = 0.f;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P * C; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        float d = 0.f;
        if (c < used) {
            d = out[i] - __bfloat162float(tgt[i]);
            s += d * d;
        }
        dOut[i] = __float2bfloat16((float)(2.0 * inv) * d);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = (float)(red[0] * inv);
}

// Adam (Kingma & Ba) on FP32 master weights; BF16 copy refreshed
// (weights [9][ci][co]: wbt, when given, receives the transposed copy [9][co][ci])
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       bf16* __restrict__ wb, bf16* __restrict__ wbt, int ci_n, int co_n, long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
        if (wbt) {
            const long co = i % co_n, ci = (i / co_n) % ci_n, tap = i / ((long)co_n * ci_n);
            wbt[(tap * co_n + co) * ci_n + ci] = __float2bfloat16(wi);
        }
    }
}

// BF16 copies of the FP32 weights [9][ci][co]: wb in place, wbt transposed [9][co][ci]
__global__ void k_to_bf16(const float* __restrict__ a, bf16* __restrict__ b, bf16* __restrict__ bt, int ci_n, int co_n,
                          long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const bf16 v = __float2bfloat16(a[i]);
        b[i] = v;
        const long co = i % co_n, ci = (i / co_n) % ci_n, tap = i / ((long)co_n * ci_n);
        bt[(tap * co_n + co) * ci_n + ci] = v;
    }
}

// deterministic weight init: uniform(-a, a) from a counter hash (splitmix64)
__global__ void k_init_uniform(float* __restrict__ w, long n, unsigned long long seed, float a) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float u = (float)((z >> 40) * (1.0 / 16777216.0));
        w[i] = (2.f * u - 1.f) * a;
    }
}

// ---------------------------------------------------------------------------
// features and output mapping for the RTE solve (2D mode fields, L <= 7)
//   channels: b_c / s (2L+1 real channels of b = K~ g), f / fmax, log(mu_t)/4,
//   mu_s/mu_t, g, zeros to CIN
//   u0 = b + s * net_c  (first 2L+1 output channels)
// ---------------------------------------------------------------------------
// sc[0] = RMS of the 2L+1 real channels of b, sc[1] = max |f|  (one block)
__global__ void k_guess_scales(const double* __restrict__ bmode, const double* __restrict__ f, int n, int L,
                               double* __restrict__ sc) {
    __shared__ double r1[1024], r2[1024];
    const long P = (long)n * n;
    const long nb = 2L * (L + 1) * P;
    double s = 0.0, m = 0.0;
    for (long i = threadIdx.x; i < nb; i += blockDim.x) s += bmode[i] * bmode[i];
    for (long i = threadIdx.x; i < P; i += blockDim.x) m = fmax(m, fabs(f[i]));
    r1[threadIdx.x] = s;
    r2[threadIdx.x] = m;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            r1[threadIdx.x] += r1[threadIdx.x + k];
            r2[threadIdx.x] = fmax(r2[threadIdx.x], r2[threadIdx.x + k]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc[0] = sqrt(r1[0] / ((2.0 * L + 1.0) * P));
        sc[1] = r2[0];
    }
}

__global__ void k_features(const double* __restrict__ bmode, const double* __restrict__ f, int n, int L,
                           const double* __restrict__ sc, float p0, float p1, float p2, int CIN, bf16* __restrict__ X) {
    const long P = (long)n * n;
    const double s_b = sc[0], fmax = sc[1];
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
        bf16* xp = X + p * CIN;
        int c = 0;
        const double inv = s_b > 0 ? 1.0 / s_b : 0.0;
        xp[c++] = __float2bfloat16((float)(bmode[2 * p] * inv));
        for (int k = 1; k <= L; ++k) {
            xp[c++] = __float2bfloat16((float)(bmode[2 * (k * P + p)] * inv));
            xp[c++] = __float2bfloat16((float)(bmode[2 * (k * P + p) + 1] * inv));
        }
        xp[c++] = __float2bfloat16((float)(fmax > 0 ? f[p] / fmax : 0.0));
        xp[c++] = __float2bfloat16(p0);
        xp[c++] = __float2bfloat16(p1);
        xp[c++] = __float2bfloat16(p2);
        while (c < CIN) xp[c++] = __float2bfloat16(0.f);
    }
}

// multi-scale context (inputs with room for it, CIN >= 3 (2L+1) + 4): the
// means of the 2L+1 scaled channels of b over the 8 x 8 and the 32 x 32 tile
// that contain the pixel, in channels 2L+5 + c and 2L+5 + (2L+1) + c.  A 3x3
// network sees 13 cells; these give every pixel the field's coarse shape
// over 32 (resp. 128) cells around it at no extra layers.  One CTA per 32 x 32
// tile (partial tiles at the border average their own cells).
__global__ void __launch_bounds__(256) k_features_pooled(const double* __restrict__ bmode, int n, int L,
                                                         const double* __restrict__ sc, int CIN, bf16* __restrict__ X) {
    __shared__ float s8[16][2 * RTE_MAX_L_DIRECT + 1];
    __shared__ float s32[2 * RTE_MAX_L_DIRECT + 1];
    const long P = (long)n * n;
    const int nch = 2 * L + 1;
    const int tx0 = blockIdx.x * 32, ty0 = blockIdx.y * 32;
    const double inv = sc[0] > 0 ? 1.0 / sc[0] : 0.0;
    // channel c, sub-tile q (4 x 4 of 8 x 8 cells): one thread each, summing its cells
    for (int job = threadIdx.x; job < 16 * nch; job += blockDim.x) {
        const int c = job / 16, q = job % 16;
        const int k = c == 0 ? 0 : (c + 1) / 2, im = c > 0 && (c % 2 == 0);
        const int x0 = tx0 + (q % 4) * 8, y0 = ty0 + (q / 4) * 8;
        double sum = 0.0;
        int cnt = 0;
        for (int yy = y0; yy < y0 + 8 && yy < n; ++yy)
            for (int xx = x0; xx < x0 + 8 && xx < n; ++xx) {
                sum += bmode[2 * (k * P + (long)yy * n + xx) + im];
                ++cnt;
            }
        s8[q][c] = cnt ? (float)(sum * inv / cnt) : 0.f;
    }
    __syncthreads();
    if (threadIdx.x < nch) {
        const int c = threadIdx.x;
        double sum = 0.0;
        int cnt = 0;
        for (int q = 0; q < 16; ++q) {
            const int x0 = tx0 + (q % 4) * 8, y0 = ty0 + (q / 4) * 8;
            const int wq = max(0, min(8, n - x0)) * max(0, min(8, n - y0));
            sum += (double)s8[q][c] * wq;
            cnt += wq;
        }
        s32[c] = cnt ? (float)(sum / cnt) : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
        const int xx = tx0 + (i % 32), yy = ty0 + (i / 32);
        if (xx >= n || yy >= n) continue;
        const int q = ((i / 32) / 8) * 4 + (i % 32) / 8;
        bf16* xp = X + ((long)yy * n + xx) * CIN + nch + 4;
        for (int c = 0; c < nch; ++c) {
            xp[c] = __float2bfloat16(s8[q][c]);
            xp[nch + c] = __float2bfloat16(s32[c]);
        }
    }
}

__global__ void k_targets(const double* __restrict__ umode, const double* __restrict__ bmode, int n, int L,
                          const double* __restrict__ sc, int COUT, bf16* __restrict__ Yt) {
    const long P = (long)n * n;
    const double s_b = sc[0];
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
        bf16* yp = Yt + p * COUT;
        int c = 0;
        const double inv = s_b > 0 ? 1.0 / s_b : 0.0;
        yp[c++] = __float2bfloat16((float)((umode[2 * p] - bmode[2 * p]) * inv));
        for (int k = 1; k <= L; ++k) {
            const long o = 2 * (k * P + p);
            yp[c++] = __float2bfloat16((float)((umode[o] - bmode[o]) * inv));
            yp[c++] = __float2bfloat16((float)((umode[o + 1] - bmode[o + 1]) * inv));
        }
        while (c < COUT) yp[c++] = __float2bfloat16(0.f);
    }
}

__global__ void k_guess_out(const float* __restrict__ net, const double* __restrict__ bmode, int n, int L,
                            const double* __restrict__ sc, int COUT, double* __restrict__ u0) {
    const long P = (long)n * n;
    const double s_b = sc[0];
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
        const float* np = net + p * COUT;
        u0[2 * p] = bmode[2 * p] + s_b * np[0];
        u0[2 * p + 1] = 0.0;
        int c = 1;
        for (int k = 1; k <= L; ++k) {
            const long o = 2 * (k * P + p);
            u0[o] = bmode[o] + s_b * np[c++];
            u0[o + 1] = bmode[o + 1] + s_b * np[c++];
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct CnnLayer {
    int cin, cout;   // padded channel counts
    float* w = nullptr;
    float* bias = nullptr;
    bf16* wb = nullptr;    // BF16 copy [9][cin][cout]
    bf16* wbt = nullptr;   // BF16 copy transposed [9][cout][cin] (forward MMA operand)
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr, *gw = nullptr, *gb = nullptr;
};

struct rte_cnn_s {
    int cin = 16, width = 64, depth = 6, cout = 16;
    std::vector<CnnLayer> layers;
    // activations for the current batch shape
    int B = 0, H = 0, W = 0;
    std::vector<bf16*> act;    // act[0] = input, act[l+1] = output of layer l (bf16), last layer f32 in out_f
    float* out_f = nullptr;
    bf16* g0 = nullptr;        // gradient buffers (ping-pong), size P * max(width, cin, cout)
    bf16* g1 = nullptr;
    float* part = nullptr;     // weight-gradient partials
    long part_cap = 0;
    float* loss_part = nullptr;
    float* loss_host = nullptr;
    int* err = nullptr;        // set by a tensor-core convolution whose barrier wait gave up
    int nsm = 152;             // SMs of the device (the weight gradient's CTA count)
    long step = 0;
};

static int nblk_pix(int B, int H) {
    long rows = (long)B * H;
    int rpb = 16;
    return (int)((rows + rpb - 1) / rpb);
}

template <int CX, int NOUT>
static cudaError_t launch_conv_tc(dim3 grid, const bf16* X, const bf16* Wk, int flip, const float* bias, int relu,
                                  bf16* Ybf, float* Yf, int H, int W, int* err, cudaStream_t s) {
    using C = ConvTc<CX, NOUT>;
    static bool once = false;
    if (!once) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CX, NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return e;
        once = true;
    }
    k_conv_tc<CX, NOUT><<<grid, 128, C::SMEM, s>>>(X, Wk, flip, bias, relu, Ybf, Yf, H, W, err);
    return cudaGetLastError();
}

// CX, NOUT in {16, 32, 64}
static cudaError_t conv_tc(int CX, int NOUT, const bf16* X, const bf16* Wk, int flip, const float* bias, int relu,
                           bf16* Ybf, float* Yf, int B, int H, int W, int* err, cudaStream_t s) {
    const dim3 grid((W + CNN_TILE - 1) / CNN_TILE, H, B);
#define CONV_TC_CASE(a, b) \
    if (CX == a && NOUT == b) return launch_conv_tc<a, b>(grid, X, Wk, flip, bias, relu, Ybf, Yf, H, W, err, s);
    CONV_TC_CASE(16, 16) CONV_TC_CASE(16, 32) CONV_TC_CASE(16, 64)
    CONV_TC_CASE(32, 16) CONV_TC_CASE(32, 32) CONV_TC_CASE(32, 64)
    CONV_TC_CASE(64, 16) CONV_TC_CASE(64, 32) CONV_TC_CASE(64, 64)
#undef CONV_TC_CASE
    return cudaErrorInvalidValue;
}

// Y[p][co] = act(sum_tap sum_ci X[p + d(tap)][ci] W[tap][ci][co] + bias[co]),
// the weights read transposed (wbt[tap][co][ci]: K-major for the MMA)
static cudaError_t conv_fwd(const bf16* X, const CnnLayer& Lr, bool relu, bf16* Ybf, float* Yf, int B, int H, int W,
                            int* err, cudaStream_t s) {
    rte_count_launches(1);
    return conv_tc(Lr.cin, Lr.cout, X, Lr.wbt, 0, Lr.bias, relu, Ybf, Yf, B, H, W, err, s);
}

// dX[p][ci] = sum_tap sum_co dY[p - d(tap)][co] W[tap][ci][co]  (W[tap] is K-major in co)
static cudaError_t conv_dgrad(const bf16* dY, const CnnLayer& Lr, bf16* dX, int B, int H, int W, int* err,
                              cudaStream_t s) {
    rte_count_launches(1);
    return conv_tc(Lr.cout, Lr.cin, dY, Lr.wb, 1, nullptr, 0, dX, nullptr, B, H, W, err, s);
}

template <int CI, int CO>
static cudaError_t launch_wgrad_tc(int nb, const bf16* X, const bf16* dY, float* part, int B, int H, int W, int* err,
                                   cudaStream_t s) {
    using C = WgTc<CI, CO>;
    static bool once = false;
    if (!once) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad_tc<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::SMEM);
        if (e != cudaSuccess) return e;
        once = true;
    }
    k_conv_wgrad_tc<CI, CO><<<nb, 128, C::SMEM, s>>>(X, dY, part, B, H, W, err);
    return cudaGetLastError();
}

// dW = sum over pixels of X[p + d(tap)] dY[p]^T on tcgen05 (k_conv_wgrad_tc),
// one CTA per SM at most (partials reduced in a fixed order)
static cudaError_t conv_wgrad(rte_cnn c, const bf16* X, const bf16* dY, CnnLayer& Lr, int B, int H, int W,
                              cudaStream_t s) {
    const long tiles = (long)B * H * ((W + 127) / 128);
    const int nb = (int)(tiles < c->nsm ? tiles : c->nsm);
    const long per = 9L * Lr.cin * Lr.cout;
    if ((long)nb * per > c->part_cap) return cudaErrorInvalidValue;
    cudaError_t e;
    if (Lr.cin == 64 && Lr.cout == 64) e = launch_wgrad_tc<64, 64>(nb, X, dY, c->part, B, H, W, c->err, s);
    else if (Lr.cin == 16 && Lr.cout == 64) e = launch_wgrad_tc<16, 64>(nb, X, dY, c->part, B, H, W, c->err, s);
    else if (Lr.cin == 32 && Lr.cout == 64) e = launch_wgrad_tc<32, 64>(nb, X, dY, c->part, B, H, W, c->err, s);
    else if (Lr.cin == 64 && Lr.cout == 16) e = launch_wgrad_tc<64, 16>(nb, X, dY, c->part, B, H, W, c->err, s);
    else if (Lr.cin == 64 && Lr.cout == 32) e = launch_wgrad_tc<64, 32>(nb, X, dY, c->part, B, H, W, c->err, s);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    k_reduce_parts<<<(unsigned)((per + 255) / 256), 256, 0, s>>>(c->part, nb, per, Lr.gw);
    k_bias_grad<<<Lr.cout, 256, 0, s>>>(dY, (long)B * H * W, Lr.cout, Lr.gb);
    rte_count_launches(3);
    return cudaGetLastError();
}

static void cnn_free_acts(rte_cnn c) {
    for (bf16* a : c->act) if (a) rte_dev_free(a);
    c->act.clear();
    if (c->out_f) rte_dev_free(c->out_f);
    if (c->g0) rte_dev_free(c->g0);
    if (c->g1) rte_dev_free(c->g1);
    if (c->part) rte_dev_free(c->part);
    if (c->loss_part) rte_dev_free(c->loss_part);
    c->out_f = nullptr;
    c->g0 = c->g1 = nullptr;
    c->part = nullptr;
    c->loss_part = nullptr;
    c->B = c->H = c->W = 0;
}

static rte_status cnn_ensure(rte_cnn c, int B, int H, int W) {
    if (c->B == B && c->H == H && c->W == W) return RTE_OK;
    cnn_free_acts(c);
    const long P = (long)B * H * W;
    c->act.assign(c->depth + 1, nullptr);
    for (int l = 0; l <= c->depth; ++l) {
        const int ch = l == 0 ? c->cin : c->layers[l - 1].cout;
        if (rte_dev_malloc((void**)&c->act[l], P * ch * sizeof(bf16)) != cudaSuccess) { cudaGetLastError(); return RTE_ENOMEM; }
    }
    const int wmax = c->width > c->cin ? c->width : c->cin;
    if (rte_dev_malloc((void**)&c->out_f, P * c->cout * sizeof(float)) != cudaSuccess ||
        rte_dev_malloc((void**)&c->g0, P * wmax * sizeof(bf16)) != cudaSuccess ||
        rte_dev_malloc((void**)&c->g1, P * wmax * sizeof(bf16)) != cudaSuccess) {
        cudaGetLastError();
        return RTE_ENOMEM;
    }
    c->part_cap = (long)c->nsm * 9 * 64 * 64;
    if (rte_dev_malloc((void**)&c->part, c->part_cap * sizeof(float)) != cudaSuccess ||
        rte_dev_malloc((void**)&c->loss_part, 1024 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return RTE_ENOMEM;
    }
    c->B = B;
    c->H = H;
    c->W = W;
    return RTE_OK;
}

extern "C" rte_status rte_cnn_destroy(rte_cnn c) {
    if (!c) return RTE_OK;
    cudaDeviceSynchronize();
    cnn_free_acts(c);
    for (CnnLayer& L : c->layers) {
        void* ptrs[] = {L.w, L.bias, L.wb, L.wbt, L.mw, L.vw, L.mb, L.vb, L.gw, L.gb};
        for (void* p : ptrs) if (p) rte_dev_free(p);
    }
    if (c->loss_host) rte_host_free(c->loss_host);
    if (c->err) rte_dev_free(c->err);
    delete c;
    return RTE_OK;
}

extern "C" rte_status rte_cnn_create(rte_cnn* out, int cin, int width, int depth, int cout, unsigned long long seed,
                                     void* stream) {
    if (!out || depth < 2 || (cin != 16 && cin != 32) || (width != 64) || (cout != 16 && cout != 32)) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_cnn c = new rte_cnn_s();
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
        if (c->nsm < 1) c->nsm = 1;
    }
    c->cin = cin;
    c->width = width;
    c->depth = depth;
    c->cout = cout;
    c->layers.resize(depth);
    for (int l = 0; l < depth; ++l) {
        CnnLayer& L = c->layers[l];
        L.cin = l == 0 ? cin : width;
        L.cout = l == depth - 1 ? cout : width;
        const long nw = 9L * L.cin * L.cout;
        bool ok = rte_dev_malloc((void**)&L.w, nw * 4) == cudaSuccess && rte_dev_malloc((void**)&L.wb, nw * 2) == cudaSuccess &&
                  rte_dev_malloc((void**)&L.wbt, nw * 2) == cudaSuccess &&
                  rte_dev_malloc((void**)&L.mw, nw * 4) == cudaSuccess && rte_dev_malloc((void**)&L.vw, nw * 4) == cudaSuccess &&
                  rte_dev_malloc((void**)&L.gw, nw * 4) == cudaSuccess && rte_dev_malloc((void**)&L.bias, L.cout * 4) == cudaSuccess &&
                  rte_dev_malloc((void**)&L.mb, L.cout * 4) == cudaSuccess && rte_dev_malloc((void**)&L.vb, L.cout * 4) == cudaSuccess &&
                  rte_dev_malloc((void**)&L.gb, L.cout * 4) == cudaSuccess;
        if (!ok) { cudaGetLastError(); rte_cnn_destroy(c); return RTE_ENOMEM; }
        // He-uniform init; the last layer starts small so the first guess is ~b
        const float a = (l == depth - 1 ? 0.1f : 1.0f) * sqrtf(6.f / (9.f * L.cin));
        k_init_uniform<<<256, 256, 0, s>>>(L.w, nw, seed * 131 + l, a);
        k_to_bf16<<<256, 256, 0, s>>>(L.w, L.wb, L.wbt, L.cin, L.cout, nw);
        cudaMemsetAsync(L.bias, 0, L.cout * 4, s);
        cudaMemsetAsync(L.mw, 0, nw * 4, s);
        cudaMemsetAsync(L.vw, 0, nw * 4, s);
        cudaMemsetAsync(L.mb, 0, L.cout * 4, s);
        cudaMemsetAsync(L.vb, 0, L.cout * 4, s);
        rte_count_launches(2);
    }
    if (rte_host_malloc((void**)&c->loss_host, 1024 * sizeof(float)) != cudaSuccess ||
        rte_dev_malloc((void**)&c->err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        rte_cnn_destroy(c);
        return RTE_ENOMEM;
    }
    cudaMemsetAsync(c->err, 0, sizeof(int), s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rte_cnn_destroy(c); return rte_cuda_fail(e, "rte_cnn_create"); }
    *out = c;
    return RTE_OK;
}

static rte_status cnn_forward_internal(rte_cnn c, const bf16* X, int B, int H, int W, cudaStream_t s) {
    rte_status st = cnn_ensure(c, B, H, W);
    if (st != RTE_OK) return st;
    const long P = (long)B * H * W;
    RTE_CUDA_TRY(cudaMemcpyAsync(c->act[0], X, P * c->cin * sizeof(bf16), cudaMemcpyDeviceToDevice, s));
    for (int l = 0; l < c->depth; ++l) {
        const CnnLayer& L = c->layers[l];
        const bool last = l == c->depth - 1;
        cudaError_t e = conv_fwd(c->act[l], L, !last, last ? nullptr : c->act[l + 1], last ? c->out_f : nullptr,
                                 B, H, W, c->err, s);
        if (e != cudaSuccess) return rte_cuda_fail(e, "cnn forward");
    }
    return RTE_OK;
}

// y_out (device, f32 [B][H][W][cout]) = net(X)
extern "C" rte_status rte_cnn_forward(rte_cnn c, const void* X_dev, int B, int H, int W, float* y_dev, void* stream) {
    if (!c || !X_dev || !y_dev || B < 1 || H < 1 || W < 1) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_status st = cnn_forward_internal(c, (const bf16*)X_dev, B, H, W, s);
    if (st != RTE_OK) return st;
    RTE_CUDA_TRY(cudaMemcpyAsync(y_dev, c->out_f, (long)B * H * W * c->cout * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return RTE_OK;
}

// backward from dOut (bf16 [P][cout]) through all layers into the weight gradients
static rte_status cnn_backward(rte_cnn c, const bf16* dOut, int B, int H, int W, cudaStream_t s) {
    const long P = (long)B * H * W;
    RTE_CUDA_TRY(cudaMemcpyAsync(c->g0, dOut, P * c->cout * sizeof(bf16), cudaMemcpyDeviceToDevice, s));
    bf16* gcur = c->g0;
    bf16* gnext = c->g1;
    for (int l = c->depth - 1; l >= 0; --l) {
        CnnLayer& L = c->layers[l];
        if (l < c->depth - 1) {
            k_relu_bwd<<<1024, 256, 0, s>>>(gcur, c->act[l + 1], P * L.cout);
            rte_count_launches(1);
        }
        cudaError_t e = conv_wgrad(c, c->act[l], gcur, L, B, H, W, s);
        if (e != cudaSuccess) return rte_cuda_fail(e, "cnn wgrad");
        if (l > 0) {
            e = conv_dgrad(gcur, L, gnext, B, H, W, c->err, s);
            if (e != cudaSuccess) return rte_cuda_fail(e, "cnn dgrad");
            bf16* t = gcur;
            gcur = gnext;
            gnext = t;
        }
    }
    return RTE_OK;
}

// gradients of 0.5 * sum ... are exposed for testing: loss = mean over P x used
// of (net - target)^2; one Adam step when lr > 0.  X, T: bf16 [B][H][W][16].
extern "C" rte_status rte_cnn_train_step(rte_cnn c, const void* X_dev, const void* T_dev, int B, int H, int W,
                                         int used, float lr, float* loss_out, void* stream) {
    if (!c || !X_dev || !T_dev || B < 1 || used < 1 || used > c->cout) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_status st = cnn_forward_internal(c, (const bf16*)X_dev, B, H, W, s);
    if (st != RTE_OK) return st;
    const long P = (long)B * H * W;
    const int nb = 512;
    k_mse<<<nb, 256, 0, s>>>(c->out_f, (const bf16*)T_dev, P, c->cout, used, c->g1, c->loss_part);
    RTE_CUDA_TRY(cudaGetLastError());
    rte_count_launches(1);
    // dOut sits in g1; backward copies it into g0 first
    st = cnn_backward(c, c->g1, B, H, W, s);
    if (st != RTE_OK) return st;
    if (lr > 0.f) {
        c->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
        for (CnnLayer& L : c->layers) {
            const long nw = 9L * L.cin * L.cout;
            k_adam<<<256, 256, 0, s>>>(L.w, L.mw, L.vw, L.gw, L.wb, L.wbt, L.cin, L.cout, nw, lr, b1, b2, 1e-8f, c1,
                                       c2);
            k_adam<<<1, 256, 0, s>>>(L.bias, L.mb, L.vb, L.gb, nullptr, nullptr, 1, 1, L.cout, lr, b1, b2, 1e-8f, c1,
                                     c2);
            rte_count_launches(2);
        }
        RTE_CUDA_TRY(cudaGetLastError());
    }
    if (loss_out) {
        int* err_host = reinterpret_cast<int*>(c->loss_host + 1000);  // spare pinned words past the partials
        RTE_CUDA_TRY(cudaMemcpyAsync(c->loss_host, c->loss_part, nb * sizeof(float), cudaMemcpyDeviceToHost, s));
        RTE_CUDA_TRY(cudaMemcpyAsync(err_host, c->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        RTE_CUDA_TRY(cudaStreamSynchronize(s));
        if (*err_host) return rte_fail(RTE_ETIMEOUT, "cnn: a tensor-core convolution gave up waiting for its MMAs");
        double t = 0.0;
        for (int i = 0; i < nb; ++i) t += c->loss_host[i];
        *loss_out = (float)t;
    }
    return RTE_OK;
}

// layer access for checks and checkpoints: weights [9][cin][cout] f32, bias [cout]
extern "C" rte_status rte_cnn_layer(rte_cnn c, int l, int* cin, int* cout, float** w_dev, float** bias_dev,
                                    float** gw_dev, float** gb_dev) {
    if (!c || l < 0 || l >= c->depth) return RTE_EINVAL;
    CnnLayer& L = c->layers[l];
    if (cin) *cin = L.cin;
    if (cout) *cout = L.cout;
    if (w_dev) *w_dev = L.w;
    if (bias_dev) *bias_dev = L.bias;
    if (gw_dev) *gw_dev = L.gw;
    if (gb_dev) *gb_dev = L.gb;
    return RTE_OK;
}

// refresh the BF16 weights after the FP32 ones were written from outside
extern "C" rte_status rte_cnn_sync_weights(rte_cnn c, void* stream) {
    if (!c) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (CnnLayer& L : c->layers) {
        k_to_bf16<<<256, 256, 0, s>>>(L.w, L.wb, L.wbt, L.cin, L.cout, 9L * L.cin * L.cout);
        rte_count_launches(1);
    }
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// ---------------------------------------------------------------------------
// weights file: "RTECNN01", int32 cin, width, depth, cout, then per layer
// int32 cin_l, cout_l, f32 w[9][cin_l][cout_l], f32 bias[cout_l]
// (host byte order)
// ---------------------------------------------------------------------------
static const char kCnnMagic[8] = {'R', 'T', 'E', 'C', 'N', 'N', '0', '1'};

extern "C" rte_status rte_cnn_save(rte_cnn c, const char* path) {
    if (!c || !path) return RTE_EINVAL;
    RTE_CUDA_TRY(cudaDeviceSynchronize());
    FILE* f = fopen(path, "wb");
    if (!f) return rte_fail(RTE_EINVAL, "rte_cnn_save: cannot open the file");
    bool ok = fwrite(kCnnMagic, 1, 8, f) == 8;
    const int hdr[4] = {c->cin, c->width, c->depth, c->cout};
    ok = ok && fwrite(hdr, sizeof(int), 4, f) == 4;
    std::vector<float> buf;
    for (const CnnLayer& L : c->layers) {
        if (!ok) break;
        const int dims[2] = {L.cin, L.cout};
        ok = fwrite(dims, sizeof(int), 2, f) == 2;
        const size_t nw = 9ull * L.cin * L.cout;
        buf.resize(nw + L.cout);
        if (cudaMemcpy(buf.data(), L.w, nw * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(buf.data() + nw, L.bias, L.cout * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
            fclose(f);
            return rte_cuda_fail(cudaGetLastError(), "rte_cnn_save");
        }
        ok = ok && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) return rte_fail(RTE_EINVAL, "rte_cnn_save: writing the file failed");
    return RTE_OK;
}

extern "C" rte_status rte_cnn_load(rte_cnn c, const char* path, void* stream) {
    if (!c || !path) return RTE_EINVAL;
    FILE* f = fopen(path, "rb");
    if (!f) return rte_fail(RTE_EINVAL, "rte_cnn_load: cannot open the file");
    char magic[8];
    int hdr[4];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kCnnMagic, 8) == 0 && fread(hdr, sizeof(int), 4, f) == 4 &&
              hdr[0] == c->cin && hdr[1] == c->width && hdr[2] == c->depth && hdr[3] == c->cout;
    std::vector<std::vector<float>> host(c->layers.size());
    for (size_t l = 0; ok && l < c->layers.size(); ++l) {
        const CnnLayer& L = c->layers[l];
        int dims[2];
        ok = fread(dims, sizeof(int), 2, f) == 2 && dims[0] == L.cin && dims[1] == L.cout;
        if (!ok) break;
        host[l].resize(9ull * L.cin * L.cout + L.cout);
        ok = fread(host[l].data(), sizeof(float), host[l].size(), f) == host[l].size();
    }
    fclose(f);
    if (!ok) return rte_fail(RTE_EINVAL, "rte_cnn_load: not a weights file of this network's shape");
    // nothing on the device changes unless the whole file was valid
    for (size_t l = 0; l < c->layers.size(); ++l) {
        const CnnLayer& L = c->layers[l];
        const size_t nw = 9ull * L.cin * L.cout;
        RTE_CUDA_TRY(cudaMemcpy(L.w, host[l].data(), nw * sizeof(float), cudaMemcpyHostToDevice));
        RTE_CUDA_TRY(cudaMemcpy(L.bias, host[l].data() + nw, L.cout * sizeof(float), cudaMemcpyHostToDevice));
    }
    return rte_cnn_sync_weights(c, stream);
}

// Training checkpoint: the weights file's contents plus, per layer, the Adam
// moments of the weights and biases, and the optimizer's step count, so that a
// resumed run continues the same trajectory:
//   "RTECNS01", int32 cin, width, depth, cout, int64 step, then per layer
//   int32 cin_l, cout_l and f32 w, bias, m_w, v_w, m_b, v_b.
static const char kCnnStateMagic[8] = {'R', 'T', 'E', 'C', 'N', 'S', '0', '1'};

extern "C" rte_status rte_cnn_save_state(rte_cnn c, const char* path) {
    if (!c || !path) return RTE_EINVAL;
    RTE_CUDA_TRY(cudaDeviceSynchronize());
    FILE* f = fopen(path, "wb");
    if (!f) return rte_fail(RTE_EINVAL, "rte_cnn_save_state: cannot open the file");
    bool ok = fwrite(kCnnStateMagic, 1, 8, f) == 8;
    const int hdr[4] = {c->cin, c->width, c->depth, c->cout};
    const long long step = c->step;
    ok = ok && fwrite(hdr, sizeof(int), 4, f) == 4 && fwrite(&step, sizeof(step), 1, f) == 1;
    std::vector<float> buf;
    for (const CnnLayer& L : c->layers) {
        if (!ok) break;
        const int dims[2] = {L.cin, L.cout};
        ok = fwrite(dims, sizeof(int), 2, f) == 2;
        const size_t nw = 9ull * L.cin * L.cout, nb = (size_t)L.cout;
        const float* src[6] = {L.w, L.bias, L.mw, L.vw, L.mb, L.vb};
        const size_t cnt[6] = {nw, nb, nw, nw, nb, nb};
        for (int k = 0; k < 6 && ok; ++k) {
            buf.resize(cnt[k]);
            if (cudaMemcpy(buf.data(), src[k], cnt[k] * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
                fclose(f);
                return rte_cuda_fail(cudaGetLastError(), "rte_cnn_save_state");
            }
            ok = fwrite(buf.data(), sizeof(float), cnt[k], f) == cnt[k];
        }
    }
    ok = (fclose(f) == 0) && ok;
    if (!ok) return rte_fail(RTE_EINVAL, "rte_cnn_save_state: writing the file failed");
    return RTE_OK;
}

extern "C" rte_status rte_cnn_load_state(rte_cnn c, const char* path, void* stream) {
    if (!c || !path) return RTE_EINVAL;
    FILE* f = fopen(path, "rb");
    if (!f) return rte_fail(RTE_EINVAL, "rte_cnn_load_state: cannot open the file");
    char magic[8];
    int hdr[4];
    long long step = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kCnnStateMagic, 8) == 0 &&
              fread(hdr, sizeof(int), 4, f) == 4 && hdr[0] == c->cin && hdr[1] == c->width && hdr[2] == c->depth &&
              hdr[3] == c->cout && fread(&step, sizeof(step), 1, f) == 1 && step >= 0;
    std::vector<std::vector<float>> host(c->layers.size());
    for (size_t l = 0; ok && l < c->layers.size(); ++l) {
        const CnnLayer& L = c->layers[l];
        int dims[2];
        ok = fread(dims, sizeof(int), 2, f) == 2 && dims[0] == L.cin && dims[1] == L.cout;
        if (!ok) break;
        const size_t nw = 9ull * L.cin * L.cout, nb = (size_t)L.cout;
        host[l].resize(3 * nw + 3 * nb);
        ok = fread(host[l].data(), sizeof(float), host[l].size(), f) == host[l].size();
    }
    fclose(f);
    if (!ok) return rte_fail(RTE_EINVAL, "rte_cnn_load_state: not a training checkpoint of this network's shape");
    // nothing on the device changes unless the whole file was valid
    for (size_t l = 0; l < c->layers.size(); ++l) {
        const CnnLayer& L = c->layers[l];
        const size_t nw = 9ull * L.cin * L.cout, nb = (size_t)L.cout;
        float* dst[6] = {L.w, L.bias, L.mw, L.vw, L.mb, L.vb};
        const size_t cnt[6] = {nw, nb, nw, nw, nb, nb};
        const float* src = host[l].data();
        for (int k = 0; k < 6; ++k) {
            RTE_CUDA_TRY(cudaMemcpy(dst[k], src, cnt[k] * sizeof(float), cudaMemcpyHostToDevice));
            src += cnt[k];
        }
    }
    c->step = (long)step;
    return rte_cnn_sync_weights(c, stream);
}

// ---------------------------------------------------------------------------
// the learned guess for a plan: u0 = b + s_b * net(features(b, f, params))
// (scales s_b, fmax computed on the device into the plan's dscal[2..3])
// ---------------------------------------------------------------------------
static rte_status guess_scales(rte_plan p, const double* f_dev, const double* b_dev, cudaStream_t s) {
    k_guess_scales<<<1, 1024, 0, s>>>(b_dev, f_dev, p->n, p->L, p->dscal + 2);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

extern "C" rte_status rte_guess_features(rte_plan p, int cin, const double* f_dev, const double* b_dev, void* X_dev,
                                         void* stream) {
    if (!p || p->dim != 2 || !f_dev || !b_dev || !X_dev || (cin != 16 && cin != 32) || 2 * p->L + 5 > cin)
        return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_status st = guess_scales(p, f_dev, b_dev, s);
    if (st != RTE_OK) return st;
    const float p0 = (float)(log(p->mu_t > 1e-30 ? p->mu_t : 1e-30) / 4.0);
    const float p1 = (float)(p->mu_t > 0 ? p->mu_s / p->mu_t : 0.0);
    const float p2 = (float)(p->L >= 1 ? p->sigma_hat[1] : 0.0);
    k_features<<<512, 256, 0, s>>>(b_dev, f_dev, p->n, p->L, p->dscal + 2, p0, p1, p2, cin, (bf16*)X_dev);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    if (3 * p->nch + 4 <= cin && p->L <= RTE_MAX_L_DIRECT) {
        const dim3 tiles((p->n + 31) / 32, (p->n + 31) / 32);
        k_features_pooled<<<tiles, 256, 0, s>>>(b_dev, p->n, p->L, p->dscal + 2, cin, (bf16*)X_dev);
        rte_count_launches(1);
        RTE_CUDA_TRY(cudaGetLastError());
    }
    return RTE_OK;
}

extern "C" rte_status rte_guess_targets(rte_plan p, int cout, const double* f_dev, const double* u_dev,
                                        const double* b_dev, void* T_dev, void* stream) {
    if (!p || p->dim != 2 || !f_dev || !u_dev || !b_dev || !T_dev || (cout != 16 && cout != 32) ||
        2 * p->L + 1 > cout)
        return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_status st = guess_scales(p, f_dev, b_dev, s);
    if (st != RTE_OK) return st;
    k_targets<<<512, 256, 0, s>>>(u_dev, b_dev, p->n, p->L, p->dscal + 2, cout, (bf16*)T_dev);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// b_out: caller buffer for b = K~ g (FP64 mode field), computed here
extern "C" rte_status rte_cnn_guess_apply(rte_cnn c, rte_plan p, const double* f_dev, double* b_out_dev,
                                          void* X_scratch_dev, void* u0_dev, void* stream) {
    if (!c || !p || p->dim != 2 || !f_dev || !b_out_dev || !X_scratch_dev || !u0_dev || 2 * p->L + 1 > c->cout)
        return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // b = K~ g for the features and the guess base: the float-float
    // application (FP64-accurate, on the FP32 units)
    rte_status st = plan_apply64e(p, MIX_RHS, f_dev, b_out_dev, 0.0, 1.0, 0.0, nullptr, s);
    if (st != RTE_OK) return st;
    st = rte_guess_features(p, c->cin, f_dev, b_out_dev, X_scratch_dev, stream);
    if (st != RTE_OK) return st;
    st = cnn_forward_internal(c, (const bf16*)X_scratch_dev, 1, p->n, p->n, s);
    if (st != RTE_OK) return st;
    k_guess_out<<<512, 256, 0, s>>>(c->out_f, b_out_dev, p->n, p->L, p->dscal + 2, c->cout, (double*)u0_dev);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

// ---------------------------------------------------------------------------
// rte_guess: a trained network loaded from its weights file, with its own
// scratch (features and b = K~ g), sized on first use for a plan's grid
// ---------------------------------------------------------------------------
struct rte_guess_s {
    rte_cnn net = nullptr;
    void* X = nullptr;     // bf16 [n][n][cin]
    double* b = nullptr;   // FP64 mode field [L+1][n][n] complex
    size_t X_bytes = 0, b_bytes = 0;
};

extern "C" rte_status rte_guess_destroy(rte_guess g) {
    if (!g) return RTE_OK;
    if (g->X || g->b) cudaDeviceSynchronize();
    if (g->X) rte_dev_free(g->X);
    if (g->b) rte_dev_free(g->b);
    rte_status st = rte_cnn_destroy(g->net);
    delete g;
    return st;
}

extern "C" rte_status rte_guess_load(rte_guess* out, const char* weights_path) {
    if (!out || !weights_path) return RTE_EINVAL;
    *out = nullptr;
    FILE* f = fopen(weights_path, "rb");
    if (!f) return rte_fail(RTE_EINVAL, "rte_guess_load: cannot open the file");
    char magic[8];
    int hdr[4];
    const bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kCnnMagic, 8) == 0 && fread(hdr, sizeof(int), 4, f) == 4;
    fclose(f);
    if (!ok) return rte_fail(RTE_EINVAL, "rte_guess_load: not a network weights file");
    rte_guess g = new rte_guess_s();
    rte_status st = rte_cnn_create(&g->net, hdr[0], hdr[1], hdr[2], hdr[3], 0, nullptr);
    if (st == RTE_OK) st = rte_cnn_load(g->net, weights_path, nullptr);
    if (st == RTE_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) st = rte_cuda_fail(cudaGetLastError(), "rte_guess_load");
    if (st != RTE_OK) {
        rte_guess_destroy(g);
        return st;
    }
    *out = g;
    return RTE_OK;
}

extern "C" rte_status rte_guess_apply(rte_guess g, rte_plan p, const double* f_dev, void* u0_dev, void* stream) {
    if (!g || !p || p->dim != 2 || !f_dev || !u0_dev) return RTE_EINVAL;
    if (2 * p->L + 5 > g->net->cin || 2 * p->L + 1 > g->net->cout) return RTE_EINVAL;
    const size_t xb = (size_t)p->n * p->n * g->net->cin * sizeof(bf16);
    const size_t bb = (size_t)p->nr * sizeof(double);
    if (xb > g->X_bytes || bb > g->b_bytes) {
        // grow the scratch (synchronises the device: earlier calls may still use it)
        cudaDeviceSynchronize();
        if (xb > g->X_bytes) {
            if (g->X) rte_dev_free(g->X);
            g->X = nullptr;
            g->X_bytes = 0;
            if (rte_dev_malloc(&g->X, xb) != cudaSuccess) return rte_cuda_fail(cudaErrorMemoryAllocation, "rte_guess_apply");
            g->X_bytes = xb;
        }
        if (bb > g->b_bytes) {
            if (g->b) rte_dev_free(g->b);
            g->b = nullptr;
            g->b_bytes = 0;
            if (rte_dev_malloc((void**)&g->b, bb) != cudaSuccess)
                return rte_cuda_fail(cudaErrorMemoryAllocation, "rte_guess_apply");
            g->b_bytes = bb;
        }
    }
    return rte_cnn_guess_apply(g->net, p, f_dev, g->b, g->X, u0_dev, stream);
}
