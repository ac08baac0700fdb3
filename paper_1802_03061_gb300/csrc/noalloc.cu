// rte_apply_K_noalloc: y = K x for small 2D grids without any device
// allocation.  Intended for callers that may not allocate device memory at
// the point of the call: plug-ins whose host application owns and caps the
// device memory, real-time loops that forbid allocator calls after start-up,
// code that runs while another component holds the whole device allocator.
// They cannot create a plan (rte_plan_create allocates), so this call rebuilds
// everything a plan would hold -- twiddles, cell weights, kernel samples,
// spectra -- plus the pass intermediates in one fixed static device array,
// then runs the same FP64 passes as rte_apply_K.
//
// The scratch is a file-scope __device__ array of RTE_NOALLOC_BYTES bytes.
// This translation unit is its own CUDA module (the library is built without
// relocatable device code), and under the runtime's default lazy module
// loading that module -- and with it the array's device memory -- is loaded
// on a device at the first cudaGetSymbolAddress below, i.e. during the first
// call on that device; from then on the device holds the array until the
// process exits.  Callers therefore make their first call where taking that
// memory is allowed (start-up) and before any stream capture.
// All calls share it: two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.  Every call writes each scratch byte it reads before reading
// it (kernel samples and padding are written in full), so no clearing is
// needed between calls.
#include <math.h>
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "internal.h"

#define RTE_NOALLOC_MAX_N 64
#define RTE_NOALLOC_MAX_L 4
#define NA_QMAX 128
#define NA_HMAX (NA_QMAX / 2 + 1)
#define NA_NM (2 * RTE_NOALLOC_MAX_L + 1)
// layout in double2 units
#define NA_G_ELEMS ((long)NA_NM * NA_QMAX * NA_QMAX)        // sampled kernels, full grid
#define NA_S64_ELEMS ((long)NA_HMAX * NA_NM * NA_QMAX)      // FP64 spectra
#define NA_S32_ELEMS ((NA_S64_ELEMS + 1) / 2)                // FP32 copy (float2)
#define NA_S16_ELEMS ((NA_S64_ELEMS + 3) / 4)                // BF16 copy (bf16x2)
#define NA_T_ELEMS ((long)NA_NM * NA_HMAX * RTE_NOALLOC_MAX_N)  // pass intermediate
#define NA_TW_ELEMS (NA_QMAX + NA_QMAX / 2)                 // tw64 + tw32
#define NA_D_ELEMS 16                                       // cell weights (doubles, 2 per double2)
#define NA_TOTAL (NA_G_ELEMS + NA_S64_ELEMS + NA_S32_ELEMS + NA_S16_ELEMS + NA_T_ELEMS + NA_TW_ELEMS + NA_D_ELEMS)
#define RTE_NOALLOC_BYTES (NA_TOTAL * 16)

static __device__ __align__(256) double2 g_rte_noalloc_scratch[NA_TOTAL];

static std::mutex g_na_mu;
static double2* g_na_addr[64];  // device address of the scratch, per device ordinal
static bool g_na_ready[64];

// Once per device, with that device current: the host-side symbol is only a
// stand-in, the kernels need the device address.
static rte_status na_scratch(double2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_apply_K_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return RTE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ready[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rte_noalloc_scratch);
        if (e != cudaSuccess) return rte_cuda_fail(e, "rte_apply_K_noalloc: cudaGetSymbolAddress");
        g_na_addr[dev] = (double2*)p;
        g_na_ready[dev] = true;
    }
    *out = g_na_addr[dev];
    return RTE_OK;
}

extern "C" long long rte_noalloc_scratch_bytes(void) { return (long long)RTE_NOALLOC_BYTES; }

extern "C" rte_status rte_apply_K_noalloc(int n, double h, double mu_t, double mu_s, int L, const double* sigma_hat,
                                          const void* x_dev, void* y_dev, void* cuda_stream) {
    if (!x_dev || !y_dev || x_dev == y_dev) return RTE_EINVAL;
    if (n < 1 || !(h > 0) || !isfinite(h)) return RTE_EINVAL;
    if (!(mu_t >= 0) || !(mu_s >= 0) || !(mu_s <= mu_t) || !isfinite(mu_t)) return RTE_EINVAL;
    if (L < 0 || (L > 0 && !sigma_hat)) return RTE_EINVAL;
    if (n > RTE_NOALLOC_MAX_N || L > RTE_NOALLOC_MAX_L) {
        return RTE_EUNSUPPORTED;  // beyond the fixed static scratch: use rte_plan_create + rte_apply_K
    }
    if (sigma_hat) {
        if (fabs(sigma_hat[0] - 1.0) > 1e-12) return RTE_EINVAL;
        for (int k = 1; k <= L; ++k)
            if (!(fabs(sigma_hat[k]) <= 1.0)) return RTE_EINVAL;
    }
    double2* base = nullptr;
    rte_status st = na_scratch(&base);
    if (st != RTE_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // a plan on the stack whose buffers all point into the static scratch
    rte_plan_s p;
    p.dim = 2;
    p.n = n;
    p.Q = choose_Q(n);
    p.H = p.Q / 2 + 1;
    p.L = L;
    p.nch = 2 * L + 1;
    p.h = h;
    p.mu_t = mu_t;
    p.mu_s = mu_s;
    for (int k = 0; k <= RTE_MAX_L; ++k) p.sigma_hat[k] = (k <= L && sigma_hat) ? sigma_hat[k] : (k == 0 ? 1.0 : 0.0);
    make_sched(&p.sched, p.Q);
    p.ncell = (long)n * n;
    p.nr = 2L * (L + 1) * n * n;
    const int Q = p.Q, H = p.H, nm = 2 * L + 1;
    double2* G = base;
    double2* S64 = G + NA_G_ELEMS;
    float2* S32 = (float2*)(S64 + NA_S64_ELEMS);
    __nv_bfloat162* S16 = (__nv_bfloat162*)(S64 + NA_S64_ELEMS + NA_S32_ELEMS);
    double2* T = S64 + NA_S64_ELEMS + NA_S32_ELEMS + NA_S16_ELEMS;
    double2* tw64 = T + NA_T_ELEMS;
    float2* tw32 = (float2*)(tw64 + NA_QMAX);
    double* Dm = (double*)(tw64 + NA_TW_ELEMS);

    k_twiddles<<<(Q + 255) / 256, 256, 0, s>>>(tw64, tw32, Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_apply_K_noalloc: twiddles");
    k_cell_weights_2d<<<1, 64, 0, s>>>(mu_t, h, 2 * L, Dm);
    const long P = (long)Q * Q;
    k_sample_2d<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(G, n, Q, 2 * L, h, mu_t, Dm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_apply_K_noalloc: sampling");
    rte_count_launches(3);
    st = fft_lines_host(G, p.sched, tw64, (long)nm * Q, (long)nm * Q, Q, 0, 1, s);
    if (st != RTE_OK) return st;
    st = fft_lines_host(G, p.sched, tw64, (long)nm * Q, Q, 1, P, Q, s);
    if (st != RTE_OK) return st;
    const long tot = (long)H * nm * Q;
    k_extract_2d<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, Q, H, nm, S64, S32, S16);
    e = cudaGetLastError();
    if (e != cudaSuccess) return rte_cuda_fail(e, "rte_apply_K_noalloc: spectra");
    rte_count_launches(3);
    return op2d_apply64_buffers(&p, (const double*)x_dev, (double*)y_dev, T, S64, tw64, s);
}
