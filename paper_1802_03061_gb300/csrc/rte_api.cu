// C ABI entry points (include/rte.h): plan lifetime, operator application,
// right-hand side, solve.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>

#include "internal.h"

static thread_local char g_last_error[256] = "";

rte_status rte_cuda_fail(cudaError_t e, const char* what) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();  // clear a sticky non-fatal error state where possible
    return e == cudaErrorMemoryAllocation ? RTE_ENOMEM : RTE_ECUDA;
}

rte_status rte_fail(rte_status st, const char* msg) {
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
    return st;
}

extern "C" const char* rte_last_error(void) { return g_last_error; }

// ---------------------------------------------------------------------------
// Every device and pinned-host allocation of the library goes through these
// wrappers: they count the live allocations and, for tests of the error
// paths, can make the k-th allocation fail as if the device were full
// (rte_debug_fail_alloc).  A simulated failure touches no CUDA state.
// ---------------------------------------------------------------------------
static std::atomic<long> g_alloc_seen{0}, g_alloc_fail_at{0}, g_live_dev{0}, g_live_host{0};

static bool alloc_injected_failure() {
    const long k = ++g_alloc_seen;
    const long at = g_alloc_fail_at.load();
    return at > 0 && k == at;
}

cudaError_t rte_dev_malloc(void** p, size_t bytes) {
    if (alloc_injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live_dev;
    return e;
}

cudaError_t rte_dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    if (alloc_injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) ++g_live_dev;
    return e;
}

cudaError_t rte_host_malloc(void** p, size_t bytes) {
    if (alloc_injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) ++g_live_host;
    return e;
}

cudaError_t rte_dev_free(void* p) {
    if (!p) return cudaSuccess;
    --g_live_dev;
    return cudaFree(p);
}

cudaError_t rte_dev_free_async(void* p, cudaStream_t s) {
    if (!p) return cudaSuccess;
    --g_live_dev;
    return cudaFreeAsync(p, s);
}

cudaError_t rte_host_free(void* p) {
    if (!p) return cudaSuccess;
    --g_live_host;
    return cudaFreeHost(p);
}

extern "C" rte_status rte_debug_fail_alloc(long k, long* seen_out, long* live_dev_out, long* live_host_out) {
    if (seen_out) *seen_out = g_alloc_seen.load();
    if (live_dev_out) *live_dev_out = g_live_dev.load();
    if (live_host_out) *live_host_out = g_live_host.load();
    g_alloc_seen = 0;
    g_alloc_fail_at = k > 0 ? k : 0;
    return RTE_OK;
}

static long long g_launches = 0;
void rte_count_launches(long k) { __atomic_add_fetch(&g_launches, (long long)k, __ATOMIC_RELAXED); }
extern "C" long long rte_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

extern "C" rte_status rte_time_passes(rte_plan p, int inner, int reps, double* ms_out, void* stream) {
    if (!p || !ms_out || reps < 1) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->dim != 2) return RTE_EUNSUPPORTED;
    if (inner == 2) return op2d_time_ff(p, reps, ms_out, s);
    if (inner == 3) return plan_time_pc(p, reps, ms_out, s);
    return inner ? op2d_time32(p, reps, ms_out, s) : op2d_time64(p, reps, ms_out, s);
}

extern "C" const char* rte_status_str(rte_status s) {
    switch (s) {
        case RTE_OK: return "ok";
        case RTE_EINVAL: return "invalid argument";
        case RTE_EUNSUPPORTED: return "unsupported configuration";
        case RTE_ENOMEM: return "device out of memory";
        case RTE_ECUDA: return "CUDA error";
        case RTE_ENOCONV: return "solver did not reach the tolerance";
        case RTE_ETIMEOUT: return "device wait timed out";
        case RTE_ENAN: return "non-finite value";
    }
    return "unknown status";
}

static bool smooth23(int q) {
    if (q < 1) return false;
    while (q % 2 == 0) q /= 2;
    while (q % 3 == 0) q /= 3;
    return q == 1;
}

static void fill_defaults(rte_opts* o) {
    if (o->tol <= 0) o->tol = 1e-8;
    if (o->restart <= 0) o->restart = 40;
    if (o->restart > 128) o->restart = 128;
    if (o->maxit <= 0) o->maxit = 2000;
    if (o->inner_tol <= 0) o->inner_tol = 1e-4;
}

template <typename P> static rte_status dalloc(P** p, size_t bytes) {
    if (rte_dev_malloc((void**)p, bytes) != cudaSuccess) {
        cudaGetLastError();
        snprintf(g_last_error, sizeof(g_last_error), "cudaMalloc(%zu) failed", bytes);
        return RTE_ENOMEM;
    }
    return RTE_OK;
}

// the operator's inputs by kind: x is the field (MIX_K, MIX_KF) or the source
// (MIX_RHS); MIX_KF adds the plan's source f
static const double* op_x(MixKind kind, const double* x) { return kind == MIX_RHS ? nullptr : x; }
static const double* op_f(const rte_plan p, MixKind kind, const double* x) {
    return kind == MIX_RHS ? x : kind == MIX_KF ? p->f_dev : nullptr;
}

rte_status plan_apply64(rte_plan p, MixKind kind, const double* x, double* out, double a, double b, double c,
                        const double* z, cudaStream_t s) {
    if (p->dim == 2) return op2d_apply64(p, kind, op_x(kind, x), op_f(p, kind, x), out, a, b, c, z, s);
    return op3d_apply64(p, kind, x, out, a, b, c, z, s);
}

// FP64-accurate application in float-float arithmetic (used by the mixed
// refinement for the right-hand side and the residual)
rte_status plan_apply64e(rte_plan p, MixKind kind, const double* x, double* out, double a, double b, double c,
                         const double* z, cudaStream_t s) {
    if (p->dim == 2) return op2d_apply_ff(p, kind, op_x(kind, x), op_f(p, kind, x), out, a, b, c, z, s);
    return op3d_apply_ff(p, kind, x, out, a, b, c, z, s);
}

// b = K~ f in FP32 into the FP32 field layout (3D uses the plan's d32 as
// scratch for the rounded source)
rte_status plan_rhs32(rte_plan p, float* out, cudaStream_t s) {
    if (p->dim == 2) return op2d_rhs32(p, out, s);
    return op3d_rhs32(p, p->d32, out, s);
}

rte_status plan_apply32(rte_plan p, const float* x, float* out, float a, float b, float c, const float* z,
                        cudaStream_t s) {
    if (p->dim == 2) return op2d_apply32(p, x, out, a, b, c, z, s);
    return op3d_apply32(p, x, out, a, b, c, z, s);
}

extern "C" rte_status rte_destroy(rte_plan p) {
    if (!p) return RTE_OK;
    cudaDeviceSynchronize();
    krylov_free(p);
    void* bufs[] = {p->twm64, p->twm32, p->twmff, p->Sm64, p->Sm32, p->Smff, p->S3p, p->Pp, p->pv1, p->pv2, p->tw64, p->tw32, p->twff, p->Sff, p->Sffp, p->S3ff, p->S64, p->S32, p->S16, p->S32p, p->S16p, p->Tz32, p->S3_64, p->S3_32, p->Dm, p->T64, p->T32,
                    p->U64, p->U32, p->Tsplit, p->Tsplit32, p->b64, p->r64, p->x64, p->t64, p->r32,
                    p->d32, p->dscal, p->part64, p->f_dev, p->u_dev, p->ref};
    for (void* b : bufs)
        if (b) rte_dev_free(b);
    if (p->hst) rte_host_free(p->hst);
    delete p;
    return RTE_OK;
}

extern "C" rte_status rte_plan_create(rte_plan* out, rte_grid grid, double h, double mu_t, double mu_s, int L,
                                      const double* sigma_hat, const rte_opts* opts, void* cuda_stream) {
    if (!out) return RTE_EINVAL;
    *out = nullptr;
    if (grid.dim != 2 && grid.dim != 3) return RTE_EINVAL;
    const int n = grid.n[0];
    if (n < 1 || !(h > 0) || !isfinite(h)) return RTE_EINVAL;
    if (!(mu_t >= 0) || !(mu_s >= 0) || !(mu_s <= mu_t) || !isfinite(mu_t)) return RTE_EINVAL;
    if (L < 0 || L > RTE_MAX_L) return RTE_EINVAL;
    if (L > 0 && !sigma_hat) return RTE_EINVAL;
    if (sigma_hat) {
        if (fabs(sigma_hat[0] - 1.0) > 1e-12) return RTE_EINVAL;
        for (int k = 1; k <= L; ++k)
            if (!(fabs(sigma_hat[k]) <= 1.0)) return RTE_EINVAL;
    }
    if (grid.dim == 3 && L > 0) return RTE_EUNSUPPORTED;
    rte_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    fill_defaults(&o);
    if (o.prec < RTE_PREC_FP64 || o.prec > RTE_PREC_MIXED_BF16SPEC) return RTE_EINVAL;
    if (o.mode_mix < 0 || o.mode_mix > 2) return RTE_EINVAL;
    if (o.mode_mix == 1 && L > RTE_MAX_L_DIRECT) return RTE_EINVAL;
    int Q = choose_Q(n);
    if (o.q_policy > 0) {
        Q = o.q_policy;
        if (Q < 2 * n - 1 || (Q & 1) || !smooth23(Q)) return RTE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rte_plan p = new rte_plan_s();
    p->dim = grid.dim;
    p->n = n;
    p->Q = Q;
    p->H = Q / 2 + 1;
    p->L = L;
    p->nch = 2 * L + 1;
    p->h = h;
    p->mu_t = mu_t;
    p->mu_s = mu_s;
    for (int k = 0; k <= RTE_MAX_L; ++k) p->sigma_hat[k] = (k <= L && sigma_hat) ? sigma_hat[k] : (k == 0 ? 1.0 : 0.0);
    p->opts = o;
    make_sched(&p->sched, Q);
    p->mix_fft = grid.dim == 2 && (o.mode_mix == 2 || (o.mode_mix == 0 && L > RTE_MAX_L_DIRECT));
    if (p->mix_fft) {
        p->Pm = choose_P(L);
        make_sched(&p->sched_m, p->Pm);
    }
    p->ncell = grid.dim == 2 ? (long)n * n : (long)n * n * n;
    p->nr = grid.dim == 2 ? 2L * (L + 1) * n * n : p->ncell;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);

    rte_status st = RTE_OK;
    const int H = p->H, nch = p->nch;
#define TRY(x)                      \
    do {                            \
        st = (x);                   \
        if (st != RTE_OK) goto fail; \
    } while (0)
    TRY(dalloc(&p->tw64, Q * sizeof(double2)));
    TRY(dalloc(&p->tw32, Q * sizeof(float2)));
    TRY(dalloc(&p->twff, Q * sizeof(ffc)));
    TRY(dalloc(&p->Dm, (2 * RTE_MAX_L + 1) * sizeof(double)));
    if (grid.dim == 2) {
        const size_t ns = (size_t)H * nch * Q;
        TRY(dalloc(&p->S64, ns * sizeof(double2)));
        TRY(dalloc(&p->S32, ns * sizeof(float2)));
        if (p->mix_fft) {
            // the column passes use only the mode-axis DFTs of the spectra
            const int P = p->Pm;
            const size_t nf = (size_t)H * Q * P;
            TRY(dalloc(&p->twm64, P * sizeof(double2)));
            TRY(dalloc(&p->twm32, P * sizeof(float2)));
            TRY(dalloc(&p->twmff, P * sizeof(ffc)));
            TRY(dalloc(&p->Sm64, nf * sizeof(double2)));
            TRY(dalloc(&p->Sm32, nf * sizeof(float2)));
            TRY(dalloc(&p->Smff, nf * sizeof(ffc)));
        } else if (Q == 64 || Q == 128 || Q == 256 || Q == 512 || Q == 1024) {
            TRY(dalloc(&p->S16, ns * sizeof(__nv_bfloat162)));
            TRY(dalloc(&p->S32p, ns * sizeof(float2)));
            TRY(dalloc(&p->S16p, ns * sizeof(__nv_bfloat162)));
            TRY(dalloc(&p->Sffp, ns * sizeof(ffc)));
            // Q = 1024: the column passes run two 512-point residues; the
            // first residue's result waits here
            if (Q == 1024) TRY(dalloc(&p->Tz32, (size_t)nch * H * n * sizeof(float2)));
        } else {
            TRY(dalloc(&p->S16, ns * sizeof(__nv_bfloat162)));
            TRY(dalloc(&p->Sff, ns * sizeof(ffc)));
        }
        const size_t nt = (size_t)nch * H * n;
        TRY(dalloc((double2**)&p->T64, nt * sizeof(double2)));
        TRY(dalloc((float2**)&p->T32, nt * sizeof(float2)));
        p->col_split64 = (size_t)(Q + nch * Q + Q) * sizeof(double2) > 200 * 1024;
        p->col_split32 = (size_t)(Q + nch * Q + Q) * sizeof(float2) > 200 * 1024;
        // the float-float passes always take the split column path
        TRY(dalloc((double2**)&p->Tsplit, (size_t)nch * H * Q * sizeof(double2)));
        if (p->col_split32 || p->mix_fft) TRY(dalloc((float2**)&p->Tsplit32, (size_t)nch * H * Q * sizeof(float2)));
    } else {
        const size_t ns = (size_t)H * H * H;
        TRY(dalloc(&p->S3_64, ns * sizeof(double)));
        TRY(dalloc(&p->S3_32, ns * sizeof(float)));
        TRY(dalloc(&p->S3ff, ns * sizeof(ff)));
        const size_t n1 = (size_t)n * H * n;   // after x pass: [z][xi_x][y]
        const size_t n2 = (size_t)H * Q * n;   // after y pass: [xi_x][xi_y][z]
        TRY(dalloc((double2**)&p->T64, n1 * sizeof(double2)));
        TRY(dalloc((double2**)&p->U64, n2 * sizeof(double2)));
        TRY(dalloc((float2**)&p->T32, n1 * sizeof(float2)));
        TRY(dalloc((float2**)&p->U32, n2 * sizeof(float2)));
    }
    TRY(dalloc(&p->b64, p->nr * sizeof(double)));
    TRY(dalloc(&p->r64, p->nr * sizeof(double)));
    TRY(dalloc(&p->x64, p->nr * sizeof(double)));
    TRY(dalloc(&p->t64, p->nr * sizeof(double)));
    TRY(dalloc(&p->r32, p->nr * sizeof(float)));
    TRY(dalloc(&p->d32, p->nr * sizeof(float)));
    TRY(dalloc(&p->dscal, 8 * sizeof(double)));
    TRY(dalloc(&p->part64, (size_t)((p->nr + 2047) / 2048 + 1) * sizeof(double)));
    TRY(dalloc(&p->f_dev, p->ncell * sizeof(double)));
    TRY(dalloc(&p->u_dev, p->nr * sizeof(double)));
    TRY(dalloc((char**)&p->ref, refdev_size()));
    if (rte_host_malloc((void**)&p->hst, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        st = RTE_ENOMEM;
        goto fail;
    }
    TRY(plan_build_spectra(p, s));
    TRY(plan_build_modefft(p, s));
    if (grid.dim == 2) TRY(op2d_permute_spectra(p, s));
    TRY(plan_split_ff(p, s));
    // one application in each precision: validates the launch shapes and
    // sets the kernels' shared-memory attributes before any graph capture
    if (cudaMemsetAsync(p->x64, 0, p->nr * sizeof(double), s) != cudaSuccess) { st = RTE_ECUDA; goto fail; }
    if (cudaMemsetAsync(p->r32, 0, p->nr * sizeof(float), s) != cudaSuccess) { st = RTE_ECUDA; goto fail; }
    TRY(plan_apply64(p, MIX_K, p->x64, p->t64, 1.0, -1.0, 0.0, nullptr, s));
    TRY(plan_apply32(p, p->r32, p->d32, 1.0f, -1.0f, 0.0f, nullptr, s));
    TRY(plan_apply64e(p, MIX_K, p->x64, p->t64, 1.0, -1.0, 0.0, nullptr, s));
    {
        cudaError_t ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { st = rte_cuda_fail(ce, "plan_create"); goto fail; }
    }
#undef TRY
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        p->ms_pre = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = p;
    return RTE_OK;
fail:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rte_destroy(p);
    return st;
}

extern "C" rte_status rte_apply_K(rte_plan p, const void* x, void* y, void* stream) {
    if (!p || !x || !y || x == y) return RTE_EINVAL;
    return plan_apply64(p, MIX_K, (const double*)x, (double*)y, 0.0, 1.0, 0.0, nullptr, (cudaStream_t)stream);
}

extern "C" rte_status rte_apply_A(rte_plan p, const void* x, void* y, void* stream) {
    if (!p || !x || !y || x == y) return RTE_EINVAL;
    return plan_apply64(p, MIX_K, (const double*)x, (double*)y, 1.0, -1.0, 0.0, nullptr, (cudaStream_t)stream);
}

extern "C" rte_status rte_apply_K64e(rte_plan p, const void* x, void* y, void* stream) {
    if (!p || !x || !y || x == y) return RTE_EINVAL;
    return plan_apply64e(p, MIX_K, (const double*)x, (double*)y, 0.0, 1.0, 0.0, nullptr, (cudaStream_t)stream);
}

extern "C" rte_status rte_apply_K32(rte_plan p, const void* x, void* y, void* stream) {
    if (!p || !x || !y || x == y) return RTE_EINVAL;
    return plan_apply32(p, (const float*)x, (float*)y, 0.0f, 1.0f, 0.0f, nullptr, (cudaStream_t)stream);
}

extern "C" rte_status rte_precond_info(rte_plan p, int* lmax_out) {
    if (!p || !lmax_out || !p->pc_ready) return RTE_EINVAL;
    *lmax_out = p->dim == 2 ? (p->pc_nl - 1) / 2 : 0;
    return RTE_OK;
}

extern "C" rte_status rte_apply_precond32(rte_plan p, const void* x, void* y, void* stream) {
    if (!p || !x || !y || x == y) return RTE_EINVAL;
    if (!plan_precond_supported(p)) return RTE_EUNSUPPORTED;
    rte_status st = plan_precond_build(p, (cudaStream_t)stream);
    if (st != RTE_OK) return st;
    return plan_apply_pc32(p, (const float*)x, (float*)y, (cudaStream_t)stream);
}

extern "C" rte_status rte_rhs(rte_plan p, const double* f, void* b, void* stream) {
    if (!p || !f || !b) return RTE_EINVAL;
    return plan_apply64(p, MIX_RHS, f, (double*)b, 0.0, 1.0, 0.0, nullptr, (cudaStream_t)stream);
}

// f and u are copied to / from the plan's own buffers so that the captured
// solve graph (bound to those buffers) serves every call
extern "C" rte_status rte_solve(rte_plan p, const double* f, void* u, const rte_opts* opts, rte_stats* stats,
                                void* stream) {
    if (!p || !f || !u) return RTE_EINVAL;
    rte_opts o = opts ? *opts : p->opts;
    fill_defaults(&o);
    if (o.prec < RTE_PREC_FP64 || o.prec > RTE_PREC_MIXED_BF16SPEC) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    RTE_CUDA_TRY(cudaMemcpyAsync(p->f_dev, f, p->ncell * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (o.use_guess) RTE_CUDA_TRY(cudaMemcpyAsync(p->u_dev, u, p->nr * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return krylov_solve(p, &o, stats, s, u, cudaMemcpyDeviceToDevice);
}

extern "C" rte_status rte_solve_host(rte_plan p, const double* f_host, void* u_host, const rte_opts* opts,
                                     rte_stats* stats, void* stream) {
    if (!p || !f_host || !u_host) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_opts o = opts ? *opts : p->opts;
    fill_defaults(&o);
    if (o.prec < RTE_PREC_FP64 || o.prec > RTE_PREC_MIXED_BF16SPEC) return RTE_EINVAL;
    RTE_CUDA_TRY(cudaMemcpyAsync(p->f_dev, f_host, p->ncell * sizeof(double), cudaMemcpyHostToDevice, s));
    if (o.use_guess)
        RTE_CUDA_TRY(cudaMemcpyAsync(p->u_dev, u_host, p->nr * sizeof(double), cudaMemcpyHostToDevice, s));
    return krylov_solve(p, &o, stats, s, u_host, cudaMemcpyDeviceToHost);
}

extern "C" rte_status rte_plan_info(rte_plan p, int* n, int* Q, int* L, long* nreal) {
    if (!p) return RTE_EINVAL;
    if (n) *n = p->n;
    if (Q) *Q = p->Q;
    if (L) *L = p->L;
    if (nreal) *nreal = p->nr;
    return RTE_OK;
}

extern "C" rte_status rte_plan_cell_weights(rte_plan p, double* out) {
    if (!p || !out) return RTE_EINVAL;
    const int cnt = p->dim == 2 ? 2 * p->L + 1 : 1;
    RTE_CUDA_TRY(cudaMemcpy(out, p->Dm, cnt * sizeof(double), cudaMemcpyDeviceToHost));
    return RTE_OK;
}

// ---------------------------------------------------------------------------
// autotuner: padded length Q and row tile by measurement
// ---------------------------------------------------------------------------
extern "C" rte_status rte_autotune(int n, int L, int prec, int reps, int* Q_out, int* rb_out, double* ms_out,
                                   void* stream) {
    if (n < 1 || L < 0 || L > RTE_MAX_L || reps < 1) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double sig[RTE_MAX_L + 1];
    for (int k = 0; k <= L; ++k) sig[k] = k == 0 ? 1.0 : 0.5;
    // the three smallest admissible Q, and the smallest Q whose column passes
    // run on the warp-register FFT (64, 128, ..., 1024) when it is not among them
    int cands[4];
    int nc = 0;
    int q = choose_Q(n);
    while (nc < 3) {
        cands[nc++] = q;
        ++q;
        while (q % 2 || !smooth23(q)) ++q;
    }
    for (int w = 64; w <= 1024; w *= 2)
        if (w >= 2 * n - 1) {
            if (w > cands[nc - 1]) cands[nc++] = w;
            break;
        }
    double best = 1e30;
    int bq = cands[0], brb = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c = 0; c < nc; ++c) {
        rte_opts o;
        memset(&o, 0, sizeof(o));
        o.prec = (rte_prec)(prec == RTE_PREC_FP64 ? RTE_PREC_MIXED_FP32 : prec);
        o.q_policy = cands[c];
        rte_grid g;
        g.dim = 2;
        g.n[0] = g.n[1] = g.n[2] = n;
        rte_plan p = nullptr;
        rte_status st = rte_plan_create(&p, g, 1.0 / n, 1.0, 0.5, L, sig, &o, stream);
        if (st != RTE_OK) continue;
        // 0 = the default row passes (warp-register FFT where Q allows it)
        const int rbs[5] = {0, 2, 4, 8, 16};
        for (int r = 0; r < 5; ++r) {
            p->rb_force = rbs[r];
            st = plan_apply32(p, p->r32, p->d32, 1.0f, -1.0f, 0.0f, nullptr, s);  // warm-up
            if (st != RTE_OK) break;
            cudaEventRecord(e0, s);
            for (int i = 0; i < reps && st == RTE_OK; ++i)
                st = plan_apply32(p, p->r32, p->d32, 1.0f, -1.0f, 0.0f, nullptr, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double t = ms / reps;
            if (st == RTE_OK && t < best) {
                best = t;
                bq = cands[c];
                brb = rbs[r];
            }
        }
        rte_destroy(p);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best >= 1e30) return RTE_ECUDA;
    if (Q_out) *Q_out = bq;
    if (rb_out) *rb_out = brb;
    if (ms_out) *ms_out = best;
    return RTE_OK;
}
