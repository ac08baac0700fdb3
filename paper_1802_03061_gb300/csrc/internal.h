// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/rte.h"
#include "common.cuh"

rte_status rte_cuda_fail(cudaError_t e, const char* what);
// records msg as the last error text and returns st
rte_status rte_fail(rte_status st, const char* msg);
// allocation wrappers (rte_api.cu): cudaMalloc / cudaMallocAsync /
// cudaMallocHost and their frees, with a live-allocation count and the
// simulated failures of rte_debug_fail_alloc
cudaError_t rte_dev_malloc(void** p, size_t bytes);
cudaError_t rte_dev_malloc_async(void** p, size_t bytes, cudaStream_t s);
cudaError_t rte_host_malloc(void** p, size_t bytes);
cudaError_t rte_dev_free(void* p);
cudaError_t rte_dev_free_async(void* p, cudaStream_t s);
cudaError_t rte_host_free(void* p);
template <typename T> inline cudaError_t rte_dev_malloc(T** p, size_t bytes) { return rte_dev_malloc((void**)p, bytes); }
template <typename T> inline cudaError_t rte_host_malloc(T** p, size_t bytes) { return rte_host_malloc((void**)p, bytes); }
// host-side count of kernel launches issued by the library (graph replays
// add the kernel nodes they contain)
void rte_count_launches(long k);
extern "C" long long rte_kernel_launches(void);

// Which linear map a pass sequence applies (Sec. 3.3, steps T.1 and T.2).
// MIX_K: K x;  MIX_RHS: K~ applied to the source f (mode 0);  MIX_KF: K x + K~ f
// in one application (the source joins mode 0 of the input after the
// mu_s sigma_hat weighting)
enum MixKind { MIX_K = 0, MIX_RHS = 1, MIX_KF = 2 };

// Krylov workspace of one precision.
struct KrylovWs {
    int m = 0;               // restart length (basis holds m+2 vectors; slot m+1 = matvec input)
    void* V = nullptr;       // (m+2) x nr reals (float or double)
    void* w = nullptr;       // nr reals
    double* part = nullptr;  // partial sums [(m+1)][tiles]
    double* st = nullptr;    // device GMRES state (see krylov.cu)
    void* Z = nullptr;       // preconditioned inner solves: (m+1) x nr floats, z_j = M v_j
};
void krylov_free_ws(KrylovWs& ws);

// kernels per graph segment of a captured solve (for launch accounting)
struct SolveGraphInfo {
    long long k_fixed = 0, k_guess = 0, k_outer = 0, k_cycle = 0, k_step = 0, k_restart = 0;
};
// The operator and the vectors a solve graph is built on (krylov.cu): the
// plan's J-symmetric channels, or the spherical-harmonic operator's moments.
// Each callback enqueues its kernels on the given stream (it is captured).
struct KrylovOp {
    void* ctx = nullptr;
    long nr = 0;       // vector length (reals)
    long nw1 = 0;      // elements [0, nw1) weigh 1 in the inner product, the rest 2
    double* u = nullptr;       // solution
    double* b64 = nullptr;     // right-hand side
    double* r64 = nullptr;     // residual
    double* x64 = nullptr;     // FP64 mode: correction of one refinement step
    double* part64 = nullptr;  // reduction partials, krylov_tiles(nr)
    float* r32 = nullptr;      // mixed mode: inner right-hand side
    float* d32 = nullptr;      // mixed mode: inner solution
    float* pv1 = nullptr;      // preconditioned steps: M v (with pcA32 only)
    void* ref = nullptr;       // device refinement state, refdev_size() bytes
    // y = (I - K) x
    rte_status (*A32)(void* ctx, const float* x, float* y, cudaStream_t s) = nullptr;
    rte_status (*A64)(void* ctx, const double* x, double* y, cudaStream_t s) = nullptr;
    // y = (I - K) M x with z = M x (right preconditioning), or null
    rte_status (*pcA32)(void* ctx, const float* x, float* z, float* y, cudaStream_t s) = nullptr;
    // b64 = K~ f (FP32-accurate suffices when mixed: residuals are exact in b)
    rte_status (*rhs)(void* ctx, int mixed, cudaStream_t s) = nullptr;
    // r64 = b - (I - K) u, FP64-accurate
    rte_status (*resid)(void* ctx, int mixed, cudaStream_t s) = nullptr;
};
long krylov_tiles(long nr);
// graph of a whole solve of op (GMRES inner solves, no preconditioner) into *exec
rte_status krylov_op_graph(const KrylovOp& op, KrylovWs& ws, int prec, int m, cudaStream_t s, void** exec,
                           SolveGraphInfo* info);
// options into op.ref (host staging `hst`, refdev_size() bytes), launch, read back
// the state into hst + refdev_size(), collect statistics and the status
rte_status krylov_op_run(const KrylovOp& op, void* exec, const SolveGraphInfo& info, const rte_opts* o, void* hst,
                         double rho, double ms_pre, rte_stats* stats, cudaStream_t s);

struct SolveGraph {
    void* exec = nullptr;  // cudaGraphExec_t of the whole solve
    int m = 0;
    bool minres = false;   // inner solves by MINRES (else GMRES)
    bool pc = false;       // inner GMRES with the periodic preconditioner
    SolveGraphInfo info;
};

struct rte_plan_s {
    int dim = 2;
    int n = 0;             // cells per side
    int Q = 0;             // padded FFT length per dimension (even, >= 2n-1)
    int H = 0;             // Q/2 + 1 half-spectrum columns
    int L = 0;
    int nch = 1;           // real channels 2L+1
    long ncell = 0;        // n^dim
    long nr = 0;           // reals per field vector: 2D 2(L+1)n^2, 3D n^3
    double h = 0, mu_t = 0, mu_s = 0;
    double sigma_hat[RTE_MAX_L + 1];
    rte_opts opts;
    FftSched sched;
    // twiddle tables exp(-2 pi i t/Q), t < Q
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    // kernel spectra (already scaled by 1/Q^dim).
    // 2D: [H][2L+1][Q] complex for m = 0..2L.  3D: real octant [H][H][H].
    double2* S64 = nullptr;
    float2* S32 = nullptr;
    __nv_bfloat162* S16 = nullptr;
    ffc* Sff = nullptr;              // float-float copy of S64 (FP64-accurate passes on FP32 units)
    ffc* Sffp = nullptr;             // the same in the warp column pass's slot order (Q = 32 * 2^j)
    ff* S3ff = nullptr;
    ffc* twff = nullptr;
    float2* S32p = nullptr;          // FP32 / BF16 spectra in the warp column pass's slot order
    float2* Tz32 = nullptr;          // Q = 1024: first-residue column results [nch][H][n]
    __nv_bfloat162* S16p = nullptr;
    double* S3_64 = nullptr;
    float* S3_32 = nullptr;
    // periodic preconditioner (precond.cu), built on first use: 3D inverse
    // spectrum [H][H][H]; 2D tagged inverse matrices [H][nch][nch][Q] (BF16)
    float* S3p = nullptr;
    __nv_bfloat16* Pp = nullptr;
    float* pv1 = nullptr;      // FP32 field temporaries of the preconditioned solve
    float* pv2 = nullptr;
    bool pc_ready = false;
    int pc_nl = 0;                   // 2D: channels the preconditioner inverts (2 lmax + 1)
    // mode coupling by a circular convolution along the mode axis (2D,
    // rte_opts.mode_mix): length P >= 4L+1, twiddles exp(-2 pi i t/P) and
    // per frequency the P-point DFT of S_m (m = -2L..2L at m mod P), scaled
    // by 1/P: [H*Q][P] complex in FP64, FP32 and float-float
    bool mix_fft = false;
    int Pm = 0;
    FftSched sched_m;
    double2* twm64 = nullptr;
    float2* twm32 = nullptr;
    ffc* twmff = nullptr;
    double2* Sm64 = nullptr;
    float2* Sm32 = nullptr;
    ffc* Smff = nullptr;
    // cell weights D_m, m = 0..2L (2D) or D (3D), computed on the device
    double* Dm = nullptr;
    // pass intermediates: 2D [nch][H][n] complex; 3D T1 [n][H][n], T2 [H][Q][n]
    void* T64 = nullptr;
    void* T32 = nullptr;
    void* U64 = nullptr;   // second 3D intermediate (FP64)
    void* U32 = nullptr;   // second 3D intermediate (FP32)
    void* Tsplit = nullptr;    // [nch][H][Q] complex FP64 for the split column path
    void* Tsplit32 = nullptr;  // same, FP32
    bool col_split64 = false;
    bool col_split32 = false;
    // solve buffers (FP64): b, r, u, tmp
    double* b64 = nullptr;
    double* r64 = nullptr;
    double* x64 = nullptr;
    double* t64 = nullptr;
    float* r32 = nullptr;
    float* d32 = nullptr;
    double* dscal = nullptr;  // device scalar (residual norm)
    double* part64 = nullptr; // partial sums of plan-level norms
    // host-side staging for rte_solve_host
    double* f_dev = nullptr;
    double* u_dev = nullptr;
    KrylovWs k64, k32;
    SolveGraph graphs[3];    // per precision mode
    void* ev[2] = {nullptr, nullptr};  // cudaEvent_t pair timing the solve graph (created on first use)
    void* ref = nullptr;     // device refinement state (krylov.cu)
    double* hst = nullptr;   // pinned host mirror of small device state (64 doubles)
    double ms_pre = 0.0;
    int rb_force = 0;        // row-pass rows per block chosen by the autotuner (0 = default)
    int nsm = 152;
};

// spectra.cu
rte_status plan_build_spectra(rte_plan p, cudaStream_t s);
// the mode-axis DFTs of the spectra (p->mix_fft plans), from p->S64
rte_status plan_build_modefft(rte_plan p, cudaStream_t s);
int choose_P(int L);
rte_status fft_lines_host(double2* data, const FftSched& sc, const double2* tw, long nlines, long nA, long sA,
                          long sB, long sE, cudaStream_t s);
__global__ void k_twiddles(double2* tw64, float2* tw32, int Q);
__global__ void k_cell_weights_2d(double mu, double h, int mmax, double* D);
__global__ void k_sample_2d(double2* G, int n, int Q, int mmax, double h, double mu, const double* D);
__global__ void k_extract_2d(const double2* G, int Q, int H, int nm, double2* S64, float2* S32,
                             __nv_bfloat162* S16);
void make_sched(FftSched* s, int Q);
int choose_Q(int n);

// op2d.cu : out = a*x + b*(K x) + c*z   (K replaced by K~g for MIX_RHS)
rte_status op2d_apply64(rte_plan p, MixKind kind, const double* x, const double* xin_real,
                        double* out, double a, double b, double c, const double* z, cudaStream_t s);
rte_status op2d_apply32(rte_plan p, const float* x, float* out, float a, float b, float c,
                        const float* z, cudaStream_t s);
rte_status op2d_time64(rte_plan p, int reps, double* ms, cudaStream_t s);
rte_status op2d_time_ff(rte_plan p, int reps, double* ms, cudaStream_t s);
rte_status op2d_permute_spectra(rte_plan p, cudaStream_t s);
// op2d_ff.cu / op3d.cu: FP64-accurate applications in float-float arithmetic
rte_status op2d_apply_ff(rte_plan p, MixKind kind, const double* x, const double* f, double* out, double a, double b,
                         double c, const double* z, cudaStream_t s);
rte_status op3d_apply_ff(rte_plan p, MixKind kind, const double* x, double* out, double a, double b, double c,
                         const double* z, cudaStream_t s);
rte_status plan_split_ff(rte_plan p, cudaStream_t s);
rte_status plan_apply64e(rte_plan p, MixKind kind, const double* x, double* out, double a, double b, double c,
                         const double* z, cudaStream_t s);
rte_status op2d_time32(rte_plan p, int reps, double* ms, cudaStream_t s);
// op2d_64.cu: the FP64 passes on explicit buffers (no plan-owned scratch)
rte_status op2d_apply64_buffers(rte_plan p, const double* x, double* out, double2* Tb, const double2* S64,
                                const double2* tw64, cudaStream_t s);
// op3d.cu
rte_status op3d_apply64(rte_plan p, MixKind kind, const double* x, double* out, double a, double b,
                        double c, const double* z, cudaStream_t s);
// precond.cu
bool plan_precond_supported(const rte_plan p);
rte_status plan_precond_build(rte_plan p, cudaStream_t s);
rte_status plan_apply_pc32(rte_plan p, const float* x, float* out, cudaStream_t s);
rte_status plan_time_pc(rte_plan p, int reps, double* ms, cudaStream_t s);
// w = A M v and pv = M v for one preconditioned inner step (FP32)
rte_status plan_apply_pcA32(rte_plan p, const float* v, float* pv, float* w, cudaStream_t s);
rte_status op2d_apply32_stage(rte_plan p, const float* x, float* out, float a, float b, float c, int stage,
                              cudaStream_t s);
cudaError_t op3d_run_pc32(rte_plan p, const float* x, float* out, cudaStream_t s);
rte_status op3d_apply32(rte_plan p, const float* x, float* out, float a, float b, float c,
                        const float* z, cudaStream_t s);

// krylov.cu: the solve reads p->f_dev and writes p->u_dev
// one solve of the plan's f_dev into u_dev; u_out (optional) receives a copy
// of u_dev of kind `kind`, enqueued before the one synchronisation
rte_status krylov_solve(rte_plan p, const rte_opts* o, rte_stats* st, cudaStream_t s, void* u_out = nullptr,
                        cudaMemcpyKind kind = cudaMemcpyDeviceToDevice);
rte_status krylov_free(rte_plan p);
size_t refdev_size();
bool solve_uses_minres(const rte_plan p, const rte_opts* o);
bool solve_uses_precond(const rte_plan p, const rte_opts* o);
rte_status solve_graph_append(rte_plan p, int prec, int m, bool minres, bool pc, cudaGraph_t g,
                              cudaGraphNode_t* dep, cudaStream_t cs, SolveGraphInfo* info);
rte_status solve_set_options(rte_plan p, const rte_opts* o, cudaStream_t s);
struct RefDev;
rte_status solve_collect(rte_plan p, int prec, const RefDev* host_ref, rte_stats* stats, double ms);
void launch_ref_load(rte_plan p, const void* tmpl, cudaStream_t s);
void launch_ref_store(rte_plan p, void* dst, cudaStream_t s);
void launch_copy(const double* src, double* dst, long n, cudaStream_t s);
void fill_ref_template(void* host, const rte_opts* o);

// dispatch helpers (rte_api.cu)
rte_status plan_apply64(rte_plan p, MixKind kind, const double* x, double* out, double a, double b,
                        double c, const double* z, cudaStream_t s);
rte_status op2d_rhs32(rte_plan p, float* out, cudaStream_t s);
rte_status op3d_rhs32(rte_plan p, float* f32, float* out, cudaStream_t s);
rte_status plan_rhs32(rte_plan p, float* out, cudaStream_t s);
rte_status plan_apply32(rte_plan p, const float* x, float* out, float a, float b, float c,
                        const float* z, cudaStream_t s);
