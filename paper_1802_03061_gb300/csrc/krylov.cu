// Device GMRES (Saad & Schultz) for (I - K) u = b, plus the mixed-precision
// iterative refinement driver.
//
// The paper solves step T.2 (Sec. 3.3.1) -- and S.2 for L = 0 (Sec. 2.3.1) --
// with GMRES/MINRES on the FFT matvec.  Here the Krylov vectors are the real
// channels of J-symmetric fields (u_{-k} = conj(u_k)), with the inner
// product of the full complex vector over modes -L..L:
//   <u, v> = sum_{mode 0} u v + 2 sum_{modes k>=1} Re(conj(u_k) v_k),
// so residual norms equal those of the paper's NM-dimensional system.
//
// Arnoldi: classical Gram-Schmidt with one re-orthogonalisation (CGS2) as
// multi-dot / multi-axpy kernels over the basis; the Hessenberg column,
// Givens rotations and the residual estimate live in device memory (FP64)
// and are updated by a one-thread kernel.  One Arnoldi step is captured once
// into a CUDA graph (every kernel reads the step index from device memory)
// and replayed; the host reads a 16-byte status word after each step.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "internal.h"

#define GM_MMAX 128
#define DOT_CHUNK 8
#define DOT_NBLK 304  // 2 x 152 SMs

struct GmresDev {
    int j;          // index of the basis vector being orthogonalised against (step j builds V_{j+1})
    int its;        // iterations in this solve
    int stop;       // 1: end of cycle (converged, breakdown or j == m)
    int conv;       // 1: estimated residual <= target
    int m;          // restart length
    int pad;
    double target;  // absolute residual target tol * ||b||
    double beta;
    double res;     // |g_{j+1}|, the residual estimate
    double cs[GM_MMAX], sn[GM_MMAX], g[GM_MMAX + 1];
    double Hc[(GM_MMAX + 1) * GM_MMAX];  // H[i + j*(m+1)]
    double hA[GM_MMAX + 1], hB[GM_MMAX + 1], y[GM_MMAX];
    double nrm;     // scratch scalar (norm results)
};

// --------------------------------------------------------------------------
// vector kernels (T = float or double storage; FP64 accumulation)
// --------------------------------------------------------------------------
// part[i * nblk + blk] = sum_{e in blk} wt(e) V_i[e] w[e],  i < count
// count = (*cnt_src) + cnt_add ; elements e < nw1 have weight 1, others 2
template <typename T>
__global__ void __launch_bounds__(256) k_dot_part(const T* __restrict__ V, long nr, const T* __restrict__ w,
                                                  const int* __restrict__ cnt_src, int cnt_add, long nw1,
                                                  double* __restrict__ part) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    const int i0 = blockIdx.y * DOT_CHUNK;
    if (i0 >= count) return;
    const int ni = min(DOT_CHUNK, count - i0);
    double acc[DOT_CHUNK];
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; ++i) acc[i] = 0.0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x) {
        const double we = (double)w[e] * (e < nw1 ? 1.0 : 2.0);
#pragma unroll
        for (int i = 0; i < DOT_CHUNK; ++i)
            if (i < ni) acc[i] += (double)V[(long)(i0 + i) * nr + e] * we;
    }
    __shared__ double red[DOT_CHUNK][256 / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < DOT_CHUNK; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[i][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < ni) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += red[threadIdx.x][q];
        part[(long)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
    }
}

// out[i] = sum_b part[i][b] for i < count (fixed order); optional sqrt of out[0]
__global__ void k_dot_finish(const double* __restrict__ part, int nblk, const int* __restrict__ cnt_src,
                             int cnt_add, double* __restrict__ out, int do_sqrt) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    __shared__ double red[256];
    for (int i = 0; i < count; ++i) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) t += part[(long)i * nblk + b];
        red[threadIdx.x] = t;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[i] = do_sqrt ? sqrt(red[0]) : red[0];
        __syncthreads();
    }
}

// w[e] += sgn * sum_{i < count} coef[i] V_i[e]
template <typename T>
__global__ void __launch_bounds__(256) k_multi_axpy(const T* __restrict__ V, long nr, T* __restrict__ w,
                                                    const double* __restrict__ coef, const int* __restrict__ cnt_src,
                                                    int cnt_add, double sgn) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < count; ++i) acc += coef[i] * (double)V[(long)i * nr + e];
        w[e] = (T)((double)w[e] + sgn * acc);
    }
}

// w[e] = rhs[e] - w[e]
template <typename T>
__global__ void k_rsub(const T* __restrict__ rhs, T* __restrict__ w, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        w[e] = rhs[e] - w[e];
}

// u[e] += d[e]
__global__ void k_add64(double* __restrict__ u, const double* __restrict__ d, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        u[e] += d[e];
}

// dst[e] = src[e] * (1 / *s)   (0 if *s == 0)
template <typename T, typename U>
__global__ void k_scale_inv(const T* __restrict__ src, U* __restrict__ dst, long nr, const double* __restrict__ s) {
    const double inv = (*s != 0.0) ? 1.0 / *s : 0.0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = (U)((double)src[e] * inv);
}

// dst = V_{j+1} slot: pointer computed from device j
template <typename T>
__global__ void k_scale_to_basis(const T* __restrict__ w, T* __restrict__ V, long nr, const GmresDev* __restrict__ st) {
    const int j = st->j;
    const double nrm = st->hA[j + 1];
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    T* dst = V + (long)(j + 1) * nr;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = (T)((double)w[e] * inv);
}

// copy V_j into the matvec input is not needed: the matvec reads V + j*nr via
// this pointer-producing trick -- the operator kernels take a fixed pointer,
// so the Arnoldi step first copies V_j to a fixed slot.
template <typename T>
__global__ void k_copy_vj(const T* __restrict__ V, T* __restrict__ dst, long nr, const GmresDev* __restrict__ st) {
    const T* src = V + (long)st->j * nr;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = src[e];
}

// Init a cycle: V_0 = r / ||r||, g = (beta, 0, ...)
__global__ void k_cycle_init(GmresDev* st, int m, double target) {
    st->j = 0;
    st->m = m;
    st->stop = 0;
    st->conv = 0;
    st->target = target;
    st->beta = st->nrm;
    st->res = st->nrm;
    for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
    st->g[0] = st->nrm;
    if (!(st->nrm > target)) { st->stop = 1; st->conv = 1; }
    if (!isfinite(st->nrm)) { st->stop = 1; st->conv = 0; }
}

// One Givens update after the CGS2 column h = hA + hB (entries 0..j), h_{j+1} = ||w||
__global__ void k_givens(GmresDev* st) {
    const int j = st->j, m = st->m, ld = m + 1;
    double* Hc = st->Hc + (long)j * ld;
    for (int i = 0; i <= j; ++i) Hc[i] = st->hA[i] + st->hB[i];
    const double hn = st->nrm;
    Hc[j + 1] = hn;
    st->hA[j + 1] = hn;  // read by the basis scaling kernel
    for (int i = 0; i < j; ++i) {
        const double t = st->cs[i] * Hc[i] + st->sn[i] * Hc[i + 1];
        Hc[i + 1] = -st->sn[i] * Hc[i] + st->cs[i] * Hc[i + 1];
        Hc[i] = t;
    }
    const double a = Hc[j], b = Hc[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    st->cs[j] = c;
    st->sn[j] = s;
    Hc[j] = r;
    Hc[j + 1] = 0.0;
    st->g[j + 1] = -s * st->g[j];
    st->g[j] = c * st->g[j];
    st->res = fabs(st->g[j + 1]);
    st->its += 1;
    if (st->res <= st->target) { st->stop = 1; st->conv = 1; }
    if (!(hn > 1e-300) || !isfinite(st->res)) st->stop = 1;  // breakdown / non-finite
    if (j + 1 >= m) st->stop = 1;
}

// after the step: advance j unless the cycle stopped
__global__ void k_advance(GmresDev* st) {
    st->j += 1;  // number of columns = j afterwards
}

// back substitution H(0:k,0:k) y = g(0:k), k = j (number of columns)
__global__ void k_solve_tri(GmresDev* st) {
    const int k = st->j, ld = st->m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double t = st->g[i];
        for (int q = i + 1; q < k; ++q) t -= st->Hc[i + (long)q * ld] * st->y[q];
        const double d = st->Hc[i + (long)i * ld];
        st->y[i] = d != 0.0 ? t / d : 0.0;
    }
}

// u += scale * dvec (FP64 u, T-typed d), then optional scaling
template <typename T>
__global__ void k_axpy_scaled(double* __restrict__ u, const T* __restrict__ d, long nr, const double* __restrict__ sc) {
    const double a = *sc;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        u[e] += a * (double)d[e];
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
static int grid_for(long nr) {
    long g = (nr + 255) / 256;
    return (int)(g < 1216 ? (g < 1 ? 1 : g) : 1216);
}

template <typename T> struct Gm {
    rte_plan p;
    KrylovWs* ws;
    T* V;
    T* w;
    T* vin;        // fixed matvec input slot
    GmresDev* st;  // device state
    double* part;
    long nr, nw1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// norm of a vector into st->nrm (weighted)
template <typename T>
static rte_status dev_norm(const T* v, long nr, long nw1, double* part, double* out, cudaStream_t s) {
    dim3 g(DOT_NBLK, 1);
    k_dot_part<T><<<g, 256, 0, s>>>(v, nr, v, nullptr, 1, nw1, part);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_dot_finish<<<1, 256, 0, s>>>(part, DOT_NBLK, nullptr, 1, out, 1);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

static rte_status apply_A_T(rte_plan p, const double* x, double* y, cudaStream_t s) {
    return plan_apply64(p, MIX_K, x, y, 1.0, -1.0, 0.0, nullptr, s);
}
static rte_status apply_A_T(rte_plan p, const float* x, float* y, cudaStream_t s) {
    return plan_apply32(p, x, y, 1.0f, -1.0f, 0.0f, nullptr, s);
}

// enqueue one Arnoldi step (CGS2) for step index st->j
template <typename T>
static rte_status arnoldi_step(Gm<T>& G, cudaStream_t s) {
    const long nr = G.nr;
    const int gr = grid_for(nr);
    k_copy_vj<T><<<gr, 256, 0, s>>>(G.V, G.vin, nr, G.st);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    rte_status e = apply_A_T(G.p, G.vin, G.w, s);
    if (e != RTE_OK) return e;
    const int* jp = &G.st->j;
    const dim3 gd(DOT_NBLK, GM_MMAX / DOT_CHUNK);
    // pass 1
    k_dot_part<T><<<gd, 256, 0, s>>>(G.V, nr, G.w, jp, 1, G.nw1, G.part);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_dot_finish<<<1, 256, 0, s>>>(G.part, DOT_NBLK, jp, 1, G.st->hA, 0);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_multi_axpy<T><<<gr, 256, 0, s>>>(G.V, nr, G.w, G.st->hA, jp, 1, -1.0);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    // pass 2 (re-orthogonalisation)
    k_dot_part<T><<<gd, 256, 0, s>>>(G.V, nr, G.w, jp, 1, G.nw1, G.part);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_dot_finish<<<1, 256, 0, s>>>(G.part, DOT_NBLK, jp, 1, G.st->hB, 0);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_multi_axpy<T><<<gr, 256, 0, s>>>(G.V, nr, G.w, G.st->hB, jp, 1, -1.0);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    // norm, Givens, new basis vector
    rte_status e2 = dev_norm<T>(G.w, nr, G.nw1, G.part, &G.st->nrm, s);
    if (e2 != RTE_OK) return e2;
    k_givens<<<1, 1, 0, s>>>(G.st);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_scale_to_basis<T><<<gr, 256, 0, s>>>(G.w, G.V, nr, G.st);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_advance<<<1, 1, 0, s>>>(G.st);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

template <typename T>
static rte_status gm_setup(Gm<T>& G, rte_plan p, KrylovWs& ws, int m, cudaStream_t s) {
    G.p = p;
    G.ws = &ws;
    G.nr = p->nr;
    G.nw1 = p->dim == 2 ? 2L * p->n * p->n : p->nr;
    if (ws.m != m || !ws.V) {
        if (ws.V) cudaFree(ws.V);
        if (ws.w) cudaFree(ws.w);
        if (ws.part) cudaFree(ws.part);
        if (ws.st) cudaFree(ws.st);
        if (ws.exec) cudaGraphExecDestroy((cudaGraphExec_t)ws.exec);
        ws.exec = nullptr;
        ws.V = ws.w = nullptr;
        ws.part = ws.st = nullptr;
        if (cudaMalloc(&ws.V, (size_t)(m + 2) * p->nr * sizeof(T)) != cudaSuccess) return RTE_ENOMEM;
        if (cudaMalloc(&ws.w, (size_t)p->nr * sizeof(T)) != cudaSuccess) return RTE_ENOMEM;
        if (cudaMalloc((void**)&ws.part, (size_t)(GM_MMAX + 1) * DOT_NBLK * sizeof(double)) != cudaSuccess)
            return RTE_ENOMEM;
        if (cudaMalloc((void**)&ws.st, sizeof(GmresDev)) != cudaSuccess) return RTE_ENOMEM;
        RTE_CUDA_TRY(cudaMemsetAsync(ws.st, 0, sizeof(GmresDev), s));
        ws.m = m;
    }
    G.V = (T*)ws.V;
    G.vin = G.V + (long)(m + 1) * p->nr;  // slot m+1 is the matvec input
    G.w = (T*)ws.w;
    G.st = (GmresDev*)ws.st;
    G.part = ws.part;
    return RTE_OK;
}

struct HostStatus { int j, its, stop, conv; double res; };

static rte_status read_status(const GmresDev* st, HostStatus* hs, double* pinned, cudaStream_t s) {
    RTE_CUDA_TRY(cudaMemcpyAsync(pinned, st, 4 * sizeof(int) + 0, cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaMemcpyAsync(pinned + 2, &st->res, sizeof(double), cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    const int* ip = (const int*)pinned;
    hs->j = ip[0];
    hs->its = ip[1];
    hs->stop = ip[2];
    hs->conv = ip[3];
    hs->res = pinned[2];
    return RTE_OK;
}

// GMRES(m) on A = I - K in precision T: solves A x = rhs, x in/out (T).
// x is assumed zero on entry when x_zero.  Returns iterations in *its.
template <typename T>
static rte_status gmres_T(rte_plan p, KrylovWs& ws, const T* rhs, T* x, bool x_zero, double tol_rel, int m,
                          int maxit, int* its_out, double* relres_est, cudaStream_t s) {
    Gm<T> G;
    rte_status e = gm_setup<T>(G, p, ws, m, s);
    if (e != RTE_OK) return e;
    const long nr = G.nr;
    const int gr = grid_for(nr);
    double* pinned = p->hst;
    // ||rhs||
    e = dev_norm<T>(rhs, nr, G.nw1, G.part, &G.st->nrm, s);
    if (e != RTE_OK) return e;
    RTE_CUDA_TRY(cudaMemcpyAsync(pinned, &G.st->nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    const double bnorm = pinned[0];
    *its_out = 0;
    *relres_est = 0.0;
    if (!(bnorm > 0.0)) {
        if (!isfinite(bnorm)) return RTE_ENAN;
        return RTE_OK;
    }
    const double target = tol_rel * bnorm;
    int its = 0;
    RTE_CUDA_TRY(cudaMemsetAsync(&G.st->its, 0, sizeof(int), s));
    // one Arnoldi step captured once per workspace (kernels read j from device state)
    if (!ws.exec) {
        cudaGraph_t graph = nullptr;
        cudaStream_t cs;
        RTE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        RTE_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const long long before = rte_kernel_launches();
        rte_status ce = arnoldi_step<T>(G, cs);
        const long long captured = rte_kernel_launches() - before;
        rte_count_launches(-captured);  // captured, not executed
        ws.nodes = captured;
        cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (ce != RTE_OK) { if (graph) cudaGraphDestroy(graph); return ce; }
        if (ee != cudaSuccess) return rte_cuda_fail(ee, "capture arnoldi");
        cudaGraphExec_t ex = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return rte_cuda_fail(ie, "instantiate arnoldi");
        ws.exec = ex;
    }
    cudaGraphExec_t exec = (cudaGraphExec_t)ws.exec;
    rte_status result = RTE_OK;
    bool first = true;
    double last_res = bnorm;
    while (true) {
        // r = rhs - A x  -> w  (or rhs when x == 0)
        if (first && x_zero) {
            RTE_CUDA_TRY(cudaMemcpyAsync(G.w, rhs, nr * sizeof(T), cudaMemcpyDeviceToDevice, s));
        } else {
            e = apply_A_T(p, x, G.w, s);
            if (e != RTE_OK) { result = e; break; }
            k_rsub<T><<<gr, 256, 0, s>>>(rhs, G.w, nr);
            rte_count_launches(1);
            RTE_CUDA_TRY(cudaGetLastError());
        }
        first = false;
        e = dev_norm<T>(G.w, nr, G.nw1, G.part, &G.st->nrm, s);
        if (e != RTE_OK) { result = e; break; }
        k_cycle_init<<<1, 1, 0, s>>>(G.st, m, target);
        rte_count_launches(1);
        RTE_CUDA_TRY(cudaGetLastError());
        k_scale_inv<T, T><<<gr, 256, 0, s>>>(G.w, G.V, nr, &G.st->nrm);
        rte_count_launches(1);
        RTE_CUDA_TRY(cudaGetLastError());
        HostStatus hs;
        e = read_status(G.st, &hs, pinned, s);
        if (e != RTE_OK) { result = e; break; }
        last_res = hs.res;
        if (hs.stop) {
            if (!isfinite(hs.res)) result = RTE_ENAN;
            break;  // converged at cycle start (or non-finite)
        }
        int steps = 0;
        while (true) {
            RTE_CUDA_TRY(cudaGraphLaunch(exec, s));
            rte_count_launches(ws.nodes);
            ++steps;
            e = read_status(G.st, &hs, pinned, s);
            if (e != RTE_OK) { result = e; break; }
            if (hs.stop || its + steps >= maxit) break;
        }
        if (result != RTE_OK) break;
        its += steps;
        last_res = hs.res;
        // x += V y
        k_solve_tri<<<1, 1, 0, s>>>(G.st);
        rte_count_launches(1);
        RTE_CUDA_TRY(cudaGetLastError());
        k_multi_axpy<T><<<gr, 256, 0, s>>>(G.V, nr, x, G.st->y, &G.st->j, 0, 1.0);
        rte_count_launches(1);
        RTE_CUDA_TRY(cudaGetLastError());
        if (!isfinite(hs.res)) { result = RTE_ENAN; break; }
        if (hs.conv) break;
        if (its >= maxit) { result = RTE_ENOCONV; break; }
        // otherwise restart: true residual recomputed at the loop head
    }
    *its_out = its;
    *relres_est = last_res / bnorm;
    return result;
}

// --------------------------------------------------------------------------
// residual helpers (FP64): r = b - (u - K u) = -u + K u + b
// --------------------------------------------------------------------------
static rte_status residual64(rte_plan p, const double* b, const double* u, double* r, cudaStream_t s) {
    return plan_apply64(p, MIX_K, u, r, -1.0, 1.0, 1.0, b, s);
}

static rte_status norm64(rte_plan p, const double* v, double* out_host, cudaStream_t s) {
    const long nw1 = p->dim == 2 ? 2L * p->n * p->n : p->nr;
    double* part = p->k64.part ? p->k64.part : p->k32.part;
    double* dst = p->k64.st ? (double*)&((GmresDev*)p->k64.st)->nrm : (double*)&((GmresDev*)p->k32.st)->nrm;
    rte_status e = dev_norm<double>(v, p->nr, nw1, part, dst, s);
    if (e != RTE_OK) return e;
    RTE_CUDA_TRY(cudaMemcpyAsync(p->hst + 8, dst, sizeof(double), cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    *out_host = p->hst[8];
    return RTE_OK;
}

rte_status krylov_solve(rte_plan p, const double* f, double* u, const rte_opts* o, rte_stats* stats,
                        cudaStream_t s) {
    const long nr = p->nr;
    const int gr = grid_for(nr);
    const int m = o->restart;
    cudaEvent_t ev0, ev1;
    RTE_CUDA_TRY(cudaEventCreate(&ev0));
    RTE_CUDA_TRY(cudaEventCreate(&ev1));
    RTE_CUDA_TRY(cudaEventRecord(ev0, s));
    // workspaces (the FP64 one also provides scratch for norms)
    {
        Gm<double> G64;
        rte_status e = gm_setup<double>(G64, p, p->k64, o->prec == RTE_PREC_FP64 ? m : 1, s);
        if (e != RTE_OK) return e;
    }
    // T.1: b = K~ g in FP64
    rte_status e = plan_apply64(p, MIX_RHS, f, p->b64, 0.0, 1.0, 0.0, nullptr, s);
    if (e != RTE_OK) return e;
    double bnorm = 0.0;
    e = norm64(p, p->b64, &bnorm, s);
    if (e != RTE_OK) return e;
    if (!isfinite(bnorm)) return RTE_ENAN;
    if (!o->use_guess) RTE_CUDA_TRY(cudaMemsetAsync(u, 0, nr * sizeof(double), s));
    int iters = 0, outer = 0;
    double relres = 0.0;
    rte_status result = RTE_OK;
    if (bnorm == 0.0) {
        RTE_CUDA_TRY(cudaMemsetAsync(u, 0, nr * sizeof(double), s));
    } else if (o->prec == RTE_PREC_FP64) {
        // plain FP64 GMRES; restarts recompute the true residual
        double est = 0.0;
        int its = 0;
        // solve A d = r with r = b - A u0, then u = u0 + d (handles a guess uniformly)
        e = residual64(p, p->b64, u, p->r64, s);
        if (e != RTE_OK) return e;
        RTE_CUDA_TRY(cudaMemsetAsync(p->x64, 0, nr * sizeof(double), s));
        double rn = 0.0;
        e = norm64(p, p->r64, &rn, s);
        if (e != RTE_OK) return e;
        if (rn > o->tol * bnorm) {
            const double tol_in = o->tol * bnorm / rn;
            result = gmres_T<double>(p, p->k64, p->r64, p->x64, true, tol_in * 0.5, m, o->maxit, &its, &est, s);
            k_add64<<<gr, 256, 0, s>>>(u, p->x64, nr);
            rte_count_launches(1);
            RTE_CUDA_TRY(cudaGetLastError());
        }
        iters = its;
        e = residual64(p, p->b64, u, p->r64, s);
        if (e != RTE_OK) return e;
        e = norm64(p, p->r64, &rn, s);
        if (e != RTE_OK) return e;
        relres = rn / bnorm;
    } else {
        // mixed: FP64 residual, FP32 inner GMRES on the unit-scaled residual, FP64 update
        const int max_outer = 40;
        while (true) {
            e = residual64(p, p->b64, u, p->r64, s);
            if (e != RTE_OK) return e;
            double rn = 0.0;
            e = norm64(p, p->r64, &rn, s);
            if (e != RTE_OK) return e;
            relres = rn / bnorm;
            if (!isfinite(rn)) { result = RTE_ENAN; break; }
            if (relres <= o->tol) break;
            if (outer >= max_outer || iters >= o->maxit) { result = RTE_ENOCONV; break; }
            // r32 = r / ||r||
            p->hst[9] = rn;
            RTE_CUDA_TRY(cudaMemcpyAsync(p->dscal, p->hst + 9, sizeof(double), cudaMemcpyHostToDevice, s));
            k_scale_inv<double, float><<<gr, 256, 0, s>>>(p->r64, p->r32, nr, p->dscal);
            rte_count_launches(1);
            RTE_CUDA_TRY(cudaGetLastError());
            float* d32 = p->d32;
            RTE_CUDA_TRY(cudaMemsetAsync(d32, 0, nr * sizeof(float), s));
            int its = 0;
            double est = 0.0;
            double tin = o->inner_tol;
            // never ask the inner solve for more than the outer target needs
            const double need = o->tol / relres * 0.5;
            if (need > tin) tin = need;
            rte_status ie = gmres_T<float>(p, p->k32, p->r32, d32, true, tin, m, o->maxit - iters, &its, &est, s);
            iters += its;
            ++outer;
            if (ie != RTE_OK && ie != RTE_ENOCONV) { result = ie; break; }
            // u += rn * d32
            k_axpy_scaled<float><<<gr, 256, 0, s>>>(u, d32, nr, p->dscal);
            rte_count_launches(1);
            RTE_CUDA_TRY(cudaGetLastError());
        }
    }
    RTE_CUDA_TRY(cudaEventRecord(ev1, s));
    RTE_CUDA_TRY(cudaEventSynchronize(ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (stats) {
        const double rho = p->mu_t > 0 ? p->mu_s / p->mu_t : 0.0;
        const double cond = rho < 1.0 ? (1.0 + rho) / (1.0 - rho) : INFINITY;
        stats->iters = iters;
        stats->outer = outer;
        stats->relres_true = relres;
        stats->converged = relres <= o->tol ? 1 : 0;
        stats->ms_total = ms;
        stats->ms_pre = p->ms_pre;
        stats->est_err_bound = cond * relres;
    }
    if (result == RTE_OK && !(relres <= o->tol)) result = RTE_ENOCONV;
    return result;
}

rte_status krylov_free(rte_plan p) {
    KrylovWs* w[2] = {&p->k64, &p->k32};
    for (int i = 0; i < 2; ++i) {
        if (w[i]->V) cudaFree(w[i]->V);
        if (w[i]->w) cudaFree(w[i]->w);
        if (w[i]->part) cudaFree(w[i]->part);
        if (w[i]->st) cudaFree(w[i]->st);
        if (w[i]->exec) cudaGraphExecDestroy((cudaGraphExec_t)w[i]->exec);
        *w[i] = KrylovWs();
    }
    return RTE_OK;
}
