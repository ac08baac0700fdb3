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
// Arnoldi: classical Gram-Schmidt, once (FP32 inner solves) or twice (FP64),
// as a single-pass multi-dot over the basis and a fused multi-axpy + norm.
// The Hessenberg matrix, Givens rotations and residual estimate live in
// device memory (FP64) and are updated by one warp.  A whole restart cycle is
// one CUDA graph: residual, normalisation, then a conditional WHILE node whose
// body is one Arnoldi step (the Givens kernel clears the condition when the
// cycle ends), then the triangular solve and the update of x.  The host waits
// once per cycle.
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "internal.h"

#define GM_MMAX 128
#define TILE 2048   // elements per block in the vector kernels (256 threads x 8)

struct GmresDev {
    int j;       // Arnoldi index (number of finished columns after the step)
    int its;     // iterations in this solve
    int stop;    // 1: end of cycle
    int conv;    // 1: estimated residual <= target
    int m;       // restart length
    int maxit;
    int cgs2;    // 1: re-orthogonalise
    int pad;
    double tol;     // relative tolerance (set by the host before each solve)
    double target;  // absolute residual target tol * ||rhs||
    double beta;
    double res;     // |g_{j}|, the residual estimate
    double nrm;     // last norm result
    double bnorm;   // ||rhs||
    double cs[GM_MMAX], sn[GM_MMAX], g[GM_MMAX + 1];
    double Hc[(GM_MMAX + 1) * GM_MMAX];  // H[i + j*(m+1)]
    double hA[GM_MMAX + 1], hB[GM_MMAX + 1], y[GM_MMAX];
};

// --------------------------------------------------------------------------
// vector kernels (T = float or double storage; FP64 accumulation)
// element e has weight 1 when e < nw1 (mode 0), else 2
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_mdot(const T* __restrict__ V, long nr, const T* __restrict__ w,
                                              const int* __restrict__ cnt_src, int cnt_add, long nw1,
                                              double* __restrict__ part) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    __shared__ double red[GM_MMAX + 1][8];
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    double wv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        wv[q] = e < nr ? (double)w[e] * (e < nw1 ? 1.0 : 2.0) : 0.0;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = 0; i < count; ++i) {
        const T* v = V + (long)i * nr;
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            if (e < nr) s += (double)v[e] * wv[q];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[i][wid] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[i][q];
        part[(long)i * gridDim.x + blockIdx.x] = t;
    }
}

// out[i] = sum_b part[i][b] (fixed order), i < count; one block per i
__global__ void k_reduce(const double* __restrict__ part, int nblk, const int* __restrict__ cnt_src, int cnt_add,
                         double* __restrict__ out, int do_sqrt) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    const int i = blockIdx.x;
    if (i >= count) return;
    __shared__ double red[256];
    double t = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) t += part[(long)i * nblk + b];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = do_sqrt ? sqrt(red[0]) : red[0];
}

// w += sgn * sum_{i<count} coef[i] V_i ; optionally partial ||w||^2 per block
template <typename T>
__global__ void __launch_bounds__(256) k_maxpy(const T* __restrict__ V, long nr, T* __restrict__ w,
                                               const double* __restrict__ coef, const int* __restrict__ cnt_src,
                                               int cnt_add, double sgn, long nw1, double* __restrict__ part) {
    const int count = (cnt_src ? *cnt_src : 0) + cnt_add;
    __shared__ double c[GM_MMAX + 1];
    __shared__ double red[8];
    for (int i = threadIdx.x; i < count; i += blockDim.x) c[i] = sgn * coef[i];
    __syncthreads();
    const long base = (long)blockIdx.x * TILE + threadIdx.x;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int i = 0; i < count; ++i) {
        const T* v = V + (long)i * nr;
        const double ci = c[i];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long e = base + 256 * q;
            if (e < nr) acc[q] += ci * (double)v[e];
        }
    }
    double sq = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long e = base + 256 * q;
        if (e < nr) {
            const T nv = (T)((double)w[e] + acc[q]);
            w[e] = nv;
            sq += (double)nv * (double)nv * (e < nw1 ? 1.0 : 2.0);
        }
    }
    if (part) {
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += red[q];
            part[blockIdx.x] = t;
        }
    }
}

// w = rhs - w
template <typename T>
__global__ void k_rsub(const T* __restrict__ rhs, T* __restrict__ w, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        w[e] = rhs[e] - w[e];
}

// u += d (FP64)
__global__ void k_add64(double* __restrict__ u, const double* __restrict__ d, long nr) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        u[e] += d[e];
}

// dst = src * (1 / *s)  (0 if *s == 0)
template <typename T, typename U>
__global__ void k_scale_inv(const T* __restrict__ src, U* __restrict__ dst, long nr, const double* __restrict__ s) {
    const double inv = (*s != 0.0) ? 1.0 / *s : 0.0;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        dst[e] = (U)((double)src[e] * inv);
}

// u += (*a) * d
template <typename T>
__global__ void k_axpy_scaled(double* __restrict__ u, const T* __restrict__ d, long nr, const double* __restrict__ a) {
    const double s = *a;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x)
        u[e] += s * (double)d[e];
}

// V_{j+off} = w / nrm and the matvec input slot gets the same vector
template <typename T>
__global__ void k_scale_basis(const T* __restrict__ w, T* __restrict__ V, T* __restrict__ vin, long nr,
                              const GmresDev* __restrict__ st, int off) {
    const int slot = st->j + off;
    const double nrm = st->nrm;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    T* dst = V + (long)slot * nr;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nr; e += (long)gridDim.x * blockDim.x) {
        const T v = (T)((double)w[e] * inv);
        dst[e] = v;
        vin[e] = v;
    }
}

// start of a cycle: the residual norm is in st->nrm
__global__ void k_cycle_init(GmresDev* st, int first, cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0) return;
    const double nrm = st->nrm;
    if (first) {
        st->bnorm = nrm;
        st->target = st->tol * nrm;
    }
    st->j = 0;
    st->stop = 0;
    st->conv = 0;
    st->beta = nrm;
    st->res = nrm;
    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
    st->g[0] = nrm;
    bool skip = false;
    if (!isfinite(nrm)) { st->stop = 1; skip = true; }
    else if (!(nrm > st->target)) { st->stop = 1; st->conv = 1; skip = true; }
    if (st->its >= st->maxit) { st->stop = 1; skip = true; }
    cudaGraphSetConditional(loop, skip ? 0u : 1u);
}

// One Givens update; column h = hA (+ hB), h_{j+1} = st->nrm.  One warp.
__global__ void k_givens(GmresDev* st, cudaGraphConditionalHandle loop) {
    __shared__ double col[GM_MMAX + 2], cs[GM_MMAX], sn[GM_MMAX];
    const int j = st->j, m = st->m, ld = m + 1;
    const int two = st->cgs2;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = st->hA[i] + (two ? st->hB[i] : 0.0);
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        cs[i] = st->cs[i];
        sn[i] = st->sn[i];
    }
    __syncwarp();
    if (threadIdx.x != 0) return;
    const double hn = st->nrm;
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double a = col[j], b = col[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    st->cs[j] = c;
    st->sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    double* Hc = st->Hc + (long)j * ld;
    for (int i = 0; i <= j + 1; ++i) Hc[i] = col[i];
    const double gj = st->g[j];
    st->g[j + 1] = -s * gj;
    st->g[j] = c * gj;
    st->res = fabs(st->g[j + 1]);
    st->its += 1;
    st->j = j + 1;
    int stop = 0;
    if (st->res <= st->target) { stop = 1; st->conv = 1; }
    if (!(hn > 1e-300) || !isfinite(st->res)) stop = 1;  // breakdown or non-finite
    if (j + 1 >= m || st->its >= st->maxit) stop = 1;
    st->stop = stop;
    cudaGraphSetConditional(loop, stop ? 0u : 1u);
}

// back substitution H(0:k,0:k) y = g(0:k), k = st->j
__global__ void k_solve_tri(GmresDev* st) {
    if (threadIdx.x != 0) return;
    const int k = st->j, ld = st->m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double t = st->g[i];
        for (int q = i + 1; q < k; ++q) t -= st->Hc[i + (long)q * ld] * st->y[q];
        const double d = st->Hc[i + (long)i * ld];
        st->y[i] = d != 0.0 ? t / d : 0.0;
    }
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
static int grid_for(long nr) {
    long g = (nr + 255) / 256;
    return (int)(g < 1216 ? (g < 1 ? 1 : g) : 1216);
}
static int tiles(long nr) { return (int)((nr + TILE - 1) / TILE); }

static rte_status apply_A_T(rte_plan p, const double* x, double* y, cudaStream_t s) {
    return plan_apply64(p, MIX_K, x, y, 1.0, -1.0, 0.0, nullptr, s);
}
static rte_status apply_A_T(rte_plan p, const float* x, float* y, cudaStream_t s) {
    return plan_apply32(p, x, y, 1.0f, -1.0f, 0.0f, nullptr, s);
}

template <typename T> struct Gm {
    rte_plan p;
    KrylovWs* ws;
    T* V;
    T* w;
    T* vin;
    GmresDev* st;
    double* part;
    long nr, nw1;
    int m;
};

// weighted norm of v into *out (device)
template <typename T>
static rte_status dev_norm(const T* v, long nr, long nw1, double* part, double* out, cudaStream_t s) {
    const int nb = tiles(nr);
    k_mdot<T><<<nb, 256, 0, s>>>(v, nr, v, nullptr, 1, nw1, part);
    RTE_CUDA_TRY(cudaGetLastError());
    k_reduce<<<1, 256, 0, s>>>(part, nb, nullptr, 1, out, 1);
    RTE_CUDA_TRY(cudaGetLastError());
    rte_count_launches(2);
    return RTE_OK;
}

// one Arnoldi step (graph body)
template <typename T>
static rte_status arnoldi_body(Gm<T>& G, bool cgs2, cudaGraphConditionalHandle loop, cudaStream_t s) {
    const long nr = G.nr;
    const int nb = tiles(nr), gr = grid_for(nr);
    rte_status e = apply_A_T(G.p, G.vin, G.w, s);
    if (e != RTE_OK) return e;
    const int* jp = &G.st->j;
    k_mdot<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, jp, 1, G.nw1, G.part);
    RTE_CUDA_TRY(cudaGetLastError());
    k_reduce<<<G.m + 1, 256, 0, s>>>(G.part, nb, jp, 1, G.st->hA, 0);
    RTE_CUDA_TRY(cudaGetLastError());
    rte_count_launches(2);
    if (cgs2) {
        k_maxpy<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, G.st->hA, jp, 1, -1.0, G.nw1, nullptr);
        RTE_CUDA_TRY(cudaGetLastError());
        k_mdot<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, jp, 1, G.nw1, G.part);
        RTE_CUDA_TRY(cudaGetLastError());
        k_reduce<<<G.m + 1, 256, 0, s>>>(G.part, nb, jp, 1, G.st->hB, 0);
        RTE_CUDA_TRY(cudaGetLastError());
        k_maxpy<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, G.st->hB, jp, 1, -1.0, G.nw1, G.part);
        RTE_CUDA_TRY(cudaGetLastError());
        rte_count_launches(4);
    } else {
        k_maxpy<T><<<nb, 256, 0, s>>>(G.V, nr, G.w, G.st->hA, jp, 1, -1.0, G.nw1, G.part);
        RTE_CUDA_TRY(cudaGetLastError());
        rte_count_launches(1);
    }
    k_reduce<<<1, 256, 0, s>>>(G.part, nb, nullptr, 1, &G.st->nrm, 1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_scale_basis<T><<<gr, 256, 0, s>>>(G.w, G.V, G.vin, nr, G.st, 1);
    RTE_CUDA_TRY(cudaGetLastError());
    k_givens<<<1, 32, 0, s>>>(G.st, loop);
    RTE_CUDA_TRY(cudaGetLastError());
    rte_count_launches(3);
    return RTE_OK;
}

// sink node of a graph (the node without dependents)
static cudaGraphNode_t graph_sink(cudaGraph_t g) {
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    if (n == 0) return nullptr;
    cudaGraphNode_t* nodes = new cudaGraphNode_t[n];
    cudaGraphGetNodes(g, nodes, &n);
    cudaGraphNode_t last = nullptr;
    for (size_t i = 0; i < n; ++i) {
        size_t nd = 0;
        cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd);
        if (nd == 0) last = nodes[i];
    }
    delete[] nodes;
    return last;
}

// Capture one restart cycle: first = true means x == 0 (residual = rhs).
template <typename T>
static rte_status build_cycle(Gm<T>& G, const T* rhs, T* x, bool first, bool cgs2, cudaGraphExec_t* out,
                              long long* nodes_out, long long* body_nodes_out) {
    const long nr = G.nr;
    const int nb = tiles(nr), gr = grid_for(nr);
    cudaGraph_t g = nullptr;
    RTE_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle loop;
    cudaStream_t cs = nullptr;
    rte_status st = RTE_OK;
    const long long c0 = rte_kernel_launches();
    long long pre = 0, body = 0, post = 0;
    cudaGraphNode_t last = nullptr;
    cudaError_t e = cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { st = rte_cuda_fail(e, "conditional handle"); goto done; }
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { st = rte_cuda_fail(e, "capture stream"); goto done; }
    // head: residual, norm, init, V_0
    e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { st = rte_cuda_fail(e, "capture head"); goto done; }
    if (first) {
        cudaMemcpyAsync(G.w, rhs, nr * sizeof(T), cudaMemcpyDeviceToDevice, cs);
    } else {
        st = apply_A_T(G.p, x, G.w, cs);
        if (st == RTE_OK) {
            k_rsub<T><<<gr, 256, 0, cs>>>(rhs, G.w, nr);
            rte_count_launches(1);
        }
    }
    if (st == RTE_OK) st = dev_norm<T>(G.w, nr, G.nw1, G.part, &G.st->nrm, cs);
    if (st == RTE_OK) {
        k_cycle_init<<<1, 32, 0, cs>>>(G.st, first ? 1 : 0, loop);
        k_scale_basis<T><<<gr, 256, 0, cs>>>(G.w, G.V, G.vin, nr, G.st, 0);
        rte_count_launches(2);
    }
    {
        cudaGraph_t gg = nullptr;
        e = cudaStreamEndCapture(cs, &gg);
    }
    if (st == RTE_OK && e != cudaSuccess) st = rte_cuda_fail(e, "capture head end");
    if (st != RTE_OK) goto done;
    last = graph_sink(g);
    pre = rte_kernel_launches() - c0;
    // WHILE node with the Arnoldi body
    {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode;
        e = cudaGraphAddNode(&wnode, g, &last, nullptr, 1, &cp);
        if (e != cudaSuccess) { st = rte_cuda_fail(e, "add while node"); goto done; }
        cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { st = rte_cuda_fail(e, "capture body"); goto done; }
        const long long b0 = rte_kernel_launches();
        st = arnoldi_body<T>(G, cgs2, loop, cs);
        body = rte_kernel_launches() - b0;
        cudaGraph_t gb = nullptr;
        e = cudaStreamEndCapture(cs, &gb);
        if (st == RTE_OK && e != cudaSuccess) st = rte_cuda_fail(e, "capture body end");
        if (st != RTE_OK) goto done;
        last = wnode;
    }
    // tail: x += V y
    {
        const long long t0 = rte_kernel_launches();
        e = cudaStreamBeginCaptureToGraph(cs, g, &last, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { st = rte_cuda_fail(e, "capture tail"); goto done; }
        k_solve_tri<<<1, 32, 0, cs>>>(G.st);
        k_maxpy<T><<<nb, 256, 0, cs>>>(G.V, nr, x, G.st->y, &G.st->j, 0, 1.0, G.nw1, nullptr);
        rte_count_launches(2);
        cudaGraph_t gt = nullptr;
        e = cudaStreamEndCapture(cs, &gt);
        if (e != cudaSuccess) { st = rte_cuda_fail(e, "capture tail end"); goto done; }
        post = rte_kernel_launches() - t0;
    }
    {
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) { st = rte_cuda_fail(e, "instantiate cycle"); goto done; }
        *out = ex;
        *nodes_out = pre + post;
        *body_nodes_out = body;
    }
done:
    rte_count_launches(-(rte_kernel_launches() - c0));  // captured, not executed
    if (cs) cudaStreamDestroy(cs);
    cudaGraphDestroy(g);
    return st;
}

template <typename T>
static rte_status gm_setup(Gm<T>& G, rte_plan p, KrylovWs& ws, int m, cudaStream_t s) {
    G.p = p;
    G.ws = &ws;
    G.nr = p->nr;
    G.nw1 = p->dim == 2 ? 2L * p->n * p->n : p->nr;
    G.m = m;
    if (ws.m != m || !ws.V) {
        krylov_free_ws(ws);
        if (cudaMalloc(&ws.V, (size_t)(m + 2) * p->nr * sizeof(T)) != cudaSuccess) return RTE_ENOMEM;
        if (cudaMalloc(&ws.w, (size_t)p->nr * sizeof(T)) != cudaSuccess) return RTE_ENOMEM;
        if (cudaMalloc((void**)&ws.part, (size_t)(GM_MMAX + 1) * tiles(p->nr) * sizeof(double)) != cudaSuccess)
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

struct HostStatus { int j, its, stop, conv; double res, bnorm; };

static rte_status read_status(const GmresDev* st, HostStatus* hs, double* pinned, cudaStream_t s) {
    RTE_CUDA_TRY(cudaMemcpyAsync(pinned, st, offsetof(GmresDev, cs), cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    const GmresDev* h = (const GmresDev*)pinned;
    hs->j = h->j;
    hs->its = h->its;
    hs->stop = h->stop;
    hs->conv = h->conv;
    hs->res = h->res;
    hs->bnorm = h->bnorm;
    return RTE_OK;
}

// GMRES(m) on A = I - K in precision T: solves A x = rhs with x = 0 on entry,
// tol relative to ||rhs||.  rhs and x must be the same buffers on every call
// for one workspace (the cycle graphs bind them).
template <typename T>
static rte_status gmres_T(rte_plan p, KrylovWs& ws, const T* rhs, T* x, double tol_rel, int m, int maxit, bool cgs2,
                          int* its_out, double* relres_est, cudaStream_t s) {
    Gm<T> G;
    rte_status e = gm_setup<T>(G, p, ws, m, s);
    if (e != RTE_OK) return e;
    const int key = (int)p->opts.prec * 2 + (cgs2 ? 1 : 0);
    if (!ws.exec_first || ws.key != key || ws.rhs != (const void*)rhs || ws.x != (void*)x) {
        if (ws.exec_first) cudaGraphExecDestroy((cudaGraphExec_t)ws.exec_first);
        if (ws.exec_restart) cudaGraphExecDestroy((cudaGraphExec_t)ws.exec_restart);
        ws.exec_first = ws.exec_restart = nullptr;
        cudaGraphExec_t a = nullptr, b = nullptr;
        e = build_cycle<T>(G, rhs, x, true, cgs2, &a, &ws.nodes_first, &ws.nodes_body);
        if (e != RTE_OK) return e;
        e = build_cycle<T>(G, rhs, x, false, cgs2, &b, &ws.nodes_restart, &ws.nodes_body);
        if (e != RTE_OK) { cudaGraphExecDestroy(a); return e; }
        ws.exec_first = a;
        ws.exec_restart = b;
        ws.key = key;
        ws.rhs = (const void*)rhs;
        ws.x = (void*)x;
    }
    // tolerance, restart, iteration budget into the device state
    GmresDev* h0 = (GmresDev*)(p->hst + 32);
    memset(h0, 0, offsetof(GmresDev, cs));
    h0->m = m;
    h0->maxit = maxit < 1 ? 1 : maxit;
    h0->cgs2 = cgs2 ? 1 : 0;
    h0->tol = tol_rel;
    RTE_CUDA_TRY(cudaMemcpyAsync(G.st, h0, offsetof(GmresDev, cs), cudaMemcpyHostToDevice, s));
    *its_out = 0;
    *relres_est = 0.0;
    rte_status result = RTE_OK;
    HostStatus hs;
    bool first = true;
    int last_its = 0;
    while (true) {
        cudaGraphExec_t ex = (cudaGraphExec_t)(first ? ws.exec_first : ws.exec_restart);
        RTE_CUDA_TRY(cudaGraphLaunch(ex, s));
        e = read_status(G.st, &hs, p->hst + 8, s);
        if (e != RTE_OK) return e;
        rte_count_launches((first ? ws.nodes_first : ws.nodes_restart) + ws.nodes_body * (hs.its - last_its));
        last_its = hs.its;
        first = false;
        if (!isfinite(hs.res)) { result = RTE_ENAN; break; }
        if (hs.conv) break;
        if (hs.its >= maxit) { result = RTE_ENOCONV; break; }
        if (hs.j == 0) { result = RTE_ENOCONV; break; }  // cycle made no step
    }
    *its_out = hs.its;
    *relres_est = hs.bnorm > 0 ? hs.res / hs.bnorm : 0.0;
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
    rte_status e = dev_norm<double>(v, p->nr, nw1, p->part64, p->dscal, s);
    if (e != RTE_OK) return e;
    RTE_CUDA_TRY(cudaMemcpyAsync(p->hst + 4, p->dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    *out_host = p->hst[4];
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
        // plain FP64 GMRES on r = b - A u0 (u0 = guess or 0); u = u0 + d
        double rn = bnorm;
        if (o->use_guess) {
            e = residual64(p, p->b64, u, p->r64, s);
            if (e != RTE_OK) return e;
            e = norm64(p, p->r64, &rn, s);
            if (e != RTE_OK) return e;
        } else {
            RTE_CUDA_TRY(cudaMemcpyAsync(p->r64, p->b64, nr * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        if (rn > o->tol * bnorm) {
            RTE_CUDA_TRY(cudaMemsetAsync(p->x64, 0, nr * sizeof(double), s));
            double est = 0.0;
            int its = 0;
            const double tol_in = o->tol * bnorm / rn * 0.5;
            result = gmres_T<double>(p, p->k64, p->r64, p->x64, tol_in, m, o->maxit, true, &its, &est, s);
            iters = its;
            if (result != RTE_OK && result != RTE_ENOCONV) return result;
            k_add64<<<gr, 256, 0, s>>>(u, p->x64, nr);
            RTE_CUDA_TRY(cudaGetLastError());
            rte_count_launches(1);
        }
        e = residual64(p, p->b64, u, p->r64, s);
        if (e != RTE_OK) return e;
        e = norm64(p, p->r64, &rn, s);
        if (e != RTE_OK) return e;
        relres = rn / bnorm;
    } else {
        // mixed: FP64 residual, FP32 inner GMRES on the unit-scaled residual, FP64 update
        const int max_outer = 40;
        bool u_zero = !o->use_guess;
        while (true) {
            double rn = 0.0;
            if (u_zero) {
                // r = b when u = 0: no FP64 operator application needed
                RTE_CUDA_TRY(cudaMemcpyAsync(p->r64, p->b64, nr * sizeof(double), cudaMemcpyDeviceToDevice, s));
                e = norm64(p, p->r64, &rn, s);
                u_zero = false;
            } else {
                e = residual64(p, p->b64, u, p->r64, s);
                if (e != RTE_OK) return e;
                e = norm64(p, p->r64, &rn, s);
            }
            if (e != RTE_OK) return e;
            relres = rn / bnorm;
            if (!isfinite(rn)) { result = RTE_ENAN; break; }
            if (relres <= o->tol) break;
            if (outer >= max_outer || iters >= o->maxit) { result = RTE_ENOCONV; break; }
            // r32 = r / ||r||   (p->dscal holds ||r|| on the device)
            k_scale_inv<double, float><<<gr, 256, 0, s>>>(p->r64, p->r32, nr, p->dscal);
            RTE_CUDA_TRY(cudaGetLastError());
            RTE_CUDA_TRY(cudaMemsetAsync(p->d32, 0, nr * sizeof(float), s));
            rte_count_launches(1);
            int its = 0;
            double est = 0.0;
            double tin = o->inner_tol;
            // never ask the inner solve for more than the outer target needs
            const double need = o->tol / relres * 0.5;
            if (need > tin) tin = need;
            rte_status ie = gmres_T<float>(p, p->k32, p->r32, p->d32, tin, m, o->maxit - iters, false, &its, &est, s);
            iters += its;
            ++outer;
            if (ie != RTE_OK && ie != RTE_ENOCONV) { result = ie; break; }
            // u += ||r|| d32
            k_axpy_scaled<float><<<gr, 256, 0, s>>>(u, p->d32, nr, p->dscal);
            RTE_CUDA_TRY(cudaGetLastError());
            rte_count_launches(1);
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

void krylov_free_ws(KrylovWs& ws) {
    if (ws.V) cudaFree(ws.V);
    if (ws.w) cudaFree(ws.w);
    if (ws.part) cudaFree(ws.part);
    if (ws.st) cudaFree(ws.st);
    if (ws.exec_first) cudaGraphExecDestroy((cudaGraphExec_t)ws.exec_first);
    if (ws.exec_restart) cudaGraphExecDestroy((cudaGraphExec_t)ws.exec_restart);
    ws = KrylovWs();
}

rte_status krylov_free(rte_plan p) {
    krylov_free_ws(p->k64);
    krylov_free_ws(p->k32);
    return RTE_OK;
}
