// Batched solves of many independent 2D instances of uneven size in one
// CUDA graph launch.
//
// Every instance gets its own plan (spectra, intermediates, Krylov
// workspace).  The batch graph holds, for every instance, an independent
// branch: copy its source out of the packed input array, the whole
// device-controlled solve (refinement / GMRES / Arnoldi conditional loops),
// copy the solution into the packed output array and the final solver state
// into a packed state array.  The graph executor runs the branches
// concurrently, so small instances fill the GPU together.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "internal.h"

struct rte_batch_s {
    int count = 0;
    int prec = 0;
    int m = 0;
    rte_opts opts;
    std::vector<rte_plan> plans;
    std::vector<long> f_off, u_off;   // count + 1 prefix offsets (doubles)
    std::vector<SolveGraphInfo> info;
    double* f_all = nullptr;
    double* u_all = nullptr;
    void* ref_tmpl = nullptr;         // device options template
    void* ref_all = nullptr;          // device [count] final states
    void* ref_host = nullptr;         // pinned copy of ref_all
    void* tmpl_host = nullptr;        // pinned options template
    size_t ref_sz = 0;
    void* exec = nullptr;
    // rte_batch_solve with one device buffer per instance: the prefix
    // offsets on the device, the two pointer tables (device) and their
    // pinned host staging
    long* off_dev = nullptr;          // [2][count + 1]: f offsets, then u offsets
    void** ptr_dev = nullptr;         // [2][count]: f pointers, then u pointers
    void** ptr_host = nullptr;
};

// dst_base[off[i] + e] = src[i][e] (gather) or dst[i][e] = src_base[off[i] + e]
// (scatter) for every instance i = blockIdx.y
__global__ void k_batch_gather(const double* const* src, const long* off, double* dst_base) {
    const int i = blockIdx.y;
    const long n = off[i + 1] - off[i];
    const double* a = src[i];
    double* d = dst_base + off[i];
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) d[e] = a[e];
}
__global__ void k_batch_scatter(const double* src_base, const long* off, double* const* dst) {
    const int i = blockIdx.y;
    const long n = off[i + 1] - off[i];
    const double* a = src_base + off[i];
    double* d = dst[i];
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) d[e] = a[e];
}

extern "C" rte_status rte_batch_destroy(rte_batch b) {
    if (!b) return RTE_OK;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy((cudaGraphExec_t)b->exec);
    for (rte_plan p : b->plans) rte_destroy(p);
    if (b->f_all) rte_dev_free(b->f_all);
    if (b->u_all) rte_dev_free(b->u_all);
    if (b->ref_tmpl) rte_dev_free(b->ref_tmpl);
    if (b->ref_all) rte_dev_free(b->ref_all);
    if (b->ref_host) rte_host_free(b->ref_host);
    if (b->tmpl_host) rte_host_free(b->tmpl_host);
    if (b->off_dev) rte_dev_free(b->off_dev);
    if (b->ptr_dev) rte_dev_free(b->ptr_dev);
    if (b->ptr_host) rte_host_free(b->ptr_host);
    delete b;
    return RTE_OK;
}

extern "C" rte_status rte_batch_create(rte_batch* out, int count, const rte_instance_desc* descs,
                                       const rte_opts* opts, void* stream) {
    if (!out || count < 1 || !descs) return RTE_EINVAL;
    *out = nullptr;
    rte_batch b = new rte_batch_s();
    rte_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.tol <= 0) o.tol = 1e-8;
    if (o.restart <= 0) o.restart = 30;
    if (o.restart > 128) o.restart = 128;
    if (o.maxit <= 0) o.maxit = 2000;
    if (o.inner_tol <= 0) o.inner_tol = 1e-4;
    if (o.prec < RTE_PREC_FP64 || o.prec > RTE_PREC_MIXED_BF16SPEC) { delete b; return RTE_EINVAL; }
    b->count = count;
    b->opts = o;
    b->prec = (int)o.prec;
    b->m = o.restart;
    b->f_off.assign(count + 1, 0);
    b->u_off.assign(count + 1, 0);
    rte_status st = RTE_OK;
    for (int i = 0; i < count; ++i) {
        const rte_instance_desc& d = descs[i];
        rte_grid g;
        g.dim = 2;
        g.n[0] = g.n[1] = g.n[2] = d.n;
        rte_opts po = o;
        po.q_policy = d.q > 0 ? d.q : o.q_policy;
        rte_plan p = nullptr;
        st = rte_plan_create(&p, g, d.h, d.mu_t, d.mu_s, d.L, d.sigma_hat, &po, stream);
        if (st != RTE_OK) { rte_batch_destroy(b); return st; }
        if (d.rows_per_block > 0) p->rb_force = d.rows_per_block;
        b->plans.push_back(p);
        b->f_off[i + 1] = b->f_off[i] + p->ncell;
        b->u_off[i + 1] = b->u_off[i] + p->nr;
    }
    b->ref_sz = refdev_size();
    if (rte_dev_malloc((void**)&b->f_all, b->f_off[count] * sizeof(double)) != cudaSuccess ||
        rte_dev_malloc((void**)&b->u_all, b->u_off[count] * sizeof(double)) != cudaSuccess ||
        rte_dev_malloc(&b->ref_tmpl, b->ref_sz) != cudaSuccess || rte_dev_malloc(&b->ref_all, b->ref_sz * count) != cudaSuccess ||
        rte_host_malloc(&b->ref_host, b->ref_sz * count) != cudaSuccess ||
        rte_host_malloc(&b->tmpl_host, b->ref_sz) != cudaSuccess ||
        rte_dev_malloc((void**)&b->off_dev, 2 * (count + 1) * sizeof(long)) != cudaSuccess ||
        rte_dev_malloc((void**)&b->ptr_dev, 2 * count * sizeof(void*)) != cudaSuccess ||
        rte_host_malloc((void**)&b->ptr_host, 2 * count * sizeof(void*)) != cudaSuccess) {
        cudaGetLastError();
        rte_batch_destroy(b);
        return RTE_ENOMEM;
    }
    if (cudaMemcpy(b->off_dev, b->f_off.data(), (count + 1) * sizeof(long), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->off_dev + count + 1, b->u_off.data(), (count + 1) * sizeof(long), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        st = rte_cuda_fail(cudaGetLastError(), "rte_batch_create: offsets");
        rte_batch_destroy(b);
        return st;
    }
    // preconditioner data (allocates): before any capture
    for (int i = 0; i < count && st == RTE_OK; ++i)
        if (solve_uses_precond(b->plans[i], &b->opts)) st = plan_precond_build(b->plans[i], (cudaStream_t)stream);
    if (st == RTE_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) st = RTE_ECUDA;
    if (st != RTE_OK) {
        rte_batch_destroy(b);
        return st;
    }
    // build the batch graph: one independent branch per instance
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr;
    b->info.resize(count);
    const long long c0 = rte_kernel_launches();
    if (cudaGraphCreate(&g, 0) != cudaSuccess || cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        rte_batch_destroy(b);
        return RTE_ECUDA;
    }
    for (int i = 0; i < count && st == RTE_OK; ++i) {
        rte_plan p = b->plans[i];
        cudaGraphNode_t dep = nullptr;
        // head: options and source in
        {
            cudaError_t e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) { st = rte_cuda_fail(e, "batch capture"); break; }
            launch_ref_load(p, b->ref_tmpl, cs);
            launch_copy(b->f_all + b->f_off[i], p->f_dev, p->ncell, cs);
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
            dep = nd == 1 ? deps[0] : nullptr;
            cudaGraph_t gg;
            e = cudaStreamEndCapture(cs, &gg);
            if (e != cudaSuccess || nd != 1) { st = rte_cuda_fail(e, "batch capture end"); break; }
        }
        st = solve_graph_append(p, b->prec, b->m, solve_uses_minres(p, &b->opts), solve_uses_precond(p, &b->opts), g,
                                &dep, cs, &b->info[i]);
        if (st != RTE_OK) break;
        // tail: solution and state out
        {
            cudaError_t e = cudaStreamBeginCaptureToGraph(cs, g, &dep, nullptr, 1, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) { st = rte_cuda_fail(e, "batch capture tail"); break; }
            launch_copy(p->u_dev, b->u_all + b->u_off[i], p->nr, cs);
            launch_ref_store(p, (char*)b->ref_all + b->ref_sz * i, cs);
            cudaGraph_t gg;
            e = cudaStreamEndCapture(cs, &gg);
            if (e != cudaSuccess) { st = rte_cuda_fail(e, "batch capture tail end"); break; }
        }
    }
    rte_count_launches(-(rte_kernel_launches() - c0));  // captured, not executed
    if (cs) cudaStreamDestroy(cs);
    if (st == RTE_OK) {
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) st = rte_cuda_fail(e, "batch instantiate");
        else b->exec = ex;
    }
    cudaGraphDestroy(g);
    if (st != RTE_OK) { rte_batch_destroy(b); return st; }
    *out = b;
    return RTE_OK;
}

extern "C" rte_status rte_batch_layout(rte_batch b, long* f_offsets, long* u_offsets) {
    if (!b) return RTE_EINVAL;
    for (int i = 0; i <= b->count; ++i) {
        if (f_offsets) f_offsets[i] = b->f_off[i];
        if (u_offsets) u_offsets[i] = b->u_off[i];
    }
    return RTE_OK;
}

// the graph launch and the statistics, shared by both solve entry points;
// `scatter` (may be null) runs after the graph, before the states come back
static rte_status batch_run(rte_batch b, rte_stats* stats, double* ms_out, cudaStream_t s,
                            rte_status (*scatter)(rte_batch, void*, cudaStream_t), void* scatter_arg) {
    cudaEvent_t e0, e1;
    RTE_CUDA_TRY(cudaEventCreate(&e0));
    RTE_CUDA_TRY(cudaEventCreate(&e1));
    RTE_CUDA_TRY(cudaEventRecord(e0, s));
    RTE_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)b->exec, s));
    RTE_CUDA_TRY(cudaEventRecord(e1, s));
    rte_status sst = scatter(b, scatter_arg, s);
    if (sst != RTE_OK) return sst;
    RTE_CUDA_TRY(cudaMemcpyAsync(b->ref_host, b->ref_all, b->ref_sz * b->count, cudaMemcpyDeviceToHost, s));
    RTE_CUDA_TRY(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_out) *ms_out = ms;
    rte_status worst = RTE_OK;
    rte_count_launches(2L * b->count);  // ref load + copy in/out per branch
    for (int i = 0; i < b->count; ++i) {
        rte_stats one;
        rte_plan p = b->plans[i];
        // per-instance accounting uses the batch graph's segment counts
        const SolveGraphInfo saved = p->graphs[b->prec].info;
        p->graphs[b->prec].info = b->info[i];
        rte_status st = solve_collect(p, b->prec, (const RefDev*)((char*)b->ref_host + b->ref_sz * i), &one, ms);
        p->graphs[b->prec].info = saved;
        if (stats) stats[i] = one;
        if (st != RTE_OK && worst == RTE_OK) worst = st;
    }
    return worst;
}

static rte_status batch_options_in(rte_batch b, cudaStream_t s) {
    fill_ref_template(b->tmpl_host, &b->opts);
    RTE_CUDA_TRY(cudaMemcpyAsync(b->ref_tmpl, b->tmpl_host, b->ref_sz, cudaMemcpyHostToDevice, s));
    return RTE_OK;
}

static rte_status scatter_packed(rte_batch b, void* u_packed, cudaStream_t s) {
    RTE_CUDA_TRY(cudaMemcpyAsync(u_packed, b->u_all, b->u_off[b->count] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return RTE_OK;
}

static rte_status scatter_ptrs(rte_batch b, void*, cudaStream_t s) {
    dim3 grid(64, b->count);
    k_batch_scatter<<<grid, 256, 0, s>>>(b->u_all, b->off_dev + b->count + 1, (double* const*)(b->ptr_dev + b->count));
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
}

extern "C" rte_status rte_batch_solve_packed(rte_batch b, const double* f_packed, double* u_packed, rte_stats* stats,
                                             double* ms_out, void* stream) {
    if (!b || !f_packed || !u_packed) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    rte_status st = batch_options_in(b, s);
    if (st != RTE_OK) return st;
    RTE_CUDA_TRY(cudaMemcpyAsync(b->f_all, f_packed, b->f_off[b->count] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return batch_run(b, stats, ms_out, s, scatter_packed, u_packed);
}

extern "C" rte_status rte_batch_solve(rte_batch b, const double* const* f, void* const* u, rte_stats* stats,
                                      void* stream) {
    if (!b || !f || !u) return RTE_EINVAL;
    for (int i = 0; i < b->count; ++i)
        if (!f[i] || !u[i]) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // the pinned staging is rewritten only after the previous call's copy of
    // it has finished (every solve synchronises the stream before returning)
    for (int i = 0; i < b->count; ++i) {
        b->ptr_host[i] = (void*)f[i];
        b->ptr_host[b->count + i] = u[i];
    }
    rte_status st = batch_options_in(b, s);
    if (st != RTE_OK) return st;
    RTE_CUDA_TRY(cudaMemcpyAsync(b->ptr_dev, b->ptr_host, 2 * b->count * sizeof(void*), cudaMemcpyHostToDevice, s));
    dim3 grid(64, b->count);
    k_batch_gather<<<grid, 256, 0, s>>>((const double* const*)b->ptr_dev, b->off_dev, b->f_all);
    rte_count_launches(1);
    RTE_CUDA_TRY(cudaGetLastError());
    return batch_run(b, stats, nullptr, s, scatter_ptrs, nullptr);
}

extern "C" rte_status rte_batch_plan(rte_batch b, int i, rte_plan* out) {
    if (!b || !out || i < 0 || i >= b->count) return RTE_EINVAL;
    *out = b->plans[i];
    return RTE_OK;
}
