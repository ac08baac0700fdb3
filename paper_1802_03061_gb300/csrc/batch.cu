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
};

extern "C" rte_status rte_batch_destroy(rte_batch b) {
    if (!b) return RTE_OK;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy((cudaGraphExec_t)b->exec);
    for (rte_plan p : b->plans) rte_destroy(p);
    if (b->f_all) cudaFree(b->f_all);
    if (b->u_all) cudaFree(b->u_all);
    if (b->ref_tmpl) cudaFree(b->ref_tmpl);
    if (b->ref_all) cudaFree(b->ref_all);
    if (b->ref_host) cudaFreeHost(b->ref_host);
    if (b->tmpl_host) cudaFreeHost(b->tmpl_host);
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
    if (cudaMalloc((void**)&b->f_all, b->f_off[count] * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&b->u_all, b->u_off[count] * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->ref_tmpl, b->ref_sz) != cudaSuccess || cudaMalloc(&b->ref_all, b->ref_sz * count) != cudaSuccess ||
        cudaMallocHost(&b->ref_host, b->ref_sz * count) != cudaSuccess ||
        cudaMallocHost(&b->tmpl_host, b->ref_sz) != cudaSuccess) {
        cudaGetLastError();
        rte_batch_destroy(b);
        return RTE_ENOMEM;
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

extern "C" rte_status rte_batch_solve(rte_batch b, const double* f_packed, double* u_packed, rte_stats* stats,
                                      double* ms_out, void* stream) {
    if (!b || !f_packed || !u_packed) return RTE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    fill_ref_template(b->tmpl_host, &b->opts);
    RTE_CUDA_TRY(cudaMemcpyAsync(b->ref_tmpl, b->tmpl_host, b->ref_sz, cudaMemcpyHostToDevice, s));
    RTE_CUDA_TRY(cudaMemcpyAsync(b->f_all, f_packed, b->f_off[b->count] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    RTE_CUDA_TRY(cudaEventCreate(&e0));
    RTE_CUDA_TRY(cudaEventCreate(&e1));
    RTE_CUDA_TRY(cudaEventRecord(e0, s));
    RTE_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)b->exec, s));
    RTE_CUDA_TRY(cudaEventRecord(e1, s));
    RTE_CUDA_TRY(cudaMemcpyAsync(u_packed, b->u_all, b->u_off[b->count] * sizeof(double), cudaMemcpyDeviceToDevice, s));
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

extern "C" rte_status rte_batch_plan(rte_batch b, int i, rte_plan* out) {
    if (!b || !out || i < 0 || i >= b->count) return RTE_EINVAL;
    *out = b->plans[i];
    return RTE_OK;
}
