// FP32 instantiation of the 2D passes: dispatch on the spectra precision
// (FP32 spectra here, BF16 spectra in op2d_32b.cu).
#include "op2d_launch.cuh"

rte_status op2d_apply32_bf16(rte_plan p, const float2* x, float2* out, float a, float b, float c, const float2* z,
                             cudaStream_t s);
rte_status op2d_time32_bf16(rte_plan p, int reps, double* ms, cudaStream_t s);
rte_status op2d_apply32_bf16_stage(rte_plan p, const float2* x, float2* out, float a, float b, float c, int stage,
                                   cudaStream_t s);

rte_status op2d_apply32(rte_plan p, const float* x, float* out, float a, float b, float c, const float* z,
                        cudaStream_t s) {
    const float2* xx = reinterpret_cast<const float2*>(x);
    const float2* zz = reinterpret_cast<const float2*>(z);
    float2* oo = reinterpret_cast<float2*>(out);
    // plans with the mode-axis FFT coupling keep FP32 spectra only
    if (p->opts.prec == RTE_PREC_MIXED_BF16SPEC && !p->mix_fft) return op2d_apply32_bf16(p, xx, oo, a, b, c, zz, s);
    float2* Tb = reinterpret_cast<float2*>(p->T32);
    float2* Ts = reinterpret_cast<float2*>(p->Tsplit32);
    cudaError_t e = op2d_run<float2, float2>(p, MIX_K, xx, nullptr, oo, a, b, c, zz, Tb, Ts, p->S32, p->tw32,
                                             p->col_split32, s, -1, p->S32p);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply32");
    return RTE_OK;
}

// b = K~ f in FP32 (FP32 spectra): the inner solves' first right-hand side
rte_status op2d_rhs32(rte_plan p, float* out, cudaStream_t s) {
    cudaError_t e = op2d_run<float2, float2, float2>(p, MIX_RHS, nullptr, p->f_dev, reinterpret_cast<float2*>(out), 0.0, 1.0,
                                             0.0, nullptr, reinterpret_cast<float2*>(p->T32),
                                             reinterpret_cast<float2*>(p->Tsplit32), p->S32, p->tw32,
                                             p->col_split32, s, -1, p->S32p);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_rhs32");
    return RTE_OK;
}

// one stage of the FP32 application (0 row, 1 column, 2 inverse row + epilogue)
rte_status op2d_apply32_stage(rte_plan p, const float* x, float* out, float a, float b, float c, int stage,
                              cudaStream_t s) {
    const float2* xx = reinterpret_cast<const float2*>(x);
    float2* oo = reinterpret_cast<float2*>(out);
    if (p->opts.prec == RTE_PREC_MIXED_BF16SPEC && !p->mix_fft)
        return op2d_apply32_bf16_stage(p, xx, oo, a, b, c, stage, s);
    cudaError_t e = op2d_run<float2, float2, float2>(p, MIX_K, xx, nullptr, oo, a, b, c, nullptr, reinterpret_cast<float2*>(p->T32),
                                             reinterpret_cast<float2*>(p->Tsplit32), p->S32, p->tw32, p->col_split32,
                                             s, stage, p->S32p);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply32_stage");
    return RTE_OK;
}

rte_status op2d_time32(rte_plan p, int reps, double* ms, cudaStream_t s) {
    if (p->opts.prec == RTE_PREC_MIXED_BF16SPEC && !p->mix_fft) return op2d_time32_bf16(p, reps, ms, s);
    const float2* xx = reinterpret_cast<const float2*>(p->r32);
    float2* oo = reinterpret_cast<float2*>(p->d32);
    float2* Tb = reinterpret_cast<float2*>(p->T32);
    float2* Ts = reinterpret_cast<float2*>(p->Tsplit32);
    cudaError_t e = op2d_time<float2, float2>(p, xx, oo, Tb, Ts, p->S32, p->tw32, p->col_split32, reps, ms, s, p->S32p);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_time32");
    return RTE_OK;
}

// plan time: spectra copies in the warp column pass's slot order
rte_status op2d_permute_spectra(rte_plan p, cudaStream_t s) {
    if (!p->S32p) return RTE_OK;
    const long rows = (long)p->H * p->nch;
    k_permute_spec<float2><<<1024, 256, 0, s>>>(p->S32, p->S32p, rows, p->Q);
    k_permute_spec<__nv_bfloat162><<<1024, 256, 0, s>>>(p->S16, p->S16p, rows, p->Q);
    rte_count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_permute_spectra");
    return RTE_OK;
}
