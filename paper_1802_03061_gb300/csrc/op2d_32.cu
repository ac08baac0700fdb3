// FP32 instantiation of the 2D passes (FP32 or BF16 spectra).
#include "op2d_launch.cuh"

rte_status op2d_apply32(rte_plan p, const float* x, float* out, float a, float b, float c, const float* z,
                        cudaStream_t s) {
    cudaError_t e;
    const float2* xx = reinterpret_cast<const float2*>(x);
    const float2* zz = reinterpret_cast<const float2*>(z);
    float2* oo = reinterpret_cast<float2*>(out);
    float2* Tb = reinterpret_cast<float2*>(p->T32);
    float2* Ts = reinterpret_cast<float2*>(p->Tsplit32);
    if (p->opts.prec == RTE_PREC_MIXED_BF16SPEC)
        e = op2d_run<float2, __nv_bfloat162>(p, MIX_K, xx, nullptr, oo, a, b, c, zz, Tb, Ts, p->S16, p->tw32,
                                             p->col_split32, s);
    else
        e = op2d_run<float2, float2>(p, MIX_K, xx, nullptr, oo, a, b, c, zz, Tb, Ts, p->S32, p->tw32,
                                     p->col_split32, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply32");
    return RTE_OK;
}

rte_status op2d_time32(rte_plan p, int reps, double* ms, cudaStream_t s) {
    cudaError_t e;
    const float2* xx = reinterpret_cast<const float2*>(p->r32);
    float2* oo = reinterpret_cast<float2*>(p->d32);
    float2* Tb = reinterpret_cast<float2*>(p->T32);
    float2* Ts = reinterpret_cast<float2*>(p->Tsplit32);
    if (p->opts.prec == RTE_PREC_MIXED_BF16SPEC)
        e = op2d_time<float2, __nv_bfloat162>(p, xx, oo, Tb, Ts, p->S16, p->tw32, p->col_split32, reps, ms, s);
    else
        e = op2d_time<float2, float2>(p, xx, oo, Tb, Ts, p->S32, p->tw32, p->col_split32, reps, ms, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_time32");
    return RTE_OK;
}
