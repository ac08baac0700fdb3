// FP32 passes with BF16 kernel spectra.
#include "op2d_launch.cuh"

rte_status op2d_apply32_bf16(rte_plan p, const float2* x, float2* out, float a, float b, float c, const float2* z,
                             cudaStream_t s) {
    float2* Tb = reinterpret_cast<float2*>(p->T32);
    float2* Ts = reinterpret_cast<float2*>(p->Tsplit32);
    cudaError_t e = op2d_run<float2, __nv_bfloat162>(p, MIX_K, x, nullptr, out, a, b, c, z, Tb, Ts, p->S16, p->tw32,
                                                     p->col_split32, s, -1, p->S16p);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply32_bf16");
    return RTE_OK;
}

rte_status op2d_apply32_bf16_stage(rte_plan p, const float2* x, float2* out, float a, float b, float c, int stage,
                                   cudaStream_t s) {
    float2* Tb = reinterpret_cast<float2*>(p->T32);
    float2* Ts = reinterpret_cast<float2*>(p->Tsplit32);
    cudaError_t e = op2d_run<float2, __nv_bfloat162, float2>(p, MIX_K, x, nullptr, out, a, b, c, nullptr, Tb, Ts, p->S16,
                                                     p->tw32, p->col_split32, s, stage, p->S16p);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply32_bf16_stage");
    return RTE_OK;
}

rte_status op2d_time32_bf16(rte_plan p, int reps, double* ms, cudaStream_t s) {
    const float2* xx = reinterpret_cast<const float2*>(p->r32);
    float2* oo = reinterpret_cast<float2*>(p->d32);
    float2* Tb = reinterpret_cast<float2*>(p->T32);
    float2* Ts = reinterpret_cast<float2*>(p->Tsplit32);
    cudaError_t e = op2d_time<float2, __nv_bfloat162>(p, xx, oo, Tb, Ts, p->S16, p->tw32, p->col_split32, reps, ms, s,
                                                      p->S16p);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_time32_bf16");
    return RTE_OK;
}
