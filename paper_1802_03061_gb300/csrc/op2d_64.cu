// FP64 instantiation of the 2D passes (FP64 spectra).
#include "op2d_launch.cuh"

rte_status op2d_apply64(rte_plan p, MixKind kind, const double* x, const double* f, double* out, double a,
                        double b, double c, const double* z, cudaStream_t s) {
    cudaError_t e = op2d_run<double2, double2>(
        p, kind, reinterpret_cast<const double2*>(x), f, reinterpret_cast<double2*>(out), a, b, c,
        reinterpret_cast<const double2*>(z), reinterpret_cast<double2*>(p->T64),
        reinterpret_cast<double2*>(p->Tsplit), p->S64, p->tw64, p->col_split64, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply64");
    return RTE_OK;
}

rte_status op2d_time64(rte_plan p, int reps, double* ms, cudaStream_t s) {
    cudaError_t e = op2d_time<double2, double2>(
        p, reinterpret_cast<const double2*>(p->x64), reinterpret_cast<double2*>(p->t64),
        reinterpret_cast<double2*>(p->T64), reinterpret_cast<double2*>(p->Tsplit), p->S64, p->tw64,
        p->col_split64, reps, ms, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_time64");
    return RTE_OK;
}

rte_status op2d_apply64_buffers(rte_plan p, const double* x, double* out, double2* Tb, const double2* S64,
                                const double2* tw64, cudaStream_t s) {
    cudaError_t e = op2d_run<double2, double2, double2>(p, MIX_K, reinterpret_cast<const double2*>(x), nullptr,
                                               reinterpret_cast<double2*>(out), 0.0, 1.0, 0.0, nullptr, Tb,
                                               nullptr, S64, tw64, false, s);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply64_buffers");
    return RTE_OK;
}
