// Float-float instantiation of the 2D passes: FP64-accurate K applications
// (the refinement residual and the right-hand side) on the FP32 units.
// Fields stay FP64 (double2) in memory; intermediates and spectra are
// float-float pairs of the same 16-byte size.
#include "op2d_launch.cuh"

rte_status op2d_apply_ff(rte_plan p, MixKind kind, const double* x, const double* f, double* out, double a, double b,
                         double c, const double* z, cudaStream_t s) {
    cudaError_t e = op2d_run<ffc, ffc, double2>(
        p, kind, reinterpret_cast<const double2*>(x), f, reinterpret_cast<double2*>(out), a, b, c,
        reinterpret_cast<const double2*>(z), reinterpret_cast<ffc*>(p->T64), reinterpret_cast<ffc*>(p->Tsplit),
        p->Sff, p->twff, true, s, -1, p->Sffp);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_apply_ff");
    return RTE_OK;
}

rte_status op2d_time_ff(rte_plan p, int reps, double* ms, cudaStream_t s) {
    cudaError_t e = op2d_time<ffc, ffc, double2>(
        p, reinterpret_cast<const double2*>(p->x64), reinterpret_cast<double2*>(p->t64),
        reinterpret_cast<ffc*>(p->T64), reinterpret_cast<ffc*>(p->Tsplit), p->Sff, p->twff, true, reps, ms, s,
        p->Sffp);
    if (e != cudaSuccess) return rte_cuda_fail(e, "op2d_time_ff");
    return RTE_OK;
}

__global__ void k_split_ff2(const double2* __restrict__ src, ffc* __restrict__ dst, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = to_ffc(src[i]);
}
// the same into the float-float column passes' slot order:
// dst[row][sl] = src[row][slot_freq_ff(sl, Q)]
__global__ void k_split_ff2_slot(const double2* __restrict__ src, ffc* __restrict__ dst, long rows, int Q) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < rows * Q; i += (long)gridDim.x * blockDim.x) {
        const long row = i / Q;
        const int sl = (int)(i % Q);
        dst[i] = to_ffc(src[row * Q + slot_freq_ff(sl, Q)]);
    }
}
__global__ void k_split_ff(const double* __restrict__ src, ff* __restrict__ dst, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = ff(src[i]);
}

// plan time: float-float copies of the twiddles and spectra
rte_status plan_split_ff(rte_plan p, cudaStream_t s) {
    k_split_ff2<<<64, 256, 0, s>>>(p->tw64, p->twff, p->Q);
    if (p->dim == 2) {
        // plans with the mode-axis FFT coupling hold neither copy (their
        // float-float spectra are the mode-axis DFTs, built with them)
        if (p->Sffp) k_split_ff2_slot<<<1024, 256, 0, s>>>(p->S64, p->Sffp, (long)p->H * p->nch, p->Q);
        else if (p->Sff) k_split_ff2<<<1024, 256, 0, s>>>(p->S64, p->Sff, (long)p->H * p->nch * p->Q);
    } else {
        k_split_ff<<<1024, 256, 0, s>>>(p->S3_64, p->S3ff, (long)p->H * p->H * p->H);
    }
    rte_count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rte_cuda_fail(e, "plan_split_ff");
    return RTE_OK;
}
