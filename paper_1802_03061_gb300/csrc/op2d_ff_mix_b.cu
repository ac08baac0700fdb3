// Float-float mode-mix kernels (float-float column passes), L = 6..7
// (separate units keep each compilation short).
#include "op2d.cuh"
#include "op2d_launch.cuh"

cudaError_t launch_mix_ff_b(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s) {
    const long tot = (long)cp.H * cp.Q;
    const unsigned g = (unsigned)((tot + 31) / 32);
    switch (L) {
        case 6: k_mix_ff<6><<<g, 128, 0, s>>>(Ts, S, cp); break;
        case 7: k_mix_ff<7><<<g, 128, 0, s>>>(Ts, S, cp); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
