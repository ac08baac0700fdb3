// Float-float mode-mix kernels (split column path), L = 6..7
// (separate units keep each compilation short).
#include "op2d.cuh"
#include "op2d_launch.cuh"

cudaError_t launch_mix_ff_b(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s) {
    const long tot = (long)cp.H * cp.Q;
    const unsigned g = (unsigned)((tot + 255) / 256);
    switch (L) {
        case 6: k_mix_pointwise<6, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        case 7: k_mix_pointwise<7, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
