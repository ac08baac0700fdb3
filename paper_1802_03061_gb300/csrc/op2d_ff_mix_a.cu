// Float-float mode-mix kernels (split column path), L = 0..5
// (separate units keep each compilation short).
#include "op2d.cuh"
#include "op2d_launch.cuh"

cudaError_t launch_mix_ff_a(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s) {
    const long tot = (long)cp.H * cp.Q;
    const unsigned g = (unsigned)((tot + 255) / 256);
    switch (L) {
        case 0: k_mix_pointwise<0, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        case 1: k_mix_pointwise<1, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        case 2: k_mix_pointwise<2, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        case 3: k_mix_pointwise<3, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        case 4: k_mix_pointwise<4, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        case 5: k_mix_pointwise<5, ffc, ffc><<<g, 256, 0, s>>>(Ts, S, cp); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
