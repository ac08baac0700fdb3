// Float-float mode-mix kernels (float-float column passes), L = 0..5
// (separate units keep each compilation short).
#include "op2d.cuh"
#include "op2d_launch.cuh"

cudaError_t launch_mix_ff_a(int L, ffc* Ts, const ffc* S, const ColParams& cp, cudaStream_t s) {
    const long tot = (long)cp.H * cp.Q;
    const unsigned g = (unsigned)((tot + 31) / 32);
    switch (L) {
        case 0: k_mix_ff<0><<<g, 128, 0, s>>>(Ts, S, cp); break;
        case 1: k_mix_ff<1><<<g, 128, 0, s>>>(Ts, S, cp); break;
        case 2: k_mix_ff<2><<<g, 128, 0, s>>>(Ts, S, cp); break;
        case 3: k_mix_ff<3><<<g, 128, 0, s>>>(Ts, S, cp); break;
        case 4: k_mix_ff<4><<<g, 128, 0, s>>>(Ts, S, cp); break;
        case 5: k_mix_ff<5><<<g, 128, 0, s>>>(Ts, S, cp); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
