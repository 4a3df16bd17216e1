// k_ax1_impl.cuh -- launchers of the element-wise kernels of passes 1 and 5
// (gradient / CG direction update, divergence / CG residual update).
#pragma once
#include "launch.h"

namespace dbfft {

template <typename T, int NC>
cudaError_t launch_grad_nc(int mode, const Ax1InvArgs<T>& a, cudaStream_t s) {
    const dim3 grid((unsigned)pw_blocks(a.d.H, a.d.B), (unsigned)a.d.B);
    if (mode == AX1_CG) return launch_k(k_grad<T, NC, AX1_CG>, grid, dim3(PW_THREADS), 0, s, a);
    k_grad<T, NC, AX1_PLAIN><<<grid, PW_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int NC>
cudaError_t launch_div_nc(int mode, const Ax1FwdArgs<T>& a, cudaStream_t s) {
    const dim3 grid((unsigned)pw_blocks(a.d.H, a.d.B), (unsigned)a.d.B);
    // the CG form runs one wave: its block reduction and last-block hand-off then
    // cover twice the frequencies per block (measured faster at 64^3 x 6 and 256^3)
    if (mode == AX5_CG)
        return launch_k(k_div<T, NC, AX5_CG>, dim3((unsigned)pw_blocks(a.d.H, a.d.B, 1), (unsigned)a.d.B),
                        dim3(PW_THREADS), 0, s, a);
    if (mode == AX5_RESID) k_div<T, NC, AX5_RESID><<<grid, PW_THREADS, 0, s>>>(a);
    else k_div<T, NC, AX5_PLAIN><<<grid, PW_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dbfft
