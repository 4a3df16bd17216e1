// k_ax1_impl.cuh -- launchers of the element-wise kernels of passes 1 and 5
// (gradient / CG direction update, divergence / CG residual update).
#pragma once
#include "launch.h"

namespace dbfft {

// resident blocks per SM of a kernel at PW_THREADS threads (queried once)
template <typename K>
int pw_resident(K kern) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, PW_THREADS, 0) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 4;
    }
    return n;
}

template <typename T, int NC>
cudaError_t launch_grad_nc(int mode, const Ax1InvArgs<T>& a, cudaStream_t s) {
    const dim3 grid((unsigned)pw_blocks(a.d.H, a.d.B), (unsigned)a.d.B);
    // (two whole waves of resident blocks measured slower at 256^3: 0.229 against 0.216 ms)
    if (mode == AX1_CG) return launch_k(k_grad<T, NC, AX1_CG>, grid, dim3(PW_THREADS), 0, s, a);
    k_grad<T, NC, AX1_PLAIN><<<grid, PW_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int NC>
cudaError_t launch_div_nc(int mode, const Ax1FwdArgs<T>& a, cudaStream_t s) {
    const dim3 grid((unsigned)pw_blocks(a.d.H, a.d.B), (unsigned)a.d.B);
    // the CG form runs one whole wave: its block reduction and last-block hand-off
    // then cover twice the frequencies per block (measured faster at 256^3)
    if (mode == AX5_CG) {
        static const int occ = pw_resident(k_div<T, NC, AX5_CG>);
        return launch_k(k_div<T, NC, AX5_CG>, dim3((unsigned)pw_blocks_resident(a.d.H, a.d.B, 1, occ), (unsigned)a.d.B),
                        dim3(PW_THREADS), 0, s, a);
    }
    if (mode == AX5_RESID) k_div<T, NC, AX5_RESID><<<grid, PW_THREADS, 0, s>>>(a);
    else k_div<T, NC, AX5_PLAIN><<<grid, PW_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dbfft
