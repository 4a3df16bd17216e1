// k_ax3_odd_impl.cuh -- launcher of the odd-n3 pass 3 for one (length, components, operation).
#pragma once
#include "launch.h"
#include "pass3_odd.cuh"

namespace dbfft {

template <typename T, int N3, int NC, int OPK>
static cudaError_t ax3_odd_n(const Ax3Args<T>& a0, cudaStream_t s) {
    Ax3Args<T> a = a0;
    a.RB = 1;  // one right-hand side per CTA
    a.L = ax3_odd_lines(N3, NC, sizeof(T) == 8);
    const long long nlines = (long long)a.d.n1 * a.d.n2;
    const size_t smem = (size_t)((NC + 1) / 2) * a.L * 2 * N3 * sizeof(cplx<T>);
    static bool opted = false;
    if (!opted) {
        cudaError_t e = cudaFuncSetAttribute(k_axis3_odd<T, N3, NC, OPK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             96 * 1024);
        if (e != cudaSuccess) return e;
        opted = true;
    }
    const dim3 grid((unsigned)((nlines + a.L - 1) / a.L), (unsigned)a.d.B);
    return launch_k(k_axis3_odd<T, N3, NC, OPK>, grid, dim3(kOddThreads), smem, s, a);
}

}  // namespace dbfft
