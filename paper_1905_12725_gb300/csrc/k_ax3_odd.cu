// Pass 3 for odd n3 (linear isotropic phases), FP32 and FP64.
#include "launch.h"
#include "pass3_odd.cuh"

namespace dbfft {

template <typename T, int N3>
static cudaError_t ax3_odd_n(const Ax3Args<T>& a0, cudaStream_t s) {
    Ax3Args<T> a = a0;
    a.RB = 1;  // one right-hand side per CTA
    a.L = ax3_odd_lines(N3, sizeof(T) == 8);
    const long long nlines = (long long)a.d.n1 * a.d.n2;
    const size_t smem = (size_t)3 * a.L * 2 * N3 * sizeof(cplx<T>);
    static bool opted = false;
    if (!opted) {
        cudaError_t e = cudaFuncSetAttribute(k_axis3_odd<T, N3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             96 * 1024);
        if (e != cudaSuccess) return e;
        opted = true;
    }
    const dim3 grid((unsigned)((nlines + a.L - 1) / a.L), (unsigned)a.d.B);
    return launch_k(k_axis3_odd<T, N3>, grid, dim3(kOddThreads), smem, s, a);
}

template <typename T>
cudaError_t launch_ax3_odd(int opk, const Ax3Args<T>& a, cudaStream_t s) {
    if (opk != OP_ISO || a.d.nc != 6) return cudaErrorInvalidValue;
#define DBFFT_ODD_AX3(N) \
    case N: return ax3_odd_n<T, N>(a, s);
    switch (a.d.n3) {
        DBFFT_ODD_SIZES(DBFFT_ODD_AX3)
        default: return cudaErrorInvalidValue;
    }
#undef DBFFT_ODD_AX3
}

template cudaError_t launch_ax3_odd<float>(int, const Ax3Args<float>&, cudaStream_t);
template cudaError_t launch_ax3_odd<double>(int, const Ax3Args<double>&, cudaStream_t);

}  // namespace dbfft
