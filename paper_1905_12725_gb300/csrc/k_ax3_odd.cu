// Pass 3 for odd n3: linear isotropic phases (every odd length), FP32 and FP64;
// the nonlinear operations dispatch to their own translation units.
#include "k_ax3_odd_impl.cuh"

namespace dbfft {

template <typename T>
cudaError_t launch_ax3_odd(int opk, const Ax3Args<T>& a, cudaStream_t s) {
    if (opk != OP_ISO) return launch_ax3_odd_nl<T>(opk, a, s);
    if (a.d.nc != 6) return cudaErrorInvalidValue;
#define DBFFT_ODD_AX3(N) \
    case N: return ax3_odd_n<T, N, 6, OP_ISO>(a, s);
    switch (a.d.n3) {
        DBFFT_ODD_SIZES(DBFFT_ODD_AX3)
        default: return cudaErrorInvalidValue;
    }
#undef DBFFT_ODD_AX3
}

template cudaError_t launch_ax3_odd<float>(int, const Ax3Args<float>&, cudaStream_t);
template cudaError_t launch_ax3_odd<double>(int, const Ax3Args<double>&, cudaStream_t);

}  // namespace dbfft
