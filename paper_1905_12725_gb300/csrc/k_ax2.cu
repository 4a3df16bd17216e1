// Passes 2 and 4 (axis 2, both directions) in FP32 and FP64.
#include "launch.h"

namespace dbfft {

template <typename T, int N2, int DIR>
static cudaError_t ax2_n(const Ax2Args<T>& a, cudaStream_t s) {
    constexpr int R = RadixFor<T, N2>::value;
    constexpr int P = N2 / R;
    const int TW = ax2_tile(N2, sizeof(T) == 8);
    const long long ncols = (long long)a.d.B * a.d.nc * a.d.n1 * a.d.h;
    const dim3 block(TW, P);
    const dim3 grid((unsigned)((ncols + TW - 1) / TW));
    const size_t smem = (ColFFT<T, N2, R, DIR>::NST > 1) ? (size_t)N2 * TW * sizeof(cplx<T>) : 0;
    k_axis2<T, N2, DIR><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ax2(int dir, const Ax2Args<T>& a, cudaStream_t s) {
#define DBFFT_AX2(N) case N: return dir > 0 ? ax2_n<T, N, +1>(a, s) : ax2_n<T, N, -1>(a, s);
    switch (a.d.n2) {
        DBFFT_AX2(8) DBFFT_AX2(16) DBFFT_AX2(32) DBFFT_AX2(64) DBFFT_AX2(128) DBFFT_AX2(256)
        default: return cudaErrorInvalidValue;
    }
#undef DBFFT_AX2
}

template cudaError_t launch_ax2<float>(int, const Ax2Args<float>&, cudaStream_t);
template cudaError_t launch_ax2<double>(int, const Ax2Args<double>&, cudaStream_t);

}  // namespace dbfft
