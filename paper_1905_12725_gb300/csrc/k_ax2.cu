// Pure C2C transforms along axis 1 (passes 2, 4) and axis 2 (passes 1b, 5a), both directions, FP32 and FP64.
#include "launch.h"

namespace dbfft {

template <typename T, int N, int DIR>
static cudaError_t fft_n(Ax2Args<T> a, int axis, cudaStream_t s) {
    constexpr int R = RadixFor<T, N>::value;
    constexpr int P = N / R;
    const int want = axis == 1 ? a.tw_ax1 : a.tw_ax2;
    int TW = want > 0 ? want : ax2_tile(N, sizeof(T) == 8);
    if (TW * P > 512) TW = 512 / P;
    if (axis == 1) {  // element (b, c, t, j): (b nc + c) n1 plane + t plane + j
        a.tab = a.tw.t1;
        a.inner = a.d.plane;
        a.ncols = (long long)a.d.B * a.d.nc * a.d.plane;
        a.cols_per_b = (long long)a.d.nc * a.d.plane;
    } else {  // element (b, c, k1, t, k3): ((b nc + c) n1 + k1) plane + t h + k3
        a.tab = a.tw.t2;
        a.inner = a.d.h;
        a.ncols = (long long)a.d.B * a.d.nc * a.d.n1 * a.d.h;
        a.cols_per_b = (long long)a.d.nc * a.d.n1 * a.d.h;
    }
    if (a.ncols >= (1LL << 32) - 512) return cudaErrorInvalidValue;  // 32-bit column indices
    a.div_inner = make_fastdiv((unsigned)a.inner);
    a.div_cpb = make_fastdiv((unsigned)a.cols_per_b);
    const dim3 block(TW, P);
    const dim3 grid((unsigned)((a.ncols + TW - 1) / TW));
    const size_t smem = (ColFFT<T, N, R, DIR>::NST > 1) ? (size_t)N * TW * sizeof(cplx<T>) : 0;
    return launch_k(k_fft_strided<T, N, DIR>, grid, block, smem, s, a);
}

#define DBFFT_FFT(N, AX) case N: return dir > 0 ? fft_n<T, N, +1>(a, AX, s) : fft_n<T, N, -1>(a, AX, s);
template <typename T>
cudaError_t launch_fft_ax1(int dir, const Ax2Args<T>& a, cudaStream_t s) {
    switch (a.d.n1) {
        DBFFT_FFT(8, 1) DBFFT_FFT(16, 1) DBFFT_FFT(32, 1) DBFFT_FFT(64, 1) DBFFT_FFT(128, 1) DBFFT_FFT(256, 1)
        default: return (a.d.n1 & 1) ? launch_fft_odd<T>(dir, 1, a, s) : cudaErrorInvalidValue;
    }
}
template <typename T>
cudaError_t launch_fft_ax2(int dir, const Ax2Args<T>& a, cudaStream_t s) {
    switch (a.d.n2) {
        DBFFT_FFT(8, 2) DBFFT_FFT(16, 2) DBFFT_FFT(32, 2) DBFFT_FFT(64, 2) DBFFT_FFT(128, 2) DBFFT_FFT(256, 2)
        default: return (a.d.n2 & 1) ? launch_fft_odd<T>(dir, 2, a, s) : cudaErrorInvalidValue;
    }
}
#undef DBFFT_FFT

template cudaError_t launch_fft_ax1<float>(int, const Ax2Args<float>&, cudaStream_t);
template cudaError_t launch_fft_ax1<double>(int, const Ax2Args<double>&, cudaStream_t);
template cudaError_t launch_fft_ax2<float>(int, const Ax2Args<float>&, cudaStream_t);
template cudaError_t launch_fft_ax2<double>(int, const Ax2Args<double>&, cudaStream_t);

}  // namespace dbfft
