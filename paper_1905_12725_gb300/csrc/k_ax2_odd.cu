// Strided C2C transforms along axis 1 or 2 for odd lengths, FP32 and FP64.
#include "launch.h"
#include "pass3_odd.cuh"

namespace dbfft {

template <typename T, int N, int DIR>
static cudaError_t fft_odd_n(Ax2Args<T> a, int axis, cudaStream_t s) {
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
    // columns per CTA: a power of two <= 32 whose two column buffers fit in 96 KB
    const size_t col_bytes = 2 * (size_t)N * sizeof(cplx<T>);
    int TW = 32;
    while (TW > 1 && TW * col_bytes > 96 * 1024) TW /= 2;
    const int G = kOddThreads / TW;
    const size_t smem = TW * col_bytes;
    static bool opted = false;
    if (!opted) {
        cudaError_t e = cudaFuncSetAttribute(k_fft_odd<T, N, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             96 * 1024);
        if (e != cudaSuccess) return e;
        opted = true;
    }
    const dim3 grid((unsigned)((a.ncols + TW - 1) / TW));
    return launch_k(k_fft_odd<T, N, DIR>, grid, dim3(TW, G), smem, s, a);
}

template <typename T>
cudaError_t launch_fft_odd(int dir, int axis, Ax2Args<T> a, cudaStream_t s) {
    const int n = axis == 1 ? a.d.n1 : a.d.n2;
#define DBFFT_ODD_FFT(N) \
    case N: return dir > 0 ? fft_odd_n<T, N, +1>(a, axis, s) : fft_odd_n<T, N, -1>(a, axis, s);
    switch (n) {
        DBFFT_ODD_SIZES(DBFFT_ODD_FFT)
        default: return cudaErrorInvalidValue;
    }
#undef DBFFT_ODD_FFT
}

template cudaError_t launch_fft_odd<float>(int, int, Ax2Args<float>, cudaStream_t);
template cudaError_t launch_fft_odd<double>(int, int, Ax2Args<double>, cudaStream_t);

}  // namespace dbfft
