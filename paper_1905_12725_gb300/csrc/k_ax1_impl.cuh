// k_ax1_impl.cuh -- launchers of passes 1 and 5 (axis 1) for one precision.
#pragma once
#include "launch.h"

namespace dbfft {

template <typename K>
static void allow_smem(K kernel, size_t smem) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int N1>
static size_t ax1_smem() {
    constexpr int R = RadixAx1<T, N1>::value;
    constexpr int P = N1 / R;
    constexpr int TW = AX1_THREADS / P;
    return ((size_t)N1 * TW + 3 * (size_t)R * AX1_THREADS) * sizeof(cplx<T>);
}

template <typename T, int N1, int NC>
static cudaError_t ax1_inv_n(int mode, const Ax1InvArgs<T>& a, cudaStream_t s) {
    constexpr int R = RadixAx1<T, N1>::value;
    constexpr int P = N1 / R;
    constexpr int TW = AX1_THREADS / P;
    const dim3 block(TW, P);
    const dim3 grid((unsigned)((a.d.plane + TW - 1) / TW), (unsigned)a.d.B);
    const size_t smem = ax1_smem<T, N1>();
    if (mode == AX1_CG) {
        allow_smem(k_axis1_inv<T, N1, NC, AX1_CG>, smem);
        k_axis1_inv<T, N1, NC, AX1_CG><<<grid, block, smem, s>>>(a);
    } else {
        allow_smem(k_axis1_inv<T, N1, NC, AX1_PLAIN>, smem);
        k_axis1_inv<T, N1, NC, AX1_PLAIN><<<grid, block, smem, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename T, int N1, int NC>
static cudaError_t ax1_fwd_n(int mode, const Ax1FwdArgs<T>& a, cudaStream_t s) {
    constexpr int R = RadixAx1<T, N1>::value;
    constexpr int P = N1 / R;
    constexpr int TW = AX1_THREADS / P;
    const dim3 block(TW, P);
    const dim3 grid((unsigned)((a.d.plane + TW - 1) / TW), (unsigned)a.d.B);
    const size_t smem = ax1_smem<T, N1>();
    if (mode == AX5_CG) {
        allow_smem(k_axis1_fwd<T, N1, NC, AX5_CG>, smem);
        k_axis1_fwd<T, N1, NC, AX5_CG><<<grid, block, smem, s>>>(a);
    } else if (mode == AX5_RESID) {
        allow_smem(k_axis1_fwd<T, N1, NC, AX5_RESID>, smem);
        k_axis1_fwd<T, N1, NC, AX5_RESID><<<grid, block, smem, s>>>(a);
    } else {
        allow_smem(k_axis1_fwd<T, N1, NC, AX5_PLAIN>, smem);
        k_axis1_fwd<T, N1, NC, AX5_PLAIN><<<grid, block, smem, s>>>(a);
    }
    return cudaGetLastError();
}

#define DBFFT_AX1_CASES(FN, NC, ...)                       \
    switch (a.d.n1) {                                      \
        case 8: return FN<T, 8, NC>(__VA_ARGS__);          \
        case 16: return FN<T, 16, NC>(__VA_ARGS__);        \
        case 32: return FN<T, 32, NC>(__VA_ARGS__);        \
        case 64: return FN<T, 64, NC>(__VA_ARGS__);        \
        case 128: return FN<T, 128, NC>(__VA_ARGS__);      \
        case 256: return FN<T, 256, NC>(__VA_ARGS__);      \
        default: return cudaErrorInvalidValue;             \
    }

template <typename T, int NC>
cudaError_t launch_ax1_inv_nc(int mode, const Ax1InvArgs<T>& a, cudaStream_t s) {
    DBFFT_AX1_CASES(ax1_inv_n, NC, mode, a, s)
}
template <typename T, int NC>
cudaError_t launch_ax1_fwd_nc(int mode, const Ax1FwdArgs<T>& a, cudaStream_t s) {
    DBFFT_AX1_CASES(ax1_fwd_n, NC, mode, a, s)
}

}  // namespace dbfft
