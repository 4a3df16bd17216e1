// k_ax3_impl.cuh -- launchers of pass 3 (axis 3 + per-voxel op) for one precision.
#pragma once
#include "launch.h"

namespace dbfft {

template <typename T, int N3, int NC, int OPK>
static cudaError_t ax3_n(const Ax3Args<T>& a, cudaStream_t s) {
    constexpr int M = N3 / 2;
    constexpr int R = RadixFor<T, M>::value;
    constexpr int P = M / R;
    const int threads = ((P * a.L * a.RB * NC + 31) / 32) * 32;  // whole warps (block reductions shuffle full warps)
    const long long nlines = (long long)a.d.n1 * a.d.n2;
    const dim3 grid((unsigned)((nlines + a.L - 1) / a.L), (unsigned)(a.d.B / a.RB));
    // one real line of N3 values per slot of P threads, padding slots included
    const size_t smem = (size_t)(threads / P) * N3 * sizeof(T) * (OPK == OP_ADJ ? 2 : 1);
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_axis3<T, N3, NC, OPK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_done = true;
    }
    k_axis3<T, N3, NC, OPK><<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int NC, int OPK>
static cudaError_t ax3_sz(const Ax3Args<T>& a, cudaStream_t s) {
    switch (a.d.n3) {
        case 8: return ax3_n<T, 8, NC, OPK>(a, s);
        case 16: return ax3_n<T, 16, NC, OPK>(a, s);
        case 32: return ax3_n<T, 32, NC, OPK>(a, s);
        case 64: return ax3_n<T, 64, NC, OPK>(a, s);
        case 128: return ax3_n<T, 128, NC, OPK>(a, s);
        case 256: return ax3_n<T, 256, NC, OPK>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dbfft
