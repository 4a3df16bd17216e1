// k_ax3_impl.cuh -- launchers of pass 3 (axis 3 + per-voxel op) for one precision.
#pragma once
#include "launch.h"

namespace dbfft {

template <typename T, int N3, int NC, int OPK, int RW>
static cudaError_t ax3_nr(const Ax3Args<T>& a, cudaStream_t s) {
    if constexpr (OpInfo<OPK>::apply) {
        if (a.pipe) return launch_ax3_pipe<T>(OPK, a, s);
    }
    const int threads = 256;
    const long long nlines = (long long)a.d.n1 * a.d.n2;
    const dim3 grid((unsigned)((nlines + a.L - 1) / a.L), (unsigned)(a.d.B / a.RB));
    const int nf = OPK == OP_ADJ ? 2 : 1;
    const size_t smem = ((size_t)nf * a.L * a.RB * NC + 1) * ax3_slot_cplx<T, N3, RW>() * sizeof(cplx<T>);
    static int max_dyn = -1;
    if (max_dyn < 0) {  // opt in to large dynamic shared memory: 227 KB per block minus the static part
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k_axis3<T, N3, NC, OPK, RW>);
        if (e != cudaSuccess) return e;
        const int md = 227 * 1024 - (int)fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(k_axis3<T, N3, NC, OPK, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize, md);
        if (e != cudaSuccess) return e;
        max_dyn = md;  // set once the attribute is in place
    }
    if (smem > (size_t)max_dyn) return cudaErrorInvalidConfiguration;
    return launch_k(k_axis3<T, N3, NC, OPK, RW>, grid, dim3(threads), smem, s, a);
}

template <typename T, int N3, int NC, int OPK>
static cudaError_t ax3_n(const Ax3Args<T>& a, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (a.radix == 16) return ax3_nr<T, N3, NC, OPK, 16>(a, s);
    }
    // radix 32: one thread per line (N3/2 <= 32), or 32 values of a line per
    // thread (N3 = 128, 256; FP32); for the operator applications (and the
    // linear residual chain in FP64)
    if constexpr ((sizeof(T) == 4 ? N3 <= 256 : N3 <= 64) && (OpInfo<OPK>::apply)) {
        if (a.radix == 32 && !a.pipe) return ax3_nr<T, N3, NC, OPK, 32>(a, s);
    }
    return ax3_nr<T, N3, NC, OPK, 8>(a, s);
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
