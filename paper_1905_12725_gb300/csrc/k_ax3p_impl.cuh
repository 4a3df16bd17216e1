// k_ax3p_impl.cuh -- launchers of the pipelined pass 3 (CG applications) for one precision.
#pragma once
#include "launch.h"
#include "pass3_pipe.cuh"

namespace dbfft {

template <typename T, int N3, int NC, int OPK, int RW, int NS>
static cudaError_t pipe_nrs(const Ax3Args<T>& a, cudaStream_t s) {
    using Plan = PipePlan<T, N3>;
    constexpr int M = N3 / 2;
    constexpr int R = RadixAx3<T, M, RW>::value;
    constexpr int P = M / R;
    const int threads = 256;
    const long long nlines = (long long)a.d.n1 * a.d.n2;
    if (a.L < 2 || (a.L & 1) || nlines % a.L != 0 || a.RB < 1 || a.RB > 8 || a.d.B % a.RB != 0)
        return cudaErrorInvalidConfiguration;
    const long long smem = Plan::total_bytes(a.L, a.RB, NC, a.scale != nullptr, P, threads / 32, NS);
    auto kern = k_axis3_pipe<T, N3, NC, OPK, RW, NS>;
    static int max_dyn = -1;
    if (max_dyn < 0) {  // opt in to large dynamic shared memory: 227 KB per block minus the static part
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        const int md = 227 * 1024 - (int)fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, md);
        if (e != cudaSuccess) return e;
        max_dyn = md;  // set once the attribute is in place
    }
    if (smem > max_dyn) return cudaErrorInvalidConfiguration;
    // persistent grid: as many CTAs as fit on the GPU at once, shared among the groups
    static long long occ_smem = -1;
    static int occ = 0, nsm = 0;
    if (occ_smem != smem) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, (size_t)smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        occ_smem = smem;
    }
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const long long ngroups = a.d.B / a.RB;
    const long long ntiles = nlines / a.L;
    long long per_group = ((long long)occ * nsm + ngroups - 1) / ngroups;
    if (per_group > ntiles) per_group = ntiles;
    if (per_group < 1) per_group = 1;
    return launch_k(kern, dim3((unsigned)per_group, (unsigned)ngroups), dim3(threads), (size_t)smem, s, a);
}

// a.pipe: 1 = two shared-memory stages, 2 = one stage
template <typename T, int N3, int NC, int OPK, int RW>
static cudaError_t pipe_nr(const Ax3Args<T>& a, cudaStream_t s) {
    if (a.pipe == 2) return pipe_nrs<T, N3, NC, OPK, RW, 1>(a, s);
    return pipe_nrs<T, N3, NC, OPK, RW, 2>(a, s);
}

template <typename T, int N3, int NC, int OPK>
static cudaError_t pipe_n(const Ax3Args<T>& a, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (a.radix == 16) return pipe_nr<T, N3, NC, OPK, 16>(a, s);
    }
    return pipe_nr<T, N3, NC, OPK, 8>(a, s);
}

template <typename T, int NC, int OPK>
static cudaError_t pipe_sz(const Ax3Args<T>& a, cudaStream_t s) {
    switch (a.d.n3) {
        case 8: return pipe_n<T, 8, NC, OPK>(a, s);
        case 16: return pipe_n<T, 16, NC, OPK>(a, s);
        case 32: return pipe_n<T, 32, NC, OPK>(a, s);
        case 64: return pipe_n<T, 64, NC, OPK>(a, s);
        case 128: return pipe_n<T, 128, NC, OPK>(a, s);
        case 256: return pipe_n<T, 256, NC, OPK>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t pipe_dispatch(int opk, const Ax3Args<T>& a, cudaStream_t s) {
    if (a.pipe == 3) {  // the line-bulk pass (FP32 only)
        if constexpr (sizeof(T) == 4) return launch_ax3_lb(opk, a, s);
        else return cudaErrorInvalidConfiguration;
    }
    switch (opk) {
        case OP_ISO: return pipe_sz<T, 6, OP_ISO>(a, s);
        case OP_NH_APPLY: return pipe_sz<T, 9, OP_NH_APPLY>(a, s);
        case OP_CP_APPLY: return pipe_sz<T, 6, OP_CP_APPLY>(a, s);
        case OP_SVK_APPLY: return launch_ax3_svk<T>(opk, a, s);
        case OP_FCP_APPLY: return launch_ax3_fcp<T>(opk, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dbfft
