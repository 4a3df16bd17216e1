// Pass 3 for odd n3: finite-strain crystal plasticity, the tangent application
// (FP32 and FP64) and the update (FP64 pass; FP64 or FP32 tangent data).
#include "k_ax3_odd_impl.cuh"

namespace dbfft {

template <typename T, int N3>
static cudaError_t odd_fcp_n(int opk, const Ax3Args<T>& a, cudaStream_t s) {
    if (opk == OP_FCP_APPLY) return ax3_odd_n<T, N3, 9, OP_FCP_APPLY>(a, s);
    if constexpr (sizeof(T) == 8) {
        if (opk == OP_FCP_UPDATE) return ax3_odd_n<T, N3, 9, OP_FCP_UPDATE>(a, s);
        if (opk == OP_FCP_UPDATE32) return ax3_odd_n<T, N3, 9, OP_FCP_UPDATE32>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_ax3_odd_fcp(int opk, const Ax3Args<T>& a, cudaStream_t s) {
#define DBFFT_ODD_FCP(N) \
    case N: return odd_fcp_n<T, N>(opk, a, s);
    switch (a.d.n3) {
        DBFFT_ODD_NL_SIZES(DBFFT_ODD_FCP)
        default: return cudaErrorInvalidValue;
    }
#undef DBFFT_ODD_FCP
}

template cudaError_t launch_ax3_odd_fcp<float>(int, const Ax3Args<float>&, cudaStream_t);
template cudaError_t launch_ax3_odd_fcp<double>(int, const Ax3Args<double>&, cudaStream_t);

}  // namespace dbfft
