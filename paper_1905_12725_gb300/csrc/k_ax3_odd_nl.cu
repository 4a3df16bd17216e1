// Pass 3 for odd n3 with the nonlinear models: tangent applications (FP32 and
// FP64) and the Neo-Hookean / St. Venant-Kirchhoff updates (FP64); the
// crystal-plasticity operations dispatch to their own translation units.
#include "k_ax3_odd_impl.cuh"

namespace dbfft {

template <typename T, int N3>
static cudaError_t odd_nl_n(int opk, const Ax3Args<T>& a, cudaStream_t s) {
    switch (opk) {
        case OP_NH_APPLY: return ax3_odd_n<T, N3, 9, OP_NH_APPLY>(a, s);
        case OP_SVK_APPLY: return ax3_odd_n<T, N3, 9, OP_SVK_APPLY>(a, s);
        case OP_CP_APPLY: return ax3_odd_n<T, N3, 6, OP_CP_APPLY>(a, s);
        case OP_FCP_APPLY:
        case OP_FCP_UPDATE:
        case OP_FCP_UPDATE32: return launch_ax3_odd_fcp<T>(opk, a, s);
        default: break;
    }
    if constexpr (sizeof(T) == 8) {
        switch (opk) {
            case OP_NH_UPDATE: return ax3_odd_n<T, N3, 9, OP_NH_UPDATE>(a, s);
            case OP_SVK_UPDATE: return ax3_odd_n<T, N3, 9, OP_SVK_UPDATE>(a, s);
            case OP_CP_UPDATE:
            case OP_CP_UPDATE32: return launch_ax3_odd_cp(opk, a, s);
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_ax3_odd_nl(int opk, const Ax3Args<T>& a, cudaStream_t s) {
#define DBFFT_ODD_NL(N) \
    case N: return odd_nl_n<T, N>(opk, a, s);
    switch (a.d.n3) {
        DBFFT_ODD_NL_SIZES(DBFFT_ODD_NL)
        default: return cudaErrorInvalidValue;
    }
#undef DBFFT_ODD_NL
}

template cudaError_t launch_ax3_odd_nl<float>(int, const Ax3Args<float>&, cudaStream_t);
template cudaError_t launch_ax3_odd_nl<double>(int, const Ax3Args<double>&, cudaStream_t);

}  // namespace dbfft
