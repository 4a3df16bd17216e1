// Pass 3 for odd n3: the crystal-plasticity updates (FP64 pass; FP64 or FP32 tangent).
#include "k_ax3_odd_impl.cuh"

namespace dbfft {

template <int N3>
static cudaError_t odd_cp_n(int opk, const Ax3Args<double>& a, cudaStream_t s) {
    if (opk == OP_CP_UPDATE32) return ax3_odd_n<double, N3, 6, OP_CP_UPDATE32>(a, s);
    return ax3_odd_n<double, N3, 6, OP_CP_UPDATE>(a, s);
}

cudaError_t launch_ax3_odd_cp(int opk, const Ax3Args<double>& a, cudaStream_t s) {
#define DBFFT_ODD_CP(N) \
    case N: return odd_cp_n<N>(opk, a, s);
    switch (a.d.n3) {
        DBFFT_ODD_NL_SIZES(DBFFT_ODD_CP)
        default: return cudaErrorInvalidValue;
    }
#undef DBFFT_ODD_CP
}

}  // namespace dbfft
