// Pass 3 of finite-strain crystal plasticity in FP64: tangent applications and the update.
#include "k_ax3_impl.cuh"
#include "k_ax3p_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_fcp<double>(int opk, const Ax3Args<double>& a, cudaStream_t s) {
    if (opk == OP_FCP_APPLY) return a.pipe ? pipe_sz<double, 9, OP_FCP_APPLY>(a, s) : ax3_sz<double, 9, OP_FCP_APPLY>(a, s);
    if (opk == OP_FCP_UPDATE) return ax3_sz<double, 9, OP_FCP_UPDATE>(a, s);
    if (opk == OP_FCP_UPDATE32) return ax3_sz<double, 9, OP_FCP_UPDATE32>(a, s);
    return cudaErrorInvalidValue;
}
}  // namespace dbfft
