// Pass 3 of finite-strain crystal plasticity in FP32: the tangent applications of the inner CG.
#include "k_ax3_impl.cuh"
#include "k_ax3p_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_fcp<float>(int opk, const Ax3Args<float>& a, cudaStream_t s) {
    if (opk == OP_FCP_APPLY) return a.pipe ? pipe_sz<float, 9, OP_FCP_APPLY>(a, s) : ax3_sz<float, 9, OP_FCP_APPLY>(a, s);
    return cudaErrorInvalidValue;
}
}  // namespace dbfft
