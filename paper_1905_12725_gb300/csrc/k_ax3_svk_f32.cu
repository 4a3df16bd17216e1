// Pass 3 of the St. Venant-Kirchhoff law in FP32: the tangent applications of the inner CG.
#include "k_ax3_impl.cuh"
#include "k_ax3p_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_svk<float>(int opk, const Ax3Args<float>& a, cudaStream_t s) {
    if (opk == OP_SVK_APPLY) return a.pipe ? pipe_sz<float, 9, OP_SVK_APPLY>(a, s) : ax3_sz<float, 9, OP_SVK_APPLY>(a, s);
    return cudaErrorInvalidValue;
}
}  // namespace dbfft
