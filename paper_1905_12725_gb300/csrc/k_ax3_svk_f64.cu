// Pass 3 of the St. Venant-Kirchhoff law in FP64: tangent applications and the constitutive update.
#include "k_ax3_impl.cuh"
#include "k_ax3p_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_svk<double>(int opk, const Ax3Args<double>& a, cudaStream_t s) {
    if (opk == OP_SVK_APPLY) return a.pipe ? pipe_sz<double, 9, OP_SVK_APPLY>(a, s) : ax3_sz<double, 9, OP_SVK_APPLY>(a, s);
    if (opk == OP_SVK_UPDATE) return ax3_sz<double, 9, OP_SVK_UPDATE>(a, s);
    return cudaErrorInvalidValue;
}
}  // namespace dbfft
