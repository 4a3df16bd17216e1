// Pass 3 of the post-processing transforms in FP64: the total displacement field.
#include "k_ax3_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_post<double>(int opk, const Ax3Args<double>& a, cudaStream_t s) {
    if (opk == OP_DISP) return ax3_sz<double, 3, OP_DISP>(a, s);
    return cudaErrorInvalidValue;
}
}  // namespace dbfft
