// Pass 3 of the post-processing transforms in FP64: the total displacement field, and
// real 6-component fields in and out of the spectrum (the crystal-plasticity adjoint).
#include "k_ax3_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_post<double>(int opk, const Ax3Args<double>& a, cudaStream_t s) {
    if (opk == OP_DISP) return ax3_sz<double, 3, OP_DISP>(a, s);
    if (opk == OP_LOADW) return ax3_sz<double, 6, OP_LOADW>(a, s);
    if (opk == OP_STOREW) return ax3_sz<double, 6, OP_STOREW>(a, s);
    return cudaErrorInvalidValue;
}
}  // namespace dbfft
