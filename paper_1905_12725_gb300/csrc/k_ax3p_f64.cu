// Pipelined pass 3 in FP64: the tangent applications of the FP64 CG.
#include "k_ax3p_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_pipe<double>(int opk, const Ax3Args<double>& a, cudaStream_t s) {
    return pipe_dispatch<double>(opk, a, s);
}
}  // namespace dbfft
