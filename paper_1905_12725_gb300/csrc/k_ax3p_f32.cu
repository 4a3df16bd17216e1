// Pipelined pass 3 in FP32: the tangent applications of the inner CG.
#include "k_ax3p_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3_pipe<float>(int opk, const Ax3Args<float>& a, cudaStream_t s) {
    return pipe_dispatch<float>(opk, a, s);
}
}  // namespace dbfft
