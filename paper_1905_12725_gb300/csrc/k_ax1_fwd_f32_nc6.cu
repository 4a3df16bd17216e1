// Pass 5 (axis 1, forward) in F32, 6 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_ax1_fwd_nc<float, 6>(int, const Ax1FwdArgs<float>&, cudaStream_t);
}
