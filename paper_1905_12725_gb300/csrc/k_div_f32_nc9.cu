// Element-wise pass 5b (divergence, CG residual) in F32, 9 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_div_nc<float, 9>(int, const Ax1FwdArgs<float>&, cudaStream_t);
}
