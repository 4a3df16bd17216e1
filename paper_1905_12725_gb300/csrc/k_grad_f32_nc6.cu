// Element-wise pass 1a (gradient, CG direction) in F32, 6 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_grad_nc<float, 6>(int, const Ax1InvArgs<float>&, cudaStream_t);
}
