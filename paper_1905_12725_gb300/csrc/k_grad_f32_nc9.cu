// Element-wise pass 1a (gradient, CG direction) in F32, 9 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_grad_nc<float, 9>(int, const Ax1InvArgs<float>&, cudaStream_t);
}
