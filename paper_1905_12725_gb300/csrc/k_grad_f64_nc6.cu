// Element-wise pass 1a (gradient, CG direction) in F64, 6 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_grad_nc<double, 6>(int, const Ax1InvArgs<double>&, cudaStream_t);
}
