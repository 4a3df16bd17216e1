// Element-wise pass 5b (divergence, CG residual) in F64, 6 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_div_nc<double, 6>(int, const Ax1FwdArgs<double>&, cudaStream_t);
}
