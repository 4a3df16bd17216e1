// Pass 1 (axis 1, inverse) in F64, 9 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_ax1_inv_nc<double, 9>(int, const Ax1InvArgs<double>&, cudaStream_t);
}
