// Pass 1 (axis 1, inverse) in F32, 6 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_ax1_inv_nc<float, 6>(int, const Ax1InvArgs<float>&, cudaStream_t);
}
