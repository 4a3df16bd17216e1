// Pass 1 (axis 1, inverse) in F32, 9 field components.
#include "k_ax1_impl.cuh"
namespace dbfft {
template cudaError_t launch_ax1_inv_nc<float, 9>(int, const Ax1InvArgs<float>&, cudaStream_t);
}
