// Dispatch of the element-wise kernels of passes 1 and 5 on the number of field components.
#include "launch.h"

namespace dbfft {

template <typename T, int NC> cudaError_t launch_grad_nc(int mode, const Ax1InvArgs<T>& a, cudaStream_t s);
template <typename T, int NC> cudaError_t launch_div_nc(int mode, const Ax1FwdArgs<T>& a, cudaStream_t s);

template <typename T>
cudaError_t launch_grad(int mode, const Ax1InvArgs<T>& a, cudaStream_t s) {
    return a.d.nc == 6 ? launch_grad_nc<T, 6>(mode, a, s) : launch_grad_nc<T, 9>(mode, a, s);
}
template <typename T>
cudaError_t launch_div(int mode, const Ax1FwdArgs<T>& a, cudaStream_t s) {
    return a.d.nc == 6 ? launch_div_nc<T, 6>(mode, a, s) : launch_div_nc<T, 9>(mode, a, s);
}
template cudaError_t launch_grad<float>(int, const Ax1InvArgs<float>&, cudaStream_t);
template cudaError_t launch_grad<double>(int, const Ax1InvArgs<double>&, cudaStream_t);
template cudaError_t launch_div<float>(int, const Ax1FwdArgs<float>&, cudaStream_t);
template cudaError_t launch_div<double>(int, const Ax1FwdArgs<double>&, cudaStream_t);

}  // namespace dbfft
