// Fused first pass of the FP32 CG iteration: preconditioner, direction and
// iterate updates, gradient and the inverse axis-2 transform (launchers).
#include "launch.h"
#include "passes_fused.cuh"

namespace dbfft {

namespace {
template <int NC, int N, int TW>
cudaError_t grad_ax2_n(const Ax1InvArgs<float>& a, cudaStream_t s) {
    constexpr int P = N / FUSED_R;
    const dim3 grid((unsigned)(((long long)a.d.n1 * a.d.h + TW - 1) / TW), (unsigned)a.d.B);
    return launch_k(k_grad_ax2<float, NC, N, TW>, grid, dim3(TW, P), (size_t)N * TW * sizeof(cplx<float>), s, a);
}
template <int NC>
cudaError_t grad_ax2_nc(const Ax1InvArgs<float>& a, cudaStream_t s) {
    switch (a.d.n2) {
        case 32: return fused_tw() == 8 ? grad_ax2_n<NC, 32, 8>(a, s) : grad_ax2_n<NC, 32, 16>(a, s);
        case 64: return fused_tw() == 8 ? grad_ax2_n<NC, 64, 8>(a, s) : grad_ax2_n<NC, 64, 16>(a, s);
        case 128: return fused_tw() == 8 ? grad_ax2_n<NC, 128, 8>(a, s) : grad_ax2_n<NC, 128, 16>(a, s);
        case 256: return fused_tw() == 8 ? grad_ax2_n<NC, 256, 8>(a, s) : grad_ax2_n<NC, 256, 16>(a, s);
        default: return cudaErrorInvalidConfiguration;
    }
}
}  // namespace

cudaError_t launch_grad_ax2(const Ax1InvArgs<float>& a, cudaStream_t s) {
    return a.d.nc == 9 ? grad_ax2_nc<9>(a, s) : grad_ax2_nc<6>(a, s);
}

}  // namespace dbfft
