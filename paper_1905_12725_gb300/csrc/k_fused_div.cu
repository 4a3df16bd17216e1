// Fused last pass of the FP32 CG iteration: the forward axis-2 transform,
// divergence, null mask, residual update and the CG reductions (launchers).
#include "launch.h"
#include "passes_fused.cuh"

#include <cstdlib>

namespace dbfft {

namespace {
template <int NC, int N, int TW>
cudaError_t ax2_div_n(const Ax1FwdArgs<float>& a, cudaStream_t s) {
    constexpr int P = N / FUSED_R;
    const dim3 grid((unsigned)(((long long)a.d.n1 * a.d.h + TW - 1) / TW), (unsigned)a.d.B);
    return launch_k(k_ax2_div<float, NC, N, TW>, grid, dim3(TW, P), (size_t)N * TW * sizeof(cplx<float>), s, a);
}
template <int NC>
cudaError_t ax2_div_nc(const Ax1FwdArgs<float>& a, cudaStream_t s) {
    switch (a.d.n2) {
        case 32: return fused_tw() == 8 ? ax2_div_n<NC, 32, 8>(a, s) : ax2_div_n<NC, 32, 16>(a, s);
        case 64: return fused_tw() == 8 ? ax2_div_n<NC, 64, 8>(a, s) : ax2_div_n<NC, 64, 16>(a, s);
        case 128: return fused_tw() == 8 ? ax2_div_n<NC, 128, 8>(a, s) : ax2_div_n<NC, 128, 16>(a, s);
        case 256: return fused_tw() == 8 ? ax2_div_n<NC, 256, 8>(a, s) : ax2_div_n<NC, 256, 16>(a, s);
        default: return cudaErrorInvalidConfiguration;
    }
}
}  // namespace

cudaError_t launch_ax2_div(const Ax1FwdArgs<float>& a, cudaStream_t s) {
    return a.d.nc == 9 ? ax2_div_nc<9>(a, s) : ax2_div_nc<6>(a, s);
}

long long fused_ax2_blocks(int n1, int h) { return ((long long)n1 * h + 7) / 8; }  // the narrowest tile
int fused_tw() {
    static int tw = 0;
    if (tw == 0) {
        const char* e = std::getenv("DBFFT_FUSED_TW");
        tw = (e && std::atoi(e) == 8) ? 8 : 16;
    }
    return tw;
}
bool fused_ax2_supported(int n2) { return n2 == 32 || n2 == 64 || n2 == 128 || n2 == 256; }

}  // namespace dbfft
