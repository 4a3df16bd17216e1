// Pass 3 in FP32: the tangent applications of the inner CG.
#include "k_ax3_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3<float>(int opk, const Ax3Args<float>& a, cudaStream_t s) {
    if (a.d.n3 & 1) return launch_ax3_odd<float>(opk, a, s);
    switch (opk) {
        case OP_ISO: return ax3_sz<float, 6, OP_ISO>(a, s);
        case OP_NH_APPLY: return ax3_sz<float, 9, OP_NH_APPLY>(a, s);
        case OP_CP_APPLY: return ax3_sz<float, 6, OP_CP_APPLY>(a, s);
        case OP_SVK_APPLY: return launch_ax3_svk<float>(opk, a, s);
        case OP_FCP_APPLY: return launch_ax3_fcp<float>(opk, a, s);
        default: return cudaErrorInvalidValue;
    }
}
}
