// Pass 3 in FP64: tangent applications, constitutive updates and the adjoint assembly.
#include "k_ax3_impl.cuh"
namespace dbfft {
template <>
cudaError_t launch_ax3<double>(int opk, const Ax3Args<double>& a, cudaStream_t s) {
    if (a.d.n3 & 1) return launch_ax3_odd<double>(opk, a, s);
    switch (opk) {
        case OP_ISO: return ax3_sz<double, 6, OP_ISO>(a, s);
        case OP_NH_APPLY: return ax3_sz<double, 9, OP_NH_APPLY>(a, s);
        case OP_CP_APPLY: return ax3_sz<double, 6, OP_CP_APPLY>(a, s);
        case OP_NH_UPDATE: return ax3_sz<double, 9, OP_NH_UPDATE>(a, s);
        case OP_CP_UPDATE: return ax3_sz<double, 6, OP_CP_UPDATE>(a, s);
        case OP_CP_UPDATE32: return ax3_sz<double, 6, OP_CP_UPDATE32>(a, s);
        case OP_ADJ: return ax3_sz<double, 6, OP_ADJ>(a, s);
        case OP_SVK_APPLY:
        case OP_SVK_UPDATE: return launch_ax3_svk<double>(opk, a, s);
        case OP_FCP_APPLY:
        case OP_FCP_UPDATE:
        case OP_FCP_UPDATE32: return launch_ax3_fcp<double>(opk, a, s);
        default: return cudaErrorInvalidValue;
    }
}
}
