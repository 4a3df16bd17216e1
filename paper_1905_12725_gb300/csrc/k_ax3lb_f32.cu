// Line-bulk pass 3 (FP32 CG applications, n3 = 64, 128 and 256): launchers.
#include "launch.h"
#include "pass3_lb.cuh"

namespace dbfft {

namespace {

template <int N3, int NC, int OPK, int WL>
cudaError_t lb_launch(const Ax3Args<float>& a, cudaStream_t s) {
    using Plan = LbPlan<N3>;
    const long long nlines = (long long)a.d.n1 * a.d.n2;
    if (a.L < 2 || (a.L & 1) || nlines % a.L != 0 || a.RB < 1 || a.RB > 8 || a.d.B % a.RB != 0)
        return cudaErrorInvalidConfiguration;
    if ((WL == 1 && a.L != 16) || (WL == 2 && a.L != LbShape<N3 / 2>::P)) return cudaErrorInvalidConfiguration;
    const long long smem = Plan::total_bytes(a.L, a.RB, NC, a.scale != nullptr);
    auto kern = k_axis3_lb<N3, NC, OPK, WL>;
    static int max_dyn = -1;
    if (max_dyn < 0) {  // opt in to large dynamic shared memory: 227 KB per block minus the static part
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        const int md = 227 * 1024 - (int)fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, md);
        if (e != cudaSuccess) return e;
        max_dyn = md;  // set once the attribute is in place
    }
    if (smem > max_dyn) return cudaErrorInvalidConfiguration;
    // a.radix: the thread cap (0: 384); -1, -2: warp lines (WL = 1: P warps; WL = 2: P / 2 warps)
    constexpr int P = LbShape<N3 / 2>::P;
    const int threads = WL == 1 ? 32 * P : (WL == 2 ? 16 * P : lb_threads<N3>(a.RB * NC * a.L, a.radix));
    return launch_k(kern, dim3((unsigned)(nlines / a.L), (unsigned)(a.d.B / a.RB)), dim3(threads), (size_t)smem, s, a);
}

template <int NC, int OPK>
cudaError_t lb_n(const Ax3Args<float>& a, cudaStream_t s) {
    switch (a.d.n3) {
        case 64:
            return a.radix == -2 ? lb_launch<64, NC, OPK, 2>(a, s)
                 : a.radix < 0   ? lb_launch<64, NC, OPK, 1>(a, s)
                                 : lb_launch<64, NC, OPK, 0>(a, s);
        case 128:
            return a.radix == -2 ? lb_launch<128, NC, OPK, 2>(a, s)
                 : a.radix < 0   ? lb_launch<128, NC, OPK, 1>(a, s)
                                 : lb_launch<128, NC, OPK, 0>(a, s);
        case 256:
            return a.radix == -2 ? lb_launch<256, NC, OPK, 2>(a, s)
                 : a.radix < 0   ? lb_launch<256, NC, OPK, 1>(a, s)
                                 : lb_launch<256, NC, OPK, 0>(a, s);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace

cudaError_t launch_ax3_lb(int opk, const Ax3Args<float>& a, cudaStream_t s) {
    switch (opk) {
        case OP_ISO: return lb_n<6, OP_ISO>(a, s);
        case OP_CP_APPLY: return lb_n<6, OP_CP_APPLY>(a, s);
        case OP_NH_APPLY: return lb_n<9, OP_NH_APPLY>(a, s);
        default: return cudaErrorInvalidConfiguration;
    }
}

long long ax3_lb_smem(int n3, int nc, int rb, bool scale, int L, long long nlines) {
    if (L < 2 || (L & 1) || nlines % L != 0 || rb < 1 || rb > 8 || (nc != 6 && nc != 9)) return -1;
    if (lb_threads<256>(rb * nc * L) > 384) return -1;
    switch (n3) {
        case 64: return LbPlan<64>::total_bytes(L, rb, nc, scale);
        case 128: return LbPlan<128>::total_bytes(L, rb, nc, scale);
        case 256: return LbPlan<256>::total_bytes(L, rb, nc, scale);
        default: return -1;
    }
}

}  // namespace dbfft
