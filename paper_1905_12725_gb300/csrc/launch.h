// launch.h -- host-side launchers of the pass kernels. Each translation unit
// instantiates the kernels of one pass and precision for the compiled
// transform lengths and dispatches on the runtime sizes.
#pragma once
#include "pass3.cuh"

#include <utility>

namespace dbfft {
// Kernels of the PCG loop are launched with programmatic stream serialisation
// while this is set (the CG graph body is captured that way).
extern thread_local bool g_pdl_launch;

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if (g_pdl_launch) {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
}  // namespace dbfft

namespace dbfft {

// Launch geometry shared by the launchers and the buffer sizing.
long long pw_blocks(long long H, int B, int waves = 2);     // grid (per right-hand side) of the element-wise kernels
long long pw_blocks_resident(long long H, int B, int waves, int per_sm);  // the same in whole waves of per_sm blocks per SM
int ax2_tile(int n, bool dbl);                       // columns per CTA of the strided transforms
int ax3_lines(int n3, int nc, int rb, bool dbl, int nfields = 1, int radix = 8);  // default lines per CTA of pass 3
int ax3_threads_per_line(int n3, int nc, int rb, bool dbl);
size_t ax3_smem(int n3, int nc, int rb, int lines, bool dbl, bool two_fields);
bool supported_len(int n);   // powers of two in [8, 256] or the odd lengths below
bool supported_pow2(int n);  // powers of two in [8, 256]

template <typename T> cudaError_t launch_grad(int mode, const Ax1InvArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_div(int mode, const Ax1FwdArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_fft_ax1(int dir, const Ax2Args<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_fft_ax2(int dir, const Ax2Args<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_ax3(int opk, const Ax3Args<T>& a, cudaStream_t s);
// the pipelined pass 3 of the CG applications (OP_ISO, OP_NH_APPLY, OP_CP_APPLY, OP_SVK_APPLY)
template <typename T> cudaError_t launch_ax3_pipe(int opk, const Ax3Args<T>& a, cudaStream_t s);
// pass 3 of the St. Venant-Kirchhoff law (OP_SVK_APPLY in both precisions, OP_SVK_UPDATE in FP64),
// plain and pipelined; compiled in translation units of their own
template <typename T> cudaError_t launch_ax3_svk(int opk, const Ax3Args<T>& a, cudaStream_t s);
// pass 3 of finite-strain crystal plasticity (OP_FCP_APPLY in both precisions, OP_FCP_UPDATE[32] in FP64)
template <typename T> cudaError_t launch_ax3_fcp(int opk, const Ax3Args<T>& a, cudaStream_t s);
// compatibility of the gradient field W (small: curl curl eps; finite: curl F):
// per-RHS partial sums of |.|^2 over the spectrum into partials [B][nblk]
cudaError_t launch_compat(const Dims& d, const Freq<double>& f, const cplx<double>* W, double* partials, int nblk,
                          cudaStream_t s);
// odd transform lengths (prime factors 3, 5, 7; Sec. 2.1's odd grids), compiled in
// translation units of their own: strided C2C along axis 1 or 2, and pass 3
// for linear isotropic phases (OP_ISO) with odd n3
#define DBFFT_ODD_SIZES(X) X(9) X(15) X(21) X(25) X(27) X(35) X(45) X(49) X(63) X(75) X(81) X(105) \
    X(125) X(135) X(147) X(175) X(189) X(225) X(243) X(245)
// odd n3 with the nonlinear models (their pass-3 instantiations)
#define DBFFT_ODD_NL_SIZES(X) X(9) X(15) X(21) X(27) X(45) X(63) X(81)
bool supported_odd(int n);
bool supported_odd_nl(int n);
template <typename T> cudaError_t launch_fft_odd(int dir, int axis, Ax2Args<T> a, cudaStream_t s);
template <typename T> cudaError_t launch_ax3_odd(int opk, const Ax3Args<T>& a, cudaStream_t s);
// the nonlinear operations of the odd pass 3 (translation units of their own)
template <typename T> cudaError_t launch_ax3_odd_nl(int opk, const Ax3Args<T>& a, cudaStream_t s);
cudaError_t launch_ax3_odd_cp(int opk, const Ax3Args<double>& a, cudaStream_t s);
template <typename T> cudaError_t launch_ax3_odd_fcp(int opk, const Ax3Args<T>& a, cudaStream_t s);
// lines per CTA of the odd pass 3 (one right-hand side per CTA; nc components)
int ax3_odd_lines(int n3, int nc, bool dbl);
// pass 3 of the post-processing transforms (OP_DISP, FP64 only)
template <typename T> cudaError_t launch_ax3_post(int opk, const Ax3Args<T>& a, cudaStream_t s);
// the first and the last pass of the FP32 CG iteration with the element-wise work fused into
// the axis-2 transforms (n2 = 32 .. 256): k_grad + inverse axis-2 C2C, forward axis-2 C2C + k_div
cudaError_t launch_grad_ax2(const Ax1InvArgs<float>& a, cudaStream_t s);
cudaError_t launch_ax2_div(const Ax1FwdArgs<float>& a, cudaStream_t s);
long long fused_ax2_blocks(int n1, int h);  // CTAs per right-hand side of both
bool fused_ax2_supported(int n2);
int fused_tw();  // columns per CTA of the fused passes
// pass 3 of the FP32 CG applications on long lines (n3 = 128, 256; OP_ISO, OP_CP_APPLY, OP_NH_APPLY):
// one tile of a.L grid lines per CTA moved by bulk copies, two-stage transforms in registers (pipe = 3)
cudaError_t launch_ax3_lb(int opk, const Ax3Args<float>& a, cudaStream_t s);
// shared memory of one such CTA, or -1 when (n3, nc, L) is not a valid tile
long long ax3_lb_smem(int n3, int nc, int rb, bool scale, int L, long long nlines);
// shared memory of one pipelined CTA (pipe 1: two stages, 2: one stage), or -1 when (n3, L) is not a valid tile
long long ax3_pipe_smem(int n3, int nc, int rb, bool dbl, bool scale, int radix, int L, long long nlines, int pipe);

}  // namespace dbfft
