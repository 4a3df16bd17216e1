// misc.h -- launchers of the small kernels in k_misc.cu.
#pragma once
#include "launch.h"

namespace dbfft {
cudaError_t launch_macro(int B, int nc, const int* activeflag, const double* fU, const double* e, double* macroW,
                         float* macroWf, cudaStream_t s);
template <typename Ti>
cudaError_t launch_to_inner(const Dims& d, const cplx<double>* r64, const double* re64, const double* sc, cplx<Ti>* ri,
                            double* re_i, cplx<Ti>* xi, double* xe_i, cudaStream_t s);
template <typename Ti>
cudaError_t launch_from_inner(const Dims& d, const cplx<Ti>* xi, const cplx<Ti>* pi, const CgState* cg,
                              const double* xe_i, const double* sb, cplx<double>* x64, double* xe64, cudaStream_t s);
template <typename T>
cudaError_t launch_precond_field(const Dims& d, const Freq<T>& f, const PrecondData* pre, const cplx<T>* u,
                                 cplx<T>* out, const double* e_in, double* e_out, cudaStream_t s);
template <typename TT>
cudaError_t launch_mean_tangent(int kind, int B, long long V, const TT* tan, const uint16_t* phase, const double* lam,
                                const double* mu, double* partials, int nblk, cudaStream_t s);
template <typename T>
cudaError_t launch_herm_planes(const Dims& d, cplx<T>* v, cudaStream_t s);
// n row-major 3x3 identity matrices at m[9 n]
cudaError_t launch_fill_identity(double* m, long long n, cudaStream_t s);
// device-resident material maps: per-map phase counts [Bm][np] (ids >= np counted in *bad), and the FP32
// copy of the stiffness scale with its non-finite count and per-block sums of lam(id) s, mu(id) s
cudaError_t launch_phase_counts(const uint16_t* phase, int Bm, long long V, int np, unsigned long long* counts,
                                unsigned long long* bad, cudaStream_t s);
cudaError_t launch_scale_stats(const uint16_t* phase, const double* scale, float* scale_f, int Bm, long long V, int np,
                               const double* lam, const double* mu, double* partials, int nblk,
                               unsigned long long* bad, cudaStream_t s);
// effective-stiffness sensitivity: six-term combinations of the six solutions of each
// material map (out[g 6 + I] = sum_J G[g][I][J] x[g 6 + J], n complex values each), and
// the sum of the six per-right-hand-side fields of each map
cudaError_t launch_combine6(const cplx<double>* x, const double* G, cplx<double>* out, long long n, int Bm,
                            cudaStream_t s);
cudaError_t launch_sum6(const double* tmp, double* out, long long V, int Bm, cudaStream_t s);
// sigma-hat of every right-hand side from the unit-strain stress spectra of each
// material map (linear isotropic phases, zero fluctuation; Bm <= 8, nc = 6)
cudaError_t launch_affine_combine(const Dims& d, int Bm, cplx<double>* W, const double* macroW, cudaStream_t s);
// per-voxel steps of the crystal-plasticity adjoint (k_cpadj.cu): post = 0 writes the
// tangent T_n (tan, may be null) and, with write_w, w = q + T_n (a - S q); post = 1
// reads e_lam from w, accumulates dJds and updates q
cudaError_t launch_cp_adj(int post, int B, int Rm, long long V, const uint16_t* phase, const CpGrain* grains,
                          const CpParams& cp, const double* sig, double* q, const double* aw, double* w, double* tan,
                          double* dJds, unsigned* err, int write_w, cudaStream_t s);
// the calling thread's last failure message of dbfft_apply_iso_noalloc ("" if none)
const char* noalloc_last_error();
}  // namespace dbfft
