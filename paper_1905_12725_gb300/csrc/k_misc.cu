// k_misc.cu -- small kernels around the passes: macro fields, precision
// conversion between the FP64 outer loop and the inner CG, the
// preconditioner as a stand-alone operator, and the mean tangent.
#include <algorithm>

#include "../../include/dbfft.h"
#include "launch.h"
#include "misc.h"

namespace dbfft {

__global__ void k_macro(int B, int nc, const int* activeflag, const double* fU, const double* e, double* macroW,
                        float* macroWf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 9) return;
    const int q = i % 9;
    double v = fU ? fU[i] : 0.0;
    if (e && activeflag[q]) v += ((nc == 6 && q >= 3) ? 0.70710678118654752440084436210485 : 1.0) * e[i];
    macroW[i] = v;
    if (macroWf) macroWf[i] = (float)v;
}

cudaError_t launch_macro(int B, int nc, const int* activeflag, const double* fU, const double* e, double* macroW,
                         float* macroWf, cudaStream_t s) {
    k_macro<<<(B * 9 + 127) / 128, 128, 0, s>>>(B, nc, activeflag, fU, e, macroW, macroWf);
    return cudaGetLastError();
}

template <typename Ti>
__global__ void k_to_inner(long long n3H, int B, const cplx<double>* r64, const double* re64, const double* sc,
                           cplx<Ti>* ri, double* re_i, cplx<Ti>* xi, double* xe_i) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    const double s = sc[b];
    if (i < n3H) {
        const cplx<double> v = r64[(long long)b * n3H + i];
        cplx<Ti> o;
        o.x = (Ti)(v.x * s);
        o.y = (Ti)(v.y * s);
        ri[(long long)b * n3H + i] = o;
        cplx<Ti> z;
        z.x = Ti(0);
        z.y = Ti(0);
        xi[(long long)b * n3H + i] = z;
    }
    if (blockIdx.x == 0 && threadIdx.x < 9) {
        re_i[b * 9 + threadIdx.x] = re64[b * 9 + threadIdx.x] * s;
        xe_i[b * 9 + threadIdx.x] = 0.0;
    }
}

// x64 += s (x_i + alpha p_i): the inner PCG applies each iterate update one
// iteration late (in the next pass 1), so the last alpha p is added here.
template <typename Ti>
__global__ void k_from_inner(long long n3H, int B, const cplx<Ti>* xi, const cplx<Ti>* pi, const CgState* cg,
                             const double* xe_i, const double* sb, cplx<double>* x64, double* xe64) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    const double s = sb[b];
    const Ti al = (Ti)cg[b].alpha;
    if (i < n3H) {
        cplx<double> v = x64[(long long)b * n3H + i];
        const cplx<Ti> dx = xi[(long long)b * n3H + i];
        const cplx<Ti> dp = pi[(long long)b * n3H + i];
        v.x += s * (double)(dx.x + al * dp.x);
        v.y += s * (double)(dx.y + al * dp.y);
        x64[(long long)b * n3H + i] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x < 9) xe64[b * 9 + threadIdx.x] += s * xe_i[b * 9 + threadIdx.x];
}

template <typename Ti>
cudaError_t launch_to_inner(const Dims& d, const cplx<double>* r64, const double* re64, const double* sc, cplx<Ti>* ri,
                            double* re_i, cplx<Ti>* xi, double* xe_i, cudaStream_t s) {
    const long long n = 3 * d.H;
    k_to_inner<Ti><<<dim3((unsigned)((n + 255) / 256), d.B), 256, 0, s>>>(n, d.B, r64, re64, sc, ri, re_i, xi, xe_i);
    return cudaGetLastError();
}
template <typename Ti>
cudaError_t launch_from_inner(const Dims& d, const cplx<Ti>* xi, const cplx<Ti>* pi, const CgState* cg,
                              const double* xe_i, const double* sb, cplx<double>* x64, double* xe64, cudaStream_t s) {
    const long long n = 3 * d.H;
    k_from_inner<Ti><<<dim3((unsigned)((n + 255) / 256), d.B), 256, 0, s>>>(n, d.B, xi, pi, cg, xe_i, sb, x64, xe64);
    return cudaGetLastError();
}
template cudaError_t launch_to_inner<float>(const Dims&, const cplx<double>*, const double*, const double*,
                                            cplx<float>*, double*, cplx<float>*, double*, cudaStream_t);
template cudaError_t launch_to_inner<double>(const Dims&, const cplx<double>*, const double*, const double*,
                                             cplx<double>*, double*, cplx<double>*, double*, cudaStream_t);
template cudaError_t launch_from_inner<float>(const Dims&, const cplx<float>*, const cplx<float>*, const CgState*,
                                              const double*, const double*, cplx<double>*, double*, cudaStream_t);
template cudaError_t launch_from_inner<double>(const Dims&, const cplx<double>*, const cplx<double>*, const CgState*,
                                               const double*, const double*, cplx<double>*, double*, cudaStream_t);

// out = M u: N Q(xi)^-1 u per frequency (zero on the null set), macro block Me e.
template <typename T>
__global__ void k_precond_field(Dims d, Freq<T> f, const PrecondData* pre, const cplx<T>* u, cplx<T>* out,
                                const double* e_in, double* e_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    const PrecondData& pd = pre[b / d.Rm];
    if (i < d.H) {
        const long long k1 = i / d.plane;
        const long long rem = i - k1 * d.plane;
        const int k2 = (int)(rem / d.h), k3 = (int)(rem - (long long)k2 * d.h);
        cplx<T> r[3], z[3];
        for (int c = 0; c < 3; ++c) r[c] = u[(long long)(b * 3 + c) * d.H + i];
        precond_pd<T>(pd, f.xi1[k1], f.xi2[k2], f.xi3[k3], (T)(1.0 / d.invN), r, z);
        for (int c = 0; c < 3; ++c) out[(long long)(b * 3 + c) * d.H + i] = z[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && e_out) {
        for (int q = 0; q < 9; ++q) e_out[b * 9 + q] = 0.0;
        for (int k = 0; k < d.ne; ++k) {
            double acc = 0.0;
            for (int l = 0; l < d.ne; ++l) acc += pd.Me[k][l] * (e_in ? e_in[b * 9 + d.active[l]] : 0.0);
            e_out[b * 9 + d.active[k]] = acc;
        }
    }
}

template <typename T>
cudaError_t launch_precond_field(const Dims& d, const Freq<T>& f, const PrecondData* pre, const cplx<T>* u,
                                 cplx<T>* out, const double* e_in, double* e_out, cudaStream_t s) {
    k_precond_field<T><<<dim3((unsigned)((d.H + 255) / 256), d.B), 256, 0, s>>>(d, f, pre, u, out, e_in, e_out);
    return cudaGetLastError();
}
template cudaError_t launch_precond_field<float>(const Dims&, const Freq<float>&, const PrecondData*,
                                                 const cplx<float>*, cplx<float>*, const double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_precond_field<double>(const Dims&, const Freq<double>&, const PrecondData*,
                                                  const cplx<double>*, cplx<double>*, const double*, double*,
                                                  cudaStream_t);

// Mean of the fourth-order tangent K_ijkl over the voxels of one right-hand
// side (81 components), from the stored tangent data:
//   kind 0: Neo-Hookean data (F^-T, mu - lam ln J) with per-phase mu, lam;
//   kind 1: 21-entry Mandel tangent;
//   kind 2: St. Venant-Kirchhoff data (F, S) with per-phase mu, lam;
//   kind 3: finite-strain crystal-plasticity data (45 values).
template <typename TT>
__global__ void k_mean_tangent(int kind, long long V, const TT* tan, const uint16_t* phase, const double* lam,
                               const double* mu, double* partials /* [B][gridDim.x][81] */) {
    __shared__ double acc[81];
    const int b = blockIdx.y;
    for (int q = threadIdx.x; q < 81; q += blockDim.x) acc[q] = 0.0;
    __syncthreads();
    if (kind == 0) {
        double loc[81];
        for (int q = 0; q < 81; ++q) loc[q] = 0.0;
        for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
            const TT* t = tan + ((long long)b * V + v) * 10;
            const int ph = phase[(long long)b * V + v];
            double A[9];
            for (int q = 0; q < 9; ++q) A[q] = (double)t[q];
            const double c1 = (double)t[9];
            // K_iJkL = mu d_ik d_JL + c1 A_iL A_kJ + lam A_iJ A_kL
            for (int i = 0; i < 3; ++i)
                for (int J = 0; J < 3; ++J)
                    for (int k = 0; k < 3; ++k)
                        for (int L = 0; L < 3; ++L) {
                            double val = c1 * A[3 * i + L] * A[3 * k + J] + lam[ph] * A[3 * i + J] * A[3 * k + L];
                            if (i == k && J == L) val += mu[ph];
                            loc[((i * 3 + J) * 3 + k) * 3 + L] += val;
                        }
        }
        for (int q = 0; q < 81; ++q) atomicAdd(&acc[q], loc[q]);
        __syncthreads();
    } else if (kind == 2) {
        // St. Venant-Kirchhoff, data (F, S):
        // K_iJkL = d_ik S_JL + lam F_iJ F_kL + mu (F_iL F_kJ + (F F^T)_ik d_JL)
        double loc[81];
        for (int q = 0; q < 81; ++q) loc[q] = 0.0;
        for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
            const TT* t = tan + ((long long)b * V + v) * 15;
            const int ph = phase[(long long)b * V + v];
            double F[9];
            for (int q = 0; q < 9; ++q) F[q] = (double)t[q];
            const int sidx[9] = {0, 5, 4, 5, 1, 3, 4, 3, 2};
            for (int i = 0; i < 3; ++i)
                for (int J = 0; J < 3; ++J)
                    for (int k = 0; k < 3; ++k)
                        for (int L = 0; L < 3; ++L) {
                            double val = lam[ph] * F[3 * i + J] * F[3 * k + L] + mu[ph] * F[3 * i + L] * F[3 * k + J];
                            if (i == k) val += (double)t[9 + sidx[3 * J + L]];
                            if (J == L)
                                val += mu[ph] * (F[3 * i] * F[3 * k] + F[3 * i + 1] * F[3 * k + 1] + F[3 * i + 2] * F[3 * k + 2]);
                            loc[((i * 3 + J) * 3 + k) * 3 + L] += val;
                        }
        }
        for (int q = 0; q < 81; ++q) atomicAdd(&acc[q], loc[q]);
        __syncthreads();
    } else if (kind == 3) {
        // finite-strain crystal plasticity, 45 values: column (k, L) of K is
        // the response to the unit gradient e_k (x) e_L
        double loc[81];
        for (int q = 0; q < 81; ++q) loc[q] = 0.0;
        for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
            const TT* t = tan + ((long long)b * V + v) * 45;
            double td[45];
            for (int q = 0; q < 45; ++q) td[q] = (double)t[q];
            for (int kl = 0; kl < 9; ++kl) {
                double G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, out[9];
                G[kl] = 1.0;
                fcp_apply<double>(td, G, out);
                for (int iJ = 0; iJ < 9; ++iJ) loc[iJ * 9 + kl] += out[iJ];
            }
        }
        for (int q = 0; q < 81; ++q) atomicAdd(&acc[q], loc[q]);
        __syncthreads();
    } else {
        // the mean is linear in the 21 Mandel entries: sum them (in TT per
        // thread, FP64 across threads), then expand the block's sums to the
        // fourth-order tensor once
        __shared__ double m21[21];
        for (int q = threadIdx.x; q < 21; q += blockDim.x) m21[q] = 0.0;
        __syncthreads();
        TT loc[21];
#pragma unroll
        for (int q = 0; q < 21; ++q) loc[q] = TT(0);
        for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
            const TT* t = tan + ((long long)b * V + v) * 21;
#pragma unroll
            for (int q = 0; q < 21; ++q) loc[q] += t[q];
        }
#pragma unroll
        for (int q = 0; q < 21; ++q) {
            double x = (double)loc[q];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&m21[q], x);
        }
        __syncthreads();
        if (threadIdx.x == 0) {  // Mandel -> tensor: K_ijkl = sum_mn Psi_m,ij Cm_mn Psi_n,kl
            const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
            for (int m = 0; m < 6; ++m)
                for (int n = 0; n < 6; ++n) {
                    const double c = m21[sym6(m, n)] * (m >= 3 ? 0.70710678118654752440 : 1.0) *
                                     (n >= 3 ? 0.70710678118654752440 : 1.0);
                    const int ii[2] = {pi[m], pj[m]}, jj[2] = {pj[m], pi[m]};
                    const int kk[2] = {pi[n], pj[n]}, ll[2] = {pj[n], pi[n]};
                    for (int s1 = 0; s1 < (m >= 3 ? 2 : 1); ++s1)
                        for (int s2 = 0; s2 < (n >= 3 ? 2 : 1); ++s2)
                            acc[((ii[s1] * 3 + jj[s1]) * 3 + kk[s2]) * 3 + ll[s2]] += c;
                }
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < 81; q += blockDim.x)
        partials[((long long)b * gridDim.x + blockIdx.x) * 81 + q] = acc[q];
}

template <typename TT>
cudaError_t launch_mean_tangent(int kind, int B, long long V, const TT* tan, const uint16_t* phase, const double* lam,
                                const double* mu, double* partials, int nblk, cudaStream_t s) {
    k_mean_tangent<TT><<<dim3(nblk, B), 256, 0, s>>>(kind, V, tan, phase, lam, mu, partials);
    return cudaGetLastError();
}
template cudaError_t launch_mean_tangent<float>(int, int, long long, const float*, const uint16_t*, const double*,
                                                const double*, double*, int, cudaStream_t);
template cudaError_t launch_mean_tangent<double>(int, int, long long, const double*, const uint16_t*,
                                                 const double*, const double*, double*, int, cudaStream_t);

// Project [B][3][H] half spectra onto Hermitian-consistent vectors: on the
// planes k3 = 0 and (even n3) k3 = n3/2 the pair (k1, k2) / (-k1, -k2) is replaced by
// its conjugate-symmetric part (one thread per pair).
template <typename T>
__global__ void k_herm_planes(Dims d, cplx<T>* v) {
    const long long per = (long long)d.n1 * d.n2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per * (d.n3 % 2 == 0 ? 2 : 1)) return;  // odd n3: the plane k3 = 0 only
    const int plane = (int)(i / per);
    const long long j = i - plane * per;
    const int k1 = (int)(j / d.n2), k2 = (int)(j - (long long)k1 * d.n2);
    const int q1 = (d.n1 - k1) % d.n1, q2 = (d.n2 - k2) % d.n2;
    const long long jq = (long long)q1 * d.n2 + q2;
    if (jq < j) return;
    const int k3 = plane == 0 ? 0 : d.m;
    const int bc = blockIdx.y;  // b * 3 + c
    cplx<T>* base = v + (long long)bc * d.H;
    const long long a = ((long long)k1 * d.n2 + k2) * d.h + k3;
    const long long bq = ((long long)q1 * d.n2 + q2) * d.h + k3;
    cplx<T> x = base[a], y = base[bq];
    cplx<T> s;
    s.x = T(0.5) * (x.x + y.x);
    s.y = T(0.5) * (x.y - y.y);
    if (jq == j) s.y = T(0);
    base[a] = s;
    s.y = -s.y;
    base[bq] = s;
}

template <typename T>
cudaError_t launch_herm_planes(const Dims& d, cplx<T>* v, cudaStream_t s) {
    const long long n = 2LL * d.n1 * d.n2;
    k_herm_planes<T><<<dim3((unsigned)((n + 255) / 256), d.B * 3), 256, 0, s>>>(d, v);
    return cudaGetLastError();
}
template cudaError_t launch_herm_planes<double>(const Dims&, cplx<double>*, cudaStream_t);
template cudaError_t launch_herm_planes<float>(const Dims&, cplx<float>*, cudaStream_t);

__global__ void k_fill_identity(double* m, long long n9) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n9) m[i] = (i % 9 == 0 || i % 9 == 4 || i % 9 == 8) ? 1.0 : 0.0;
}

cudaError_t launch_fill_identity(double* m, long long n, cudaStream_t s) {
    const long long n9 = 9 * n;
    if (n9 == 0) return cudaSuccess;
    k_fill_identity<<<(unsigned)((n9 + 255) / 256), 256, 0, s>>>(m, n9);
    return cudaGetLastError();
}

}  // namespace dbfft

namespace dbfft {

// Levi-Civita symbol e_ijk.
__device__ __forceinline__ int levi(int i, int j, int k) {
    return (i == j || j == k || i == k) ? 0 : (((j - i + 3) % 3 == 1) ? 1 : -1);
}

// Compatibility of the gradient field W ([B][nc][H], Fourier coefficients of the
// real field; Sec. 3's compatibility check): small strain eta = curl (curl eps)^T,
// eta_ij = -e_ikl e_jmn xi_k xi_m eps_ln; finite strain (curl F)_iJ =
// i e_JKL xi_K F_iL. Per right-hand side the whole-spectrum sum of |.|^2 (half
// spectrum with weights), i.e. the mean of |.|^2 over the cell (Parseval).
template <int NC>
__global__ void k_compat(Dims d, Freq<double> f, const cplx<double>* W, double* partials) {
    __shared__ double red[32];
    const int b = blockIdx.y;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.H;
         i += (long long)gridDim.x * blockDim.x) {
        const FreqIdx fi = freq_idx(d, i);
        const double xi[3] = {f.xi1[fi.k1], f.xi2[fi.k2], f.xi3[fi.k3]};
        const double wgt = hweight(fi.k3, d.m);
        cplx<double> w[NC];
        for (int c = 0; c < NC; ++c) w[c] = W[(long long)(b * NC + c) * d.H + i];
        double s = 0.0;
        if (NC == 6) {
            const int ci[6] = {0, 1, 2, 1, 0, 0}, cj[6] = {0, 1, 2, 2, 2, 1};
            cplx<double> E[3][3];
            for (int c = 0; c < 6; ++c) E[ci[c]][cj[c]] = E[cj[c]][ci[c]] = w[c];
            for (int ii = 0; ii < 3; ++ii)
                for (int jj = 0; jj < 3; ++jj) {
                    double er = 0.0, ei = 0.0;
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) {
                            const int e1 = levi(ii, k, l);
                            if (!e1) continue;
                            for (int m = 0; m < 3; ++m)
                                for (int n = 0; n < 3; ++n) {
                                    const int e2 = levi(jj, m, n);
                                    if (!e2) continue;
                                    const double c = -(double)(e1 * e2) * xi[k] * xi[m];
                                    er += c * E[l][n].x;
                                    ei += c * E[l][n].y;
                                }
                        }
                    s += er * er + ei * ei;
                }
        } else {
            for (int ii = 0; ii < 3; ++ii)
                for (int J = 0; J < 3; ++J) {
                    double er = 0.0, ei = 0.0;
                    for (int K = 0; K < 3; ++K)
                        for (int L = 0; L < 3; ++L) {
                            const int e1 = levi(J, K, L);
                            if (!e1) continue;
                            er += e1 * xi[K] * w[3 * ii + L].x;
                            ei += e1 * xi[K] * w[3 * ii + L].y;
                        }
                    s += er * er + ei * ei;  // |i (er + i ei)|^2
                }
        }
        acc += wgt * s;
    }
    double v1[1] = {acc};
    block_sum<1>(v1, red);
    if (threadIdx.x == 0) partials[(long long)b * gridDim.x + blockIdx.x] = v1[0];
}

cudaError_t launch_compat(const Dims& d, const Freq<double>& f, const cplx<double>* W, double* partials, int nblk,
                          cudaStream_t s) {
    if (d.nc == 6) k_compat<6><<<dim3(nblk, d.B), 256, 0, s>>>(d, f, W, partials);
    else k_compat<9><<<dim3(nblk, d.B), 256, 0, s>>>(d, f, W, partials);
    return cudaGetLastError();
}

}  // namespace dbfft

namespace dbfft {

// Device-resident material maps (dbfft_materials.device_arrays): what the host
// path computes from host arrays at creation, computed where the maps are.
// k_phase_counts: voxels of each phase id per material map (a block histogram
// in shared memory, added to counts [Bm][np]); ids at or beyond np counted in *bad.
constexpr int kHistShared = 8192;  // phase ids counted in shared memory (more: global atomics)

__global__ void k_phase_counts(const uint16_t* __restrict__ phase, long long V, int np,
                               unsigned long long* counts, unsigned long long* bad) {
    __shared__ unsigned hist[kHistShared];
    const int g = blockIdx.y;
    const bool sh = np <= kHistShared;
    if (sh)
        for (int k = threadIdx.x; k < np; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    unsigned nbad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        const int id = phase[(long long)g * V + i];
        if (id >= np) ++nbad;
        else if (sh) atomicAdd(&hist[id], 1u);
        else atomicAdd(&counts[(long long)g * np + id], 1ull);
    }
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
    __syncthreads();
    if (sh)
        for (int k = threadIdx.x; k < np; k += blockDim.x)
            if (hist[k]) atomicAdd(&counts[(long long)g * np + k], (unsigned long long)hist[k]);
}

// k_scale_stats: FP32 copy of the per-voxel stiffness scale, a count of
// non-finite values, and per-block partial sums of lam(id) s and mu(id) s
// (partials [Bm][nblk][2], summed in a fixed order on the host).
__global__ void k_scale_stats(const uint16_t* __restrict__ phase, const double* __restrict__ scale, float* scale_f,
                              long long V, int np, const double* lam, const double* mu, double* partials,
                              unsigned long long* bad) {
    __shared__ double red[32 * 2];
    const int g = blockIdx.y;
    double v[2] = {0.0, 0.0};
    unsigned nbad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
        const long long j = (long long)g * V + i;
        const double s = scale[j];
        scale_f[j] = (float)s;
        if (!isfinite(s)) ++nbad;
        const int id = phase[j];
        if (id < np) {
            v[0] += lam[id] * s;
            v[1] += mu[id] * s;
        }
    }
    if (nbad) atomicAdd(bad, (unsigned long long)nbad);
    block_sum<2>(v, red);
    if (threadIdx.x == 0) {
        partials[((long long)g * gridDim.x + blockIdx.x) * 2 + 0] = v[0];
        partials[((long long)g * gridDim.x + blockIdx.x) * 2 + 1] = v[1];
    }
}

cudaError_t launch_phase_counts(const uint16_t* phase, int Bm, long long V, int np, unsigned long long* counts,
                                unsigned long long* bad, cudaStream_t s) {
    const long long nb = std::min<long long>((V + 255) / 256, 1024);
    k_phase_counts<<<dim3((unsigned)nb, (unsigned)Bm), 256, 0, s>>>(phase, V, np, counts, bad);
    return cudaGetLastError();
}

cudaError_t launch_scale_stats(const uint16_t* phase, const double* scale, float* scale_f, int Bm, long long V, int np,
                               const double* lam, const double* mu, double* partials, int nblk,
                               unsigned long long* bad, cudaStream_t s) {
    k_scale_stats<<<dim3((unsigned)nblk, (unsigned)Bm), 256, 0, s>>>(phase, scale, scale_f, V, np, lam, mu, partials,
                                                                    bad);
    return cudaGetLastError();
}

}  // namespace dbfft

namespace dbfft {

// Effective-stiffness sensitivity: out[g 6 + I] = sum_J G[g][I][J] x[g 6 + J]
// over the n = 3 H complex values of each right-hand side (six per material map).
__global__ void k_combine6(const cplx<double>* __restrict__ x, const double* __restrict__ G, cplx<double>* out,
                           long long n) {
    const int g = blockIdx.y / 6, I = blockIdx.y % 6;
    double c[6];
#pragma unroll
    for (int J = 0; J < 6; ++J) c[J] = G[(g * 6 + I) * 6 + J];
    const cplx<double>* xg = x + (long long)g * 6 * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        cplx<double> s = zero_c<double>();
#pragma unroll
        for (int J = 0; J < 6; ++J) s = s + c[J] * ldc(xg + J * n + i);
        stc(out + (long long)blockIdx.y * n + i, s);
    }
}

// out[g][v] = sum over the six right-hand sides of map g of tmp[g 6 + I][v]
__global__ void k_sum6(const double* __restrict__ tmp, double* out, long long V) {
    const int g = blockIdx.y;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
#pragma unroll
        for (int I = 0; I < 6; ++I) s += tmp[((long long)g * 6 + I) * V + v];
        out[(long long)g * V + v] = s;
    }
}

cudaError_t launch_combine6(const cplx<double>* x, const double* G, cplx<double>* out, long long n, int Bm,
                            cudaStream_t s) {
    const long long nb = std::min<long long>((n + 255) / 256, 512);
    k_combine6<<<dim3((unsigned)nb, (unsigned)(6 * Bm)), 256, 0, s>>>(x, G, out, n);
    return cudaGetLastError();
}

// The stress spectra of all right-hand sides at zero fluctuation, for linear
// isotropic phases: sigma(x) = lambda(x) tr(E) I + 2 mu(x) E is linear in the two
// fields lambda(x), mu(x), so with s the stress of the unit strain e11 of the
// same material map (s11 = lambda + 2 mu, s22 = lambda), every right-hand side
// is sigma = tr(E) s22 I + (s11 - s22) E, component by component and, the
// transform being linear, frequency by frequency. W holds the transformed s of
// map m in the slots of right-hand side m (components 0 and 1); all of them are
// read before any right-hand side is written (Bm <= 8).
__global__ void k_affine_combine(Dims d, int Bm, cplx<double>* W, const double* __restrict__ macroW) {
    const long long H = d.H;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < H; i += (long long)gridDim.x * blockDim.x) {
        cplx<double> s22[8], dif[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if (m >= Bm) break;
            s22[m] = ldc(W + (long long)(m * 6 + 1) * H + i);
            dif[m] = ldc(W + (long long)(m * 6 + 0) * H + i) - s22[m];
        }
        for (int b = 0; b < d.B; ++b) {
            const int m = b / d.Rm;
            cplx<double> sm = s22[0], dm = dif[0];  // the map's values by selection (no arithmetic)
#pragma unroll
            for (int mm = 1; mm < 8; ++mm)
                if (mm == m) {
                    sm = s22[mm];
                    dm = dif[mm];
                }
            const double* E = macroW + b * 9;
            const cplx<double> iso = (E[0] + E[1] + E[2]) * sm;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const cplx<double> v = c < 3 ? iso + E[c] * dm : E[c] * dm;
                stc(W + (long long)(b * 6 + c) * H + i, v);
            }
        }
    }
}

cudaError_t launch_affine_combine(const Dims& d, int Bm, cplx<double>* W, const double* macroW, cudaStream_t s) {
    if (Bm < 1 || Bm > 8 || d.nc != 6) return cudaErrorInvalidValue;
    const long long nb = std::min<long long>((d.H + 255) / 256, 1216);
    k_affine_combine<<<(unsigned)nb, 256, 0, s>>>(d, Bm, W, macroW);
    return cudaGetLastError();
}

cudaError_t launch_sum6(const double* tmp, double* out, long long V, int Bm, cudaStream_t s) {
    const long long nb = std::min<long long>((V + 255) / 256, 1024);
    k_sum6<<<dim3((unsigned)nb, (unsigned)Bm), 256, 0, s>>>(tmp, out, V);
    return cudaGetLastError();
}

}  // namespace dbfft

namespace dbfft {

// FP64 fused multiply-add rate: eight independent dependency chains per
// thread, so that the FP64 pipe, not the latency of one chain, sets the pace.
__global__ void k_fp64_fma(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// L2 copy rate: every thread copies float4 elements of a buffer that fits in
// L2, reps times over, so that after the first sweep reads and writes hit L2.
__global__ void k_l2_copy(const float4* __restrict__ src, float4* __restrict__ dst, long long n, int reps) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            float4 v = __ldcg(src + i);
            v.x += 1.0f;
            __stcg(dst + i, v);
        }
}

}  // namespace dbfft

extern "C" dbfft_status dbfft_l2_copy_rate(double* gbs, void* stream) {
    using namespace dbfft;
    if (!gbs) return DBFFT_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DBFFT_E_CUDA;
    const long long bytes = 16LL << 20;  // each of source and destination: 32 MB in all
    const long long n = bytes / (long long)sizeof(float4);
    const int reps = 32;
    float4* buf = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&buf), 2 * (size_t)bytes, s) != cudaSuccess) return DBFFT_E_NOMEM;
    cudaMemsetAsync(buf, 0, 2 * (size_t)bytes, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, s);
        k_l2_copy<<<nsm * 8, 256, 0, s>>>(buf, buf + n, n, reps);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = ms < best ? ms : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    const bool ok = cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    *gbs = 2.0 * (double)bytes * reps / (best * 1e-3) / 1e9;
    return ok ? DBFFT_OK : DBFFT_E_CUDA;
}

extern "C" dbfft_status dbfft_fp64_fma_rate(double* tflops, void* stream) {
    using namespace dbfft;
    if (!tflops) return DBFFT_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DBFFT_E_CUDA;
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    double* out = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&out), (size_t)blocks * threads * sizeof(double), s) != cudaSuccess)
        return DBFFT_E_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, s);
        k_fp64_fma<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = ms < best ? ms : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    const bool ok = cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
    return ok ? DBFFT_OK : DBFFT_E_CUDA;
}
