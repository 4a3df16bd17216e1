// passes.cuh -- the five passes of one DBFFT operator application and the
// small kernels of the preconditioned CG around them.
//
// Layout of the work buffer W: [B][nc][n1][n2][h] interleaved complex with
// h = n3/2 + 1 (nc = 6 strain components 11,22,33,23,13,12 at small strain,
// nc = 9 components 3i+j of the displacement gradient at finite strain).
//
//   pass 1  axis 2, inverse : u (3 comps) -> s.u or g.u (nc comps), C2C   [k_pass1]
//   pass 2  axis 1, inverse : C2C                                         [k_fft_strided]
//   pass 3  axis 3          : C2R, per-voxel tangent / constitutive, R2C  [k_axis3]
//   pass 4  axis 1, forward : C2C                                         [k_fft_strided]
//   pass 5  axis 2, forward : C2C, divergence d:sigma, null mask, CG      [k_pass5]
//
// The fused passes run along axis 2, whose stride (n3/2 + 1 entries) keeps a
// column tile inside one compact region; the pure transforms run along
// axis 1 (stride n2 (n3/2 + 1)) with wide tiles.
//
// Inside CG, pass 1 also forms the new search direction p = M r + beta p
// (the preconditioner of Sec. 2.5 evaluated on the fly from the frequency),
// pass 3 accumulates the curvature <p, K p> = sum_x eps : C : eps and its last
// block sets alpha, and pass 5 applies x += alpha p, r -= alpha q, evaluates
// <r, M r> and ||r||^2 and its last block sets beta and the stop flag. The
// product q = K p never reaches memory.
#pragma once
#include "dbfft_dev.cuh"

namespace dbfft {

// ------------------------------------------------------------------ helpers
template <typename T>
__device__ __forceinline__ cplx<T> zero_c() { return mk<T>(T(0), T(0)); }

// Stored weight of a half-spectrum entry in the full-spectrum inner product.
__device__ __forceinline__ int hweight(int k3, int m) { return (k3 == 0 || k3 == m) ? 1 : 2; }

// z = N Q(xi)^-1 r (zero on the null set), Q from the mean tangent.
// 1/x: the correctly rounded FP32 reciprocal instruction, or an FP64 division.
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }

template <typename T>
__device__ __forceinline__ void precond_apply(const T (*coef)[6], T x1, T x2, T x3, T N,
                                              const cplx<T>* r, cplx<T>* z) {
    const T k2 = x1 * x1 + x2 * x2 + x3 * x3;
    if (k2 == T(0)) {
        z[0] = z[1] = z[2] = zero_c<T>();
        return;
    }
    const T ik2 = rcp_t(k2);
    const T mono[6] = {x1 * x1 * ik2, x2 * x2 * ik2, x3 * x3 * ik2,
                       x2 * x3 * ik2, x1 * x3 * ik2, x1 * x2 * ik2};
    T q[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < 6; ++b) s += coef[a][b] * mono[b];
        q[a] = s;
    }
    // Q = [[q0 q5 q4] [q5 q1 q3] [q4 q3 q2]], inverse by cofactors
    const T A00 = q[1] * q[2] - q[3] * q[3];
    const T A11 = q[0] * q[2] - q[4] * q[4];
    const T A22 = q[0] * q[1] - q[5] * q[5];
    const T A01 = q[4] * q[3] - q[5] * q[2];
    const T A02 = q[5] * q[3] - q[4] * q[1];
    const T A12 = q[5] * q[4] - q[0] * q[3];
    const T det = q[0] * A00 + q[5] * A01 + q[4] * A02;
    const T s = N * ik2 * rcp_t(det);
    z[0] = s * (A00 * r[0] + (A01 * r[1] + A02 * r[2]));
    z[1] = s * (A01 * r[0] + (A11 * r[1] + A12 * r[2]));
    z[2] = s * (A02 * r[0] + (A12 * r[1] + A22 * r[2]));
}

// The preconditioner of one material group: the closed form for an isotropic
// mean tangent, z = N / |xi|^2 (r - c (xi . r) xi / |xi|^2) / mu0 (the same
// operator as the general 3x3 inverse above, up to rounding), else the general form.
template <typename T>
__device__ __forceinline__ void precond_pd(const PrecondData& pd, T x1, T x2, T x3, T N, const cplx<T>* r,
                                           cplx<T>* z) {
    if (pd.iso) {
        const T k2 = x1 * x1 + x2 * x2 + x3 * x3;
        if (k2 == T(0)) {
            z[0] = z[1] = z[2] = zero_c<T>();
            return;
        }
        const T* iso = piso<T>(pd);
        const T ik2 = rcp_t(k2);
        const T s = N * ik2 * iso[0];
        const cplx<T> xr = x1 * r[0] + x2 * r[1] + x3 * r[2];
        const T cc = iso[1] * ik2;
        const cplx<T> w = cc * xr;
        z[0] = s * (r[0] - x1 * w);
        z[1] = s * (r[1] - x2 * w);
        z[2] = s * (r[2] - x3 * w);
        return;
    }
    precond_apply<T>(pcoef<T>(pd), x1, x2, x3, N, r, z);
}

// scalar * complex helpers for the real-scalar product
template <typename T>
__device__ __forceinline__ cplx<T> operator*(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }

// Block-wide sum of NV doubles; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* scratch /* >= 32*NV */) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    const int lane = threadIdx.x % 32 + 0, warp = (threadIdx.x + threadIdx.y * blockDim.x) / 32;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nwarps = (blockDim.x * blockDim.y + 31) / 32;
    __syncthreads();
    if ((tid & 31) == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp * NV + k] = v[k];
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += scratch[w * NV + k];
            v[k] = s;
        }
    }
    (void)lane;
}

// Block-wide sum of NV values held in precision T: warp sums in T, the
// per-warp partials combined in FP64 by thread 0 (result valid there).
template <typename T, int NV>
__device__ __forceinline__ void block_sum_t(const T* vin, double* out, double* scratch /* >= 32*NV */) {
    T v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        v[k] = vin[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int warp = tid / 32;
    const int nwarps = (blockDim.x * blockDim.y + 31) / 32;
    __syncthreads();
    if ((tid & 31) == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) scratch[warp * NV + k] = (double)v[k];
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += scratch[w * NV + k];
            out[k] = s;
        }
    }
}

// Symmetric-gradient / gradient component m of u at xi, times (i * invN).
template <typename T, int NC, int M>
__device__ __forceinline__ cplx<T> grad_comp(const cplx<T>* u, T x1, T x2, T x3, T s) {
    if constexpr (NC == 6) {
        const T h = T(0.5) * s;
        if constexpr (M == 0) return mul_i(s * x1, u[0]);
        if constexpr (M == 1) return mul_i(s * x2, u[1]);
        if constexpr (M == 2) return mul_i(s * x3, u[2]);
        if constexpr (M == 3) return mul_i(h, x3 * u[1] + x2 * u[2]);
        if constexpr (M == 4) return mul_i(h, x3 * u[0] + x1 * u[2]);
        if constexpr (M == 5) return mul_i(h, x2 * u[0] + x1 * u[1]);
    } else {
        constexpr int i = M / 3, j = M % 3;
        const T xj = j == 0 ? x1 : (j == 1 ? x2 : x3);
        return mul_i(s * xj, u[i]);
    }
    return zero_c<T>();
}

// Accumulate the divergence contribution of stress component m:
// acc_i += xi_j sigma_ij (the factor -i/N is applied at the end).
template <typename T, int NC, int M>
__device__ __forceinline__ void div_acc(cplx<T>* acc, cplx<T> s, T x1, T x2, T x3) {
    if constexpr (NC == 6) {
        if constexpr (M == 0) acc[0] = acc[0] + x1 * s;
        if constexpr (M == 1) acc[1] = acc[1] + x2 * s;
        if constexpr (M == 2) acc[2] = acc[2] + x3 * s;
        if constexpr (M == 3) { acc[1] = acc[1] + x3 * s; acc[2] = acc[2] + x2 * s; }
        if constexpr (M == 4) { acc[0] = acc[0] + x3 * s; acc[2] = acc[2] + x1 * s; }
        if constexpr (M == 5) { acc[0] = acc[0] + x2 * s; acc[1] = acc[1] + x1 * s; }
    } else {
        constexpr int i = M / 3, j = M % 3;
        const T xj = j == 0 ? x1 : (j == 1 ? x2 : x3);
        acc[i] = acc[i] + xj * s;
    }
}

// Macro basis: W-component value of unit macro coefficient m, and the
// coefficient of a stress tensor on basis m (E^T sigma).
template <int NC>
__host__ __device__ __forceinline__ double macro_to_w(int m) {
    return (NC == 6 && m >= 3) ? 0.70710678118654752440084436210485 : 1.0;
}
template <int NC>
__host__ __device__ __forceinline__ double w_to_macro(int m) {
    return (NC == 6 && m >= 3) ? 1.41421356237309504880168872420970 : 1.0;
}

// ------------------------------------------------------------------ pass 1
enum { AX1_PLAIN = 0, AX1_CG = 1 };

template <typename T>
struct Ax1InvArgs {
    Dims d;
    Freq<T> f;
    Twiddles<T> tw;
    const cplx<T>* in;   // PLAIN: u [B][3][H]; CG: r [B][3][H]
    cplx<T>* p;          // CG: search direction [B][3][H], updated in place
    cplx<T>* x;          // CG: iterate [B][3][H]; x += alpha_prev p_old is applied here
    cplx<T>* W;          // [B][nc][H]
    const CgState* cg;   // CG (beta, done)
    const PrecondData* pre;  // [B / Rm] per material group
};

// Threads per CTA of the element-wise kernels of passes 1 and 5.
constexpr int PW_THREADS = 256;

// Frequency indices of half-spectrum entry i (k3 fastest).
struct FreqIdx {
    int k1, k2, k3;
};
__device__ __forceinline__ FreqIdx freq_idx(const Dims& d, long long i) {
    FreqIdx f;
    const unsigned u = (unsigned)i;  // i < H < 2^32
    const unsigned k1 = fastdiv(u, d.div_plane);
    const unsigned rem = u - k1 * d.div_plane.d;
    const unsigned k2 = fastdiv(rem, d.div_h);
    f.k1 = (int)k1;
    f.k2 = (int)k2;
    f.k3 = (int)(rem - k2 * d.div_h.d);
    return f;
}

// Pass 1a, element-wise over frequencies: the Fourier (symmetric) gradient of
// u scaled by 1/N (the inverse transforms that follow are unnormalised).
// In CG mode u is the new search direction p = M r + beta p_old, formed here
// from r, together with the deferred iterate update x += alpha_prev p_old.
template <typename T, int NC, int MODE>
__global__ void __launch_bounds__(PW_THREADS) k_grad(Ax1InvArgs<T> a) {
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    const int b = blockIdx.y;
    if (MODE == AX1_CG && a.cg[b].done) return;
    const Dims& d = a.d;
    const T s = (T)d.invN;
    T beta = T(0), alpha = T(0), N = T(0);
    const PrecondData* pd = nullptr;
    if constexpr (MODE == AX1_CG) {
        beta = (T)a.cg[b].beta;
        alpha = (T)a.cg[b].alpha;
        N = (T)(1.0 / d.invN);
        pd = a.pre + b / d.Rm;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.H; i += (long long)gridDim.x * blockDim.x) {
        const FreqIdx fi = freq_idx(d, i);
        const T x1 = a.f.xi1[fi.k1], x2 = a.f.xi2[fi.k2], x3 = a.f.xi3[fi.k3];
        cplx<T> u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = ldc(a.in + (long long)(b * 3 + c) * d.H + i);
        if constexpr (MODE == AX1_CG) {
            cplx<T> z[3], po[3], xo[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                po[c] = ldc(a.p + (long long)(b * 3 + c) * d.H + i);
                xo[c] = ldc(a.x + (long long)(b * 3 + c) * d.H + i);
            }
            precond_pd<T>(*pd, x1, x2, x3, N, u, z);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                u[c] = z[c] + po[c] * beta;
                stc(a.p + (long long)(b * 3 + c) * d.H + i, u[c]);
                stc(a.x + (long long)(b * 3 + c) * d.H + i, xo[c] + po[c] * alpha);
            }
        }
        cplx<T>* Wb = a.W + (long long)b * NC * d.H + i;
        stc(Wb + 0 * d.H, grad_comp<T, NC, 0>(u, x1, x2, x3, s));
        stc(Wb + 1 * d.H, grad_comp<T, NC, 1>(u, x1, x2, x3, s));
        stc(Wb + 2 * d.H, grad_comp<T, NC, 2>(u, x1, x2, x3, s));
        stc(Wb + 3 * d.H, grad_comp<T, NC, 3>(u, x1, x2, x3, s));
        stc(Wb + 4 * d.H, grad_comp<T, NC, 4>(u, x1, x2, x3, s));
        stc(Wb + 5 * d.H, grad_comp<T, NC, 5>(u, x1, x2, x3, s));
        if constexpr (NC == 9) {
            stc(Wb + 6 * d.H, grad_comp<T, NC, 6>(u, x1, x2, x3, s));
            stc(Wb + 7 * d.H, grad_comp<T, NC, 7>(u, x1, x2, x3, s));
            stc(Wb + 8 * d.H, grad_comp<T, NC, 8>(u, x1, x2, x3, s));
        }
    }
}

// ------------------------------------------------------------------ pass 2/4
// Pure C2C transform of length N along a strided axis: column col = outer *
// inner + in (in < inner), element t at outer * N * inner + t * inner + in.
// Axis 1: inner = n2 h, outer = b * nc + c. A warp covers consecutive
// columns, so every row segment of a tile is contiguous.
template <typename T>
struct Ax2Args {
    Dims d;
    Twiddles<T> tw;
    cplx<T>* W;
    const CgState* cg;  // may be null: right-hand sides with done set are skipped
    const cplx<T>* tab; // twiddle table of this axis (length N)
    long long inner;    // stride of the transformed axis (in entries)
    long long ncols;    // columns in total
    long long cols_per_b;
    FastDiv div_inner, div_cpb;  // by inner and cols_per_b (set with them; ncols < 2^32)
    int tw_ax1, tw_ax2; // columns per CTA along axis 1 / axis 2 (0: default)
};

template <typename T, int N, int DIR>
__global__ void __launch_bounds__(512) k_fft_strided(Ax2Args<T> a) {
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    constexpr int R = RadixFor<T, N>::value;
    constexpr int P = N / R;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smraw);
    const int TW = blockDim.x;
    const int w = threadIdx.x, p = threadIdx.y;
    const unsigned c0 = blockIdx.x * (unsigned)TW;  // columns < 2^32 (checked by the launcher)
    if (a.cg) {  // skip tiles whose right-hand sides are all finished
        const int bfirst = (int)fastdiv(c0, a.div_cpb);
        const unsigned clast = (unsigned)min((long long)c0 + TW, a.ncols) - 1u;
        const int blast = (int)fastdiv(clast, a.div_cpb);
        bool all_done = true;
        for (int bb = bfirst; bb <= blast; ++bb) all_done &= (a.cg[bb].done != 0);
        if (all_done) return;
    }
    const unsigned col = c0 + w;
    const bool valid = col < a.ncols;
    const unsigned outer = valid ? fastdiv(col, a.div_inner) : 0u;
    const unsigned in = valid ? col - outer * a.div_inner.d : 0u;
    const long long base = (long long)outer * N * a.inner + in;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = valid ? ldc(a.W + base + (long long)(p + r * P) * a.inner) : zero_c<T>();
    ColFFT<T, N, R, DIR>::run(v, sm + w, TW, p, a.tab);
    if (valid) {
#pragma unroll
        for (int r = 0; r < R; ++r) stc(a.W + base + (long long)(p + r * P) * a.inner, v[r]);
    }
}

// ------------------------------------------------------------------ pass 5
enum { AX5_PLAIN = 0, AX5_CG = 1, AX5_RESID = 2 };


template <typename T>
struct Ax1FwdArgs {
    Dims d;
    Freq<T> f;
    Twiddles<T> tw;
    const cplx<T>* W;
    cplx<T>* out;        // PLAIN: K u; RESID: residual r (= -K-part); CG: unused
    cplx<T>* x;          // CG
    cplx<T>* p;          // CG
    cplx<T>* r;          // CG
    double* e_out;       // PLAIN: [B][9] E^T sigma-hat(0) part of K u (may be null)
    double* sig0;        // RESID: [B][9] sigma-hat(0) / N (mean stress), W components
    const double* sig_f; // RESID: [B][9] stress targets on the macro basis
    double* r_e;         // RESID/CG: macro residual [B][9]
    double* x_e;         // CG: [B][9]
    double* p_e;         // CG: [B][9]
    double* macroW;      // CG: [B][9] (output: E p_e for the next pass 3)
    float* macroWf;      // CG: FP32 copy of macroW
    CgState* cg;
    const PrecondData* pre;
    double* partials;    // [B][nblk][2]
    unsigned* counters;  // [B]
};

// Pass 5b, element-wise over frequencies, after the forward transforms:
// q = B^H sigma = -(i/N) xi_j sigma-hat_ij (zero on the null set), then
//  PLAIN: out = q (and E^T sigma-hat(0) into e_out);
//  RESID: out = -q, the mean stress and the macro residual, ||r||^2 partials;
//  CG:    r -= alpha q (the iterate update is deferred to the next pass 1),
//         <r, M r> and ||r||^2; the last block sets beta and the stop flag.
template <typename T, int NC, int MODE>
__global__ void __launch_bounds__(PW_THREADS) k_div(Ax1FwdArgs<T> a) {
    __shared__ double red[32 * 2];
    __shared__ bool is_last;
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    const int b = blockIdx.y;
    const int tid = threadIdx.x;
    const Dims& d = a.d;
    if (MODE == AX5_CG && a.cg[b].done) return;
    const T ms = -(T)d.invN;
    T alpha = T(0), N = T(0);
    const PrecondData* pd = a.pre ? a.pre + b / d.Rm : nullptr;
    if constexpr (MODE == AX5_CG) {
        alpha = (T)a.cg[b].alpha;
        N = (T)(1.0 / d.invN);
    }
    T acc0 = T(0), acc1 = T(0);  // CG: <r, M r>, ||r||^2 ; RESID: ||r_u||^2
    const cplx<T>* Wb = a.W + (long long)b * NC * d.H;
    for (long long i = (long long)blockIdx.x * blockDim.x + tid; i < d.H; i += (long long)gridDim.x * blockDim.x) {
        const FreqIdx fi = freq_idx(d, i);
        const T x1 = a.f.xi1[fi.k1], x2 = a.f.xi2[fi.k2], x3 = a.f.xi3[fi.k3];
        cplx<T> q[3] = {zero_c<T>(), zero_c<T>(), zero_c<T>()};
        div_acc<T, NC, 0>(q, ldc(Wb + 0 * d.H + i), x1, x2, x3);
        div_acc<T, NC, 1>(q, ldc(Wb + 1 * d.H + i), x1, x2, x3);
        div_acc<T, NC, 2>(q, ldc(Wb + 2 * d.H + i), x1, x2, x3);
        div_acc<T, NC, 3>(q, ldc(Wb + 3 * d.H + i), x1, x2, x3);
        div_acc<T, NC, 4>(q, ldc(Wb + 4 * d.H + i), x1, x2, x3);
        div_acc<T, NC, 5>(q, ldc(Wb + 5 * d.H + i), x1, x2, x3);
        if constexpr (NC == 9) {
            div_acc<T, NC, 6>(q, ldc(Wb + 6 * d.H + i), x1, x2, x3);
            div_acc<T, NC, 7>(q, ldc(Wb + 7 * d.H + i), x1, x2, x3);
            div_acc<T, NC, 8>(q, ldc(Wb + 8 * d.H + i), x1, x2, x3);
        }
        const bool zmode = (x1 == T(0)) && (x2 == T(0)) && (x3 == T(0));
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c] = zmode ? zero_c<T>() : mul_i(ms, q[c]);
        const T wgt = (T)hweight(fi.k3, d.m);
        if constexpr (MODE == AX5_PLAIN) {
#pragma unroll
            for (int c = 0; c < 3; ++c) stc(a.out + (long long)(b * 3 + c) * d.H + i, q[c]);
        } else if constexpr (MODE == AX5_RESID) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const cplx<T> v = mk(-q[c].x, -q[c].y);
                stc(a.out + (long long)(b * 3 + c) * d.H + i, v);
                acc0 += wgt * (v.x * v.x + v.y * v.y);
            }
        } else {
            cplx<T> rv[3], z[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long idx = (long long)(b * 3 + c) * d.H + i;
                rv[c] = ldc(a.r + idx) - q[c] * alpha;
                stc(a.r + idx, rv[c]);
            }
            precond_pd<T>(*pd, x1, x2, x3, N, rv, z);
            T lrz = T(0), lrr = T(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lrz += rv[c].x * z[c].x + rv[c].y * z[c].y;
                lrr += rv[c].x * rv[c].x + rv[c].y * rv[c].y;
            }
            acc0 += wgt * lrz;
            acc1 += wgt * lrr;
        }
    }
    const bool has0 = blockIdx.x == 0 && tid == 0;  // k = (0,0,0) is entry 0
    // sigma-hat(0) of the nc components, W components (mean stress = this / N)
    auto s0 = [&](int m) { return (double)ldc(Wb + (long long)m * d.H).x; };

    if constexpr (MODE == AX5_PLAIN) {
        if (has0 && a.e_out) {
            for (int q = 0; q < 9; ++q) a.e_out[b * 9 + q] = 0.0;
            for (int k = 0; k < d.ne; ++k) {
                const int m = d.active[k];
                a.e_out[b * 9 + m] = w_to_macro<NC>(m) * s0(m);
            }
        }
        return;
    }
    if constexpr (MODE == AX5_RESID) {
        double v2[2];  // ||r_u||^2 and ||r_e||^2
        {
            const T in2[2] = {acc0, T(0)};
            block_sum_t<T, 2>(in2, v2, red);
        }
        if (has0) {
            const double Nd = 1.0 / d.invN;
            for (int q = 0; q < 9; ++q) a.sig0[b * 9 + q] = q < NC ? s0(q) * d.invN : 0.0;
            for (int q = 0; q < 9; ++q) a.r_e[b * 9 + q] = 0.0;
            for (int k = 0; k < d.ne; ++k) {
                const int m = d.active[k];
                const double re = Nd * a.sig_f[b * 9 + m] - w_to_macro<NC>(m) * s0(m);
                a.r_e[b * 9 + m] = re;
                v2[1] += re * re;
            }
        }
        if (tid == 0) {
            a.partials[((long long)b * gridDim.x + blockIdx.x) * 2 + 0] = v2[0];
            a.partials[((long long)b * gridDim.x + blockIdx.x) * 2 + 1] = v2[1];
        }
        return;
    }
    if constexpr (MODE == AX5_CG) {
        double v2[2];
        {
            const T in2[2] = {acc0, acc1};
            block_sum_t<T, 2>(in2, v2, red);
        }
        if (has0) {  // macro part: q_e = E^T sigma-hat(0); x_e += alpha p_e; r_e -= alpha q_e
            const double al = a.cg[b].alpha;
            double re[9];
            for (int k = 0; k < d.ne; ++k) {
                const int m = d.active[k];
                const double qe = w_to_macro<NC>(m) * s0(m);
                a.x_e[b * 9 + m] += al * a.p_e[b * 9 + m];
                re[k] = a.r_e[b * 9 + m] - al * qe;
                a.r_e[b * 9 + m] = re[k];
            }
            const double(*Me)[9] = pd->Me;
            for (int k = 0; k < d.ne; ++k) {
                double ze = 0.0;
                for (int l = 0; l < d.ne; ++l) ze += Me[k][l] * re[l];
                v2[0] += re[k] * ze;
                v2[1] += re[k] * re[k];
            }
        }
        const int nblk = gridDim.x;
        if (tid == 0) {
            a.partials[((long long)b * nblk + blockIdx.x) * 2 + 0] = v2[0];
            a.partials[((long long)b * nblk + blockIdx.x) * 2 + 1] = v2[1];
            __threadfence();
            const unsigned prev = atomicAdd(a.counters + b, 1u);
            is_last = (prev == (unsigned)nblk - 1);
        }
        __syncthreads();
        if (is_last) {
            __threadfence();
            // the whole last block reduces the partials (fixed order: deterministic)
            double t2[2] = {0.0, 0.0};
            for (int k = tid; k < nblk; k += blockDim.x) {
                t2[0] += __ldcg(a.partials + ((long long)b * nblk + k) * 2 + 0);
                t2[1] += __ldcg(a.partials + ((long long)b * nblk + k) * 2 + 1);
            }
            block_sum<2>(t2, red);
            if (tid == 0) {
                const double srz = t2[0], srr = t2[1];
                CgState& cs = a.cg[b];
                cs.iter += 1;
                cs.rnorm2 = srr;
                const double beta = srz / cs.rho;
                cs.rho = srz;
                cs.beta = beta;
                if (!(srr == srr) || !(srz == srz)) { cs.flags |= 2; cs.done = 1; }
                if (srr <= cs.tol2 * cs.bnorm2 || cs.iter >= cs.max_iter) cs.done = 1;
                if (!cs.done) {  // p_e = z_e + beta p_e, and E p_e for the next pass 3
                    const double(*Me)[9] = pd->Me;
                    double pe[9];
                    for (int k = 0; k < d.ne; ++k) {
                        double ze = 0.0;
                        for (int l = 0; l < d.ne; ++l) ze += Me[k][l] * a.r_e[b * 9 + d.active[l]];
                        pe[k] = ze + beta * a.p_e[b * 9 + d.active[k]];
                    }
                    for (int q = 0; q < 9; ++q) { a.macroW[b * 9 + q] = 0.0; a.macroWf[b * 9 + q] = 0.f; }
                    for (int k = 0; k < d.ne; ++k) {
                        const int m = d.active[k];
                        a.p_e[b * 9 + m] = pe[k];
                        a.macroW[b * 9 + m] = macro_to_w<NC>(m) * pe[k];
                        a.macroWf[b * 9 + m] = (float)a.macroW[b * 9 + m];
                    }
                }
                a.counters[b] = 0u;
            }
        }
    }
}

// ------------------------------------------------------------------ CG start
// rho = <r, M r>, bnorm2 = ||r||^2 (x = 0, p = 0 preset); macro: p_e = 0.
template <typename T>
struct CgInitArgs {
    Dims d;
    Freq<T> f;
    const cplx<T>* r;
    const double* r_e;
    double* p_e;
    double* macroW;
    float* macroWf;
    CgState* cg;
    const PrecondData* pre;
    double* partials;
    unsigned* counters;
    double tol;
    int max_iter;
};

template <typename T>
__global__ void __launch_bounds__(PW_THREADS) k_cg_init(CgInitArgs<T> a) {
    __shared__ double red[32 * 2];
    __shared__ bool is_last;
    const Dims& d = a.d;
    const int b = blockIdx.y;
    const int tid = threadIdx.x;
    const PrecondData& pd = a.pre[b / d.Rm];
    const T N = (T)(1.0 / d.invN);
    T lrz = T(0), lrr = T(0);
    for (long long i = (long long)blockIdx.x * blockDim.x + tid; i < d.H; i += (long long)gridDim.x * blockDim.x) {
        const FreqIdx fi = freq_idx(d, i);
        cplx<T> rv[3], z[3];
        for (int c = 0; c < 3; ++c) rv[c] = ldc(a.r + (long long)(b * 3 + c) * d.H + i);
        precond_pd<T>(pd, a.f.xi1[fi.k1], a.f.xi2[fi.k2], a.f.xi3[fi.k3], N, rv, z);
        const T wgt = (T)hweight(fi.k3, d.m);
        for (int c = 0; c < 3; ++c) {
            lrz += wgt * (rv[c].x * z[c].x + rv[c].y * z[c].y);
            lrr += wgt * (rv[c].x * rv[c].x + rv[c].y * rv[c].y);
        }
    }
    double v2[2] = {(double)lrz, (double)lrr};
    if (blockIdx.x == 0 && tid == 0) {
        for (int k = 0; k < d.ne; ++k) {
            double ze = 0.0;
            for (int l = 0; l < d.ne; ++l) ze += pd.Me[k][l] * a.r_e[b * 9 + d.active[l]];
            const double re = a.r_e[b * 9 + d.active[k]];
            v2[0] += re * ze;
            v2[1] += re * re;
        }
    }
    block_sum<2>(v2, red);
    const int nblk = gridDim.x;
    if (tid == 0) {
        a.partials[((long long)b * nblk + blockIdx.x) * 2 + 0] = v2[0];
        a.partials[((long long)b * nblk + blockIdx.x) * 2 + 1] = v2[1];
        __threadfence();
        const unsigned prev = atomicAdd(a.counters + b, 1u);
        is_last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double t2[2] = {0.0, 0.0};
    for (int k = tid; k < nblk; k += blockDim.x) {
        t2[0] += __ldcg(a.partials + ((long long)b * nblk + k) * 2 + 0);
        t2[1] += __ldcg(a.partials + ((long long)b * nblk + k) * 2 + 1);
    }
    block_sum<2>(t2, red);
    if (tid == 0) {
        const double srz = t2[0], srr = t2[1];
        CgState& cs = a.cg[b];
        cs.rho = srz;
        cs.bnorm2 = srr;
        cs.rnorm2 = srr;
        cs.beta = 0.0;
        cs.alpha = 0.0;
        cs.iter = 0;
        cs.flags = 0;
        cs.tol2 = a.tol * a.tol;
        cs.max_iter = a.max_iter;
        cs.done = (srr == 0.0) ? 1 : 0;
        if (!(srr == srr)) { cs.done = 1; cs.flags |= 2; }
        // first direction's macro part: p_e = z_e (beta = 0)
        for (int q = 0; q < 9; ++q) { a.p_e[b * 9 + q] = 0.0; a.macroW[b * 9 + q] = 0.0; a.macroWf[b * 9 + q] = 0.f; }
        for (int k = 0; k < d.ne; ++k) {
            double ze = 0.0;
            for (int l = 0; l < d.ne; ++l) ze += pd.Me[k][l] * a.r_e[b * 9 + d.active[l]];
            const int m = d.active[k];
            a.p_e[b * 9 + m] = ze;
            a.macroW[b * 9 + m] = (d.nc == 6 && m >= 3 ? 0.70710678118654752440084436210485 : 1.0) * ze;
            a.macroWf[b * 9 + m] = (float)a.macroW[b * 9 + m];
        }
        a.counters[b] = 0u;
    }
}

}  // namespace dbfft
