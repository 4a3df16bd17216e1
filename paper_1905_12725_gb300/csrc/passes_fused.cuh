// passes_fused.cuh -- the first and the last pass of a CG iteration with the
// element-wise work fused into the axis-2 transform (Sec. 2.2, Eqs. s-hat and
// d-hat; Sec. 2.5, the preconditioner).
//
//   k_grad_ax2: p = M r + beta p, x += alpha p_old, eps-hat = s-hat . p / N
//               (or g-hat . p at finite strain), then the inverse C2C of each
//               strain component along axis 2;
//   k_ax2_div:  the forward C2C of each stress component along axis 2, the
//               divergence -d-hat : sigma-hat / N on the fly, the null mask,
//               r -= alpha q, <r, M r>, ||r||^2; the last block sets beta and
//               the stop flag (and the macro rows from sigma-hat(0)).
//
// A CTA owns TW columns (k1, k3) of one right-hand side and all n2 rows of
// them: a warp covers TW consecutive k3 (rows of TW complex values, 128 bytes
// in FP32 for TW = 16) and P = n2 / 8 threads share each column's transform,
// eight values per thread in registers, exchanging through shared memory.
// Both kernels touch each vector once: k_grad_ax2 reads r, p, x and writes
// p, x and the nc strain components (the 15 + nc component passes of the
// element-wise pass 1 alone), k_ax2_div reads the nc stress components and r
// and writes r (6 + nc): the separate axis-2 passes (2 nc each) disappear.
#pragma once
#include "passes.cuh"

namespace dbfft {

constexpr int FUSED_R = 8;   // values per thread of the axis-2 transform
constexpr int FUSED_TW = 16; // columns per CTA (one 128-byte row segment in FP32)

template <typename T, int NC, int N, int TWC>
__global__ void __launch_bounds__(TWC * N / FUSED_R, TWC * N / FUSED_R >= 512 ? 1 : 2) k_grad_ax2(Ax1InvArgs<T> a) {
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    constexpr int R = FUSED_R;
    constexpr int P = N / R;
    extern __shared__ __align__(16) unsigned char smfz[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smfz);
    constexpr int TW = TWC;
    const int w = threadIdx.x, p = threadIdx.y;
    const int b = blockIdx.y;
    if (a.cg[b].done) return;
    const Dims& d = a.d;
    const long long col = (long long)blockIdx.x * TW + w;  // (k1, k3) of this thread's column
    const bool valid = col < (long long)d.n1 * d.h;
    const unsigned k1 = valid ? fastdiv((unsigned)col, d.div_h) : 0u;
    const unsigned k3 = valid ? (unsigned)col - k1 * d.div_h.d : 0u;
    const T s = (T)d.invN;
    const T beta = (T)a.cg[b].beta, alpha = (T)a.cg[b].alpha, Nn = (T)(1.0 / d.invN);
    const PrecondData* pd = a.pre + b / d.Rm;
    const T x1 = a.f.xi1[k1], x3 = a.f.xi3[k3];
    const long long base = ((long long)(b * 3) * d.n1 + k1) * d.plane + k3;  // component c: + c H
    cplx<T> u[3][R];
    T x2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k2 = p + P * r;
        x2[r] = a.f.xi2[k2];
        if (valid) {
            const long long o = base + (long long)k2 * d.h;
            cplx<T> rv[3], po[3], xo[3], z[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rv[c] = ldc(a.in + o + c * d.H);
                po[c] = ldc(a.p + o + c * d.H);
                xo[c] = ldc(a.x + o + c * d.H);
            }
            precond_pd<T>(*pd, x1, x2[r], x3, Nn, rv, z);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                u[c][r] = z[c] + po[c] * beta;
                stc(a.p + o + c * d.H, u[c][r]);
                stc(a.x + o + c * d.H, xo[c] + po[c] * alpha);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c][r] = zero_c<T>();
        }
    }
    cplx<T>* Wb = a.W + ((long long)(b * NC) * d.n1 + k1) * d.plane + k3;
    sfor<0, NC>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const cplx<T> uu[3] = {u[0][r], u[1][r], u[2][r]};
            v[r] = grad_comp<T, NC, m>(uu, x1, x2[r], x3, s);
        }
        ColFFT<T, N, R, +1>::run(v, sm + w, TW, p, a.tw.t2);
        if (valid) {
#pragma unroll
            for (int r = 0; r < R; ++r) stc(Wb + m * d.H + (long long)(p + P * r) * d.h, v[r]);
        }
    });
}

template <typename T, int NC, int N, int TWC>
__global__ void __launch_bounds__(TWC * N / FUSED_R, TWC * N / FUSED_R >= 512 ? 1 : 2) k_ax2_div(Ax1FwdArgs<T> a) {
    constexpr int R = FUSED_R;
    constexpr int P = N / R;
    extern __shared__ __align__(16) unsigned char smfz[];
    cplx<T>* sm = reinterpret_cast<cplx<T>*>(smfz);
    __shared__ double red[32 * 2];
    __shared__ double s_sig0[9];
    __shared__ bool is_last;
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    constexpr int TW = TWC;
    const int w = threadIdx.x, p = threadIdx.y;
    const int tid = w + TW * p;
    const int b = blockIdx.y;
    if (a.cg[b].done) return;
    const Dims& d = a.d;
    const long long col = (long long)blockIdx.x * TW + w;
    const bool valid = col < (long long)d.n1 * d.h;
    const unsigned k1 = valid ? fastdiv((unsigned)col, d.div_h) : 0u;
    const unsigned k3 = valid ? (unsigned)col - k1 * d.div_h.d : 0u;
    const T ms = -(T)d.invN;
    const T alpha = (T)a.cg[b].alpha, Nn = (T)(1.0 / d.invN);
    const PrecondData* pd = a.pre + b / d.Rm;
    const T x1 = a.f.xi1[k1], x3 = a.f.xi3[k3];
    T x2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x2[r] = a.f.xi2[p + P * r];
    const bool owns0 = valid && col == 0 && p == 0;  // holds frequency (0, 0, 0) after the transform
    cplx<T> q[3][R];
#pragma unroll
    for (int r = 0; r < R; ++r) q[0][r] = q[1][r] = q[2][r] = zero_c<T>();
    const cplx<T>* Wb = a.W + ((long long)(b * NC) * d.n1 + k1) * d.plane + k3;
    sfor<0, NC>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = valid ? ldc(Wb + m * d.H + (long long)(p + P * r) * d.h) : zero_c<T>();
        ColFFT<T, N, R, -1>::run(v, sm + w, TW, p, a.tw.t2);
        if (owns0) s_sig0[m] = (double)v[0].x;  // sigma-hat(0) of component m (k2 = 0 is r = 0 of p = 0)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            cplx<T> qq[3] = {q[0][r], q[1][r], q[2][r]};
            div_acc<T, NC, m>(qq, v[r], x1, x2[r], x3);
            q[0][r] = qq[0];
            q[1][r] = qq[1];
            q[2][r] = qq[2];
        }
    });
    // q = B^H sigma = -(i/N) xi_j sigma-hat_ij (0 on the null set); r -= alpha q; <r, M r>, ||r||^2
    T acc0 = T(0), acc1 = T(0);
    if (valid) {
        const T wgt = (T)hweight((int)k3, d.m);
        const long long base = ((long long)(b * 3) * d.n1 + k1) * d.plane + k3;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k2 = p + P * r;
            const bool zmode = (x1 == T(0)) && (x2[r] == T(0)) && (x3 == T(0));
            const long long o = base + (long long)k2 * d.h;
            cplx<T> rv[3], z[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const cplx<T> qc = zmode ? zero_c<T>() : mul_i(ms, q[c][r]);
                rv[c] = ldc(a.r + o + c * d.H) - qc * alpha;
                stc(a.r + o + c * d.H, rv[c]);
            }
            precond_pd<T>(*pd, x1, x2[r], x3, Nn, rv, z);
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
    double v2[2];
    {
        const T in2[2] = {acc0, acc1};
        block_sum_t<T, 2>(in2, v2, red);  // result in thread 0; its barriers also publish s_sig0
    }
    if (blockIdx.x == 0 && tid == 0) {  // macro part: q_e = E^T sigma-hat(0); x_e += alpha p_e; r_e -= alpha q_e
        const double al = a.cg[b].alpha;
        double re[9];
        for (int k = 0; k < d.ne; ++k) {
            const int m = d.active[k];
            const double qe = w_to_macro<NC>(m) * s_sig0[m];
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
    if (!is_last) return;
    __threadfence();
    // the whole last block reduces the partials (fixed order: deterministic)
    double t2[2] = {0.0, 0.0};
    const int nthr = TW * blockDim.y;
    for (int k = tid; k < nblk; k += nthr) {
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
            for (int qq = 0; qq < 9; ++qq) { a.macroW[b * 9 + qq] = 0.0; a.macroWf[b * 9 + qq] = 0.f; }
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

}  // namespace dbfft
