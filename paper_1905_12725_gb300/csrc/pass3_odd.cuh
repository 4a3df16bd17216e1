// pass3_odd.cuh -- the transforms of odd grid lengths (Sec. 2.1 uses odd
// grids, whose frequency set has no Nyquist index).
//
//  * k_fft_odd: C2C along axis 1 or 2 (the strided passes) for an odd length,
//    mixed-radix (3, 5, 7) Stockham in shared memory.
//  * k_axis3_odd: pass 3 for an odd n3 and linear isotropic phases. An odd
//    real line has no half-length packing, so two real components share one
//    complex transform of length n3: Z[k] = Xa[k] + i Xb[k] over the whole
//    spectrum (X[n3-k] = conj X[k]) gives z = xa + i xb; after the per-voxel
//    stress, Z = DFT(z) and Xa[k] = (Z[k] + conj Z[-k]) / 2,
//    Xb[k] = (Z[k] - conj Z[-k]) / (2 i). The six strain components make
//    three such pairs per grid line and right-hand side.
#pragma once
#include "fft_odd.cuh"
#include "pass3.cuh"

namespace dbfft {

constexpr int kOddThreads = 256;  // threads per CTA of both kernels
constexpr int kOddG = 8;          // threads per transformed line in k_axis3_odd

template <typename T, int N, int DIR>
__global__ void __launch_bounds__(kOddThreads) k_fft_odd(Ax2Args<T> a) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smraw[];
    const int TW = blockDim.x, G = blockDim.y;
    const int w = threadIdx.x, p = threadIdx.y;
    cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smraw);
    cplx<T>* b1 = b0 + (long long)N * TW;
    const long long c0 = (long long)blockIdx.x * TW;
    if (a.cg) {  // skip tiles whose right-hand sides are all finished
        const int bfirst = (int)(c0 / a.cols_per_b);
        const long long clast = min(c0 + TW, a.ncols) - 1;
        const int blast = (int)(clast / a.cols_per_b);
        bool all_done = true;
        for (int bb = bfirst; bb <= blast; ++bb) all_done &= (a.cg[bb].done != 0);
        if (all_done) return;
    }
    const long long col = c0 + w;
    const bool valid = col < a.ncols;
    const long long outer = valid ? col / a.inner : 0;
    const long long in = valid ? col - outer * a.inner : 0;
    const long long base = outer * (long long)N * a.inner + in;
    for (int i = p; i < N; i += G) b0[i * TW + w] = valid ? ldc(a.W + base + (long long)i * a.inner) : zero_c<T>();
    __syncthreads();
    const cplx<T>* res = OddFFT<T, N, DIR>::run(b0 + w, b1 + w, TW, p, G, a.tab);
    if (valid)
        for (int i = p; i < N; i += G) stc(a.W + base + (long long)i * a.inner, res[i * TW]);
}

// Pass 3 for odd n3, OP_ISO (6 components): CTA = L grid lines of one
// right-hand side (a.RB = 1), 3 L component pairs, kOddG threads per pair;
// two buffers of n3 complex values per pair.
template <typename T, int N3>
__global__ void __launch_bounds__(kOddThreads) k_axis3_odd(Ax3Args<T> a) {
    pdl_wait();
    pdl_trigger();
    constexpr int H = (N3 + 1) / 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* sbuf = reinterpret_cast<cplx<T>*>(smraw);
    __shared__ double red[32 * 8];
    __shared__ bool is_last;
    __shared__ T s_macro[9];
    const Dims& d = a.d;
    const int L = a.L;
    const int t = threadIdx.x;
    const int b = blockIdx.y;  // right-hand side
    const long long nlines = (long long)d.n1 * d.n2;
    const long long line0 = (long long)blockIdx.x * L;
    const int lines_here = (int)min((long long)L, nlines - line0);
    const bool done = a.cg != nullptr && a.cg[b].done != 0;
    if (done) return;  // uniform over the CTA
    if (t < 9) s_macro[t] = a.macroW[b * 9 + t];
    const int NP = 3 * L;           // component pairs of this CTA
    const int pr = t / kOddG, p = t % kOddG;
    const bool own = pr < NP;       // this thread works on pair pr
    const int ll = pr / 3, q = pr - (pr / 3) * 3;
    const bool live = own && ll < lines_here;
    cplx<T>* b0 = sbuf + (long long)(own ? pr : 0) * 2 * N3;
    cplx<T>* b1 = b0 + N3;
    const int pf = own ? p : N3;  // threads without a pair take part in the barriers only

    // ---- whole spectra of the pairs: Z[k] = Xa[k] + i Xb[k], Z[n3-k] = conj Xa[k] + i conj Xb[k]
    cplx<T>* res;
    if (a.zero_in) {
        if (own)
            for (int k = p; k < N3; k += kOddG) b0[k] = zero_c<T>();
        __syncthreads();
        res = b0;
    } else {
        if (live) {
            const cplx<T>* xa = a.W + ((long long)(b * 6 + 2 * q) * nlines + line0 + ll) * H;
            const cplx<T>* xb = a.W + ((long long)(b * 6 + 2 * q + 1) * nlines + line0 + ll) * H;
            for (int k = p; k < H; k += kOddG) {
                const cplx<T> A = ldc(xa + k), Bv = ldc(xb + k);
                b0[k] = mk(A.x - Bv.y, A.y + Bv.x);
                if (k > 0) b0[N3 - k] = mk(A.x + Bv.y, Bv.x - A.y);
            }
        } else if (own) {
            for (int k = p; k < N3; k += kOddG) b0[k] = zero_c<T>();
        }
        __syncthreads();
        res = OddFFT<T, N3, +1>::run(b0, b1, 1, pf, kOddG, a.tw.t3);
    }
    const long long roff = res - b0;  // 0 or N3, the same for every pair

    // ---- per-voxel stress sigma = C (eps + macro) and the CG curvature
    T eacc = T(0);
    for (int idx = t; idx < lines_here * N3; idx += kOddThreads) {
        const int lv = idx / N3, x3 = idx - lv * N3;
        const long long vox = (line0 + lv) * N3 + x3;
        const long long mv = (long long)(b / d.Rm) * d.V + vox;
        const int ph = a.phase[mv];
        const T sc = a.scale ? a.scale[mv] : T(1);
        const T lam = a.lam[ph] * sc, mu = a.mu[ph] * sc;
        cplx<T>* z[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) z[c] = sbuf + (long long)(lv * 3 + c) * 2 * N3 + roff + x3;
        T e[6], sg[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cplx<T> v = *z[c];
            e[2 * c] = v.x + s_macro[2 * c];
            e[2 * c + 1] = v.y + s_macro[2 * c + 1];
        }
        iso_stress<T, 6>(e, lam, mu, sg);
        if (a.cg) {
#pragma unroll
            for (int c = 0; c < 6; ++c) eacc += (c >= 3 ? T(2) : T(1)) * e[c] * sg[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) *z[c] = mk(sg[2 * c], sg[2 * c + 1]);
    }

    // ---- CG curvature <p, K p>; the last CTA of this right-hand side sets alpha
    if (a.cg) {
        double v1[1];
        const T in1[1] = {eacc};
        block_sum_t<T, 1>(in1, v1, red);
        const int nblk = gridDim.x;
        if (t == 0) {
            a.partials[(long long)b * nblk + blockIdx.x] = v1[0];
            __threadfence();
            const unsigned prev = atomicAdd(a.counters + b, 1u);
            is_last = (prev == (unsigned)nblk - 1);
        }
        __syncthreads();
        if (is_last) {
            __threadfence();
            double s1[1] = {0.0};
            for (int k = t; k < nblk; k += kOddThreads) s1[0] += __ldcg(a.partials + (long long)b * nblk + k);
            block_sum<1>(s1, red);
            if (t == 0) {
                const double sum = s1[0];
                CgState& cs = a.cg[b];
                if (!cs.done) {
                    cs.pq = sum;
                    if (sum > 0.0 && sum == sum) {
                        cs.alpha = cs.rho / sum;
                    } else {
                        cs.alpha = 0.0;
                        cs.flags |= (sum == sum) ? 1 : 2;
                        cs.done = 1;
                    }
                }
                a.counters[b] = 0u;
            }
        }
    }
    __syncthreads();

    // ---- forward transform and unpacking of the two half spectra of each pair
    cplx<T>* rb = sbuf + (long long)(own ? pr : 0) * 2 * N3 + roff;
    cplx<T>* ob = sbuf + (long long)(own ? pr : 0) * 2 * N3 + (N3 - roff);
    const cplx<T>* f = OddFFT<T, N3, -1>::run(rb, ob, 1, pf, kOddG, a.tw.t3);
    if (live) {
        cplx<T>* xa = a.W + ((long long)(b * 6 + 2 * q) * nlines + line0 + ll) * H;
        cplx<T>* xb = a.W + ((long long)(b * 6 + 2 * q + 1) * nlines + line0 + ll) * H;
        const T half = T(0.5);
        for (int k = p; k < H; k += kOddG) {
            const cplx<T> Zk = f[k], Zm = f[k == 0 ? 0 : N3 - k];
            // Xa = (Zk + conj Zm) / 2, Xb = (Zk - conj Zm) / (2 i)
            stc(xa + k, mk(half * (Zk.x + Zm.x), half * (Zk.y - Zm.y)));
            stc(xb + k, mk(half * (Zk.y + Zm.y), -half * (Zk.x - Zm.x)));
        }
    }
}

}  // namespace dbfft
