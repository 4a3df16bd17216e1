// pass3_odd.cuh -- the transforms of odd grid lengths (Sec. 2.1 uses odd
// grids, whose frequency set has no Nyquist index).
//
//  * k_fft_odd: C2C along axis 1 or 2 (the strided passes) for an odd length,
//    mixed-radix (3, 5, 7) Stockham in shared memory.
//  * k_axis3_odd: pass 3 for an odd n3 (every model). An odd
//    real line has no half-length packing, so two real components share one
//    complex transform of length n3: Z[k] = Xa[k] + i Xb[k] over the whole
//    spectrum (X[n3-k] = conj X[k]) gives z = xa + i xb; after the per-voxel
//    stress, Z = DFT(z) and Xa[k] = (Z[k] + conj Z[-k]) / 2,
//    Xb[k] = (Z[k] - conj Z[-k]) / (2 i). The six strain components make
//    three such pairs per grid line and right-hand side, the nine gradient
//    components five (the last with a zero partner).
#pragma once
#include "fft_odd.cuh"
#include "pass3_pipe.cuh"

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

// Constitutive update of one voxel in the odd pass 3 (the update ops of
// k_axis3, on a voxel's components gathered in e[NC]): the stress replaces e,
// tangent and state go to their arrays.
template <typename T, int NC, int OPK>
__device__ __forceinline__ void update_voxel(const Ax3Args<T>& a, int bb, long long vox, long long mv, T* e) {
    if constexpr (OPK == OP_NH_UPDATE || OPK == OP_SVK_UPDATE) {
        constexpr int NT = OPK == OP_SVK_UPDATE ? 15 : 10;
        const int ph = a.phase[mv];
        double F[9], Pk[9], tn[NT];
#pragma unroll
        for (int q = 0; q < 9; ++q) F[q] = (double)e[q] + a.macroW[bb * 9 + q];
        bool ok;
        if constexpr (OPK == OP_SVK_UPDATE)
            ok = svk_stress(F, a.mu[ph], a.lam[ph], Pk, tn);
        else
            ok = nh_stress(F, a.mu[ph], a.lam[ph], Pk, tn);
        if (!ok) atomicOr(a.err, 1u);
        const long long to = ((long long)bb * a.d.V + vox) * NT;
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            if (a.tan_out_f) a.tan_out_f[to + q] = (float)tn[q];
            if (a.tan_out_d) a.tan_out_d[to + q] = tn[q];
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) e[q] = (T)Pk[q];
    } else if constexpr (OPK == OP_CP_UPDATE || OPK == OP_CP_UPDATE32) {
        const int gr = a.phase[mv];
        double ev[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) ev[q] = (double)e[q] + a.macroW[bb * 9 + q];
        const long long so = ((long long)bb * a.d.V + vox) * 6;
        double sg[6], ep[6], guess[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) guess[q] = (a.guess_trial ? a.sig_t : a.sig_prev)[so + q];
        const long long to = ((long long)bb * a.d.V + vox) * 21;
        bool ok;
        if constexpr (OPK == OP_CP_UPDATE32) {
            float tn[21];
            ok = cp_update<float>(a.grains[gr], a.grains_f[gr], a.cp, ev, a.eps_p + so, guess, sg, tn, ep);
#pragma unroll
            for (int q = 0; q < 21; ++q) a.tan_out_f[to + q] = tn[q];
        } else {
            double tn[21];
            ok = cp_update<double>(a.grains[gr], a.grains_f[gr], a.cp, ev, a.eps_p + so, guess, sg, tn, ep);
#pragma unroll
            for (int q = 0; q < 21; ++q) a.tan_out_d[to + q] = tn[q];
        }
        if (!ok) atomicOr(a.err, 1u);
#pragma unroll
        for (int q = 0; q < 6; ++q) { a.eps_p_t[so + q] = ep[q]; a.sig_t[so + q] = sg[q]; }
        const double ir2 = 0.70710678118654752440084436210485;
#pragma unroll
        for (int q = 0; q < 6; ++q) e[q] = (T)(q < 3 ? sg[q] : ir2 * sg[q]);
    } else if constexpr (OPK == OP_FCP_UPDATE || OPK == OP_FCP_UPDATE32) {
        const int gr = a.phase[mv];
        const long long vo = (long long)bb * a.d.V + vox;
        double F[9], Pk[9], Fpn[9], Fpo[9], Tn[6], guess[6], tn[45];
#pragma unroll
        for (int q = 0; q < 9; ++q) F[q] = (double)e[q] + a.macroW[bb * 9 + q];
#pragma unroll
        for (int q = 0; q < 9; ++q) Fpo[q] = a.fp_old[vo * 9 + q];
#pragma unroll
        for (int q = 0; q < 6; ++q) guess[q] = (a.guess_trial ? a.sig_t : a.sig_prev)[vo * 6 + q];
                const bool ok = fcp_update<OPK == OP_FCP_UPDATE32>(a.grains[gr], a.grains_f[gr], a.cp, F, Fpo, guess, Pk, Fpn, Tn, tn);
        if (!ok) atomicOr(a.err, 1u);
#pragma unroll
        for (int q = 0; q < 9; ++q) a.fp_new[vo * 9 + q] = Fpn[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) a.sig_t[vo * 6 + q] = Tn[q];
#pragma unroll
        for (int q = 0; q < 45; ++q) {
            if (a.tan_out_f) a.tan_out_f[vo * 45 + q] = (float)tn[q];
            if (a.tan_out_d) a.tan_out_d[vo * 45 + q] = tn[q];
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) e[q] = (T)Pk[q];
    }
}

// Pass 3 for odd n3: CTA = L grid lines of one right-hand side (a.RB = 1),
// NP = ceil(NC/2) component pairs per line (the last of nine components rides
// with a zero), kOddG threads per pair, two buffers of n3 complex values per
// pair. Every operation of k_axis3 but the adjoint assembly and the
// displacement output.
template <typename T, int N3, int NC, int OPK>
__global__ void __launch_bounds__(kOddThreads) k_axis3_odd(Ax3Args<T> a) {
    pdl_wait();
    pdl_trigger();
    constexpr int H = (N3 + 1) / 2;
    constexpr int NPL = (NC + 1) / 2;  // pairs per line
    extern __shared__ __align__(16) unsigned char smraw[];
    cplx<T>* sbuf = reinterpret_cast<cplx<T>*>(smraw);
    __shared__ double red[32 * 8];
    __shared__ bool is_last;
    const Dims& d = a.d;
    const int L = a.L;
    const int t = threadIdx.x;
    const int b = blockIdx.y;  // right-hand side
    const long long nlines = (long long)d.n1 * d.n2;
    const long long line0 = (long long)blockIdx.x * L;
    const int lines_here = (int)min((long long)L, nlines - line0);
    const bool done = a.cg != nullptr && a.cg[b].done != 0;
    if (done) return;  // uniform over the CTA
    const int NP = NPL * L;         // component pairs of this CTA
    const int pr = t / kOddG, p = t % kOddG;
    const bool own = pr < NP;       // this thread works on pair pr
    const int ll = pr / NPL, q = pr - (pr / NPL) * NPL;
    const bool live = own && ll < lines_here;
    const bool has_b = 2 * q + 1 < NC;  // the pair's second component exists
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
            const cplx<T>* xa = a.W + ((long long)(b * NC + 2 * q) * nlines + line0 + ll) * H;
            const cplx<T>* xb = a.W + ((long long)(b * NC + 2 * q + 1) * nlines + line0 + ll) * H;
            for (int k = p; k < H; k += kOddG) {
                const cplx<T> A = ldc(xa + k), Bv = has_b ? ldc(xb + k) : zero_c<T>();
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

    // ---- per-voxel operation (and the CG curvature for the applications)
    T eacc = T(0);
    for (int idx = t; idx < lines_here * N3; idx += kOddThreads) {
        const int lv = idx / N3, x3 = idx - lv * N3;
        const long long vox = (line0 + lv) * N3 + x3;
        const long long mv = (long long)(b / d.Rm) * d.V + vox;
        cplx<T>* z[NPL];
#pragma unroll
        for (int c = 0; c < NPL; ++c) z[c] = sbuf + (long long)(lv * NPL + c) * 2 * N3 + roff + x3;
        T e[2 * NPL];
#pragma unroll
        for (int c = 0; c < NPL; ++c) {
            const cplx<T> v = *z[c];
            e[2 * c] = v.x;
            e[2 * c + 1] = v.y;
        }
        if constexpr (OpInfo<OPK>::apply) {
            const int ph = a.phase[mv];
            const T sc = (OPK == OP_ISO && a.scale) ? a.scale[mv] : T(1);
            const T en = apply_voxel<T, NC, OPK>(a, b, vox, ph, sc, e, 1);
            if (a.cg) eacc += en;
        } else {
            update_voxel<T, NC, OPK>(a, b, vox, mv, e);
        }
        if constexpr (NC % 2 == 1) e[NC] = T(0);  // the zero partner of the last component
#pragma unroll
        for (int c = 0; c < NPL; ++c) *z[c] = mk(e[2 * c], e[2 * c + 1]);
    }

    // ---- CG curvature <p, K p>; the last CTA of this right-hand side sets alpha
    if constexpr (OpInfo<OPK>::apply) {
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
    }
    __syncthreads();

    // ---- forward transform and unpacking of the two half spectra of each pair
    cplx<T>* rb = sbuf + (long long)(own ? pr : 0) * 2 * N3 + roff;
    cplx<T>* ob = sbuf + (long long)(own ? pr : 0) * 2 * N3 + (N3 - roff);
    const cplx<T>* f = OddFFT<T, N3, -1>::run(rb, ob, 1, pf, kOddG, a.tw.t3);
    if (live) {
        cplx<T>* xa = a.W + ((long long)(b * NC + 2 * q) * nlines + line0 + ll) * H;
        cplx<T>* xb = a.W + ((long long)(b * NC + 2 * q + 1) * nlines + line0 + ll) * H;
        const T half = T(0.5);
        for (int k = p; k < H; k += kOddG) {
            const cplx<T> Zk = f[k], Zm = f[k == 0 ? 0 : N3 - k];
            // Xa = (Zk + conj Zm) / 2, Xb = (Zk - conj Zm) / (2 i)
            stc(xa + k, mk(half * (Zk.x + Zm.x), half * (Zk.y - Zm.y)));
            if (has_b) stc(xb + k, mk(half * (Zk.y + Zm.y), -half * (Zk.x - Zm.x)));
        }
    }
}

}  // namespace dbfft
