// pass3.cuh -- axis-3 pass: C2R along the contiguous, halved axis, the
// per-voxel operation in real space, and R2C back. Real-space fields live only
// in shared memory. One CTA carries L grid lines (i1, i2) for the RB
// right-hand sides that share one material map, so the material of a voxel
// is read once for all of them.
//
// Real transform of length n via a complex transform of length m = n/2
// (the standard even/odd packing z[j] = x[2j] + i x[2j+1]):
//   C2R: Z[k] = (X[k] + conj X[m-k]) + i e^{+2 pi i k/n} (X[k] - conj X[m-k]),
//        z = IDFT_m(Z) gives x[2j] = Re z[j], x[2j+1] = Im z[j] (unnormalised);
//   R2C: Z = DFT_m(z), X[k] = (Z[k] + conj Z[m-k]) / 2
//                            - (i/2) e^{-2 pi i k/n} (Z[k] - conj Z[m-k]).
#pragma once
#include "constitutive.cuh"
#include "passes.cuh"

namespace dbfft {

enum {
    OP_ISO = 0,        // sigma = C (eps + macro): linear isotropic phases
    OP_NH_APPLY = 1,   // dP = K(F) : (G + macro) from the stored NH tangent data
    OP_NH_UPDATE = 2,  // P(F), F = macro (incl. I) + G; stores tangent data
    OP_CP_APPLY = 3,   // sigma = C_tan (eps + macro), stored 21-entry Mandel tangent
    OP_CP_UPDATE = 4,  // backward-Euler crystal plasticity at eps = macro + eps~
    OP_ADJ = 5         // dJ/dE(x) = (1/N) eps_adj : C1 : eps_fwd (no forward R2C)
};

template <typename T>
struct Ax3Args {
    Dims d;
    Twiddles<T> tw;
    cplx<T>* W;            // [B][nc][H]
    const cplx<T>* W2;     // OP_ADJ: adjoint strain field in W layout
    int RB;                // right-hand sides per CTA (divides Rm)
    int L;                 // grid lines per CTA
    const double* macroW;  // [B][9] constant field added before the op (W components)
    const double* macroW2; // OP_ADJ: macro part of the adjoint field
    // CG curvature (apply ops only; null outside CG)
    CgState* cg;
    double* partials;      // [B][nblk]
    unsigned* counters;    // [B / RB]
    // materials
    const uint16_t* phase; // [Bm][V]
    const double* scale;   // [Bm][V] or null
    const double* lam;     // per phase
    const double* mu;
    // nonlinear tangent / state
    const T* tan_in;       // apply ops: [B][V][ntan]
    float* tan_out_f;      // update ops: tangent written in FP32 (or null)
    double* tan_out_d;     // update ops: tangent written in FP64 (or null)
    const CpGrain* grains; // CP per-grain data
    CpParams cp;
    const double* eps_p;   // [B][V][6] committed plastic strain
    const double* sig_prev;// [B][V][6] committed stress (Newton start)
    double* eps_p_t;       // trial plastic strain
    double* sig_t;         // trial stress
    unsigned* err;         // error bits (bit 0: local Newton failure)
    double* dJdE;          // OP_ADJ output [B][V]
};

template <int OPK> struct OpInfo {
    static constexpr bool forward = OPK != OP_ADJ;
    static constexpr bool apply = OPK == OP_ISO || OPK == OP_NH_APPLY || OPK == OP_CP_APPLY;
};

template <typename T, int N3, int NC, int OPK>
__global__ void __launch_bounds__(256) k_axis3(Ax3Args<T> a) {
    constexpr int M = N3 / 2;
    constexpr int R = RadixFor<T, M>::value;
    constexpr int P = M / R;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sreal = reinterpret_cast<T*>(smraw);
    __shared__ double red[32 * 8];
    __shared__ double ecc[8];
    __shared__ bool is_last;
    const Dims& d = a.d;
    const int RB = a.RB, L = a.L;
    const int NSLOT = L * RB * NC;
    const int NSLOT_ALLOC = blockDim.x / P;  // padding threads of the last warp get scratch slots
    const int t = threadIdx.x;
    const int p = t % P, slot = t / P;
    const bool slot_ok = slot < NSLOT;
    const int c = slot % NC, rl = (slot / NC) % RB, ll = slot / (NC * RB);
    const int g = blockIdx.y;
    const int b = g * RB + rl;
    const long long nlines = (long long)d.n1 * d.n2;
    const long long line = (long long)blockIdx.x * L + ll;
    const bool act_b = (a.cg == nullptr) || (a.cg[b].done == 0);
    const bool valid = slot_ok && line < nlines && act_b;
    T* my = sreal + (long long)slot * N3;
    cplx<T>* myc = reinterpret_cast<cplx<T>*>(my);
    const long long base = ((long long)(b * NC + c) * nlines + line) * d.h;

    // ---- C2R (and for OP_ADJ the second field in the second half of the slots)
    {
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = p + r * P;
            if (valid) {
                const cplx<T> X = ldc(a.W + base + k);
                const cplx<T> Xc = conjg(ldc(a.W + base + (M - k)));
                const cplx<T> e = conjg(ldg_c(a.tw.t3 + k));  // e^{+2 pi i k / n}
                const cplx<T> dlt = e * (X - Xc);
                v[r] = (X + Xc) + mk(-dlt.y, dlt.x);
            } else {
                v[r] = zero_c<T>();
            }
        }
        ColFFT<T, M, R, +1>::run(v, myc, 1, p, a.tw.tm);
        __syncthreads();
        if (slot_ok) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int jj = p + r * P;
                my[2 * jj] = v[r].x;
                my[2 * jj + 1] = v[r].y;
            }
        }
    }
    T* sreal2 = sreal + (long long)NSLOT_ALLOC * N3;  // OP_ADJ second field
    if constexpr (OPK == OP_ADJ) {
        cplx<T> v[R];
        T* my2 = sreal2 + (long long)slot * N3;
        cplx<T>* myc2 = reinterpret_cast<cplx<T>*>(my2);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = p + r * P;
            if (valid) {
                const cplx<T> X = ldc(a.W2 + base + k);
                const cplx<T> Xc = conjg(ldc(a.W2 + base + (M - k)));
                const cplx<T> e = conjg(ldg_c(a.tw.t3 + k));
                const cplx<T> dlt = e * (X - Xc);
                v[r] = (X + Xc) + mk(-dlt.y, dlt.x);
            } else {
                v[r] = zero_c<T>();
            }
        }
        ColFFT<T, M, R, +1>::run(v, myc2, 1, p, a.tw.tm);
        __syncthreads();
        if (slot_ok) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int jj = p + r * P;
                my2[2 * jj] = v[r].x;
                my2[2 * jj + 1] = v[r].y;
            }
        }
    }
    __syncthreads();

    // ---- per-voxel operation
    double eacc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) eacc[q] = 0.0;
    const int mat = (g * RB) / d.Rm;
    for (int idx = t; idx < L * N3; idx += blockDim.x) {
        const int lv = idx / N3, x3 = idx - lv * N3;
        const long long ln = (long long)blockIdx.x * L + lv;
        if (ln >= nlines) continue;
        const long long vox = ln * N3 + x3;
        if constexpr (OPK == OP_ISO || OPK == OP_ADJ) {
            const long long mv = (long long)mat * d.V + vox;
            const int ph = a.phase[mv];
            double sc = a.scale ? a.scale[mv] : 1.0;
            const T lam = (T)(a.lam[ph] * sc), mu = (T)(a.mu[ph] * sc);
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                if (a.cg && a.cg[bb].done) continue;
                T* f = sreal + (long long)((lv * RB + rr) * NC) * N3 + x3;
                T e[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) e[q] = f[q * N3] + (T)a.macroW[bb * 9 + q];
                if constexpr (OPK == OP_ADJ) {
                    // dJ/dE = (1/N) eps_adj : C1 : eps_fwd, C1 = C / E: for this
                    // op the phase tables hold lam, mu per unit Young's modulus
                    const T* f2 = sreal2 + (long long)((lv * RB + rr) * NC) * N3 + x3;
                    T e2[NC];
#pragma unroll
                    for (int q = 0; q < NC; ++q) e2[q] = f2[q * N3] + (T)a.macroW2[bb * 9 + q];
                    T sg[NC];
                    iso_stress<T, NC>(e, (T)a.lam[ph], (T)a.mu[ph], sg);
                    T acc = T(0);
#pragma unroll
                    for (int q = 0; q < NC; ++q) acc += (q >= 3 && NC == 6 ? T(2) : T(1)) * e2[q] * sg[q];
                    a.dJdE[(long long)bb * d.V + vox] = (double)acc * d.invN;
                } else {
                    T sg[NC];
                    iso_stress<T, NC>(e, lam, mu, sg);
                    if (OpInfo<OPK>::apply && a.cg) {
                        T en = T(0);
#pragma unroll
                        for (int q = 0; q < NC; ++q) en += (q >= 3 && NC == 6 ? T(2) : T(1)) * e[q] * sg[q];
                        eacc[rr] += (double)en;
                    }
#pragma unroll
                    for (int q = 0; q < NC; ++q) f[q * N3] = sg[q];
                }
            }
        } else if constexpr (OPK == OP_NH_APPLY) {
            const long long mv = (long long)mat * d.V + vox;
            const int ph = a.phase[mv];
            const T lam = (T)a.lam[ph], mu = (T)a.mu[ph];
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                if (a.cg && a.cg[bb].done) continue;
                T* f = sreal + (long long)((lv * RB + rr) * NC) * N3 + x3;
                T G[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) G[q] = f[q * N3] + (T)a.macroW[bb * 9 + q];
                const T* tn = a.tan_in + ((long long)bb * d.V + vox) * 10;
                T sg[9];
                nh_apply<T>(tn, mu, lam, G, sg);
                if (a.cg) {
                    T en = T(0);
#pragma unroll
                    for (int q = 0; q < 9; ++q) en += G[q] * sg[q];
                    eacc[rr] += (double)en;
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) f[q * N3] = sg[q];
            }
        } else if constexpr (OPK == OP_NH_UPDATE) {
            const long long mv = (long long)mat * d.V + vox;
            const int ph = a.phase[mv];
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                T* f = sreal + (long long)((lv * RB + rr) * NC) * N3 + x3;
                double F[9], Pk[9], tn[10];
#pragma unroll
                for (int q = 0; q < 9; ++q) F[q] = (double)f[q * N3] + a.macroW[bb * 9 + q];
                const bool ok = nh_stress(F, a.mu[ph], a.lam[ph], Pk, tn);
                if (!ok) atomicOr(a.err, 1u);
                const long long to = ((long long)bb * d.V + vox) * 10;
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    if (a.tan_out_f) a.tan_out_f[to + q] = (float)tn[q];
                    if (a.tan_out_d) a.tan_out_d[to + q] = tn[q];
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) f[q * N3] = (T)Pk[q];
            }
        } else if constexpr (OPK == OP_CP_APPLY) {
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                if (a.cg && a.cg[bb].done) continue;
                T* f = sreal + (long long)((lv * RB + rr) * NC) * N3 + x3;
                T e[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) e[q] = f[q * N3] + (T)a.macroW[bb * 9 + q];
                const T* tn = a.tan_in + ((long long)bb * d.V + vox) * 21;
                T sg[6];
                cp_apply<T>(tn, e, sg);
                if (a.cg) {
                    T en = T(0);
#pragma unroll
                    for (int q = 0; q < 6; ++q) en += (q >= 3 ? T(2) : T(1)) * e[q] * sg[q];
                    eacc[rr] += (double)en;
                }
#pragma unroll
                for (int q = 0; q < 6; ++q) f[q * N3] = sg[q];
            }
        } else if constexpr (OPK == OP_CP_UPDATE) {
            const long long mv = (long long)mat * d.V + vox;
            const int gr = a.phase[mv];
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                T* f = sreal + (long long)((lv * RB + rr) * NC) * N3 + x3;
                double e[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) e[q] = (double)f[q * N3] + a.macroW[bb * 9 + q];
                const long long so = ((long long)bb * d.V + vox) * 6;
                double sg[6], tn[21], ep[6];
                const bool ok = cp_update(a.grains[gr], a.cp, e, a.eps_p + so, a.sig_prev + so, sg, tn, ep);
                if (!ok) atomicOr(a.err, 1u);
#pragma unroll
                for (int q = 0; q < 6; ++q) { a.eps_p_t[so + q] = ep[q]; a.sig_t[so + q] = sg[q]; }
                const long long to = ((long long)bb * d.V + vox) * 21;
#pragma unroll
                for (int q = 0; q < 21; ++q) {
                    if (a.tan_out_f) a.tan_out_f[to + q] = (float)tn[q];
                    if (a.tan_out_d) a.tan_out_d[to + q] = tn[q];
                }
                const double ir2 = 0.70710678118654752440084436210485;
#pragma unroll
                for (int q = 0; q < 6; ++q) f[q * N3] = (T)(q < 3 ? sg[q] : ir2 * sg[q]);
            }
        }
    }

    // ---- CG curvature <p, K p> = sum_x eps : sigma, per right-hand side
    if constexpr (OpInfo<OPK>::apply) {
        if (a.cg) {
            for (int rr = 0; rr < RB; ++rr) {
                double v1[1] = {eacc[rr]};
                block_sum<1>(v1, red);
                if (t == 0) ecc[rr] = v1[0];
            }
            const int nblk = gridDim.x;
            if (t == 0) {
                for (int rr = 0; rr < RB; ++rr)
                    a.partials[(long long)(g * RB + rr) * nblk + blockIdx.x] = ecc[rr];
                __threadfence();
                const unsigned prev = atomicAdd(a.counters + g, 1u);
                is_last = (prev == (unsigned)nblk - 1);
            }
            __syncthreads();
            if (is_last && t < RB) {
                __threadfence();
                const int bb = g * RB + t;
                double s = 0.0;
                for (int k = 0; k < nblk; ++k) s += __ldcg(a.partials + (long long)bb * nblk + k);
                CgState& cs = a.cg[bb];
                if (!cs.done) {
                    cs.pq = s;
                    if (s > 0.0 && s == s) {
                        cs.alpha = cs.rho / s;
                    } else {
                        cs.alpha = 0.0;
                        cs.flags |= (s == s) ? 1 : 2;
                        cs.done = 1;
                    }
                }
            }
            if (is_last && t == 0) a.counters[g] = 0u;
        }
    }
    if constexpr (!OpInfo<OPK>::forward) return;
    __syncthreads();

    // ---- R2C
    {
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int jj = p + r * P;
            v[r] = mk(my[2 * jj], my[2 * jj + 1]);
        }
        ColFFT<T, M, R, -1>::run(v, myc, 1, p, a.tw.tm);
        __syncthreads();
        if (slot_ok) {
#pragma unroll
            for (int r = 0; r < R; ++r) myc[p + r * P] = v[r];
        }
        __syncthreads();
        if (valid) {
            const T half = T(0.5);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = p + r * P;
                const cplx<T> Zk = myc[k];
                const cplx<T> Zc = conjg(myc[(M - k) & (M - 1)]);
                const cplx<T> e = ldg_c(a.tw.t3 + k);  // e^{-2 pi i k / n}
                const cplx<T> dlt = e * (Zk - Zc);
                // X = (Zk + Zc)/2 - (i/2) dlt
                stc(a.W + base + k, mk(half * (Zk.x + Zc.x) + half * dlt.y, half * (Zk.y + Zc.y) - half * dlt.x));
            }
            if (p == 0) {
                const cplx<T> Z0 = myc[0];
                stc(a.W + base + M, mk(Z0.x - Z0.y, T(0)));
            }
        }
    }
}

}  // namespace dbfft
