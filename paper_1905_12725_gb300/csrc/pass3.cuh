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
    OP_ADJ = 5,        // dJ/dE(x) = (1/N) eps_adj : C1 : eps_fwd (no forward R2C)
    OP_CP_UPDATE32 = 6, // OP_CP_UPDATE for an FP32 inner solve: FP32 Newton start, FP32 tangent
    OP_SVK_APPLY = 7,   // dP = K(F) : (G + macro) from the stored SVK tangent data (F, S)
    OP_SVK_UPDATE = 8,  // St. Venant-Kirchhoff P(F), F = macro (incl. I) + G; stores F and S
    OP_DISP = 9,        // total displacement Hbar x + u~ from the 3 inverse-transformed components (no R2C)
    OP_FCP_APPLY = 10,  // dP = K : (G + macro) from the stored finite-strain crystal-plasticity data (45)
    OP_FCP_UPDATE = 11, // finite-strain crystal plasticity, F = Fe Fp: P, Fp, T and the tangent data
    OP_FCP_UPDATE32 = 12, // OP_FCP_UPDATE for an FP32 inner solve: FP32 start of the local solve
    OP_LOADW = 13,        // real field from real_in ([B][V][6], Mandel) into the lines, then R2C (zero_in)
    OP_STOREW = 14        // C2R, then the real field plus the macro part to real_out ([B][V][6], Mandel)
};

template <typename T>
struct Ax3Args {
    Dims d;
    Twiddles<T> tw;
    cplx<T>* W;            // [B][nc][H]
    const cplx<T>* W2;     // OP_ADJ: adjoint strain field in W layout
    int RB;                // right-hand sides per CTA (divides Rm)
    int L;                 // grid lines per CTA (per tile for the pipelined pass)
    int pipe;              // CG applications: 1 = pipelined pass (k_axis3_pipe), 0 = k_axis3
    int zero_in;           // the input field is known to be zero: no load, no C2R (real fields start at 0)
    int radix;             // radix of the half-length transform (FP32: 8 or 16; FP64: 4)
    const T* macroW;       // [B][9] constant field added before the op (W components)
    const T* macroW2;      // OP_ADJ: macro part of the adjoint field
    // CG curvature (apply ops only; null outside CG)
    CgState* cg;
    double* partials;      // [B][nblk]
    unsigned* counters;    // [B / RB]
    // materials
    const uint16_t* phase; // [Bm][V]
    const T* scale;        // [Bm][V] or null
    const T* lam;          // per phase (in the pass precision)
    const T* mu;
    // nonlinear tangent / state
    const T* tan_in;       // apply ops: [B][V][ntan]
    float* tan_out_f;      // update ops: tangent written in FP32 (or null)
    double* tan_out_d;     // update ops: tangent written in FP64 (or null)
    const CpGrain* grains; // CP per-grain data
    const CpGrainF* grains_f; // the same in FP32
    CpParams cp;
    int guess_trial;       // CP: start the local Newton from the trial stress (not the committed one)
    const double* eps_p;   // [B][V][6] committed plastic strain
    const double* sig_prev;// [B][V][6] committed stress (Newton start)
    double* eps_p_t;       // trial plastic strain
    double* sig_t;         // trial stress
    unsigned* err;         // error bits (bit 0: local Newton failure)
    double* dJdE;          // OP_ADJ output [B][V]
    double* real_out;      // OP_DISP output [B][3][V]; macroW holds Hbar row-major [B][9]
    const double* fp_old;  // OP_FCP_UPDATE: committed Fp [B][V][9]
    double* fp_new;        // OP_FCP_UPDATE: trial Fp [B][V][9]
    double hx[3];          // OP_DISP: voxel edge lengths L_a / n_a
    long long wait_limit;  // polls of a bulk-copy wait before it gives up (0: the default, 2^26)
    const double* real_in; // OP_LOADW input [B][V][6] (Mandel components)
};

template <int OPK> struct OpInfo {
    static constexpr bool forward = OPK != OP_ADJ && OPK != OP_DISP && OPK != OP_STOREW;
    static constexpr bool apply =
        OPK == OP_ISO || OPK == OP_NH_APPLY || OPK == OP_CP_APPLY || OPK == OP_SVK_APPLY || OPK == OP_FCP_APPLY;
};

// Complex entries per slot buffer: room for the half-spectrum line (M + 1),
// the real line (M complex) and, when a line's transform is shared among
// threads, the padded FFT exchange. Several threads per line: the slot
// stride is 16 banks modulo 32 (neighbouring slots of a half-warp then use
// disjoint banks). One thread per line (radix = M, no exchange): the stride
// is an odd number of 8- or 16-byte words, so the lanes of a warp, each on
// its own line, read the same position of 32 lines without bank conflicts.
template <typename T, int N3, int RW = 8>
__host__ __device__ constexpr int ax3_slot_cplx() {
    constexpr int M = N3 / 2;
    constexpr int R = radix_ax3(M, sizeof(T) == 8, RW);
    if constexpr (R == M) {
        int n = M + 1;
        const int words = (int)sizeof(cplx<T>) / 4;  // 2 (FP32) or 4 (FP64)
        while (((n * words) & 31) != words) ++n;
        return n;
    } else {
        int n = padded_len<T>(M) > M + 1 ? padded_len<T>(M) : M + 1;
        while (((n * (int)sizeof(cplx<T>) / 4) & 31) != 16) ++n;
        return n;
    }
}

// Shared-memory layout: one buffer of SB = N3 + 2 values per slot
// (slot = grid line x right-hand side x component), holding either the
// half-spectrum line (N3/2 + 1 complex values) or the real line (N3 values),
// plus one scratch buffer for idle threads of the last FFT round. Global
// loads and stores are done cooperatively: for one (right-hand side,
// component) the L lines of a CTA are L h contiguous complex values.
template <typename T, int N3, int NC, int OPK, int RW>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? (RW == 32 ? 2 : (RW == 16 ? 2 : 3)) : ((RW == 32 || OPK == OP_CP_UPDATE || OPK == OP_CP_UPDATE32 || OPK == OP_NH_UPDATE || OPK == OP_SVK_UPDATE || OPK == OP_FCP_UPDATE || OPK == OP_FCP_UPDATE32) ? 1 : 2))) k_axis3(Ax3Args<T> a) {
    constexpr bool CPU_ = OPK == OP_CP_UPDATE || OPK == OP_CP_UPDATE32;  // crystal-plasticity update
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    constexpr int M = N3 / 2;
    constexpr int H = M + 1;
    constexpr int R = RadixAx3<T, M, RW>::value;
    constexpr int P = M / R;
    constexpr int SB = 2 * ax3_slot_cplx<T, N3, RW>();  // in T values
    static_assert(P <= 32 && (32 % P) == 0, "a slot's threads must sit inside one warp");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sbuf = reinterpret_cast<T*>(smraw);
    __shared__ double red[32 * 8];
    __shared__ double ecc[8];
    __shared__ bool is_last;
    const Dims& d = a.d;
    const int RB = a.RB, L = a.L;
    const int NSLOT = L * RB * NC;
    const int NF = (OPK == OP_ADJ) ? 2 : 1;  // fields carried (the adjoint reads two)
    const int t = threadIdx.x;
    const int nthr = blockDim.x;
    const int per_round = nthr / P;
    const int rounds = (NSLOT + per_round - 1) / per_round;
    const int g = blockIdx.y;
    const long long nlines = (long long)d.n1 * d.n2;
    const long long line0 = (long long)blockIdx.x * L;
    const int lines_here = (int)min((long long)L, nlines - line0);
    T* scratch = sbuf + (long long)NF * NSLOT * SB;
    // slot s = (ll * RB + rl) * NC + c ; field f at offset f * NSLOT
    auto slot_ptr = [&](int f, int sl) { return sbuf + ((long long)f * NSLOT + sl) * SB; };
    // stopped right-hand sides of this group, read once (bit rl)
    // (kept in shared memory, so that no register holds it through the kernel)
    __shared__ unsigned s_done;
    {
        unsigned done_mask = 0;
        if (a.cg != nullptr)
            for (int rl = 0; rl < RB; ++rl) done_mask |= (a.cg[g * RB + rl].done != 0 ? 1u : 0u) << rl;
        if (a.cg != nullptr && done_mask == (1u << RB) - 1u) return;  // the whole group has stopped
        if (t == 0) s_done = done_mask;
        __syncthreads();
    }
    auto rhs_done = [&](int rl) { return (s_done >> rl) & 1u; };
    // the macro parts of the group's right-hand sides, staged once per CTA
    // (visible after the barrier that ends the load / C2R phase)
    __shared__ T s_macro[8 * 9];
    for (int i = t; i < RB * 9; i += nthr) s_macro[i] = a.macroW[(long long)g * RB * 9 + i];

    if (a.zero_in) {  // real-space input fields are zero: clear the real lines instead
        for (int i = t; i < NF * NSLOT * N3; i += nthr) {
            const int sl = i / N3, x3 = i - sl * N3;
            sbuf[(long long)sl * SB + x3] = T(0);
        }
        __syncthreads();
    } else {
    // ---- cooperative load of the half-spectrum lines: for each (rhs, comp)
    // the lines of this CTA are lines_here * H contiguous complex values
    for (int f = 0; f < NF; ++f) {
        const cplx<T>* src = f == 0 ? a.W : a.W2;
        const int per_rc = lines_here * H;
        for (int rc = 0; rc < RB * NC; ++rc) {
            const int rl = rc / NC, c = rc - rl * NC;
            if (rhs_done(rl)) continue;
            const int b = g * RB + rl;
            const cplx<T>* gsrc = src + ((long long)(b * NC + c) * nlines + line0) * H;
            for (int i = t; i < per_rc; i += nthr) {
                const int ll = i / H, k = i - ll * H;  // H is a compile-time constant
                cp_async_c(reinterpret_cast<cplx<T>*>(slot_ptr(f, (ll * RB + rl) * NC + c)) + k, gsrc + i);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- C2R per slot: Z[k] = (X[k] + conj X[M-k]) + i e^{+2 pi i k/n} (X[k] - conj X[M-k])
    for (int f = 0; f < NF; ++f) {
        for (int rd = 0; rd < rounds; ++rd) {
            const int sl = rd * per_round + t / P;
            const int p = t % P;
            const bool ok = sl < NSLOT && t / P < per_round;
            T* my = ok ? slot_ptr(f, sl) : scratch;
            cplx<T>* myc = reinterpret_cast<cplx<T>*>(my);
            cplx<T> v[R];
            if constexpr (P == 1) {
                // the whole line in this thread: X[k] and X[M-k] read once for both
                // Z[k] and Z[M-k] (Z[M-k] = conj(A) - i e_{M-k}^* conj(B) with A, B of k),
                // twiddles as compile-time constants
                sfor<0, M / 2 + 1>([&](auto kc) {
                    constexpr int k = decltype(kc)::value;
                    constexpr int km = M - k;
                    const cplx<T> X = myc[k];
                    const cplx<T> Xc = conjg(myc[km]);
                    const cplx<T> A = X + Xc, Bd = X - Xc;
                    const cplx<T> dl = conjg(tw_const<T, N3, k>()) * Bd;
                    v[k] = A + mk(-dl.y, dl.x);
                    if constexpr (k != 0 && k != km) {
                        const cplx<T> dl2 = conjg(tw_const<T, N3, km>()) * mk(-Bd.x, Bd.y);  // -conj(Bd)
                        v[km] = conjg(A) + mk(-dl2.y, dl2.x);
                    }
                });
            } else {
                // pairs (k, M - k): with S = X[k] + conj X[M-k] and Q = e^{+2 pi i k/n} (X[k] - conj X[M-k]),
                // Z[k] = S + i Q and Z[M - k] = conj(S) + i conj(Q). Each thread takes its registers
                // r < R/2; Z[M - k] is register R - 1 - r of the partner thread P - p (the P threads
                // of a slot are consecutive lanes), which receives it by shuffle. Thread 0 is its own
                // partner: its Z[M - P r] belongs in register R - r (moved below), Z[M/2] = 2 conj X[M/2].
                const int lane = t & 31;
                const int partner = (lane & ~(P - 1)) | ((P - p) & (P - 1));
#pragma unroll
                for (int r = 0; r < R / 2; ++r) {
                    const int k = p + r * P;
                    const cplx<T> X = myc[k];
                    const cplx<T> Xc = conjg(myc[M - k]);
                    const cplx<T> e = conjg(ldg_c(a.tw.t3 + k));
                    const cplx<T> S = X + Xc, Q = e * (X - Xc);
                    v[r] = S + mk(-Q.y, Q.x);
                    const cplx<T> zp = mk(S.x + Q.y, Q.x - S.y);
                    v[R - 1 - r].x = __shfl_sync(0xffffffffu, zp.x, partner);
                    v[R - 1 - r].y = __shfl_sync(0xffffffffu, zp.y, partner);
                }
                const bool p0 = p == 0;
#pragma unroll
                for (int j = R - 1; j > R / 2; --j) v[j] = p0 ? v[j - 1] : v[j];
                const cplx<T> xm = myc[M / 2];
                if (p0) v[R / 2] = mk(T(2) * xm.x, T(-2) * xm.y);
            }
            __syncwarp();  // the slot's threads (one warp-aligned group) have read their line
            ColFFT<T, M, R, +1, true, true>::run(v, myc, 1, p, a.tw.tm);
            __syncwarp();
            // real values x[2j], x[2j+1] = Re, Im z[j]: one complex store per j
#pragma unroll
            for (int r = 0; r < R; ++r) myc[p + r * P] = v[r];
        }
    }
    __syncthreads();
    }  // !zero_in

    // ---- per-voxel operation
    T eacc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) eacc[q] = T(0);
    const int mat = (g * RB) / d.Rm;
    for (int idx = t; idx < lines_here * N3; idx += nthr) {
        const int lv = idx / N3, x3 = idx - lv * N3;
        const long long vox = (line0 + lv) * N3 + x3;
        if constexpr (OPK == OP_ISO || OPK == OP_ADJ) {
            const long long mv = (long long)mat * d.V + vox;
            const int ph = a.phase[mv];
            const T sc = a.scale ? a.scale[mv] : T(1);
            const T lam = a.lam[ph] * sc, mu = a.mu[ph] * sc;
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                if (rhs_done(rr)) continue;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                T e[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) e[q] = f[q * SB] + s_macro[rr * 9 + q];
                if constexpr (OPK == OP_ADJ) {
                    // dJ/dE = (1/N) eps_adj : C1 : eps_fwd, C1 = C / E: for this
                    // op the phase tables hold lam, mu per unit Young's modulus
                    const T* f2 = slot_ptr(1, (lv * RB + rr) * NC) + x3;
                    T e2[NC];
#pragma unroll
                    for (int q = 0; q < NC; ++q) e2[q] = f2[q * SB] + a.macroW2[bb * 9 + q];
                    T sg[NC];
                    iso_stress<T, NC>(e, a.lam[ph], a.mu[ph], sg);
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
                        eacc[rr] += en;
                    }
#pragma unroll
                    for (int q = 0; q < NC; ++q) f[q * SB] = sg[q];
                }
            }
        } else if constexpr (OPK == OP_NH_APPLY || OPK == OP_SVK_APPLY) {
            constexpr int NT = OPK == OP_SVK_APPLY ? 15 : 10;  // tangent data per voxel
            const long long mv = (long long)mat * d.V + vox;
            const int ph = a.phase[mv];
            const T lam = a.lam[ph], mu = a.mu[ph];
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                if (rhs_done(rr)) continue;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                T G[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) G[q] = f[q * SB] + s_macro[rr * 9 + q];
                const T* tn = a.tan_in + ((long long)bb * d.V + vox) * NT;
                T sg[9];
                if constexpr (OPK == OP_SVK_APPLY)
                    svk_apply<T>(tn, mu, lam, G, sg);
                else
                    nh_apply<T>(tn, mu, lam, G, sg);
                if (a.cg) {
                    T en = T(0);
#pragma unroll
                    for (int q = 0; q < 9; ++q) en += G[q] * sg[q];
                    eacc[rr] += en;
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) f[q * SB] = sg[q];
            }
        } else if constexpr (OPK == OP_NH_UPDATE || OPK == OP_SVK_UPDATE) {
            constexpr int NT = OPK == OP_SVK_UPDATE ? 15 : 10;
            const long long mv = (long long)mat * d.V + vox;
            const int ph = a.phase[mv];
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                double F[9], Pk[9], tn[NT];
#pragma unroll
                for (int q = 0; q < 9; ++q) F[q] = (double)f[q * SB] + s_macro[rr * 9 + q];
                bool ok;
                if constexpr (OPK == OP_SVK_UPDATE)
                    ok = svk_stress(F, a.mu[ph], a.lam[ph], Pk, tn);
                else
                    ok = nh_stress(F, a.mu[ph], a.lam[ph], Pk, tn);
                if (!ok) atomicOr(a.err, 1u);
                const long long to = ((long long)bb * d.V + vox) * NT;
#pragma unroll
                for (int q = 0; q < NT; ++q) {
                    if (a.tan_out_f) a.tan_out_f[to + q] = (float)tn[q];
                    if (a.tan_out_d) a.tan_out_d[to + q] = tn[q];
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) f[q * SB] = (T)Pk[q];
            }
        } else if constexpr (OPK == OP_FCP_APPLY) {
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                if (rhs_done(rr)) continue;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                T G[9], sg[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) G[q] = f[q * SB] + s_macro[rr * 9 + q];
                fcp_apply<T>(a.tan_in + ((long long)bb * d.V + vox) * 45, G, sg);
                if (a.cg) {
                    T en = T(0);
#pragma unroll
                    for (int q = 0; q < 9; ++q) en += G[q] * sg[q];
                    eacc[rr] += en;
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) f[q * SB] = sg[q];
            }
        } else if constexpr (OPK == OP_FCP_UPDATE || OPK == OP_FCP_UPDATE32) {
            const long long mv = (long long)mat * d.V + vox;
            const int gr = a.phase[mv];
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                double F[9], Pk[9], Fpn[9], Fpo[9], Tn[6], guess[6], tn[45];
#pragma unroll
                for (int q = 0; q < 9; ++q) F[q] = (double)f[q * SB] + s_macro[rr * 9 + q];
                const long long vo = (long long)bb * d.V + vox;
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
                for (int q = 0; q < 9; ++q) f[q * SB] = (T)Pk[q];
            }
        } else if constexpr (OPK == OP_LOADW || OPK == OP_STOREW) {
            // real 6-component fields in Mandel components (shear sqrt(2) x the tensor
            // component); the lines hold W components (the tensor components)
            const double r2 = 1.41421356237309504880168872420970;
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                const long long o = ((long long)bb * d.V + vox) * 6;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    if constexpr (OPK == OP_LOADW) {
                        f[q * SB] = (T)(q < 3 ? a.real_in[o + q] : a.real_in[o + q] / r2);
                    } else {
                        const double v = (double)f[q * SB] + (double)s_macro[rr * 9 + q];
                        a.real_out[o + q] = q < 3 ? v : r2 * v;
                    }
                }
            }
        } else if constexpr (OPK == OP_DISP) {
            // u = Hbar x + u~ at the voxel centre x = (i + 1/2) h; u~ = the real line / N
            const long long ln = line0 + lv;
            const long long i1 = ln / d.n2;
            const double X[3] = {((double)i1 + 0.5) * a.hx[0], ((double)(ln - i1 * d.n2) + 0.5) * a.hx[1],
                                 ((double)x3 + 0.5) * a.hx[2]};
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                const T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double v = (double)f[c * SB] * d.invN + (double)s_macro[rr * 9 + 3 * c] * X[0] +
                                     (double)s_macro[rr * 9 + 3 * c + 1] * X[1] + (double)s_macro[rr * 9 + 3 * c + 2] * X[2];
                    a.real_out[((long long)bb * 3 + c) * d.V + vox] = v;
                }
            }
        } else if constexpr (OPK == OP_CP_APPLY) {
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                if (rhs_done(rr)) continue;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                T e[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) e[q] = f[q * SB] + s_macro[rr * 9 + q];
                const T* tn = a.tan_in + ((long long)bb * d.V + vox) * 21;
                T sg[6];
                cp_apply<T>(tn, e, sg);
                if (a.cg) {
                    T en = T(0);
#pragma unroll
                    for (int q = 0; q < 6; ++q) en += (q >= 3 ? T(2) : T(1)) * e[q] * sg[q];
                    eacc[rr] += en;
                }
#pragma unroll
                for (int q = 0; q < 6; ++q) f[q * SB] = sg[q];
            }
        } else if constexpr (CPU_) {
            const long long mv = (long long)mat * d.V + vox;
            const int gr = a.phase[mv];
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                T* f = slot_ptr(0, (lv * RB + rr) * NC) + x3;
                double e[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) e[q] = (double)f[q * SB] + s_macro[rr * 9 + q];
                const long long so = ((long long)bb * d.V + vox) * 6;
                double sg[6], ep[6], guess[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) guess[q] = (a.guess_trial ? a.sig_t : a.sig_prev)[so + q];
                const long long to = ((long long)bb * d.V + vox) * 21;
                bool ok;
                if constexpr (OPK == OP_CP_UPDATE32) {
                    float tn[21];
                    ok = cp_update<float>(a.grains[gr], a.grains_f[gr], a.cp, e, a.eps_p + so, guess, sg, tn, ep);
#pragma unroll
                    for (int q = 0; q < 21; ++q) a.tan_out_f[to + q] = tn[q];
                } else {
                    double tn[21];
                    ok = cp_update<double>(a.grains[gr], a.grains_f[gr], a.cp, e, a.eps_p + so, guess, sg, tn, ep);
#pragma unroll
                    for (int q = 0; q < 21; ++q) a.tan_out_d[to + q] = tn[q];
                }
                if (!ok) atomicOr(a.err, 1u);
#pragma unroll
                for (int q = 0; q < 6; ++q) { a.eps_p_t[so + q] = ep[q]; a.sig_t[so + q] = sg[q]; }
                const double ir2 = 0.70710678118654752440084436210485;
#pragma unroll
                for (int q = 0; q < 6; ++q) f[q * SB] = (T)(q < 3 ? sg[q] : ir2 * sg[q]);
            }
        }
    }

    // ---- CG curvature <p, K p> = sum_x eps : sigma, per right-hand side
    if constexpr (OpInfo<OPK>::apply) {
        if (a.cg) {
            for (int rr = 0; rr < RB; ++rr) {
                double v1[1];
                const T in1[1] = {eacc[rr]};
                block_sum_t<T, 1>(in1, v1, red);
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
            if (is_last) {  // the whole last block reduces the partials (fixed order)
                __threadfence();
                for (int rr = 0; rr < RB; ++rr) {
                    const int bb = g * RB + rr;
                    double v1[1] = {0.0};
                    for (int k = t; k < nblk; k += nthr) v1[0] += __ldcg(a.partials + (long long)bb * nblk + k);
                    block_sum<1>(v1, red);
                    if (t == 0) {
                        const double sum = v1[0];
                        CgState& cs = a.cg[bb];
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
                    }
                }
                if (t == 0) a.counters[g] = 0u;
            }
        }
    }
    if constexpr (!OpInfo<OPK>::forward) return;
    __syncthreads();

    // ---- R2C per slot, result staged back into the slot buffer
    for (int rd = 0; rd < rounds; ++rd) {
        const int sl = rd * per_round + t / P;
        const int p = t % P;
        const bool ok = sl < NSLOT && t / P < per_round;
        T* my = ok ? slot_ptr(0, sl) : scratch;
        cplx<T>* myc = reinterpret_cast<cplx<T>*>(my);
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = myc[p + r * P];  // z[j] = x[2j] + i x[2j+1]
        __syncwarp();
        ColFFT<T, M, R, -1, true, true>::run(v, myc, 1, p, a.tw.tm);
        __syncwarp();
        if constexpr (P == 1) {
            // the whole line is in this thread's registers: X[k] and X[M-k] from
            // Z[k] and Z[M-k] directly, written pairwise
            const T half = T(0.5);
            sfor<0, M / 2 + 1>([&](auto kk) {
                constexpr int k = decltype(kk)::value;
                constexpr int kc = (M - k) & (M - 1);
                const cplx<T> Zk = v[k], Zc = conjg(v[kc]);
                const cplx<T> dl = tw_const<T, N3, k>() * (Zk - Zc);
                myc[k] = mk(half * (Zk.x + Zc.x) + half * dl.y, half * (Zk.y + Zc.y) - half * dl.x);
                if constexpr (k != 0 && k != M - k) {
                    const cplx<T> Zk2 = v[kc], Zc2 = conjg(v[k]);
                    const cplx<T> dl2 = tw_const<T, N3, M - k>() * (Zk2 - Zc2);
                    myc[M - k] = mk(half * (Zk2.x + Zc2.x) + half * dl2.y, half * (Zk2.y + Zc2.y) - half * dl2.x);
                }
            });
            myc[M] = mk(v[0].x - v[0].y, T(0));
            continue;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) myc[p + r * P] = v[r];
        __syncwarp();
        // pairs (k, M - k): with S = Z[k] + conj Z[M-k] and Q = e^{-2 pi i k/n} (Z[k] - conj Z[M-k]),
        // X[k] = (S - i Q) / 2 and X[M - k] = (conj S - i conj Q) / 2; each thread takes r < R/2
        // (thread 0: r = 0 gives X[0] and the Nyquist X[M]) and thread 0 adds X[M/2] = conj Z[M/2]
        cplx<T> Xa[R / 2], Xb[R / 2];
        const T half = T(0.5);
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
            const int k = p + r * P;
            const cplx<T> Zk = myc[k];
            const cplx<T> Zc = conjg(myc[(M - k) & (M - 1)]);
            const cplx<T> e = ldg_c(a.tw.t3 + k);  // e^{-2 pi i k / n}
            const cplx<T> S = Zk + Zc, Q = e * (Zk - Zc);
            Xa[r] = mk(half * (S.x + Q.y), half * (S.y - Q.x));
            Xb[r] = mk(half * (S.x - Q.y), -half * (S.y + Q.x));
        }
        const cplx<T> Xmid = conjg(myc[M / 2]);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R / 2; ++r) {
            myc[p + r * P] = Xa[r];
            myc[M - p - r * P] = Xb[r];
        }
        if (p == 0) myc[M / 2] = Xmid;
    }
    __syncthreads();

    // ---- cooperative store
    {
        const int per_rc = lines_here * H;
        for (int rc = 0; rc < RB * NC; ++rc) {
            const int rl = rc / NC, c = rc - rl * NC;
            if (rhs_done(rl)) continue;
            const int b = g * RB + rl;
            cplx<T>* gdst = a.W + ((long long)(b * NC + c) * nlines + line0) * H;
            for (int i = t; i < per_rc; i += nthr) {
                const int ll = i / H, k = i - ll * H;
                stc(gdst + i, reinterpret_cast<const cplx<T>*>(slot_ptr(0, (ll * RB + rl) * NC + c))[k]);
            }
        }
    }
}

}  // namespace dbfft
