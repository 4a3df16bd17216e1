// constitutive.cuh -- per-voxel material laws evaluated inside pass 3.
//
//  * linear isotropic elasticity: sigma = lam tr(eps) I + mu (eps + eps^T)
//  * compressible Neo-Hookean (finite strain), W = mu/2 (tr F^T F - 3)
//    - mu ln J + lam/2 (ln J)^2:  P = mu (F - F^-T) + lam ln J F^-T and
//    dP = mu G + (mu - lam ln J) F^-T G^T F^-T + lam (F^-T : G) F^-T
//  * small-strain FCC crystal plasticity with power-law slip rates,
//    backward Euler on the stress (Mandel 6-vectors):
//      R(s) = S s + dt sum_a gdot_a(s) P_a - (eps_{n+1} - eps_p,n) = 0,
//    solved by Newton (stopped on the full Newton step) with backtracking,
//    far from the solution, on the convex potential whose gradient R is;
//    consistent tangent (S + dt sum_a gdot'_a P_a P_a^T)^-1;
//  * finite-strain crystal plasticity, F = Fe Fp: the same local problem on
//    the second Piola-Kirchhoff stress of the intermediate configuration with
//    the trial Green strain as the strain, then the update of Fp.
// The converged stress is FP64; a mixed-precision context runs the first
// Newton iterations in FP32.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace dbfft {

struct CpGrain {
    double S[21];     // Mandel compliance, upper triangle row-major
    double P[12][6];  // Schmid tensors sym(s x n), Mandel, sample frame
    double sv[12][3]; // slip directions and plane normals, sample frame (finite strain)
    double nv[12][3];
};

struct CpGrainF {  // the same in FP32
    float S[21];
    float P[12][6];
};

template <typename R>
struct CpScalars {
    R gdot0, inv_m, tau_c, dt;
    R inv_tc;    // 1 / tau_c
    R dtg;       // dt gdot0
    R dtg_n_tc;  // dt gdot0 (1/m) / tau_c
    R dtk;       // dt gdot0 tau_c m / (1 + m): potential coefficient
};

struct CpParams {
    CpScalars<double> d;
    CpScalars<float> f;
    double rtol;
    int max_it;
    int n_int;  // 1/m when it is an integer in [1, 127] (powers by products), else 0
};

__host__ __device__ __forceinline__ constexpr int sym6(int i, int j) {
    if (i > j) { int t = i; i = j; j = t; }
    return i * 6 - (i * (i - 1)) / 2 + (j - i);
}

template <typename T, int NC>
__device__ __forceinline__ void iso_stress(const T* e, T lam, T mu, T* s) {
    if constexpr (NC == 6) {
        const T tr = e[0] + e[1] + e[2];
        s[0] = lam * tr + T(2) * mu * e[0];
        s[1] = lam * tr + T(2) * mu * e[1];
        s[2] = lam * tr + T(2) * mu * e[2];
        s[3] = T(2) * mu * e[3];
        s[4] = T(2) * mu * e[4];
        s[5] = T(2) * mu * e[5];
    } else {
        const T tr = e[0] + e[4] + e[8];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) s[3 * i + j] = mu * (e[3 * i + j] + e[3 * j + i]) + (i == j ? lam * tr : T(0));
    }
}

// Neo-Hookean: P(F) and the data of its tangent (F^-T, mu - lam ln J).
__device__ __forceinline__ bool nh_stress(const double* F, double mu, double lam, double* P, double* tn) {
    const double a = F[0], b = F[1], c = F[2], d = F[3], e = F[4], f = F[5], g = F[6], h = F[7], i = F[8];
    const double A00 = e * i - f * h, A01 = -(d * i - f * g), A02 = d * h - e * g;
    const double J = a * A00 + b * A01 + c * A02;
    if (!(J > 0.0)) {
        for (int q = 0; q < 9; ++q) P[q] = 0.0;
        for (int q = 0; q < 10; ++q) tn[q] = 0.0;
        return false;
    }
    const double iJ = 1.0 / J;
    // F^-T = cof(F) / J
    double A[9];
    A[0] = A00 * iJ; A[1] = A01 * iJ; A[2] = A02 * iJ;
    A[3] = -(b * i - c * h) * iJ; A[4] = (a * i - c * g) * iJ; A[5] = -(a * h - b * g) * iJ;
    A[6] = (b * f - c * e) * iJ; A[7] = -(a * f - c * d) * iJ; A[8] = (a * e - b * d) * iJ;
    const double lnJ = log(J);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        P[q] = mu * (F[q] - A[q]) + lam * lnJ * A[q];
        tn[q] = A[q];
    }
    tn[9] = mu - lam * lnJ;
    return true;
}

template <typename T>
__device__ __forceinline__ void nh_apply(const T* tn, T mu, T lam, const T* G, T* out) {
    T A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = tn[q];
    const T c1 = tn[9];
    // Bm = A G^T : Bm_ik = sum_L A_iL G_kL
    T Bm[9];
    T AG = T(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) AG += A[q] * G[q];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            Bm[3 * i + k] = A[3 * i + 0] * G[3 * k + 0] + A[3 * i + 1] * G[3 * k + 1] + A[3 * i + 2] * G[3 * k + 2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T bga = Bm[3 * i + 0] * A[0 * 3 + j] + Bm[3 * i + 1] * A[1 * 3 + j] + Bm[3 * i + 2] * A[2 * 3 + j];
            out[3 * i + j] = mu * G[3 * i + j] + c1 * bga + lam * AG * A[3 * i + j];
        }
}

// St. Venant-Kirchhoff: E = (F^T F - I)/2, S = lam tr(E) I + 2 mu E,
// P = F S. The tangent data are F (9) and S (6, order 11,22,33,23,13,12).
// The law is defined for every F; a non-finite P is reported as a failure.
__device__ __forceinline__ bool svk_stress(const double* F, double mu, double lam, double* P, double* tn) {
    double C[6];  // F^T F, same component order as S
    const int ci[6] = {0, 1, 2, 1, 0, 0}, cj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int q = 0; q < 6; ++q)
        C[q] = F[ci[q]] * F[cj[q]] + F[3 + ci[q]] * F[3 + cj[q]] + F[6 + ci[q]] * F[6 + cj[q]];
    const double trE = 0.5 * (C[0] + C[1] + C[2] - 3.0);
    double S[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) S[q] = mu * (C[q] - (q < 3 ? 1.0 : 0.0)) + (q < 3 ? lam * trE : 0.0);
    const double Sm[9] = {S[0], S[5], S[4], S[5], S[1], S[3], S[4], S[3], S[2]};
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double p = F[3 * i] * Sm[j] + F[3 * i + 1] * Sm[3 + j] + F[3 * i + 2] * Sm[6 + j];
            ok = ok && isfinite(p);
            P[3 * i + j] = p;
        }
#pragma unroll
    for (int q = 0; q < 9; ++q) tn[q] = F[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) tn[9 + q] = S[q];
    return ok;
}

// dP = K(F) : G = G S + F dS with dS = lam tr(dE) I + 2 mu dE, dE = sym(F^T G).
template <typename T>
__device__ __forceinline__ void svk_apply(const T* tn, T mu, T lam, const T* G, T* out) {
    T F[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) F[q] = tn[q];
    const T Sm[9] = {tn[9], tn[14], tn[13], tn[14], tn[10], tn[12], tn[13], tn[12], tn[11]};
    T H[9];  // F^T G
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) H[3 * i + j] = F[i] * G[j] + F[3 + i] * G[3 + j] + F[6 + i] * G[6 + j];
    const T tr = H[0] + H[4] + H[8];
    T dS[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dS[3 * i + j] = mu * (H[3 * i + j] + H[3 * j + i]) + (i == j ? lam * tr : T(0));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            out[3 * i + j] = G[3 * i] * Sm[j] + G[3 * i + 1] * Sm[3 + j] + G[3 * i + 2] * Sm[6 + j] +
                             F[3 * i] * dS[j] + F[3 * i + 1] * dS[3 + j] + F[3 * i + 2] * dS[6 + j];
}

// Finite-strain crystal plasticity (F = Fe Fp): tangent data per voxel, 45
// values: Fe_tr = F a (9), a = Fp_old^-1 (9), B = a T a^T (6, order
// 11,22,33,23,13,12), C_tan = dT/dE_tr (21, Mandel). dP = G B + Fe_tr dT a^T,
// dT = C_tan : sym(Fe_tr^T G a): the derivative of F a T(E(F)) a^T with the
// plastic state held (major-symmetric).
template <typename T>
__device__ __forceinline__ void fcp_apply(const T* tn, const T* G, T* out) {
    const T* Fe = tn;
    const T* A = tn + 9;
    const T Bm[9] = {tn[18], tn[23], tn[22], tn[23], tn[19], tn[21], tn[22], tn[21], tn[20]};
    const T* Ct = tn + 24;
    T Y[9];  // G a
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Y[3 * i + j] = G[3 * i] * A[j] + G[3 * i + 1] * A[3 + j] + G[3 * i + 2] * A[6 + j];
    T H[9];  // Fe^T G a
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) H[3 * i + j] = Fe[i] * Y[j] + Fe[3 + i] * Y[3 + j] + Fe[6 + i] * Y[6 + j];
    const T r2h = T(0.70710678118654752440);  // sqrt(2) / 2
    const T e6[6] = {H[0], H[4], H[8], r2h * (H[5] + H[7]), r2h * (H[2] + H[6]), r2h * (H[1] + H[3])};
    T d6[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += Ct[sym6(i, j)] * e6[j];
        d6[i] = acc;
    }
    const T dT[9] = {d6[0], r2h * d6[5], r2h * d6[4], r2h * d6[5], d6[1], r2h * d6[3], r2h * d6[4], r2h * d6[3], d6[2]};
    T Z[9];  // Fe dT
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Z[3 * i + j] = Fe[3 * i] * dT[j] + Fe[3 * i + 1] * dT[3 + j] + Fe[3 * i + 2] * dT[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            out[3 * i + j] = G[3 * i] * Bm[j] + G[3 * i + 1] * Bm[3 + j] + G[3 * i + 2] * Bm[6 + j] +
                             Z[3 * i] * A[3 * j] + Z[3 * i + 1] * A[3 * j + 1] + Z[3 * i + 2] * A[3 * j + 2];
}

// Inverse of a 3x3 matrix (row-major) by cofactors; false when singular.
__device__ __forceinline__ bool inv3(const double* M, double* R) {
    const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    if (!(det != 0.0) || !isfinite(det)) return false;
    const double id = 1.0 / det;
    R[0] = c00 * id; R[1] = (M[2] * M[7] - M[1] * M[8]) * id; R[2] = (M[1] * M[5] - M[2] * M[4]) * id;
    R[3] = c01 * id; R[4] = (M[0] * M[8] - M[2] * M[6]) * id; R[5] = (M[2] * M[3] - M[0] * M[5]) * id;
    R[6] = c02 * id; R[7] = (M[1] * M[6] - M[0] * M[7]) * id; R[8] = (M[0] * M[4] - M[1] * M[3]) * id;
    return true;
}

// sigma (W components 11,22,33,23,13,12) = C_mandel eps, 21-entry tangent.
template <typename T>
__device__ __forceinline__ void cp_apply(const T* tn, const T* e, T* s) {
    const T r2 = T(1.41421356237309504880168872420970);
    const T ir2 = T(0.70710678118654752440084436210485);
    const T em[6] = {e[0], e[1], e[2], r2 * e[3], r2 * e[4], r2 * e[5]};
    T sm[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += tn[sym6(i, j)] * em[j];
        sm[i] = acc;
    }
    s[0] = sm[0]; s[1] = sm[1]; s[2] = sm[2];
    s[3] = ir2 * sm[3]; s[4] = ir2 * sm[4]; s[5] = ir2 * sm[5];
}

// ---- crystal plasticity, local problem
// Index of (i, j), i > j, in a strictly lower 6x6 triangle stored by rows.
__host__ __device__ __forceinline__ constexpr int lo6(int i, int j) { return i * (i - 1) / 2 + j; }

template <typename R> struct CpGrainOf;
template <> struct CpGrainOf<double> { using type = CpGrain; };
template <> struct CpGrainOf<float> { using type = CpGrainF; };

template <typename R>
__device__ __forceinline__ const CpScalars<R>& cp_scalars(const CpParams& cp) {
    if constexpr (sizeof(R) == 8) return cp.d;
    else return cp.f;
}

// x^k, 0 <= k < 128, by binary powering (exact products, no pow call).
template <typename R>
__device__ __forceinline__ R ipow(R x, int k) {
    R r = R(1), b = x;
#pragma unroll
    for (int bit = 0; bit < 7; ++bit) {
        if (k & (1 << bit)) r *= b;
        if ((k >> (bit + 1)) == 0) break;
        b *= b;
    }
    return r;
}

// xn = x^(1/m) and xn1 = x^(1/m - 1) for x = |tau| / tau_c >= 0.
template <typename R>
__device__ __forceinline__ void cp_powers(const CpParams& cp, R x, R& xn, R& xn1) {
    if (cp.n_int > 0) {
        xn1 = ipow<R>(x, cp.n_int - 1);
        xn = xn1 * x;
    } else {
        const CpScalars<R>& c = cp_scalars<R>(cp);
        xn = pow(x, c.inv_m);
        xn1 = x > R(0) ? xn / x : pow(x, c.inv_m - R(1));
    }
}

// Residual R(s) = S s + dt sum_a gdot_a(s) P_a - tg, optionally its Jacobian
// J = S + dt sum_a gdot'_a P_a P_a^T (21 packed entries, symmetric) and the
// convex potential phi(s) = 1/2 s.S.s - s.tg + dt sum_a k |tau_a / tau_c|^(1+1/m)
// whose gradient R is. All in precision R.
template <typename R, bool JAC, bool POT>
__device__ __forceinline__ void cp_eval(const typename CpGrainOf<R>::type& G, const CpParams& cp, const R (&s)[6],
                                        const R (&tg)[6], R (&Rv)[6], R (&J)[21], R& pot) {
    const CpScalars<R>& c = cp_scalars<R>(cp);
    if (POT) pot = R(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        R acc = R(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += G.S[sym6(i, j)] * s[j];
        Rv[i] = acc - tg[i];
        if (POT) pot += s[i] * (R(0.5) * acc - tg[i]);
    }
    if (JAC) {
#pragma unroll
        for (int q = 0; q < 21; ++q) J[q] = G.S[q];
    }
    R ppot = R(0);
#pragma unroll 1
    for (int al = 0; al < 12; ++al) {
        R Pa[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) Pa[j] = G.P[al][j];
        R tau = R(0);
#pragma unroll
        for (int j = 0; j < 6; ++j) tau += Pa[j] * s[j];
        const R x = fabs(tau) * c.inv_tc;
        R xn, xn1;
        cp_powers<R>(cp, x, xn, xn1);
        const R g = tau < R(0) ? -c.dtg * xn : c.dtg * xn;  // dt gdot_a (0 at tau = 0)
#pragma unroll
        for (int i = 0; i < 6; ++i) Rv[i] += g * Pa[i];
        if (JAC) {
            const R f = c.dtg_n_tc * xn1;  // dt d gdot_a / d tau
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const R fi = f * Pa[i];
#pragma unroll
                for (int j = i; j < 6; ++j) J[sym6(i, j)] += fi * Pa[j];
            }
        }
        if (POT) ppot += xn * x;
    }
    if (POT) pot += c.dtk * ppot;
}

// Compile-time loop: f(std::integral_constant<int, k>) for k = B .. E-1, so
// that every array index below is a constant and the arrays stay in registers.
template <int B, int E, typename F>
__device__ __forceinline__ void sfor(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// L D L^T factorisation of a packed symmetric 6x6 matrix; false unless
// positive definite (or on a non-finite entry).
template <typename R>
__device__ __forceinline__ bool ldl6(const R (&A)[21], R (&L)[15], R (&Di)[6]) {
    R D[6];
    bool ok = true;
    sfor<0, 6>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        R d = A[sym6(j, j)];
        sfor<0, j>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            d -= L[lo6(j, k)] * L[lo6(j, k)] * D[k];
        });
        ok = ok && (d > R(0));
        D[j] = d;
        Di[j] = R(1) / d;
        sfor<j + 1, 6>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            R t = A[sym6(j, i)];
            sfor<0, j>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                t -= L[lo6(i, k)] * L[lo6(j, k)] * D[k];
            });
            L[lo6(i, j)] = t * Di[j];
        });
    });
    return ok;
}

template <typename R>
__device__ __forceinline__ void ldl6_solve(const R (&L)[15], const R (&Di)[6], const R (&b)[6], R (&x)[6]) {
    R y[6];
    sfor<0, 6>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        R t = b[i];
        sfor<0, i>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            t -= L[lo6(i, k)] * y[k];
        });
        y[i] = t;
    });
    sfor<0, 6>([&](auto rc) {
        constexpr int i = 5 - decltype(rc)::value;
        R t = y[i] * Di[i];
        sfor<i + 1, 6>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            t -= L[lo6(k, i)] * x[k];
        });
        x[i] = t;
    });
}

// Newton on R(s) = 0 in precision R, from s (in/out). Stops once the full
// Newton step is below rtol (|s| + tau_c) (the step is then applied).
// Far from the solution (step > 1e-3 scale) the step is backtracked on the
// convex potential, with an allowance armijo |phi| for its round-off.
// Returns 1 when converged, 0 at the iteration cap, -1 on a non-SPD
// Jacobian or a non-finite step.
template <typename R>
__device__ __forceinline__ int cp_newton(const typename CpGrainOf<R>::type& G, const CpParams& cp, const R (&tg)[6],
                                         R (&s)[6], R rtol, R armijo, int max_it) {
    const R tau_c = cp_scalars<R>(cp).tau_c;
    for (int it = 0; it < max_it; ++it) {
        R Rv[6], J[21], L[15], Di[6], st[6], unused;
        cp_eval<R, true, false>(G, cp, s, tg, Rv, J, unused);
        if (!ldl6<R>(J, L, Di)) return -1;
        R mR[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) mR[i] = -Rv[i];
        ldl6_solve<R>(L, Di, mR, st);
        R slope = R(0), ns = R(0), sn = R(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            slope += Rv[i] * st[i];
            ns += st[i] * st[i];
            sn += s[i] * s[i];
        }
        if (!(ns <= R(3e38))) return -1;  // NaN or overflow
        const R scale = sqrt(sn) + tau_c;
        ns = sqrt(ns);
        R t = R(1);
        if (ns > R(1e-3) * scale) {
            R f0, Rj[6], Jj[21];
            cp_eval<R, false, true>(G, cp, s, tg, Rj, Jj, f0);
            for (int ls = 0; ls < 60; ++ls) {
                R trial[6], f;
#pragma unroll
                for (int i = 0; i < 6; ++i) trial[i] = s[i] + t * st[i];
                cp_eval<R, false, true>(G, cp, trial, tg, Rj, Jj, f);
                if (!(f > f0 + R(1e-4) * t * slope + armijo * fabs(f0))) break;
                t *= R(0.5);
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) s[i] += t * st[i];
        if (ns <= rtol * scale) return 1;
    }
    return 0;
}

// Simplified Newton in FP64 with a fixed FP32 factorisation (L, Di): the
// residual is evaluated in FP64, the step solved in FP32. Stops, like
// cp_newton, once the step is below rtol (|s| + tau_c). Returns 1 when
// converged, 0 otherwise (then s is left where the iteration stopped).
__device__ __forceinline__ int cp_refine64(const CpGrain& G, const CpParams& cp, const double (&tg)[6], double (&s)[6],
                                           const float (&L)[15], const float (&Di)[6], double rtol, int max_it) {
    for (int it = 0; it < max_it; ++it) {
        double Rv[6], J[21], unused;
        cp_eval<double, false, false>(G, cp, s, tg, Rv, J, unused);
        float mR[6], st[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) mR[i] = (float)(-Rv[i]);
        ldl6_solve<float>(L, Di, mR, st);
        double ns = 0.0, sn = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            ns += (double)st[i] * (double)st[i];
            sn += s[i] * s[i];
        }
        if (!(ns <= 1e300)) return 0;
#pragma unroll
        for (int i = 0; i < 6; ++i) s[i] += (double)st[i];
        if (ns <= rtol * rtol * (sqrt(sn) + cp.d.tau_c) * (sqrt(sn) + cp.d.tau_c)) return 1;
    }
    return 0;
}

// Backward-Euler update of one voxel. eps_w: total strain in W components
// (11,22,33,23,13,12); ep_old, s_guess, s_out, ep_new: Mandel 6-vectors;
// tan: 21-entry Mandel tangent (J^-1 at the solution) in precision TT.
// With TT = float (the FP32 inner-CG mode) Newton first runs in FP32 from
// s_guess; FP64 then finishes with simplified Newton steps (FP64 residual,
// FP32 Jacobian factors), falling back to FP64 Newton if those do not
// settle; the stored FP32 tangent is built in FP32. With TT = double
// everything runs in FP64 Newton. Both stop when the FP64 step is below the
// same tolerance, so both return the same stress to that tolerance.
// F32START = true with TT = double takes the FP32 start and builds the
// tangent in FP64.
// Returns false when the local Newton fails (outputs stay finite).
template <typename TT, bool F32START = (sizeof(TT) == 4)>
__device__ __forceinline__ bool cp_update(const CpGrain& G, const CpGrainF& Gf, const CpParams& cp,
                                          const double* eps_w, const double* ep_old, const double* s_guess,
                                          double* s_out, TT* tan, double* ep_new) {
    const double r2 = 1.41421356237309504880168872420970;
    const double em[6] = {eps_w[0], eps_w[1], eps_w[2], r2 * eps_w[3], r2 * eps_w[4], r2 * eps_w[5]};
    double tg[6], s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        tg[i] = em[i] - ep_old[i];
        s[i] = s_guess[i];
    }
    int r = 0;
    if constexpr (F32START) {
        float tgf[6], sf[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            tgf[i] = (float)tg[i];
            sf[i] = (float)s[i];
        }
        if (cp_newton<float>(Gf, cp, tgf, sf, 3e-6f, 1e-6f, 40) >= 0) {
            // FP64 finish with the FP32 Jacobian at the FP32 solution: each step
            // takes the FP64 residual and an FP32 solve, and the iteration
            // contracts by about cond(J) times the Jacobian's relative error
            float Rf[6], Jf[21], Lf[15], Dif[6], unused;
            cp_eval<float, true, false>(Gf, cp, sf, tgf, Rf, Jf, unused);
            if (ldl6<float>(Jf, Lf, Dif)) {
#pragma unroll
                for (int i = 0; i < 6; ++i) s[i] = sf[i];
                r = cp_refine64(G, cp, tg, s, Lf, Dif, cp.rtol, 8);
            }
            if (r != 1) {  // the simplified iteration did not settle: plain FP64 Newton from the FP32 point
#pragma unroll
                for (int i = 0; i < 6; ++i) s[i] = sf[i];
            }
        }
    }
    if (r != 1) r = cp_newton<double>(G, cp, tg, s, cp.rtol, 1e-13, cp.max_it);
    bool ok = r == 1;
    // plastic strain from the converged residual: eps_p = eps - S s
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double acc = em[i];
#pragma unroll
        for (int j = 0; j < 6; ++j) acc -= G.S[sym6(i, j)] * s[j];
        ep_new[i] = acc;
        s_out[i] = s[i];
    }
    // consistent tangent J^-1 at the solution, column by column
    using RT = TT;
    RT sT[6], tgT[6], Rv[6], J[21], L[15], Di[6], unused;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        sT[i] = (RT)s[i];
        tgT[i] = (RT)tg[i];
    }
    if constexpr (sizeof(TT) == 4) cp_eval<float, true, false>(Gf, cp, sT, tgT, Rv, J, unused);
    else cp_eval<double, true, false>(G, cp, sT, tgT, Rv, J, unused);
    const bool spd = ldl6<RT>(J, L, Di);
    ok = ok && spd;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        RT e[6], col[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) e[i] = RT(i == j ? 1 : 0);
        ldl6_solve<RT>(L, Di, e, col);
#pragma unroll
        for (int i = 0; i <= j; ++i) tan[sym6(i, j)] = spd ? col[i] : RT(0);
    }
    return ok;
}

// Finite-strain crystal-plasticity update at one voxel (FP64): F (9), the
// committed Fp_old (9), a start guess of T (Mandel 6). With a = Fp_old^-1,
// Fe_tr = F a and E_tr = (Fe_tr^T Fe_tr - I)/2, T solves the small-strain
// backward-Euler problem with E_tr as the strain (cp_update, no plastic strain
// at the start of the step); then Fp = (I + dt sum_a gdot_a s_a n_a) Fp_old,
// P = F Fp^-1 T Fp^-T. Writes P (9), Fp (9), T (Mandel 6) and the 45 tangent
// values (fcp_apply). False when the local solve or an inverse fails. F32START
// starts the local solve in FP32, as cp_update does for the mixed-precision
// inner solve, with the same FP64 stop rule on T; C_tan = J^-1 stays FP64
// (J has condition numbers of several hundred in plastic flow, so an FP32
// inverse would lose about 1e-5 of the tangent).
template <bool F32START>
__device__ __forceinline__ bool fcp_update(const CpGrain& G, const CpGrainF& Gf, const CpParams& cp, const double* F,
                                           const double* Fp_old, const double* T_guess, double* P, double* Fp,
                                           double* T, double* tn) {
    double a[9];
    bool ok = inv3(Fp_old, a);
    double Fe[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Fe[3 * i + j] = F[3 * i] * a[j] + F[3 * i + 1] * a[3 + j] + F[3 * i + 2] * a[6 + j];
    double A[9];  // Fe^T Fe
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[3 * i + j] = Fe[i] * Fe[j] + Fe[3 + i] * Fe[3 + j] + Fe[6 + i] * Fe[6 + j];
    // E_tr in W components (tensor 11, 22, 33, 23, 13, 12)
    const double Ew[6] = {0.5 * (A[0] - 1.0), 0.5 * (A[4] - 1.0), 0.5 * (A[8] - 1.0), 0.5 * A[5], 0.5 * A[2], 0.5 * A[1]};
    const double zero6[6] = {0, 0, 0, 0, 0, 0};
    double dep[6], Ct[21];
    ok = cp_update<double, F32START>(G, Gf, cp, Ew, zero6, T_guess, T, Ct, dep) && ok;
    // slip increments dt gdot_a(tau_a), tau_a = P_a . T
    double L[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    const CpScalars<double>& c = cp_scalars<double>(cp);
    for (int al = 0; al < 12; ++al) {
        double tau = 0.0;
#pragma unroll
        for (int m = 0; m < 6; ++m) tau += G.P[al][m] * T[m];
        const double x = fabs(tau) * c.inv_tc;
        double xn, xn1;
        cp_powers<double>(cp, x, xn, xn1);
        const double dg = tau < 0.0 ? -c.dtg * xn : c.dtg * xn;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) L[3 * i + j] += dg * G.sv[al][i] * G.nv[al][j];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Fp[3 * i + j] = L[3 * i] * Fp_old[j] + L[3 * i + 1] * Fp_old[3 + j] + L[3 * i + 2] * Fp_old[6 + j];
    double Fpi[9];
    ok = inv3(Fp, Fpi) && ok;
    const double r2h = 0.70710678118654752440084436210485;
    const double Tm[9] = {T[0], r2h * T[5], r2h * T[4], r2h * T[5], T[1], r2h * T[3], r2h * T[4], r2h * T[3], T[2]};
    double W1[9], W2[9];  // F Fp^-1, then (F Fp^-1) T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) W1[3 * i + j] = F[3 * i] * Fpi[j] + F[3 * i + 1] * Fpi[3 + j] + F[3 * i + 2] * Fpi[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) W2[3 * i + j] = W1[3 * i] * Tm[j] + W1[3 * i + 1] * Tm[3 + j] + W1[3 * i + 2] * Tm[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double v = W2[3 * i] * Fpi[3 * j] + W2[3 * i + 1] * Fpi[3 * j + 1] + W2[3 * i + 2] * Fpi[3 * j + 2];
            ok = ok && isfinite(v);
            P[3 * i + j] = v;
        }
    // tangent data: Fe_tr, a, B = a T a^T, C_tan
    double aT[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) aT[3 * i + j] = a[3 * i] * Tm[j] + a[3 * i + 1] * Tm[3 + j] + a[3 * i + 2] * Tm[6 + j];
    const int bi[6] = {0, 1, 2, 1, 0, 0}, bj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        tn[q] = Fe[q];
        tn[9 + q] = a[q];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
        tn[18 + q] = aT[3 * bi[q]] * a[3 * bj[q]] + aT[3 * bi[q] + 1] * a[3 * bj[q] + 1] + aT[3 * bi[q] + 2] * a[3 * bj[q] + 2];
#pragma unroll
    for (int q = 0; q < 21; ++q) tn[24 + q] = Ct[q];
    return ok;
}

}  // namespace dbfft
