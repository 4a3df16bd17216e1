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
//    consistent tangent (S + dt sum_a gdot'_a P_a P_a^T)^-1.
// The stress-side math runs in FP64.
#pragma once
#include <cuda_runtime.h>

namespace dbfft {

struct CpGrain {
    double S[21];     // Mandel compliance, upper triangle row-major
    double P[12][6];  // Schmid tensors sym(s x n), Mandel, sample frame
};

struct CpParams {
    double gdot0, inv_m, tau_c, dt, rtol;
    int max_it;
};

__host__ __device__ __forceinline__ int sym6(int i, int j) {
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

// Cholesky solve / inverse of a 6x6 SPD matrix (full storage).
__device__ __forceinline__ bool chol6(double (*A)[6], double (*L)[6]) {
    for (int j = 0; j < 6; ++j) {
        double s = A[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0)) return false;
        const double ljj = sqrt(s);
        L[j][j] = ljj;
        for (int i = j + 1; i < 6; ++i) {
            double t = A[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / ljj;
        }
    }
    return true;
}
__device__ __forceinline__ void chol6_solve(double (*L)[6], const double* b, double* x) {
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
        y[i] = t / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < 6; ++k) t -= L[k][i] * x[k];
        x[i] = t / L[i][i];
    }
}

struct CpEval {
    double R[6];
    double Jm[6][6];
};

__device__ __forceinline__ void cp_residual(const CpGrain& G, const CpParams& cp, const double* s,
                                            const double* target, double* R, double (*Jm)[6], double* gd_out) {
    for (int i = 0; i < 6; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 6; ++j) acc += G.S[sym6(i, j)] * s[j];
        R[i] = acc - target[i];
        if (Jm)
            for (int j = 0; j < 6; ++j) Jm[i][j] = G.S[sym6(i, j)];
    }
    for (int al = 0; al < 12; ++al) {
        double tau = 0.0;
        for (int j = 0; j < 6; ++j) tau += G.P[al][j] * s[j];
        const double x = fabs(tau) / cp.tau_c;
        const double pw = pow(x, cp.inv_m);
        const double gd = cp.gdot0 * pw * (tau > 0.0 ? 1.0 : (tau < 0.0 ? -1.0 : 0.0));
        if (gd_out) gd_out[al] = gd;
        for (int i = 0; i < 6; ++i) R[i] += cp.dt * gd * G.P[al][i];
        if (Jm) {
            const double dgd = cp.gdot0 * cp.inv_m / cp.tau_c * pow(x, cp.inv_m - 1.0);
            const double f = cp.dt * dgd;
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) Jm[i][j] += f * G.P[al][i] * G.P[al][j];
        }
    }
}

__device__ __forceinline__ double cp_potential(const CpGrain& G, const CpParams& cp, const double* s,
                                               const double* target) {
    double v = 0.0;
    for (int i = 0; i < 6; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 6; ++j) acc += G.S[sym6(i, j)] * s[j];
        v += 0.5 * s[i] * acc - s[i] * target[i];
    }
    const double m = 1.0 / cp.inv_m;
    const double k = cp.gdot0 * cp.tau_c * m / (1.0 + m);
    double pot = 0.0;
    for (int al = 0; al < 12; ++al) {
        double tau = 0.0;
        for (int j = 0; j < 6; ++j) tau += G.P[al][j] * s[j];
        pot += k * pow(fabs(tau) / cp.tau_c, 1.0 + cp.inv_m);
    }
    return v + cp.dt * pot;
}

// eps_w: total strain in W components (11,22,33,23,13,12); ep_old, s_guess,
// s_out, ep_new: Mandel; tan: 21-entry Mandel tangent. Returns false when
// the local Newton fails.
__device__ __forceinline__ bool cp_update(const CpGrain& G, const CpParams& cp, const double* eps_w,
                                          const double* ep_old, const double* s_guess, double* s_out,
                                          double* tan, double* ep_new) {
    const double r2 = 1.41421356237309504880168872420970;
    double target[6];
    const double em[6] = {eps_w[0], eps_w[1], eps_w[2], r2 * eps_w[3], r2 * eps_w[4], r2 * eps_w[5]};
    for (int i = 0; i < 6; ++i) target[i] = em[i] - ep_old[i];
    double s[6];
    for (int i = 0; i < 6; ++i) s[i] = s_guess[i];
    bool conv = false;
    double R[6], Jm[6][6], L[6][6], step[6];
    for (int it = 0; it < cp.max_it; ++it) {
        cp_residual(G, cp, s, target, R, Jm, nullptr);
        if (!chol6(Jm, L)) return false;
        double mR[6];
        for (int i = 0; i < 6; ++i) mR[i] = -R[i];
        chol6_solve(L, mR, step);
        double slope = 0.0, ns = 0.0, sn = 0.0;
        for (int i = 0; i < 6; ++i) {
            slope += R[i] * step[i];
            ns += step[i] * step[i];
            sn += s[i] * s[i];
        }
        const double scale = sqrt(sn) + cp.tau_c;
        ns = sqrt(ns);
        double t = 1.0;
        if (ns > 1e-3 * scale) {  // backtracking on the convex potential, far from the solution only
            const double f0 = cp_potential(G, cp, s, target);
            for (int ls = 0; ls < 60; ++ls) {
                double trial[6];
                for (int i = 0; i < 6; ++i) trial[i] = s[i] + t * step[i];
                if (!(cp_potential(G, cp, trial, target) > f0 + 1e-4 * t * slope + 1e-13 * fabs(f0))) break;
                t *= 0.5;
            }
        }
        for (int i = 0; i < 6; ++i) s[i] += t * step[i];
        if (ns <= cp.rtol * scale) { conv = true; break; }  // full Newton step below tolerance
    }
    double gd[12];
    cp_residual(G, cp, s, target, R, Jm, gd);
    if (!chol6(Jm, L)) return false;
    // tangent = Jm^-1 (symmetric), column by column
    for (int j = 0; j < 6; ++j) {
        double e[6] = {0, 0, 0, 0, 0, 0}, col[6];
        e[j] = 1.0;
        chol6_solve(L, e, col);
        for (int i = 0; i <= j; ++i) tan[sym6(i, j)] = col[i];
    }
    for (int i = 0; i < 6; ++i) {
        double acc = ep_old[i];
        for (int al = 0; al < 12; ++al) acc += cp.dt * gd[al] * G.P[al][i];
        ep_new[i] = acc;
    }
    for (int i = 0; i < 6; ++i) s_out[i] = s[i];
    return conv;
}

}  // namespace dbfft
