// k_cpadj.cu -- per-voxel steps of the adjoint of the small-strain
// crystal-plasticity increments (R14 flow rule, Sec. 2.4 increments).
//
// For J = g : <sigma> after the last increment, s(x) a factor on the elastic
// stiffness of voxel x (derivative at s = 1), the reverse sweep over the
// increments n = N .. 1 keeps per voxel the state adjoint q (dJ / d eps_p of
// the increment's result) and uses the increment's converged stress sigma_n
// (its checkpoint), from which the consistent tangent
// T_n = (S + dt sum_a gdot'_a P_a P_a^T)^-1 follows. With a = g / N at the last
// increment (0 before), in Mandel components:
//   before the solve:  h = a - S q,  w = q + T_n h   (right-hand side B^H w);
//   after the solve K_n lam = B^H w, with e_lam = B lam:
//     d = h - e_lam,  dJ/ds += d . T_n S sigma_n + q . S sigma_n,  q = -T_n d.
#include <algorithm>

#include "launch.h"
#include "misc.h"

namespace dbfft {

namespace {

// T = (S + dt sum_a gdot'_a P_a P_a^T)^-1 at the stress s (21 packed entries);
// false when the Jacobian is not positive definite (T = 0 then).
__device__ __forceinline__ bool cp_tangent_at(const CpGrain& G, const CpParams& cp, const double (&s)[6],
                                              double (&T)[21]) {
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    double Rv[6], J[21], L[15], Di[6], unused;
    cp_eval<double, true, false>(G, cp, s, zero, Rv, J, unused);
    const bool spd = ldl6<double>(J, L, Di);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double e[6], col[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) e[i] = i == j ? 1.0 : 0.0;
        ldl6_solve<double>(L, Di, e, col);
#pragma unroll
        for (int i = 0; i <= j; ++i) T[sym6(i, j)] = spd ? col[i] : 0.0;
    }
    return spd;
}

// y = A x for a packed symmetric 6x6 A
__device__ __forceinline__ void sym_mv(const double* A, const double (&x)[6], double (&y)[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) acc += A[sym6(i, j)] * x[j];
        y[i] = acc;
    }
}

struct CpAdjArgs {
    int B, Rm;
    long long V;
    const uint16_t* phase;  // [Bm][V] grain ids
    const CpGrain* grains;
    CpParams cp;
    const double* sig;      // [B][V][6] checkpoint of the increment (Mandel)
    double* q;              // [B][V][6] state adjoint
    const double* a;        // [B][6] weight of sigma at this increment (g / N or 0)
    double* w;              // pre: out, the stress-like field w; post: in, e_lam = B lam
    double* tan;            // pre: out, T_n [B][V][21] (may be null)
    double* dJds;           // post: accumulated [B][V]
    unsigned* err;          // bit 0: a tangent that is not positive definite
    int write_w;            // pre: 0 = only the tangent
};

__global__ void k_cp_adj_pre(CpAdjArgs a) {
    const int b = blockIdx.y;
    const int mat = b / a.Rm;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.V; v += (long long)gridDim.x * blockDim.x) {
        const CpGrain& G = a.grains[a.phase[(long long)mat * a.V + v]];
        const long long o = (long long)b * a.V + v;
        double s[6], T[21];
#pragma unroll
        for (int i = 0; i < 6; ++i) s[i] = a.sig[o * 6 + i];
        if (!cp_tangent_at(G, a.cp, s, T) && a.err) atomicOr(a.err, 1u);
        if (a.tan) {
#pragma unroll
            for (int k = 0; k < 21; ++k) a.tan[o * 21 + k] = T[k];
        }
        if (!a.write_w) continue;
        double q[6], Sq[6], h[6], Th[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) q[i] = a.q[o * 6 + i];
        sym_mv(G.S, q, Sq);
#pragma unroll
        for (int i = 0; i < 6; ++i) h[i] = a.a[b * 6 + i] - Sq[i];
        sym_mv(T, h, Th);
#pragma unroll
        for (int i = 0; i < 6; ++i) a.w[o * 6 + i] = q[i] + Th[i];
    }
}

__global__ void k_cp_adj_post(CpAdjArgs a) {
    const int b = blockIdx.y;
    const int mat = b / a.Rm;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < a.V; v += (long long)gridDim.x * blockDim.x) {
        const CpGrain& G = a.grains[a.phase[(long long)mat * a.V + v]];
        const long long o = (long long)b * a.V + v;
        double s[6], T[21], q[6], Sq[6], d[6], Ss[6], sigs[6], qn[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            s[i] = a.sig[o * 6 + i];
            q[i] = a.q[o * 6 + i];
        }
        if (!cp_tangent_at(G, a.cp, s, T) && a.err) atomicOr(a.err, 1u);
        sym_mv(G.S, q, Sq);
        sym_mv(G.S, s, Ss);
#pragma unroll
        for (int i = 0; i < 6; ++i) d[i] = a.a[b * 6 + i] - Sq[i] - a.w[o * 6 + i];
        sym_mv(T, Ss, sigs);  // d sigma / d s at fixed strain and plastic strain
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) acc += d[i] * sigs[i] + q[i] * Ss[i];
        a.dJds[o] += acc;
        sym_mv(T, d, qn);
#pragma unroll
        for (int i = 0; i < 6; ++i) a.q[o * 6 + i] = -qn[i];
    }
}

dim3 grid_of(long long V, int B) {
    return dim3((unsigned)std::min<long long>((V + 255) / 256, 2048), (unsigned)B);
}

}  // namespace

cudaError_t launch_cp_adj(int post, int B, int Rm, long long V, const uint16_t* phase, const CpGrain* grains,
                          const CpParams& cp, const double* sig, double* q, const double* aw, double* w, double* tan,
                          double* dJds, unsigned* err, int write_w, cudaStream_t s) {
    CpAdjArgs a{B, Rm, V, phase, grains, cp, sig, q, aw, w, tan, dJds, err, write_w};
    if (post) k_cp_adj_post<<<grid_of(V, B), 256, 0, s>>>(a);
    else k_cp_adj_pre<<<grid_of(V, B), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dbfft
