// dbfft_dev.cuh -- device-side data structures shared by the pass kernels and
// the host driver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace dbfft {

enum { KIN_SMALL = 0, KIN_FINITE = 1 };

// Per-solve CG scalars (one per right-hand side), always FP64.
struct CgState {
    double rho;      // <r, M r>
    double alpha;    // rho / <p, K p>
    double beta;
    double bnorm2;   // ||b||^2 of this inner solve
    double rnorm2;   // ||r||^2 after the last update
    double pq;       // <p, K p>
    double tol2;     // stop when rnorm2 <= tol2 * bnorm2
    int iter;        // iterations done
    int done;        // 1: converged (or stopped); kernels skip this RHS
    int flags;       // bit 0: breakdown (non-positive curvature), bit 1: non-finite
    int max_iter;
};

// Preconditioner constants of one material group (Sec. 2.5, Eqs. pred2-pred3):
// Q(xi)_ik = sum_mono coef[ik][mono] mono(xi), with ik over (11,22,33,23,13,12)
// and mono over (x1^2, x2^2, x3^2, x2 x3, x1 x3, x1 x2); z = N Q^-1 r.
// Macro block: z_e = Me r_e with Me = (N Cbar_ee)^-1 on the active basis.
struct PrecondData {
    double coef[6][6];
    double Me[9][9];
    float coef_f[6][6];  // FP32 copy for the FP32 passes (no FP64 work per frequency)
    // isotropic mean tangent (lambda0, mu0): Q(xi) / |xi|^2 = mu0 I + (lambda0 + mu0) n n^T has the
    // closed-form inverse (I - c n n^T) / mu0 with c = (lambda0 + mu0) / (lambda0 + 2 mu0);
    // iso_d / iso_f hold 1 / mu0 and c
    int iso;
    double iso_d[2];
    float iso_f[2];
};

template <typename T>
__host__ __device__ __forceinline__ const T (*pcoef(const PrecondData& pd))[6] {
    if constexpr (sizeof(T) == 4) return pd.coef_f;
    else return pd.coef;
}
template <typename T>
__host__ __device__ __forceinline__ const T* piso(const PrecondData& pd) {
    if constexpr (sizeof(T) == 4) return pd.iso_f;
    else return pd.iso_d;
}

// Everything a pass needs about the grid and the macro basis.
// Division by a loop-invariant unsigned 32-bit divisor with one multiply-high
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994, round-up variant): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> s1)) >> s2 for
// t = mulhi(m, n), s1 = min(l, 1), s2 = max(l - 1, 0); exact for all n < 2^32.
struct FastDiv {
    unsigned d, m, s1, s2;
};

__host__ __device__ inline FastDiv make_fastdiv(unsigned d) {
    unsigned l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

__host__ __device__ __forceinline__ unsigned fastdiv(unsigned n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
    const unsigned t = __umulhi(f.m, n);
#else
    const unsigned t = (unsigned)(((unsigned long long)f.m * n) >> 32);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor finishes; it waits here,
// before touching anything the predecessor wrote (a no-op otherwise).
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
// Let the successor start launching (called once a block's main work is issued).
__device__ __forceinline__ void pdl_trigger() {
#if defined(__CUDA_ARCH__)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

struct Dims {
    int n1, n2, n3, h, m;   // h = n3/2 + 1, m = n3/2
    long long H;            // n1 n2 h
    long long V;            // n1 n2 n3
    long long plane;        // n2 h (one k1 plane of the half spectrum)
    int B;                  // right-hand sides
    int Rm;                 // right-hand sides per material map
    int nc;                 // 6 (small) or 9 (finite)
    int kin;
    int ne;                 // number of active macro unknowns
    int active[9];          // active macro basis indices (Mandel or 3i+j)
    double invN;
    FastDiv div_plane, div_h;  // half-spectrum index -> (k1, k2, k3); H < 2^32
};

template <typename T>
struct Freq {
    const T* xi1;  // [n1]
    const T* xi2;  // [n2]
    const T* xi3;  // [h]
};

template <typename T>
struct Twiddles {
    const cplx<T>* t1;  // [n1]
    const cplx<T>* t2;  // [n2]
    const cplx<T>* t3;  // [n3]  exp(-2 pi i k / n3)
    const cplx<T>* tm;  // [m]
};

}  // namespace dbfft
