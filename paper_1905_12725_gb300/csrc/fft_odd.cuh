// fft_odd.cuh -- mixed-radix (3, 5, 7) Stockham FFTs in shared memory for odd
// transform lengths (the paper's odd grids, Sec. 2.1).
//
// A length-N column lives in shared memory (element i at buf[i * es]). Each
// stage of radix R (span Ns = product of the earlier radices) has N / R
// butterflies; butterfly j reads x[j + r N/R], twiddles by w_{Ns R}^{r (j mod
// Ns)}, does a radix-R DFT in registers and writes y[(j / Ns) Ns R + j mod Ns +
// q Ns] into the other buffer (self-sorting: natural order in and out). G
// threads share one column and loop over its butterflies. The radix-R DFT
// pairs x_r with x_{R-r}, so that each output needs (R-1)/2 real-by-complex
// products of each kind.
#pragma once
#include "fft.cuh"

#include <type_traits>

namespace dbfft {

// compile-time loop: f(std::integral_constant<int, i>) for i in [B, E)
template <int B, int E, typename F>
__device__ __forceinline__ void sfor_odd(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor_odd<B + 1, E>(f);
    }
}

// cos and sin of 2 pi m / R (R = 3, 5, 7; 1 <= m <= (R-1)/2), mathematical constants.
__host__ __device__ constexpr double cosR(int R, int m) {
    return R == 3 ? -0.5000000000000000000000000000000000
         : R == 5 ? (m == 1 ? 0.3090169943749474241022934171828191 : -0.8090169943749474241022934171828191)
         : (m == 1 ? 0.6234898018587335305250048840042398
            : m == 2 ? -0.2225209339563144042889025644967948 : -0.9009688679024191262361023195074451);
}
__host__ __device__ constexpr double sinR(int R, int m) {
    return R == 3 ? 0.8660254037844386467637231707529362
         : R == 5 ? (m == 1 ? 0.9510565162951535721164393333793821 : 0.5877852522924731291687059546390728)
         : (m == 1 ? 0.7818314824680298087084445266740578
            : m == 2 ? 0.9749279121818236070181316829939312 : 0.4338837391175581204757683328483588);
}

// y_q = sum_r x_r exp(SIGMA 2 pi i q r / R) in place, R odd (3, 5, 7).
template <int R, int SIGMA, typename T>
__device__ __forceinline__ void odd_dft(cplx<T> (&x)[R]) {
    constexpr int HR = (R - 1) / 2;
    cplx<T> a[HR], b[HR];
    cplx<T> y0 = x[0];
#pragma unroll
    for (int r = 1; r <= HR; ++r) {
        a[r - 1] = x[r] + x[R - r];
        b[r - 1] = x[r] - x[R - r];
        y0 = y0 + a[r - 1];
    }
    cplx<T> y[R];
    y[0] = y0;
    sfor_odd<1, HR + 1>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        cplx<T> c = x[0], s = mk(T(0), T(0));
        sfor_odd<1, HR + 1>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            constexpr int m0 = (q * r) % R;
            constexpr int m = m0 <= HR ? m0 : R - m0;        // cos(2 pi m0/R) = cos(2 pi m/R)
            constexpr double sg = m0 <= HR ? 1.0 : -1.0;      // sin(2 pi m0/R) = sg sin(2 pi m/R)
            const T cv = (T)cosR(R, m), sv = (T)(sg * sinR(R, m));
            c = c + cv * a[r - 1];
            s = s + sv * b[r - 1];
        });
        // y_q = c + SIGMA i s, y_{R-q} = c - SIGMA i s
        const cplx<T> is = SIGMA > 0 ? mk(-s.y, s.x) : mk(s.y, -s.x);
        y[q] = c + is;
        y[R - q] = c - is;
    });
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = y[q];
}

// Radices of the stages of an odd length: sevens, then fives, then threes.
__host__ __device__ constexpr int odd_radix(int N, int s) {
    int n = N, r = 1;
    for (int k = 0; k <= s; ++k) {
        r = (n % 7 == 0) ? 7 : (n % 5 == 0) ? 5 : (n % 3 == 0) ? 3 : 1;
        if (r == 1) return 1;
        n /= r;
    }
    return r;
}
__host__ __device__ constexpr int odd_stages(int N) {
    int s = 0;
    while (odd_radix(N, s) != 1) ++s;
    return s;
}
__host__ __device__ constexpr bool odd_len_ok(int N) {
    int n = N;
    while (n % 7 == 0) n /= 7;
    while (n % 5 == 0) n /= 5;
    while (n % 3 == 0) n /= 3;
    return N > 1 && (N & 1) && n == 1;
}

template <typename T, int N, int DIR>
struct OddFFT {
    static_assert(odd_len_ok(N), "odd lengths with prime factors 3, 5 and 7 only");
    static constexpr int NST = odd_stages(N);

    template <int S, int NS>
    __device__ __forceinline__ static cplx<T>* stage(cplx<T>* in, cplx<T>* out, int es, int p, int G,
                                                     const cplx<T>* tab) {
        if constexpr (S == NST) {
            return in;
        } else {
            constexpr int R = odd_radix(N, S);
            constexpr int NB = N / R;
            for (int j = p; j < NB; j += G) {
                const int k = j % NS;
                cplx<T> x[R];
#pragma unroll
                for (int r = 0; r < R; ++r) x[r] = in[(j + r * NB) * es];
                if constexpr (S > 0) {
#pragma unroll
                    for (int r = 1; r < R; ++r) x[r] = twmul<DIR>(x[r], ldg_c(tab + r * k * (N / (NS * R))));
                }
                odd_dft<R, DIR>(x);
                const int o = (j / NS) * NS * R + k;
#pragma unroll
                for (int q = 0; q < R; ++q) out[(o + q * NS) * es] = x[q];
            }
            __syncthreads();
            return stage<S + 1, NS * R>(out, in, es, p, G, tab);
        }
    }
    // Transform the column held in b0 (b1: scratch of the same size). Returns
    // the buffer that holds the result. Every thread of the block must call it
    // (it synchronises the block after each stage); tab is the forward twiddle
    // table of length N.
    __device__ __forceinline__ static cplx<T>* run(cplx<T>* b0, cplx<T>* b1, int es, int p, int G,
                                                   const cplx<T>* tab) {
        return stage<0, 1>(b0, b1, es, p, G, tab);
    }
};

}  // namespace dbfft
