// fft.cuh -- register-resident Stockham FFT building blocks for sm_103a.
//
// A length-N transform of one column is carried by P = N / R threads; each
// thread holds R complex values in registers. Stage s (radix R, span
// Ns = R^s) reads x[p + r P], twiddles by w_{Ns R}^{r (p mod Ns)}, does a
// radix-R DFT in registers and writes y[(p / Ns) Ns R + p mod Ns + q Ns]
// (the Stockham autosort schedule); consecutive stages exchange through
// shared memory. When log2 N is not a multiple of log2 R, the last stage uses
// a smaller radix and each thread does R / R_last of them. Before the first
// and after the last stage a thread holds the elements p + r P, r < R, so
// global loads and stores are strided the same way on both sides and a warp
// that spans consecutive columns touches contiguous memory.
//
// Twiddles come from a table tw[k] = exp(-2 pi i k / N) computed on the host
// in extended precision; radix-R butterflies use the constants cos/sin of
// 2 pi m / 32 written out below.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dbfft {

template <typename T> struct cplx { T x, y; };
template <typename T> struct vec2 {};
template <> struct vec2<float> { typedef float2 type; };
template <> struct vec2<double> { typedef double2 type; };

template <typename T> __device__ __forceinline__ cplx<T> mk(T a, T b) { cplx<T> c; c.x = a; c.y = b; return c; }
template <typename T> __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk(s * a.x, s * a.y); }
template <typename T> __device__ __forceinline__ cplx<T> conjg(cplx<T> a) { return mk(a.x, -a.y); }
// multiply by i * s (s real)
template <typename T> __device__ __forceinline__ cplx<T> mul_i(T s, cplx<T> a) { return mk(-s * a.y, s * a.x); }
// a * conj(w) when INV, else a * w  (w from the forward table)
template <int DIR, typename T> __device__ __forceinline__ cplx<T> twmul(cplx<T> a, cplx<T> w) {
    if (DIR > 0) w.y = -w.y;
    return a * w;
}

template <typename T> __device__ __forceinline__ cplx<T> ldc(const cplx<T>* p) {
    typename vec2<T>::type v = *reinterpret_cast<const typename vec2<T>::type*>(p);
    return mk<T>(v.x, v.y);
}
template <typename T> __device__ __forceinline__ void stc(cplx<T>* p, cplx<T> a) {
    typename vec2<T>::type v; v.x = a.x; v.y = a.y;
    *reinterpret_cast<typename vec2<T>::type*>(p) = v;
}
template <typename T> __device__ __forceinline__ cplx<T> ldg_c(const cplx<T>* p) {
    typename vec2<T>::type v = __ldg(reinterpret_cast<const typename vec2<T>::type*>(p));
    return mk<T>(v.x, v.y);
}

// Asynchronous global -> shared copy of one complex value (cp.async): the
// copies of a thread stay in flight together until cp_async_wait_all().
template <typename T>
__device__ __forceinline__ void cp_async_c(cplx<T>* smem_dst, const cplx<T>* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(T) == 4) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
    } else {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
    }
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// cos(2 pi m / 32) for m = 0..8 (first octant), mathematical constants.
__device__ __forceinline__ constexpr double c32(int m) {
    return m == 0 ? 1.0
         : m == 1 ? 0.98078528040323044912618223613424
         : m == 2 ? 0.92387953251128675612818318939679
         : m == 3 ? 0.83146961230254523707878837761791
         : m == 4 ? 0.70710678118654752440084436210485
         : m == 5 ? 0.55557023301960222474283081394853
         : m == 6 ? 0.38268343236508977172845998403040
         : m == 7 ? 0.19509032201612826784828486847702
         : 0.0;
}
// cos and sin of 2 pi m / 32 for any m in [0, 32)
__device__ __forceinline__ constexpr double cos32(int m) {
    return m <= 8 ? c32(m) : m <= 16 ? -c32(16 - m) : m <= 24 ? -c32(m - 16) : c32(32 - m);
}
__device__ __forceinline__ constexpr double sin32(int m) { return cos32((m + 24) & 31); }

// Multiply by exp(DIR * 2 pi i k / L) with k, L compile-time.
template <int DIR, int L, int K, typename T>
__device__ __forceinline__ cplx<T> rot(cplx<T> a) {
    constexpr int k = ((K % L) + L) % L;
    if constexpr (k == 0) {
        return a;
    } else if constexpr (4 * k == L) {  // * (DIR i)
        return DIR > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
    } else if constexpr (2 * k == L) {
        return mk(-a.x, -a.y);
    } else if constexpr (4 * k == 3 * L) {
        return DIR > 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
    } else {
        constexpr int m = k * (32 / L);
        const T c = (T)cos32(m);
        const T s = (T)(DIR * sin32(m));
        return mk(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

template <int N> struct ilog2 { static constexpr int value = 1 + ilog2<N / 2>::value; };
template <> struct ilog2<1> { static constexpr int value = 0; };

template <int R> __host__ __device__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1, rb = R >> 1; b < R; b <<= 1, rb >>= 1)
        if (i & b) r |= rb;
    return r;
}

// In-register DFT of length R (2..32), natural order in and out, on the
// elements v[OFF + STRIDE * r]. DIR = -1 forward, +1 inverse (unnormalised).
template <int R, int DIR, int STRIDE, int OFF, typename T>
struct RegDFT {
    template <int LEN, int I, int K>
    __device__ __forceinline__ static void bfly(cplx<T>* v) {
        constexpr int a = OFF + STRIDE * (I + K), b = OFF + STRIDE * (I + K + LEN / 2);
        cplx<T> t = rot<DIR, LEN, K>(v[b]);
        cplx<T> u = v[a];
        v[a] = u + t;
        v[b] = u - t;
    }
    template <int LEN, int I, int K>
    __device__ __forceinline__ static void inner(cplx<T>* v) {
        if constexpr (K < LEN / 2) {
            bfly<LEN, I, K>(v);
            inner<LEN, I, K + 1>(v);
        }
    }
    template <int LEN, int I>
    __device__ __forceinline__ static void groups(cplx<T>* v) {
        if constexpr (I < R) {
            inner<LEN, I, 0>(v);
            groups<LEN, I + LEN>(v);
        }
    }
    template <int LEN>
    __device__ __forceinline__ static void stages(cplx<T>* v) {
        if constexpr (LEN <= R) {
            groups<LEN, 0>(v);
            stages<LEN * 2>(v);
        }
    }
    template <int I>
    __device__ __forceinline__ static void perm(cplx<T>* v) {
        if constexpr (I < R) {
            constexpr int j = bitrev<R>(I);
            if constexpr (j > I) {
                cplx<T> t = v[OFF + STRIDE * I];
                v[OFF + STRIDE * I] = v[OFF + STRIDE * j];
                v[OFF + STRIDE * j] = t;
            }
            perm<I + 1>(v);
        }
    }
    __device__ __forceinline__ static void run(cplx<T>* v) {
        perm<0>(v);
        stages<2>(v);
    }
};

// Padded position of a contiguous (SS = 1) exchange buffer: one spare entry
// after every 128 bytes, so that the Stockham write pattern (stride R
// entries between neighbouring threads) spreads over the shared-memory banks.
template <typename T>
__host__ __device__ constexpr int pad_shift() { return sizeof(T) == 8 ? 3 : 4; }
template <typename T>
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> pad_shift<T>()) + 1; }

// Column FFT of length N with P = N / R threads per column.
//  v:   the thread's R registers, holding x[p + r P] on entry and X[p + r P]
//       on exit.
//  sm:  shared exchange buffer for this column: element i lives at
//       sm[i * SS] (SS = stride between positions) or, when PAD, at
//       sm[i + i / (128 bytes)] (SS must be 1 then; the buffer needs
//       padded_len(N) entries); it is only touched when there is more than
//       one stage.
//  tw:  twiddle table of length N (forward sign).
// Every thread of the block (of the warp, when WARP) must call this, including
// threads whose column is out of range.
template <typename T, int N, int R, int DIR, bool PAD = false, bool WARP = false>
struct ColFFT {
    static_assert(N >= R, "radix larger than the transform");
    static constexpr int P = N / R;
    static constexpr int LOGN = ilog2<N>::value;
    static constexpr int LOGR = ilog2<R>::value;
    static constexpr int NST = (LOGN + LOGR - 1) / LOGR;
    static constexpr int LASTR = 1 << (LOGN - (NST - 1) * LOGR);

    // WARP: the P threads of a column are one aligned group inside a warp, so
    // the exchange only needs the warp to agree.
    __device__ __forceinline__ static void sync() {
        if constexpr (WARP) __syncwarp();
        else __syncthreads();
    }
    __device__ __forceinline__ static int at(int i, int SS) {
        if constexpr (PAD) return i + (i >> pad_shift<T>());
        return i * SS;
    }
    template <int S, int NS>
    __device__ __forceinline__ static void stage(cplx<T>* v, cplx<T>* sm, int SS, int p, const cplx<T>* tw) {
        if constexpr (S < NST) {
            if constexpr (S == NST - 1 && LASTR != R) {
                // smaller last radix: sub-transform t uses v[t + rp (R/LASTR)]
                constexpr int G = R / LASTR;
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int jp = p + t * P;
#pragma unroll
                    for (int rp = 1; rp < LASTR; ++rp)
                        v[t + rp * G] = twmul<DIR>(v[t + rp * G], ldg_c(tw + (rp * jp) % N));
                }
                sub_dft<0, G>(v);
            } else {
                if constexpr (S > 0) {
                    const int k = p % NS;
#pragma unroll
                    for (int r = 1; r < R; ++r)
                        v[r] = twmul<DIR>(v[r], ldg_c(tw + r * k * (N / (NS * R))));
                }
                RegDFT<R, DIR, 1, 0, T>::run(v);
                if constexpr (S < NST - 1) {
                    const int base = (p / NS) * NS * R + (p % NS);
                    sync();
#pragma unroll
                    for (int q = 0; q < R; ++q) sm[at(base + q * NS, SS)] = v[q];
                    sync();
#pragma unroll
                    for (int r = 0; r < R; ++r) v[r] = sm[at(p + r * P, SS)];
                }
            }
            stage<S + 1, NS * R>(v, sm, SS, p, tw);
        }
    }
    template <int TI, int G>
    __device__ __forceinline__ static void sub_dft(cplx<T>* v) {
        if constexpr (TI < G) {
            RegDFT<LASTR, DIR, G, TI, T>::run(v);
            sub_dft<TI + 1, G>(v);
        }
    }
    __device__ __forceinline__ static void run(cplx<T>* v, cplx<T>* sm, int SS, int p, const cplx<T>* tw) {
        stage<0, 1>(v, sm, SS, p, tw);
    }
};

// Radix per pass, transform length and precision (host and device agree on it).
//  axis 1 (passes 1 and 5) and the half-length transform of axis 3 keep
//  their radix small so that several CTAs fit on an SM; axis 2 (a pure
//  transform) uses radix 16 in FP32 and 8 in FP64.
__host__ __device__ constexpr int radix_ax1(int n, bool dbl) { return dbl ? (n < 4 ? n : 4) : (n < 8 ? n : 8); }
__host__ __device__ constexpr int radix_ax2(int n, bool dbl) { return dbl ? (n < 8 ? n : 8) : (n < 16 ? n : 16); }
__host__ __device__ constexpr int radix_ax3(int m, bool dbl, int want = 8) {
    // want = 32: whole lines (m <= 32) or halves of lines per thread, in either precision
    return want == 32 ? (m < 32 ? m : 32) : dbl ? (m < 4 ? m : 4) : (m < want ? m : want);
}
template <typename T, int N> struct RadixAx1 { static constexpr int value = radix_ax1(N, sizeof(T) == 8); };
template <typename T, int M, int WANT> struct RadixAx3 { static constexpr int value = radix_ax3(M, sizeof(T) == 8, WANT); };
template <typename T, int N> struct RadixFor { static constexpr int value = radix_ax2(N, sizeof(T) == 8); };

}  // namespace dbfft
