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

// FP32 complex sums and differences as one packed two-lane instruction each
// (Blackwell's float2 add): the butterflies' additions take half the issue
// slots. Round-to-nearest on each lane, the same results as two scalar adds.
__device__ __forceinline__ cplx<float> operator+(cplx<float> a, cplx<float> b) {
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return mk(r.x, r.y);
}
__device__ __forceinline__ cplx<float> operator-(cplx<float> a, cplx<float> b) {
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(-b.x, -b.y));
    return mk(r.x, r.y);
}
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

// cos(2 pi m / 256) for m = 0..64 (first quadrant), mathematical constants
// (34 decimals), for twiddles whose index is known at compile time.
__host__ __device__ constexpr double c256(int m) {
    switch (m) {
        case 0: return 1.0000000000000000000000000000000000;
        case 1: return 0.9996988186962042201157656496661722;
        case 2: return 0.9987954562051723927147716047591007;
        case 3: return 0.9972904566786902161355971401825678;
        case 4: return 0.9951847266721968862448369531094799;
        case 5: return 0.9924795345987099981567672516611178;
        case 6: return 0.9891765099647809734516737380162431;
        case 7: return 0.9852776423889412447740184331785478;
        case 8: return 0.9807852804032304491261822361342390;
        case 9: return 0.9757021300385285444603957664195280;
        case 10: return 0.9700312531945439926039842072861003;
        case 11: return 0.9637760657954398666864643555078352;
        case 12: return 0.9569403357322088649357978869802700;
        case 13: return 0.9495281805930366671959360741893450;
        case 14: return 0.9415440651830207784125094025995024;
        case 15: return 0.9329927988347388877116602555433025;
        case 16: return 0.9238795325112867561281831893967883;
        case 17: return 0.9142097557035306546350148293935774;
        case 18: return 0.9039892931234433315862002972305370;
        case 19: return 0.8932243011955153203424164474933980;
        case 20: return 0.8819212643483550297127568636603883;
        case 21: return 0.8700869911087114186522924044838488;
        case 22: return 0.8577286100002720699022699842847701;
        case 23: return 0.8448535652497070732595712051049571;
        case 24: return 0.8314696123025452370787883776179058;
        case 25: return 0.8175848131515836965049208841306338;
        case 26: return 0.8032075314806449098066765129631419;
        case 27: return 0.7883464276266062620091647053596893;
        case 28: return 0.7730104533627369608109066097584698;
        case 29: return 0.7572088465064845475754640536057845;
        case 30: return 0.7409511253549590911756168974951627;
        case 31: return 0.7242470829514669209410692432905532;
        case 32: return 0.7071067811865475244008443621048490;
        case 33: return 0.6895405447370669246167306299574847;
        case 34: return 0.6715589548470184006253768504274218;
        case 35: return 0.6531728429537767640842030136563054;
        case 36: return 0.6343932841636454982151716132254934;
        case 37: return 0.6152315905806268454849135634139843;
        case 38: return 0.5956993044924333434670365288299699;
        case 39: return 0.5758081914178453007459724538157308;
        case 40: return 0.5555702330196022247428308139485329;
        case 41: return 0.5349976198870972106630769046370179;
        case 42: return 0.5141027441932217265936938389688158;
        case 43: return 0.4928981922297840368730266887588093;
        case 44: return 0.4713967368259976485563876259052544;
        case 45: return 0.4496113296546066000462945794242271;
        case 46: return 0.4275550934302820943209668568887985;
        case 47: return 0.4052413140049898709084813055050525;
        case 48: return 0.3826834323650897717284599840303989;
        case 49: return 0.3598950365349881487751045723267564;
        case 50: return 0.3368898533922200506892532126191476;
        case 51: return 0.3136817403988914766564788459941003;
        case 52: return 0.2902846772544623676361923758173953;
        case 53: return 0.2667127574748983863252865151164364;
        case 54: return 0.2429801799032638899482741620774711;
        case 55: return 0.2191012401568697972277375474973578;
        case 56: return 0.1950903220161282678482848684770222;
        case 57: return 0.1709618887603012263636423572082635;
        case 58: return 0.1467304744553617516588501296467178;
        case 59: return 0.1224106751992161984987044741509458;
        case 60: return 0.0980171403295606019941955638886418;
        case 61: return 0.0735645635996674235294656215752343;
        case 62: return 0.0490676743274180142549549769426827;
        case 63: return 0.0245412285229122880317345294592829;
        default: return 0.0;  // m = 64
    }
}
// cos and sin of 2 pi m / 256 for any m in [0, 256)
__host__ __device__ constexpr double cos256(int m) {
    return m <= 64 ? c256(m) : m <= 128 ? -c256(128 - m) : m <= 192 ? -c256(m - 128) : c256(256 - m);
}
__host__ __device__ constexpr double sin256(int m) { return cos256((m + 192) & 255); }

// exp(-2 pi i K / N) as compile-time constants (N a power of two <= 256): the
// entry K of the forward twiddle table of length N.
template <typename T, int N, int K>
__device__ __forceinline__ cplx<T> tw_const() {
    static_assert(N <= 256 && 256 % N == 0, "twiddle constants cover lengths dividing 256");
    constexpr int m = ((K % N + N) % N) * (256 / N);
    return mk((T)cos256(m), (T)(-sin256(m)));
}

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
