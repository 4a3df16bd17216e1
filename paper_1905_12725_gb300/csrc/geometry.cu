// geometry.cu -- launch geometry of the passes (shared by host code).
#include "launch.h"
#include "pass3_pipe.cuh"

namespace dbfft {

thread_local bool g_pdl_launch = false;

bool supported_pow2(int n) { return n == 8 || n == 16 || n == 32 || n == 64 || n == 128 || n == 256; }
bool supported_odd(int n) {
#define DBFFT_ODD_CASE(N) case N:
    switch (n) {
        DBFFT_ODD_SIZES(DBFFT_ODD_CASE) return true;
        default: return false;
    }
#undef DBFFT_ODD_CASE
}
bool supported_odd_nl(int n) {
#define DBFFT_ODD_CASE(N) case N:
    switch (n) {
        DBFFT_ODD_NL_SIZES(DBFFT_ODD_CASE) return true;
        default: return false;
    }
#undef DBFFT_ODD_CASE
}
bool supported_len(int n) { return supported_pow2(n) || supported_odd(n); }
int ax3_odd_lines(int n3, int nc, bool dbl) {
    // ceil(nc/2) component pairs per line, two buffers of n3 complex values each,
    // at most 96 KB of shared memory and 256 / 8 threads' worth of pairs per CTA
    const int npl = (nc + 1) / 2;
    const long long per_line = (long long)npl * 2 * n3 * (dbl ? 16 : 8);
    long long L = (96LL * 1024) / per_line;
    if (L > 32 / npl) L = 32 / npl;
    if (L < 1) L = 1;
    return (int)L;
}

static int radix_for(int n, bool dbl) { return radix_ax2(n, dbl); }

long long pw_blocks(long long H, int B, int waves) {
    // about `waves` waves of blocks over the whole GPU, shared among the right-hand
    // sides: the element-wise kernels end with a block reduction, whose cost
    // is amortised over several frequencies per thread (grid-stride loops)
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            nsm < 1)
            nsm = 152;
    }
    const long long target = (long long)waves * 5 * nsm;  // ~5 resident 256-thread blocks per SM
    long long per = (target + (B > 0 ? B : 1) - 1) / (B > 0 ? B : 1);
    const long long need = (H + PW_THREADS - 1) / PW_THREADS;
    if (per > need) per = need;
    if (per < 1) per = 1;
    return per;
}

long long pw_blocks_resident(long long H, int B, int waves, int per_sm) {
    // whole waves: `waves` times the blocks that fit on the GPU at once (per_sm
    // resident blocks of the kernel on each SM), split evenly among the right-hand
    // sides and rounded down, so that no block starts a wave of its own
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            nsm < 1)
            nsm = 152;
    }
    const int b = B > 0 ? B : 1;
    long long per = (long long)waves * (per_sm > 0 ? per_sm : 1) * nsm / b;
    const long long need = (H + PW_THREADS - 1) / PW_THREADS;
    if (per > need) per = need;
    if (per < 1) per = 1;
    return per;
}

int ax2_tile(int n2, bool dbl) {
    const int P = n2 / radix_ax2(n2, dbl);
    int tw = 256 / P;
    if (tw < 8) tw = 8;
    if (tw > 256) tw = 256;
    return tw;
}

static int slot_bytes(int n3, bool dbl, int radix) {
    // mirrors ax3_slot_cplx<T, N3, RW>() in pass3.cuh
    const int m = n3 / 2;
    const int csz = dbl ? 16 : 8;
    const int r = radix_ax3(m, dbl, radix);
    if (r == m) {  // one thread per line: an odd number of words of the element size
        const int words = csz / 4;
        int n = m + 1;
        while (((n * words) & 31) != words) ++n;
        return n * csz;
    }
    const int pl = m + (m >> (dbl ? 3 : 4)) + 1;
    int n = pl > m + 1 ? pl : m + 1;
    while (((n * csz / 4) & 31) != 16) ++n;
    return n * csz;
}

int ax3_lines(int n3, int nc, int rb, bool dbl, int nfields, int radix) {
    // lines per CTA: real-space tiles within ~72 KB (three CTAs per SM), chosen
    // so that the slot FFT rounds (256 / P slots each) are well filled
    const size_t sb = (size_t)slot_bytes(n3, dbl, radix);
    long long Lmax = (long long)(72 * 1024) / ((long long)sb * rb * nc * nfields);
    if (Lmax < 1) Lmax = 1;
    if (Lmax > 32) Lmax = 32;
    const int m = n3 / 2;
    const int per_round = 256 / (m / radix_ax3(m, dbl, radix));
    int best = 1;
    double best_u = -1.0;
    for (int L = (int)Lmax; L >= 1; --L) {
        const int slots = L * rb * nc * nfields;
        const int rounds = (slots + per_round - 1) / per_round;
        const double u = (double)slots / (rounds * per_round);
        if (u > best_u + 0.02) {
            best_u = u;
            best = L;
        }
    }
    return best;
}

int ax3_threads_per_line(int n3, int nc, int rb, bool dbl) {
    const int m = n3 / 2;
    return (m / radix_ax3(m, dbl, 8)) * rb * nc;
}

size_t ax3_smem(int n3, int nc, int rb, int lines, bool dbl, bool two_fields) {
    return (size_t)lines * rb * nc * n3 * (dbl ? 8 : 4) * (two_fields ? 2 : 1);
}

}  // namespace dbfft

namespace dbfft {

namespace {
template <typename T, int N3>
long long pipe_smem_t(int nc, int rb, bool scale, int radix, int L, int nstage) {
    constexpr int M = N3 / 2;
    const int R = radix_ax3(M, sizeof(T) == 8, radix);
    const int P = M / R;
    return PipePlan<T, N3>::total_bytes(L, rb, nc, scale, P, 256 / 32, nstage);
}
template <typename T>
long long pipe_smem_n(int n3, int nc, int rb, bool scale, int radix, int L, int ns) {
    switch (n3) {
        case 8: return pipe_smem_t<T, 8>(nc, rb, scale, radix, L, ns);
        case 16: return pipe_smem_t<T, 16>(nc, rb, scale, radix, L, ns);
        case 32: return pipe_smem_t<T, 32>(nc, rb, scale, radix, L, ns);
        case 64: return pipe_smem_t<T, 64>(nc, rb, scale, radix, L, ns);
        case 128: return pipe_smem_t<T, 128>(nc, rb, scale, radix, L, ns);
        case 256: return pipe_smem_t<T, 256>(nc, rb, scale, radix, L, ns);
        default: return -1;
    }
}
}  // namespace

long long ax3_pipe_smem(int n3, int nc, int rb, bool dbl, bool scale, int radix, int L, long long nlines, int pipe) {
    if (L < 2 || (L & 1) || nlines % L != 0 || rb < 1 || rb > 8 || (pipe != 1 && pipe != 2)) return -1;
    const int ns = pipe == 2 ? 1 : 2;
    return dbl ? pipe_smem_n<double>(n3, nc, rb, scale, radix, L, ns) : pipe_smem_n<float>(n3, nc, rb, scale, radix, L, ns);
}

}  // namespace dbfft
