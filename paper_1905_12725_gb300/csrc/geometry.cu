// geometry.cu -- launch geometry of the passes (shared by host code).
#include "launch.h"

namespace dbfft {

bool supported_len(int n) { return n == 8 || n == 16 || n == 32 || n == 64 || n == 128 || n == 256; }

static int radix_for(int n, bool dbl) { return radix_ax2(n, dbl); }

long long pw_blocks(long long H) {
    const long long nb = (H + PW_THREADS - 1) / PW_THREADS;
    return nb < 2048 ? nb : 2048;  // grid-stride loops beyond 2048 blocks per right-hand side
}

int ax2_tile(int n2, bool dbl) {
    const int P = n2 / radix_ax2(n2, dbl);
    int tw = 256 / P;
    if (tw < 8) tw = 8;
    if (tw > 256) tw = 256;
    return tw;
}

static int slot_bytes(int n3, bool dbl) {
    // mirrors ax3_slot_cplx<T, N3>() in pass3.cuh
    const int m = n3 / 2;
    const int csz = dbl ? 16 : 8;
    const int pl = m + (m >> (dbl ? 3 : 4)) + 1;
    int n = pl > m + 1 ? pl : m + 1;
    while (((n * csz / 4) & 31) != 16) ++n;
    return n * csz;
}

int ax3_lines(int n3, int nc, int rb, bool dbl, int nfields) {
    // real-space tiles of one CTA within ~56 KB so that four CTAs fit on an SM
    const size_t sb = (size_t)slot_bytes(n3, dbl);
    long long L = (long long)(56 * 1024) / ((long long)sb * rb * nc * nfields);
    if (L < 1) L = 1;
    if (L > 32) L = 32;
    return (int)L;
}

int ax3_threads_per_line(int n3, int nc, int rb, bool dbl) {
    const int m = n3 / 2;
    return (m / radix_ax3(m, dbl)) * rb * nc;
}

size_t ax3_smem(int n3, int nc, int rb, int lines, bool dbl, bool two_fields) {
    return (size_t)lines * rb * nc * n3 * (dbl ? 8 : 4) * (two_fields ? 2 : 1);
}

}  // namespace dbfft
