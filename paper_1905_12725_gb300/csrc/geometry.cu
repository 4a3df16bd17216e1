// geometry.cu -- launch geometry of the passes (shared by host code).
#include "launch.h"

namespace dbfft {

bool supported_len(int n) { return n == 8 || n == 16 || n == 32 || n == 64 || n == 128 || n == 256; }

static int radix_for(int n, bool dbl) { return dbl ? (n < 8 ? n : 8) : (n < 16 ? n : 16); }

int ax1_tile(int n1, bool dbl) {
    const int P = n1 / radix_for(n1, dbl);
    int tw = 256 / P;
    if (tw < 8) tw = 8;
    if (tw > 256) tw = 256;
    return tw;
}
int ax2_tile(int n2, bool dbl) { return ax1_tile(n2, dbl); }

int ax3_lines(int n3, int nc, int rb, bool dbl) {
    const int m = n3 / 2;
    const int P = m / radix_for(m, dbl);
    const int per_line = P * rb * nc;
    int L = 256 / per_line;
    if (L < 1) L = 1;
    while (L > 1 && ((per_line * L + 31) / 32) * 32 > 256) --L;
    // keep the real-space tiles within 96 KB
    const size_t per = (size_t)rb * nc * n3 * (dbl ? 8 : 4);
    while (L > 1 && per * L > 96 * 1024) --L;
    return L;
}

int ax3_threads_per_line(int n3, int nc, int rb, bool dbl) {
    const int m = n3 / 2;
    return (m / radix_for(m, dbl)) * rb * nc;
}

size_t ax3_smem(int n3, int nc, int rb, int lines, bool dbl, bool two_fields) {
    return (size_t)lines * rb * nc * n3 * (dbl ? 8 : 4) * (two_fields ? 2 : 1);
}

}  // namespace dbfft
