// noalloc.cu -- operator application that performs no device allocation.
//
// dbfft_apply_iso_noalloc runs the same five passes as dbfft_apply (FP64,
// small strain, linear isotropic phases, full strain control) without a
// context: the work buffer of the passes and the frequency / twiddle tables
// live in file-scope static device arrays, so the call itself never asks
// the CUDA runtime (or any allocator) for memory. Host code never dereferences
// those arrays: their device addresses are looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/dbfft.h"
#include "launch.h"

using namespace dbfft;

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // work buffer: 16 MiB
constexpr int kMaxLen = 256;                        // longest axis supported by the passes
constexpr int kMaxBatch = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) double g_xi[3 * kMaxLen];           // xi per axis
static __device__ __align__(256) cplx<double> g_tw[4 * kMaxLen];     // n1, n2, n3, n3/2 tables
static __device__ __align__(256) double g_zero_macro[kMaxBatch * 9];  // zero macro strain, never written

struct DeviceSymbols {
    bool ready = false;
    void* scratch = nullptr;
    double* xi = nullptr;
    cplx<double>* tw = nullptr;
    double* zero_macro = nullptr;
};
DeviceSymbols g_dev[kMaxDevices];
std::mutex g_mu;

// Device addresses of the static arrays for the current device, looked up the
// first time this device is used (with the device current).
dbfft_status symbols_for_current_device(DeviceSymbols** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DBFFT_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSymbols& s = g_dev[dev];
    if (!s.ready) {
        if (cudaGetSymbolAddress(&s.scratch, g_scratch) != cudaSuccess) return DBFFT_E_CUDA;
        if (cudaGetSymbolAddress(reinterpret_cast<void**>(&s.xi), g_xi) != cudaSuccess) return DBFFT_E_CUDA;
        if (cudaGetSymbolAddress(reinterpret_cast<void**>(&s.tw), g_tw) != cudaSuccess) return DBFFT_E_CUDA;
        if (cudaGetSymbolAddress(reinterpret_cast<void**>(&s.zero_macro), g_zero_macro) != cudaSuccess)
            return DBFFT_E_CUDA;
        s.ready = true;
    }
    *out = &s;
    return DBFFT_OK;
}

}  // namespace

extern "C" dbfft_status dbfft_apply_iso_noalloc(const int n[3], const double L[3], int batch,
                                                const uint16_t* phase_id, const double* lam, const double* mu,
                                                const void* u_hat, void* out, void* stream) {
    if (!n || !phase_id || !lam || !mu || !u_hat || !out || batch < 1) return DBFFT_E_ARG;
    for (int a = 0; a < 3; ++a)
        if (!supported_pow2(n[a])) return DBFFT_E_UNSUPPORTED_GRID;
    const int n1 = n[0], n2 = n[1], n3 = n[2], m = n3 / 2, h = m + 1;
    const long long H = (long long)n1 * n2 * h;
    const size_t need = (size_t)batch * 6 * (size_t)H * sizeof(cplx<double>);
    if (batch > kMaxBatch || need > kScratchBytes) {
        std::fprintf(stderr,
                     "dbfft_apply_iso_noalloc: batch * 6 * n1 * n2 * (n3/2+1) * 16 bytes = %zu exceeds the "
                     "static work buffer of %zu bytes (or batch > %d)\n",
                     need, kScratchBytes, kMaxBatch);
        return DBFFT_E_ARG;
    }
    if (u_hat == out) return DBFFT_E_ARG;
    DeviceSymbols* sym = nullptr;
    dbfft_status st = symbols_for_current_device(&sym);
    if (st != DBFFT_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // frequency and twiddle tables of this grid (host-built, copied into the static arrays)
    double xi[3 * kMaxLen];
    cplx<double> tw[4 * kMaxLen];
    const int lens[4] = {n1, n2, n3, m};
    for (int t = 0; t < 4; ++t)
        for (int k = 0; k < lens[t]; ++k) {
            const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)lens[t];
            tw[t * kMaxLen + k].x = (double)cosl(ang);
            tw[t * kMaxLen + k].y = (double)sinl(ang);
        }
    const int nax[3] = {n1, n2, n3};
    for (int ax = 0; ax < 3; ++ax) {
        const int len = nax[ax], cnt = ax == 2 ? h : len;
        const double Lx = (L && L[ax] > 0) ? L[ax] : 1.0;
        for (int k = 0; k < cnt; ++k) {
            const int kk = (k < (len + 1) / 2) ? k : k - len;
            xi[ax * kMaxLen + k] = (len % 2 == 0 && k == len / 2) ? 0.0
                                   : 2.0 * 3.14159265358979323846264338327950288 * (double)kk / Lx;
        }
    }
    if (cudaMemcpyAsync(sym->xi, xi, sizeof(xi), cudaMemcpyHostToDevice, s) != cudaSuccess) return DBFFT_E_CUDA;
    if (cudaMemcpyAsync(sym->tw, tw, sizeof(tw), cudaMemcpyHostToDevice, s) != cudaSuccess) return DBFFT_E_CUDA;

    Dims d{};
    d.n1 = n1; d.n2 = n2; d.n3 = n3; d.h = h; d.m = m;
    d.H = H; d.V = (long long)n1 * n2 * n3; d.plane = (long long)n2 * h;
    d.div_plane = make_fastdiv((unsigned)d.plane);
    d.div_h = make_fastdiv((unsigned)h);
    d.B = batch; d.Rm = 1; d.nc = 6; d.kin = KIN_SMALL; d.ne = 0;
    d.invN = 1.0 / (double)d.V;
    const Freq<double> f{sym->xi, sym->xi + kMaxLen, sym->xi + 2 * kMaxLen};
    const Twiddles<double> twd{sym->tw, sym->tw + kMaxLen, sym->tw + 2 * kMaxLen, sym->tw + 3 * kMaxLen};
    cplx<double>* W = reinterpret_cast<cplx<double>*>(sym->scratch);  // fully overwritten by pass 1

    Ax1InvArgs<double> a1{d, f, twd, reinterpret_cast<const cplx<double>*>(u_hat), nullptr, nullptr, W, nullptr, nullptr};
    Ax2Args<double> a2{d, twd, W, nullptr};
    if (launch_grad<double>(AX1_PLAIN, a1, s) != cudaSuccess) return DBFFT_E_CUDA;
    if (launch_fft_ax2<double>(+1, a2, s) != cudaSuccess) return DBFFT_E_CUDA;
    if (launch_fft_ax1<double>(+1, a2, s) != cudaSuccess) return DBFFT_E_CUDA;
    Ax3Args<double> a3{};
    a3.d = d;
    a3.tw = twd;
    a3.W = W;
    a3.RB = 1;
    a3.L = ax3_lines(n3, 6, 1, true);
    a3.macroW = sym->zero_macro;
    a3.phase = phase_id;
    a3.lam = lam;
    a3.mu = mu;
    if (launch_ax3<double>(OP_ISO, a3, s) != cudaSuccess) return DBFFT_E_CUDA;
    if (launch_fft_ax1<double>(-1, a2, s) != cudaSuccess) return DBFFT_E_CUDA;
    if (launch_fft_ax2<double>(-1, a2, s) != cudaSuccess) return DBFFT_E_CUDA;
    Ax1FwdArgs<double> a5{};
    a5.d = d;
    a5.f = f;
    a5.tw = twd;
    a5.W = W;
    a5.out = reinterpret_cast<cplx<double>*>(out);
    if (launch_div<double>(AX5_PLAIN, a5, s) != cudaSuccess) return DBFFT_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DBFFT_E_CUDA;
    return DBFFT_OK;
}
