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
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dbfft.h"
#include "launch.h"

using namespace dbfft;

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // work buffer: 16 MiB
constexpr int kMaxLen = 256;                        // longest axis supported by the passes
constexpr int kMaxBatch = 1024;
constexpr int kMaxDevices = 64;
constexpr int kPhaseTable = 65536;                  // one entry per uint16 phase id

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) double g_xi[3 * kMaxLen];           // xi per axis
static __device__ __align__(256) cplx<double> g_tw[4 * kMaxLen];     // n1, n2, n3, n3/2 tables
static __device__ __align__(256) double g_zero_macro[kMaxBatch * 9];  // zero macro strain, never written
// Lame constants indexed by phase id: every uint16 id reads inside the table,
// so an id at or beyond the caller's n_phases cannot read past an array; such
// ids are reported through g_bad_phase instead.
static __device__ __align__(256) double g_lam[kPhaseTable];
static __device__ __align__(256) double g_mu[kPhaseTable];
static __device__ __align__(16) unsigned g_bad_phase;

struct DeviceSymbols {
    bool ready = false;
    void* scratch = nullptr;
    double* xi = nullptr;
    cplx<double>* tw = nullptr;
    double* zero_macro = nullptr;
    double* lam = nullptr;
    double* mu = nullptr;
    unsigned* bad_phase = nullptr;
    // grid and box lengths whose tables are in g_xi / g_tw (n1 = 0: none yet)
    int tab_n[3] = {0, 0, 0};
    double tab_L[3] = {0.0, 0.0, 0.0};
};
DeviceSymbols g_dev[kMaxDevices];
std::mutex g_mu_lock;
thread_local std::string g_message;  // last failure of this thread's context-free calls

dbfft_status fail(dbfft_status st, const std::string& msg) {
    g_message = "dbfft_apply_iso_noalloc: " + msg;
    return st;
}

template <typename Sym>
bool symbol_address(void** p, const Sym& sym) {
    return cudaGetSymbolAddress(p, sym) == cudaSuccess;
}

// Device addresses of the static arrays for the current device, looked up the
// first time this device is used (with the device current).
dbfft_status symbols_for_current_device(DeviceSymbols** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(DBFFT_E_CUDA, "no usable device");
    std::lock_guard<std::mutex> lock(g_mu_lock);
    DeviceSymbols& s = g_dev[dev];
    if (!s.ready) {
        if (!symbol_address(&s.scratch, g_scratch) || !symbol_address(reinterpret_cast<void**>(&s.xi), g_xi) ||
            !symbol_address(reinterpret_cast<void**>(&s.tw), g_tw) ||
            !symbol_address(reinterpret_cast<void**>(&s.zero_macro), g_zero_macro) ||
            !symbol_address(reinterpret_cast<void**>(&s.lam), g_lam) ||
            !symbol_address(reinterpret_cast<void**>(&s.mu), g_mu) ||
            !symbol_address(reinterpret_cast<void**>(&s.bad_phase), g_bad_phase))
            return fail(DBFFT_E_CUDA, "cudaGetSymbolAddress failed");
        s.ready = true;
    }
    *out = &s;
    return DBFFT_OK;
}

// Flags phase ids at or beyond n_phases (the passes then read the static
// tables, whose entries past n_phases are stale but in bounds).
__global__ void k_check_phase(const uint16_t* __restrict__ phase, long long n, int n_phases, unsigned* bad) {
    bool any = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        any |= phase[i] >= n_phases;
    if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

}  // namespace

namespace dbfft {
const char* noalloc_last_error() { return g_message.c_str(); }
}  // namespace dbfft

extern "C" dbfft_status dbfft_apply_iso_noalloc(const int n[3], const double L[3], int batch,
                                                const uint16_t* phase_id, int n_phases, const double* lam,
                                                const double* mu, const void* u_hat, void* out, void* stream) {
    g_message.clear();
    if (!n || !phase_id || !lam || !mu || !u_hat || !out) return fail(DBFFT_E_ARG, "null pointer argument");
    if (batch < 1) return fail(DBFFT_E_ARG, "batch must be at least 1");
    if (n_phases < 1 || n_phases > kPhaseTable) return fail(DBFFT_E_ARG, "n_phases must lie in [1, 65536]");
    for (int a = 0; a < 3; ++a)
        if (!supported_pow2(n[a])) return fail(DBFFT_E_UNSUPPORTED_GRID, "grid lengths must be powers of two in [8, 256]");
    const int n1 = n[0], n2 = n[1], n3 = n[2], m = n3 / 2, h = m + 1;
    const long long H = (long long)n1 * n2 * h;
    const size_t need = (size_t)batch * 6 * (size_t)H * sizeof(cplx<double>);
    if (batch > kMaxBatch || need > kScratchBytes) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "batch * 6 * n1 * n2 * (n3/2+1) * 16 bytes = %zu exceeds the static work buffer of %zu bytes "
                      "(or batch > %d)",
                      need, kScratchBytes, kMaxBatch);
        return fail(DBFFT_E_ARG, buf);
    }
    if (u_hat == out) return fail(DBFFT_E_ARG, "out may not alias u_hat");
    double Lx[3];
    for (int ax = 0; ax < 3; ++ax) {
        Lx[ax] = L ? L[ax] : 1.0;
        if (!(Lx[ax] > 0.0) || !std::isfinite(Lx[ax])) return fail(DBFFT_E_ARG, "box lengths must be positive");
    }
    DeviceSymbols* sym = nullptr;
    dbfft_status st = symbols_for_current_device(&sym);
    if (st != DBFFT_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto cuda_fail = [&](const char* what) { return fail(DBFFT_E_CUDA, what); };

    // frequency and twiddle tables of this grid, host-built in extended
    // precision; uploaded only when the grid or the box differs from the last
    // upload on this device
    const bool same_tables = sym->tab_n[0] == n1 && sym->tab_n[1] == n2 && sym->tab_n[2] == n3 &&
                             sym->tab_L[0] == Lx[0] && sym->tab_L[1] == Lx[1] && sym->tab_L[2] == Lx[2];
    if (!same_tables) {
        double xi[3 * kMaxLen];
        cplx<double> tw[4 * kMaxLen];
        const int lens[4] = {n1, n2, n3, m};
        for (int t = 0; t < 4; ++t)
            for (int k = 0; k < lens[t]; ++k) {
                const long double ang =
                    -2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)lens[t];
                tw[t * kMaxLen + k].x = (double)cosl(ang);
                tw[t * kMaxLen + k].y = (double)sinl(ang);
            }
        const int nax[3] = {n1, n2, n3};
        for (int ax = 0; ax < 3; ++ax) {
            const int len = nax[ax], cnt = ax == 2 ? h : len;
            for (int k = 0; k < cnt; ++k) {
                const int kk = (k < (len + 1) / 2) ? k : k - len;
                xi[ax * kMaxLen + k] = (len % 2 == 0 && k == len / 2)
                                           ? 0.0
                                           : 2.0 * 3.14159265358979323846264338327950288 * (double)kk / Lx[ax];
            }
        }
        sym->tab_n[0] = 0;  // marked valid only once both copies are done
        if (cudaMemcpyAsync(sym->xi, xi, sizeof(xi), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(sym->tw, tw, sizeof(tw), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_fail("table upload failed");
        for (int ax = 0; ax < 3; ++ax) {
            sym->tab_n[ax] = nax[ax];
            sym->tab_L[ax] = Lx[ax];
        }
    }
    // the caller's Lame constants into the full-range phase tables, and the
    // phase-id check (its flag cleared first: the flag keeps the last call's value)
    const long long nvox = (long long)batch * n1 * n2 * n3;
    if (cudaMemcpyAsync(sym->lam, lam, (size_t)n_phases * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sym->mu, mu, (size_t)n_phases * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(sym->bad_phase, 0, sizeof(unsigned), s) != cudaSuccess)
        return cuda_fail("material table copy failed");
    {
        const long long blocks = std::min<long long>((nvox + 255) / 256, 2048);
        k_check_phase<<<(unsigned)blocks, 256, 0, s>>>(phase_id, nvox, n_phases, sym->bad_phase);
        if (cudaGetLastError() != cudaSuccess) return cuda_fail("phase check launch failed");
    }

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
    if (launch_grad<double>(AX1_PLAIN, a1, s) != cudaSuccess) return cuda_fail("pass 1 launch failed");
    if (launch_fft_ax2<double>(+1, a2, s) != cudaSuccess) return cuda_fail("axis-2 transform launch failed");
    if (launch_fft_ax1<double>(+1, a2, s) != cudaSuccess) return cuda_fail("axis-1 transform launch failed");
    Ax3Args<double> a3{};
    a3.d = d;
    a3.tw = twd;
    a3.W = W;
    a3.RB = 1;
    a3.L = ax3_lines(n3, 6, 1, true);
    a3.macroW = sym->zero_macro;
    a3.phase = phase_id;
    a3.lam = sym->lam;
    a3.mu = sym->mu;
    if (launch_ax3<double>(OP_ISO, a3, s) != cudaSuccess) return cuda_fail("pass 3 launch failed");
    if (launch_fft_ax1<double>(-1, a2, s) != cudaSuccess) return cuda_fail("axis-1 transform launch failed");
    if (launch_fft_ax2<double>(-1, a2, s) != cudaSuccess) return cuda_fail("axis-2 transform launch failed");
    Ax1FwdArgs<double> a5{};
    a5.d = d;
    a5.f = f;
    a5.tw = twd;
    a5.W = W;
    a5.out = reinterpret_cast<cplx<double>*>(out);
    if (launch_div<double>(AX5_PLAIN, a5, s) != cudaSuccess) return cuda_fail("pass 5 launch failed");
    // the call returns after the work is done, so that it can report the phase check
    unsigned bad = 0;
    if (cudaMemcpyAsync(&bad, sym->bad_phase, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_fail("stream synchronisation failed");
    if (bad) return fail(DBFFT_E_ARG, "a phase id is at or beyond n_phases; out is unspecified");
    return DBFFT_OK;
}
