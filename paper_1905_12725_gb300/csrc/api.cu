// api.cu -- host driver and C ABI of the DBFFT library (declared in dbfft.h).
//
// A context owns device buffers for one batch of right-hand sides. A solve
// (dbfft_solve_increment) runs an outer loop in FP64: the residual
// r = b - K x (or the Newton residual -B^H P(F) + macro rows) is formed by the
// FP64 pass chain with the constitutive update in pass 3, then an inner
// preconditioned CG (FP64, or FP32 for the MIXED precision mode) solves
// K d = r / ||r|| and x += ||r|| d in FP64. Linear problems in FP64 solve the
// inner system straight to the tolerance; MIXED is iterative refinement;
// nonlinear problems are Newton steps with an inexact inner solve
// (Sec. 2.4, Eqs. lineariz and nonlineqf).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dbfft.h"
#include "launch.h"
#include "misc.h"

using namespace dbfft;

namespace {

const double kPi = 3.14159265358979323846264338327950288;

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};


}  // namespace

struct dbfft_ctx {
    // ---- configuration
    dbfft_grid grid{};
    int n1 = 0, n2 = 0, n3 = 0, h = 0, m = 0;
    long long H = 0, V = 0;
    int B = 0, Bm = 0, Rm = 0, RB = 1;
    int kin = 0, nc = 6, prec = 0, model = 0;
    Dims dims{};
    unsigned stress_mask = 0;
    int activeflag_h[9] = {0};
    std::vector<double> target;  // [B][9]
    int n_inc = 1;
    double total_time = 1.0;
    int cur_inc = -1;
    cudaStream_t stream = nullptr;
    dbfft_allocator alloc{};
    bool use_cb = false;
    std::string err;
    size_t bytes = 0;
    std::vector<DevBuf> bufs;

    // ---- tables
    double* xi_d[3] = {nullptr, nullptr, nullptr};
    float* xi_f[3] = {nullptr, nullptr, nullptr};
    cplx<double>* tw_d[4] = {nullptr, nullptr, nullptr, nullptr};
    cplx<float>* tw_f[4] = {nullptr, nullptr, nullptr, nullptr};
    int* activeflag = nullptr;

    // ---- materials
    uint16_t* phase = nullptr;
    double* scale = nullptr;
    double* lam = nullptr;
    double* mu = nullptr;
    double* lam1 = nullptr;  // per unit Young's modulus (adjoint)
    double* mu1 = nullptr;
    float* lam_f = nullptr;  // FP32 copies for the FP32 passes
    float* mu_f = nullptr;
    float* scale_f = nullptr;
    std::vector<double> lam_h, mu_h, E_h;
    CpGrain* grains = nullptr;
    CpGrainF* grains_f = nullptr;
    int cp_guess_trial = 0;  // next CP update starts from the trial stress
    CpParams cp{};
    PrecondData* pre = nullptr;
    std::vector<PrecondData> pre_h;
    std::vector<PrecondData> pre_init_h;  // the preconditioner of the initial stiffness
    int pre_refresh = DBFFT_PRECOND_PER_INCREMENT;
    bool pre_is_init = true;  // the device holds pre_init_h
    long long wait_limit = 0;  // polls of the bulk-copy waits of pass 3 (0: the kernels' default)
    bool fwd_inc0 = false;     // x64 holds the converged solve of increment 0 (the adjoint reuses it)
    bool tangent_ready = false;  // x64 holds the six unit-strain solves of dbfft_homogenized_tangent
    std::vector<double> tangent_C;  // their C_eff [Bm][6][6]
    double* sens_tmp = nullptr;  // [B][V] per right-hand side sensitivity terms
    double* sens_G = nullptr;    // [Bm][6][6] weights on the device
    // checkpoints of the crystal-plasticity increments (the adjoint's forward record)
    bool ckpt_on = false;
    double* ckpt = nullptr;      // [n_inc][B][V][6] converged stress of each increment (Mandel)
    int ckpt_n = 0;              // increments 0 .. ckpt_n - 1 recorded
    double* adj_q = nullptr;     // [B][V][6] state adjoint
    double* adj_w = nullptr;     // [B][V][6] w, then B lam
    double* adj_a = nullptr;     // [B][6]

    // ---- vectors
    cplx<double>* x64 = nullptr;
    cplx<double>* r64 = nullptr;
    double* xe64 = nullptr;
    double* re64 = nullptr;
    void* xi = nullptr;  // inner precision
    void* ri = nullptr;
    void* pi = nullptr;
    double* xe_i = nullptr;
    double* re_i = nullptr;
    double* pe_i = nullptr;
    void* W = nullptr;   // [B][nc][H] sized for FP64
    void* W2 = nullptr;  // adjoint assembly
    cplx<double>* xfwd = nullptr;
    double* fU = nullptr;
    double* hbar = nullptr;  // [B][9] macro displacement gradient (displacement output)
    void* stage_h = nullptr;  // page-locked staging of the phase maps
    size_t stage_n = 0;
    char* small_cur = nullptr;  // small-object arena: next free byte and bytes left in the block
    size_t small_left = 0;
    double* sigf = nullptr;
    double* sig0 = nullptr;
    double* macroW = nullptr;
    double* macro_unit = nullptr;  // [Bm][9]: the unit strain e11 per material map (zero-fluctuation shortcut)
    float* macroWf = nullptr;  // FP32 copy read by the FP32 passes
    double* macroW2 = nullptr;
    double* scal = nullptr;  // [B] scale factors
    CgState* cg = nullptr;
    double* partials = nullptr;
    size_t partials_n = 0;
    unsigned* counters = nullptr;
    unsigned* errw = nullptr;

    // ---- nonlinear
    void* tan = nullptr;  // [B][V][ntan] inner precision
    int ntan = 0;
    double* eps_p = nullptr;
    double* sig_prev = nullptr;
    double* eps_p_t = nullptr;
    double* sig_t = nullptr;
    double* fp_c = nullptr;  // finite-strain CP: committed Fp [B][V][9]
    double* fp_t = nullptr;  // finite-strain CP: trial Fp [B][V][9]

    // ---- pinned host staging
    CgState* cg_h = nullptr;
    double* part_h = nullptr;
    double* small_h = nullptr;  // [B][9] + [B]

    bool have_solution = false;
    int nblk_max = 0;

    // ---- profiling: launch count and per-pass device time (CUDA events on the stream)
    long long launches = 0;
    bool prof = false;
    struct ProfRec {
        int slot;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<std::string> prof_name;
    std::vector<long long> prof_n;
    std::vector<double> prof_ms, prof_bytes;
    int active_b = 0;  // right-hand sides still iterating (bytes accounting)

    // ---- tuned launch shapes (0: built-in default), index 0 FP32 / 1 FP64
    int ax3_radix[2] = {8, 4};
    int ax3_L[2] = {0, 0};
    int fft_tw[2][2] = {{0, 0}, {0, 0}};  // [precision][axis 1, axis 2]
    // pipelined pass 3 for the CG applications: [precision] on/off, radix, lines per tile
    int pipe_on[2] = {0, 0}, pipe_R[2] = {8, 4}, pipe_L[2] = {0, 0};
    int lb_RB = 0;  // right-hand sides per CTA of the line-bulk pass (0: RB)
    std::string tune_note;

    // ---- inner PCG as one CUDA graph (WHILE node), per inner precision
    bool use_graphs = true;
    bool use_pdl = false;    // programmatic dependent launch inside the CG graph
    bool fuse_ax2 = false;   // FP32 CG: element-wise passes 1 and 5 fused into the axis-2 transforms
    bool graph_warm[2] = {false, false};
    cudaGraphExec_t cg_exec[2] = {nullptr, nullptr};
};

namespace {

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            ctx->err = std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " #call;          \
            return DBFFT_E_CUDA;                                                                     \
        }                                                                                            \
    } while (0)

#define TRY(expr)                                 \
    do {                                          \
        dbfft_status s_ = (expr);                 \
        if (s_ != DBFFT_OK) return s_;            \
    } while (0)

dbfft_status fail(dbfft_ctx* ctx, dbfft_status s, const std::string& msg) {
    ctx->err = msg;
    return s;
}

cudaEvent_t get_event(dbfft_ctx* ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int prof_slot(dbfft_ctx* ctx, const char* name) {
    for (size_t i = 0; i < ctx->prof_name.size(); ++i)
        if (ctx->prof_name[i] == name) return (int)i;
    ctx->prof_name.push_back(name);
    ctx->prof_n.push_back(0);
    ctx->prof_ms.push_back(0.0);
    ctx->prof_bytes.push_back(0.0);
    return (int)ctx->prof_name.size() - 1;
}

// Launch through f(), counting it; when profiling, bracket it with events.
// bytes: algorithmic DRAM bytes of this launch (reads + writes it must do).
template <class F>
dbfft_status run(dbfft_ctx* ctx, const char* name, double bytes, F&& f) {
    cudaEvent_t a = nullptr;
    if (ctx->prof) {
        a = get_event(ctx);
        CK(cudaEventRecord(a, ctx->stream));
    }
    CK(f());
    ctx->launches++;
    if (ctx->prof) {
        cudaEvent_t b = get_event(ctx);
        CK(cudaEventRecord(b, ctx->stream));
        ctx->pending.push_back({prof_slot(ctx, name), a, b, bytes});
    }
    return DBFFT_OK;
}

// Resolve pending event pairs (call after the stream has been synchronised).
void prof_flush(dbfft_ctx* ctx) {
    for (auto& r : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ctx->prof_ms[r.slot] += ms;
            ctx->prof_n[r.slot] += 1;
            ctx->prof_bytes[r.slot] += r.bytes;
        }
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->pending.clear();
    cudaGetLastError();
}

// Bytes of one component pass (one complex component over the half spectrum).
double cpass(const dbfft_ctx* ctx, bool dbl, int nb) { return (double)nb * ctx->H * (dbl ? 16.0 : 8.0); }

double mat_bytes(const dbfft_ctx* ctx, bool dbl, bool update) {
    const double V = (double)ctx->V;
    if (ctx->model == DBFFT_ISO_ELASTIC) return (double)ctx->Bm * V * (2.0 + (ctx->scale ? 8.0 : 0.0));
    const double t = dbl ? 8.0 : 4.0;
    if (!update) return (double)ctx->B * V * (2.0 + ctx->ntan * t);
    const double tw = ctx->prec == DBFFT_FP64 ? 8.0 : 4.0;
    if (ctx->model == DBFFT_CP_FCC_FINITE)  // Fp and T: read the committed, write the trial
        return (double)ctx->B * V * (2.0 + ctx->ntan * tw + 2 * (9 + 6) * 8.0);
    if (ctx->model != DBFFT_CP_FCC_POWERLAW) return (double)ctx->B * V * (2.0 + ctx->ntan * tw);
    return (double)ctx->B * V * (2.0 + ctx->ntan * tw + 4 * 6 * 8.0);
}

// Pinned host buffers (CG state, partial sums) outlive their context in a
// process-wide cache keyed by size: page-locking memory costs far more than a
// context's whole set-up, and repeated contexts of one problem reuse the same
// sizes. At most kPinnedCacheBytes stay cached.
constexpr size_t kPinnedCacheBytes = 64u << 20;
std::mutex g_pinned_mu;
std::multimap<size_t, void*> g_pinned_free;
size_t g_pinned_cached = 0;

void* pinned_alloc(size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(g_pinned_mu);
        auto it = g_pinned_free.find(bytes);
        if (it != g_pinned_free.end()) {
            void* p = it->second;
            g_pinned_free.erase(it);
            g_pinned_cached -= bytes;
            return p;
        }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_free(void* p, size_t bytes) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_pinned_mu);
        if (g_pinned_cached + bytes <= kPinnedCacheBytes) {
            g_pinned_free.emplace(bytes, p);
            g_pinned_cached += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

constexpr size_t kSmallMax = 64 * 1024;     // requests up to this size ...
constexpr size_t kSmallBlock = 1024 * 1024;  // ... are carved from blocks of this size

dbfft_status dalloc_raw(dbfft_ctx* ctx, size_t bytes, void** out);

dbfft_status dalloc(dbfft_ctx* ctx, size_t bytes, void** out) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes <= kSmallMax) {  // the many small tables of a context share a few allocations
        if (ctx->small_left < bytes) {
            void* blk = nullptr;
            TRY(dalloc_raw(ctx, kSmallBlock, &blk));
            ctx->small_cur = static_cast<char*>(blk);
            ctx->small_left = kSmallBlock;
        }
        *out = ctx->small_cur;
        ctx->small_cur += bytes;
        ctx->small_left -= bytes;
        return DBFFT_OK;
    }
    return dalloc_raw(ctx, bytes, out);
}

dbfft_status dalloc_raw(dbfft_ctx* ctx, size_t bytes, void** out) {
    void* p = nullptr;
    if (ctx->use_cb) {
        p = ctx->alloc.alloc(bytes, ctx->alloc.user);
        if (!p) return fail(ctx, DBFFT_E_NOMEM, "allocator callback returned NULL");
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, DBFFT_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        }
    }
    ctx->bufs.push_back(DevBuf{p, bytes});
    ctx->bytes += bytes;
    *out = p;
    return DBFFT_OK;
}

template <typename P>
dbfft_status dalloc_t(dbfft_ctx* ctx, size_t count, P** out) {
    void* p = nullptr;
    TRY(dalloc(ctx, count * sizeof(P), &p));
    *out = reinterpret_cast<P*>(p);
    return DBFFT_OK;
}

// ---------------------------------------------------------------- host math
void iso_C(double lam, double mu, double C[3][3][3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    C[i][j][k][l] = lam * (i == j) * (k == l) + mu * ((i == k) * (j == l) + (i == l) * (j == k));
}

// Macro basis tensor m (Mandel for small strain, e_i x e_j for finite).
void basis_tensor(int nc, int m, double T[3][3]) {
    std::memset(T, 0, sizeof(double) * 9);
    if (nc == 9) {
        T[m / 3][m % 3] = 1.0;
        return;
    }
    static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
    if (m < 3) {
        T[m][m] = 1.0;
    } else {
        T[pi[m]][pj[m]] = T[pj[m]][pi[m]] = 1.0 / std::sqrt(2.0);
    }
}

bool invert(int n, std::vector<double>& A) {  // Gauss-Jordan with partial pivoting, row-major n x n
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        for (int k = 0; k < n; ++k) {
            std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(I[c * n + k], I[piv * n + k]);
        }
        const double d = A[c * n + c];
        for (int k = 0; k < n; ++k) {
            A[c * n + k] /= d;
            I[c * n + k] /= d;
        }
        for (int r = 0; r < n; ++r)
            if (r != c) {
                const double f = A[r * n + c];
                if (f != 0.0)
                    for (int k = 0; k < n; ++k) {
                        A[r * n + k] -= f * A[c * n + k];
                        I[r * n + k] -= f * I[c * n + k];
                    }
            }
    }
    A = I;
    return true;
}

// Preconditioner constants from a mean fourth-order tangent (Sec. 2.5):
// Q_ik(xi) = sum_jl xi_j Cbar_ijkl xi_l written on the six monomials, and the
// macro block (N Cbar_ee)^-1 on the active basis (R4 reading of M(0)).
bool precond_from(const dbfft_ctx* ctx, const double C[3][3][3][3], PrecondData& pd) {
    std::memset(&pd, 0, sizeof(pd));
    static const int ik[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
    static const int jl[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            const int i = ik[a][0], k = ik[a][1], j = jl[b][0], l = jl[b][1];
            pd.coef[a][b] = (j == l) ? C[i][j][k][j] : (C[i][j][k][l] + C[i][l][k][j]);
            pd.coef_f[a][b] = (float)pd.coef[a][b];
        }
    {  // an isotropic mean tangent (to rounding) takes the closed-form inverse
        const double lam = C[0][0][1][1], mu = C[0][1][0][1];
        double cmax = 0.0, dev = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        const double iso = lam * (i == j && k == l) + mu * ((i == k && j == l) + (i == l && j == k));
                        cmax = std::max(cmax, std::fabs(C[i][j][k][l]));
                        dev = std::max(dev, std::fabs(C[i][j][k][l] - iso));
                    }
        if (mu > 0.0 && lam + 2.0 * mu > 0.0 && dev <= 1e-13 * cmax) {
            pd.iso = 1;
            pd.iso_d[0] = 1.0 / mu;
            pd.iso_d[1] = (lam + mu) / (lam + 2.0 * mu);
            pd.iso_f[0] = (float)pd.iso_d[0];
            pd.iso_f[1] = (float)pd.iso_d[1];
        }
    }
    const int ne = ctx->dims.ne;
    if (ne > 0) {
        std::vector<double> A(ne * ne);
        const double N = (double)ctx->V;
        for (int p = 0; p < ne; ++p)
            for (int q = 0; q < ne; ++q) {
                double Tp[3][3], Tq[3][3];
                basis_tensor(ctx->nc, ctx->dims.active[p], Tp);
                basis_tensor(ctx->nc, ctx->dims.active[q], Tq);
                double s = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        for (int k = 0; k < 3; ++k)
                            for (int l = 0; l < 3; ++l) s += Tp[i][j] * C[i][j][k][l] * Tq[k][l];
                A[p * ne + q] = N * s;
            }
        if (!invert(ne, A)) return false;
        for (int p = 0; p < ne; ++p)
            for (int q = 0; q < ne; ++q) pd.Me[p][q] = A[p * ne + q];
    }
    return true;
}

void quat_rot(const double* q0, double R[3][3]) {
    double n = std::sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
    const double w = q0[0] / n, x = q0[1] / n, y = q0[2] / n, z = q0[3] / n;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

void to_mandel(const double C[3][3][3][3], double Cm[6][6]) {
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
            double Ta[3][3], Tb[3][3];
            basis_tensor(6, a, Ta);
            basis_tensor(6, b, Tb);
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) s += Ta[i][j] * C[i][j][k][l] * Tb[k][l];
            Cm[a][b] = s;
        }
}

// Crystal data of one grain: Mandel compliance of the rotated cubic
// stiffness and the Schmid tensors of the 12 {111}<110> systems.
bool cp_grain(const dbfft_phase& ph, CpGrain& g) {
    static const double planes[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
    static const double dirs[4][3][3] = {{{0, 1, -1}, {1, 0, -1}, {1, -1, 0}},
                                         {{0, 1, -1}, {1, 0, 1}, {1, 1, 0}},
                                         {{0, 1, 1}, {1, 0, -1}, {1, 1, 0}},
                                         {{0, 1, 1}, {1, 0, 1}, {1, -1, 0}}};
    double R[3][3];
    quat_rot(ph.quat, R);
    double Cc[3][3][3][3], Cg[3][3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double v = 0.0;
                    if (i == j && k == l) v = (i == k) ? ph.C11 : ph.C12;
                    else if ((i == k && j == l) || (i == l && j == k)) v = ph.C44;
                    Cc[i][j][k][l] = v;
                }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double s = 0.0;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            for (int c = 0; c < 3; ++c)
                                for (int d = 0; d < 3; ++d)
                                    s += R[i][a] * R[j][b] * R[k][c] * R[l][d] * Cc[a][b][c][d];
                    Cg[i][j][k][l] = s;
                }
    double Cm[6][6];
    to_mandel(Cg, Cm);
    std::vector<double> A(36);
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) A[a * 6 + b] = Cm[a][b];
    if (!invert(6, A)) return false;
    for (int a = 0; a < 6; ++a)
        for (int b = a; b < 6; ++b) g.S[sym6(a, b)] = 0.5 * (A[a * 6 + b] + A[b * 6 + a]);
    for (int p = 0; p < 4; ++p)
        for (int dd = 0; dd < 3; ++dd) {
            double n[3], s[3], nr[3] = {0, 0, 0}, sr[3] = {0, 0, 0};
            for (int i = 0; i < 3; ++i) {
                n[i] = planes[p][i] / std::sqrt(3.0);
                s[i] = dirs[p][dd][i] / std::sqrt(2.0);
            }
            for (int i = 0; i < 3; ++i)
                for (int k = 0; k < 3; ++k) {
                    nr[i] += R[i][k] * n[k];
                    sr[i] += R[i][k] * s[k];
                }
            for (int i = 0; i < 3; ++i) {
                g.sv[p * 3 + dd][i] = sr[i];
                g.nv[p * 3 + dd][i] = nr[i];
            }
            double Pt[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Pt[i][j] = 0.5 * (sr[i] * nr[j] + nr[i] * sr[j]);
            for (int mm = 0; mm < 6; ++mm) {
                double Tm[3][3];
                basis_tensor(6, mm, Tm);
                double v = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) v += Tm[i][j] * Pt[i][j];
                g.P[p * 3 + dd][mm] = v;
            }
        }
    return true;
}

// ---------------------------------------------------------------- tables
template <typename T>
Freq<T> freq(dbfft_ctx* ctx);
template <>
Freq<double> freq<double>(dbfft_ctx* ctx) { return Freq<double>{ctx->xi_d[0], ctx->xi_d[1], ctx->xi_d[2]}; }
template <>
Freq<float> freq<float>(dbfft_ctx* ctx) { return Freq<float>{ctx->xi_f[0], ctx->xi_f[1], ctx->xi_f[2]}; }
template <typename T>
Twiddles<T> twid(dbfft_ctx* ctx);
template <>
Twiddles<double> twid<double>(dbfft_ctx* ctx) {
    return Twiddles<double>{ctx->tw_d[0], ctx->tw_d[1], ctx->tw_d[2], ctx->tw_d[3]};
}
template <>
Twiddles<float> twid<float>(dbfft_ctx* ctx) {
    return Twiddles<float>{ctx->tw_f[0], ctx->tw_f[1], ctx->tw_f[2], ctx->tw_f[3]};
}

dbfft_status upload_tables(dbfft_ctx* ctx) {
    // All tables go to the device in one copy: host staging with 256-byte aligned
    // offsets, one device block, pointers into it.
    std::vector<unsigned char> host;
    auto place = [&](size_t bytes) {
        const size_t off = (host.size() + 255) & ~(size_t)255;
        host.resize(off + bytes);
        return off;
    };
    // twiddles exp(-2 pi i k / n) per axis; tm: the half-length transform of an even
    // axis 3 (unused for odd n3)
    const int lens[4] = {ctx->n1, ctx->n2, ctx->n3, ctx->n3 % 2 == 0 ? ctx->m : 1};
    size_t off_td[4], off_tf[4], off_xd[3], off_xf[3];
    for (int t = 0; t < 4; ++t) {
        off_td[t] = place(lens[t] * sizeof(cplx<double>));
        off_tf[t] = place(lens[t] * sizeof(cplx<float>));
    }
    // frequencies xi_i = 2 pi k_i / L_i in FFT order, Nyquist index set to 0
    const int nax[3] = {ctx->n1, ctx->n2, ctx->n3};
    int cnts[3];
    for (int ax = 0; ax < 3; ++ax) {
        cnts[ax] = (ax == 2) ? ctx->h : nax[ax];
        off_xd[ax] = place(cnts[ax] * sizeof(double));
        off_xf[ax] = place(cnts[ax] * sizeof(float));
    }
    for (int t = 0; t < 4; ++t) {
        const int n = lens[t];
        cplx<double>* td = reinterpret_cast<cplx<double>*>(host.data() + off_td[t]);
        cplx<float>* tf = reinterpret_cast<cplx<float>*>(host.data() + off_tf[t]);
        for (int k = 0; k < n; ++k) {
            const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)k / (long double)n;
            td[k].x = (double)cosl(ang);
            td[k].y = (double)sinl(ang);
            tf[k].x = (float)td[k].x;
            tf[k].y = (float)td[k].y;
        }
    }
    for (int ax = 0; ax < 3; ++ax) {
        const int n = nax[ax];
        const double L = ctx->grid.L[ax] > 0 ? ctx->grid.L[ax] : 1.0;
        double* xd = reinterpret_cast<double*>(host.data() + off_xd[ax]);
        float* xf = reinterpret_cast<float*>(host.data() + off_xf[ax]);
        for (int k = 0; k < cnts[ax]; ++k) {
            const int kk = (k < (n + 1) / 2) ? k : k - n;
            double v = 2.0 * kPi * (double)kk / L;
            if (n % 2 == 0 && (k == n / 2)) v = 0.0;
            xd[k] = v;
            xf[k] = (float)v;
        }
    }
    void* blk = nullptr;
    TRY(dalloc(ctx, host.size(), &blk));
    unsigned char* dev = static_cast<unsigned char*>(blk);
    for (int t = 0; t < 4; ++t) {
        ctx->tw_d[t] = reinterpret_cast<cplx<double>*>(dev + off_td[t]);
        ctx->tw_f[t] = reinterpret_cast<cplx<float>*>(dev + off_tf[t]);
    }
    for (int ax = 0; ax < 3; ++ax) {
        ctx->xi_d[ax] = reinterpret_cast<double*>(dev + off_xd[ax]);
        ctx->xi_f[ax] = reinterpret_cast<float*>(dev + off_xf[ax]);
    }
    CK(cudaMemcpyAsync(blk, host.data(), host.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DBFFT_OK;
}

// ---------------------------------------------------------------- load
// Prescribed macro field (W components) and stress targets (macro basis) of
// increment inc: fraction (inc+1)/n of the ramp from 0 (small) / I (finite).
dbfft_status set_load(dbfft_ctx* ctx, int inc, const double* tgt /* [B][9] */) {
    const double f = (double)(inc + 1) / (double)ctx->n_inc;
    std::vector<double> fU(ctx->B * 9, 0.0), sf(ctx->B * 9, 0.0);
    static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
    for (int b = 0; b < ctx->B; ++b) {
        const double* t = tgt + b * 9;
        if (ctx->nc == 6) {
            for (int mm = 0; mm < 6; ++mm) {
                const double sym = 0.5 * (t[3 * pi[mm] + pj[mm]] + t[3 * pj[mm] + pi[mm]]);
                if (ctx->activeflag_h[mm]) sf[b * 9 + mm] = f * sym * (mm >= 3 ? std::sqrt(2.0) : 1.0);
                else fU[b * 9 + mm] = f * sym;
            }
        } else {
            for (int q = 0; q < 9; ++q) {
                const double id = (q / 3 == q % 3) ? 1.0 : 0.0;
                if (ctx->activeflag_h[q]) {
                    sf[b * 9 + q] = f * t[q];
                    fU[b * 9 + q] = id;
                } else {
                    fU[b * 9 + q] = id + f * (t[q] - id);
                }
            }
        }
    }
    CK(cudaMemcpyAsync(ctx->fU, fU.data(), fU.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sigf, sf.data(), sf.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DBFFT_OK;
}

// ---------------------------------------------------------------- chains
template <typename T>
Dims dims_of(dbfft_ctx* ctx) { return ctx->dims; }

int opk_apply(const dbfft_ctx* ctx) {
    switch (ctx->model) {
        case DBFFT_ISO_ELASTIC: return OP_ISO;
        case DBFFT_NEO_HOOKE: return OP_NH_APPLY;
        case DBFFT_SVK: return OP_SVK_APPLY;
        case DBFFT_CP_FCC_FINITE: return OP_FCP_APPLY;
        default: return OP_CP_APPLY;
    }
}
int opk_update(const dbfft_ctx* ctx) {
    if (ctx->model == DBFFT_CP_FCC_POWERLAW) return ctx->prec == DBFFT_MIXED ? OP_CP_UPDATE32 : OP_CP_UPDATE;
    if (ctx->model == DBFFT_SVK) return OP_SVK_UPDATE;
    if (ctx->model == DBFFT_CP_FCC_FINITE) return ctx->prec == DBFFT_MIXED ? OP_FCP_UPDATE32 : OP_FCP_UPDATE;
    return ctx->model == DBFFT_ISO_ELASTIC ? OP_ISO : OP_NH_UPDATE;
}

template <typename T>
Ax2Args<T> fft_args(dbfft_ctx* ctx, cplx<T>* W, const CgState* cg) {
    Ax2Args<T> a;
    std::memset(&a, 0, sizeof(a));
    a.d = ctx->dims;
    a.tw = twid<T>(ctx);
    a.W = W;
    a.cg = cg;
    const int pi_ = sizeof(T) == 8 ? 1 : 0;
    a.tw_ax1 = ctx->fft_tw[pi_][0];
    a.tw_ax2 = ctx->fft_tw[pi_][1];
    return a;
}

template <typename T>
Ax3Args<T> ax3_base(dbfft_ctx* ctx, cplx<T>* W) {
    Ax3Args<T> a;
    std::memset(&a, 0, sizeof(a));
    a.d = ctx->dims;
    a.tw = twid<T>(ctx);
    a.W = W;
    a.RB = ctx->RB;
    const int pi_ = sizeof(T) == 8 ? 1 : 0;
    a.radix = ctx->ax3_radix[pi_];
    a.L = ctx->ax3_L[pi_] > 0 ? ctx->ax3_L[pi_] : ax3_lines(ctx->n3, ctx->nc, ctx->RB, sizeof(T) == 8, 1, a.radix);
    a.phase = ctx->phase;
    if constexpr (sizeof(T) == 4) {
        a.scale = ctx->scale_f;
        a.lam = ctx->lam_f;
        a.mu = ctx->mu_f;
    } else {
        a.scale = ctx->scale;
        a.lam = ctx->lam;
        a.mu = ctx->mu;
    }
    a.grains = ctx->grains;
    a.grains_f = ctx->grains_f;
    a.cp = ctx->cp;
    a.err = ctx->errw;
    a.wait_limit = ctx->wait_limit;
    return a;
}

// Launch shape of the CG applications of pass 3 (the pipelined kernel when tuned in).
template <typename T>
void apply_shape(const dbfft_ctx* ctx, Ax3Args<T>& a) {
    const int pi_ = sizeof(T) == 8 ? 1 : 0;
    if (ctx->pipe_on[pi_]) {
        a.pipe = ctx->pipe_on[pi_];
        a.radix = ctx->pipe_R[pi_];
        a.L = ctx->pipe_L[pi_];
        if (a.pipe == 3 && ctx->lb_RB > 0) a.RB = ctx->lb_RB;
    }
}

// One operator application in precision T: out = K u (flags: macro e_in/e_out).
template <typename T>
dbfft_status chain_apply(dbfft_ctx* ctx, const cplx<T>* u, const T* macroW, cplx<T>* out, double* e_out) {
    cplx<T>* W = reinterpret_cast<cplx<T>*>(ctx->W);
    const bool dbl = sizeof(T) == 8;
    const double cp = cpass(ctx, dbl, ctx->B);
    const int nc = ctx->nc;
    Ax1InvArgs<T> a1{ctx->dims, freq<T>(ctx), twid<T>(ctx), u, nullptr, nullptr, W, nullptr, ctx->pre};
    Ax2Args<T> a2 = fft_args<T>(ctx, W, nullptr);
    TRY(run(ctx, dbl ? "pass1_grad_f64" : "pass1_grad_f32", (3 + nc) * cp,
            [&] { return launch_grad<T>(AX1_PLAIN, a1, ctx->stream); }));
    TRY(run(ctx, dbl ? "fft_ax2_f64" : "fft_ax2_f32", 2 * nc * cp, [&] { return launch_fft_ax2<T>(+1, a2, ctx->stream); }));
    TRY(run(ctx, dbl ? "fft_ax1_f64" : "fft_ax1_f32", 2 * nc * cp, [&] { return launch_fft_ax1<T>(+1, a2, ctx->stream); }));
    Ax3Args<T> a3 = ax3_base<T>(ctx, W);
    apply_shape<T>(ctx, a3);
    a3.macroW = macroW;
    a3.tan_in = reinterpret_cast<const T*>(ctx->tan);
    TRY(run(ctx, dbl ? "pass3_tangent_f64" : "pass3_tangent_f32", 2 * nc * cp + mat_bytes(ctx, dbl, false),
            [&] { return launch_ax3<T>(opk_apply(ctx), a3, ctx->stream); }));
    TRY(run(ctx, dbl ? "fft_ax1_f64" : "fft_ax1_f32", 2 * nc * cp, [&] { return launch_fft_ax1<T>(-1, a2, ctx->stream); }));
    TRY(run(ctx, dbl ? "fft_ax2_f64" : "fft_ax2_f32", 2 * nc * cp, [&] { return launch_fft_ax2<T>(-1, a2, ctx->stream); }));
    Ax1FwdArgs<T> a5;
    std::memset(&a5, 0, sizeof(a5));
    a5.d = ctx->dims;
    a5.f = freq<T>(ctx);
    a5.tw = twid<T>(ctx);
    a5.W = W;
    a5.out = out;
    a5.e_out = e_out;
    TRY(run(ctx, dbl ? "pass5_div_f64" : "pass5_div_f32", (3 + nc) * cp,
            [&] { return launch_div<T>(AX5_PLAIN, a5, ctx->stream); }));
    return DBFFT_OK;
}

dbfft_status chain_div_resid(dbfft_ctx* ctx, cplx<double>* W, std::vector<double>& ru2, std::vector<double>& re2);

// FP64 residual of the current state: r64 = -B^H sigma(fU + E x_e + B x) + (0, N sigma_f),
// constitutive update in pass 3 (tangent written in the inner precision).
// Returns per-RHS ||r_u||^2 and ||r_e||^2 on the host and fills sig0.
// x_zero: the fluctuation x is known to be zero (the first residual of a
// linear solve); its gradient and inverse transforms are exact zeros, so the
// chain starts in pass 3 from the macro field alone.
dbfft_status chain_residual(dbfft_ctx* ctx, const cplx<double>* x, const double* xe, std::vector<double>& ru2,
                            std::vector<double>& re2, bool x_zero = false) {
    cplx<double>* W = reinterpret_cast<cplx<double>*>(ctx->W);
    const double cp = cpass(ctx, true, ctx->B);
    const int nc = ctx->nc;
    TRY(run(ctx, "macro", 0.0,
            [&] { return launch_macro(ctx->B, ctx->nc, ctx->activeflag, ctx->fU, xe, ctx->macroW, ctx->macroWf, ctx->stream); }));
    Ax1InvArgs<double> a1{ctx->dims, freq<double>(ctx), twid<double>(ctx), x, nullptr, nullptr, W, nullptr, ctx->pre};
    Ax2Args<double> a2 = fft_args<double>(ctx, W, nullptr);
    if (!x_zero) {
        TRY(run(ctx, "pass1_grad_f64", (3 + nc) * cp, [&] { return launch_grad<double>(AX1_PLAIN, a1, ctx->stream); }));
        TRY(run(ctx, "fft_ax2_f64", 2 * nc * cp, [&] { return launch_fft_ax2<double>(+1, a2, ctx->stream); }));
        TRY(run(ctx, "fft_ax1_f64", 2 * nc * cp, [&] { return launch_fft_ax1<double>(+1, a2, ctx->stream); }));
    }
    // Zero fluctuation and linear isotropic phases: the stress is linear in the
    // fields lambda(x), mu(x), so one unit-strain stress per material map goes
    // through pass 3 and the two strided transforms and every right-hand side's
    // spectrum is a combination of it (exact up to rounding; Rm times less
    // FP64 transform work).
    if (x_zero && ctx->model == DBFFT_ISO_ELASTIC && nc == 6 && ctx->n3 % 2 == 0 && ctx->Bm <= 8 && ctx->Rm > 1) {
        Dims d1 = ctx->dims;
        d1.B = ctx->Bm;
        d1.Rm = 1;
        const double cp1 = cpass(ctx, true, ctx->Bm);
        Ax3Args<double> u3 = ax3_base<double>(ctx, W);
        u3.d = d1;
        u3.RB = 1;
        u3.zero_in = 1;
        u3.macroW = ctx->macro_unit;
        Ax2Args<double> u2 = a2;
        u2.d = d1;
        CK(cudaMemsetAsync(ctx->errw, 0, sizeof(unsigned), ctx->stream));
        TRY(run(ctx, "pass3_unit_f64", 2 * nc * cp1,
                [&] { return launch_ax3<double>(OP_ISO, u3, ctx->stream); }));
        TRY(run(ctx, "fft_ax1_f64", 2 * nc * cp1, [&] { return launch_fft_ax1<double>(-1, u2, ctx->stream); }));
        TRY(run(ctx, "fft_ax2_f64", 2 * nc * cp1, [&] { return launch_fft_ax2<double>(-1, u2, ctx->stream); }));
        TRY(run(ctx, "affine_combine_f64", (2.0 * ctx->Bm + 6.0 * ctx->B) * cpass(ctx, true, 1),
                [&] { return launch_affine_combine(ctx->dims, ctx->Bm, W, ctx->macroW, ctx->stream); }));
        return chain_div_resid(ctx, W, ru2, re2);
    }
    Ax3Args<double> a3 = ax3_base<double>(ctx, W);
    a3.zero_in = x_zero ? 1 : 0;
    a3.macroW = ctx->macroW;
    if (ctx->model != DBFFT_ISO_ELASTIC) {
        if (ctx->prec == DBFFT_MIXED) a3.tan_out_f = reinterpret_cast<float*>(ctx->tan);
        else a3.tan_out_d = reinterpret_cast<double*>(ctx->tan);
        a3.eps_p = ctx->eps_p;
        a3.sig_prev = ctx->sig_prev;
        a3.eps_p_t = ctx->eps_p_t;
        a3.sig_t = ctx->sig_t;
        a3.guess_trial = ctx->cp_guess_trial;
        a3.fp_old = ctx->fp_c;
        a3.fp_new = ctx->fp_t;
    }
    CK(cudaMemsetAsync(ctx->errw, 0, sizeof(unsigned), ctx->stream));
    TRY(run(ctx, "pass3_update_f64", 2 * nc * cp + mat_bytes(ctx, true, true),
            [&] { return launch_ax3<double>(opk_update(ctx), a3, ctx->stream); }));
    TRY(run(ctx, "fft_ax1_f64", 2 * nc * cp, [&] { return launch_fft_ax1<double>(-1, a2, ctx->stream); }));
    TRY(run(ctx, "fft_ax2_f64", 2 * nc * cp, [&] { return launch_fft_ax2<double>(-1, a2, ctx->stream); }));
    return chain_div_resid(ctx, W, ru2, re2);
}

// The end of the FP64 residual chain: r64 = -B^H sigma-hat (with the macro
// rows), the per-RHS norms on the host, and the error words of pass 3.
dbfft_status chain_div_resid(dbfft_ctx* ctx, cplx<double>* W, std::vector<double>& ru2, std::vector<double>& re2) {
    const double cp = cpass(ctx, true, ctx->B);
    const int nc = ctx->nc;
    Ax1FwdArgs<double> a5;
    std::memset(&a5, 0, sizeof(a5));
    a5.d = ctx->dims;
    a5.f = freq<double>(ctx);
    a5.tw = twid<double>(ctx);
    a5.W = W;
    a5.out = ctx->r64;
    a5.sig0 = ctx->sig0;
    a5.sig_f = ctx->sigf;
    a5.r_e = ctx->re64;
    a5.partials = ctx->partials;
    TRY(run(ctx, "pass5_div_resid_f64", (3 + nc) * cp,
            [&] { return launch_div<double>(AX5_RESID, a5, ctx->stream); }));
    // the unknowns are Hermitian-consistent spectra: drop the round-off that breaks it
    TRY(run(ctx, "hermitian_planes", 0.0, [&] { return launch_herm_planes<double>(ctx->dims, ctx->r64, ctx->stream); }));
    const int nblk = (int)pw_blocks(ctx->H, ctx->B);
    CK(cudaMemcpyAsync(ctx->part_h, ctx->partials, (size_t)ctx->B * nblk * 2 * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    unsigned* errh = reinterpret_cast<unsigned*>(ctx->small_h + ctx->B * 10);
    CK(cudaMemcpyAsync(errh, ctx->errw, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    prof_flush(ctx);
    ru2.assign(ctx->B, 0.0);
    re2.assign(ctx->B, 0.0);
    for (int b = 0; b < ctx->B; ++b)
        for (int k = 0; k < nblk; ++k) {
            ru2[b] += ctx->part_h[((size_t)b * nblk + k) * 2 + 0];
            re2[b] += ctx->part_h[((size_t)b * nblk + k) * 2 + 1];
        }
    if (*errh & 2u) return fail(ctx, DBFFT_E_TIMEOUT, "a device wait gave up (pass 3 copy pipeline)");
    if (*errh) return fail(ctx, DBFFT_E_MATERIAL, "local constitutive update failed (non-positive J or local Newton)");
    for (int b = 0; b < ctx->B; ++b)
        if (!std::isfinite(ru2[b]) || !std::isfinite(re2[b])) return fail(ctx, DBFFT_E_NONFINITE, "non-finite residual");
    return DBFFT_OK;
}

// Loop condition of the inner-PCG graph: keep iterating while any
// right-hand side is still active (each stops by tolerance or iteration cap).
__global__ void k_cg_continue(cudaGraphConditionalHandle h, const CgState* cg, int B) {
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    int any = 0;
    for (int b = threadIdx.x; b < B; b += 32) any |= (cg[b].done == 0);
    any = __any_sync(0xffffffffu, any);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

// Capture one PCG iteration (passes 1-5 + the loop condition) as the body of
// a WHILE conditional node: one graph launch runs the whole inner solve.
// The FP32 CG iteration runs passes 1 and 5 fused into the axis-2 transforms
// (5 kernels per iteration instead of 7) where the fused kernels exist.
template <typename T>
bool fused_cg(const dbfft_ctx* ctx) {
    return sizeof(T) == 4 && ctx->fuse_ax2 && fused_ax2_supported(ctx->n2);
}

template <typename T>
dbfft_status build_cg_graph(dbfft_ctx* ctx, const Ax1InvArgs<T>& a1, const Ax2Args<T>& a2, const Ax3Args<T>& a3,
                            const Ax1FwdArgs<T>& a5, int opk, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    std::memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // capture on a private stream (the context's stream may be the legacy
    // default stream, which cannot capture); the graph runs on the context's stream
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // consecutive kernels of the iteration are joined by programmatic
        // dependencies: each may launch while its predecessor drains and waits
        // (pdl_wait) before reading the predecessor's output
        g_pdl_launch = ctx->use_pdl;
        if (fused_cg<T>(ctx)) {
            if constexpr (sizeof(T) == 4) {
                e = launch_grad_ax2(a1, cs);
                if (e == cudaSuccess) e = launch_fft_ax1<T>(+1, a2, cs);
                if (e == cudaSuccess) e = launch_ax3<T>(opk, a3, cs);
                if (e == cudaSuccess) e = launch_fft_ax1<T>(-1, a2, cs);
                if (e == cudaSuccess) e = launch_ax2_div(a5, cs);
            }
        } else {
            e = launch_grad<T>(AX1_CG, a1, cs);
            if (e == cudaSuccess) e = launch_fft_ax2<T>(+1, a2, cs);
            if (e == cudaSuccess) e = launch_fft_ax1<T>(+1, a2, cs);
            if (e == cudaSuccess) e = launch_ax3<T>(opk, a3, cs);
            if (e == cudaSuccess) e = launch_fft_ax1<T>(-1, a2, cs);
            if (e == cudaSuccess) e = launch_fft_ax2<T>(-1, a2, cs);
            if (e == cudaSuccess) e = launch_div<T>(AX5_CG, a5, cs);
        }
        if (e == cudaSuccess) e = launch_k(k_cg_continue, dim3(1), dim3(32), 0, cs, h, (const CgState*)ctx->cg, ctx->B);
        g_pdl_launch = false;
        cudaGraph_t captured = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
        if (e == cudaSuccess) e = e2;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        if (ctx->use_pdl) {  // capture without programmatic dependencies instead
            ctx->use_pdl = false;
            return build_cg_graph<T>(ctx, a1, a2, a3, a5, opk, out);
        }
        CK(e);
    }
    cudaError_t e3 = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e3);
    return DBFFT_OK;
}

// Inner PCG in precision T on K d = ri (already scaled), x = xi.
template <typename T>
dbfft_status inner_cg(dbfft_ctx* ctx, double tol, long long& it_sum, int& it_max) {
    cplx<T>* W = reinterpret_cast<cplx<T>*>(ctx->W);
    cplx<T>* xi = reinterpret_cast<cplx<T>*>(ctx->xi);
    cplx<T>* ri = reinterpret_cast<cplx<T>*>(ctx->ri);
    cplx<T>* pi = reinterpret_cast<cplx<T>*>(ctx->pi);
    CK(cudaMemsetAsync(pi, 0, (size_t)ctx->B * 3 * ctx->H * sizeof(cplx<T>), ctx->stream));
    CgInitArgs<T> ai;
    ai.d = ctx->dims;
    ai.f = freq<T>(ctx);
    ai.r = ri;
    ai.r_e = ctx->re_i;
    ai.p_e = ctx->pe_i;
    ai.macroW = ctx->macroW;
    ai.macroWf = ctx->macroWf;
    ai.cg = ctx->cg;
    ai.pre = ctx->pre;
    ai.partials = ctx->partials;
    ai.counters = ctx->counters;
    ai.tol = tol;
    ai.max_iter = ctx->grid.max_iter;
    const dim3 gi((unsigned)pw_blocks(ctx->H, ctx->B), ctx->B);
    const bool dbl = sizeof(T) == 8;
    TRY(run(ctx, dbl ? "cg_init_f64" : "cg_init_f32", 3 * cpass(ctx, dbl, ctx->B), [&] {
        k_cg_init<T><<<gi, PW_THREADS, 0, ctx->stream>>>(ai);
        return cudaGetLastError();
    }));

    Ax1InvArgs<T> a1{ctx->dims, freq<T>(ctx), twid<T>(ctx), ri, pi, xi, W, ctx->cg, ctx->pre};
    Ax2Args<T> a2 = fft_args<T>(ctx, W, ctx->cg);
    Ax3Args<T> a3 = ax3_base<T>(ctx, W);
    apply_shape<T>(ctx, a3);
    if constexpr (sizeof(T) == 4) a3.macroW = ctx->macroWf;
    else a3.macroW = ctx->macroW;
    a3.cg = ctx->cg;
    a3.partials = ctx->partials;
    a3.counters = ctx->counters;
    a3.tan_in = reinterpret_cast<const T*>(ctx->tan);
    Ax1FwdArgs<T> a5;
    std::memset(&a5, 0, sizeof(a5));
    a5.d = ctx->dims;
    a5.f = freq<T>(ctx);
    a5.tw = twid<T>(ctx);
    a5.W = W;
    a5.x = xi;
    a5.p = pi;
    a5.r = ri;
    a5.r_e = ctx->re_i;
    a5.x_e = ctx->xe_i;
    a5.p_e = ctx->pe_i;
    a5.macroW = ctx->macroW;
    a5.macroWf = ctx->macroWf;
    a5.cg = ctx->cg;
    a5.pre = ctx->pre;
    a5.partials = ctx->partials;
    a5.counters = ctx->counters;
    const int opk = opk_apply(ctx);

    const int pi_ = dbl ? 1 : 0;
    if (ctx->use_graphs && !ctx->prof && !ctx->graph_warm[pi_] && !ctx->cg_exec[pi_]) {
        // first inner solve of this context: capture it right away. A launcher whose
        // one-time set-up cannot run under capture makes this fail; the solve then
        // runs launch by launch once (which does that set-up) and captures next time.
        const std::string keep = ctx->err;
        const bool pdl = ctx->use_pdl;
        if (build_cg_graph<T>(ctx, a1, a2, a3, a5, opk_apply(ctx), &ctx->cg_exec[pi_]) != DBFFT_OK) {
            ctx->cg_exec[pi_] = nullptr;
            ctx->err = keep;
            ctx->use_pdl = pdl;
            cudaGetLastError();
        }
    }
    if (ctx->use_graphs && !ctx->prof && (ctx->graph_warm[pi_] || ctx->cg_exec[pi_])) {
        // the whole inner solve as one graph launch
        if (!ctx->cg_exec[pi_]) TRY(build_cg_graph<T>(ctx, a1, a2, a3, a5, opk_apply(ctx), &ctx->cg_exec[pi_]));
        CK(cudaGraphLaunch(ctx->cg_exec[pi_], ctx->stream));
        CK(cudaMemcpyAsync(ctx->cg_h, ctx->cg, ctx->B * sizeof(CgState), cudaMemcpyDeviceToHost, ctx->stream));
        unsigned* errh = reinterpret_cast<unsigned*>(ctx->small_h + ctx->B * 10);
        CK(cudaMemcpyAsync(errh, ctx->errw, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (*errh & 2u) return fail(ctx, DBFFT_E_TIMEOUT, "a device wait gave up (pass 3 copy pipeline)");
        int mx = 1;
        for (int b = 0; b < ctx->B; ++b) mx = std::max(mx, ctx->cg_h[b].iter);
        ctx->launches += (fused_cg<T>(ctx) ? 6LL : 8LL) * mx;
        it_max = 0;
        for (int b = 0; b < ctx->B; ++b) {
            it_sum += ctx->cg_h[b].iter;
            if (ctx->cg_h[b].iter > it_max) it_max = ctx->cg_h[b].iter;
            if (ctx->cg_h[b].flags & 2) return fail(ctx, DBFFT_E_NONFINITE, "non-finite value in the inner CG");
        }
        return DBFFT_OK;
    }
    int launched = 0;
    int chunk = 4;
    const int nc = ctx->nc;
    const char* n_p1 = dbl ? "pass1_grad_cg_f64" : "pass1_grad_cg_f32";
    const char* n_a2 = dbl ? "fft_ax2_f64" : "fft_ax2_f32";
    const char* n_a1 = dbl ? "fft_ax1_f64" : "fft_ax1_f32";
    const char* n_p3 = dbl ? "pass3_tangent_f64" : "pass3_tangent_f32";
    const char* n_p5 = dbl ? "pass5_div_cg_f64" : "pass5_div_cg_f32";
    const bool fused = fused_cg<T>(ctx);
    const char* n_p1f = "pass1_grad_ax2_cg_f32";  // fused: pass 1 + inverse axis-2 transform
    const char* n_p5f = "pass5_ax2_div_cg_f32";   // fused: forward axis-2 transform + pass 5
    std::vector<int> it_before(ctx->B, 0);
    while (true) {
        // launches are timed here; their algorithmic bytes are credited after
        // the chunk, from the iterations each right-hand side really made (a
        // right-hand side that stops inside a chunk skips the later launches)
        for (int k = 0; k < chunk; ++k) {
            if (fused) {
                if constexpr (sizeof(T) == 4) {
                    TRY(run(ctx, n_p1f, 0.0, [&] { return launch_grad_ax2(a1, ctx->stream); }));
                    TRY(run(ctx, n_a1, 0.0, [&] { return launch_fft_ax1<T>(+1, a2, ctx->stream); }));
                    TRY(run(ctx, n_p3, 0.0, [&] { return launch_ax3<T>(opk, a3, ctx->stream); }));
                    TRY(run(ctx, n_a1, 0.0, [&] { return launch_fft_ax1<T>(-1, a2, ctx->stream); }));
                    TRY(run(ctx, n_p5f, 0.0, [&] { return launch_ax2_div(a5, ctx->stream); }));
                }
                continue;
            }
            TRY(run(ctx, n_p1, 0.0, [&] { return launch_grad<T>(AX1_CG, a1, ctx->stream); }));
            TRY(run(ctx, n_a2, 0.0, [&] { return launch_fft_ax2<T>(+1, a2, ctx->stream); }));
            TRY(run(ctx, n_a1, 0.0, [&] { return launch_fft_ax1<T>(+1, a2, ctx->stream); }));
            TRY(run(ctx, n_p3, 0.0, [&] { return launch_ax3<T>(opk, a3, ctx->stream); }));
            TRY(run(ctx, n_a1, 0.0, [&] { return launch_fft_ax1<T>(-1, a2, ctx->stream); }));
            TRY(run(ctx, n_a2, 0.0, [&] { return launch_fft_ax2<T>(-1, a2, ctx->stream); }));
            TRY(run(ctx, n_p5, 0.0, [&] { return launch_div<T>(AX5_CG, a5, ctx->stream); }));
        }
        launched += chunk;
        CK(cudaMemcpyAsync(ctx->cg_h, ctx->cg, ctx->B * sizeof(CgState), cudaMemcpyDeviceToHost, ctx->stream));
        unsigned* errh = reinterpret_cast<unsigned*>(ctx->small_h + ctx->B * 10);
        CK(cudaMemcpyAsync(errh, ctx->errw, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        prof_flush(ctx);
        if (*errh & 2u) return fail(ctx, DBFFT_E_TIMEOUT, "a device wait gave up (pass 3 copy pipeline)");
        if (ctx->prof) {
            const double cp1 = cpass(ctx, dbl, 1);
            double sum_it = 0.0, mat = 0.0;
            for (int g = 0; g < ctx->Bm; ++g) {  // material tables: once per launch in which a group iterates
                int mx = 0;
                for (int r = 0; r < ctx->Rm; ++r) {
                    const int b = g * ctx->Rm + r;
                    mx = std::max(mx, ctx->cg_h[b].iter - it_before[b]);
                    sum_it += ctx->cg_h[b].iter - it_before[b];
                }
                mat += (ctx->model == DBFFT_ISO_ELASTIC ? (double)mx : 0.0) * mat_bytes(ctx, dbl, false) / ctx->Bm;
            }
            if (ctx->model != DBFFT_ISO_ELASTIC) mat = sum_it * mat_bytes(ctx, dbl, false) / ctx->B;
            ctx->prof_bytes[prof_slot(ctx, fused ? n_p1f : n_p1)] += sum_it * (15 + nc) * cp1;
            if (!fused) ctx->prof_bytes[prof_slot(ctx, n_a2)] += sum_it * 2 * (2 * nc * cp1);
            ctx->prof_bytes[prof_slot(ctx, n_a1)] += sum_it * 2 * (2 * nc * cp1);
            ctx->prof_bytes[prof_slot(ctx, n_p3)] += sum_it * 2 * nc * cp1 + mat;
            ctx->prof_bytes[prof_slot(ctx, fused ? n_p5f : n_p5)] += sum_it * (6 + nc) * cp1;
        }
        bool all = true;
        for (int b = 0; b < ctx->B; ++b) {
            all &= (ctx->cg_h[b].done != 0);
            it_before[b] = ctx->cg_h[b].iter;
        }
        if (all || launched >= ctx->grid.max_iter + 1) break;
        chunk = chunk < 16 ? chunk * 2 : 16;
    }
    ctx->graph_warm[pi_] = true;
    it_max = 0;
    for (int b = 0; b < ctx->B; ++b) {
        it_sum += ctx->cg_h[b].iter;
        if (ctx->cg_h[b].iter > it_max) it_max = ctx->cg_h[b].iter;
        if (ctx->cg_h[b].flags & 2) return fail(ctx, DBFFT_E_NONFINITE, "non-finite value in the inner CG");
    }
    return DBFFT_OK;
}

constexpr int kMeanTangentBlocks = 456;  // blocks per right-hand side of the mean-tangent reduction

// Mean tangent of the current state -> preconditioner (R10), nonlinear only.
dbfft_status refresh_precond(dbfft_ctx* ctx) {
    const int nblk = kMeanTangentBlocks;
    const int kind = ctx->model == DBFFT_NEO_HOOKE ? 0
                   : ctx->model == DBFFT_SVK         ? 2
                   : ctx->model == DBFFT_CP_FCC_FINITE ? 3
                                                       : 1;
    TRY(run(ctx, "mean_tangent", 0.0, [&] {
        if (ctx->prec == DBFFT_MIXED)
            return launch_mean_tangent<float>(kind, ctx->B, ctx->V, reinterpret_cast<const float*>(ctx->tan),
                                              ctx->phase, ctx->lam, ctx->mu, ctx->partials, nblk, ctx->stream);
        return launch_mean_tangent<double>(kind, ctx->B, ctx->V, reinterpret_cast<const double*>(ctx->tan),
                                           ctx->phase, ctx->lam, ctx->mu, ctx->partials, nblk, ctx->stream);
    }));
    std::vector<double> ph((size_t)ctx->B * nblk * 81);
    CK(cudaMemcpyAsync(ph.data(), ctx->partials, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int b = 0; b < ctx->B; ++b) {
        double C[3][3][3][3];
        double* Cf = &C[0][0][0][0];
        for (int q = 0; q < 81; ++q) {
            double s = 0.0;
            for (int k = 0; k < nblk; ++k) s += ph[((size_t)b * nblk + k) * 81 + q];
            Cf[q] = s / (double)ctx->V;
        }
        if (!precond_from(ctx, C, ctx->pre_h[b / ctx->Rm]))
            return fail(ctx, DBFFT_E_NONFINITE, "singular macro block of the mean tangent");
    }
    CK(cudaMemcpyAsync(ctx->pre, ctx->pre_h.data(), ctx->pre_h.size() * sizeof(PrecondData), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->pre_is_init = false;
    return DBFFT_OK;
}

// Back to the preconditioner of the initial stiffness (refresh policy INITIAL).
dbfft_status restore_initial_precond(dbfft_ctx* ctx) {
    ctx->pre_h = ctx->pre_init_h;
    CK(cudaMemcpyAsync(ctx->pre, ctx->pre_h.data(), ctx->pre_h.size() * sizeof(PrecondData), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->pre_is_init = true;
    return DBFFT_OK;
}

dbfft_status set_scales(dbfft_ctx* ctx, const std::vector<double>& s) {
    std::memcpy(ctx->small_h, s.data(), ctx->B * sizeof(double));
    CK(cudaMemcpyAsync(ctx->scal, ctx->small_h, ctx->B * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    return DBFFT_OK;
}

// Outer FP64 loop of one increment (linear refinement or Newton).
dbfft_status solve_current(dbfft_ctx* ctx, dbfft_report* rep) {
    const bool linear = ctx->model == DBFFT_ISO_ELASTIC;
    const bool inner64 = ctx->prec == DBFFT_FP64;
    std::vector<double> ru2, re2, bn(ctx->B, 0.0);
    std::vector<char> done(ctx->B, 0);
    long long it_sum = 0;
    int it_max_all = 0;
    int outer = 0, steps = 0;
    bool converged = false;
    double worst_eq = 0.0, worst_ld = 0.0, worst_rel = 0.0;
    if (linear) {
        CK(cudaMemsetAsync(ctx->x64, 0, (size_t)ctx->B * 3 * ctx->H * sizeof(cplx<double>), ctx->stream));
        CK(cudaMemsetAsync(ctx->xe64, 0, (size_t)ctx->B * 9 * sizeof(double), ctx->stream));
    }
    const int max_steps = ctx->grid.max_newton > 0 ? ctx->grid.max_newton : 50;
    for (int step = 0; step <= max_steps; ++step) {
        ctx->cp_guess_trial = step > 0;  // later Newton steps start the local solves from the last trial stress
        const dbfft_status rs = chain_residual(ctx, ctx->x64, ctx->xe64, ru2, re2, linear && step == 0);
        ctx->cp_guess_trial = 0;
        TRY(rs);
        ++outer;
        // convergence per right-hand side
        CK(cudaMemcpyAsync(ctx->small_h, ctx->sig0, ctx->B * 9 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        bool all = true;
        worst_eq = worst_ld = worst_rel = 0.0;
        for (int b = 0; b < ctx->B; ++b) {
            const double rn = std::sqrt(ru2[b] + re2[b]);
            double sn = 0.0;
            for (int q = 0; q < ctx->nc; ++q) {
                const double v = ctx->small_h[b * 9 + q];
                sn += (ctx->nc == 6 && q >= 3 ? 2.0 : 1.0) * v * v;
            }
            sn = std::sqrt(sn);
            const double eq = sn > 0 ? std::sqrt(ru2[b]) / sn : std::sqrt(ru2[b]);
            const double ld = (sn > 0 && ctx->dims.ne) ? std::sqrt(re2[b]) / ((double)ctx->V * sn) : 0.0;
            if (linear) {
                if (step == 0) bn[b] = rn;
                const double rel = bn[b] > 0 ? rn / bn[b] : 0.0;
                done[b] = (bn[b] == 0.0) || rel <= ctx->grid.tol;
                worst_rel = std::max(worst_rel, rel);
            } else {
                done[b] = eq <= ctx->grid.newton_tol && ld <= ctx->grid.load_tol;
            }
            worst_eq = std::max(worst_eq, eq);
            worst_ld = std::max(worst_ld, ld);
            all &= done[b] != 0;
        }
        if (all) { converged = true; break; }
        if (step == max_steps) break;
        if (!linear) {  // reference stiffness of the preconditioner (R10 and its alternatives)
            if (ctx->pre_refresh == DBFFT_PRECOND_INITIAL) {
                if (!ctx->pre_is_init) TRY(restore_initial_precond(ctx));
            } else if (step == 0 || ctx->pre_refresh == DBFFT_PRECOND_PER_NEWTON) {
                TRY(refresh_precond(ctx));
            }
        }
        // inner solve on r / ||r||
        std::vector<double> sc(ctx->B), sb(ctx->B);
        for (int b = 0; b < ctx->B; ++b) {
            const double rn = std::sqrt(ru2[b] + re2[b]);
            sc[b] = (!done[b] && rn > 0) ? 1.0 / rn : 0.0;
            sb[b] = (!done[b] && rn > 0) ? rn : 0.0;
        }
        TRY(set_scales(ctx, sc));
        const double itol = (linear && inner64) ? ctx->grid.tol : ctx->grid.eta_inner;
        int itm = 0;
        const double c64 = cpass(ctx, true, ctx->B), ci = cpass(ctx, inner64, ctx->B);
        if (inner64) {
            TRY(run(ctx, "to_inner", 3 * (c64 + 2 * ci), [&] {
                return launch_to_inner<double>(ctx->dims, ctx->r64, ctx->re64, ctx->scal,
                                               reinterpret_cast<cplx<double>*>(ctx->ri), ctx->re_i,
                                               reinterpret_cast<cplx<double>*>(ctx->xi), ctx->xe_i, ctx->stream);
            }));
            TRY(inner_cg<double>(ctx, itol, it_sum, itm));
        } else {
            TRY(run(ctx, "to_inner", 3 * (c64 + 2 * ci), [&] {
                return launch_to_inner<float>(ctx->dims, ctx->r64, ctx->re64, ctx->scal,
                                              reinterpret_cast<cplx<float>*>(ctx->ri), ctx->re_i,
                                              reinterpret_cast<cplx<float>*>(ctx->xi), ctx->xe_i, ctx->stream);
            }));
            TRY(inner_cg<float>(ctx, itol, it_sum, itm));
        }
        it_max_all += itm;
        TRY(set_scales(ctx, sb));
        TRY(run(ctx, "from_inner", 3 * (2 * c64 + 2 * ci), [&] {
            if (inner64)
                return launch_from_inner<double>(ctx->dims, reinterpret_cast<const cplx<double>*>(ctx->xi),
                                                 reinterpret_cast<const cplx<double>*>(ctx->pi), ctx->cg, ctx->xe_i,
                                                 ctx->scal, ctx->x64, ctx->xe64, ctx->stream);
            return launch_from_inner<float>(ctx->dims, reinterpret_cast<const cplx<float>*>(ctx->xi),
                                            reinterpret_cast<const cplx<float>*>(ctx->pi), ctx->cg, ctx->xe_i,
                                            ctx->scal, ctx->x64, ctx->xe64, ctx->stream);
        }));
        // keep the iterate a Hermitian-consistent spectrum (R5b): FP32 corrections
        // carry round-off off that subspace on the k3 = 0 and k3 = n3/2 planes
        TRY(run(ctx, "hermitian_planes", 0.0, [&] { return launch_herm_planes<double>(ctx->dims, ctx->x64, ctx->stream); }));
        ++steps;
    }
    ctx->have_solution = true;
    if (rep) {
        rep->newton_iters = steps;
        rep->outer_iters = outer;
        rep->cg_iters = it_sum;
        rep->cg_iters_max = it_max_all;
        rep->eps_eq = worst_eq;
        rep->load_res = worst_ld;
        rep->true_rel_res = worst_rel;
    }
    if (!converged) return fail(ctx, DBFFT_E_NOT_CONVERGED, "iteration cap reached before the tolerance");
    return DBFFT_OK;
}

dbfft_status commit_state(dbfft_ctx* ctx) {
    if (ctx->model == DBFFT_CP_FCC_POWERLAW) {
        std::swap(ctx->eps_p, ctx->eps_p_t);
        std::swap(ctx->sig_prev, ctx->sig_t);
    } else if (ctx->model == DBFFT_CP_FCC_FINITE) {
        std::swap(ctx->fp_c, ctx->fp_t);
        std::swap(ctx->sig_prev, ctx->sig_t);
    }
    return DBFFT_OK;
}

// Time one launch shape: two warm launches, then the best of five (CUDA events).
template <class F>
float time_launch(dbfft_ctx* ctx, F&& f) {
    cudaEvent_t a = get_event(ctx), b = get_event(ctx);
    float best = 1e30f;
    bool ok = true;
    for (int k = 0; k < 7 && ok; ++k) {
        cudaEventRecord(a, ctx->stream);
        ok = f() == cudaSuccess;
        cudaEventRecord(b, ctx->stream);
        if (cudaEventSynchronize(b) != cudaSuccess) ok = false;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ok && k >= 2) best = std::min(best, ms);
    }
    cudaGetLastError();
    ctx->pool.push_back(a);
    ctx->pool.push_back(b);
    return ok ? best : 1e30f;
}

// The line-bulk pass 3 serves the FP32 applications of the linear, small-strain
// crystal-plasticity and Neo-Hookean models on lines of 64, 128 or 256 values.
bool lb_supported(const dbfft_ctx* ctx) {
    const int opk = opk_apply(ctx);
    return (ctx->n3 == 64 || ctx->n3 == 128 || ctx->n3 == 256) && (opk == OP_ISO || opk == OP_CP_APPLY || opk == OP_NH_APPLY);
}

template <typename T>
void tune_pass3(dbfft_ctx* ctx, int pi_, cplx<T>* W) {
    char buf[256];
    // FP32 (the CG applications): each candidate runs as in the CG iteration,
    // with its curvature reduction (the CG states cleared first, so that no
    // right-hand side counts as stopped) and right after the axis-1 transform that
    // precedes it; the clearing and the transform's own time are subtracted.
    // Isolated timings without the reduction ranked the line-bulk forms
    // differently from the solve at 64^3 x 6. The CG states are set again by the
    // next solve's start.
    const Ax2Args<T> a2p = fft_args<T>(ctx, W, nullptr);
    const bool chained = sizeof(T) == 4;
    auto pre = [&]() {
        const cudaError_t e = cudaMemsetAsync(ctx->cg, 0, (size_t)ctx->B * sizeof(CgState), ctx->stream);
        return e != cudaSuccess ? e : launch_fft_ax1<T>(+1, a2p, ctx->stream);
    };
    const float t_pre = chained ? time_launch(ctx, pre) : 0.f;
    auto time_p3 = [&](Ax3Args<T> a3) {
        if (!chained) return time_launch(ctx, [&] { return launch_ax3<T>(opk_apply(ctx), a3, ctx->stream); });
        a3.cg = ctx->cg;
        a3.partials = ctx->partials;
        a3.counters = ctx->counters;
        const float ms = time_launch(ctx, [&] {
            const cudaError_t e = pre();
            return e != cudaSuccess ? e : launch_ax3<T>(opk_apply(ctx), a3, ctx->stream);
        });
        return ms >= 1e29f ? ms : std::max(ms - t_pre, 1e-4f);
    };
    // pass 3: radix x lines per CTA (radix 32 = one thread per line, lines of up to 32 complex values)
    const int radices[3] = {8, 16, 32};
    const int radices64[2] = {4, 32};
    const bool r32 = sizeof(T) == 4 ? ctx->n3 <= 256 : ctx->n3 <= 64;
    const int nrad = sizeof(T) == 4 ? (r32 ? 3 : 2) : (r32 ? 2 : 1);
    float best = 1e30f;
    int bestR = ctx->ax3_radix[pi_], bestL = 0;
    std::string per_radix;
    for (int ri = 0; ri < nrad; ++ri) {
        const int R = sizeof(T) == 4 ? radices[ri] : radices64[ri];
        float bR = 1e30f;
        const int Ld = ax3_lines(ctx->n3, ctx->nc, ctx->RB, sizeof(T) == 8, 1, R);
        const int cand[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, Ld};
        for (int L : cand) {
            if (L > Ld * 2 || (long long)L > (long long)ctx->n1 * ctx->n2) continue;
            Ax3Args<T> a3 = ax3_base<T>(ctx, W);
            a3.radix = R;
            a3.L = L;
            if constexpr (sizeof(T) == 4) a3.macroW = ctx->macroWf;
            else a3.macroW = ctx->macroW;
            a3.tan_in = reinterpret_cast<const T*>(ctx->tan);
            const float ms = time_p3(a3);
            bR = std::min(bR, ms);
            if (ms < best * 0.98f) {
                best = ms;
                bestR = R;
                bestL = L;
            }
        }
        std::snprintf(buf, sizeof(buf), "%s%d: %.4f", per_radix.empty() ? "" : ", ", R, bR);
        per_radix += buf;
    }
    ctx->ax3_radix[pi_] = bestR;
    ctx->ax3_L[pi_] = bestL;
    std::snprintf(buf, sizeof(buf), "pass3 radix %d lines %d (%.4f ms; best per radix %s); ", bestR, bestL, best,
                  per_radix.c_str());
    ctx->tune_note += buf;
    // the pipelined pass for the CG applications: radix x lines per tile
    {
        const long long nlines = (long long)ctx->n1 * ctx->n2;
        float bp = 1e30f;
        int bpR = 0, bpL = 0, bpS = 0;
        for (int ps : {1, 2})
        for (int ri = 0; ri < (sizeof(T) == 4 ? 2 : 1); ++ri) {
            const int R = sizeof(T) == 4 ? radices[ri] : 4;
            for (int L : {2, 4, 6, 8, 12, 16, 24, 32}) {
                const long long sm = ax3_pipe_smem(ctx->n3, ctx->nc, ctx->RB, sizeof(T) == 8, ctx->scale != nullptr, R,
                                                   L, nlines, ps);
                if (sm < 0 || sm > 200 * 1024) continue;
                Ax3Args<T> a3 = ax3_base<T>(ctx, W);
                a3.pipe = ps;
                a3.radix = R;
                a3.L = L;
                if constexpr (sizeof(T) == 4) a3.macroW = ctx->macroWf;
                else a3.macroW = ctx->macroW;
                a3.tan_in = reinterpret_cast<const T*>(ctx->tan);
                const float ms = time_p3(a3);
                if (ms < bp * 0.98f) {
                    bp = ms;
                    bpR = R;
                    bpL = L;
                    bpS = ps;
                }
            }
        }
        // the line-bulk pass (FP32 applications on lines of 64, 128 or 256 values)
        float blb = 1e30f;
        int blbL = 0;
        int blbT = 0;
        int blbB = 0;
        if (sizeof(T) == 4 && lb_supported(ctx)) {
            for (int rb = std::min(ctx->Rm, 8); rb >= 1; --rb)  // right-hand sides per CTA
            for (int cap : {384, 192, -1, -2})  // threads per CTA (more, smaller CTAs overlap each
                                                  // other's phases); -1, -2: warp lines
            for (int L : {2, 4, 6, 8, 12, 16}) {
                if (ctx->Rm % rb != 0) continue;
                if (cap == -1 && L != 16) continue;
                if (cap == -2 && L != (ctx->n3 == 256 ? 8 : 4)) continue;
                const long long sm = ax3_lb_smem(ctx->n3, ctx->nc, rb, ctx->scale != nullptr, L, nlines);
                if (sm < 0 || sm > 110 * 1024) continue;
                Ax3Args<T> a3 = ax3_base<T>(ctx, W);
                a3.pipe = 3;
                a3.radix = cap;
                a3.L = L;
                a3.RB = rb;
                if constexpr (sizeof(T) == 4) a3.macroW = ctx->macroWf;
                else a3.macroW = ctx->macroW;
                a3.tan_in = reinterpret_cast<const T*>(ctx->tan);
                const float ms = time_p3(a3);
                if (ms < blb * 0.98f) {
                    blb = ms;
                    blbL = L;
                    blbT = cap;
                    blbB = rb;
                }
            }
            if (blbL > 0 && blb < bp) {
                bp = blb;
                bpS = 3;
                bpR = blbT;
                bpL = blbL;
            }
        }
        ctx->pipe_on[pi_] = (bpL > 0 && bp < best) ? bpS : 0;
        ctx->pipe_R[pi_] = bpR;
        ctx->pipe_L[pi_] = bpL;
        if (sizeof(T) == 4) ctx->lb_RB = ctx->pipe_on[pi_] == 3 ? blbB : 0;
        std::snprintf(buf, sizeof(buf), "pass3 bulk-copy %s radix %d lines %d (%.4f ms)%s; ",
                      bpS == 3 ? "line-bulk" : bpS == 2 ? "one-stage" : "two-stage", bpR, bpL, bp,
                      ctx->pipe_on[pi_] ? " used" : "");
        ctx->tune_note += buf;
        if (blbL > 0) {
            std::snprintf(buf, sizeof(buf), "pass3 line-bulk lines %d threads<=%d rhs/CTA %d (%.4f ms); ", blbL, blbT,
                          blbB, blb);
            ctx->tune_note += buf;
        }
    }
}

template <typename T>
void tune_precision(dbfft_ctx* ctx, int pi_, bool pass3) {
    cplx<T>* W = reinterpret_cast<cplx<T>*>(ctx->W);
    cudaMemsetAsync(ctx->W, 0, (size_t)ctx->B * ctx->nc * ctx->H * sizeof(cplx<T>), ctx->stream);
    char buf[256];
    if (pass3) tune_pass3<T>(ctx, pi_, W);
    // strided transforms: columns per CTA along axes 1 and 2
    for (int ax = 0; ax < 2; ++ax) {
        float bt = 1e30f;
        int btw = 0;
        for (int tw : {4, 8, 16, 32, 64}) {
            Ax2Args<T> a2 = fft_args<T>(ctx, W, nullptr);
            a2.tw_ax1 = a2.tw_ax2 = tw;
            const float ms = time_launch(ctx, [&] {
                return ax == 0 ? launch_fft_ax1<T>(+1, a2, ctx->stream) : launch_fft_ax2<T>(+1, a2, ctx->stream);
            });
            if (ms < bt * 0.98f) {
                bt = ms;
                btw = tw;
            }
        }
        ctx->fft_tw[pi_][ax] = btw;
        std::snprintf(buf, sizeof(buf), "fft axis %d tile %d (%.4f ms); ", ax + 1, btw, bt);
        ctx->tune_note += buf;
    }
}

std::string tune_key(const dbfft_ctx* ctx) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == ' ') c = '_';
    char buf[256];
    std::snprintf(buf, sizeof(buf), "v2 %s n=%dx%dx%d B=%d RB=%d nc=%d prec=%d model=%d scale=%d", name.c_str(), ctx->n1,
                  ctx->n2, ctx->n3, ctx->B, ctx->RB, ctx->nc, ctx->prec, ctx->model, ctx->scale != nullptr ? 1 : 0);
    return buf;
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

const char* dbfft_status_string(dbfft_status s) {
    switch (s) {
        case DBFFT_OK: return "DBFFT_OK";
        case DBFFT_E_ARG: return "DBFFT_E_ARG";
        case DBFFT_E_UNSUPPORTED_GRID: return "DBFFT_E_UNSUPPORTED_GRID";
        case DBFFT_E_NOMEM: return "DBFFT_E_NOMEM";
        case DBFFT_E_CUDA: return "DBFFT_E_CUDA";
        case DBFFT_E_NOT_CONVERGED: return "DBFFT_E_NOT_CONVERGED";
        case DBFFT_E_NONFINITE: return "DBFFT_E_NONFINITE";
        case DBFFT_E_TIMEOUT: return "DBFFT_E_TIMEOUT";
        case DBFFT_E_MATERIAL: return "DBFFT_E_MATERIAL";
        case DBFFT_E_STATE: return "DBFFT_E_STATE";
    }
    return "unknown";
}

const char* dbfft_last_error(const dbfft_ctx* ctx) { return ctx ? ctx->err.c_str() : noalloc_last_error(); }

long long dbfft_launch_count(const dbfft_ctx* ctx) { return ctx ? ctx->launches : 0; }

dbfft_status dbfft_autotune(dbfft_ctx* ctx, const char* cache_path) {
    if (!ctx) return DBFFT_E_ARG;
    ctx->fwd_inc0 = false;  // timing runs the passes on the context's buffers
    ctx->tangent_ready = false;
    if ((ctx->n1 & 1) || (ctx->n2 & 1) || (ctx->n3 & 1)) {  // the odd-length kernels have one shape each
        ctx->tune_note = "odd grid: fixed launch shapes";
        return DBFFT_OK;
    }
    const std::string key = tune_key(ctx);
    // precisions to tune: the inner solve's, and in the MIXED mode also the
    // FP64 passes of the outer residual chain
    std::vector<int> pis;
    if (ctx->prec == DBFFT_FP64) pis = {1};
    else pis = {0, 1};
    auto drop_graphs = [&] {
        for (int k = 0; k < 2; ++k)
            if (ctx->cg_exec[k]) { cudaGraphExecDestroy(ctx->cg_exec[k]); ctx->cg_exec[k] = nullptr; }
    };
    if (cache_path) {
        if (FILE* f = std::fopen(cache_path, "r")) {
            char line[512];
            while (std::fgets(line, sizeof(line), f)) {
                std::string ln(line);
                if (ln.compare(0, key.size(), key) != 0 || ln.size() <= key.size() || ln[key.size()] != '|') continue;
                const char* p = ln.c_str() + key.size() + 1;
                int v[2][8];
                int n = 0;
                for (size_t k = 0; k < pis.size(); ++k) {
                    int used = 0;
                    if (std::sscanf(p, "%d %d %d %d %d %d %d %d%n", &v[k][0], &v[k][1], &v[k][2], &v[k][3], &v[k][4],
                                    &v[k][5], &v[k][6], &v[k][7], &used) != 8)
                        break;
                    p += used;
                    ++n;
                }
                if (n != (int)pis.size()) continue;
                for (size_t k = 0; k < pis.size(); ++k) {
                    const int pi_ = pis[k];
                    ctx->ax3_radix[pi_] = v[k][0];
                    ctx->ax3_L[pi_] = v[k][1];
                    ctx->fft_tw[pi_][0] = v[k][2];
                    ctx->fft_tw[pi_][1] = v[k][3];
                    ctx->pipe_on[pi_] = v[k][4];
                    ctx->pipe_R[pi_] = v[k][5];
                    ctx->pipe_L[pi_] = v[k][6];
                    if (pi_ == 0) ctx->lb_RB = v[k][7];
                }
                ctx->tune_note = "from cache:";
                for (int pi_ : pis) {  // the shapes in force, as the tuner reports them
                    char b[160];
                    std::snprintf(b, sizeof(b), " [%s] pass3 %s radix %d lines %d rhs/CTA %d, fft tiles %d/%d;",
                                  pi_ ? "FP64" : "FP32",
                                  ctx->pipe_on[pi_] == 3   ? "line-bulk"
                                  : ctx->pipe_on[pi_] == 2 ? "bulk-copy one-stage"
                                  : ctx->pipe_on[pi_] == 1 ? "bulk-copy two-stage"
                                                           : "plain",
                                  ctx->pipe_on[pi_] ? ctx->pipe_R[pi_] : ctx->ax3_radix[pi_],
                                  ctx->pipe_on[pi_] ? ctx->pipe_L[pi_] : ctx->ax3_L[pi_],
                                  ctx->pipe_on[pi_] == 3 && ctx->lb_RB > 0 ? ctx->lb_RB : ctx->RB,
                                  ctx->fft_tw[pi_][0], ctx->fft_tw[pi_][1]);
                    ctx->tune_note += b;
                }
                std::fclose(f);
                drop_graphs();
                return DBFFT_OK;
            }
            std::fclose(f);
        }
    }
    ctx->tune_note.clear();
    for (int pi_ : pis) {
        if (pi_ == 0) {
            tune_precision<float>(ctx, 0, true);
        } else {
            // the FP64 operator application of pass 3 reads an FP64 tangent, which a
            // MIXED context of a nonlinear model does not hold: there only the
            // strided transforms are tuned for FP64
            const bool p3 = ctx->prec == DBFFT_FP64 || ctx->model == DBFFT_ISO_ELASTIC;
            if (ctx->prec != DBFFT_FP64) ctx->tune_note += "[FP64 residual chain] ";
            tune_precision<double>(ctx, 1, p3);
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graphs();
    if (cache_path) {
        if (FILE* f = std::fopen(cache_path, "a")) {
            std::fprintf(f, "%s|", key.c_str());
            for (int pi_ : pis)
                std::fprintf(f, " %d %d %d %d %d %d %d %d", ctx->ax3_radix[pi_], ctx->ax3_L[pi_], ctx->fft_tw[pi_][0],
                             ctx->fft_tw[pi_][1], ctx->pipe_on[pi_], ctx->pipe_R[pi_], ctx->pipe_L[pi_],
                             pi_ == 0 ? ctx->lb_RB : 0);
            std::fprintf(f, "\n");
            std::fclose(f);
        }
    }
    return DBFFT_OK;
}

const char* dbfft_tuning(const dbfft_ctx* ctx) { return ctx ? ctx->tune_note.c_str() : ""; }

dbfft_status dbfft_set_pass3_shape(dbfft_ctx* ctx, int fp64, int pipelined, int radix, int lines) {
    if (!ctx || (fp64 != 0 && fp64 != 1) || lines < 1) return DBFFT_E_ARG;
    const bool dbl = fp64 == 1;
    const long long nlines = (long long)ctx->n1 * ctx->n2;
    const int pi_ = dbl ? 1 : 0;
    if (pipelined == 3) {  // line-bulk pass: its transform shape is fixed, radix is ignored
        const int rb = ctx->lb_RB > 0 ? ctx->lb_RB : ctx->RB;
        const long long sm = ax3_lb_smem(ctx->n3, ctx->nc, rb, ctx->scale != nullptr, lines, nlines);
        if (dbl || !lb_supported(ctx) || sm < 0 || sm > 200 * 1024)
            return fail(ctx, DBFFT_E_ARG,
                        "line-bulk pass 3: FP32, n3 = 64, 128 or 256, linear / crystal-plasticity / Neo-Hookean "
                        "model, lines even and dividing n1*n2");
        if (radix == -1 && lines != 16) return fail(ctx, DBFFT_E_ARG, "line-bulk warp lines (-1) need 16-line tiles");
        if (radix == -2 && lines != (ctx->n3 == 256 ? 8 : 4))
            return fail(ctx, DBFFT_E_ARG,
                        "line-bulk warp lines (-2) need tiles of 8 (n3 = 256) or 4 (n3 = 64, 128) lines");
        if (radix < -2) return fail(ctx, DBFFT_E_ARG, "line-bulk: radix is a thread cap, -1 or -2");
        ctx->pipe_on[pi_] = 3;
        ctx->pipe_R[pi_] = radix < 0 ? radix : (radix > 0 && radix < 384 ? radix : 0);  // thread cap / warp lines
        ctx->pipe_L[pi_] = lines;
        for (int k = 0; k < 2; ++k)
            if (ctx->cg_exec[k]) { cudaGraphExecDestroy(ctx->cg_exec[k]); ctx->cg_exec[k] = nullptr; }
        return DBFFT_OK;
    }
    if (pipelined < 0 || pipelined > 3) return fail(ctx, DBFFT_E_ARG, "pipelined: 0, 1, 2 or 3");
    const bool r32 = radix == 32 && !pipelined && ctx->n3 <= (dbl ? 64 : 256);
    if (dbl ? (radix != 4 && !r32) : (radix != 8 && radix != 16 && !r32))
        return fail(ctx, DBFFT_E_ARG,
                    "radix: 8 or 16 (FP32), 4 (FP64), or 32 with the plain kernel (n3 <= 256 FP32, <= 64 FP64)");
    if (lines > nlines) return fail(ctx, DBFFT_E_ARG, "more lines per CTA than grid lines");
    if (pipelined) {
        const long long sm =
            ax3_pipe_smem(ctx->n3, ctx->nc, ctx->RB, dbl, ctx->scale != nullptr, radix, lines, nlines, pipelined);
        if (sm < 0 || sm > 200 * 1024)
            return fail(ctx, DBFFT_E_ARG, "pipelined pass 3: lines must be even, divide n1*n2 and fit in shared memory");
        ctx->pipe_on[pi_] = pipelined;
        ctx->pipe_R[pi_] = radix;
        ctx->pipe_L[pi_] = lines;
    } else {
        ctx->pipe_on[pi_] = 0;
        ctx->ax3_radix[pi_] = radix;
        ctx->ax3_L[pi_] = lines;
    }
    for (int k = 0; k < 2; ++k)  // graphs captured with the old shape
        if (ctx->cg_exec[k]) { cudaGraphExecDestroy(ctx->cg_exec[k]); ctx->cg_exec[k] = nullptr; }
    return DBFFT_OK;
}

dbfft_status dbfft_set_pass3_rhs_group(dbfft_ctx* ctx, int rhs) {
    if (!ctx) return DBFFT_E_ARG;
    if (rhs < 0 || rhs > 8 || (rhs > 0 && ctx->Rm % rhs != 0))
        return fail(ctx, DBFFT_E_ARG, "line-bulk right-hand sides per CTA: 0, or 1 to 8 dividing those of a material map");
    if (rhs > 0 && ctx->pipe_on[0] == 3 &&
        ax3_lb_smem(ctx->n3, ctx->nc, rhs, ctx->scale != nullptr, ctx->pipe_L[0], (long long)ctx->n1 * ctx->n2) >
            200 * 1024)
        return fail(ctx, DBFFT_E_ARG, "line-bulk tile does not fit in shared memory with that many right-hand sides");
    ctx->lb_RB = rhs;
    for (int k = 0; k < 2; ++k)
        if (ctx->cg_exec[k]) { cudaGraphExecDestroy(ctx->cg_exec[k]); ctx->cg_exec[k] = nullptr; }
    return DBFFT_OK;
}

dbfft_status dbfft_set_precond_refresh(dbfft_ctx* ctx, int policy) {
    if (!ctx) return DBFFT_E_ARG;
    if (policy != DBFFT_PRECOND_PER_INCREMENT && policy != DBFFT_PRECOND_INITIAL && policy != DBFFT_PRECOND_PER_NEWTON)
        return fail(ctx, DBFFT_E_ARG, "unknown preconditioner refresh policy");
    ctx->pre_refresh = policy;
    return DBFFT_OK;
}

dbfft_status dbfft_profile(dbfft_ctx* ctx, int enable) {
    if (!ctx) return DBFFT_E_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    prof_flush(ctx);
    ctx->prof = enable != 0;
    ctx->prof_name.clear();
    ctx->prof_n.clear();
    ctx->prof_ms.clear();
    ctx->prof_bytes.clear();
    return DBFFT_OK;
}

int dbfft_profile_read(dbfft_ctx* ctx, dbfft_profile_entry* out, int max_entries) {
    if (!ctx) return 0;
    cudaStreamSynchronize(ctx->stream);
    prof_flush(ctx);
    const int n = (int)ctx->prof_name.size();
    for (int i = 0; i < n && i < max_entries; ++i) {
        std::memset(out[i].name, 0, sizeof(out[i].name));
        std::strncpy(out[i].name, ctx->prof_name[i].c_str(), sizeof(out[i].name) - 1);
        out[i].launches = ctx->prof_n[i];
        out[i].ms = ctx->prof_ms[i];
        out[i].bytes = ctx->prof_bytes[i];
    }
    return n;
}

size_t dbfft_device_bytes(const dbfft_ctx* ctx) { return ctx ? ctx->bytes : 0; }

void dbfft_destroy(dbfft_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    prof_flush(ctx);
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k)
        if (ctx->cg_exec[k]) cudaGraphExecDestroy(ctx->cg_exec[k]);
    for (auto& b : ctx->bufs) {
        if (ctx->use_cb) ctx->alloc.free(b.p, ctx->alloc.user);
        else cudaFree(b.p);
    }
    pinned_free(ctx->cg_h, ctx->B * sizeof(CgState));
    pinned_free(ctx->part_h, ctx->partials_n * sizeof(double));
    pinned_free(ctx->small_h, (ctx->B * 10 + 8) * sizeof(double));
    pinned_free(ctx->stage_h, ctx->stage_n);
    delete ctx;
}

static dbfft_status create_impl(dbfft_ctx* ctx, const dbfft_grid* grid, const dbfft_materials* mat,
                                const dbfft_load* load) {
    ctx->grid = *grid;
    // DBFFT_CUDA_GRAPHS=0 runs every inner PCG launch by launch (same kernels,
    // same order), e.g. for profilers that cannot look inside conditional graphs
    if (const char* g = std::getenv("DBFFT_CUDA_GRAPHS")) ctx->use_graphs = g[0] != '0';
    // programmatic dependent launch inside the CG graph (DBFFT_PDL=1): the
    // early-launched successor holds SM resources while it waits. Measured in
    // graph order on the current kernels: 64^3 x 6 RHS mixed step 10.75 ms with
    // it against 10.65 ms without, the FP64 CG of 64^3 x 1 RHS 23.8 against
    // 18.5 ms per solve, 256^3 x 1 FP32 iteration 1.080 ms either way; off.
    ctx->use_pdl = false;
    if (const char* g = std::getenv("DBFFT_PDL")) ctx->use_pdl = g[0] != '0';
    // DBFFT_FUSE_AX2=0 keeps passes 1 and 5 as element-wise kernels around separate
    // axis-2 transforms in the FP32 CG (for comparison; the results agree to rounding)
    if (const char* g = std::getenv("DBFFT_FUSE_AX2")) ctx->fuse_ax2 = g[0] != '0';
    // DBFFT_WAIT_POLLS=n bounds the first bulk-copy wait of the line-bulk pass 3
    // to n polls (a test setting: a limit that runs out makes the solve return
    // E_TIMEOUT while the copies still land before the CTA exits)
    if (const char* g = std::getenv("DBFFT_WAIT_POLLS")) ctx->wait_limit = std::atoll(g);
    ctx->n1 = grid->n[0];
    ctx->n2 = grid->n[1];
    ctx->n3 = grid->n[2];
    for (int a = 0; a < 3; ++a)
        if (!supported_len(grid->n[a]))
            return fail(ctx, DBFFT_E_UNSUPPORTED_GRID,
                        "grid sizes must be powers of two in [8, 256] or odd with prime factors 3, 5, 7 (9 .. 245)");
    // m: the Nyquist index of an even axis 3 (weight-1 plane of the half spectrum);
    // 0 for odd n3, whose only weight-1 plane is k3 = 0
    ctx->m = ctx->n3 % 2 == 0 ? ctx->n3 / 2 : 0;
    ctx->h = ctx->n3 / 2 + 1;
    ctx->H = (long long)ctx->n1 * ctx->n2 * ctx->h;
    ctx->V = (long long)ctx->n1 * ctx->n2 * ctx->n3;
    ctx->B = grid->batch;
    ctx->Bm = grid->n_materials;
    if (ctx->B < 1 || ctx->Bm < 1 || ctx->B % ctx->Bm) return fail(ctx, DBFFT_E_ARG, "batch must be a multiple of n_materials");
    if (ctx->B > 65535) return fail(ctx, DBFFT_E_ARG, "batch too large");
    ctx->Rm = ctx->B / ctx->Bm;
    ctx->kin = grid->kinematics;
    if (ctx->kin != DBFFT_SMALL && ctx->kin != DBFFT_FINITE) return fail(ctx, DBFFT_E_ARG, "kinematics");
    ctx->nc = ctx->kin == DBFFT_SMALL ? 6 : 9;
    ctx->prec = grid->precision;
    if (ctx->prec != DBFFT_FP64 && ctx->prec != DBFFT_MIXED) return fail(ctx, DBFFT_E_ARG, "precision");
    if (!(grid->tol > 0) || grid->max_iter < 1) return fail(ctx, DBFFT_E_ARG, "tol / max_iter");
    if (!mat || !mat->phase_id || mat->n_phases < 1 || !mat->phases) return fail(ctx, DBFFT_E_ARG, "materials");
    ctx->model = mat->phases[0].model;
    for (int p = 0; p < mat->n_phases; ++p)
        if (mat->phases[p].model != ctx->model) return fail(ctx, DBFFT_E_ARG, "all phases must use one model kind");
    if ((ctx->model == DBFFT_NEO_HOOKE || ctx->model == DBFFT_SVK || ctx->model == DBFFT_CP_FCC_FINITE) !=
        (ctx->kin == DBFFT_FINITE))
        return fail(ctx, DBFFT_E_ARG,
                    "NEO_HOOKE, SVK and CP_FCC_FINITE need FINITE kinematics; ISO_ELASTIC and CP need SMALL");
    if ((ctx->n3 & 1) && ctx->model != DBFFT_ISO_ELASTIC && !supported_odd_nl(ctx->n3))
        return fail(ctx, DBFFT_E_UNSUPPORTED_GRID, "odd n3 with nonlinear phases: 9, 15, 21, 27, 45, 63 or 81");
    if (ctx->model != DBFFT_ISO_ELASTIC && ctx->Rm != 1)
        return fail(ctx, DBFFT_E_ARG, "nonlinear models need one material map per right-hand side");
    if (!load || !load->target || load->n_increments < 1) return fail(ctx, DBFFT_E_ARG, "load");
    ctx->stress_mask = load->stress_mask;
    ctx->n_inc = load->n_increments;
    ctx->total_time = load->total_time > 0 ? load->total_time : 1.0;
    ctx->target.assign(load->target, load->target + ctx->B * 9);
    for (double v : ctx->target)
        if (!std::isfinite(v)) return fail(ctx, DBFFT_E_NONFINITE, "non-finite load target");

    // macro unknowns (R8)
    Dims& d = ctx->dims;
    std::memset(&d, 0, sizeof(d));
    d.n1 = ctx->n1; d.n2 = ctx->n2; d.n3 = ctx->n3; d.h = ctx->h; d.m = ctx->m;
    d.H = ctx->H; d.V = ctx->V; d.plane = (long long)ctx->n2 * ctx->h;
    d.div_plane = make_fastdiv((unsigned)d.plane);
    d.div_h = make_fastdiv((unsigned)ctx->h);
    d.B = ctx->B; d.Rm = ctx->Rm; d.nc = ctx->nc; d.kin = ctx->kin;
    d.invN = 1.0 / (double)ctx->V;
    if (ctx->nc == 6) {
        static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (((ctx->stress_mask >> (3 * i + j)) & 1u) != ((ctx->stress_mask >> (3 * j + i)) & 1u))
                    return fail(ctx, DBFFT_E_ARG, "small-strain stress mask must be symmetric");
        for (int mm = 0; mm < 6; ++mm)
            if ((ctx->stress_mask >> (3 * pi[mm] + pj[mm])) & 1u) {
                ctx->activeflag_h[mm] = 1;
                d.active[d.ne++] = mm;
            }
    } else {
        for (int q = 0; q < 9; ++q)
            if ((ctx->stress_mask >> q) & 1u) {
                ctx->activeflag_h[q] = 1;
                d.active[d.ne++] = q;
            }
    }
    // right-hand sides per CTA of pass 3: a divisor of Rm that keeps the CTA within 256 threads
    ctx->RB = 1;
    for (int rb = std::min(ctx->Rm, 8); rb >= 1; --rb)
        if (ctx->Rm % rb == 0 && ax3_threads_per_line(ctx->n3, ctx->nc, rb, true) <= 256 &&
            ax3_threads_per_line(ctx->n3, ctx->nc, rb, false) <= 256) {
            ctx->RB = rb;
            break;
        }

    TRY(upload_tables(ctx));
    TRY(dalloc_t(ctx, 9, &ctx->activeflag));
    CK(cudaMemcpyAsync(ctx->activeflag, ctx->activeflag_h, 9 * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));

    // materials
    const size_t nvox = (size_t)ctx->Bm * ctx->V;
    TRY(dalloc_t(ctx, nvox, &ctx->phase));
    const bool dev_maps = mat->device_arrays != 0;
    std::vector<long long> pcount((size_t)ctx->Bm * mat->n_phases, 0);
    if (dev_maps) {
        // the maps live on the device: copy them there, count the phases and check
        // the ids with a kernel (the stiffness scale is checked once lam and mu are
        // uploaded, below)
        CK(cudaMemcpyAsync(ctx->phase, mat->phase_id, nvox * sizeof(uint16_t), cudaMemcpyDeviceToDevice, ctx->stream));
        unsigned long long* cnt_d = nullptr;
        const size_t ncnt = (size_t)ctx->Bm * mat->n_phases + 1;  // counts, then the bad-id count
        TRY(dalloc_t(ctx, ncnt, &cnt_d));
        CK(cudaMemsetAsync(cnt_d, 0, ncnt * sizeof(unsigned long long), ctx->stream));
        CK(launch_phase_counts(ctx->phase, ctx->Bm, ctx->V, mat->n_phases, cnt_d, cnt_d + ncnt - 1, ctx->stream));
        std::vector<unsigned long long> cnt_h(ncnt);
        CK(cudaMemcpyAsync(cnt_h.data(), cnt_d, ncnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (cnt_h[ncnt - 1]) return fail(ctx, DBFFT_E_ARG, "phase id out of range");
        for (size_t k = 0; k + 1 < ncnt; ++k) pcount[k] = (long long)cnt_h[k];
        if (mat->E_scale) {
            TRY(dalloc_t(ctx, nvox, &ctx->scale));
            TRY(dalloc_t(ctx, nvox, &ctx->scale_f));
            CK(cudaMemcpyAsync(ctx->scale, mat->E_scale, nvox * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        }
    } else {
        // one pass over the maps: range check and the voxel count of every phase per material group
        // (four interleaved count arrays, so that runs of one phase id do not chain their increments)
        {
            const size_t np4 = (size_t)mat->n_phases;
            std::vector<uint32_t> c4(4 * np4);
            for (int g = 0; g < ctx->Bm; ++g) {
                const uint16_t* ids = mat->phase_id + (size_t)g * ctx->V;
                std::fill(c4.begin(), c4.end(), 0u);
                unsigned mx = 0;
                long long v = 0;
                for (; v + 4 <= ctx->V; v += 4) {
                    const unsigned a = ids[v], b = ids[v + 1], c = ids[v + 2], d = ids[v + 3];
                    mx = std::max(mx, std::max(std::max(a, b), std::max(c, d)));
                    if (mx >= (unsigned)mat->n_phases) return fail(ctx, DBFFT_E_ARG, "phase id out of range");
                    ++c4[a];
                    ++c4[np4 + b];
                    ++c4[2 * np4 + c];
                    ++c4[3 * np4 + d];
                }
                for (; v < ctx->V; ++v) {
                    const unsigned a = ids[v];
                    if (a >= (unsigned)mat->n_phases) return fail(ctx, DBFFT_E_ARG, "phase id out of range");
                    ++c4[a];
                }
                long long* cg = pcount.data() + (size_t)g * np4;
                for (size_t p = 0; p < np4; ++p) cg[p] = (long long)c4[p] + c4[np4 + p] + c4[2 * np4 + p] + c4[3 * np4 + p];
            }
        }
        // through a page-locked staging copy: the transfer then runs while the host
        // goes on with the set-up (the buffer returns to the cache at destroy)
        ctx->stage_n = nvox * sizeof(uint16_t);
        ctx->stage_h = pinned_alloc(ctx->stage_n);
        if (ctx->stage_h) {
            std::memcpy(ctx->stage_h, mat->phase_id, ctx->stage_n);
            CK(cudaMemcpyAsync(ctx->phase, ctx->stage_h, ctx->stage_n, cudaMemcpyHostToDevice, ctx->stream));
        } else {
            CK(cudaMemcpyAsync(ctx->phase, mat->phase_id, ctx->stage_n, cudaMemcpyHostToDevice, ctx->stream));
        }
        if (mat->E_scale) {
            for (size_t i = 0; i < nvox; ++i)
                if (!std::isfinite(mat->E_scale[i])) return fail(ctx, DBFFT_E_NONFINITE, "non-finite E_scale");
            TRY(dalloc_t(ctx, nvox, &ctx->scale));
            CK(cudaMemcpyAsync(ctx->scale, mat->E_scale, nvox * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
            std::vector<float> sf(mat->E_scale, mat->E_scale + nvox);
            TRY(dalloc_t(ctx, nvox, &ctx->scale_f));
            CK(cudaMemcpyAsync(ctx->scale_f, sf.data(), nvox * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        }
    }
    const int np = mat->n_phases;
    ctx->lam_h.assign(np, 0.0);
    ctx->mu_h.assign(np, 0.0);
    ctx->E_h.assign(np, 1.0);
    std::vector<double> lam1(np, 0.0), mu1(np, 0.0);
    for (int p = 0; p < np; ++p) {
        const dbfft_phase& ph = mat->phases[p];
        if (ctx->model == DBFFT_ISO_ELASTIC) {
            if (!std::isfinite(ph.E) || !std::isfinite(ph.nu)) return fail(ctx, DBFFT_E_NONFINITE, "non-finite E or nu");
            if (!(ph.E > 0) || !(ph.nu > -1 && ph.nu < 0.5)) return fail(ctx, DBFFT_E_ARG, "E > 0 and -1 < nu < 1/2 required");
            ctx->lam_h[p] = ph.E * ph.nu / ((1 + ph.nu) * (1 - 2 * ph.nu));
            ctx->mu_h[p] = ph.E / (2 * (1 + ph.nu));
            ctx->E_h[p] = ph.E;
            lam1[p] = ctx->lam_h[p] / ph.E;
            mu1[p] = ctx->mu_h[p] / ph.E;
        } else if (ctx->model == DBFFT_NEO_HOOKE || ctx->model == DBFFT_SVK) {
            if (!std::isfinite(ph.mu) || !std::isfinite(ph.lambda)) return fail(ctx, DBFFT_E_NONFINITE, "non-finite mu or lambda");
            if (!(ph.mu > 0)) return fail(ctx, DBFFT_E_ARG, "mu > 0 required");
            if (ctx->model == DBFFT_SVK && !(3.0 * ph.lambda + 2.0 * ph.mu > 0))
                return fail(ctx, DBFFT_E_ARG, "3 lambda + 2 mu > 0 required");
            ctx->lam_h[p] = ph.lambda;
            ctx->mu_h[p] = ph.mu;
        } else if (ctx->model == DBFFT_CP_FCC_POWERLAW || ctx->model == DBFFT_CP_FCC_FINITE) {
            const double vals[9] = {ph.C11, ph.C12, ph.C44, ph.gdot0, ph.m, ph.tau_c, ph.quat[0], ph.quat[1], ph.quat[2]};
            for (double v : vals)
                if (!std::isfinite(v)) return fail(ctx, DBFFT_E_NONFINITE, "non-finite crystal parameter");
        } else {
            return fail(ctx, DBFFT_E_ARG, "unknown model");
        }
    }
    TRY(dalloc_t(ctx, np, &ctx->lam));
    TRY(dalloc_t(ctx, np, &ctx->mu));
    TRY(dalloc_t(ctx, np, &ctx->lam1));
    TRY(dalloc_t(ctx, np, &ctx->mu1));
    CK(cudaMemcpyAsync(ctx->lam, ctx->lam_h.data(), np * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->mu, ctx->mu_h.data(), np * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    {
        std::vector<float> lf(ctx->lam_h.begin(), ctx->lam_h.end()), mf(ctx->mu_h.begin(), ctx->mu_h.end());
        TRY(dalloc_t(ctx, np, &ctx->lam_f));
        TRY(dalloc_t(ctx, np, &ctx->mu_f));
        CK(cudaMemcpyAsync(ctx->lam_f, lf.data(), np * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->mu_f, mf.data(), np * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->lam1, lam1.data(), np * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->mu1, mu1.data(), np * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->model == DBFFT_CP_FCC_POWERLAW || ctx->model == DBFFT_CP_FCC_FINITE) {
        std::vector<CpGrain> gr(np);
        for (int p = 0; p < np; ++p)
            if (!cp_grain(mat->phases[p], gr[p])) return fail(ctx, DBFFT_E_ARG, "singular crystal stiffness");
        std::vector<CpGrainF> grf(np);
        for (int p = 0; p < np; ++p) {
            for (int q = 0; q < 21; ++q) grf[p].S[q] = (float)gr[p].S[q];
            for (int a = 0; a < 12; ++a)
                for (int q = 0; q < 6; ++q) grf[p].P[a][q] = (float)gr[p].P[a][q];
        }
        TRY(dalloc_t(ctx, np, &ctx->grains));
        TRY(dalloc_t(ctx, np, &ctx->grains_f));
        CK(cudaMemcpyAsync(ctx->grains, gr.data(), np * sizeof(CpGrain), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->grains_f, grf.data(), np * sizeof(CpGrainF), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const dbfft_phase& p0 = mat->phases[0];
        CpScalars<double>& c = ctx->cp.d;
        c.gdot0 = p0.gdot0;
        c.inv_m = 1.0 / p0.m;
        c.tau_c = p0.tau_c;
        c.dt = ctx->total_time / ctx->n_inc;
        c.inv_tc = 1.0 / c.tau_c;
        c.dtg = c.dt * c.gdot0;
        c.dtg_n_tc = c.dtg * c.inv_m / c.tau_c;
        c.dtk = c.dtg * c.tau_c * p0.m / (1.0 + p0.m);
        CpScalars<float>& cf = ctx->cp.f;
        cf.gdot0 = (float)c.gdot0;
        cf.inv_m = (float)c.inv_m;
        cf.tau_c = (float)c.tau_c;
        cf.dt = (float)c.dt;
        cf.inv_tc = (float)c.inv_tc;
        cf.dtg = (float)c.dtg;
        cf.dtg_n_tc = (float)c.dtg_n_tc;
        cf.dtk = (float)c.dtk;
        const double ni = std::round(c.inv_m);
        ctx->cp.n_int = (ni >= 1.0 && ni <= 127.0 && std::fabs(c.inv_m - ni) <= 1e-12 * ni) ? (int)ni : 0;
        ctx->cp.rtol = 1e-12;
        ctx->cp.max_it = 100;
    }

    // device-resident stiffness scale: FP32 copy, finite check and the per-map
    // sums of lam s and mu s for the mean stiffness, on the device
    std::vector<double> scaled_sums;  // [Bm][2]
    if (dev_maps && mat->E_scale) {
        const int nblk = (int)std::min<long long>((ctx->V + 255) / 256, 1024);
        double* part_d = nullptr;
        unsigned long long* bad_d = nullptr;
        TRY(dalloc_t(ctx, (size_t)ctx->Bm * nblk * 2, &part_d));
        TRY(dalloc_t(ctx, 1, &bad_d));
        CK(cudaMemsetAsync(bad_d, 0, sizeof(unsigned long long), ctx->stream));
        CK(launch_scale_stats(ctx->phase, ctx->scale, ctx->scale_f, ctx->Bm, ctx->V, np, ctx->lam, ctx->mu, part_d, nblk,
                              bad_d, ctx->stream));
        std::vector<double> part_h((size_t)ctx->Bm * nblk * 2);
        unsigned long long bad_h = 0;
        CK(cudaMemcpyAsync(part_h.data(), part_d, part_h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&bad_h, bad_d, sizeof(bad_h), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (bad_h) return fail(ctx, DBFFT_E_NONFINITE, "non-finite E_scale");
        scaled_sums.assign((size_t)ctx->Bm * 2, 0.0);
        for (int g = 0; g < ctx->Bm; ++g)
            for (int k = 0; k < nblk; ++k) {  // fixed order: the same sums on every run
                scaled_sums[g * 2 + 0] += part_h[((size_t)g * nblk + k) * 2 + 0];
                scaled_sums[g * 2 + 1] += part_h[((size_t)g * nblk + k) * 2 + 1];
            }
    }

    // preconditioner of the linear problem: mean stiffness (Sec. 2.5, R10)
    ctx->pre_h.assign(ctx->Bm, PrecondData{});
    for (int g = 0; g < ctx->Bm; ++g) {
        double C[3][3][3][3];
        const long long* cnt = pcount.data() + (size_t)g * np;
        if (ctx->model == DBFFT_ISO_ELASTIC || ctx->model == DBFFT_NEO_HOOKE || ctx->model == DBFFT_SVK) {
            // ISO: mean stiffness; NH, SVK: initial tangent K(I) = isotropic C of the mean moduli
            double sl = 0.0, sm = 0.0;
            if (ctx->model == DBFFT_ISO_ELASTIC && mat->E_scale && dev_maps) {
                sl = scaled_sums[g * 2 + 0];
                sm = scaled_sums[g * 2 + 1];
            } else if (ctx->model == DBFFT_ISO_ELASTIC && mat->E_scale) {
                for (long long v = 0; v < ctx->V; ++v) {
                    const int p = mat->phase_id[(size_t)g * ctx->V + v];
                    const double s = mat->E_scale[(size_t)g * ctx->V + v];
                    sl += ctx->lam_h[p] * s;
                    sm += ctx->mu_h[p] * s;
                }
            } else {
                for (int p = 0; p < np; ++p) {
                    sl += (double)cnt[p] * ctx->lam_h[p];
                    sm += (double)cnt[p] * ctx->mu_h[p];
                }
            }
            iso_C(sl / ctx->V, sm / ctx->V, C);
        } else {  // elastic stiffness of the grains
            double Cs[3][3][3][3] = {};
            for (int p = 0; p < np; ++p) {
                if (!cnt[p]) continue;
                CpGrain gg;
                cp_grain(mat->phases[p], gg);
                std::vector<double> A(36);
                for (int a = 0; a < 6; ++a)
                    for (int b = 0; b < 6; ++b) A[a * 6 + b] = gg.S[sym6(a, b)];
                invert(6, A);
                for (int a = 0; a < 6; ++a)
                    for (int b = 0; b < 6; ++b) {
                        double Ta[3][3], Tb[3][3];
                        basis_tensor(6, a, Ta);
                        basis_tensor(6, b, Tb);
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j)
                                for (int k = 0; k < 3; ++k)
                                    for (int l = 0; l < 3; ++l)
                                        Cs[i][j][k][l] += (double)cnt[p] / ctx->V * Ta[i][j] * A[a * 6 + b] * Tb[k][l];
                    }
            }
            std::memcpy(C, Cs, sizeof(C));
        }
        if (!precond_from(ctx, C, ctx->pre_h[g])) return fail(ctx, DBFFT_E_ARG, "singular mean stiffness");
    }
    TRY(dalloc_t(ctx, ctx->Bm, &ctx->pre));
    CK(cudaMemcpyAsync(ctx->pre, ctx->pre_h.data(), ctx->Bm * sizeof(PrecondData), cudaMemcpyHostToDevice, ctx->stream));
    ctx->pre_init_h = ctx->pre_h;

    // vectors and work buffers
    const size_t nU = (size_t)ctx->B * 3 * ctx->H;
    const size_t isz = ctx->prec == DBFFT_FP64 ? sizeof(cplx<double>) : sizeof(cplx<float>);
    TRY(dalloc_t(ctx, nU, &ctx->x64));
    TRY(dalloc_t(ctx, nU, &ctx->r64));
    TRY(dalloc(ctx, nU * isz, &ctx->xi));
    TRY(dalloc(ctx, nU * isz, &ctx->ri));
    TRY(dalloc(ctx, nU * isz, &ctx->pi));
    TRY(dalloc(ctx, (size_t)ctx->B * ctx->nc * ctx->H * sizeof(cplx<double>), &ctx->W));
    double** smalls[] = {&ctx->xe64, &ctx->re64, &ctx->xe_i, &ctx->re_i, &ctx->pe_i, &ctx->fU,
                         &ctx->sigf, &ctx->sig0, &ctx->macroW, &ctx->macroW2, &ctx->hbar};
    for (double** s : smalls) TRY(dalloc_t(ctx, (size_t)ctx->B * 9, s));
    TRY(dalloc_t(ctx, (size_t)ctx->B * 9, &ctx->macroWf));
    {
        std::vector<double> unit((size_t)ctx->Bm * 9, 0.0);
        for (int m = 0; m < ctx->Bm; ++m) unit[(size_t)m * 9] = 1.0;
        TRY(dalloc_t(ctx, unit.size(), &ctx->macro_unit));
        CK(cudaMemcpyAsync(ctx->macro_unit, unit.data(), unit.size() * sizeof(double), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));  // the host vector goes out of scope
    }
    TRY(dalloc_t(ctx, (size_t)ctx->B, &ctx->scal));
    TRY(dalloc_t(ctx, (size_t)ctx->B, &ctx->cg));
    TRY(dalloc_t(ctx, (size_t)ctx->B, &ctx->counters));
    TRY(dalloc_t(ctx, 1, &ctx->errw));
    CK(cudaMemsetAsync(ctx->errw, 0, sizeof(unsigned), ctx->stream));
    CK(cudaMemsetAsync(ctx->counters, 0, ctx->B * sizeof(unsigned), ctx->stream));
    CK(cudaMemsetAsync(ctx->x64, 0, nU * sizeof(cplx<double>), ctx->stream));
    CK(cudaMemsetAsync(ctx->xe64, 0, ctx->B * 9 * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(ctx->macroW2, 0, ctx->B * 9 * sizeof(double), ctx->stream));
    // reduction partials: the largest grid of any reducing kernel
    {
        const long long nb1 = pw_blocks(ctx->H, 1);  // element-wise kernels of passes 1 and 5
        const long long nb1d = nb1;
        const long long nlines = (long long)ctx->n1 * ctx->n2;
        const long long nb3 = nlines;  // pass 3 with one line per CTA (any tuned shape fits)
        const long long nb3d = nlines;
        const long long nbi = (ctx->H + 255) / 256;
        const long long nbf = fused_ax2_blocks(ctx->n1, ctx->n3 / 2 + 1);  // fused pass 5
        long long nb = std::max(std::max(std::max(nb1, nb1d), nbf), std::max(std::max(nb3, nb3d), nbi));
        ctx->nblk_max = (int)nb;
        ctx->partials_n = std::max((size_t)ctx->B * (size_t)nb * 2, (size_t)ctx->B * kMeanTangentBlocks * 81);
        TRY(dalloc_t(ctx, ctx->partials_n, &ctx->partials));
        if (!(ctx->part_h = static_cast<double*>(pinned_alloc(ctx->partials_n * sizeof(double)))))
            return fail(ctx, DBFFT_E_NOMEM, "pinned host allocation failed");
    }
    if (!(ctx->cg_h = static_cast<CgState*>(pinned_alloc(ctx->B * sizeof(CgState)))) ||
        !(ctx->small_h = static_cast<double*>(pinned_alloc((ctx->B * 10 + 8) * sizeof(double)))))
        return fail(ctx, DBFFT_E_NOMEM, "pinned host allocation failed");
    // nonlinear tangent and state
    if (ctx->model != DBFFT_ISO_ELASTIC) {
        ctx->ntan = ctx->model == DBFFT_NEO_HOOKE       ? 10
                  : ctx->model == DBFFT_SVK              ? 15
                  : ctx->model == DBFFT_CP_FCC_FINITE    ? 45
                                                         : 21;
        const size_t tsz = ctx->prec == DBFFT_FP64 ? 8 : 4;
        TRY(dalloc(ctx, (size_t)ctx->B * ctx->V * ctx->ntan * tsz, &ctx->tan));
        if (ctx->model == DBFFT_CP_FCC_POWERLAW) {
            const size_t ns = (size_t)ctx->B * ctx->V * 6;
            TRY(dalloc_t(ctx, ns, &ctx->eps_p));
            TRY(dalloc_t(ctx, ns, &ctx->sig_prev));
            TRY(dalloc_t(ctx, ns, &ctx->eps_p_t));
            TRY(dalloc_t(ctx, ns, &ctx->sig_t));
            CK(cudaMemsetAsync(ctx->eps_p, 0, ns * sizeof(double), ctx->stream));
            CK(cudaMemsetAsync(ctx->sig_prev, 0, ns * sizeof(double), ctx->stream));
        } else if (ctx->model == DBFFT_CP_FCC_FINITE) {
            const size_t ns = (size_t)ctx->B * ctx->V * 6, nf = (size_t)ctx->B * ctx->V * 9;
            TRY(dalloc_t(ctx, ns, &ctx->sig_prev));
            TRY(dalloc_t(ctx, ns, &ctx->sig_t));
            TRY(dalloc_t(ctx, nf, &ctx->fp_c));
            TRY(dalloc_t(ctx, nf, &ctx->fp_t));
            CK(cudaMemsetAsync(ctx->sig_prev, 0, ns * sizeof(double), ctx->stream));
            CK(launch_fill_identity(ctx->fp_c, (long long)ctx->B * ctx->V, ctx->stream));
        }
    }
    TRY(set_load(ctx, 0, ctx->target.data()));
    ctx->cur_inc = -1;
    CK(cudaStreamSynchronize(ctx->stream));
    return DBFFT_OK;
}

dbfft_status dbfft_create(const dbfft_grid* grid, const dbfft_materials* mat, const dbfft_load* load,
                          const dbfft_allocator* alloc, void* stream, dbfft_ctx** out) {
    if (!out || !grid) return DBFFT_E_ARG;
    *out = nullptr;
    dbfft_ctx* ctx = new dbfft_ctx();
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    if (alloc && alloc->alloc && alloc->free) {
        ctx->alloc = *alloc;
        ctx->use_cb = true;
    }
    dbfft_status s = create_impl(ctx, grid, mat, load);
    if (s != DBFFT_OK) {
        std::fprintf(stderr, "dbfft_create: %s\n", ctx->err.c_str());
        dbfft_destroy(ctx);
        return s;
    }
    *out = ctx;
    return DBFFT_OK;
}

dbfft_status dbfft_solve_increment(dbfft_ctx* ctx, int inc, dbfft_report* rep) {
    if (!ctx) return DBFFT_E_ARG;
    if (inc < 0 || inc >= ctx->n_inc) return fail(ctx, DBFFT_E_ARG, "increment out of range");
    if (ctx->model != DBFFT_ISO_ELASTIC && inc != ctx->cur_inc + 1)
        return fail(ctx, DBFFT_E_STATE, "path-dependent solves must run increments in order");
    const auto t0 = std::chrono::steady_clock::now();
    if (rep) std::memset(rep, 0, sizeof(*rep));
    ctx->fwd_inc0 = false;
    ctx->tangent_ready = false;
    TRY(set_load(ctx, inc, ctx->target.data()));
    dbfft_status s = solve_current(ctx, rep);
    if (s == DBFFT_OK || s == DBFFT_E_NOT_CONVERGED) {
        commit_state(ctx);
        ctx->cur_inc = inc;
    }
    ctx->fwd_inc0 = s == DBFFT_OK && inc == 0;
    if (ctx->ckpt_on && ctx->model == DBFFT_CP_FCC_POWERLAW) {
        // the converged stress of this increment: the adjoint's checkpoint
        if (s == DBFFT_OK && inc == ctx->ckpt_n) {
            const size_t per = (size_t)ctx->B * ctx->V * 6;
            if (!ctx->ckpt) TRY(dalloc_t(ctx, per * ctx->n_inc, &ctx->ckpt));
            CK(cudaMemcpyAsync(ctx->ckpt + per * inc, ctx->sig_prev, per * sizeof(double), cudaMemcpyDeviceToDevice,
                               ctx->stream));
            ctx->ckpt_n = inc + 1;
        } else {
            ctx->ckpt_n = 0;  // a gap in the record: no adjoint for this path
        }
    }
    if (rep) rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return s;
}

dbfft_status dbfft_homogenized_stress(dbfft_ctx* ctx, double* out) {
    if (!ctx || !out) return DBFFT_E_ARG;
    if (!ctx->have_solution) return fail(ctx, DBFFT_E_STATE, "no solution yet");
    std::vector<double> s(ctx->B * 9);
    CK(cudaMemcpyAsync(s.data(), ctx->sig0, s.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
    for (int b = 0; b < ctx->B; ++b) {
        if (ctx->nc == 9) {
            for (int q = 0; q < 9; ++q) out[b * 9 + q] = s[b * 9 + q];
        } else {
            for (int mm = 0; mm < 6; ++mm) {
                out[b * 9 + 3 * pi[mm] + pj[mm]] = s[b * 9 + mm];
                out[b * 9 + 3 * pj[mm] + pi[mm]] = s[b * 9 + mm];
            }
        }
    }
    return DBFFT_OK;
}

dbfft_status dbfft_get_solution(dbfft_ctx* ctx, void* u_hat, double* e) {
    if (!ctx) return DBFFT_E_ARG;
    if (u_hat)
        CK(cudaMemcpyAsync(u_hat, ctx->x64, (size_t)ctx->B * 3 * ctx->H * sizeof(cplx<double>),
                           cudaMemcpyDeviceToDevice, ctx->stream));
    if (e) CK(cudaMemcpyAsync(e, ctx->xe64, (size_t)ctx->B * 9 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DBFFT_OK;
}

// Hbar per right-hand side, row-major [B][9]: the whole macro strain (small) or
// Fbar - I (finite), from the prescribed part fU (W components) and the solved
// stress-controlled unknowns.
dbfft_status macro_hbar(dbfft_ctx* ctx, std::vector<double>& hb) {
    std::vector<double> fU((size_t)ctx->B * 9), xe((size_t)ctx->B * 9);
    hb.assign((size_t)ctx->B * 9, 0.0);
    CK(cudaMemcpyAsync(fU.data(), ctx->fU, fU.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(xe.data(), ctx->xe64, xe.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
    for (int b = 0; b < ctx->B; ++b) {
        double* H = &hb[(size_t)b * 9];
        if (ctx->nc == 6) {
            for (int mm = 0; mm < 6; ++mm) {
                double v = fU[(size_t)b * 9 + mm];
                if (ctx->activeflag_h[mm]) v += (mm >= 3 ? std::sqrt(0.5) : 1.0) * xe[(size_t)b * 9 + mm];
                H[3 * pi[mm] + pj[mm]] = v;
                H[3 * pj[mm] + pi[mm]] = v;
            }
        } else {
            for (int q = 0; q < 9; ++q) {
                double v = fU[(size_t)b * 9 + q];
                if (ctx->activeflag_h[q]) v += xe[(size_t)b * 9 + q];
                H[q] = v - ((q / 3 == q % 3) ? 1.0 : 0.0);
            }
        }
    }
    return DBFFT_OK;
}

dbfft_status dbfft_compatibility(dbfft_ctx* ctx, double* out) {
    if (!ctx || !out) return DBFFT_E_ARG;
    if (!ctx->have_solution) return fail(ctx, DBFFT_E_STATE, "no solution yet");
    cplx<double>* W = reinterpret_cast<cplx<double>*>(ctx->W);
    Ax1InvArgs<double> a1{ctx->dims, freq<double>(ctx), twid<double>(ctx), ctx->x64, nullptr, nullptr, W, nullptr,
                          ctx->pre};
    TRY(run(ctx, "pass1_grad_f64", (3 + ctx->nc) * cpass(ctx, true, ctx->B),
            [&] { return launch_grad<double>(AX1_PLAIN, a1, ctx->stream); }));
    const int nblk = (int)std::min<long long>(256, ctx->nblk_max);
    TRY(run(ctx, "compatibility", 0.0,
            [&] { return launch_compat(ctx->dims, freq<double>(ctx), W, ctx->partials, nblk, ctx->stream); }));
    std::vector<double> ph((size_t)ctx->B * nblk);
    CK(cudaMemcpyAsync(ph.data(), ctx->partials, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<double> hb;
    TRY(macro_hbar(ctx, hb));
    for (int b = 0; b < ctx->B; ++b) {
        double s = 0.0, h2 = 0.0;
        for (int k = 0; k < nblk; ++k) s += ph[(size_t)b * nblk + k];
        for (int q = 0; q < 9; ++q) h2 += hb[(size_t)b * 9 + q] * hb[(size_t)b * 9 + q];
        out[b] = h2 > 0.0 ? std::sqrt(s) / std::sqrt(h2) : std::sqrt(s);
    }
    return DBFFT_OK;
}

dbfft_status dbfft_displacement(dbfft_ctx* ctx, double* out) {
    if (!ctx || !out) return DBFFT_E_ARG;
    if (ctx->n3 & 1) return fail(ctx, DBFFT_E_UNSUPPORTED_GRID, "displacement output: even n3 only");
    std::vector<double> hb;
    TRY(macro_hbar(ctx, hb));
    CK(cudaMemcpyAsync(ctx->hbar, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // the fluctuation: inverse transforms of the three components of u-hat
    cplx<double>* W = reinterpret_cast<cplx<double>*>(ctx->W);
    CK(cudaMemcpyAsync(W, ctx->x64, (size_t)ctx->B * 3 * ctx->H * sizeof(cplx<double>), cudaMemcpyDeviceToDevice,
                       ctx->stream));
    Ax2Args<double> a2 = fft_args<double>(ctx, W, nullptr);
    a2.d.nc = 3;
    const double cp = cpass(ctx, true, ctx->B);
    TRY(run(ctx, "fft_ax2_f64", 2 * 3 * cp, [&] { return launch_fft_ax2<double>(+1, a2, ctx->stream); }));
    TRY(run(ctx, "fft_ax1_f64", 2 * 3 * cp, [&] { return launch_fft_ax1<double>(+1, a2, ctx->stream); }));
    Ax3Args<double> a3 = ax3_base<double>(ctx, W);
    a3.d.nc = 3;
    a3.radix = 4;
    a3.L = ax3_lines(ctx->n3, 3, ctx->RB, true, 1, 4);
    a3.pipe = 0;
    a3.macroW = ctx->hbar;
    a3.real_out = out;
    const double Ls[3] = {ctx->grid.L[0] > 0 ? ctx->grid.L[0] : 1.0, ctx->grid.L[1] > 0 ? ctx->grid.L[1] : 1.0,
                          ctx->grid.L[2] > 0 ? ctx->grid.L[2] : 1.0};
    a3.hx[0] = Ls[0] / ctx->n1;
    a3.hx[1] = Ls[1] / ctx->n2;
    a3.hx[2] = Ls[2] / ctx->n3;
    TRY(run(ctx, "pass3_displacement_f64", 3 * cp + (double)ctx->B * 3 * ctx->V * 8.0,
            [&] { return launch_ax3_post<double>(OP_DISP, a3, ctx->stream); }));
    CK(cudaStreamSynchronize(ctx->stream));
    return DBFFT_OK;
}

dbfft_status dbfft_apply(dbfft_ctx* ctx, int flags, const void* u_hat, const void* e_in, void* out, void* e_out) {
    if (!ctx || !u_hat || !out) return DBFFT_E_ARG;
    if (u_hat == out) return fail(ctx, DBFFT_E_ARG, "out may not alias u_hat");
    const bool f32 = (flags & DBFFT_APPLY_FP32) != 0;
    const double* ein = reinterpret_cast<const double*>(e_in);
    double* eout = reinterpret_cast<double*>(e_out);
    if (flags & DBFFT_APPLY_RESIDUAL) {
        if (f32) return fail(ctx, DBFFT_E_ARG, "the residual is formed in FP64 only");
        // copy e_in into the macro unknown buffer used by the residual chain
        std::vector<double> ru2, re2;
        if (ein) CK(cudaMemcpyAsync(ctx->xe_i, ein, ctx->B * 9 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        else CK(cudaMemsetAsync(ctx->xe_i, 0, ctx->B * 9 * sizeof(double), ctx->stream));
        cplx<double>* save = ctx->r64;
        ctx->r64 = reinterpret_cast<cplx<double>*>(out);
        dbfft_status s = chain_residual(ctx, reinterpret_cast<const cplx<double>*>(u_hat), ctx->xe_i, ru2, re2);
        ctx->r64 = save;
        TRY(s);
        if (eout) CK(cudaMemcpyAsync(eout, ctx->re64, ctx->B * 9 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return DBFFT_OK;
    }
    if (flags & DBFFT_APPLY_PRECOND) {
        TRY(run(ctx, "precond", 0.0, [&] {
            if (f32)
                return launch_precond_field<float>(ctx->dims, freq<float>(ctx), ctx->pre,
                                                   reinterpret_cast<const cplx<float>*>(u_hat),
                                                   reinterpret_cast<cplx<float>*>(out), ein, eout, ctx->stream);
            return launch_precond_field<double>(ctx->dims, freq<double>(ctx), ctx->pre,
                                                reinterpret_cast<const cplx<double>*>(u_hat),
                                                reinterpret_cast<cplx<double>*>(out), ein, eout, ctx->stream);
        }));
        CK(cudaStreamSynchronize(ctx->stream));
        return DBFFT_OK;
    }
    if (ctx->model != DBFFT_ISO_ELASTIC) {
        const bool stored64 = ctx->prec == DBFFT_FP64;
        if (stored64 == f32) return fail(ctx, DBFFT_E_STATE, "the tangent is stored in the other precision");
    }
    TRY(run(ctx, "macro", 0.0,
            [&] { return launch_macro(ctx->B, ctx->nc, ctx->activeflag, nullptr, ein, ctx->macroW, ctx->macroWf, ctx->stream); }));
    if (f32)
        TRY(chain_apply<float>(ctx, reinterpret_cast<const cplx<float>*>(u_hat), ctx->macroWf,
                               reinterpret_cast<cplx<float>*>(out), eout));
    else
        TRY(chain_apply<double>(ctx, reinterpret_cast<const cplx<double>*>(u_hat), ctx->macroW,
                                reinterpret_cast<cplx<double>*>(out), eout));
    CK(cudaStreamSynchronize(ctx->stream));
    return DBFFT_OK;
}

dbfft_status dbfft_homogenized_tangent(dbfft_ctx* ctx, double* out, dbfft_report* rep) {
    if (ctx) ctx->fwd_inc0 = false;  // the unit-strain solves replace the state
    if (!ctx || !out) return DBFFT_E_ARG;
    if (ctx->model != DBFFT_ISO_ELASTIC || ctx->nc != 6 || ctx->dims.ne != 0 || ctx->B != 6 * ctx->Bm)
        return fail(ctx, DBFFT_E_STATE, "homogenized tangent needs linear small strain, strain control, B = 6 n_materials");
    const auto t0 = std::chrono::steady_clock::now();
    if (rep) std::memset(rep, 0, sizeof(*rep));
    std::vector<double> tgt(ctx->B * 9, 0.0);
    static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
    for (int b = 0; b < ctx->B; ++b) {
        const int mm = b % 6;
        const double v = mm < 3 ? 1.0 : 1.0 / std::sqrt(2.0);  // unit Mandel strain
        tgt[b * 9 + 3 * pi[mm] + pj[mm]] = v;
        tgt[b * 9 + 3 * pj[mm] + pi[mm]] = v;
    }
    const int save_n = ctx->n_inc;
    ctx->n_inc = 1;
    dbfft_status s = set_load(ctx, 0, tgt.data());
    if (s == DBFFT_OK) s = solve_current(ctx, rep);
    ctx->n_inc = save_n;
    if (s != DBFFT_OK && s != DBFFT_E_NOT_CONVERGED) return s;
    std::vector<double> sg(ctx->B * 9);
    CK(cudaMemcpyAsync(sg.data(), ctx->sig0, sg.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int g = 0; g < ctx->Bm; ++g)
        for (int j = 0; j < 6; ++j)
            for (int i = 0; i < 6; ++i)
                out[(g * 6 + i) * 6 + j] = sg[(g * 6 + j) * 9 + i] * (i >= 3 ? std::sqrt(2.0) : 1.0);
    ctx->tangent_ready = s == DBFFT_OK;
    ctx->tangent_C.assign(out, out + (size_t)ctx->Bm * 36);
    TRY(set_load(ctx, 0, ctx->target.data()));
    if (rep) rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return s;
}

dbfft_status dbfft_adjoint(dbfft_ctx* ctx, const double* dJ_dsigma, double* dJ_dE, dbfft_report* rep) {
    if (!ctx || !dJ_dsigma || !dJ_dE) return DBFFT_E_ARG;
    if (ctx->model != DBFFT_ISO_ELASTIC || ctx->dims.ne != 0)
        return fail(ctx, DBFFT_E_STATE, "adjoint needs linear elastic phases under full strain control");
    if (ctx->n3 & 1) return fail(ctx, DBFFT_E_UNSUPPORTED_GRID, "adjoint: even n3 only");
    const auto t0 = std::chrono::steady_clock::now();
    if (rep) std::memset(rep, 0, sizeof(*rep));
    dbfft_report r1{}, r2{};
    // forward solve of increment 0, unless the context holds it already (a
    // dbfft_solve_increment(ctx, 0) that converged, or an earlier adjoint)
    ctx->tangent_ready = false;  // the solves below replace the state
    dbfft_status s = DBFFT_OK;
    if (!ctx->fwd_inc0) {
        TRY(set_load(ctx, 0, ctx->target.data()));
        s = solve_current(ctx, &r1);
        if (s != DBFFT_OK && s != DBFFT_E_NOT_CONVERGED) return s;
    }
    const bool fwd_ok = s == DBFFT_OK;
    const size_t nU = (size_t)ctx->B * 3 * ctx->H;
    if (!ctx->xfwd) TRY(dalloc_t(ctx, nU, &ctx->xfwd));
    if (!ctx->W2) TRY(dalloc(ctx, (size_t)ctx->B * ctx->nc * ctx->H * sizeof(cplx<double>), &ctx->W2));
    CK(cudaMemcpyAsync(ctx->xfwd, ctx->x64, nU * sizeof(cplx<double>), cudaMemcpyDeviceToDevice, ctx->stream));
    std::vector<double> fUfwd(ctx->B * 9);
    CK(cudaMemcpyAsync(fUfwd.data(), ctx->fU, fUfwd.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    // adjoint problem: strain control with macro strain g = sym(dJ/dsigma); lam' = its fluctuation
    std::vector<double> g(ctx->B * 9);
    for (int b = 0; b < ctx->B; ++b)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) g[b * 9 + 3 * i + j] = 0.5 * (dJ_dsigma[b * 9 + 3 * i + j] + dJ_dsigma[b * 9 + 3 * j + i]);
    const int save_n = ctx->n_inc;
    ctx->n_inc = 1;
    s = set_load(ctx, 0, g.data());
    if (s == DBFFT_OK) s = solve_current(ctx, &r2);
    ctx->n_inc = save_n;
    if (s != DBFFT_OK && s != DBFFT_E_NOT_CONVERGED) return s;
    // assembly: dJ/dE = (1/N) (g + B lam')(x) : C1 : (epsbar + B u)(x)
    CK(cudaMemcpyAsync(ctx->macroW2, ctx->fU, ctx->B * 9 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->macroW, fUfwd.data(), ctx->B * 9 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    cplx<double>* W = reinterpret_cast<cplx<double>*>(ctx->W);
    cplx<double>* W2 = reinterpret_cast<cplx<double>*>(ctx->W2);
    Ax1InvArgs<double> a1{ctx->dims, freq<double>(ctx), twid<double>(ctx), ctx->xfwd, nullptr, nullptr, W, nullptr, ctx->pre};
    Ax2Args<double> a2 = fft_args<double>(ctx, W, nullptr);
    TRY(run(ctx, "pass1_grad_f64", 0.0, [&] { return launch_grad<double>(AX1_PLAIN, a1, ctx->stream); }));
    TRY(run(ctx, "fft_ax2_f64", 0.0, [&] { return launch_fft_ax2<double>(+1, a2, ctx->stream); }));
    TRY(run(ctx, "fft_ax1_f64", 0.0, [&] { return launch_fft_ax1<double>(+1, a2, ctx->stream); }));
    Ax1InvArgs<double> b1{ctx->dims, freq<double>(ctx), twid<double>(ctx), ctx->x64, nullptr, nullptr, W2, nullptr, ctx->pre};
    Ax2Args<double> b2 = fft_args<double>(ctx, W2, nullptr);
    TRY(run(ctx, "pass1_grad_f64", 0.0, [&] { return launch_grad<double>(AX1_PLAIN, b1, ctx->stream); }));
    TRY(run(ctx, "fft_ax2_f64", 0.0, [&] { return launch_fft_ax2<double>(+1, b2, ctx->stream); }));
    TRY(run(ctx, "fft_ax1_f64", 0.0, [&] { return launch_fft_ax1<double>(+1, b2, ctx->stream); }));
    Ax3Args<double> a3 = ax3_base<double>(ctx, W);
    a3.L = ax3_lines(ctx->n3, ctx->nc, ctx->RB, true, 2, a3.radix);
    a3.W2 = W2;
    a3.macroW = ctx->macroW;
    a3.macroW2 = ctx->macroW2;
    a3.lam = ctx->lam1;
    a3.mu = ctx->mu1;
    a3.scale = nullptr;
    a3.dJdE = dJ_dE;
    TRY(run(ctx, "pass3_adjoint_f64", 0.0, [&] { return launch_ax3<double>(OP_ADJ, a3, ctx->stream); }));
    // restore the forward state
    CK(cudaMemcpyAsync(ctx->x64, ctx->xfwd, nU * sizeof(cplx<double>), cudaMemcpyDeviceToDevice, ctx->stream));
    TRY(set_load(ctx, 0, ctx->target.data()));
    std::vector<double> ru2, re2;
    TRY(chain_residual(ctx, ctx->x64, ctx->xe64, ru2, re2));  // restores sig0 of the forward solution
    ctx->fwd_inc0 = fwd_ok;
    if (rep) {
        rep->cg_iters = r1.cg_iters + r2.cg_iters;
        rep->cg_iters_max = std::max(r1.cg_iters_max, r2.cg_iters_max);
        rep->outer_iters = r1.outer_iters + r2.outer_iters + 1;
        rep->newton_iters = r1.newton_iters + r2.newton_iters;
        rep->true_rel_res = std::max(r1.true_rel_res, r2.true_rel_res);
        rep->eps_eq = std::max(r1.eps_eq, r2.eps_eq);
        rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return s;
}

dbfft_status dbfft_tangent_sensitivity(dbfft_ctx* ctx, const double* G, double* dJ_dE, double* C_eff,
                                       dbfft_report* rep) {
    if (!ctx || !G || !dJ_dE) return DBFFT_E_ARG;
    if (ctx->model != DBFFT_ISO_ELASTIC || ctx->nc != 6 || ctx->dims.ne != 0 || ctx->B != 6 * ctx->Bm)
        return fail(ctx, DBFFT_E_STATE,
                    "stiffness sensitivity needs linear small strain, strain control, B = 6 n_materials");
    if (ctx->n3 & 1) return fail(ctx, DBFFT_E_UNSUPPORTED_GRID, "stiffness sensitivity: even n3 only");
    const auto t0 = std::chrono::steady_clock::now();
    if (rep) std::memset(rep, 0, sizeof(*rep));
    // the six unit-strain solves of every map, unless the context holds them
    // (a converged dbfft_homogenized_tangent, or an earlier call of this one)
    std::vector<double> C((size_t)ctx->Bm * 36);
    if (!ctx->tangent_ready) {
        const dbfft_status s = dbfft_homogenized_tangent(ctx, C.data(), rep);
        if (s != DBFFT_OK) return s;
    } else {
        C = ctx->tangent_C;
    }
    const size_t nU = (size_t)ctx->B * 3 * ctx->H;
    if (!ctx->xfwd) TRY(dalloc_t(ctx, nU, &ctx->xfwd));
    if (!ctx->W2) TRY(dalloc(ctx, (size_t)ctx->B * ctx->nc * ctx->H * sizeof(cplx<double>), &ctx->W2));
    if (!ctx->sens_tmp) TRY(dalloc_t(ctx, (size_t)ctx->B * ctx->V, &ctx->sens_tmp));
    if (!ctx->sens_G) TRY(dalloc_t(ctx, (size_t)ctx->Bm * 36, &ctx->sens_G));
    CK(cudaMemcpyAsync(ctx->sens_G, G, (size_t)ctx->Bm * 36 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // dJ/dE(x) = (1/N) sum_I eps^I(x) : C1(x) : eta^I(x), eta^I = sum_J G_IJ eps^J: the
    // strain fields of the unit strains and their combinations, both through pass 3
    // (C_IJ = (1/N) sum_x eps^I : C : eps^J is stationary in the fluctuations, so no
    // adjoint solve is needed: the adjoint fields are the forward ones)
    TRY(run(ctx, "combine6", 0.0, [&] { return launch_combine6(ctx->x64, ctx->sens_G, ctx->xfwd, 3 * ctx->H, ctx->Bm,
                                                             ctx->stream); }));
    std::vector<double> mw((size_t)ctx->B * 9, 0.0), mw2((size_t)ctx->B * 9, 0.0);
    for (int b = 0; b < ctx->B; ++b) mw[b * 9 + b % 6] = b % 6 < 3 ? 1.0 : 0.70710678118654752440084436210485;
    for (int g = 0; g < ctx->Bm; ++g)
        for (int I = 0; I < 6; ++I)
            for (int J = 0; J < 6; ++J) mw2[(g * 6 + I) * 9 + J] = G[(g * 6 + I) * 6 + J] * mw[(g * 6 + J) * 9 + J];
    CK(cudaMemcpyAsync(ctx->macroW, mw.data(), mw.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->macroW2, mw2.data(), mw2.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    cplx<double>* W = reinterpret_cast<cplx<double>*>(ctx->W);
    cplx<double>* W2 = reinterpret_cast<cplx<double>*>(ctx->W2);
    Ax1InvArgs<double> a1{ctx->dims, freq<double>(ctx), twid<double>(ctx), ctx->x64, nullptr, nullptr, W, nullptr, ctx->pre};
    Ax2Args<double> a2 = fft_args<double>(ctx, W, nullptr);
    TRY(run(ctx, "pass1_grad_f64", 0.0, [&] { return launch_grad<double>(AX1_PLAIN, a1, ctx->stream); }));
    TRY(run(ctx, "fft_ax2_f64", 0.0, [&] { return launch_fft_ax2<double>(+1, a2, ctx->stream); }));
    TRY(run(ctx, "fft_ax1_f64", 0.0, [&] { return launch_fft_ax1<double>(+1, a2, ctx->stream); }));
    Ax1InvArgs<double> b1{ctx->dims, freq<double>(ctx), twid<double>(ctx), ctx->xfwd, nullptr, nullptr, W2, nullptr, ctx->pre};
    Ax2Args<double> b2 = fft_args<double>(ctx, W2, nullptr);
    TRY(run(ctx, "pass1_grad_f64", 0.0, [&] { return launch_grad<double>(AX1_PLAIN, b1, ctx->stream); }));
    TRY(run(ctx, "fft_ax2_f64", 0.0, [&] { return launch_fft_ax2<double>(+1, b2, ctx->stream); }));
    TRY(run(ctx, "fft_ax1_f64", 0.0, [&] { return launch_fft_ax1<double>(+1, b2, ctx->stream); }));
    Ax3Args<double> a3 = ax3_base<double>(ctx, W);
    a3.L = ax3_lines(ctx->n3, ctx->nc, ctx->RB, true, 2, a3.radix);
    a3.W2 = W2;
    a3.macroW = ctx->macroW;
    a3.macroW2 = ctx->macroW2;
    a3.lam = ctx->lam1;
    a3.mu = ctx->mu1;
    a3.scale = nullptr;
    a3.dJdE = ctx->sens_tmp;
    TRY(run(ctx, "pass3_adjoint_f64", 0.0, [&] { return launch_ax3<double>(OP_ADJ, a3, ctx->stream); }));
    TRY(run(ctx, "sum6", 0.0, [&] { return launch_sum6(ctx->sens_tmp, dJ_dE, ctx->V, ctx->Bm, ctx->stream); }));
    TRY(set_load(ctx, 0, ctx->target.data()));  // the context's own macro fields again
    CK(cudaStreamSynchronize(ctx->stream));
    if (C_eff) std::memcpy(C_eff, C.data(), C.size() * sizeof(double));
    if (rep) rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return DBFFT_OK;
}

dbfft_status dbfft_set_checkpointing(dbfft_ctx* ctx, int enable) {
    if (!ctx) return DBFFT_E_ARG;
    if (ctx->model != DBFFT_CP_FCC_POWERLAW)
        return fail(ctx, DBFFT_E_STATE, "checkpoints are kept for the small-strain crystal-plasticity model");
    if (enable && ctx->cur_inc >= 0)
        return fail(ctx, DBFFT_E_STATE, "enable checkpoints before the first increment");
    ctx->ckpt_on = enable != 0;
    ctx->ckpt_n = 0;
    return DBFFT_OK;
}

dbfft_status dbfft_cp_adjoint(dbfft_ctx* ctx, const double* dJ_dsigma, double* dJ_ds, dbfft_report* rep) {
    if (!ctx || !dJ_dsigma || !dJ_ds) return DBFFT_E_ARG;
    if (ctx->model != DBFFT_CP_FCC_POWERLAW || ctx->prec != DBFFT_FP64)
        return fail(ctx, DBFFT_E_STATE, "the increment adjoint needs the small-strain crystal-plasticity model in FP64");
    if (ctx->n3 & 1) return fail(ctx, DBFFT_E_UNSUPPORTED_GRID, "increment adjoint: even n3 only");
    if (!ctx->ckpt_on || ctx->cur_inc < 0 || ctx->ckpt_n != ctx->cur_inc + 1)
        return fail(ctx, DBFFT_E_STATE, "no checkpoint of every increment up to the current one");
    const auto t0 = std::chrono::steady_clock::now();
    if (rep) std::memset(rep, 0, sizeof(*rep));
    ctx->fwd_inc0 = false;
    ctx->tangent_ready = false;
    const size_t per = (size_t)ctx->B * ctx->V * 6;
    const size_t nU = (size_t)ctx->B * 3 * ctx->H;
    if (!ctx->adj_q) TRY(dalloc_t(ctx, per, &ctx->adj_q));
    if (!ctx->adj_w) TRY(dalloc_t(ctx, per, &ctx->adj_w));
    if (!ctx->adj_a) TRY(dalloc_t(ctx, (size_t)ctx->B * 6, &ctx->adj_a));
    if (!ctx->xfwd) TRY(dalloc_t(ctx, nU, &ctx->xfwd));
    CK(cudaMemsetAsync(ctx->adj_q, 0, per * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(dJ_ds, 0, (size_t)ctx->B * ctx->V * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(ctx->errw, 0, sizeof(unsigned), ctx->stream));
    // the forward state, restored at the end
    CK(cudaMemcpyAsync(ctx->xfwd, ctx->x64, nU * sizeof(cplx<double>), cudaMemcpyDeviceToDevice, ctx->stream));
    std::vector<double> xe_save((size_t)ctx->B * 9), sig0_save((size_t)ctx->B * 9);
    CK(cudaMemcpyAsync(xe_save.data(), ctx->xe64, xe_save.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(sig0_save.data(), ctx->sig0, sig0_save.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    // a = sym(dJ/dsigma) / N in Mandel components at the last increment
    static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
    std::vector<double> a_last((size_t)ctx->B * 6), a_zero((size_t)ctx->B * 6, 0.0);
    for (int b = 0; b < ctx->B; ++b)
        for (int m = 0; m < 6; ++m) {
            const double gs = 0.5 * (dJ_dsigma[b * 9 + 3 * pi[m] + pj[m]] + dJ_dsigma[b * 9 + 3 * pj[m] + pi[m]]);
            a_last[b * 6 + m] = (m < 3 ? gs : std::sqrt(2.0) * gs) * ctx->dims.invN;
        }
    cplx<double>* W = reinterpret_cast<cplx<double>*>(ctx->W);
    double* tan = reinterpret_cast<double*>(ctx->tan);
    long long it_sum = 0;
    int it_max = 0;
    for (int n = ctx->cur_inc; n >= 0; --n) {
        const double* sig_n = ctx->ckpt + per * n;
        CK(cudaMemcpyAsync(ctx->adj_a, (n == ctx->cur_inc ? a_last : a_zero).data(), a_last.size() * sizeof(double),
                           cudaMemcpyHostToDevice, ctx->stream));
        // w = q + T_n (a - S q), and T_n as the context's tangent
        TRY(run(ctx, "cp_adjoint_pre", 0.0, [&] {
            return launch_cp_adj(0, ctx->B, ctx->Rm, ctx->V, ctx->phase, ctx->grains, ctx->cp, sig_n, ctx->adj_q,
                                 ctx->adj_a, ctx->adj_w, tan, nullptr, ctx->errw, 1, ctx->stream);
        }));
        TRY(refresh_precond(ctx));
        // right-hand side B^H w: the real field through R2C, the forward transforms and the divergence
        Ax3Args<double> a3 = ax3_base<double>(ctx, W);
        a3.zero_in = 1;
        a3.real_in = ctx->adj_w;
        a3.macroW = ctx->macroW;
        TRY(run(ctx, "pass3_loadw_f64", 0.0, [&] { return launch_ax3_post<double>(OP_LOADW, a3, ctx->stream); }));
        Ax2Args<double> a2 = fft_args<double>(ctx, W, nullptr);
        TRY(run(ctx, "fft_ax1_f64", 0.0, [&] { return launch_fft_ax1<double>(-1, a2, ctx->stream); }));
        TRY(run(ctx, "fft_ax2_f64", 0.0, [&] { return launch_fft_ax2<double>(-1, a2, ctx->stream); }));
        Ax1FwdArgs<double> a5;
        std::memset(&a5, 0, sizeof(a5));
        a5.d = ctx->dims;
        a5.f = freq<double>(ctx);
        a5.tw = twid<double>(ctx);
        a5.W = W;
        a5.out = ctx->r64;
        a5.e_out = ctx->re64;
        TRY(run(ctx, "pass5_div_f64", 0.0, [&] { return launch_div<double>(AX5_PLAIN, a5, ctx->stream); }));
        TRY(run(ctx, "hermitian_planes", 0.0, [&] { return launch_herm_planes<double>(ctx->dims, ctx->r64, ctx->stream); }));
        // K_n lam = B^H w by PCG in FP64 (x = 0 start, tolerance grid.tol)
        CK(cudaMemsetAsync(ctx->x64, 0, nU * sizeof(cplx<double>), ctx->stream));
        CK(cudaMemsetAsync(ctx->xe64, 0, (size_t)ctx->B * 9 * sizeof(double), ctx->stream));
        TRY(set_scales(ctx, std::vector<double>(ctx->B, 1.0)));
        TRY(run(ctx, "to_inner", 0.0, [&] {
            return launch_to_inner<double>(ctx->dims, ctx->r64, ctx->re64, ctx->scal,
                                           reinterpret_cast<cplx<double>*>(ctx->ri), ctx->re_i,
                                           reinterpret_cast<cplx<double>*>(ctx->xi), ctx->xe_i, ctx->stream);
        }));
        int itm = 0;
        TRY(inner_cg<double>(ctx, ctx->grid.tol, it_sum, itm));
        it_max = std::max(it_max, itm);
        TRY(run(ctx, "from_inner", 0.0, [&] {
            return launch_from_inner<double>(ctx->dims, reinterpret_cast<const cplx<double>*>(ctx->xi),
                                             reinterpret_cast<const cplx<double>*>(ctx->pi), ctx->cg, ctx->xe_i,
                                             ctx->scal, ctx->x64, ctx->xe64, ctx->stream);
        }));
        // e_lam = B lam as a real field (fluctuation and macro part)
        TRY(run(ctx, "macro", 0.0, [&] {
            return launch_macro(ctx->B, ctx->nc, ctx->activeflag, nullptr, ctx->xe64, ctx->macroW, ctx->macroWf,
                                ctx->stream);
        }));
        Ax1InvArgs<double> a1{ctx->dims, freq<double>(ctx), twid<double>(ctx), ctx->x64, nullptr, nullptr, W, nullptr,
                              ctx->pre};
        TRY(run(ctx, "pass1_grad_f64", 0.0, [&] { return launch_grad<double>(AX1_PLAIN, a1, ctx->stream); }));
        TRY(run(ctx, "fft_ax2_f64", 0.0, [&] { return launch_fft_ax2<double>(+1, a2, ctx->stream); }));
        TRY(run(ctx, "fft_ax1_f64", 0.0, [&] { return launch_fft_ax1<double>(+1, a2, ctx->stream); }));
        Ax3Args<double> b3 = ax3_base<double>(ctx, W);
        b3.real_out = ctx->adj_w;
        b3.macroW = ctx->macroW;
        TRY(run(ctx, "pass3_storew_f64", 0.0, [&] { return launch_ax3_post<double>(OP_STOREW, b3, ctx->stream); }));
        // dJ/ds += d . T_n S sigma_n + q . S sigma_n, q = -T_n d
        TRY(run(ctx, "cp_adjoint_post", 0.0, [&] {
            return launch_cp_adj(1, ctx->B, ctx->Rm, ctx->V, ctx->phase, ctx->grains, ctx->cp, sig_n, ctx->adj_q,
                                 ctx->adj_a, ctx->adj_w, nullptr, dJ_ds, ctx->errw, 0, ctx->stream);
        }));
    }
    unsigned errh = 0;
    CK(cudaMemcpyAsync(&errh, ctx->errw, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    // the forward state again: solution, macro fields, mean stress and the tangent of the
    // last increment (from its checkpoint; a constitutive update here would start a new step)
    CK(cudaMemcpyAsync(ctx->x64, ctx->xfwd, nU * sizeof(cplx<double>), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->xe64, xe_save.data(), xe_save.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->sig0, sig0_save.data(), sig0_save.size() * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->stream));
    TRY(set_load(ctx, ctx->cur_inc, ctx->target.data()));
    TRY(run(ctx, "cp_adjoint_pre", 0.0, [&] {
        return launch_cp_adj(0, ctx->B, ctx->Rm, ctx->V, ctx->phase, ctx->grains, ctx->cp, ctx->ckpt + per * ctx->cur_inc,
                             ctx->adj_q, ctx->adj_a, ctx->adj_w, tan, nullptr, ctx->errw, 0, ctx->stream);
    }));
    CK(cudaStreamSynchronize(ctx->stream));
    if (errh & 1u) return fail(ctx, DBFFT_E_MATERIAL, "a checkpoint gave a tangent that is not positive definite");
    if (rep) {
        rep->cg_iters = it_sum;
        rep->cg_iters_max = it_max;
        rep->outer_iters = ctx->cur_inc + 1;
        rep->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return DBFFT_OK;
}

}  // extern "C"
