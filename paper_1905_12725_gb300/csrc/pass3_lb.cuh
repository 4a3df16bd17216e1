// pass3_lb.cuh -- axis-3 pass of the FP32 CG operator applications for the
// long lines (n3 = 64, 128, 256), built to cut the instructions per voxel:
//
//  * data movement by the copy engine only: for one (right-hand side,
//    component) the half-spectrum lines of a tile of L grid lines are
//    L (n3/2 + 1) contiguous complex values in global memory and stay
//    contiguous in shared memory, so each moves as one bulk copy (in, and out
//    again after the R2C); the phase ids of the tile come the same way;
//  * every transform works in place inside its own line buffer, so shared
//    memory holds only the tile;
//  * the half-length complex transform (M = n3/2 = R x P values, P threads
//    per line, R values per thread) has exactly two register stages and one
//    exchange. Inverse: stage A is P DFTs of length R over x[n2 + P n1]
//    (thread p = n2), stage B is R DFTs of length P over n2, G = R / P of them
//    per thread (k1 = G p + g); the forward transform runs the same stages in
//    the transposed order. The exchange moves G complex values (16 or 32
//    bytes) per access through an XOR-swizzled chunk layout that keeps the
//    P threads of a line on distinct banks;
//  * twiddles are registers: the stage-B factors W_M^(n2 k1) of a thread are
//    read once per CTA, the pre/post factors e^(-2 pi i k / n3) of
//    k = p + P r are one per-thread value times compile-time constants;
//  * the pre- and post-processing take each (k, M - k) pair once: a thread
//    forms both values of its pairs and hands the partner thread (P - p)
//    its half by shuffle;
//  * the per-voxel operation reads and writes four voxels per access, and the
//    isotropic contraction runs two voxels per packed FP32x2 instruction
//    (complex sums and differences everywhere are packed too, fft.cuh);
//  * the 2 (n3 = 256) or 4 (n3 = 64, 128) line slots that share a half-warp
//    sit 8 (or 4) line buffers apart; a line buffer is 8 bytes long modulo
//    128, so they are 64 (or 32) bytes apart modulo 128 and the 64-bit
//    accesses of the C2R/R2C pre- and post-processing are free of bank
//    conflicts.
//
// Real transform of length n via the half-length complex transform, as in
// pass3.cuh:
//   C2R: Z[k] = (X[k] + conj X[M-k]) + i e^{+2 pi i k/n} (X[k] - conj X[M-k]),
//        z = IDFT_M(Z), x[2j] = Re z[j], x[2j+1] = Im z[j];
//   R2C: Z = DFT_M(z), X[k] = (Z[k] + conj Z[M-k]) / 2
//                            - (i/2) e^{-2 pi i k/n} (Z[k] - conj Z[M-k]).
// Alignment: a bulk copy needs 16-byte aligned addresses and sizes; a line
// is (M + 1) * 8 bytes, 8 modulo 16, so L must be even (and divide n1 n2).
// Inside an odd line buffer the exchange and the real line start 8 bytes in,
// which keeps every 16-byte access aligned.
#pragma once
#include "pass3_pipe.cuh"
#include "tma.cuh"

namespace dbfft {

// values per thread (stage-A radix) and threads per line of the half-length transform
template <int M> struct LbShape;
template <> struct LbShape<128> { static constexpr int R = 16, P = 8; };
template <> struct LbShape<64> { static constexpr int R = 16, P = 4; };
template <> struct LbShape<32> { static constexpr int R = 8, P = 4; };

// Shared-memory plan of one CTA (bytes), shared by host and device:
// [RB][NC][L] line buffers of M + 1 complex values, phase ids [L][N3],
// the optional per-voxel scale [L][N3], one mbarrier.
template <int N3>
struct LbPlan {
    static constexpr int M = N3 / 2;
    static constexpr int H = M + 1;
    __host__ __device__ static constexpr long long field_bytes(int L, int RB, int NC) {
        return (long long)RB * NC * L * H * 8;
    }
    __host__ __device__ static constexpr long long phase_bytes(int L) { return ((long long)L * N3 * 2 + 15) / 16 * 16; }
    __host__ __device__ static constexpr long long scale_bytes(int L, bool sc) { return sc ? (long long)L * N3 * 4 : 0; }
    __host__ __device__ static constexpr long long total_bytes(int L, int RB, int NC, bool sc) {
        return field_bytes(L, RB, NC) + phase_bytes(L) + scale_bytes(L, sc) + 16;
    }
};

// Threads per CTA: every (padded) line slot gets P threads, in as few rounds
// as keep the CTA at or below max_thr (at most 384) threads.
template <int N3>
__host__ __device__ constexpr int lb_threads(int nslot, int max_thr = 384) {
    constexpr int P = LbShape<N3 / 2>::P;
    const int cap = max_thr > 0 && max_thr < 384 ? max_thr : 384;
    const int ns16 = (nslot + 15) / 16 * 16;
    for (int rounds = 1; rounds <= ns16; ++rounds) {
        const int groups = (ns16 + rounds - 1) / rounds;
        const int thr = (groups * P + 31) / 32 * 32;
        if (thr <= cap) return thr;
    }
    return 32;
}

// line slot of group gi: inside each block of 16 slots, the GH = 16 / P groups
// of one half-warp take slots P apart
template <int P>
__device__ __forceinline__ int lb_slot(int gi) {
    constexpr int GH = 16 / P;
    const int w = gi & 15;
    return (gi & ~15) + w / GH + P * (w % GH);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// WL (warp lines): every warp takes its own lines alone through C2R,
// contraction and R2C, so only warp barriers separate the phases.
//  WL = 1: a tile of 16 lines, P warps; warp w owns the 16 / P lines w + P j,
//          a half-warp does one (rhs, component) slot of each of them per round;
//          they are P line buffers apart (64 or 32 bytes modulo 128).
//  WL = 2: a tile of L = P lines, L / 2 warps; warp w owns lines 2w and 2w + 1
//          (one per half-warp), a half-warp does 16 / P components of its line
//          per round; those are L line buffers apart (again 64 or 32 bytes
//          modulo 128). Smaller CTAs, more of them per SM.
// Either way the 64-bit accesses of a half-warp are free of bank conflicts.
template <int N3, int NC, int OPK, int WL = 0>
__global__ void __launch_bounds__(WL == 0 ? 384 : (WL == 1 ? 256 : 128), WL == 2 ? 4 : 2) k_axis3_lb(Ax3Args<float> a) {
    using T = float;
    static_assert(OpInfo<OPK>::apply, "the line-bulk pass serves the CG applications");
    constexpr int M = N3 / 2;
    constexpr int H = M + 1;
    constexpr int R = LbShape<M>::R;
    constexpr int P = LbShape<M>::P;
    constexpr int G = R / P;  // stage-B transforms (and exchange chunk, complex values) per thread
    static_assert(R * P == M && G * P == R && (G == 2 || G == 4), "supported line shapes");
    using Plan = LbPlan<N3>;
    extern __shared__ __align__(16) unsigned char smlb[];
    __shared__ double red[32];  // block_sum<1> scratch (kept small: four CTAs per SM at 8-line tiles)
    __shared__ double s_eacc[8];
    __shared__ float s_macro[8 * 9];
    __shared__ bool is_last;
    __shared__ int s_abort;

    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    const Dims& d = a.d;
    const int RB = a.RB, L = a.L;
    const int t = threadIdx.x, nthr = blockDim.x, lane = t & 31;
    const int g = blockIdx.y;
    const long long nlines = (long long)d.n1 * d.n2;
    const long long line0 = (long long)blockIdx.x * L;
    const int mat = (g * RB) / d.Rm;
    const bool has_scale = a.scale != nullptr;
    unsigned done_mask = 0;
    if (a.cg != nullptr)
        for (int rl = 0; rl < RB; ++rl) done_mask |= (a.cg[g * RB + rl].done != 0 ? 1u : 0u) << rl;
    if (a.cg != nullptr && done_mask == (1u << RB) - 1u) return;  // the whole group has stopped

    cplx<T>* lines = reinterpret_cast<cplx<T>*>(smlb);
    const uint16_t* phs = reinterpret_cast<const uint16_t*>(smlb + Plan::field_bytes(L, RB, NC));
    const T* scs = reinterpret_cast<const T*>(smlb + Plan::field_bytes(L, RB, NC) + Plan::phase_bytes(L));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smlb + Plan::total_bytes(L, RB, NC, has_scale) - 16);

    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        s_abort = 0;
        const uint32_t chunk = (uint32_t)((long long)L * H * 8);
        uint32_t tx = (uint32_t)(Plan::phase_bytes(L) + Plan::scale_bytes(L, has_scale));
        for (int rl = 0; rl < RB; ++rl)
            if (!((done_mask >> rl) & 1u)) tx += chunk * NC;
        mbar_arrive_expect_tx(bar, tx);
        for (int rl = 0; rl < RB; ++rl) {
            if ((done_mask >> rl) & 1u) continue;
            const int b = g * RB + rl;
            for (int c = 0; c < NC; ++c)
                bulk_load(smlb + (long long)(rl * NC + c) * chunk, a.W + ((long long)(b * NC + c) * nlines + line0) * H,
                          chunk, bar);
        }
        bulk_load(smlb + Plan::field_bytes(L, RB, NC), a.phase + (long long)mat * d.V + line0 * N3,
                  (uint32_t)Plan::phase_bytes(L), bar);
        if (has_scale)
            bulk_load(smlb + Plan::field_bytes(L, RB, NC) + Plan::phase_bytes(L),
                      a.scale + (long long)mat * d.V + line0 * N3, (uint32_t)Plan::scale_bytes(L, true), bar);
        // a short, exactly counted limit (a test setting) polls right after the issue
        if (a.wait_limit > 0 && !mbar_poll_bounded(bar, 0u, a.wait_limit)) s_abort = 1;
    }
    for (int i = t; i < RB * 9; i += nthr) s_macro[i] = a.macroW[(long long)g * RB * 9 + i];
    if (t < 8) s_eacc[t] = 0.0;

    // per-thread twiddles (independent of the line), read at the start of each
    // transform phase: stage B needs W_M^(n2 (G p + g)) = W_M^(n2 G p) W_M^(n2 g)
    // for n2 = 1..P-1 (forward sign; the inverse conjugates), the first factor
    // from the table, the second a compile-time constant; and e^(-2 pi i p / n3)
    const int p = t % P;
    cplx<T> twB[P - 1];
    auto load_twB = [&]() {
#pragma unroll
        for (int n2 = 1; n2 < P; ++n2) twB[n2 - 1] = ldg_c(a.tw.tm + (n2 * G * p) % M);
    };
    const cplx<T> ep = ldg_c(a.tw.t3 + p);

    __syncthreads();  // the mbarrier is initialised before anyone waits on it
    // the wait: at most 2^26 blocking polls (unless the short limit above ran out)
    if (!s_abort && !mbar_wait_bounded(bar, 0u)) s_abort = 1;
    __syncthreads();
    if (s_abort) {  // a wait gave up: record it and let the copies land (bounded wait);
                    // the CTA still takes part in the curvature reduction below
        if (t == 0) {
            if (a.err) atomicOr(a.err, 2u);
            mbar_wait_bounded(bar, 0u);
        }
    } else {

    const int nslot = RB * NC * L;
    const int ngr = nthr / P;  // line slots per round
    const int warp = t >> 5;
    constexpr int GH = 16 / P;  // line slots (groups) per half-warp
    const int nrounds = WL == 1   ? (RB * NC + 1) / 2
                        : WL == 2 ? (RB * NC + GH - 1) / GH
                                  : ((nslot + 15) / 16 * 16 + ngr - 1) / ngr;
    // slot -> (ok, line buffer); the aligned region of an odd slot starts 8 bytes in
    auto slot_of = [&](int rd, bool& ok, int& sig) {
        if constexpr (WL == 1) {
            const int cs = 2 * rd + (lane >> 4);            // (rhs, component) slot of this half-warp
            const int ll = warp + P * ((lane & 15) / P);    // one of the warp's lines
            sig = cs * L + ll;
            ok = cs < RB * NC && !((done_mask >> (cs / NC)) & 1u);
        } else if constexpr (WL == 2) {
            const int cs = GH * rd + (lane & 15) / P;       // one of this half-warp's components
            const int ll = 2 * warp + (lane >> 4);          // the half-warp's line
            sig = cs * L + ll;
            ok = cs < RB * NC && !((done_mask >> (cs / NC)) & 1u);
        } else {
            sig = lb_slot<P>(rd * ngr + t / P);
            ok = sig < nslot && !((done_mask >> (sig / (NC * L))) & 1u);
        }
        if (!ok) sig = 0;
    };
    auto phase_sync = [&]() {
        if constexpr (WL != 0) __syncwarp();
        else __syncthreads();
    };

    // ---------------------------------------------------------------- C2R
    load_twB();
    for (int rd = 0; rd < nrounds; ++rd) {
        bool ok;
        int sig;
        slot_of(rd, ok, sig);
        cplx<T>* line = lines + (long long)sig * H;
        T* xr = reinterpret_cast<T*>(line + (sig & 1));  // aligned exchange / real line
        cplx<T> v[R];
        // Z[k], k = p + P r, and Z[M - k] from the same pair: with S = X[k] + conj X[M-k],
        // Q = e^{+2 pi i k / n3} (X[k] - conj X[M-k]) (e = conj(ep) conj(e^{-2 pi i P r / n3})),
        // Z[k] = S + i Q and Z[M - k] = conj(S) + i conj(Q). Each thread takes the pairs of
        // its registers r < R/2; Z[M - k] is register R - 1 - r of the partner thread P - p,
        // which receives it by shuffle. Thread 0 is its own partner: its Z[M - P r] is its
        // register R - r (moved into place below), Z[M/2] = 2 conj X[M/2] is computed apart,
        // and the r = 0 pair (k = 0 with the Nyquist value X[M]) has no partner register.
        const int partner = (lane & ~(P - 1)) | ((P - p) & (P - 1));
        sfor<0, R / 2>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            const int k = p + P * r;
            const cplx<T> X = line[k];
            const cplx<T> Xc = conjg(line[M - k]);
            const cplx<T> e = conjg(ep * tw_const<T, N3, P * r>());
            const cplx<T> S = X + Xc, Q = e * (X - Xc);
            v[r] = S + mk(-Q.y, Q.x);
            const cplx<T> zp = mk(S.x + Q.y, Q.x - S.y);
            v[R - 1 - r].x = __shfl_sync(0xffffffffu, zp.x, partner);
            v[R - 1 - r].y = __shfl_sync(0xffffffffu, zp.y, partner);
        });
        {
            const bool p0 = p == 0;
#pragma unroll
            for (int j = R - 1; j > R / 2; --j) v[j] = p0 ? v[j - 1] : v[j];
            const cplx<T> xm = line[M / 2];
            if (p0) v[R / 2] = mk(T(2) * xm.x, T(-2) * xm.y);
        }
        __syncwarp();
        RegDFT<R, +1, 1, 0, T>::run(v);  // stage A over n1; v[k1] = Y[n2 = p][k1]
        // exchange: block n2 = p, chunk c (k1 = cG .. cG + G - 1) at slot n2 P + (c ^ n2)
        if (ok) {
#pragma unroll
            for (int c = 0; c < P; ++c) {
                T* dst = xr + 2 * G * (p * P + (c ^ p));
#pragma unroll
                for (int h = 0; h < G / 2; ++h)
                    st4(dst + 4 * h, make_float4(v[c * G + 2 * h].x, v[c * G + 2 * h].y, v[c * G + 2 * h + 1].x,
                                                 v[c * G + 2 * h + 1].y));
            }
        }
        __syncwarp();
#pragma unroll
        for (int n2 = 0; n2 < P; ++n2) {  // chunk p of every block: v[g + G n2] = Y[n2][G p + g]
            const T* src = xr + 2 * G * (n2 * P + (p ^ n2));
#pragma unroll
            for (int h = 0; h < G / 2; ++h) {
                const float4 q = ld4(src + 4 * h);
                v[2 * h + G * n2] = mk(q.x, q.y);
                v[2 * h + 1 + G * n2] = mk(q.z, q.w);
            }
        }
        // stage B: twiddle W_M^{-n2 k1} (inverse), DFT of length P over n2
        sfor<1, P>([&](auto nc) {
            constexpr int n2 = decltype(nc)::value;
            sfor<0, G>([&](auto gc) {
                constexpr int gg = decltype(gc)::value;
                v[gg + G * n2] = v[gg + G * n2] * conjg(twB[n2 - 1]);
                if constexpr (gg > 0) v[gg + G * n2] = v[gg + G * n2] * conjg(tw_const<T, M, n2 * gg>());
            });
        });
        sfor<0, G>([&](auto gc) { RegDFT<P, +1, G, decltype(gc)::value, T>::run(v); });
        __syncwarp();
        // z[j], j = G p + g + R k2 -> reals x[2j], x[2j+1]
        if (ok) {
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) {
                T* dst = xr + 2 * (G * p + R * k2);
#pragma unroll
                for (int h = 0; h < G / 2; ++h)
                    st4(dst + 4 * h, make_float4(v[2 * h + G * k2].x, v[2 * h + G * k2].y, v[2 * h + 1 + G * k2].x,
                                                 v[2 * h + 1 + G * k2].y));
            }
        }
    }
    phase_sync();

    // ---------------------------------------------------------------- per-voxel operation
    // one right-hand side at a time (its curvature share is reduced before the next)
    for (int rr = 0; rr < RB; ++rr) {
        if ((done_mask >> rr) & 1u) continue;
        constexpr int Q4 = N3 / 4;
        const int CS = 2 * L * H;  // floats between the components of one line
        T en = T(0);
        // all lines of the tile (block-strided), or the warp's own 16 / P lines (lane-strided)
        const int it0 = WL ? lane : t, itn = WL == 1 ? (16 / P) * Q4 : (WL == 2 ? 2 * Q4 : L * Q4);
        const int its = WL ? 32 : nthr;
        float2 mac[NC];  // the macro strain of this right-hand side, in both lanes (warp-lines forms;
                         // the 384-thread form rereads it, having no registers to spare)
#pragma unroll
        for (int q = 0; q < NC; ++q) mac[q] = make_float2(s_macro[rr * 9 + q], s_macro[rr * 9 + q]);
        auto macro_of = [&](int q) {
            return WL == 0 ? make_float2(s_macro[rr * 9 + q], s_macro[rr * 9 + q]) : mac[q];
        };
        for (int it = it0; it < itn; it += its) {
            const int ll = WL == 1 ? warp + P * (it / Q4) : (WL == 2 ? 2 * warp + it / Q4 : it / Q4);
            const int x4 = (it % Q4) * 4;
            const uint2 pp = *reinterpret_cast<const uint2*>(phs + ll * N3 + x4);
            const float4 s4 = has_scale ? ld4(scs + ll * N3 + x4) : make_float4(1.f, 1.f, 1.f, 1.f);
            const int sig0 = (rr * NC) * L + ll;  // component 0; all components share its parity
            T* f = reinterpret_cast<T*>(lines + (long long)sig0 * H + (sig0 & 1)) + x4;
            if constexpr (OPK == OP_ISO) {
                // two voxels per packed instruction: lanes (x, y) and (z, w) of the
                // float4 of each component are neighbouring voxels
                static_assert(NC == 6, "small-strain isotropic contraction");
                float4 e4[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) e4[q] = ld4(f + q * CS);
                float2* ev = reinterpret_cast<float2*>(e4);
                const float2 two = make_float2(2.f, 2.f);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const unsigned pw = h == 0 ? pp.x : pp.y;
                    const float2 sc = h == 0 ? make_float2(s4.x, s4.y) : make_float2(s4.z, s4.w);
                    const float2 lam = __fmul2_rn(make_float2(__ldg(a.lam + (pw & 0xffffu)), __ldg(a.lam + (pw >> 16))), sc);
                    const float2 mu2 = __fmul2_rn(
                        __fmul2_rn(make_float2(__ldg(a.mu + (pw & 0xffffu)), __ldg(a.mu + (pw >> 16))), sc), two);
                    float2 e[NC];
#pragma unroll
                    for (int q = 0; q < NC; ++q) e[q] = __fadd2_rn(ev[2 * q + h], macro_of(q));
                    const float2 ltr = __fmul2_rn(lam, __fadd2_rn(__fadd2_rn(e[0], e[1]), e[2]));
                    float2 en_n = make_float2(0.f, 0.f), en_s = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float2 sg = __ffma2_rn(mu2, e[q], ltr);  // lambda tr + 2 mu e
                        en_n = __ffma2_rn(e[q], sg, en_n);
                        ev[2 * q + h] = sg;
                    }
#pragma unroll
                    for (int q = 3; q < 6; ++q) {
                        const float2 sg = __fmul2_rn(mu2, e[q]);  // 2 mu e (shear, Mandel weight 2 in the energy)
                        en_s = __ffma2_rn(e[q], sg, en_s);
                        ev[2 * q + h] = sg;
                    }
                    en += (en_n.x + en_n.y) + T(2) * (en_s.x + en_s.y);
                }
#pragma unroll
                for (int q = 0; q < NC; ++q) st4(f + q * CS, e4[q]);
            } else {
                const long long vox0 = (line0 + ll) * N3 + x4;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int ph = (int)(((j < 2 ? pp.x : pp.y) >> (16 * (j & 1))) & 0xffffu);
                    const T sc = j == 0 ? s4.x : j == 1 ? s4.y : j == 2 ? s4.z : s4.w;
                    en += apply_voxel<T, NC, OPK>(a, g * RB + rr, vox0 + j, ph, sc, f + j, CS);
                }
            }
        }
        if (a.cg) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) en += __shfl_xor_sync(0xffffffffu, en, o);
            if (lane == 0) atomicAdd(&s_eacc[rr], (double)en);
        }
    }
    phase_sync();

    // ---------------------------------------------------------------- R2C
    load_twB();
    for (int rd = 0; rd < nrounds; ++rd) {
        bool ok;
        int sig;
        slot_of(rd, ok, sig);
        cplx<T>* line = lines + (long long)sig * H;
        T* xr = reinterpret_cast<T*>(line + (sig & 1));
        cplx<T> v[R];
        // stage 1 input: v[g + G n2] = z[n1 + R n2], n1 = G p + g
#pragma unroll
        for (int n2 = 0; n2 < P; ++n2) {
            const T* src = xr + 2 * (G * p + R * n2);
#pragma unroll
            for (int h = 0; h < G / 2; ++h) {
                const float4 q = ld4(src + 4 * h);
                v[2 * h + G * n2] = mk(q.x, q.y);
                v[2 * h + 1 + G * n2] = mk(q.z, q.w);
            }
        }
        __syncwarp();
        sfor<0, G>([&](auto gc) { RegDFT<P, -1, G, decltype(gc)::value, T>::run(v); });
        // twiddle W_M^{n1 k2} (forward), then exchange: block k2, chunk p
        sfor<1, P>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            sfor<0, G>([&](auto gc) {
                constexpr int gg = decltype(gc)::value;
                v[gg + G * k2] = v[gg + G * k2] * twB[k2 - 1];
                if constexpr (gg > 0) v[gg + G * k2] = v[gg + G * k2] * tw_const<T, M, k2 * gg>();
            });
        });
        if (ok) {
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) {
                T* dst = xr + 2 * G * (k2 * P + (p ^ k2));
#pragma unroll
                for (int h = 0; h < G / 2; ++h)
                    st4(dst + 4 * h, make_float4(v[2 * h + G * k2].x, v[2 * h + G * k2].y, v[2 * h + 1 + G * k2].x,
                                                 v[2 * h + 1 + G * k2].y));
            }
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < P; ++c) {  // block p: v[n1] = Y[n1][k2 = p]
            const T* src = xr + 2 * G * (p * P + (c ^ p));
#pragma unroll
            for (int h = 0; h < G / 2; ++h) {
                const float4 q = ld4(src + 4 * h);
                v[c * G + 2 * h] = mk(q.x, q.y);
                v[c * G + 2 * h + 1] = mk(q.z, q.w);
            }
        }
        RegDFT<R, -1, 1, 0, T>::run(v);  // stage 2 over n1: v[r] = Z[p + P r]
        // R2C post-processing: Z[M - k] of k = p + P r sits in thread P - p,
        // register R - 1 - r (thread 0: its own register (R - r) mod R); the
        // results go straight to the line buffer once every thread of the
        // line has read the exchange
        const int src_lane = (lane & ~(P - 1)) | ((P - p) & (P - 1));
        const T half = T(0.5);
        // Both X[k] and X[M - k] come from the pair (Z[k], Z[M - k]): with S = Z[k] + conj Z[M-k]
        // and Q = e^{-2 pi i k / n3} (Z[k] - conj Z[M-k]), X[k] = (S - i Q) / 2 and
        // X[M - k] = (conj S - i conj Q) / 2; each thread takes its registers r < R/2 (for
        // thread 0, r = 0 gives X[0] and the Nyquist value X[M]) and thread 0 adds X[M/2].
        __syncwarp();
        sfor<0, R / 2>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            cplx<T> zc;
            zc.x = __shfl_sync(0xffffffffu, v[R - 1 - r].x, src_lane);
            zc.y = __shfl_sync(0xffffffffu, v[R - 1 - r].y, src_lane);
            if (p == 0) zc = v[(R - r) % R];
            const cplx<T> Zk = v[r], Zc = conjg(zc);
            const cplx<T> e = ep * tw_const<T, N3, P * r>();  // e^{-2 pi i k / n3}
            const cplx<T> S = Zk + Zc, Q = e * (Zk - Zc);
            if (ok) {
                line[p + P * r] = mk(half * (S.x + Q.y), half * (S.y - Q.x));
                line[M - p - P * r] = mk(half * (S.x - Q.y), -half * (S.y + Q.x));
            }
        });
        if (ok && p == 0) line[M / 2] = conjg(v[R / 2]);
    }
    fence_proxy_async_smem();  // this thread's generic writes before the bulk stores read them
    __syncthreads();

    // ---------------------------------------------------------------- bulk stores
    if (t == 0) {
        const uint32_t chunk = (uint32_t)((long long)L * H * 8);
        for (int rl = 0; rl < RB; ++rl) {
            if ((done_mask >> rl) & 1u) continue;
            const int b = g * RB + rl;
            for (int c = 0; c < NC; ++c)
                bulk_store(a.W + ((long long)(b * NC + c) * nlines + line0) * H, smlb + (long long)(rl * NC + c) * chunk,
                           chunk);
        }
        bulk_commit();
    }
    }  // !s_abort

    // ---------------------------------------------------------------- CG curvature
    if (a.cg) {
        const int nblk = gridDim.x;
        if (t == 0) {
            for (int rr = 0; rr < RB; ++rr) a.partials[(long long)(g * RB + rr) * nblk + blockIdx.x] = s_eacc[rr];
            __threadfence();
            const unsigned prev = atomicAdd(a.counters + g, 1u);
            is_last = (prev == (unsigned)nblk - 1);
        }
        __syncthreads();
        if (is_last) {  // the whole last block reduces the partials (fixed order) and sets alpha
            __threadfence();
            for (int rr = 0; rr < RB; ++rr) {
                const int bb = g * RB + rr;
                double v1[1] = {0.0};
                for (int k = t; k < nblk; k += nthr) v1[0] += __ldcg(a.partials + (long long)bb * nblk + k);
                block_sum<1>(v1, red);
                if (t == 0) {
                    const double sum = v1[0];
                    CgState& cs = a.cg[bb];
                    if (!cs.done) {
                        cs.pq = sum;
                        if (sum > 0.0 && sum == sum) {
                            cs.alpha = cs.rho / sum;
                        } else {
                            cs.alpha = 0.0;
                            cs.flags |= (sum == sum) ? 1 : 2;
                            cs.done = 1;
                        }
                    }
                }
            }
            if (t == 0) a.counters[g] = 0u;
        }
    }
    if (t == 0 && !s_abort) bulk_wait_read_all();  // the tile leaves shared memory before the CTA does
}

}  // namespace dbfft
