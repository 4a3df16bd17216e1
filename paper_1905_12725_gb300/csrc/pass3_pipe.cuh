// pass3_pipe.cuh -- axis-3 pass for the CG operator applications, as a
// persistent, double-buffered pipeline fed by bulk copies.
//
// Same arithmetic as k_axis3 (C2R along the halved contiguous axis, the
// per-voxel contraction, R2C back, and the CG curvature <p, K p>), with a
// different data movement:
//  * a tile is L consecutive grid lines of one material group; for one
//    (right-hand side, component) its half-spectrum lines are L * (N3/2+1)
//    contiguous complex values in global memory and are kept contiguous in
//    shared memory, so each one moves as a single bulk copy (no per-element
//    address arithmetic); the phase ids (and per-voxel scale) of the tile
//    come the same way;
//  * each CTA loops over tiles with two shared-memory stages: while it
//    transforms tile i in one stage, the copy engine loads tile i+1 into the
//    other, and the results of tile i leave by bulk stores;
//  * the FFT exchanges go through a small padded scratch per warp instead of
//    padding the line buffers.
// Alignment: a bulk copy needs 16-byte aligned addresses and sizes, which
// holds when L is even (FP32: (N3/2+1) * 8 bytes is 8 modulo 16) and L
// divides n1 * n2; the host only selects this kernel then.
#pragma once
#include "pass3.cuh"
#include "tma.cuh"

namespace dbfft {

// Per-voxel operation of the CG applications. f points at the real value of
// component 0 of this voxel, components CS apart; returns eps : sigma.
template <typename T, int NC, int OPK>
__device__ __forceinline__ T apply_voxel(const Ax3Args<T>& a, int bb, long long vox, int ph, T sc, T* f, int CS) {
    T en = T(0);
    if constexpr (OPK == OP_ISO) {
        const T lam = a.lam[ph] * sc, mu = a.mu[ph] * sc;
        T e[NC], sg[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) e[q] = f[q * CS] + a.macroW[bb * 9 + q];
        iso_stress<T, NC>(e, lam, mu, sg);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            en += (q >= 3 && NC == 6 ? T(2) : T(1)) * e[q] * sg[q];
            f[q * CS] = sg[q];
        }
    } else if constexpr (OPK == OP_NH_APPLY || OPK == OP_SVK_APPLY) {
        const T lam = a.lam[ph], mu = a.mu[ph];
        T G[9], sg[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) G[q] = f[q * CS] + a.macroW[bb * 9 + q];
        if constexpr (OPK == OP_SVK_APPLY)
            svk_apply<T>(a.tan_in + ((long long)bb * a.d.V + vox) * 15, mu, lam, G, sg);
        else
            nh_apply<T>(a.tan_in + ((long long)bb * a.d.V + vox) * 10, mu, lam, G, sg);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            en += G[q] * sg[q];
            f[q * CS] = sg[q];
        }
    } else if constexpr (OPK == OP_FCP_APPLY) {
        T G[9], sg[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) G[q] = f[q * CS] + a.macroW[bb * 9 + q];
        fcp_apply<T>(a.tan_in + ((long long)bb * a.d.V + vox) * 45, G, sg);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            en += G[q] * sg[q];
            f[q * CS] = sg[q];
        }
    } else if constexpr (OPK == OP_CP_APPLY) {
        T e[6], sg[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) e[q] = f[q * CS] + a.macroW[bb * 9 + q];
        cp_apply<T>(a.tan_in + ((long long)bb * a.d.V + vox) * 21, e, sg);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            en += (q >= 3 ? T(2) : T(1)) * e[q] * sg[q];
            f[q * CS] = sg[q];
        }
    }
    return en;
}

// Shared-memory plan of one CTA (bytes), shared by host and device.
template <typename T, int N3>
struct PipePlan {
    static constexpr int M = N3 / 2;
    static constexpr int H = M + 1;
    // per stage: fields [RB][NC][L][H] complex, then phase ids [L][N3] u16
    // (rounded to 16 bytes), then the optional scale [L][N3] T
    __host__ __device__ static constexpr long long field_bytes(int L, int RB, int NC) {
        return (long long)RB * NC * L * H * (long long)sizeof(cplx<T>);
    }
    __host__ __device__ static constexpr long long phase_bytes(int L) { return ((long long)L * N3 * 2 + 15) / 16 * 16; }
    __host__ __device__ static constexpr long long scale_bytes(int L, bool sc) {
        return sc ? (long long)L * N3 * (long long)sizeof(T) : 0;
    }
    __host__ __device__ static constexpr long long stage_bytes(int L, int RB, int NC, bool sc) {
        return field_bytes(L, RB, NC) + phase_bytes(L) + scale_bytes(L, sc);
    }
    // FFT exchange scratch: per warp, 32 / P lines of padded_len(M) complex
    __host__ __device__ static constexpr long long scratch_bytes(int P, int nwarps) {
        return (long long)nwarps * (32 / P) * padded_len<T>(M) * (long long)sizeof(cplx<T>);
    }
    __host__ __device__ static constexpr long long total_bytes(int L, int RB, int NC, bool sc, int P, int nwarps,
                                                               int nstage) {
        return nstage * stage_bytes(L, RB, NC, sc) + scratch_bytes(P, nwarps) + 16;  // + 2 mbarriers
    }
};

// NS = 2: two stages, the loads of the next tile overlap this tile's work;
// NS = 1: one stage (half the shared memory, so more CTAs per SM overlap
// each other instead).
template <typename T, int N3, int NC, int OPK, int RW, int NS>
__global__ void __launch_bounds__(256) k_axis3_pipe(Ax3Args<T> a) {
    static_assert(OpInfo<OPK>::apply, "the pipelined pass serves the CG applications");
    pdl_wait();
    pdl_trigger();  // the successor may start launching; it waits for this grid to finish
    constexpr int M = N3 / 2;
    constexpr int H = M + 1;
    constexpr int R = RadixAx3<T, M, RW>::value;
    constexpr int P = M / R;
    constexpr int LPW = 32 / P;  // lines a warp transforms at once
    static_assert(P <= 32 && (32 % P) == 0, "a line's threads must sit inside one warp");
    using Plan = PipePlan<T, N3>;
    extern __shared__ __align__(16) unsigned char smpipe[];
    __shared__ double red[32 * 8];
    __shared__ bool is_last;
    __shared__ int abort_flag;

    const Dims& d = a.d;
    const int RB = a.RB, L = a.L;
    const int t = threadIdx.x, nthr = blockDim.x, warp = t >> 5, lane = t & 31;
    const int g = blockIdx.y;
    const long long nlines = (long long)d.n1 * d.n2;
    const long long ntiles = nlines / L;
    const bool has_scale = a.scale != nullptr;
    const long long sbytes = Plan::stage_bytes(L, RB, NC, has_scale);
    cplx<T>* scratch = reinterpret_cast<cplx<T>*>(smpipe + NS * sbytes) + (long long)warp * LPW * padded_len<T>(M);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smpipe + NS * sbytes + Plan::scratch_bytes(P, nthr / 32));
    const int mat = (g * RB) / d.Rm;
    // right-hand sides of this group that have stopped (the flags do not change while the pass runs)
    unsigned done_mask = 0;
    if (a.cg != nullptr)
        for (int rl = 0; rl < RB; ++rl) done_mask |= (a.cg[g * RB + rl].done != 0 ? 1u : 0u) << rl;
    auto rhs_done = [&](int rl) { return (done_mask >> rl) & 1u; };
    if (a.cg != nullptr && done_mask == (RB >= 32 ? ~0u : ((1u << RB) - 1u))) return;  // the whole group has stopped

    __shared__ double s_eacc[8];  // <p, K p> of this CTA per right-hand side (tile shares formed in T)
    if (t < 8) s_eacc[t] = 0.0;
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();

    // issue the loads of one tile into one stage (thread 0 only)
    auto issue_loads = [&](long long tile, int s) {
        unsigned char* sb = smpipe + s * sbytes;
        const long long line0 = tile * L;
        const uint32_t chunk = (uint32_t)((long long)L * H * sizeof(cplx<T>));
        uint32_t tx = (uint32_t)(Plan::phase_bytes(L) + Plan::scale_bytes(L, has_scale));
        for (int rl = 0; rl < RB; ++rl)
            if (!rhs_done(rl)) tx += chunk * NC;
        mbar_arrive_expect_tx(&bars[s], tx);
        for (int rl = 0; rl < RB; ++rl) {
            if (rhs_done(rl)) continue;
            const int b = g * RB + rl;
            for (int c = 0; c < NC; ++c)
                bulk_load(sb + (long long)(rl * NC + c) * chunk, a.W + ((long long)(b * NC + c) * nlines + line0) * H,
                          chunk, &bars[s]);
        }
        unsigned char* ph = sb + Plan::field_bytes(L, RB, NC);
        bulk_load(ph, a.phase + (long long)mat * d.V + line0 * N3, (uint32_t)Plan::phase_bytes(L), &bars[s]);
        if (has_scale)
            bulk_load(ph + Plan::phase_bytes(L), a.scale + (long long)mat * d.V + line0 * N3,
                      (uint32_t)Plan::scale_bytes(L, true), &bars[s]);
    };


    long long tile = blockIdx.x;
    if (NS == 2 && t == 0 && tile < ntiles) issue_loads(tile, 0);
    const int nslot = L * RB * NC;  // (line, rhs, component) lines of a tile
    const int rounds = (nslot + LPW * (nthr / 32) - 1) / (LPW * (nthr / 32));
    int ab_it = -1;  // iteration at which a wait gave up (then the pass stops early)
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const int s = NS == 2 ? (it & 1) : 0;
        const long long next = tile + gridDim.x;
        if (t == 0) {
            if (NS == 2 && next < ntiles) {
                bulk_wait_read_all();  // the stores of the other stage have left shared memory
                issue_loads(next, s ^ 1);
            } else if (NS == 1) {
                bulk_wait_read_all();  // the previous tile's stores have left the stage
                issue_loads(tile, 0);
            }
        }
        if (!mbar_wait_bounded(&bars[s], (uint32_t)(NS == 2 ? ((it >> 1) & 1) : (it & 1)))) {
            if (a.err) atomicOr(a.err, 2u);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) {
            ab_it = it;
            break;
        }
        unsigned char* sb = smpipe + s * sbytes;
        cplx<T>* fc = reinterpret_cast<cplx<T>*>(sb);          // [RB][NC][L][H]
        T* fr = reinterpret_cast<T*>(sb);                       // the same as reals, line stride 2H
        const uint16_t* phs = reinterpret_cast<const uint16_t*>(sb + Plan::field_bytes(L, RB, NC));
        const T* scs = has_scale ? reinterpret_cast<const T*>(sb + Plan::field_bytes(L, RB, NC) + Plan::phase_bytes(L))
                                 : nullptr;

        // ---- C2R per line: Z[k] = (X[k] + conj X[M-k]) + i e^{+2 pi i k/n} (X[k] - conj X[M-k])
        for (int rd = 0; rd < rounds; ++rd) {
            const int sl = (rd * (nthr / 32) + warp) * LPW + lane / P;  // slot = (rl * NC + c) * L + ll
            const int p = lane % P;
            const bool ok = sl < nslot && !rhs_done(sl / (NC * L));
            cplx<T>* line = fc + (long long)(ok ? sl : 0) * H;
            cplx<T>* sm = scratch + (lane / P) * padded_len<T>(M);
            cplx<T> v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = p + r * P;
                const cplx<T> X = line[k];
                const cplx<T> Xc = conjg(line[M - k]);
                const cplx<T> e = conjg(ldg_c(a.tw.t3 + k));
                const cplx<T> dl = e * (X - Xc);
                v[r] = (X + Xc) + mk(-dl.y, dl.x);
            }
            ColFFT<T, M, R, +1, true, true>::run(v, sm, 1, p, a.tw.tm);
            __syncwarp();
            if (ok) {
#pragma unroll
                for (int r = 0; r < R; ++r) line[p + r * P] = v[r];  // x[2j], x[2j+1] = Re, Im z[j]
            }
            __syncwarp();
        }
        __syncthreads();

        // ---- per-voxel operation, components L * 2H reals apart
        T etile[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) etile[q] = T(0);
        for (int idx = t; idx < L * N3; idx += nthr) {
            const int lv = idx / N3, x3 = idx - lv * N3;
            const long long vox = (tile * L + lv) * N3 + x3;
            const int ph = phs[idx];
            const T sc = has_scale ? scs[idx] : T(1);
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {  // compile-time index into eacc (RB <= 8)
                if (rr >= RB) break;
                if (done_mask & (1u << rr)) continue;
                T* f = fr + ((long long)(rr * NC) * L + lv) * (2 * H) + x3;
                etile[rr] += apply_voxel<T, NC, OPK>(a, g * RB + rr, vox, ph, sc, f, L * 2 * H);
            }
        }
        if (a.cg) {
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                if (rr >= RB) break;
                T v = etile[rr];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) atomicAdd(&s_eacc[rr], (double)v);
            }
        }
        __syncthreads();

        // ---- R2C per line, X written back over the line
        for (int rd = 0; rd < rounds; ++rd) {
            const int sl = (rd * (nthr / 32) + warp) * LPW + lane / P;
            const int p = lane % P;
            const bool ok = sl < nslot && !rhs_done(sl / (NC * L));
            cplx<T>* line = fc + (long long)(ok ? sl : 0) * H;
            cplx<T>* sm = scratch + (lane / P) * padded_len<T>(M);
            cplx<T> v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = line[p + r * P];  // z[j] = x[2j] + i x[2j+1]
            ColFFT<T, M, R, -1, true, true>::run(v, sm, 1, p, a.tw.tm);
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r) sm[ColFFT<T, M, R, -1, true, true>::at(p + r * P, 1)] = v[r];
            __syncwarp();
            cplx<T> X[R];
            const T half = T(0.5);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = p + r * P;
                const cplx<T> Zk = sm[ColFFT<T, M, R, -1, true, true>::at(k, 1)];
                const cplx<T> Zc = conjg(sm[ColFFT<T, M, R, -1, true, true>::at((M - k) & (M - 1), 1)]);
                const cplx<T> e = ldg_c(a.tw.t3 + k);  // e^{-2 pi i k / n}
                const cplx<T> dl = e * (Zk - Zc);
                X[r] = mk(half * (Zk.x + Zc.x) + half * dl.y, half * (Zk.y + Zc.y) - half * dl.x);
            }
            if (ok) {
#pragma unroll
                for (int r = 0; r < R; ++r) line[p + r * P] = X[r];
                if (p == 0) {
                    const cplx<T> Z0 = sm[0];
                    line[M] = mk(Z0.x - Z0.y, T(0));
                }
            }
            __syncwarp();
        }
        fence_proxy_async_smem();  // generic writes of this stage before the bulk stores read it
        __syncthreads();

        // ---- bulk stores of the tile (thread 0), left in flight
        if (t == 0) {
            const uint32_t chunk = (uint32_t)((long long)L * H * sizeof(cplx<T>));
            for (int rl = 0; rl < RB; ++rl) {
                if (rhs_done(rl)) continue;
                const int b = g * RB + rl;
                for (int c = 0; c < NC; ++c)
                    bulk_store(a.W + ((long long)(b * NC + c) * nlines + tile * L) * H, sb + (long long)(rl * NC + c) * chunk,
                               chunk);
            }
            bulk_commit();
        }
    }
    if (t == 0) {
        if (ab_it >= 0) {  // give the loads still in flight a bounded time to land before the CTA exits
            if (NS == 1) {
                mbar_wait_bounded(&bars[0], (uint32_t)(ab_it & 1));
            } else {
                mbar_wait_bounded(&bars[ab_it & 1], (uint32_t)((ab_it >> 1) & 1));
                if (blockIdx.x + (long long)(ab_it + 1) * gridDim.x < ntiles)
                    mbar_wait_bounded(&bars[(ab_it + 1) & 1], (uint32_t)(((ab_it + 1) >> 1) & 1));
            }
        }
        bulk_wait_all();
    }

    // ---- CG curvature <p, K p> = sum_x eps : sigma, per right-hand side; the last
    // CTA of the group reduces the partials in a fixed order and sets alpha
    if (a.cg) {
        __syncthreads();  // every warp's atomics into s_eacc are done
        const int nblk = gridDim.x;
        if (t == 0) {
            for (int rr = 0; rr < RB; ++rr) a.partials[(long long)(g * RB + rr) * nblk + blockIdx.x] = s_eacc[rr];
            __threadfence();
            const unsigned prev = atomicAdd(a.counters + g, 1u);
            is_last = (prev == (unsigned)nblk - 1);
        }
        __syncthreads();
        if (is_last) {
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
}

}  // namespace dbfft
