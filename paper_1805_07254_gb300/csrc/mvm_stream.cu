// Persistent streaming MVM d = M s fused with the leaky integrator
// a <- leak * a + g * d (Fig. 3 (c)-(d)) -- the path's bandwidth-bound bulk
// (Sec. 1.1.1: each frame streams the whole control matrix from memory).
//
// Layout of the work.  The matrix is [nact][kpad] row-major in its stored type;
// rows are taken four at a time ("row groups") so that each slope chunk read
// serves four matrix chunks.  The space of (row group, 16-byte column chunk)
// units is cut into G equal contiguous ranges, one per block, G = min(#SMs,
// #row groups), so every SM streams the same number of bytes and no block is
// left to finish alone.  A block's range is a list of jobs: row groups it owns
// whole, plus at most a head (leading chunks) and a tail (trailing chunks) of a
// row group it shares with a neighbour.
//
// Movement.  One producer thread streams each job as tiles of 4 row segments x
// 512 chunks (32 KB) into shared-memory stages with bulk asynchronous copies
// (TMA, `cp.async.bulk`) that complete on per-stage mbarriers.  Two teams of 8
// consumer warps take alternate row groups, so one team's reduction and
// integrator update overlap the other's tiles.  Each team has its own ring of 2-3
// stages, its own producer thread and its own full/empty barriers, and consumes
// its ring in order (a shared ring consumed out of order would let a wait on a
// later phase pass early); 128-192 KB per SM is in flight.  Each consumer thread takes two chunks per row of a tile and
// issues all its shared-memory loads before its FMAs.  The slope vector is copied
// once per block into shared memory (bank-swizzled) when it fits in 64 KB.
//
// Arithmetic.  Stored values are widened to FP32 just before the FMA (BF16 by a
// shift, E4M3 by the hardware fp8x2 -> f16x2 conversion; the FP8 row scale is
// applied once after the sum), as Sec. 2.3.4 widens its 16-bit matrix.  Partial
// sums are combined in a fixed order -- xor butterfly in each warp, pairwise
// tree over the 8 warps, and for a shared row group head + tail, added by
// whichever of the two blocks finishes second -- the GPU form of the
// partial-DM-vector tree of Sec. 2.3.5.  Results do not depend on scheduling.
//
// Every wait is bounded (200 ms of %globaltimer); a wait that expires records
// RTC_ETIMEDOUT in the status word, lets the block's copies land and returns.

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "rtc_internal.h"

namespace {

constexpr int kTeams = 2;                          // consumer teams, taking alternate row groups
constexpr int kTeamWarps = 8;
constexpr int kTeamThreads = kTeamWarps * 32;
constexpr int kConsumerWarps = kTeams * kTeamWarps;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + kTeams * 32;  // + one producer warp per team
constexpr int kRows = kMvmRows;                    // rows per row group
constexpr int kU = 2;                              // chunks per consumer thread per row per tile
constexpr int kCH = kTeamThreads * kU;             // 16-byte chunks per row segment per tile
constexpr int kMaxTeamStages = 3;                  // stages per team ring (2 or 3 at run time)
constexpr int kStageBytes = kRows * kCH * 16;      // 32 KB
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;
constexpr int kMaxPrefetchBytes = 16 * 1024;       // integrator state + scales of a block's rows
constexpr int kMaxSBytes = 64 * 1024;              // slope vector kept in shared memory up to this
constexpr size_t kDynSmemBudget = 227 * 1024 - 1024; // dynamic shared memory per block (static ~0.5 KB)

template <int DT> struct Epc;
template <> struct Epc<RTC_F32> { static constexpr int v = 4; };
template <> struct Epc<RTC_BF16> { static constexpr int v = 8; };
template <> struct Epc<RTC_FP8_E4M3> { static constexpr int v = 16; };

// ---- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts128(uint32_t addr, const float4& v) {
    asm volatile("st.shared.v4.f32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}
// Bank swizzle of the shared slope copy (see the staging loop in the kernel).
template <int E>
__device__ __forceinline__ int s_swizzle(int chunk) {
    return E == 16 ? ((chunk >> 1) & 3) : E == 8 ? ((chunk >> 2) & 1) : 0;
}
__device__ __forceinline__ void consumer_sync() {          // all consumer warps
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
}
__device__ __forceinline__ void team_sync(int team) {      // the 8 warps of one team
    asm volatile("bar.sync %0, %1;" ::"r"(2 + team), "n"(kTeamThreads) : "memory");
}

// Bounded wait on an mbarrier phase; false if it expired or (when abort is given)
// the block aborted.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort && *abort) return false;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

// ---- widening dot products (acc += <16-byte chunk, s values>) ------------------
__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t two) {
    __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(two), __NV_E4M3);
    return __half22float2(*reinterpret_cast<__half2*>(&hr));
}

template <int DT>
__device__ __forceinline__ float chunk_dot(float acc, const uint4& m, const float* sv) {
    const uint32_t w[4] = {m.x, m.y, m.z, m.w};
    if (DT == RTC_F32) {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc = fmaf(__uint_as_float(w[j]), sv[j], acc);
    } else if (DT == RTC_BF16) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc = fmaf(__uint_as_float(w[j] << 16), sv[2 * j], acc);
            acc = fmaf(__uint_as_float(w[j] & 0xffff0000u), sv[2 * j + 1], acc);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 a = e4m3x2_to_float2(w[j] & 0xffffu);
            const float2 b = e4m3x2_to_float2(w[j] >> 16);
            acc = fmaf(a.x, sv[4 * j + 0], acc);
            acc = fmaf(a.y, sv[4 * j + 1], acc);
            acc = fmaf(b.x, sv[4 * j + 2], acc);
            acc = fmaf(b.y, sv[4 * j + 3], acc);
        }
    }
    return acc;
}

struct Range {
    long long u0, u1;       // [u0, u1) in units of (row group, chunk), row-group major
};

__device__ __forceinline__ Range block_range(long long total, int G, int b) {
    return Range{total * b / G, total * (b + 1) / G};
}

// Integrator update of one actuator from its previous state and FP8 row scale.
template <int DT>
__device__ __forceinline__ void integrate_row(int row, float d, float a_prev, float sc,
                                              float* __restrict__ a, float* __restrict__ dm_out,
                                              float gain, float leak) {
    if (DT == RTC_FP8_E4M3) d *= sc;
    const float an = fmaf(leak, a_prev, gain * d);
    a[row] = an;
    if (dm_out) dm_out[row] = an;
}

// S_SMEM: the slope vector is copied once into shared memory (kpad * 4 <= kMaxSBytes);
// otherwise it is read through L1/L2.
template <int DT, bool S_SMEM>
__global__ void __launch_bounds__(kThreads, 1)
mvm_stream_kernel(const unsigned char* __restrict__ M, int cpr, int nact, int nst,
                  const float* __restrict__ s, const float* __restrict__ scale,
                  float* __restrict__ slots, unsigned* __restrict__ counters,
                  float* __restrict__ a, float* __restrict__ dm_out, float gain, float leak,
                  int* __restrict__ status) {
    constexpr int E = Epc<DT>::v;
    extern __shared__ __align__(128) unsigned char smem[];
    // each team owns a ring of nst stages with its own full/empty barriers and its own
    // producer, and consumes it strictly in order, so no wait can run a phase ahead
    __shared__ __align__(8) unsigned long long full_bar[kTeams][kMaxTeamStages];
    __shared__ __align__(8) unsigned long long empty_bar[kTeams][kMaxTeamStages];
    __shared__ float red[kTeams][kRows][kTeamWarps];
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int nrg = (nact + kRows - 1) / kRows;
    const long long total = static_cast<long long>(nrg) * cpr;
    const Range rg_range = block_range(total, gridDim.x, blockIdx.x);
    const size_t pitch = static_cast<size_t>(cpr) * 16;     // bytes per matrix row

    if (tid == 0) {
        for (int t = 0; t < kTeams; ++t)
            for (int i = 0; i < kMaxTeamStages; ++i) {
                mbar_init(smem_addr(&full_bar[t][i]), 1);
                mbar_init(smem_addr(&empty_bar[t][i]), kTeamWarps);
            }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (rg_range.u1 <= rg_range.u0) return;

    const int rg_first = static_cast<int>(rg_range.u0 / cpr);
    const int rg_last = static_cast<int>((rg_range.u1 - 1) / cpr);
    const uint32_t smem_base = smem_addr(smem);
    const int ring_bytes = kTeams * nst * kStageBytes;
    const uint32_t s_smem = smem_base + ring_bytes;                  // slope copy (S_SMEM)
    const int s_bytes = S_SMEM ? cpr * E * 4 : 0;
    // integrator state (and FP8 scales) of the block's rows, read once at the start:
    // a demand miss at the end of every row group would queue behind the matrix stream
    const int row_lo = rg_first * kRows;
    const int nrow_blk = min(nact, (rg_last + 1) * kRows) - row_lo;
    float* a_pre = reinterpret_cast<float*>(smem + ring_bytes + s_bytes);
    float* sc_pre = a_pre + nrow_blk;

    if (warp >= kConsumerWarps) {
        // ------------------------------------------------------------ producers
        if (lane != 0) return;
        const int team = warp - kConsumerWarps;
        const uint32_t ring = smem_base + team * nst * kStageBytes;
        int tl = 0;                                                  // team-local tile index
        bool ok = true;
        for (int rg = rg_first + team; rg <= rg_last && ok; rg += kTeams) {
            const int kb = (rg == rg_first) ? static_cast<int>(rg_range.u0 % cpr) : 0;
            const int ke = (rg == rg_last) ? static_cast<int>((rg_range.u1 - 1) % cpr) + 1 : cpr;
            const int nrows = min(kRows, nact - rg * kRows);
            for (int k = kb; k < ke; k += kCH, ++tl) {
                const int st = tl % nst;
                const int use = tl / nst;
                if (use > 0 &&
                    !wait_phase(smem_addr(&empty_bar[team][st]), (use - 1) & 1, &abort_flag)) {
                    ok = false;
                    break;
                }
                const int nck = min(kCH, ke - k);
                const uint32_t bytes = static_cast<uint32_t>(nck) * 16;
                const uint32_t fb = smem_addr(&full_bar[team][st]);
                mbar_expect_tx(fb, bytes * nrows);
                for (int r = 0; r < nrows; ++r) {
                    const unsigned char* src = M + static_cast<size_t>(rg * kRows + r) * pitch +
                                               static_cast<size_t>(k) * 16;
                    bulk_g2s(ring + st * kStageBytes + r * kCH * 16, src, bytes, fb);
                }
            }
        }
        if (!ok) {
            atomicExch(status, RTC_ETIMEDOUT);
            abort_flag = 1;
        }
        // let every issued copy land before the block can exit
        for (int t = max(0, tl - nst); t < tl; ++t)
            wait_phase(smem_addr(&full_bar[team][t % nst]), (t / nst) & 1, nullptr);
        return;
    }

    // ---------------------------------------------------------------- consumers
    for (int i = tid; i < nrow_blk; i += kConsumers) {   // visible after the consumer_sync below
        a_pre[i] = a[row_lo + i];
        sc_pre[i] = (DT == RTC_FP8_E4M3) ? scale[row_lo + i] : 1.f;
    }
    if (S_SMEM) {
        // copy s into shared memory once; piece j (16 bytes) of chunk c goes to slot
        // j ^ swz(c), so that the 16-byte pieces the lanes of a warp read together fall
        // in different banks although their chunks are E*4 bytes apart
        constexpr int P = E / 4;
        for (int p = tid; p < cpr * P; p += kConsumers) {
            const int c = p / P;
            const int j = p - c * P;
            const float4 v = __ldg(reinterpret_cast<const float4*>(s) + p);
            sts128(s_smem + static_cast<uint32_t>(c * P + (j ^ s_swizzle<E>(c))) * 16, v);
        }
    }
    consumer_sync();

    // team t takes the block's row groups (jobs) t, t + kTeams, ... from its own ring
    const int team = warp / kTeamWarps;
    const int twarp = warp - team * kTeamWarps;
    const int ttid = tid - team * kTeamThreads;
    const uint32_t ring = smem_base + team * nst * kStageBytes;
    int tile = 0;                                                    // team-local tile index
    for (int rg = rg_first + team; rg <= rg_last; rg += kTeams) {
        const int kb = (rg == rg_first) ? static_cast<int>(rg_range.u0 % cpr) : 0;
        const int ke = (rg == rg_last) ? static_cast<int>((rg_range.u1 - 1) % cpr) + 1 : cpr;
        const int nrows = min(kRows, nact - rg * kRows);
        float acc[kU][kRows];
#pragma unroll
        for (int u = 0; u < kU; ++u)
#pragma unroll
            for (int r = 0; r < kRows; ++r) acc[u][r] = 0.f;
        for (int k = kb; k < ke; k += kCH, ++tile) {
            const int st = tile % nst;
            const bool ok = __all_sync(0xffffffffu, wait_phase(smem_addr(&full_bar[team][st]),
                                                                (tile / nst) & 1, &abort_flag));
            if (!ok) {
                if (lane == 0 && !abort_flag) {
                    atomicExch(status, RTC_ETIMEDOUT);
                    abort_flag = 1;
                }
                continue;     // skip the work but keep reaching the block's barriers
            }
            const int nck = min(kCH, ke - k);
            // issue every shared-memory load of this tile before any FMA; rows past
            // nact hold stale bytes and their sums are never used
            uint4 m[kU][kRows];
            float sv[kU][E];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int c = ttid + u * kTeamThreads;
                if (c < nck) {
                    if (S_SMEM) {
                        const uint32_t sp = s_smem + static_cast<uint32_t>(k + c) * (E * 4);
                        const int sw = s_swizzle<E>(k + c);
#pragma unroll
                        for (int j = 0; j < E / 4; ++j) {
                            const uint4 v = lds128(sp + ((j ^ sw) * 16));
                            sv[u][4 * j] = __uint_as_float(v.x);
                            sv[u][4 * j + 1] = __uint_as_float(v.y);
                            sv[u][4 * j + 2] = __uint_as_float(v.z);
                            sv[u][4 * j + 3] = __uint_as_float(v.w);
                        }
                    } else {
                        const float4* sp = reinterpret_cast<const float4*>(s) + static_cast<size_t>(k + c) * (E / 4);
#pragma unroll
                        for (int j = 0; j < E / 4; ++j) {
                            const float4 v = __ldg(sp + j);
                            sv[u][4 * j] = v.x;
                            sv[u][4 * j + 1] = v.y;
                            sv[u][4 * j + 2] = v.z;
                            sv[u][4 * j + 3] = v.w;
                        }
                    }
                    const uint32_t sb = ring + st * kStageBytes + c * 16;
#pragma unroll
                    for (int r = 0; r < kRows; ++r) m[u][r] = lds128(sb + r * kCH * 16);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (ttid + u * kTeamThreads < nck)
#pragma unroll
                    for (int r = 0; r < kRows; ++r) acc[u][r] = chunk_dot<DT>(acc[u][r], m[u][r], sv[u]);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&empty_bar[team][st]));
        }

        // fixed-order reduction of the row group's 4 partial sums over the team
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            float v = acc[0][r];
#pragma unroll
            for (int u = 1; u < kU; ++u) v += acc[u][r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[team][r][twarp] = v;
        }
        team_sync(team);
        if (twarp == 0 && !abort_flag) {
            float d = 0.f;
            if (lane < kRows) {
                float v[kTeamWarps];
#pragma unroll
                for (int w = 0; w < kTeamWarps; ++w) v[w] = red[team][lane][w];
#pragma unroll
                for (int width = 1; width < kTeamWarps; width <<= 1)
#pragma unroll
                    for (int i = 0; i + width < kTeamWarps; i += 2 * width) v[i] += v[i + width];
                d = v[0];
            }
            const int row = rg * kRows + lane;
            if (kb == 0 && ke == cpr) {
                if (lane < nrows)
                    integrate_row<DT>(row, d, a_pre[row - row_lo], sc_pre[row - row_lo], a, dm_out,
                                      gain, leak);
            } else {
                // shared row group: head (kb == 0) -> slot 0, tail -> slot 1
                const int part = (kb == 0) ? 0 : 1;
                if (lane < kRows) slots[(static_cast<size_t>(rg) * 2 + part) * kRows + lane] = d;
                __threadfence();
                __syncwarp();
                unsigned prev = 0;
                if (lane == 0) prev = atomicAdd(counters + rg, 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev == 1) {
                    __threadfence();
                    if (lane < nrows) {
                        const float h = __ldcg(slots + (static_cast<size_t>(rg) * 2 + 0) * kRows + lane);
                        const float t = __ldcg(slots + (static_cast<size_t>(rg) * 2 + 1) * kRows + lane);
                        integrate_row<DT>(row, h + t, a[row],
                                          DT == RTC_FP8_E4M3 ? scale[row] : 1.f, a, dm_out, gain, leak);
                    }
                    if (lane == 0) counters[rg] = 0u;
                }
            }
        }
        team_sync(team);
    }
}

// With no slopes, d = 0: only the leak acts.
__global__ void decay_kernel(int nact, float* __restrict__ a, float* __restrict__ dm_out,
                             float leak) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nact) {
        const float an = leak * a[i];
        a[i] = an;
        if (dm_out) dm_out[i] = an;
    }
}

template <int DT>
cudaError_t launch_stream(const rtc_handle* h, const float* d_s, float* d_dm_out, cudaStream_t st) {
    const int nact = h->cfg.nact;
    const int cpr = h->kpad / Epc<DT>::v;
    const int nrg = (nact + kRows - 1) / kRows;
    const int G = std::min(h->num_sms, nrg);
    // stage ring + slope copy + prefetched state of the at most ceil(nrg / G) + 2 row groups
    const size_t pre = static_cast<size_t>((nrg + G - 1) / G + 2) * kRows * 2 * sizeof(float);
    if (pre > static_cast<size_t>(kMaxPrefetchBytes)) return cudaErrorInvalidValue;
    const size_t s_bytes = static_cast<size_t>(h->kpad) * sizeof(float);
    const bool s_in_smem = s_bytes <= static_cast<size_t>(kMaxSBytes);
    const size_t extra = (s_in_smem ? s_bytes : 0) + pre;
    // three stages per team when they fit beside the slope copy, else two
    const int nst = (static_cast<size_t>(kTeams) * 3 * kStageBytes + extra <= kDynSmemBudget) ? 3 : 2;
    const size_t bytes = static_cast<size_t>(kTeams) * nst * kStageBytes + extra;
    if (bytes > kDynSmemBudget) return cudaErrorInvalidValue;
    if (s_in_smem) {
        mvm_stream_kernel<DT, true><<<G, kThreads, bytes, st>>>(
            static_cast<const unsigned char*>(h->d_M), cpr, nact, nst, d_s, h->d_scale, h->d_partial,
            h->d_count, h->d_a, d_dm_out, h->gain, h->leak, h->d_status);
    } else {
        mvm_stream_kernel<DT, false><<<G, kThreads, bytes, st>>>(
            static_cast<const unsigned char*>(h->d_M), cpr, nact, nst, d_s, h->d_scale, h->d_partial,
            h->d_count, h->d_a, d_dm_out, h->gain, h->leak, h->d_status);
    }
    return cudaGetLastError();
}

}  // namespace

template <int DT, bool S>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(mvm_stream_kernel<DT, S>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kDynSmemBudget));
}

cudaError_t mvm_stream_configure() {
    cudaError_t e = configure_one<RTC_F32, true>();
    if (e == cudaSuccess) e = configure_one<RTC_F32, false>();
    if (e == cudaSuccess) e = configure_one<RTC_BF16, true>();
    if (e == cudaSuccess) e = configure_one<RTC_BF16, false>();
    if (e == cudaSuccess) e = configure_one<RTC_FP8_E4M3, true>();
    if (e == cudaSuccess) e = configure_one<RTC_FP8_E4M3, false>();
    return e;
}

cudaError_t launch_mvm_integrate(const rtc_handle* h, const float* d_s, float* d_dm_out,
                                 cudaStream_t st) {
    if (h->kpad == 0) {
        decay_kernel<<<(h->cfg.nact + 255) / 256, 256, 0, st>>>(h->cfg.nact, h->d_a, d_dm_out,
                                                                h->leak);
        return cudaGetLastError();
    }
    switch (h->store) {
        case RTC_F32: return launch_stream<RTC_F32>(h, d_s, d_dm_out, st);
        case RTC_BF16: return launch_stream<RTC_BF16>(h, d_s, d_dm_out, st);
        case RTC_FP8_E4M3: return launch_stream<RTC_FP8_E4M3>(h, d_s, d_dm_out, st);
        default: return cudaErrorInvalidValue;
    }
}
