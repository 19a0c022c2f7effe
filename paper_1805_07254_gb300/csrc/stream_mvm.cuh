// Device code of the streaming reconstruction d = M s fused with the leaky
// integrator a <- leak * a + g * d (Fig. 3 (c)-(d)), shared by the stand-alone
// reconstruction kernel, the fused frame kernel and the persistent loop kernel.
//
// The MVM is the path's bandwidth-bound bulk (Sec. 1.1.1: every frame streams the
// whole control matrix from memory), so it runs on CUDA cores as a GEMV.
//
// Work.  The matrix is [nact][kpad] row-major in its stored type; rows are taken
// four at a time ("row groups") so that each slope chunk serves four matrix
// chunks.  The (row group, 16-byte column chunk) units are cut into G equal
// contiguous ranges, one per block (one block per SM), so every SM streams the
// same number of bytes.  A block's range is a list of jobs: row groups it owns
// whole, plus at most a head (leading chunks) and a tail (trailing chunks) of a
// row group it shares with a neighbour.
//
// Movement.  Tiles of 4 row segments x tw chunks are copied into shared memory
// with bulk asynchronous copies (TMA, `cp.async.bulk`) that complete on per-stage
// mbarriers.  tw splits a row into the fewest equal tiles of at most 448 chunks
// (28 KB per tile), so a row gives no small remainder tile, and the rings take as
// many stages (up to 8 per team) as shared memory holds: short reduced-precision
// rows get deeper rings, so the bytes in flight per SM, which hide the HBM
// latency, stay at 150-190 KB for every stored type.  Two teams of 7 consumer
// warps take alternate jobs; each team has its own ring, its own producer thread
// and its own full/empty barriers, and consumes its ring in order (a ring shared
// by teams that consume out of order would let a wait on a later phase pass
// early).  One team's reduction overlaps the other's tiles.  Each consumer thread
// takes two chunks per row of a tile and issues all of its shared-memory loads
// before its FMAs.  (Deferring the reductions to the end of a block's work, so
// that a team's warps never meet between row groups, measured slower: the tail
// grows.)  The slope vector is copied once per block into shared memory
// (bank-swizzled) when it fits in 64 KB, else read through L1/L2.
//
// Arithmetic.  Stored values are widened to FP32 just before the FMA (BF16 by a
// shift, FP16 by the half2 -> float2 conversion, E4M3 by the hardware fp8x2 ->
// f16x2 conversion, INT8 exactly through the mantissa of 2^23; the FP8 and INT8
// row scales are applied once after the sum), as Sec. 2.3.4 widens its 16-bit
// matrix.  Partial sums are combined in a fixed order -- xor butterfly in each
// warp, pairwise tree over the team's 7 warps, and for a shared row group head +
// tail, added by whichever of the two blocks finishes second -- the GPU form of
// the partial-DM-vector tree of Sec. 2.3.5.  Results do not depend on scheduling.
//
// Every wait is bounded (200 ms of %globaltimer); a wait that expires records
// RTC_ETIMEDOUT in the status word, the block skips the rest of its work, lets its
// copies land and returns.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "rtc_internal.h"

namespace rtc_mvm {

constexpr int kTeams = 2;                          // consumer teams, taking alternate row groups
constexpr int kTeamWarps = 7;                      // 2 x 7 consumer + 1 producer warp: 15 warps,
                                                   // so 128 registers per thread are available
constexpr int kTeamThreads = kTeamWarps * 32;
constexpr int kConsumerWarps = kTeams * kTeamWarps;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;          // + one producer warp (lane t feeds team t)
constexpr int kRows = kMvmRows;                    // rows per row group
constexpr int kU = 2;                              // chunks per consumer thread per row per tile
constexpr int kCH = kTeamThreads * kU;             // most 16-byte chunks per row segment per tile
constexpr int kMaxTeamStages = 8;                  // stages per team ring (2..8 at run time)
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;
constexpr int kMaxPrefetchBytes = 16 * 1024;       // integrator state + scales of a block's rows
constexpr int kMaxSBytes = 64 * 1024;              // slope vector kept in shared memory up to this
constexpr size_t kDynSmemBudget = 227 * 1024 - 2048;  // dynamic shared memory per block

template <int DT> struct Epc;
template <> struct Epc<RTC_F32> { static constexpr int v = 4; };
template <> struct Epc<RTC_BF16> { static constexpr int v = 8; };
template <> struct Epc<RTC_F16> { static constexpr int v = 8; };
template <> struct Epc<RTC_FP8_E4M3> { static constexpr int v = 16; };
template <> struct Epc<RTC_INT8> { static constexpr int v = 16; };

// Stored types whose rows carry one FP32 scale, applied once after the row's sum.
template <int DT> struct RowScaled { static constexpr bool v = DT == RTC_FP8_E4M3 || DT == RTC_INT8; };

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

// Bank swizzle of the shared slope copy: piece j (16 bytes) of chunk c sits in
// slot j ^ swz(c), so the pieces the lanes of a warp read together fall in
// different banks although their chunks are E*4 bytes apart.
template <int E>
__device__ __forceinline__ int s_swizzle(int chunk) {
    return E == 16 ? ((chunk >> 1) & 3) : E == 8 ? ((chunk >> 2) & 1) : 0;
}

// ---- widening dot products (acc += <16-byte chunk, s values>) ------------------
__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t two) {
    __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(two), __NV_E4M3);
    return __half22float2(*reinterpret_cast<__half2*>(&hr));
}

// Four signed 8-bit codes (bias-flipped by xor 0x80) -> exact floats: the byte
// goes into the low mantissa bits of 2^23, so the float is 2^23 + code + 128.
__device__ __forceinline__ float i8_to_float(uint32_t flipped, int k) {
    return __uint_as_float(__byte_perm(flipped, 0x4B000000u, 0x7650 + k)) - 8388736.0f;
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
    } else if (DT == RTC_F16) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __half2_raw hr;
            hr.x = static_cast<unsigned short>(w[j] & 0xffffu);
            hr.y = static_cast<unsigned short>(w[j] >> 16);
            const float2 f = __half22float2(*reinterpret_cast<__half2*>(&hr));
            acc = fmaf(f.x, sv[2 * j], acc);
            acc = fmaf(f.y, sv[2 * j + 1], acc);
        }
    } else if (DT == RTC_INT8) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t x = w[j] ^ 0x80808080u;
#pragma unroll
            for (int k = 0; k < 4; ++k) acc = fmaf(i8_to_float(x, k), sv[4 * j + k], acc);
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

// Integrator update of one actuator from its previous state and row scale.
template <int DT>
__device__ __forceinline__ void integrate_row(int row, float d, float a_prev, float sc,
                                              float* __restrict__ a, float* __restrict__ dm_out,
                                              float gain, float leak) {
    if (RowScaled<DT>::v) d *= sc;
    const float an = fmaf(leak, a_prev, gain * d);
    a[row] = an;
    if (dm_out) dm_out[row] = an;
}

struct Args {
    const unsigned char* M;  // [nact][cpr * 16 bytes]
    int cpr, nact, nst;      // chunks per row, rows, stages per team ring
    int tw, stage_bytes;     // tile width in chunks (<= kCH), bytes of one stage (kRows * tw * 16)
    const float* s;          // [cpr * E] slopes, zero padded
    const float* scale;      // [nact] row scales (FP8, INT8)
    float* slots;            // [nrg][2][4] partials of shared row groups (scratch)
    unsigned* counters;      // [nrg] arrival counters (scratch, self-resetting)
    float* a;                // [nact] integrator state
    float* dm_out;           // [nact] or nullptr
    float gain, leak;
    int* status;             // device error word
    int region;              // bytes of shared memory between the rings and the prefetch
                             // area: the slope copy, or a fused phase's scratch before it
};

struct Shared {
    unsigned long long full_bar[kTeams][kMaxTeamStages];
    unsigned long long empty_bar[kTeams][kMaxTeamStages];
    float red[kTeams][kRows][kTeamWarps];
    volatile int abort_flag;
    volatile int release;    // set once the slopes are known (see produce's hold)
};

// What one block does, from its share of the (row group, chunk) space.
struct Plan {
    long long u0, u1;        // [u0, u1) units, row-group major
    int rg_first, rg_last;
    int row_lo, nrow_blk;    // rows touched by the block
    uint32_t smem_base;      // stage rings (kTeams * nst * stage_bytes)
    uint32_t s_smem;         // slope copy (S_SMEM)
    unsigned char* scratch;  // the same region, free until consumer_prologue
    float* a_pre;            // [nrow_blk] integrator state of the block's rows
    float* sc_pre;           // [nrow_blk] row scales of the block's rows
};

__device__ __forceinline__ void init_shared(Shared& sh) {
    for (int t = 0; t < kTeams; ++t)
        for (int i = 0; i < kMaxTeamStages; ++i) {
            mbar_init(smem_addr(&sh.full_bar[t][i]), 1);
            mbar_init(smem_addr(&sh.empty_bar[t][i]), kTeamWarps);
        }
    sh.abort_flag = 0;
    sh.release = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <int DT, bool S_SMEM>
__device__ __forceinline__ Plan make_plan(const Args& g, unsigned char* smem) {
    Plan pl;
    const int nrg = (g.nact + kRows - 1) / kRows;
    const long long total = static_cast<long long>(nrg) * g.cpr;
    pl.u0 = total * blockIdx.x / gridDim.x;
    pl.u1 = total * (blockIdx.x + 1) / gridDim.x;
    pl.rg_first = static_cast<int>(pl.u0 / g.cpr);
    pl.rg_last = static_cast<int>((pl.u1 - 1) / g.cpr);
    pl.row_lo = pl.rg_first * kRows;
    pl.nrow_blk = min(g.nact, (pl.rg_last + 1) * kRows) - pl.row_lo;
    pl.smem_base = smem_addr(smem);
    const int ring_bytes = kTeams * g.nst * g.stage_bytes;
    pl.s_smem = pl.smem_base + ring_bytes;
    pl.scratch = smem + ring_bytes;
    pl.a_pre = reinterpret_cast<float*>(smem + ring_bytes + g.region);
    pl.sc_pre = pl.a_pre + pl.nrow_blk;
    return pl;
}

__device__ __forceinline__ void job_bounds(const Args& g, const Plan& pl, int rg, int& kb, int& ke) {
    kb = (rg == pl.rg_first) ? static_cast<int>(pl.u0 % g.cpr) : 0;
    ke = (rg == pl.rg_last) ? static_cast<int>((pl.u1 - 1) % g.cpr) + 1 : g.cpr;
}

// Bounded wait for a shared-memory flag; false if it expired or the block aborted.
__device__ __forceinline__ bool wait_flag(volatile int* flag, volatile int* abort) {
    const unsigned long long t0 = global_ns();
    while (!*flag) {
        if (*abort) return false;
        if (global_ns() - t0 > kWaitNs) return false;
        __nanosleep(64);
    }
    return true;
}

// One team's producer (a single thread): stream the team's jobs into its ring.
// tl0: the team's running tile count at entry (barrier phases continue across
// calls, e.g. frame after frame in a persistent kernel); returns the count at exit.
// drain: wait for the last copies to land before returning (a block must not exit
// with copies in flight).  hold > 0: after the first `hold` tiles, wait until the
// consumers set sh.release (the latency-critical pixel stage and grid barrier
// then run in a memory system that is not flooded by the matrix stream).
__device__ __forceinline__ int produce(const Args& g, const Plan& pl, Shared& sh, int team,
                                       int tl0 = 0, bool drain = true, int hold = 0) {
    const size_t pitch = static_cast<size_t>(g.cpr) * 16;
    const uint32_t ring = pl.smem_base + team * g.nst * g.stage_bytes;
    int tl = tl0;
    bool ok = true;
    for (int rg = pl.rg_first + team; rg <= pl.rg_last && ok; rg += kTeams) {
        int kb, ke;
        job_bounds(g, pl, rg, kb, ke);
        const int nrows = min(kRows, g.nact - rg * kRows);
        for (int k = kb; k < ke; k += g.tw, ++tl) {
            if (hold > 0 && tl - tl0 == hold && !wait_flag(&sh.release, &sh.abort_flag)) {
                ok = false;
                break;
            }
            const int st = tl % g.nst;
            const int use = tl / g.nst;
            if (use > 0 &&
                !wait_phase(smem_addr(&sh.empty_bar[team][st]), (use - 1) & 1, &sh.abort_flag)) {
                ok = false;
                break;
            }
            const int nck = min(g.tw, ke - k);
            const uint32_t bytes = static_cast<uint32_t>(nck) * 16;
            const uint32_t fb = smem_addr(&sh.full_bar[team][st]);
            mbar_expect_tx(fb, bytes * nrows);
            for (int r = 0; r < nrows; ++r) {
                const unsigned char* src = g.M + static_cast<size_t>(rg * kRows + r) * pitch +
                                           static_cast<size_t>(k) * 16;
                bulk_g2s(ring + st * g.stage_bytes + r * g.tw * 16, src, bytes, fb);
            }
        }
    }
    if (!ok && !sh.abort_flag) {
        atomicExch(g.status, RTC_ETIMEDOUT);
        sh.abort_flag = 1;
    }
    // let every issued copy land before the block can exit
    if (drain || !ok)
        for (int t = max(tl0, tl - g.nst); t < tl; ++t)
            wait_phase(smem_addr(&sh.full_bar[team][t % g.nst]), (t / g.nst) & 1, nullptr);
    return tl;
}

// Consumers, before their first tile: integrator state and scales of the block's
// rows into shared memory (a demand miss at the end of every row group would queue
// behind the matrix stream), and the slope copy.  FRESH: read s from L2 (it was
// written by other blocks of the same kernel).  Ends with a consumer barrier.
template <int DT, bool S_SMEM, bool FRESH>
__device__ __forceinline__ void consumer_prologue(const Args& g, const Plan& pl, int tid,
                                                  const float* __restrict__ s_vec) {
    constexpr int E = Epc<DT>::v;
    for (int i = tid; i < pl.nrow_blk; i += kConsumers) {
        pl.a_pre[i] = FRESH ? __ldcg(g.a + pl.row_lo + i) : g.a[pl.row_lo + i];
        pl.sc_pre[i] = RowScaled<DT>::v ? g.scale[pl.row_lo + i] : 1.f;
    }
    if (S_SMEM) {
        // up to kBatch loads in flight per thread before the first store: the copy
        // costs about one L2 round trip, not one per piece
        constexpr int P = E / 4;
        constexpr int kBatch = 4;
        const int npieces = g.cpr * P;
        for (int p0 = tid; p0 < npieces; p0 += kBatch * kConsumers) {
            float4 v[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int p = p0 + b * kConsumers;
                if (p < npieces) {
                    const float4* src = reinterpret_cast<const float4*>(s_vec) + p;
                    v[b] = FRESH ? __ldcg(src) : __ldg(src);
                }
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int p = p0 + b * kConsumers;
                if (p < npieces) {
                    const int c = p / P;
                    const int j = p - c * P;
                    sts128(pl.s_smem + static_cast<uint32_t>(c * P + (j ^ s_swizzle<E>(c))) * 16, v[b]);
                }
            }
        }
    }
    consumer_sync();
}

// The consumer teams: multiply every tile of the team's jobs and finalise each
// row group (integrator, or the shared head/tail exchange).
// tile0: the team's running tile count at entry; returns the count at exit.
// s_vec: the slope vector; dm_out: where the new commands go besides g.a (or null).
template <int DT, bool S_SMEM, bool FRESH>
__device__ __forceinline__ int consume(const Args& g, const Plan& pl, Shared& sh, int tid,
                                       int tile0, const float* __restrict__ s_vec,
                                       float* __restrict__ dm_out) {
    constexpr int E = Epc<DT>::v;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int team = warp / kTeamWarps;
    const int twarp = warp - team * kTeamWarps;
    const int ttid = tid - team * kTeamThreads;
    const uint32_t ring = pl.smem_base + team * g.nst * g.stage_bytes;
    int tile = tile0;                                                // team-local tile index
    for (int rg = pl.rg_first + team; rg <= pl.rg_last; rg += kTeams) {
        int kb, ke;
        job_bounds(g, pl, rg, kb, ke);
        const int nrows = min(kRows, g.nact - rg * kRows);
        float acc[kU][kRows];
#pragma unroll
        for (int u = 0; u < kU; ++u)
#pragma unroll
            for (int r = 0; r < kRows; ++r) acc[u][r] = 0.f;
        for (int k = kb; k < ke; k += g.tw, ++tile) {
            const int st = tile % g.nst;
            const bool ok = __all_sync(0xffffffffu, wait_phase(smem_addr(&sh.full_bar[team][st]),
                                                                (tile / g.nst) & 1, &sh.abort_flag));
            if (!ok) {
                if (lane == 0 && !sh.abort_flag) {
                    atomicExch(g.status, RTC_ETIMEDOUT);
                    sh.abort_flag = 1;
                }
                continue;     // skip the work but keep reaching the block's barriers
            }
            const int nck = min(g.tw, ke - k);
            // issue every shared-memory load of this tile before any FMA; rows past
            // nact hold stale bytes and their sums are never used
            uint4 m[kU][kRows];
            float sv[kU][E];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int c = ttid + u * kTeamThreads;
                if (c < nck) {
                    if (S_SMEM) {
                        const uint32_t sp = pl.s_smem + static_cast<uint32_t>(k + c) * (E * 4);
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
                        const float4* sp =
                            reinterpret_cast<const float4*>(s_vec) + static_cast<size_t>(k + c) * (E / 4);
#pragma unroll
                        for (int j = 0; j < E / 4; ++j) {
                            const float4 v = FRESH ? __ldcg(sp + j) : __ldg(sp + j);
                            sv[u][4 * j] = v.x;
                            sv[u][4 * j + 1] = v.y;
                            sv[u][4 * j + 2] = v.z;
                            sv[u][4 * j + 3] = v.w;
                        }
                    }
                    const uint32_t sb = ring + st * g.stage_bytes + c * 16;
#pragma unroll
                    for (int r = 0; r < kRows; ++r) m[u][r] = lds128(sb + r * g.tw * 16);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (ttid + u * kTeamThreads < nck)
#pragma unroll
                    for (int r = 0; r < kRows; ++r) acc[u][r] = chunk_dot<DT>(acc[u][r], m[u][r], sv[u]);
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&sh.empty_bar[team][st]));
        }

        // fixed-order reduction of the row group's 4 partial sums over the team
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            float v = acc[0][r];
#pragma unroll
            for (int u = 1; u < kU; ++u) v += acc[u][r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) sh.red[team][r][twarp] = v;
        }
        team_sync(team);
        if (twarp == 0 && !sh.abort_flag) {
            float d = 0.f;
            if (lane < kRows) {
                float v[kTeamWarps];
#pragma unroll
                for (int w = 0; w < kTeamWarps; ++w) v[w] = sh.red[team][lane][w];
#pragma unroll
                for (int width = 1; width < kTeamWarps; width <<= 1)
#pragma unroll
                    for (int i = 0; i + width < kTeamWarps; i += 2 * width) v[i] += v[i + width];
                d = v[0];
            }
            const int row = rg * kRows + lane;
            if (kb == 0 && ke == g.cpr) {
                if (lane < nrows)
                    integrate_row<DT>(row, d, pl.a_pre[row - pl.row_lo], pl.sc_pre[row - pl.row_lo],
                                      g.a, dm_out, g.gain, g.leak);
            } else {
                // shared row group: head (kb == 0) -> slot 0, tail -> slot 1
                const int part = (kb == 0) ? 0 : 1;
                if (lane < kRows) g.slots[(static_cast<size_t>(rg) * 2 + part) * kRows + lane] = d;
                __threadfence();
                __syncwarp();
                unsigned prev = 0;
                if (lane == 0) prev = atomicAdd(g.counters + rg, 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev == 1) {
                    __threadfence();
                    if (lane < nrows) {
                        const float h = __ldcg(g.slots + (static_cast<size_t>(rg) * 2 + 0) * kRows + lane);
                        const float t = __ldcg(g.slots + (static_cast<size_t>(rg) * 2 + 1) * kRows + lane);
                        integrate_row<DT>(row, h + t, __ldcg(g.a + row),
                                          RowScaled<DT>::v ? g.scale[row] : 1.f, g.a, dm_out,
                                          g.gain, g.leak);
                    }
                    if (lane == 0) g.counters[rg] = 0u;
                }
            }
        }
        team_sync(team);
    }
    return tile;
}

// Grid barrier over co-resident blocks: one thread per block, after a block-level
// barrier.  The counter only grows; the caller passes the arrival count that
// completes this barrier.  False (and RTC_ETIMEDOUT in the status word) if it
// did not complete within kWaitNs.
__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long target,
                                             int* status, volatile int* abort) {
    __threadfence();
    atomicAdd(bar, 1ull);
    const unsigned long long t0 = global_ns();
    while (true) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(bar) : "memory");
        if (v >= target) break;
        if (global_ns() - t0 > kWaitNs) {
            atomicExch(status, RTC_ETIMEDOUT);
            *abort = 1;
            return false;
        }
    }
    __threadfence();
    return true;
}

// Grid, stages per team ring and dynamic shared memory of a launch for one handle.
struct Launch {
    int G, nst;
    int tw, stage_bytes;     // tile width (chunks) and stage size
    size_t smem;
    size_t region;           // slope copy / fused-phase scratch bytes
    bool s_in_smem;
    bool ok;
};

// min_region: shared-memory scratch a fused phase needs before the reconstruction.
inline Launch plan_launch(const rtc_handle* h, int elems_per_chunk, size_t min_region = 0) {
    Launch L{};
    const int nrg = (h->cfg.nact + kRows - 1) / kRows;
    L.G = nrg < h->num_sms ? nrg : h->num_sms;
    const size_t pre = static_cast<size_t>((nrg + L.G - 1) / L.G + 2) * kRows * 2 * sizeof(float);
    const size_t s_bytes = static_cast<size_t>(h->kpad) * sizeof(float);
    L.s_in_smem = s_bytes <= static_cast<size_t>(kMaxSBytes);
    L.region = L.s_in_smem ? s_bytes : 0;
    if (L.region < min_region) L.region = (min_region + 15) / 16 * 16;
    const size_t extra = L.region + pre;
    // a row splits into the fewest equal tiles of at most kCH chunks (no small
    // remainder tile), and the rings take as many stages as fit
    const int cpr = elems_per_chunk > 0 ? h->kpad / elems_per_chunk : 0;
    const int ntile = cpr > 0 ? (cpr + kCH - 1) / kCH : 1;
    L.tw = cpr > 0 ? (cpr + ntile - 1) / ntile : kCH;
    const size_t room = kDynSmemBudget > extra ? kDynSmemBudget - extra : 0;
    L.stage_bytes = kRows * L.tw * 16;
    const size_t fit = room / (static_cast<size_t>(kTeams) * L.stage_bytes);
    L.nst = static_cast<int>(fit < static_cast<size_t>(kMaxTeamStages) ? fit : kMaxTeamStages);
    L.smem = static_cast<size_t>(kTeams) * L.nst * L.stage_bytes + extra;
    L.ok = L.nst >= 2 && pre <= static_cast<size_t>(kMaxPrefetchBytes) && L.smem <= kDynSmemBudget &&
           h->kpad % (16 * 4 / 4) == 0 && elems_per_chunk > 0;
    return L;
}

inline Args make_args(const rtc_handle* h, const float* d_s, float* d_dm_out, const Launch& L, int epc) {
    return Args{static_cast<const unsigned char*>(h->d_M), h->kpad / epc, h->cfg.nact, L.nst,
                L.tw, L.stage_bytes, d_s, h->d_scale, h->d_partial, h->d_count, h->d_a, d_dm_out,
                h->gain, h->leak, h->d_status, static_cast<int>(L.region)};
}

}  // namespace rtc_mvm
