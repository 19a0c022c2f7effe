// Device code of the reconstruction d = M s fused with the leaky integrator
// a <- leak * a + g * d (Fig. 3 (c)-(d)), shared by the stand-alone reconstruction
// kernel, the fused frame kernel and the persistent loop kernel.
//
// Decomposition (Sec. 2.3, 2.3.5).  As in the paper, where each thread takes a set
// of subapertures, multiplies the matrix columns of their slopes and leaves a
// partial DM vector that a tree then sums, the slope columns are cut into S slices
// of consecutive subapertures (S = the SM count, or the number of subapertures if
// smaller).  rtc_load_cmat stores the matrix slice by slice: slice s is one
// contiguous [nact][w_s] block, its w_s = 2 n_s columns being the slice's x slopes
// then its y slopes, each row padded to a multiple of 4 bytes.  A block of a fused
// kernel takes a run of whole slices and computes those subapertures' slopes
// itself, so its share of the product starts as soon as its own pixels are done,
// without waiting for any other block; it writes one partial vector per slice.
// After one grid barrier every block sums the S partials of its share of the rows
// in a fixed order (warp w sums the slices w, w+14, w+28, ... in turn for 32
// consecutive rows with coalesced loads, then a fixed pairwise tree over the 14
// warps), applies the FP8/INT8 row scale and the integrator.
// The result does not depend on the number of blocks or on their timing.
//
// Movement.  A slice streams in tiles of R rows, bulk asynchronous copies
// (`cp.async.bulk`) completing on a per-stage mbarrier, through a ring of up to 8
// stages in shared memory that one producer thread fills and 14 consumer warps
// drain.  T consecutive lanes take one row of a tile (T = 1 for ELT-sized slices,
// more when rows are long, so that at least two stages fit) and read it in units of
// 16, 8 or 4 bytes, the widest that divides the row an odd number of times (rows
// are padded until one does), so that the rows a warp reads at once fall in
// different banks; all lanes read the same units of the slice's slopes at the same
// time (shared-memory broadcasts).
//
// Arithmetic.  Stored values are widened to FP32 just before the FMA (BF16 by a
// shift, FP16 by the half2 -> float2 conversion, E4M3 by the hardware fp8x2 ->
// f16x2 conversion, INT8 exactly through the mantissa of 2^23), as Sec. 2.3.4
// widens its 16-bit matrix; the FP8 and INT8 row scales are applied once per row
// after the sum over slices.
//
// Every wait is bounded (200 ms of %globaltimer); a wait that expires records
// RTC_ETIMEDOUT in the status word, the block skips the rest of its work, lets its
// copies land and returns.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "rtc_internal.h"

namespace rtc_mvm {

constexpr int kConsumerWarps = 14;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;          // + one producer warp
constexpr int kMaxStages = 32;
// Smallest ring stage the launch plan aims for, in bytes (two stages of ~96 KB
// measured faster than more, smaller ones: fewer per-tile handshakes).
constexpr size_t kMinTileBytes = 96 * 1024;
// Rows of one slice's tile per consumer thread, at most (narrow slices pack several
// rows into a stage sized for the widest one).
constexpr int kMaxRowsPerThread = 32;
// Largest matrix streamed with the default L2 policy (of the 126 MB L2).
constexpr long long kL2KeepBytes = 80ll << 20;
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;
constexpr int kMaxLocalFloats = 8192;              // slopes of a block's slices (32 KB)
constexpr int kMaxRowFloats = 4096;                // rows a block reduces, at most
constexpr size_t kDynSmemBudget = 227 * 1024 - 2048;  // dynamic shared memory per block
constexpr int kMaxSlices = 256;
constexpr int kSlicesPerWarp = (kMaxSlices + kConsumerWarps - 1) / kConsumerWarps;
constexpr uint32_t kCopyBytes = 8192;              // largest single bulk copy of a tile

template <int DT> struct Esize;
template <> struct Esize<RTC_F32> { static constexpr int v = 4; };
template <> struct Esize<RTC_BF16> { static constexpr int v = 2; };
template <> struct Esize<RTC_F16> { static constexpr int v = 2; };
template <> struct Esize<RTC_FP8_E4M3> { static constexpr int v = 1; };
template <> struct Esize<RTC_INT8> { static constexpr int v = 1; };

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
// Bulk copy global -> shared completing on an mbarrier, with an L2 eviction policy.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar, unsigned long long policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}
// L2 policies for the matrix stream.  A matrix larger than L2 goes through without
// displacing the calibration maps, frames and partial vectors (evict_first); one
// that fits beside them keeps the default policy, so that frame after frame it can
// stay in L2.
enum L2Policy { kL2Normal = 0, kL2Stream = 1 };
__device__ __forceinline__ unsigned long long matrix_policy(int mode) {
    unsigned long long p;
    if (mode == kL2Stream)
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Bulk prefetch of global bytes into L2 (no shared memory, no completion).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint2 lds64(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}

// Access unit of a slice row of rb bytes: the widest of 16, 8, 4 bytes that divides
// the row an odd number of times, so that the rows a warp reads at once (rb bytes
// apart) fall in different banks.  rtc_load_cmat pads rows until one exists.
__host__ __device__ __forceinline__ int row_unit(int rb) {
    if (rb % 16 == 0 && (rb / 16) % 2 == 1) return 16;
    if (rb % 8 == 0 && (rb / 8) % 2 == 1) return 8;
    if (rb % 4 == 0 && (rb / 4) % 2 == 1) return 4;
    return 0;
}
// Byte offset of byte cb of row `row` of a slice (at byte off, rb bytes per row,
// nact rows).  Row-major, or in the plane layout: rows in groups of 32, and within a
// group the rows' first 16-byte units, then their second ones, ..., then their
// (rb % 16)-byte tails.  A group of ng rows takes ng * rb bytes either way, so tiles
// of whole groups are the same byte ranges in both layouts.
__host__ __device__ __forceinline__ size_t slice_elem_offset(long long off, int rb, int nact, int row, int cb,
                                                             int plane) {
    if (!plane) return static_cast<size_t>(off) + static_cast<size_t>(row) * rb + cb;
    const int g0 = row & ~31;
    const int ng = nact - g0 < 32 ? nact - g0 : 32;
    const int li = row - g0, q = rb >> 4, t = rb & 15, k = cb >> 4;
    const size_t base = static_cast<size_t>(off) + static_cast<size_t>(g0) * rb;
    if (k < q) return base + static_cast<size_t>(k) * ng * 16 + li * 16 + (cb & 15);
    return base + static_cast<size_t>(q) * ng * 16 + static_cast<size_t>(li) * t + (cb - 16 * q);
}

__device__ __forceinline__ void consumer_sync() {          // all consumer warps
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
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

// ---- widening dot products: acc += <one 4-byte word of a row, its slopes> -------
__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t two) {
    __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(two), __NV_E4M3);
    return __half22float2(*reinterpret_cast<__half2*>(&hr));
}

// Four signed 8-bit codes (bias-flipped by xor 0x80) -> exact floats: the byte
// goes into the low mantissa bits of 2^23, so the float is 2^23 + code + 128.
__device__ __forceinline__ float i8_to_float(uint32_t flipped, int k) {
    return __uint_as_float(__byte_perm(flipped, 0x4B000000u, 0x7650 + k)) - 8388736.0f;
}

// acc += <word w, its EPW slopes s>.  (Placing FP8 / FP16 bits at the top of an FP32
// mantissa and pre-scaling the slopes by 2^120 / 2^112 avoids the conversion
// instructions but measured slower than the hardware conversions.)
template <int DT>
__device__ __forceinline__ float word_dot(float acc, uint32_t w, const float* s) {
    if (DT == RTC_F32) {
        acc = fmaf(__uint_as_float(w), s[0], acc);
    } else if (DT == RTC_BF16) {
        acc = fmaf(__uint_as_float(w << 16), s[0], acc);
        acc = fmaf(__uint_as_float(w & 0xffff0000u), s[1], acc);
    } else if (DT == RTC_F16) {
        __half2_raw hr;
        hr.x = static_cast<unsigned short>(w & 0xffffu);
        hr.y = static_cast<unsigned short>(w >> 16);
        const float2 f = __half22float2(*reinterpret_cast<__half2*>(&hr));
        acc = fmaf(f.x, s[0], acc);
        acc = fmaf(f.y, s[1], acc);
    } else if (DT == RTC_FP8_E4M3) {
        const float2 a = e4m3x2_to_float2(w & 0xffffu);
        const float2 b = e4m3x2_to_float2(w >> 16);
        acc = fmaf(a.x, s[0], acc);
        acc = fmaf(a.y, s[1], acc);
        acc = fmaf(b.x, s[2], acc);
        acc = fmaf(b.y, s[3], acc);
    } else {
        const uint32_t x = w ^ 0x80808080u;
        acc = fmaf(i8_to_float(x, 0), s[0], acc);
        acc = fmaf(i8_to_float(x, 1), s[1], acc);
        acc = fmaf(i8_to_float(x, 2), s[2], acc);
        acc = fmaf(i8_to_float(x, 3), s[3], acc);
    }
    return acc;
}

// Integrator update of one actuator from its previous state and row scale.
template <int DT>
__device__ __forceinline__ float integrate_row(int row, float d, float a_prev, float sc,
                                               float* __restrict__ a, float* __restrict__ dm_out,
                                               float gain, float leak) {
    if (RowScaled<DT>::v) d *= sc;
    const float an = fmaf(leak, a_prev, gain * d);
    a[row] = an;
    if (dm_out) dm_out[row] = an;
    return an;
}

// ---- plan ----------------------------------------------------------------------

// The slice table of a loaded matrix (device arrays).
struct Slices {
    const long long* off;    // [S] byte offset of slice s in the matrix (16-byte aligned)
    const int* rowbytes;     // [S] bytes per row of slice s (multiple of 4)
    const int* g0;           // [S + 1] first subaperture (w * n_valid + i) of slice s
    const int* loc;          // [S + 1] float offset of slice s's slopes in a local vector
    int S;
    int nt;                  // subapertures over all WFS
    int equal;               // g0[s] = nt s / S (the default cut): computed, not loaded
};

struct Args {
    const unsigned char* M;  // slice-major matrix
    Slices sl;
    int nact, n_valid;       // rows; valid subapertures per WFS
    int T, R;                // lanes per row, rows per tile (T * R = kConsumers)
    int stage_bytes, nst;    // the ring: nst stages of stage_bytes (R rows of the widest slice)
    int l2_policy;           // L2Policy of the matrix stream
    int region;              // shared scratch bytes of a fused phase (before the slopes)
    int loc_floats;          // floats of the largest block-local slope vector
    int row_floats;          // rows a block reduces, at most
    int plane;               // slices in the plane layout (T = 1; see slice_elem_offset)
    const float* s;          // stand-alone reconstruction: the full slope vector (else unused)
    const float* scale;      // [nact] row scales (FP8, INT8)
    float* partial;          // [S][nact] partial DM vectors
    float* a;                // [nact] integrator state
    float* dm_out;           // [nact] or nullptr
    float gain, leak;
    int* status;             // device error word
};

struct Shared {
    unsigned long long full_bar[kMaxStages];
    unsigned long long empty_bar[kMaxStages];
    volatile int abort_flag;
    volatile int release;    // set once the block's slopes are known (see produce's hold)
};

// What one block does.
struct Plan {
    int sb0, sb1;            // slices [sb0, sb1)
    int g0, g1;              // subapertures [g0, g1)
    int r0, r1;              // rows the block reduces
    int rb0, n0, loc0;       // first slice: bytes per row, subapertures, local offset
    uint32_t ring;           // shared address of the ring
    unsigned char* scratch;  // fused-phase scratch (region bytes)
    float* loc;              // block-local slopes: each slice's x then y block, zero padded
    float* a_pre;            // [r1 - r0] integrator state of the rows the block reduces
    float* sc_pre;           // [r1 - r0] their row scales
    float* red;              // [kConsumerWarps][32] warp sums of the sum over slices
};

__device__ __forceinline__ void init_shared(Shared& sh) {
    for (int i = 0; i < kMaxStages; ++i) {
        mbar_init(smem_addr(&sh.full_bar[i]), 1);
        mbar_init(smem_addr(&sh.empty_bar[i]), kConsumerWarps);
    }
    sh.abort_flag = 0;
    sh.release = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ Plan make_plan(const Args& g, unsigned char* smem) {
    Plan pl;
    const int S = g.sl.S;
    pl.sb0 = static_cast<int>(static_cast<long long>(S) * blockIdx.x / gridDim.x);
    pl.sb1 = static_cast<int>(static_cast<long long>(S) * (blockIdx.x + 1) / gridDim.x);
    // the block's subapertures: with the default cut computed, so that the pixel
    // stage does not wait for a table load before it can fetch positions
    if (g.sl.equal) {
        pl.g0 = static_cast<int>(static_cast<long long>(g.sl.nt) * pl.sb0 / S);
        pl.g1 = static_cast<int>(static_cast<long long>(g.sl.nt) * pl.sb1 / S);
        pl.n0 = static_cast<int>(static_cast<long long>(g.sl.nt) * (pl.sb0 + 1) / S) - pl.g0;
    } else {
        pl.g0 = g.sl.g0[pl.sb0];
        pl.g1 = g.sl.g0[pl.sb1];
        pl.n0 = g.sl.g0[pl.sb0 + 1] - pl.g0;
    }
    // the first slice's layout, read once here rather than on the frame's critical path
    pl.rb0 = g.sl.rowbytes[pl.sb0];
    pl.loc0 = g.sl.loc[pl.sb0];
    pl.r0 = static_cast<int>(static_cast<long long>(g.nact) * blockIdx.x / gridDim.x);
    pl.r1 = static_cast<int>(static_cast<long long>(g.nact) * (blockIdx.x + 1) / gridDim.x);
    const int ring_bytes = g.nst * g.stage_bytes;
    pl.ring = smem_addr(smem);
    pl.scratch = smem + ring_bytes;
    pl.loc = reinterpret_cast<float*>(smem + ring_bytes + g.region);
    pl.a_pre = pl.loc + g.loc_floats;
    pl.sc_pre = pl.a_pre + g.row_floats;
    pl.red = pl.sc_pre + g.row_floats;
    return pl;
}

// Where subaperture gi (one of the block's) puts its x and y slopes in the
// block-local vector.
__device__ __forceinline__ void local_index(const Args& g, const Plan& pl, int gi, int& ix, int& iy) {
    if (gi < pl.g0 + pl.n0) {           // the first slice
        ix = gi - pl.g0;
        iy = ix + pl.n0;
        return;
    }
    int s = pl.sb0 + 1;
    while (s + 1 < pl.sb1 && g.sl.g0[s + 1] <= gi) ++s;
    const int base = g.sl.loc[s] - pl.loc0;
    const int n = g.sl.g0[s + 1] - g.sl.g0[s];
    ix = base + (gi - g.sl.g0[s]);
    iy = ix + n;
}

// Consumers: clear the block-local slope vector (its padding stays zero).
__device__ __forceinline__ void clear_local(const Args& g, const Plan& pl, int tid) {
    for (int i = tid; i < g.loc_floats; i += kConsumers) pl.loc[i] = 0.f;
}

// Consumers: the block's slopes from a full slope vector s (x block then y block per
// WFS).  fresh: s was written by other blocks of the same kernel (read from L2).
__device__ __forceinline__ void gather_local(const Args& g, const Plan& pl, int tid,
                                             const float* __restrict__ s, bool fresh) {
    for (int gi = pl.g0 + tid; gi < pl.g1; gi += kConsumers) {
        const int w = gi / g.n_valid, i = gi - w * g.n_valid;
        const size_t bx = static_cast<size_t>(w) * 2 * g.n_valid + i;
        int ix, iy;
        local_index(g, pl, gi, ix, iy);
        pl.loc[ix] = fresh ? __ldcg(s + bx) : __ldg(s + bx);
        pl.loc[iy] = fresh ? __ldcg(s + bx + g.n_valid) : __ldg(s + bx + g.n_valid);
    }
}

// 4-byte global -> shared copy that does not hold up the issuing thread.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// Consumers: integrator state and row scales of the rows the block reduces, as
// asynchronous copies, so that the block's first tiles need not wait for them (a
// cold load here held every frame's stream back by about a round trip).  The
// copies are complete once rows_landed() and a consumer barrier have followed.
template <int DT>
__device__ __forceinline__ void prefetch_rows(const Args& g, const Plan& pl, int tid) {
    for (int r = pl.r0 + tid; r < pl.r1; r += kConsumers) {
        cp_async4(pl.a_pre + (r - pl.r0), g.a + r);
        if (RowScaled<DT>::v) cp_async4(pl.sc_pre + (r - pl.r0), g.scale + r);
        else pl.sc_pre[r - pl.r0] = 1.f;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The calling thread's prefetch_rows copies have landed.  Every consumer calls it
// before the barrier that precedes reduce_rows, aborted or not (no copy may still
// be writing shared memory when the block exits).
__device__ __forceinline__ void rows_landed() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Rows of slice tiles with rb bytes per row: R rows for the widest slice, a multiple
// of R that still fits in a stage for narrower ones.  A row is always summed by
// the same T lanes, so the tile height does not change any result.
__device__ __forceinline__ int tile_rows(const Args& g, int rb) {
    const int m = g.stage_bytes / (g.R * rb);
    return g.R * (m < 1 ? 1 : m > kMaxRowsPerThread ? kMaxRowsPerThread : m);
}

// Source and size of tile t of the block (counted from the start of its first
// slice); false past its last tile.
__device__ __forceinline__ bool tile_src(const Args& g, const Plan& pl, int t, const unsigned char*& src,
                                         uint32_t& bytes) {
    for (int s = pl.sb0; s < pl.sb1; ++s) {
        const int rb = g.sl.rowbytes[s];
        const int tr = tile_rows(g, rb);
        const int nt = (g.nact + tr - 1) / tr;
        if (t < nt) {
            const int row0 = t * tr;
            src = g.M + g.sl.off[s] + static_cast<size_t>(row0) * rb;
            bytes = (static_cast<uint32_t>(min(tr, g.nact - row0)) * rb + 15u) & ~15u;
            return true;
        }
        t -= nt;
    }
    return false;
}

// One producer thread: stream the block's slices tile by tile into the ring.
// tl0: the running tile count at entry (barrier phases continue across calls, e.g.
// frame after frame in a persistent kernel); returns the count at exit.  drain: wait
// for the last copies to land before returning (a block must not exit with copies
// in flight).  hold > 0: after the first `hold` tiles, wait until the consumers set
// sh.release (the latency-critical pixel loads then do not queue behind the
// stream).  hold_l2: tiles prefetched into L2 right before that wait (a long wait,
// such as the predictor's, then leaves the HBM streaming).
__device__ __forceinline__ int produce(const Args& g, const Plan& pl, Shared& sh, int tl0 = 0,
                                       bool drain = true, int hold = 0, int hold_l2 = 0) {
    int tl = tl0;
    bool ok = true;
    const unsigned long long policy = matrix_policy(g.l2_policy);
    for (int s = pl.sb0; s < pl.sb1 && ok; ++s) {
        const unsigned char* base = g.M + g.sl.off[s];
        const int rb = g.sl.rowbytes[s];
        const int tr = tile_rows(g, rb);
        for (int row0 = 0; row0 < g.nact; row0 += tr, ++tl) {
            if (hold > 0 && tl - tl0 == hold) {
                for (int j = 0; j < hold_l2; ++j) {
                    const unsigned char* psrc;
                    uint32_t pbytes;
                    if (tile_src(g, pl, hold + j, psrc, pbytes)) bulk_prefetch_l2(psrc, pbytes);
                }
                if (!wait_flag(&sh.release, &sh.abort_flag)) {
                    ok = false;
                    break;
                }
            }
            const int st = tl % g.nst;
            const int use = tl / g.nst;
            if (use > 0 && !wait_phase(smem_addr(&sh.empty_bar[st]), (use - 1) & 1, &sh.abort_flag)) {
                ok = false;
                break;
            }
            const int rows = min(tr, g.nact - row0);
            // the slice is padded to 16 bytes, so the last tile may round up; the tile
            // goes as several copies
            const uint32_t bytes = (static_cast<uint32_t>(rows) * rb + 15u) & ~15u;
            const uint32_t fb = smem_addr(&sh.full_bar[st]);
            mbar_expect_tx(fb, bytes);
            const unsigned char* src = base + static_cast<size_t>(row0) * rb;
            for (uint32_t o = 0; o < bytes; o += kCopyBytes)
                bulk_g2s(pl.ring + st * g.stage_bytes + o, src + o, min(kCopyBytes, bytes - o), fb, policy);
        }
    }
    if (!ok && !sh.abort_flag) {
        atomicExch(g.status, RTC_ETIMEDOUT);
        sh.abort_flag = 1;
    }
    if (drain || !ok)
        for (int t = max(tl0, tl - g.nst); t < tl; ++t)
            wait_phase(smem_addr(&sh.full_bar[t % g.nst]), (t / g.nst) & 1, nullptr);
    return tl;
}

// The EPU slopes of one unit into registers with vector loads (shared-memory
// broadcasts: every lane of the warp reads the same unit at the same time).
template <int EPU>
__device__ __forceinline__ void load_unit(const float* s, float* r) {
    if constexpr (EPU % 4 == 0) {
#pragma unroll
        for (int j = 0; j < EPU; j += 4) {
            const float4 v = *reinterpret_cast<const float4*>(s + j);
            r[j] = v.x;
            r[j + 1] = v.y;
            r[j + 2] = v.z;
            r[j + 3] = v.w;
        }
    } else if constexpr (EPU == 2) {
        const float2 v = *reinterpret_cast<const float2*>(s);
        r[0] = v.x;
        r[1] = v.y;
    } else {
        r[0] = s[0];
    }
}

// acc += <one U-byte unit of a row at shared address a, its slopes r>, word by word.
template <int DT, int U>
__device__ __forceinline__ float unit_dot(float acc, uint32_t a, const float* r) {
    constexpr int EPW = 4 / Esize<DT>::v;                    // elements per 4-byte word
    if constexpr (U == 16) {
        const uint4 m = lds128(a);
        acc = word_dot<DT>(acc, m.x, r);
        acc = word_dot<DT>(acc, m.y, r + EPW);
        acc = word_dot<DT>(acc, m.z, r + 2 * EPW);
        acc = word_dot<DT>(acc, m.w, r + 3 * EPW);
    } else if constexpr (U == 8) {
        const uint2 m = lds64(a);
        acc = word_dot<DT>(acc, m.x, r);
        acc = word_dot<DT>(acc, m.y, r + EPW);
    } else {
        acc = word_dot<DT>(acc, lds32(a), r);
    }
    return acc;
}

// Slope floats a consumer lane keeps in registers for one slice.
constexpr int kSlopeRegs = 16;
// Units of a row a lane can hold the slopes of: kSlopeRegs / (elements per unit).
template <int DT, int U>
struct LaneUnits {
    static constexpr int v = kSlopeRegs * Esize<DT>::v / U > 0 ? kSlopeRegs * Esize<DT>::v / U : 1;
};

// The tiles of one slice (rb bytes per row, its slopes at pl.loc + lo); returns the
// running tile count.  Lane `part` of a row's T lanes takes the row's units part,
// part + T, ..., in that order, and the T partial sums meet in an xor butterfly.
// When a lane's units fit (LaneUnits), their slopes stay in registers for the
// whole slice and the tile is read once; otherwise every unit's slopes come from
// shared memory.  Both ways add the same terms in the same order.
template <int DT, int U>
__device__ __forceinline__ int consume_slice(const Args& g, const Plan& pl, Shared& sh, int tid,
                                             int tile, int s, int rb, int lo) {
    constexpr int EPU = U / Esize<DT>::v;                    // elements per unit
    constexpr int JM = LaneUnits<DT, U>::v;
    // launch constants in registers for the row loops
    const int T = g.T, R = g.R, nact = g.nact, nst = g.nst, stage_bytes = g.stage_bytes;
    const int lane = tid & 31;
    const int rt = tid / T;                                  // row of the tile
    const int part = tid - rt * T;                           // lane within the row's group
    const int nunits = rb / U;
    const float* sv = pl.loc + lo;
    float* out = g.partial + static_cast<size_t>(s) * nact;
    const int tr = tile_rows(g, rb);
    const bool in_regs = (nunits + T - 1) / T <= JM;     // the same for the whole block
    float sr[JM][EPU];
#pragma unroll
    for (int j = 0; j < JM; ++j) {
        const int k = part + j * T;
        if (in_regs && k < nunits) {
            load_unit<EPU>(sv + k * EPU, sr[j]);
        } else {
#pragma unroll
            for (int e = 0; e < EPU; ++e) sr[j][e] = 0.f;
        }
    }
    for (int row0 = 0; row0 < nact; row0 += tr, ++tile) {
        const int st = tile % nst;
        const bool ok = __all_sync(0xffffffffu, wait_phase(smem_addr(&sh.full_bar[st]),
                                                            (tile / nst) & 1, &sh.abort_flag));
        if (!ok) {
            if (lane == 0 && !sh.abort_flag) {
                atomicExch(g.status, RTC_ETIMEDOUT);
                sh.abort_flag = 1;
            }
            continue;     // skip the work but keep reaching the block's barriers
        }
        const uint32_t stage = pl.ring + st * stage_bytes;
        // rows of this tile per lane group: the same count on every lane
        const int iters = (min(tr, nact - row0) + R - 1) / R;
        if (in_regs) {
            int i = 0;
            for (; i + 2 <= iters; i += 2) {                 // two rows in flight
                const int ra = rt + i * R, rbw = ra + R;
                const bool va = row0 + ra < nact, vb = row0 + rbw < nact;
                float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
                for (int j = 0; j < JM; ++j) {
                    const int k = part + j * T;
                    if (k < nunits) {
                        if (va) acc0 = unit_dot<DT, U>(acc0, stage + ra * rb + k * U, sr[j]);
                        if (vb) acc1 = unit_dot<DT, U>(acc1, stage + rbw * rb + k * U, sr[j]);
                    }
                }
                for (int off = T >> 1; off > 0; off >>= 1) {
                    acc0 += __shfl_xor_sync(0xffffffffu, acc0, off);
                    acc1 += __shfl_xor_sync(0xffffffffu, acc1, off);
                }
                if (part == 0 && va) out[row0 + ra] = acc0;
                if (part == 0 && vb) out[row0 + rbw] = acc1;
            }
            if (i < iters) {
                const int ra = rt + i * R;
                const bool va = row0 + ra < nact;
                float acc0 = 0.f;
#pragma unroll
                for (int j = 0; j < JM; ++j) {
                    const int k = part + j * T;
                    if (k < nunits && va) acc0 = unit_dot<DT, U>(acc0, stage + ra * rb + k * U, sr[j]);
                }
                for (int off = T >> 1; off > 0; off >>= 1) acc0 += __shfl_xor_sync(0xffffffffu, acc0, off);
                if (part == 0 && va) out[row0 + ra] = acc0;
            }
        } else {
            for (int i = 0; i < iters; ++i) {
                const int ra = rt + i * R;
                const bool va = row0 + ra < nact;
                float acc = 0.f;
                if (va) {
#pragma unroll 4
                    for (int k = part; k < nunits; k += T) {
                        float r[EPU];
                        load_unit<EPU>(sv + k * EPU, r);
                        acc = unit_dot<DT, U>(acc, stage + ra * rb + k * U, r);
                    }
                }
                for (int off = T >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if (part == 0 && va) out[row0 + ra] = acc;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&sh.empty_bar[st]));
    }
    return tile;
}

// The tiles of one slice in the plane layout (T = 1, R = kConsumers rows a tile step):
// warp w takes rows 32 w .. 32 w + 31 of each step, one group, so every 16-byte load
// of the warp reads 512 consecutive bytes, and the (rb % 16)-byte tails follow the
// group's units.  Rows are taken two at a time, sharing each unit's slope loads.
// Each row's terms are added in element order, the order of the row-major form.
template <int DT>
__device__ __forceinline__ int consume_slice_plane(const Args& g, const Plan& pl, Shared& sh, int tid,
                                                   int tile, int s, int rb, int lo) {
    constexpr int E16 = 16 / Esize<DT>::v;                   // elements per 16-byte unit
    constexpr int EPW = 4 / Esize<DT>::v;                    // elements per word
    const int R = g.R, nact = g.nact, nst = g.nst, stage_bytes = g.stage_bytes;
    const int lane = tid & 31;
    const int q = rb >> 4, tb = rb & 15;
    const float* sv = pl.loc + lo;
    const float* st_tail = sv + q * E16;
    float* out = g.partial + static_cast<size_t>(s) * nact;
    const int tr = tile_rows(g, rb);
    for (int row0 = 0; row0 < nact; row0 += tr, ++tile) {
        const int st = tile % nst;
        const bool ok = __all_sync(0xffffffffu, wait_phase(smem_addr(&sh.full_bar[st]),
                                                            (tile / nst) & 1, &sh.abort_flag));
        if (!ok) {
            if (lane == 0 && !sh.abort_flag) {
                atomicExch(g.status, RTC_ETIMEDOUT);
                sh.abort_flag = 1;
            }
            continue;     // skip the work but keep reaching the block's barriers
        }
        const uint32_t stage = pl.ring + st * stage_bytes;
        const int iters = (min(tr, nact - row0) + R - 1) / R;
        for (int i = 0; i < iters; i += 2) {
            const int ra = tid + i * R, rbw = ra + R;
            const bool va = row0 + ra < nact;
            const bool vb = i + 1 < iters && row0 + rbw < nact;
            const int ga = ra & ~31, gb = rbw & ~31;
            const int na = min(32, nact - row0 - ga), nb = min(32, nact - row0 - gb);
            const uint32_t pa = stage + ga * rb + lane * 16, pb = stage + gb * rb + lane * 16;
            float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 2
            for (int k = 0; k < q; ++k) {
                float r[E16];
                load_unit<E16>(sv + k * E16, r);
                if (va) acc0 = unit_dot<DT, 16>(acc0, pa + k * na * 16, r);
                if (vb) acc1 = unit_dot<DT, 16>(acc1, pb + k * nb * 16, r);
            }
            if (tb) {
                const uint32_t ta = stage + ga * rb + q * na * 16 + lane * tb;
                const uint32_t tbb = stage + gb * rb + q * nb * 16 + lane * tb;
                if (tb == 8) {
                    float r[2 * EPW];
                    load_unit<2 * EPW>(st_tail, r);
                    if (va) acc0 = unit_dot<DT, 8>(acc0, ta, r);
                    if (vb) acc1 = unit_dot<DT, 8>(acc1, tbb, r);
                } else {
                    for (int w = 0; w < tb / 4; ++w) {
                        float r[EPW];
                        load_unit<EPW>(st_tail + w * EPW, r);
                        if (va) acc0 = word_dot<DT>(acc0, lds32(ta + 4 * w), r);
                        if (vb) acc1 = word_dot<DT>(acc1, lds32(tbb + 4 * w), r);
                    }
                }
            }
            if (va) out[row0 + ra] = acc0;
            if (vb) out[row0 + rbw] = acc1;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&sh.empty_bar[st]));
    }
    return tile;
}

// The consumer warps: every tile of the block's slices, one partial vector per
// slice (partial[s][row] = the row's dot product with the slice's slopes, in unit
// order).  tile0: the running tile count at entry; returns the count at exit.  The
// next slice's layout is fetched while the present one is consumed.
template <int DT>
__device__ __forceinline__ int consume(const Args& g, const Plan& pl, Shared& sh, int tid, int tile0) {
    int tile = tile0;
    int rb = pl.rb0, lo = 0;
    for (int s = pl.sb0; s < pl.sb1; ++s) {
        int rb_next = 0, lo_next = 0;
        if (s + 1 < pl.sb1) {
            rb_next = __ldg(g.sl.rowbytes + s + 1);
            lo_next = __ldg(g.sl.loc + s + 1) - pl.loc0;
        }
        const int u = row_unit(rb);
        if (g.plane) tile = consume_slice_plane<DT>(g, pl, sh, tid, tile, s, rb, lo);
        else if (u == 16) tile = consume_slice<DT, 16>(g, pl, sh, tid, tile, s, rb, lo);
        else if (u == 8) tile = consume_slice<DT, 8>(g, pl, sh, tid, tile, s, rb, lo);
        else tile = consume_slice<DT, 4>(g, pl, sh, tid, tile, s, rb, lo);
        rb = rb_next;
        lo = lo_next;
    }
    return tile;
}

// After the grid barrier that follows every block's partials: the rows [r0, r1) of
// the block, 32 at a time (one per lane), each summed over the S slices in a fixed
// order -- warp w adds the slices w, w+14, w+28, ... in turn (coalesced loads of 32
// consecutive rows of one slice), then warp 0 adds the 14 warp sums in a pairwise
// tree -- then the row scale and the integrator.  dm_out: where the new commands go
// besides g.a.
template <int DT>
__device__ __forceinline__ void reduce_rows(const Args& g, const Plan& pl, int tid,
                                            float* __restrict__ dm_out) {
    const int warp = tid >> 5, lane = tid & 31;
    for (int base = pl.r0; base < pl.r1; base += 32) {
        const int row = base + lane;
        float v = 0.f;
        if (row < pl.r1) {
            float p[kSlicesPerWarp];
#pragma unroll
            for (int j = 0; j < kSlicesPerWarp; ++j) {
                const int s = warp + j * kConsumerWarps;
                p[j] = s < g.sl.S ? __ldcg(g.partial + static_cast<size_t>(s) * g.nact + row) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < kSlicesPerWarp; ++j)
                if (warp + j * kConsumerWarps < g.sl.S) v += p[j];
        }
        pl.red[warp * 32 + lane] = v;
        consumer_sync();
        if (warp == 0 && row < pl.r1) {
            float t[kConsumerWarps];
#pragma unroll
            for (int w = 0; w < kConsumerWarps; ++w) t[w] = pl.red[w * 32 + lane];
#pragma unroll
            for (int width = 1; width < kConsumerWarps; width <<= 1)
#pragma unroll
                for (int i = 0; i + width < kConsumerWarps; i += 2 * width) t[i] += t[i + width];
            // the shared copy of the state stays current for a persistent kernel
            pl.a_pre[row - pl.r0] = integrate_row<DT>(row, t[0], pl.a_pre[row - pl.r0], pl.sc_pre[row - pl.r0],
                                                      g.a, dm_out, g.gain, g.leak);
        }
        consumer_sync();
    }
}

// Grid barrier over co-resident blocks: one thread per block, between two
// block-level barriers.  The arrival is a release and the polling an acquire at
// GPU scope, so the block's writes before the first block barrier are visible to
// every block after its second one (no separate fences).  The counter only grows;
// the caller passes the arrival count that completes this barrier.  False (and
// RTC_ETIMEDOUT in the status word) if it did not complete within kWaitNs.
//
// The two halves may also be called apart (grid_arrive, then grid_wait): loads the
// thread issues in between do not hold up its arrival, which a release would
// otherwise wait for.
__device__ __forceinline__ void grid_arrive(unsigned long long* bar) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
}

__device__ __forceinline__ bool grid_wait(unsigned long long* bar, unsigned long long target, int* status,
                                          volatile int* abort) {
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
    return true;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long target,
                                             int* status, volatile int* abort) {
    grid_arrive(bar);
    return grid_wait(bar, target, status, abort);
}

// Grid, tiles, stages and dynamic shared memory of a launch for one handle.
struct Launch {
    int G, T, R, nst, stage_bytes, loc_floats, row_floats;
    size_t smem, region;
    bool ok;
};

// min_region: shared-memory scratch a fused phase needs.  Uses the handle's slice
// table, built when the matrix was loaded.
inline Launch plan_launch(const rtc_handle* h, size_t min_region = 0) {
    Launch L{};
    const int S = h->sl_S;
    L.G = S < h->num_sms ? S : h->num_sms;
    if (L.G < 1 || S < 1 || static_cast<int>(h->sl_rowbytes.size()) != S) return L;
    // largest row and largest block-local slope vector over the blocks
    int max_rb = 0, max_loc = 0;
    for (int b = 0; b < L.G; ++b) {
        const int s0 = static_cast<int>(static_cast<long long>(S) * b / L.G);
        const int s1 = static_cast<int>(static_cast<long long>(S) * (b + 1) / L.G);
        max_loc = std::max(max_loc, h->sl_loc[s1] - h->sl_loc[s0]);
        for (int s = s0; s < s1; ++s) max_rb = std::max(max_rb, h->sl_rowbytes[s]);
    }
    L.loc_floats = (max_loc + 3) / 4 * 4;
    L.row_floats = (h->cfg.nact + L.G - 1) / L.G;
    L.region = (min_region + 15) / 16 * 16;
    const size_t extra = L.region + 4 * static_cast<size_t>(L.loc_floats) +
                         8 * static_cast<size_t>(L.row_floats) + 4 * kConsumerWarps * 32;
    const size_t room = kDynSmemBudget > extra ? kDynSmemBudget - extra : 0;
    // lanes per row: the fewest for which two stages of R = kConsumers / T rows fit
    // (splitting rows further to keep the slopes in registers measured slower for
    // every store type: more tiles and butterflies cost more than the slope reads
    // they save).  Only the slices decide it, not the block count, so the order of
    // every row's sum is the same for any launch of the handle.
    auto stage = [&](int T) { return (static_cast<size_t>(kConsumers / T) * max_rb + 15) / 16 * 16; };
    L.T = 1;
    while (L.T < 16 && 2 * stage(L.T) > room) L.T *= 2;      // R stays a multiple of 4
    L.R = kConsumers / L.T;
    // stages of at least kMinTileBytes (whole multiples of R rows of the widest
    // slice), so that the per-tile handshakes stay a small part of the work
    const size_t st1 = stage(L.T);
    size_t m = st1 > 0 ? std::max<size_t>(1, kMinTileBytes / st1) : 1;
    while (m > 1 && 2 * m * st1 > room) --m;
    L.stage_bytes = static_cast<int>(m * st1);
    const size_t fit = L.stage_bytes > 0 ? room / L.stage_bytes : 0;
    L.nst = static_cast<int>(fit < static_cast<size_t>(kMaxStages) ? fit : kMaxStages);
    L.smem = static_cast<size_t>(L.nst) * L.stage_bytes + extra;
    L.ok = L.nst >= 2 && L.loc_floats <= kMaxLocalFloats && L.row_floats <= kMaxRowFloats &&
           S <= kMaxSlices && L.smem <= kDynSmemBudget && (!h->sl_plane || L.T == 1);
    return L;
}

inline Args make_args(const rtc_handle* h, const float* d_s, float* d_dm_out, const Launch& L) {
    Args g{};
    g.M = static_cast<const unsigned char*>(h->d_M);
    g.sl = Slices{h->d_sl_off, h->d_sl_rowbytes, h->d_sl_g0, h->d_sl_loc, h->sl_S,
                  h->sl_S > 0 ? h->sl_g0[h->sl_S] : 0, h->sl_equal ? 1 : 0};
    g.nact = h->cfg.nact;
    g.n_valid = h->n_valid;
    g.T = L.T;
    g.R = L.R;
    g.stage_bytes = L.stage_bytes;
    g.nst = L.nst;
    g.l2_policy = h->m_bytes <= kL2KeepBytes ? kL2Normal : kL2Stream;
    g.region = static_cast<int>(L.region);
    g.plane = h->sl_plane ? 1 : 0;
    g.loc_floats = L.loc_floats;
    g.row_floats = L.row_floats;
    g.s = d_s;
    g.scale = h->d_scale;
    g.partial = h->d_partial;
    g.a = h->d_a;
    g.dm_out = d_dm_out;
    g.gain = h->gain;
    g.leak = h->leak;
    g.status = h->d_status;
    return g;
}

}  // namespace rtc_mvm
