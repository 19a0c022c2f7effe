// Persistent real-time loop kernel: the per-frame pipeline of Sec. 2.1 / Fig. 3,
// frame after frame, in one cooperative launch.
//
// The paper's RTC keeps its worker threads running and synchronises them by
// spinning on flags instead of sleeping (Sec. 2.3.2), and starts on the pixels of
// a frame while the camera is still reading it out (Sec. 2.2).  Here every block
// keeps running across frames:
//   1. thread 0 of each block spins (bounded, 2 s) on the frame slot's sequence
//      word in pinned host memory (a system-scope acquire load) until the band of
//      pixel rows that completes the block's subapertures has been published; a
//      stop value ends the loop;
//   2. the consumer warps copy the block's own pixels -- the sorted list of
//      copy units (16 bytes for ELT frames) that its subapertures' rows cover,
//      built on the host at launch -- from the host slot into a device staging
//      buffer, bypassing the caches (the slot is rewritten between its uses), and
//      compute the block's slopes from it through L2 into shared memory.  No block
//      waits for another: a frame's early bands are turned into slopes and into
//      partial DM vectors while later bands are still arriving;
//   3. with the learned predictor on (PRED), the measured slopes go to the next
//      row of the handle's history ring, a grid barrier makes them visible, and
//      each block replaces its subapertures' slopes by their prediction
//      (pred_tile.cuh);
//   4. each block multiplies its matrix slices by its own slopes, a grid barrier
//      publishes the partial DM vectors, and each block sums and integrates its
//      share of the rows (stream_mvm.cuh); DM commands go to the device state and
//      to the frame's slot in mapped host memory.  The partial vectors alternate
//      between two buffers frame by frame (see below);
//   5. the last block to finish publishes the completion record (sequence, the
//      latest device time at which a block had its rows, device time the commands
//      were written).
// The producer warp streams the matrix frame after frame; its barrier phases
// continue across frames, so the next frame's first tiles are already in flight
// while the kernel waits for the frame.
//
// Two blocks may both copy a unit that straddles their subapertures; they write
// the same bytes of the same frame.  A block only starts copying frame k + 1 after
// the grid barrier of frame k, which every block reaches after its pixel stage, so
// no copy overwrites pixels another block is still reading.  In the same way a
// block writes frame k + 2's partials (the buffer of frame k) only after the grid
// barrier of frame k + 1, which every block reaches after summing its rows of
// frame k (the barrier's release orders a block's earlier reads too).

#include <algorithm>
#include <vector>

#include "pixel.cuh"
#include "pred_tile.cuh"
#include "stream_mvm.cuh"

#ifdef RTC_PHASE_STAMPS
// Diagnostic build only: %globaltimer at the phases of each block's last frame.
__device__ unsigned long long g_rtc_loop_stamps[256][8];
#define RTC_LOOP_STAMP(i)                                                        \
    do {                                                                         \
        if (tid == 0) g_rtc_loop_stamps[blockIdx.x][i] = rtc_mvm::global_ns();   \
    } while (0)
extern "C" int rtc_probe_loop_stamps(unsigned long long* out, int n) {
    return cudaMemcpyFromSymbol(out, g_rtc_loop_stamps, sizeof(unsigned long long) * 8 * (n < 256 ? n : 256)) ==
                   cudaSuccess
               ? 0
               : -1;
}
#else
#define RTC_LOOP_STAMP(i) \
    do {                  \
    } while (0)
#endif

namespace {

using namespace rtc_mvm;
using rtc_pixel::copy_units;
using rtc_pixel::kNoUnit;
using rtc_pixel::kUnitRegs;

constexpr unsigned long long kFrameWaitNs = 2000ull * 1000 * 1000;   // 2 s for a frame to arrive
constexpr unsigned long long kStop = ~0ull;

#ifndef RTC_LOOP_POLLERS
#define RTC_LOOP_POLLERS 1
#endif
// Warps whose lane 0 polls host memory for the frame, their first polls spread over
// about one round trip.  One per polling block: four (to see a publication sooner)
// measured 6 us worse host to host.
constexpr int kPollers = RTC_LOOP_POLLERS;
#ifndef RTC_HOST_POLL_STRIDE
#define RTC_HOST_POLL_STRIDE 8
#endif
// With whole frames, one block in this many polls host memory for the frame.
constexpr int kHostPollStride = RTC_HOST_POLL_STRIDE;
constexpr unsigned long long kPollSpreadNs = 1200;

struct LoopArgs {
    rtc_pixel::PixelArgs px;           // frame and s are set per frame
    Args mv;                           // s and dm_out are set per frame
    const uint16_t* frames;            // mapped host ring [nslot][frame_elems]
    unsigned long long frame_elems;
    uint16_t* stage;                   // device [frame_elems]: this frame's pixels
    int copy_unit;                     // bytes per copy unit: 16, 4 or 2
    const unsigned* units;             // copy units (frame offset / copy_unit) of all blocks
    const int4* blk;                   // [G] first unit, end unit, band that completes the block
    int n_bands;                       // bands per frame: frame k band j is k * n_bands + j + 1
    const unsigned long long* seq;     // mapped host [nslot]: bands published
    const unsigned long long* ptrs;    // mapped host [nslot][2] or null: the frame's own
                                       // frame and DM buffers (device views; resident mode)
    int host_poll_stride;              // blocks b with b % stride == 0 poll host memory; the
                                       // others poll the device mirror (whole frames only)
    unsigned long long* mirror;        // device [nslot]: highest published value seen
    unsigned long long* mirror_ptrs;   // device [nslot][2]: the frame's buffers, copied
    float* dm_ring;                    // mapped host [nslot][nact]
    rtc_loop_done* done;               // mapped host [nslot]
    float* s_buf;                      // device [2][kpad]
    unsigned long long* gridbar;       // device, zero at launch
    size_t partial_stride;             // floats between the two partial-vector buffers
    unsigned long long* donectr;       // device, zero at launch
    unsigned long long* t_seen;        // device [2], zero at launch
    unsigned long long n_frames;
    int nslot;
    int kpad;
    rtc_pred::PredArgs pa;             // PRED only
    int head0;                         // PRED: ring row of the newest vector at launch
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu_max(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int DT, int NPX, bool PRED>
__global__ void __launch_bounds__(kThreads, 1) loop_kernel(LoopArgs L) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ int poll_state;               // this frame: 0 waiting, 1 published, 2 stop
    __shared__ const uint16_t* frame_in;     // this frame's pixels (ring slot or caller's buffer)
    __shared__ float* dm_to;                 // where this frame's DM commands go
    const int tid = threadIdx.x;
    const unsigned long long G = gridDim.x;
    // the block's plan lives in shared memory: kept in registers across the frame
    // loop it would push the reconstruction's working set into local memory
    __shared__ Plan pl;
    if (tid == 0) {
        init_shared(sh);
        pl = make_plan(L.mv, smem);
        poll_state = 0;
    }
    __syncthreads();

    if (tid >= kConsumers) {
        // producer: the matrix does not depend on the frame, so the next frame's
        // first tiles stream while the kernel waits for it
        if ((tid & 31) == 0) {
            int tl = 0;
            for (unsigned long long k = 0; k < L.n_frames && !sh.abort_flag; ++k)
                tl = produce(L.mv, pl, sh, tl, k + 1 == L.n_frames);
        }
        return;
    }

    clear_local(L.mv, pl, tid);         // the padding of the local slopes stays zero
    // integrator state and row scales of the block's rows: the reduction keeps the
    // shared copy of the state current from frame to frame
    prefetch_rows<DT>(L.mv, pl, tid);
    rows_landed();                      // once per loop: no need to overlap it
    // the block's calibration data (subaperture-major, contiguous), 128-byte lines
    const int npp = L.px.npx * L.px.npx;
    const long long cal_lines = (static_cast<long long>(pl.g1 - pl.g0) * npp * 4 + 127) / 128;
    const int slot_lane = 2 * (tid >> 5) + ((tid >> 4) & 1);
    // the grid position of the thread's first subaperture: the same every frame
    const int2 pos0 = rtc_pixel::subap_pos(L.px, pl.g0 + slot_lane, pl.g0 + slot_lane < pl.g1);
    constexpr unsigned long long kBarriers = PRED ? 2 : 1;     // grid barriers per frame
    int tile = 0;
    for (unsigned long long k = 0; k < L.n_frames; ++k) {
        const int slot = static_cast<int>(k % L.nslot);
        // the block's first copy units, fetched while thread 0 waits for the frame
        // (reloaded every frame, so that they hold no registers across the rest)
        const int4 bk = __ldg(L.blk + blockIdx.x);
        // warm L2 with the block's dark and gain values while the frame is awaited
        for (long long c = tid; c < 2 * cal_lines; c += kConsumers) {
            const float* base = c < cal_lines ? L.px.dark : L.px.gainmap;
            const long long line = c < cal_lines ? c : c - cal_lines;
            asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(
                reinterpret_cast<const char*>(base + static_cast<size_t>(pl.g0) * npp) + line * 128));
        }
        unsigned ur[kUnitRegs];
#pragma unroll
        for (int j = 0; j < kUnitRegs; ++j) {
            const int f = bk.x + tid + j * kConsumers;
            ur[j] = f < bk.y ? __ldg(L.units + f) : kNoUnit;
        }
        // 1. wait for the band of frame k that completes the block's subapertures:
        //    the pollers' first loads are staggered; whichever sees the band first
        //    (an acquire) reads the frame's buffers and tells the others.  With whole
        //    frames only every host_poll_stride-th block polls host memory; it copies
        //    what it saw into a device mirror (a release), which the other blocks
        //    poll in L2, so that the host link carries a few polls instead of one per
        //    block
        if ((tid & 31) == 0 && (tid >> 5) < kPollers) {
            volatile int* state = &poll_state;
            const unsigned long long want = k * static_cast<unsigned long long>(L.n_bands) + bk.z + 1;
            const bool host = blockIdx.x % L.host_poll_stride == 0;
            const bool mirrored = L.host_poll_stride > 1;
            const unsigned long long t0 = global_ns();
            const unsigned long long delay = (tid >> 5) * kPollSpreadNs / kPollers;
            while (*state == 0 && global_ns() - t0 < delay) {
            }
            while (*state == 0) {
                const unsigned long long v = host ? ld_acquire_sys(L.seq + slot) : ld_acquire_gpu(L.mirror + slot);
                const unsigned long long t = global_ns();
                if (v == kStop) {
                    if (host && mirrored) red_release_gpu_max(L.mirror + slot, v);
                    *state = 2;
                    break;
                }
                if (v >= want) {
                    // the frame's buffers: written by the host before it published the frame
                    const uint16_t* fr = L.frames + static_cast<size_t>(slot) * L.frame_elems;
                    float* dm = L.dm_ring + static_cast<size_t>(slot) * L.mv.nact;
                    if (L.ptrs) {
                        const unsigned long long* src = host ? L.ptrs : L.mirror_ptrs;
                        const unsigned long long a = host ? ld_relaxed_sys(src + 2 * slot) : ld_relaxed_gpu(src + 2 * slot);
                        const unsigned long long b =
                            host ? ld_relaxed_sys(src + 2 * slot + 1) : ld_relaxed_gpu(src + 2 * slot + 1);
                        fr = reinterpret_cast<const uint16_t*>(a);
                        dm = reinterpret_cast<float*>(b);
                        if (host && mirrored) {
                            L.mirror_ptrs[2 * slot] = a;
                            L.mirror_ptrs[2 * slot + 1] = b;
                        }
                    }
                    if (host && mirrored) red_release_gpu_max(L.mirror + slot, v);
                    frame_in = fr;
                    dm_to = dm;
                    atomicMax(L.t_seen + (k & 1), t);
                    *state = 1;
                    break;
                }
                if (t - t0 > kFrameWaitNs) {
                    atomicExch(L.mv.status, RTC_ETIMEDOUT);
                    *state = 2;
                    break;
                }
            }
        }
        consumer_sync();
        if (poll_state == 2) {
            if (tid == 0) sh.abort_flag = 1;        // the producer stops too
            break;
        }
        // every thread has read the state (a late reader may see the reset: it only
        // tests for a stop), and the next frame's pollers start after later barriers
        if (tid == 0) poll_state = 0;
        RTC_LOOP_STAMP(0);

        // 2. the block's pixels into device memory, then the block's slopes from
        //    them, into the local vector (and the global one)
        const uint16_t* frame = frame_in;
        const int f_over = bk.x + tid + kUnitRegs * kConsumers;
        if (L.copy_unit == 16)
            copy_units<uint4, kConsumers>(frame, L.stage, L.units, bk.y, ur, f_over);
        else if (L.copy_unit == 4)
            copy_units<unsigned, kConsumers>(frame, L.stage, L.units, bk.y, ur, f_over);
        else
            copy_units<unsigned short, kConsumers>(frame, L.stage, L.units, bk.y, ur, f_over);
        consumer_sync();
        RTC_LOOP_STAMP(1);
        const int head = (L.head0 + 1 + static_cast<int>(k & 3)) & 3;
        float* s_k = PRED ? L.pa.ring + static_cast<size_t>(head) * L.kpad
                          : L.s_buf + static_cast<size_t>(k & 1) * L.kpad;
        for (int base = pl.g0; base < pl.g1; base += 2 * kConsumerWarps) {
            const int gi = base + slot_lane;
            const bool valid = gi < pl.g1;
            const int2 pos = base == pl.g0 ? pos0 : rtc_pixel::subap_pos(L.px, gi, valid);
            const float2 sxy = rtc_pixel::subap_slopes_at<NPX, rtc_pixel::kPixelL2, 16>(
                L.px, L.stage, s_k, gi, valid, tid & 31, pos);
            if (valid && (tid & 15) == 0) {
                int ix, iy;
                local_index(L.mv, pl, gi, ix, iy);
                pl.loc[ix] = sxy.x;
                pl.loc[iy] = sxy.y;
            }
        }

        // 3. with the predictor: every block's measured slopes in the history ring,
        //    then the prediction of the block's own subapertures
        if (PRED) {
            consumer_sync();
            if (tid == 0) grid_arrive(L.gridbar);
            rtc_pred::Regs pr;
            rtc_pred::prefetch(L.pa, pl.scratch, tid, pl.g0, pl.g1, head, pr);   // overlaps the barrier's wait
            if (tid == 0) grid_wait(L.gridbar, G * (kBarriers * k + 1), L.mv.status, &sh.abort_flag);
            consumer_sync();
            if (sh.abort_flag) {
                rows_landed();          // the prefetch's copies, before the block exits
                break;
            }
            // the predictions replace the block's local slopes as they are made
            auto slot_of = [&](int gi, int axis) {
                int ix, iy;
                local_index(L.mv, pl, gi, ix, iy);
                return axis ? iy : ix;
            };
            rtc_pred::predict(
                L.pa, pl.scratch, tid, pl.g0, pl.g1, head, pr,
                [&](int gi, int axis) { return pl.loc[slot_of(gi, axis)]; },
                [&](int gi, int axis, float v) { pl.loc[slot_of(gi, axis)] = v; });
        }
        consumer_sync();

        // 4. the block's partial DM vectors (this frame's buffer), then its rows summed
        //    and integrated; DM commands to the device state and the frame's host slot
        Args mv = L.mv;
        mv.partial = L.mv.partial + (k & 1) * L.partial_stride;
        RTC_LOOP_STAMP(2);
        tile = consume<DT>(mv, pl, sh, tid, tile);
        RTC_LOOP_STAMP(3);
        consumer_sync();
        if (tid == 0) grid_barrier(L.gridbar, G * (kBarriers * k + kBarriers), L.mv.status, &sh.abort_flag);
        consumer_sync();
        if (sh.abort_flag) break;
        RTC_LOOP_STAMP(4);
        reduce_rows<DT>(mv, pl, tid, dm_to);
        RTC_LOOP_STAMP(5);

        // 5. the last block to finish publishes the completion record
        consumer_sync();
        if (tid == 0) {
            __threadfence_system();
            const unsigned long long prev = atomicAdd(L.donectr, 1ull);
            if (prev + 1 == G * (k + 1)) {
                rtc_loop_done* d = L.done + slot;
                // the latest time a block had its rows; cleared for frame k + 2, whose
                // blocks start after the grid barrier of frame k + 1
                d->t_seen = atomicExch(L.t_seen + (k & 1), 0ull);
                d->t_done = global_ns();
                __threadfence_system();
                st_release_sys(&d->seq, k + 1);
            }
        }
    }
}

template <int DT, int NPX, bool PRED>
cudaError_t launch_t(const Launch& Lc, LoopArgs a, cudaStream_t st) {
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(loop_kernel<DT, NPX, PRED>),
                                       dim3(Lc.G), dim3(kThreads), args, Lc.smem, st);
}

}  // namespace

// The copy units and the completing band of every block of a G-block launch
// (plan_ingest: for each run of the block's subapertures that are neighbours in
// one row of the subaperture grid, the units its pixel rows cover; sorted and
// without repeats, so that neighbouring threads read neighbouring units).
int build_ingest(rtc_handle* h, int G, int unit, int n_bands) {
    if (h->ingest_G == G && h->ingest_unit == unit && h->ingest_bands == n_bands) return RTC_OK;
    h->ingest_G = -1;
    std::vector<unsigned> units;
    std::vector<int> b4;
    plan_ingest(h->rc.data(), h->n_valid, h->cfg.npx, h->side, h->sl_g0.data(), h->sl_S, G, unit, n_bands,
                units, b4);
    std::vector<int4> blk(G);
    for (int b = 0; b < G; ++b) blk[b] = make_int4(b4[4 * b], b4[4 * b + 1], b4[4 * b + 2], 0);
    if (units.empty()) units.push_back(0);
    if (units.size() > h->units_cap) {
        if (h->d_units) cudaFree(h->d_units);
        h->d_units = nullptr;
        h->units_cap = 0;
        if (cudaMalloc(&h->d_units, units.size() * sizeof(unsigned)) != cudaSuccess) return RTC_ENOMEM;
        h->units_cap = units.size();
    }
    if (!h->d_blk && cudaMalloc(&h->d_blk, static_cast<size_t>(h->dev_sms) * sizeof(int4)) != cudaSuccess)
        return RTC_ENOMEM;
    if (cudaMemcpy(h->d_units, units.data(), units.size() * sizeof(unsigned), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(h->d_blk, blk.data(), G * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return RTC_EDEVICE;
    h->ingest_G = G;
    h->ingest_unit = unit;
    h->ingest_bands = n_bands;
    return RTC_OK;
}

namespace {

template <int DT>
cudaError_t launch_dt(rtc_handle* h, const LoopLaunch& ll, cudaStream_t st) {
    const bool pred = h->pred_on;
    const Launch Lc = plan_launch(h, pred ? rtc_pred::kSmemBytes : 0);
    if (!Lc.ok || Lc.G > h->dev_sms) return cudaErrorInvalidValue;
    LoopArgs a{};
    a.px = pixel_args(h, nullptr, nullptr);
    a.mv = make_args(h, nullptr, nullptr, Lc);
    if (ll.l2_stream) a.mv.l2_policy = kL2Stream;
    a.frames = ll.d_frames;
    a.frame_elems = ll.frame_elems;
    a.stage = h->d_frame;
    const size_t fbytes = ll.frame_elems * 2;
    const uintptr_t bases = reinterpret_cast<uintptr_t>(ll.d_frames) | reinterpret_cast<uintptr_t>(h->d_frame);
    a.copy_unit = (fbytes % 16 == 0 && bases % 16 == 0) ? 16 : (fbytes % 4 == 0 && bases % 4 == 0) ? 4 : 2;
    const int rc = build_ingest(h, Lc.G, a.copy_unit, ll.n_bands);
    if (rc == RTC_ENOMEM) return cudaErrorMemoryAllocation;
    if (rc != RTC_OK) return cudaErrorUnknown;
    a.units = h->d_units;
    a.blk = h->d_blk;
    a.n_bands = ll.n_bands;
    a.seq = ll.d_seq;
    a.ptrs = ll.d_ptrs;
    a.host_poll_stride = ll.n_bands == 1 ? kHostPollStride : 1;
    a.mirror = h->d_mirror;
    a.mirror_ptrs = h->d_mirror + RTC_LOOP_SLOTS;
    a.dm_ring = ll.d_dm;
    a.done = ll.d_done;
    a.s_buf = h->d_sbuf;
    a.gridbar = h->d_gridbar;
    a.partial_stride = static_cast<size_t>(h->dev_sms) * h->cfg.nact;
    a.donectr = h->d_donectr;
    a.t_seen = h->d_tseen;
    a.n_frames = ll.n_frames;
    a.nslot = ll.nslot;
    a.kpad = h->kpad;
    const bool npx10 = h->cfg.npx == 10;
    if (pred) {
        a.pa = pred_args(h);
        a.head0 = h->ring_head;
        return npx10 ? launch_t<DT, 10, true>(Lc, a, st) : launch_t<DT, 0, true>(Lc, a, st);
    }
    return npx10 ? launch_t<DT, 10, false>(Lc, a, st) : launch_t<DT, 0, false>(Lc, a, st);
}

template <int DT, int NPX, bool PRED>
cudaError_t configure_t() {
    return cudaFuncSetAttribute(loop_kernel<DT, NPX, PRED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kDynSmemBudget));
}

template <int DT>
cudaError_t configure_dt() {
    cudaError_t e = configure_t<DT, 10, false>();
    if (e == cudaSuccess) e = configure_t<DT, 0, false>();
    if (e == cudaSuccess) e = configure_t<DT, 10, true>();
    if (e == cudaSuccess) e = configure_t<DT, 0, true>();
    return e;
}

}  // namespace

cudaError_t loop_kernel_configure() {
    cudaError_t e = configure_dt<RTC_F32>();
    if (e == cudaSuccess) e = configure_dt<RTC_BF16>();
    if (e == cudaSuccess) e = configure_dt<RTC_F16>();
    if (e == cudaSuccess) e = configure_dt<RTC_FP8_E4M3>();
    if (e == cudaSuccess) e = configure_dt<RTC_INT8>();
    return e;
}

cudaError_t launch_loop(rtc_handle* h, const LoopLaunch& ll, cudaStream_t st) {
    switch (h->store) {
        case RTC_F32: return launch_dt<RTC_F32>(h, ll, st);
        case RTC_BF16: return launch_dt<RTC_BF16>(h, ll, st);
        case RTC_F16: return launch_dt<RTC_F16>(h, ll, st);
        case RTC_FP8_E4M3: return launch_dt<RTC_FP8_E4M3>(h, ll, st);
        case RTC_INT8: return launch_dt<RTC_INT8>(h, ll, st);
        default: return cudaErrorInvalidValue;
    }
}
