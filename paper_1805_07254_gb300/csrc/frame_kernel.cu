// Fused frame kernel: the whole per-frame pipeline of Sec. 2.1 / Fig. 3 in one
// cooperative launch.
//
// Each block owns a run of matrix slices (stream_mvm.cuh) and the subapertures
// whose slopes those slices multiply.  While its producer warp streams the slices'
// matrix tiles into shared memory (the matrix does not depend on the frame), the
// consumer warps compute the block's slopes (pixel.cuh) into shared memory and
// multiply them straight away: no block waits for another before its share of the
// product, as in the paper's per-thread column blocks (Sec. 2.3).  Each block
// writes one partial DM vector per slice; a bounded grid barrier then lets every
// block sum its share of the rows over the slices in a fixed order and apply the
// integrator (the partial-DM-vector tree of Sec. 2.3.5).
//
// The producer warp starts streaming at once: the ring's first tiles are in flight
// during the launch's cold start (instruction, parameter and table fetches after
// an L2 flush take the first ~3.5 us before a block can issue its pixel loads), and
// it holds the rest until the block's slopes are known.  (Measured: waiting for the
// pixel loads to be issued first, which kept them from queueing behind the bulk
// copies, came out 0.7-1 us later at the end of the stream.)
//
// With the learned slope predictor on (PRED), the measured slopes go into the
// history ring, a grid barrier makes them visible, each block predicts the next
// slopes of its own subapertures from their neighbourhoods (pred_tile.cuh, in the
// shared scratch before the slopes), writing them straight into its local slope
// vector, and multiplies the prediction.  The block arrives at the barrier before it
// fetches the network's weights (a release would wait for those loads), and the
// producer's hold lasts through the barrier and the prediction.
//
// For rtc_process_frame with pinned host buffers (HOST) the frame is read in place
// from mapped host memory and the DM commands are written there; the last block to
// finish writes the caller's completion record, so the host needs no copies and no
// stream synchronisation.  This is a separate instantiation: the device-frame kernel
// carries none of its code.
//
// The grid barrier counts block arrivals on a 64-bit counter that only grows;
// each barrier waits for the running total of arrivals expected up to and
// including its own, so the counter never needs a reset between launches (even
// when the block count changes).  All blocks are co-resident (cooperative
// launch, one block per SM).

#include "mlp.h"
#include "pixel.cuh"

#ifdef RTC_PHASE_STAMPS
// Diagnostic build only: %globaltimer at the sub-phases of the fused prediction of
// each block of the last launch (pred_tile.cuh).
__device__ unsigned long long g_rtc_pred_stamps[256][8];
#define RTC_PRED_STAMP(i)                                                          \
    do {                                                                           \
        unsigned long long t_;                                                     \
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                     \
        if (tid == 0) g_rtc_pred_stamps[blockIdx.x][i] = t_;                       \
    } while (0)
extern "C" int rtc_probe_pred_stamps(unsigned long long* out, int n) {
    return cudaMemcpyFromSymbol(out, g_rtc_pred_stamps, sizeof(unsigned long long) * 8 * (n < 256 ? n : 256)) ==
                   cudaSuccess
               ? 0
               : -1;
}
#endif

#include "pred_tile.cuh"
#include "stream_mvm.cuh"

#ifndef RTC_PRED_L2_TILES
#define RTC_PRED_L2_TILES 0
#endif
#ifndef RTC_PRED_PREFETCH_TILES
#define RTC_PRED_PREFETCH_TILES 1
#endif
#ifndef RTC_PREFETCH_TILES
#define RTC_PREFETCH_TILES 2
#endif

#ifdef RTC_PHASE_STAMPS
// Diagnostic build only: %globaltimer at the phases of each block of the last launch.
__device__ unsigned long long g_rtc_stamps[256][16];
#define RTC_STAMP(i)                                                   \
    do {                                                               \
        if (tid == 0) g_rtc_stamps[blockIdx.x][i] = rtc_mvm::global_ns(); \
    } while (0)
// the SM the block runs on, in the last entry
#define RTC_STAMP_SM()                                                 \
    do {                                                               \
        unsigned sm_;                                                  \
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm_));               \
        if (tid == 0) g_rtc_stamps[blockIdx.x][7] = sm_;               \
    } while (0)
extern "C" int rtc_probe_stamps(unsigned long long* out, int n) {
    return cudaMemcpyFromSymbol(out, g_rtc_stamps, sizeof(unsigned long long) * 16 * (n < 256 ? n : 256)) ==
                   cudaSuccess
               ? 0
               : -1;
}
#else
#define RTC_STAMP(i) \
    do {             \
    } while (0)
#define RTC_STAMP_SM() \
    do {               \
    } while (0)
#endif

namespace {

using namespace rtc_mvm;

// Matrix tiles the producer streams before the block's slopes are known (the
// ring's two stages).
constexpr int kPrefetchTiles = RTC_PREFETCH_TILES;
// With the predictor the hold lasts through the grid barrier and the prediction:
// this many tiles go to the ring, and this many further ones into L2, meanwhile.
// (Measured: four L2 tiles made the whole frame 3 us slower than none, their
// traffic queueing the prediction's latency-bound loads behind it.)
constexpr int kPredPrefetchTiles = RTC_PRED_PREFETCH_TILES;
constexpr int kPredL2Tiles = RTC_PRED_L2_TILES;

// HOST: the frame is in mapped host memory (rtc_process_frame with pinned buffers):
// each block copies its pixel rows into device staging (uncached 16-byte loads over
// the host link), and the last block to finish writes the caller's completion
// record (fh).
template <int DT, int NPX, bool PRED, bool HOST>
__global__ void __launch_bounds__(kThreads, 1)
frame_kernel(rtc_pixel::PixelArgs px, Args g, rtc_pred::PredArgs pa, int head,
             unsigned long long* gridbar, unsigned long long target, FrameHost fh) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    RTC_STAMP(0);
    RTC_STAMP_SM();
    const Plan pl = make_plan(g, smem);
    // the grid position of a consumer's first subaperture, loaded before the
    // block's set-up so that its latency overlaps it
    const int slot = 2 * (tid >> 5) + ((tid >> 4) & 1);
    const int2 pos0 = rtc_pixel::subap_pos(px, pl.g0 + slot, tid < kConsumers && pl.g0 + slot < pl.g1);
    if (tid == 0) init_shared(sh);
    __syncthreads();
    RTC_STAMP(8);
    if (tid >= kConsumers) {
        if ((tid & 31) == 0)
            produce(g, pl, sh, 0, true, PRED ? kPredPrefetchTiles : kPrefetchTiles, PRED ? kPredL2Tiles : 0);
        return;
    }
    clear_local(g, pl, tid);
    consumer_sync();
    RTC_STAMP(9);

    auto issued = [tid]() { RTC_STAMP(6); };   // the pixel loads are in flight
    // a frame in host memory: the block's pixel rows into device staging first, in
    // 16-byte units over the host link, while the matrix stream already runs (the
    // host link and HBM do not compete); the pixel stage then reads them through L2
    if (HOST) {
        rtc_pixel::ingest_block<kConsumers>(px.frame, fh.stage, fh.units, __ldg(fh.blk + blockIdx.x), fh.unit,
                                            tid);
        consumer_sync();
    }
    const uint16_t* frame = HOST ? fh.stage : px.frame;

    // pixel stage: the block's subapertures, one half-warp each (the ~26
    // subapertures of a block on the ELT frame take a single round)
    constexpr int kLoad = HOST ? rtc_pixel::kPixelL2 : rtc_pixel::kPixelReadOnly;
    for (int base = pl.g0; base < pl.g1; base += 2 * kConsumerWarps) {
        const int gi = base + slot;
        const bool valid = gi < pl.g1;
        const int2 pos = base == pl.g0 ? pos0 : rtc_pixel::subap_pos(px, gi, valid);
        const float2 sxy =
            rtc_pixel::subap_slopes_at<NPX, kLoad, 16>(px, frame, px.s, gi, valid, tid & 31, pos, issued);
        if (valid && (tid & 15) == 0) {
            int ix, iy;
            local_index(g, pl, gi, ix, iy);
            pl.loc[ix] = sxy.x;
            pl.loc[iy] = sxy.y;
        }
    }
    RTC_STAMP(1);
    prefetch_rows<DT>(g, pl, tid);

    unsigned long long next = target;   // arrivals that complete the next grid barrier
    if (PRED) {
        // every block's measured slopes in the history ring, then the prediction of
        // the block's own subapertures, which replaces their local slopes; the
        // network's weights are fetched after the block's arrival, while it waits
        consumer_sync();
        if (tid == 0) grid_arrive(gridbar);
        RTC_PRED_STAMP(5);
        rtc_pred::Regs pr;
        rtc_pred::prefetch(pa, pl.scratch, tid, pl.g0, pl.g1, head, pr);
        RTC_PRED_STAMP(6);
        if (tid == 0) grid_wait(gridbar, next, g.status, &sh.abort_flag);
        RTC_PRED_STAMP(7);
        consumer_sync();
        next += gridDim.x;
        if (!sh.abort_flag) {
            // the predictions replace the block's local slopes as they are made
            auto slot_of = [&](int gi, int axis) {
                int ix, iy;
                local_index(g, pl, gi, ix, iy);
                return axis ? iy : ix;
            };
            rtc_pred::predict(
                pa, pl.scratch, tid, pl.g0, pl.g1, head, pr,
                [&](int gi, int axis) { return pl.loc[slot_of(gi, axis)]; },
                [&](int gi, int axis, float v) { pl.loc[slot_of(gi, axis)] = v; });
        } else {
            rows_landed();              // the prefetch's copies, before the block exits
        }
    }
    consumer_sync();
    RTC_STAMP(2);
    if (tid == 0) sh.release = 1;       // the rest of the matrix stream may start
    consume<DT>(g, pl, sh, tid, 0);
    RTC_STAMP(3);
    rows_landed();

    // every block's partial vectors before any block sums them
    consumer_sync();
    if (tid == 0 && !sh.abort_flag) grid_barrier(gridbar, next, g.status, &sh.abort_flag);
    consumer_sync();
    RTC_STAMP(4);
    if (!sh.abort_flag) reduce_rows<DT>(g, pl, tid, g.dm_out);
    RTC_STAMP(5);

    if (HOST) {
        // the last block to finish writes the completion record (every block, aborted
        // or not, counts itself once)
        consumer_sync();
        if (tid == 0) {
            __threadfence_system();
            const unsigned long long prev = atomicAdd(fh.ctr, 1ull);
            if (prev + 1 == fh.target) {
                __threadfence_system();
                fh.done->status = *reinterpret_cast<volatile int*>(g.status);
                __threadfence_system();
                asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(&fh.done->seq), "l"(fh.seq) : "memory");
            }
        }
    }
}

template <int DT, int NPX, bool PRED, bool HOST>
cudaError_t launch_t(const Launch& L, rtc_pixel::PixelArgs px, Args g, rtc_pred::PredArgs pa, int head,
                     unsigned long long* bar, unsigned long long target, FrameHost fh, cudaStream_t st) {
    void* args[] = {&px, &g, &pa, &head, &bar, &target, &fh};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(frame_kernel<DT, NPX, PRED, HOST>),
                                       dim3(L.G), dim3(kThreads), args, L.smem, st);
}

template <int DT, bool PRED, bool HOST>
cudaError_t launch_npx(const rtc_handle* h, const Launch& L, rtc_pixel::PixelArgs px, Args g,
                       rtc_pred::PredArgs pa, int head, unsigned long long target, const FrameHost& fh,
                       cudaStream_t st) {
    if (h->cfg.npx == 10) return launch_t<DT, 10, PRED, HOST>(L, px, g, pa, head, h->d_gridbar, target, fh, st);
    return launch_t<DT, 0, PRED, HOST>(L, px, g, pa, head, h->d_gridbar, target, fh, st);
}

template <int DT, bool HOST>
cudaError_t launch_pred(const rtc_handle* h, const Launch& L, rtc_pixel::PixelArgs px, Args g, bool pred,
                        int head, unsigned long long target, const FrameHost& fh, cudaStream_t st) {
    if (pred) return launch_npx<DT, true, HOST>(h, L, px, g, pred_args(h), head, target, fh, st);
    const rtc_pred::PredArgs pa{};
    return launch_npx<DT, false, HOST>(h, L, px, g, pa, 0, target, fh, st);
}

template <int DT>
cudaError_t launch_dt(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, float* d_s_meas,
                      int head, cudaStream_t st, FrameHost* fhp) {
    const bool pred = d_s_meas != nullptr;
    const Launch L = plan_launch(h, pred ? rtc_pred::kSmemBytes : 0);
    if (!L.ok) return cudaErrorInvalidValue;
    const rtc_pixel::PixelArgs px = pixel_args(h, d_frame, pred ? d_s_meas : h->d_s);
    const Args g = make_args(h, h->d_s, d_dm_out, L);
    // the block count may change between launches (e.g. a server slot limits it), so
    // each target is the running total of expected arrivals, not launches x blocks
    const unsigned long long G = static_cast<unsigned long long>(L.G);
    const unsigned long long target = h->grid_epoch + G;
    FrameHost fh{};
    if (fhp) {
        fh = *fhp;
        fh.target = h->pf_arrivals + G;
        // the copy units of each block's pixel rows (16 bytes when the frame allows)
        const size_t fbytes = static_cast<size_t>(h->cfg.n_wfs) * h->side * h->side * 2;
        const uintptr_t bases = reinterpret_cast<uintptr_t>(d_frame) | reinterpret_cast<uintptr_t>(h->d_frame);
        fh.unit = (fbytes % 16 == 0 && bases % 16 == 0) ? 16 : (fbytes % 4 == 0 && bases % 4 == 0) ? 4 : 2;
        const int rc = build_ingest(h, L.G, fh.unit, 1);
        if (rc == RTC_ENOMEM) return cudaErrorMemoryAllocation;
        if (rc != RTC_OK) return cudaErrorUnknown;
        fh.units = h->d_units;
        fh.blk = h->d_blk;
        fh.stage = h->d_frame;
    }
    const cudaError_t e = fhp ? launch_pred<DT, true>(h, L, px, g, pred, head, target, fh, st)
                              : launch_pred<DT, false>(h, L, px, g, pred, head, target, fh, st);
    if (e == cudaSuccess) {
        h->grid_epoch = target + (pred ? G : 0);
        if (fhp) h->pf_arrivals = fh.target;
    }
    return e;
}

template <int DT, int NPX, bool PRED, bool HOST>
cudaError_t configure_t() {
    return cudaFuncSetAttribute(frame_kernel<DT, NPX, PRED, HOST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kDynSmemBudget));
}

template <int DT, bool HOST>
cudaError_t configure_host() {
    cudaError_t e = configure_t<DT, 10, false, HOST>();
    if (e == cudaSuccess) e = configure_t<DT, 0, false, HOST>();
    if (e == cudaSuccess) e = configure_t<DT, 10, true, HOST>();
    if (e == cudaSuccess) e = configure_t<DT, 0, true, HOST>();
    return e;
}

template <int DT>
cudaError_t configure_dt() {
    cudaError_t e = configure_host<DT, false>();
    if (e == cudaSuccess) e = configure_host<DT, true>();
    return e;
}

}  // namespace

cudaError_t frame_kernel_configure() {
    cudaError_t e = configure_dt<RTC_F32>();
    if (e == cudaSuccess) e = configure_dt<RTC_BF16>();
    if (e == cudaSuccess) e = configure_dt<RTC_F16>();
    if (e == cudaSuccess) e = configure_dt<RTC_FP8_E4M3>();
    if (e == cudaSuccess) e = configure_dt<RTC_INT8>();
    return e;
}

rtc_pred::PredArgs pred_args(const rtc_handle* h) {
    rtc_pred::PredArgs pa{};
    pa.w1 = h->pred->w1_bf16;
    pa.w2 = h->pred->w2_bf16;
    pa.params = h->pred->master;
    pa.nbr = h->d_nbr;
    pa.ring = h->d_ring;
    pa.s_pred = h->d_spred;
    pa.kpad = h->kpad;
    pa.nv = h->n_valid;
    pa.sigma = h->pred_sigma;
    pa.inv_sigma = 1.f / h->pred_sigma;
    return pa;
}

cudaError_t launch_frame(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, float* d_s_meas,
                         int head, cudaStream_t st, FrameHost* fh) {
    if (h->kpad == 0) return launch_decay(h, d_dm_out, st);
    switch (h->store) {
        case RTC_F32: return launch_dt<RTC_F32>(h, d_frame, d_dm_out, d_s_meas, head, st, fh);
        case RTC_BF16: return launch_dt<RTC_BF16>(h, d_frame, d_dm_out, d_s_meas, head, st, fh);
        case RTC_F16: return launch_dt<RTC_F16>(h, d_frame, d_dm_out, d_s_meas, head, st, fh);
        case RTC_FP8_E4M3: return launch_dt<RTC_FP8_E4M3>(h, d_frame, d_dm_out, d_s_meas, head, st, fh);
        case RTC_INT8: return launch_dt<RTC_INT8>(h, d_frame, d_dm_out, d_s_meas, head, st, fh);
        default: return cudaErrorInvalidValue;
    }
}
