// Fused frame kernel: the whole per-frame pipeline of Sec. 2.1 / Fig. 3 in one
// cooperative launch.
//
// While the producer warps of every block start streaming matrix tiles into
// shared memory (the matrix does not depend on the frame), the consumer warps
// compute the block's share of the slopes (pixel.cuh); a bounded grid barrier then
// makes the whole slope vector visible, and the consumers run the streaming
// reconstruction and integrator (stream_mvm.cuh).  The pixel work and the
// launch of the reconstruction are hidden under the first matrix tiles, much as
// DARC's horizontal processing overlaps work with pixel arrival (Sec. 2.2).
//
// With the learned slope predictor on (PRED), the measured slopes go into the
// history ring, a second phase between two grid barriers predicts the next
// slopes of every subaperture (pred_tile.cuh, in the shared memory the slope copy
// takes later), and the reconstruction multiplies the prediction.
//
// The grid barrier counts block arrivals on a 64-bit counter that only grows;
// each barrier waits for the running total of arrivals expected up to and
// including its own, so the counter never needs a reset between launches (even
// when the block count changes).  All blocks are co-resident (cooperative
// launch, one block per SM).

#include "mlp.h"
#include "pixel.cuh"
#include "pred_tile.cuh"
#include "stream_mvm.cuh"

namespace {

using namespace rtc_mvm;

// Named barrier on which the producer warp waits until every consumer warp has
// issued its first pixel loads: the matrix prefetch fills the memory system for
// microseconds, and pixel loads queued behind it would delay the whole frame.
constexpr int kGateBar = 4;
// Matrix tiles each team's producer streams before the slopes are known; the rest
// follows once they are (a flood of bulk copies would slow the pixel loads and the
// grid barrier's round trips, which are on the frame's critical path).
constexpr int kPrefetchTiles = 1;

template <int DT, bool S_SMEM, int NPX, bool PRED>
__global__ void __launch_bounds__(kThreads, 1)
frame_kernel(rtc_pixel::PixelArgs px, Args g, rtc_pred::PredArgs pa, int head,
             unsigned long long* gridbar, unsigned long long target) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    if (tid == 0) init_shared(sh);
    __syncthreads();
    const Plan pl = make_plan<DT, S_SMEM>(g, smem);
    if (tid >= kConsumers) {
        asm volatile("bar.sync %0, %1;" ::"n"(kGateBar), "n"(kThreads) : "memory");
        if ((tid & 31) < kTeams) produce(g, pl, sh, tid & 31, 0, true, kPrefetchTiles);
        return;
    }
    // pixel stage: this block's share of the subapertures, one half-warp each (so
    // the ~26 subapertures of a block on the ELT frame take a single round)
    const int nt = px.n_valid * px.n_wfs;
    const int i0 = static_cast<int>(static_cast<long long>(nt) * blockIdx.x / gridDim.x);
    const int i1 = static_cast<int>(static_cast<long long>(nt) * (blockIdx.x + 1) / gridDim.x);
    const int slot = 2 * (tid >> 5) + ((tid >> 4) & 1);
    bool gate_open = false;             // every consumer warp arrives exactly once
    auto open_gate = [&gate_open]() {
        if (!gate_open) {
            asm volatile("bar.arrive %0, %1;" ::"n"(kGateBar), "n"(kThreads) : "memory");
            gate_open = true;
        }
    };
    for (int base = i0; base < i1; base += 2 * kConsumerWarps) {
        const int gi = base + slot;
        rtc_pixel::subap_slopes<NPX, rtc_pixel::kPixelReadOnly, 16>(px, px.frame, px.s, gi, gi < i1,
                                                                    tid & 31, open_gate);
    }
    open_gate();                        // a warp without pixel work
    // every block's slopes must be visible before any block reads s
    consumer_sync();
    if (tid == 0) grid_barrier(gridbar, target, g.status, &sh.abort_flag);
    consumer_sync();
    const float* s_vec = g.s;
    if (PRED) {
        // next slopes of the block's subapertures from the 4 newest measured vectors
        if (!sh.abort_flag) rtc_pred::predict(pa, pl.scratch, tid, i0, i1, head);
        if (tid == 0 && !sh.abort_flag)
            grid_barrier(gridbar, target + gridDim.x, g.status, &sh.abort_flag);
        consumer_sync();
        s_vec = pa.s_pred;
    }
    consumer_prologue<DT, S_SMEM, true>(g, pl, tid, s_vec);
    if (tid == 0) sh.release = 1;       // the rest of the matrix stream may start
    consume<DT, S_SMEM, true>(g, pl, sh, tid, 0, s_vec, g.dm_out);
}

template <int DT, bool S, int NPX, bool PRED>
cudaError_t launch_t(const Launch& L, rtc_pixel::PixelArgs px, Args g, rtc_pred::PredArgs pa, int head,
                     unsigned long long* bar, unsigned long long target, cudaStream_t st) {
    void* args[] = {&px, &g, &pa, &head, &bar, &target};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(frame_kernel<DT, S, NPX, PRED>),
                                       dim3(L.G), dim3(kThreads), args, L.smem, st);
}

template <int DT, bool S, bool PRED>
cudaError_t launch_npx(const rtc_handle* h, const Launch& L, rtc_pixel::PixelArgs px, Args g,
                       rtc_pred::PredArgs pa, int head, unsigned long long target, cudaStream_t st) {
    if (h->cfg.npx == 10) return launch_t<DT, S, 10, PRED>(L, px, g, pa, head, h->d_gridbar, target, st);
    return launch_t<DT, S, 0, PRED>(L, px, g, pa, head, h->d_gridbar, target, st);
}

template <int DT>
cudaError_t launch_dt(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, float* d_s_meas,
                      int head, cudaStream_t st) {
    const bool pred = d_s_meas != nullptr;
    const Launch L = plan_launch(h, Epc<DT>::v, pred ? rtc_pred::kSmemBytes : 0);
    if (!L.ok || (pred && !L.s_in_smem)) return cudaErrorInvalidValue;
    const rtc_pixel::PixelArgs px = pixel_args(h, d_frame, pred ? d_s_meas : h->d_s);
    const Args g = make_args(h, h->d_s, d_dm_out, L, Epc<DT>::v);
    // the block count may change between launches (e.g. a server slot limits it), so
    // each target is the running total of expected arrivals, not launches x blocks
    const unsigned long long G = static_cast<unsigned long long>(L.G);
    const unsigned long long target = h->grid_epoch + G;
    cudaError_t e;
    if (pred) {
        const rtc_pred::PredArgs pa = pred_args(h);
        e = launch_npx<DT, true, true>(h, L, px, g, pa, head, target, st);
    } else {
        const rtc_pred::PredArgs pa{};
        e = L.s_in_smem ? launch_npx<DT, true, false>(h, L, px, g, pa, 0, target, st)
                        : launch_npx<DT, false, false>(h, L, px, g, pa, 0, target, st);
    }
    if (e == cudaSuccess) h->grid_epoch = target + (pred ? G : 0);
    return e;
}

template <int DT, bool S, int NPX, bool PRED>
cudaError_t configure_t() {
    return cudaFuncSetAttribute(frame_kernel<DT, S, NPX, PRED>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kDynSmemBudget));
}

template <int DT>
cudaError_t configure_dt() {
    cudaError_t e = configure_t<DT, true, 10, false>();
    if (e == cudaSuccess) e = configure_t<DT, true, 0, false>();
    if (e == cudaSuccess) e = configure_t<DT, false, 10, false>();
    if (e == cudaSuccess) e = configure_t<DT, false, 0, false>();
    if (e == cudaSuccess) e = configure_t<DT, true, 10, true>();
    if (e == cudaSuccess) e = configure_t<DT, true, 0, true>();
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
                         int head, cudaStream_t st) {
    if (h->kpad == 0) return launch_decay(h, d_dm_out, st);
    switch (h->store) {
        case RTC_F32: return launch_dt<RTC_F32>(h, d_frame, d_dm_out, d_s_meas, head, st);
        case RTC_BF16: return launch_dt<RTC_BF16>(h, d_frame, d_dm_out, d_s_meas, head, st);
        case RTC_F16: return launch_dt<RTC_F16>(h, d_frame, d_dm_out, d_s_meas, head, st);
        case RTC_FP8_E4M3: return launch_dt<RTC_FP8_E4M3>(h, d_frame, d_dm_out, d_s_meas, head, st);
        case RTC_INT8: return launch_dt<RTC_INT8>(h, d_frame, d_dm_out, d_s_meas, head, st);
        default: return cudaErrorInvalidValue;
    }
}
