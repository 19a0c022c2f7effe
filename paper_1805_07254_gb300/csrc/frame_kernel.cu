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
// The grid barrier counts block arrivals on a 64-bit counter that only grows;
// each launch waits for the running total of arrivals expected up to and
// including its own blocks, so the counter never needs a reset between launches
// (even when the block count changes).  All blocks are co-resident (cooperative
// launch, one block per SM).

#include "pixel.cuh"
#include "stream_mvm.cuh"

namespace {

using namespace rtc_mvm;

template <int DT, bool S_SMEM, int NPX>
__global__ void __launch_bounds__(kThreads, 1)
frame_kernel(rtc_pixel::PixelArgs px, Args g, unsigned long long* gridbar,
             unsigned long long target) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    if (tid == 0) init_shared(sh);
    __syncthreads();
    const Plan pl = make_plan<DT, S_SMEM>(g, smem);
    if (tid >= kConsumers) {
        if ((tid & 31) < kTeams) produce(g, pl, sh, tid & 31);
        return;
    }
    // pixel stage: this block's share of the subapertures, one half-warp each (so
    // the ~26 subapertures of a block on the ELT frame take a single round)
    const int nt = px.n_valid * px.n_wfs;
    const int i0 = static_cast<int>(static_cast<long long>(nt) * blockIdx.x / gridDim.x);
    const int i1 = static_cast<int>(static_cast<long long>(nt) * (blockIdx.x + 1) / gridDim.x);
    const int slot = 2 * (tid >> 5) + ((tid >> 4) & 1);
    for (int base = i0; base < i1; base += 2 * kConsumerWarps) {
        const int gi = base + slot;
        rtc_pixel::subap_slopes<NPX, rtc_pixel::kPixelReadOnly, 16>(px, px.frame, px.s, gi, gi < i1,
                                                                    tid & 31);
    }
    // every block's slopes must be visible before any block reads s
    consumer_sync();
    if (tid == 0) grid_barrier(gridbar, target, g.status, &sh.abort_flag);
    consumer_sync();
    consumer_prologue<DT, S_SMEM, true>(g, pl, tid, g.s);
    consume<DT, S_SMEM, true>(g, pl, sh, tid, 0, g.s, g.dm_out);
}

template <int DT, bool S, int NPX>
cudaError_t launch_t(const Launch& L, rtc_pixel::PixelArgs px, Args g, unsigned long long* bar,
                     unsigned long long target, cudaStream_t st) {
    void* args[] = {&px, &g, &bar, &target};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(frame_kernel<DT, S, NPX>),
                                       dim3(L.G), dim3(kThreads), args, L.smem, st);
}

template <int DT, bool S>
cudaError_t launch_npx(const rtc_handle* h, const Launch& L, rtc_pixel::PixelArgs px, Args g,
                       unsigned long long target, cudaStream_t st) {
    if (h->cfg.npx == 10) return launch_t<DT, S, 10>(L, px, g, h->d_gridbar, target, st);
    return launch_t<DT, S, 0>(L, px, g, h->d_gridbar, target, st);
}

template <int DT>
cudaError_t launch_dt(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, cudaStream_t st) {
    const Launch L = plan_launch(h, Epc<DT>::v);
    if (!L.ok) return cudaErrorInvalidValue;
    const rtc_pixel::PixelArgs px = pixel_args(h, d_frame, h->d_s);
    const Args g = make_args(h, h->d_s, d_dm_out, L.nst, Epc<DT>::v);
    // the block count may change between launches (e.g. a server slot limits it), so
    // the target is the running total of expected arrivals, not launches x blocks
    const unsigned long long target = h->grid_epoch + static_cast<unsigned long long>(L.G);
    const cudaError_t e = L.s_in_smem ? launch_npx<DT, true>(h, L, px, g, target, st)
                                      : launch_npx<DT, false>(h, L, px, g, target, st);
    if (e == cudaSuccess) h->grid_epoch = target;
    return e;
}

template <int DT, bool S, int NPX>
cudaError_t configure_t() {
    return cudaFuncSetAttribute(frame_kernel<DT, S, NPX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kDynSmemBudget));
}

template <int DT>
cudaError_t configure_dt() {
    cudaError_t e = configure_t<DT, true, 10>();
    if (e == cudaSuccess) e = configure_t<DT, true, 0>();
    if (e == cudaSuccess) e = configure_t<DT, false, 10>();
    if (e == cudaSuccess) e = configure_t<DT, false, 0>();
    return e;
}

}  // namespace

cudaError_t frame_kernel_configure() {
    cudaError_t e = configure_dt<RTC_F32>();
    if (e == cudaSuccess) e = configure_dt<RTC_BF16>();
    if (e == cudaSuccess) e = configure_dt<RTC_FP8_E4M3>();
    return e;
}

cudaError_t launch_frame(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, cudaStream_t st) {
    if (h->kpad == 0) return launch_decay(h, d_dm_out, st);
    switch (h->store) {
        case RTC_F32: return launch_dt<RTC_F32>(h, d_frame, d_dm_out, st);
        case RTC_BF16: return launch_dt<RTC_BF16>(h, d_frame, d_dm_out, st);
        case RTC_FP8_E4M3: return launch_dt<RTC_FP8_E4M3>(h, d_frame, d_dm_out, st);
        default: return cudaErrorInvalidValue;
    }
}
