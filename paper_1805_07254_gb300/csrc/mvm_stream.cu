// Stand-alone reconstruction kernel (d = M s and the leaky integrator, Fig. 3
// (c)-(d)) on a full slope vector; the device code is in stream_mvm.cuh.  Used by
// rtc_reconstruct_async; rtc_process_frame runs the fused frame kernel, which gives
// the same results bit for bit (same slices, same partials, same sum).  One
// cooperative launch: each block gathers its slices' slopes, streams their matrix
// bytes into partial vectors, and after a grid barrier reduces its share of rows.

#include "stream_mvm.cuh"

namespace {

using namespace rtc_mvm;

template <int DT>
__global__ void __launch_bounds__(kThreads, 1)
mvm_stream_kernel(Args g, unsigned long long* gridbar, unsigned long long target) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    if (tid == 0) init_shared(sh);
    __syncthreads();
    const Plan pl = make_plan(g, smem);
    if (tid >= kConsumers) {
        if ((tid & 31) == 0) produce(g, pl, sh);
        return;
    }
    clear_local(g, pl, tid);
    consumer_sync();
    gather_local(g, pl, tid, g.s, false);
    prefetch_rows<DT>(g, pl, tid);
    consumer_sync();
    consume<DT>(g, pl, sh, tid, 0);
    rows_landed();
    // every block's partial vectors before any block sums them
    consumer_sync();
    if (tid == 0) grid_barrier(gridbar, target, g.status, &sh.abort_flag);
    consumer_sync();
    if (!sh.abort_flag) reduce_rows<DT>(g, pl, tid, g.dm_out);
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
cudaError_t launch_stream(rtc_handle* h, const float* d_s, float* d_dm_out, cudaStream_t st) {
    const Launch L = plan_launch(h);
    if (!L.ok) return cudaErrorInvalidValue;
    Args g = make_args(h, d_s, d_dm_out, L);
    unsigned long long* bar = h->d_gridbar;
    unsigned long long target = h->grid_epoch + static_cast<unsigned long long>(L.G);
    void* args[] = {&g, &bar, &target};
    const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(mvm_stream_kernel<DT>),
                                                      dim3(L.G), dim3(kThreads), args, L.smem, st);
    if (e == cudaSuccess) h->grid_epoch = target;
    return e;
}

template <int DT>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(mvm_stream_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kDynSmemBudget));
}

}  // namespace

cudaError_t mvm_stream_configure() {
    cudaError_t e = configure_one<RTC_F32>();
    if (e == cudaSuccess) e = configure_one<RTC_BF16>();
    if (e == cudaSuccess) e = configure_one<RTC_F16>();
    if (e == cudaSuccess) e = configure_one<RTC_FP8_E4M3>();
    if (e == cudaSuccess) e = configure_one<RTC_INT8>();
    return e;
}

cudaError_t launch_decay(const rtc_handle* h, float* d_dm_out, cudaStream_t st) {
    decay_kernel<<<(h->cfg.nact + 255) / 256, 256, 0, st>>>(h->cfg.nact, h->d_a, d_dm_out, h->leak);
    return cudaGetLastError();
}

cudaError_t launch_mvm_integrate(rtc_handle* h, const float* d_s, float* d_dm_out, cudaStream_t st) {
    if (h->kpad == 0) return launch_decay(h, d_dm_out, st);
    switch (h->store) {
        case RTC_F32: return launch_stream<RTC_F32>(h, d_s, d_dm_out, st);
        case RTC_BF16: return launch_stream<RTC_BF16>(h, d_s, d_dm_out, st);
        case RTC_F16: return launch_stream<RTC_F16>(h, d_s, d_dm_out, st);
        case RTC_FP8_E4M3: return launch_stream<RTC_FP8_E4M3>(h, d_s, d_dm_out, st);
        case RTC_INT8: return launch_stream<RTC_INT8>(h, d_s, d_dm_out, st);
        default: return cudaErrorInvalidValue;
    }
}
