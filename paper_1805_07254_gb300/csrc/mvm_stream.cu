// Stand-alone streaming reconstruction kernel (d = M s and the leaky integrator,
// Fig. 3 (c)-(d)); the device code is in stream_mvm.cuh.  Used by
// rtc_reconstruct_async; rtc_process_frame runs the fused frame kernel.

#include "stream_mvm.cuh"

namespace {

using namespace rtc_mvm;

template <int DT, bool S_SMEM>
__global__ void __launch_bounds__(kThreads, 1) mvm_stream_kernel(Args g) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    if (tid == 0) init_shared(sh);
    __syncthreads();
    const Plan pl = make_plan<DT, S_SMEM>(g, smem);
    if (pl.u1 <= pl.u0) return;
    if (tid >= kConsumers) {
        if ((tid & 31) < kTeams) produce(g, pl, sh, tid & 31);
        return;
    }
    consumer_prologue<DT, S_SMEM, false>(g, pl, tid, g.s);
    consume<DT, S_SMEM, false>(g, pl, sh, tid, 0, g.s, g.dm_out);
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
    const Launch L = plan_launch(h, Epc<DT>::v);
    if (!L.ok) return cudaErrorInvalidValue;
    const Args g = make_args(h, d_s, d_dm_out, L, Epc<DT>::v);
    if (L.s_in_smem)
        mvm_stream_kernel<DT, true><<<L.G, kThreads, L.smem, st>>>(g);
    else
        mvm_stream_kernel<DT, false><<<L.G, kThreads, L.smem, st>>>(g);
    return cudaGetLastError();
}

template <int DT, bool S>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(mvm_stream_kernel<DT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kDynSmemBudget));
}

}  // namespace

cudaError_t mvm_stream_configure() {
    cudaError_t e = configure_one<RTC_F32, true>();
    if (e == cudaSuccess) e = configure_one<RTC_F32, false>();
    if (e == cudaSuccess) e = configure_one<RTC_BF16, true>();
    if (e == cudaSuccess) e = configure_one<RTC_BF16, false>();
    if (e == cudaSuccess) e = configure_one<RTC_F16, true>();
    if (e == cudaSuccess) e = configure_one<RTC_F16, false>();
    if (e == cudaSuccess) e = configure_one<RTC_FP8_E4M3, true>();
    if (e == cudaSuccess) e = configure_one<RTC_FP8_E4M3, false>();
    if (e == cudaSuccess) e = configure_one<RTC_INT8, true>();
    if (e == cudaSuccess) e = configure_one<RTC_INT8, false>();
    return e;
}

cudaError_t launch_decay(const rtc_handle* h, float* d_dm_out, cudaStream_t st) {
    decay_kernel<<<(h->cfg.nact + 255) / 256, 256, 0, st>>>(h->cfg.nact, h->d_a, d_dm_out, h->leak);
    return cudaGetLastError();
}

cudaError_t launch_mvm_integrate(const rtc_handle* h, const float* d_s, float* d_dm_out,
                                 cudaStream_t st) {
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
