// Reconstruction + integrator for callers that cannot allocate device memory.
//
// Some hosts of this code must never call cudaMalloc: a hard-real-time control
// thread cannot risk the implicit device synchronisation and unbounded latency
// of the allocator inside its loop, and a plugin embedded in a larger RTC
// framework may be handed all of its device buffers by that framework and be
// forbidden to allocate its own.  rtc_mvm_integrate_noalloc serves them: it runs
// the same split-K MVM + leaky-integrator kernel as the handle-based path, but
// takes its split-K scratch (block partials and arrival counters) from one
// file-scope __device__ array instead of from an allocation.
//
// The array is sized for at most RTC_NOALLOC_MAX_NACT actuators and
// RTC_NOALLOC_MAX_KSPLIT split-K blocks per row group (about 520 KiB); every GPU
// that loads the library holds it until the process exits.  All calls on a device
// share it, and it keeps the contents of the last call: the arrival counters are
// cleared by each call before its kernel runs, so two calls whose work overlaps on
// the GPU (different streams without ordering) race on the scratch and must not be
// issued.

#include <mutex>

#include "rtc_internal.h"

namespace {

constexpr size_t kPartialBytes =
    static_cast<size_t>(RTC_NOALLOC_MAX_KSPLIT) * RTC_NOALLOC_MAX_NACT * sizeof(float);
constexpr size_t kCounterBytes =
    static_cast<size_t>((RTC_NOALLOC_MAX_NACT + kMvmRows - 1) / kMvmRows) * sizeof(unsigned);

static __device__ __align__(256) unsigned char g_mvm_scratch[kPartialBytes + kCounterBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

int noalloc_fail(int code, const char* msg) {
    rtc_set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int rtc_mvm_integrate_noalloc(const void* d_M, int32_t store, const float* d_row_scales,
                                         int32_t nact, int32_t kpad, const float* d_s, float* d_a,
                                         float* d_dm_out, float gain, float leak, int32_t ksplit,
                                         void* stream) {
    if (nact <= 0 || nact > RTC_NOALLOC_MAX_NACT)
        return noalloc_fail(RTC_EINVAL, "nact must be in 1..RTC_NOALLOC_MAX_NACT (8192)");
    if (ksplit < 1 || ksplit > RTC_NOALLOC_MAX_KSPLIT)
        return noalloc_fail(RTC_EINVAL, "ksplit must be in 1..RTC_NOALLOC_MAX_KSPLIT (16)");
    if (kpad < 0 || kpad % 16 != 0) return noalloc_fail(RTC_EINVAL, "kpad must be a multiple of 16");
    if (store != RTC_F32 && store != RTC_BF16 && store != RTC_F16 && store != RTC_FP8_E4M3 &&
        store != RTC_INT8)
        return noalloc_fail(RTC_EINVAL, "unknown store type");
    if (!d_s || !d_a || (kpad > 0 && !d_M)) return noalloc_fail(RTC_EINVAL, "NULL buffer");
    if ((store == RTC_FP8_E4M3 || store == RTC_INT8) && !d_row_scales)
        return noalloc_fail(RTC_EINVAL, "FP8 and INT8 need row scales");
    if ((reinterpret_cast<uintptr_t>(d_M) | reinterpret_cast<uintptr_t>(d_s)) & 15)
        return noalloc_fail(RTC_EINVAL, "d_M and d_s must be 16-byte aligned");

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(RTC_EDEVICE, "no usable current CUDA device");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            // The array's host-side name is only a stand-in; the kernel needs the
            // device address, looked up once per device with that device current.
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_mvm_scratch);
            if (e != cudaSuccess) return noalloc_fail(RTC_EDEVICE, cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    float* partial = static_cast<float*>(base);
    unsigned* counter = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(base) + kPartialBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nrb = (static_cast<size_t>(nact) + kMvmRows - 1) / kMvmRows;
    cudaError_t e = cudaMemsetAsync(counter, 0, nrb * sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = launch_mvm_raw(store, d_M, d_row_scales, nact, kpad, d_s, ksplit, partial, counter, d_a,
                           d_dm_out, gain, leak, st);
    if (e != cudaSuccess) return noalloc_fail(RTC_EDEVICE, cudaGetErrorString(e));
    return RTC_OK;
}
