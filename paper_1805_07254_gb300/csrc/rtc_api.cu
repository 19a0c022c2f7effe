// C-ABI entry points of librtc.so: handle lifecycle, loading of the subaperture
// map, calibration maps and control matrix, and the per-frame step.
// Declarations and their contracts are in include/rtc.h.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>
#include <vector>

#include "mlp.h"
#include "pred_tile.cuh"
#include "rtc_internal.h"
#include "stream_mvm.cuh"

namespace {

thread_local std::string g_create_error;

int fail(rtc_handle* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return code;
}

// Makes the handle's device current for the scope and restores the caller's.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define RTC_CUDA(h, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), RTC_EDEVICE, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
void free_dev(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void free_predictor(rtc_handle* h) {
    if (h->pred) {
        mlp_free(*h->pred);
        delete h->pred;
        h->pred = nullptr;
    }
    free_dev(h->d_nbr);
    free_dev(h->d_ring);
    free_dev(h->d_spred);
    h->pred_on = false;
}

void free_slices(rtc_handle* h) {
    free_dev(h->d_sl_off);
    free_dev(h->d_sl_rowbytes);
    free_dev(h->d_sl_g0);
    free_dev(h->d_sl_loc);
    h->sl_S = 0;
    h->sl_off.clear();
    h->sl_rowbytes.clear();
    h->sl_g0.clear();
    h->sl_loc.clear();
    h->sl_equal = false;
    h->m_bytes = 0;
}

int dtype_size(int dt) {
    switch (dt) {
        case RTC_F32: return 4;
        case RTC_BF16: return 2;
        case RTC_F16: return 2;
        case RTC_FP8_E4M3: return 1;
        case RTC_INT8: return 1;
        default: return 0;
    }
}

// First subaperture of each slice for the handle's readout model (plan.cu).
std::vector<int> slice_bounds(const rtc_handle* h, int esz) {
    return plan_slices(h->rc.data(), h->n_valid, h->cfg.n_wfs, h->cfg.npx, h->side, h->cfg.nact, esz,
                       h->dev_sms, h->ro_bands, h->ro_interval_ns);
}

// The slice table for slice bounds g0, in the handle's host vectors: each slice one
// contiguous [nact][2 n_s] block (x slopes, then y slopes), rows padded to a
// multiple of 4 bytes with an access unit (16, 8 or 4 bytes) that divides them an
// odd number of times.  colmap: column c (WFS w, axis, subaperture i) -> (slice,
// column within the slice).
void cut_slices(rtc_handle* h, const std::vector<int>& g0, int esz, std::vector<int2>& colmap) {
    const int S = static_cast<int>(g0.size()) - 1;
    const int nact = h->cfg.nact;
    h->sl_S = S;
    h->sl_g0 = g0;
    h->sl_equal = true;
    for (int s = 0; s <= S; ++s)
        if (g0[s] != static_cast<int>(static_cast<long long>(g0[S]) * s / S)) h->sl_equal = false;
    h->sl_off.resize(S);
    h->sl_rowbytes.resize(S);
    h->sl_loc.resize(S + 1);
    long long off = 0;
    int loc = 0;
    for (int s = 0; s < S; ++s) {
        const int n = g0[s + 1] - g0[s];
        int rb = (2 * n * esz + 3) / 4 * 4;
        while (rtc_mvm::row_unit(rb) == 0) rb += 4;       // a bank-conflict-free access unit
        h->sl_off[s] = off;
        h->sl_rowbytes[s] = rb;
        off += (static_cast<long long>(nact) * rb + 15) / 16 * 16;
        h->sl_loc[s] = loc;
        loc += (rb / esz + 3) / 4 * 4;
    }
    h->sl_loc[S] = loc;
    h->m_bytes = off;
    h->ingest_G = -1;                                   // the frame ingest follows the slices
    // 1-byte stores take the plane layout when one lane per row holds (two ring
    // stages of kConsumers rows leave a generous margin of shared memory): their
    // rows then load as 16-byte units (measured: FP8 frame 21.0 against 22.5 us on
    // ELT; 2-byte stores, which keep up with the HBM anyway, gained nothing)
    int max_rb = 0;
    for (int s = 0; s < S; ++s) max_rb = std::max(max_rb, h->sl_rowbytes[s]);
    h->sl_plane = esz == 1 && 2 * static_cast<long long>(rtc_mvm::kConsumers) * max_rb + (64 << 10) <=
                                  static_cast<long long>(rtc_mvm::kDynSmemBudget);
    const int nv = h->n_valid, nt = nv * h->cfg.n_wfs;
    std::vector<int> slice_of(nt);
    for (int s = 0; s < S; ++s)
        for (int gi = g0[s]; gi < g0[s + 1]; ++gi) slice_of[gi] = s;
    colmap.resize(h->nslopes);
    for (int c = 0; c < h->nslopes; ++c) {
        const int w = c / (2 * nv), rem = c - w * 2 * nv;
        const int axis = rem >= nv ? 1 : 0;
        const int gi = w * nv + (rem - axis * nv);
        const int sl = slice_of[gi];
        const int n = g0[sl + 1] - g0[sl];
        colmap[c] = make_int2(sl, axis * n + (gi - g0[sl]));
    }
}

// The slice table to the device.
cudaError_t upload_slices(rtc_handle* h) {
    const int S = h->sl_S;
    cudaError_t e = cudaMalloc(&h->d_sl_off, S * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_sl_rowbytes, S * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_sl_g0, (S + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_sl_loc, (S + 1) * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_sl_off, h->sl_off.data(), S * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_sl_rowbytes, h->sl_rowbytes.data(), S * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_sl_g0, h->sl_g0.data(), (S + 1) * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_sl_loc, h->sl_loc.data(), (S + 1) * sizeof(int), cudaMemcpyHostToDevice);
    return e;
}

// Default map: subaperture centres inside the annulus obs*n/2 <= r <= n/2,
// radii in subaperture pitches from the grid centre, row-major order.
std::vector<int32_t> default_subaps(int n, float obs) {
    std::vector<int32_t> rc;
    const double ro2 = (n / 2.0) * (n / 2.0);
    const double ri = static_cast<double>(obs) * n / 2.0;
    const double ri2 = ri * ri;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            const double y = r + 0.5 - n / 2.0, x = c + 0.5 - n / 2.0;
            const double d2 = x * x + y * y;
            if (d2 <= ro2 && d2 >= ri2) {
                rc.push_back(r);
                rc.push_back(c);
            }
        }
    return rc;
}

// (Re)build everything whose size depends on the subaperture map.
int apply_subaps(rtc_handle* h, const std::vector<int32_t>& rc) {
    const int n = h->cfg.nsub;
    const int nv = static_cast<int>(rc.size() / 2);
    for (int i = 0; i < nv; ++i) {
        const int r = rc[2 * i], c = rc[2 * i + 1];
        if (r < 0 || r >= n || c < 0 || c >= n)
            return fail(h, RTC_EINVAL, "subap %d at (%d,%d) lies outside the %dx%d grid", i, r, c, n, n);
        if (i > 0) {
            const long prev = static_cast<long>(rc[2 * i - 2]) * n + rc[2 * i - 1];
            if (static_cast<long>(r) * n + c <= prev)
                return fail(h, RTC_EINVAL, "subap map must be strictly increasing in row-major order (entry %d)", i);
        }
    }
    free_predictor(h);        // its neighbour table and history depend on the map
    free_dev(h->d_rc);
    free_dev(h->d_dark);
    free_dev(h->d_gainmap);
    free_dev(h->d_M);
    free_dev(h->d_scale);
    free_dev(h->d_s);
    free_slices(h);
    h->rc = rc;
    h->n_valid = nv;
    h->nslopes = 2 * nv * h->cfg.n_wfs;
    h->kpad = (h->nslopes + 15) / 16 * 16;
    h->store = -1;
    h->calib_loaded = false;
    if (nv > 0) {
        RTC_CUDA(h, cudaMalloc(&h->d_rc, nv * sizeof(int2)));
        RTC_CUDA(h, cudaMemcpy(h->d_rc, rc.data(), nv * sizeof(int2), cudaMemcpyHostToDevice));
    }
    RTC_CUDA(h, cudaMalloc(&h->d_s, std::max(h->kpad, 16) * sizeof(float)));
    RTC_CUDA(h, cudaMemset(h->d_s, 0, std::max(h->kpad, 16) * sizeof(float)));
    return RTC_OK;
}

}  // namespace

int fail_handle(rtc_handle* h, int code, const char* msg) { return fail(h, code, "%s", msg); }

int handle_busy(rtc_handle* h) {
    if (h->in_slot.load()) return fail(h, RTC_ESTATE, "the handle's job is in a server slot");
    if (h->resident) return fail(h, RTC_ESTATE, "the handle is resident (rtc_resident_stop first)");
    return RTC_OK;
}

// Read (and clear) the device status word after the stream has drained.

int take_status(rtc_handle* h, cudaStream_t st) {
    RTC_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    RTC_CUDA(h, cudaStreamSynchronize(st));
    const int code = *h->h_status;
    if (code != 0) {
        // an aborted launch may leave the grid-barrier count short: start it afresh
        RTC_CUDA(h, cudaMemsetAsync(h->d_gridbar, 0, sizeof(unsigned long long), st));
        h->grid_epoch = 0;
        RTC_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), st));
        RTC_CUDA(h, cudaStreamSynchronize(st));
        return fail(h, code, "a bounded device wait expired (results of this step are invalid)");
    }
    return RTC_OK;
}

namespace {

int check_ready(rtc_handle* h) {
    if (!h) return RTC_EINVAL;
    if (!h->calib_loaded) return fail(h, RTC_ESTATE, "calibration maps not loaded");
    if (h->store < 0) return fail(h, RTC_ESTATE, "control matrix not loaded");
    return RTC_OK;
}

// s_used (optional) receives the device buffer that holds this frame's measured slopes.
int enqueue_step(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, float* d_slopes_out,
                 cudaStream_t st, const float** s_used = nullptr, FrameHost* fh = nullptr) {
    if (s_used) *s_used = h->d_s;
    if (h->pred_on && h->kpad > 0) {
        // measured slopes into the next row of the history ring, the prediction from
        // the 4 newest rows, the reconstruction from the prediction: one launch
        const int head = (h->ring_head + 1) & 3;
        float* s_meas = h->d_ring + static_cast<size_t>(head) * h->kpad;
        RTC_CUDA(h, launch_frame(h, d_frame, d_dm_out, s_meas, head, st, fh));
        h->ring_head = head;
        if (s_used) *s_used = s_meas;
        if (d_slopes_out)
            RTC_CUDA(h, cudaMemcpyAsync(d_slopes_out, s_meas, h->nslopes * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st));
        return RTC_OK;
    }
    RTC_CUDA(h, launch_frame(h, d_frame, d_dm_out, nullptr, 0, st, fh));
    if (d_slopes_out)
        RTC_CUDA(h, cudaMemcpyAsync(d_slopes_out, h->d_s, h->nslopes * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
    return RTC_OK;
}

// Device view of a pinned, mapped host buffer; nullptr for pageable or device memory.
const void* mapped_view(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();             // clear the error of a pointer CUDA does not know
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
void* mapped_view(void* p) { return const_cast<void*>(mapped_view(static_cast<const void*>(p))); }

constexpr double kHostWaitS = 2.0;      // bound on the host's wait for a frame's record

#ifdef RTC_HOST_STAMPS
// Diagnostic build only: steady-clock times (ns) of the last rtc_process_frame call
// with pinned buffers: entry, buffers resolved, launch enqueued, record seen, return.
long long g_host_stamps[5];
#define RTC_HOST_STAMP(i) \
    g_host_stamps[i] = std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch()).count()
#else
#define RTC_HOST_STAMP(i) \
    do {                  \
    } while (0)
#endif

// rtc_process_frame on pinned host buffers: one launch reads the frame over the host
// link and writes the DM commands there; the host waits for the completion record.
int process_mapped(rtc_handle* h, const uint16_t* d_frame_host, float* d_dm_host, float* slopes_out) {
    if (!h->h_pf_done) {
        void* p = nullptr;
        RTC_CUDA(h, cudaHostAlloc(&p, sizeof(rtc_pf_done), cudaHostAllocMapped));
        h->h_pf_done = static_cast<rtc_pf_done*>(p);
        memset(h->h_pf_done, 0, sizeof(rtc_pf_done));
        RTC_CUDA(h, cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->d_pf_done), h->h_pf_done, 0));
        RTC_CUDA(h, cudaMalloc(&h->d_pf_ctr, sizeof(unsigned long long)));
        RTC_CUDA(h, cudaMemset(h->d_pf_ctr, 0, sizeof(unsigned long long)));
        h->pf_arrivals = 0;
    }
    FrameHost fh{h->d_pf_done, h->d_pf_ctr, 0, ++h->pf_seq};
    const float* s_used = nullptr;
    const int rc = enqueue_step(h, d_frame_host, d_dm_host, nullptr, h->stream, &s_used, &fh);
    if (rc != RTC_OK) return rc;
    RTC_HOST_STAMP(2);
    const auto t0 = std::chrono::steady_clock::now();
    while (__atomic_load_n(&h->h_pf_done->seq, __ATOMIC_ACQUIRE) != fh.seq) {
        if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > kHostWaitS) {
            const cudaError_t e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return fail(h, RTC_EDEVICE, "%s", cudaGetErrorString(e));
            if (__atomic_load_n(&h->h_pf_done->seq, __ATOMIC_ACQUIRE) == fh.seq) break;
            return fail(h, RTC_ETIMEDOUT, "the frame's completion record did not arrive");
        }
    }
    RTC_HOST_STAMP(3);
    if (__atomic_load_n(&h->h_pf_done->status, __ATOMIC_RELAXED) != RTC_OK) return take_status(h, h->stream);
    if (slopes_out) {
        RTC_CUDA(h, cudaMemcpyAsync(slopes_out, s_used, h->nslopes * sizeof(float), cudaMemcpyDeviceToHost,
                                    h->stream));
        RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return RTC_OK;
}

}  // namespace

void rtc_set_global_error(const char* msg) { g_create_error = msg; }

namespace {
std::mutex g_loop_mu;
int g_loops = 0;
std::vector<std::function<void()>> g_deferred;
}  // namespace

void loop_begin() {
    std::lock_guard<std::mutex> lock(g_loop_mu);
    ++g_loops;
}

void loop_end() {
    std::vector<std::function<void()>> run;
    {
        std::lock_guard<std::mutex> lock(g_loop_mu);
        if (--g_loops > 0) return;
        run.swap(g_deferred);
    }
    for (auto& f : run) f();
}

bool release_or_defer(std::function<void()> f) {
    std::lock_guard<std::mutex> lock(g_loop_mu);
    if (g_loops == 0) return false;
    g_deferred.push_back(std::move(f));
    return true;
}

extern "C" {

const char* rtc_version(void) { return "librtc 0.1 (sm_103a)"; }

const char* rtc_last_error(const rtc_handle* h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

int rtc_create(const rtc_config* cfg, rtc_handle** out) {
    if (!cfg || !out) return fail(nullptr, RTC_EINVAL, "cfg and out must be non-NULL");
    *out = nullptr;
    const rtc_config& c = *cfg;
    if (c.nsub <= 0 || c.npx <= 0 || c.n_wfs <= 0 || c.nact <= 0)
        return fail(nullptr, RTC_EINVAL, "nsub, npx, n_wfs and nact must be positive");
    if (static_cast<long long>(c.nsub) * c.npx > 16384)
        return fail(nullptr, RTC_EINVAL, "frame side %lld exceeds 16384", (long long)c.nsub * c.npx);
    if (!(c.obs >= 0.f && c.obs < 1.f)) return fail(nullptr, RTC_EINVAL, "obs must be in [0, 1)");
    if (!isfinite(c.gain) || !isfinite(c.leak) || !isfinite(c.thr))
        return fail(nullptr, RTC_EINVAL, "gain, leak and thr must be finite");
    if (c.thr_mode != 0 && c.thr_mode != 1) return fail(nullptr, RTC_EINVAL, "thr_mode must be 0 or 1");
    if (c.reserved != 0) return fail(nullptr, RTC_EINVAL, "reserved must be 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev)
        return fail(nullptr, RTC_EINVAL, "device %d not available", c.device);

    rtc_handle* h = new rtc_handle();
    h->cfg = c;
    h->side = c.nsub * c.npx;
    h->gain = c.gain;
    h->leak = c.leak;
    h->thr_mode = c.thr_mode;
    h->thr = c.thr;
    DeviceScope ds(c.device);
    int rcode = RTC_OK;
    cudaDeviceGetAttribute(&h->dev_sms, cudaDevAttrMultiProcessorCount, c.device);
    if (h->dev_sms < 1) h->dev_sms = 1;
    h->num_sms = h->dev_sms;
    if (mvm_stream_configure() != cudaSuccess || frame_kernel_configure() != cudaSuccess ||
        loop_kernel_configure() != cudaSuccess) {
        rcode = fail(nullptr, RTC_EDEVICE, "cannot configure the reconstruction kernel");
    } else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        rcode = fail(nullptr, RTC_EDEVICE, "cudaStreamCreate failed");
    } else {
        const size_t frame_elems = static_cast<size_t>(c.n_wfs) * h->side * h->side;
        if (cudaMalloc(&h->d_a, c.nact * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&h->d_partial, 2 * static_cast<size_t>(h->dev_sms) * c.nact * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&h->d_frame, frame_elems * sizeof(uint16_t)) != cudaSuccess ||
            cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&h->d_gridbar, sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&h->h_status, sizeof(int)) != cudaSuccess) {
            rcode = fail(nullptr, RTC_ENOMEM, "device allocation failed");
        } else if (cudaMemset(h->d_a, 0, c.nact * sizeof(float)) != cudaSuccess ||
                   cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess ||
                   cudaMemset(h->d_gridbar, 0, sizeof(unsigned long long)) != cudaSuccess) {
            rcode = fail(nullptr, RTC_EDEVICE, "cudaMemset failed");
        } else {
            rcode = apply_subaps(h, default_subaps(c.nsub, c.obs));
            if (rcode != RTC_OK) g_create_error = h->err;
        }
    }
    if (rcode != RTC_OK) {
        rtc_destroy(h);
        return rcode;
    }
    *out = h;
    return RTC_OK;
}

int rtc_destroy(rtc_handle* h) {
    if (!h) return RTC_OK;
    if (h->in_slot.load()) return fail(h, RTC_ESTATE, "the handle's job is in a server slot");
    if (h->resident) {
        DeviceScope ds(h->cfg.device);
        resident_stop(h);
    }
    if (release_or_defer([h] { rtc_destroy(h); })) return RTC_OK;
    DeviceScope ds(h->cfg.device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_predictor(h);
    free_dev(h->d_rc);
    free_dev(h->d_dark);
    free_dev(h->d_gainmap);
    free_dev(h->d_M);
    free_dev(h->d_scale);
    free_dev(h->d_s);
    free_dev(h->d_a);
    free_dev(h->d_partial);
    free_slices(h);
    free_dev(h->d_frame);
    free_dev(h->d_status);
    free_dev(h->d_gridbar);
    free_dev(h->d_sbuf);
    free_dev(h->d_donectr);
    free_dev(h->d_mirror);
    free_dev(h->d_tseen);
    free_dev(h->d_units);
    free_dev(h->d_blk);
    free_dev(h->d_pf_ctr);
    if (h->h_pf_done) cudaFreeHost(h->h_pf_done);
    if (h->h_ring) cudaFreeHost(h->h_ring);
    if (h->h_seq) cudaFreeHost(h->h_seq);
    if (h->h_dm_ring) cudaFreeHost(h->h_dm_ring);
    if (h->h_done) cudaFreeHost(h->h_done);
    if (h->h_ptrs) cudaFreeHost(h->h_ptrs);
    if (h->h_status) cudaFreeHost(h->h_status);
    h->h_status = nullptr;
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return RTC_OK;
}

int rtc_load_subaps(rtc_handle* h, const int32_t* rc, int32_t n_valid) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (n_valid < 0 || (n_valid > 0 && !rc)) return fail(h, RTC_EINVAL, "bad subap map");
    DeviceScope ds(h->cfg.device);
    RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<int32_t> v(rc, rc + 2 * static_cast<size_t>(n_valid));
    return apply_subaps(h, v);
}

int rtc_load_calib(rtc_handle* h, const float* dark, const float* flat, int64_t npix) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    const int side = h->side, npx = h->cfg.npx, nw = h->cfg.n_wfs, nv = h->n_valid;
    const int64_t want = static_cast<int64_t>(nw) * side * side;
    if (!dark || !flat || npix != want)
        return fail(h, RTC_EINVAL, "calibration maps must hold n_wfs*H*W = %lld pixels", (long long)want);
    const int npp = npx * npx;
    std::vector<float> dk(static_cast<size_t>(nw) * nv * npp), gk(dk.size());
    for (int w = 0; w < nw; ++w)
        for (int i = 0; i < nv; ++i) {
            const int r = h->rc[2 * i], c = h->rc[2 * i + 1];
            for (int y = 0; y < npx; ++y)
                for (int x = 0; x < npx; ++x) {
                    const size_t src = static_cast<size_t>(w) * side * side +
                                       static_cast<size_t>(r * npx + y) * side + (c * npx + x);
                    const size_t dst = (static_cast<size_t>(w) * nv + i) * npp + y * npx + x;
                    const float f = flat[src];
                    if (!(f != 0.f) || !isfinite(f) || !isfinite(dark[src]))
                        return fail(h, RTC_EINVAL, "flat must be finite and non-zero, dark finite (pixel %zu)", src);
                    dk[dst] = dark[src];
                    gk[dst] = 1.0f / f;
                }
        }
    DeviceScope ds(h->cfg.device);
    RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    free_dev(h->d_dark);
    free_dev(h->d_gainmap);
    h->calib_loaded = false;
    if (!dk.empty()) {
        RTC_CUDA(h, cudaMalloc(&h->d_dark, dk.size() * sizeof(float)));
        RTC_CUDA(h, cudaMalloc(&h->d_gainmap, gk.size() * sizeof(float)));
        RTC_CUDA(h, cudaMemcpy(h->d_dark, dk.data(), dk.size() * sizeof(float), cudaMemcpyHostToDevice));
        RTC_CUDA(h, cudaMemcpy(h->d_gainmap, gk.data(), gk.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    h->calib_loaded = true;
    return RTC_OK;
}

int rtc_set_threshold(rtc_handle* h, int32_t mode, float thr) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if ((mode != 0 && mode != 1) || !isfinite(thr)) return fail(h, RTC_EINVAL, "bad threshold");
    h->thr_mode = mode;
    h->thr = thr;
    return RTC_OK;
}

int rtc_load_cmat(rtc_handle* h, const void* M, int32_t nact, int32_t nslopes, int32_t src,
                  int32_t store, const float* row_scales) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (!M) return fail(h, RTC_EINVAL, "M is NULL");
    if (nact != h->cfg.nact || nslopes != h->nslopes)
        return fail(h, RTC_EINVAL, "matrix is %dx%d, handle expects %dx%d", nact, nslopes, h->cfg.nact, h->nslopes);
    if (dtype_size(src) == 0 || dtype_size(store) == 0) return fail(h, RTC_EINVAL, "unknown dtype");
    if (src != RTC_F32 && src != store) return fail(h, RTC_EINVAL, "only an FP32 source can be converted");
    const bool scaled = store == RTC_FP8_E4M3 || store == RTC_INT8;
    if (src == store && scaled && !row_scales) return fail(h, RTC_EINVAL, "FP8 and INT8 sources need row_scales");
    DeviceScope ds(h->cfg.device);
    RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    free_dev(h->d_M);
    free_dev(h->d_scale);
    free_slices(h);
    h->store = -1;
    RTC_CUDA(h, cudaMalloc(&h->d_scale, nact * sizeof(float)));
    if (nslopes == 0) {          // no valid subapertures: an empty matrix, d = 0
        h->store = store;
        return RTC_OK;
    }
    const int esz = dtype_size(store);
    std::vector<int2> colmap;
    cut_slices(h, slice_bounds(h, esz), esz, colmap);
    if (upload_slices(h) != cudaSuccess) {
        free_slices(h);
        return fail(h, RTC_ENOMEM, "cannot allocate the slice table");
    }
    if (cudaMalloc(&h->d_M, static_cast<size_t>(h->m_bytes)) != cudaSuccess) {
        h->d_M = nullptr;
        free_slices(h);
        return fail(h, RTC_ENOMEM, "cannot allocate %lld bytes for the matrix", h->m_bytes);
    }
    RTC_CUDA(h, cudaMemset(h->d_M, 0, static_cast<size_t>(h->m_bytes)));
    if (src == store && scaled)
        RTC_CUDA(h, cudaMemcpy(h->d_scale, row_scales, nact * sizeof(float), cudaMemcpyHostToDevice));
    // the host matrix through a staging buffer into the slice layout
    void* staging = nullptr;
    int2* d_colmap = nullptr;
    const size_t sbytes = static_cast<size_t>(nact) * nslopes * dtype_size(src);
    if (cudaMalloc(&staging, sbytes) != cudaSuccess ||
        cudaMalloc(&d_colmap, nslopes * sizeof(int2)) != cudaSuccess) {
        if (staging) cudaFree(staging);
        return fail(h, RTC_ENOMEM, "cannot allocate %zu bytes of staging", sbytes);
    }
    cudaError_t e = cudaMemcpy(staging, M, sbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_colmap, colmap.data(), nslopes * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_layout(src, store, staging, nact, nslopes, d_colmap, h->d_sl_off, h->d_sl_rowbytes,
                          h->sl_plane ? 1 : 0, h->d_scale, h->d_M, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(staging);
    cudaFree(d_colmap);
    if (e != cudaSuccess) return fail(h, RTC_EDEVICE, "matrix conversion failed: %s", cudaGetErrorString(e));
    h->store = store;
    return RTC_OK;
}

int rtc_set_readout(rtc_handle* h, int32_t n_bands, double band_interval_us) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (n_bands < 0 || n_bands > h->side || !(band_interval_us >= 0.0) || !(band_interval_us <= 1e6))
        return fail(h, RTC_EINVAL, "n_bands must be 0 .. frame height and band_interval_us in [0, 1e6]");
    DeviceScope ds(h->cfg.device);
    RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    h->ro_bands = n_bands;
    h->ro_interval_ns = static_cast<long long>(band_interval_us * 1e3 + 0.5);
    if (h->store < 0 || h->sl_S == 0) return RTC_OK;       // the next rtc_load_cmat cuts
    // the resident matrix from its present slices into the new ones, on the device
    const int esz = dtype_size(h->store);
    const int nact = h->cfg.nact, ncol = h->nslopes;
    std::vector<int2> old_map, new_map;
    cut_slices(h, h->sl_g0, esz, old_map);                  // the present cut's column map
    const int old_plane = h->sl_plane ? 1 : 0;
    const std::vector<int> g0 = slice_bounds(h, esz);
    void* old_M = h->d_M;
    long long* old_off = h->d_sl_off;
    int* old_rb = h->d_sl_rowbytes;
    int* old_g0 = h->d_sl_g0;
    int* old_loc = h->d_sl_loc;
    h->d_M = nullptr;
    h->d_sl_off = nullptr;
    h->d_sl_rowbytes = nullptr;
    h->d_sl_g0 = nullptr;
    h->d_sl_loc = nullptr;
    cut_slices(h, g0, esz, new_map);
    int2* d_maps = nullptr;
    cudaError_t e = upload_slices(h);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_M, static_cast<size_t>(h->m_bytes));
    if (e == cudaSuccess) e = cudaMemset(h->d_M, 0, static_cast<size_t>(h->m_bytes));
    if (e == cudaSuccess) e = cudaMalloc(&d_maps, 2 * static_cast<size_t>(ncol) * sizeof(int2));
    if (e == cudaSuccess)
        e = cudaMemcpy(d_maps, old_map.data(), ncol * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_maps + ncol, new_map.data(), ncol * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_relayout(esz, old_plane, h->sl_plane ? 1 : 0, old_M, d_maps, old_off, old_rb, nact, ncol, d_maps + ncol,
                            h->d_sl_off, h->d_sl_rowbytes, h->d_M, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (d_maps) cudaFree(d_maps);
    cudaFree(old_M);
    cudaFree(old_off);
    cudaFree(old_rb);
    cudaFree(old_g0);
    cudaFree(old_loc);
    if (e != cudaSuccess) {
        free_dev(h->d_M);
        free_slices(h);
        h->store = -1;
        return fail(h, e == cudaErrorMemoryAllocation ? RTC_ENOMEM : RTC_EDEVICE,
                    "matrix re-cut failed (the matrix must be loaded again): %s", cudaGetErrorString(e));
    }
    return RTC_OK;
}

int rtc_set_gain(rtc_handle* h, float gain, float leak) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (!isfinite(gain) || !isfinite(leak)) return fail(h, RTC_EINVAL, "gain and leak must be finite");
    h->gain = gain;
    h->leak = leak;
    return RTC_OK;
}

int rtc_reset(rtc_handle* h) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    DeviceScope ds(h->cfg.device);
    RTC_CUDA(h, cudaMemsetAsync(h->d_a, 0, h->cfg.nact * sizeof(float), h->stream));
    if (h->d_ring)
        RTC_CUDA(h, cudaMemsetAsync(h->d_ring, 0, 4 * static_cast<size_t>(h->kpad) * sizeof(float), h->stream));
    h->ring_head = 3;
    RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    return RTC_OK;
}

int rtc_load_predictor(rtc_handle* h, const float* params, int64_t n, float sigma) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (!params || n != RTC_MLP_NPARAMS || !(sigma > 0.f) || !isfinite(sigma))
        return fail(h, RTC_EINVAL, "need RTC_MLP_NPARAMS parameters and sigma > 0");
    if (h->cfg.n_wfs != 1) return fail(h, RTC_EINVAL, "the predictor is for single-WFS handles");
    if (h->kpad > 16384)   // the fused kernels keep the slope vector in shared memory
        return fail(h, RTC_EINVAL, "the predictor supports up to 16384 slopes");
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(params[i])) return fail(h, RTC_EINVAL, "parameters must be finite");
    DeviceScope ds(h->cfg.device);
    RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    free_predictor(h);
    RTC_CUDA(h, mlp_configure());
    h->pred = new MlpDev();
    if (mlp_alloc(*h->pred) != RTC_OK) {
        free_predictor(h);
        return fail(h, RTC_ENOMEM, "cannot allocate the predictor");
    }
    if (mlp_upload(*h->pred, params, h->stream) != RTC_OK) {
        free_predictor(h);
        return fail(h, RTC_EDEVICE, "predictor upload failed");
    }
    const std::vector<int> nbr = mlp_neighbours(h->rc.data(), h->n_valid, h->cfg.nsub);
    const size_t ring = 4 * static_cast<size_t>(std::max(h->kpad, 16)) * sizeof(float);
    if ((!nbr.empty() && cudaMalloc(&h->d_nbr, nbr.size() * sizeof(int)) != cudaSuccess) ||
        cudaMalloc(&h->d_ring, ring) != cudaSuccess ||
        cudaMalloc(&h->d_spred, std::max(h->kpad, 16) * sizeof(float)) != cudaSuccess) {
        free_predictor(h);
        return fail(h, RTC_ENOMEM, "cannot allocate the predictor state");
    }
    if (!nbr.empty())
        RTC_CUDA(h, cudaMemcpy(h->d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
    RTC_CUDA(h, cudaMemset(h->d_ring, 0, ring));
    RTC_CUDA(h, cudaMemset(h->d_spred, 0, std::max(h->kpad, 16) * sizeof(float)));
    h->ring_head = 3;
    h->pred_sigma = sigma;
    return RTC_OK;
}

int rtc_set_predictor(rtc_handle* h, int32_t on) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (on && !h->pred) return fail(h, RTC_ESTATE, "no predictor loaded");
    h->pred_on = on != 0;
    return RTC_OK;
}

int rtc_get_dm(rtc_handle* h, float* out) {
    if (!h || !out) return h ? fail(h, RTC_EINVAL, "out is NULL") : RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    DeviceScope ds(h->cfg.device);
    RTC_CUDA(h, cudaMemcpyAsync(out, h->d_a, h->cfg.nact * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    RTC_CUDA(h, cudaStreamSynchronize(h->stream));
    return RTC_OK;
}

int rtc_get_info(const rtc_handle* h, rtc_info* out) {
    if (!h || !out) return RTC_EINVAL;
    out->n_valid = h->n_valid;
    out->nslopes = h->nslopes;
    out->nact = h->cfg.nact;
    out->kpad = h->kpad;
    out->store = h->store;
    out->blocks = out->tile_rows = out->ring_stages = 0;
    out->slices = h->sl_S;
    if (h->store >= 0 && h->sl_S > 0) {
        const rtc_mvm::Launch L = rtc_mvm::plan_launch(h, h->pred_on ? rtc_pred::kSmemBytes : 0);
        out->blocks = L.G;
        out->tile_rows = L.R;
        out->ring_stages = L.nst;
    }
    const int64_t entries = static_cast<int64_t>(h->cfg.nact) * h->nslopes;
    int64_t mb = 0;
    if (h->store >= 0) mb = entries * dtype_size(h->store) + (h->store == RTC_FP8_E4M3 || h->store == RTC_INT8 ? 4LL * h->cfg.nact : 0);
    out->matrix_bytes = mb;
    out->frame_bytes = static_cast<int64_t>(h->cfg.n_wfs) * h->side * h->side * 2;
    out->calib_bytes = 2LL * 4 * h->cfg.n_wfs * h->n_valid * h->cfg.npx * h->cfg.npx;
    return RTC_OK;
}

int rtc_process_frame(rtc_handle* h, const uint16_t* frame, float* dm_out, float* slopes_out) {
    RTC_HOST_STAMP(0);
    int rc = check_ready(h);
    if (rc != RTC_OK) return rc;
    if (!frame || !dm_out) return fail(h, RTC_EINVAL, "frame and dm_out must be non-NULL");
    if (h->resident) {
        // the resident kernel takes the frame: pinned buffers only, no slopes
        const uint16_t* d_frame = static_cast<const uint16_t*>(mapped_view(frame));
        float* d_dm = static_cast<float*>(mapped_view(dm_out));
        if (!d_frame || !d_dm || slopes_out)
            return fail(h, RTC_ESTATE, "a resident handle takes pinned frame and dm buffers and no slopes_out");
        DeviceScope ds(h->cfg.device);
        return resident_frame(h, d_frame, d_dm);
    }
    if (const int busy = handle_busy(h)) return busy;
    DeviceScope ds(h->cfg.device);
    // pinned (page-locked, mapped) host buffers: the kernel reads the frame and writes
    // the commands over the host link, no copies and no stream synchronisation
    const uint16_t* d_frame_host = static_cast<const uint16_t*>(mapped_view(frame));
    float* d_dm_host = static_cast<float*>(mapped_view(dm_out));
    RTC_HOST_STAMP(1);
    if (d_frame_host && d_dm_host && h->kpad > 0) {
        rc = process_mapped(h, d_frame_host, d_dm_host, slopes_out);
        RTC_HOST_STAMP(4);
        return rc;
    }
    const size_t fbytes = static_cast<size_t>(h->cfg.n_wfs) * h->side * h->side * sizeof(uint16_t);
    RTC_CUDA(h, cudaMemcpyAsync(h->d_frame, frame, fbytes, cudaMemcpyHostToDevice, h->stream));
    const float* s_used = nullptr;
    rc = enqueue_step(h, h->d_frame, nullptr, nullptr, h->stream, &s_used);
    if (rc != RTC_OK) return rc;
    RTC_CUDA(h, cudaMemcpyAsync(dm_out, h->d_a, h->cfg.nact * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (slopes_out)
        RTC_CUDA(h, cudaMemcpyAsync(slopes_out, s_used, h->nslopes * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    return take_status(h, h->stream);
}

}  // extern "C"

int rtc_enqueue_frame(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, cudaStream_t st) {
    return enqueue_step(h, d_frame, d_dm_out, nullptr, st);
}

bool rtc_handle_ready(const rtc_handle* h) { return h && h->calib_loaded && h->store >= 0; }

int64_t rtc_handle_device_bytes(const rtc_handle* h) {
    const int64_t nact = h->cfg.nact, kpad = h->kpad, nw = h->cfg.n_wfs;
    const int64_t npp = static_cast<int64_t>(h->cfg.npx) * h->cfg.npx;
    int64_t b = h->m_bytes + 4 * nact;                                         // matrix + scales
    b += 2 * 4 * nw * h->n_valid * npp;                                        // dark + gain
    b += nw * static_cast<int64_t>(h->side) * h->side * 2;                     // frame staging
    b += 4 * (kpad + nact) + 8 * static_cast<int64_t>(h->dev_sms) * nact + 4 * nact;  // s, a, partials
    if (h->pred) b += 4 * (5 * kpad) + 4 * 25 * h->n_valid + 3 * 4 * RTC_MLP_NPARAMS + 2 * (64 * 208 + 64 * 64);
    return b;
}

extern "C" {

int rtc_process_frame_async(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out,
                            float* d_slopes_out, void* stream) {
    int rc = check_ready(h);
    if (rc != RTC_OK) return rc;
    if (const int busy = handle_busy(h)) return busy;
    if (!d_frame) return fail(h, RTC_EINVAL, "d_frame is NULL");
    if (reinterpret_cast<uintptr_t>(d_frame) & 15) return fail(h, RTC_EINVAL, "d_frame must be 16-byte aligned");
    DeviceScope ds(h->cfg.device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    return enqueue_step(h, d_frame, d_dm_out, d_slopes_out, st);
}

int rtc_centroid_async(rtc_handle* h, const uint16_t* d_frame, float* d_slopes_out, void* stream) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (!h->calib_loaded) return fail(h, RTC_ESTATE, "calibration maps not loaded");
    if (!d_frame) return fail(h, RTC_EINVAL, "d_frame is NULL");
    if (reinterpret_cast<uintptr_t>(d_frame) & 15) return fail(h, RTC_EINVAL, "d_frame must be 16-byte aligned");
    DeviceScope ds(h->cfg.device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    RTC_CUDA(h, launch_calib_cog(h, d_frame, h->d_s, st));
    if (d_slopes_out)
        RTC_CUDA(h, cudaMemcpyAsync(d_slopes_out, h->d_s, h->nslopes * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
    return RTC_OK;
}

int rtc_reconstruct_async(rtc_handle* h, const float* d_slopes, float* d_dm_out, void* stream) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (h->store < 0) return fail(h, RTC_ESTATE, "control matrix not loaded");
    DeviceScope ds(h->cfg.device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    if (d_slopes && d_slopes != h->d_s)
        RTC_CUDA(h, cudaMemcpyAsync(h->d_s, d_slopes, h->nslopes * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
    RTC_CUDA(h, launch_mvm_integrate(h, h->d_s, d_dm_out, st));
    return RTC_OK;
}

int rtc_synchronize(rtc_handle* h, void* stream) {
    if (!h) return RTC_EINVAL;
    if (h->resident) return fail(h, RTC_ESTATE, "the handle is resident (rtc_resident_stop first)");
    DeviceScope ds(h->cfg.device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    RTC_CUDA(h, cudaStreamSynchronize(st));
    RTC_CUDA(h, cudaGetLastError());
    return take_status(h, st);
}

}  // extern "C"

#ifdef RTC_HOST_STAMPS
extern "C" void rtc_probe_host_stamps(long long* out) {
    for (int i = 0; i < 5; ++i) out[i] = g_host_stamps[i];
}
#endif
