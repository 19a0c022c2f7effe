// rtc_run_loop: host side of the persistent real-time loop (see loop_kernel.cu).
//
// A ring of RTC_LOOP_SLOTS frame slots lives in pinned host memory mapped into the
// device's address space.  A filler thread writes frame k into slot k % nslot
// (through the caller's source callback) once the device is done with the frame
// that used the slot before; the calling thread publishes frame k at its time,
// band by band (n_bands bands of pixel rows, n_bands = 1 for a whole frame), by
// release stores of k * n_bands + j + 1 into the slot's sequence word, then spins
// on the slot's completion record and takes the frame's latency from the last
// band.  With a preloaded frame set the slots are filled once and only
// republished.  The pixels are in the slot before the first band is published;
// the bands only gate when each part of the kernel may read them, as the rows of
// a rolling readout would.

#include <math.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "rtc_internal.h"

namespace {

constexpr unsigned long long kStop = ~0ull;
constexpr long long kHostWaitNs = 5ll * 1000 * 1000 * 1000;   // host gives a frame up to 5 s

long long mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return static_cast<long long>(ts.tv_sec) * 1000000000ll + ts.tv_nsec;
}

unsigned long long load_acquire(const unsigned long long* p) {
    return __atomic_load_n(p, __ATOMIC_ACQUIRE);
}
void store_release(unsigned long long* p, unsigned long long v) {
    __atomic_store_n(p, v, __ATOMIC_RELEASE);
}

// Percentiles, mean, standard deviation (RMS jitter) and peak-to-peak of ns samples, in us.
void summarise(std::vector<long long> v, double& p50, double& p99, double& p999, double& mean,
               double& rms, double& p2p) {
    p50 = p99 = p999 = mean = rms = p2p = 0.0;
    if (v.empty()) return;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        const double k = (v.size() - 1) * q;
        const size_t lo = static_cast<size_t>(floor(k)), hi = static_cast<size_t>(ceil(k));
        return (v[lo] + (v[hi] - v[lo]) * (k - lo)) / 1e3;
    };
    p50 = pct(0.5);
    p99 = pct(0.99);
    p999 = pct(0.999);
    double s = 0.0;
    for (long long x : v) s += static_cast<double>(x);
    mean = s / v.size();
    double ss = 0.0;
    for (long long x : v) ss += (x - mean) * (x - mean);
    rms = v.size() > 1 ? sqrt(ss / (v.size() - 1)) / 1e3 : 0.0;
    mean /= 1e3;
    p2p = (v.back() - v.front()) / 1e3;
}

#define LOOP_CUDA(call)                                                                      \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail_handle(h, RTC_EDEVICE, cudaGetErrorString(e_));   \
    } while (0)

int ensure_buffers(rtc_handle* h) {
    const size_t frame_bytes = static_cast<size_t>(h->cfg.n_wfs) * h->side * h->side * 2;
    if (!h->h_ring) {
        LOOP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&h->h_ring), RTC_LOOP_SLOTS * frame_bytes,
                                cudaHostAllocMapped | cudaHostAllocPortable));
        LOOP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&h->h_seq),
                                RTC_LOOP_SLOTS * sizeof(unsigned long long), cudaHostAllocMapped));
        LOOP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&h->h_dm_ring),
                                static_cast<size_t>(RTC_LOOP_SLOTS) * h->cfg.nact * sizeof(float),
                                cudaHostAllocMapped));
        LOOP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&h->h_done),
                                RTC_LOOP_SLOTS * sizeof(rtc_loop_done), cudaHostAllocMapped));
        LOOP_CUDA(cudaMalloc(&h->d_donectr, sizeof(unsigned long long)));
        LOOP_CUDA(cudaMalloc(&h->d_mirror, 3 * RTC_LOOP_SLOTS * sizeof(unsigned long long)));
        LOOP_CUDA(cudaMalloc(&h->d_tseen, 2 * sizeof(unsigned long long)));
    }
    if (h->sbuf_kpad != h->kpad) {
        if (h->d_sbuf) cudaFree(h->d_sbuf);
        h->d_sbuf = nullptr;
        LOOP_CUDA(cudaMalloc(&h->d_sbuf, 2 * static_cast<size_t>(std::max(h->kpad, 16)) * sizeof(float)));
        LOOP_CUDA(cudaMemset(h->d_sbuf, 0, 2 * static_cast<size_t>(std::max(h->kpad, 16)) * sizeof(float)));
        h->sbuf_kpad = h->kpad;
    }
    return RTC_OK;
}

}  // namespace

extern "C" int rtc_run_loop(rtc_handle* h, const rtc_loop_config* cfg, rtc_stats* stats) {
    if (!h) return RTC_EINVAL;
    if (const int busy = handle_busy(h)) return busy;
    if (!cfg || !stats) return fail_handle(h, RTC_EINVAL, "cfg and stats must be non-NULL");
    if (!h->calib_loaded || h->store < 0)
        return fail_handle(h, RTC_ESTATE, "calibration maps and control matrix must be loaded");
    if (h->kpad == 0) return fail_handle(h, RTC_ESTATE, "the loop needs at least one valid subaperture");
    if (cfg->n_frames == 0 || !(cfg->rate_hz >= 0.0) || !isfinite(cfg->rate_hz))
        return fail_handle(h, RTC_EINVAL, "n_frames must be > 0 and rate_hz finite and >= 0");
    if (!cfg->source && (!cfg->preload || cfg->n_preload < 1 || cfg->n_preload > RTC_LOOP_SLOTS))
        return fail_handle(h, RTC_EINVAL, "give a source callback or 1..RTC_LOOP_SLOTS preloaded frames");
    if (cfg->n_bands < 0 || cfg->n_bands > h->side || !(cfg->band_interval_us >= 0.0) ||
        !isfinite(cfg->band_interval_us))
        return fail_handle(h, RTC_EINVAL, "n_bands must be 0 .. frame height and band_interval_us finite and >= 0");
    const int nb = std::max(cfg->n_bands, 1);
    const long long band_ns = static_cast<long long>(cfg->band_interval_us * 1e3);
    memset(stats, 0, sizeof *stats);

    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != h->cfg.device) cudaSetDevice(h->cfg.device);
    struct Restore {
        int d;
        ~Restore() {
            int cur = -1;
            if (d >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != d) cudaSetDevice(d);
        }
    } restore{dev_prev};

    // releases requested while the loop runs wait for its end
    struct LoopScope {
        LoopScope() { loop_begin(); }
        ~LoopScope() { loop_end(); }
    } loop_scope;

    int rc = ensure_buffers(h);
    if (rc != RTC_OK) return rc;
    LOOP_CUDA(cudaStreamSynchronize(h->stream));

    const size_t frame_elems = static_cast<size_t>(h->cfg.n_wfs) * h->side * h->side;
    const int nslot = cfg->source ? RTC_LOOP_SLOTS : cfg->n_preload;
    const unsigned long long n = cfg->n_frames;
    for (int i = 0; i < RTC_LOOP_SLOTS; ++i) {
        h->h_seq[i] = 0;
        memset(&h->h_done[i], 0, sizeof(rtc_loop_done));
    }
    if (!cfg->source)
        for (int i = 0; i < nslot; ++i)
            memcpy(h->h_ring + i * frame_elems, cfg->preload + i * frame_elems, frame_elems * 2);
    LOOP_CUDA(cudaMemsetAsync(h->d_gridbar, 0, sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_donectr, 0, sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_mirror, 0, 3 * RTC_LOOP_SLOTS * sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_tseen, 0, 2 * sizeof(unsigned long long), h->stream));
    h->grid_epoch = 0;

    LoopLaunch ll{};
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(const_cast<uint16_t**>(&ll.d_frames)), h->h_ring, 0));
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(const_cast<unsigned long long**>(&ll.d_seq)), h->h_seq, 0));
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ll.d_dm), h->h_dm_ring, 0));
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ll.d_done), h->h_done, 0));
    ll.frame_elems = frame_elems;
    ll.n_frames = n;
    ll.nslot = nslot;
    ll.n_bands = nb;
    ll.l2_stream = cfg->matrix_l2 == 1 ? 1 : 0;
    LOOP_CUDA(launch_loop(h, ll, h->stream));

    // filler: frame k into slot k % nslot once frame k - nslot has left it
    std::atomic<unsigned long long> filled{cfg->source ? 0ull : n};
    std::atomic<bool> stop{false};
    std::atomic<unsigned long long> source_end{n};
    std::thread filler;
    if (cfg->source) {
        filler = std::thread([&] {
            for (unsigned long long k = 0; k < n && !stop.load(); ++k) {
                const int slot = static_cast<int>(k % nslot);
                if (k >= static_cast<unsigned long long>(nslot)) {
                    const unsigned long long need = k - nslot + 1;
                    while (load_acquire(&h->h_done[slot].seq) < need && !stop.load()) {
                    }
                    if (stop.load()) break;
                }
                if (cfg->source(cfg->source_user, k, h->h_ring + slot * frame_elems) != 0) {
                    source_end.store(k);
                    break;
                }
                filled.store(k + 1, std::memory_order_release);
            }
        });
    }

    std::vector<long long> e2e, dev;
    e2e.reserve(n);
    dev.reserve(n);
    const long long period = cfg->rate_hz > 0 ? static_cast<long long>(1e9 / cfg->rate_hz) : 0;
    const long long t_start = mono_ns();
    long long t_first_pub = 0, t_last_done = 0;
    int result = RTC_OK;
    unsigned long long k = 0;
    for (; k < n; ++k) {
        const int slot = static_cast<int>(k % nslot);
        // the frame must be in its slot
        const long long w0 = mono_ns();
        while (filled.load(std::memory_order_acquire) <= k && k < source_end.load()) {
            if (mono_ns() - w0 > kHostWaitNs) break;
        }
        if (k >= source_end.load() || filled.load(std::memory_order_acquire) <= k) break;
        if (period) {
            const long long due = t_start + static_cast<long long>(k) * period;
            while (mono_ns() < due) {
            }
        }
        // bands 0 .. nb - 2 at their times, then the last one, from which the
        // frame's latency is taken
        const long long t_band0 = mono_ns();
        if (k == 0) t_first_pub = t_band0;
        for (int j = 0; j + 1 < nb; ++j) {
            while (mono_ns() < t_band0 + j * band_ns) {
            }
            store_release(&h->h_seq[slot], k * nb + j + 1);
        }
        while (mono_ns() < t_band0 + (nb - 1) * band_ns) {
        }
        const long long t_pub = mono_ns();
        store_release(&h->h_seq[slot], (k + 1) * nb);
        // completion record of frame k
        bool ok = true;
        while (load_acquire(&h->h_done[slot].seq) != k + 1) {
            if (mono_ns() - t_pub > kHostWaitNs || cudaStreamQuery(h->stream) != cudaErrorNotReady) {
                ok = load_acquire(&h->h_done[slot].seq) == k + 1;
                break;
            }
        }
        if (!ok) {
            result = RTC_ETIMEDOUT;
            break;
        }
        const long long t_done = mono_ns();
        t_last_done = t_done;
        e2e.push_back(t_done - t_pub);
        dev.push_back(static_cast<long long>(h->h_done[slot].t_done - h->h_done[slot].t_seen));
        if (cfg->e2e_ns) cfg->e2e_ns[k] = e2e.back();
        if (cfg->dev_ns) cfg->dev_ns[k] = dev.back();
        if (cfg->sink) cfg->sink(cfg->sink_user, k, h->h_dm_ring + static_cast<size_t>(slot) * h->cfg.nact);
    }
    // a loop that ends early tells the kernel to stop at the next frame it waits for
    if (k < n) store_release(&h->h_seq[k % nslot], kStop);
    stop.store(true);
    if (filler.joinable()) filler.join();
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail_handle(h, RTC_EDEVICE, cudaGetErrorString(e));
    const int st = take_status(h, h->stream);
    LOOP_CUDA(cudaMemsetAsync(h->d_gridbar, 0, sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaStreamSynchronize(h->stream));
    h->grid_epoch = 0;

    // with the predictor on, every frame the kernel took pushed one measured vector
    // into the history ring
    if (h->pred_on) h->ring_head = static_cast<int>((h->ring_head + e2e.size()) & 3);
    stats->frames = e2e.size();
    if (!e2e.empty() && t_last_done > t_first_pub)
        stats->frames_per_s = e2e.size() / ((t_last_done - t_first_pub) / 1e9);
    summarise(e2e, stats->e2e_p50_us, stats->e2e_p99_us, stats->e2e_p999_us, stats->e2e_mean_us,
              stats->e2e_rms_jitter_us, stats->e2e_p2p_us);
    summarise(dev, stats->dev_p50_us, stats->dev_p99_us, stats->dev_p999_us, stats->dev_mean_us,
              stats->dev_rms_jitter_us, stats->dev_p2p_us);
    if (st != RTC_OK) return st;
    if (result != RTC_OK) return fail_handle(h, result, "a loop frame did not complete in time");
    return RTC_OK;
}

// ---- resident per-frame calls ---------------------------------------------------
// The loop kernel launched for an unbounded run of frames; rtc_process_frame then
// publishes one frame per call into slot k % RTC_LOOP_SLOTS, with the device views
// of the caller's frame and DM buffers in the slot's pointer pair, and waits for
// the slot's completion record.  Calls are synchronous, so a slot is free again
// by the time it comes round.

namespace {

constexpr unsigned long long kResidentFrames = ~0ull >> 1;   // "until stopped"
constexpr long long kResidentCheckNs = 20ll * 1000 * 1000;   // look at the kernel after 20 ms

// The status word of an ended resident kernel, cleared.  A kernel whose frame wait
// expired (the caller was idle) reports RTC_ETIMEDOUT, which is not an error here.
int resident_status(rtc_handle* h, int& code) {
    LOOP_CUDA(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_gridbar, 0, sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaStreamSynchronize(h->stream));
    h->grid_epoch = 0;
    code = *h->h_status;
    // every frame the kernel finished pushed one measured vector into the history ring
    if (h->pred_on) h->ring_head = static_cast<int>((h->res_head0 + h->res_k) & 3);
    h->res_k = 0;
    return RTC_OK;
}

int resident_launch(rtc_handle* h) {
    for (int i = 0; i < RTC_LOOP_SLOTS; ++i) {
        h->h_seq[i] = 0;
        memset(&h->h_done[i], 0, sizeof(rtc_loop_done));
    }
    LOOP_CUDA(cudaMemsetAsync(h->d_gridbar, 0, sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_donectr, 0, sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_mirror, 0, 3 * RTC_LOOP_SLOTS * sizeof(unsigned long long), h->stream));
    LOOP_CUDA(cudaMemsetAsync(h->d_tseen, 0, 2 * sizeof(unsigned long long), h->stream));
    h->grid_epoch = 0;
    LoopLaunch ll{};
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(const_cast<uint16_t**>(&ll.d_frames)), h->h_ring, 0));
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(const_cast<unsigned long long**>(&ll.d_seq)), h->h_seq, 0));
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(const_cast<unsigned long long**>(&ll.d_ptrs)), h->h_ptrs, 0));
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ll.d_dm), h->h_dm_ring, 0));
    LOOP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ll.d_done), h->h_done, 0));
    ll.frame_elems = static_cast<size_t>(h->cfg.n_wfs) * h->side * h->side;
    ll.n_frames = kResidentFrames;
    ll.nslot = RTC_LOOP_SLOTS;
    ll.n_bands = 1;
    ll.l2_stream = 0;
    h->res_k = 0;
    h->res_head0 = h->ring_head;
    LOOP_CUDA(launch_loop(h, ll, h->stream));
    return RTC_OK;
}

}  // namespace

extern "C" int rtc_resident_start(rtc_handle* h) {
    if (!h) return RTC_EINVAL;
    if (h->in_slot.load()) return fail_handle(h, RTC_ESTATE, "the handle's job is in a server slot");
    if (h->resident) return fail_handle(h, RTC_ESTATE, "the handle is already resident");
    if (!h->calib_loaded || h->store < 0)
        return fail_handle(h, RTC_ESTATE, "calibration maps and control matrix must be loaded");
    if (h->kpad == 0) return fail_handle(h, RTC_ESTATE, "the resident kernel needs at least one valid subaperture");
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != h->cfg.device) cudaSetDevice(h->cfg.device);
    struct Restore {
        int d;
        ~Restore() {
            int cur = -1;
            if (d >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != d) cudaSetDevice(d);
        }
    } restore{dev_prev};
    int rc = ensure_buffers(h);
    if (rc != RTC_OK) return rc;
    if (!h->h_ptrs) {
        LOOP_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&h->h_ptrs),
                                2 * RTC_LOOP_SLOTS * sizeof(unsigned long long), cudaHostAllocMapped));
        memset(h->h_ptrs, 0, 2 * RTC_LOOP_SLOTS * sizeof(unsigned long long));
    }
    LOOP_CUDA(cudaStreamSynchronize(h->stream));
    loop_begin();                       // releases of any handle wait for rtc_resident_stop
    rc = resident_launch(h);
    if (rc != RTC_OK) {
        loop_end();
        return rc;
    }
    h->resident = true;
    return RTC_OK;
}

int resident_frame(rtc_handle* h, const uint16_t* d_frame, float* d_dm) {
    if (reinterpret_cast<uintptr_t>(d_frame) % 16 != 0 || reinterpret_cast<uintptr_t>(d_dm) % 4 != 0)
        return fail_handle(h, RTC_EINVAL, "resident mode: the frame buffer must be 16-byte aligned, dm_out 4-byte");
    for (int attempt = 0; attempt < 2; ++attempt) {
        // a kernel whose frame wait expired while the caller was idle has ended:
        // launch it again (a grid barrier that expired is an error)
        if (cudaStreamQuery(h->stream) != cudaErrorNotReady) {
            int code = RTC_OK;
            int rc = resident_status(h, code);
            if (rc != RTC_OK) return rc;
            if (code != RTC_OK && code != RTC_ETIMEDOUT)
                return fail_handle(h, code, "the resident kernel ended with an error");
            rc = resident_launch(h);
            if (rc != RTC_OK) return rc;
        }
        const unsigned long long k = h->res_k;
        const int slot = static_cast<int>(k % RTC_LOOP_SLOTS);
        h->h_ptrs[2 * slot] = reinterpret_cast<uintptr_t>(d_frame);
        h->h_ptrs[2 * slot + 1] = reinterpret_cast<uintptr_t>(d_dm);
        store_release(&h->h_seq[slot], k + 1);
        const long long t0 = mono_ns();
        bool ended = false;
        while (load_acquire(&h->h_done[slot].seq) != k + 1) {
            const long long dt = mono_ns() - t0;
            if (dt > kResidentCheckNs && cudaStreamQuery(h->stream) != cudaErrorNotReady) {
                ended = load_acquire(&h->h_done[slot].seq) != k + 1;
                break;
            }
            if (dt > kHostWaitNs) {
                // the kernel neither finished the frame nor ended: stop it
                store_release(&h->h_seq[slot], kStop);
                cudaStreamSynchronize(h->stream);
                int code = RTC_OK;
                resident_status(h, code);
                return fail_handle(h, RTC_ETIMEDOUT, "the resident kernel did not finish the frame in time");
            }
        }
        if (!ended) {
            h->res_k = k + 1;
            return RTC_OK;
        }
        // the kernel ended (its frame wait expired) just before this frame was seen:
        // relaunch and publish it again
    }
    return fail_handle(h, RTC_EDEVICE, "the resident kernel could not be restarted");
}

int resident_stop(rtc_handle* h) {
    if (!h->resident) return RTC_OK;
    if (cudaStreamQuery(h->stream) == cudaErrorNotReady)
        store_release(&h->h_seq[h->res_k % RTC_LOOP_SLOTS], kStop);
    const cudaError_t e = cudaStreamSynchronize(h->stream);
    h->resident = false;
    loop_end();
    if (e != cudaSuccess) return fail_handle(h, RTC_EDEVICE, cudaGetErrorString(e));
    int code = RTC_OK;
    const int rc = resident_status(h, code);
    if (rc != RTC_OK) return rc;
    if (code != RTC_OK && code != RTC_ETIMEDOUT)
        return fail_handle(h, code, "the resident kernel ended with an error");
    return RTC_OK;
}

extern "C" int rtc_resident_stop(rtc_handle* h) {
    if (!h) return RTC_EINVAL;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != h->cfg.device) cudaSetDevice(h->cfg.device);
    const int rc = resident_stop(h);
    int cur = -1;
    if (dev_prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != dev_prev) cudaSetDevice(dev_prev);
    return rc;
}
