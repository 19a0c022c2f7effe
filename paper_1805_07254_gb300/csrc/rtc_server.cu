// Serving several independent real-time controllers on one GPU with continuous
// batching (rtc_server_* / rtc_slot_* in include/rtc.h).
//
// A job (one handle + a run of frames) is admitted into a free slot when the
// server's device-memory budget has room for the handle, while other jobs keep
// running.  Admission enqueues all of the job's frames on the slot's own stream:
// host->device copy of the frame, the fused frame kernel, device->host copy of the
// DM commands.  The handle's frame kernel is limited to num_SMs / max_slots
// blocks while it is in the slot, so the kernels of different slots fit on the
// device together and overlap (one block per SM each), and a job computes the
// same results whatever runs beside it.  Checkpoint events give the progress;
// the last one frees the slot.

#include <mutex>
#include <vector>

#include "rtc_internal.h"

namespace {

constexpr int kMaxSlots = 32;
constexpr int kCheckpoints = 64;      // progress events per job

struct Job {
    bool active = false;
    rtc_handle* h = nullptr;
    int saved_sms = 0;
    int64_t bytes = 0;
    uint64_t n_frames = 0;
    std::vector<cudaEvent_t> marks;    // events after frame (checkpoint index + 1) * step - 1
    std::vector<uint64_t> mark_frame;  // frames done when each event completes
};

int sfail(int code, const char* msg) {
    rtc_set_global_error(msg);
    return code;
}

}  // namespace

struct rtc_server {
    int device = 0;
    int max_slots = 1;
    int share = 1;                     // SMs (frame-kernel blocks) per slot
    int64_t budget = 0;
    int64_t in_use = 0;
    std::vector<Job> jobs;
    std::vector<cudaStream_t> streams;
    mutable std::mutex mu;
};

namespace {

struct Dev {
    int prev = -1;
    explicit Dev(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~Dev() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void release(rtc_server* s, Job& j) {
    for (cudaEvent_t e : j.marks) cudaEventDestroy(e);
    j.marks.clear();
    j.mark_frame.clear();
    if (j.h) {
        j.h->num_sms = j.saved_sms;
        j.h->in_slot = false;
    }
    s->in_use -= j.bytes;
    j = Job{};
}

}  // namespace

extern "C" {

int rtc_server_create(int32_t device, int32_t max_slots, int64_t mem_budget_bytes, rtc_server** out) {
    if (!out) return sfail(RTC_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return sfail(RTC_EINVAL, "device not available");
    if (max_slots < 1 || max_slots > kMaxSlots || mem_budget_bytes <= 0)
        return sfail(RTC_EINVAL, "max_slots must be 1..32 and the budget positive");
    Dev d(device);
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    rtc_server* s = new rtc_server();
    s->device = device;
    s->max_slots = max_slots;
    s->share = nsm / max_slots > 0 ? nsm / max_slots : 1;
    s->budget = mem_budget_bytes;
    s->jobs.resize(max_slots);
    s->streams.resize(max_slots, nullptr);
    for (int i = 0; i < max_slots; ++i)
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            rtc_server_destroy(s);
            return sfail(RTC_ENOMEM, "cannot create the slot streams");
        }
    *out = s;
    return RTC_OK;
}

int rtc_server_destroy(rtc_server* s) {
    if (!s) return RTC_OK;
    if (release_or_defer([s] { rtc_server_destroy(s); })) return RTC_OK;
    Dev d(s->device);
    for (size_t i = 0; i < s->streams.size(); ++i) {
        if (s->streams[i]) cudaStreamSynchronize(s->streams[i]);
        if (s->jobs[i].active) release(s, s->jobs[i]);
        if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    }
    delete s;
    return RTC_OK;
}

int rtc_slot_submit(rtc_server* s, rtc_handle* h, const uint16_t* frames, uint64_t n_frames,
                    float* dm_out, int32_t* slot) {
    if (!s || !h || !frames || !dm_out || !slot || n_frames == 0)
        return sfail(RTC_EINVAL, "server, handle, frames, dm_out and slot must be given, n_frames > 0");
    if (h->cfg.device != s->device) return sfail(RTC_ESTATE, "handle is on another device");
    if (!rtc_handle_ready(h)) return sfail(RTC_ESTATE, "handle has no calibration or matrix");
    std::lock_guard<std::mutex> lock(s->mu);
    if (h->in_slot) return sfail(RTC_ESTATE, "handle is already in a slot");
    if (h->resident) return sfail(RTC_ESTATE, "handle is resident (rtc_resident_stop first)");
    int free_slot = -1;
    for (int i = 0; i < s->max_slots; ++i)
        if (!s->jobs[i].active) {
            free_slot = i;
            break;
        }
    const int64_t bytes = rtc_handle_device_bytes(h);
    if (free_slot < 0) return sfail(RTC_EBUSY, "all slots are busy");
    if (s->in_use + bytes > s->budget) return sfail(RTC_EBUSY, "not enough memory budget now");

    Dev d(s->device);
    Job& j = s->jobs[free_slot];
    j.active = true;
    j.h = h;
    j.bytes = bytes;
    j.n_frames = n_frames;
    j.saved_sms = h->num_sms;
    h->num_sms = s->share;
    h->in_slot = true;
    s->in_use += bytes;

    cudaStream_t st = s->streams[free_slot];
    const size_t elems = static_cast<size_t>(h->cfg.n_wfs) * h->side * h->side;
    const uint64_t step = (n_frames + kCheckpoints - 1) / kCheckpoints;
    int rc = RTC_OK;
    for (uint64_t k = 0; k < n_frames && rc == RTC_OK; ++k) {
        if (cudaMemcpyAsync(h->d_frame, frames + k * elems, elems * sizeof(uint16_t),
                            cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = RTC_EDEVICE;
            break;
        }
        rc = rtc_enqueue_frame(h, h->d_frame, nullptr, st);
        if (rc != RTC_OK) break;
        if (cudaMemcpyAsync(dm_out + k * h->cfg.nact, h->d_a, h->cfg.nact * sizeof(float),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            rc = RTC_EDEVICE;
            break;
        }
        if ((k + 1) % step == 0 || k + 1 == n_frames) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(e, st) != cudaSuccess) {
                rc = RTC_EDEVICE;
                break;
            }
            j.marks.push_back(e);
            j.mark_frame.push_back(k + 1);
        }
    }
    if (rc != RTC_OK) {
        cudaStreamSynchronize(st);
        release(s, j);
        return sfail(rc, "job submission failed");
    }
    *slot = free_slot;
    return RTC_OK;
}

int rtc_slot_poll(rtc_server* s, int32_t slot, uint64_t* frames_done) {
    if (!s || slot < 0 || slot >= s->max_slots) return sfail(RTC_EINVAL, "bad slot");
    std::lock_guard<std::mutex> lock(s->mu);
    Job& j = s->jobs[slot];
    if (!j.active) return sfail(RTC_EINVAL, "slot is not running a job");
    Dev d(s->device);
    uint64_t done = 0;
    cudaError_t last = cudaSuccess;
    for (size_t i = 0; i < j.marks.size(); ++i) {
        last = cudaEventQuery(j.marks[i]);
        if (last != cudaSuccess) break;
        done = j.mark_frame[i];
    }
    if (frames_done) *frames_done = done;
    if (last == cudaErrorNotReady) return RTC_EBUSY;
    int rc = RTC_OK;
    if (last != cudaSuccess) rc = sfail(RTC_EDEVICE, cudaGetErrorString(last));
    else {
        const int st = take_status(j.h, s->streams[slot]);
        if (st != RTC_OK) rc = sfail(st, "a bounded device wait expired in this job");
    }
    release(s, j);
    return rc;
}

int rtc_server_info(const rtc_server* s, int32_t* active_slots, int64_t* mem_in_use) {
    if (!s) return RTC_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);    // submit and poll change both fields under it
    int n = 0;
    for (const Job& j : s->jobs) n += j.active ? 1 : 0;
    if (active_slots) *active_slots = n;
    if (mem_in_use) *mem_in_use = s->in_use;
    return RTC_OK;
}

}  // extern "C"
