// Internal state and kernel launchers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <string>
#include <vector>

#include "rtc.h"

// Threads per block of the pixel stage and of the reconstruction stage.
constexpr int kCalibThreads = 256;
constexpr int kMvmThreads = 256;
// Matrix rows handled together by one reconstruction block.
constexpr int kMvmRows = 4;
// Largest split-K factor (partials per actuator summed by the fixed-order tree).
constexpr int kMaxKsplit = 32;

// Completion record of one loop frame, written by the device into mapped host memory.
struct rtc_loop_done {
    unsigned long long seq;      // k + 1 once frame k's DM commands are in host memory
    unsigned long long t_seen;   // device %globaltimer: the latest time a block had its pixel rows
    unsigned long long t_done;   // device %globaltimer when the last block finished
    unsigned long long pad;
};

// Completion record of one rtc_process_frame call whose buffers are in pinned host
// memory, written by the last block of the frame kernel into mapped host memory.
struct rtc_pf_done {
    unsigned long long seq;      // the call's sequence number once its DM commands are written
    int status;                  // the device status word at that time (RTC_OK or an error)
    int pad;
};

// What the frame kernel does for a caller waiting on the host (rtc_process_frame with
// pinned buffers): the frame is read from mapped host memory, and the last block to
// finish writes the completion record.
struct FrameHost {
    rtc_pf_done* done;           // device view of the mapped completion record
    unsigned long long* ctr;     // device count of finished blocks (only grows)
    unsigned long long target;   // the count that completes this launch (set by launch_frame)
    unsigned long long seq;      // value of the record's seq for this call
    const unsigned* units;       // the blocks' copy units of the frame (build_ingest)
    const int4* blk;             // [G] first unit, end unit of each block
    uint16_t* stage;             // device staging of the frame's copied pixels
    int unit;                    // bytes per copy unit
};

// Device-visible addresses of the host ring for one rtc_run_loop call.
struct LoopLaunch {
    const uint16_t* d_frames;
    unsigned long long frame_elems;
    const unsigned long long* d_seq;
    const unsigned long long* d_ptrs;   // [nslot][2] frame and DM device views, or null (ring)
    float* d_dm;
    rtc_loop_done* d_done;
    unsigned long long n_frames;
    int nslot;
    int n_bands;                 // >= 1 bands of pixel rows per frame
    int l2_stream;               // stream the matrix with L2 evict_first whatever its size
};

struct rtc_handle {
    rtc_config cfg{};
    int side = 0;               // frame side in pixels (nsub * npx)
    int n_valid = 0;            // valid subapertures per WFS
    int nslopes = 0;            // 2 * n_valid * n_wfs
    int kpad = 0;               // padded matrix row length (elements)
    int store = -1;             // rtc_dtype of the resident matrix, -1 when none
    int ro_bands = 0;           // readout model of the slice cut (rtc_set_readout): bands,
    long long ro_interval_ns = 0;   // and time between bands
    float gain = 0.f, leak = 1.f;
    int thr_mode = 0;
    float thr = 0.f;
    bool calib_loaded = false;

    cudaStream_t stream = nullptr;
    int num_sms = 1;                // blocks the fused kernels may use (a server slot lowers it)
    int dev_sms = 1;                // streaming multiprocessors of the device

    std::vector<int32_t> rc;    // host copy of the subaperture map (row, col) pairs

    // device buffers (owned)
    int2* d_rc = nullptr;           // [n_valid] (row, col) grid position of each valid subap
    float* d_dark = nullptr;        // [n_wfs][n_valid][npx*npx] dark, subap-major
    float* d_gainmap = nullptr;     // [n_wfs][n_valid][npx*npx] 1/flat, subap-major
    void* d_M = nullptr;            // slice-major matrix in the stored type (see stream_mvm.cuh)
    int64_t m_bytes = 0;            // bytes of d_M
    float* d_scale = nullptr;       // [nact] FP8 / INT8 row scales
    // slice table of the loaded matrix: S slices of consecutive subapertures
    int sl_S = 0;
    std::vector<long long> sl_off;  // [S] byte offset of each slice (16-byte aligned)
    std::vector<int> sl_rowbytes;   // [S] bytes per row (multiple of 4)
    std::vector<int> sl_g0;         // [S + 1] first subaperture of each slice
    std::vector<int> sl_loc;        // [S + 1] float offset of each slice's slopes in a local vector
    bool sl_equal = false;          // sl_g0[s] == nt * s / S for every s
    bool sl_plane = false;          // slices stored in the plane layout (1- and 2-byte stores)
    long long* d_sl_off = nullptr;
    int* d_sl_rowbytes = nullptr;
    int* d_sl_g0 = nullptr;
    int* d_sl_loc = nullptr;
    float* d_s = nullptr;           // [kpad] slope vector, zero padded
    float* d_a = nullptr;           // [nact] integrator state
    float* d_partial = nullptr;     // [2][dev_sms][nact] partial DM vectors, one per slice (scratch;
                                    // the persistent loop alternates the halves frame by frame)
    uint16_t* d_frame = nullptr;    // [n_wfs][side][side] staging for host frames
    int* d_status = nullptr;        // device-side error word (RTC_ETIMEDOUT from bounded waits)
    unsigned long long* d_gridbar = nullptr;  // grid-barrier arrival counter (only grows)
    unsigned long long grid_epoch = 0;        // block arrivals expected so far on d_gridbar

    // persistent loop (allocated by the first rtc_run_loop)
    float* d_sbuf = nullptr;                  // [2][kpad] slope vectors by frame parity
    unsigned long long* d_donectr = nullptr;  // finished-block counter
    unsigned long long* d_tseen = nullptr;    // [2] device time the last block had its frame rows
    unsigned* d_units = nullptr;              // frame copy units of each block (see loop_kernel.cu)
    size_t units_cap = 0;                     // entries d_units holds
    int4* d_blk = nullptr;                    // [dev_sms] per block: first unit, end, band, 0
    int ingest_G = -1, ingest_unit = 0, ingest_bands = 0;   // what d_units / d_blk were built for
    uint16_t* h_ring = nullptr;               // pinned mapped [RTC_LOOP_SLOTS][n_wfs][H][W]
    unsigned long long* h_seq = nullptr;      // pinned mapped [RTC_LOOP_SLOTS]
    float* h_dm_ring = nullptr;               // pinned mapped [RTC_LOOP_SLOTS][nact]
    rtc_loop_done* h_done = nullptr;          // pinned mapped [RTC_LOOP_SLOTS]
    unsigned long long* h_ptrs = nullptr;     // pinned mapped [RTC_LOOP_SLOTS][2]: resident frame/DM views
    unsigned long long* d_mirror = nullptr;   // device [RTC_LOOP_SLOTS] + [RTC_LOOP_SLOTS][2]: the loop's
                                              // device copy of the published flags and buffers
    bool resident = false;                    // rtc_resident_start .. rtc_resident_stop
    unsigned long long res_k = 0;             // frames the present resident kernel has finished
    int res_head0 = 0;                        // predictor ring head when it was launched
    int sbuf_kpad = -1;                       // kpad d_sbuf was sized for

    std::atomic<bool> in_slot{false};         // owned by a server slot (rtc_slot_submit)

    // learned slope predictor (rtc_load_predictor)
    struct MlpDev* pred = nullptr;            // network weights on the device
    bool pred_on = false;
    float pred_sigma = 1.f;
    int* d_nbr = nullptr;                     // [n_valid][25] neighbour table
    float* d_ring = nullptr;                  // [4][kpad] last measured slope vectors
    int ring_head = 3;                        // row of the newest vector
    float* d_spred = nullptr;                 // [kpad] predicted slopes, zero padded
    int* h_status = nullptr;        // pinned host mirror of d_status
    // rtc_process_frame with pinned host buffers (allocated at its first such call)
    rtc_pf_done* h_pf_done = nullptr;         // pinned mapped completion record
    rtc_pf_done* d_pf_done = nullptr;         // its device view
    unsigned long long* d_pf_ctr = nullptr;   // finished-block count of those launches
    unsigned long long pf_arrivals = 0;       // block arrivals expected so far on d_pf_ctr
    unsigned long long pf_seq = 0;            // calls made so far

    std::string err;
};

// Pixel calibration + centre of gravity + slope packing for every valid
// subaperture of every WFS frame.  Writes s[0 .. nslopes).
cudaError_t launch_calib_cog(const rtc_handle* h, const uint16_t* d_frame, float* d_s,
                             cudaStream_t st);

// Slice-by-slice reconstruction (TMA bulk copies) with the fixed-order sum of the
// partial DM vectors and the leaky integrator (see stream_mvm.cuh).
cudaError_t mvm_stream_configure();
cudaError_t launch_decay(const rtc_handle* h, float* d_dm_out, cudaStream_t st);

// Fused frame kernel (pixel stage + grid barrier + streaming MVM + integrator),
// one cooperative launch per frame; the slopes land in h->d_s.
cudaError_t frame_kernel_configure();

// The per-block copy units of a frame for a G-block launch (loop_kernel.cu); rebuilt
// only when G, the unit or the bands change, or the slices were cut again.
int build_ingest(rtc_handle* h, int G, int unit, int n_bands);

// Persistent loop kernel (see loop_kernel.cu).
cudaError_t loop_kernel_configure();
cudaError_t launch_loop(rtc_handle* h, const LoopLaunch& ll, cudaStream_t st);
// One frame through the fused kernel.  d_s_meas == nullptr: the plain path (slopes in
// h->d_s).  Otherwise the predictor path: measured slopes into d_s_meas = ring row
// `head` of h->d_ring, predicted slopes into h->d_spred, reconstruction from those.
// fh (optional): the frame and d_dm_out are device views of mapped host memory, and
// the launch writes fh->done when its commands are out.
cudaError_t launch_frame(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, float* d_s_meas,
                         int head, cudaStream_t st, FrameHost* fh = nullptr);
cudaError_t launch_mvm_integrate(rtc_handle* h, const float* d_s, float* d_dm_out,
                                 cudaStream_t st);

// The same split-K MVM + integrator on caller-described buffers: matrix [nact][kpad]
// in the stored type, s [kpad], partial scratch [ksplit][nact], counters
// [ceil(nact/kMvmRows)] that must be zero on entry.
cudaError_t launch_mvm_raw(int store, const void* d_M, const float* d_scale, int nact, int kpad,
                           const float* d_s, int ksplit, float* d_partial, unsigned* d_count,
                           float* d_a, float* d_dm_out, float gain, float leak, cudaStream_t st);

// Store a device matrix [nact][ncol] (FP32, or already in the stored type when
// src == store) into the slice-major layout: column c goes to slice colmap[c].x,
// local column colmap[c].y.  From FP32, the FP8 / INT8 row scales are computed
// into d_scale first.
cudaError_t launch_layout(int src, int store, const void* d_src, int nact, int ncol,
                          const int2* d_colmap, const long long* d_off, const int* d_rowbytes, int plane,
                          float* d_scale, void* d_dst, cudaStream_t st);

// Move a matrix between two slice layouts of the same store (esize bytes per
// entry): column c from (old_colmap[c]) to (new_colmap[c]).
cudaError_t launch_relayout(int esize, int old_plane, int new_plane, const void* d_old, const int2* d_old_colmap,
                            const long long* d_old_off, const int* d_old_rowbytes, int nact, int ncol,
                            const int2* d_new_colmap, const long long* d_new_off, const int* d_new_rowbytes,
                            void* d_new, cudaStream_t st);

// Read and clear the device status word after `st` drains (RTC_OK or the recorded
// error, which also restarts the grid-barrier count); set the handle's message.
int take_status(rtc_handle* h, cudaStream_t st);

// One frame through the whole path on device buffers, enqueued on st (the work of
// rtc_process_frame_async after its checks); and whether the handle is ready for it.
int rtc_enqueue_frame(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out, cudaStream_t st);
bool rtc_handle_ready(const rtc_handle* h);
// Device memory the handle holds (matrix, calibration, state, staging).
int64_t rtc_handle_device_bytes(const rtc_handle* h);
int fail_handle(rtc_handle* h, int code, const char* msg);

// Resident mode (rtc_loop.cu): one frame through the resident kernel (pinned
// buffers, device views); stop the kernel (rtc_resident_stop's body).
int resident_frame(rtc_handle* h, const uint16_t* d_frame, float* d_dm);
int resident_stop(rtc_handle* h);
// RTC_ESTATE (with the reason recorded) if the handle's device work is owned by a
// server slot or a resident kernel, else RTC_OK.
int handle_busy(rtc_handle* h);

// Host planning (plan.cu).  plan_slices: first subaperture of each slice (then
// the subaperture count): equal slices, or with n_bands > 1 the asymmetric cut
// for that readout.  plan_ingest: the persistent loop's per-block copy units and
// completing band (blk: 4 ints per block) for G blocks over slices g0[0..S].
std::vector<int> plan_slices(const int32_t* rc, int nv, int nw, int npx, int side, int nact, int esz,
                             int max_slices, int n_bands, long long interval_ns);
void plan_ingest(const int32_t* rc, int nv, int npx, int side, const int* g0, int S, int G, int unit,
                 int n_bands, std::vector<unsigned>& units, std::vector<int>& blk);

// While a persistent loop runs, a release (rtc_destroy, rtc_mlp_destroy,
// rtc_server_destroy) would wait for the device and so for the loop, whose kernel
// in turn waits for frames from the host thread: called from a source or sink
// callback, or from a garbage collector that runs inside one, it would deadlock
// until the loop's bounded waits expire.  Releases made while any loop runs are
// therefore queued and carried out when the last loop has ended.
void loop_begin();
void loop_end();
// Run f now, or queue it if a loop is running; true when queued.
bool release_or_defer(std::function<void()> f);

// Message returned by rtc_last_error(NULL) for failures of calls without a handle.
void rtc_set_global_error(const char* msg);
