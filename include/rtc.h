/*
 * rtc.h -- C ABI of the GB300 single-conjugate adaptive-optics real-time
 * controller (librtc.so).
 *
 * The library runs, on one CUDA device, the per-frame pipeline of Sec. 2.1 /
 * Fig. 3 of Jenkins, Basden & Myers (2018):
 *   (a) pixel calibration   p = (raw - dark) * (1/flat), then a threshold;
 *   (b) centre-of-gravity   one (x, y) gradient per valid subaperture;
 *       slope packing       all x gradients first, then all y (Fig. 3 caption);
 *   (c) reconstruction      d = M s, a dense matrix-vector product (Sec. 1.1.1,
 *                           memory-bandwidth bound);
 *   (d) gain                a <- leak * a + g * d  (Sec. 2.1's gain factor,
 *                           with a leak; leak = 1 gives the plain gain).
 * The partial products of (c) are summed in a fixed-order tree, the GPU form of
 * the tree-like partial-vector addition of Sec. 2.3.5.
 *
 * Conventions for every entry point:
 *   - Every function returns an int status: RTC_OK (0) or a negative RTC_E*
 *     code.  The library never aborts the process.  rtc_last_error() gives a
 *     human-readable message for the last failure on a handle.
 *   - Pointers documented as "host" are ordinary (pageable or pinned) host
 *     memory; "device" pointers are CUDA device memory on the handle's device.
 *     Input pointers are borrowed for the duration of the call only; the library
 *     copies what it keeps.  Output buffers are allocated by the caller.
 *   - All arrays are dense and row-major.  Frames are uint16, (n_wfs, H, W) with
 *     H = W = nsub * npx.  Slope vectors are float32, per WFS the x block then
 *     the y block (length 2 * n_valid), WFS after WFS.
 *   - A handle is not thread-safe: calls on one handle must be serialised by the
 *     caller.  Different handles are independent.
 *   - Device-side errors (a failed launch, a fault reported by the runtime)
 *     return RTC_EDEVICE; a bounded device wait that ran out returns
 *     RTC_ETIMEDOUT.
 */
#ifndef RTC_H
#define RTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTC_OK          0
#define RTC_EINVAL     (-1)   /* bad argument or inconsistent sizes */
#define RTC_ENOMEM     (-2)   /* device or pinned-host allocation failed */
#define RTC_EDEVICE    (-3)   /* CUDA reported an error */
#define RTC_ETIMEDOUT  (-4)   /* a bounded device-side wait expired */
#define RTC_ESTATE     (-5)   /* call not valid in the handle's current state */
#define RTC_EBUSY      (-6)   /* resource in use (e.g. all serving slots taken) */

/* Storage type of the control matrix.  Accumulation is always FP32. */
typedef enum rtc_dtype {
    RTC_F32 = 0,        /* IEEE binary32 */
    RTC_BF16 = 1,       /* bfloat16, round-to-nearest-even from FP32 */
    RTC_FP8_E4M3 = 2,   /* E4M3 ("fn": bias 7, max 448) codes with one FP32 scale per row */
    RTC_F16 = 3,        /* IEEE binary16, round-to-nearest-even (Sec. 2.3.4's 16-bit format) */
    RTC_INT8 = 4        /* signed 8-bit codes in [-127, 127] with one FP32 scale per row */
} rtc_dtype;

typedef struct rtc_config {
    int32_t nsub;       /* subapertures across the square grid (e.g. 74) */
    int32_t npx;        /* pixels per subaperture side (e.g. 10); frame side = nsub*npx */
    int32_t n_wfs;      /* wavefront-sensor frames per step, stacked (1 for SCAO) */
    int32_t nact;       /* actuators = rows of the control matrix */
    float   obs;        /* central obscuration (fraction of the diameter) for the
                           default subaperture map; see rtc_load_subaps */
    float   gain;       /* integrator gain g */
    float   leak;       /* integrator leak */
    int32_t thr_mode;   /* 0: p < thr -> 0;  1: p -> max(p - thr, 0) */
    float   thr;        /* threshold in calibrated ADU */
    int32_t device;     /* CUDA device ordinal */
    int32_t reserved;   /* must be 0 */
} rtc_config;

typedef struct rtc_info {
    int32_t n_valid;        /* valid subapertures per WFS */
    int32_t nslopes;        /* 2 * n_valid * n_wfs */
    int32_t nact;
    int32_t kpad;           /* matrix row length after padding to a multiple of 16 */
    int32_t store;          /* rtc_dtype of the loaded matrix, -1 if none */
    /* layout and launch plan of the loaded matrix (0 while none): */
    int32_t slices;         /* column slices (consecutive subapertures), each stored
                               contiguously and multiplied by one block */
    int32_t blocks;         /* blocks of the fused kernels, one per SM */
    int32_t tile_rows;      /* matrix rows per streamed tile */
    int32_t ring_stages;    /* tiles in flight per block */
    int64_t matrix_bytes;   /* algorithmic bytes of the stored matrix (unpadded, incl. scales) */
    int64_t frame_bytes;    /* n_wfs * H * W * 2 */
    int64_t calib_bytes;    /* bytes of the per-pixel calibration data read per frame */
} rtc_info;

typedef struct rtc_handle rtc_handle;

/* Build/version string of the library (static storage; never NULL). */
const char* rtc_version(void);

/* Message of the last failure on h (or, when h is NULL, of the last failed call
 * without a handle: rtc_create, rtc_mvm_integrate_noalloc).  Static or
 * handle-owned storage valid until the next call on h. */
const char* rtc_last_error(const rtc_handle* h);

/* Validate cfg and allocate the handle's resident device state.  The default
 * subaperture map is the set whose centres lie in the annulus
 * obs*nsub/2 <= r <= nsub/2 (row-major order); the integrator starts at zero.
 * Errors: RTC_EINVAL (bad geometry or parameters), RTC_ENOMEM, RTC_EDEVICE. */
int rtc_create(const rtc_config* cfg, rtc_handle** out);

/* Release everything the handle owns.  NULL is accepted.  RTC_ESTATE while the
 * handle's job is in a server slot (rtc_slot_submit).  Called while any
 * rtc_run_loop is running (from its callbacks, or from another thread), the
 * release is queued and carried out when the last running loop returns: freeing
 * device memory waits for the device, which would wait for the loop. */
int rtc_destroy(rtc_handle* h);

/* Replace the subaperture map.  rc: host int32 [n_valid][2] of (row, col) grid
 * positions, strictly increasing in row-major order, each inside the grid.
 * Invalidates the loaded calibration maps and control matrix (their sizes
 * depend on n_valid), which must be loaded again.  Errors: RTC_EINVAL. */
int rtc_load_subaps(rtc_handle* h, const int32_t* rc, int32_t n_valid);

/* Calibration maps for Fig. 3 (a).  dark, flat: host float32 [n_wfs][H][W]
 * (npix must equal n_wfs*H*W).  The library inverts flat in FP32
 * (gain = 1.0f/flat, correctly rounded) and keeps, per valid subaperture, the
 * dark and gain values it needs.  flat entries must be finite and non-zero.
 * Errors: RTC_EINVAL, RTC_EDEVICE. */
int rtc_load_calib(rtc_handle* h, const float* dark, const float* flat, int64_t npix);

/* Threshold of Fig. 3 (a): mode 0 zeroes pixels with p < thr; mode 1 maps p to
 * p - thr when p > thr and to 0 otherwise.  The comparison is made on the FP32
 * calibrated value.  Errors: RTC_EINVAL. */
int rtc_set_threshold(rtc_handle* h, int32_t mode, float thr);

/* Control matrix for Fig. 3 (c).  M: host, row-major [nact][nslopes] of type
 * src (float32, bf16 or binary16 bits as uint16, E4M3 codes as uint8, or int8
 * codes).  nact and nslopes must match the handle.  store selects the device
 * storage: from an RTC_F32 source the library quantises on the device (BF16 and
 * F16: round to nearest even; FP8: per-row scale = max|M_r| / 448, codes =
 * e4m3_rn_satfinite(M_rj / scale); INT8: per-row scale = max|M_r| / 127, codes =
 * clamp(rint(M_rj / scale), -127, 127); every division one FP32 operation; a zero
 * row gets scale 1); otherwise store must equal src and, for FP8 and INT8,
 * row_scales (host float32 [nact]) must be given.  The dot product of a scaled
 * row is scale_r * sum_j code_rj s_j.  Rows are padded with zeros to kpad
 * entries.  Errors: RTC_EINVAL, RTC_ENOMEM, RTC_EDEVICE. */
int rtc_load_cmat(rtc_handle* h, const void* M, int32_t nact, int32_t nslopes,
                  int32_t src, int32_t store, const float* row_scales);

/* Integrator parameters of Fig. 3 (d).  Errors: RTC_EINVAL (non-finite). */
int rtc_set_gain(rtc_handle* h, float gain, float leak);

/* Zero the integrator state (and the predictor's slope history). */
int rtc_reset(rtc_handle* h);

/* Copy the integrator state (float32 [nact]) to host memory. */
int rtc_get_dm(rtc_handle* h, float* out);

/* Sizes and byte counts of the loaded configuration. */
int rtc_get_info(const rtc_handle* h, rtc_info* out);

/* One frame through (a)-(d), synchronously, with host buffers.
 * frame: host uint16 [n_wfs][H][W]; dm_out: host float32 [nact] receives the
 * updated integrator state; slopes_out: host float32 [nslopes] or NULL.
 * The frame is copied to the device, processed on the handle's stream and the
 * results copied back before the call returns.
 * Errors: RTC_ESTATE (calibration or matrix not loaded), RTC_EDEVICE. */
int rtc_process_frame(rtc_handle* h, const uint16_t* frame, float* dm_out, float* slopes_out);

/* The same step on device buffers, enqueued on `stream` (a cudaStream_t; NULL
 * means the handle's own non-blocking stream, which does not wait for work on the
 * legacy default stream: pass cudaStreamLegacy to order the call after such
 * work) without synchronising.  d_frame must be 16-byte
 * aligned.  d_dm_out (float32 [nact]) and d_slopes_out (float32 [nslopes]) may
 * be NULL.  The integrator state lives on the device; consecutive calls on one
 * stream form the closed loop.  Errors: RTC_EINVAL, RTC_ESTATE, RTC_EDEVICE. */
int rtc_process_frame_async(rtc_handle* h, const uint16_t* d_frame, float* d_dm_out,
                            float* d_slopes_out, void* stream);

/* Stage (a)-(b) alone: calibrate d_frame and write the slope vector into the
 * handle's resident slope buffer (and into d_slopes_out, float32 [nslopes], when
 * not NULL), enqueued on `stream` (NULL: own stream).  d_frame must be 16-byte
 * aligned.  Errors: RTC_EINVAL, RTC_ESTATE, RTC_EDEVICE. */
int rtc_centroid_async(rtc_handle* h, const uint16_t* d_frame, float* d_slopes_out, void* stream);

/* Stage (c)-(d) alone: d = M s and the integrator update, enqueued on `stream`.
 * d_slopes: device float32 [nslopes] to reconstruct from, or NULL to use the
 * resident slope buffer written by the last rtc_centroid_async on this handle.
 * d_dm_out: device float32 [nact] or NULL.  Errors: RTC_EINVAL, RTC_ESTATE,
 * RTC_EDEVICE. */
int rtc_reconstruct_async(rtc_handle* h, const float* d_slopes, float* d_dm_out, void* stream);

/* Block until all work enqueued by the handle on `stream` (NULL: own stream) is
 * done, and report any device error.  Errors: RTC_EDEVICE. */
int rtc_synchronize(rtc_handle* h, void* stream);

/* Asymmetric subaperture allocation (Sec. 2.3.3, Fig. 6 (d)) for frames that
 * arrive in n_bands bands of pixel rows, band_interval_us apart (the banded
 * publication of rtc_run_loop).  The matrix is cut into slices of consecutive
 * subapertures, one per block of the fused kernels; by default the slices are
 * equal.  With a readout model the cut gives the subapertures of the last rows
 * small slices of their own and those that arrive early large ones (at most twice
 * the mean), so that every block finishes at about the same time after the last
 * band and last pixel -> DM latency drops.  The resident matrix, if any, is
 * re-laid out on the device; the model also applies to later rtc_load_cmat calls.
 * n_bands = 0 or 1 restores equal slices.  Results depend on the cut only through
 * the order of the partial sums, and are the same for rtc_process_frame and
 * rtc_run_loop under any cut.  Errors: RTC_EINVAL (n_bands outside 0 .. H,
 * band_interval_us outside [0, 1e6]), RTC_ENOMEM, RTC_EDEVICE (the matrix is then
 * unloaded). */
int rtc_set_readout(rtc_handle* h, int32_t n_bands, double band_interval_us);

/* ---- planning helpers (host only) ------------------------------------------
 * What rtc_set_readout and rtc_run_loop work out on the host, without a handle or
 * a device, for inspection and tests.  rc: int32 [n_valid][2] (row, col) grid
 * positions of one WFS's valid subapertures, as for rtc_load_subaps; with n_wfs
 * WFS the subapertures are numbered WFS by WFS (gi = w * n_valid + i). */

/* The slice cut: g0_out[0 .. *n_slices] receives the first subaperture of each of
 * at most max_slices slices of consecutive subapertures, then their count.  With
 * n_bands <= 1 the slices are equal; otherwise the asymmetric cut of
 * rtc_set_readout for n_bands bands band_interval_us apart, with the cost model
 * of a `store` (rtc_dtype) matrix of nact rows.  g0_out holds max_slices + 1
 * entries.  Errors: RTC_EINVAL. */
int rtc_plan_slices(const int32_t* rc, int32_t n_valid, int32_t n_wfs, int32_t nsub, int32_t npx,
                    int32_t nact, int32_t store, int32_t max_slices, int32_t n_bands,
                    double band_interval_us, int32_t* g0_out, int32_t* n_slices);

/* The persistent loop's ingest table for `blocks` blocks over the slices g0[0 ..
 * n_slices] (block b takes slices n_slices*b/blocks .. n_slices*(b+1)/blocks - 1):
 * blk_out[4b .. 4b+3] = {first unit, end unit, band that completes the block, 0}
 * and units_out[first .. end) the block's copy units, sorted and distinct: frame
 * byte offset / unit_bytes (2, 4 or 16) of every unit that the pixel rows of its
 * subapertures touch, the frame being uint16 [n_wfs][H][W], H = W = nsub * npx.
 * *n_units receives the total; units_out may be NULL to ask for it, else it holds
 * units_cap entries.  Errors: RTC_EINVAL (bad geometry, slices that are empty or
 * do not cover 0 .. n_wfs * n_valid, units_cap too small). */
int rtc_plan_ingest(const int32_t* rc, int32_t n_valid, int32_t n_wfs, int32_t nsub, int32_t npx,
                    const int32_t* g0, int32_t n_slices, int32_t blocks, int32_t unit_bytes,
                    int32_t n_bands, int32_t* blk_out, uint32_t* units_out, int64_t units_cap,
                    int64_t* n_units);

/* ---- persistent real-time loop ---------------------------------------------
 * The paper's RTC runs its threads continuously and hands work over through
 * spinning on flags rather than sleeping (Sec. 2.3.2); latency is measured from
 * the last pixel to the DM demand being ready, jitter is its variation (Sec. 3).
 * rtc_run_loop is the GPU form: one persistent kernel keeps calibration, matrix
 * and integrator resident and loops over frames.  A host thread publishes each
 * frame in a ring of pinned, device-mapped buffers by setting a sequence flag;
 * the kernel's blocks spin (bounded) on that flag, each copies the pixels of its
 * own subapertures from host memory, computes its share of the DM commands, and
 * the commands go to mapped host memory with a completion record carrying device
 * timestamps. */

#define RTC_LOOP_SLOTS 8            /* frame slots in the host ring */

/* Fill dst (pinned host memory, uint16 [n_wfs][H][W]) with frame k.  Return 0,
 * or non-zero to end the loop early.  Called on a library-owned thread.  The
 * source and sink callbacks must not make CUDA calls that wait for the device
 * (cudaDeviceSynchronize, cudaFree, ...): the device is running the loop, which
 * waits for them.  The library's own release calls are safe (they are queued). */
typedef int (*rtc_frame_source)(void* user, uint64_t k, uint16_t* dst);

/* Receives the DM commands (float32 [nact], valid during the call) of frame k,
 * on the thread that called rtc_run_loop, after the frame's latency is taken. */
typedef void (*rtc_dm_sink)(void* user, uint64_t k, const float* dm);

typedef struct rtc_loop_config {
    uint64_t n_frames;           /* frames to process (> 0) */
    double rate_hz;              /* publish at this rate; 0: each frame as soon as the
                                    previous one's DM commands are out */
    rtc_frame_source source;     /* fills each frame, or NULL to cycle `preload` */
    void* source_user;
    const uint16_t* preload;     /* host frames [n_preload][n_wfs][H][W] (source == NULL) */
    int32_t n_preload;           /* 1 .. RTC_LOOP_SLOTS */
    rtc_dm_sink sink;            /* or NULL */
    void* sink_user;
    int64_t* e2e_ns;             /* [n_frames] publication (of the last band) -> DM visible
                                    on the host, or NULL */
    int64_t* dev_ns;             /* [n_frames] the last block has its pixel rows -> DM
                                    written, device clock, or NULL */
    int32_t n_bands;             /* 0 or 1: each frame is published whole.  2 .. H: in
                                    n_bands bands of pixel rows, top to bottom, as a
                                    rolling-shutter camera reads out; band j holds rows
                                    floor(H j / n_bands) .. floor(H (j+1) / n_bands) - 1 of
                                    every WFS.  Each block of the kernel starts as soon as
                                    the rows its subapertures cover have arrived (the
                                    paper's processing of pixels during readout, Sec. 2.2). */
    double band_interval_us;     /* host time between the publication of successive bands */
    int32_t matrix_l2;           /* 0: a matrix of at most 80 MB is streamed with the default
                                    L2 policy, so that it can stay in L2 from frame to frame,
                                    a larger one with L2 evict_first; 1: evict_first whatever
                                    its size (lines may still hit L2 when nothing else
                                    competes for it) */
} rtc_loop_config;

/* Latency statistics of one rtc_run_loop call.  "e2e": host clock, from the flag
 * that publishes the frame (with bands: its last band) to the moment the host
 * sees the completion record (the DM commands are in host memory).  "dev": device
 * clock, from the moment the last block has the pixel rows it needs to the last
 * block finishing its DM commands: last pixel seen -> DM demand written. */
typedef struct rtc_stats {
    uint64_t frames;             /* frames completed */
    double frames_per_s;         /* completed frames / (last completion - first publish) */
    double e2e_p50_us, e2e_p99_us, e2e_p999_us, e2e_mean_us, e2e_rms_jitter_us, e2e_p2p_us;
    double dev_p50_us, dev_p99_us, dev_p999_us, dev_mean_us, dev_rms_jitter_us, dev_p2p_us;
} rtc_stats;

/* Run the persistent loop for cfg->n_frames frames and return when they are done
 * (or the source stopped).  The handle must have calibration and matrix loaded;
 * the integrator state carries over from and to the per-frame calls.  One loop at
 * a time per handle.  Every device wait is bounded: a frame that is not published
 * within 2 s, or a grid barrier that does not complete within 200 ms, ends the
 * loop with RTC_ETIMEDOUT.  Errors: RTC_EINVAL, RTC_ESTATE, RTC_ENOMEM,
 * RTC_EDEVICE, RTC_ETIMEDOUT. */
int rtc_run_loop(rtc_handle* h, const rtc_loop_config* cfg, rtc_stats* stats);

/* ---- resident per-frame calls --------------------------------------------------
 * The same persistent kernel, driven one frame at a time by the caller's own
 * thread (a camera callback, say) instead of by a frame source: after
 * rtc_resident_start, each rtc_process_frame call on pinned (page-locked, mapped)
 * buffers publishes the frame and waits for its DM commands, with no kernel launch
 * per frame (the paper's continuously running RTC threads, Sec. 2.3.2).  The
 * kernel reads the frame from the caller's buffer and writes the commands into
 * the caller's dm_out; both must stay valid until the call returns, the frame
 * buffer must be 16-byte aligned and dm_out 4-byte aligned.  Results are those of
 * the per-frame launches bit for bit, the integrator (and predictor history) carry
 * over in both directions, and the learned predictor runs if it is on.
 *
 * While resident the kernel occupies every SM of the handle's device, spinning on
 * the next frame's flag.  If no frame comes for 2 s its bounded wait expires and
 * it exits; the next rtc_process_frame relaunches it transparently.  Other calls
 * on the handle that touch the device (loading maps or a matrix, the stage and
 * async calls, rtc_run_loop, a server slot, rtc_process_frame with pageable
 * buffers or slopes_out) return RTC_ESTATE until rtc_resident_stop; device
 * memory releases of any handle are queued until then (as during rtc_run_loop).
 * rtc_destroy stops a resident handle first.
 * Errors: RTC_EINVAL, RTC_ESTATE (not ready, in a server slot, already resident),
 * RTC_ENOMEM, RTC_EDEVICE. */
int rtc_resident_start(rtc_handle* h);

/* Stop the resident kernel (no-op if the handle is not resident).  Errors:
 * RTC_EINVAL, RTC_EDEVICE, RTC_ETIMEDOUT (a grid barrier of the kernel expired). */
int rtc_resident_stop(rtc_handle* h);

/* ---- serving several loops on one GPU (continuous batching) --------------------
 * A server runs independent controllers (handles, each with its own calibration,
 * matrix, integrator and predictor history) side by side on one device.  A job
 * is one handle plus a run of frames.  Jobs are admitted into slots while other
 * jobs are running, as long as a slot is free and the handle's device memory fits
 * in the server's budget; otherwise rtc_slot_submit returns RTC_EBUSY and the
 * caller retries once rtc_slot_poll has freed a slot.  Each admitted job gets its
 * own stream and a fixed share of the SMs (num_SMs / max_slots blocks per frame
 * kernel), so the work of different jobs overlaps on the device, and a job's
 * results do not depend on which other jobs run beside it. */

typedef struct rtc_server rtc_server;

/* Errors: RTC_EINVAL (max_slots < 1 or > 32, budget <= 0, device), RTC_ENOMEM. */
int rtc_server_create(int32_t device, int32_t max_slots, int64_t mem_budget_bytes, rtc_server** out);

/* Wait for running jobs, then release the server (not the handles).  Queued
 * like rtc_destroy while an rtc_run_loop is running. */
int rtc_server_destroy(rtc_server* s);

/* Admit a job: frames host uint16 [n_frames][n_wfs][H][W] (pinned memory keeps the
 * submission asynchronous), dm_out host float32 [n_frames][nact] receives each
 * frame's DM commands.  Both stay owned by the caller and must stay valid until
 * rtc_slot_poll reports the job done; meanwhile the handle's own calls (rtc_destroy
 * included) return RTC_ESTATE, since the job's kernels use its device state.
 * *slot receives the slot id.  Errors: RTC_EINVAL, RTC_ESTATE (handle not ready
 * or already in a slot, or on another device), RTC_EBUSY (no slot or not enough
 * memory budget now), RTC_EDEVICE. */
int rtc_slot_submit(rtc_server* s, rtc_handle* h, const uint16_t* frames, uint64_t n_frames,
                    float* dm_out, int32_t* slot);

/* RTC_OK when the job in `slot` is complete (its results are in dm_out and the slot
 * and its memory budget are free again), RTC_EBUSY while it runs.  frames_done (may
 * be NULL) receives the frames completed so far.  Errors: RTC_EINVAL,
 * RTC_ETIMEDOUT or RTC_EDEVICE (the job failed; the slot is freed). */
int rtc_slot_poll(rtc_server* s, int32_t slot, uint64_t* frames_done);

/* Jobs running and device bytes they account for. */
int rtc_server_info(const rtc_server* s, int32_t* active_slots, int64_t* mem_in_use);

/* ---- learned slope predictor --------------------------------------------------
 * An addition to the paper's pipeline: a shared MLP predicts each subaperture's
 * next slopes from its 5x5 neighbourhood over the last 4 frames, to offset the
 * integrator's one-frame servo lag.  Definition (both the kernels and the FP64
 * oracle follow it):
 *   features  x_f, f = ((lag*2 + axis)*5 + (dr+2))*5 + (dc+2), 200 values: the
 *             slope (axis 0 = x, 1 = y) of the neighbour at grid offset (dr, dc)
 *             in the frame `lag` frames ago (0 = newest), divided by sigma; 0 off
 *             the grid or off the pupil;
 *   network   z1 = W1 x + b1, h1 = GELU(z1), z2 = W2 h1 + b2, h2 = GELU(z2),
 *             y = W3 h2 + b3; 200 -> 64 -> 64 -> 2; exact GELU z*Phi(z);
 *   output    predicted next slopes = s_k + sigma * y;
 *   loss      sum over the batch of |y - t|^2 / (2B), t = (s_{k+1} - s_k) / sigma;
 *   update    Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 * Parameters are one float32 vector of RTC_MLP_NPARAMS values: W1 [64][200],
 * b1 [64], W2 [64][64], b2 [64], W3 [2][64], b3 [2], each row-major.  The GEMMs
 * run on the tensor cores with BF16 operands and FP32 accumulation; the master
 * weights and Adam state are FP32. */

#define RTC_MLP_NPARAMS 17154
#define RTC_MLP_NFEAT 200

typedef struct rtc_mlp rtc_mlp;

/* A network on `device` with all parameters zero.  Errors: RTC_EINVAL, RTC_ENOMEM. */
int rtc_mlp_create(int32_t device, rtc_mlp** out);
/* Release the network; queued like rtc_destroy while an rtc_run_loop is running. */
int rtc_mlp_destroy(rtc_mlp* m);

/* Host float32 [RTC_MLP_NPARAMS] in/out; setting resets the Adam state and step. */
int rtc_mlp_set_params(rtc_mlp* m, const float* params, int64_t n);
int rtc_mlp_get_params(rtc_mlp* m, float* params, int64_t n);

/* Subaperture geometry used by rtc_mlp_train_seq: host int32 [n_valid][2] (row,
 * col), row-major order, on an nsub x nsub grid.  Errors: RTC_EINVAL. */
int rtc_mlp_set_geometry(rtc_mlp* m, const int32_t* rc, int32_t n_valid, int32_t nsub);

/* y = net(X) for device X float32 [B][200] -> device Y float32 [B][2]. */
int rtc_mlp_forward(rtc_mlp* m, const float* d_X, int32_t B, float* d_Y, void* stream);

/* Gradient of the loss at the current parameters for the batch (X [B][200],
 * targets T [B][2], device): d_grad float32 [RTC_MLP_NPARAMS] (device), d_loss
 * float32 [1] (device, may be NULL).  No update. */
int rtc_mlp_gradient(rtc_mlp* m, const float* d_X, const float* d_T, int32_t B, float* d_grad,
                     float* d_loss, void* stream);

/* One Adam step with learning rate lr on the batch; d_loss (device, may be NULL)
 * receives the batch loss before the step. */
int rtc_mlp_train_step(rtc_mlp* m, const float* d_X, const float* d_T, int32_t B, float lr,
                       float* d_loss, void* stream);

/* One Adam step on samples drawn from a slope sequence: d_S device float32
 * [n_frames][2 n_valid] (x block then y block per frame), d_samples device int32
 * [B][2] of (subaperture, frame k) with 3 <= k <= n_frames - 2.  Features come
 * from frames k..k-3, targets from k+1.  Needs rtc_mlp_set_geometry. */
int rtc_mlp_train_seq(rtc_mlp* m, const float* d_S, int32_t n_frames, const int32_t* d_samples,
                      int32_t B, float sigma, float lr, float* d_loss, void* stream);

/* Predictions over a slope sequence (geometry from rtc_mlp_set_geometry): for
 * every frame k with 3 <= k <= n_frames - 2, row k + 1 of d_out (device float32
 * [n_frames][2 n_valid]) receives s_k + sigma * y from the features of frames
 * k..k-3 of d_S; other rows are not written. */
int rtc_mlp_predict_seq(rtc_mlp* m, const float* d_S, int32_t n_frames, float sigma, float* d_out,
                        void* stream);

/* Use a predictor in the per-frame path of a handle (SCAO only, n_wfs == 1, up to
 * 16384 slopes): params host float32 [RTC_MLP_NPARAMS], sigma the slope scale of
 * the features.  The handle keeps the last 4 measured slope vectors; with the
 * predictor on, the reconstruction uses the predicted next slopes
 * s_k + sigma * y instead of the measured ones, in rtc_process_frame(_async) and
 * in rtc_run_loop alike (the prediction runs inside the same kernel launch as the
 * rest of the frame), and slopes_out still receives the measured slopes.
 * rtc_reset clears the history.  Errors: RTC_EINVAL, RTC_ENOMEM, RTC_EDEVICE. */
int rtc_load_predictor(rtc_handle* h, const float* params, int64_t n, float sigma);
int rtc_set_predictor(rtc_handle* h, int32_t on);

/* Largest sizes rtc_mvm_integrate_noalloc accepts (its scratch is fixed at load). */
#define RTC_NOALLOC_MAX_NACT   8192
#define RTC_NOALLOC_MAX_KSPLIT 16

/* Reconstruction + leaky integrator (the work of rtc_reconstruct_async) for
 * callers that must not allocate device memory.  The paper has no counterpart:
 * this entry point exists for hosts such as a hard-real-time control thread,
 * which cannot afford the implicit device synchronisation and unbounded latency
 * of cudaMalloc inside its loop, or a plugin inside a larger RTC framework that
 * receives every device buffer from the framework and may not allocate its own.
 * It needs no handle and allocates nothing: the split-K scratch lives in a
 * static device array of about 520 KiB, held by every GPU that loads the library
 * until the process exits.
 *
 * Buffers (all device memory on the current device, owned by the caller):
 *   d_M          [nact][kpad] matrix in the stored type `store` (rtc_dtype),
 *                rows zero-padded, 16-byte aligned; kpad a multiple of 16;
 *   d_row_scales [nact] FP32 row scales (FP8 and INT8, else may be NULL);
 *   d_s          [kpad] FP32 slopes, zero-padded, 16-byte aligned;
 *   d_a          [nact] FP32 integrator state, updated in place:
 *                a <- leak * a + gain * (M s);
 *   d_dm_out     [nact] FP32 copy of the new state, or NULL.
 * nact must be in 1..RTC_NOALLOC_MAX_NACT and ksplit in 1..RTC_NOALLOC_MAX_KSPLIT;
 * larger sizes are rejected with RTC_EINVAL (message in rtc_last_error(NULL)).
 * The work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 * stream) without synchronising.
 *
 * The first call on a device looks up the scratch array's device address (this
 * may load the library's device code); make that first call before any stream
 * capture.  Every call on a device shares the one scratch array, which keeps the
 * last call's contents; each call clears the counters it needs before its kernel.
 * Calls whose work overlaps on the GPU (unordered streams) race on the scratch
 * and give wrong results: order them on one stream.
 * Errors: RTC_EINVAL, RTC_EDEVICE. */
int rtc_mvm_integrate_noalloc(const void* d_M, int32_t store, const float* d_row_scales,
                              int32_t nact, int32_t kpad, const float* d_s, float* d_a,
                              float* d_dm_out, float gain, float leak, int32_t ksplit,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RTC_H */
