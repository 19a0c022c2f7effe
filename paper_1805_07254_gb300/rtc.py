"""ctypes binding of librtc.so (include/rtc.h) -- argument marshalling only.

Every computation happens in the library's CUDA kernels; this module converts
numpy arrays / torch tensors to pointers, checks status codes and raises
``RtcError``.  If the library has not been built the import of ``Rtc`` fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librtc.so")

RTC_OK, RTC_EINVAL, RTC_ENOMEM, RTC_EDEVICE, RTC_ETIMEDOUT, RTC_ESTATE, RTC_EBUSY = 0, -1, -2, -3, -4, -5, -6
DTYPES = {"f32": 0, "bf16": 1, "fp8": 2, "f16": 3, "int8": 4}
_ERRNAMES = {0: "RTC_OK", -1: "RTC_EINVAL", -2: "RTC_ENOMEM", -3: "RTC_EDEVICE",
             -4: "RTC_ETIMEDOUT", -5: "RTC_ESTATE", -6: "RTC_EBUSY"}


class RtcConfig(C.Structure):
    _fields_ = [("nsub", C.c_int32), ("npx", C.c_int32), ("n_wfs", C.c_int32), ("nact", C.c_int32),
                ("obs", C.c_float), ("gain", C.c_float), ("leak", C.c_float),
                ("thr_mode", C.c_int32), ("thr", C.c_float), ("device", C.c_int32),
                ("reserved", C.c_int32)]


class RtcInfo(C.Structure):
    _fields_ = [("n_valid", C.c_int32), ("nslopes", C.c_int32), ("nact", C.c_int32),
                ("kpad", C.c_int32), ("store", C.c_int32), ("slices", C.c_int32),
                ("blocks", C.c_int32), ("tile_rows", C.c_int32), ("ring_stages", C.c_int32),
                ("matrix_bytes", C.c_int64), ("frame_bytes", C.c_int64), ("calib_bytes", C.c_int64)]


SOURCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_uint64, C.c_void_p)
SINK_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_uint64, C.POINTER(C.c_float))
LOOP_SLOTS = 8


class RtcLoopConfig(C.Structure):
    _fields_ = [("n_frames", C.c_uint64), ("rate_hz", C.c_double), ("source", SOURCE_FN),
                ("source_user", C.c_void_p), ("preload", C.c_void_p), ("n_preload", C.c_int32),
                ("sink", SINK_FN), ("sink_user", C.c_void_p), ("e2e_ns", C.c_void_p),
                ("dev_ns", C.c_void_p), ("n_bands", C.c_int32), ("band_interval_us", C.c_double),
                ("matrix_l2", C.c_int32)]


class RtcStats(C.Structure):
    _fields_ = [("frames", C.c_uint64), ("frames_per_s", C.c_double)] + [
        (f"{a}_{b}", C.c_double) for a in ("e2e", "dev")
        for b in ("p50_us", "p99_us", "p999_us", "mean_us", "rms_jitter_us", "p2p_us")]


_P = C.c_void_p
_I = C.c_int
# name -> (restype, argtypes); mirrors include/rtc.h
SIGNATURES = {
    "rtc_version": (C.c_char_p, []),
    "rtc_last_error": (C.c_char_p, [_P]),
    "rtc_create": (_I, [C.POINTER(RtcConfig), C.POINTER(_P)]),
    "rtc_destroy": (_I, [_P]),
    "rtc_load_subaps": (_I, [_P, _P, C.c_int32]),
    "rtc_load_calib": (_I, [_P, _P, _P, C.c_int64]),
    "rtc_set_threshold": (_I, [_P, C.c_int32, C.c_float]),
    "rtc_load_cmat": (_I, [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P]),
    "rtc_set_gain": (_I, [_P, C.c_float, C.c_float]),
    "rtc_set_readout": (_I, [_P, C.c_int32, C.c_double]),
    "rtc_plan_slices": (_I, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                             C.c_int32, C.c_int32, C.c_double, _P, _P]),
    "rtc_plan_ingest": (_I, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int32, C.c_int32,
                             C.c_int32, C.c_int32, _P, _P, C.c_int64, _P]),
    "rtc_reset": (_I, [_P]),
    "rtc_get_dm": (_I, [_P, _P]),
    "rtc_get_info": (_I, [_P, C.POINTER(RtcInfo)]),
    "rtc_process_frame": (_I, [_P, _P, _P, _P]),
    "rtc_process_frame_async": (_I, [_P, _P, _P, _P, _P]),
    "rtc_synchronize": (_I, [_P, _P]),
    "rtc_centroid_async": (_I, [_P, _P, _P, _P]),
    "rtc_reconstruct_async": (_I, [_P, _P, _P, _P]),
    "rtc_mvm_integrate_noalloc": (_I, [_P, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P, _P,
                                       C.c_float, C.c_float, C.c_int32, _P]),
    "rtc_run_loop": (_I, [_P, C.POINTER(RtcLoopConfig), C.POINTER(RtcStats)]),
    "rtc_resident_start": (_I, [_P]),
    "rtc_resident_stop": (_I, [_P]),
    "rtc_server_create": (_I, [C.c_int32, C.c_int32, C.c_int64, C.POINTER(_P)]),
    "rtc_server_destroy": (_I, [_P]),
    "rtc_slot_submit": (_I, [_P, _P, _P, C.c_uint64, _P, C.POINTER(C.c_int32)]),
    "rtc_slot_poll": (_I, [_P, C.c_int32, C.POINTER(C.c_uint64)]),
    "rtc_server_info": (_I, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "rtc_mlp_create": (_I, [C.c_int32, C.POINTER(_P)]),
    "rtc_mlp_destroy": (_I, [_P]),
    "rtc_mlp_set_params": (_I, [_P, _P, C.c_int64]),
    "rtc_mlp_get_params": (_I, [_P, _P, C.c_int64]),
    "rtc_mlp_set_geometry": (_I, [_P, _P, C.c_int32, C.c_int32]),
    "rtc_mlp_forward": (_I, [_P, _P, C.c_int32, _P, _P]),
    "rtc_mlp_gradient": (_I, [_P, _P, _P, C.c_int32, _P, _P, _P]),
    "rtc_mlp_train_step": (_I, [_P, _P, _P, C.c_int32, C.c_float, _P, _P]),
    "rtc_mlp_train_seq": (_I, [_P, _P, C.c_int32, _P, C.c_int32, C.c_float, C.c_float, _P, _P]),
    "rtc_mlp_predict_seq": (_I, [_P, _P, C.c_int32, C.c_float, _P, _P]),
    "rtc_load_predictor": (_I, [_P, _P, C.c_int64, C.c_float]),
    "rtc_set_predictor": (_I, [_P, C.c_int32]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load librtc.so and declare its signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librtc.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RtcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to librtc must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to librtc must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot pass {type(x)} to librtc")


# cudaStreamLegacy: the legacy default stream as an explicit handle.  A torch stream
# object whose handle is 0 (torch's default stream) is passed as this, because a
# NULL stream means "the handle's own stream" to the library.
_CUDA_STREAM_LEGACY = 1


def _stream_ptr(stream):
    """cudaStream_t for a torch stream, a raw handle, or None (the library default)."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or _CUDA_STREAM_LEGACY
    return int(stream)


class Rtc:
    """One real-time-controller instance on one GPU (a librtc handle)."""

    def __init__(self, nsub: int, npx: int, nact: int, n_wfs: int = 1, obs: float = 0.0,
                 gain: float = 0.4, leak: float = 0.99, thr_mode: int = 0, thr: float = 0.0,
                 device: int = 0):
        self._lib = load_library()
        cfg = RtcConfig(nsub, npx, n_wfs, nact, obs, gain, leak, thr_mode, thr, device, 0)
        h = _P()
        rc = self._lib.rtc_create(C.byref(cfg), C.byref(h))
        if rc != RTC_OK:
            raise RtcError(rc, self._lib.rtc_last_error(None).decode())
        self._h = h
        self.cfg = cfg

    # -- helpers ---------------------------------------------------------------
    def _check(self, rc: int):
        if rc != RTC_OK:
            raise RtcError(rc, self._lib.rtc_last_error(self._h).decode())

    def close(self):
        """Release the handle (rtc_destroy); raises RtcError (RTC_ESTATE) while its job is
        in a server slot, keeping the handle."""
        if getattr(self, "_h", None):
            rc = self._lib.rtc_destroy(self._h)
            if rc == RTC_ESTATE:
                raise RtcError(rc, self._lib.rtc_last_error(self._h).decode())
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- loading -------------------------------------------------------------------
    def info(self) -> dict:
        inf = RtcInfo()
        self._check(self._lib.rtc_get_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in RtcInfo._fields_}

    def load_subaps(self, rc):
        rc = np.ascontiguousarray(rc, dtype=np.int32).reshape(-1, 2)
        self._check(self._lib.rtc_load_subaps(self._h, _ptr(rc), rc.shape[0]))

    def load_calib(self, dark, flat):
        d = np.ascontiguousarray(dark, dtype=np.float32)
        f = np.ascontiguousarray(flat, dtype=np.float32)
        if d.size != f.size:
            raise ValueError("dark and flat must have the same size")
        self._check(self._lib.rtc_load_calib(self._h, _ptr(d), _ptr(f), d.size))

    def set_threshold(self, mode: int, thr: float):
        self._check(self._lib.rtc_set_threshold(self._h, mode, thr))

    def load_cmat(self, M, store: str = "f32", src: str = "f32", row_scales=None):
        if src == "f32":
            m = np.ascontiguousarray(M, dtype=np.float32)
        elif src == "bf16":
            m = np.ascontiguousarray(M, dtype=np.uint16)
        elif src == "f16":
            m = np.ascontiguousarray(M, dtype=np.float16)
        elif src == "fp8":
            m = np.ascontiguousarray(M, dtype=np.uint8)
        elif src == "int8":
            m = np.ascontiguousarray(M, dtype=np.int8)
        else:
            raise ValueError(src)
        sc = None if row_scales is None else np.ascontiguousarray(row_scales, dtype=np.float32)
        self._check(self._lib.rtc_load_cmat(self._h, _ptr(m), m.shape[0], m.shape[1],
                                            DTYPES[src], DTYPES[store], _ptr(sc)))

    def set_gain(self, gain: float, leak: float):
        self._check(self._lib.rtc_set_gain(self._h, gain, leak))

    def set_readout(self, bands: int, band_interval_us: float = 0.0):
        """Asymmetric subaperture allocation for a rolling readout of `bands` bands of
        pixel rows, band_interval_us apart (rtc_set_readout); bands = 0 restores
        equal slices."""
        self._check(self._lib.rtc_set_readout(self._h, int(bands), float(band_interval_us)))

    def reset(self):
        self._check(self._lib.rtc_reset(self._h))

    def get_dm(self) -> np.ndarray:
        out = np.empty(self.cfg.nact, np.float32)
        self._check(self._lib.rtc_get_dm(self._h, _ptr(out)))
        return out

    # -- per frame -----------------------------------------------------------------
    def resident_start(self):
        """Keep the persistent kernel resident: process_frame on pinned buffers then
        hands each frame to it without a launch (rtc_resident_start)."""
        self._check(self._lib.rtc_resident_start(self._h))

    def resident_stop(self):
        self._check(self._lib.rtc_resident_stop(self._h))

    def process_frame(self, frame, dm_out=None, slopes_out=None, want_slopes: bool = False):
        """One synchronous step with host buffers.  ``frame`` is a uint16 numpy array or a
        (pinned) CPU tensor; returns dm (and slopes if requested)."""
        if isinstance(frame, np.ndarray):
            frame = np.ascontiguousarray(frame, dtype=np.uint16)
        inf = None
        if dm_out is None:
            dm_out = np.empty(self.cfg.nact, np.float32)
        if want_slopes and slopes_out is None:
            inf = inf or self.info()
            slopes_out = np.empty(inf["nslopes"], np.float32)
        self._check(self._lib.rtc_process_frame(self._h, _ptr(frame), _ptr(dm_out), _ptr(slopes_out)))
        return (dm_out, slopes_out) if (want_slopes or slopes_out is not None) else dm_out

    def process_frame_async(self, d_frame, d_dm_out=None, d_slopes_out=None, stream=None):
        """Enqueue one step on device buffers (torch CUDA tensors) on ``stream``."""
        self._check(self._lib.rtc_process_frame_async(self._h, _ptr(d_frame), _ptr(d_dm_out),
                                                      _ptr(d_slopes_out), _stream_ptr(stream)))

    def centroid_async(self, d_frame, d_slopes_out=None, stream=None):
        """Enqueue the pixel stage (calibration + centroids) on device buffers."""
        self._check(self._lib.rtc_centroid_async(self._h, _ptr(d_frame), _ptr(d_slopes_out),
                                                 _stream_ptr(stream)))

    def reconstruct_async(self, d_slopes=None, d_dm_out=None, stream=None):
        """Enqueue MVM + integrator from ``d_slopes`` (None: the resident slope buffer)."""
        self._check(self._lib.rtc_reconstruct_async(self._h, _ptr(d_slopes), _ptr(d_dm_out),
                                                    _stream_ptr(stream)))

    def run_loop(self, n_frames: int, rate_hz: float = 0.0, frames=None, source=None, sink=None,
                 record: bool = True, bands: int = 0, band_interval_us: float = 0.0,
                 matrix_l2: int = 0):
        """Persistent real-time loop (rtc_run_loop).

        frames: uint16 array (n, [n_wfs,] H, W), 1 <= n <= 8, cycled; or source(k) -> frame
        array for frame k (None stops the loop).  sink(k, dm) receives each frame's DM
        commands (a float32 array valid during the call).  bands > 1 publishes each
        frame in that many bands of pixel rows, band_interval_us apart (a rolling
        readout).  matrix_l2=1 streams the matrix with L2 evict_first whatever its size.
        Returns (stats dict, e2e_ns, dev_ns) with per-frame latencies when record is
        true."""
        n_frames = int(n_frames)
        cfg = RtcLoopConfig()
        cfg.n_frames = n_frames
        cfg.rate_hz = float(rate_hz)
        cfg.n_bands = int(bands)
        cfg.band_interval_us = float(band_interval_us)
        cfg.matrix_l2 = int(matrix_l2)
        keep = []
        if source is not None:
            nbytes = [None]

            def _src(user, k, dst):
                try:
                    f = source(int(k))
                    if f is None:
                        return 1
                    f = np.ascontiguousarray(f, dtype=np.uint16)
                    C.memmove(dst, f.ctypes.data, f.nbytes)
                    return 0
                except Exception:          # a failing source ends the loop
                    return 1
            cfg.source = SOURCE_FN(_src)
            keep.append(cfg.source)
        else:
            if frames is None:
                raise ValueError("give frames or a source")
            fr = np.ascontiguousarray(frames, dtype=np.uint16)
            cfg.preload = fr.ctypes.data
            cfg.n_preload = fr.shape[0]
            keep.append(fr)
        if sink is not None:
            nact = self.cfg.nact

            def _sink(user, k, dm):
                sink(int(k), np.ctypeslib.as_array(dm, shape=(nact,)).copy())
            cfg.sink = SINK_FN(_sink)
            keep.append(cfg.sink)
        e2e = dev = None
        if record:
            e2e = np.zeros(n_frames, np.int64)
            dev = np.zeros(n_frames, np.int64)
            cfg.e2e_ns = e2e.ctypes.data
            cfg.dev_ns = dev.ctypes.data
        st = RtcStats()
        rc = self._lib.rtc_run_loop(self._h, C.byref(cfg), C.byref(st))
        stats = {k: getattr(st, k) for k, _ in RtcStats._fields_}
        if rc != RTC_OK:
            err = RtcError(rc, self._lib.rtc_last_error(self._h).decode())
            err.stats = stats
            raise err
        n = int(st.frames)
        return stats, (e2e[:n] if record else None), (dev[:n] if record else None)

    def load_predictor(self, params, sigma: float):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        self._check(self._lib.rtc_load_predictor(self._h, _ptr(p), p.size, sigma))

    def set_predictor(self, on: bool):
        self._check(self._lib.rtc_set_predictor(self._h, 1 if on else 0))

    def synchronize(self, stream=None):
        self._check(self._lib.rtc_synchronize(self._h, _stream_ptr(stream)))


def mvm_integrate_noalloc(d_M, store: str, d_row_scales, nact: int, kpad: int, d_s, d_a,
                          d_dm_out=None, gain: float = 0.4, leak: float = 0.99, ksplit: int = 1,
                          stream=None):
    """Reconstruction + integrator on caller-owned device buffers, with no device
    allocation by the library (see rtc_mvm_integrate_noalloc in include/rtc.h)."""
    lib = load_library()
    rc = lib.rtc_mvm_integrate_noalloc(_ptr(d_M), DTYPES[store], _ptr(d_row_scales), nact, kpad,
                                       _ptr(d_s), _ptr(d_a), _ptr(d_dm_out), gain, leak, ksplit,
                                       _stream_ptr(stream))
    if rc != RTC_OK:
        raise RtcError(rc, lib.rtc_last_error(None).decode())


class Server:
    """Several controllers served side by side on one GPU (rtc_server_* / rtc_slot_*)."""

    def __init__(self, device: int = 0, max_slots: int = 4, mem_budget: int = 1 << 36):
        self._lib = load_library()
        h = _P()
        rc = self._lib.rtc_server_create(device, max_slots, mem_budget, C.byref(h))
        if rc != RTC_OK:
            raise RtcError(rc, self._lib.rtc_last_error(None).decode())
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rtc_server_destroy(self._h)
            self._h = None
            self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, rtc: "Rtc", frames) -> int:
        """Admit a job; returns its slot.  Raises RtcError (code RTC_EBUSY) when no slot
        or memory budget is free now.  Results: see result(slot)."""
        import torch
        fr = torch.from_numpy(np.ascontiguousarray(frames, dtype=np.uint16)).pin_memory()
        n = fr.shape[0]
        dm = torch.empty((n, rtc.cfg.nact), dtype=torch.float32).pin_memory()
        slot = C.c_int32(-1)
        rc = self._lib.rtc_slot_submit(self._h, rtc.handle, _ptr(fr), n, _ptr(dm), C.byref(slot))
        if rc != RTC_OK:
            raise RtcError(rc, self._lib.rtc_last_error(None).decode())
        self._keep[slot.value] = (fr, dm)
        return slot.value

    def poll(self, slot: int):
        """(done, frames_done); raises RtcError if the job failed."""
        done = C.c_uint64(0)
        rc = self._lib.rtc_slot_poll(self._h, slot, C.byref(done))
        if rc == RTC_EBUSY:
            return False, done.value
        if rc != RTC_OK:
            raise RtcError(rc, self._lib.rtc_last_error(None).decode())
        return True, done.value

    def wait(self, slot: int, timeout_s: float = 120.0) -> np.ndarray:
        """Block until the job in `slot` is done; returns its DM commands [n_frames][nact]."""
        import time
        t0 = time.time()
        while True:
            done, _ = self.poll(slot)
            if done:
                return self._keep.pop(slot)[1].numpy().copy()
            if time.time() - t0 > timeout_s:
                raise TimeoutError(f"slot {slot} not done after {timeout_s} s")
            time.sleep(0.0005)

    def info(self):
        a = C.c_int32(0)
        b = C.c_int64(0)
        self._lib.rtc_server_info(self._h, C.byref(a), C.byref(b))
        return {"active_slots": a.value, "mem_in_use": b.value}


MLP_NPARAMS = 17154


class Mlp:
    """The slope-predictor network (rtc_mlp_*): training and evaluation on device tensors."""

    def __init__(self, device: int = 0, params=None):
        self._lib = load_library()
        h = _P()
        self._check(self._lib.rtc_mlp_create(device, C.byref(h)))
        self._h = h
        if params is not None:
            self.set_params(params)

    def _check(self, rc):
        if rc != RTC_OK:
            raise RtcError(rc, self._lib.rtc_last_error(None).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rtc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        self._check(self._lib.rtc_mlp_set_params(self._h, _ptr(p), p.size))

    def get_params(self) -> np.ndarray:
        out = np.empty(MLP_NPARAMS, np.float32)
        self._check(self._lib.rtc_mlp_get_params(self._h, _ptr(out), out.size))
        return out

    def set_geometry(self, rc, nsub: int):
        rc = np.ascontiguousarray(rc, dtype=np.int32).reshape(-1, 2)
        self._check(self._lib.rtc_mlp_set_geometry(self._h, _ptr(rc), rc.shape[0], nsub))

    def forward(self, d_X, d_Y, stream=None):
        self._check(self._lib.rtc_mlp_forward(self._h, _ptr(d_X), d_X.shape[0], _ptr(d_Y),
                                              _stream_ptr(stream)))

    def gradient(self, d_X, d_T, d_grad, d_loss=None, stream=None):
        self._check(self._lib.rtc_mlp_gradient(self._h, _ptr(d_X), _ptr(d_T), d_X.shape[0],
                                               _ptr(d_grad), _ptr(d_loss), _stream_ptr(stream)))

    def train_step(self, d_X, d_T, lr: float, d_loss=None, stream=None):
        self._check(self._lib.rtc_mlp_train_step(self._h, _ptr(d_X), _ptr(d_T), d_X.shape[0], lr,
                                                 _ptr(d_loss), _stream_ptr(stream)))

    def train_seq(self, d_S, d_samples, sigma: float, lr: float, d_loss=None, stream=None):
        self._check(self._lib.rtc_mlp_train_seq(self._h, _ptr(d_S), d_S.shape[0], _ptr(d_samples),
                                                d_samples.shape[0], sigma, lr, _ptr(d_loss),
                                                _stream_ptr(stream)))

    def predict_seq(self, d_S, sigma: float, d_out, stream=None):
        self._check(self._lib.rtc_mlp_predict_seq(self._h, _ptr(d_S), d_S.shape[0], sigma,
                                                  _ptr(d_out), _stream_ptr(stream)))


def version() -> str:
    return load_library().rtc_version().decode()


def plan_slices(rc, nsub: int, npx: int, nact: int, store: str = "f32", max_slices: int = 152,
                bands: int = 0, band_interval_us: float = 0.0, n_wfs: int = 1) -> np.ndarray:
    """The slice cut (rtc_plan_slices): first subaperture of each slice, then the
    subaperture count.  Host only."""
    lib = load_library()
    rc = np.ascontiguousarray(rc, dtype=np.int32).reshape(-1, 2)
    g0 = np.zeros(max_slices + 1, np.int32)
    n = C.c_int32(0)
    rc_ = lib.rtc_plan_slices(_ptr(rc), rc.shape[0], n_wfs, nsub, npx, nact, DTYPES[store], max_slices,
                              int(bands), float(band_interval_us), _ptr(g0), C.byref(n))
    if rc_ != RTC_OK:
        raise RtcError(rc_, "rtc_plan_slices rejected its arguments")
    return g0[:n.value + 1].copy()


def plan_ingest(rc, nsub: int, npx: int, g0, blocks: int, unit_bytes: int = 16, bands: int = 1,
                n_wfs: int = 1):
    """The persistent loop's ingest table (rtc_plan_ingest): (blk [blocks][4] int32,
    units uint32).  Host only."""
    lib = load_library()
    rc = np.ascontiguousarray(rc, dtype=np.int32).reshape(-1, 2)
    g0 = np.ascontiguousarray(g0, dtype=np.int32)
    blk = np.zeros((blocks, 4), np.int32)
    n = C.c_int64(0)
    args = (_ptr(rc), rc.shape[0], n_wfs, nsub, npx, _ptr(g0), g0.shape[0] - 1, blocks, unit_bytes, int(bands),
            _ptr(blk))
    rc_ = lib.rtc_plan_ingest(*args, None, 0, C.byref(n))
    if rc_ != RTC_OK:
        raise RtcError(rc_, "rtc_plan_ingest rejected its arguments")
    units = np.zeros(max(n.value, 1), np.uint32)
    rc_ = lib.rtc_plan_ingest(*args, _ptr(units), units.shape[0], C.byref(n))
    if rc_ != RTC_OK:
        raise RtcError(rc_, "rtc_plan_ingest rejected its arguments")
    return blk, units[:n.value]
