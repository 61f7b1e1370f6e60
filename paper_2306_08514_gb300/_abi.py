"""ctypes binding of libsrp (include/libsrp.h): the same entry points under the same
names, plus a thin ``Plan`` wrapper that allocates outputs with PyTorch and passes raw
pointers and the current CUDA stream.  Argument marshalling only: every step of the SRP
path runs in libsrp's CUDA kernels, and importing this module fails loudly when the
library has not been built."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsrp.so")

SRP_OK, SRP_EINVAL, SRP_ENOMEM, SRP_ECUDA, SRP_ETIMEOUT, SRP_EUNSUPPORTED, SRP_EAGAIN = 0, 1, 2, 3, 4, 5, 6
SRP_CONV, SRP_SLRI, SRP_SSPI, SRP_SI, SRP_TD, SRP_LR = 0, 1, 2, 3, 4, 5
SRP_FP32, SRP_BF16, SRP_FP16, SRP_BF16X3, SRP_FP16X3, SRP_TF32X3, SRP_TF32 = 0, 1, 2, 3, 4, 5, 6
SRP_WIN_HANN, SRP_WIN_SQRT_HANN, SRP_WIN_RECT = 0, 1, 2

METHODS = {"conv": SRP_CONV, "slri": SRP_SLRI, "sspi": SRP_SSPI, "si": SRP_SI, "td": SRP_TD,
           "lr": SRP_LR}
PRECISIONS = {"fp32": SRP_FP32, "bf16": SRP_BF16, "fp16": SRP_FP16, "bf16x3": SRP_BF16X3,
              "fp16x3": SRP_FP16X3, "tf32x3": SRP_TF32X3, "tf32": SRP_TF32}
WINDOWS = {"hann": SRP_WIN_HANN, "sqrt-hann": SRP_WIN_SQRT_HANN, "rect": SRP_WIN_RECT}


class srp_plan_desc(C.Structure):
    _fields_ = [
        ("M", C.c_int), ("mic_xyz", C.POINTER(C.c_double)),
        ("J", C.c_int), ("grid_xyz", C.POINTER(C.c_double)),
        ("fs", C.c_double), ("N", C.c_int), ("window", C.c_int), ("c", C.c_double),
        ("n_aux", C.c_int), ("method", C.c_int), ("rank", C.c_int),
        ("taps_per_loc_pair", C.c_double), ("precision", C.c_int), ("max_frames", C.c_int),
        ("far_field", C.c_int), ("h_on_the_fly", C.c_int),
    ]


class srp_plan_info_t(C.Structure):
    _fields_ = [
        ("M", C.c_int), ("P", C.c_int), ("J", C.c_int), ("N", C.c_int), ("K", C.c_int),
        ("L", C.c_int), ("rank", C.c_int), ("nnz", C.c_longlong), ("tied_at_cut", C.c_longlong),
        ("device_bytes", C.c_size_t), ("fit_seconds", C.c_double), ("launches", C.c_longlong),
    ]


class srp_server_desc(C.Structure):
    _fields_ = [
        ("hbm_budget", C.c_size_t), ("max_sessions", C.c_int), ("max_batch", C.c_int),
        ("streams", C.c_int), ("slots_per_session", C.c_int), ("pending_frames", C.c_int),
        ("use_graphs", C.c_int), ("group_launches", C.c_int),
    ]


class srp_server_stats_t(C.Structure):
    _fields_ = [
        ("frames_done", C.c_longlong), ("frames_launched", C.c_longlong),
        ("launches", C.c_longlong), ("graph_launches", C.c_longlong),
        ("device_bytes", C.c_size_t), ("sessions_active", C.c_int), ("sessions_queued", C.c_int),
        ("latency_p50_s", C.c_double), ("latency_p99_s", C.c_double), ("latency_max_s", C.c_double),
        ("group_launches", C.c_longlong), ("group_frames", C.c_longlong),
        ("group_sessions", C.c_longlong),
    ]


SESSION_STATES = {0: "queued", 1: "active", 2: "closing", 3: "closed", 4: "failed"}


class srp_tune_report_t(C.Structure):
    _fields_ = [("variant", C.c_int), ("ms", C.c_float * 12)]


_TUNE_BASE = {0: "128x256 4-stage", 1: "128x256 2-stage 4-box", 2: "128x128 4-stage",
              3: "128x256 hi+lo per stage"}
# variants 4..7 / 8..11: variants 0..3 in clusters of 2 CTAs sharing the B tiles / of 2 x 2
# sharing the B and the A tiles
TUNE_VARIANTS = {-1: "fp32", **_TUNE_BASE, **{v + 4: name + " cluster 2" for v, name in _TUNE_BASE.items()},
                 **{v + 8: name + " cluster 2x2" for v, name in _TUNE_BASE.items()}}

# every symbol include/libsrp.h declares, with (restype, argtypes)
SIGNATURES = {
    "srp_plan_create": (C.c_int, [C.POINTER(srp_plan_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "srp_plan_info": (C.c_int, [C.c_void_p, C.POINTER(srp_plan_info_t)]),
    "srp_plan_lags": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "srp_map": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "srp_map_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "srp_map_peaks": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double,
                                C.c_void_p, C.c_void_p, C.c_void_p]),
    "srp_gcc_samples": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "srp_plan_sspi_taps": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                     C.POINTER(C.c_float)]),
    "srp_plan_slri_sigma": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int]),
    "srp_plan_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "srp_plan_stage_ms": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_int)]),
    "srp_plan_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "srp_debug_fail_allocations": (C.c_int, [C.c_int, C.c_int]),
    "srp_plan_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "srp_plan_create_from_file": (C.c_int, [C.POINTER(srp_plan_desc), C.c_char_p, C.c_void_p,
                                            C.POINTER(C.c_void_p)]),
    "srp_debug_stall_next_contraction": (C.c_int, [C.c_void_p]),
    "srp_slri_apply_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                        C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "srp_stream_push": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "srp_stream_reset": (C.c_int, [C.c_void_p]),
    "srp_plan_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(srp_tune_report_t)]),
    "srp_plan_set_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "srp_plan_estimate_bytes": (C.c_int, [C.POINTER(srp_plan_desc), C.POINTER(C.c_size_t)]),
    "srp_server_create": (C.c_int, [C.POINTER(srp_server_desc), C.POINTER(C.c_void_p)]),
    "srp_server_open": (C.c_int, [C.c_void_p, C.POINTER(srp_plan_desc), C.c_int, C.POINTER(C.c_int)]),
    "srp_server_push": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double]),
    "srp_server_poll": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.POINTER(C.c_int)]),
    "srp_server_session_info": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                          C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "srp_server_close": (C.c_int, [C.c_void_p, C.c_int]),
    "srp_server_stats": (C.c_int, [C.c_void_p, C.POINTER(srp_server_stats_t)]),
    "srp_server_reset_stats": (C.c_int, [C.c_void_p]),
    "srp_server_now": (C.c_double, []),
    "srp_server_destroy": (None, [C.c_void_p]),
    "srp_destroy": (None, [C.c_void_p]),
    "srp_last_error": (C.c_char_p, []),
}

_lib = None


def lib():
    """Load libsrp.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsrp.so not built at {LIB_PATH}: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SrpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libsrp status {status}: {msg}")
        self.status = status


def _check(st):
    if st != SRP_OK:
        raise SrpError(st, lib().srp_last_error().decode())


# ---- the C entry points under their own names -------------------------------------
def srp_last_error() -> str:
    return lib().srp_last_error().decode()


def srp_plan_create(desc: srp_plan_desc, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().srp_plan_create(C.byref(desc), stream, C.byref(h)))
    return h


def srp_plan_create_from_file(desc: srp_plan_desc, path, stream=None) -> C.c_void_p:
    """srp_plan_create with the method's fit read from a file written by srp_plan_save."""
    h = C.c_void_p()
    _check(lib().srp_plan_create_from_file(C.byref(desc), os.fsencode(path), stream, C.byref(h)))
    return h


def srp_plan_save(plan, path) -> None:
    _check(lib().srp_plan_save(plan, os.fsencode(path)))


def srp_plan_info(plan) -> srp_plan_info_t:
    info = srp_plan_info_t()
    _check(lib().srp_plan_info(plan, C.byref(info)))
    return info


def srp_plan_lags(plan, P: int) -> np.ndarray:
    out = (C.c_int * P)()
    _check(lib().srp_plan_lags(plan, out))
    return np.array(out[:], dtype=np.int64)


def srp_map(plan, frames_ptr, F, maps_ptr, argmax_ptr, stream) -> None:
    _check(lib().srp_map(plan, frames_ptr, F, maps_ptr, argmax_ptr, stream))


def srp_map_peaks(plan, frames_ptr, F, maps_ptr, K, d_min, peaks_ptr, values_ptr, stream) -> None:
    _check(lib().srp_map_peaks(plan, frames_ptr, F, maps_ptr, int(K), float(d_min), peaks_ptr,
                               values_ptr, stream))


def srp_map_host(plan, frames_ptr, F, maps_ptr, argmax_ptr, stream) -> None:
    _check(lib().srp_map_host(plan, frames_ptr, F, maps_ptr, argmax_ptr, stream))


def srp_gcc_samples(plan, frames_ptr, F, xi_ptr, stream) -> None:
    _check(lib().srp_gcc_samples(plan, frames_ptr, F, xi_ptr, stream))


def srp_plan_sspi_taps(plan, J: int, nnz: int):
    row_ptr = np.zeros(J + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.float32)
    _check(lib().srp_plan_sspi_taps(plan, row_ptr.ctypes.data_as(C.POINTER(C.c_longlong)),
                                    col.ctypes.data_as(C.POINTER(C.c_int)),
                                    val.ctypes.data_as(C.POINTER(C.c_float))))
    return row_ptr, col, val


def srp_plan_slri_sigma(plan, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _check(lib().srp_plan_slri_sigma(plan, out.ctypes.data_as(C.POINTER(C.c_double)), n))
    return out


SRP_NSTAGES = 4
STAGES = ("frontend", "spectra", "contract", "argmax")


def srp_plan_set_profiling(plan, enable: bool) -> None:
    _check(lib().srp_plan_set_profiling(plan, 1 if enable else 0))


def srp_plan_stage_ms(plan) -> dict:
    """Summed milliseconds per stage since profiling was enabled, plus 'chunks'."""
    out = (C.c_float * SRP_NSTAGES)()
    n = C.c_int(0)
    _check(lib().srp_plan_stage_ms(plan, out, C.byref(n)))
    d = dict(zip(STAGES, [float(v) for v in out]))
    d["chunks"] = int(n.value)
    return d


def srp_plan_status(plan, stream=None) -> None:
    """Raise SrpError(SRP_ETIMEOUT) if a bounded wait in one of the plan's kernels ran out."""
    _check(lib().srp_plan_status(plan, stream))


def srp_debug_fail_allocations(after, n) -> None:
    """Failure-detection test hook: the next n device allocations of libsrp fail (as out of
    memory) after `after` more succeed; n = 0 clears."""
    _check(lib().srp_debug_fail_allocations(int(after), int(n)))


def srp_slri_apply_static(xi_ptr, fat_ptr, tall_ptr, F, L, R, J, maps_ptr, argmax_ptr,
                          stream) -> None:
    """Allocation-free SLRI interpolation (pointers are device addresses)."""
    _check(lib().srp_slri_apply_static(xi_ptr, fat_ptr, tall_ptr, F, L, R, J, maps_ptr,
                                       argmax_ptr, stream))


def srp_destroy(plan) -> None:
    lib().srp_destroy(plan)


# ---- convenience wrapper ----------------------------------------------------------
def make_desc(mic_xyz, grid_xyz, fs, N, method="conv", rank=0, taps=0.0, precision="fp32",
              window="hann", c=340.0, n_aux=2, max_frames=256, far_field=False,
              h_on_the_fly=0):
    mic = np.ascontiguousarray(mic_xyz, dtype=np.float64)
    grid = np.ascontiguousarray(grid_xyz, dtype=np.float64)
    d = srp_plan_desc()
    d.M = mic.shape[0]
    d.mic_xyz = mic.ctypes.data_as(C.POINTER(C.c_double))
    d.J = grid.shape[0]
    d.grid_xyz = grid.ctypes.data_as(C.POINTER(C.c_double))
    d.fs, d.N, d.window, d.c, d.n_aux = float(fs), int(N), WINDOWS[window], float(c), int(n_aux)
    d.method = METHODS[method] if isinstance(method, str) else int(method)
    d.rank, d.taps_per_loc_pair = int(rank), float(taps)
    d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    d.max_frames = int(max_frames)
    d.far_field = 1 if far_field else 0
    d.h_on_the_fly = int(h_on_the_fly)
    d._keep = (mic, grid)  # keep the arrays alive while the struct is used
    return d


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Plan:
    """An SRP plan on the current CUDA device.  Outputs are torch CUDA tensors."""

    def __init__(self, mic_xyz, grid_xyz, fs, N, method="conv", rank=0, taps=0.0,
                 precision="fp32", window="hann", c=340.0, n_aux=2, max_frames=256,
                 stream=None, far_field=False, h_on_the_fly=0, plan_file=None):
        """plan_file: create from a file written by save() (the fit is read, not computed)."""
        self.desc = make_desc(mic_xyz, grid_xyz, fs, N, method, rank, taps, precision, window,
                              c, n_aux, max_frames, far_field, h_on_the_fly)
        if plan_file is None:
            self.handle = srp_plan_create(self.desc, _stream_handle(stream))
        else:
            self.handle = srp_plan_create_from_file(self.desc, plan_file, _stream_handle(stream))
        self.info = srp_plan_info(self.handle)
        self.M, self.J, self.N, self.L, self.P = (self.info.M, self.info.J, self.info.N,
                                                  self.info.L, self.info.P)

    def map(self, frames, maps=None, argmax=None, stream=None, want_argmax=True,
            want_maps=True):
        """want_maps=False: estimates only (argmax, no map written; srp_map with maps NULL)."""
        import torch
        assert frames.is_cuda and frames.dtype == torch.float32 and frames.is_contiguous()
        F = frames.shape[0]
        if maps is None and want_maps:
            maps = torch.empty((F, self.J), dtype=torch.float32, device=frames.device)
        if argmax is None and (want_argmax or not want_maps):
            argmax = torch.empty((F,), dtype=torch.int32, device=frames.device)
        srp_map(self.handle, C.c_void_p(frames.data_ptr()), F,
                C.c_void_p(maps.data_ptr()) if maps is not None else None,
                C.c_void_p(argmax.data_ptr()) if argmax is not None else None,
                _stream_handle(stream))
        return maps, argmax

    def peaks(self, frames, K, d_min, maps=None, want_maps=True, stream=None):
        """Several estimates per frame (srp_map_peaks): returns (peaks [F][K] int32, values
        [F][K] float32, maps [F][J] or None).  want_maps=False: estimates only."""
        import torch
        assert frames.is_cuda and frames.dtype == torch.float32 and frames.is_contiguous()
        F = frames.shape[0]
        if maps is None and want_maps:
            maps = torch.empty((F, self.J), dtype=torch.float32, device=frames.device)
        peaks = torch.empty((F, K), dtype=torch.int32, device=frames.device)
        values = torch.empty((F, K), dtype=torch.float32, device=frames.device)
        srp_map_peaks(self.handle, C.c_void_p(frames.data_ptr()), F,
                      C.c_void_p(maps.data_ptr()) if maps is not None else None, K, d_min,
                      C.c_void_p(peaks.data_ptr()), C.c_void_p(values.data_ptr()),
                      _stream_handle(stream))
        return peaks, values, maps

    def map_host(self, frames, maps=None, argmax=None, stream=None):
        """frames, maps, argmax: host arrays (numpy or pinned CPU tensors)."""
        F = frames.shape[0]

        def ptr(a):
            return C.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)

        if maps is None:
            maps = np.empty((F, self.J), dtype=np.float32)
        if argmax is None:
            argmax = np.empty((F,), dtype=np.int32)
        srp_map_host(self.handle, ptr(frames), F, ptr(maps), ptr(argmax), _stream_handle(stream))
        return maps, argmax

    def autotune(self, F=None, stream=None):
        """srp_plan_autotune: time the tensor-core variants at F frames, keep the fastest.
        Returns {"variant": name, "ms": {name: ms}}."""
        rep = srp_tune_report_t()
        F = int(F or self.desc.max_frames)
        _check(lib().srp_plan_autotune(self.handle, F, _stream_handle(stream), C.byref(rep)))
        return {"variant": TUNE_VARIANTS.get(rep.variant, rep.variant),
                "ms": {TUNE_VARIANTS[v]: rep.ms[v] for v in range(12) if rep.ms[v] >= 0}}

    def set_variant(self, variant):
        _check(lib().srp_plan_set_variant(self.handle, int(variant)))

    def stream_push(self, hops, maps=None, argmax=None, stream=None):
        """hops: CUDA float32 [B][M][hop] (consecutive blocks of new samples); the plan keeps
        the overlap between calls (srp_stream_push)."""
        import torch
        assert hops.is_cuda and hops.dtype == torch.float32 and hops.is_contiguous()
        B, hop = hops.shape[0], hops.shape[2]
        if maps is None:
            maps = torch.empty((B, self.J), dtype=torch.float32, device=hops.device)
        if argmax is None:
            argmax = torch.empty((B,), dtype=torch.int32, device=hops.device)
        _check(lib().srp_stream_push(self.handle, C.c_void_p(hops.data_ptr()), B, hop,
                                     C.c_void_p(maps.data_ptr()), C.c_void_p(argmax.data_ptr()),
                                     _stream_handle(stream)))
        return maps, argmax

    def stream_reset(self):
        _check(lib().srp_stream_reset(self.handle))

    def gcc_samples(self, frames, stream=None):
        import torch
        F = frames.shape[0]
        xi = torch.empty((F, self.L), dtype=torch.float32, device=frames.device)
        srp_gcc_samples(self.handle, C.c_void_p(frames.data_ptr()), F, C.c_void_p(xi.data_ptr()),
                        _stream_handle(stream))
        return xi

    def set_profiling(self, enable=True):
        srp_plan_set_profiling(self.handle, enable)

    def info_now(self):
        """srp_plan_info as of now (launch counter included)."""
        return srp_plan_info(self.handle)

    def stage_ms(self):
        return srp_plan_stage_ms(self.handle)

    def status(self, stream=None):
        srp_plan_status(self.handle, _stream_handle(stream))

    def save(self, path):
        """srp_plan_save: write the plan's fit (checkpoint) to path."""
        srp_plan_save(self.handle, path)

    def debug_stall_next_contraction(self):
        """Failure-detection test hook: the next tensor-core contraction's bounded waits run
        out (SRP_ETIMEOUT from status(); the plan stays usable)."""
        _check(lib().srp_debug_stall_next_contraction(self.handle))

    def lags(self):
        return srp_plan_lags(self.handle, self.P)

    def sspi_taps(self):
        return srp_plan_sspi_taps(self.handle, self.J, self.info.nnz)

    def slri_sigma(self, n=None):
        return srp_plan_slri_sigma(self.handle, self.L if n is None else n)

    def close(self):
        if getattr(self, "handle", None):
            srp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving ----------------------------------------------------------------------
def srp_plan_estimate_bytes(desc: srp_plan_desc) -> int:
    b = C.c_size_t()
    _check(lib().srp_plan_estimate_bytes(C.byref(desc), C.byref(b)))
    return b.value


def srp_server_now() -> float:
    return lib().srp_server_now()


class Server:
    """Many concurrent SRP sessions on the current CUDA device (libsrp's serving runtime):
    admission by HBM footprint, host framing with overlap, continuous batching over
    streams, CUDA-graph replay.  Host numpy in, host numpy out."""

    def __init__(self, hbm_budget=8 << 30, max_sessions=64, max_batch=16, streams=8,
                 slots_per_session=2, pending_frames=None, use_graphs=True, group_launches=True):
        d = srp_server_desc()
        d.hbm_budget, d.max_sessions, d.max_batch = int(hbm_budget), int(max_sessions), int(max_batch)
        d.streams, d.slots_per_session = int(streams), int(slots_per_session)
        d.pending_frames = int(pending_frames or 8 * max_batch)
        d.use_graphs = 1 if use_graphs else 0
        d.group_launches = 1 if group_launches else 0
        self.desc = d
        self.handle = C.c_void_p()
        _check(lib().srp_server_create(C.byref(d), C.byref(self.handle)))
        self.sessions = {}

    def open(self, mic_xyz, grid_xyz, fs, N, hop, method="slri", rank=0, taps=0.0,
             precision="bf16", window="hann", c=340.0, n_aux=2, far_field=False):
        desc = make_desc(mic_xyz, grid_xyz, fs, N, method, rank, taps, precision, window, c,
                         n_aux, max_frames=self.desc.max_batch, far_field=far_field)
        sid = C.c_int()
        _check(lib().srp_server_open(self.handle, C.byref(desc), int(hop), C.byref(sid)))
        self.sessions[sid.value] = (desc.M, desc.J)
        return sid.value

    def push(self, sid, samples, t_arrival=-1.0):
        """samples: [M][n] float32 (channel major).  Returns False if the queue is full."""
        a = np.ascontiguousarray(samples, dtype=np.float32)
        st = lib().srp_server_push(self.handle, sid, C.c_void_p(a.ctypes.data), a.shape[1],
                                   float(t_arrival))
        if st == SRP_EAGAIN:
            return False
        _check(st)
        return True

    def poll(self, sid, max_frames=None, want_maps=True):
        """-> (maps [n][J] or None, argmax [n], frame_index [n], latency_s [n])"""
        M, J = self.sessions[sid]
        n = int(max_frames or 4 * self.desc.max_batch)
        maps = np.empty((n, J), np.float32) if want_maps else None
        am = np.empty((n,), np.int32)
        idx = np.empty((n,), np.int64)
        lat = np.empty((n,), np.float64)
        got = C.c_int()
        _check(lib().srp_server_poll(self.handle, sid, n,
                                     C.c_void_p(maps.ctypes.data) if want_maps else None,
                                     C.c_void_p(am.ctypes.data), C.c_void_p(idx.ctypes.data),
                                     C.c_void_p(lat.ctypes.data), C.byref(got)))
        k = got.value
        return (maps[:k] if want_maps else None), am[:k], idx[:k], lat[:k]

    def session_info(self, sid):
        st, b, pend = C.c_int(), C.c_size_t(), C.c_int()
        _check(lib().srp_server_session_info(self.handle, sid, C.byref(st), C.byref(b), C.byref(pend)))
        return {"state": SESSION_STATES.get(st.value, st.value), "device_bytes": b.value,
                "pending": pend.value}

    def close_session(self, sid):
        _check(lib().srp_server_close(self.handle, sid))

    def stats(self):
        s = srp_server_stats_t()
        _check(lib().srp_server_stats(self.handle, C.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def reset_stats(self):
        _check(lib().srp_server_reset_stats(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().srp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
