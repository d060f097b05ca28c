"""Python binding of libkoma (ctypes; argument marshalling only).

Every function named ``koma_*`` here calls the C entry point of the same name
declared in ``include/koma.h``; all simulation work runs in the library's CUDA
kernels. PyTorch is used only for device memory and streams (``Simulator``).
There is no fallback: if ``libkoma.so`` is missing or fails to load, every
call raises ``KomaError``.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkoma.so")

KOMA_OK, KOMA_E_INVALID, KOMA_E_NOMEM, KOMA_E_CUDA, KOMA_E_TIMEOUT, KOMA_E_BUSY, KOMA_E_INTERNAL = range(7)
STATUS_NAMES = {0: "KOMA_OK", 1: "KOMA_E_INVALID", 2: "KOMA_E_NOMEM", 3: "KOMA_E_CUDA",
                4: "KOMA_E_TIMEOUT", 5: "KOMA_E_BUSY", 6: "KOMA_E_INTERNAL"}
KOMA_FP64 = 0
KOMA_FP32_SPLITPHASE = 1
PRECISIONS = {"fp64": KOMA_FP64, "fp32": KOMA_FP32_SPLITPHASE}

#: every entry point include/koma.h declares
EXPORTS = (
    "koma_gamma", "koma_version", "koma_init", "koma_destroy", "koma_last_error", "koma_mem_used",
    "koma_phantom_upload", "koma_phantom_n_spins", "koma_phantom_n_groups", "koma_phantom_free",
    "koma_phantom_set_motion",
    "koma_sequence_upload", "koma_sequence_n_adc", "koma_sequence_n_steps", "koma_sequence_get_info",
    "koma_sequence_free", "koma_sequence_plan", "koma_simulate", "koma_sync", "koma_set_timing",
    "koma_get_timing", "koma_get_launch_info", "koma_simulate_host", "koma_simulate_host_batch",
    "koma_simulate_static", "koma_tune",
    "koma_server_create", "koma_server_submit", "koma_server_wait", "koma_server_get_stats",
    "koma_server_last_error", "koma_server_destroy", "koma_check_bounded_wait", "koma_get_stage_timing",
    "koma_set_mma", "koma_set_rf_maps", "koma_get_map_timing",
)


class KomaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class HostJob(ctypes.Structure):
    """koma_host_job: one simulation of koma_simulate_host_batch."""
    _fields_ = ([("n", ctypes.c_int64)] + [(f, ctypes.POINTER(ctypes.c_double)) for f in
                                          ("x", "y", "z", "pd", "t1", "t2", "dw")] +
                [("group_offsets", ctypes.POINTER(ctypes.c_int64)), ("n_groups", ctypes.c_int64),
                 ("n_steps", ctypes.c_int64)] +
                [(f, ctypes.POINTER(ctypes.c_double)) for f in ("dt", "gx", "gy", "gz", "b1_re", "b1_im")] +
                [("adc", ctypes.POINTER(ctypes.c_uint8)), ("sig_host", ctypes.POINTER(ctypes.c_double))])


class LaunchInfo(ctypes.Structure):
    _fields_ = [("kernels", ctypes.c_int32), ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("spins_per_thread", ctypes.c_int32), ("spins_per_cta", ctypes.c_int64),
                ("n_records", ctypes.c_int64), ("partial_bytes", ctypes.c_int64),
                ("bloch_stream", ctypes.c_void_p), ("split", ctypes.c_int32), ("mma_grid", ctypes.c_int32),
                ("tile_records", ctypes.c_int32), ("phase_mode", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SequenceInfo(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int64), ("n_rf", ctypes.c_int64), ("n_adc", ctypes.c_int64),
                ("n_precess", ctypes.c_int64), ("n_records", ctypes.c_int64),
                ("n_adc_runs", ctypes.c_int64), ("n_materialize", ctypes.c_int64),
                ("n_mma_groups", ctypes.c_int64), ("n_mma_runs", ctypes.c_int64),
                ("n_mma_samples", ctypes.c_int64), ("n_rf_maps", ctypes.c_int64),
                ("n_rf_map_runs", ctypes.c_int64), ("n_rf_map_steps", ctypes.c_int64),
                ("n_rf_map_pulse_steps", ctypes.c_int64), ("z_dict", ctypes.c_int64),
                ("z_kmax", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_active", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("launch_work", ctypes.c_double), ("chunk_records", ctypes.c_int64),
                ("plain_spins", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("n_spins", ctypes.c_int64), ("n_steps", ctypes.c_int64),
                ("n_adc", ctypes.c_int64), ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("launches", ctypes.c_int32),
                ("status", ctypes.c_int), ("n_groups", ctypes.c_int64), ("lane", ctypes.c_int32),
                ("prep_s", ctypes.c_double), ("upload_s", ctypes.c_double), ("run_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("active", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("mem_used", ctypes.c_size_t), ("mem_peak", ctypes.c_size_t),
                ("lane_runs", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def load(path: Optional[str] = None):
    """Load libkoma.so and declare its signatures (raises KomaError if absent)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise KomaError(KOMA_E_CUDA, f"{p} is not built; run `python -m paper_2301_02702_b300.build`")
        try:
            lib = ctypes.CDLL(p)
        except OSError as e:
            raise KomaError(KOMA_E_CUDA, f"cannot load {p}: {e}") from e
        st = ctypes.c_int
        lib.koma_gamma.restype = ctypes.c_double
        lib.koma_gamma.argtypes = []
        lib.koma_version.restype = ctypes.c_char_p
        lib.koma_version.argtypes = []
        lib.koma_init.restype = st
        lib.koma_init.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_vp)]
        lib.koma_destroy.restype = st
        lib.koma_destroy.argtypes = [_vp]
        lib.koma_last_error.restype = ctypes.c_char_p
        lib.koma_last_error.argtypes = [_vp]
        lib.koma_mem_used.restype = ctypes.c_size_t
        lib.koma_mem_used.argtypes = [_vp]
        lib.koma_phantom_upload.restype = st
        lib.koma_phantom_upload.argtypes = [_vp, ctypes.c_int64] + [_dp] * 7 + [_i64p, ctypes.c_int64,
                                                                                 ctypes.POINTER(_vp)]
        lib.koma_phantom_n_spins.restype = ctypes.c_int64
        lib.koma_phantom_n_spins.argtypes = [_vp]
        lib.koma_phantom_n_groups.restype = ctypes.c_int64
        lib.koma_phantom_n_groups.argtypes = [_vp]
        lib.koma_phantom_free.restype = st
        lib.koma_phantom_free.argtypes = [_vp]
        lib.koma_phantom_set_motion.restype = st
        lib.koma_phantom_set_motion.argtypes = [_vp, _dp, _dp, _dp]
        lib.koma_sequence_upload.restype = st
        lib.koma_sequence_upload.argtypes = [_vp, ctypes.c_int64] + [_dp] * 6 + [_u8p, ctypes.POINTER(_vp)]
        lib.koma_sequence_n_adc.restype = ctypes.c_int64
        lib.koma_sequence_n_adc.argtypes = [_vp]
        lib.koma_sequence_n_steps.restype = ctypes.c_int64
        lib.koma_sequence_n_steps.argtypes = [_vp]
        lib.koma_sequence_get_info.restype = st
        lib.koma_sequence_get_info.argtypes = [_vp, ctypes.POINTER(SequenceInfo)]
        lib.koma_sequence_free.restype = st
        lib.koma_sequence_free.argtypes = [_vp]
        lib.koma_sequence_plan.restype = st
        lib.koma_sequence_plan.argtypes = ([ctypes.c_int64] + [_dp] * 6 + [_u8p, ctypes.POINTER(SequenceInfo),
                                           _dp, ctypes.c_int64])
        lib.koma_simulate.restype = st
        lib.koma_simulate.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]
        lib.koma_sync.restype = st
        lib.koma_sync.argtypes = [_vp, _vp]
        lib.koma_set_timing.restype = st
        lib.koma_set_timing.argtypes = [_vp, ctypes.c_int]
        lib.koma_get_timing.restype = st
        lib.koma_get_timing.argtypes = [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
        lib.koma_get_stage_timing.restype = st
        lib.koma_get_stage_timing.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_float)] * 3
        lib.koma_set_mma.restype = st
        lib.koma_set_mma.argtypes = [_vp, ctypes.c_int]
        lib.koma_set_rf_maps.restype = st
        lib.koma_set_rf_maps.argtypes = [_vp, ctypes.c_int]
        lib.koma_get_map_timing.restype = st
        lib.koma_get_map_timing.argtypes = [_vp, ctypes.POINTER(ctypes.c_float)]
        lib.koma_get_launch_info.restype = st
        lib.koma_get_launch_info.argtypes = [_vp, ctypes.POINTER(LaunchInfo)]
        lib.koma_server_create.restype = st
        lib.koma_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]
        lib.koma_server_submit.restype = st
        lib.koma_server_submit.argtypes = ([_vp, ctypes.c_int64] + [_dp] * 7 + [_i64p, ctypes.c_int64,
                                           ctypes.c_int64] + [_dp] * 6 + [_u8p, ctypes.POINTER(ctypes.c_uint64)])
        lib.koma_server_wait.restype = st
        lib.koma_server_wait.argtypes = [_vp, ctypes.c_uint64, ctypes.c_double, _dp, ctypes.c_int64,
                                         ctypes.POINTER(RequestInfo)]
        lib.koma_server_get_stats.restype = st
        lib.koma_server_get_stats.argtypes = [_vp, ctypes.POINTER(ServerStats)]
        lib.koma_server_last_error.restype = ctypes.c_char_p
        lib.koma_server_last_error.argtypes = [_vp]
        lib.koma_server_destroy.restype = st
        lib.koma_server_destroy.argtypes = [_vp]
        lib.koma_tune.restype = st
        lib.koma_tune.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(LaunchInfo)]
        lib.koma_check_bounded_wait.restype = st
        lib.koma_check_bounded_wait.argtypes = [_vp, ctypes.c_int64, _vp]
        lib.koma_simulate_static.restype = st
        lib.koma_simulate_static.argtypes = [_vp, _vp, _vp, _vp]
        lib.koma_simulate_host_batch.restype = st
        lib.koma_simulate_host_batch.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(HostJob), ctypes.c_int]
        lib.koma_simulate_host.restype = st
        lib.koma_simulate_host.argtypes = ([_vp, ctypes.c_int64] + [_dp] * 7 + [_i64p, ctypes.c_int64,
                                           ctypes.c_int64] + [_dp] * 6 + [_u8p, ctypes.c_int, _dp])
        if path is None:
            _lib = lib
        return lib


def _check(ctx, rc: int, what: str):
    if rc != KOMA_OK:
        msg = load().koma_last_error(ctx).decode() if ctx else ""
        raise KomaError(rc, f"{what}: {msg}")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


# --------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------

def koma_gamma() -> float:
    return load().koma_gamma()


def koma_version() -> str:
    return load().koma_version().decode()


def koma_init(device: int = 0, mem_budget_bytes: int = 0):
    out = _vp()
    rc = load().koma_init(int(device), int(mem_budget_bytes), ctypes.byref(out))
    if rc != KOMA_OK:
        raise KomaError(rc, f"koma_init(device={device}) failed")
    return out


def koma_destroy(ctx):
    _check(ctx, load().koma_destroy(ctx), "koma_destroy")


def koma_last_error(ctx) -> str:
    return load().koma_last_error(ctx).decode()


def koma_mem_used(ctx) -> int:
    return int(load().koma_mem_used(ctx))


def koma_phantom_upload(ctx, phantom):
    """Upload a phantom (object with x, y, z, pd, t1, t2, dw and optional
    group_offsets and velocity [3, n]). Returns the phantom handle."""
    arrs = [_f64(getattr(phantom, f)) for f in ("x", "y", "z", "pd", "t1", "t2", "dw")]
    n = arrs[0].shape[0]
    go = getattr(phantom, "group_offsets", None)
    go_arr = None if go is None else np.ascontiguousarray(go, dtype=np.int64)
    n_groups = 1 if go_arr is None else go_arr.shape[0] - 1
    out = _vp()
    rc = load().koma_phantom_upload(ctx, n, *[_ptr(a) for a in arrs],
                                    None if go_arr is None else _ptr(go_arr, ctypes.c_int64),
                                    n_groups, ctypes.byref(out))
    _check(ctx, rc, "koma_phantom_upload")
    vel = getattr(phantom, "velocity", None)
    if vel is not None:
        try:
            koma_phantom_set_motion(ctx, out, vel)
        except KomaError:
            load().koma_phantom_free(out)
            raise
    return out


def koma_phantom_set_motion(ctx, ph, velocity):
    """Give an uploaded phantom constant per-spin velocities ``velocity``
    [3, n] (m/s; x(t) = x + v t), or make it static again with None."""
    lib = load()
    if velocity is None:
        _check(ctx, lib.koma_phantom_set_motion(ph, None, None, None), "koma_phantom_set_motion")
        return
    v = [_f64(a) for a in velocity]
    if len(v) != 3 or any(a.shape != (koma_phantom_n_spins(ph),) for a in v):
        raise KomaError(KOMA_E_INVALID, "koma_phantom_set_motion: velocity must be [3, n_spins]")
    _check(ctx, lib.koma_phantom_set_motion(ph, *[_ptr(a) for a in v]), "koma_phantom_set_motion")


def koma_phantom_n_spins(ph) -> int:
    return int(load().koma_phantom_n_spins(ph))


def koma_phantom_n_groups(ph) -> int:
    return int(load().koma_phantom_n_groups(ph))


def koma_phantom_free(ph):
    load().koma_phantom_free(ph)


def _seq_arrays(seq):
    b1 = np.asarray(seq.b1, dtype=np.complex128)
    return (_f64(seq.dt), _f64(seq.gx), _f64(seq.gy), _f64(seq.gz), _f64(b1.real), _f64(b1.imag),
            np.ascontiguousarray(seq.adc, dtype=np.uint8))


def koma_sequence_upload(ctx, seq):
    """Upload a discretised sequence (object with dt, gx, gy, gz, b1, adc)."""
    dt, gx, gy, gz, bre, bim, adc = _seq_arrays(seq)
    out = _vp()
    rc = load().koma_sequence_upload(ctx, dt.shape[0], _ptr(dt), _ptr(gx), _ptr(gy), _ptr(gz),
                                     _ptr(bre), _ptr(bim), _ptr(adc, ctypes.c_uint8), ctypes.byref(out))
    _check(ctx, rc, "koma_sequence_upload")
    return out


def koma_sequence_n_adc(seq) -> int:
    return int(load().koma_sequence_n_adc(seq))


def koma_sequence_n_steps(seq) -> int:
    return int(load().koma_sequence_n_steps(seq))


def koma_sequence_get_info(seq) -> dict:
    info = SequenceInfo()
    rc = load().koma_sequence_get_info(seq, ctypes.byref(info))
    if rc != KOMA_OK:
        raise KomaError(rc, "koma_sequence_get_info")
    return info.as_dict()


def koma_sequence_free(seq):
    load().koma_sequence_free(seq)


def koma_sequence_plan(seq, with_records: bool = False):
    """Host-only preprocessing of a sequence (no GPU needed). Returns the
    step-class counts, and with ``with_records`` also the FP64 records as a
    [n_records, 17] array ([type, count, first sample, 14 payload values])."""
    dt, gx, gy, gz, bre, bim, adc = _seq_arrays(seq)
    info = SequenceInfo()
    lib = load()
    rc = lib.koma_sequence_plan(dt.shape[0], _ptr(dt), _ptr(gx), _ptr(gy), _ptr(gz), _ptr(bre), _ptr(bim),
                                _ptr(adc, ctypes.c_uint8), ctypes.byref(info), None, 0)
    if rc != KOMA_OK:
        raise KomaError(rc, "koma_sequence_plan rejected the sequence")
    if not with_records:
        return info.as_dict()
    rec = np.zeros((max(info.n_records, 1), 17), dtype=np.float64)
    rc = lib.koma_sequence_plan(dt.shape[0], _ptr(dt), _ptr(gx), _ptr(gy), _ptr(gz), _ptr(bre), _ptr(bim),
                                _ptr(adc, ctypes.c_uint8), ctypes.byref(info), _ptr(rec), rec.shape[0])
    if rc != KOMA_OK:
        raise KomaError(rc, "koma_sequence_plan")
    return info.as_dict(), rec[:info.n_records]


def koma_simulate(ctx, ph, seq, precision: int, sig_dev_ptr: int, stream_ptr: int):
    rc = load().koma_simulate(ctx, ph, seq, int(precision), ctypes.c_void_p(int(sig_dev_ptr)),
                              ctypes.c_void_p(int(stream_ptr)))
    _check(ctx, rc, "koma_simulate")


def koma_tune(ctx, ph, seq, sig_dev_ptr: int, stream_ptr: int) -> dict:
    """Autotune the FP32 launch for (ph, seq); returns the chosen launch."""
    info = LaunchInfo()
    rc = load().koma_tune(ctx, ph, seq, ctypes.c_void_p(int(sig_dev_ptr)), ctypes.c_void_p(int(stream_ptr)),
                          ctypes.byref(info))
    _check(ctx, rc, "koma_tune")
    return info.as_dict()


def koma_simulate_static(ctx, ph, seq, sig_dev_ptr: int, stream_ptr: int):
    """Allocation-free simulation (FP32 path): partial sums in the library's
    static device array. ``ctx`` is only used to fetch the error message."""
    rc = load().koma_simulate_static(ph, seq, ctypes.c_void_p(int(sig_dev_ptr)), ctypes.c_void_p(int(stream_ptr)))
    _check(ctx, rc, "koma_simulate_static")


def koma_sync(ctx, stream_ptr: int):
    _check(ctx, load().koma_sync(ctx, ctypes.c_void_p(int(stream_ptr))), "koma_sync")


def koma_set_timing(ctx, enable: bool = True):
    _check(ctx, load().koma_set_timing(ctx, int(bool(enable))), "koma_set_timing")


def koma_get_timing(ctx):
    """(bloch_ms, reduce_ms) of the last timed koma_simulate."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(ctx, load().koma_get_timing(ctx, ctypes.byref(a), ctypes.byref(b)), "koma_get_timing")
    return a.value, b.value


def koma_get_stage_timing(ctx):
    """(bloch_ms, mma_ms, reduce_ms) of the last timed koma_simulate; mma_ms
    is the tensor-core readout (0 when it did not run)."""
    a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(ctx, load().koma_get_stage_timing(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "koma_get_stage_timing")
    return a.value, b.value, c.value


def koma_set_mma(ctx, enable: bool = True):
    _check(ctx, load().koma_set_mma(ctx, int(bool(enable))), "koma_set_mma")


def koma_set_rf_maps(ctx, enable: bool = True):
    _check(ctx, load().koma_set_rf_maps(ctx, int(bool(enable))), "koma_set_rf_maps")


def koma_get_map_timing(ctx) -> float:
    """Milliseconds of the repeated-pulse map pre-pass of the last timed
    koma_simulate (0 when it had none)."""
    a = ctypes.c_float()
    _check(ctx, load().koma_get_map_timing(ctx, ctypes.byref(a)), "koma_get_map_timing")
    return a.value


def koma_get_launch_info(ctx) -> dict:
    info = LaunchInfo()
    _check(ctx, load().koma_get_launch_info(ctx, ctypes.byref(info)), "koma_get_launch_info")
    return info.as_dict()


def koma_simulate_host(ctx, phantom, seq, precision: int = KOMA_FP32_SPLITPHASE, out=None):
    """Host arrays in, host signal out (complex128 [n_groups, n_adc])."""
    arrs = [_f64(getattr(phantom, f)) for f in ("x", "y", "z", "pd", "t1", "t2", "dw")]
    go = getattr(phantom, "group_offsets", None)
    go_arr = None if go is None else np.ascontiguousarray(go, dtype=np.int64)
    n_groups = 1 if go_arr is None else go_arr.shape[0] - 1
    dt, gx, gy, gz, bre, bim, adc = _seq_arrays(seq)
    n_adc = int(np.count_nonzero(adc))
    if out is None:
        out = np.empty((n_groups, n_adc), dtype=np.complex128)
    assert out.dtype == np.complex128 and out.flags.c_contiguous and out.size == n_groups * n_adc
    rc = load().koma_simulate_host(ctx, arrs[0].shape[0], *[_ptr(a) for a in arrs],
                                   None if go_arr is None else _ptr(go_arr, ctypes.c_int64), n_groups,
                                   dt.shape[0], _ptr(dt), _ptr(gx), _ptr(gy), _ptr(gz), _ptr(bre),
                                   _ptr(bim), _ptr(adc, ctypes.c_uint8), int(precision),
                                   out.ctypes.data_as(_dp))
    _check(ctx, rc, "koma_simulate_host")
    return out


def koma_simulate_host_batch(ctx, jobs, precision: int = KOMA_FP32_SPLITPHASE):
    """koma_simulate_host for each (phantom, seq, out) of `jobs`, one job's
    host work overlapped with the previous job's simulation; `out` as for
    koma_simulate_host (allocated when None). Returns the outputs."""
    keep, arr, outs = [], (HostJob * max(1, len(jobs)))(), []
    for i, (phantom, seq, out) in enumerate(jobs):
        ph = [_f64(getattr(phantom, f)) for f in ("x", "y", "z", "pd", "t1", "t2", "dw")]
        go = getattr(phantom, "group_offsets", None)
        go_arr = None if go is None else np.ascontiguousarray(go, dtype=np.int64)
        n_groups = 1 if go_arr is None else go_arr.shape[0] - 1
        sq = _seq_arrays(seq)
        n_adc = int(np.count_nonzero(sq[6]))
        if out is None:
            out = np.empty((n_groups, n_adc), dtype=np.complex128)
        assert out.dtype == np.complex128 and out.flags.c_contiguous and out.size == n_groups * n_adc
        keep += ph + list(sq) + [go_arr, out]
        j = arr[i]
        j.n = ph[0].shape[0]
        for f, a in zip(("x", "y", "z", "pd", "t1", "t2", "dw"), ph):
            setattr(j, f, _ptr(a))
        j.group_offsets = None if go_arr is None else _ptr(go_arr, ctypes.c_int64)
        j.n_groups = n_groups
        j.n_steps = sq[0].shape[0]
        for f, a in zip(("dt", "gx", "gy", "gz", "b1_re", "b1_im"), sq[:6]):
            setattr(j, f, _ptr(a))
        j.adc = _ptr(sq[6], ctypes.c_uint8)
        j.sig_host = out.ctypes.data_as(_dp)
        outs.append(out)
    rc = load().koma_simulate_host_batch(ctx, len(jobs), arr, int(precision))
    _check(ctx, rc, "koma_simulate_host_batch")
    del keep
    return outs


# --------------------------------------------------------------------------
# convenience layer over torch device memory / streams
# --------------------------------------------------------------------------

class Simulator:
    """Owns a context on one CUDA device; uploads and simulates.

    >>> sim = Simulator()
    >>> ph = sim.upload_phantom(phantom); sq = sim.upload_sequence(seq)
    >>> sig = sim.simulate(ph, sq)          # torch complex128 [n_groups, n_adc] on the device
    """

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        import torch  # noqa: F401  (device memory and streams)
        self.device = device
        self.ctx = koma_init(device, mem_budget_bytes)

    def upload_phantom(self, phantom):
        return koma_phantom_upload(self.ctx, phantom)

    def upload_sequence(self, seq):
        return koma_sequence_upload(self.ctx, seq)

    def simulate(self, ph, seq, precision="fp32", out=None, stream=None):
        import torch
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        n_adc = koma_sequence_n_adc(seq)
        n_groups = koma_phantom_n_groups(ph)
        if out is None:
            out = torch.empty((n_groups, n_adc), dtype=torch.complex128, device=f"cuda:{self.device}")
        assert out.dtype == torch.complex128 and out.is_contiguous() and out.numel() == n_groups * n_adc
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        koma_simulate(self.ctx, ph, seq, prec, out.data_ptr() if out.numel() else 0, st.cuda_stream)
        return out

    def sync(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        koma_sync(self.ctx, st.cuda_stream)

    def tune(self, ph, seq, stream=None) -> dict:
        import torch
        n_adc = koma_sequence_n_adc(seq)
        out = torch.empty((koma_phantom_n_groups(ph), n_adc), dtype=torch.complex128, device=f"cuda:{self.device}")
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        return koma_tune(self.ctx, ph, seq, out.data_ptr() if out.numel() else 0, st.cuda_stream)

    def launch_info(self) -> dict:
        return koma_get_launch_info(self.ctx)

    def close(self):
        if self.ctx is not None:
            koma_destroy(self.ctx)
            self.ctx = None


# --------------------------------------------------------------------------
# continuous-batching server
# --------------------------------------------------------------------------

def koma_server_create(device: int = 0, mem_budget_bytes: int = 0, max_active: int = 0, launch_work: float = 0.0,
                       chunk_records: int = 0, plain_spins: int = 0):
    cfg = ServerConfig(int(device), int(max_active), int(mem_budget_bytes), float(launch_work), int(chunk_records),
                       int(plain_spins))
    out = _vp()
    rc = load().koma_server_create(ctypes.byref(cfg), ctypes.byref(out))
    if rc != KOMA_OK:
        raise KomaError(rc, "koma_server_create failed")
    return out


def koma_server_last_error(srv) -> str:
    return load().koma_server_last_error(srv).decode()


def koma_server_submit(srv, phantom, seq) -> int:
    arrs = [_f64(getattr(phantom, f)) for f in ("x", "y", "z", "pd", "t1", "t2", "dw")]
    go = getattr(phantom, "group_offsets", None)
    go_arr = None if go is None else np.ascontiguousarray(go, dtype=np.int64)
    n_groups = 1 if go_arr is None else int(go_arr.shape[0] - 1)
    dt, gx, gy, gz, bre, bim, adc = _seq_arrays(seq)
    rid = ctypes.c_uint64()
    rc = load().koma_server_submit(srv, arrs[0].shape[0], *[_ptr(a) for a in arrs],
                                   None if go_arr is None else _ptr(go_arr, ctypes.c_int64), n_groups,
                                   dt.shape[0], _ptr(dt), _ptr(gx), _ptr(gy), _ptr(gz), _ptr(bre), _ptr(bim),
                                   _ptr(adc, ctypes.c_uint8), ctypes.byref(rid))
    if rc != KOMA_OK:
        raise KomaError(rc, "koma_server_submit: " + koma_server_last_error(srv))
    return int(rid.value)


def koma_server_wait(srv, rid: int, n_adc: int, timeout_s: float = -1.0, n_groups: int = 1):
    """(signal complex128 [n_adc], or [n_groups, n_adc] for a grouped request;
    info dict) of request `rid`."""
    out = np.empty(max(n_groups * n_adc, 1), dtype=np.complex128)
    info = RequestInfo()
    rc = load().koma_server_wait(srv, int(rid), float(timeout_s), out.ctypes.data_as(_dp), n_groups * n_adc,
                                 ctypes.byref(info))
    if rc != KOMA_OK:
        raise KomaError(rc, "koma_server_wait: " + koma_server_last_error(srv))
    sig = out[:n_groups * n_adc]
    return (sig.reshape(n_groups, n_adc) if n_groups > 1 else sig), info.as_dict()


def koma_check_bounded_wait(ctx, limit_us: int, stream_handle: int = 0):
    """Enqueue the self-check of the device-side timeout path (see koma.h);
    the next koma_sync on the stream raises KomaError(KOMA_E_TIMEOUT)."""
    _check(ctx, load().koma_check_bounded_wait(ctx, int(limit_us), stream_handle or None),
           "koma_check_bounded_wait")


def koma_server_get_stats(srv) -> dict:
    st = ServerStats()
    rc = load().koma_server_get_stats(srv, ctypes.byref(st))
    if rc != KOMA_OK:
        raise KomaError(rc, "koma_server_get_stats")
    return st.as_dict()


def koma_server_destroy(srv):
    load().koma_server_destroy(srv)


class Server:
    """Continuous-batching simulation server on one device (native worker
    threads: shared launches for small requests, the koma_simulate lane for
    large and grouped ones)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_active: int = 0, launch_work: float = 0.0,
                 chunk_records: int = 0, plain_spins: int = 0):
        self.srv = koma_server_create(device, mem_budget_bytes, max_active, launch_work, chunk_records, plain_spins)
        self._shape = {}

    def submit(self, phantom, seq) -> int:
        rid = koma_server_submit(self.srv, phantom, seq)
        go = getattr(phantom, "group_offsets", None)
        self._shape[rid] = (int(np.count_nonzero(seq.adc)), 1 if go is None else int(len(go) - 1))
        return rid

    def wait(self, rid: int, timeout_s: float = -1.0):
        n_adc, n_groups = self._shape[rid]
        sig, info = koma_server_wait(self.srv, rid, n_adc, timeout_s, n_groups)
        del self._shape[rid]
        return sig, info

    def stats(self) -> dict:
        return koma_server_get_stats(self.srv)

    def close(self):
        if self.srv is not None:
            koma_server_destroy(self.srv)
            self.srv = None
