"""FP64 CPU oracle for the Bloch-simulation hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline / reference leg, never by the library.
The C source (``koma_oracle.c``) states, step by step, which equation of the
KomaMRI.jl paper each operation follows; it shares no code with the CUDA path.

Parity status per function:
* ``simulate``  pinned by closed forms (FID, flip angle, spin echo, Ernst
  steady state, k-space = 2-D DFT), by invariants and by ``rk4``.
* ``rk4``       a direct integration of the Bloch equation; pinned by the same
  closed forms in the precession regime (where it must agree to ~1e-9).
Excitation with a soft pulse under a simultaneous gradient and relaxation has
no closed form: there the oracle is pinned only through convergence to
``rk4`` as the RF step shrinks (parity unpinned beyond that).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "koma_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

#: the oracle's γ (rad/s/T); the tests check the library reports the same value
GAMMA = 2.0 * np.pi * 42.577478518e6


def build(force: bool = False) -> str:
    """Compile ``koma_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # KOMA_ORACLE_LIB points at a deliberately broken build of this
            # oracle (mutation tests check that the pins reject it)
            lib = ctypes.CDLL(os.environ.get("KOMA_ORACLE_LIB") or build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_simulate.restype = ctypes.c_int
            lib.oracle_simulate.argtypes = ([ctypes.c_int64] + [dp] * 7 + [i64p, ctypes.c_int64,
                                            ctypes.c_int64] + [dp] * 6 + [u8p, ctypes.c_int, dp, dp])
            lib.oracle_simulate_moving.restype = ctypes.c_int
            lib.oracle_simulate_moving.argtypes = ([ctypes.c_int64] + [dp] * 10 + [i64p, ctypes.c_int64,
                                                   ctypes.c_int64] + [dp] * 6 + [u8p, ctypes.c_int, dp, dp])
            lib.oracle_rk4_moving.restype = ctypes.c_int
            lib.oracle_rk4_moving.argtypes = ([ctypes.c_double] * 10 + [ctypes.c_int64] + [dp] * 6
                                              + [u8p, ctypes.c_int64, dp, dp])
            lib.oracle_rk4.restype = ctypes.c_int
            lib.oracle_rk4.argtypes = ([ctypes.c_double] * 7 + [ctypes.c_int64] + [dp] * 6
                                       + [u8p, ctypes.c_int64, dp, dp])
            _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _seq_arrays(seq):
    b1 = np.asarray(seq.b1, dtype=np.complex128)
    return (_d(seq.dt), _d(seq.gx), _d(seq.gy), _d(seq.gz), _d(b1.real), _d(b1.imag),
            np.ascontiguousarray(seq.adc, dtype=np.uint8))


def simulate(phantom, seq, threads: int = 0, return_state: bool = False):
    """Signal of ``phantom`` under ``seq``: complex128 array [n_groups, n_adc]
    (grouped phantoms sum within each group). A phantom attribute
    ``velocity = (vx, vy, vz)`` (m/s per spin) moves the spins, x(t) = x + v t.
    With ``return_state`` also the final magnetisation [n, 3] = (Mx, My, Mz)."""
    lib = _load()
    ph = [_d(getattr(phantom, f)) for f in ("x", "y", "z", "pd", "t1", "t2", "dw")]
    n = ph[0].shape[0]
    go = getattr(phantom, "group_offsets", None)
    n_groups = 1 if go is None else int(len(go) - 1)
    go_arr = None if go is None else np.ascontiguousarray(go, dtype=np.int64)
    dt, gx, gy, gz, b1re, b1im, adc = _seq_arrays(seq)
    n_steps = dt.shape[0]
    n_adc = int(np.count_nonzero(adc))
    sig = np.zeros((n_groups, max(n_adc, 0), 2), dtype=np.float64)
    mf = np.zeros((n, 3), dtype=np.float64) if return_state else None
    vel = getattr(phantom, "velocity", None)
    vel = None if vel is None else [_d(v) for v in vel]  # kept alive through the call
    vptr = [None, None, None] if vel is None else [_ptr(v) for v in vel]
    rc = lib.oracle_simulate_moving(
        n, *[_ptr(a) for a in ph], *vptr,
        None if go_arr is None else _ptr(go_arr, ctypes.c_int64), n_groups,
        n_steps, _ptr(dt), _ptr(gx), _ptr(gy), _ptr(gz), _ptr(b1re), _ptr(b1im),
        _ptr(adc, ctypes.c_uint8), int(threads),
        _ptr(sig) if sig.size else _ptr(np.zeros(2)),
        None if mf is None else _ptr(mf))
    if rc != 0:
        raise ValueError("oracle_simulate rejected its arguments")
    out = sig[..., 0] + 1j * sig[..., 1]
    return (out, mf) if return_state else out


def rk4(spin, seq, substeps: int):
    """Brute-force RK4 of the Bloch equation for ONE spin (a mapping or object
    with scalar x, y, z, pd, t1, t2, dw and optionally vx, vy, vz for a
    constant velocity). Returns (signal [n_adc] complex128, final
    magnetisation [3])."""
    lib = _load()
    get = (lambda k: float(spin[k])) if isinstance(spin, dict) else (lambda k: float(getattr(spin, k)))
    dt, gx, gy, gz, b1re, b1im, adc = _seq_arrays(seq)
    n_adc = int(np.count_nonzero(adc))
    sig = np.zeros((max(n_adc, 1), 2))
    mf = np.zeros(3)
    v = [float(spin.get(k, 0.0)) if isinstance(spin, dict) else float(getattr(spin, k, 0.0))
         for k in ("vx", "vy", "vz")]
    rc = lib.oracle_rk4_moving(get("x"), get("y"), get("z"), get("pd"), get("t1"), get("t2"), get("dw"),
                               *v, dt.shape[0], _ptr(dt), _ptr(gx), _ptr(gy), _ptr(gz), _ptr(b1re),
                               _ptr(b1im), _ptr(adc, ctypes.c_uint8), int(substeps), _ptr(sig), _ptr(mf))
    if rc != 0:
        raise ValueError("oracle_rk4 rejected its arguments")
    return (sig[:n_adc, 0] + 1j * sig[:n_adc, 1]), mf
