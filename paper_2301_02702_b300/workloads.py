"""Seeded synthetic phantoms and discretised pulse sequences.

This module only builds the arrays a Bloch simulation consumes; it contains no
Bloch-equation arithmetic and is shared by the CUDA path's tests and the
oracle's tests alike (neither side imports the other).

Objects follow the paper's input types (Section "Overview"): a *phantom* is a
set of spins with position x, proton density M0 (``pd``), T1, T2 and
off-resonance Δω; a *sequence* is the discretised form the solver steps
through ("Sequence-aware time stepping"): time points t_0..t_N with

* ``dt[n]``            step length t_{n+1} - t_n                      [s]
* ``gx/gy/gz[i]``      gradient value at time point t_i (vertices; the
                       waveform is piecewise linear between them)     [T/m]
* ``b1[n]``            complex RF B1 = B1x + i B1y, constant over step n [T]
* ``adc[i]``           1 where the ADC samples the signal at t_i

Units are SI (m, s, T, rad/s). All randomness comes from numpy PCG64 with an
explicit seed.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence as Seq

import numpy as np

#: proton gyromagnetic ratio / 2π (CODATA 2018), Hz/T
GAMMA_BAR = 42.577478518e6
#: proton gyromagnetic ratio, rad/s/T
GAMMA = 2.0 * np.pi * GAMMA_BAR


@dataclasses.dataclass
class Phantom:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    pd: np.ndarray
    t1: np.ndarray
    t2: np.ndarray
    dw: np.ndarray  # off-resonance Δω, rad/s
    group_offsets: Optional[np.ndarray] = None  # int64 [n_groups + 1]
    # motion u(x, t) = v t: per-spin constant velocity [3, n] (m/s), or None
    velocity: Optional[np.ndarray] = None

    def __post_init__(self):
        for f in ("x", "y", "z", "pd", "t1", "t2", "dw"):
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.float64))
        if self.group_offsets is not None:
            self.group_offsets = np.ascontiguousarray(self.group_offsets, dtype=np.int64)
        if self.velocity is not None:
            self.velocity = np.ascontiguousarray(np.broadcast_to(self.velocity, (3, self.x.shape[0])),
                                                 dtype=np.float64)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_groups(self) -> int:
        return 1 if self.group_offsets is None else int(self.group_offsets.shape[0] - 1)

    def subset(self, idx) -> "Phantom":
        idx = np.asarray(idx)
        return Phantom(*(getattr(self, f)[idx] for f in ("x", "y", "z", "pd", "t1", "t2", "dw")),
                       velocity=None if self.velocity is None else self.velocity[:, idx])

    def arrays(self):
        return self.x, self.y, self.z, self.pd, self.t1, self.t2, self.dw


@dataclasses.dataclass
class Sequence:
    dt: np.ndarray
    gx: np.ndarray
    gy: np.ndarray
    gz: np.ndarray
    b1: np.ndarray
    adc: np.ndarray

    def __post_init__(self):
        for f in ("dt", "gx", "gy", "gz"):
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.float64))
        self.b1 = np.ascontiguousarray(self.b1, dtype=np.complex128)
        self.adc = np.ascontiguousarray(self.adc, dtype=np.uint8)
        n = self.dt.shape[0]
        assert self.gx.shape == (n + 1,) and self.gy.shape == (n + 1,) and self.gz.shape == (n + 1,)
        assert self.b1.shape == (n,) and self.adc.shape == (n + 1,)

    @property
    def n_steps(self) -> int:
        return int(self.dt.shape[0])

    @property
    def n_adc(self) -> int:
        return int(np.count_nonzero(self.adc))

    @property
    def n_rf(self) -> int:
        return int(np.count_nonzero(self.b1))

    @property
    def duration(self) -> float:
        return float(self.dt.sum())

    def arrays(self):
        return (self.dt, self.gx, self.gy, self.gz,
                np.ascontiguousarray(self.b1.real), np.ascontiguousarray(self.b1.imag), self.adc)

    def concat(self, other: "Sequence") -> "Sequence":
        """Play ``other`` right after ``self`` (the joining vertex must agree)."""
        g_self = np.array([self.gx[-1], self.gy[-1], self.gz[-1]])
        g_other = np.array([other.gx[0], other.gy[0], other.gz[0]])
        assert np.array_equal(g_self, g_other), "gradient waveform must be continuous"
        adc = self.adc.copy()
        adc[-1] = adc[-1] | other.adc[0]
        return Sequence(np.concatenate([self.dt, other.dt]),
                        np.concatenate([self.gx, other.gx[1:]]),
                        np.concatenate([self.gy, other.gy[1:]]),
                        np.concatenate([self.gz, other.gz[1:]]),
                        np.concatenate([self.b1, other.b1]),
                        np.concatenate([adc, other.adc[1:]]))


class SequenceBuilder:
    """Appends steps to a discretised sequence.

    Every call adds ``n`` steps of length ``dt``; the gradient moves linearly
    from its current vertex value to ``g_end`` over those steps (``None``
    keeps it constant), so the waveform stays continuous and piecewise linear.
    """

    def __init__(self):
        self._dt: List[np.ndarray] = []
        self._g: List[np.ndarray] = [np.zeros((1, 3))]
        self._b1: List[np.ndarray] = []
        self._adc: List[np.ndarray] = [np.zeros(1, dtype=np.uint8)]
        self.g = np.zeros(3)
        self.t = 0.0

    def steps(self, n: int, dt: float, g_end=None, b1=None, adc: bool = False):
        n = int(n)
        if n <= 0:
            return self
        g_end = self.g.copy() if g_end is None else np.asarray(g_end, dtype=np.float64)
        frac = (np.arange(1, n + 1, dtype=np.float64) / n)[:, None]
        self._g.append(self.g[None, :] * (1.0 - frac) + g_end[None, :] * frac)
        self._dt.append(np.full(n, float(dt)))
        if b1 is None:
            self._b1.append(np.zeros(n, dtype=np.complex128))
        else:
            b1 = np.broadcast_to(np.asarray(b1, dtype=np.complex128), (n,))
            self._b1.append(np.array(b1))
        self._adc.append(np.full(n, 1 if adc else 0, dtype=np.uint8))
        self.g = g_end.copy()
        self.t += n * dt
        return self

    def idle_until(self, t_end: float, g_end=None):
        """One step (gradient vertex only) up to time ``t_end``."""
        if t_end - self.t > 1e-12:
            self.steps(1, t_end - self.t, g_end)
        return self

    def trapezoid(self, area_turns_per_m, ramp_steps: int, flat_steps: int, dt: float):
        """Gradient lobe whose moment γ̄∫G dt equals ``area_turns_per_m``
        (per axis), with ``ramp_steps`` on each ramp and ``flat_steps`` flat.
        The lobe must start from zero gradient and returns to zero."""
        area = np.asarray(area_turns_per_m, dtype=np.float64)
        amp = area / (GAMMA_BAR * (flat_steps + ramp_steps) * dt)
        self.steps(ramp_steps, dt, amp)
        self.steps(flat_steps, dt, amp)
        self.steps(ramp_steps, dt, np.zeros(3))
        return self

    def build(self) -> Sequence:
        g = np.concatenate(self._g, axis=0)
        return Sequence(np.concatenate(self._dt) if self._dt else np.zeros(0),
                        g[:, 0], g[:, 1], g[:, 2],
                        np.concatenate(self._b1) if self._b1 else np.zeros(0, np.complex128),
                        np.concatenate(self._adc))


def sinc_pulse(n: int, dt: float, flip_deg: float, tbw: float = 4.0, phase: float = 0.0) -> np.ndarray:
    """Hann-windowed sinc RF samples (one per step) whose hard-pulse flip
    angle γ Σ|B1| Δt equals ``flip_deg``. Returns complex B1 in tesla."""
    tc = (np.arange(n) + 0.5) / n - 0.5
    shape = np.sinc(tbw * tc) * (0.5 + 0.5 * np.cos(2.0 * np.pi * tc))
    amp = np.deg2rad(flip_deg) / (GAMMA * dt * shape.sum())
    return amp * shape * np.exp(1j * phase)


def hard_pulse_b1(flip_rad: float, duration: float, phase: float = 0.0) -> complex:
    """Constant B1 (tesla) giving rotation angle ``flip_rad`` in ``duration``
    on resonance, about the axis at angle ``phase`` from x in the xy plane."""
    return complex(flip_rad / (GAMMA * duration) * np.exp(1j * phase))


# --------------------------------------------------------------------------
# smooth off-resonance field
# --------------------------------------------------------------------------

def _smooth_field(rng, coords: np.ndarray, extent: float, std_hz: float,
                  n_bumps: int = 16, sigma: float = 0.04) -> np.ndarray:
    """Δω (rad/s) as a sum of Gaussian bumps, rescaled to a given std in Hz."""
    dim = coords.shape[1]
    centres = rng.uniform(-extent / 2, extent / 2, size=(n_bumps, dim))
    weights = rng.standard_normal(n_bumps)
    f = np.zeros(coords.shape[0])
    for c, w in zip(centres, weights):
        r2 = np.sum((coords - c[None, :]) ** 2, axis=1)
        f += w * np.exp(-r2 / (2 * sigma ** 2))
    f = f - f.mean()
    sd = f.std()
    if sd > 0:
        f *= std_hz / sd
    return 2.0 * np.pi * f


# --------------------------------------------------------------------------
# Workload 1: 32x32 grid phantom, spoiled GRE, uniform 10 us grid
# --------------------------------------------------------------------------

def gre_grid_phantom(n: int = 32, fov: float = 0.2, seed: int = 1001) -> Phantom:
    rng = np.random.Generator(np.random.PCG64(seed))
    c = (np.arange(n) - n // 2) * (fov / n)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    m = n * n
    return Phantom(x=xx.ravel(), y=yy.ravel(), z=np.zeros(m),
                   pd=rng.uniform(0.0, 1.0, m), t1=rng.uniform(0.2, 2.0, m),
                   t2=rng.uniform(0.02, 0.2, m), dw=np.zeros(m))


def spoiled_gre(n: int = 32, fov: float = 0.2, tr: float = 10e-3, dt: float = 10e-6,
                flip_deg: float = 30.0, rf_steps: int = 100, n_tr: Optional[int] = None,
                rf_spoil_deg: float = 117.0) -> Sequence:
    """Cartesian spoiled gradient echo on a uniform ``dt`` grid: per TR a
    Hann-sinc RF (with quadratic RF-spoiling phase), prephaser + phase encode,
    an ``n``-sample readout, rewinder + spoiler (2 cycles across the FOV),
    then free precession to the end of the TR."""
    n_tr = n if n_tr is None else n_tr
    per_tr = int(round(tr / dt))
    dk = 1.0 / fov
    ramp, flat = 10, 30
    b = SequenceBuilder()
    for j in range(n_tr):
        t0 = b.t
        ph = np.deg2rad(rf_spoil_deg) * j * (j + 1) / 2.0
        b.steps(rf_steps, dt, b1=sinc_pulse(rf_steps, dt, flip_deg, phase=ph))
        ky = ((j % n) - n // 2) * dk
        # readout ramp adds ramp/2 samples of moment; first sample lands at -n/2
        kx_pre = -(n // 2 + 1 + ramp / 2) * dk
        b.trapezoid([kx_pre, ky, 0.0], ramp, flat, dt)
        g_read = dk / (GAMMA_BAR * dt)
        b.steps(ramp, dt, [g_read, 0, 0])
        b.steps(n, dt, adc=True)
        b.steps(ramp, dt, [0, 0, 0])
        b.trapezoid([2.0 * dk, -ky, 0.0], ramp, flat, dt)
        used = int(round((b.t - t0) / dt))
        b.steps(per_tr - used, dt)
    return b.build()


# --------------------------------------------------------------------------
# Workload 2: 512x512 ellipse phantom, single-shot EPI
# --------------------------------------------------------------------------

def ellipse_phantom(n: int = 512, fov: float = 0.256, n_ellipses: int = 10,
                    df_std_hz: float = 20.0, seed: int = 1002) -> Phantom:
    rng = np.random.Generator(np.random.PCG64(seed))
    c = (np.arange(n) - n // 2) * (fov / n)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    x, y = xx.ravel(), yy.ravel()
    m = x.shape[0]
    pd = np.zeros(m)
    t1 = np.full(m, 1.0)
    t2 = np.full(m, 0.1)
    s = fov / 0.256
    head = (x / (0.09 * s)) ** 2 + (y / (0.11 * s)) ** 2 <= 1.0
    pd[head], t1[head], t2[head] = 0.8, 0.8, 0.08
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(-0.08 * s, 0.08 * s, 2)
        a, bb = rng.uniform(0.01 * s, 0.06 * s, 2)
        th = rng.uniform(0, np.pi)
        xr = (x - cx) * np.cos(th) + (y - cy) * np.sin(th)
        yr = -(x - cx) * np.sin(th) + (y - cy) * np.cos(th)
        inside = (xr / a) ** 2 + (yr / bb) ** 2 <= 1.0
        pd[inside] = rng.uniform(0.5, 1.0)
        t1[inside] = rng.uniform(0.3, 2.0)
        t2[inside] = rng.uniform(0.03, 0.3)
    dw = _smooth_field(rng, np.stack([x, y], axis=1), fov, df_std_hz)
    return Phantom(x=x, y=y, z=np.zeros(m), pd=pd, t1=t1, t2=t2, dw=dw)


def epi(n_read: int = 128, n_lines: int = 128, fov: float = 0.256, dwell: float = 4e-6,
        rf_dt: float = 4e-6, rf_steps: int = 500, flip_deg: float = 90.0,
        blip_steps: int = 8, kz: float = 0.0) -> Sequence:
    """Single-shot gradient-echo EPI: a Hann-sinc excitation, a prephaser to
    the k-space corner, then ``n_lines`` readouts of ``n_read`` samples with
    alternating readout gradient and a triangular phase blip between lines.
    ``kz`` (1/m) adds a partition-encoding moment to the prephaser (one
    partition of a 3-D EPI)."""
    dk = 1.0 / fov
    g_read = dk / (GAMMA_BAR * dwell)
    half = blip_steps // 2
    b = SequenceBuilder()
    b.steps(rf_steps, rf_dt, b1=sinc_pulse(rf_steps, rf_dt, flip_deg))
    kx_pre = -(n_read // 2 + 1 + half / 2) * dk
    ky_pre = -(n_lines // 2) * dk
    b.trapezoid([kx_pre, ky_pre, kz], 10, 30, dwell)
    b.steps(half, dwell, [g_read, 0, 0])
    g_blip = dk / (GAMMA_BAR * half * dwell)
    sign = 1.0
    for line in range(n_lines):
        b.steps(n_read, dwell, adc=True)
        if line + 1 < n_lines:
            b.steps(half, dwell, [0.0, g_blip, 0.0])
            b.steps(half, dwell, [-sign * g_read, 0.0, 0.0])
            sign = -sign
    b.steps(half, dwell, [0, 0, 0])
    return b.build()


# --------------------------------------------------------------------------
# Workload 3: 128^3 ellipsoid phantom, multi-shot spin echo
# --------------------------------------------------------------------------

def ellipsoid_phantom(n: int = 128, fov: float = 0.256, df_std_hz: float = 50.0,
                      seed: int = 1003) -> Phantom:
    rng = np.random.Generator(np.random.PCG64(seed))
    c = (np.arange(n) - n // 2) * (fov / n)
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    r = fov / 2
    inside = (xx / r) ** 2 + (yy / r) ** 2 + (zz / r) ** 2 <= 1.0
    x, y, z = xx[inside], yy[inside], zz[inside]
    m = x.shape[0]
    pd = np.full(m, 0.8)
    t1 = np.full(m, 1.0)
    t2 = np.full(m, 0.08)
    s = fov / 0.256
    inner = (x / (0.06 * s)) ** 2 + (y / (0.08 * s)) ** 2 + (z / (0.05 * s)) ** 2 <= 1.0
    pd[inner], t1[inner], t2[inner] = 1.0, 1.5, 0.15
    dw = _smooth_field(rng, np.stack([x, y, z], axis=1), fov, df_std_hz)
    return Phantom(x=x, y=y, z=z, pd=pd, t1=t1, t2=t2, dw=dw)


def spin_echo(n_shots: int = 64, n_read: int = 256, fov: float = 0.256, te: float = 20e-3,
              tr: float = 50e-3, rf_dt: float = 2e-6, rf_steps: int = 500,
              dwell: float = 4e-6, slice_thickness: float = 0.005, tbw: float = 4.0) -> Sequence:
    """Multi-shot slice-selective spin echo: per shot a 90°x sinc with slice
    select and rephaser, crushers around a 180°y sinc at TE/2, then one phase
    encoded ``n_read``-sample readout centred on TE. Gradients elsewhere are
    trapezoid vertices only (one step per corner)."""
    dk = 1.0 / fov
    t_rf = rf_steps * rf_dt
    g_ss = (tbw / t_rf) / (GAMMA_BAR * slice_thickness)
    g_read = dk / (GAMMA_BAR * dwell)
    tg = 100e-6  # ramp / flat step of a trapezoid corner
    crush = 2.0 / slice_thickness
    b = SequenceBuilder()
    for shot in range(n_shots):
        t_start = b.t
        # 90 degrees about x, centred at t_start + tg + t_rf/2
        b.steps(1, tg, [0, 0, g_ss])
        t90 = b.t + t_rf / 2
        b.steps(rf_steps, rf_dt, b1=sinc_pulse(rf_steps, rf_dt, 90.0, tbw))
        b.steps(1, tg, [0, 0, 0])
        # slice rephaser: half of the slice-select moment (the plateau only)
        area_ss = GAMMA_BAR * g_ss * (t_rf / 2 + tg / 2)
        amp = -area_ss / (GAMMA_BAR * 2 * tg)
        b.steps(1, tg, [0, 0, amp]).steps(1, tg).steps(1, tg, [0, 0, 0])
        # 180 degrees about y at TE/2 with crushers on both sides
        t180 = t90 + te / 2
        amp_c = crush / (GAMMA_BAR * 2 * tg)
        b.idle_until(t180 - t_rf / 2 - 4 * tg)
        b.steps(1, tg, [0, 0, amp_c]).steps(1, tg).steps(1, tg, [0, 0, 0])
        b.steps(1, tg, [0, 0, g_ss])
        b.steps(rf_steps, rf_dt, b1=sinc_pulse(rf_steps, rf_dt, 180.0, tbw, phase=np.pi / 2))
        b.steps(1, tg, [0, 0, 0])
        b.steps(1, tg, [0, 0, amp_c]).steps(1, tg).steps(1, tg, [0, 0, 0])
        # readout centred on TE: sample n_read/2 at t90 + te
        ky = (shot - n_shots // 2) * dk
        t_first = t90 + te - (n_read // 2) * dwell  # time of sample 0
        t_flat = t_first - dwell
        kx_pre = -(n_read // 2 + 1) * dk - GAMMA_BAR * g_read * tg / 2
        amp_pre = np.array([kx_pre, ky, 0.0]) / (GAMMA_BAR * 2 * tg)
        b.idle_until(t_flat - 4 * tg)
        b.steps(1, tg, amp_pre).steps(1, tg).steps(1, tg, [0, 0, 0])
        b.steps(1, tg, [g_read, 0, 0])
        b.steps(n_read, dwell, adc=True)
        b.steps(1, tg, [0, 0, 0])
        # spoiler, then wait for the next shot
        b.steps(1, tg, [2 * amp_pre[0], 0, amp_c]).steps(1, tg).steps(1, tg, [0, 0, 0])
        b.idle_until(t_start + tr)
    return b.build()


# --------------------------------------------------------------------------
# Workload 4: MRF dictionary (grouped isochromats), FISP train
# --------------------------------------------------------------------------

def mrf_dictionary_phantom(n_t1: int = 250, n_t2: int = 200, n_iso=(50, 400), voxel: float = 1e-3,
                           t1_range=(0.3, 2.5), t2_range=(0.04, 0.35), seed: int = 1004) -> Phantom:
    """One group of isochromats per (T1, T2) dictionary entry on a log grid.
    Group g has n_e ~ U{n_iso} spins at z_k = L (k + 1/2) / n_e - L/2 inside a
    voxel of length L (PD = 1 / n_e each, so a group's signal is the voxel
    average scaled to M0 = 1); x = y = 0, no off-resonance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t1s = np.geomspace(t1_range[0], t1_range[1], n_t1)
    t2s = np.geomspace(t2_range[0], t2_range[1], n_t2)
    T1, T2 = np.meshgrid(t1s, t2s, indexing="ij")
    T1, T2 = T1.ravel(), T2.ravel()
    counts = rng.integers(n_iso[0], n_iso[1] + 1, size=T1.size)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n = int(offs[-1])
    z = np.empty(n)
    pd = np.empty(n)
    for g, c in enumerate(counts):
        k = np.arange(c)
        z[offs[g]:offs[g + 1]] = voxel * (k + 0.5) / c - voxel / 2
        pd[offs[g]:offs[g + 1]] = 1.0 / c
    return Phantom(x=np.zeros(n), y=np.zeros(n), z=z, pd=pd, t1=np.repeat(T1, counts),
                   t2=np.repeat(T2, counts), dw=np.zeros(n), group_offsets=offs)


def mrf_fisp(n_tr: int = 1000, voxel: float = 1e-3, te: float = 3e-3, rf_dur: float = 100e-6,
             ti: float = 50e-3, seed: int = 1014) -> Sequence:
    """FISP fingerprinting train: an inversion (hard 180 deg) and TI, then
    n_tr TRs of a hard pulse with flip FA_j = 37.5 - 32.5 cos(2 pi j / 250)
    degrees (5..70), one ADC sample at TE, an unbalanced z gradient lobe whose
    moment dephases one full turn across the voxel, free precession to the
    end of the TR (TR_j ~ U[10, 15] ms)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    trs = rng.uniform(10e-3, 15e-3, n_tr)
    tg = 200e-6
    amp = (1.0 / voxel) / (GAMMA_BAR * 2 * tg)  # trapezoid of 1 ramp + 1 flat + 1 ramp step
    b = SequenceBuilder()
    b.steps(1, rf_dur, b1=hard_pulse_b1(np.pi, rf_dur))
    b.steps(1, ti - rf_dur)
    for j in range(n_tr):
        t0 = b.t
        fa = np.deg2rad(37.5 - 32.5 * np.cos(2 * np.pi * j / 250.0))
        b.steps(1, rf_dur, b1=hard_pulse_b1(fa, rf_dur))
        b.steps(1, te - rf_dur / 2, adc=True)            # TE from the pulse centre
        b.steps(1, tg, [0, 0, amp]).steps(1, tg).steps(1, tg, [0, 0, 0])
        b.idle_until(t0 + trs[j])
    return b.build()


# --------------------------------------------------------------------------
# named workloads (sizes of the benchmark configurations)
# --------------------------------------------------------------------------

def workload(name: str, scale: str = "full"):
    """Return ``(phantom, sequence)`` for a named workload.

    ``scale='full'`` gives the benchmark sizes; ``scale='small'`` a reduced
    version of the same construction (same shapes of waveforms and value
    distributions, fewer spins / lines) that the oracle finishes in seconds.
    """
    full = scale == "full"
    if name == "gre32":
        return gre_grid_phantom(), spoiled_gre()
    if name == "epi512":
        if full:
            return ellipse_phantom(), epi()
        return ellipse_phantom(n=48), epi(n_read=32, n_lines=16, rf_steps=100)
    if name == "se128":
        if full:
            return ellipsoid_phantom(), spin_echo()
        return ellipsoid_phantom(n=12), spin_echo(n_shots=4, n_read=32, rf_steps=100)
    if name == "mrf":
        if full:
            return mrf_dictionary_phantom(), mrf_fisp()
        return mrf_dictionary_phantom(n_t1=10, n_t2=8), mrf_fisp(n_tr=100)
    if name in ("paper_a", "paper_b"):
        # the paper's experiments (a)/(b): fully specified phantoms, single-shot
        # EPI (FOV 230 mm, 100 x 100, TE 100 ms, hard pulse) built from events
        from .discretize import discretize, epi_blocks, paper_phantom_a, paper_phantom_b
        ph = paper_phantom_a() if name == "paper_a" else paper_phantom_b()
        seq = discretize(epi_blocks() if full else epi_blocks(n=20, te=20e-3))
        if not full:
            ph = ph.subset(np.arange(0, ph.n, 4))
        return ph, seq
    if name == "paper_d":
        # the paper's experiment (d): a head at the phantoms' 1 mm resolution
        # (the ellipse head stands in for the BrainWeb brain), no
        # off-resonance, displaced along y by u_y = v_y t with v_y = 0.1 m/s,
        # single-shot EPI as in (a)/(b)
        from .discretize import discretize, epi_blocks
        ph = ellipse_phantom(n=230 if full else 58, fov=0.23)
        ph = ph.subset(np.flatnonzero(ph.pd > 0))
        ph.dw[:] = 0.0
        v = np.zeros((3, ph.n))
        v[1] = 0.1
        ph.velocity = v
        return ph, discretize(epi_blocks() if full else epi_blocks(n=20, te=20e-3))
    raise KeyError(name)


WORKLOADS = ("gre32", "epi512", "se128", "mrf")


def random_spins(n: int, seed: int, extent: float = 0.1, dim: int = 3,
                 dw_std: float = 2 * np.pi * 50.0) -> Phantom:
    """Unstructured spins with random properties (used by edge-case tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.uniform(-extent, extent, size=(3, n))
    if dim < 3:
        pos[dim:] = 0.0
    return Phantom(x=pos[0], y=pos[1], z=pos[2], pd=rng.uniform(0.2, 1.0, n),
                   t1=rng.uniform(0.1, 2.0, n), t2=rng.uniform(0.01, 0.3, n),
                   dw=rng.normal(0.0, dw_std, n))


def random_sequence(n_steps: int, seed: int, rf_frac: float = 0.3, adc_frac: float = 0.3,
                    dt_range=(1e-6, 50e-6), g_max: float = 0.03, b1_max: float = 2e-5) -> Sequence:
    """Unstructured sequence with random step lengths, gradient vertices, RF
    and ADC (used by edge-case tests). RF steps appear in runs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dt = rng.uniform(dt_range[0], dt_range[1], n_steps)
    g = rng.uniform(-g_max, g_max, size=(3, n_steps + 1))
    rf = np.zeros(n_steps, dtype=bool)
    i = 0
    while i < n_steps:
        run = int(rng.integers(1, 12))
        if rng.uniform() < rf_frac:
            rf[i:i + run] = True
        i += run
    b1 = np.where(rf, rng.uniform(0, b1_max, n_steps) * np.exp(1j * rng.uniform(0, 2 * np.pi, n_steps)), 0)
    adc = (rng.uniform(size=n_steps + 1) < adc_frac).astype(np.uint8)
    return Sequence(dt, g[0], g[1], g[2], b1, adc)
