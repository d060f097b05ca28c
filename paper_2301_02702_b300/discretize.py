"""Sequence-aware time stepping: events -> discretised sequence.

The paper's simulator computes the time points a sequence needs instead of a
uniform grid (Section "Simulation blocks, Regime Switching, and
Sequence-Aware Time Stepping"): with piecewise-linear gradients the
precession phase is exact when integrated by the trapezoid rule over the
gradient's vertices, with piecewise-constant RF the excitation rotation is
exact per RF sample, and intermediate points are only needed for the ADC
samples (and, optionally, at most every ``dt`` to bound the step, and every
``dt_rf`` inside RF pulses). This module builds that discretisation from a
list of blocks of events and returns the arrays ``koma_sequence_upload``
takes (``workloads.Sequence``).

Events of a block (times relative to the block start, SI units):

* ``Trap(amp, rise, flat, fall, delay)``: trapezoid gradient on one axis;
* ``Arb(samples, raster, delay)``: gradient through ``samples`` at times
  ``delay + i * raster`` (linear in between, zero outside);
* ``RF(samples, dwell, delay)``: complex B1 (T), ``samples[i]`` held over
  ``[delay + i dwell, delay + (i+1) dwell)``;
* ``ADC(n, dwell, delay)``: samples at ``delay + (k + 1/2) dwell``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence as Seq, Union

import numpy as np

from .workloads import Sequence


@dataclasses.dataclass
class Trap:
    amp: float
    rise: float
    flat: float
    fall: float
    delay: float = 0.0

    def vertices(self):
        t = np.array([0.0, self.rise, self.rise + self.flat, self.rise + self.flat + self.fall]) + self.delay
        return t, np.array([0.0, self.amp, self.amp, 0.0])

    @property
    def end(self):
        return self.delay + self.rise + self.flat + self.fall

    @property
    def area(self):
        return self.amp * (self.flat + 0.5 * (self.rise + self.fall))


@dataclasses.dataclass
class Arb:
    samples: np.ndarray
    raster: float
    delay: float = 0.0

    def vertices(self):
        s = np.asarray(self.samples, dtype=np.float64)
        return self.delay + self.raster * np.arange(s.size), s

    @property
    def end(self):
        return self.delay + self.raster * (len(self.samples) - 1)


@dataclasses.dataclass
class RF:
    samples: np.ndarray
    dwell: float
    delay: float = 0.0

    @property
    def end(self):
        return self.delay + self.dwell * len(self.samples)


@dataclasses.dataclass
class ADC:
    n: int
    dwell: float
    delay: float = 0.0

    def times(self):
        return self.delay + (np.arange(self.n) + 0.5) * self.dwell

    @property
    def end(self):
        return self.delay + self.n * self.dwell


Grad = Optional[Union[Trap, Arb]]


@dataclasses.dataclass
class Block:
    gx: Grad = None
    gy: Grad = None
    gz: Grad = None
    rf: Optional[RF] = None
    adc: Optional[ADC] = None
    duration: Optional[float] = None

    def length(self) -> float:
        ends = [e.end for e in (self.gx, self.gy, self.gz, self.rf, self.adc) if e is not None]
        d = max(ends) if ends else 0.0
        return max(d, self.duration or 0.0)


def _grad_at(g: Grad, t: np.ndarray) -> np.ndarray:
    if g is None:
        return np.zeros_like(t)
    tv, gv = g.vertices()
    return np.interp(t, tv, gv, left=0.0, right=0.0)


def discretize(blocks: Seq[Block], dt: float = 1e-3, dt_rf: Optional[float] = None,
               tol: float = 1e-12) -> Sequence:
    """Time points of ``blocks`` played back to back, and the per-step
    gradient vertices, RF values and ADC mask at them.

    ``dt``: longest step outside RF pulses (the paper's Δt); ``dt_rf``: longest
    step inside RF pulses (Δt_rf; None: the RF samples' own dwell)."""
    pts: List[np.ndarray] = []
    adc_t: List[np.ndarray] = []
    rf_spans = []  # (t0, t1, rf, block start)
    t0 = 0.0
    g_at_end = np.zeros(3)
    for bi, b in enumerate(blocks):
        dur = b.length()
        if dur <= 0:
            raise ValueError(f"block {bi} has no duration")
        # continuity of the gradient waveform across block boundaries
        g_start = np.array([_grad_at(g, np.array([0.0]))[0] for g in (b.gx, b.gy, b.gz)])
        if np.max(np.abs(g_start - g_at_end)) > 1e-9:
            raise ValueError(f"gradient jumps at the start of block {bi}")
        g_at_end = np.array([_grad_at(g, np.array([dur]))[0] for g in (b.gx, b.gy, b.gz)])
        local = [np.array([0.0, dur])]
        for g in (b.gx, b.gy, b.gz):
            if g is not None:
                tv, _ = g.vertices()
                local.append(tv[(tv >= 0) & (tv <= dur)])
        if b.rf is not None:
            local.append(b.rf.delay + b.rf.dwell * np.arange(len(b.rf.samples) + 1))
            rf_spans.append((t0 + b.rf.delay, t0 + b.rf.end, b.rf, t0))
        if b.adc is not None:
            at = b.adc.times()
            local.append(at)
            adc_t.append(t0 + at)
        pts.append(t0 + np.concatenate(local))
        t0 += dur
    t = np.unique(np.round(np.concatenate(pts) / tol) * tol)
    # subdivide long steps: dt_rf inside RF pulses, dt elsewhere
    out = [t[:1]]
    for a, b_ in zip(t[:-1], t[1:]):
        mid = 0.5 * (a + b_)
        in_rf = any(s0 <= mid < s1 for s0, s1, _, _ in rf_spans)
        lim = (dt_rf if dt_rf is not None else np.inf) if in_rf else dt
        k = int(np.ceil((b_ - a) / lim - 1e-9)) if np.isfinite(lim) else 1
        k = max(k, 1)
        out.append(a + (b_ - a) * np.arange(1, k + 1) / k)
    t = np.concatenate(out)
    steps = np.diff(t)
    if np.any(steps <= 0):
        raise ValueError("non-increasing time points")
    # gradient vertices: sum of each block's waveform at its local time
    g = np.zeros((3, t.size))
    starts = np.concatenate([[0.0], np.cumsum([b.length() for b in blocks])])
    for bi, b in enumerate(blocks):
        lo, hi = starts[bi], starts[bi + 1]
        m = (t >= lo - tol) & (t <= hi + tol)
        for d, gg in enumerate((b.gx, b.gy, b.gz)):
            if gg is not None:
                g[d, m] = _grad_at(gg, t[m] - lo)
    # RF: the value held at each step's midpoint
    b1 = np.zeros(steps.size, dtype=np.complex128)
    mids = 0.5 * (t[:-1] + t[1:])
    for s0, s1, rf, tb in rf_spans:
        m = (mids >= s0) & (mids < s1)
        i = np.floor((mids[m] - tb - rf.delay) / rf.dwell).astype(np.int64)
        b1[m] = np.asarray(rf.samples, dtype=np.complex128)[np.clip(i, 0, len(rf.samples) - 1)]
    # ADC: the time points at the sample times
    adc = np.zeros(t.size, dtype=np.uint8)
    if adc_t:
        at = np.concatenate(adc_t)
        idx = np.searchsorted(t, at - tol)
        if np.any(idx >= t.size) or np.any(np.abs(t[np.minimum(idx, t.size - 1)] - at) > 10 * tol):
            raise ValueError("an ADC sample fell between time points")
        adc[idx] = 1
    return Sequence(steps, g[0], g[1], g[2], b1, adc)


# --------------------------------------------------------------------------
# Sequences of the paper's comparison experiments, built from events
# --------------------------------------------------------------------------

def epi_blocks(fov: float = 0.23, n: int = 100, te: float = 100e-3, dwell: float = 4e-6,
               rf_dur: float = 100e-6, flip_deg: float = 90.0, ramp: float = 40e-6,
               gamma_bar: float = 42.577478518e6) -> List[Block]:
    """Single-shot gradient-echo EPI with a hard excitation (the paper's
    experiments (a)-(d): FOV 230 mm, 100 x 100 matrix, TE 100 ms, hard RF):
    sample k of line l sits at k-space ((k - n/2) dk, (l - n/2) dk), mirrored
    in x on odd lines, with the centre of k-space at TE after the pulse
    centre. Readout lobes are trapezoids with the ADC on their flat part; the
    phase blip sits in each lobe's ramp-down."""
    dk = 1.0 / fov
    b1 = np.deg2rad(flip_deg) / (2 * np.pi * gamma_bar * rf_dur)
    g_read = dk / (gamma_bar * dwell)
    t_line = n * dwell
    pre_flat = 10 * ramp
    area_x = -(n / 2 + 0.5) * dk - gamma_bar * g_read * ramp / 2  # turns/m
    area_y = -(n // 2) * dk
    pre = Block(gx=Trap(area_x / (gamma_bar * (pre_flat + ramp)), ramp, pre_flat, ramp),
                gy=Trap(area_y / (gamma_bar * (pre_flat + ramp)), ramp, pre_flat, ramp))
    t_lobe = t_line + 2 * ramp
    t_centre = rf_dur + pre.length() + (n // 2) * t_lobe + ramp + (n // 2 + 0.5) * dwell  # without the wait
    wait = te + rf_dur / 2 - t_centre
    blocks = [Block(rf=RF(np.array([b1 + 0j]), rf_dur))]
    if wait > 0:
        blocks.append(Block(duration=wait))
    blocks.append(pre)
    blip_amp = dk / (gamma_bar * ramp / 2)
    sign = 1.0
    for line in range(n):
        gy = Trap(blip_amp, ramp / 2, 0.0, ramp / 2, delay=ramp + t_line) if line + 1 < n else None
        blocks.append(Block(gx=Trap(sign * g_read, ramp, t_line, ramp), gy=gy, adc=ADC(n, dwell, delay=ramp)))
        sign = -sign
    return blocks


def paper_phantom_a(res: float = 1e-3):
    """Experiment (a): a column of spins in four 50 mm segments with
    M0 = [1, 0.5, 1, 0.5] and T1 = T2 = [100, 50, 100, 50] ms."""
    from .workloads import Phantom
    l = 0.05
    y = np.arange(-2 * l + res / 2, 2 * l, res)
    seg = np.clip(((y + 2 * l) // l).astype(int), 0, 3)
    m0 = np.array([1.0, 0.5, 1.0, 0.5])[seg]
    t = np.array([100e-3, 50e-3, 100e-3, 50e-3])[seg]
    nn = y.size
    return Phantom(x=np.zeros(nn), y=y, z=np.zeros(nn), pd=m0, t1=t, t2=t.copy(), dw=np.zeros(nn))


def paper_phantom_b(res: float = 1e-3):
    """Experiment (b): two concentric circles, R = 50 mm and r = 25 mm,
    M0 = 1, T1 = T2 = 100 ms outside and 50 ms inside, and a 200 rad/s
    frequency offset in the inner circle."""
    from .workloads import Phantom
    c = np.arange(-0.05 + res / 2, 0.05, res)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    rr = np.hypot(xx, yy)
    m = rr <= 0.05
    inner = rr[m] <= 0.025
    x, y = xx[m], yy[m]
    t = np.where(inner, 50e-3, 100e-3)
    return Phantom(x=x, y=y, z=np.zeros(x.size), pd=np.ones(x.size), t1=t, t2=t.copy(),
                   dw=np.where(inner, 200.0, 0.0))
