"""Sequence-aware time stepping (events -> discretised sequence)."""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300.discretize import ADC, RF, Arb, Block, Trap, discretize, epi_blocks
from paper_2301_02702_b300.workloads import GAMMA_BAR, Phantom


def moments(seq):
    """gammabar * integral of G over each step (trapezoid on vertices)."""
    g = np.stack([seq.gx, seq.gy, seq.gz])
    return GAMMA_BAR * 0.5 * (g[:, :-1] + g[:, 1:]) * seq.dt


def test_trapezoids_need_only_their_corners():
    blocks = [Block(gx=Trap(0.02, 1e-4, 3e-4, 2e-4), gz=Trap(-0.01, 2e-4, 0.0, 2e-4, delay=1e-4)),
              Block(gy=Arb(np.array([0.0, 0.004, 0.001, 0.0]), 1e-4))]
    seq = discretize(blocks, dt=1.0)
    assert seq.n_steps <= 8
    m = moments(seq).sum(axis=1)
    assert m[0] == pytest.approx(GAMMA_BAR * blocks[0].gx.area, rel=1e-12)
    assert m[2] == pytest.approx(GAMMA_BAR * blocks[0].gz.area, rel=1e-12)
    assert m[1] == pytest.approx(GAMMA_BAR * 1e-4 * (0.004 + 0.001), rel=1e-12)


def test_step_limits_and_rf_area():
    rf = RF(np.array([1e-6, 2e-6 + 1e-6j, 3e-6]), 1e-4, delay=5e-5)
    blocks = [Block(rf=rf, gz=Trap(0.01, 1e-4, 3e-4, 1e-4)), Block(duration=5e-3), Block(adc=ADC(16, 1e-5))]
    seq = discretize(blocks, dt=2e-4, dt_rf=1e-5)
    rf_steps = seq.b1 != 0
    assert np.max(seq.dt[rf_steps]) <= 1e-5 + 1e-15
    assert np.max(seq.dt[~rf_steps]) <= 2e-4 + 1e-15
    assert np.sum(seq.b1 * seq.dt) == pytest.approx(np.sum(rf.samples) * rf.dwell, rel=1e-12)
    assert seq.n_adc == 16


def test_jump_in_gradient_is_rejected():
    with pytest.raises(ValueError):
        discretize([Block(gx=Arb(np.array([0.0, 0.01]), 1e-4)), Block(gx=Arb(np.array([0.0, 0.0]), 1e-4))])


def test_epi_from_events_samples_the_dft_grid():
    """A 90x hard pulse, no relaxation or off-resonance, then the event-built
    EPI: line l, sample k equals i * DFT of the PD image at
    ((k - n/2), (l - n/2)) / FOV, mirrored in x on odd lines."""
    n, fov = 16, 0.2
    rng = np.random.default_rng(3)
    img = rng.uniform(0, 1, (n, n))
    c = (np.arange(n) - n // 2) * (fov / n)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    ph = Phantom(x=xx.ravel(), y=yy.ravel(), z=np.zeros(n * n), pd=img.ravel(),
                 t1=np.full(n * n, np.inf), t2=np.full(n * n, np.inf), dw=np.zeros(n * n))
    seq = discretize(epi_blocks(fov=fov, n=n, te=5e-3))
    sig = oracle.simulate(ph, seq).reshape(n, n)
    F = 1j * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(img)))
    expect = F.copy()
    expect[1::2] = F[1::2, ::-1]
    assert np.max(np.abs(sig - expect)) < 1e-9 * np.max(np.abs(F))
