"""GPU parity of repeated RF pulses taken by their maps.

A run of RF steps is one affine map of the magnetisation (the composition of
its steps' rotations, Eq. Rot_exc, and relaxations); for pulses that recur
unchanged the pre-pass kernel computes the map per spin and the Bloch kernel
applies it at every occurrence. These tests compare that path with the FP64
oracle (which steps every RF step) and with the stepped GPU path, on each
rotation path of the pre-pass (series of 1, 2 and 4 terms, the general path),
pulses longer than a record tile, pulses at t = 0, interleaved pulses, spins
without relaxation or proton density, and ragged spin counts.
"""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import SequenceBuilder, random_spins, sinc_pulse, workload

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    koma.koma_set_timing(s.ctx, True)
    yield s
    s.close()


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def run(sim, ph, seq, maps=True):
    """(signal, map pre-pass ms) of one FP32 simulation."""
    koma.koma_set_rf_maps(sim.ctx, maps)
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        out = sim.simulate(hp, hs, "fp32")
        sim.sync()
        return out.cpu().numpy(), koma.koma_get_map_timing(sim.ctx)
    finally:
        koma.koma_set_rf_maps(sim.ctx, True)
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def pulse_train(pulses, order, seed=0, lead_in=True):
    """Pulses (n, dt, b1, gradient) in `order`, each between gradient ramps,
    followed by a lobe whose area changes per occurrence and a short
    readout; lead_in=False starts the first pulse at t = 0."""
    rng = np.random.default_rng(seed)
    b = SequenceBuilder()
    for k, p in enumerate(order):
        n, dt, b1, g = pulses[p]
        if k > 0 or lead_in or np.any(np.asarray(g) != 0):
            b.steps(1, 20e-6, g)
        b.steps(n, dt, g, b1=b1)
        b.steps(1, 20e-6, [0.0, 0.0, 0.0])
        b.steps(2, 40e-6, [rng.uniform(-0.02, 0.02), 0.006 * (k % 5) - 0.012, 0.0])
        b.steps(1, 40e-6, [0.0, 0.0, 0.0])
        b.steps(24, 8e-6, [0.01, 0.0, 0.0], adc=True)
        b.steps(1, 8e-6, [0.0, 0.0, 0.0])
        b.steps(1, rng.uniform(1e-3, 4e-3))
    return b.build()


def check(sim, ph, seq, expect_maps=True):
    info = koma.koma_sequence_plan(seq)
    assert (info["n_rf_maps"] > 0) == expect_maps
    ref = oracle.simulate(ph, seq)
    got, t_maps = run(sim, ph, seq, maps=True)
    stepped, t_none = run(sim, ph, seq, maps=False)
    assert t_none == 0.0
    if expect_maps:
        assert t_maps > 0.0, "the map pre-pass did not run"
    e_maps, e_step = rel_err(got, ref), rel_err(stepped, ref)
    assert e_maps < TOL32, (e_maps, e_step)
    assert e_step < TOL32, e_step
    assert rel_err(got, stepped) < TOL32
    return e_maps


# (pulse half-angle regime, gradient during the pulse): with spins up to 4 cm
# from the centre, 0.01 T/m over 4 us steps reaches ~0.21 rad per step (four
# series terms), 0.05 T/m ~1.1 rad (the general path); without a gradient the
# off-resonance alone leaves small angles (one or two terms)
@pytest.mark.parametrize("g,flip,n_steps", [
    (0.0, 30.0, 40),      # no gradient: smallest angles
    (0.0, 180.0, 16),     # no gradient, large B1 per step
    (0.002, 90.0, 60),    # small slice gradient
    (0.01, 90.0, 300),    # series with four terms, longer than a record tile
    (0.05, 90.0, 120),    # general path (rsqrt and exact sine)
])
def test_repeated_pulse_paths(sim, g, flip, n_steps):
    ph = random_spins(1000, seed=31, extent=0.04)
    p = (n_steps, 4e-6, sinc_pulse(n_steps, 4e-6, flip), [0.0, 0.0, g])
    seq = pulse_train([p], [0] * 6, seed=2)
    check(sim, ph, seq)


def test_interleaved_pulses_from_t0(sim):
    """Two pulses A (90 deg, slice gradient) and B (180 deg about y) in the
    order A B A B A B A, the first A at t = 0; ragged spin counts."""
    a = (70, 4e-6, sinc_pulse(70, 4e-6, 90.0), [0.0, 0.0, 0.008])
    b = (90, 4e-6, sinc_pulse(90, 4e-6, 180.0, phase=np.pi / 2), [0.0, 0.0, 0.008])
    seq = pulse_train([a, b], [0, 1, 0, 1, 0, 1, 0], seed=3, lead_in=False)
    for n, seed in ((1, 1), (33, 2), (4099, 3)):
        check(sim, random_spins(n, seed=seed, extent=0.03), seq)


def test_maps_with_infinite_relaxation_and_zero_pd(sim):
    ph = random_spins(700, seed=10, extent=0.03)
    ph.t1[::3] = np.inf
    ph.t2[::4] = np.inf
    ph.pd[::5] = 0.0
    p = (50, 4e-6, sinc_pulse(50, 4e-6, 60.0), [0.0, 0.0, 0.01])
    check(sim, ph, pulse_train([p], [0] * 5, seed=4))


def test_only_repeated_pulses_take_maps(sim):
    """A pulse played once and one played twice are stepped; the one played
    four times takes its map, in the same launch."""
    a = (40, 4e-6, sinc_pulse(40, 4e-6, 45.0), [0.0, 0.0, 0.01])
    b = (30, 4e-6, sinc_pulse(30, 4e-6, 20.0), [0.0, 0.0, 0.01])
    c = (20, 4e-6, sinc_pulse(20, 4e-6, 70.0), [0.0, 0.0, 0.0])
    seq = pulse_train([a, b, c], [0, 1, 0, 2, 1, 0, 0], seed=5)
    info = koma.koma_sequence_plan(seq)
    assert (info["n_rf_maps"], info["n_rf_map_runs"]) == (1, 4)
    check(sim, random_spins(500, seed=6, extent=0.03), seq)


def test_se128_small_with_and_without_maps(sim):
    ph, seq = workload("se128", "small")
    check(sim, ph, seq)


def test_maps_deterministic_and_capturable(sim):
    import torch
    ph, seq = workload("se128", "small")
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        s = torch.cuda.Stream()
        out = torch.empty((1, seq.n_adc), dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(s):
            sim.simulate(hp, hs, out=out, stream=s)
        sim.sync(s)
        ref = out.clone()
        with torch.cuda.stream(s):
            sim.simulate(hp, hs, out=out, stream=s)
        sim.sync(s)
        assert torch.equal(out, ref), "two runs must be bitwise identical"
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            sim.simulate(hp, hs, out=out, stream=s)
        out.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        del g
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)
