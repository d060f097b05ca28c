"""GPU parity of moving phantoms (x(t) = x + v t) against the FP64 oracle.

Motion is the phantom's motion field u(x, t) of Section "Overview" with the
constant-velocity displacement of the paper's experiment (d). Same error
metric and tolerances as the static parity tests: FP32 1e-4, FP64 1e-9 of
the reference maximum.
"""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import (SequenceBuilder, hard_pulse_b1, random_sequence, random_spins,
                                             workload)

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL64 = 1e-9


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    yield s
    s.close()


def gpu_signal(sim, ph, seq, precision="fp32"):
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        out = sim.simulate(hp, hs, precision)
        sim.sync()
        return out.cpu().numpy()
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def rel_err(got, ref):
    scale = np.max(np.abs(ref))
    assert scale > 0
    return float(np.max(np.abs(got - ref)) / scale)


def moving(ph, seed, vmax=0.5):
    rng = np.random.default_rng(seed)
    ph.velocity = rng.uniform(-vmax, vmax, (3, ph.n))
    return ph


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_paper_experiment_d_full_size(sim, precision):
    """Experiment (d): head phantom without off-resonance moving at
    v_y = 0.1 m/s, single-shot EPI (FOV 230 mm, 100 x 100, TE 100 ms), full
    size. The motion changes the signal well beyond the tolerance."""
    ph, seq = workload("paper_d", "full")
    ref = oracle.simulate(ph, seq)
    got = gpu_signal(sim, ph, seq, precision)
    assert rel_err(got, ref) < (TOL32 if precision == "fp32" else TOL64)
    if precision == "fp32":
        ph.velocity = None
        still = oracle.simulate(ph, seq)
        assert rel_err(still, ref) > 100 * TOL32
        info = sim.launch_info()
        assert info["spins_per_thread"] == 2 and info["grid"] >= 148


@pytest.mark.parametrize("seed,n", [(1, 1), (2, 33), (3, 257), (4, 4099)])
def test_random_moving_spins(sim, seed, n):
    ph = moving(random_spins(n, seed=seed), seed + 50, vmax=1.0)
    seq = random_sequence(700, seed=seed + 100)
    ref = oracle.simulate(ph, seq)
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        assert rel_err(gpu_signal(sim, ph, seq, prec), ref) < tol, (seed, n, prec)


@pytest.mark.parametrize("name", ["epi512", "se128", "gre32"])
def test_workloads_with_motion(sim, name):
    """The static workloads' sequences with moving spins: long EPI readouts
    (quadratic per-sample phase), spin echoes over ~0.3 s and the 32,000-step
    GRE (late absolute times, so K1.v spans many turns)."""
    ph, seq = workload(name, "small" if name != "gre32" else "full")
    ph = moving(ph, 7, vmax=0.3)
    ref = oracle.simulate(ph, seq)
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        assert rel_err(gpu_signal(sim, ph, seq, prec), ref) < tol, prec


def test_zero_velocity_matches_static_path(sim):
    """A phantom moving at v = 0 runs the motion kernel and agrees with the
    static kernel; removing the motion goes back to the static kernel."""
    ph, seq = workload("epi512", "small")
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        still = sim.simulate(hp, hs).cpu().numpy()
        assert sim.launch_info()["spins_per_thread"] == 4
        koma.koma_phantom_set_motion(sim.ctx, hp, np.zeros((3, ph.n)))
        mov = sim.simulate(hp, hs).cpu().numpy()
        assert sim.launch_info()["spins_per_thread"] == 2
        assert rel_err(mov, still) < 1e-5
        koma.koma_phantom_set_motion(sim.ctx, hp, None)
        back = sim.simulate(hp, hs).cpu().numpy()
        assert np.array_equal(back, still)
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def test_moving_grouped_phantom(sim):
    """Groups of moving spins (each group's signal separately)."""
    ph = moving(random_spins(600, seed=31), 32)
    ph.group_offsets = np.array([0, 5, 5, 300, 301, 600])
    seq = random_sequence(400, seed=33)
    ref = oracle.simulate(ph, seq)
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        got = gpu_signal(sim, ph, seq, prec)
        assert got.shape == (5, seq.n_adc)
        assert np.all(got[1] == 0)
        for g in (0, 2, 3, 4):
            assert np.max(np.abs(got[g] - ref[g])) < tol * np.max(np.abs(ref[g])), (g, prec)


def test_fast_motion_and_soft_pulse(sim):
    """Spins at up to 3 m/s through a slice-selective soft pulse (RF steps
    see the midpoint position; the series path's bound includes the motion)
    and a readout with 128-sample runs."""
    b = SequenceBuilder()
    b.steps(1, 1e-6, [0.0, 0.0, 0.01])
    b.steps(100, 4e-6, b1=hard_pulse_b1(np.pi / 2, 400e-6, 0.3))
    b.steps(10, 20e-6, [0.008, 0.0, -0.01])
    b.steps(300, 4e-6, [0.008, 0.0, 0.0], adc=True)
    seq = b.build()
    ph = moving(random_spins(2000, seed=41, extent=0.05), 42, vmax=3.0)
    ref = oracle.simulate(ph, seq)
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        assert rel_err(gpu_signal(sim, ph, seq, prec), ref) < tol, prec


def test_motion_errors(sim):
    ph = random_spins(10, seed=1)
    hp = sim.upload_phantom(ph)
    try:
        bad = np.zeros((3, 10))
        bad[1, 4] = np.inf
        with pytest.raises(koma.KomaError) as e:
            koma.koma_phantom_set_motion(sim.ctx, hp, bad)
        assert e.value.status == koma.KOMA_E_INVALID
        import torch
        hs = sim.upload_sequence(random_sequence(30, seed=2))
        koma.koma_phantom_set_motion(sim.ctx, hp, np.ones((3, 10)))
        out = torch.zeros((1, koma.koma_sequence_n_adc(hs)), dtype=torch.complex128, device="cuda")
        with pytest.raises(koma.KomaError) as e:
            koma.koma_simulate_static(sim.ctx, hp, hs, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert e.value.status == koma.KOMA_E_INVALID
        koma.koma_sequence_free(hs)
    finally:
        koma.koma_phantom_free(hp)
