"""GPU parity of the tensor-core readout (matrix form of ADC runs that share
their per-sample rotator) against the FP64 oracle.

The signal of such runs is sum_s E_s(r) z_s^l, evaluated as a complex matrix
product on the tensor cores in FP16 hi/lo operand pairs with FP32
accumulation; the oracle steps every sample. Same error metric and FP32
tolerance as the other parity tests (1e-4 of the reference maximum); the
readout on and off must agree far inside it.
"""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import SequenceBuilder, epi, random_sequence, random_spins, workload

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    yield s
    s.close()


def run(sim, ph, seq, mma=True):
    koma.koma_set_mma(sim.ctx, mma)
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        out = sim.simulate(hp, hs)
        sim.sync()
        return out.cpu().numpy(), sim.launch_info()
    finally:
        koma.koma_set_mma(sim.ctx, True)
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def rel_err(got, ref):
    scale = np.max(np.abs(ref))
    assert scale > 0
    return float(np.max(np.abs(got - ref)) / scale)


def head_like(n, seed, fov=0.23):
    """2-D spins inside the field of view with a smooth off-resonance."""
    ph = random_spins(n, seed=seed, extent=0.45 * fov, dim=2, dw_std=2 * np.pi * 20.0)
    return ph


@pytest.mark.parametrize("n_read,n_lines,n_spins,seed", [
    (128, 128, 3000, 1),   # the benchmark's readout: 2 groups of 64 full runs
    (100, 70, 1001, 2),    # ragged runs (100 samples), 35 runs a group
    (200, 150, 517, 3),    # lines split into 128 + 72 samples; 64 + 64 + ... runs, a short last group
    (64, 40, 1, 4),        # one spin
    (40, 60, 33, 5),       # spins not a multiple of 32
    (96, 130, 333, 6),     # 65 runs a direction: a last group of a single run
])
def test_epi_readouts_match_oracle(sim, n_read, n_lines, n_spins, seed):
    seq = epi(n_read=n_read, n_lines=n_lines, fov=0.23, rf_steps=100)
    info = koma.koma_sequence_plan(seq)
    assert info["n_mma_groups"] >= 2 and info["n_mma_runs"] == info["n_adc_runs"]
    ph = head_like(n_spins, seed)
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] >= 1 and li["kernels"] == 3
    assert rel_err(got, ref) < TOL32
    off, li_off = run(sim, ph, seq, mma=False)
    assert li_off["mma_grid"] == 0 and li_off["kernels"] == 2
    assert rel_err(off, ref) < TOL32
    assert rel_err(got, off) < 2e-5


def test_mixed_sequence_combines_both_sources(sim):
    """Readout lines that form groups next to runs that do not (a few lone
    samples and a short run at another gradient): each sample comes from the
    kernel that took it."""
    b = SequenceBuilder()
    b.steps(50, 4e-6, b1=2e-6)
    b.steps(10, 10e-6, [0.0, 0.004, 0.0])
    b.steps(5, 4e-6, [0.0, 0.0, 0.0])
    for line in range(12):
        b.steps(2, 4e-6, [0.01, 0.0, 0.0])
        b.steps(96, 4e-6, adc=True)
        b.steps(2, 4e-6, [0.0, 0.0, 0.0])
        b.steps(3, 4e-6, [0.0, 0.002, 0.0])
        b.steps(3, 4e-6, [0.0, 0.0, 0.0])
    b.steps(7, 4e-6, [0.003, 0.0, 0.001], adc=True)
    b.steps(1, 30e-6, adc=True)
    seq = b.build()
    info = koma.koma_sequence_plan(seq)
    assert info["n_mma_groups"] == 1 and 0 < info["n_mma_runs"] < info["n_adc_runs"]
    ph = random_spins(700, seed=9, extent=0.08)
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] >= 1
    assert rel_err(got, ref) < TOL32


@pytest.mark.parametrize("pd_scale", [1e-3, 1.0, 3e3])
def test_proton_density_scale(sim, pd_scale):
    """E is scaled by a power of two from the phantom's largest pd so its
    FP16 parts neither overflow nor lose their low bits; a spin of zero pd
    adds nothing."""
    seq = epi(n_read=64, n_lines=32, fov=0.2, rf_steps=50)
    ph = head_like(300, 11, fov=0.2)
    ph.pd = ph.pd * pd_scale
    ph.pd[::7] = 0.0
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] >= 1
    assert rel_err(got, ref) < TOL32


def test_fast_decay_and_wide_off_resonance(sim):
    """Short T2 (the rotator's magnitude falls far below 1 within a run) and
    off-resonance of several kHz (many turns per run)."""
    seq = epi(n_read=128, n_lines=16, fov=0.2, rf_steps=50)
    ph = random_spins(257, seed=21, extent=0.09, dim=2, dw_std=2 * np.pi * 3000.0)
    ph.t2 = np.full(ph.n, 2e-3)
    ref = oracle.simulate(ph, seq)
    got, _ = run(sim, ph, seq)
    assert rel_err(got, ref) < TOL32


def test_spin_echo_lines_across_rf(sim):
    """Cartesian spin-echo lines: one readout per repetition, all with the
    same rotator, separated by refocusing pulses (E of each line comes from
    the state after its own pulses)."""
    ph, seq = workload("se128", "full")
    info = koma.koma_sequence_plan(seq)
    assert info["n_mma_groups"] >= 1
    rng = np.random.default_rng(5)
    sub = ph.subset(rng.choice(ph.n, 1500, replace=False))
    ref = oracle.simulate(sub, seq)
    got, li = run(sim, sub, seq)
    assert li["mma_grid"] >= 1
    assert rel_err(got, ref) < TOL32


def test_deterministic_and_order_free(sim):
    """Two calls give the same bits; the readout's partial rows are summed in
    a fixed order."""
    seq = epi(n_read=128, n_lines=64, fov=0.23, rf_steps=100)
    ph = head_like(5000, 31)
    a, _ = run(sim, ph, seq)
    b, _ = run(sim, ph, seq)
    assert np.array_equal(a, b)


def test_grouped_and_moving_phantoms_do_not_use_it(sim):
    seq = epi(n_read=64, n_lines=32, fov=0.2, rf_steps=50)
    ph = head_like(200, 41, fov=0.2)
    ph.group_offsets = np.array([0, 120, 200])
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] == 0
    assert np.max(np.abs(got - ref)) < TOL32 * np.max(np.abs(ref))
    ph2 = head_like(200, 42, fov=0.2)
    ph2.velocity = np.zeros((3, ph2.n))
    ph2.velocity[1] = 0.1
    ref2 = oracle.simulate(ph2, seq)
    got2, li2 = run(sim, ph2, seq)
    assert li2["mma_grid"] == 0
    assert rel_err(got2, ref2) < TOL32


def test_full_size_benchmark_readout(sim):
    """The benchmark's full launch (262,144 spins, 128 x 128 EPI): all ADC
    runs on the tensor cores, checked on a random spin sample (the other
    spins' pd set to zero so the oracle computes only the sample)."""
    ph, seq = workload("epi512", "full")
    rng = np.random.default_rng(123)
    keep = rng.choice(ph.n, 1536, replace=False)
    pd = np.zeros(ph.n)
    pd[keep] = ph.pd[keep]
    ph.pd = pd
    ref = oracle.simulate(ph.subset(keep), seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] >= 100
    assert rel_err(got, ref) < TOL32


def test_graph_capture_with_readout(sim):
    import torch
    seq = epi(n_read=128, n_lines=32, fov=0.23, rf_steps=100)
    ph = head_like(4000, 51)
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        s = torch.cuda.Stream()
        out = torch.empty((1, seq.n_adc), dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(s):
            sim.simulate(hp, hs, out=out, stream=s)
        sim.sync(s)
        assert sim.launch_info()["mma_grid"] >= 1
        ref = out.clone()
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


def test_random_sequences_unaffected(sim):
    """Unstructured sequences form no groups and run as before."""
    seq = random_sequence(800, seed=61)
    assert koma.koma_sequence_plan(seq)["n_mma_groups"] == 0
    ph = random_spins(300, seed=62)
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] == 0
    assert rel_err(got, ref) < TOL32


def test_stage_timing_splits_the_bloch_time(sim):
    """koma_get_stage_timing splits koma_get_timing's Bloch time into the
    Bloch kernel and the readout; the readout is 0 when it does not run."""
    seq = epi(n_read=128, n_lines=32, fov=0.23, rf_steps=100)
    ph = head_like(3000, 71)
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        koma.koma_set_timing(sim.ctx, True)
        for mma in (True, False):
            koma.koma_set_mma(sim.ctx, mma)
            sim.simulate(hp, hs)
            sim.sync()
            b, m, r = koma.koma_get_stage_timing(sim.ctx)
            tb, tr = koma.koma_get_timing(sim.ctx)
            assert b > 0 and r > 0 and (m > 0.003 if mma else m < 0.003)
            assert abs((b + m) - tb) <= 0.005 and abs(r - tr) <= 0.005
    finally:
        koma.koma_set_timing(sim.ctx, False)
        koma.koma_set_mma(sim.ctx, True)
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def test_multi_shot_epi_groups_span_blocks(sim):
    """Four EPI shots of 30-degree excitations: each readout direction's group
    holds runs of four RF-separated blocks (four snapshot rows, magnetisation
    carried from shot to shot)."""
    one = epi(n_read=64, n_lines=16, fov=0.2, rf_steps=40, flip_deg=30.0)
    seq = one.concat(one).concat(one).concat(one)
    info = koma.koma_sequence_plan(seq)
    assert info["n_mma_groups"] == 2 and info["n_mma_runs"] == 64
    ph = head_like(777, 81, fov=0.2)
    ph.t1 = np.full(ph.n, 0.3)
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] >= 1
    assert rel_err(got, ref) < TOL32
    off, _ = run(sim, ph, seq, mma=False)
    assert rel_err(got, off) < 2e-5


@pytest.mark.parametrize("seed", range(8))
def test_random_readout_shapes(sim, seed):
    """Random EPI shapes: line lengths from 8 to 300 samples (runs of up to
    128, a short last run), 8 to 140 lines (groups of 64 runs and a short
    last group, down to a single run), random spin counts."""
    rng = np.random.default_rng(900 + seed)
    n_read = int(rng.integers(8, 301))
    n_lines = int(rng.integers(8, 141))
    n_read = max(n_read, -(-2048 // n_lines))  # enough samples for a group
    seq = epi(n_read=n_read, n_lines=n_lines, fov=0.2, rf_steps=int(rng.integers(1, 60)),
              flip_deg=float(rng.uniform(10, 90)))
    info = koma.koma_sequence_plan(seq)
    ph = head_like(int(rng.integers(1, 700)), 1000 + seed, fov=0.2)
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert (li["mma_grid"] > 0) == (info["n_mma_groups"] > 0)
    assert rel_err(got, ref) < TOL32, (n_read, n_lines, info)


@pytest.mark.parametrize("dim,df_hz,kz", [
    (2, 0.0, 0.0),      # x, y terms only
    (2, 40.0, 0.0),     # + off-resonance
    (3, 0.0, 37.0),     # + a z moment on every line (one partition of a 3-D EPI)
    (3, 40.0, -23.0),   # all four terms
])
def test_phase_term_instances(sim, dim, df_hz, kz):
    """The readout kernel is compiled per set of phase terms the phantom
    needs (z, off-resonance); each instance against the oracle."""
    seq = epi(n_read=64, n_lines=48, fov=0.2, rf_steps=40, kz=kz)
    ph = random_spins(700, seed=61 + dim, extent=0.09, dim=dim, dw_std=2 * np.pi * df_hz)
    if df_hz == 0.0:
        ph.dw = np.zeros(ph.n)
    ref = oracle.simulate(ph, seq)
    got, li = run(sim, ph, seq)
    assert li["mma_grid"] >= 1
    assert rel_err(got, ref) < TOL32
    off, _ = run(sim, ph, seq, mma=False)
    assert rel_err(got, off) < 2e-5
