"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Error metric (the paper compares signals normalised by the reference maximum):
rel_err = max_k |s_gpu[k] - s_ref[k]| / max_k |s_ref[k]|.
Tolerances: FP32 split-phase path 1e-4; FP64 path 1e-9 (FP64 rounding of a
different but mathematically equal formulation, over up to ~1e5 steps).
"""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import (WORKLOADS, Phantom, Sequence, SequenceBuilder, hard_pulse_b1,
                                             random_sequence, random_spins, workload)

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


@pytest.mark.parametrize("name", WORKLOADS)
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_workloads_small(sim, name, precision):
    ph, seq = workload(name, "small")
    ref = oracle.simulate(ph, seq)
    got = gpu_signal(sim, ph, seq, precision)
    assert got.shape == ref.shape
    err = rel_err(got, ref)
    assert err < (TOL32 if precision == "fp32" else TOL64), err


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_gre32_full_size(sim, precision):
    """The 1,024-spin, 32,000-step spoiled GRE at its full size."""
    ph, seq = workload("gre32", "full")
    ref = oracle.simulate(ph, seq)
    err = rel_err(gpu_signal(sim, ph, seq, precision), ref)
    assert err < (TOL32 if precision == "fp32" else TOL64), err


@pytest.mark.parametrize("name", ["epi512", "se128"])
def test_full_size_launch_sampled_spins(sim, name):
    """Full-size phantom in the benchmark's launch configuration; all spins
    but a random sample of 1,536 get PD = 0, so the signal is that sample's
    signal (linearity in PD) and the oracle computes it directly."""
    ph, seq = workload(name, "full")
    rng = np.random.default_rng(5)
    keep = np.sort(rng.choice(ph.n, 1536, replace=False))
    pd = np.zeros(ph.n)
    pd[keep] = ph.pd[keep]
    masked = Phantom(ph.x, ph.y, ph.z, pd, ph.t1, ph.t2, ph.dw)
    got = gpu_signal(sim, masked, seq)
    info = sim.launch_info()
    ref = oracle.simulate(ph.subset(keep), seq)
    err = rel_err(got, ref)
    assert err < TOL32, err
    assert info["grid"] >= 148


def test_random_sequences_and_ragged_sizes(sim):
    for seed, n in ((1, 1), (2, 31), (3, 33), (4, 257), (5, 1000), (6, 4099)):
        ph = random_spins(n, seed=seed)
        seq = random_sequence(700, seed=seed + 100)
        ref = oracle.simulate(ph, seq)
        for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
            err = rel_err(gpu_signal(sim, ph, seq, prec), ref)
            assert err < tol, (seed, n, prec, err)


def test_edge_cases(sim):
    ph = random_spins(70, seed=9)
    # ADC at t0 only: equilibrium has no transverse magnetisation
    seq0 = Sequence(np.zeros(0), np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(0, complex), np.ones(1, np.uint8))
    assert np.all(gpu_signal(sim, ph, seq0) == 0)
    # no ADC at all: an empty signal
    seq1 = random_sequence(50, seed=3, adc_frac=0.0)
    seq1.adc[:] = 0
    assert gpu_signal(sim, ph, seq1).shape == (1, 0)
    # no RF: nothing is ever excited
    seq2 = random_sequence(80, seed=4, rf_frac=0.0)
    assert np.all(gpu_signal(sim, ph, seq2) == 0)
    # infinite T1/T2 and zero PD spins mixed in
    ph3 = random_spins(100, seed=10)
    ph3.t1[::3] = np.inf
    ph3.t2[::4] = np.inf
    ph3.pd[::5] = 0.0
    seq3 = random_sequence(400, seed=11)
    ref = oracle.simulate(ph3, seq3)
    assert rel_err(gpu_signal(sim, ph3, seq3), ref) < TOL32
    # RF with every step sampled (samples inside an excitation block)
    b = SequenceBuilder()
    b.steps(50, 4e-6, b1=hard_pulse_b1(np.pi / 2, 200e-6, 0.3), adc=True)
    b.steps(30, 4e-6, [0.01, 0.0, 0.0], adc=True)
    seq4 = b.build()
    ref = oracle.simulate(ph3, seq4)
    assert rel_err(gpu_signal(sim, ph3, seq4), ref) < TOL32
    # large per-step angles (range reduction of the half angle)
    b = SequenceBuilder()
    b.steps(20, 50e-6, [0.0, 0.0, 0.2], b1=hard_pulse_b1(3.0, 1e-3))
    b.steps(10, 20e-6, adc=True)
    seq5 = b.build()
    ref = oracle.simulate(ph3, seq5)
    assert rel_err(gpu_signal(sim, ph3, seq5), ref) < TOL32



@pytest.mark.parametrize("theta", [0.004, 0.0125, 0.0175, 0.06, 0.095, 0.12, 0.4, 0.74])
@pytest.mark.parametrize("slice_grad", [False, True])
def test_rf_series_lengths(sim, theta, slice_grad):
    """The series path's length follows the RF run's largest half angle
    (terms to t^2 up to 0.015, to t^4 up to 0.1, to t^10 up to 0.754): pulses
    whose per-step half angle (plus the off-resonance and slice-gradient
    share) falls in each band and next to its edges, spins off resonance so
    the rotation axis is per spin."""
    n, dt = 40, 10e-6
    ph = random_spins(300, seed=77, extent=0.004, dim=3, dw_std=2 * np.pi * 40.0)
    b = SequenceBuilder()
    g_rf = [0.0, 0.0, 0.001] if slice_grad else None
    b.steps(n, dt, g_rf, b1=hard_pulse_b1(2 * n * theta, n * dt, 0.4))
    b.steps(4, dt, [0.0, 0.0, 0.0])
    b.steps(64, dt, [0.02, 0.0, 0.0], adc=True)
    seq = b.build()
    ref = oracle.simulate(ph, seq)
    assert rel_err(gpu_signal(sim, ph, seq), ref) < TOL32

def test_grouped_phantom(sim):
    ph = random_spins(300, seed=21)
    offs = np.array([0, 7, 7, 100, 101, 240, 300])
    seq = random_sequence(300, seed=22)
    phg = random_spins(300, seed=21)
    phg.group_offsets = offs
    ref = oracle.simulate(phg, seq)
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        got = gpu_signal(sim, phg, seq, prec)
        assert got.shape == (6, seq.n_adc)
        for g in range(6):
            if offs[g + 1] == offs[g]:
                assert np.all(got[g] == 0)
            else:
                assert np.max(np.abs(got[g] - ref[g])) < tol * np.max(np.abs(ref[g])), (g, prec)
    del ph


def test_deterministic_and_additive(sim):
    ph, seq = workload("epi512", "small")
    a = gpu_signal(sim, ph, seq)
    b = gpu_signal(sim, ph, seq)
    assert np.array_equal(a, b), "two runs must be bitwise identical"
    half = ph.n // 2
    s1 = gpu_signal(sim, ph.subset(np.arange(half)), seq)
    s2 = gpu_signal(sim, ph.subset(np.arange(half, ph.n)), seq)
    assert rel_err(s1 + s2, a) < TOL32


def test_simulate_host_matches_device_path(sim):
    ph, seq = workload("se128", "small")
    dev = gpu_signal(sim, ph, seq)
    host = koma.koma_simulate_host(sim.ctx, ph, seq, koma.KOMA_FP32_SPLITPHASE)
    assert np.array_equal(dev, host)


@pytest.mark.parametrize("case", ["se128", "epi512", "random"])
def test_host_call_equals_device_path_on_long_sequences(sim, case):
    """The host call builds the FP32 stream alone in parallel chunks, gathers
    it straight into the staging buffer and lets the readout and pulse plans
    mark it there; the device path's upload builds all three streams and
    concatenates them. Same records, so bitwise the same signal (long
    sequences: 40,000 to 81,920 steps, many chunks)."""
    if case == "random":
        ph, seq = random_spins(1500, seed=31), random_sequence(40_000, seed=32)
    else:
        ph, seq = workload(case, "small")[0], workload(case, "full")[1]
    dev = gpu_signal(sim, ph, seq)
    host = koma.koma_simulate_host(sim.ctx, ph, seq, koma.KOMA_FP32_SPLITPHASE)
    assert np.max(np.abs(dev)) > 0
    assert np.array_equal(dev, host)


def test_abi_errors(sim):
    bad = random_spins(10, seed=1)
    bad.t2[3] = 0.0
    with pytest.raises(koma.KomaError) as e:
        sim.upload_phantom(bad)
    assert e.value.status == koma.KOMA_E_INVALID
    bad = random_spins(10, seed=1)
    bad.x[2] = np.nan
    with pytest.raises(koma.KomaError):
        sim.upload_phantom(bad)
    small = koma.Simulator(0, mem_budget_bytes=1 << 16)
    try:
        with pytest.raises(koma.KomaError) as e:
            small.upload_phantom(random_spins(100000, seed=2))
        assert e.value.status == koma.KOMA_E_NOMEM
    finally:
        small.close()
    # objects of one context are rejected by another
    other = koma.Simulator(0)
    try:
        hp = other.upload_phantom(random_spins(10, seed=3))
        hs = sim.upload_sequence(random_sequence(10, seed=4))
        with pytest.raises(koma.KomaError) as e:
            sim.simulate(hp, hs)
        assert e.value.status == koma.KOMA_E_INVALID
        koma.koma_phantom_free(hp)
        koma.koma_sequence_free(hs)
    finally:
        other.close()


def test_mrf_dictionary_full_size_sampled_groups(sim):
    """The 50,000-entry dictionary (11.3 M isochromats) in one launch of the
    work-item kernel; 500 random groups checked against the oracle (groups are
    independent outputs, so each sampled row is compared exactly)."""
    from paper_2301_02702_b300.workloads import Phantom as Ph
    ph, seq = workload("mrf", "full")
    got = gpu_signal(sim, ph, seq)
    assert got.shape == (50000, seq.n_adc)
    rng = np.random.default_rng(11)
    groups = np.sort(rng.choice(ph.n_groups, 500, replace=False))
    idx = np.concatenate([np.arange(ph.group_offsets[g], ph.group_offsets[g + 1]) for g in groups])
    offs = np.concatenate([[0], np.cumsum(np.diff(ph.group_offsets)[groups])])
    sub = Ph(ph.x[idx], ph.y[idx], ph.z[idx], ph.pd[idx], ph.t1[idx], ph.t2[idx], ph.dw[idx], group_offsets=offs)
    ref = oracle.simulate(sub, seq)
    err = np.max(np.abs(got[groups] - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert np.max(err) < TOL32, np.max(err)


def test_grouped_kernel_deterministic_and_tuned(sim):
    import torch
    ph, seq = workload("mrf", "small")
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        a = sim.simulate(hp, hs).cpu().numpy()
        b = sim.simulate(hp, hs).cpu().numpy()
        assert np.array_equal(a, b)
        choice = sim.tune(hp, hs)
        assert choice["spins_per_thread"] in (2, 4, 8) and choice["block"] in (128, 256)
        assert choice["tile_records"] in (64, 128, 256)  # the sequence-tile length is tuned too
        c = sim.simulate(hp, hs).cpu().numpy()
        sim.sync()
        info = sim.launch_info()
        assert info["spins_per_thread"] == choice["spins_per_thread"]
        assert info["tile_records"] == choice["tile_records"]
        assert rel_err(c, a) < TOL32
        ref = oracle.simulate(ph, seq)
        assert rel_err(c, ref) < TOL32
        # ungrouped phantoms tune the Bloch kernel's spins per thread
        ph2, seq2 = workload("epi512", "small")
        hp2 = sim.upload_phantom(ph2)
        hs2 = sim.upload_sequence(seq2)
        ch2 = sim.tune(hp2, hs2)
        assert ch2["spins_per_thread"] in (2, 4)
        out = sim.simulate(hp2, hs2).cpu().numpy()
        assert rel_err(out, oracle.simulate(ph2, seq2)) < TOL32
        koma.koma_sequence_free(hs2)
        koma.koma_phantom_free(hp2)
        del torch
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


@pytest.mark.parametrize("name", ["paper_a", "paper_b"])
def test_paper_experiments_full_size(sim, name):
    """The paper's fully specified phantoms (experiments (a) column of four
    segments, (b) concentric circles with a 200 rad/s offset), single-shot
    EPI (FOV 230 mm, 100 x 100, TE 100 ms, hard pulse) built by the
    discretiser, at full size against the oracle."""
    ph, seq = workload(name, "full")
    ref = oracle.simulate(ph, seq)
    for prec, tol in (("fp32", TOL32), ("fp64", TOL64)):
        assert rel_err(gpu_signal(sim, ph, seq, prec), ref) < tol


def test_invalid_spin_reported_by_index(sim):
    """The device-side input check names the first offending spin."""
    bad = random_spins(5000, seed=7)
    bad.t1[4321] = -1.0
    bad.pd[4400] = -0.5
    with pytest.raises(koma.KomaError) as e:
        sim.upload_phantom(bad)
    assert e.value.status == koma.KOMA_E_INVALID
    assert "4321" in str(e.value)
    bad = random_spins(300, seed=8)
    bad.dw[299] = np.inf
    with pytest.raises(koma.KomaError) as e:
        sim.upload_phantom(bad)
    assert "299" in str(e.value)


def test_upload_cycles_reuse_memory(sim):
    """Upload / simulate / free cycles return the context's accounted memory
    to where it was and do not grow the device footprint (pooled blocks are
    reused)."""
    import torch
    ph, seq = workload("epi512", "small")
    first = None
    used = None
    for i in range(4):
        hp = sim.upload_phantom(ph)
        hs = sim.upload_sequence(seq)
        sim.simulate(hp, hs)
        sim.sync()
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)
        # what stays accounted is the context's partial-sum scratch
        if used is None:
            used = koma.koma_mem_used(sim.ctx)
        assert koma.koma_mem_used(sim.ctx) == used
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        if i == 1:
            first = free
        elif i > 1:
            assert free == first, "device footprint grew across identical cycles"


def test_tuned_shape_is_reused_by_other_phantoms(sim):
    """A shape tuned once is reused, without tuning, by another phantom of
    the same size bucket (the autotuner's cache on the context)."""
    ph, seq = workload("mrf", "small")
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        choice = sim.tune(hp, hs)
        # a second dictionary of the same shape: same sizes, other relaxation values
        ph2, _ = workload("mrf", "small")
        ph2.t2 = ph2.t2 * 1.1
        hp2 = sim.upload_phantom(ph2)
        try:
            got = sim.simulate(hp2, hs).cpu().numpy()
            info = sim.launch_info()
            assert (info["spins_per_thread"], info["block"], info["tile_records"]) == (
                choice["spins_per_thread"], choice["block"], choice["tile_records"])
            ref = oracle.simulate(ph2, seq)
            assert rel_err(got, ref) < TOL32
        finally:
            koma.koma_phantom_free(hp2)
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


@pytest.mark.parametrize("name", ["epi512", "mrf", "paper_d"])
def test_simulate_captures_into_a_cuda_graph(sim, name):
    """After one warm call (scratch and launch tables in place) a simulation
    is capturable: the Bloch, grouped and motion launches replay from a CUDA
    graph bitwise identical to the direct call."""
    import torch
    ph, seq = workload(name, "small")
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        s = torch.cuda.Stream()
        out = torch.empty((ph.n_groups, seq.n_adc), dtype=torch.complex128, device="cuda")
        with torch.cuda.stream(s):
            sim.simulate(hp, hs, out=out, stream=s)
        sim.sync(s)
        ref = out.clone()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            sim.simulate(hp, hs, out=out, stream=s)
        out.zero_()
        torch.cuda.synchronize()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        del g
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def test_adc_run_split_for_small_single_shot_problems(sim):
    """A phantom that fills few warps under a single-shot readout gets CTAs
    that share its spin ranges and divide the ADC runs (the launch reports
    the split); the signal matches the oracle and is deterministic. A launch
    that fills the GPU, or an RF-dominated sequence, does not split."""
    ph, seq = workload("paper_b", "full")
    a = gpu_signal(sim, ph, seq)
    info = sim.launch_info()
    assert info["split"] > 1
    b = gpu_signal(sim, ph, seq)
    assert np.array_equal(a, b)
    assert rel_err(a, oracle.simulate(ph, seq)) < TOL32
    gpu_signal(sim, *workload("epi512", "full"))
    assert sim.launch_info()["split"] == 1
    gpu_signal(sim, *workload("gre32", "full"))
    assert sim.launch_info()["split"] == 1
