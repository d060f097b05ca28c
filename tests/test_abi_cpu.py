"""C-ABI checks that need no GPU: the library loads, exports every entry point
include/koma.h declares, validates its inputs, and its host preprocessing
(regime classification, cumulative moments, uniform ADC runs) reproduces the
per-sample gradient moments computed independently here with numpy."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import (GAMMA_BAR, Sequence, SequenceBuilder, random_sequence,
                                             workload)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return koma.load()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "koma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(koma_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/koma.h but not exported"
    assert sorted(koma.EXPORTS) == names


def test_gamma_and_version(lib):
    assert koma.koma_gamma() == pytest.approx(oracle.GAMMA, rel=1e-15)
    assert "sm_103a" in koma.koma_version()


def test_init_without_gpu_fails_cleanly(lib, cuda_available):
    if cuda_available:
        pytest.skip("a GPU is present")
    with pytest.raises(koma.KomaError) as e:
        koma.koma_init(0)
    assert e.value.status == koma.KOMA_E_CUDA
    assert lib.koma_destroy(None) == koma.KOMA_OK


def test_plan_rejects_bad_sequences(lib):
    good = random_sequence(20, seed=1)
    koma.koma_sequence_plan(good)
    for mutate in (lambda s: s.dt.__setitem__(3, 0.0), lambda s: s.dt.__setitem__(3, -1e-6),
                   lambda s: s.dt.__setitem__(3, np.nan), lambda s: s.gx.__setitem__(5, np.inf),
                   lambda s: s.b1.__setitem__(2, complex(np.nan, 0)), lambda s: s.adc.__setitem__(4, 2)):
        s = random_sequence(20, seed=1)
        mutate(s)
        with pytest.raises(koma.KomaError) as e:
            koma.koma_sequence_plan(s)
        assert e.value.status == koma.KOMA_E_INVALID


def test_plan_rejects_bad_long_sequences(lib):
    """Sequences of >= 65,536 steps are checked by a parallel pass before the
    serial one names the first offence: an invalid value anywhere, up to the
    last step and the last time point, is still refused."""
    n = 70_000
    koma.koma_sequence_plan(random_sequence(n, seed=3))
    for i in (0, 33_001, n - 1):
        for mutate in (lambda s: s.dt.__setitem__(i, 0.0), lambda s: s.dt.__setitem__(i, np.nan),
                       lambda s: s.b1.__setitem__(i, complex(0, np.inf)), lambda s: s.gz.__setitem__(i, np.nan),
                       lambda s: s.gy.__setitem__(n, -np.inf), lambda s: s.adc.__setitem__(n, 3)):
            s = random_sequence(n, seed=3)
            mutate(s)
            with pytest.raises(koma.KomaError) as e:
                koma.koma_sequence_plan(s)
            assert e.value.status == koma.KOMA_E_INVALID


def _reference_samples(seq: Sequence):
    """(K [turns/m], tau [s], K1 [turns s/m]) of every ADC sample relative
    to the end of the last RF step before it, by a plain loop over steps:
    the trapezoid rule for K, and for K1 = gammabar * integral of G(s) s ds
    Gauss-Legendre quadrature with two nodes per step (exact for the
    quadratic integrand)."""
    K = np.zeros(3)
    K1 = np.zeros(3)
    tau = 0.0
    t = 0.0
    out = []
    nodes = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    if seq.adc[0]:
        out.append((K.copy(), tau, K1.copy()))
    for n in range(seq.n_steps):
        g0 = np.array([seq.gx[n], seq.gy[n], seq.gz[n]])
        g1 = np.array([seq.gx[n + 1], seq.gy[n + 1], seq.gz[n + 1]])
        dt = seq.dt[n]
        if seq.b1[n] != 0:
            K[:] = 0.0
            K1[:] = 0.0
            tau = 0.0
        else:
            K += GAMMA_BAR * dt * 0.5 * (g0 + g1)
            for u in nodes:
                f = 0.5 * (1.0 + u)
                s = t + f * dt
                K1 += GAMMA_BAR * 0.5 * dt * ((1.0 - f) * g0 + f * g1) * s
            tau += dt
        t += dt
        if seq.adc[n + 1]:
            out.append((K.copy(), tau, K1.copy()))
    return out


def _decode_samples(rec):
    out = {}
    for r in rec:
        if int(r[0]) != 2:
            continue
        count, k0 = int(r[1]), int(r[2])
        a = r[3:]
        assert 1 <= count <= 128
        for l in range(count):
            out[k0 + l] = (a[0:3] + l * a[4:7], a[3] + l * a[7],
                           a[8:11] + l * a[11:14] + 0.5 * l * (l - 1) * a[7] * a[4:7])
    return [out[k] for k in range(len(out))]


@pytest.mark.parametrize("name", ["gre32", "epi512", "se128", "random"])
def test_plan_reproduces_sample_moments(lib, name):
    seq = random_sequence(3000, seed=7) if name == "random" else workload(name, "small")[1]
    info, rec = koma.koma_sequence_plan(seq, with_records=True)
    assert info["n_steps"] == seq.n_steps
    assert info["n_adc"] == seq.n_adc
    assert info["n_rf"] == seq.n_rf
    assert info["n_rf"] + info["n_precess"] == seq.n_steps
    assert info["n_records"] == info["n_rf"] + info["n_adc_runs"] + info["n_materialize"]
    ref = _reference_samples(seq)
    got = _decode_samples(rec)
    assert len(got) == len(ref)
    for (kr, tr, k1r), (kg, tg, k1g) in zip(ref, got):
        assert np.max(np.abs(kr - kg)) <= 1e-9 * (1 + np.max(np.abs(kr)))
        assert abs(tr - tg) <= 1e-12 * (1 + tr)
        assert np.max(np.abs(k1r - k1g)) <= 1e-9 * (1 + np.max(np.abs(k1r)))
    # the types appear in the order the steps do: every RF step is a record
    assert int(np.sum(rec[:, 0] == 0)) == seq.n_rf


@pytest.mark.parametrize("name", ["se128", "epi512", "random_long"])
def test_long_sequences_built_in_chunks_reproduce_sample_moments(lib, name):
    """Sequences of 16,384 steps and more are built in parallel chunks cut
    after RF steps; every sample's moments (K with absolute-time first
    moments K1) and index must still match the reference walk, and the
    record counts must add up."""
    seq = random_sequence(60000, seed=11) if name == "random_long" else workload(name, "full")[1]
    assert seq.n_steps >= 16384
    info, rec = koma.koma_sequence_plan(seq, with_records=True)
    assert info["n_adc"] == seq.n_adc and info["n_rf"] == seq.n_rf
    assert info["n_rf"] + info["n_precess"] == seq.n_steps
    assert info["n_records"] == info["n_rf"] + info["n_adc_runs"] + info["n_materialize"]
    ref = _reference_samples(seq)
    got = _decode_samples(rec)
    assert len(got) == len(ref)
    kr = np.array([r[0] for r in ref]); kg = np.array([g[0] for g in got])
    tr = np.array([r[1] for r in ref]); tg = np.array([g[1] for g in got])
    k1r = np.array([r[2] for r in ref]); k1g = np.array([g[2] for g in got])
    assert np.all(np.abs(kr - kg) <= 1e-9 * (1 + np.max(np.abs(kr), axis=1, keepdims=True)))
    assert np.all(np.abs(tr - tg) <= 1e-12 * (1 + tr))
    assert np.all(np.abs(k1r - k1g) <= 1e-9 * (1 + np.max(np.abs(k1r), axis=1, keepdims=True)))
    assert int(np.sum(rec[:, 0] == 0)) == seq.n_rf
    # the same records on every call (the chunks' order does not depend on timing)
    info2, rec2 = koma.koma_sequence_plan(seq, with_records=True)
    assert np.array_equal(rec, rec2)


def test_plan_merges_uniform_readouts(lib):
    """A Cartesian readout of n samples at constant gradient becomes
    ceil(n / 128) ADC records."""
    b = SequenceBuilder()
    b.steps(1, 1e-6, b1=1e-5)
    b.steps(5, 10e-6, [0.01, 0, 0])
    b.steps(200, 4e-6, adc=True)
    info = koma.koma_sequence_plan(b.build())
    assert info["n_adc"] == 200 and info["n_adc_runs"] == 2


def test_plan_empty_and_adc_at_t0(lib):
    seq = Sequence(np.zeros(0), np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(0, complex), np.ones(1, np.uint8))
    info = koma.koma_sequence_plan(seq)
    assert info["n_adc"] == 1 and info["n_records"] == 1


def test_server_create_without_gpu_fails_cleanly(lib, cuda_available):
    if cuda_available:
        pytest.skip("a GPU is present")
    with pytest.raises(koma.KomaError) as e:
        koma.koma_server_create(0)
    assert e.value.status == koma.KOMA_E_CUDA


def test_plan_groups_readout_lines(lib):
    """Matrix-form readout plan: runs sharing (dK, dtau) form groups of at
    most 64 runs when a bucket has >= 8 runs and >= 1,024 samples; the two
    readout directions of an EPI are two buckets."""
    from paper_2301_02702_b300.workloads import epi
    info = koma.koma_sequence_plan(epi(n_read=128, n_lines=128, fov=0.23, rf_steps=100))
    assert (info["n_mma_groups"], info["n_mma_runs"], info["n_mma_samples"]) == (2, 128, 16384)
    # lines longer than a run: 128 + 72 samples, 150 runs a direction -> 64 + 64 + 22
    info = koma.koma_sequence_plan(epi(n_read=200, n_lines=150, fov=0.23, rf_steps=100))
    assert (info["n_mma_groups"], info["n_mma_runs"], info["n_mma_samples"]) == (6, 300, 30000)
    # thresholds: 8 runs of 128 samples a direction qualify, of 127 (1,016 samples) not;
    # 7 runs a direction not
    assert koma.koma_sequence_plan(epi(n_read=128, n_lines=16, fov=0.23, rf_steps=100))["n_mma_groups"] == 2
    assert koma.koma_sequence_plan(epi(n_read=127, n_lines=16, fov=0.23, rf_steps=100))["n_mma_groups"] == 0
    assert koma.koma_sequence_plan(epi(n_read=128, n_lines=14, fov=0.23, rf_steps=100))["n_mma_groups"] == 0
    # unstructured sequences: none
    assert koma.koma_sequence_plan(random_sequence(3000, seed=7))["n_mma_groups"] == 0


def _pulse_train(pulses, order, seed=0):
    """Pulses (n, dt, b1 samples, gradient during the pulse) played in
    `order`, each preceded by a gradient ramp to its own gradient and
    followed by a ramp down, a lobe whose area changes per occurrence and a
    few samples: only the pulses repeat."""
    rng = np.random.default_rng(seed)
    b = SequenceBuilder()
    for k, p in enumerate(order):
        n, dt, b1, g = pulses[p]
        b.steps(1, 20e-6, g)
        b.steps(n, dt, g, b1=b1)
        b.steps(1, 20e-6, [0.0, 0.0, 0.0])
        b.steps(2, 40e-6, [rng.uniform(-0.01, 0.01), 0.004 * (k % 5), 0.0]).steps(1, 40e-6, [0.0, 0.0, 0.0])
        b.steps(4, 10e-6, adc=True)
    return b.build()


def test_plan_on_long_streams_follows_the_rule(lib):
    """Streams of >= 16,384 records find their RF runs, hash them and check
    their equality in parallel slices; the plan is still the rule's: pulses
    of >= 4 steps that recur unchanged >= 3 times, at most 8, the ones saving
    the most stepped RF steps first (ties: first occurrence)."""
    from paper_2301_02702_b300.workloads import sinc_pulse
    rng = np.random.default_rng(5)
    lens = [3] + [4 * i for i in range(1, 12)]  # pulse 0 is too short for a map
    pulses = [(m, 4e-6, sinc_pulse(m, 4e-6, 15.0 + 5 * i), [0.0, 0.0, 0.002 * (i % 3)]) for i, m in enumerate(lens)]
    order = [int(p) for p in rng.choice(10, size=900)]
    order += [10, 10, 11]  # pulse 10 three times more, pulse 11 once
    seq = _pulse_train(pulses, order, seed=6)
    info = koma.koma_sequence_plan(seq)
    assert info["n_records"] >= 16384
    counts = {p: order.count(p) for p in set(order)}
    first = {p: order.index(p) for p in counts}
    cls = [p for p, c in counts.items() if c >= 3 and pulses[p][0] >= 4]
    cls.sort(key=lambda p: (-(counts[p] - 1) * pulses[p][0], first[p]))
    cls = cls[:8]
    assert info["n_rf_maps"] == len(cls)
    assert info["n_rf_map_runs"] == sum(counts[p] for p in cls)
    assert info["n_rf_map_steps"] == sum(counts[p] * pulses[p][0] for p in cls)
    assert info["n_rf_map_pulse_steps"] == sum(pulses[p][0] for p in cls)


def test_plan_reports_the_dictionary_kernels_stream_condition(lib):
    """The record stream's half of the dictionary kernel's condition (no RF step
    with a z gradient, one sample per ADC record) and the largest |Kz| of the
    phase records, which picks its one-product phase: the FISP dictionary
    train qualifies with max |Kz| = the unbalanced lobe's moment, one turn per
    voxel length; slice-selective pulses (se128), multi-sample readouts
    (epi512) and a FISP train sampling twice per TR do not."""
    from paper_2301_02702_b300.workloads import mrf_fisp
    info = koma.koma_sequence_plan(mrf_fisp(n_tr=40, voxel=1e-3))
    assert info["z_dict"] == 1
    assert info["z_kmax"] == pytest.approx(1.0 / 1e-3, rel=1e-6)
    assert koma.koma_sequence_plan(mrf_fisp(n_tr=40, voxel=2e-3))["z_kmax"] == pytest.approx(500.0, rel=1e-6)
    for name in ("se128", "epi512"):
        info = koma.koma_sequence_plan(workload(name, "small")[1])
        assert info["z_dict"] == 0 and info["z_kmax"] == 0.0, name
    b = SequenceBuilder()
    for _ in range(5):
        b.steps(1, 1e-4, b1=2e-6).steps(1, 3e-3).steps(2, 1e-5, adc=True)
        b.steps(1, 2e-4, [0, 0, 0.01]).steps(1, 2e-4, [0, 0, 0]).steps(1, 8e-3)
    assert koma.koma_sequence_plan(b.build())["z_dict"] == 0


def test_plan_finds_repeated_pulses(lib):
    """Runs of RF steps that recur unchanged at least 3 times (and are at
    least 4 steps long) get a map slot; at most 8 slots, the ones saving the
    most steps first."""
    from paper_2301_02702_b300.workloads import sinc_pulse
    info = koma.koma_sequence_plan(workload("se128", "full")[1])
    assert (info["n_rf_maps"], info["n_rf_map_runs"], info["n_rf_map_steps"],
            info["n_rf_map_pulse_steps"]) == (2, 128, 64000, 1000)
    a = (60, 4e-6, sinc_pulse(60, 4e-6, 90.0), [0.0, 0.0, 0.01])
    b = (40, 4e-6, sinc_pulse(40, 4e-6, 30.0), [0.0, 0.0, 0.01])
    c = (3, 4e-6, sinc_pulse(3, 4e-6, 10.0), [0.0, 0.0, 0.0])
    a_g = (60, 4e-6, sinc_pulse(60, 4e-6, 90.0), [0.0, 0.0, 0.012])  # A under another gradient
    info = koma.koma_sequence_plan(_pulse_train([a, b, c, a_g], [0, 1, 0, 2, 2, 2, 2, 3, 0, 1]))
    # A three times (the other gradient is another pulse), B only twice, C too short
    assert (info["n_rf_maps"], info["n_rf_map_runs"], info["n_rf_map_steps"]) == (1, 3, 180)
    assert info["n_rf_map_pulse_steps"] == 60
    # nine distinct pulses repeated 3 times each: the eight longest get maps
    ps = [(10 + 2 * i, 4e-6, sinc_pulse(10 + 2 * i, 4e-6, 20.0 + i), [0.0, 0.0, 0.0]) for i in range(9)]
    info = koma.koma_sequence_plan(_pulse_train(ps, [i for _ in range(3) for i in range(9)]))
    assert info["n_rf_maps"] == 8 and info["n_rf_map_runs"] == 24
    assert info["n_rf_map_pulse_steps"] == sum(10 + 2 * i for i in range(1, 9))
    # unstructured sequences: none
    assert koma.koma_sequence_plan(random_sequence(3000, seed=7))["n_rf_maps"] == 0
