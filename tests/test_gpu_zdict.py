"""The dictionary kernel for isochromats along z (K3z) against the oracle.

K3z runs when a grouped phantom's spins differ only in z (x = y = 0, no
off-resonance), every group has one T1 and one T2, no RF step has a z
gradient and every ADC record holds one sample: a FISP fingerprinting
dictionary (the MRF showcase, Section "Magnetic Resonance Fingerprinting"). These
tests check:

* eligible dictionaries with ragged groups (empty, 1, 127/128/129 spins: a
  K3z thread takes a unit of up to 8 spins of one group and a warp 32 units,
  so groups end inside and at a unit, and span warps),
  pulses on both sides of the series/closed-form switch, multi-step pulses,
  complex B1 and streams of several record tiles, group by group against the
  oracle, and bitwise repeatable;
* that each broken condition sends the same problem to the general grouped
  kernel (K3), whose result also matches the oracle;
* the tuner's pick among K3 and K3z shapes.
"""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import (GAMMA_BAR, Phantom, SequenceBuilder, hard_pulse_b1, sinc_pulse,
                                             workload)

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    yield s
    s.close()


def run(sim, ph, seq):
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        out = sim.simulate(hp, hs, "fp32").cpu().numpy()
        sim.sync()
        return out, sim.launch_info()
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def z_dictionary(sizes, seed, voxel=1e-3):
    """Groups of isochromats spread along z over one voxel, one (T1, T2) each."""
    rng = np.random.default_rng(seed)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    z = np.empty(n)
    pd = np.empty(n)
    t1 = np.empty(n)
    t2 = np.empty(n)
    for g, c in enumerate(sizes):
        sl = slice(offs[g], offs[g + 1])
        z[sl] = voxel * (np.arange(c) + rng.uniform(0.2, 0.8, c)) / max(c, 1) - voxel / 2
        pd[sl] = rng.uniform(0.5, 1.5, c) / max(c, 1)
        T2 = rng.uniform(0.03, 0.3)
        t1[sl] = T2 + rng.uniform(0.2, 2.0)
        t2[sl] = T2
    return Phantom(x=np.zeros(n), y=np.zeros(n), z=z, pd=pd, t1=t1, t2=t2, dw=np.zeros(n), group_offsets=offs)


def fisp_train(n_tr, seed, voxel=1e-3, sinc_steps=0, adc_samples=1, rf_gz=0.0, lobe_turns=1.0):
    """Inversion, then TRs of a pulse (hard, or a sinc of `sinc_steps` steps,
    with a random B1 phase), one ADC step at TE, a z lobe that dephases
    `lobe_turns` turns across the voxel, free precession. `adc_samples` > 1 or
    `rf_gz` != 0 break K3z's condition on the stream; with the spins inside
    the voxel |z Kz| <= lobe_turns / 2, so lobe_turns > 2 takes K3z's hi/lo
    phase."""
    rng = np.random.default_rng(seed)
    rf_dur, te, tg = 100e-6, 3e-3, 200e-6
    amp = (lobe_turns / voxel) / (GAMMA_BAR * 2 * tg)
    b = SequenceBuilder()
    b.steps(1, rf_dur, b1=hard_pulse_b1(np.pi, rf_dur))  # half angle pi/2: the closed form
    b.steps(1, 20e-3)
    for j in range(n_tr):
        t0 = b.t
        fa = np.deg2rad(rng.uniform(5.0, 120.0))  # small and large angles
        ph = np.exp(1j * rng.uniform(0, 2 * np.pi))
        if sinc_steps:
            b1 = sinc_pulse(sinc_steps, rf_dur / sinc_steps, np.rad2deg(fa)) * ph
            b.steps(sinc_steps, rf_dur / sinc_steps, [0, 0, rf_gz], b1=b1)
        else:
            b.steps(1, rf_dur, [0, 0, rf_gz], b1=hard_pulse_b1(fa, rf_dur) * ph)
        b.steps(1, te - rf_dur / 2)
        b.steps(adc_samples, 10e-6, adc=True)
        b.steps(1, tg, [0, 0, amp]).steps(1, tg).steps(1, tg, [0, 0, 0])
        b.idle_until(t0 + rng.uniform(6e-3, 9e-3))
    return b.build()


def check_groups(got, ref, offs):
    assert got.shape == ref.shape
    for g in range(len(offs) - 1):
        if offs[g + 1] == offs[g]:
            assert np.all(got[g] == 0), g
        else:
            scale = np.max(np.abs(ref[g]))
            assert scale > 0, g
            assert np.max(np.abs(got[g] - ref[g])) < TOL32 * scale, (g, np.max(np.abs(got[g] - ref[g])) / scale)


SIZES = [1, 0, 127, 128, 129, 300, 5, 256, 64, 383, 2, 129]


@pytest.mark.parametrize("sinc_steps,lobe_turns", [(0, 1.0), (24, 1.0), (0, 6.0), (24, 2.5)])
def test_z_dictionary_matches_oracle(sim, sinc_steps, lobe_turns):
    ph = z_dictionary(SIZES, seed=3)
    seq = fisp_train(60 if sinc_steps else 150, seed=4, sinc_steps=sinc_steps, lobe_turns=lobe_turns)
    assert seq.n_steps > 512  # several record tiles of the walk
    got, info = run(sim, ph, seq)
    assert info["spins_per_thread"] == 8, info  # K3z
    # one FP32 product for the phase while |z Kz| <= 1 turn, else hi/lo
    assert info["phase_mode"] == (1 if lobe_turns <= 2.0 else 0), info
    check_groups(got, oracle.simulate(ph, seq), ph.group_offsets)
    again, _ = run(sim, ph, seq)
    assert np.array_equal(got, again)


def test_many_small_groups_fill_whole_batches(sim):
    """700 groups packed as 8-spin units across warps and CTAs: segments of
    several groups in one warp, groups split between warps, the last batch
    partly empty."""
    rng = np.random.default_rng(8)
    sizes = list(rng.integers(1, 260, size=700))
    ph = z_dictionary(sizes, seed=9)
    seq = fisp_train(40, seed=10)
    got, info = run(sim, ph, seq)
    assert info["spins_per_thread"] == 8
    check_groups(got, oracle.simulate(ph, seq), ph.group_offsets)


def _broken(kind):
    ph = z_dictionary(SIZES, seed=5)
    seq_kw = {}
    if kind == "t1_in_group":
        ph.t1[ph.group_offsets[5] + 3] *= 1.5
    elif kind == "x":
        ph.x[ph.group_offsets[2]] = 1e-4
    elif kind == "df":
        ph.dw[ph.group_offsets[3] + 1] = 2 * np.pi * 5.0
    elif kind == "rf_gz":
        seq_kw["rf_gz"] = 1e-3
    elif kind == "adc2":
        seq_kw["adc_samples"] = 2
    return ph, fisp_train(40, seed=6, **seq_kw)


@pytest.mark.parametrize("kind", ["t1_in_group", "x", "df", "rf_gz", "adc2"])
def test_broken_condition_takes_the_general_grouped_kernel(sim, kind):
    ph, seq = _broken(kind)
    got, info = run(sim, ph, seq)
    assert info["spins_per_thread"] in (2, 4) and info["phase_mode"] == 0, (kind, info)
    check_groups(got, oracle.simulate(ph, seq), ph.group_offsets)


def test_tuner_includes_k3z(sim):
    ph, seq = workload("mrf", "small")
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        choice = sim.tune(hp, hs)
        assert (choice["spins_per_thread"], choice["block"]) in {(s, b) for s in (2, 4, 8) for b in (128, 256)}
        got = sim.simulate(hp, hs).cpu().numpy()
        sim.sync()
        assert sim.launch_info()["spins_per_thread"] == choice["spins_per_thread"]
        check_groups(got, oracle.simulate(ph, seq), ph.group_offsets)
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)
