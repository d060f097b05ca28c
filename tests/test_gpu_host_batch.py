"""koma_simulate_host_batch: host-buffer simulations with one job's host work
overlapped with the previous job's simulation (jobs alternate between the
context and a second one on the same device). Each job's result is bitwise
the one koma_simulate_host gives for it alone; a failing job stops the batch
with its error, and the context stays usable."""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import random_sequence, random_spins, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    build.build()
    c = koma.koma_init(0)
    yield c
    koma.koma_destroy(c)


def _jobs():
    return [workload("se128", "small"), workload("epi512", "small"), workload("mrf", "small"),
            (random_spins(700, seed=41), random_sequence(9000, seed=42)), workload("gre32", "small")]


def test_batch_equals_one_call_per_job(ctx):
    jobs = _jobs()
    single = [koma.koma_simulate_host(ctx, ph, seq, koma.KOMA_FP32_SPLITPHASE) for ph, seq in jobs]
    for rep in range(2):  # the second batch reuses the second context
        outs = koma.koma_simulate_host_batch(ctx, [(ph, seq, None) for ph, seq in jobs])
        assert len(outs) == len(jobs)
        for a, b in zip(outs, single):
            assert a.shape == b.shape and np.array_equal(a, b)
    ph, seq = jobs[2]
    ref = oracle.simulate(ph, seq)
    err = np.max(np.abs(outs[2] - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert np.max(err) < 1e-4


def test_empty_and_single_job_batches(ctx):
    assert koma.koma_simulate_host_batch(ctx, []) == []
    ph, seq = workload("epi512", "small")
    (one,) = koma.koma_simulate_host_batch(ctx, [(ph, seq, None)])
    assert np.array_equal(one, koma.koma_simulate_host(ctx, ph, seq, koma.KOMA_FP32_SPLITPHASE))


@pytest.mark.parametrize("bad_at", [1, 2])
def test_failing_job_stops_the_batch(ctx, bad_at):
    """A job with an invalid spin (T2 < 0) fails the batch with its message,
    whichever of the two contexts ran it; the next batch runs normally."""
    jobs = [(ph, seq, None) for ph, seq in _jobs()[:4]]
    bad = random_spins(500, seed=7)
    bad.t2[123] = -1.0
    jobs[bad_at] = (bad, random_sequence(300, seed=8), None)
    with pytest.raises(koma.KomaError) as e:
        koma.koma_simulate_host_batch(ctx, jobs)
    assert e.value.status == koma.KOMA_E_INVALID
    assert "123" in str(e.value), str(e.value)
    ph, seq = workload("se128", "small")
    (out,) = koma.koma_simulate_host_batch(ctx, [(ph, seq, None)])
    assert np.array_equal(out, koma.koma_simulate_host(ctx, ph, seq, koma.KOMA_FP32_SPLITPHASE))


def test_batch_follows_the_context_switches_and_fp64(ctx):
    """Switches set on the context after its second context exists apply to
    every job of the next batch (readout on the tensor cores off, repeated
    pulses stepped), and an FP64 batch equals FP64 single calls."""
    jobs = [workload("se128", "small"), workload("epi512", "small"), workload("se128", "small")]
    koma.koma_simulate_host_batch(ctx, [(ph, seq, None) for ph, seq in jobs])  # the second context exists
    lib = koma.load()
    try:
        lib.koma_set_mma(ctx, 0)
        lib.koma_set_rf_maps(ctx, 0)
        single = [koma.koma_simulate_host(ctx, ph, seq, koma.KOMA_FP32_SPLITPHASE) for ph, seq in jobs]
        outs = koma.koma_simulate_host_batch(ctx, [(ph, seq, None) for ph, seq in jobs])
        for a, b in zip(outs, single):
            assert np.array_equal(a, b)
    finally:
        lib.koma_set_mma(ctx, 1)
        lib.koma_set_rf_maps(ctx, 1)
    ph, seq = workload("gre32", "small")
    one = koma.koma_simulate_host(ctx, ph, seq, koma.KOMA_FP64)
    outs = koma.koma_simulate_host_batch(ctx, [(ph, seq, None), (ph, seq, None)], koma.KOMA_FP64)
    assert all(np.array_equal(o, one) for o in outs)
    assert np.max(np.abs(one - oracle.simulate(ph, seq))) < 1e-9 * np.max(np.abs(one))
