"""Failure detection on the device without a fault: every wait in the kernels
is bounded by the global timer, and a wait that gives up sets a status word
that the host reads at koma_sync (KOMA_E_TIMEOUT); the context stays usable.
The self-check kernel waits on a barrier that nothing completes, with a
short bound, so the path runs for real without hanging anything."""
import time

import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    yield s
    s.close()


def test_bounded_wait_times_out_and_context_survives(sim):
    import torch
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    koma.koma_check_bounded_wait(sim.ctx, 20000, stream.cuda_stream)
    with pytest.raises(koma.KomaError) as e:
        sim.sync(stream)
    assert e.value.status == koma.KOMA_E_TIMEOUT
    assert time.perf_counter() - t0 >= 0.015, "the wait ended before its bound"
    # the flag was cleared by the sync that reported it
    sim.sync(stream)
    # and the context still simulates correctly
    ph, seq = workload("epi512", "small")
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        got = sim.simulate(hp, hs, stream=stream)
        sim.sync(stream)
        ref = oracle.simulate(ph, seq)
        assert np.max(np.abs(got.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-4
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def test_bounded_wait_limits_are_checked(sim):
    for bad in (0, -5, 2000001):
        with pytest.raises(koma.KomaError) as e:
            koma.koma_check_bounded_wait(sim.ctx, bad)
        assert e.value.status == koma.KOMA_E_INVALID
