"""Several contexts used at once from host threads, each uploading its
inputs and simulating on its own non-blocking stream straight after the
uploads return (the pattern of the server's second lane, where four such
threads run next to the shared launches). Every result is bitwise the one a
lone, serial run gives.

This guards the rule that an upload has landed in device memory when the
call returns: a copy that merely staged its data (a plain cudaMemcpy from
pageable memory, on the legacy stream) lets a kernel on a non-blocking
stream read records that have not arrived, which the kernels' own bounds
checks then report (KOMA_E_INTERNAL) instead of reading out of bounds.
"""
import threading

import numpy as np
import pytest

from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import random_sequence, random_spins, workload

pytestmark = pytest.mark.gpu


def _cases():
    cases = [workload("se128", "small"), workload("epi512", "small")]
    for i in range(6):
        # long record streams (up to ~1.3 MB each) and ragged spin counts
        cases.append((random_spins(3000 + 517 * i, seed=90 + i), random_sequence(12000 + 2000 * i, seed=70 + i)))
    return cases


def _run(sim, ph, seq, stream):
    import torch
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        out = torch.empty((1, seq.n_adc), dtype=torch.complex128, device="cuda")
        sim.simulate(hp, hs, "fp32", out=out, stream=stream)
        sim.sync(stream)
        return out.cpu().numpy()
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def test_concurrent_contexts_match_serial():
    import torch
    build.build()
    cases = _cases()
    sim0 = koma.Simulator(0)
    try:
        s0 = torch.cuda.Stream()
        ref = [_run(sim0, ph, seq, s0) for ph, seq in cases]
    finally:
        sim0.close()
    errors, results = [], {}

    def worker(t):
        sim = koma.Simulator(0)
        try:
            st = torch.cuda.Stream()
            for rep in range(3):
                for k in range(len(cases)):
                    i = (k + t) % len(cases)
                    results[(t, rep, i)] = _run(sim, cases[i][0], cases[i][1], st)
        except Exception as e:  # reported below
            errors.append(repr(e))
        finally:
            sim.close()

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    assert len(results) == 4 * 3 * len(cases)
    for (t, rep, i), r in results.items():
        assert np.array_equal(r, ref[i]), (t, rep, i)
