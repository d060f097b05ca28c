"""Spin sharding, the multi-GPU partition (spins are independent, Section
"Physical and Mathematical Background"), run as k shards on one GPU: each
shard (a contiguous spin range, or whole groups of a dictionary) is simulated
by its own launch, and the shards' signals combined as the ranks' all-reduce
would (a sum; disjoint group rows for a grouped phantom) equal the whole
launch and the oracle within the FP32 tolerance. The cross-rank exchange
itself is covered by the two-rank gloo tests on CPU."""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.shard import shard_phantom
from paper_2301_02702_b300.workloads import workload

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    yield s
    s.close()


def run(sim, ph, seq):
    hp, hs = sim.upload_phantom(ph), sim.upload_sequence(seq)
    try:
        out = sim.simulate(hp, hs, "fp32").cpu().numpy()
        sim.sync()
        return out
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def rows_rel_err(got, ref):
    return float(np.max(np.max(np.abs(got - ref), axis=1) / np.max(np.abs(ref), axis=1)))


@pytest.mark.parametrize("name,k", [("epi512", 3), ("se128", 2), ("mrf", 4)])
def test_k_shards_on_one_gpu_combine_to_the_whole(sim, name, k):
    ph, seq = workload(name, "small")
    whole = run(sim, ph, seq)
    combined = np.zeros_like(whole)
    for rank in range(k):
        part, (g_lo, g_hi) = shard_phantom(ph, rank, k)
        sig = run(sim, part, seq)
        if ph.group_offsets is None:
            combined[0] += sig[0]
        else:
            assert sig.shape[0] == g_hi - g_lo
            combined[g_lo:g_hi] = sig
    assert rows_rel_err(combined, whole) < TOL32
    assert rows_rel_err(combined, oracle.simulate(ph, seq)) < TOL32
