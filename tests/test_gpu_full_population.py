"""GPU parity at full population: every spin of a benchmark launch contributes.

The signal is the plain sum of Mxy over all spins (Section "GPU/CPU
Parallelization"), so these tests check the accumulation itself: per-thread
and warp sums, the per-CTA partial rows, the tensor-core readout's
accumulators and the cross-CTA reduction, with whole CTAs and 32-spin readout
blocks full of real spins. The oracle sums the same spins in FP64.

* epi512: all 262,144 spins, in the benchmark's launch configuration (the
  readout on the tensor cores) and with every sample stepped by the Bloch
  kernel (readout off).
* se128: the full 1.1 M-spin launch with a contiguous slab of 65,536 spins
  around the excited slice kept (spins are stored slice by slice, so the slab
  fills whole CTAs and readout blocks) and PD = 0 elsewhere: by linearity in
  PD the signal is the slab's, which the oracle computes directly.
"""
import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import Phantom, workload

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
_ref_cache = {}


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    yield s
    s.close()


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def gpu_signal(sim, ph, seq, mma=True):
    koma.koma_set_mma(sim.ctx, mma)
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        out = sim.simulate(hp, hs, "fp32")
        sim.sync()
        info = sim.launch_info()
        return out.cpu().numpy(), info
    finally:
        koma.koma_set_mma(sim.ctx, True)
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def central_slab(ph, n_keep):
    lo = ph.n // 2 - n_keep // 2
    return np.arange(lo, lo + n_keep)


@pytest.mark.parametrize("mma", [True, False])
def test_epi512_every_spin(sim, mma):
    ph, seq = workload("epi512", "full")
    if "epi512" not in _ref_cache:
        _ref_cache["epi512"] = oracle.simulate(ph, seq)
    ref = _ref_cache["epi512"]
    got, info = gpu_signal(sim, ph, seq, mma)
    assert (info["mma_grid"] > 0) == mma
    assert info["grid"] >= 148
    err = rel_err(got, ref)
    print(f"epi512 all {ph.n} spins, readout {'tensor cores' if mma else 'Bloch kernel'}: rel err {err:.3e}")
    assert err < TOL32, err


def test_se128_full_launch_contiguous_slab(sim):
    ph, seq = workload("se128", "full")
    keep = central_slab(ph, 65536)
    pd = np.zeros(ph.n)
    pd[keep] = ph.pd[keep]
    masked = Phantom(ph.x, ph.y, ph.z, pd, ph.t1, ph.t2, ph.dw)
    got, info = gpu_signal(sim, masked, seq)
    assert info["mma_grid"] > 0 and info["grid"] >= 148
    ref = oracle.simulate(ph.subset(keep), seq)
    # the slab holds the excited slice: its signal is far from zero
    assert np.max(np.abs(ref)) > 100.0
    err = rel_err(got, ref)
    print(f"se128 full launch, central slab of {len(keep)} spins: rel err {err:.3e}")
    assert err < TOL32, err
