"""koma_simulate_static: the simulation entry point that allocates nothing.

It exists for callers that cannot allocate device memory when they simulate
(an allocator that owns the whole device, a loop that must not pay
cudaMalloc's implicit synchronisation, or no allocator at all): its per-CTA
partial sums live in a static device array inside libkoma. This file runs
last so that a failure here leaves every other test already run; it passes
alone in a fresh process as well as after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import random_sequence, random_spins, workload

pytestmark = pytest.mark.gpu

TOL32 = 1e-4  # the FP32 path's parity tolerance used by the other GPU tests


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def sim():
    build.build()
    s = koma.Simulator(0)
    yield s
    s.close()


@pytest.mark.parametrize("name,scale", [("epi512", "small"), ("se128", "small"), ("epi512", "full")])
def test_static_entry_matches_simulate_on_two_calls(sim, name, scale):
    import torch
    ph, seq = workload(name, scale)
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        ref = sim.simulate(hp, hs, "fp32")
        sim.sync()
        ref = ref.cpu().numpy()
        stream = torch.cuda.current_stream()
        held = koma.koma_mem_used(sim.ctx)
        for call in range(2):
            out = torch.full((1, seq.n_adc), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            koma.koma_simulate_static(sim.ctx, hp, hs, out.data_ptr(), stream.cuda_stream)
            sim.sync()
            free_after = torch.cuda.mem_get_info()[0]
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), f"call {call}: output not fully written"
            err = rel_err(got, ref)
            assert err < TOL32, f"call {call}: rel err {err:.3g} vs koma_simulate"
            assert koma.koma_mem_used(sim.ctx) == held
            info = sim.launch_info()  # describes this call, not the koma_simulate before it
            assert info["kernels"] == 2 and info["mma_grid"] == 0 and info["grid"] >= 1
            if call == 1:
                assert free_after == free_before, "the call took device memory"
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)


def test_static_entry_rejects_what_does_not_fit(sim):
    import torch
    stream = torch.cuda.current_stream()
    out = torch.zeros((1, 4097), dtype=torch.complex128, device="cuda")
    # 2^20 spins need at least 1,024 CTAs; x 4,097 samples > 4,194,304 partials
    ph = random_spins(1 << 20, seed=3)
    seq = random_sequence(4097, seed=4, rf_frac=0.3, adc_frac=0.0)
    seq.adc[:] = 0
    seq.adc[1:] = 1
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    try:
        with pytest.raises(koma.KomaError) as e:
            koma.koma_simulate_static(sim.ctx, hp, hs, out.data_ptr(), stream.cuda_stream)
        assert e.value.status == koma.KOMA_E_INVALID
        assert "static scratch" in str(e.value)
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)
    # grouped phantoms are refused (their launch needs a device CTA table)
    phg = random_spins(64, seed=5)
    phg.group_offsets = np.array([0, 30, 64])
    hp = sim.upload_phantom(phg)
    hs = sim.upload_sequence(random_sequence(40, seed=6))
    try:
        with pytest.raises(koma.KomaError) as e:
            koma.koma_simulate_static(sim.ctx, hp, hs, out.data_ptr(), stream.cuda_stream)
        assert e.value.status == koma.KOMA_E_INVALID
    finally:
        koma.koma_sequence_free(hs)
        koma.koma_phantom_free(hp)
