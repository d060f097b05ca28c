"""The continuous-batching server: results against the oracle and against the
single-simulation path, the same result alone and in a mix (bitwise), and
admission under a device-memory budget."""
import threading

import numpy as np
import pytest

import oracle
from paper_2301_02702_b300 import build, koma
from paper_2301_02702_b300.workloads import random_sequence, random_spins, workload

pytestmark = pytest.mark.gpu
TOL32 = 1e-4


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def server():
    build.build()
    srv = koma.Server(0)
    yield srv
    srv.close()


def _mix(seed, k):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        n = int(rng.integers(1, 3000))
        out.append((random_spins(n, seed=1000 * seed + i), random_sequence(int(rng.integers(20, 600)), seed=77 * seed + i)))
    return out


def test_server_matches_oracle(server):
    reqs = [workload("epi512", "small"), workload("se128", "small"), workload("gre32", "small")] + _mix(3, 5)
    ids = [server.submit(ph, seq) for ph, seq in reqs]
    for (ph, seq), rid in zip(reqs, ids):
        sig, info = server.wait(rid)
        assert info["status"] == 0 and info["latency_s"] > 0 and info["launches"] >= 1
        ref = oracle.simulate(ph, seq)[0]
        assert rel_err(sig, ref) < TOL32


def test_same_result_alone_and_in_a_mix(server):
    ph, seq = workload("epi512", "small")
    alone, _ = server.wait(server.submit(ph, seq))
    mix = _mix(7, 12)
    ids = []
    for i, (p, s) in enumerate(mix):
        ids.append(server.submit(p, s))
        if i == 5:
            target = server.submit(ph, seq)
    with_mix, info = server.wait(target)
    for rid in ids:
        server.wait(rid)
    assert np.array_equal(alone, with_mix), "a request's result must not depend on the mix"
    # and both agree with the single-simulation path within tolerance
    sim = koma.Simulator(0)
    try:
        hp, hs = sim.upload_phantom(ph), sim.upload_sequence(seq)
        direct = sim.simulate(hp, hs).cpu().numpy()[0]
        koma.koma_phantom_free(hp)
        koma.koma_sequence_free(hs)
    finally:
        sim.close()
    assert rel_err(alone, direct) < TOL32


def test_concurrent_submitters(server):
    mix = _mix(11, 16)
    results = {}

    def worker(lo, hi):
        for i in range(lo, hi):
            rid = server.submit(*mix[i])
            results[i] = server.wait(rid)[0]

    th = [threading.Thread(target=worker, args=(4 * t, 4 * t + 4)) for t in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i, (ph, seq) in enumerate(mix):
        ref = oracle.simulate(ph, seq)[0]
        if np.max(np.abs(ref)) > 0:
            assert rel_err(results[i], ref) < TOL32


def test_admission_by_memory_budget():
    """A small budget admits requests one or two at a time; all complete, the
    peak stays under the budget; a request larger than the whole budget fails."""
    reqs = _mix(21, 6)
    srv = koma.Server(0, mem_budget_bytes=400 << 10)
    try:
        ids = [srv.submit(p, s) for p, s in reqs]
        for (ph, seq), rid in zip(reqs, ids):
            sig, _ = srv.wait(rid)
            ref = oracle.simulate(ph, seq)[0]
            if np.max(np.abs(ref)) > 0:
                assert rel_err(sig, ref) < TOL32
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["mem_peak"] <= 400 << 10
        big_ph, big_seq = workload("epi512", "full")
        rid = srv.submit(big_ph, big_seq)
        with pytest.raises(koma.KomaError) as e:
            srv.wait(rid)
        assert e.value.status == koma.KOMA_E_NOMEM
    finally:
        srv.close()


def test_checkpointed_chunks_equal_unsplit_walk(server):
    """Walking a sequence in chunks of 7 step records, with the spin state
    checkpointed in device memory between launches (cuts fall inside RF runs
    and between samples), gives bitwise the result of the unsplit walk. The
    spin echo's repeated pulses are taken by their maps: a pulse is one
    record of the walked stream."""
    reqs = [workload("se128", "small"), workload("epi512", "small"), (random_spins(700, seed=4),
                                                                       random_sequence(900, seed=5))]
    assert koma.koma_sequence_plan(reqs[0][1])["n_rf_maps"] == 2
    whole = [server.wait(server.submit(ph, seq))[0] for ph, seq in reqs]
    small = koma.Server(0, chunk_records=7)
    try:
        parts = [small.wait(small.submit(ph, seq)) for ph, seq in reqs]
    finally:
        small.close()
    for (ph, seq), a, (b, info) in zip(reqs, whole, parts):
        assert info["launches"] > 1
        assert np.array_equal(a, b)
        assert rel_err(b, oracle.simulate(ph, seq)[0]) < TOL32


def test_grouped_request_served_alone_and_in_a_mix(server):
    """A dictionary (one signal per group, with an empty group) is served by
    the koma_simulate lane: it matches the oracle group by group, and its
    result is bitwise the same alone and while shared launches run."""
    ph, seq = workload("mrf", "small")
    ph.group_offsets = ph.group_offsets.copy()
    alone, info = server.wait(server.submit(ph, seq))
    assert info["lane"] == 1 and info["n_groups"] == ph.n_groups
    assert alone.shape == (ph.n_groups, seq.n_adc)
    ref = oracle.simulate(ph, seq)
    err = np.max(np.abs(alone - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert np.max(err) < TOL32
    mix = _mix(5, 10)
    ids = [server.submit(p, s) for p, s in mix[:5]]
    target = server.submit(ph, seq)
    ids += [server.submit(p, s) for p, s in mix[5:]]
    with_mix, info = server.wait(target)
    for rid in ids:
        server.wait(rid)
    assert np.array_equal(alone, with_mix)
    # groups that are empty give zero signal
    phe = random_spins(50, seed=3)
    phe.group_offsets = np.array([0, 20, 20, 50])
    sig, info = server.wait(server.submit(phe, random_sequence(200, seed=4)))
    assert sig.shape[0] == 3 and np.all(sig[1] == 0) and info["lane"] == 1


def test_large_requests_take_the_simulate_lane():
    """With a low threshold, requests of at least plain_spins spins run the
    koma_simulate path in the second lane (bitwise what a fresh context's
    koma_simulate gives, so the tensor-core readout and the maps of repeated
    pulses apply), while smaller ones share the persistent kernel's launches
    at the same time; both match the oracle."""
    big = [workload("se128", "small"), workload("epi512", "small")]  # 922 and 2,304 spins
    small = [(random_spins(n, seed=40 + i), random_sequence(300 + 50 * i, seed=60 + i))
             for i, n in enumerate((1, 17, 300, 640, 800, 899))]
    srv = koma.Server(0, plain_spins=900)
    try:
        ids = [srv.submit(*r) for r in big] + [srv.submit(*r) for r in small]
        res = [srv.wait(rid) for rid in ids]
        st = srv.stats()
    finally:
        srv.close()
    assert st["lane_runs"] == 2
    sim = koma.Simulator(0)
    try:
        for (ph, seq), (sig, info) in zip(big, res[:2]):
            assert info["lane"] == 1
            hp, hs = sim.upload_phantom(ph), sim.upload_sequence(seq)
            direct = sim.simulate(hp, hs).cpu().numpy()[0]
            koma.koma_phantom_free(hp)
            koma.koma_sequence_free(hs)
            assert np.array_equal(sig, direct)
            assert rel_err(sig, oracle.simulate(ph, seq)[0]) < TOL32
    finally:
        sim.close()
    for (ph, seq), (sig, info) in zip(small, res[2:]):
        assert info["lane"] == 0
        ref = oracle.simulate(ph, seq)[0]
        if np.max(np.abs(ref)) > 0:
            assert rel_err(sig, ref) < TOL32


def test_submit_rejects_bad_group_offsets(server):
    ph = random_spins(10, seed=1)
    ph.group_offsets = np.array([0, 6, 4, 10])
    with pytest.raises(koma.KomaError) as e:
        server.submit(ph, random_sequence(20, seed=2))
    assert e.value.status == koma.KOMA_E_INVALID


def test_large_request_checked_on_the_device_at_submit():
    """A large request's phantom goes to device memory at submit, where the
    conversion kernel checks every spin: invalid spins are refused by submit
    itself, with the offending spin's index, and the server keeps serving."""
    srv = koma.Server(0, plain_spins=900)
    try:
        seq = random_sequence(150, seed=9)
        for field, j, value in (("t2", 1234, -1.0), ("x", 77, np.nan), ("pd", 1999, -0.5)):
            ph = random_spins(2000, seed=8)
            getattr(ph, field)[j] = value
            with pytest.raises(koma.KomaError) as e:
                srv.submit(ph, seq)
            assert e.value.status == koma.KOMA_E_INVALID
            assert str(j) in str(e.value), str(e.value)
        ph, seq = workload("epi512", "small")
        sig, info = srv.wait(srv.submit(ph, seq))
        assert info["lane"] == 1
        assert rel_err(sig, oracle.simulate(ph, seq)[0]) < TOL32
        assert srv.stats()["mem_used"] == 0  # the device phantom is released with the request
    finally:
        srv.close()


def test_large_request_over_budget_keeps_a_host_copy():
    """When the memory budget has no room for a large request's phantom at
    submit, its spins are checked on the host and the lane uploads a host
    copy once the request is admitted; the result is bitwise the device
    path's. The budget is just under two phantoms: while the first request
    (a long pulse, ~50 ms on the GPU) holds its phantom, the second cannot
    place its own and takes the host path."""
    from paper_2301_02702_b300.workloads import SequenceBuilder, sinc_pulse
    ph = random_spins(600_000, seed=12, extent=0.05)
    b = SequenceBuilder()
    b.steps(50_000, 2e-6, [0.0, 0.0, 0.002], b1=sinc_pulse(50_000, 2e-6, 30.0))
    b.steps(1, 1e-4)
    b.steps(128, 8e-6, [0.01, 0.0, 0.0], adc=True)
    b.steps(1, 1e-5)
    seq = b.build()
    n_pad = (ph.n + 31) // 32 * 32
    ph_bytes = n_pad * (7 * 8 + 11 * 4)  # FP64 and FP32 phantom blocks
    roomy = koma.Server(0, plain_spins=900)
    try:
        a, info_a = roomy.wait(roomy.submit(ph, seq))
    finally:
        roomy.close()
    tight = koma.Server(0, plain_spins=900, mem_budget_bytes=2 * ph_bytes - 1)
    try:
        ids = [tight.submit(ph, seq) for _ in range(2)]
        res = [tight.wait(i) for i in ids]
        st = tight.stats()
    finally:
        tight.close()
    assert info_a["lane"] == 1 and st["failed"] == 0 and st["mem_peak"] <= 2 * ph_bytes - 1
    for b_sig, info in res:
        assert info["lane"] == 1
        assert np.array_equal(a, b_sig)
