#!/usr/bin/env python3
"""Benchmark of the Bloch-simulation hot path: spin-steps/s on one B300.

One *step* is one complete simulation of the workload (every spin through
every discretised sequence step, with the per-ADC-sample signal sum), i.e. one
``koma_simulate`` call: the Bloch kernel, the tensor-core readout when the
sequence has matrix-form readout groups, and the fixed-order reduction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload se128]
    python bench.py --workload serve ...     # the serving workload on its own
    python bench.py --impl reference ...     # the FP64 CPU oracle, host cores

The default workload is the largest single-GPU configuration, the 128^3
spin echo (se128). Its line also carries a ``serving`` object: a Poisson
stream of mixed requests through the continuous-batching server, with
p50/p99 latency and served spin-steps/s.

Under torchrun (N > 1) every rank simulates its own replica of the workload
(the path has no data exchange: spins are independent); ``value`` is the
spin-steps of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Bloch spin-steps/s at <=1e-4 rel err vs FP64 oracle"
UNIT = "spin-steps/s"
TOL = 1e-4

# Algorithmic FP32 work per unit (FMA = 2 flops): an excitation step rotates
# M about the step's constant field and relaxes it (50 flops per spin), an ADC
# sample advances Mxy by one complex rotation-with-decay and adds it to the
# signal (8 flops per spin). Steps without RF and without ADC cost nothing
# (the closed form of the merged precession is evaluated where it is observed).
FLOPS_RF_STEP = 50
FLOPS_ADC_SAMPLE = 8
# moving spins: the RF step's field also moves the position (3 FMA), and an
# ADC sample also turns the per-sample rotator by its own increment (one
# more complex product)
FLOPS_RF_STEP_MOVING = 56
FLOPS_ADC_SAMPLE_MOVING = 16
# FP32 peak of the part: 148 SMs x 128 lanes x 2 flops x 2032 MHz (max SM clock)
SM_COUNT = 148
PEAK_FP32_TFLOPS = SM_COUNT * 128 * 2 * 2032e6 / 1e12
# repeated RF pulses taken by their maps: the pre-pass steps four vectors
# (the three columns of A and c) through each distinct pulse, sharing the
# step's rotation: per spin-step the field, |a|^2, |a| and the axis (14
# flops) once; per vector the rotation (two cross products, w p + q and the
# update: 30) and the relaxation (6); the columns of A, carried as FP32
# pairs, also rotate their low parts (30) and add each component's increment
# by TwoSum (6 per component: 18). Applying a map is 9 FMA per spin.
FLOPS_MAP_STEP = 14 + 3 * (30 + 6 + 30 + 18) + (30 + 6)
FLOPS_MAP_APPLY = 18
# tensor-core readout: per 32-spin block and matrix-form group, 4 K slices x
# 3 FP16 products (hi hi, hi lo, lo hi) of one M = N = 128, K = 16 MMA
MMA_FLOPS_PER_BLOCK_GROUP = 12 * 2 * 128 * 128 * 16
# dense FP16/BF16 tensor peak and HBM bandwidth when MEASURED_PEAKS.json is absent (fallback)
PEAK_TENSOR_FALLBACK = 1800.0
PEAK_HBM_FALLBACK = 6400.0
# contiguous spins kept for the se128 parity check (the rest get PD = 0)
SE128_PARITY_SLAB = 65536

WORKLOAD_TEXT = {
    "gre32": "gre32: 32x32 grid phantom (1,024 spins), spoiled GRE 32 TRs x 10 ms on a 10 us grid "
             "(32,000 steps, 30-deg 1 ms sinc RF, 1,024 ADC samples)",
    "epi512": "epi512: 512x512 ellipse phantom (262,144 spins, dB0 ~ 20 Hz smooth field), single-shot "
              "128x128 EPI, 4 us dwell, 90-deg 2 ms sinc at 4 us (17,958 steps, 16,384 ADC samples)",
    "se128": "se128: 128^3 ellipsoid phantom (1,097,914 spins, dB0 ~ 50 Hz smooth field), 64-shot spin echo, "
             "90/180-deg 1 ms sinc at 2 us, 256-sample readouts (81,920 steps, 16,384 ADC samples)",
    "serve": "serve: Poisson stream (200 req/s) of simulations with 1e3-1e6 spins (random subsets of the epi512 "
             "and se128 phantoms) and 1e3-1e5 steps (the workloads' sequences truncated or repeated), both "
             "log-uniform, served under a 150 GB device-memory budget",
    "paper_d": "paper_d: the paper's experiment (d): 230x230 mm head phantom at 1 mm (26,874 spins, no "
               "off-resonance) moving along y at v_y = 0.1 m/s, single-shot EPI FOV 230 mm 100x100 TE 100 ms with "
               "a hard 90-deg pulse (10,479 steps, 10,000 ADC samples), motion kernel",
    "mrf": "mrf: FISP fingerprinting dictionary, 250 T1 x 200 T2 log grid = 50,000 entries of U{50..400} "
           "isochromats over one voxel (11,282,781 spins), inversion + 1,000 TRs of 10-15 ms, flip 5-70 deg "
           "(6,002 steps, 1,000 ADC samples per entry), one persistent autotuned launch",
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# --------------------------------------------------------------------------
# clocks during the timed region (NVML; read only)
# --------------------------------------------------------------------------
class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml.so.1 ships with
    the driver; the Python wrapper package may be absent)."""

    def __init__(self, index: int):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex failed")
        try:
            self._reasons = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self._reasons = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sm_clock(self) -> int:
        v = self.ct.c_uint()
        self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(v))  # NVML_CLOCK_SM
        return v.value

    def sm_max_clock(self) -> int:
        v = self.ct.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.ct.byref(v))
        return v.value

    def reasons(self) -> int:
        v = self.ct.c_ulonglong()
        self._reasons(self.h, self.ct.byref(v))
        return v.value


class ClockSampler:
    """Samples the SM clock and the clock-event reasons while running."""
    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
               "sw_power_cap": 0x4, "hw_power_brake_slowdown": 0x80}

    def __init__(self, device_index: int, interval_s: float = 0.002):
        self.interval = interval_s
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self.error = None
        try:
            self._nv = _Nvml(device_index)
            self.max_mhz = self._nv.sm_max_clock()
        except Exception as e:  # no NVML: report the absence
            self._nv = None
            self.error = repr(e)

    def _run(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self._nv.sm_clock())
                r = self._nv.reasons()
                for name, bit in self.REASONS.items():
                    if r & bit:
                        self.reasons.add(name)
            except Exception as e:
                self.error = repr(e)
                return
            time.sleep(self.interval)

    def start(self):
        if self._nv is not None:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join()
        out = {"sm_mhz": float(statistics.median(self.samples)) if self.samples else None,
               "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons), "samples": len(self.samples),
               "source": "NVML (libnvidia-ml, read only)"}
        if self.error:
            out["error"] = self.error
        return out


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in ("paper_2301_02702_b300/csrc/koma_kernels.cu", "paper_2301_02702_b300/csrc/koma_internal.h"):
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes per launch of the Bloch kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "bloch_fp32_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(workload)
    if not e or e.get("kernel_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def tensor_peak():
    """(TFLOP/s, source) of the dense 16-bit tensor peak: the measured cuBLAS
    BF16 burst rate of this pool's parts (FP16 has the same nominal rate)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["bf16_tflops"])
        return v, "measured dense BF16 GEMM burst (MEASURED_PEAKS.json; FP16 same nominal rate)"
    except (OSError, KeyError, ValueError, TypeError):
        return PEAK_TENSOR_FALLBACK, "fallback 1.8 PFLOP/s dense BF16 (no measured peaks file)"


def hbm_peak():
    """(GB/s, source) of the measured HBM copy bandwidth of this pool's parts."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured HBM copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError, TypeError):
        return PEAK_HBM_FALLBACK, "fallback 6.4 TB/s (no measured peaks file)"


def algorithmic_flops(info: dict, n_spins: int, moving: bool = False) -> float:
    if moving:
        return float(n_spins) * (info["n_rf"] * FLOPS_RF_STEP_MOVING + info["n_adc"] * FLOPS_ADC_SAMPLE_MOVING)
    return float(n_spins) * (info["n_rf"] * FLOPS_RF_STEP + info["n_adc"] * FLOPS_ADC_SAMPLE)


def cpu_sample_run(ph, seq, target_s: float, threads: int):
    """Time the oracle on a random spin sample sized for ~target_s seconds."""
    import oracle
    rng = np.random.default_rng(123)
    # two calibration sizes: the slope is the per-spin cost, the rest the
    # per-call cost (sequence conversion, threads), which a one-point
    # estimate would spread over the spins
    n_cal = min(ph.n, max(16 * threads, 64))
    t = []
    for n in (n_cal, 2 * n_cal):
        idx = np.sort(rng.choice(ph.n, min(ph.n, n), replace=False))
        t0 = time.perf_counter()
        oracle.simulate(ph.subset(idx), seq, threads=threads)
        t.append(time.perf_counter() - t0)
    per_spin = max((t[1] - t[0]) / n_cal, t[1] / (2 * n_cal) * 0.25, 1e-9)
    fixed = max(t[0] - per_spin * n_cal, 0.0)
    n = int(min(ph.n, max(threads, (target_s - fixed) / per_spin)))
    idx = np.sort(rng.choice(ph.n, n, replace=False))
    return idx


def reduce_max(x: float, world: int):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# --------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_2301_02702_b300.workloads import workload
    ph, seq = workload(args.workload, "full")
    threads = os.cpu_count() or 1
    per_step = max(1.0, min(30.0, args.reference_budget_s / max(1, args.steps + args.warmup)))
    idx = cpu_sample_run(ph, seq, per_step, threads)
    sub = ph.subset(idx)
    for _ in range(args.warmup):
        oracle.simulate(sub, seq, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.simulate(sub, seq, threads=threads)
        times.append(time.perf_counter() - t0)
    units = len(idx) * seq.n_steps
    value = units * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "spins": ph.n, "steps_per_sim": seq.n_steps,
                   "n_adc": seq.n_adc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{len(idx)} of {ph.n} spins (random, seed 123) x all {seq.n_steps} steps "
                                   f"per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0




# --------------------------------------------------------------------------
# serving workload
# --------------------------------------------------------------------------
def make_requests(n_req: int, seed: int = 1005):
    """Request mix of the serving workload (phantom, sequence, spin-steps):
    spins log-uniform in [1e3, 1e6] (random subsets of the epi512 and se128
    phantoms), steps log-uniform in [1e3, 1e5] (the gre32, epi512, se128 and
    MRF sequences truncated or repeated)."""
    from paper_2301_02702_b300.workloads import Sequence, workload
    rng = np.random.default_rng(seed)
    phs = [workload("epi512", "full")[0], workload("se128", "full")[0]]
    seqs = [workload(w, "full")[1] for w in ("epi512", "se128", "gre32", "mrf")]

    def take(seq, steps):
        reps = -(-steps // seq.n_steps)
        s = seq
        for _ in range(reps - 1):
            s = s.concat(seq)
        return Sequence(s.dt[:steps], s.gx[:steps + 1], s.gy[:steps + 1], s.gz[:steps + 1], s.b1[:steps],
                        s.adc[:steps + 1])

    out = []
    for _ in range(n_req):
        n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e6)))))
        steps = int(round(np.exp(rng.uniform(np.log(1e3), np.log(1e5)))))
        ph = phs[int(rng.integers(len(phs)))]
        idx = np.sort(rng.choice(ph.n, min(n, ph.n), replace=False))
        seq = take(seqs[int(rng.integers(len(seqs)))], steps)
        out.append((ph.subset(idx), seq, len(idx) * steps))
    return out


def fifo_latencies(arrivals, service):
    """Latencies of requests served one at a time in arrival order."""
    free_at, lat = 0.0, []
    for a, sv in zip(arrivals, service):
        start = max(a, free_at)
        free_at = start + sv
        lat.append(free_at - a)
    return lat


def serve_measure(local: int, n_req: int, rate: float, plain_host: bool = False, n_clients: int = 4,
                  floods: int = 3):
    """Serve a Poisson stream of mixed requests (open loop) and measure
    latency and throughput; then the same requests as floods (saturated
    throughput) and, for comparison, one plain koma_simulate per request on
    device-resident inputs (and optionally koma_simulate_host per request)."""
    import torch
    from paper_2301_02702_b300 import koma
    reqs = make_requests(n_req)
    rng = np.random.default_rng(77)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    total_units = sum(r[2] for r in reqs)
    srv = koma.Server(local, mem_budget_bytes=int(150e9))
    for ph, seq, _ in reqs[:3]:  # warm-up
        srv.wait(srv.submit(ph, seq))

    # open loop: submit at the Poisson arrival times from several client
    # threads (arrival i -> client i % n_clients), collect latencies
    ids = [None] * len(reqs)
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()

    def client(c):
        for i in range(c, len(reqs), n_clients):
            d = t0 + arrivals[i] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids[i] = srv.submit(reqs[i][0], reqs[i][1])

    ths = [threading.Thread(target=client, args=(c,)) for c in range(n_clients)]
    for th in ths:
        th.start()
    lat, infos = [], []
    for i in range(len(reqs)):
        while ids[i] is None:
            time.sleep(0.0005)
        _, info = srv.wait(ids[i])
        lat.append(info["latency_s"])
        infos.append(info)
    for th in ths:
        th.join()
    t_open = time.perf_counter() - t0
    clk = clocks.stop()
    stats = srv.stats()

    # saturation: everything submitted at once by the same client threads;
    # the median of the floods (host threads make single floods noisy)
    sid = [None] * len(reqs)

    def flood(c):
        for i in range(c, len(reqs), n_clients):
            sid[i] = srv.submit(reqs[i][0], reqs[i][1])

    t_floods = []
    for _ in range(floods):
        t1 = time.perf_counter()
        ths = [threading.Thread(target=flood, args=(c,)) for c in range(n_clients)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for rid in sid:
            srv.wait(rid)
        t_floods.append(time.perf_counter() - t1)
    t_sat = statistics.median(t_floods)
    launches = int(srv.stats()["launches"])
    srv.close()

    # plain, device resident: every request's phantom and sequence uploaded
    # beforehand, then one koma_simulate per request back to back on one
    # stream (the readout on the tensor cores where the sequence has
    # matrix-form groups), device time per call from CUDA events
    sim = koma.Simulator(local)
    stream = torch.cuda.Stream(local)
    service_dev = []
    chunk = 64
    for c0 in range(0, len(reqs), chunk):
        part = reqs[c0:c0 + chunk]
        hs_ = [(sim.upload_phantom(ph), sim.upload_sequence(seq), seq.n_adc) for ph, seq, _ in part]
        outs = [torch.empty((1, n_adc), dtype=torch.complex128, device=f"cuda:{local}") for _, _, n_adc in hs_]
        for (hp, hq, _), o in zip(hs_, outs):  # warm: scratch grown, launch tables in place
            sim.simulate(hp, hq, "fp32", out=o, stream=stream)
        sim.sync(stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in hs_]
        for (hp, hq, _), o, (e0, e1) in zip(hs_, outs, evs):
            e0.record(stream)
            sim.simulate(hp, hq, "fp32", out=o, stream=stream)
            e1.record(stream)
        sim.sync(stream)
        service_dev += [e0.elapsed_time(e1) / 1e3 for e0, e1 in evs]
        for hp, hq, _ in hs_:
            koma.koma_sequence_free(hq)
            koma.koma_phantom_free(hp)
    sim.close()
    t_plain_dev = sum(service_dev)
    plain_lat = fifo_latencies(arrivals, service_dev)
    # served roofline: the FP32 flops the kernels execute for the stream (stepped RF
    # steps, pulse steps of the maps and their applications, stepped samples; samples
    # summed on the tensor cores, in the koma_simulate lane, are not FP32 work) over
    # the saturated time, against the FP32 peak
    fp32 = 0.0
    for (ph, seq, _), f in zip(reqs, infos):
        p = koma.koma_sequence_plan(seq)
        per_spin = ((p["n_rf"] - p["n_rf_map_steps"]) * FLOPS_RF_STEP + p["n_rf_map_pulse_steps"] * FLOPS_MAP_STEP
                    + p["n_rf_map_runs"] * FLOPS_MAP_APPLY
                    + (p["n_adc"] - (p["n_mma_samples"] if f["lane"] == 1 else 0)) * FLOPS_ADC_SAMPLE)
        fp32 += float(ph.n) * per_spin
    served_roof = {"bound": "alu", "achieved": fp32 / t_sat / 1e12, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                   "frac": fp32 / t_sat / 1e12 / PEAK_FP32_TFLOPS,
                   "how": "FP32 flops the kernels execute for the whole stream (50 per stepped RF spin-step, "
                          "302 per pulse step of a repeated pulse's map, 18 per map application, 8 per stepped "
                          "sample; samples summed on the tensor cores not counted) / the saturated time"}
    out = {
        "requests": len(reqs), "rate_per_s": rate,
        "mean_spin_steps_per_request": total_units / len(reqs),
        "offered_spin_steps_per_s": total_units / arrivals[-1],
        "served": {"value": total_units / t_open, "unit": UNIT, "seconds": t_open},
        "latency": {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "mean_s": float(np.mean(lat)), "max_s": float(np.max(lat))},
        "saturated": {"value": total_units / t_sat, "unit": UNIT, "seconds": t_sat,
                      "floods_s": [round(t, 4) for t in t_floods], "statistic": f"median of {floods} floods"},
        "plain_device": {"value": total_units / t_plain_dev, "unit": UNIT, "seconds": t_plain_dev,
                         "p50_s": float(np.percentile(plain_lat, 50)),
                         "p99_s": float(np.percentile(plain_lat, 99)),
                         "plain": "one koma_simulate per request on device-resident inputs, back to back on one "
                                  "stream (device time, CUDA events); latencies under the same arrivals"},
        "ratio_saturated_vs_plain_device": t_plain_dev / t_sat,
        "roofline": served_roof,
        "server": {k: stats[k] for k in ("batches", "mem_peak", "completed", "failed", "lane_runs")},
        "lanes": {"requests": [sum(1 for f in infos if f["lane"] == k) for k in (0, 1)],
                  "spin_steps": [sum(r[2] for r, f in zip(reqs, infos) if f["lane"] == k) for k in (0, 1)],
                  "prep_s_total": sum(f["prep_s"] for f in infos),
                  "prep_s_by_lane": [sum(f["prep_s"] for f in infos if f["lane"] == k) for k in (0, 1)],
                  "upload_s_total": sum(f["upload_s"] for f in infos),
                  "run_s_total": sum(f["run_s"] for f in infos),
                  "how": "open-loop stream: requests and spin-steps per lane (0 shared launches, 1 koma_simulate "
                         "lane); host seconds summed over requests"},
        "server_launches": launches,
        "clocks": clk,
    }
    if plain_host:
        # plain through the host API: one koma_simulate_host per request
        # (upload, simulate, copy back), one at a time in arrival order
        ctx = koma.koma_init(local)
        service = []
        for ph, seq, _ in reqs:
            buf = np.empty((1, seq.n_adc), dtype=np.complex128)
            ts = time.perf_counter()
            koma.koma_simulate_host(ctx, ph, seq, koma.KOMA_FP32_SPLITPHASE, out=buf)
            service.append(time.perf_counter() - ts)
        koma.koma_destroy(ctx)
        hl = fifo_latencies(arrivals, service)
        out["plain_host"] = {"value": total_units / sum(service), "unit": UNIT, "seconds": sum(service),
                             "p50_s": float(np.percentile(hl, 50)), "p99_s": float(np.percentile(hl, 99)),
                             "plain": "koma_simulate_host per request (upload, simulate, copy back), one at a "
                                      "time in arrival order; latencies under the same arrivals"}
    return out


def run_serve(args, rank, world, local):
    import torch
    from paper_2301_02702_b300 import build, koma
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(koma.LIB_PATH):
        build.build()
    barrier(world)
    r = serve_measure(local, args.requests, args.rate, plain_host=True)
    # replicas: every rank serves its own stream; the slowest rank's time counts
    t_open = reduce_max(r["served"]["seconds"], world)
    value = r["served"]["value"] * r["served"]["seconds"] / t_open * world
    if rank == 0:
        line = {
            "metric": "Bloch spin-steps/s served (open-loop Poisson load); p50/p99 latency", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": r["requests"], "warmup": 3,
            "ms_per_step": 1e3 * r["served"]["seconds"] / r["requests"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["serve"], "requests": r["requests"], "rate_per_s": args.rate,
                       "parallelism": f"replicas x{world}"},
            "serving": r,
            "gpu_launches": r["server_launches"],
            "clocks": r["clocks"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def parity_case(name, ph, seq):
    """(phantom to launch, phantom the oracle runs, description, group rows)
    of the parity check in the benchmark's launch configuration. Every spin
    contributes except for se128 (a contiguous slab of 65,536 spins around
    the excited slice, PD = 0 elsewhere: the signal is then the slab's) and
    the MRF dictionary (200 random entries, each an independent output)."""
    from paper_2301_02702_b300.workloads import Phantom
    if ph.n_groups > 1:
        rng = np.random.default_rng(11)
        groups = np.sort(rng.choice(ph.n_groups, min(ph.n_groups, 200), replace=False))
        idx = np.concatenate([np.arange(ph.group_offsets[g], ph.group_offsets[g + 1]) for g in groups])
        offs = np.concatenate([[0], np.cumsum(np.diff(ph.group_offsets)[groups])])
        sub = Phantom(ph.x[idx], ph.y[idx], ph.z[idx], ph.pd[idx], ph.t1[idx], ph.t2[idx], ph.dw[idx],
                      group_offsets=offs)
        return ph, sub, (f"{len(groups)} random dictionary entries of the full launch vs FP64 oracle "
                         f"(per-entry max-abs error over the entry's maximum)"), groups
    if name == "se128":
        lo = ph.n // 2 - SE128_PARITY_SLAB // 2
        keep = np.arange(lo, lo + SE128_PARITY_SLAB)
        pd = np.zeros(ph.n)
        pd[keep] = ph.pd[keep]
        masked = Phantom(ph.x, ph.y, ph.z, pd, ph.t1, ph.t2, ph.dw, velocity=ph.velocity)
        return masked, ph.subset(keep), (f"full {ph.n}-spin launch with a contiguous slab of {len(keep)} spins "
                                         f"around the excited slice kept (PD = 0 elsewhere) vs FP64 oracle on the "
                                         f"slab"), None
    return ph, ph, f"every spin ({ph.n}) of the full launch vs FP64 oracle", None


def rel_err_of(got, ref, groups):
    if groups is not None:
        return float(np.max(np.max(np.abs(got[groups] - ref), axis=1) / np.max(np.abs(ref), axis=1)))
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def run_ours(args, rank, world, local):
    import torch
    from paper_2301_02702_b300 import build, koma
    from paper_2301_02702_b300.workloads import Phantom, Sequence, workload

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(koma.LIB_PATH):
        build.build()
    barrier(world)

    ph, seq = workload(args.workload, "full")
    sim = koma.Simulator(local)
    hp = sim.upload_phantom(ph)
    hs = sim.upload_sequence(seq)
    info = koma.koma_sequence_get_info(hs)
    stream = torch.cuda.Stream(local)
    out = torch.empty((ph.n_groups, seq.n_adc), dtype=torch.complex128, device=f"cuda:{local}")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")  # > 126 MB L2
    grouped = ph.n_groups > 1
    moving = ph.velocity is not None
    tuned = sim.tune(hp, hs, stream) if (grouped or args.tune) else None

    def run_once(handle, mma=True):
        koma.koma_set_mma(sim.ctx, mma)
        with torch.cuda.stream(stream):
            sim.simulate(handle, hs, "fp32", out=out, stream=stream)
        sim.sync(stream)
        koma.koma_set_mma(sim.ctx, True)
        return out.cpu().numpy()

    # parity in this launch configuration against the FP64 oracle
    parity = None
    par_handle, par_ref, par_groups = None, None, None
    if rank == 0 and not args.no_parity:
        import oracle
        launch_ph, oracle_ph, desc, par_groups = parity_case(args.workload, ph, seq)
        par_handle = hp if launch_ph is ph else sim.upload_phantom(launch_ph)
        got = run_once(par_handle)
        t0 = time.perf_counter()
        par_ref = oracle.simulate(oracle_ph, seq)
        t_or = time.perf_counter() - t0
        err = rel_err_of(got, par_ref, par_groups)
        parity = {"rel_err": err, "tol": TOL, "pass": err <= TOL, "sample": desc,
                  "oracle_s": round(t_or, 1)}

    koma.koma_set_timing(sim.ctx, True)
    for _ in range(args.warmup):
        sim.simulate(hp, hs, "fp32", out=out, stream=stream)
    sim.sync(stream)
    launch = sim.launch_info()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_ms = []
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(local)
    clocks.start()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()                       # L2 flush between timed steps (not timed)
            ev[i][0].record(stream)
            sim.simulate(hp, hs, "fp32", out=out, stream=stream)
            ev[i][1].record(stream)
        if args.kernel_timing:
            stage_ms.append(koma.koma_get_stage_timing(sim.ctx) + (koma.koma_get_map_timing(sim.ctx),))
    torch.cuda.synchronize(local)
    barrier(world)
    clk = clocks.stop()
    sim.sync(stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms_max = reduce_max(ms, world)
    units = ph.n * seq.n_steps
    value = units * world / (ms_max / 1e3)

    # the same step with every ADC sample stepped by the Bloch kernel (no
    # tensor cores), with its own parity against the same oracle result
    no_mma = None
    if rank == 0 and launch.get("mma_grid", 0) > 0:
        koma.koma_set_mma(sim.ctx, False)
        for _ in range(2):
            sim.simulate(hp, hs, "fp32", out=out, stream=stream)
        sim.sync(stream)
        n_nm = max(1, min(args.steps, 5))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_nm)]
        for e0, e1 in evs:
            with torch.cuda.stream(stream):
                flush.zero_()
                e0.record(stream)
                sim.simulate(hp, hs, "fp32", out=out, stream=stream)
                e1.record(stream)
        sim.sync(stream)
        nm_ms = sum(a.elapsed_time(b) for a, b in evs) / n_nm
        koma.koma_set_mma(sim.ctx, True)
        no_mma = {"value": units / (nm_ms / 1e3), "unit": UNIT, "ms_per_step": nm_ms, "steps": n_nm,
                  "path": "koma_set_mma(ctx, 0): every ADC sample stepped by the Bloch kernel (FP32 pipes only)"}
        if par_handle is not None:
            err = rel_err_of(run_once(par_handle, mma=False), par_ref, par_groups)
            no_mma["rel_err"] = err
            no_mma["pass"] = err <= TOL
    # gre32 is specified in FP64: the same step through KOMA_FP64 (one spin per
    # thread, every sample evaluated in FP64), with its own parity
    fp64_leg = None
    if rank == 0 and args.workload == "gre32":
        for _ in range(2):
            sim.simulate(hp, hs, "fp64", out=out, stream=stream)
        sim.sync(stream)
        n64 = max(1, min(args.steps, 5))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n64)]
        for e0, e1 in evs:
            with torch.cuda.stream(stream):
                flush.zero_()
                e0.record(stream)
                sim.simulate(hp, hs, "fp64", out=out, stream=stream)
                e1.record(stream)
        sim.sync(stream)
        ms64 = sum(a.elapsed_time(b) for a, b in evs) / n64
        fp64_leg = {"value": units / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": n64, "dtype": "f64",
                    "path": "KOMA_FP64: every operation in FP64, one spin per thread, every sample evaluated"}
        if par_handle is hp and par_ref is not None:
            with torch.cuda.stream(stream):
                sim.simulate(hp, hs, "fp64", out=out, stream=stream)
            sim.sync(stream)
            err = rel_err_of(out.cpu().numpy(), par_ref, par_groups)
            fp64_leg["rel_err"] = err
            fp64_leg["pass"] = err <= 1e-9
    # the same step with every RF step stepped (repeated pulses not taken by
    # their maps), with its own parity
    no_maps = None
    if rank == 0 and info.get("n_rf_maps", 0) > 0 and not grouped and not moving:
        koma.koma_set_rf_maps(sim.ctx, False)
        for _ in range(2):
            sim.simulate(hp, hs, "fp32", out=out, stream=stream)
        sim.sync(stream)
        n_nm = max(1, min(args.steps, 5))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_nm)]
        for e0, e1 in evs:
            with torch.cuda.stream(stream):
                flush.zero_()
                e0.record(stream)
                sim.simulate(hp, hs, "fp32", out=out, stream=stream)
                e1.record(stream)
        sim.sync(stream)
        nm_ms = sum(a.elapsed_time(b) for a, b in evs) / n_nm
        no_maps = {"value": units / (nm_ms / 1e3), "unit": UNIT, "ms_per_step": nm_ms, "steps": n_nm,
                   "path": "koma_set_rf_maps(ctx, 0): every RF step of the repeated pulses stepped by the Bloch "
                           "kernel"}
        if par_handle is not None:
            got = None
            koma.koma_set_rf_maps(sim.ctx, False)
            got = run_once(par_handle)
            err = rel_err_of(got, par_ref, par_groups)
            no_maps["rel_err"] = err
            no_maps["pass"] = err <= TOL
        koma.koma_set_rf_maps(sim.ctx, True)
    if par_handle is not None and par_handle is not hp:
        koma.koma_phantom_free(par_handle)

    # the plain path for a dictionary: one koma_simulate per entry (sample)
    vs_plain = None
    if grouped and rank == 0:
        rng = np.random.default_rng(3)
        groups = rng.choice(ph.n_groups, min(ph.n_groups, 200), replace=False)
        handles = []
        for g in groups:
            lo, hi = int(ph.group_offsets[g]), int(ph.group_offsets[g + 1])
            handles.append((sim.upload_phantom(ph.subset(np.arange(lo, hi))), hi - lo))
        one = torch.empty((1, seq.n_adc), dtype=torch.complex128, device=f"cuda:{local}")
        for h, _ in handles[:5]:
            sim.simulate(h, hs, "fp32", out=one, stream=stream)
        sim.sync(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for h, _ in handles:
            sim.simulate(h, hs, "fp32", out=one, stream=stream)
        e1.record(stream)
        sim.sync(stream)
        plain_ms = e0.elapsed_time(e1)
        plain_units = sum(c for _, c in handles) * seq.n_steps
        plain_value = plain_units / (plain_ms / 1e3)
        for h, _ in handles:
            koma.koma_phantom_free(h)
        vs_plain = {"plain_value": plain_value, "unit": UNIT, "ratio": value / plain_value,
                    "plain": f"one koma_simulate per dictionary entry, {len(handles)} random entries back to back "
                             f"on one stream ({plain_ms:.1f} ms)"}

    # end to end through the public host API: host arrays in, host signal out. The
    # inputs and the result live in pinned host memory (as a serving front end keeps
    # them); every step copies them to and from the device inside the timed region.
    e2e = None
    pinned_keep = []

    def pinned(a):
        a = np.ascontiguousarray(a)
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0].copy()).dtype, pin_memory=True)
        out_ = t.numpy()
        out_[...] = a
        pinned_keep.append(t)
        return out_

    if not args.no_e2e:
        ph_host = Phantom(*(pinned(getattr(ph, f)) for f in ("x", "y", "z", "pd", "t1", "t2", "dw")),
                          group_offsets=None if ph.group_offsets is None else pinned(ph.group_offsets),
                          velocity=None if ph.velocity is None else pinned(ph.velocity))
        seq_host = Sequence(*(pinned(a) for a in (seq.dt, seq.gx, seq.gy, seq.gz, seq.b1, seq.adc)))
    if not args.no_e2e and moving:
        # moving phantoms: upload (with the velocities), simulate, copy the
        # signal back and free, every step, through the Simulator API
        host_sig = pinned(np.empty((ph.n_groups, seq.n_adc), dtype=np.complex128))

        def e2e_step():
            p_ = sim.upload_phantom(ph_host)
            s_ = sim.upload_sequence(seq_host)
            sig = sim.simulate(p_, s_, "fp32", stream=stream)
            sim.sync(stream)
            host_sig[...] = sig.cpu().numpy()
            koma.koma_sequence_free(s_)
            koma.koma_phantom_free(p_)

        for _ in range(max(3, args.warmup)):
            e2e_step()
        n_e2e = max(1, min(args.steps, args.e2e_steps))
        barrier(world)
        gc.collect()
        gc.disable()  # no interpreter collection pause inside the timed calls
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        t_e2e = time.perf_counter() - t0
        gc.enable()
        t_e2e = reduce_max(t_e2e / n_e2e, world)
        n_pad = max(32, (ph.n + 31) // 32 * 32)
        # raw FP64 phantom rows, velocity blocks (FP32 hi/lo + FP64), three record streams
        h2d = ph.n * 7 * 8 + n_pad * (6 * 4 + 3 * 8) + info["n_records"] * (64 + 128 + 128)
        e2e = {"value": units * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(ph.n_groups * seq.n_adc * 16),
               "path": "Simulator from pinned host arrays: phantom + velocity upload, sequence preprocessing + "
                       "upload, simulate, signal copy-back into pinned memory, free"}
    elif not args.no_e2e:
        sim2 = koma.Simulator(local)  # a context of its own
        ctx2 = sim2.ctx
        if tuned is not None:
            # a user tunes a shape once; later host calls of that shape reuse the choice
            hp2, hs2 = sim2.upload_phantom(ph), sim2.upload_sequence(seq)
            sim2.tune(hp2, hs2, stream)
            koma.koma_sequence_free(hs2)
            koma.koma_phantom_free(hp2)
        host_sig = pinned(np.empty((ph.n_groups, seq.n_adc), dtype=np.complex128))
        n_e2e = max(1, min(args.steps, args.e2e_steps))
        # one pinned signal buffer per job of the batch
        sigs = [pinned(np.empty((ph.n_groups, seq.n_adc), dtype=np.complex128)) for _ in range(n_e2e)]
        for _ in range(max(3, args.warmup)):  # warm-up calls, as for the device-timed steps
            koma.koma_simulate_host(ctx2, ph_host, seq_host, koma.KOMA_FP32_SPLITPHASE, out=host_sig)
        koma.koma_simulate_host_batch(ctx2, [(ph_host, seq_host, sigs[i]) for i in range(min(4, n_e2e))])
        barrier(world)
        gc.collect()
        gc.disable()  # no interpreter collection pause inside the timed calls
        # the timed region: one batch of n_e2e host-buffer simulations (each
        # job's inputs copied up and its signal copied back; one job's host
        # work overlapped with the previous job's simulation)
        t0 = time.perf_counter()
        koma.koma_simulate_host_batch(ctx2, [(ph_host, seq_host, sigs[i]) for i in range(n_e2e)])
        t_e2e = (time.perf_counter() - t0) / n_e2e
        # one call at a time, for the latency of a single simulation
        calls = []
        for _ in range(n_e2e):
            c0 = time.perf_counter()
            koma.koma_simulate_host(ctx2, ph_host, seq_host, koma.KOMA_FP32_SPLITPHASE, out=host_sig)
            calls.append(time.perf_counter() - c0)
        gc.enable()
        t_e2e = reduce_max(t_e2e, world)
        assert all(np.array_equal(sg, host_sig) for sg in sigs)  # every job's signal arrived
        sim2.close()
        # raw FP64 phantom rows (the FP32 block is built on the device), the FP32 record
        # stream (the host call builds no FP64 or motion stream for an FP32 static
        # simulation), the compacted stream of the mapped pulses, the readout tables
        n_rec_c = (info["n_records"] - info.get("n_rf_map_steps", 0) + info.get("n_rf_map_runs", 0)
                   if info.get("n_rf_maps", 0) else 0)
        h2d = (ph.n * 7 * 8 + 64 * (info["n_records"] + n_rec_c) + 64 * info.get("n_mma_runs", 0)
               + info["n_adc"] + 16 * info.get("n_rf_maps", 0))
        e2e = {"value": units * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(ph.n_groups * seq.n_adc * 16),
               "ms_per_step": 1e3 * t_e2e, "steps": n_e2e,
               "path": "koma_simulate_host_batch of the steps from pinned host arrays: per step validation + "
                       "preprocessing + uploads + simulate + signal copy-back into pinned memory, one step's "
                       "host work overlapped with the previous step's simulation",
               "single_call": {"ms_median": 1e3 * float(np.median(calls)), "ms_max": 1e3 * max(calls),
                               "calls": n_e2e, "value": units * world / float(np.median(calls)),
                               "path": "koma_simulate_host, one call at a time"}}

    # CPU baseline: the oracle on a bounded spin sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        threads = os.cpu_count() or 1
        idx = cpu_sample_run(ph, seq, args.cpu_target_s, threads)
        t0 = time.perf_counter()
        oracle.simulate(ph.subset(idx), seq, threads=threads)
        dt = time.perf_counter() - t0
        cpu = {"value": len(idx) * seq.n_steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{len(idx)} of {ph.n} spins (random, seed 123) x all {seq.n_steps} steps, "
                         f"{dt:.1f} s"}

    # serving: a Poisson stream of mixed requests through the server (rank 0)
    serving = None
    if rank == 0 and args.workload == "se128" and args.serving_requests > 0:
        serving = serve_measure(local, args.serving_requests, args.rate)

    line = None
    if rank == 0:
        line = result_line(args, world, ph, seq, info, launch, stage_ms, clk, value, ms_max, tuned, moving,
                           grouped)
        line.update({"cpu_baseline": cpu, "e2e": e2e, "parity": parity})
        if no_mma is not None:
            line["no_tensor_cores"] = no_mma
        if fp64_leg is not None:
            line["fp64"] = fp64_leg
        if no_maps is not None:
            line["no_rf_maps"] = no_maps
        if vs_plain is not None:
            line["vs_plain"] = vs_plain
        if serving is not None:
            line["serving"] = serving
        print(json.dumps(line), flush=True)
    koma.koma_sequence_free(hs)
    koma.koma_phantom_free(hp)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def result_line(args, world, ph, seq, info, launch, stage_ms, clk, value, ms_max, tuned, moving, grouped):
    """The JSON line of our arm: the metric, the launch, and the roofline of
    each kernel of the step (with the step's time-weighted fraction)."""
    k1 = k6 = k2 = k7 = None
    if stage_ms:
        k7 = sum(t[3] for t in stage_ms) / len(stage_ms)
        k1 = sum(t[0] for t in stage_ms) / len(stage_ms) - k7  # the stage includes the map pre-pass
        k6 = sum(t[1] for t in stage_ms) / len(stage_ms)
        k2 = sum(t[2] for t in stage_ms) / len(stage_ms)
    mma = launch.get("mma_grid", 0) > 0
    mma_samples = info.get("n_mma_samples", 0) if mma else 0
    maps = bool(k7) and info.get("n_rf_maps", 0) > 0
    flops_all = algorithmic_flops(info, ph.n, moving)
    # the Bloch kernel's share: the RF steps and samples it steps, and the
    # maps it applies
    flops = flops_all - float(ph.n) * mma_samples * FLOPS_ADC_SAMPLE
    if maps:
        flops -= float(ph.n) * info["n_rf_map_steps"] * FLOPS_RF_STEP
        flops += float(ph.n) * info["n_rf_map_runs"] * FLOPS_MAP_APPLY
    achieved = flops / (k1 / 1e3) / 1e12 if k1 else None
    kname = "bloch_motion_kernel" if moving else ("bloch_items_kernel" if grouped else "bloch_fp32_kernel")
    if grouped and launch["spins_per_thread"] == 8:
        kname = "bloch_items_z_kernel"  # the dictionary kernel for isochromats along z, 8 spins per thread
    roofs = []
    if maps:
        mflops = float(ph.n) * info["n_rf_map_pulse_steps"] * FLOPS_MAP_STEP
        roofs.append({"bound": "alu", "kernel": "rf_map_kernel", "achieved": mflops / (k7 / 1e3) / 1e12,
                      "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                      "frac": mflops / (k7 / 1e3) / 1e12 / PEAK_FP32_TFLOPS,
                      "traffic": measured_traffic(args.workload + ":rf_map"), "kernel_ms": k7,
                      "algorithmic_flops_per_launch": mflops,
                      # 7 FP32 phantom rows read, 12 map floats per spin and pulse written
                      "algorithmic_bytes_per_launch": 4.0 * ph.n * (7 + 12 * info["n_rf_maps"]),
                      "peak_source": "FP32 peak 148 SMs x 128 lanes x 2 x 2032 MHz (unit counts, max SM clock)",
                      "pulses": info["n_rf_maps"], "pulse_steps": info["n_rf_map_pulse_steps"],
                      "replaces_rf_steps": info["n_rf_map_steps"]})
    kfull = kname if kname == "bloch_items_z_kernel" else f"{kname}<{launch['spins_per_thread']}>"
    roof1 = {"bound": "alu", "kernel": kfull,
             "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
             "frac": (achieved / PEAK_FP32_TFLOPS) if achieved else None,
             "traffic": measured_traffic(args.workload),
             "kernel_ms": k1, "algorithmic_flops_per_launch": flops,
             "peak_source": "FP32 peak 148 SMs x 128 lanes x 2 x 2032 MHz (unit counts, max SM clock)"}
    if kname == "bloch_items_z_kernel":
        # its partial rows, plus z, M0, 1/T1, 1/T2 (FP32) per spin and 12 B per
        # unit of <= 8 spins of one group (the work table)
        units = int(np.sum((np.diff(ph.group_offsets) + 7) // 8))
        roof1["algorithmic_bytes_per_launch"] = float(launch["partial_bytes"]) + 16.0 * ph.n + 12.0 * units
    roofs.append(roof1)
    if mma and k6:
        peak_t, peak_src = tensor_peak()
        blocks = (ph.n + 31) // 32
        tflops = float(blocks) * info["n_mma_groups"] * MMA_FLOPS_PER_BLOCK_GROUP
        direct = float(ph.n) * mma_samples * FLOPS_ADC_SAMPLE
        roofs.append({"bound": "tensor", "kernel": "readout_mma_kernel", "achieved": tflops / (k6 / 1e3) / 1e12,
                      "peak": peak_t, "unit": "TFLOP/s", "frac": tflops / (k6 / 1e3) / 1e12 / peak_t,
                      "traffic": measured_traffic(args.workload + ":readout"), "kernel_ms": k6,
                      "tensor_flops_per_launch": tflops, "peak_source": peak_src + " (of measured)",
                      "samples": mma_samples, "direct_sum_flops_per_launch": direct,
                      "direct_sum_tflops": direct / (k6 / 1e3) / 1e12})
    if k2 and not grouped:
        # the reduction reads each sample's partial rows once (8 B per row and
        # sample) and writes the FP64 signal (16 B per sample)
        peak_h, hsrc = hbm_peak()
        rows1 = launch["grid"] // max(1, launch.get("split", 1))
        n_adc = info["n_adc"]
        rb = 8.0 * (rows1 * (n_adc - mma_samples) + launch.get("mma_grid", 0) * mma_samples) + 16.0 * n_adc
        if mma:
            rb += n_adc  # the per-sample source map
        roofs.append({"bound": "hbm", "kernel": "reduce_partials_kernel", "achieved": rb / (k2 / 1e3) / 1e9,
                      "peak": peak_h, "unit": "GB/s", "frac": rb / (k2 / 1e3) / 1e9 / peak_h,
                      "traffic": None, "kernel_ms": k2, "algorithmic_bytes_per_launch": rb,
                      "peak_source": hsrc + " (of measured)"})
    roofs.sort(key=lambda r: -(r["kernel_ms"] or 0.0))
    step = None
    if k1:
        tot = sum(r["kernel_ms"] for r in roofs)
        step = {"kernels_ms": tot, "frac": sum(r["kernel_ms"] * r["frac"] for r in roofs) / tot,
                "how": "kernel-time-weighted mean of the step's kernels' roofline fractions"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "spins": ph.n, "steps_per_sim": seq.n_steps,
                   "n_adc": seq.n_adc, "n_rf": info["n_rf"], "records": info["n_records"],
                   "precision": "KOMA_FP32_SPLITPHASE", "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world}",
                   "launch": {k: launch[k] for k in ("grid", "block", "spins_per_thread", "spins_per_cta",
                                                     "mma_grid")}},
        "roofline": roofs[0],
        "roofline_other": roofs[1:],
        "roofline_step": step,
        "gpu_launches": launch["kernels"] * args.steps,
        "clocks": clk,
    }
    if tuned is not None:
        line["config"]["tuned"] = {k: tuned[k] for k in ("grid", "block", "spins_per_thread", "tile_records")}
    return line


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOAD_TEXT), default="se128")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--cpu-target-s", type=float, default=15.0)
    ap.add_argument("--reference-budget-s", type=float, default=150.0)
    ap.add_argument("--no-kernel-timing", dest="kernel_timing", action="store_false")
    ap.add_argument("--tune", action="store_true", help="autotune the launch first (grouped workloads always do)")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: number of requests")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests of the serving stream in the se128 line (0: none)")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: Poisson arrival rate, 1/s")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        if args.workload == "serve":
            args.workload = "se128"
        return run_reference(args, rank, world)
    if args.workload == "serve":
        return run_serve(args, rank, world, local)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
