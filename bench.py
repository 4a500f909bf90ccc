"""Benchmark: phase-space cell-updates/s of the per-step VFP update on B300.

Default (N=1 GPU): a batched scan of N=256 grids shaped like the paper's
current scans (S_csr on a grid in [0.2, 1.5] x Pi in {1, 2, 3}, 1000 steps per
synchrotron period, FP32 psi with FP64 sums), with enough instances that the
double-buffered state (2 x instances x 256 KB) exceeds the 126 MB L2, so every
step streams psi through HBM.  One timed step = one fused launch that advances
every instance by one time step (rotation, kick, Fokker-Planck, projection,
FFT wake, CSR power, renormalisation).

Printed (one JSON line on rank 0): value (cell-updates/s over all ranks),
the plain single-simulation path at N=256 for comparison, a roofline object
for the fused kernel (algorithmic 8 B per cell per step over the kernel's
CUDA-event time, against the measured HBM copy bandwidth), the FP64 oracle
timed on the host cores on a bounded sample (cpu_baseline), an end-to-end
figure through the C ABI with host buffers (e2e) and the SM clocks sampled
during the timed region.

--impl reference times the FP64 CPU oracle (the method's reference
implementation here) on the same workload shape, bounded to a few minutes.
Multi-GPU (torchrun): one independent batch per rank, no collective; the
barrier-bracketed time is the max over ranks (weak scaling, replicas).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6400.0

PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_kernel_f32_batched_n256.md")


def kernel_source_digest() -> str:
    """sha256 (16 hex digits) of the CUDA sources the step kernels are built from."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1611_05293_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def measured_traffic_per_launch():
    """DRAM bytes (read + write) of one launch of the batched step kernel, from
    the ncu summary of the headline kernel -- only if that capture was taken of
    the kernel sources built now (its `kernel-sources` digest matches);
    otherwise None."""
    try:
        kv = {}
        for line in open(PROFILE_SUMMARY):
            if line.startswith("<!-- ") and ":" in line:
                k, v = line[5:].split("-->")[0].split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel-sources") == kernel_source_digest():
            return float(kv["dram-bytes-per-launch"]), kv.get("launch-shape", "")
    except (OSError, KeyError, ValueError):
        pass
    return None, ""


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [x for x in (num(r[0]) for r in self.rows) if x is not None]
        mx = [x for x in (num(r[1]) for r in self.rows) if x is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def head_start(torch, stream, ms: float = 3.0):
    """A few milliseconds of dense GEMMs on `stream`, queued right before the
    first event of a timed region: the SMs are busy (and clocked up) while the
    host queues the timed steps, so the region measures the steps and not the
    GPU's wake-up from idle or the host's launch pace (measured: 20 steps
    after a 0.3 s idle gap 149 us per step, after busy work 114, steady
    state 113.5)."""
    a = torch.randn(4096, 4096, device="cuda", dtype=torch.bfloat16)
    with torch.cuda.stream(stream):
        for _ in range(max(1, int(ms / 0.1))):  # ~0.1 ms per 4096^3 GEMM
            torch.mm(a, a)


def scan_points(count: int, rank: int = 0, world: int = 1):
    """(S, Pi) of this rank's `count` instances: ranks take consecutive,
    disjoint slices of one scan of count * world points (replicas, weak
    scaling: every rank runs its own simulations, no collective)."""
    from paper_1611_05293_b300 import workloads as W
    base = W.scan_grid()
    return [base[i % len(base)] for i in range(rank * count, (rank + 1) * count)]


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time is the slowest rank's (all_reduce MAX; no-op alone)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


PIN_SHAPE = None  # (W, tiles per strip) from --shape: fixed launch shape instead of the autotuner's
PAIRING = False   # --pairing: simulations of one geometry two at a time (pair kernel)


def build_batch(V, count, n, spp, beta, stream, seed=1612, rotation=0, rank=0, world=1):
    from paper_1611_05293_b300 import workloads as W
    b = V.Batch(count, 0, stream)
    if PIN_SHAPE:
        b.pin_shape(*PIN_SHAPE)
    b.pairing(PAIRING)
    psi0 = W.noisy_gaussian(n, seed, 1e-6)
    for S, Pi in scan_points(count, rank, world):
        b.add(V.Params(n=n, steps_per_period=spp, beta=beta, rotation=rotation), psi0, V.IMPEDANCE_PARALLEL_PLATES,
              Pi, S, nsteps=1 << 40)
    return b


def calibrate(V, torch, stream, count, n=256, spp=1000, beta=1e-2, rotation=0, steps=480):
    """Let the library's autotuner time its candidate launch shapes for this
    batch configuration on a throwaway batch (480 steps), so that the timed
    batch built next starts with the tuned shape (the choice is cached per
    configuration for the process)."""
    b = build_batch(V, count, n, spp, beta, stream, rotation=rotation)
    b.run(steps)
    torch.cuda.synchronize()
    b.close()


def manhattan_scan(V, torch, stream, warmup, count=512, steps=200):
    """The headline scan with the Manhattan rotation (drift, then RF kick; two
    1-D cubic interpolations instead of one 2-D) in place of the standard one."""
    calibrate(V, torch, stream, count, rotation=1)
    b = build_batch(V, count, 256, 1000, 1e-2, stream, rotation=1)
    b.run(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    head_start(torch, stream)
    e0.record(stream)
    b.run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    b.close()
    value = count * 65536 * steps / dt
    return {"value": value, "unit": "cell-updates/s", "ms_per_step": 1e3 * dt / steps,
            "roofline_frac": 8.0 * value / 1e9 / measured_peaks()[0],
            "workload": f"{count} x N=256 scan, Manhattan rotation"}


def serving(V, torch, stream, count=500, seed=1613, budget_mb=64):
    """The served uneven batch: a Poisson stream of `count` requests shaped like
    the paper's scans (N in {128, 256, 512, 1024}, S in U[0.2, 2], Pi in
    U[0.5, 4], 1000-4000 steps per period, 5-50 periods), an admission cap
    of budget_mb of device memory (so that requests queue for memory) and 64
    slots.  The arrival rate is 0.9 x the capacity measured first on the
    same cap -- a throwaway batch filled from the stream's own first
    requests -- and the middle fifth of the stream arrives at twice that
    rate (an overload burst)."""
    from paper_1611_05293_b300 import workloads as W
    from paper_1611_05293_b300.serve import Server
    budget = budget_mb << 20
    probe = W.request_stream(count, 1.0, seed)
    mean_cells = float(np.mean([r.cell_updates for r in probe]))
    # capacity under the cap: admit in stream order until the cap refuses,
    # then time a few chunks of the mix
    cal = V.Batch(64, budget, stream)
    for r in probe:
        if cal.try_add(V.Params(n=r.n, steps_per_period=r.steps_per_period, beta=1e-2), None,
                       V.IMPEDANCE_PARALLEL_PLATES, r.Pi, r.s_csr, nsteps=1 << 40) is None:
            break
    cal.run(256)
    torch.cuda.synchronize()
    cells = sum(p_.n * p_.n for p_ in cal.params.values())
    t0 = time.perf_counter()
    cal.run(2048)
    cal.poll()
    cap_cells = cells * 2048 / (time.perf_counter() - t0)
    cal.close()
    rate = 0.9 * cap_cells / mean_cells
    reqs = W.request_stream(count, rate, seed)
    # the burst: arrivals lo .. hi-1 come at twice the rate (their gaps are
    # halved), and everything after them moves up by the time saved
    lo, hi = (2 * count) // 5, (3 * count) // 5
    a = [r.arrival_s for r in reqs]
    saved = 0.5 * (a[hi] - a[lo])
    for i in range(lo, count):
        reqs[i].arrival_s = a[lo] + 0.5 * (a[i] - a[lo]) if i < hi else a[i] - saved
    srv = Server(max_slots=64, budget_bytes=budget, chunk_steps=1000, beta=1e-2, stream=stream, keep_psi=False)
    stats = srv.run(reqs, realtime=True)
    srv.close()
    out = stats.summary()
    out.update({"arrival_rate_per_s": rate, "burst": f"requests {lo}-{hi - 1} at 2x the rate",
                "capacity_cell_updates_per_s": cap_cells, "budget_bytes": budget,
                "unit": "s (time to result)",
                "workload": f"{count} Poisson requests, N in {{128,256,512,1024}}, 1000-4000 steps/period, "
                            f"5-50 periods, 64 slots, {budget_mb} MB admission cap"})
    return out


def moments_cost(V, torch, stream, warmup, count=512, steps=200, every=10):
    """What recording the bunch moments in the step epilogue costs: the
    headline scan with every slot recording {<q>, sigma_q, <p>, sigma_p}
    every `every` steps, against the same scan without."""
    out = {}
    for rec in (0, every):
        b = build_batch(V, count, 256, 1000, 1e-2, stream)
        if rec:
            for sl in range(count):
                b.record_moments(sl, rec)
        b.run(max(warmup, 64))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        head_start(torch, stream)
        e0.record(stream)
        b.run(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        out["every_%d" % rec if rec else "off"] = e0.elapsed_time(e1) / steps * 1e3
        b.close()
    return {"us_per_step": out, "workload": f"{count} x N=256 scan, moments recorded every {every} steps vs off",
            "cost_per_recorded_step_us": (out[f"every_{every}"] - out["off"]) * every}


def spectrogram_cost(V, torch, stream, count=512, length=1024, hop=512, windows=16):
    """One vfps_batch_spectrogram call over every slot of the headline scan:
    `windows` windows of `length` CSR-power values each, in one launch."""
    b = build_batch(V, count, 256, 1000, 1e-2, stream)
    b.run(length + (windows - 1) * hop)
    torch.cuda.synchronize()
    slots = list(range(count))
    b.spectrogram(slots, length, hop, windows)  # warm-up (kernel attributes, memory pool)
    t0 = time.perf_counter()
    b.spectrogram(slots, length, hop, windows)
    dt = time.perf_counter() - t0
    b.close()
    return {"ms_per_call": 1e3 * dt, "windows": count * windows,
            "workload": f"{count} slots x {windows} windows of {length} values (hop {hop}), one launch, wall clock "
                        "including the copy of the spectra to the host"}


def c3_scan_64(V, torch, stream, warmup, steps=100):
    """The 64-instance N=256 scan itself: its state (32 MiB) fits in L2, so L2 is
    flushed (a 256 MiB write) before every timed step and only the steps are timed."""
    calibrate(V, torch, stream, 64)
    b = build_batch(V, 64, 256, 1000, 1e-2, stream)
    b.run(warmup)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    total = 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(1)
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1) / 1e3
    b.close()
    return {"value": 64 * 65536 * steps / total, "unit": "cell-updates/s", "ms_per_step": 1e3 * total / steps,
            "l2": "flushed before every timed step"}


GRAPH_STEPS = 32  # batches replay CUDA graphs of this many steps; timed step counts are whole graphs


def solo_warmup(sim, warmup):
    """Warm-up of a lone simulation before its timed region (it steps in
    persistent launches, or in CUDA graphs of GRAPH_STEPS steps where those do
    not apply): at least 2 GRAPH_STEPS steps."""
    sim.step(max(warmup, 2 * GRAPH_STEPS))


def c3_n1024_64(V, torch, stream, warmup, steps=64):
    """A 64-instance copy of the scan at N=1024 (4000 steps/period): its state
    (2 x 268 MB) exceeds L2, so the batched step is timed back to back for a
    pure-HBM number."""
    calibrate(V, torch, stream, 64, n=1024, spp=4000, steps=1024)  # ~21 candidate shapes of 32 steps
    b = build_batch(V, 64, 1024, 4000, 1e-2, stream)
    b.run(max(warmup, 2 * GRAPH_STEPS))
    torch.cuda.synchronize()
    head_start(torch, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    b.close()
    cells = 64 * 1024 * 1024
    return {"value": cells * steps / dt, "unit": "cell-updates/s", "ms_per_step": 1e3 * dt / steps,
            "roofline_frac": 8.0 * cells / (dt / steps) / 1e9 / measured_peaks()[0],
            "workload": "64 x N=1024 scan, 4000 steps/period, state larger than L2"}


def c5_single(V, torch, stream, warmup, steps=512):
    """Large-grid single simulation: N=1024, 4000 steps/period, Pi=1, S=3."""
    sim = V.Simulation(V.Params(n=1024, steps_per_period=4000, beta=1e-2), None, stream)
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 1.0, 3.0)
    solo_warmup(sim, warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    head_start(torch, stream)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    sim.close()
    return {"value": 1024 * 1024 * steps / dt, "unit": "cell-updates/s", "ms_per_step": 1e3 * dt / steps,
            "roofline_frac": 8.0 * 1024 * 1024 / (dt / steps) / 1e9 / measured_peaks()[0]}


def m6_rotation(V, torch, stream, warmup, steps=1024):
    """The paper's rotation benchmark set-up (Fig. sm-performance): one N=512
    grid, 1000 steps (1024 timed here: whole 32-step graphs), no wake and no damping, for the standard and the
    Manhattan rotation (the kick and Fokker-Planck passes still run, with
    identity weights, inside the same fused kernel)."""
    out = {}
    for name, rot in (("standard", 0), ("manhattan", 1)):
        sim = V.Simulation(V.Params(n=512, steps_per_period=1000, beta=0.0, rotation=rot), None, stream)
        solo_warmup(sim, warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        head_start(torch, stream)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        sim.close()
        out[name] = {"value": 512 * 512 * steps / dt, "unit": "cell-updates/s", "ms_per_step": 1e3 * dt / steps}
    out["workload"] = "single simulation N=512, 1024 timed steps after a graph warm-up, no wake, beta=0"
    return out


def cpu_baseline(n, spp, beta, budget_s=12.0):
    """FP64 oracle on the host cores: one N=n instance of the scan for as many
    steps as fit in budget_s (after one untimed step)."""
    from oracle import oracle as O
    from paper_1611_05293_b300 import workloads as W
    O.build()
    S, Pi = scan_points(1)[0]
    pr = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S)
    zr, zi = O.impedance(pr, 2, Pi)
    psi = O.normalize(pr, W.noisy_gaussian(n, 1612, 1e-6))
    psi, _, _ = O.run(pr, zr, zi, psi, 1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        psi, _, _ = O.run(pr, zr, zi, psi, 8)
        steps += 8
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n * n * steps / dt, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"1 instance N={n} (S={S:.3f}, Pi={Pi:g}), {steps} steps, {dt:.1f} s",
            "cpu_model": cpu_model(), "single_thread": cpu_single_thread(n, spp, beta)}


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_single_thread(n, spp, beta, budget_s=4.0):
    """The same oracle sample on one thread (a subprocess with OMP_NUM_THREADS=1)."""
    import subprocess
    code = (f"import sys, time; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(bench.cpu_baseline_value({n}, {spp}, {beta}, {budget_s}))")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        return {"value": float(out.stdout.strip().splitlines()[-1]), "unit": "cell-updates/s", "cores": 1}
    except Exception as e:  # the single-thread figure is context only
        return {"value": None, "error": str(e)[:200]}


def cpu_baseline_value(n, spp, beta, budget_s):
    from oracle import oracle as O
    from paper_1611_05293_b300 import workloads as W
    S, Pi = scan_points(1)[0]
    pr = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S)
    zr, zi = O.impedance(pr, 2, Pi)
    psi = O.normalize(pr, W.noisy_gaussian(n, 1612, 1e-6))
    psi, _, _ = O.run(pr, zr, zi, psi, 1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        psi, _, _ = O.run(pr, zr, zi, psi, 2)
        steps += 2
    return n * n * steps / (time.perf_counter() - t0)


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the benchmark's workload shape."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    n, spp, beta = args.n, 1000, 1e-2
    from oracle import oracle as O
    from paper_1611_05293_b300 import workloads as W
    O.build()
    sims = []
    for S, Pi in scan_points(2):
        pr = O.Params(n=n, steps_per_period=spp, beta=beta, s_csr=S)
        zr, zi = O.impedance(pr, 2, Pi)
        sims.append([pr, zr, zi, O.normalize(pr, W.noisy_gaussian(n, 1612, 1e-6))])
    # bounded sample per timed step, long enough that the oracle's per-call
    # set-up does not dominate (about 40 ms per timed step on 16 cores)
    per_step = 32 if args.steps > 20 else 64
    for _ in range(args.warmup):
        for s in sims:
            s[3], _, _ = O.run(s[0], s[1], s[2], s[3], 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in sims:
            s[3], _, _ = O.run(s[0], s[1], s[2], s[3], per_step)
    dt = time.perf_counter() - t0
    value = n * n * per_step * len(sims) * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{len(sims)} instances of N={n}, {per_step} steps each per timed step"
    print(json.dumps({
        "impl": "reference", "metric": "phase-space cell-updates/s", "value": value,
        "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batched N={n} parallel-plates scan (oracle sample: {sample})",
                   "grid": n, "steps_per_period": spp},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def measure_e2e(V, torch, args, n, spp, beta, stream):
    """The scan end to end through the C ABI with host buffers, wall clock:
    vfps_batch_add_many of every slot from one pinned host block of FP64
    starting states (one host-to-device copy; normalisation and FP32
    conversion on the device), the run, and vfps_batch_take_many of every
    final state (gathered and converted on the device, one device-to-host
    copy into a pinned host block) with its CSR-power series.  Run before the
    clock sampler is first used: after an nvidia-smi process ends, the driver
    calls of the next ~0.2 s run two to three times slower (measured)."""
    from paper_1611_05293_b300 import workloads as W
    count = args.instances
    pts = scan_points(count)
    host_in = torch.empty((count, n, n), dtype=torch.float64, pin_memory=True).numpy()
    host_in[:] = W.noisy_gaussian(n, 1612, 1e-6)
    host_out = torch.empty((count, n, n), dtype=torch.float64, pin_memory=True).numpy()
    Pi = np.array([p[1] for p in pts])
    S = np.array([p[0] for p in pts])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bb = V.Batch(count, 0, stream)
    if PIN_SHAPE:
        bb.pin_shape(*PIN_SHAPE)
    slots = bb.add_many(V.Params(n=n, steps_per_period=spp, beta=beta), host_in, V.IMPEDANCE_PARALLEL_PLATES,
                        Pi, S, nsteps=1 << 40)
    t_add = time.perf_counter()
    bb.run(args.steps)
    bb.poll()  # waits for the run
    t_run = time.perf_counter()
    power = bb.take_many(slots, psi_out=host_out, power_cap=args.steps)
    t_take = time.perf_counter()
    bb.close()
    e2e_dt = t_take - t0
    h2d = host_in.nbytes / args.steps
    d2h = (host_out.nbytes + sum(p_.nbytes for p_ in power)) / args.steps
    return {"value": count * n * n * args.steps / e2e_dt, "unit": "cell-updates/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "what": "vfps_batch_add_many from one pinned host block of fp64 states + run + vfps_batch_take_many "
                    "of every state (into one pinned block) and P(t), wall clock",
            "split_ms": {"add": 1e3 * (t_add - t0), "run": 1e3 * (t_run - t_add), "take": 1e3 * (t_take - t_run)}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the serving / C3 / C5 side measurements")
    ap.add_argument("--shape", default="", help="W,tps: fixed batch launch shape (profiling runs)")
    ap.add_argument("--pairing", action="store_true", help="pair kernel for simulations of one geometry")
    ap.add_argument("--rotation", type=int, default=0, choices=[0, 1],
                    help="1: the Manhattan rotation for the batched scan (profiling runs)")
    args = ap.parse_args()
    global PIN_SHAPE, PAIRING
    PAIRING = args.pairing
    if args.shape:
        PIN_SHAPE = tuple(int(v) for v in args.shape.split(","))
    if args.impl == "reference":
        run_reference(args)
        return
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1611_05293_b300 import vfps as V

    n, spp, beta = args.n, 1000, 1e-2
    stream = torch.cuda.Stream()
    hbm, peak_kind = measured_peaks()

    # ---- batched scan (the headline)
    if not PIN_SHAPE:
        calibrate(V, torch, stream, args.instances, n, spp, beta, rotation=args.rotation)
    e2e = measure_e2e(V, torch, args, n, spp, beta, stream) if rank == 0 else None
    b = build_batch(V, args.instances, n, spp, beta, stream, rotation=args.rotation, rank=rank, world=world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        b.run(args.warmup)
        launches = b.launches_per_step()
        shapes = b.shapes()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        head_start(torch, stream)
        t0 = time.perf_counter()
        e0.record(stream)
        b.run(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    dt = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist if world > 1 else None, "cuda")
    if world > 1:
        dist.barrier()
    cells_step = args.instances * n * n
    value = world * cells_step * args.steps / dt
    # every launch of a step runs concurrently with the others of that step (one
    # stream each): the algorithmic bytes of all of them over the step time
    achieved = 8.0 * cells_step / (dt / args.steps) / 1e9  # GB/s
    b.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- plain single-simulation path (N=256, FP32, Pi=2, S=0.9)
    sim = V.Simulation(V.Params(n=n, steps_per_period=spp, beta=1.25e-2), None, stream)
    sim.set_impedance(V.IMPEDANCE_PARALLEL_PLATES, 2.0, 0.9)
    solo_warmup(sim, args.warmup)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_steps = -(-max(args.steps, 256) // GRAPH_STEPS) * GRAPH_STEPS  # whole graphs
    head_start(torch, stream)
    p0.record(stream)
    sim.step(plain_steps)
    p1.record(stream)
    torch.cuda.synchronize()
    pdt = p0.elapsed_time(p1) / 1e3
    sim.close()
    plain = {"value": n * n * plain_steps / pdt, "unit": "cell-updates/s",
             "ms_per_step": 1e3 * pdt / plain_steps, "workload": "single simulation N=256 FP32, Pi=2, S=0.9"}

    tpl, tshape = measured_traffic_per_launch()
    shape_now = ",".join(f"{g['W']}x{g['tps']}" for g in shapes)
    traffic, traffic_src = None, "no ncu capture of the kernel sources built now"
    if tpl and args.instances == 512 and n == 256 and not args.rotation and not PAIRING and tshape == shape_now:
        traffic, traffic_src = tpl * launches, "ncu capture of this kernel build and launch shape"
    line = {
        "metric": "phase-space cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched N={n} parallel-plates scan, {args.instances} instances per GPU "
                               f"(S in [0.2,1.5] x Pi in {{1,2,3}}), {spp} steps/period, FP32 psi + FP64 sums"
                               + (", Manhattan rotation" if args.rotation else ""),
                   "instances": args.instances, "grid": n, "steps_per_period": spp, "beta": beta,
                   "l2": f"inputs larger than L2: state {2 * cells_step * 4 / 2**20:.0f} MiB > 126 MiB",
                   "parallelism": f"replicas x{world}"},
        "plain": plain,
        "batched_vs_plain": value / world / plain["value"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": traffic,
                     "traffic_unit": "DRAM bytes per step (all launches of the step, ncu)",
                     "traffic_source": traffic_src,
                     "algorithmic_bytes_per_step": 8 * cells_step,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_cell": 8,
                     "frac_vs_nominal_8tbs": achieved / 8000.0},
        "gpu_launches": args.steps * launches,
        "launches_per_step": launches,
        "launch_shapes": shapes,
        "clocks": clk.summary(),
        "e2e": e2e,
        "wall_s_timed": wall,
    }
    if not args.no_extra:
        line["c3_scan_64"] = c3_scan_64(V, torch, stream, args.warmup)
        line["c5_n1024"] = c5_single(V, torch, stream, args.warmup)
        line["c3_n1024_64"] = c3_n1024_64(V, torch, stream, args.warmup)
        line["manhattan_scan"] = manhattan_scan(V, torch, stream, args.warmup)
        line["m6_rotation_n512"] = m6_rotation(V, torch, stream, args.warmup)
        line["moments_cost"] = moments_cost(V, torch, stream, args.warmup)
        line["spectrogram"] = spectrogram_cost(V, torch, stream)
        line["serving"] = serving(V, torch, stream)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(n, spp, beta)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
