#!/usr/bin/env python3
"""Benchmark of the multi-spin-coded checkerboard Metropolis sweep on GB300.

Workload: the largest single-GPU lattice, L = 524288 (2^38 spins, 64 spins per
64-bit word, 32 GiB), cold start, T = 2.0, seed 5, M and E recorded after every
sweep.  A step is 10 sweeps (the 200-sweep run is 20 steps).  Metric: spin-flip
attempts per ns (N = L^2 attempts per sweep).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--parallelism replicas|strips]

--gpus N with N > 1 starts N ranks itself (torch.distributed.run on this node)
unless it already runs under a launcher that set WORLD_SIZE, which must then
equal N.  Ranks:
  replicas  every rank sweeps its own L = 524288 lattice (stream_id = rank); the
            units of all ranks over the slowest rank's time (weak scaling);
  strips    one L = 524288 lattice in row strips, one per rank, with a halo
            row exchanged with each ring neighbour before every checkerboard
            step and an int64 all-reduce of the counts at every recorded sweep
            (the paper's border exchange, Sec. 6.1; strong scaling).

One JSON line on rank 0:
  value          device-timed attempts/ns, lattice resident in HBM
  e2e            the same through the C ABI from pinned host memory: each step
                 creates the lattice from the host copy (H2D), sweeps, reads
                 the M/E samples back (D2H) and destroys it
  roofline       the dominant kernel (the half-sweep) against the integer-ALU
                 bound (16 int32 ops per attempt at 128 lanes per SM per clock),
                 with the measured draw-generation rates beside it
  cpu_baseline   the oracle on this host's cores (all, and one) on a bounded
                 light-cone sample of the same lattice (rank 0, N = 1 only)
  extras         the L = 32768 lattice, small lattices, the 128-lattice batch,
                 the served request stream, the field, the paper's shape
The reference arm (--impl reference) times the oracle itself on that sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import socket
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L = 524288
T = 2.0
SEED = 5
WORD_BITS = 64
SWEEPS_PER_STEP = 10
METRIC = "spin-flip attempts/ns"
UNIT = "attempts/ns"
# canonical integer operations per attempt (Philox 10, counter 0.5, compares and
# bit insertion 4, bit-sliced logic / mask / XOR 1, popcount reductions 0.5)
OPS_PER_ATTEMPT = 16
INT32_LANES_PER_SM = 128
CONFIG = {
    "workload": "L=524288 (2^38 spins, u64 words, 32 GiB), cold start, T=2.0, seed 5, "
                "10 sweeps per step (the 200-sweep run in 20 steps), M/E every sweep",
    "L": L, "T": T, "seed": SEED, "sweeps_per_step": SWEEPS_PER_STEP, "word_bits": WORD_BITS,
    "record_every": 1,
    "l2": "no flush: the lattice (32 GiB) is far larger than L2 (129 MB) and is read and "
          "written twice per sweep",
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------- distributed --
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def spawn_ranks(n: int) -> int:
    """Re-runs this command as n ranks under torch.distributed.run on this node."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(n),
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.abspath(__file__)]
    cmd += sys.argv[1:]
    return subprocess.call(cmd)


# ------------------------------------------------------------------ clocks --
def gpu_local_cpus(gpu_index: int):
    """The CPUs next to a GPU (sysfs local_cpulist of its PCI device), or None."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip()
        dom, rest = bus.split(":", 1)
        path = "/sys/bus/pci/devices/%04x:%s/local_cpulist" % (int(dom, 16) & 0xFFFF, rest.lower())
        with open(path) as f:
            text = f.read().strip()
        cpus = set()
        for part in text.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        cpus &= os.sched_getaffinity(0)
        return cpus or None
    except Exception:
        return None


def compact_cpus(cpus) -> str:
    out, run = [], []
    for c in sorted(cpus):
        if run and c == run[-1] + 1:
            run.append(c)
        else:
            if run:
                out.append("%d-%d" % (run[0], run[-1]) if len(run) > 1 else str(run[0]))
            run = [c]
    if run:
        out.append("%d-%d" % (run[0], run[-1]) if len(run) > 1 else str(run[0]))
    return ",".join(out)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: the upper part of the distribution
        loaded = [s for s in sm if s >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- profiles --
KERNEL_SOURCES = ("kernels.cu", "sweep_device.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "half_sweep_traffic.json")


def kernel_source_hash() -> str:
    """sha256[:16] of the half-sweep kernel's sources, concatenated in order."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1007_3726_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_kernel():
    """The committed ncu figures of the half-sweep (DRAM bytes per launch at the
    captured size, thread instructions per attempt), if they were taken on the
    current kernel source; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_sources_sha16") != kernel_source_hash():
        return None
    return d


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------- CPU oracle ---
def oracle_window_sample(target_s: float, rows: int = 256, max_sweeps: int | None = None):
    """Time the oracle on a light-cone window of the workload lattice: rows
    [0, rows) of the L = 524288 cold start, sweeps until about target_s
    seconds.  Each sweep counts (rows - 2) x L attempts (the window's edge rows
    are its fixed boundary).  Returns (attempts, seconds, sweeps, threads)."""
    import numpy as np

    import oracle

    oracle.build()
    thr4, thr8 = oracle.thresholds(T)
    s = np.ones((rows, L), dtype=np.int8)
    attempts = 0
    sweeps = 0
    t0 = time.perf_counter()
    while True:
        oracle.run_window(s, L, 0, 1, SEED, 0, thr4, thr8, t0=sweeps)
        sweeps += 1
        attempts += (rows - 2) * L
        el = time.perf_counter() - t0
        if el >= target_s or (max_sweeps and sweeps >= max_sweeps):
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return attempts, el, sweeps, threads


def oracle_one_core(target_s: float, rows: int = 64):
    """The same sample on one host thread, in a child process (OMP_NUM_THREADS=1)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = ("import json, bench; a, el, sw, thr = bench.oracle_window_sample(%r, rows=%d); "
            "print(json.dumps([a, el, sw, thr]))" % (target_s, rows))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_configs(one_thread: bool = False) -> dict:
    """The oracle on the other workloads (bounded samples, each a few seconds
    at most): the L = 64 case in full (1000 sweeps, one thread), the L = 32768
    case (two whole-lattice sweeps on all cores; a 10-sweep light-cone window of
    256 rows on one thread) and one lattice per size of the 128-lattice batch
    (200 sweeps each, all cores).  With one_thread, only the one-thread parts."""
    import numpy as np

    import oracle
    from paper_1007_3726_gb300 import workloads as WL

    oracle.build()
    out = {}
    if one_thread:
        thr4, thr8 = oracle.thresholds(2.269185)
        s = oracle.init_cold(64)
        t = time.perf_counter()
        oracle.run(s, 1000, 1, 0, thr4, thr8, check=False)
        el = time.perf_counter() - t
        out["L64_1000_sweeps_1_thread"] = {"value": 64 * 64 * 1000 / el / 1e9, "seconds": el}
        w = WL.large_L32768()
        thr4, thr8 = oracle.thresholds(w["T"])
        s = oracle.init_hot(w["L"], w["seed"], w["stream_id"], 0, 256)
        t = time.perf_counter()
        oracle.run_window(s, w["L"], 0, 10, w["seed"], w["stream_id"], thr4, thr8)
        el = time.perf_counter() - t
        out["L32768_window_1_thread"] = {"value": 254 * w["L"] * 10 / el / 1e9, "seconds": el,
                                         "sample": "rows 0-255, 10 sweeps (light-cone mode)"}
        return out
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    w = WL.large_L32768()
    thr4, thr8 = oracle.thresholds(w["T"])
    s = oracle.init_hot(w["L"], w["seed"], w["stream_id"])
    t = time.perf_counter()
    oracle.run(s, 2, w["seed"], w["stream_id"], thr4, thr8, check=False)
    el = time.perf_counter() - t
    out["L32768_2_sweeps"] = {"value": w["L"] ** 2 * 2 / el / 1e9, "seconds": el, "cores": threads}
    del s
    attempts, el = 0, 0.0
    for sp in WL.fss_batch()[::32]:  # the first temperature of each size
        thr4, thr8 = oracle.thresholds(sp["T"])
        s = oracle.init_hot(sp["L"], sp["seed"], sp["stream_id"])
        t = time.perf_counter()
        oracle.run(s, 200, sp["seed"], sp["stream_id"], thr4, thr8, check=False)
        el += time.perf_counter() - t
        attempts += sp["L"] ** 2 * 200
    out["fss_one_lattice_per_L_200_sweeps"] = {"value": attempts / el / 1e9, "seconds": el, "cores": threads}
    return out


def oracle_configs_one_thread() -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = "import json, bench; print(json.dumps(bench.oracle_configs(one_thread=True)))"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def msc_sample(target_s: float):
    """The paper's CPU multi-spin-coding program (Sec. 4, a Boltzmann-pattern pool
    of 2^22 entries) on its Table 1 shape, L = 4096 at T = 0.99 T_c, hot start:
    sweeps until about target_s seconds.  Returns (attempts, seconds, sweeps,
    threads)."""
    from oracle import msc

    import oracle

    L4 = 4096
    pool = msc.Pool(0.99 * 2.269185, 1 << 22, seed=1)
    lat = msc.pack(oracle.init_hot(L4, 11, 0))
    msc.sweeps(lat, pool, 1, seed=1, record=False)
    n, t0 = 0, time.perf_counter()
    while True:
        msc.sweeps(lat, pool, 1, seed=1, t0=1 + n, record=False)
        n += 1
        el = time.perf_counter() - t0
        if el >= target_s:
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return L4 * L4 * n, el, n, threads


def msc_one_core(target_s: float):
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = "import json, bench; print(json.dumps(bench.msc_sample(%r)))" % target_s
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(target_s=10.0):
    a, el, sw, thr = oracle_window_sample(target_s)
    a1, el1, sw1, thr1 = oracle_one_core(target_s)
    m, elm, swm, thrm = msc_sample(5.0)
    m1, elm1, swm1, thrm1 = msc_one_core(5.0)
    msc = {"kind": "the paper's CPU multi-spin coding (Sec. 4), Boltzmann-pattern pool of 2^22, one address "
                   "per 32-spin word; not bit-exact (another random-number scheme), pinned statistically",
           "workload": "L=4096, T=0.99 T_c, hot start (the paper's Table 1 shape)", "unit": UNIT,
           "all_cores": {"value": m / elm / 1e9, "cores": thrm, "sweeps": swm, "seconds": elm},
           "one_core": {"value": m1 / elm1 / 1e9, "cores": thrm1, "sweeps": swm1, "seconds": elm1},
           "paper_one_core": {"value": 0.2267, "hardware": "Intel Xeon X5560 2.80 GHz, 1 core (Table 1)"}}
    per_config = dict(oracle_configs(), **oracle_configs_one_thread())
    return {"value": a / el / 1e9, "unit": UNIT, "cores": thr, "kind": "oracle", "paper_cpu_msc": msc,
            "per_config": dict(per_config, unit=UNIT),
            "sample": "oracle (one int8 per spin, plain C, OpenMP over rows) on rows 0-255 of the "
                      "L=524288 cold start, %d sweeps in light-cone mode, %.1f s wall, %d threads"
                      % (sw, el, thr),
            "one_core": {"value": a1 / el1 / 1e9, "unit": UNIT, "cores": thr1,
                         "sample": "rows 0-63 of the same lattice, %d sweeps, %.1f s wall, 1 thread"
                                   % (sw1, el1)}}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_window_sample(0.0, max_sweeps=1)
    total_a, total_t, sweeps, threads = 0, 0.0, 0, 1
    for _ in range(args.steps):
        a, el, sw, threads = oracle_window_sample(2.0)
        total_a += a
        total_t += el
        sweeps += sw
    v = total_a / total_t / 1e9
    line = {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_t * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i8",
        "data": "synthetic", "config": CONFIG, "impl": "reference",
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "each step: oracle on rows 0-255 of the L=524288 cold start "
                                   "for about 2 s (%d sweeps in total)" % sweeps},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- ours --
def timed_sweeps(P, lat, stream, sweeps, record_every=1, reps=1):
    """Device time (CUDA events on the lattice's stream) of `sweeps` sweeps."""
    import torch

    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.sweep(sweeps, record_every)
        e1.record(stream)
        lat.measure()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best / 1e3


def mix_peaks(P, stream):
    """The integer-mix microbenchmark (ising_bench_mix), draws per ns."""
    out = {}
    for form, name in ((0, "full_philox_rounds"), (1, "kernel_philox_form"), (2, "kernel_form_with_masks")):
        P.ising_bench_mix(form, 2000, stream=stream)
        best = 0.0
        for _ in range(2):
            _, r = P.ising_bench_mix(form, 40000, stream=stream)
            best = max(best, r)
        out[name] = best
    return out


def served_extras(P):
    """The served stream, shortened: an overload stream (200 requests/s for 10 s,
    then up to 40 s to drain) and a stream at 60 % of the capacity the overload
    run measured; and the first 120 requests of the stream served together
    against the same requests run one after another with plain launches."""
    from paper_1007_3726_gb300 import serve

    out = {}
    reqs = serve.poisson_requests(rate=200.0, duration=10.0, seed=4)
    with P.Server(hbm_budget_bytes=64 * 10 ** 9, epoch_sweeps=1000) as srv:
        over = serve.run_stream(srv, reqs, drain_s=40.0)
    out["overload_200_per_s_10s"] = over
    mean_work = sum(r["L"] ** 2 * r["nsweeps"] for r in reqs) / len(reqs)
    cap = over["server_attempts_per_ns"] * 1e9  # attempts per second
    rate = 0.6 * cap / mean_work
    reqs60 = serve.poisson_requests(rate=rate, duration=20.0, seed=4)
    with P.Server(hbm_budget_bytes=64 * 10 ** 9, epoch_sweeps=1000) as srv:
        r60 = serve.run_stream(srv, reqs60, drain_s=40.0)
    r60["offered_rate_per_s"] = rate
    r60["offered_attempts_per_ns"] = rate * mean_work / 1e9
    out["at_60pct_of_capacity"] = r60
    # the same requests served together vs sequential plain launches
    same = [dict(r, t=0.0) for r in reqs[:120]]
    work = sum(r["L"] ** 2 * r["nsweeps"] for r in same)
    with P.Server(hbm_budget_bytes=64 * 10 ** 9, epoch_sweeps=1000) as srv:
        t = time.perf_counter()
        s = serve.run_stream(srv, same, drain_s=600.0)
        t_served = time.perf_counter() - t
    t = time.perf_counter()
    for r in same:
        with P.Lattice(r["L"], r["T"], seed=r["seed"], init="hot") as lat:
            lat.sweep(r["nsweeps"], r["record_every"])
            lat.measure()
    t_seq = time.perf_counter() - t
    out["same_120_requests"] = {
        "served_attempts_per_ns": work / t_served / 1e9, "sequential_plain_attempts_per_ns": work / t_seq / 1e9,
        "served_over_sequential": t_seq / t_served, "completed": s["completed"],
        "note": "all 120 submitted at once; sequential: one Lattice per request, ising_sweep's default "
                "launch, in submission order"}
    return out


def extras(P, stream, peaks, mix):
    """Other workloads, on rank 0 at N = 1."""
    import torch

    from paper_1007_3726_gb300 import workloads as WL

    out = {}
    # the L = 32768 lattice (hot start, T = T_c): 1000 sweeps, device-timed
    w = WL.large_L32768()
    lat = P.Lattice(**WL.lattice_kwargs(w), stream=stream)
    cfg, _ = lat.autotune(reps=3)
    timed_sweeps(P, lat, stream, 20)
    t = timed_sweeps(P, lat, stream, w["sweeps"], reps=2)
    rate = w["L"] ** 2 * w["sweeps"] / t / 1e9
    mean_launch = t / (2 * w["sweeps"])
    out["L32768_1000_sweeps"] = {
        "attempts_per_ns": rate, "launch": cfg, "mean_launch_us": mean_launch * 1e6,
        "frac_nominal_int32": OPS_PER_ATTEMPT * rate * 1e9 / (peaks["int32_tops"] * 1e12),
        "frac_of_measured_draw_rate": rate / mix["kernel_philox_form"],
        "frac_of_measured_draws_with_masks": rate / mix["kernel_form_with_masks"],
        "note": "the previous headline workload: 2^30 spins, u32 storage, hot start seed 7, T=2.269185, "
                "M/E every sweep; best of 2 device-timed 1000-sweep runs"}
    lat.close()

    def wall_call(lat, sweeps):
        lat.sweep(20, 1)
        lat.measure()
        t = time.perf_counter()
        lat.sweep(sweeps, 1)
        lat.measure()
        return time.perf_counter() - t

    # small lattices: one CTA (L = 64) and an 8-CTA cluster (L = 256)
    for Ls in (64, 128, 256, 512):
        name = "L%d_1000_sweeps" % Ls
        a = P.Lattice(Ls, 2.269185, seed=1, init="cold_up")
        ta = min(wall_call(a, 1000) for _ in range(3))
        n = Ls * Ls * 1000
        d = {"attempts_per_ns": n / ta / 1e9, "launch": a.launch,
             "note": "wall time of one ising_sweep call (launch, 1000 sweeps, read-back of 1000 M/E samples), "
                     "best of 3"}
        s = P.Lattice(Ls, 2.269185, seed=1, init="cold_up")
        s.set_launch(proc_bits=32, regcap=0, insert=0, block=128, rows_per_item=4, grid=0)
        d["step_launches_attempts_per_ns"] = n / wall_call(s, 1000) / 1e9
        ctas = max(1, a.launch["grid"])
        d["issue_bound_attempts_per_ns"] = ctas * INT32_LANES_PER_SM * peaks["sm_max_ghz"] / OPS_PER_ATTEMPT
        # the SMs that draw the acceptance masks (the warp-specialised form
        # draws in all CTAs but the first) at the measured per-SM draw rate
        drawing = ctas - 1 if a.launch["block"] == 1024 and ctas > 1 else ctas
        d["draw_bound_attempts_per_ns"] = drawing * mix["kernel_form_with_masks"] / torch.cuda.get_device_properties(
            torch.cuda.current_device()).multi_processor_count
        d["frac_of_draw_bound"] = d["attempts_per_ns"] / d["draw_bound_attempts_per_ns"]
        out[name] = d
        a.close()
        s.close()

    # the 128-lattice finite-size-scaling batch: one tuned persistent launch
    specs = WL.fss_batch()
    lats = [P.Lattice(**WL.lattice_kwargs(sp)) for sp in specs]
    sweeps = [sp["sweeps"] for sp in specs]
    N = sum(sp["L"] ** 2 for sp in specs)
    opts, _ = P.ising_batch_tune(lats, sweeps, 20)
    torch.cuda.synchronize()
    with P.Batch(lats, sweeps, specs[0]["record_every"], **opts) as b:
        info = b.info()
        t = time.perf_counter()
        b.run(1)
        t_b = time.perf_counter() - t
    t = time.perf_counter()
    for lat in lats:
        lat.sweep(200, 10)
    for lat in lats:
        lat.measure()
    t_p = time.perf_counter() - t
    out["fss_batch_128_lattices"] = {
        "persistent_attempts_per_ns": N * sweeps[0] / t_b / 1e9,
        "sequential_plain_attempts_per_ns": N * 200 / t_p / 1e9,
        "seconds": t_b, "plan": info, "options": opts,
        "note": "10^4 sweeps of 128 lattices in one launch (wall time incl. sample read-back); "
                "plain: each lattice's default launch, 200 sweeps each, one after another"}
    for lat in lats:
        lat.close()

    # the L = 32768 lattice in a field H = 0.1 (ten acceptance classes)
    f = P.Lattice(32768, 2.269185, seed=7, init="hot", H=0.1)
    t_f = wall_call(f, 200)
    out["field_L32768_H0.1"] = {"attempts_per_ns": 32768 ** 2 * 200 / t_f / 1e9,
                                "note": "200 sweeps, M/E every sweep, wall time of one call"}
    f.close()

    # the shape of the paper's single-GPU comparison (Table 1): L = 4096 at T = 0.99 T_c
    w = WL.paper_benchmark()
    q = P.Lattice(**WL.lattice_kwargs(w))
    q.autotune(reps=2)
    t_q = wall_call(q, w["sweeps"])
    out["paper_shape_L4096_0.99Tc"] = {
        "attempts_per_ns": 4096 ** 2 * w["sweeps"] / t_q / 1e9, "launch": q.launch,
        "note": "1000 sweeps, M/E every sweep, wall time of one call; the paper's best single-GPU "
                "figure on this shape is 7.98 attempts/ns (Tesla C1060, another RNG): context only"}
    q.close()

    out["served"] = served_extras(P)
    return out


class StripsRun:
    """The workload lattice as row strips over the ranks (NCCL halo exchange)."""

    def __init__(self, P, ws, rank, stream):
        from paper_1007_3726_gb300.distributed import StripLattice, TorchDistExchange

        self.strip = StripLattice(L, T, seed=SEED, init="cold_up", rank=rank, world=ws, word_bits=WORD_BITS)
        self.ex = TorchDistExchange()

    def sweep(self, n, record_every):
        from paper_1007_3726_gb300.distributed import sweep_strips

        return sweep_strips([self.strip], self.ex, L, n, record_every)

    def close(self):
        self.strip = None


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1007_3726_gb300 as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    P.load()
    stream = torch.cuda.Stream(device=dev)
    N = L * L
    strips = args.parallelism == "strips" and ws > 1
    units_per_step = N * SWEEPS_PER_STEP * (1 if strips else ws)

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if ws == 1:
            return x
        import torch.distributed as dist

        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---------------- device-resident timing
    tuned, tuned_us = None, None
    if strips:
        with torch.cuda.stream(stream):
            lat = StripsRun(P, ws, rank, stream)
    else:
        lat = P.Lattice(L, T, seed=SEED, stream_id=rank, init="cold_up", word_bits=WORD_BITS, stream=stream)
        tuned, tuned_us = lat.autotune(reps=2)   # launch shape only: results are identical
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            lat.sweep(SWEEPS_PER_STEP, 1)
            if not strips:
                lat.measure()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            ev[i][0].record(stream)
            lat.sweep(SWEEPS_PER_STEP, 1)   # 2 half-sweep launches per sweep
            ev[i][1].record(stream)
        if not strips:
            lat.measure()                   # harvests the samples, FP64 moments on the host
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = max_over_ranks(sum(step_ms) / 1e3)
    value = units_per_step * args.steps / t_dev / 1e9
    obs = None if strips else lat.measure()
    lat.close()
    launches = 2 * SWEEPS_PER_STEP * args.steps
    mean_launch_s = sum(step_ms) / 1e3 / launches

    # ---------------- end to end through the C ABI from pinned host memory
    nbytes = N // 8
    e2e_value, h2d, d2h = None, 0, 0
    local_cpus_used, raw_h2d_gbs = None, None
    if not strips:
        # the pinned buffer on the CPU socket next to this GPU (its pages are
        # placed where they are first touched): bind to the GPU's local CPUs
        # while allocating and filling it, then restore the affinity
        local_cpus_used = gpu_local_cpus(local)
        saved = os.sched_getaffinity(0)
        if local_cpus_used:
            os.sched_setaffinity(0, local_cpus_used)
        try:
            host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
            host.fill_(0xFF)                              # the cold start, packed
        finally:
            os.sched_setaffinity(0, saved)
        hp = host.numpy().view(np.uint64).reshape(L, L // 64)
        Mh = np.zeros(SWEEPS_PER_STEP, dtype=np.int64)
        Eh = np.zeros(SWEEPS_PER_STEP, dtype=np.int64)

        phases = []
        # two lattices in flight: step k + 1's lattice is created (its upload on
        # its own stream, from a second host thread) while step k sweeps, as a
        # pipeline of jobs would run; every upload, every sweep and every sample
        # read-back is inside the timed region
        streams = [stream, torch.cuda.Stream(device=dev)]

        def create(k):
            torch.cuda.set_device(dev)  # the library creates on the calling thread's device
            t0 = time.perf_counter()
            lt = P.Lattice(L, T, seed=SEED, stream_id=rank, packed=hp, word_bits=WORD_BITS,
                           stream=streams[k % 2])
            return lt, time.perf_counter() - t0

        def e2e_run(nsteps):
            from concurrent.futures import ThreadPoolExecutor

            with ThreadPoolExecutor(max_workers=1) as pool:
                fut = pool.submit(create, 0)
                for k in range(nsteps):
                    lt, t_create = fut.result()
                    if k + 1 < nsteps:
                        fut = pool.submit(create, k + 1)
                    t1 = time.perf_counter()
                    P.ising_sweep(lt.handle, SWEEPS_PER_STEP, 1, Mh, Eh, SWEEPS_PER_STEP)
                    t2 = time.perf_counter()
                    lt.close()
                    phases.append((t_create, t2 - t1, time.perf_counter() - t2))

        # the library's device memory from PyTorch's caching allocator, as a
        # caller that runs job after job would set it up: the two 32 GiB
        # lattices are allocated once, not cudaMalloc'd and freed in every step
        # the bare copy from this buffer (torch, outside the timed region): the
        # reference for the upload phase below
        dev_probe = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        tc = time.perf_counter()
        dev_probe.copy_(host, non_blocking=True)
        torch.cuda.synchronize()
        raw_h2d_gbs = nbytes / (time.perf_counter() - tc) / 1e9
        del dev_probe
        torch.cuda.empty_cache()
        P.use_torch_allocator()
        e2e_clocks = ClockSampler(local)
        try:
            e2e_run(2)
            barrier()
            e2e_clocks.start()
            del phases[:]
            t0 = time.perf_counter()
            e2e_run(args.steps)
            torch.cuda.synchronize()
            t_e2e = max_over_ranks(time.perf_counter() - t0)
            e2e_clk = e2e_clocks.stop()
        finally:
            P.ising_set_allocator(None)
            torch.cuda.empty_cache()
        e2e_phases = {k: round(float(np.median([ph[j] for ph in phases])), 4)
                      for j, k in enumerate(("create_upload_s", "sweeps_s", "close_s"))}
        e2e_value = units_per_step * args.steps / t_e2e / 1e9
        h2d, d2h = nbytes, int(Mh.nbytes + Eh.nbytes)
        del host

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max_ghz = (peaks.get("sm_max_mhz") or 2070.0) / 1e3
    peak_tops = sms * INT32_LANES_PER_SM * sm_max_ghz * 1e9 / 1e12
    per_rank_attempts = N / 2 / (ws if strips else 1)
    achieved_tops = OPS_PER_ATTEMPT * per_rank_attempts / mean_launch_s / 1e12
    rate_per_gpu = per_rank_attempts / mean_launch_s / 1e9  # attempts/ns of one GPU's launches
    mix = mix_peaks(P, stream) if ws == 1 else None
    prof = profiled_kernel()
    traffic = None
    if prof and not strips:
        # DRAM bytes of one launch at the captured size, scaled by the sites of this one
        traffic = prof["dram_bytes_per_launch"] * (N / float(prof["L"]) ** 2)
    roof = {
        "bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s (int32)",
        "frac": achieved_tops / peak_tops, "traffic": traffic,
        "kernel": "k_half_sweep (proc_bits=%s, regcap=%s)" % (
            tuned["proc_bits"] if tuned else "default", tuned["regcap"] if tuned else "default"),
        "peak_basis": "%d SMs x %d int32 lanes x %.2f GHz (max SM clock), derived" % (
            sms, INT32_LANES_PER_SM, sm_max_ghz),
        "achieved_basis": "%d ops/attempt x %d attempts per launch / mean launch time %.1f us (CUDA events "
                          "over the timed region)" % (OPS_PER_ATTEMPT, per_rank_attempts, mean_launch_s * 1e6),
        "hbm_view": {"bytes_per_launch_algorithmic": per_rank_attempts * 2 / 8 * 2,
                     "achieved_gbs": per_rank_attempts * 2 / 8 * 2 / mean_launch_s / 1e9,
                     "peak_gbs": peaks.get("hbm_gbs"), "peak_note": "of measured"},
    }
    if traffic is not None:
        roof["traffic_basis"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch at L=%d, "
                                 "scaled by the sites per launch (%s)" % (prof["L"], prof["source"]))
        roof["ncu_thread_instructions_per_attempt"] = prof.get("thread_inst_per_attempt")
    if mix:
        roof["measured_mix"] = dict(mix, unit="draws/ns", how="ising_bench_mix: one wave of resident 512-thread "
                                    "blocks, 32 draws per thread per word, CUDA events",
                                    frac_of_kernel_philox_form=rate_per_gpu / mix["kernel_philox_form"],
                                    frac_of_kernel_form_with_masks=rate_per_gpu / mix["kernel_form_with_masks"],
                                    peak_tops_equivalent=OPS_PER_ATTEMPT * mix["kernel_philox_form"] / 1e3,
                                    frac_of_peak_tops_equivalent=achieved_tops / (
                                        OPS_PER_ATTEMPT * mix["kernel_philox_form"] / 1e3))
    config = dict(CONFIG, parallelism=("strips" if strips else "replicas") if ws > 1 else "single")
    if strips:
        config["workload"] += "; one lattice in %d row strips, NCCL halo exchange" % ws
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "strong" if strips else "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic", "config": config,
        "roofline": roof,
        "e2e": ({"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "how": "per step: ising_create from the pinned packed cold start (H2D), ising_sweep of 10 "
                        "sweeps returning the 10 M/E samples (D2H), ising_destroy; the next step's lattice is "
                        "created (uploaded on a second stream by a second host thread) while this one sweeps; "
                        "device memory from PyTorch's caching allocator (ising_set_allocator)",
                 "phases_median": e2e_phases, "clocks": e2e_clk, "raw_h2d_GBs": raw_h2d_gbs,
                 "host_buffer_cpus": "the GPU's local CPUs %s" % compact_cpus(local_cpus_used)
                 if local_cpus_used else "not bound (no local CPU list found)"}
                if e2e_value is not None else None),
        "gpu_launches": launches,
        "launch": dict(tuned, autotune_us_per_step=tuned_us) if tuned else None,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if obs is not None:
        line["observables_last_step"] = {"mean_abs_m": obs["mean_abs_m"], "mean_e": obs["mean_e"],
                                         "n_samples": obs["n_samples"]}
    if ws == 1 and not args.no_extras:
        line["extras"] = extras(P, stream, {"int32_tops": peak_tops, "sm_max_ghz": sm_max_ghz}, mix)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_fss(args):
    """Finite-size scaling: U4 crossings of L = 64, 128, 256, 512 in [2.24, 2.30]
    after 2e5 sweeps (20 % dropped), against Onsager's T_c = 2/ln(1 + sqrt 2)."""
    import math

    import numpy as np

    from paper_1007_3726_gb300 import fss

    Ls = (64, 128, 256, 512)
    if args.fss_long:
        # sweeps ~ L^2.17 (the Metropolis autocorrelation time at T_c), 2e5 at L = 64;
        # each lattice of these sizes runs on one CTA, so L = 512 (2e7 sweeps) is left out
        Ls = (64, 128, 256)
        sweeps = {L: int(round(2e5 * (L / 64) ** 2.17, -4)) for L in Ls}
        temps = np.linspace(2.255, 2.285, 16)
        record_every = 100
    else:
        sweeps = {L: args.fss_sweeps for L in Ls}
        temps = None
        record_every = 10
    t = time.perf_counter()
    res = fss.run_fss(Ls=Ls, temps=temps, sweeps=sweeps, record_every=record_every)
    el = time.perf_counter() - t
    cr = fss.crossings(res)
    tc = 2.0 / math.log(1.0 + math.sqrt(2.0))
    nT = len(next(iter(res.values()))[0])
    work = sum(L * L * nT * sweeps[L] for L in res)
    line = {"metric": "finite-size-scaling T_c from U4 crossings", "value": cr[-1]["T_cross"],
            "unit": "T", "onsager_tc": tc, "crossings": cr, "seconds": el,
            "attempts_per_ns": work / el / 1e9, "sweeps": {str(L): n for L, n in sweeps.items()},
            "U4": {str(L): [float(x) for x in v[1]] for L, v in res.items()},
            "temps": [float(x) for x in next(iter(res.values()))[0]],
            "config": {"workload": "L in %s x %d T in [%.3f, %.3f], cold start, sweeps %s, "
                                   "sample every %d, 20%% burn-in, block bootstrap"
                                   % (list(Ls), nT, res[64][0][0], res[64][0][-1], sweeps, record_every)}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--parallelism", choices=["replicas", "strips"], default="replicas",
                    help="N > 1: a lattice per rank (replicas) or one lattice in row strips (strips)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads")
    ap.add_argument("--fss-sweeps", type=int, default=200000)
    ap.add_argument("--fss-long", action="store_true",
                    help="--workload fss on L = 64, 128, 256 with sweeps ~ L^2.17 (2e5 at L = 64) "
                         "on 16 T in [2.255, 2.285]")
    ap.add_argument("--workload", default="default", choices=["default", "fss"],
                    help="default: the L=524288 line; fss: the U4 crossings")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("--steps must be >= 1 and --warmup >= 0")
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        return spawn_ranks(args.gpus)
    ws, rank, local = dist_setup()
    if ws != args.gpus:
        print("bench.py: WORLD_SIZE=%d but --gpus %d" % (ws, args.gpus), file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload == "fss":
        return run_fss(args)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
