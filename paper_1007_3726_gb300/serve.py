"""Served request stream: a seeded Poisson load generator driving the request
server (ising_server_*), with latency percentiles and aggregate throughput.

The stream follows the served workload: arrivals at `rate` requests per second
for `duration` seconds, L uniform on the powers of two 64 .. 4096, T uniform in
[1.5, 3.5], sweeps log-uniform in [10^2, 10^5] (rounded), a per-request seed,
all drawn from numpy's PCG64 with seed 4.  Each request is admitted against
the server's device-memory budget.  The generator itself does none of the
method's arithmetic.
"""
from __future__ import annotations

import threading
import time

import numpy as np


def poisson_requests(rate: float, duration: float, seed: int = 4, Ls=(64, 128, 256, 512, 1024, 2048, 4096),
                     T_range=(1.5, 3.5), log10_sweeps=(2.0, 5.0), record_every: int = 10):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        out.append(dict(t=t, L=int(rng.choice(Ls)), T=float(rng.uniform(*T_range)),
                        nsweeps=int(round(10 ** rng.uniform(*log10_sweeps))),
                        seed=int(rng.integers(0, 2 ** 63)), record_every=record_every))
    return out


def percentile(xs, q):
    if not xs:
        return None
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


def run_stream(server, requests, drain_s: float = 60.0, poll_s: float = 0.05):
    """Submits `requests` at their arrival times (seconds from now), collects the
    results until all are done or `drain_s` seconds after the last arrival.

    Returns a summary: completed / outstanding counts, p50 / p99 latency
    (finish - arrival) of the completed requests, the same with the outstanding
    ones counted at the end of the window (a lower bound for them), and the
    aggregate attempts per ns of the completed requests over the makespan.
    """
    t0 = time.perf_counter()
    ids = {}
    done = {}
    stop = threading.Event()

    def feeder():
        for i, r in enumerate(requests):
            delay = r["t"] - (time.perf_counter() - t0)
            if delay > 0:
                if stop.wait(delay):
                    return
            rid = server.submit(r["L"], r["T"], r["nsweeps"], seed=r["seed"], init="hot",
                                record_every=r["record_every"], tag=i)
            ids[i] = (rid, time.perf_counter() - t0)

    th = threading.Thread(target=feeder, daemon=True)
    th.start()
    last_arrival = requests[-1]["t"] if requests else 0.0
    deadline = last_arrival + drain_s
    while True:
        for res in server.poll(cap=1024, wait_s=poll_s):
            done[res["tag"]] = res
        now = time.perf_counter() - t0
        if len(done) == len(requests) and not th.is_alive():
            break
        if now > deadline:
            break
    stop.set()
    th.join(timeout=5)
    end = time.perf_counter() - t0
    lat, lat_all, attempts = [], [], 0
    first_submit = None
    for i, r in enumerate(requests):
        if i in done and done[i]["status"] == 0:
            # the server's clock started at its creation: measure from the submit
            res = done[i]
            lat.append(res["t_finish"] - res["t_submit"])
            lat_all.append(lat[-1])
            attempts += r["L"] * r["L"] * r["nsweeps"]
        elif i in ids:
            lat_all.append(end - ids[i][1])
    st = server.stats()
    return {
        "requests": len(requests), "submitted": len(ids), "completed": len(lat),
        "failed": sum(1 for d in done.values() if d["status"] != 0),
        "outstanding": len(ids) - len(done),
        "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
        "p50_s_censored": percentile(lat_all, 50), "p99_s_censored": percentile(lat_all, 99),
        "completed_attempts_per_ns": attempts / end / 1e9 if end > 0 else None,
        "server_attempts_per_ns": st["attempts"] / end / 1e9 if end > 0 else None,
        "gpu_busy_fraction": st["busy_seconds"] / end if end > 0 else None,
        "makespan_s": end, "epochs": st["epochs"], "peak_mem_bytes": st["peak_mem"],
    }
