"""Host loop for the served form: many concurrent Langevin trajectories
submitting MD-step requests to the library's continuous-batching server
(qmc_server_*).  The scheduling itself (admission, overlap, eviction) is native
code in csrc/server.cu; this module only generates arrivals and collects
results.

Workload of the served form (synthetic stand-in for many independent
dense-hydrogen MD runs): trajectories with N drawn uniformly from {32, 64, 128},
r_s ~ U(1.2, 1.5), T ~ U(600, 3000) K, 1024-8192 walkers each, requests
arriving as a Poisson process with a 2 ms mean inter-arrival time.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import qmcmd as q
from . import synth


@dataclass
class Trajectory:
    cfg: "q.Config"
    R: np.ndarray
    T_kelvin: float
    delta: float


def served_trajectories(n_traj=32, seed=7, sizes=(32, 64, 128), walkers=(1024, 8192), sweeps=4,
                        precision=q.QMC_MIXED) -> list[Trajectory]:
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_traj):
        N = int(rng.choice(sizes))
        rs = float(rng.uniform(1.2, 1.5))
        T = float(rng.uniform(600.0, 3000.0))
        W = int(rng.integers(walkers[0] // 256, walkers[1] // 256 + 1)) * 256
        zeta = synth.ZETA_4 if N == 128 else synth.ZETA_2
        wl = synth.Workload(name=f"serve{k}", N=N, rs=rs, zeta=zeta, walkers=W, sweeps=sweeps, warmup=4,
                            T_kelvin=T, seed=5000 + k)
        cfg = q.Config.from_workload(wl, precision=precision, warmup=4, warmup_cont=1, recompute_every=8)
        out.append(Trajectory(cfg, wl.R, T, 0.1))
    return out


def poisson_arrivals(n: int, mean_ms: float, seed: int) -> np.ndarray:
    """Arrival times (ms from start) of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(mean_ms, size=n))


def percentile(xs, p):
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = (len(xs) - 1) * p / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def run_poisson(server: "q.Server", tids: list[int], trajs: list[Trajectory], n_requests: int, mean_ms=2.0,
                seed=11, poll_sleep_s=5e-5):
    """Submit n_requests MD steps at Poisson times (trajectory drawn uniformly
    per arrival), drive the server until all finish.  Returns (results, wall_s)."""
    rng = np.random.default_rng(seed + 1)
    arrivals = poisson_arrivals(n_requests, mean_ms, seed)
    picks = rng.integers(0, len(tids), size=n_requests)
    pending = {}
    results = []
    t0 = time.perf_counter()
    nxt = 0
    while nxt < n_requests or pending:
        now_ms = (time.perf_counter() - t0) * 1e3
        while nxt < n_requests and arrivals[nxt] <= now_ms:
            k = int(picks[nxt])
            pending[server.submit(tids[k])] = k
            nxt += 1
        if server.progress() > 0 or pending:
            for ticket, k in list(pending.items()):
                r = server.fetch(ticket, tids[k])
                if r is not None:
                    r["walkers"] = trajs[k].cfg.walkers
                    r["samples"] = trajs[k].cfg.walkers * (trajs[k].cfg.sweeps // trajs[k].cfg.measure_every)
                    results.append(r)
                    del pending[ticket]
        time.sleep(poll_sleep_s)
    return results, time.perf_counter() - t0


def device_concurrency(results) -> dict:
    """From the requests' device intervals: the mean number of requests running
    on the GPU while any runs (sum of durations / length of their union) and the
    fraction of requests that overlapped another one."""
    iv = sorted((r["gpu_start_ms"], r["gpu_end_ms"]) for r in results
                if r.get("gpu_start_ms", -1) >= 0 and r.get("gpu_end_ms", -1) > r.get("gpu_start_ms", -1))
    if not iv:
        return {"mean_concurrency": None, "overlapped_fraction": None}
    total = sum(b - a for a, b in iv)
    union, cur_a, cur_b = 0.0, iv[0][0], iv[0][1]
    for a, b in iv[1:]:
        if a > cur_b:
            union += cur_b - cur_a
            cur_a, cur_b = a, b
        else:
            cur_b = max(cur_b, b)
    union += cur_b - cur_a
    over = 0
    for i, (a, b) in enumerate(iv):
        if any(max(a, c) < min(b, d) for j, (c, d) in enumerate(iv) if j != i):
            over += 1
    return {"mean_concurrency": total / union if union > 0 else None, "overlapped_fraction": over / len(iv)}


def summarize(results, wall_s) -> dict:
    lat = [r["latency_ms"] for r in results if r["status"] == 0]
    fe = sum(r["samples"] for r in results if r["status"] == 0)
    run = [r["run_ms"] for r in results if r["status"] == 0]
    return {"requests": len(results), "failed": sum(r["status"] != 0 for r in results),
            "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
            "service_p50_ms": percentile(run, 50), "service_p99_ms": percentile(run, 99),
            "completed_per_s": len(lat) / wall_s,
            "mean_wait_ms": float(np.mean([r["wait_ms"] for r in results])) if results else float("nan"),
            "force_evals_per_s": fe / wall_s, "wall_s": wall_s, **device_concurrency(results)}
