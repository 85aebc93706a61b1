"""Throughput benchmark of the VMC energy / force / covariance hot path plus the
accelerated Langevin step on GB300.

One step = one qmc_energy_forces call (warm-up continuation sweeps, measured
sweeps with a local-energy and adjoint-force sample each sweep, reductions to
E, f and S) followed by one langevin_step with S = Cov(f).  The default
workload is the N=128 dense-hydrogen system (r_s = 1.2, 4 s-Gaussians per
proton, 16384 walkers, 1000 sweeps) in the mixed-precision form.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun the walkers of one MD trajectory are sharded over the ranks
(each rank keeps the per-GPU walker count: weak scaling); every energy/force
evaluation exchanges its walker sums by two all-reduces and every rank applies
the same Langevin step; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VMC electron moves/s and force-evals/s at N=128 vs FP64 form; p50/p99 latency"
FP32_LANES_PER_SM = 128
N_SM = 152


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="h128")
    ap.add_argument("--rs", type=float, default=1.2)
    ap.add_argument("--walkers", type=int, default=None)
    ap.add_argument("--sweeps", type=int, default=None)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--recompute-every", type=int, default=8)
    ap.add_argument("--fp64-sweeps", type=int, default=50,
                    help="measured sweeps of the timed FP64-form call (0: skip the FP64-form comparison)")
    ap.add_argument("--rs-sweep", default="1.3,1.4,1.5",
                    help="other densities r_s timed at the headline size (comma list; empty: skip)")
    ap.add_argument("--rs-sweeps", type=int, default=200, help="sweeps per timed call of the r_s sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--serve-requests", type=int, default=200, help="served-form requests (0: skip)")
    ap.add_argument("--serve-trajectories", type=int, default=32)
    ap.add_argument("--serve-active", type=int, default=8)
    ap.add_argument("--no-toy", action="store_true", help="skip the toy-model integrator leg")
    ap.add_argument("--toy-only", action="store_true", help="run only the toy-model leg (one JSON line)")
    ap.add_argument("--toy-steps", type=int, default=None, help="steps per trajectory of the timed toy launch")
    ap.add_argument("--no-jastrow34", action="store_true", help="skip the e-e-n-n Jastrow (FP64 form) leg")
    ap.add_argument("--jastrow34-only", action="store_true", help="run only that leg (one JSON line)")
    ap.add_argument("--no-twist", action="store_true", help="skip the twisted-boundary-condition (FP64 form) leg")
    ap.add_argument("--twist-only", action="store_true", help="run only that leg (one JSON line)")
    ap.add_argument("--trajectory", type=int, default=0,
                    help="run only an MD trajectory of this many Langevin steps (S = Cov(f) rebuilt every step) "
                         "at the headline size and print one JSON line")
    ap.add_argument("--traj-sweeps", type=int, default=100, help="measured sweeps per MD step of --trajectory")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# Per-unit FLOP model of the measure kernel (FP32 formula operations, a
# special function -- sqrt, reciprocal, exp, erfc, sin/cos -- counted as one):
#   Jastrow value/gradient/Laplacian per ordered e-e pair        55
#   the same per e-n pair                                         55
#   real-space Ewald per unordered e-e pair: 6 + 10 per image     6 + 10 * 4.19
#     (4.19 = mean number of images with |r + nL| < L)
#   e-n pair: Jastrow third-order chain, Hessian product          130
#     plus Ewald value and gradient: 6 + 19 per image              6 + 19 * 4.19
#   reciprocal space: structure factor 14 per (electron, k),
#     force 12 per (nucleus, k)
#   g_i, l_i: 8 n per electron;  K = G Y G: 8 n^3 per walker
# DRAM traffic of a kernel comes from the committed ncu summaries under
# profiles/: a line "machine: kernel=<class> traffic_bytes_per_<unit>=<bytes>
# source=<file> sha256=<hex>" written from one capture.  It is used only while
# the kernel's source file still has that hash (null once the kernel changed).
MEASURE_UNIT = {"ee_jas": 55.0, "ep_jas": 55.0, "ee_ewald": 6.0 + 10.0 * 4.19, "ep": 130.0 + 6.0 + 19.0 * 4.19,
                "sk": 14.0, "fk": 12.0}


def _profile_traffic(cls: str):
    """(bytes per unit, unit, summary file) of kernel class `cls` from profiles/, or None."""
    import glob
    import hashlib
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            m = re.match(r"\s*machine:\s*kernel=(\S+)\s+traffic_bytes_per_(\S+?)=(\S+)\s+source=(\S+)\s+sha256=(\S+)",
                         line)
            if not m or m.group(1) != cls:
                continue
            src = os.path.join(ROOT, m.group(4))
            if not os.path.exists(src):
                continue
            if hashlib.sha256(open(src, "rb").read()).hexdigest() != m.group(5):
                return None
            return float(m.group(3)), m.group(2), os.path.relpath(path, ROOT)
    return None


def _nk(mmax: int) -> int:
    """Half-space reciprocal vectors 0 < |m|^2 <= mmax^2 (the Ewald k-sum)."""
    r = range(-mmax, mmax + 1)
    return sum(1 for x in range(0, mmax + 1) for y in r for z in r
               if (x > 0 or (x == 0 and y > 0) or (x == 0 and y == 0 and z > 0)) and x * x + y * y + z * z <= mmax * mmax)


def _flops_per_launch(cls: str, W, N, n, B, G, acc_ratio, use_tc, nk=462):
    """Algorithmic FLOPs of one launch of a kernel class (dense multiply-adds x 2)."""
    if cls == "orbitals_prop":
        return 2.0 * W * N * B * n
    if cls == "orbitals_meas":   # grad (3) + Laplacian on the tensor cores; SIMT also forms the values
        return (8.0 if use_tc else 10.0) * W * N * B * n
    if cls == "measure":
        u = MEASURE_UNIT
        # (the mixed form computes the reciprocal-space force, fk, as a GEMM
        # over walkers timed with the adjoint class)
        pairs = (u["ee_jas"] * N * (N - 1) + u["ep_jas"] * N * N + u["ee_ewald"] * N * (N - 1) / 2
                 + u["ep"] * N * N + (u["sk"] + (0.0 if use_tc else u["fk"])) * N * nk + 8.0 * n * N + 8.0 * n ** 3)
        adj = 0.0 if use_tc else 8.0 * N * G * n * n   # Z = C G, P = C K in the SIMT measure kernel
        return W * (pairs + adj)
    if cls == "adjoint":         # Z = C G and P = C (G Y G) per spin block on the tensor cores
        return 8.0 * W * N * G * n * n
    if cls == "sweep":
        return 2.0 * W * N * (n + acc_ratio * 2.0 * n * n)
    return None


def _hbm_bytes_per_launch(cls: str, W, N, n, nk, acc_ratio, t=4):
    """Algorithmic HBM bytes of one launch (state that must come from or go to
    HBM once; working precision t bytes), for the kernels whose HBM rate is
    reported beside their ALU roofline:
      sweep    per walker: G^T of both spins read and written (2 x 2 n^2 t), the
               proposals' orbital rows (N n t), their trig (6 N t) and uniforms
               (N t), positions read (24 N) and accepted ones written (24 N p_acc);
      measure  per walker: D (3 N n t), Lp (N n t), G^T (2 n^2 t), positions
               (24 N), accumulators read and written (2 x 8 (3 + 9 N)); out to
               the adjoint kernel K^T (2 n^2 t), electron data (9 N t),
               E_L (8) and the structure factor (2 nk t)."""
    if cls == "sweep":
        return W * (2 * 2 * n * n * t + N * n * t + 6 * N * t + N * t + 24 * N + 24 * N * acc_ratio)
    if cls == "measure":
        return W * (3 * N * n * t + N * n * t + 2 * n * n * t + 24 * N + 2 * 8 * (3 + 9 * N)
                    + 2 * n * n * t + 9 * N * t + 8 + 2 * nk * t)
    return None


def _cpu_baseline(wl, walkers_per_core=1):
    """The FP64 oracle on the host cores: one sweep plus one local-energy and
    force sample per walker, W = threads x walkers_per_core."""
    import numpy as np
    from oracle import oracle as orc
    threads = orc.num_threads()
    W = threads * walkers_per_core
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    t0 = time.perf_counter()
    orc.vmc(osys, wl.R, W=W, n_sweeps=1, n_warmup=0, sigma=wl.sigma, seed=wl.seed, forces=True)
    dt = time.perf_counter() - t0
    moves = W * wl.N
    return {"value": moves / dt, "unit": "electron moves/s", "cores": threads, "kind": "oracle",
            "sample": f"{W} walkers x 1 sweep of N={wl.N} (each sweep followed by one E_L + 3N-force sample), "
                      f"{dt:.1f} s", "force_evals_per_s": W / dt, "seconds": dt, "moves": moves}


# Rotating-spring toy model (SI, "A simple toy model"): the integrator comparison
# on the GPU.  Timed configuration: the adopted scheme with S = G_lambda, one
# trajectory per thread, 152 SMs x 3 resident CTAs x 256 threads.
TOY_BENCH = {"n_traj": N_SM * 3 * 256, "n_steps": 20000, "n_burn": 2000, "delta": 0.2, "seed": 11}
# FP64 operations per step of that scheme, from its formulas (a special function
# -- log, sqrt, sincos, atan2, reciprocal -- counted as one): noise 11, force 6,
# S 10, Cholesky 7, z 4, S^{-1} f 8, S-difference term and its solve 20,
# update 12, polar angle 8, radius 4, sums 7.
TOY_FLOPS_PER_STEP = 97
FP64_NOMINAL_TFLOPS = 1.25     # GB300 dense FP64, nominal (no measured FP64 peak on this machine)


def _toy_bench(stream, steps, rank, n_steps=None, table=True):
    """Time the toy-model launch; also <U> against the time step for every scheme."""
    import numpy as np
    import torch
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth
    cfg = dict(TOY_BENCH)
    if n_steps:
        cfg["n_steps"], cfg["n_burn"] = n_steps, n_steps // 10
    n = cfg["n_traj"]
    xy = torch.tensor(synth.toy_starts(n, cfg["seed"] + rank), device="cuda")
    out = torch.empty((n, q.QMC_TOY_NOUT), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")      # 256 MB > L2
    p = q.toy_params(q.QMC_TOY_ADOPTED, q.QMC_TOY_S_G, delta=cfg["delta"], n_steps=cfg["n_steps"],
                     n_burn=cfg["n_burn"], seed=cfg["seed"] + rank)
    pw = q.toy_params(q.QMC_TOY_ADOPTED, q.QMC_TOY_S_G, delta=cfg["delta"], n_steps=200, n_burn=0,
                      seed=cfg["seed"] + rank)
    for _ in range(3):
        q.toy_langevin_device(pw, xy, out, stream.cuda_stream)
    torch.cuda.synchronize()
    ms = []
    for _ in range(max(steps, 1)):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q.toy_langevin_device(p, xy, out, stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    o = out.cpu().numpy()
    avg = sum(ms) / len(ms)
    nsteps = n * cfg["n_steps"]
    value = nsteps / (avg / 1e3)
    ach = value * TOY_FLOPS_PER_STEP / 1e12
    mean_u = float(o[:, 2].sum() / (n * (cfg["n_steps"] - cfg["n_burn"])))
    # <U> versus the time step (the SI's figure): 16384 trajectories, 2000 time units each
    rows = {}
    xs = xy[:16384].contiguous()
    os_ = out[:16384]
    modes = ((q.QMC_TOY_S_G, synth.TOY_MU, "G_lambda"), (q.QMC_TOY_S_HG, 2.0, "H+2G_lambda")) if table else ()
    for s_mode, mu, tag in modes:
        for name, sc in q.TOY_SCHEMES.items():
            row = {}
            for d in (0.4, 0.2, 0.1, 0.05):
                pp = q.toy_params(sc, s_mode, mu=mu, delta=d, n_steps=int(round(2000 / d)),
                                  n_burn=int(round(200 / d)), seed=cfg["seed"] + 1)
                q.toy_langevin_device(pp, xs, os_, stream.cuda_stream)
                torch.cuda.synchronize()
                oo = os_.cpu().numpy()
                ok = oo[:, 6] == 0
                m = oo[ok, 2] / (pp.n_steps - pp.n_burn)
                row[str(d)] = {"mean_U": float(m.mean()) if ok.any() else None,
                               "err": float(m.std() / max(ok.sum(), 1) ** 0.5) if ok.any() else None,
                               "stopped": int((~ok).sum())}
            rows[f"{tag}/{name}"] = row
    return {"metric": "toy-model trajectory steps/s (adopted scheme, S = G_lambda, FP64)", "value": value,
            "unit": "trajectory steps/s", "ms_per_launch": avg, "launches_timed": len(ms),
            "config": {"workload": f"rotating spring k={synth.TOY_K}, a={synth.TOY_A}, T={synth.TOY_T}, "
                                   f"lambda={synth.TOY_LAMBDA}, alpha={synth.TOY_ALPHA}, delta={cfg['delta']}, "
                                   f"{n} trajectories x {cfg['n_steps']} steps",
                       "l2": "L2 flushed (256 MB write) before every timed launch"},
            "roofline": {"kernel": "toy_kernel", "bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach / FP64_NOMINAL_TFLOPS, "traffic": None,
                         "peak_source": "nominal GB300 dense FP64", "flops_per_step": TOY_FLOPS_PER_STEP},
            "mean_U": mean_u, "canonical_mean_U": synth.TOY_T / 2,
            "stopped_trajectories": int((o[:, 6] != 0).sum()),
            "mean_U_vs_delta": rows or None}


def _jastrow34_bench(stream, calls=8):
    """Both forms with and without the e-e-n-n Jastrow term: the FP64 form at
    N = 64 (1024 walkers) and the mixed form at N = 128 (4096 walkers), 4
    measured sweeps + 1 continuation per call, a sample every sweep: after a
    warm-up call, `calls` calls timed one by one; the median, min and max and the
    median SM clock over them."""
    import numpy as np
    import torch
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth
    out = {"metric": "electron moves/s and force-evals/s with and without U_{3+4}",
           "config": {"workload": "FP64 form: h64 (N=64, r_s=1.4, 2 s-Gaussians/proton), 1024 walkers; mixed "
                                  "form: h128 (N=128, r_s=1.2, 4 s-Gaussians/proton), 4096 walkers; 4 sweeps "
                                  "(+1 continuation) per call, sample every sweep, U_{3+4} coefficients "
                                  "symmetric U(-0.3, 0.3), exponent 0.7933844"}}
    for form, name, walkers in (("fp64", "h64", 1024), ("mixed", "h128", 4096)):
        _jastrow34_legs(stream, calls, out, form, name, walkers)
    return out


def _jastrow34_legs(stream, calls, out, form, name, walkers):
    import numpy as np
    import torch
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth
    wl = synth.workload(name, walkers=walkers, sweeps=4, warmup=2)
    A = np.random.default_rng(5).uniform(-0.3, 0.3, (wl.N, wl.N))
    fj = 0.5 * (A + A.T)
    R_dev = torch.tensor(wl.R, dtype=torch.float64, device="cuda")
    prec = q.QMC_FP64 if form == "fp64" else q.QMC_MIXED
    for tag, f in ((f"{form}_without", None), (f"{form}_with", fj)):
        cfg = q.Config.from_workload(wl, precision=prec, warmup=2, warmup_cont=1, measure_every=1,
                                     recompute_every=4, fj=f)
        sysq = q.QMCSystem(cfg, wl.R)
        sysq.set_stream(stream.cuda_stream)
        o = torch.zeros(4 + 3 * wl.N + 9 * wl.N * wl.N, dtype=torch.float64, device="cuda")
        sysq.energy_forces_device(R_dev, o)          # warm-up call
        sysq.sync()
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        ts = []
        for _ in range(calls):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sysq.energy_forces_device(R_dev, o)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        clk = clocks.stop()
        sysq.sync()
        ts.sort()
        t = ts[len(ts) // 2]
        moves = wl.walkers * wl.N * (cfg.sweeps + cfg.warmup_cont)
        out[tag] = {"electron_moves_per_s": moves / t, "force_evals_per_s": wl.walkers * cfg.sweeps / t,
                    "ms_per_call_median": 1e3 * t, "ms_per_call_min": 1e3 * ts[0], "ms_per_call_max": 1e3 * ts[-1],
                    "calls_timed": calls, "sm_mhz_median": clk.get("sm_mhz"), "clock_reasons": clk.get("reasons"),
                    "E": float(o[0].item())}
        sysq.close()


def _twist_bench(stream, calls=5):
    """Twisted boundary conditions with the k-point average (FP64 form): the
    main text's 64-atom cell with its 4 x 4 x 4 Monkhorst-Pack mesh (64 twists),
    h64 (N = 64, r_s = 1.4, 2 s-Gaussians/proton), 16 walkers per twist (1024),
    4 measured sweeps + 1 continuation per call, a sample every sweep, inverse
    recompute every 4 sweeps; after a warm-up call, `calls` calls timed one by
    one (median, min, max, median SM clock), then one profiled call for the
    per-kernel split.  The Gamma-point FP64 form at the same size, and the
    twisted form with the e-e-n-n Jastrow term (the paper's production
    wavefunction; synthetic symmetric U(-0.3, 0.3) coefficients), are timed
    the same way beside it."""
    import torch
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth
    tw = synth.monkhorst_pack(4)
    wl = synth.workload("h64", walkers=16 * len(tw), sweeps=4, warmup=2)
    R_dev = torch.tensor(wl.R, dtype=torch.float64, device="cuda")
    out = {"metric": "electron moves/s and force-evals/s, twist-averaged (64 twists) and Gamma point",
           "config": {"workload": f"h64: N=64 H, r_s=1.4, 2 s-Gaussians/proton, 4x4x4 Monkhorst-Pack twists, "
                                  f"{wl.walkers} walkers (16 per twist), 4 sweeps (+1 continuation) per call, "
                                  "sample every sweep, inverse recompute every 4 sweeps, FP64 form"}}
    import numpy as np
    A = np.random.default_rng(5).uniform(-0.3, 0.3, (wl.N, wl.N))
    fj = 0.5 * (A + A.T)        # e-e-n-n Jastrow coefficients (synthetic, symmetric)
    for tag, twists, f in (("twisted", tw, None), ("gamma", None, None), ("twisted_with_U34", tw, fj)):
        cfg = q.Config.from_workload(wl, precision=q.QMC_FP64, warmup=2, warmup_cont=1, measure_every=1,
                                     recompute_every=4, twists=twists, fj=f)
        sysq = q.QMCSystem(cfg, wl.R)
        sysq.set_stream(stream.cuda_stream)
        o = torch.zeros(4 + 3 * wl.N + 9 * wl.N * wl.N, dtype=torch.float64, device="cuda")
        sysq.energy_forces_device(R_dev, o)          # warm-up call
        sysq.sync()
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        ts = []
        for _ in range(calls):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sysq.energy_forces_device(R_dev, o)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        clk = clocks.stop()
        sysq.sync()
        sysq.set_profiling(True)
        sysq.kernel_times()
        sysq.energy_forces_device(R_dev, o)
        kt = sysq.kernel_times()
        sysq.set_profiling(False)
        sysq.sync()
        ts.sort()
        t = ts[len(ts) // 2]
        moves = wl.walkers * wl.N * (cfg.sweeps + cfg.warmup_cont)
        out[tag] = {"electron_moves_per_s": moves / t, "force_evals_per_s": wl.walkers * cfg.sweeps / t,
                    "ms_per_call_median": 1e3 * t, "ms_per_call_min": 1e3 * ts[0], "ms_per_call_max": 1e3 * ts[-1],
                    "calls_timed": calls, "sm_mhz_median": clk.get("sm_mhz"), "clock_reasons": clk.get("reasons"),
                    "kernel_ms_per_call": {k: round(v[0], 3) for k, v in kt.items() if v[1]},
                    "E": float(o[0].item()), "E_err": float(o[1].item())}
        sysq.close()
    out["twisted_over_gamma_time"] = out["twisted"]["ms_per_call_median"] / out["gamma"]["ms_per_call_median"]
    out["with_U34_over_twisted_time"] = (out["twisted_with_U34"]["ms_per_call_median"]
                                         / out["twisted"]["ms_per_call_median"])
    return out


def _empirical_bench(stream, steps=10):
    """The Langevin step at N = 128 (3N = 384) with S = H + mu I built on the
    device each step (QMC_S_EMPIRICAL: screened-Coulomb pair Hessian, then
    the step's Cholesky and solves) beside the same step with S passed in
    (QMC_S_COV); after 3 warm-up steps, `steps` steps timed one by one with
    CUDA events on the handle's stream (median)."""
    import numpy as np
    import torch
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth
    wl = synth.workload("h128", walkers=2)
    n3 = 3 * wl.N
    out = {"metric": "Langevin steps/s at N = 128", "config": {"workload": "h128 protons, T = 1500 K, Delta = 0.02, "
                                                                          "lambda = Thomas-Fermi length, mu = 1.5 "
                                                                          "(H's lowest eigenvalue here: -1.30)"}}
    for tag, mode in (("empirical_S", q.QMC_S_EMPIRICAL), ("given_S", q.QMC_S_COV)):
        sysq = q.QMCSystem(q.Config.from_workload(wl), wl.R)
        sysq.set_stream(stream.cuda_stream)
        sysq.set_empirical_s(0.0, 1.5)
        R = torch.tensor(wl.R.ravel(), dtype=torch.float64, device="cuda")
        f = torch.tensor(0.01 * np.random.default_rng(1).standard_normal(n3), dtype=torch.float64, device="cuda")
        S = torch.tensor(sysq.empirical_s(wl.R), dtype=torch.float64, device="cuda")
        ts = []
        for k in range(3 + steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sysq.langevin_step_device(R, f, S if mode == q.QMC_S_COV else None, 1500.0, 0.02, mode, 0.0)
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(e0.elapsed_time(e1))
        sysq.sync()
        ts.sort()
        out[tag] = {"ms_per_step_median": ts[len(ts) // 2], "ms_min": ts[0], "ms_max": ts[-1],
                    "steps_per_s": 1e3 / ts[len(ts) // 2], "R_finite": bool(torch.isfinite(R).all().item())}
        sysq.close()
    return out


def _toy_cpu_baseline():
    """The oracle's toy model on the host cores: 4096 trajectories x 20000 steps."""
    import numpy as np
    from oracle import oracle as orc
    from paper_1605_08423_gb300 import synth
    cfg = TOY_BENCH
    a = orc.toy_args(orc.TOY_ADOPTED, orc.TOY_S_G, delta=cfg["delta"], n_steps=cfg["n_steps"],
                     n_burn=cfg["n_burn"], seed=cfg["seed"])
    xy0 = synth.toy_starts(4096, cfg["seed"])
    orc.lib()                      # build / load outside the timed region
    t0 = time.perf_counter()
    orc.toy_run(a, xy0)
    dt = time.perf_counter() - t0
    return {"value": 4096 * cfg["n_steps"] / dt, "unit": "trajectory steps/s", "cores": orc.num_threads(),
            "kind": "oracle", "sample": f"4096 trajectories x {cfg['n_steps']} steps, {dt:.2f} s"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_1605_08423_gb300 import synth
    wl = synth.workload(args.workload, rs=args.rs)
    times = []
    last = None
    for i in range(args.warmup + args.steps):
        r = _cpu_baseline(wl)
        if i >= args.warmup:
            times.append(r)
        last = r
    tot_moves = sum(t["moves"] for t in times)
    tot_time = sum(t["seconds"] for t in times)
    value = tot_moves / tot_time
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "electron moves/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_time / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"{args.workload} (N={wl.N}, r_s={wl.rs}, {wl.n_gauss} s-Gaussians/proton); "
                                  "each step a bounded sample on the host cores"},
           "cpu_baseline": {"value": value, "unit": "electron moves/s", "cores": last["cores"], "kind": "oracle",
                            "sample": last["sample"]},
           "e2e": {"value": value, "unit": "electron moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_toy_only(args, rank, local):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    toy = _toy_bench(stream, args.steps, rank, n_steps=args.toy_steps, table=False)
    if rank == 0:
        print(json.dumps({**toy, "n_gpus": 1, "steps": args.steps, "warmup": 3, "higher_is_better": True,
                          "dtype": "f64", "data": "synthetic"}), flush=True)


def run_trajectory(args, rank, local):
    """A Langevin trajectory at T = 1500 K (the headline system's temperature),
    Delta = 0.1, S = Cov(f) rebuilt by every step's energy/force call, walkers
    carried over between steps; the whole trajectory timed with CUDA events on
    the library's stream (device API, R resident on the device)."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    over = {"rs": args.rs, "seed": 1002 + rank, "sweeps": args.traj_sweeps}
    if args.walkers:
        over["walkers"] = args.walkers
    wl = synth.workload(args.workload, **over)
    prec = q.QMC_MIXED if args.precision == "mixed" else q.QMC_FP64
    cfg = q.Config.from_workload(wl, precision=prec, warmup=20, warmup_cont=5, measure_every=1,
                                 recompute_every=args.recompute_every)
    N, W, N3 = wl.N, wl.walkers, 3 * wl.N
    system = q.QMCSystem(cfg, wl.R)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    system.set_stream(stream.cuda_stream)
    R_dev = torch.tensor(wl.R, dtype=torch.float64, device="cuda")
    steps = args.trajectory
    outs = torch.zeros((steps, 4 + N3 + N3 * N3), dtype=torch.float64, device="cuda")
    Rs = torch.zeros((steps + 1, N3), dtype=torch.float64, device="cuda")
    Rs[0] = R_dev.reshape(-1)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        system.energy_forces_device(R_dev, outs[k])
        system.langevin_step_device(R_dev, outs[k, 4:4 + N3], outs[k, 4 + N3:], wl.T_kelvin, wl.delta, q.QMC_S_COV)
        Rs[k + 1].copy_(R_dev.reshape(-1))
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    system.sync()
    ms = e0.elapsed_time(e1)
    o = outs.cpu().numpy()
    E, Eerr = o[:, 0], o[:, 1]
    R = Rs.cpu().numpy()
    d = R[1:] - R[:-1]
    d -= wl.L * np.round(d / wl.L)
    step_rms = np.sqrt(np.mean(d ** 2, axis=1))
    half = steps // 2
    slope = float(np.polyfit(np.arange(steps), E, 1)[0]) if steps > 1 else 0.0
    moves = W * N * (cfg.sweeps + cfg.warmup_cont) * steps
    out = {"metric": "MD steps/s of the accelerated Langevin dynamics (VMC E, f, S = Cov(f) every step)",
           "value": steps / (ms / 1e3), "unit": "MD steps/s", "steps": steps, "ms_per_md_step": ms / steps,
           "electron_moves_per_s": moves / (ms / 1e3), "force_evals_per_s": W * cfg.sweeps * steps / (ms / 1e3),
           "dtype": "f32" if prec == q.QMC_MIXED else "f64", "data": "synthetic", "clocks": clk,
           "config": {"workload": f"{args.workload}: N={N} H, r_s={wl.rs}, L={wl.L:.3f} bohr, {wl.n_gauss} "
                                  f"s-Gaussians/proton, {W} walkers x {cfg.sweeps} sweeps (+{cfg.warmup_cont} "
                                  f"continuation) per MD step, T={wl.T_kelvin} K, Delta={wl.delta}, adopted scheme, "
                                  f"alpha = 0.122 N_c, S = Cov(f) rebuilt every step",
                      "walkers": W, "sweeps_per_step": cfg.sweeps},
           "E_first": float(E[0]), "E_last": float(E[-1]),
           "E_mean_first_half": float(E[:half].mean()) if half else None,
           "E_mean_second_half": float(E[half:].mean()),
           "E_err_median": float(np.median(Eerr)), "E_slope_per_step": slope,
           "accept_mean": float(o[:, 3].mean()), "rms_nuclear_step_bohr": float(step_rms.mean()),
           "E_series": [float(x) for x in E]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    system.close()


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    shard = ws > 1
    if shard:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    over = {"rs": args.rs, "seed": 1002}     # one system; under torchrun its walkers are split over the ranks
    if args.walkers:
        over["walkers"] = args.walkers
    if args.sweeps:
        over["sweeps"] = args.sweeps
    wl = synth.workload(args.workload, **over)
    prec = q.QMC_MIXED if args.precision == "mixed" else q.QMC_FP64
    cfg = q.Config.from_workload(wl, precision=prec, warmup=20, warmup_cont=5, measure_every=1,
                                 recompute_every=args.recompute_every)
    N, n, G = wl.N, wl.N // 2, wl.n_gauss
    B, W, N3 = N * G, wl.walkers, 3 * wl.N
    system = q.QMCSystem(cfg, wl.R)
    if shard:
        system.set_walker_offset(rank * W)   # rank r holds walkers [r W, (r + 1) W) of W x ranks
    # a dedicated stream: the library launches on it and the timing events are recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    system.set_stream(stream.cuda_stream)
    group = q.ShardGroup(system, W * ws) if shard else None
    R_dev = torch.tensor(wl.R, dtype=torch.float64, device="cuda")
    out_dev = torch.zeros(4 + N3 + N3 * N3, dtype=torch.float64, device="cuda")
    T_K, delta = wl.T_kelvin, wl.delta

    def evaluate():
        if group is not None:
            group.energy_forces_device(R_dev, out_dev)
        else:
            system.energy_forces_device(R_dev, out_dev)

    def step():
        evaluate()
        system.langevin_step_device(R_dev, out_dev[4:4 + N3], out_dev[4 + N3:], T_K, delta, q.QMC_S_COV)

    for _ in range(args.warmup):
        step()
    system.sync()
    system.kernel_times()          # reset
    system.set_profiling(True)
    n0 = system.launch_count()
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    system.sync()
    launches = system.launch_count() - n0
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    kt = system.kernel_times()
    system.set_profiling(False)
    res = q.unpack_out(out_dev.cpu().numpy(), N)
    sweeps_per_step = cfg.warmup_cont + cfg.sweeps
    moves_per_step = W * N * sweeps_per_step
    fevals_per_step = W * (cfg.sweeps // cfg.measure_every)
    value = ws * moves_per_step * args.steps / (ms / 1e3)
    fevals = ws * fevals_per_step * args.steps / (ms / 1e3)

    # end to end through the public API with host buffers: one GPU, the
    # host-pointer C ABI (R, f, S copied in and out inside the calls); sharded,
    # R copied in from pinned host memory, the sharded evaluation and Langevin
    # step, the result (E, E_err, N_c, accept, f, S and R') copied back
    Rh = wl.R.copy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if group is None:
        for _ in range(args.e2e_steps):
            r = system.energy_forces(Rh)
            Rh = system.langevin_step(Rh, r["f"], r["S"], T_K, delta, q.QMC_S_COV).reshape(N, 3)
    else:
        R_pin = torch.tensor(Rh, dtype=torch.float64).pin_memory()
        out_pin = torch.zeros(out_dev.numel() + N3, dtype=torch.float64).pin_memory()
        for _ in range(args.e2e_steps):
            R_dev.copy_(R_pin.reshape(N, 3), non_blocking=True)
            step()
            out_pin[:out_dev.numel()].copy_(out_dev, non_blocking=True)
            out_pin[out_dev.numel():].copy_(R_dev.reshape(-1), non_blocking=True)
            torch.cuda.current_stream().synchronize()
            R_pin.copy_(out_pin[out_dev.numel():])
    t_e2e = time.perf_counter() - t0
    e2e = ws * moves_per_step * args.e2e_steps / t_e2e
    h2d = 8 * (N3 + N3 + N3 + N3 * N3)
    d2h = 8 * (4 + N3 + N3 * N3 + N3)

    # roofline of every kernel class with an algorithmic FLOP count; the dominant one is "roofline"
    peaks, peak_kind = _peaks()
    sm_clock = (clk.get("sm_max_mhz") or 2070.0) * 1e6
    fp32_peak = N_SM * FP32_LANES_PER_SM * 2 * sm_clock / 1e12
    bf16_sust = float(peaks.get("bf16_tflops_sustained", 1700.0))
    tf32_peak = bf16_sust * (1.1 / 2.25)      # nominal TF32 / BF16 dense ratio
    use_tc = prec == q.QMC_MIXED
    roofs = {}
    for cls, (cms, cl) in kt.items():
        fl = _flops_per_launch(cls, W, N, n, B, G, float(res["accept"]), use_tc, nk=_nk(cfg.mmax))
        if fl is None or cl == 0:
            continue
        avg = cms / cl
        ach = fl / (avg / 1e3) / 1e12
        if use_tc and (cls.startswith("orbitals") or cls == "adjoint"):
            # 2xTF32 pieces: three tensor products per algorithmic product
            roofs[cls] = {"kernel": cls, "bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s",
                          "frac": ach / tf32_peak, "traffic": None,
                          "peak_source": f"TF32 = {peak_kind} bf16 sustained x 1.1/2.25 (nominal ratio)",
                          "flops_per_launch": fl, "tensor_pipe_flops_per_launch": 3 * fl, "avg_launch_ms": avg}
        else:
            roofs[cls] = {"kernel": cls, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                          "frac": ach / fp32_peak, "traffic": None,
                          "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max SM clock",
                          "flops_per_launch": fl, "avg_launch_ms": avg}
            hb = _hbm_bytes_per_launch(cls, W, N, n, _nk(cfg.mmax), float(res["accept"]),
                                       4 if prec == q.QMC_MIXED else 8)
            if hb:
                gbs = hb / (avg / 1e3) / 1e9
                roofs[cls].update({"hbm_bytes_per_launch_algorithmic": hb, "hbm_gbs_achieved": gbs,
                                   "hbm_frac_of_measured_copy": gbs / float(peaks.get("hbm_gbs", 6800.0))})
    dom = max(kt, key=lambda k: kt[k][0])
    for cls in roofs:
        tr = _profile_traffic(cls) if use_tc and N == 128 and G == 4 else None
        if tr is not None:
            per_unit, unit, src = tr
            units = {"walker": W, "row": W * N}.get(unit)
            if units:
                roofs[cls]["traffic"] = per_unit * units
                roofs[cls]["traffic_source"] = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per {unit} "
                                                f"({src}), scaled to the launch; same kernel source")
    roof = roofs.get(dom, {"kernel": dom, "bound": "alu", "achieved": None, "peak": fp32_peak,
                           "unit": "TFLOP/s", "frac": None, "traffic": None})
    breakdown = {k: {"ms": v[0] / args.steps, "launches": v[1] // max(args.steps, 1)} for k, v in kt.items()}

    # FP64 form on the same system, like for like: the same walkers, sample
    # every sweep, the same continuation and recompute schedule; one warm-up
    # call (walker warm-up plus code paths), then one timed call of
    # args.fp64_sweeps measured sweeps (+ the continuation sweeps), CUDA events
    # on the same stream.
    fp64 = None
    if args.fp64_sweeps > 0 and prec == q.QMC_MIXED and rank == 0:
        wl64 = synth.workload(args.workload, **{**over, "sweeps": args.fp64_sweeps})
        cfg64 = q.Config.from_workload(wl64, precision=q.QMC_FP64, warmup=cfg.warmup_cont, warmup_cont=cfg.warmup_cont,
                                       measure_every=1, recompute_every=args.recompute_every)
        s64 = q.QMCSystem(cfg64, wl.R)
        s64.set_stream(stream.cuda_stream)
        out64 = torch.zeros_like(out_dev)
        s64.energy_forces_device(R_dev, out64)       # warm-up call
        s64.sync()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.energy_forces_device(R_dev, out64)
        f1.record(stream)
        torch.cuda.synchronize()
        s64.sync()
        t64 = f0.elapsed_time(f1) / 1e3
        sw64 = args.fp64_sweeps + cfg64.warmup_cont
        fp64 = {"value": W * N * sw64 / t64, "unit": "electron moves/s",
                "force_evals_per_s": W * args.fp64_sweeps / t64, "ms_per_call": 1e3 * t64,
                "sample": f"one call after a warm-up call: {args.fp64_sweeps} sweeps (+{cfg64.warmup_cont} "
                          f"continuation), a sample every sweep, {W} walkers, FP64 inverse recompute every "
                          f"{args.recompute_every} sweeps",
                "mixed_over_fp64_moves": value / (W * N * sw64 / t64),
                "mixed_over_fp64_force_evals": fevals / (W * args.fp64_sweeps / t64)}
        s64.close()

    # the other densities of the headline size: one warm-up call, one timed call each
    rs_rows = None
    if args.rs_sweep and prec == q.QMC_MIXED and rank == 0 and args.workload == "h128":
        rs_rows = {}
        for rs in [float(x) for x in args.rs_sweep.split(",") if x.strip()]:
            wlr = synth.workload(args.workload, **{**over, "rs": rs, "sweeps": args.rs_sweeps})
            cfgr = q.Config.from_workload(wlr, precision=prec, warmup=20, warmup_cont=cfg.warmup_cont,
                                          measure_every=1, recompute_every=args.recompute_every)
            sr = q.QMCSystem(cfgr, wlr.R)
            sr.set_stream(stream.cuda_stream)
            Rr = torch.tensor(wlr.R, dtype=torch.float64, device="cuda")
            outr = torch.zeros_like(out_dev)
            sr.energy_forces_device(Rr, outr)
            sr.sync()
            torch.cuda.synchronize()
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            sr.energy_forces_device(Rr, outr)
            r1.record(stream)
            torch.cuda.synchronize()
            sr.sync()
            tr = r0.elapsed_time(r1) / 1e3
            o = outr.cpu().numpy()
            rs_rows[f"{rs:g}"] = {"L": wlr.L, "electron_moves_per_s": W * N * (args.rs_sweeps + cfgr.warmup_cont) / tr,
                                  "force_evals_per_s": W * args.rs_sweeps / tr, "ms_per_call": 1e3 * tr,
                                  "E": float(o[0]), "E_err": float(o[1]), "accept": float(o[3])}
            sr.close()
        rs_rows[f"{wl.rs:g}"] = {"L": wl.L, "electron_moves_per_s": value, "force_evals_per_s": fevals,
                                 "ms_per_call": ms / args.steps, "E": res["E"], "E_err": res["E_err"],
                                 "accept": res["accept"], "note": "headline timed steps"}

    # served form: many concurrent trajectories, Poisson arrivals, continuous batching
    serving = None
    if args.serve_requests > 0:
        from paper_1605_08423_gb300 import serve
        system.close()
        trajs = serve.served_trajectories(n_traj=args.serve_trajectories, seed=7 + rank)
        free, _ = torch.cuda.mem_get_info()
        srv = q.Server(int(0.6 * free), args.serve_active)
        tids = [srv.add_trajectory(t.cfg, t.R, t.T_kelvin, t.delta) for t in trajs]
        sres, swall = serve.run_poisson(srv, tids, trajs, n_requests=args.serve_requests, mean_ms=2.0,
                                        seed=13 + rank)
        serving = serve.summarize(sres, swall)
        # the same mix offered below its measured capacity (60 %): latency is then
        # service time plus little queueing
        cap = serving["completed_per_s"]
        if cap > 0:
            mean_lo = 1e3 / (0.6 * cap)
            n_lo = max(20, args.serve_requests // 4)
            lres, lwall = serve.run_poisson(srv, tids, trajs, n_requests=n_lo, mean_ms=mean_lo, seed=17 + rank)
            lo = serve.summarize(lres, lwall)
            lo["mean_interarrival_ms"] = mean_lo
            serving["below_capacity"] = lo
        serving.update({"trajectories": len(trajs), "mean_interarrival_ms": 2.0, "max_active": args.serve_active,
                        "hbm_budget_gb": srv.stats()["budget"] / 1e9, "stats": srv.stats(),
                        "workload": "N in {32,64,128}, r_s~U(1.2,1.5), T~U(600,3000) K, 1024-8192 walkers, "
                                    "4 sweeps + 1 continuation per MD step (first step: 4 warm-up sweeps), "
                                    "mixed form, Langevin step with S = Cov(f)"})
        srv.close()

    toy = None
    if not args.no_toy:
        toy = _toy_bench(stream, args.steps, rank)
        toy["cpu_baseline"] = _toy_cpu_baseline() if rank == 0 and ws == 1 and not args.no_cpu_baseline else None

    j34 = None
    if not args.no_jastrow34 and rank == 0:
        try:
            j34 = _jastrow34_bench(stream)
        except Exception as exc:   # a secondary leg: report, do not lose the headline line
            j34 = {"error": f"{type(exc).__name__}: {exc}"}

    twl = None
    if not args.no_twist and rank == 0:
        try:
            twl = _twist_bench(stream)
        except Exception as exc:   # a secondary leg: report, do not lose the headline line
            twl = {"error": f"{type(exc).__name__}: {exc}"}

    emp = None
    if not args.no_twist and rank == 0:
        try:
            emp = _empirical_bench(stream)
        except Exception as exc:   # a secondary leg: report, do not lose the headline line
            emp = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(wl)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "electron moves/s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32" if prec == q.QMC_MIXED else "f64", "data": "synthetic",
               "config": {"workload": f"{args.workload}: N={N} H, r_s={wl.rs}, L={wl.L:.3f} bohr, "
                                      f"{G} s-Gaussians/proton, {W} walkers x {cfg.sweeps} sweeps "
                                      f"(+{cfg.warmup_cont} continuation), sample every sweep, "
                                      f"{'mixed' if prec == q.QMC_MIXED else 'FP64'} form, "
                                      f"FP64 Gauss-Jordan inverse recompute every {cfg.recompute_every} sweeps, "
                                      "adjoint forces, Langevin step with S = Cov(f)",
                          "walkers": W, "walkers_total": W * ws, "sweeps": cfg.sweeps,
                          "parallelism": f"walker shards x{ws} (two all-reduces per MD step)" if shard else "one GPU",
                          "force_evals_per_s": fevals,
                          "fp64_form_force_evals_per_s": fp64["force_evals_per_s"] if fp64 else None,
                          "fp64_form_electron_moves_per_s": fp64["value"] if fp64 else None,
                          "mixed_over_fp64_force_evals": fp64["mixed_over_fp64_force_evals"] if fp64 else None,
                          "rs_sweep_electron_moves_per_s": ({k: v["electron_moves_per_s"] for k, v in rs_rows.items()}
                                                            if rs_rows else None),
                          "l2": "inputs larger than L2 (walker state "
                                f"{q.footprint_bytes(cfg) / 1e9:.1f} GB per GPU)"},
               "force_evals_per_s": fevals,
               "clocks": clk,
               "e2e": {"value": e2e, "unit": "electron moves/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
               "gpu_launches": launches,
               "roofline": roof,
               "rooflines": roofs,
               "kernel_ms_per_step": breakdown,
               "fp64_form": fp64,
               "rs_sweep": rs_rows,
               "cpu_baseline": cpu,
               "serving": serving,
               "toy_langevin": toy,
               "jastrow34_fp64": j34,
               "twist_fp64": twl,
               "empirical_s_langevin": emp,
               "peaks": peak_kind,
               "result": {"E": res["E"], "E_err": res["E_err"], "accept": res["accept"], "Nc": res["Nc"]}}
        print(json.dumps(out), flush=True)
    if args.serve_requests <= 0:
        system.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = _args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.toy_only:
        run_toy_only(args, rank, local)
        return
    if args.trajectory > 0:
        run_trajectory(args, rank, local)
        return
    if args.jastrow34_only or args.twist_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        torch.cuda.set_device(local)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        if rank == 0:
            print(json.dumps(_jastrow34_bench(stream) if args.jastrow34_only else _twist_bench(stream)), flush=True)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
