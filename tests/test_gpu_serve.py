"""Served form: results are the same alone, in the mix and after evictions;
admission respects the memory budget; checkpoints restore bit-identically."""
import numpy as np
import pytest

from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu


def _traj(k, N, W, prec=q.QMC_MIXED):
    zeta = synth.ZETA_2
    wl = synth.Workload(name=f"t{k}", N=N, rs=1.2 + 0.05 * k, zeta=zeta, walkers=W, sweeps=2, warmup=2,
                        seed=300 + k)
    cfg = q.Config.from_workload(wl, precision=prec, warmup=2, warmup_cont=1, recompute_every=2)
    return cfg, wl.R, 800.0 + 300.0 * k


def _run(server, tids, steps, order):
    """Submit `steps` MD steps per trajectory in the given interleaving and drive to completion."""
    tickets = []
    for k in order:
        tickets.append((server.submit(tids[k]), k))
    out = {}
    while len(out) < len(tickets):
        server.progress()
        for t, k in tickets:
            if t in out:
                continue
            r = server.fetch(t, tids[k])
            if r is not None:
                out[t] = (k, r)
    per = {}
    for t, k in tickets:
        per.setdefault(k, []).append(out[t][1])
    return per


def _same(a, b):
    for x, y in zip(a, b):
        assert x["status"] == 0 and y["status"] == 0
        assert abs(x["E"] - y["E"]) <= 1e-12 * abs(x["E"])
        assert np.array_equal(x["f"], y["f"]) or np.max(np.abs(x["f"] - y["f"])) <= 1e-12 * np.max(np.abs(x["f"]))
        assert np.max(np.abs(x["S"] - y["S"])) <= 1e-12 * np.max(np.abs(x["S"]))
        assert np.max(np.abs(x["R_next"] - y["R_next"])) <= 1e-12


def test_result_same_alone_and_in_the_mix():
    trajs = [_traj(0, 16, 512), _traj(1, 32, 256), _traj(2, 16, 768), _traj(3, 32, 512), _traj(4, 16, 256)]
    big = 1 << 36
    alone = q.Server(big, 1)
    t0 = alone.add_trajectory(*trajs[0][:2], trajs[0][2], 0.1)
    res_alone = _run(alone, [t0], 3, [0, 0, 0])[0]
    alone.close()
    mix = q.Server(big, 3)
    tids = [mix.add_trajectory(c, R, T, 0.1) for c, R, T in trajs]
    order = [0, 1, 2, 3, 4, 0, 3, 1, 0, 2, 4, 1]
    res_mix = _run(mix, tids, 3, order)
    assert mix.stats()["completed"] == len(order)
    mix.close()
    _same(res_alone, res_mix[0])


def test_admission_by_memory_budget_with_eviction():
    trajs = [_traj(0, 16, 512), _traj(1, 32, 512), _traj(2, 16, 512), _traj(3, 32, 512)]
    fps = [q.footprint_bytes(c) for c, _, _ in trajs]
    budget = int(2.2 * max(fps))
    tight = q.Server(budget, 4)
    tids = [tight.add_trajectory(c, R, T, 0.1) for c, R, T in trajs]
    order = [0, 1, 2, 3, 0, 1, 2, 3, 3, 2, 1, 0]
    tickets = [(tight.submit(tids[k]), k) for k in order]
    out = {}
    max_used = 0
    while len(out) < len(tickets):
        tight.progress()
        st = tight.stats()
        max_used = max(max_used, st["resident_bytes"])
        assert st["resident_bytes"] <= budget
        for t, k in tickets:
            if t not in out:
                r = tight.fetch(t, tids[k])
                if r is not None:
                    out[t] = r
    st = tight.stats()
    assert st["evictions"] > 0 and max_used <= budget
    tight.close()
    loose = q.Server(1 << 36, 4)
    tids2 = [loose.add_trajectory(c, R, T, 0.1) for c, R, T in trajs]
    ref = _run(loose, tids2, 3, order)
    loose.close()
    got = {}
    for t, k in tickets:
        got.setdefault(k, []).append(out[t])
    for k in range(4):
        _same(got[k], ref[k])


def test_checkpoint_restores_bit_identically():
    cfg, R, T = _traj(0, 16, 256, prec=q.QMC_FP64)
    a = q.QMCSystem(cfg, R)
    for _ in range(2):
        r = a.energy_forces(R)
        R2 = a.langevin_step(R, r["f"], r["S"], T, 0.1).reshape(-1, 3)
    blob = a.checkpoint()
    b = q.QMCSystem(cfg, R)
    b.restore(blob)
    ra, rb = a.energy_forces(R2), b.energy_forces(R2)
    assert ra["E"] == rb["E"] and np.array_equal(ra["f"], rb["f"]) and np.array_equal(ra["S"], rb["S"])
    Ra = a.langevin_step(R2, ra["f"], ra["S"], T, 0.1)
    Rb = b.langevin_step(R2, rb["f"], rb["S"], T, 0.1)
    assert np.array_equal(Ra, Rb)
    bad = bytearray(blob)
    bad[0] ^= 1
    with pytest.raises(q.QMCError):
        b.restore(bytes(bad))


def test_served_poisson_loop_reports_latency():
    from paper_1605_08423_gb300 import serve
    trajs = serve.served_trajectories(n_traj=6, seed=3, sizes=(16, 32), walkers=(256, 768), sweeps=2)
    srv = q.Server(1 << 36, 4)
    tids = [srv.add_trajectory(t.cfg, t.R, t.T_kelvin, t.delta) for t in trajs]
    res, wall = serve.run_poisson(srv, tids, trajs, n_requests=30, mean_ms=2.0, seed=5)
    s = serve.summarize(res, wall)
    srv.close()
    assert s["requests"] == 30 and s["failed"] == 0
    assert 0 < s["p50_ms"] <= s["p99_ms"] and s["force_evals_per_s"] > 0


def test_requests_overlap_on_the_device():
    """Continuous batching, not a queue: requests of different trajectories
    admitted together run at the same time on the GPU (their start-to-end
    event intervals on their streams intersect)."""
    trajs = [_traj(k, 32, 1024) for k in range(4)]
    srv = q.Server(1 << 34, 4)
    tids = [srv.add_trajectory(c, R, T, 0.1) for c, R, T in trajs]
    res = _run(srv, tids, 1, [0, 1, 2, 3, 0, 1, 2, 3])
    srv.close()
    iv = [(r["gpu_start_ms"], r["gpu_end_ms"]) for k in res for r in res[k]]
    assert all(0 <= a < b for a, b in iv), iv
    pairs = [(i, j) for i in range(len(iv)) for j in range(i + 1, len(iv))
             if max(iv[i][0], iv[j][0]) < min(iv[i][1], iv[j][1])]
    assert pairs, iv


def test_no_device_allocation_while_serving():
    """The budget is one arena taken at creation: admissions (also after
    evictions under a tight budget) allocate no device memory."""
    import torch
    trajs = [_traj(0, 16, 512), _traj(1, 32, 512), _traj(2, 16, 512), _traj(3, 32, 512)]
    budget = int(2.2 * max(q.footprint_bytes(c) for c, _, _ in trajs))
    srv = q.Server(budget, 2)
    tids = [srv.add_trajectory(c, R, T, 0.1) for c, R, T in trajs]
    _run(srv, tids, 1, [0, 1, 2, 3])            # every kernel loaded once
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ev0 = srv.stats()["evictions"]
    _run(srv, tids, 2, [3, 2, 1, 0, 0, 1, 2, 3])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    st = srv.stats()
    srv.close()
    assert st["evictions"] > ev0 and st["admissions"] > 4
    assert free1 == free0, (free0, free1)


def test_twisted_trajectory_served_alone_and_in_the_mix():
    """A twisted FP64 trajectory (four twists, two walkers each, conventional
    S = I steps: two walkers per twist give no full-rank covariance) gives the
    same steps alone and among Gamma-point trajectories, and its first step's
    energy is that of a standalone handle with the same parameters."""
    wl = synth.workload("h16", walkers=8, sweeps=2, warmup=2)
    tw = synth.monkhorst_pack(4)[[6, 25, 40, 59]]
    cfg = q.Config.from_workload(wl, precision=q.QMC_FP64, warmup=2, warmup_cont=1, recompute_every=2, twists=tw)
    big = 1 << 36
    alone = q.Server(big, 1)
    t0 = alone.add_trajectory(cfg, wl.R, 1000.0, 0.1, s_mode=q.QMC_S_IDENTITY)
    res_alone = _run(alone, [t0], 2, [0, 0])[0]
    alone.close()
    others = [_traj(1, 16, 64, q.QMC_FP64), _traj(2, 16, 96, q.QMC_FP64)]
    mix = q.Server(big, 2)
    tids = [mix.add_trajectory(cfg, wl.R, 1000.0, 0.1, s_mode=q.QMC_S_IDENTITY)]
    tids += [mix.add_trajectory(c, R, T, 0.1) for c, R, T in others]
    res_mix = _run(mix, tids, 2, [0, 1, 2, 0, 1])
    mix.close()
    _same(res_alone, res_mix[0])
    ref = q.QMCSystem(cfg, wl.R).energy_forces(wl.R)
    assert abs(res_alone[0]["E"] - ref["E"]) <= 1e-12 * abs(ref["E"])
