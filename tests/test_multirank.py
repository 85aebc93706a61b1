"""The multi-rank paths on CPU with gloo ranks: the bench's rank set-up (one
system on every rank, walkers split by offset, max-over-ranks time) and the
walker-sharded reduction's exchange."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_1605_08423_gb300 import synth
    import bench
    wl = synth.workload("h16", seed=1002)     # one system on every rank, as bench.run_ours builds it
    ms = 10.0 + 5.0 * rank
    t = torch.tensor([ms])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    out[rank] = (float(t.item()), float(wl.R.sum()), bench._dist(), rank * wl.walkers)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_one_system_walker_offsets_and_max_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == out[1][1]                      # the same nuclei on every rank
    assert out[0][3] == 0 and out[1][3] == 256         # rank r's walkers start at r W
    assert out[0][2] == (2, 0, 0) and out[1][2][:2] == (2, 1)


class _FakeShard:
    """Host stand-in for one process's QMCSystem in the walker-sharded
    reduction: its accumulator slice (from the oracle's chains) and the three
    shard_* steps written out in numpy, with the buffer layouts of
    include/qmcmd.h.  The CUDA kernels of these steps are checked against the
    single-handle reduction on the GPU (tests/test_gpu_shard.py); this checks
    the exchange around them with real gloo collectives."""

    def __init__(self, acc, N):
        self.acc, self.N = acc, N

    def shard_sample_device(self, R_dev, sums):
        import torch
        W = self.acc.shape[0]
        s = self.acc.sum(axis=0)
        sums.copy_(torch.tensor(list(s) + [0.0, float(W), 1.0], dtype=torch.float64))

    def shard_reduce_device(self, sums, out, gram):
        import numpy as np
        import torch
        N3 = 3 * self.N
        c = sums.numpy()
        cnt, E = c[0], c[1] / c[0]
        f = -c[3 + 2 * N3:3 + 3 * N3] / cnt - 2.0 * (c[3 + N3:3 + 2 * N3] / cnt - E * c[3:3 + N3] / cnt)
        a = self.acc
        fw = -a[:, 3 + 2 * N3:3 + 3 * N3] / a[:, :1] - 2.0 * (a[:, 3 + N3:3 + 2 * N3] / a[:, :1]
                                                             - E * a[:, 3:3 + N3] / a[:, :1])
        d = fw - f
        e = a[:, 1] / a[:, 0] - E
        o = out.numpy()
        o[0], o[2], o[4:4 + N3] = E, cnt, f
        gram.copy_(torch.tensor(np.concatenate([[np.sum(e * e)], (d.T @ d).ravel()])))

    def shard_finish_device(self, sums, gram, out, walkers_total):
        N3 = 3 * self.N
        W = float(sums.numpy()[3 + 9 * self.N + 1])
        assert W == walkers_total
        g = gram.numpy()
        o = out.numpy()
        o[1] = (g[0] / (W * (W - 1))) ** 0.5
        o[4 + N3:] = g[1:] / (W * (W - 1))


def _shard_worker(rank, ws, port, out):
    import numpy as np
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import oracle as orc
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth
    wl = synth.workload("h16")
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    _, acc, _ = orc.vmc(osys, wl.R, W=11, n_sweeps=3, n_warmup=2, sigma=wl.sigma, seed=wl.seed)
    sizes = q.shard_sizes(11, ws)
    lo = sum(sizes[:rank])
    grp = q.ShardGroup(_FakeShard(acc[lo:lo + sizes[rank]], wl.N), 11)
    o = torch.zeros(4 + 3 * wl.N + 9 * wl.N * wl.N, dtype=torch.float64)
    grp.energy_forces_device(torch.zeros(wl.N, 3, dtype=torch.float64), o)
    ref = orc.reduce(acc, wl.N)
    r = o.numpy()
    N3 = 3 * wl.N
    out[rank] = (abs(r[0] - ref["E"]) / abs(ref["E"]), abs(r[1] - ref["E_err"]) / ref["E_err"],
                 float(np.max(np.abs(r[4:4 + N3] - ref["f"])) / np.max(np.abs(ref["f"]))),
                 float(np.max(np.abs(r[4 + N3:].reshape(N3, N3) - ref["S"])) / np.max(np.abs(ref["S"]))),
                 sizes)
    dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_gloo_ranks_walker_sharded_reduction_equals_single_process():
    """11 walkers split 6 + 5 over two gloo ranks: the sharded E, E_err, f and S
    equal the oracle's reduction over all 11 walkers."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(150)
        assert p.exitcode == 0
    for r in range(2):
        eE, eErr, ef, eS, sizes = out[r]
        assert sizes == [6, 5]
        assert eE < 1e-13 and eErr < 1e-10 and ef < 1e-12 and eS < 1e-11, out[r]


class _FakeTwists:
    """Host stand-in for one process's twisted QMCSystem in a TwistGroup: its
    walkers' accumulators (the oracle's chains on its twists), its own twist
    average, and the partial / combine steps written out in numpy with the
    layouts of include/qmcmd.h (their CUDA kernels are checked against a
    single handle over all twists in tests/test_gpu_twist.py)."""

    def __init__(self, acc, N, K):
        self.acc, self.N, self.K = acc, N, K

    def energy_forces_device(self, R_dev, out):
        import numpy as np
        import torch
        from oracle import oracle as orc
        r = orc.reduce_twists(self.acc, self.N, self.K)
        out.copy_(torch.tensor(np.concatenate([[r["E"], r["E_err"], r["Nc"], 0.5], r["f"], r["S"].ravel()])))

    def twist_partial_device(self, out, part):
        N3, K = 3 * self.N, float(self.K)
        o, p = out.numpy(), part.numpy()
        p[0], p[1], p[2], p[3] = K * o[0], (K * o[1]) ** 2, o[2], K * o[3]
        p[4:4 + N3] = K * o[4:4 + N3]
        p[4 + N3:] = K * K * o[4 + N3:]

    def twist_combine_device(self, part, K_total, out):
        N3, K = 3 * self.N, float(K_total)
        o, p = out.numpy(), part.numpy()
        o[0], o[1], o[2], o[3] = p[0] / K, p[1] ** 0.5 / K, p[2], p[3] / K
        o[4:4 + N3] = p[4:4 + N3] / K
        o[4 + N3:] = p[4 + N3:] / (K * K)


def _twist_worker(rank, ws, port, out):
    import numpy as np
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import oracle as orc
    from paper_1605_08423_gb300 import qmcmd as q
    from paper_1605_08423_gb300 import synth
    wl = synth.workload("h16")
    tw = synth.monkhorst_pack(2)[:4]
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, twist=tw[0])
    _, acc, _, _ = orc.vmc_twists(osys, wl.R, tw, W=12, n_sweeps=2, n_warmup=1, sigma=wl.sigma, seed=wl.seed)
    mine = q.twist_slice(tw, rank, ws)
    per = 12 // 4
    lo = rank * len(mine) * per
    grp = q.TwistGroup(_FakeTwists(acc[lo:lo + len(mine) * per], wl.N, len(mine)), 4)
    o = torch.zeros(4 + 3 * wl.N + 9 * wl.N * wl.N, dtype=torch.float64)
    grp.energy_forces_device(torch.zeros(wl.N, 3, dtype=torch.float64), o)
    ref = orc.reduce_twists(acc, wl.N, 4)
    r = o.numpy()
    N3 = 3 * wl.N
    out[rank] = (abs(r[0] - ref["E"]) / abs(ref["E"]), abs(r[1] - ref["E_err"]) / ref["E_err"], r[2] - ref["Nc"],
                 float(np.max(np.abs(r[4:4 + N3] - ref["f"])) / np.max(np.abs(ref["f"]))),
                 float(np.max(np.abs(r[4 + N3:].reshape(N3, N3) - ref["S"])) / np.max(np.abs(ref["S"]))),
                 mine.tolist())
    dist.destroy_process_group()


@pytest.mark.timeout(240)
def test_two_gloo_ranks_twist_sharded_average_equals_single_process():
    """Four twists (three walkers each) split two per gloo rank: the combined
    E, E_err, N_c, f and S equal the oracle's twist average over all four."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_twist_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(200)
        assert p.exitcode == 0
    for r in range(2):
        eE, eErr, dNc, ef, eS, mine = out[r]
        assert len(mine) == 2
        assert eE < 1e-13 and eErr < 1e-12 and dNc == 0 and ef < 1e-12 and eS < 1e-12, out[r]
    assert out[0][5] != out[1][5]
