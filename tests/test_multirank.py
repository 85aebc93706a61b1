"""The multi-rank bench path on CPU: two gloo ranks run independent replicas
(different seeds, no data-path collective) and agree on the max-over-ranks time."""
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
    wl = synth.workload("h16", seed=1002 + rank)     # per-rank replica, as bench.run_ours seeds it
    ms = 10.0 + 5.0 * rank
    t = torch.tensor([ms])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    out[rank] = (float(t.item()), float(wl.R.sum()), bench._dist())
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_independent_replicas_and_max_time():
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
    assert out[0][1] != out[1][1]                      # different synthetic replicas
    assert out[0][2] == (2, 0, 0) and out[1][2][:2] == (2, 1)
