"""Walker sharding through the C ABI on one GPU: two handles holding the
walker slices [0, W1) and [W1, W) (walker offsets 0 and W1) run one after the
other, and the buffers the processes would all-reduce are summed here; the
result must equal one handle holding all W walkers (same Philox streams, so
the same chains: walker positions bit-identical, E, f, S up to the order of
the FP64 sums)."""
import numpy as np
import pytest

from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,W,W1,prec", [("h16", 24, 13, q.QMC_FP64), ("h64", 20, 12, q.QMC_MIXED)])
def test_two_shards_equal_one_handle(name, W, W1, prec):
    import torch
    wl = synth.workload(name, walkers=W, sweeps=3, warmup=2)
    N, N3 = wl.N, 3 * wl.N
    cfg = q.Config.from_workload(wl, precision=prec, warmup=2, warmup_cont=1, recompute_every=2)
    one = q.QMCSystem(cfg, wl.R)
    # the library's work and the sums below (torch) on one stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    st = stream.cuda_stream
    one.set_stream(st)
    R_dev = torch.tensor(wl.R, dtype=torch.float64, device="cuda")
    nout = 4 + N3 + N3 * N3
    shards = []
    for lo, hi in ((0, W1), (W1, W)):
        s = q.QMCSystem(q.Config.from_workload(wl, precision=prec, warmup=2, warmup_cont=1, recompute_every=2,
                                               walkers=hi - lo), wl.R)
        s.set_stream(st)
        s.set_walker_offset(lo)
        shards.append(s)
    ref_out = torch.zeros(nout, dtype=torch.float64, device="cuda")
    for step in range(2):                    # a first call and a continuation call
        one.energy_forces_device(R_dev, ref_out)
        one.sync()
        sums = [torch.zeros(3 + 9 * N + 3, dtype=torch.float64, device="cuda") for _ in shards]
        grams = [torch.zeros(1 + 9 * N * N, dtype=torch.float64, device="cuda") for _ in shards]
        outs = [torch.zeros(nout, dtype=torch.float64, device="cuda") for _ in shards]
        for s, sm in zip(shards, sums):
            s.shard_sample_device(R_dev, sm)
        tot = sums[0] + sums[1]                 # the first all-reduce
        for s, o, g in zip(shards, outs, grams):
            s.shard_reduce_device(tot, o, g)
        gtot = grams[0] + grams[1]              # the second all-reduce
        for s, o in zip(shards, outs):
            s.shard_finish_device(tot, gtot, o, W)
            s.sync()
        Xs = np.concatenate([s.walkers() for s in shards])
        assert np.array_equal(Xs, one.walkers()), step
        ref = q.unpack_out(ref_out.cpu().numpy(), N)
        for o in outs:
            got = q.unpack_out(o.cpu().numpy(), N)
            assert abs(got["E"] - ref["E"]) <= 1e-13 * abs(ref["E"])
            assert abs(got["E_err"] - ref["E_err"]) <= 1e-10 * ref["E_err"]
            assert got["Nc"] == ref["Nc"] and abs(got["accept"] - ref["accept"]) < 1e-15
            assert np.max(np.abs(got["f"] - ref["f"])) <= 1e-12 * np.max(np.abs(ref["f"]))
            assert np.max(np.abs(got["S"] - ref["S"])) <= 1e-11 * np.max(np.abs(ref["S"]))


def test_walker_offset_rejects_negative():
    wl = synth.workload("h16", walkers=4)
    s = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    with pytest.raises(q.QMCError) as e:
        s.set_walker_offset(-1)
    assert e.value.code == -1
