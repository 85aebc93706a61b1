"""Parity of the CUDA toy-model integrators (qmc_toy_langevin, through the C ABI)
with the oracle's rotating-spring model (SI, "A simple toy model"): every scheme
and both acceleration matrices, element by element on the same Philox streams,
at a size that spans several CTAs and a ragged tail, and on sampled trajectories
of the full-size run that bench.py times."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu

# FP64 on both sides; differences are rounding-order only (fma contraction,
# closed-form versus dual-number derivatives) and stay at a few ulp per step.
TOL = 1e-9


def _both(scheme, s_mode, mu, n_traj, n_steps, n_burn, delta, seed=3, **kw):
    xy0 = synth.toy_starts(n_traj, seed)
    pg = q.toy_params(scheme, s_mode, mu=mu, delta=delta, n_steps=n_steps, n_burn=n_burn, seed=seed, **kw)
    po = orc.toy_args(scheme, s_mode, mu=mu, delta=delta, n_steps=n_steps, n_burn=n_burn, seed=seed, **kw)
    return q.toy_langevin(pg, xy0), orc.toy_run(po, xy0)


def _close(g, o):
    assert np.array_equal(g[:, 6], o[:, 6])
    scale = np.maximum(np.abs(o), 1.0)
    err = np.abs(g[:, :6] - o[:, :6]) / scale[:, :6]
    assert err.max() < TOL, err.max()


@pytest.mark.parametrize("scheme", list(q.TOY_SCHEMES.values()))
@pytest.mark.parametrize("s_mode,mu", [(q.QMC_TOY_S_G, 0.5), (q.QMC_TOY_S_HG, 2.0)])
def test_toy_schemes_match_oracle(scheme, s_mode, mu):
    g, o = _both(scheme, s_mode, mu, n_traj=600, n_steps=500, n_burn=100, delta=0.1)
    _close(g, o)


def test_toy_indefinite_S_status_matches_oracle():
    xy0 = synth.toy_starts(300, 5)
    xy0[::7] *= 1.0 / 1.4        # radius 1.0 < k a / (k + mu) = 1.12: S indefinite at once
    pg = q.toy_params(q.QMC_TOY_ADOPTED, q.QMC_TOY_S_HG, mu=0.5, delta=0.2, n_steps=3000, n_burn=0, seed=5)
    po = orc.toy_args(q.QMC_TOY_ADOPTED, q.QMC_TOY_S_HG, mu=0.5, delta=0.2, n_steps=3000, n_burn=0, seed=5)
    with pytest.raises(q.QMCError) as e:
        q.toy_langevin(pg, xy0)
    assert e.value.code == -4
    g = e.value.out
    o = orc.toy_run(po, xy0)
    assert np.all(g[::7, 6] == 1.0)
    _close(g, o)


def test_toy_device_api_and_edge_cases():
    import torch
    xy0 = synth.toy_starts(257, 9)
    p = q.toy_params(q.QMC_TOY_FIRST, q.QMC_TOY_S_G, delta=0.3, n_steps=200, n_burn=200, seed=9)
    dev_in = torch.tensor(xy0, device="cuda")
    dev_out = torch.empty((257, q.QMC_TOY_NOUT), dtype=torch.float64, device="cuda")
    q.toy_langevin_device(p, dev_in, dev_out)
    torch.cuda.synchronize()
    host = q.toy_langevin(p, xy0)
    assert np.array_equal(dev_out.cpu().numpy(), host)
    assert np.all(host[:, 2:5] == 0.0)                      # n_burn = n_steps: nothing summed
    assert q.toy_langevin(p, np.zeros((0, 2))).shape == (0, q.QMC_TOY_NOUT)
    p0 = q.toy_params(q.QMC_TOY_ADOPTED, q.QMC_TOY_S_G, n_steps=0, seed=9)
    assert np.array_equal(q.toy_langevin(p0, xy0)[:, :2], xy0)
    for bad in (dict(delta=0.0), dict(lam=-1.0), dict(T=-1.0), dict(n_steps=5, n_burn=6)):
        with pytest.raises(q.QMCError) as e:
            q.toy_langevin(q.toy_params(**bad), xy0)
        assert e.value.code == -1
    with pytest.raises(q.QMCError):
        q.toy_langevin(q.toy_params(scheme=9), xy0)


def test_toy_full_size_sampled_trajectories():
    """The bench configuration (adopted scheme, S = G_lambda): sampled trajectories
    of the full launch against the oracle run on those trajectories alone."""
    import bench
    cfg = bench.TOY_BENCH
    n, steps = cfg["n_traj"], cfg["n_steps"]
    xy0 = synth.toy_starts(n, cfg["seed"])
    p = q.toy_params(q.QMC_TOY_ADOPTED, q.QMC_TOY_S_G, delta=cfg["delta"], n_steps=steps, n_burn=cfg["n_burn"],
                     seed=cfg["seed"])
    g = q.toy_langevin(p, xy0)
    ids = np.unique(np.concatenate([[0, 1, n - 1], np.random.default_rng(1).integers(0, n, 13)]))
    po = orc.toy_args(q.QMC_TOY_ADOPTED, q.QMC_TOY_S_G, delta=cfg["delta"], n_steps=steps, n_burn=cfg["n_burn"],
                      seed=cfg["seed"])
    o = orc.toy_run_ids(po, ids, xy0[ids])
    _close(g[ids], o)
    # and the whole launch samples the canonical <U> = T/2 (SI: the adopted scheme has no time-step error here)
    mU = g[:, 2].sum() / (n * (steps - cfg["n_burn"]))
    assert abs(mU - synth.TOY_T / 2) < 0.01 * synth.TOY_T / 2, mU
