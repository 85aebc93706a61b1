"""The allocation-free Langevin step (qmc_langevin_step_static) against the
regular entry point (langevin_step), through the C ABI.

Some callers cannot call cudaMalloc (it may synchronise the device, or the
host owns all device memory); qmc_langevin_step_static serves them with a
static device workspace.  This file is collected last on purpose, and must
pass both on its own in a fresh process and after every other test.
"""
import numpy as np
import pytest

from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T / n + 0.3 * np.eye(n)


@pytest.mark.parametrize("mode", [q.QMC_S_COV, q.QMC_S_IDENTITY])
def test_static_langevin_matches_regular_entry_point(mode):
    import torch
    wl = synth.workload("h16", walkers=2)
    system = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    n = 3 * wl.N
    rng = np.random.default_rng(12)
    alpha = 41.0 if mode == q.QMC_S_COV else 0.0
    R = wl.R.ravel().copy()
    Rprev, Sprev = R.copy(), None
    dev = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    for step in range(2):                       # two calls in a row
        f = rng.standard_normal(n)
        S = _spd(n, 30 + step) * 1e-3 if mode == q.QMC_S_COV else np.eye(n)
        if Sprev is None:
            Sprev = S
        ref = system.langevin_step(R, f, S if mode == q.QMC_S_COV else None, 1500.0, 0.1, s_mode=mode, alpha=alpha)
        R_dev = dev(R)
        q.langevin_step_static(R_dev, dev(Rprev), dev(f), dev(S), dev(Sprev), 1500.0, 0.1, mode, alpha,
                               wl.seed, step, wl.L)
        got = R_dev.cpu().numpy()
        assert np.max(np.abs(got - ref)) < 1e-10, (step, np.max(np.abs(got - ref)))
        Rprev, Sprev, R = R, S, ref


def test_static_langevin_rejects_oversize_and_non_pd():
    import torch
    n = q.lib().qmc_langevin_step_static  # exported
    big = 400
    t = torch.zeros(big, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QMCError) as e:
        q.langevin_step_static(t, t, t, None, None, 1000.0, 0.1, q.QMC_S_IDENTITY, 0.0, 1, 0, 0.0)
    assert e.value.code == -1
    m = 6
    R = torch.zeros(m, dtype=torch.float64, device="cuda")
    S = -torch.eye(m, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QMCError) as e:
        q.langevin_step_static(R, R, R, S, S, 1000.0, 0.1, q.QMC_S_COV, 1.0, 1, 0, 0.0)
    assert e.value.code == -4
    assert n is not None
