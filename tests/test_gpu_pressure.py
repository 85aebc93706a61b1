"""The virial pressure through the C ABI against the oracle's on the same
chains (FP64 form: the GPU chain reproduces the oracle's on the same Philox
streams), and the mixed form within its error bars."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu


def test_pressure_matches_oracle_on_the_same_chain():
    wl = synth.workload("h16", walkers=16, sweeps=3, warmup=2)
    s = q.QMCSystem(q.Config.from_workload(wl, recompute_every=1), wl.R)
    s.energy_forces(wl.R)
    g = s.pressure(1500.0)
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    _, acc, _, vacc = orc.vmc(osys, wl.R, W=16, n_sweeps=3, n_warmup=2, sigma=wl.sigma, seed=wl.seed, potential=True)
    o = orc.pressure(acc, vacc, wl.N, wl.L ** 3, T_nuc=1500.0 * synth.K_B_HARTREE_PER_KELVIN)
    for k in ("P", "P_el", "V", "T"):
        assert abs(g[k] - o[k]) <= 1e-10 * abs(o[k]), (k, g[k], o[k])
    assert abs(g["P_err"] - o["P_err"]) <= 1e-8 * o["P_err"]
    import torch
    d = torch.zeros(5, dtype=torch.float64, device="cuda")
    s.pressure_device(1500.0, d)
    s.sync()
    assert np.allclose(d.cpu().numpy(), [g["P"], g["P_err"], g["P_el"], g["V"], g["T"]], rtol=0, atol=0)


def test_mixed_pressure_within_error_bars_of_fp64():
    wl = synth.workload("h16", walkers=256, sweeps=120, warmup=30)
    out = {}
    for prec in (q.QMC_FP64, q.QMC_MIXED):
        s = q.QMCSystem(q.Config.from_workload(wl, precision=prec), wl.R)
        s.energy_forces(wl.R)
        out[prec] = s.pressure(0.0)
    a, b = out[q.QMC_FP64], out[q.QMC_MIXED]
    assert abs(a["P"] - b["P"]) < 3 * np.hypot(a["P_err"], b["P_err"]), (a, b)
    assert a["P_err"] > 0 and b["P_err"] > 0
