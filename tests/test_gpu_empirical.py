"""Parity of the empirical acceleration matrix S = H + mu I (main text,
conclusions; H the Hessian of the screened-Coulomb proton pair potential) and
of the Langevin step that builds it on the device, against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu


def _tf_length(N, L):
    kF = (3 * math.pi ** 2 * N / L ** 3) ** (1 / 3)
    return 1 / math.sqrt(4 * kF / math.pi)


@pytest.mark.parametrize("name,lam,mu", [("h16", 0.7, 0.25), ("h16", None, 0.5)])
def test_empirical_s_matches_oracle(name, lam, mu):
    wl = synth.workload(name, walkers=2)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    if lam is not None:
        sysg.set_empirical_s(lam, mu)
    else:
        lam = _tf_length(wl.N, wl.L)        # the handle's default: Thomas-Fermi length, mu = 0.5
    Sg = sysg.empirical_s(wl.R)
    So = orc.empirical_s(wl.R, wl.L, lam, mu)
    assert np.max(np.abs(Sg - So)) < 1e-12 * np.max(np.abs(So))


def test_empirical_s_small_box_images():
    """Eight protons in a small box: pairs with several images inside one box side."""
    L = synth.box_side(8, 1.0)
    R = synth.protons(8, L, 21, min_sep=0.8)
    wl = synth.workload("h16", walkers=2)
    cfg = q.Config.from_workload(wl)
    cfg.N, cfg.L = 8, L
    cfg.coeff = synth.coefficients(8 * len(wl.zeta), 4, 21)
    sysg = q.QMCSystem(cfg, R)
    sysg.set_empirical_s(0.9, 0.05)
    So = orc.empirical_s(R, L, 0.9, 0.05)
    assert np.max(np.abs(sysg.empirical_s(R) - So)) < 1e-12 * np.max(np.abs(So))


@pytest.mark.parametrize("alpha", [0.0, 3.0])
def test_langevin_step_with_empirical_s_matches_oracle(alpha):
    """Three steps with S = H(R) + mu I rebuilt on the device each step and the
    two-time term from the previous step's S, against the oracle step fed the
    oracle's S at the same positions."""
    wl = synth.workload("h16", walkers=2)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    lam, mu = 0.7, 0.5      # H's lowest eigenvalue here is -0.35
    sysg.set_empirical_s(lam, mu)
    n = 3 * wl.N
    rng = np.random.default_rng(9)
    T_K, delta = 1500.0, 0.05
    T = T_K * synth.K_B_HARTREE_PER_KELVIN
    R = wl.R.ravel().copy()
    Rprev, Sprev = R.copy(), None
    for step in range(3):
        f = 0.05 * rng.standard_normal(n)
        S = orc.empirical_s(R, wl.L, lam, mu)
        if Sprev is None:
            Sprev = S
        xi = orc.langevin_noise(wl.seed, step, n)
        Ro = orc.langevin(R, Rprev, f, S, Sprev, T, delta, alpha, xi, box=wl.L)
        Rg = sysg.langevin_step(R, f, None, T_K, delta, s_mode=q.QMC_S_EMPIRICAL, alpha=alpha)
        assert np.max(np.abs(Rg - Ro)) < 1e-10, (step, np.max(np.abs(Rg - Ro)))
        Rprev, Sprev, R = R, S, Ro


def test_empirical_s_arguments_validated():
    wl = synth.workload("h16", walkers=2)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    with pytest.raises(q.QMCError):
        sysg.set_empirical_s(0.7, -0.1)
    with pytest.raises(q.QMCError):
        sysg.set_empirical_s(float("nan"), 0.1)
    with pytest.raises(q.QMCError):
        sysg.langevin_step(wl.R.ravel(), np.zeros(3 * wl.N), None, 1000.0, 0.1, s_mode=q.QMC_S_EMPIRICAL,
                           alpha=-1.0)
