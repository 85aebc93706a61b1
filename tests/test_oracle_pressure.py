"""Pins of the oracle's virial pressure (the paper reports P against density
along isotherms without stating its estimator; the reading is the virial of
the Coulomb system, P = (2<T> + <V>)/(3 Omega) + N T/Omega).

The pins check what that reading rests on and what fixes its value:
  * the Ewald sum is homogeneous of degree -1 in all lengths (kappa L and the
    k cutoff in units of 2 pi / L fixed), exactly;
  * for the wavefunction scaled with the cell (every length parameter scaled)
    E_L of the scaled system at the scaled configuration is T_L / lambda^2 +
    V_L / lambda, configuration by configuration -- so (2<T> + <V>) is exactly
    -dE/d ln(lambda) of the variational energy;
  * closed forms: 2<T> + <V> = 3 zeta - 2 sqrt(2 zeta / pi) for the Gaussian
    hydrogen atom (zero at the variational optimum zeta = 8 / (9 pi)), and 0
    for the exact hydrogen atom (virial theorem of an eigenstate);
  * the nuclear ideal-gas term is added exactly.
"""
import math

import numpy as np

from oracle import oracle as orc
from paper_1605_08423_gb300 import synth


def _hydrogen(zeta=0.0, jastrow=True):
    return orc.System(N=1, L=10.0, zeta=np.array([zeta]), coeff=np.array([[1.0]]), n_up=1, n_dn=0,
                      b_ee=1.0, b_ep=0.0, Z=1.0, Zj=1.0 if jastrow else 0.0, periodic=False)


def test_ewald_is_homogeneous_of_degree_minus_one():
    wl = synth.workload("h16")
    rng = np.random.default_rng(2)
    pos = np.concatenate([wl.R, rng.uniform(0, wl.L, (wl.N, 3))])
    q = np.concatenate([np.ones(wl.N), -np.ones(wl.N)])
    kappa = 5.0 / wl.L
    e1 = orc.ewald(q, pos, wl.L, kappa, 6)
    for lam in (0.9, 1.1, 1.7):
        el = orc.ewald(q, lam * pos, lam * wl.L, kappa / lam, 6)
        assert abs(el - e1 / lam) < 1e-12 * abs(e1)


def test_scaled_wavefunction_local_energy_scales_as_virial():
    """h16 with the e-e Jastrow made negligible (b_ee = 1e9; its prefactor 1/2
    is not a scaled parameter): at lambda = 1.1 every length parameter of the
    system is scaled (L, R, zeta -> zeta / lambda^2, e-n Jastrow amplitude and
    b -> / lambda, kappa -> / lambda) and E_L(lambda X) = T_L / lambda^2 + V_L / lambda."""
    wl = synth.workload("h16")
    base = dict(N=wl.N, coeff=wl.C, b_ee=1e9, b_ep=1.0, Z=1.0, Zj=1.0)
    s1 = orc.System(L=wl.L, zeta=np.array(wl.zeta), kappa=5.0 / wl.L, **base)
    X = synth.near_protons(3, wl.R, wl.N // 2, 0.6, wl.L, 4)
    for lam in (1.1, 0.93):
        sl = orc.System(L=lam * wl.L, zeta=np.array(wl.zeta) / lam ** 2, kappa=5.0 / (lam * wl.L),
                        **{**base, "b_ee": 1e9 / lam, "b_ep": 1.0 / lam, "Zj": 1.0 / lam})
        for x in X:
            o1 = orc.eval_config(s1, wl.R, x)
            ol = orc.eval_config(sl, lam * wl.R, lam * x)
            assert abs(o1["ekin"] + o1["epot"] - o1["el"]) < 1e-10 * abs(o1["epot"])
            pred = o1["ekin"] / lam ** 2 + o1["epot"] / lam
            assert abs(ol["el"] - pred) < 1e-8 * (abs(o1["ekin"]) + abs(o1["epot"])), (lam, ol["el"], pred)


def test_gaussian_hydrogen_virial_closed_form():
    """psi = exp(-zeta r^2): <T> = 3 zeta / 2, <V> = -2 sqrt(2 zeta / pi); with
    Omega = 1/3 the electronic pressure is 2<T> + <V>."""
    for zeta, seed in ((0.5, 11), (8.0 / (9.0 * math.pi), 12)):
        sysH = _hydrogen(zeta=zeta, jastrow=False)
        R = np.zeros((1, 3))
        _, acc, _, vacc = orc.vmc(sysH, R, W=512, n_sweeps=400, n_warmup=50, sigma=1.0, seed=seed,
                                  X=np.zeros((512, 1, 3)), forces=False, potential=True)
        p = orc.pressure(acc, vacc, 1, 1.0 / 3.0)
        exact = 3.0 * zeta - 2.0 * math.sqrt(2.0 * zeta / math.pi)
        assert abs(p["P_el"] - exact) < 3.5 * p["P_err"], (zeta, p, exact)
        assert abs(p["V"] + 2.0 * math.sqrt(2.0 * zeta / math.pi)) < 0.05 * abs(p["V"])
        assert p["P_err"] > 0
    assert abs(3.0 * (8.0 / (9.0 * math.pi)) - 2.0 * math.sqrt(2.0 * (8.0 / (9.0 * math.pi)) / math.pi)) < 1e-15


def test_exact_hydrogen_virial_vanishes_and_ideal_gas_term():
    sysH = _hydrogen()
    R = np.zeros((1, 3))
    X0 = np.random.default_rng(5).normal(size=(512, 1, 3))     # off the nucleus, where V_L is singular
    _, acc, _, vacc = orc.vmc(sysH, R, W=512, n_sweeps=400, n_warmup=50, sigma=1.0, seed=13,
                              X=X0, forces=False, potential=True)
    p = orc.pressure(acc, vacc, 1, 1.0 / 3.0)
    assert abs(p["P_el"]) < 3.5 * p["P_err"], p
    assert abs(p["T"] - 0.5) < 0.05 and abs(p["V"] + 1.0) < 0.05
    pt = orc.pressure(acc, vacc, 1, 1.0 / 3.0, T_nuc=0.01)
    assert abs(pt["P"] - (p["P"] + 1 * 0.01 * 3.0)) < 1e-15
