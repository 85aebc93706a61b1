"""Seeded synthetic inputs: proton configurations, orbital coefficients and the
workload table for dense liquid hydrogen.

This module only *generates inputs*; it holds none of the method's arithmetic
(no basis functions, determinants, energies or forces).  Both the CUDA path and
the CPU oracle consume its output, which is why it lives on its own.

Workloads (synthetic stand-ins for the paper's 64/128-atom liquid-hydrogen
cells at r_s ~ 1.2-1.5, whose start files and optimised wavefunctions are not
available): protons uniform in the box with a 1.0 bohr minimum-image
separation, random orbital coefficients U(-1,1) with orthonormal columns.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

K_B_HARTREE_PER_KELVIN = 3.166811563e-6   # CODATA Boltzmann constant in Ha/K

# s-Gaussian exponents (bohr^-2).  Two per proton for the small cases; the four
# retained cc-pVDZ-derived exponents of the paper's basis (all used as s-type)
# for the four-Gaussian cases.
ZETA_2 = (0.5, 1.5)
ZETA_4 = (0.122, 0.4446, 0.727, 1.962)


def box_side(n_protons: int, rs: float) -> float:
    """L = (4 pi N / 3)^(1/3) r_s for a cubic cell of N hydrogen atoms."""
    return (4.0 * math.pi * n_protons / 3.0) ** (1.0 / 3.0) * rs


def protons(n_protons: int, L: float, seed: int, min_sep: float = 1.0, max_tries: int = 1_000_000) -> np.ndarray:
    """Uniform random protons in [0,L)^3 with minimum-image separation >= min_sep."""
    rng = np.random.default_rng(seed)
    R = np.zeros((n_protons, 3))
    placed = 0
    tries = 0
    while placed < n_protons:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place protons with the requested separation")
        c = rng.uniform(0.0, L, size=3)
        if placed:
            d = R[:placed] - c
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep * min_sep:
                continue
        R[placed] = c
        placed += 1
    return R


def coefficients(n_basis: int, n_orb: int, seed: int) -> np.ndarray:
    """Random U(-1,1) coefficients [n_basis, n_orb] with orthonormal columns."""
    rng = np.random.default_rng(seed + 7919)
    C = rng.uniform(-1.0, 1.0, size=(n_basis, n_orb))
    Q, Rm = np.linalg.qr(C)
    Q = Q * np.sign(np.diag(Rm))[None, :]
    return np.ascontiguousarray(Q)


@dataclass
class Workload:
    """One synthetic dense-hydrogen system plus its VMC / MD settings."""
    name: str
    N: int
    rs: float
    zeta: tuple
    walkers: int
    sweeps: int
    warmup: int = 20
    measure_every: int = 1
    recompute_every: int = 1      # full inverse recompute period, in sweeps
    sigma: float = 0.3
    T_kelvin: float = 1000.0
    delta: float = 0.1
    seed: int = 1000
    L: float = field(init=False)
    R: np.ndarray = field(init=False, repr=False)
    C: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        self.L = box_side(self.N, self.rs)
        self.R = protons(self.N, self.L, self.seed)
        self.C = coefficients(self.N * len(self.zeta), self.N // 2, self.seed)

    @property
    def n_gauss(self) -> int:
        return len(self.zeta)

    @property
    def kappa(self) -> float:
        return 5.0 / self.L

    @property
    def T_hartree(self) -> float:
        return self.T_kelvin * K_B_HARTREE_PER_KELVIN


def workload(name: str, **over) -> Workload:
    """Named workloads.

    * ``h16``  - N=16, r_s=1.4, 2 Gaussians/proton, 256 walkers x 200 sweeps, T=1000 K, Delta=0.1.
    * ``h64``  - N=64, r_s=1.4, 2 Gaussians/proton, 4096 walkers x 500 sweeps.
    * ``h128`` - N=128, r_s in {1.2,1.3,1.4,1.5}, 4 Gaussians/proton, 16384 walkers x 1000 sweeps,
                 T=1500 K (headline throughput point).
    * ``h512`` - N=512, r_s=1.3, 2 Gaussians/proton, 32768 walkers x 500 sweeps.
    """
    table = {
        "h16": dict(N=16, rs=1.4, zeta=ZETA_2, walkers=256, sweeps=200, T_kelvin=1000.0, delta=0.1, seed=1000),
        "h64": dict(N=64, rs=1.4, zeta=ZETA_2, walkers=4096, sweeps=500, seed=1001),
        "h128": dict(N=128, rs=1.2, zeta=ZETA_4, walkers=16384, sweeps=1000, T_kelvin=1500.0, seed=1002),
        "h512": dict(N=512, rs=1.3, zeta=ZETA_2, walkers=32768, sweeps=500, seed=1004),
    }
    kw = dict(table[name])
    kw.update(over)
    return Workload(name=name, **kw)


def monkhorst_pack(q: int, time_reversal: bool = False) -> np.ndarray:
    """Twist vectors theta [q^3, 3] of the q x q x q Monkhorst-Pack mesh of a
    cubic cell (the main text's k-point sampling; q = 4 for the 64-atom runs):
    theta_mu = 2 pi (2 r - q - 1) / (2 q), r = 1..q, i.e. k = theta / L.
    For even q no point is its own negative, and with time_reversal=True one
    twist of each pair (theta, -theta) is kept (q^3 / 2 of them: the first in
    mesh order), which gives the same equal-weight average because the spin
    twists are opposite: psi(-theta) is the complex conjugate of psi(theta)."""
    u = (2.0 * np.arange(1, q + 1) - q - 1) / (2.0 * q)
    g = np.stack(np.meshgrid(u, u, u, indexing="ij"), -1).reshape(-1, 3)
    if time_reversal:
        if q % 2:
            raise ValueError("the time-reversal halving needs an even mesh")
        keep, seen = [], set()
        for i, v in enumerate(g):
            key = tuple(np.round(v * 2 * q).astype(int))
            if tuple(-k for k in key) in seen:
                continue
            seen.add(key)
            keep.append(i)
        g = g[keep]
    return 2.0 * math.pi * g


def random_electrons(n_conf: int, n_elec: int, L: float, seed: int) -> np.ndarray:
    """Uniform electron configurations [n_conf, n_elec, 3] in the box (for parity inputs)."""
    rng = np.random.default_rng(seed + 104729)
    return rng.uniform(0.0, L, size=(n_conf, n_elec, 3))


def near_protons(n_conf: int, R: np.ndarray, n_up: int, spread: float, L: float, seed: int) -> np.ndarray:
    """Electron configurations [n_conf, N, 3] scattered around the protons (typical VMC samples)."""
    rng = np.random.default_rng(seed + 15485863)
    N = R.shape[0]
    n_dn = N - n_up
    sites = np.concatenate([np.arange(n_up), n_up + np.arange(n_dn)]) % N
    X = R[sites][None, :, :] + spread * rng.standard_normal((n_conf, N, 3))
    return np.mod(X, L)


# Rotating-spring toy model (SI, "A simple toy model"): the figure's parameters.
# lambda is the parameter of the printed G_lambda; the caption's "lambda = 10"
# is read as its reciprocal (radial step reduced tenfold), which is also what
# makes alpha = 0.2 equal to k lambda, i.e. H = alpha S along the radius.
TOY_K, TOY_A, TOY_T, TOY_LAMBDA, TOY_MU, TOY_ALPHA = 2.0, 1.4, 0.01, 0.1, 0.5, 0.2


def toy_starts(n_traj: int, seed: int, a: float = TOY_A, spread: float = 0.05) -> np.ndarray:
    """Start points [n_traj, 2] of toy-model trajectories: uniform polar angle,
    radius a + N(0, spread^2) (inside the thermal ring for the figure's T)."""
    rng = np.random.default_rng(seed + 7919)
    th = rng.uniform(0.0, 2.0 * math.pi, n_traj)
    r = a + spread * rng.standard_normal(n_traj)
    return np.stack([r * np.cos(th), r * np.sin(th)], 1)
