"""Pins of the FP64 CPU oracle against things the paper and physics fix
(closed forms, textbook constants, finite differences, invariances, brute force).

None of these call the CUDA library; they make sure the oracle itself is right
before it is used as the parity reference.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    for row in _golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        assert orc.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_and_normal_moments():
    L = orc.lib()
    n = 40000
    u = np.array([L.orc_uniform(7, i, 3, 5, 3) for i in range(n)])
    z = np.array([L.orc_normal(7, i, 3, 5, 0) for i in range(n)])
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3 * math.sqrt(1 / 12 / n)
    assert abs(z.mean()) < 3 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 3 * math.sqrt(2 / n)
    # a different purpose word gives an independent stream
    z2 = np.array([L.orc_normal(7, i, 3, 5, 1) for i in range(n)])
    assert abs(np.corrcoef(z, z2)[0, 1]) < 4 / math.sqrt(n)


# ---------------------------------------------------------------- Ewald
def _nacl(L):
    d = L / 2
    q, pos = [], []
    for i in range(2):
        for j in range(2):
            for k in range(2):
                q.append((-1.0) ** (i + j + k))
                pos.append([i * d + 0.3, j * d + 0.1, k * d + 0.7])
    return np.array(q), np.array(pos), d


@pytest.mark.parametrize("kappa_L,mmax,tol", [(5.0, 6, 2e-6), (6.0, 10, 1e-10)])
def test_ewald_nacl_madelung(kappa_L, mmax, tol):
    M = float(_golden("madelung.txt")[0][1])
    L = 5.3
    q, pos, d = _nacl(L)
    E = orc.ewald(q, pos, L, kappa_L / L, mmax)
    exact = -4.0 * M / d            # 8 ions = 4 ion pairs
    assert abs(E - exact) < tol * abs(exact)


def test_ewald_simple_cubic_background():
    xi = float(_golden("madelung.txt")[1][1])
    L = 3.7
    E = orc.ewald(np.array([1.0]), np.array([[0.2, 0.4, 0.9]]), L, 6.0 / L, 10, background=True)
    assert abs(E - (-xi / (2 * L))) < 1e-8


def test_ewald_kappa_and_translation_invariance():
    rng = np.random.default_rng(3)
    L = 6.0
    q = np.array([1, 1, 1, -1, -1, -1, 1, -1], float)
    pos = rng.uniform(0, L, size=(8, 3))
    E5 = orc.ewald(q, pos, L, 5.0 / L, 6)
    E7 = orc.ewald(q, pos, L, 7.0 / L, 14)
    assert abs(E5 - E7) < 1e-6 * abs(E7)
    shifted = pos + np.array([0.37, -1.1, 2.9])
    assert abs(orc.ewald(q, shifted, L, 5.0 / L, 6) - E5) < 1e-11 * abs(E5) + 1e-12
    wrapped = pos.copy()
    wrapped[2, 1] += L
    assert abs(orc.ewald(q, wrapped, L, 5.0 / L, 6) - E5) < 1e-11 * abs(E5) + 1e-12


# ---------------------------------------------------------------- wavefunction
def _hydrogen(zeta=0.0, jastrow=True):
    return orc.System(N=1, L=10.0, zeta=np.array([zeta]), coeff=np.array([[1.0]]), n_up=1, n_dn=0,
                      b_ee=1.0, b_ep=0.0, Z=1.0, Zj=1.0 if jastrow else 0.0, periodic=False)


def test_hydrogen_exact_zero_variance():
    """psi = exp(-r) (constant orbital, u_ep = -r): E_L = -1/2 for every X, forces vanish."""
    sysH = _hydrogen()
    R = np.array([[0.3, -0.2, 0.5]])
    rng = np.random.default_rng(0)
    for _ in range(10):
        X = R + rng.normal(scale=1.5, size=(1, 3))
        o = orc.eval_config(sysH, R, X, derivs=True)
        assert abs(o["el"] + 0.5) < 1e-12
        assert np.allclose(o["del_"], 0.0, atol=1e-12)
        # translation: d lnpsi / dR = -grad_r lnpsi
        assert np.allclose(o["dlnpsi"], -o["grad"], atol=1e-12)


def test_hydrogen_gaussian_vmc_closed_form():
    """psi = exp(-zeta r^2) (no Jastrow): E = 3 zeta / 2 - 2 sqrt(2 zeta / pi) exactly."""
    zeta = 0.5
    sysH = _hydrogen(zeta=zeta, jastrow=False)
    R = np.array([[0.0, 0.0, 0.0]])
    X0 = np.zeros((512, 1, 3))
    X, acc, ar = orc.vmc(sysH, R, W=512, n_sweeps=400, n_warmup=50, sigma=1.0, seed=11, X=X0, forces=False)
    r = orc.reduce(acc, 1)
    exact = 1.5 * zeta - 2.0 * math.sqrt(2.0 * zeta / math.pi)
    assert 0.2 < ar < 0.9
    assert abs(r["E"] - exact) < 3.5 * r["E_err"], (r["E"], exact, r["E_err"])
    assert r["E"] > -0.5   # variational bound of the hydrogen atom


def _h16(seed_conf=0):
    wl = synth.workload("h16")
    sysP = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    X = synth.near_protons(1, wl.R, wl.N // 2, 0.6, wl.L, seed_conf)[0]
    return wl, sysP, X


def test_grad_and_kinetic_vs_finite_differences():
    wl, sysP, X = _h16()
    o = orc.eval_config(sysP, wl.R, X)
    h = 1e-4
    grad_fd = np.zeros_like(X)
    lap_fd = 0.0
    for i in range(X.shape[0]):
        for mu in range(3):
            Xp = X.copy(); Xp[i, mu] += h
            Xm = X.copy(); Xm[i, mu] -= h
            lp = orc.eval_config(sysP, wl.R, Xp)["lnpsi"]
            lm = orc.eval_config(sysP, wl.R, Xm)["lnpsi"]
            grad_fd[i, mu] = (lp - lm) / (2 * h)
            lap_fd += (lp + lm - 2 * o["lnpsi"]) / h ** 2
    assert np.allclose(o["grad"], grad_fd, atol=2e-6, rtol=2e-6)
    ekin_fd = -0.5 * (lap_fd + np.sum(grad_fd ** 2))
    assert abs(o["ekin"] - ekin_fd) < 1e-5 * abs(o["ekin"]) + 1e-5


def test_R_derivatives_vs_finite_differences():
    wl, sysP, X = _h16(1)
    o = orc.eval_config(sysP, wl.R, X, derivs=True)
    h = 1e-4
    for a in (0, 5, 13):
        for mu in range(3):
            Rp = wl.R.copy(); Rp[a, mu] += h
            Rm = wl.R.copy(); Rm[a, mu] -= h
            op = orc.eval_config(sysP, Rp, X)
            om = orc.eval_config(sysP, Rm, X)
            d_l = (op["lnpsi"] - om["lnpsi"]) / (2 * h)
            d_e = (op["el"] - om["el"]) / (2 * h)
            assert abs(o["dlnpsi"][a, mu] - d_l) < 1e-6 * (1 + abs(d_l))
            assert abs(o["del_"][a, mu] - d_e) < 1e-6 * (1 + abs(d_e))


def test_translation_periodicity_and_antisymmetry():
    wl, sysP, X = _h16(2)
    o = orc.eval_config(sysP, wl.R, X, derivs=True)
    # sum over nuclei of d/dR + sum over electrons of d/dr vanishes for ln psi
    assert np.allclose(o["dlnpsi"].sum(0) + o["grad"].sum(0), 0.0, atol=1e-9)
    t = np.array([0.31, -0.77, 1.9])
    o2 = orc.eval_config(sysP, wl.R + t, X + t)
    assert abs(o2["lnpsi"] - o["lnpsi"]) < 1e-10 * abs(o["lnpsi"]) + 1e-10
    assert abs(o2["el"] - o["el"]) < 1e-10 * abs(o["el"])
    # moving one electron by a lattice vector changes nothing
    Xw = X.copy(); Xw[3, 2] += wl.L; Xw[9, 0] -= wl.L
    o3 = orc.eval_config(sysP, wl.R, Xw)
    assert abs(o3["lnpsi"] - o["lnpsi"]) < 1e-10 * abs(o["lnpsi"])
    assert abs(o3["el"] - o["el"]) < 1e-10 * abs(o["el"])
    # exchanging two same-spin electrons flips the sign only
    Xs = X.copy(); Xs[[1, 4]] = Xs[[4, 1]]
    o4 = orc.eval_config(sysP, wl.R, Xs)
    assert o4["sign"] == -o["sign"]
    assert abs(o4["lnpsi"] - o["lnpsi"]) < 1e-10 * abs(o["lnpsi"])
    assert abs(o4["el"] - o["el"]) < 1e-10 * abs(o["el"])


def test_coefficient_mixing_invariance():
    """C -> C M changes ln|psi| by ln|det M| per spin and nothing physical."""
    wl, sysP, X = _h16(3)
    n = wl.N // 2
    M = np.eye(n) + 0.3 * np.random.default_rng(5).standard_normal((n, n))
    sysM = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C @ M)
    o = orc.eval_config(sysP, wl.R, X, derivs=True)
    om = orc.eval_config(sysM, wl.R, X, derivs=True)
    ldm = np.linalg.slogdet(M)[1]
    assert abs(om["lnpsi"] - o["lnpsi"] - 2 * ldm) < 1e-9
    assert abs(om["el"] - o["el"]) < 1e-9 * abs(o["el"])
    assert np.allclose(om["del_"], o["del_"], atol=1e-8)
    assert np.allclose(om["dlnpsi"], o["dlnpsi"], atol=1e-8)


@pytest.mark.parametrize("kind", ["ee", "ep"])
def test_cusps_keep_local_energy_finite(kind):
    """Kato cusps: the Pade terms cancel the 1/r Coulomb singularities."""
    wl, sysP, X = _h16(4)
    n = wl.N // 2
    direction = np.array([0.6, 0.0, 0.8])
    vals = []
    for delta in (1e-2, 1e-3, 1e-4, 1e-5):
        Xc = X.copy()
        if kind == "ee":      # up electron 0 approaches down electron n
            Xc[0] = Xc[n] + delta * direction
        else:                 # electron 0 approaches proton 2
            Xc[0] = wl.R[2] + delta * direction
        vals.append(orc.eval_config(sysP, wl.R, Xc)["el"])
    assert abs(vals[-1] - vals[-2]) < 0.02, vals
    assert abs(vals[-2] - vals[-3]) < 0.2, vals


# ---------------------------------------------------------------- force estimator
def test_force_equals_reweighted_energy_derivative():
    """f = -<dE_L> - 2(<E_L dlnpsi> - E <dlnpsi>) is exactly -dE/dR of the
    reweighted estimator E(R') = sum w E_L(R') / sum w, w = psi^2(R')/psi^2(R)."""
    wl = synth.workload("h16")
    sysP = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    X = synth.near_protons(24, wl.R, wl.N // 2, 0.7, wl.L, 9)
    lp0, el0, dl, de = orc.eval_configs(sysP, wl.R, X, derivs=True)
    N3 = 3 * wl.N
    acc = np.zeros((X.shape[0], 3 + 3 * N3))
    acc[:, 0] = 1
    acc[:, 1] = el0
    acc[:, 2] = el0 ** 2
    acc[:, 3:3 + N3] = dl.reshape(-1, N3)
    acc[:, 3 + N3:3 + 2 * N3] = el0[:, None] * dl.reshape(-1, N3)
    acc[:, 3 + 2 * N3:] = de.reshape(-1, N3)
    f = orc.reduce(acc, wl.N)["f"]
    h = 2e-5
    for a, mu in ((0, 0), (7, 2), (15, 1)):
        Es = []
        for s in (+1, -1):
            R2 = wl.R.copy(); R2[a, mu] += s * h
            lp, el, _, _ = orc.eval_configs(sysP, R2, X, derivs=False)
            w = np.exp(2 * (lp - lp0))
            Es.append(np.sum(w * el) / np.sum(w))
        dE = (Es[0] - Es[1]) / (2 * h)
        assert abs(f[3 * a + mu] + dE) < 1e-5 * (1 + abs(dE))


def test_reduce_recovers_known_covariance():
    """i.i.d. force samples with known covariance: S * N_c recovers it."""
    rng = np.random.default_rng(21)
    N = 2
    N3 = 3 * N
    W, m = 6000, 3
    Araw = rng.standard_normal((N3, N3))
    Sigma = Araw @ Araw.T / N3 + 0.5 * np.eye(N3)
    Lc = np.linalg.cholesky(Sigma)
    mu = rng.standard_normal(N3)
    dE = mu + rng.standard_normal((W, m, N3)) @ Lc.T      # E_L = 0 => f = -dE_L
    acc = np.zeros((W, 3 + 3 * N3))
    acc[:, 0] = m
    acc[:, 3 + 2 * N3:] = dE.sum(1)
    r = orc.reduce(acc, N)
    assert r["Nc"] == W * m
    assert np.allclose(r["f"], -dE.reshape(-1, N3).mean(0), atol=1e-12)
    S_full = r["S"] * r["Nc"]
    rel = np.abs(S_full - Sigma) / np.sqrt(np.outer(np.diag(Sigma), np.diag(Sigma)))
    assert rel.max() < 6 * math.sqrt(2.0 / W)


def test_vmc_samples_psi_squared_tiny_system():
    """N=2 periodic: the Metropolis estimate of <E_L> agrees with an importance-
    sampled brute-force integral over uniform configurations."""
    L = synth.box_side(2, 1.4)
    R = np.array([[0.4, 0.5, 0.6], [1.9, 1.7, 2.2]])
    C = synth.coefficients(4, 1, 5)
    sys2 = orc.System(N=2, L=L, zeta=np.array([0.5, 1.5]), coeff=C)
    X, acc, ar = orc.vmc(sys2, R, W=256, n_sweeps=400, n_warmup=40, sigma=0.6, seed=3, forces=False)
    r = orc.reduce(acc, 2)
    U = synth.random_electrons(120000, 2, L, 77)
    lp, el, _, _ = orc.eval_configs(sys2, R, U, derivs=False)
    w = np.exp(2 * (lp - lp.max()))
    E_bf = np.sum(w * el) / np.sum(w)
    # delta-method error of the ratio estimator
    wn = w / w.mean()
    err_bf = math.sqrt(np.mean(wn ** 2 * (el - E_bf) ** 2) / len(w))
    assert abs(r["E"] - E_bf) < 3.5 * math.hypot(r["E_err"], err_bf), (r["E"], E_bf, r["E_err"], err_bf)
