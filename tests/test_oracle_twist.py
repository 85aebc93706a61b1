"""Pins of the oracle's twisted-boundary-condition form (SI, basis section:
phi(r + nL) = exp(i theta.n) phi(r); main text: k-point average on a
Monkhorst-Pack mesh) against closed forms, finite differences, invariances and
brute force.  None of these call the CUDA library."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import synth


def _fourier_bloch(L, d, zeta, theta, mmax=12):
    """The Bloch-summed Gaussian by Poisson summation: per axis
    sum_n e^{i th n} e^{-zeta (d - nL)^2} = (1/L) sqrt(pi/zeta)
        sum_m exp(-(th + 2 pi m)^2 / (4 zeta L^2)) exp(i (th + 2 pi m) d / L),
    with its first and second derivatives in d (a sum of plane waves)."""
    s = np.zeros(3, complex); s1 = np.zeros(3, complex); s2 = np.zeros(3, complex)
    for mu in range(3):
        for m in range(-mmax, mmax + 1):
            k = (theta[mu] + 2 * math.pi * m) / L
            a = math.sqrt(math.pi / zeta) / L * math.exp(-(k * L) ** 2 / (4 * zeta * L * L))
            e = a * np.exp(1j * k * d[mu])
            s[mu] += e; s1[mu] += 1j * k * e; s2[mu] += -k * k * e
    chi = s[0] * s[1] * s[2]
    grad = np.array([s1[0] * s[1] * s[2], s[0] * s1[1] * s[2], s[0] * s[1] * s1[2]])
    lap = s2[0] * s[1] * s[2] + s[0] * s2[1] * s[2] + s[0] * s[1] * s2[2]
    return chi, grad, lap


@pytest.mark.parametrize("zeta", [0.5, 1.5, 0.122])
def test_bloch_gaussian_equals_its_fourier_series(zeta):
    L = synth.box_side(16, 1.4)
    rng = np.random.default_rng(11)
    M = max(1, math.ceil(math.sqrt(40 / zeta) / L - 0.5))
    for _ in range(6):
        x, Rc = rng.uniform(0, L, 3), rng.uniform(0, L, 3)
        th = rng.uniform(-math.pi, math.pi, 3)
        chi, grad, lap = orc.bloch_gaussian(L, x, Rc, zeta, th, M)
        c2, g2, l2 = _fourier_bloch(L, x - Rc, zeta, th)
        scale = max(abs(c2), 1e-3)
        assert abs(chi - c2) < 1e-12 * max(scale, 1.0)
        assert np.max(np.abs(grad - g2)) < 1e-11 * max(scale, 1.0)
        assert abs(lap - l2) < 1e-10 * max(scale, 1.0)


def test_bloch_gaussian_bloch_property():
    """chi(r + mL) = exp(i theta.m) chi(r), for value, gradient and Laplacian."""
    L, zeta, M = 5.0, 0.5, 3
    rng = np.random.default_rng(2)
    for _ in range(5):
        x, Rc = rng.uniform(0, L, 3), rng.uniform(0, L, 3)
        th = rng.uniform(-math.pi, math.pi, 3)
        m = rng.integers(-2, 3, 3)
        c0, g0, l0 = orc.bloch_gaussian(L, x, Rc, zeta, th, M)
        c1, g1, l1 = orc.bloch_gaussian(L, x + m * L, Rc, zeta, th, M)
        ph = np.exp(1j * np.dot(th, m))
        assert abs(c1 - ph * c0) < 1e-13
        assert np.max(np.abs(g1 - ph * g0)) < 1e-13
        assert abs(l1 - ph * l0) < 1e-12


def _system(wl, theta, **kw):
    return orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, twist=np.asarray(theta, float), **kw)


THETA = np.array([0.7, -1.3, 2.1])


def test_twisted_wavefunction_bloch_and_time_reversal():
    """Moving a spin-up electron by L e_mu multiplies psi by exp(i theta_mu), a
    spin-down one by exp(-i theta_mu); psi(-theta) = conj psi(theta), so ln|psi|,
    E_L and the R-derivatives are even in theta and Im E_kin is odd."""
    wl = synth.workload("h16")
    X = synth.near_protons(1, wl.R, wl.N // 2, 0.6, wl.L, 21)[0]
    s = _system(wl, THETA)
    r0 = orc.eval_config_twist(s, wl.R, X, derivs=True)
    for i, mu, sg in ((0, 0, 1), (3, 2, 1), (9, 1, -1), (15, 0, -1)):
        Xm = X.copy()
        Xm[i, mu] += wl.L
        r1 = orc.eval_config_twist(s, wl.R, Xm)
        assert abs(r1["lnpsi"] - r0["lnpsi"]) < 1e-11
        dph = math.remainder(r1["phase"] - r0["phase"] - sg * THETA[mu], 2 * math.pi)
        assert abs(dph) < 1e-10
        assert abs(r1["el"] - r0["el"]) < 1e-9
    rm = orc.eval_config_twist(_system(wl, -THETA), wl.R, X, derivs=True)
    assert abs(rm["lnpsi"] - r0["lnpsi"]) < 1e-11
    assert abs(math.remainder(rm["phase"] + r0["phase"], 2 * math.pi)) < 1e-10
    assert abs(rm["el"] - r0["el"]) < 1e-9 and abs(rm["ekin_im"] + r0["ekin_im"]) < 1e-9
    assert np.max(np.abs(rm["dlnpsi"] - r0["dlnpsi"])) < 1e-9
    assert np.max(np.abs(rm["del_"] - r0["del_"])) < 1e-8


def _psi_ratio(s, R, X, X0ref):
    r = orc.eval_config_twist(s, R, X)
    return r["lnpsi"] - X0ref["lnpsi"], r["phase"] - X0ref["phase"]


def test_twisted_kinetic_energy_vs_finite_differences():
    """-1/2 sum_i lap_i psi / psi of the complex psi by a fourth-order central
    stencil on psi(X + h e) / psi(X) = exp(d ln|psi| + i d arg psi): its real
    part is E_kin, its imaginary part Im E_kin."""
    wl = synth.workload("h16")
    X = synth.near_protons(1, wl.R, wl.N // 2, 0.6, wl.L, 33)[0]
    s = _system(wl, THETA)
    r0 = orc.eval_config_twist(s, wl.R, X)
    h = 1e-2
    lap = 0.0 + 0.0j
    for i in range(wl.N):
        for mu in range(3):
            vals = []
            for k in (-2, -1, 1, 2):
                Xk = X.copy()
                Xk[i, mu] += k * h
                dl, dp = _psi_ratio(s, wl.R, Xk, r0)
                vals.append(np.exp(dl + 1j * dp))
            fm2, fm1, fp1, fp2 = vals
            lap += (-fp2 + 16 * fp1 - 30.0 + 16 * fm1 - fm2) / (12 * h * h)
    ek = -0.5 * lap
    assert abs(ek.real - r0["ekin"]) < 2e-6 * max(1.0, abs(r0["ekin"])), (ek, r0["ekin"])
    assert abs(ek.imag - r0["ekin_im"]) < 2e-6 * max(1.0, abs(r0["ekin"])), (ek, r0["ekin_im"])


def test_twisted_R_derivatives_vs_finite_differences():
    wl = synth.workload("h16")
    X = synth.near_protons(1, wl.R, wl.N // 2, 0.6, wl.L, 44)[0]
    s = _system(wl, THETA)
    r0 = orc.eval_config_twist(s, wl.R, X, derivs=True)
    h = 1e-4
    for a, mu in ((0, 0), (5, 1), (11, 2), (15, 0)):
        Rp, Rm = wl.R.copy(), wl.R.copy()
        Rp[a, mu] += h
        Rm[a, mu] -= h
        p = orc.eval_config_twist(s, Rp, X)
        m = orc.eval_config_twist(s, Rm, X)
        fd_l = (p["lnpsi"] - m["lnpsi"]) / (2 * h)
        fd_e = (p["el"] - m["el"]) / (2 * h)
        assert abs(fd_l - r0["dlnpsi"][a, mu]) < 1e-6 * max(1.0, abs(fd_l))
        assert abs(fd_e - r0["del_"][a, mu]) < 1e-5 * max(1.0, abs(fd_e))


def test_plane_wave_limit_kinetic_energy():
    """One electron in one broad Bloch Gaussian without Jastrow: by Poisson
    summation the orbital is the plane wave exp(i theta.r / L) up to terms of
    relative size exp(-((2 pi - |theta_mu|)^2 - theta_mu^2) / (4 zeta L^2)), so
    E_kin = |theta|^2 / (2 L^2)."""
    L, zeta = 5.0, 0.01
    th = np.array([0.4, -0.9, 0.6])
    s = orc.System(N=1, L=L, zeta=np.array([zeta]), coeff=np.array([[1.0]]), n_up=1, n_dn=0, Zj=0.0,
                   twist=th)
    R = np.array([[1.0, 2.0, 3.0]])
    for x in (np.array([0.3, 4.1, 2.2]), np.array([4.9, 0.1, 3.3])):
        r = orc.eval_config_twist(s, R, x[None, :])
        assert abs(r["ekin"] - th @ th / (2 * L * L)) < 1e-11
        assert abs(r["ekin_im"]) < 1e-11


def test_reduce_twists_combination_rule():
    """K = 1 is the plain reduction; K identical blocks give the block's E and
    f, S / K and E_err / sqrt(K); the order of the blocks does not matter."""
    rng = np.random.default_rng(5)
    N, Wk, K = 2, 40, 4
    stride = 3 + 9 * N
    blk = np.zeros((Wk, stride))
    blk[:, 0] = 10.0
    blk[:, 1] = rng.normal(-1.0, 0.1, Wk) * 10
    blk[:, 2] = blk[:, 1] ** 2 / 10
    blk[:, 3:] = rng.normal(0.0, 1.0, (Wk, 9 * N))
    one = orc.reduce(blk, N)
    k1 = orc.reduce_twists(blk, N, 1)
    for key in ("E", "E_err", "Nc"):
        assert k1[key] == pytest.approx(one[key], rel=1e-14)
    assert np.allclose(k1["f"], one["f"], rtol=1e-14, atol=0) and np.allclose(k1["S"], one["S"], rtol=1e-14, atol=0)
    rep = orc.reduce_twists(np.concatenate([blk] * K), N, K)
    assert rep["E"] == pytest.approx(one["E"], rel=1e-14)
    assert rep["E_err"] == pytest.approx(one["E_err"] / math.sqrt(K), rel=1e-12)
    assert rep["Nc"] == K * one["Nc"]
    assert np.allclose(rep["f"], one["f"], rtol=1e-13, atol=1e-15)
    assert np.allclose(rep["S"], one["S"] / K, rtol=1e-12, atol=1e-18)
    blocks = [blk + rng.normal(0, 0.3, blk.shape) * (np.arange(stride) >= 3) for _ in range(K)]
    a = orc.reduce_twists(np.concatenate(blocks), N, K)
    b = orc.reduce_twists(np.concatenate(blocks[::-1]), N, K)
    assert a["E"] == pytest.approx(b["E"], rel=1e-14)
    assert np.allclose(a["f"], b["f"], rtol=1e-12, atol=1e-15) and np.allclose(a["S"], b["S"], rtol=1e-12, atol=1e-18)


def test_reduce_twists_known_covariance():
    """Per-walker block forces drawn i.i.d. with covariance Sigma in every twist
    block: the twist-averaged S estimates Sigma / W (W walkers in all)."""
    rng = np.random.default_rng(8)
    N, K, Wk = 1, 5, 400
    N3 = 3 * N
    A = rng.normal(0, 1, (N3, N3))
    Sigma = A @ A.T + N3 * np.eye(N3)
    Lc = np.linalg.cholesky(Sigma)
    acc = np.zeros((K * Wk, 3 + 3 * N3))
    for t in range(K):
        for w in range(Wk):
            row = acc[t * Wk + w]
            row[0] = 1.0
            row[1] = 0.5 * t          # E_w: the twists differ in energy
            row[2] = row[1] ** 2
            fw = Lc @ rng.normal(0, 1, N3) + t   # with dlnpsi = 0: f_w = -dE_L
            row[3 + 2 * N3:] = -fw
    r = orc.reduce_twists(acc, N, K)
    W = K * Wk
    assert r["E"] == pytest.approx(np.mean([0.5 * t for t in range(K)]), abs=1e-12)
    rel = np.abs(np.diag(r["S"]) * W / np.diag(Sigma) - 1)
    assert np.all(rel < 4 * math.sqrt(2 / (W - K)))


def test_twisted_chain_samples_psi_squared_tiny_system():
    """N = 2 periodic with a twist: the Metropolis estimate of <E_L> agrees with
    an importance-sampled brute-force integral over uniform configurations."""
    L = synth.box_side(2, 1.4)
    R = np.array([[0.4, 0.5, 0.6], [1.9, 1.7, 2.2]])
    C = synth.coefficients(4, 1, 5)
    th = np.array([[0.9, -0.4, 1.7]])
    s2 = orc.System(N=2, L=L, zeta=np.array([0.5, 1.5]), coeff=C, twist=th[0])
    X, acc, ar, _ = orc.vmc_twists(s2, R, th, W=128, n_sweeps=300, n_warmup=40, sigma=0.6, seed=3, forces=False)
    r = orc.reduce(acc, 2)
    U = synth.random_electrons(60000, 2, L, 77)
    lp, el, _, _ = orc.eval_configs_twist(s2, R, U, th, derivs=False)
    w = np.exp(2 * (lp - lp.max()))
    E_bf = np.sum(w * el) / np.sum(w)
    wn = w / w.mean()
    err_bf = math.sqrt(np.mean(wn ** 2 * (el - E_bf) ** 2) / len(w))
    assert abs(r["E"] - E_bf) < 3.5 * math.hypot(r["E_err"], err_bf), (r["E"], E_bf, r["E_err"], err_bf)


def test_monkhorst_pack_mesh_and_its_time_reversal_half():
    """The 4 x 4 x 4 mesh: 64 twists at 2 pi {-3/8, -1/8, 1/8, 3/8}^3, closed
    under negation; its halving keeps one twist of each (theta, -theta) pair,
    and every halved twist gives the oracle's E_L of its partner."""
    full = synth.monkhorst_pack(4)
    assert full.shape == (64, 3)
    assert np.allclose(np.unique(np.round(full / (2 * math.pi) * 8)), [-3, -1, 1, 3])
    half = synth.monkhorst_pack(4, time_reversal=True)
    assert half.shape == (32, 3)
    both = np.concatenate([half, -half])
    key = lambda a: sorted(map(tuple, np.round(a / (2 * math.pi) * 8).astype(int)))
    assert key(both) == key(full)
    wl = synth.workload("h16")
    X = synth.near_protons(1, wl.R, wl.N // 2, 0.6, wl.L, 4)[0]
    for th in half[:3]:
        a = orc.eval_config_twist(_system(wl, th), wl.R, X)
        b = orc.eval_config_twist(_system(wl, -th), wl.R, X)
        assert abs(a["el"] - b["el"]) < 1e-9 and abs(a["lnpsi"] - b["lnpsi"]) < 1e-11
