"""Pins of the oracle's 3- and 4-body e-e-n-n Jastrow term U_{3+4} (SI, Jastrow
section: sum over electron pairs i<j and nuclei a, b of f^{ab} phi_a(r_i)
phi_b(r_j), one periodised Gaussian per nucleus with the SI's exponent
0.7933844).  The term is checked against a closed form on one nucleus, finite
differences in the electron and nuclear coordinates, permutation invariance,
linearity in the coefficients and the Metropolis delta."""
import numpy as np

from oracle import oracle as orc
from paper_1605_08423_gb300 import synth


def _fj(N, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (N, N)) * scale
    return 0.5 * (A + A.T)


def _h16(fj, seed_conf=0):
    wl = synth.workload("h16")
    sysP = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, fj=fj)
    X = synth.near_protons(1, wl.R, wl.N // 2, 0.6, wl.L, seed_conf)[0]
    return wl, sysP, X


def _u34(wl, X, fj, R=None):
    """U_{3+4} alone: ln|psi| with the term minus ln|psi| without it (same determinants)."""
    R = wl.R if R is None else R
    on = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, fj=fj)
    off = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    return orc.eval_config(on, R, X)["lnpsi"] - orc.eval_config(off, R, X)["lnpsi"]


def test_one_nucleus_closed_form():
    """Open boundary, one nucleus, two electrons: U_{3+4} = f exp(-z r1^2) exp(-z r2^2)."""
    f, z = 0.37, 0.7933844
    base = dict(N=1, L=10.0, zeta=np.array([0.4]), coeff=np.array([[1.0]]), n_up=1, n_dn=1, b_ee=1.0, b_ep=1.0,
                periodic=False)
    R = np.array([[0.2, -0.1, 0.3]])
    X = np.array([[0.9, 0.4, -0.2], [-0.5, 0.1, 0.8]])
    on = orc.eval_config(orc.System(**base, fj=np.array([[f]])), R, X)
    off = orc.eval_config(orc.System(**base), R, X)
    r1, r2 = np.sum((X[0] - R[0]) ** 2), np.sum((X[1] - R[0]) ** 2)
    assert abs((on["lnpsi"] - off["lnpsi"]) - f * np.exp(-z * r1) * np.exp(-z * r2)) < 1e-15
    # its gradient in r_1: -2 z (r_1 - R) U
    u = f * np.exp(-z * r1) * np.exp(-z * r2)
    assert np.allclose(on["grad"][0] - off["grad"][0], -2 * z * (X[0] - R[0]) * u, atol=1e-15)


def test_zero_coefficients_switch_the_term_off():
    wl, sysP, X = _h16(np.zeros((16, 16)))
    sys0 = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    a = orc.eval_config(sysP, wl.R, X, derivs=True)
    b = orc.eval_config(sys0, wl.R, X, derivs=True)
    for k in ("lnpsi", "el"):
        assert a[k] == b[k]
    for k in ("grad", "dlnpsi", "del_"):
        assert np.array_equal(a[k], b[k])


def test_grad_and_kinetic_vs_finite_differences():
    wl, sysP, X = _h16(_fj(16, 1))
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
    wl, sysP, X = _h16(_fj(16, 2), 1)
    o = orc.eval_config(sysP, wl.R, X, derivs=True)
    h = 1e-4
    for a in (0, 7, 13):
        for mu in range(3):
            Rp = wl.R.copy(); Rp[a, mu] += h
            Rm = wl.R.copy(); Rm[a, mu] -= h
            op = orc.eval_config(sysP, Rp, X)
            om = orc.eval_config(sysP, Rm, X)
            d_l = (op["lnpsi"] - om["lnpsi"]) / (2 * h)
            d_e = (op["el"] - om["el"]) / (2 * h)
            assert abs(o["dlnpsi"][a, mu] - d_l) < 1e-6 * (1 + abs(d_l))
            assert abs(o["del_"][a, mu] - d_e) < 1e-6 * (1 + abs(d_e))


def test_permutation_invariance_and_linearity():
    # U_{3+4} is a difference of two ln|psi| of magnitude ~10, so agreement is
    # checked to 1e-11 absolute (a wrong term would be off by ~0.1)
    tol = 1e-11
    wl, _, X = _h16(None, 2)
    f1, f2 = _fj(16, 3), _fj(16, 4)
    u1, u2, u12 = _u34(wl, X, f1), _u34(wl, X, f2), _u34(wl, X, f1 + f2)
    assert abs(u12 - (u1 + u2)) < tol
    assert abs(_u34(wl, X, 2.5 * f1) - 2.5 * u1) < tol
    # any permutation of the electrons, across spins too, leaves U_{3+4} unchanged
    perm = np.random.default_rng(5).permutation(X.shape[0])
    assert abs(_u34(wl, X[perm], f1) - u1) < tol
    # a nucleus relabelling with the same relabelling of f leaves it unchanged
    q = np.random.default_rng(6).permutation(16)
    assert abs(_u34(wl, X, f1[np.ix_(q, q)], R=wl.R[q]) - u1) < tol


def test_metropolis_delta_matches_full_evaluations():
    wl, sysP, X = _h16(_fj(16, 7), 3)
    sys0 = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    rng = np.random.default_rng(8)
    for i in (0, 5, 11, 15):
        xn = X[i] + 0.3 * rng.standard_normal(3)
        Xn = X.copy(); Xn[i] = xn
        d34 = orc.jastrow_delta(sysP, wl.R, X, i, xn) - orc.jastrow_delta(sys0, wl.R, X, i, xn)
        full = _u34(wl, Xn, sysP.fj) - _u34(wl, X, sysP.fj)
        assert abs(d34 - full) < 1e-11
