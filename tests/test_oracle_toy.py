"""Pins of the oracle's rotating-spring toy model and of the integrator variants
compared on it (SI, "A simple toy model"; Eqs. standard, smartMarkov, finaldyn,
finaldyn_new, norogna).  Derivatives are checked against finite differences, the
S-difference corrections against the cumbersome term they replace (Gauss-Hermite
averages over the noise), and the sampled distributions against one-dimensional
quadratures of the canonical density and of the density the simple rule samples."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as orc

K, A, T = 2.0, 1.4, 0.01


def _pts():
    rng = np.random.default_rng(3)
    th = rng.uniform(0, 2 * np.pi, 6)
    r = rng.uniform(1.25, 1.6, 6)
    return np.stack([r * np.cos(th), r * np.sin(th)], 1)


@pytest.mark.parametrize("s_mode,mu", [(orc.TOY_S_G, 0.5), (orc.TOY_S_HG, 0.5), (orc.TOY_S_HG, 2.0)])
def test_force_hessian_and_gamma_against_finite_differences(s_mode, mu):
    a = orc.toy_args(orc.TOY_STANDARD, s_mode, mu=mu)
    h = 1e-5
    for x, y in _pts():
        e = orc.toy_eval(a, x, y)
        ev = {(dx, dy): orc.toy_eval(a, x + dx, y + dy) for dx in (-h, 0, h) for dy in (-h, 0, h)}
        fd_grad = np.array([(ev[(h, 0)]["U"] - ev[(-h, 0)]["U"]), (ev[(0, h)]["U"] - ev[(0, -h)]["U"])]) / (2 * h)
        assert np.allclose(e["f"], -fd_grad, rtol=1e-7, atol=1e-10)
        fd_H = np.stack([-(ev[(h, 0)]["f"] - ev[(-h, 0)]["f"]), -(ev[(0, h)]["f"] - ev[(0, -h)]["f"])], 1) / (2 * h)
        assert np.allclose(e["H"], fd_H, rtol=1e-6, atol=1e-8)
        assert np.allclose(e["Sinv"] @ e["S"], np.eye(2), atol=1e-12)
        # Gamma_j = sum_i d_i (S^{-1})_{ji}
        dSi_dx = (ev[(h, 0)]["Sinv"] - ev[(-h, 0)]["Sinv"]) / (2 * h)
        dSi_dy = (ev[(0, h)]["Sinv"] - ev[(0, -h)]["Sinv"]) / (2 * h)
        fd_gam = dSi_dx[:, 0] + dSi_dy[:, 1]
        assert np.allclose(e["Gamma"], fd_gam, rtol=1e-6, atol=1e-8)


def test_G_lambda_is_identity_at_one_and_scales_the_radial_direction():
    x, y = 0.9, -1.1
    r = math.hypot(x, y)
    er, et = np.array([x, y]) / r, np.array([-y, x]) / r
    assert np.allclose(orc.toy_eval(orc.toy_args(s_mode=orc.TOY_S_G, lam=1.0), x, y)["S"], np.eye(2), atol=1e-15)
    for lam in (0.1, 3.0):
        S = orc.toy_eval(orc.toy_args(s_mode=orc.TOY_S_G, lam=lam), x, y)["S"]
        assert np.allclose(S @ er, er / lam, atol=1e-14)
        assert np.allclose(S @ et, et, atol=1e-14)


def test_hessian_of_the_spring_closed_form():
    # H = k e_r e_r^T + k (1 - a/r) e_t e_t^T for U = k/2 (r - a)^2
    a = orc.toy_args(s_mode=orc.TOY_S_HG, mu=0.0)
    for x, y in _pts():
        r = math.hypot(x, y)
        er, et = np.array([x, y]) / r, np.array([-y, x]) / r
        H = K * np.outer(er, er) + K * (1 - A / r) * np.outer(et, et)
        e = orc.toy_eval(a, x, y)
        assert np.allclose(e["H"], H, atol=1e-13)
        assert np.allclose(e["S"], H, atol=1e-13)


def _gh2(n=24):
    z, w = np.polynomial.hermite_e.hermegauss(n)
    w = w / math.sqrt(2 * math.pi)
    return [(np.array([z[i], z[j]]), w[i] * w[j]) for i in range(n) for j in range(n)]


@pytest.mark.parametrize("s_mode,mu", [(orc.TOY_S_G, 0.5), (orc.TOY_S_HG, 2.0)])
def test_first_and_fast_corrections_average_to_the_cumbersome_term(s_mode, mu):
    """E_z of the S-difference term of Eq. smartMarkov (and of Eq. finaldyn with
    R_prev - R = -sqrt(2 T D) z) is T D Gamma + O(D^2) (SI, Eqs. questa, cumber)."""
    R = np.array([1.2, 0.5])
    errs = {}
    for scheme in (orc.TOY_FIRST, orc.TOY_FAST):
        for d in (0.04, 0.01):
            a = orc.toy_args(scheme, s_mode, mu=mu, delta=d, T=T)
            ref = orc.toy_args(orc.TOY_NOROGNA, s_mode, mu=mu, delta=d, T=T)
            e = orc.toy_eval(a, *R)
            Lc = np.linalg.cholesky(e["S"])
            mean = np.zeros(2)
            for xi, w in _gh2():
                if scheme == orc.TOY_FIRST:
                    c = orc.toy_step(a, R, R, xi) - orc.toy_step(ref, R, R, xi)
                else:
                    Rp = R - math.sqrt(2 * T * d) * np.linalg.solve(Lc.T, xi)
                    c = orc.toy_step(a, R, Rp, np.zeros(2)) - orc.toy_step(ref, R, R, np.zeros(2))
                mean += w * c
            errs[(scheme, d)] = np.linalg.norm(mean / (T * d) - e["Gamma"]) / np.linalg.norm(e["Gamma"])
        # relative error O(D): small, and shrinking about 4x when D shrinks 4x
        assert errs[(scheme, 0.01)] < 2e-3, errs
        assert errs[(scheme, 0.01)] < 0.4 * errs[(scheme, 0.04)], errs


def test_schemes_reduce_to_each_other_where_the_paper_says():
    rng = np.random.default_rng(5)
    R, Rp, xi = np.array([1.3, -0.4]), np.array([1.35, -0.38]), rng.standard_normal(2)
    for s_mode, mu in ((orc.TOY_S_G, 0.5), (orc.TOY_S_HG, 2.0)):
        st = lambda sc, **kw: orc.toy_step(orc.toy_args(sc, s_mode, mu=mu, **kw), R, Rp, xi)
        # T = 0: every covariant scheme is the drift step R + D S^{-1} f
        base = st(orc.TOY_NOROGNA, T=0.0)
        for sc in (orc.TOY_STANDARD, orc.TOY_FIRST):
            assert np.allclose(st(sc, T=0.0), base, atol=1e-15)
        # adopted at alpha -> 0 is the fast scheme
        assert np.allclose(st(orc.TOY_ADOPTED, alpha=1e-9), st(orc.TOY_FAST), atol=1e-9)
        # the fast scheme with R_prev = R is the simple rule
        assert np.allclose(orc.toy_step(orc.toy_args(orc.TOY_FAST, s_mode, mu=mu), R, R, xi),
                           st(orc.TOY_NOROGNA), atol=1e-15)
    # S = G_1 = I: the covariant schemes are the plain one
    st1 = lambda sc: orc.toy_step(orc.toy_args(sc, orc.TOY_S_G, lam=1.0), R, Rp, xi)
    for sc in (orc.TOY_STANDARD, orc.TOY_FIRST, orc.TOY_FAST, orc.TOY_NOROGNA):
        assert np.allclose(st1(sc), st1(orc.TOY_PLAIN), atol=1e-15)


def _quad_U(extra_log_weight):
    """<U> over the radial density r e^{-U/T} e^{extra(r)}."""
    w = lambda r: r * math.exp(-0.5 * K * (r - A) ** 2 / T + extra_log_weight(r))
    lo, hi = A - 0.65, A + 0.65      # 9 radial widths sqrt(T/k) either side
    num = integrate.quad(lambda r: 0.5 * K * (r - A) ** 2 * w(r), lo, hi, points=[A], limit=200)[0]
    return num / integrate.quad(w, lo, hi, points=[A], limit=200)[0]


def _norogna_extra(s_mode, lam, mu):
    """The simple rule samples grad ln P = f/T - S Gamma; for S = s_r P_r + s_t(r) P_t
    with constant s_r this is e^{-U/T} exp(-int (1 - s_r/s_t(r)) / r dr)."""
    if s_mode == orc.TOY_S_G:
        return lambda r: -(1.0 - 1.0 / lam) * math.log(r)
    s_r = K + mu / lam
    s_t = lambda r: K * (1 - A / r) + mu
    return lambda r: -integrate.quad(lambda q: (1 - s_r / s_t(q)) / q, A, r, limit=200)[0]


def _run_mean_U(scheme, s_mode, mu, d, n_traj=256, t_total=2000.0, seed=21):
    th = np.linspace(0, 2 * np.pi, n_traj, endpoint=False)
    xy0 = np.stack([A * np.cos(th), A * np.sin(th)], 1)
    a = orc.toy_args(scheme, s_mode, mu=mu, delta=d, n_steps=int(t_total / d), n_burn=int(100 / d), seed=seed)
    out = orc.toy_run(a, xy0)
    assert np.all(out[:, 6] == 0)
    m = out[:, 2] / (a.n_steps - a.n_burn)
    return m.mean(), m.std() / math.sqrt(n_traj)


@pytest.mark.parametrize("s_mode,mu", [(orc.TOY_S_G, 0.5), (orc.TOY_S_HG, 2.0)])
def test_stationary_mean_potential(s_mode, mu):
    """The canonical <U> is T/2 (radial harmonic well, ring Jacobian odd); the schemes
    with the S-difference term sample it as D -> 0, the simple rule does not."""
    exact = _quad_U(lambda r: 0.0)
    assert abs(exact - T / 2) < 1e-12
    wrong = _quad_U(_norogna_extra(s_mode, 0.1, mu))
    assert wrong > 1.15 * exact
    for scheme, d in ((orc.TOY_ADOPTED, 0.2), (orc.TOY_FAST, 0.05), (orc.TOY_FIRST, 0.05),
                      (orc.TOY_STANDARD, 0.05)):
        m, e = _run_mean_U(scheme, s_mode, mu, d)
        assert abs(m - exact) < 4 * e + 0.01 * exact, (scheme, m, e, exact)
    m, e = _run_mean_U(orc.TOY_NOROGNA, s_mode, mu, 0.05)
    assert abs(m - wrong) < 4 * e + 0.01 * wrong, (m, e, wrong)


def test_indefinite_S_stops_the_trajectory():
    # S = H + mu G has tangential eigenvalue k (1 - a/r) + mu < 0 for r < k a / (k + mu)
    a = orc.toy_args(orc.TOY_ADOPTED, orc.TOY_S_HG, mu=0.5, n_steps=10)
    out = orc.toy_run(a, np.array([[1.0, 0.0]]))
    assert out[0, 6] == 1.0
    with pytest.raises(ValueError):
        orc.toy_step(a, np.array([1.0, 0.0]), np.array([1.0, 0.0]), np.zeros(2))


def test_toy_noise_is_standard_normal_pairs():
    xi = np.array([orc.toy_noise(7, t, s) for t in range(20) for s in range(1000)])
    n = len(xi)
    assert np.all(np.abs(xi.mean(0)) < 4 / math.sqrt(n))
    assert np.all(np.abs(xi.var(0) - 1) < 4 * math.sqrt(2 / n))
    assert abs(np.mean(xi[:, 0] * xi[:, 1])) < 4 / math.sqrt(n)
