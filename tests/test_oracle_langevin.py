"""Pins of the oracle's accelerated Langevin step against the closed forms of the
harmonic problem and against the stationary distribution of a position-dependent
acceleration matrix (no QMC involved; forces are analytic)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc


def _spd(n, seed, cond=20.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ Q.T


def test_L1_zero_temperature_is_steepest_descent():
    K = _spd(4, 1)
    R = np.array([0.3, -1.2, 0.8, 2.0])
    d = 0.03
    out = orc.langevin(R, R, -K @ R, np.eye(4), np.eye(4), 0.0, d, 0.0, np.ones(4))
    assert np.allclose(out, (np.eye(4) - d * K) @ R, atol=1e-14)


def test_L2_hessian_preconditioner_is_one_newton_step():
    K = _spd(5, 2, cond=1e4)
    Req = np.array([0.1, 0.2, -0.3, 0.4, 0.5])
    R = Req + np.array([1.0, -2.0, 0.5, 0.3, -0.7])
    out = orc.langevin(R, R, -K @ (R - Req), K, K, 0.0, 1.0, 0.0, np.zeros(5))
    assert np.allclose(out, Req, atol=1e-10)


def _run(K, S, T, d, alpha, steps, seed, R0=None):
    n = K.shape[0]
    rng = np.random.default_rng(seed)
    R = np.zeros(n) if R0 is None else R0.copy()
    traj = np.empty((steps, n))
    for t in range(steps):
        R = orc.langevin(R, R, -K @ R, S, S, T, d, alpha, rng.standard_normal(n))
        traj[t] = R
    return traj


def _lag1(x):
    x = x - x.mean(0)
    return (x[1:] * x[:-1]).mean(0) / (x * x).mean(0)


def test_L3_cfold_stationary_variance_and_autocorrelation():
    k = np.array([0.2, 0.5, 1.0, 1.5])
    K = np.diag(k)
    T, d = 0.7, 0.8
    traj = _run(K, np.eye(4), T, d, 0.0, 60000, 3)[500:]
    var = traj.var(0)
    phi = 1 - k * d
    expect = T / (k * (1 - k * d / 2))
    err = expect * np.sqrt(2 * (1 + phi ** 2) / (1 - phi ** 2) / len(traj))
    assert np.all(np.abs(var - expect) < 4 * err), (var, expect)
    assert np.allclose(_lag1(traj), phi, atol=0.03)


def test_L4_adopted_scheme_exact_covariance_any_timestep():
    """S = K/alpha: stationary covariance T K^{-1} for any Delta, lag-1 e^{-alpha Delta}."""
    K = _spd(3, 4, cond=50.0)
    alpha = 0.9
    S = K / alpha
    T = 0.4
    for d in (0.5, 3.0):
        traj = _run(K, S, T, d, alpha, 40000, 5 + int(d))[200:]
        cov = np.cov(traj.T)
        target = T * np.linalg.inv(K)
        rel = np.abs(cov - target) / np.sqrt(np.outer(np.diag(target), np.diag(target)))
        assert rel.max() < 0.06, (d, cov, target)
        # every mode decorrelates at the same rate, independent of K's condition number
        z = traj @ np.linalg.cholesky(K)
        assert np.allclose(_lag1(z), math.exp(-alpha * d), atol=0.03)


def test_L5_autocorrelation_independent_of_temperature():
    K = np.diag([0.3, 1.2])
    a = [_lag1(_run(K, np.eye(2), T, 0.5, 0.0, 30000, 9)[300:]) for T in (0.05, 5.0)]
    assert np.allclose(a[0], a[1], atol=0.03)


def test_L6_noise_covariance_is_2T_Dbar_Sinv():
    S = _spd(3, 6, cond=10.0)
    T, d, alpha = 0.3, 0.7, 1.3
    Db = (1 - math.exp(-2 * alpha * d)) / (2 * alpha)
    rng = np.random.default_rng(7)
    draws = np.array([orc.langevin(np.zeros(3), np.zeros(3), np.zeros(3), S, S, T, d, alpha,
                                   rng.standard_normal(3)) for _ in range(30000)])
    target = 2 * T * Db * np.linalg.inv(S)
    cov = np.cov(draws.T)
    rel = np.abs(cov - target) / np.sqrt(np.outer(np.diag(target), np.diag(target)))
    assert rel.max() < 0.04


def test_noise_correction_lowers_temperature():
    T, d = 0.5, 0.2
    rng = np.random.default_rng(8)
    draws = np.array([orc.langevin(np.zeros(1), np.zeros(1), np.zeros(1), np.eye(1), np.eye(1), T, d, 0.0,
                                   rng.standard_normal(1), noise_correction=True) for _ in range(40000)])
    assert abs(draws.var() - 2 * (T - d / 2) * d) < 4 * 2 * (T - d / 2) * d * math.sqrt(2 / 40000)


def test_position_dependent_S_needs_the_two_time_term():
    """V = x^2/2, S(x) = 1 + x^2, T = 1: the canonical <x^2> is 1.  The two-time
    scheme (S difference term) samples it; the simple rule without that term
    samples S(x) e^{-V/T} instead, whose <x^2> is 2."""
    n, steps, d, T = 48, 6000, 0.02, 1.0
    rng = np.random.default_rng(10)
    results = {}
    for two_time in (True, False):
        R = rng.standard_normal(n) * 0.5
        Rprev = R.copy()
        acc = []
        for t in range(steps):
            S = np.diag(1 + R ** 2)
            Sp = np.diag(1 + Rprev ** 2) if two_time else S
            Rn = orc.langevin(R, Rprev, -R, S, Sp, T, d, 0.0, rng.standard_normal(n))
            Rprev, R = R, Rn
            if t > 1000:
                acc.append(R ** 2)
        results[two_time] = float(np.mean(acc))
    assert abs(results[True] - 1.0) < 0.15, results
    assert results[False] > 1.6, results


def test_langevin_noise_stream_is_standard_normal():
    xi = np.concatenate([orc.langevin_noise(99, m, 500) for m in range(40)])
    assert abs(xi.mean()) < 4 / math.sqrt(xi.size)
    assert abs(xi.var() - 1) < 4 * math.sqrt(2 / xi.size)


def test_non_positive_definite_S_is_rejected():
    with pytest.raises(ValueError):
        orc.langevin(np.zeros(2), np.zeros(2), np.zeros(2), np.diag([1.0, -1.0]), np.eye(2), 0.1, 0.1, 0.0,
                     np.zeros(2))


def test_fast_scheme_is_adopted_at_zero_alpha_and_ignores_alpha():
    """Eq. finaldyn is Eq. finaldyn_new at alpha = 0 (Dt = Db = Delta)."""
    rng = np.random.default_rng(11)
    n = 6
    S, Sp = _spd(n, 12), _spd(n, 13)
    R, Rp, f, xi = (rng.standard_normal(n) for _ in range(4))
    a = orc.langevin(R, Rp, f, S, Sp, 0.3, 0.4, 0.0, xi)
    b = orc.langevin(R, Rp, f, S, Sp, 0.3, 0.4, 2.5, xi, scheme=orc.LV_FAST)
    assert np.allclose(a, b, rtol=0, atol=1e-13)
    # and its S_prev term is -1/2 S^{-1} (S_prev - S)(R_prev - R) written out
    c = orc.langevin(R, Rp, f, S, S, 0.3, 0.4, 0.0, xi, scheme=orc.LV_FAST)
    assert np.allclose(b - c, -0.5 * np.linalg.solve(S, (Sp - S) @ (Rp - R)), atol=1e-12)


def test_norogna_scheme_drops_the_two_time_term():
    rng = np.random.default_rng(14)
    n = 5
    S, Sp = _spd(n, 15), _spd(n, 16)
    R, Rp, f, xi = (rng.standard_normal(n) for _ in range(4))
    a = orc.langevin(R, Rp, f, S, Sp, 0.2, 0.3, 1.0, xi, scheme=orc.LV_NOROGNA)
    b = orc.langevin(R, R, f, S, S, 0.2, 0.3, 0.0, xi)
    assert np.allclose(a, b, rtol=0, atol=1e-13)


def test_fast_scheme_stationary_covariance_closed_form():
    """Constant S = K/alpha0: the fast scheme is R' = (1 - alpha0 D) R + sqrt(2 T D) z,
    whose stationary covariance is 2 T K^{-1} / (2 - alpha0 D) (discrete Lyapunov)."""
    K = _spd(3, 17, cond=20.0)
    a0, T, d = 0.9, 0.4, 0.8
    S = K / a0
    rng = np.random.default_rng(18)
    R = np.zeros(3)
    traj = np.empty((40000, 3))
    for t in range(len(traj)):
        R = orc.langevin(R, R, -K @ R, S, S, T, d, 7.0, rng.standard_normal(3), scheme=orc.LV_FAST)
        traj[t] = R
    cov = np.cov(traj[200:].T)
    target = 2 * T * np.linalg.inv(K) / (2 - a0 * d)
    rel = np.abs(cov - target) / np.sqrt(np.outer(np.diag(target), np.diag(target)))
    assert rel.max() < 0.06, (cov, target)


def test_first_simplified_scheme_closed_forms():
    """Eq. smartMarkov: at T = 0 it is the drift step R + D S^{-1} f; with S(y) = S
    its correction vanishes; the S-difference term is written out."""
    rng = np.random.default_rng(21)
    n = 5
    S, Sy = _spd(n, 22), _spd(n, 23)
    R, f, xi = (rng.standard_normal(n) for _ in range(3))
    y0 = orc.langevin_first_predict(R, S, 0.0, 0.3, xi)
    assert np.array_equal(y0, R)
    assert np.allclose(orc.langevin_first_correct(R, f, S, Sy, y0, 0.3), R + 0.3 * np.linalg.solve(S, f), atol=1e-13)
    T, d = 0.4, 0.3
    y = orc.langevin_first_predict(R, S, T, d, xi)
    Lc = np.linalg.cholesky(S)
    assert np.allclose(y, R + math.sqrt(2 * T * d) * np.linalg.solve(Lc.T, xi), atol=1e-13)
    a = orc.langevin_first_correct(R, f, S, S, y, d)
    assert np.allclose(a, y + d * np.linalg.solve(S, f), atol=1e-12)
    b = orc.langevin_first_correct(R, f, S, Sy, y, d)
    assert np.allclose(b - a, -0.5 * np.linalg.solve(S, (Sy - S) @ (y - R)), atol=1e-12)


def test_first_simplified_scheme_samples_canonical_with_position_dependent_S():
    """V = x^2/2, S(x) = 1 + x^2, T = 1: with S evaluated at the predicted point the
    chain samples e^{-V/T} (<x^2> = 1), as the two-time scheme does."""
    n, steps, d, T = 48, 6000, 0.02, 1.0
    rng = np.random.default_rng(24)
    R = rng.standard_normal(n) * 0.5
    acc = []
    for t in range(steps):
        S = np.diag(1 + R ** 2)
        y = orc.langevin_first_predict(R, S, T, d, rng.standard_normal(n))
        R = orc.langevin_first_correct(R, -R, S, np.diag(1 + y ** 2), y, d)
        if t > 1000:
            acc.append(R ** 2)
    assert abs(float(np.mean(acc)) - 1.0) < 0.15


def test_previous_displacement_is_the_minimum_image():
    """In the periodic box the S_prev term takes the previous step's displacement
    R_prev - R as a minimum image: shifting R_prev by whole box sides leaves
    the step unchanged."""
    n, L = 12, 5.0
    rng = np.random.default_rng(12)
    R = rng.uniform(0, L, n)
    Rprev = R + 0.1 * rng.standard_normal(n)
    S, Sp = _spd(n, 3), _spd(n, 4)
    f, xi = rng.standard_normal(n), rng.standard_normal(n)
    a = orc.langevin(R, Rprev, f, S, Sp, 0.3, 0.05, 2.0, xi, box=L)
    shift = L * rng.integers(-2, 3, n)
    b = orc.langevin(R, Rprev + shift, f, S, Sp, 0.3, 0.05, 2.0, xi, box=L)
    assert np.max(np.abs(a - b)) < 1e-12


def test_position_dependent_S_in_a_periodic_box():
    """V = -A cos(2 pi x / L) with S(x) = 1 + 0.8 sin^2(2 pi x / L) on a periodic
    box where positions wrap every few hundred steps: the two-time scheme
    samples the canonical <cos(2 pi x / L)> = I_1(A/T) / I_0(A/T) (a jump of one
    box side in R_prev - R at each wrap would bias it far outside this band)."""
    from scipy.special import i0, i1
    L, A, T, d, n, steps = 4.0, 1.0, 1.0, 0.02, 64, 4000
    k = 2 * math.pi / L
    rng = np.random.default_rng(3)
    R = rng.uniform(0, L, n)
    Rprev = R.copy()
    acc = []
    for t in range(steps):
        S = np.diag(1 + 0.8 * np.sin(k * R) ** 2)
        Sp = np.diag(1 + 0.8 * np.sin(k * Rprev) ** 2)
        Rn = orc.langevin(R, Rprev, -A * k * np.sin(k * R), S, Sp, T, d, 0.0, rng.standard_normal(n), box=L)
        Rprev, R = R, Rn
        if t > 500:
            acc.append(np.cos(k * R))
    a = np.array(acc)
    err = a.mean(axis=0).std() / math.sqrt(n)
    exact = i1(A / T) / i0(A / T)
    assert abs(a.mean() - exact) < 4 * err + 0.01, (a.mean(), exact, err)
