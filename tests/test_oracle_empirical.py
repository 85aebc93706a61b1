"""Pins of the oracle's empirical acceleration matrix S = H + mu I (main text,
conclusions; reading: H the Hessian of the screened-Coulomb proton pair
potential exp(-r/lambda)/r, images within one box side) against a closed form,
finite differences of the energy and the invariances of a pair potential."""
import math

import numpy as np

from oracle import oracle as orc
from paper_1605_08423_gb300 import synth


def _v(r, lam):
    """v, v', v'' of exp(-r/lam)/r."""
    e = math.exp(-r / lam)
    return e / r, -e * (1 / r ** 2 + 1 / (lam * r)), e * (2 / r ** 3 + 2 / (lam * r ** 2) + 1 / (lam ** 2 * r))


def test_two_protons_closed_form():
    """One pair along x: the diagonal block is v'' along the bond and v'/r across
    it (plus mu); the off-diagonal block is minus the same."""
    L, lam, mu, r = 40.0, 0.7, 0.25, 1.3
    R = np.array([[5.0, 7.0, 9.0], [5.0 + r, 7.0, 9.0]])
    S = orc.empirical_s(R, L, lam, mu)
    _, v1, v2 = _v(r, lam)
    assert abs(S[0, 0] - (v2 + mu)) < 1e-13 * abs(v2)
    assert abs(S[1, 1] - (v1 / r + mu)) < 1e-13 * abs(v1)
    assert abs(S[2, 2] - (v1 / r + mu)) < 1e-13 * abs(v1)
    assert abs(S[0, 3] + v2) < 1e-13 * abs(v2) and abs(S[1, 4] + v1 / r) < 1e-13 * abs(v1)
    assert abs(S[0, 1]) < 1e-15 and abs(S[3, 3] - S[0, 0]) < 1e-13 * abs(v2)


def test_hessian_against_finite_differences_and_invariances():
    wl = synth.workload("h16")
    lam, mu = 0.7, 0.0
    S = orc.empirical_s(wl.R, wl.L, lam, mu)
    n3 = 3 * wl.N
    assert np.max(np.abs(S - S.T)) < 1e-12 * np.max(np.abs(S))
    # translation invariance: every block row sums to zero
    rows = S.reshape(wl.N, 3, wl.N, 3).sum(axis=2)
    assert np.max(np.abs(rows)) < 1e-10 * np.max(np.abs(S))
    rng = np.random.default_rng(2)
    R0 = wl.R.ravel()
    h = 1e-3
    E = lambda x: orc.empirical_energy(x, wl.L, lam)
    for _ in range(12):
        i, j = rng.integers(0, n3, 2)
        ei, ej = np.eye(n3)[i] * h, np.eye(n3)[j] * h
        fd = (E(R0 + ei + ej) - E(R0 + ei - ej) - E(R0 - ei + ej) + E(R0 - ei - ej)) / (4 * h * h)
        assert abs(fd - S[i, j]) < 1e-5 * max(1.0, abs(S[i, j])), (i, j, fd, S[i, j])


def test_mu_shifts_the_spectrum():
    wl = synth.workload("h16")
    a = np.linalg.eigvalsh(orc.empirical_s(wl.R, wl.L, 0.7, 0.0))
    b = np.linalg.eigvalsh(orc.empirical_s(wl.R, wl.L, 0.7, 0.3))
    assert np.max(np.abs(b - a - 0.3)) < 1e-10 * np.max(np.abs(a))
    # a pair potential has the three uniform translations as zero modes
    assert np.sum(np.abs(a) < 1e-9 * np.max(np.abs(a))) >= 3


def test_pair_across_half_the_box_sees_both_images():
    """Two protons L/2 + 0.3 apart along x: the images at L/2 + 0.3 and L/2 - 0.3
    both lie within one box side (the ones displaced along y or z do not), so
    the xx entry is v''(L/2 + 0.3) + v''(L/2 - 0.3) and the yy entry the sum of
    v'/r over the same two distances."""
    L, lam, mu = 6.0, 0.7, 0.1
    R = np.array([[1.0, 2.0, 3.0], [1.0 + L / 2 + 0.3, 2.0, 3.0]])
    S = orc.empirical_s(R, L, lam, mu)
    r1, r2 = L / 2 + 0.3, L / 2 - 0.3
    _, a1, a2 = _v(r1, lam)
    _, b1, b2 = _v(r2, lam)
    assert abs(S[0, 0] - (a2 + b2 + mu)) < 1e-12 * abs(a2 + b2)
    assert abs(S[1, 1] - (a1 / r1 + b1 / r2 + mu)) < 1e-12 * abs(b1 / r2)
    assert abs(S[0, 3] + (a2 + b2)) < 1e-12 * abs(a2 + b2)
