"""Host-side pieces of the served form (no GPU): arrival process and percentiles."""
import numpy as np

from paper_1605_08423_gb300 import serve


def test_poisson_arrivals_have_the_requested_mean():
    a = serve.poisson_arrivals(20000, 2.0, 1)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 2.0) < 4 * 2.0 / np.sqrt(len(gaps))
    assert abs(gaps.std() - 2.0) < 0.1          # exponential: std = mean


def test_percentiles():
    xs = list(range(1, 101))
    assert serve.percentile(xs, 50) == 50.5
    assert abs(serve.percentile(xs, 99) - 99.01) < 1e-9
    assert np.isnan(serve.percentile([], 50))


def test_served_trajectory_draws():
    trajs = serve.served_trajectories(n_traj=32, seed=7)
    Ns = {t.cfg.N for t in trajs}
    assert Ns <= {32, 64, 128}
    for t in trajs:
        assert 1024 <= t.cfg.walkers <= 8192 and t.cfg.walkers % 256 == 0
        assert 600 <= t.T_kelvin <= 3000
        rs = t.cfg.L / (4 * np.pi * t.cfg.N / 3) ** (1 / 3)
        assert 1.2 <= rs <= 1.5
