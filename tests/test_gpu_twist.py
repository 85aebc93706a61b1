"""Parity of the twisted-boundary-condition form (FP64, complex orbitals) of the
CUDA path with the FP64 CPU oracle, through the C ABI.

SI, basis section (phi(r + nL) = exp(i theta.n) phi(r), opposite twists for
opposite spins) and the main text's k-point average.  Tolerances as for the
FP64 form: 1e-10 relative per configuration; chains on the same Philox streams
reproduce the oracle's positions (1e-9) and accumulators (1e-8).
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu

MP4 = synth.monkhorst_pack(4)
DEV = "cuda"


def _osys(wl, theta):
    return orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, twist=np.asarray(theta, float))


def _configs(wl, n, seed):
    half = n // 2
    X1 = synth.near_protons(half, wl.R, wl.N // 2, 0.7, wl.L, seed)
    X2 = synth.random_electrons(n - half, wl.N, wl.L, seed)
    return np.concatenate([X1, X2])


def _rel_vec(a, b):
    return np.max(np.abs(a - b), axis=(-1, -2)) / np.max(np.abs(b), axis=(-1, -2))


@pytest.mark.parametrize("name,nconf,K", [("h16", 12, 1), ("h16", 12, 3), ("h64", 4, 2)])
def test_twisted_eval_config_matches_oracle(name, nconf, K):
    """ln|psi|, E_L, d ln|psi|/dR and dE_L/dR per configuration; configuration c
    takes twist c // (nconf / K) on both sides."""
    wl = synth.workload(name, walkers=nconf)
    tw = MP4[[7, 26, 53][:K]]
    X = _configs(wl, nconf, 31)
    sysg = q.QMCSystem(q.Config.from_workload(wl, twists=tw), wl.R)
    g = sysg.eval_config(X, wl.R)
    lp, el, dl, de = orc.eval_configs_twist(_osys(wl, tw[0]), wl.R, X, tw)
    tol = 1e-10
    assert np.all(np.abs(g["el"] - el) <= tol * np.maximum(np.abs(el), 1.0))
    assert np.all(np.abs(g["lnpsi"] - lp) <= tol * np.maximum(np.abs(lp), 1.0))
    assert np.all(_rel_vec(g["dlnpsi"], dl) < tol)
    assert np.all(_rel_vec(g["del_"], de) < tol)


def test_twisted_eval_config_full_size_values():
    """N = 128, 4 Gaussians per proton (3 Bloch images per axis, n = 64): E_L and
    ln|psi| per configuration (the oracle's R-derivatives are too slow here;
    N = 16 and 64 cover them)."""
    wl = synth.workload("h128", walkers=2)
    X = _configs(wl, 2, 12)
    tw = MP4[[45]]
    g = q.QMCSystem(q.Config.from_workload(wl, twists=tw), wl.R).eval_config(X, wl.R)
    lp, el, _, _ = orc.eval_configs_twist(_osys(wl, tw[0]), wl.R, X, tw, derivs=False)
    assert np.all(np.abs(g["el"] - el) <= 1e-10 * np.maximum(np.abs(el), 1.0))
    assert np.all(np.abs(g["lnpsi"] - lp) <= 1e-10 * np.maximum(np.abs(lp), 1.0))


@pytest.mark.parametrize("recompute_every", [1, 100])
def test_twisted_chain_reproduces_oracle(recompute_every):
    """Four twists, two walkers each, on the same Philox streams: identical
    accept sequences and positions, the same accumulators, and the twist-averaged
    E, f, S and acceptance of the oracle's reduction.  recompute_every = 100
    carries the complex Sherman-Morrison inverse (with the Bloch phase of every
    wrap into the box) through the whole call."""
    wl = synth.workload("h16", walkers=8, sweeps=3, warmup=2)
    tw = MP4[[5, 22, 41, 60]]
    sysg = q.QMCSystem(q.Config.from_workload(wl, twists=tw, recompute_every=recompute_every), wl.R)
    res = sysg.energy_forces(wl.R)
    Xg, accg = sysg.walkers(), sysg.accumulators()
    Xo, acco, ar, _ = orc.vmc_twists(_osys(wl, tw[0]), wl.R, tw, W=8, n_sweeps=3, n_warmup=2, sigma=wl.sigma,
                                     seed=wl.seed)
    assert np.allclose(Xg, Xo, atol=1e-9, rtol=0)
    scale = np.maximum(np.abs(acco), 1.0)
    assert np.max(np.abs(accg - acco) / scale) < 1e-8
    ro = orc.reduce_twists(acco, wl.N, 4)
    assert abs(res["E"] - ro["E"]) < 1e-10 * max(abs(ro["E"]), 1.0)
    assert abs(res["E_err"] - ro["E_err"]) < 1e-8 * ro["E_err"]
    assert res["Nc"] == ro["Nc"]
    assert np.max(np.abs(res["f"] - ro["f"])) < 1e-8 * np.max(np.abs(ro["f"]))
    assert np.max(np.abs(res["S"] - ro["S"])) < 1e-8 * np.max(np.abs(ro["S"]))
    assert abs(res["accept"] - ar) < 1e-12


def _fj(N, seed=5):
    A = np.random.default_rng(seed).uniform(-0.3, 0.3, (N, N))
    return 0.5 * (A + A.T)


def test_twisted_with_jastrow34_eval_config_matches_oracle():
    """The paper's production wavefunction: twisted orbitals with the e-e-n-n
    Jastrow term; per configuration as above, two twists."""
    wl = synth.workload("h16", walkers=8)
    tw = MP4[[9, 50]]
    fj = _fj(wl.N)
    X = _configs(wl, 8, 41)
    g = q.QMCSystem(q.Config.from_workload(wl, twists=tw, fj=fj), wl.R).eval_config(X, wl.R)
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, twist=tw[0], fj=fj)
    lp, el, dl, de = orc.eval_configs_twist(osys, wl.R, X, tw)
    assert np.all(np.abs(g["el"] - el) <= 1e-10 * np.maximum(np.abs(el), 1.0))
    assert np.all(np.abs(g["lnpsi"] - lp) <= 1e-10 * np.maximum(np.abs(lp), 1.0))
    assert np.all(_rel_vec(g["dlnpsi"], dl) < 1e-10)
    assert np.all(_rel_vec(g["del_"], de) < 1e-10)


def test_twisted_with_jastrow34_chain_reproduces_oracle():
    wl = synth.workload("h16", walkers=4, sweeps=3, warmup=2)
    tw = MP4[[9, 50]]
    fj = _fj(wl.N)
    sysg = q.QMCSystem(q.Config.from_workload(wl, twists=tw, fj=fj, recompute_every=100), wl.R)
    res = sysg.energy_forces(wl.R)
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, twist=tw[0], fj=fj)
    Xo, acco, ar, _ = orc.vmc_twists(osys, wl.R, tw, W=4, n_sweeps=3, n_warmup=2, sigma=wl.sigma, seed=wl.seed)
    assert np.allclose(sysg.walkers(), Xo, atol=1e-9, rtol=0)
    scale = np.maximum(np.abs(acco), 1.0)
    assert np.max(np.abs(sysg.accumulators() - acco) / scale) < 1e-8
    ro = orc.reduce_twists(acco, wl.N, 2)
    assert abs(res["E"] - ro["E"]) < 1e-10 * max(abs(ro["E"]), 1.0)
    assert np.max(np.abs(res["f"] - ro["f"])) < 1e-8 * np.max(np.abs(ro["f"]))
    assert abs(res["accept"] - ar) < 1e-12


def test_twist_average_of_single_twist_handles():
    """A two-twist handle equals the average of two one-twist handles that run
    the same walkers (the second one's Philox streams offset by W/K): E and f
    the means, S the sum over 4, E_err the root sum of squares over 2."""
    wl = synth.workload("h16", walkers=8, sweeps=4, warmup=2)
    tw = MP4[[11, 38]]
    both = q.QMCSystem(q.Config.from_workload(wl, twists=tw), wl.R).energy_forces(wl.R)
    parts = []
    for t in range(2):
        s = q.QMCSystem(q.Config.from_workload(wl, walkers=4, twists=tw[t:t + 1]), wl.R)
        s.set_walker_offset(4 * t)
        parts.append(s.energy_forces(wl.R))
    assert abs(both["E"] - 0.5 * (parts[0]["E"] + parts[1]["E"])) < 1e-12 * max(abs(both["E"]), 1.0)
    assert abs(both["E_err"] - 0.5 * np.hypot(parts[0]["E_err"], parts[1]["E_err"])) < 1e-12 * both["E_err"]
    assert np.max(np.abs(both["f"] - 0.5 * (parts[0]["f"] + parts[1]["f"]))) < 1e-12 * np.max(np.abs(both["f"]))
    assert np.max(np.abs(both["S"] - 0.25 * (parts[0]["S"] + parts[1]["S"]))) < 1e-12 * np.max(np.abs(both["S"]))
    assert both["Nc"] == parts[0]["Nc"] + parts[1]["Nc"]


def test_twist_sharded_partials_combine_to_the_single_handle():
    """The partial / combine steps of a TwistGroup on one GPU: two two-twist
    handles on the same walkers (the second one's Philox streams offset by
    W/2), their contributions summed as the all-reduce would, give the result
    of one four-twist handle."""
    import torch
    wl = synth.workload("h16", walkers=8, sweeps=3, warmup=2)
    tw = MP4[[3, 20, 44, 61]]
    n_out = 4 + 3 * wl.N + 9 * wl.N * wl.N
    R_dev = torch.tensor(wl.R, dtype=torch.float64, device=DEV)
    ref = torch.zeros(n_out, dtype=torch.float64, device=DEV)
    one = q.QMCSystem(q.Config.from_workload(wl, twists=tw), wl.R)
    one.energy_forces_device(R_dev, ref)
    one.sync()
    total = torch.zeros(n_out, dtype=torch.float64, device=DEV)
    systems = []
    for r in range(2):
        s = q.QMCSystem(q.Config.from_workload(wl, walkers=4, twists=q.twist_slice(tw, r, 2)), wl.R)
        s.set_walker_offset(4 * r)
        o = torch.zeros(n_out, dtype=torch.float64, device=DEV)
        part = torch.zeros(n_out, dtype=torch.float64, device=DEV)
        s.energy_forces_device(R_dev, o)
        s.twist_partial_device(o, part)
        s.sync()
        total += part
        systems.append(s)
    out = torch.zeros(n_out, dtype=torch.float64, device=DEV)
    if DEV == "cuda":
        torch.cuda.synchronize()      # the handles run on their own streams
    systems[0].twist_combine_device(total, 4, out)
    systems[0].sync()
    a, b = out.cpu().numpy(), ref.cpu().numpy()
    N3 = 3 * wl.N
    assert abs(a[0] - b[0]) < 1e-12 * max(abs(b[0]), 1.0) and abs(a[1] - b[1]) < 1e-12 * b[1]
    assert a[2] == b[2] and abs(a[3] - b[3]) < 1e-14
    assert np.max(np.abs(a[4:4 + N3] - b[4:4 + N3])) < 1e-12 * np.max(np.abs(b[4:4 + N3]))
    assert np.max(np.abs(a[4 + N3:] - b[4 + N3:])) < 1e-12 * np.max(np.abs(b[4 + N3:]))
    with pytest.raises(q.QMCError):
        systems[0].twist_combine_device(total, 1, out)          # fewer twists than the handle's own


def test_twisted_handles_reject_sharding():
    import torch
    wl = synth.workload("h16", walkers=4)
    s = q.QMCSystem(q.Config.from_workload(wl, twists=MP4[[0, 1]]), wl.R)
    R = torch.tensor(wl.R, dtype=torch.float64, device="cuda")
    sums = torch.zeros(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QMCError):
        s.shard_sample_device(R, sums)
