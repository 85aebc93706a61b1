"""Parity of the e-e-n-n Jastrow term (SI, U_{3+4}; FP64 form) with the oracle:
per configuration (ln|psi|, E_L and their nuclear derivatives, 1e-10) and a
Metropolis chain on the same Philox streams (positions, accumulators)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _fj(N, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (N, N)) * scale
    return 0.5 * (A + A.T)


def _rel_vec(a, b):
    return np.max(np.abs(a - b), axis=(-1, -2)) / np.max(np.abs(b), axis=(-1, -2))


@pytest.mark.parametrize("name,nconf", [("h16", 12), ("h64", 3)])
def test_eval_config_with_eenn_jastrow_matches_oracle(name, nconf):
    wl = synth.workload(name)
    fj = _fj(wl.N, 11)
    half = nconf // 2
    X = np.concatenate([synth.near_protons(half, wl.R, wl.N // 2, 0.7, wl.L, 3),
                        synth.random_electrons(nconf - half, wl.N, wl.L, 3)])
    sysg = q.QMCSystem(q.Config.from_workload(wl, walkers=max(nconf, 2), fj=fj), wl.R)
    g = sysg.eval_config(X, wl.R)
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, fj=fj)
    lp, el, dl, de = orc.eval_configs(osys, wl.R, X, derivs=True)
    assert np.all(np.abs(g["el"] - el) <= TOL * np.abs(el)), (g["el"], el)
    assert np.all(np.abs(g["lnpsi"] - lp) <= TOL * np.maximum(np.abs(lp), 1.0)), (g["lnpsi"], lp)
    assert np.all(_rel_vec(g["dlnpsi"], dl) <= TOL), _rel_vec(g["dlnpsi"], dl)
    assert np.all(_rel_vec(g["del_"], de) <= TOL), _rel_vec(g["del_"], de)
    # and the term is not negligible here
    osys0 = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)
    lp0, el0, _, _ = orc.eval_configs(osys0, wl.R, X, derivs=False)
    assert np.min(np.abs(lp - lp0)) > 1e-3


def test_fp64_chain_with_eenn_jastrow_reproduces_oracle():
    wl = synth.workload("h16", walkers=16, sweeps=3, warmup=2)
    fj = _fj(wl.N, 12)
    sysg = q.QMCSystem(q.Config.from_workload(wl, recompute_every=1, fj=fj), wl.R)
    res = sysg.energy_forces(wl.R)
    Xg, accg = sysg.walkers(), sysg.accumulators()
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, fj=fj)
    Xo, acco, ar = orc.vmc(osys, wl.R, W=16, n_sweeps=3, n_warmup=2, sigma=wl.sigma, seed=wl.seed)
    assert np.allclose(Xg, Xo, atol=1e-9, rtol=0)
    scale = np.maximum(np.abs(acco), 1.0)
    assert np.max(np.abs(accg - acco) / scale) < 1e-8
    ro = orc.reduce(acco, wl.N)
    assert abs(res["E"] - ro["E"]) < 1e-10 * abs(ro["E"])
    assert np.max(np.abs(res["f"] - ro["f"])) < 1e-8 * np.max(np.abs(ro["f"]))
    assert abs(res["accept"] - ar) < 1e-12


def _sampled(osys, R, n, seed, sweeps=8):
    X, _, _ = orc.vmc(osys, R, W=n, n_sweeps=1, n_warmup=sweeps, sigma=0.3, seed=seed, forces=False)
    return X


@pytest.mark.parametrize("name,nconf", [("h16", 12), ("h64", 4), ("h128", 2)])
def test_mixed_eval_config_with_eenn_jastrow_matches_oracle(name, nconf):
    """The mixed form (FP32 coefficients and Jastrow orbitals, tensor-core
    orbitals) with the e-e-n-n term on configurations drawn from |psi|^2 of the
    same wavefunction; 1e-4 norm-wise (E_L over the batch, forces per
    configuration, as in tests/test_gpu_h128_mixed.py)."""
    wl = synth.workload(name)
    fj = _fj(wl.N, 11)
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, fj=fj)
    X = _sampled(osys, wl.R, nconf, 7)
    sysg = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_MIXED, walkers=max(nconf, 2), fj=fj), wl.R)
    g = sysg.eval_config(X, wl.R)
    lp, el, dl, de = orc.eval_configs(osys, wl.R, X, derivs=True)
    tol = 1e-4
    assert np.max(np.abs(g["el"] - el)) <= tol * np.max(np.abs(el)), (g["el"], el)
    assert np.all(np.abs(g["lnpsi"] - lp) <= tol * np.maximum(np.abs(lp), 1.0)), (g["lnpsi"], lp)
    assert np.all(_rel_vec(g["dlnpsi"], dl) <= tol), _rel_vec(g["dlnpsi"], dl)
    assert np.all(_rel_vec(g["del_"], de) <= tol), _rel_vec(g["del_"], de)


def test_fp64_eval_config_with_eenn_jastrow_at_n128():
    wl = synth.workload("h128")
    fj = _fj(wl.N, 13)
    # one configuration: the oracle's U_{3+4} is a plain pair sum, O(N^5) over its dual-number passes
    X = synth.near_protons(1, wl.R, wl.N // 2, 0.7, wl.L, 5)
    sysg = q.QMCSystem(q.Config.from_workload(wl, walkers=2, fj=fj), wl.R)
    g = sysg.eval_config(X, wl.R)
    osys = orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, fj=fj)
    lp, el, dl, de = orc.eval_configs(osys, wl.R, X, derivs=True)
    assert np.all(np.abs(g["el"] - el) <= TOL * np.abs(el)), (g["el"], el)
    assert np.all(np.abs(g["lnpsi"] - lp) <= TOL * np.maximum(np.abs(lp), 1.0))
    assert np.all(_rel_vec(g["dlnpsi"], dl) <= TOL), _rel_vec(g["dlnpsi"], dl)
    assert np.all(_rel_vec(g["del_"], de) <= TOL), _rel_vec(g["del_"], de)


def test_mixed_chain_with_eenn_jastrow_statistically_matches_fp64():
    wl = synth.workload("h16", walkers=256, sweeps=120, warmup=30)
    fj = _fj(wl.N, 12)
    r = {}
    for prec in (q.QMC_FP64, q.QMC_MIXED):
        s = q.QMCSystem(q.Config.from_workload(wl, precision=prec, fj=fj), wl.R)
        r[prec] = s.energy_forces(wl.R)
        s.close()
    a, b = r[q.QMC_FP64], r[q.QMC_MIXED]
    err = np.hypot(a["E_err"], b["E_err"])
    assert abs(a["E"] - b["E"]) < 3 * err, (a["E"], b["E"], err)
    sig = np.sqrt(np.diag(a["S"]) + np.diag(b["S"]))
    z = np.abs(a["f"] - b["f"]) / sig
    assert np.mean(z < 3) >= 0.95 and np.max(z) < 4.03, z


def test_server_rejects_eenn_jastrow():
    wl = synth.workload("h16", walkers=4)
    srv = q.Server(1 << 30, 2)
    with pytest.raises(q.QMCError) as e:
        srv.add_trajectory(q.Config.from_workload(wl, precision=q.QMC_MIXED, fj=_fj(wl.N, 1)), wl.R, 1000.0, 0.1)
    assert e.value.code == -1
    srv.close()
