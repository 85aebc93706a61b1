"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 form 1e-10 relative, mixed form 1e-4 relative (E_L and
ln|psi| relative to their own magnitude; force vectors relative to the
largest component of the oracle's vector).  Chains on the same Philox
streams must reproduce the oracle's walker positions and accumulators.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {q.QMC_FP64: 1e-10, q.QMC_MIXED: 1e-4}


def _oracle_sys(wl):
    return orc.System(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C)


def _configs(wl, n, seed):
    """Half scattered around the protons, half uniform in the box (any configuration)."""
    half = n // 2
    X1 = synth.near_protons(half, wl.R, wl.N // 2, 0.7, wl.L, seed)
    X2 = synth.random_electrons(n - half, wl.N, wl.L, seed)
    return np.concatenate([X1, X2])


def _sampled(wl, n, seed, sweeps=12):
    """Configurations distributed as |psi|^2, drawn by the oracle's own Metropolis chains.
    The mixed form is held to 1e-4 on these: uniform configurations with nearly
    coincident same-spin electrons (Slater condition numbers ~1e3 and above,
    which |psi|^2 suppresses) amplify the FP32 input rounding beyond it."""
    X, _, _ = orc.vmc(_oracle_sys(wl), wl.R, W=n, n_sweeps=1, n_warmup=sweeps, sigma=wl.sigma, seed=seed,
                      forces=False)
    return X


def _rel_vec(a, b):
    return np.max(np.abs(a - b), axis=(-1, -2)) / np.max(np.abs(b), axis=(-1, -2))


@pytest.mark.parametrize("name,nconf,prec", [
    ("h16", 12, q.QMC_FP64), ("h16", 12, q.QMC_MIXED),
    ("h64", 4, q.QMC_FP64), ("h64", 4, q.QMC_MIXED),
])
def test_eval_config_matches_oracle(name, nconf, prec):
    wl = synth.workload(name)
    X = _configs(wl, nconf, 5) if prec == q.QMC_FP64 else _sampled(wl, nconf, 5)
    sysg = q.QMCSystem(q.Config.from_workload(wl, precision=prec, walkers=max(nconf, 2)), wl.R)
    g = sysg.eval_config(X, wl.R)
    lp, el, dl, de = orc.eval_configs(_oracle_sys(wl), wl.R, X, derivs=True)
    tol = TOL[prec]
    assert np.all(np.abs(g["el"] - el) <= tol * np.abs(el)), (g["el"], el)
    assert np.all(np.abs(g["lnpsi"] - lp) <= tol * np.maximum(np.abs(lp), 1.0)), (g["lnpsi"], lp)
    assert np.all(_rel_vec(g["dlnpsi"], dl) <= tol), _rel_vec(g["dlnpsi"], dl)
    assert np.all(_rel_vec(g["del_"], de) <= tol), _rel_vec(g["del_"], de)


def test_eval_config_full_size_fp64():
    """The N=128, 4-Gaussian headline system in the FP64 form, any configuration
    (the mixed form at this size: tests/test_gpu_h128_mixed.py)."""
    wl = synth.workload("h128", walkers=2)
    X = _configs(wl, 2, 17)
    sysg = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_FP64), wl.R)
    g = sysg.eval_config(X, wl.R)
    lp, el, dl, de = orc.eval_configs(_oracle_sys(wl), wl.R, X, derivs=True)
    tol = TOL[q.QMC_FP64]
    assert np.all(np.abs(g["el"] - el) <= tol * np.abs(el)), (g["el"], el)
    assert np.all(np.abs(g["lnpsi"] - lp) <= tol * np.abs(lp))
    assert np.all(_rel_vec(g["dlnpsi"], dl) <= tol), _rel_vec(g["dlnpsi"], dl)
    assert np.all(_rel_vec(g["del_"], de) <= tol), _rel_vec(g["del_"], de)


def test_tensor_cores_only_for_n128_four_gaussians():
    """The tcgen05 kernels are offered for N = 128 with 4 Gaussians per
    nucleus only; smaller systems run the SIMT kernels and refuse the option."""
    for name in ("h16", "h64"):
        wl = synth.workload(name)
        s = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_MIXED, walkers=4), wl.R)
        with pytest.raises(q.QMCError):
            s.set_tensor_cores(True)
        with pytest.raises(q.QMCError):
            s.set_tc_adjoint(True)
        s.close()
    wl = synth.workload("h128")
    s = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_MIXED, walkers=4), wl.R)
    s.set_tensor_cores(True)
    s.set_tc_adjoint(True)
    s.close()


def test_tensor_core_orbitals_match_simt():
    """The tcgen05 (2xTF32) orbital contraction agrees with the SIMT FP32 one."""
    wl = synth.workload("h128")
    X = _sampled(wl, 4, 21, sweeps=4)
    s = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_MIXED, walkers=4), wl.R)
    tc = s.eval_config(X, wl.R)
    s.set_tensor_cores(False)
    simt = s.eval_config(X, wl.R)
    # both are mixed-form evaluations held to 1e-4 of the oracle (norm-wise)
    # at N = 128, so they are compared at that tolerance
    assert np.abs(tc["el"] - simt["el"]).max() <= 1e-4 * np.abs(simt["el"]).max()
    assert np.all(np.abs(tc["lnpsi"] - simt["lnpsi"]) <= 1e-4 * np.abs(simt["lnpsi"]))
    assert np.all(_rel_vec(tc["del_"], simt["del_"]) <= 1e-4)
    assert np.all(_rel_vec(tc["dlnpsi"], simt["dlnpsi"]) <= 1e-4)


@pytest.mark.parametrize("name,nconf", [("h128", 2)])
def test_tensor_core_adjoint_matches_simt(name, nconf):
    """The tcgen05 form of the orbital force terms (Z = C G, P = C G Y G and
    the basis-derivative epilogue) agrees with the SIMT FP32 form."""
    wl = synth.workload(name)
    X = _sampled(wl, nconf, 23, sweeps=4)
    s = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_MIXED, walkers=nconf), wl.R)
    tc = s.eval_config(X, wl.R)
    s.set_tc_adjoint(False)
    simt = s.eval_config(X, wl.R)
    # E_L and ln psi do not depend on this choice; the two measure-kernel
    # builds may round their FP32 pair sums differently (FP32-level)
    assert np.all(np.abs(tc["el"] - simt["el"]) <= 1e-6 * np.abs(simt["el"]))
    assert np.all(np.abs(tc["lnpsi"] - simt["lnpsi"]) <= 1e-6 * np.abs(simt["lnpsi"]))
    assert np.all(_rel_vec(tc["dlnpsi"], simt["dlnpsi"]) <= 2e-5), _rel_vec(tc["dlnpsi"], simt["dlnpsi"])
    assert np.all(_rel_vec(tc["del_"], simt["del_"]) <= 2e-5), _rel_vec(tc["del_"], simt["del_"])


def test_tensor_core_adjoint_chain_matches_simt():
    """More walkers than SMs (each persistent CTA takes several walkers), four
    Gaussians (the A-operand refill path): same chain, forces and S agree."""
    wl = synth.workload("h128", walkers=320, sweeps=2, warmup=2)
    cfg = q.Config.from_workload(wl, precision=q.QMC_MIXED)
    ra = q.QMCSystem(cfg, wl.R).energy_forces(wl.R)
    b = q.QMCSystem(cfg, wl.R)
    b.set_tc_adjoint(False)
    rb = b.energy_forces(wl.R)
    assert abs(ra["E"] - rb["E"]) <= 1e-6 * abs(rb["E"]) and ra["accept"] == rb["accept"]
    assert np.max(np.abs(ra["f"] - rb["f"])) <= 2e-5 * np.max(np.abs(rb["f"]))
    assert np.max(np.abs(ra["S"] - rb["S"])) <= 1e-4 * np.max(np.abs(rb["S"]))


def test_walker_start_matches_oracle():
    wl = synth.workload("h16", walkers=32)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    Xo = orc.init_walkers(_oracle_sys(wl), wl.R, 32, wl.seed)
    assert np.allclose(sysg.walkers(), Xo, atol=1e-12, rtol=0)


def test_fp64_chain_reproduces_oracle():
    """Same Philox streams: identical accept sequences, positions and sums."""
    wl = synth.workload("h16", walkers=16, sweeps=3, warmup=2)
    cfg = q.Config.from_workload(wl, recompute_every=1)
    sysg = q.QMCSystem(cfg, wl.R)
    res = sysg.energy_forces(wl.R)
    Xg, accg = sysg.walkers(), sysg.accumulators()
    Xo, acco, ar = orc.vmc(_oracle_sys(wl), wl.R, W=16, n_sweeps=3, n_warmup=2, sigma=wl.sigma, seed=wl.seed)
    assert np.allclose(Xg, Xo, atol=1e-9, rtol=0)
    scale = np.maximum(np.abs(acco), 1.0)
    assert np.max(np.abs(accg - acco) / scale) < 1e-8
    ro = orc.reduce(acco, wl.N)
    assert abs(res["E"] - ro["E"]) < 1e-10 * abs(ro["E"])
    assert np.max(np.abs(res["f"] - ro["f"])) < 1e-8 * np.max(np.abs(ro["f"]))
    assert np.max(np.abs(res["S"] - ro["S"])) < 1e-8 * np.max(np.abs(ro["S"]))
    assert abs(res["accept"] - ar) < 1e-12


def test_mixed_chain_statistically_matches_fp64():
    wl = synth.workload("h16", walkers=256, sweeps=120, warmup=30)
    r64 = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_FP64), wl.R).energy_forces(wl.R)
    r32 = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_MIXED), wl.R).energy_forces(wl.R)
    err = np.hypot(r64["E_err"], r32["E_err"])
    assert abs(r64["E"] - r32["E"]) < 3 * err, (r64["E"], r32["E"], err)
    # 48 force components: every |z| below the Sidak threshold of a 0.27 %
    # family-wise rate (|z| < 4.03), at least 95 % within 3 sigma
    sig = np.sqrt(np.diag(r64["S"]) + np.diag(r32["S"]))
    z = np.abs(r64["f"] - r32["f"]) / sig
    assert np.mean(z < 3) >= 0.95 and np.max(z) < 4.03, z


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T / n + 0.3 * np.eye(n)


@pytest.mark.parametrize("mode", [q.QMC_S_IDENTITY, q.QMC_S_COV])
def test_langevin_step_matches_oracle(mode):
    wl = synth.workload("h16", walkers=2)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    n = 3 * wl.N
    rng = np.random.default_rng(4)
    R0 = wl.R.ravel().copy()
    T = 1000.0 * synth.K_B_HARTREE_PER_KELVIN
    alpha = 0.0 if mode == q.QMC_S_IDENTITY else 37.0
    Rprev, Sprev = R0.copy(), None
    R = R0.copy()
    for step in range(3):
        f = rng.standard_normal(n)
        S = np.eye(n) if mode == q.QMC_S_IDENTITY else _spd(n, 10 + step) * 1e-3
        if Sprev is None:
            Sprev = S
        xi = orc.langevin_noise(wl.seed, step, n)
        Ro = orc.langevin(R, Rprev, f, S, Sprev, T, 0.1, alpha, xi, box=wl.L)
        Rg = sysg.langevin_step(R, f, S if mode == q.QMC_S_COV else None, 1000.0, 0.1, s_mode=mode, alpha=alpha)
        assert np.max(np.abs(Rg - Ro)) < 1e-10, (step, np.max(np.abs(Rg - Ro)))
        Rprev, Sprev, R = R, S, Ro


@pytest.mark.parametrize("scheme,noise_corr", [(q.QMC_LV_FAST, False), (q.QMC_LV_NOROGNA, False),
                                               (q.QMC_LV_ADOPTED, True), (q.QMC_LV_FAST, True)])
def test_langevin_integrator_variants_match_oracle(scheme, noise_corr):
    wl = synth.workload("h16", walkers=2)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    sysg.set_integrator(scheme)
    sysg.set_noise_correction(noise_corr)
    n = 3 * wl.N
    rng = np.random.default_rng(5)
    T_K, delta, alpha = 1500.0, 0.004, 41.0
    T = T_K * synth.K_B_HARTREE_PER_KELVIN
    R = wl.R.ravel().copy()
    Rprev, Sprev = R.copy(), None
    oscheme = {q.QMC_LV_ADOPTED: orc.LV_ADOPTED, q.QMC_LV_FAST: orc.LV_FAST, q.QMC_LV_NOROGNA: orc.LV_NOROGNA}
    for step in range(3):
        f = rng.standard_normal(n)
        S = _spd(n, 20 + step) * 1e-3
        if Sprev is None:
            Sprev = S
        xi = orc.langevin_noise(wl.seed, step, n)
        Ro = orc.langevin(R, Rprev, f, S, Sprev, T, delta, alpha, xi, noise_correction=noise_corr, box=wl.L,
                          scheme=oscheme[scheme])
        Rg = sysg.langevin_step(R, f, S, T_K, delta, s_mode=q.QMC_S_COV, alpha=alpha)
        assert np.max(np.abs(Rg - Ro)) < 1e-10, (step, np.max(np.abs(Rg - Ro)))
        Rprev, Sprev, R = R, S, Ro
    if noise_corr:      # Delta >= 2 T leaves no temperature to correct with
        with pytest.raises(q.QMCError) as e:
            sysg.langevin_step(R, np.zeros(n), np.eye(n), T_K, 2.5 * T, s_mode=q.QMC_S_COV, alpha=alpha)
        assert e.value.code == -1
    with pytest.raises(q.QMCError):
        sysg.set_integrator(7)


def test_langevin_first_simplified_scheme_matches_oracle():
    """Eq. smartMarkov in its two halves (predict y, the caller's S(y), correct)."""
    wl = synth.workload("h16", walkers=2)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    n = 3 * wl.N
    rng = np.random.default_rng(6)
    T_K, delta = 1500.0, 0.004
    T = T_K * synth.K_B_HARTREE_PER_KELVIN
    R = wl.R.ravel().copy()
    for step in range(3):
        f = rng.standard_normal(n)
        S, Sy = _spd(n, 30 + step) * 1e-3, _spd(n, 40 + step) * 1e-3
        xi = orc.langevin_noise(wl.seed, step, n)
        yo = orc.langevin_first_predict(R, S, T, delta, xi)
        yg = sysg.langevin_first_predict(R, f, S, T_K, delta)
        assert np.max(np.abs(yg - yo)) < 1e-10, (step, np.max(np.abs(yg - yo)))
        Ro = orc.langevin_first_correct(R, f, S, Sy, yo, delta, box=wl.L)
        Rg = sysg.langevin_first_correct(yg, Sy)
        assert np.max(np.abs(Rg - Ro)) < 1e-10, (step, np.max(np.abs(Rg - Ro)))
        R = Ro
    with pytest.raises(q.QMCError) as e:          # no pending predict
        sysg.langevin_first_correct(R, np.eye(n))
    assert e.value.code == -1
    with pytest.raises(q.QMCError) as e:
        sysg.langevin_first_predict(R, np.zeros(n), -np.eye(n), T_K, delta)
    assert e.value.code == -4


def test_autograd_function_backward_is_minus_force():
    import torch
    wl = synth.workload("h16", walkers=64, sweeps=10, warmup=5)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    EF = q.energy_forces_function()
    R = torch.tensor(wl.R, dtype=torch.float64, requires_grad=True)
    E = EF.apply(R, sysg)
    E.backward()
    sys2 = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    ref = sys2.energy_forces(wl.R)
    assert abs(float(E.detach()) - ref["E"]) < 1e-12 * abs(ref["E"])
    assert np.allclose(R.grad.numpy().ravel(), -ref["f"], rtol=0, atol=1e-12 * np.max(np.abs(ref["f"])))


def test_errors_are_reported():
    wl = synth.workload("h16", walkers=2)
    sysg = q.QMCSystem(q.Config.from_workload(wl), wl.R)
    n = 3 * wl.N
    S = -np.eye(n)
    with pytest.raises(q.QMCError) as e:
        sysg.langevin_step(wl.R, np.zeros(n), S, 1000.0, 0.1, s_mode=q.QMC_S_COV, alpha=1.0)
    assert e.value.code == -4
    with pytest.raises(q.QMCError) as e:
        q.QMCSystem(q.Config.from_workload(wl, walkers=1), wl.R)
    assert e.value.code == -1


def test_adjoint_forces_vs_finite_differences_of_oracle_energy():
    """N=64 (2 Gaussians/proton), 8 seeded |psi|^2 configurations: the GPU's
    adjoint dE_L/dR and d ln psi/dR against central differences (h = 1e-4 bohr)
    of the oracle's E_L and ln|psi|, on a sample of nuclear coordinates."""
    wl = synth.workload("h64")
    X = _sampled(wl, 8, 41, sweeps=6)
    sysg = q.QMCSystem(q.Config.from_workload(wl, precision=q.QMC_FP64, walkers=8), wl.R)
    g = sysg.eval_config(X, wl.R)
    osys = _oracle_sys(wl)
    h = 1e-4
    rng = np.random.default_rng(3)
    coords = [(int(a), int(m)) for a, m in zip(rng.integers(0, wl.N, 6), rng.integers(0, 3, 6))]
    for a, m in coords:
        Rp = wl.R.copy(); Rp[a, m] += h
        Rm = wl.R.copy(); Rm[a, m] -= h
        lp_p, el_p, _, _ = orc.eval_configs(osys, Rp, X, derivs=False)
        lp_m, el_m, _, _ = orc.eval_configs(osys, Rm, X, derivs=False)
        fd_e = (el_p - el_m) / (2 * h)
        fd_l = (lp_p - lp_m) / (2 * h)
        scale_e = np.max(np.abs(g["del_"]), axis=(1, 2))
        scale_l = np.max(np.abs(g["dlnpsi"]), axis=(1, 2))
        assert np.all(np.abs(g["del_"][:, a, m] - fd_e) <= 1e-5 * scale_e), (a, m, g["del_"][:, a, m], fd_e)
        assert np.all(np.abs(g["dlnpsi"][:, a, m] - fd_l) <= 1e-5 * scale_l), (a, m)


def test_small_system_md_end_to_end_both_forms_and_both_S():
    """N=16, 256 walkers x 200 sweeps: E, 48 forces and their covariance, then 10
    Langevin steps at T = 1000 K, Delta = 0.1 with S = I and with S = Cov(f)."""
    wl = synth.workload("h16")
    res = {}
    for prec in (q.QMC_FP64, q.QMC_MIXED):
        for mode in (q.QMC_S_IDENTITY, q.QMC_S_COV):
            s = q.QMCSystem(q.Config.from_workload(wl, precision=prec, warmup=20, warmup_cont=5), wl.R)
            R = wl.R.copy()
            Es = []
            for step in range(10):
                r = s.energy_forces(R)
                assert np.isfinite(r["E"]) and np.all(np.isfinite(r["f"])) and r["f"].shape == (48,)
                S = r["S"]
                assert np.allclose(S, S.T) and np.all(np.linalg.eigvalsh(S) > 0)
                assert r["Nc"] == 256 * 200 and 0.3 < r["accept"] < 0.95
                Rn = s.langevin_step(R, r["f"], S if mode == q.QMC_S_COV else None, 1000.0, 0.1, s_mode=mode)
                disp = Rn.reshape(-1, 3) - R
                disp -= wl.L * np.round(disp / wl.L)
                assert np.all(np.abs(disp) < 0.5 * wl.L)
                R = Rn.reshape(-1, 3)
                Es.append((r["E"], r["E_err"]))
            res[(prec, mode)] = Es
            s.close()
    # first MD step (same nuclei): FP64 and mixed forms agree within their error bars
    for mode in (q.QMC_S_IDENTITY, q.QMC_S_COV):
        (e64, s64), (e32, s32) = res[(q.QMC_FP64, mode)][0], res[(q.QMC_MIXED, mode)][0]
        assert abs(e64 - e32) < 3 * np.hypot(s64, s32)
