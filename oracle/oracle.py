"""ctypes harness around the FP64 CPU oracle (oracle/qmc_oracle.cpp).

Test infrastructure only: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py may use it; the
product library never does.  Every numerical step lives in the C++ source,
which cites the passages of Sorella & Mazzola (arXiv:1605.08423) it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmc_oracle.cpp")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libqmc_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/lib/libqmc_oracle.so (g++, OpenMP, IEEE FP64)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("n_up", C.c_int32), ("n_dn", C.c_int32), ("n_orb", C.c_int32),
        ("n_gauss", C.c_int32), ("periodic", C.c_int32), ("mmax", C.c_int32), ("pad_", C.c_int32),
        ("L", C.c_double), ("b_ee", C.c_double), ("b_ep", C.c_double), ("Z", C.c_double),
        ("Zj", C.c_double), ("kappa", C.c_double),
        ("zeta", C.POINTER(C.c_double)), ("coeff", C.POINTER(C.c_double)),
        ("zeta_j", C.c_double), ("fj", C.POINTER(C.c_double)),
        ("twist", C.POINTER(C.c_double)),
    ]


class ChainArgs(C.Structure):
    _fields_ = [
        ("W", C.c_int32), ("n_sweeps", C.c_int32), ("n_warmup", C.c_int32),
        ("measure_every", C.c_int32), ("init_walkers", C.c_int32), ("forces", C.c_int32),
        ("md_step", C.c_uint32), ("pad_", C.c_int32), ("sigma", C.c_double), ("seed", C.c_uint64),
    ]


class ToyArgs(C.Structure):
    _fields_ = [
        ("k", C.c_double), ("a", C.c_double), ("T", C.c_double), ("delta", C.c_double),
        ("lam", C.c_double), ("mu", C.c_double), ("alpha", C.c_double),
        ("scheme", C.c_int32), ("s_mode", C.c_int32), ("n_steps", C.c_int32), ("n_burn", C.c_int32),
        ("seed", C.c_uint64),
    ]


_dp = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.orc_uniform.restype = C.c_double
        L.orc_uniform.argtypes = [C.c_uint64] + [C.c_uint32] * 4
        L.orc_normal.restype = C.c_double
        L.orc_normal.argtypes = [C.c_uint64] + [C.c_uint32] * 4
        L.orc_ewald.restype = C.c_double
        L.orc_ewald.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_int, C.c_int]
        L.orc_eval_config.restype = C.c_int
        L.orc_eval_config.argtypes = [C.POINTER(Params), _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_eval_configs.restype = C.c_int
        L.orc_eval_configs.argtypes = [C.POINTER(Params), _dp, C.c_int, _dp, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_init_walkers.argtypes = [C.POINTER(Params), _dp, C.c_int, C.c_uint64, _dp]
        L.orc_jastrow_delta.restype = C.c_double
        L.orc_jastrow_delta.argtypes = [C.POINTER(Params), _dp, _dp, C.c_int, _dp]
        L.orc_vmc_v.restype = None
        L.orc_vmc_v.argtypes = [C.POINTER(Params), _dp, C.POINTER(ChainArgs), _dp, _dp, _dp, C.POINTER(C.c_longlong),
                                C.POINTER(C.c_longlong)]
        L.orc_pressure.restype = None
        L.orc_pressure.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double, _dp]
        L.orc_slater_matrices.restype = None
        L.orc_slater_matrices.argtypes = [C.POINTER(Params), _dp, _dp, _dp]
        L.orc_vmc.argtypes = [C.POINTER(Params), _dp, C.POINTER(ChainArgs), _dp, _dp,
                              C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.orc_reduce.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_langevin.restype = C.c_int
        L.orc_langevin.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                   C.c_double, _dp, C.c_int, C.c_double, C.c_int, _dp]
        L.orc_langevin_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_int, _dp]
        L.orc_langevin_first_predict.restype = C.c_int
        L.orc_langevin_first_predict.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, _dp, _dp]
        L.orc_langevin_first_correct.restype = C.c_int
        L.orc_langevin_first_correct.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double, _dp]
        L.orc_num_threads.restype = C.c_int
        L.orc_toy_eval.argtypes = [C.POINTER(ToyArgs), C.c_double, C.c_double, _dp]
        L.orc_toy_step.restype = C.c_int
        L.orc_toy_step.argtypes = [C.POINTER(ToyArgs), _dp, _dp, _dp, _dp]
        L.orc_toy_run.argtypes = [C.POINTER(ToyArgs), C.c_int, _dp, _dp]
        L.orc_toy_noise.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, _dp]
        L.orc_toy_run_ids.argtypes = [C.POINTER(ToyArgs), C.c_int, C.POINTER(C.c_int), _dp, _dp]
        L.orc_reduce_twists.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_empirical_energy.restype = C.c_double
        L.orc_empirical_energy.argtypes = [C.c_int, C.c_double, _dp, C.c_double]
        L.orc_empirical_s.argtypes = [C.c_int, C.c_double, _dp, C.c_double, C.c_double, _dp]
        L.orc_bloch_images.restype = C.c_int
        L.orc_bloch_images.argtypes = [C.POINTER(Params)]
        L.orc_bloch_gaussian.argtypes = [C.c_double, _dp, _dp, C.c_double, _dp, C.c_int, _dp]
        L.orc_eval_config_twist.restype = C.c_int
        L.orc_eval_config_twist.argtypes = [C.POINTER(Params), _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_eval_configs_twist.restype = C.c_int
        L.orc_eval_configs_twist.argtypes = [C.POINTER(Params), _dp, C.c_int, _dp, C.c_int, _dp, C.c_int, _dp, _dp,
                                             _dp, _dp]
        L.orc_vmc_twists.restype = C.c_int
        L.orc_vmc_twists.argtypes = [C.POINTER(Params), _dp, C.POINTER(ChainArgs), C.c_int, _dp, _dp, _dp, _dp,
                                     C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


@dataclass
class System:
    """Wavefunction / Hamiltonian parameters of one system (oracle side)."""
    N: int
    L: float
    zeta: np.ndarray          # [G]
    coeff: np.ndarray         # [N*G][n_orb]
    n_up: int | None = None
    n_dn: int | None = None
    b_ee: float = 1.0
    b_ep: float = 1.0
    Z: float = 1.0
    Zj: float | None = None
    kappa: float | None = None
    mmax: int = 6
    periodic: bool = True
    zeta_j: float = 0.7933844        # exponent of the U_{3+4} Jastrow orbitals (SI's Z_1 = Z_2)
    fj: np.ndarray | None = None     # [N][N] symmetric U_{3+4} coefficients; None: term off
    twist: np.ndarray | None = None  # [3] twist theta of the spin-up orbitals (Bloch Gaussians); None: real form

    def cparams(self) -> Params:
        self._zeta = np.ascontiguousarray(self.zeta, dtype=np.float64)
        self._coeff = np.ascontiguousarray(self.coeff, dtype=np.float64)
        self._fj = None if self.fj is None else np.ascontiguousarray(self.fj, dtype=np.float64).reshape(self.N, self.N)
        n_up = self.N // 2 if self.n_up is None else self.n_up
        n_dn = self.N - n_up if self.n_dn is None else self.n_dn
        kappa = 5.0 / self.L if self.kappa is None else self.kappa
        self._twist = None if self.twist is None else np.ascontiguousarray(self.twist, dtype=np.float64).reshape(3)
        return Params(self.N, n_up, n_dn, self._coeff.shape[1], len(self._zeta), int(self.periodic),
                      self.mmax, 0, self.L, self.b_ee, self.b_ep, self.Z,
                      self.Z if self.Zj is None else self.Zj, kappa,
                      _ptr(self._zeta), _ptr(self._coeff), self.zeta_j,
                      _ptr(self._fj) if self._fj is not None else C.cast(None, _dp),
                      _ptr(self._twist) if self._twist is not None else C.cast(None, _dp))

    @property
    def n_elec(self) -> int:
        n_up = self.N // 2 if self.n_up is None else self.n_up
        n_dn = self.N - n_up if self.n_dn is None else self.n_dn
        return n_up + n_dn


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def ewald(q, pos, L, kappa, mmax, background=False) -> float:
    q = np.ascontiguousarray(q, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    return lib().orc_ewald(len(q), _ptr(q), _ptr(pos), L, kappa, mmax, int(background))


def eval_config(sys: System, R, X, derivs=False):
    """Return dict(lnpsi, sign, el, ekin, epot, grad[Ne,3], dlnpsi[N,3], del[N,3])."""
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    sc = np.zeros(5)
    grad = np.zeros((sys.n_elec, 3))
    dl = np.zeros((sys.N, 3))
    de = np.zeros((sys.N, 3))
    rc = lib().orc_eval_config(C.byref(p), _ptr(R), _ptr(X), int(derivs), _ptr(sc), _ptr(grad), _ptr(dl), _ptr(de))
    if rc != 0:
        raise ValueError("singular Slater block")
    out = dict(lnpsi=sc[0], sign=int(sc[1]), el=sc[2], ekin=sc[3], epot=sc[4], grad=grad)
    if derivs:
        out.update(dlnpsi=dl, del_=de)
    return out


def eval_configs(sys: System, R, X, derivs=True):
    """Walker-parallel evaluation: X [nconf, Ne, 3] -> lnpsi, el, dlnpsi, del."""
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[0]
    lp = np.zeros(n); el = np.zeros(n)
    dl = np.zeros((n, sys.N, 3)); de = np.zeros((n, sys.N, 3))
    rc = lib().orc_eval_configs(C.byref(p), _ptr(R), n, _ptr(X), int(derivs), _ptr(lp), _ptr(el), _ptr(dl), _ptr(de))
    if rc != 0:
        raise ValueError("singular Slater block")
    return lp, el, dl, de


def slater_matrices(sys: System, R, X):
    """The two Slater blocks (A_up, A_dn), A[i][j] = phi_j(r_i), at one configuration X [Ne, 3]."""
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    nu = p.n_up
    out = np.zeros((sys.n_elec, p.n_orb))
    lib().orc_slater_matrices(C.byref(p), _ptr(R), _ptr(X), _ptr(out))
    return out[:nu], out[nu:]


def slater_condition(sys: System, R, X) -> float:
    """Largest 2-norm condition number of the two Slater blocks at X [Ne, 3]."""
    return max(float(np.linalg.cond(A)) for A in slater_matrices(sys, R, X))


def jastrow_delta(sys: System, R, X, i, xn) -> float:
    """U(X with electron i at xn) - U(X), as the oracle's Metropolis step computes it."""
    p = sys.cparams()
    R, X, xn = (np.ascontiguousarray(a, dtype=np.float64) for a in (R, X, xn))
    return lib().orc_jastrow_delta(C.byref(p), _ptr(R), _ptr(X), int(i), _ptr(xn))


def init_walkers(sys: System, R, W, seed):
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    X = np.zeros((W, sys.n_elec, 3))
    lib().orc_init_walkers(C.byref(p), _ptr(R), W, seed, _ptr(X))
    return X


def vmc(sys: System, R, *, W, n_sweeps, n_warmup, measure_every=1, sigma=0.3, seed=1, md_step=0,
        X=None, forces=True, potential=False):
    """Run W Metropolis chains; returns (X, acc[W, 3+9N], accept_ratio), and with
    potential=True also vacc[W] (each walker's sum of the sampled V_L) as a fourth item."""
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    init = X is None
    Xa = np.zeros((W, sys.n_elec, 3)) if init else np.array(X, dtype=np.float64, copy=True)
    acc = np.zeros((W, 3 + 9 * sys.N))
    vacc = np.zeros(W)
    ca = ChainArgs(W, n_sweeps, n_warmup, measure_every, int(init), int(forces), md_step, 0, sigma, seed)
    na = C.c_longlong(0); nt = C.c_longlong(0)
    lib().orc_vmc_v(C.byref(p), _ptr(R), C.byref(ca), _ptr(Xa), _ptr(acc), _ptr(vacc), C.byref(na), C.byref(nt))
    ar = na.value / nt.value if nt.value else 0.0
    return (Xa, acc, ar, vacc) if potential else (Xa, acc, ar)


def pressure(acc, vacc, N, omega, T_nuc=0.0) -> dict:
    """Virial pressure of a cubic cell from the chains' accumulators (hartree / bohr^3)."""
    acc = np.ascontiguousarray(acc, dtype=np.float64)
    vacc = np.ascontiguousarray(vacc, dtype=np.float64)
    out = np.zeros(5)
    lib().orc_pressure(acc.shape[0], N, _ptr(acc), _ptr(vacc), omega, T_nuc, _ptr(out))
    return dict(P=out[0], P_err=out[1], P_el=out[2], V=out[3], T=out[4])


def reduce(acc, N):
    acc = np.ascontiguousarray(acc, dtype=np.float64)
    W = acc.shape[0]
    N3 = 3 * N
    E = C.c_double(); Ee = C.c_double(); Nc = C.c_double()
    f = np.zeros(N3); S = np.zeros((N3, N3))
    lib().orc_reduce(W, N3, _ptr(acc), C.byref(E), C.byref(Ee), _ptr(f), _ptr(S), C.byref(Nc))
    return dict(E=E.value, E_err=Ee.value, f=f, S=S, Nc=Nc.value)


def reduce_twists(acc, N, K):
    """Twist average of K contiguous walker blocks (each reduced on its own)."""
    acc = np.ascontiguousarray(acc, dtype=np.float64)
    W = acc.shape[0]
    N3 = 3 * N
    E = C.c_double(); Ee = C.c_double(); Nc = C.c_double()
    f = np.zeros(N3); S = np.zeros((N3, N3))
    lib().orc_reduce_twists(K, W, N3, _ptr(acc), C.byref(E), C.byref(Ee), _ptr(f), _ptr(S), C.byref(Nc))
    return dict(E=E.value, E_err=Ee.value, f=f, S=S, Nc=Nc.value)


# ---- empirical acceleration matrix ----

def empirical_energy(R, L, lam) -> float:
    """Screened-Coulomb proton pair energy sum_{a<b} sum_images exp(-r/lam)/r (images within L)."""
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1, 3)
    return lib().orc_empirical_energy(R.shape[0], L, _ptr(R), lam)


def empirical_s(R, L, lam, mu) -> np.ndarray:
    """S = H + mu I, H the Hessian of empirical_energy ([3N][3N])."""
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1, 3)
    n3 = 3 * R.shape[0]
    S = np.zeros((n3, n3))
    lib().orc_empirical_s(R.shape[0], L, _ptr(R), lam, mu, _ptr(S))
    return S


# ---- twisted boundary conditions ----

def bloch_images(sys: System) -> int:
    """Images per axis M of the Bloch-summed Gaussians of this system."""
    return lib().orc_bloch_images(C.byref(sys.cparams()))


def bloch_gaussian(L, x, Rc, zeta, theta, M):
    """Bloch-summed Gaussian at x: (chi, grad chi [3], lap chi), complex."""
    x, Rc, th = (np.ascontiguousarray(a, dtype=np.float64).reshape(3) for a in (x, Rc, theta))
    o = np.zeros(10)
    lib().orc_bloch_gaussian(L, _ptr(x), _ptr(Rc), zeta, _ptr(th), int(M), _ptr(o))
    return complex(o[0], o[1]), o[2:8:2] + 1j * o[3:8:2], complex(o[8], o[9])


def eval_config_twist(sys: System, R, X, derivs=False):
    """Twisted orbitals (sys.twist set): dict(lnpsi, phase, el, ekin, ekin_im, epot, grad, dlnpsi, del_)."""
    assert sys.twist is not None
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    sc = np.zeros(6)
    grad = np.zeros((sys.n_elec, 3))
    dl = np.zeros((sys.N, 3))
    de = np.zeros((sys.N, 3))
    rc = lib().orc_eval_config_twist(C.byref(p), _ptr(R), _ptr(X), int(derivs), _ptr(sc), _ptr(grad), _ptr(dl),
                                     _ptr(de))
    if rc != 0:
        raise ValueError("singular Slater block")
    out = dict(lnpsi=sc[0], phase=sc[1], el=sc[2], ekin=sc[3], ekin_im=sc[4], epot=sc[5], grad=grad)
    if derivs:
        out.update(dlnpsi=dl, del_=de)
    return out


def eval_configs_twist(sys: System, R, X, twists, derivs=True):
    """X [nconf, Ne, 3]; configuration c takes twists[c // (nconf // K)]: lnpsi, el, dlnpsi, del."""
    twists = np.ascontiguousarray(twists, dtype=np.float64).reshape(-1, 3)
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[0]
    lp = np.zeros(n); el = np.zeros(n)
    dl = np.zeros((n, sys.N, 3)); de = np.zeros((n, sys.N, 3))
    rc = lib().orc_eval_configs_twist(C.byref(p), _ptr(R), n, _ptr(X), twists.shape[0], _ptr(twists), int(derivs),
                                      _ptr(lp), _ptr(el), _ptr(dl), _ptr(de))
    if rc != 0:
        raise ValueError("singular Slater block" if rc == -1 else "configurations not a multiple of the twists")
    return lp, el, dl, de


def vmc_twists(sys: System, R, twists, *, W, n_sweeps, n_warmup, measure_every=1, sigma=0.3, seed=1, md_step=0,
               X=None, forces=True):
    """Chains with twisted orbitals, walker w on twists[w // (W // K)]; returns (X, acc, accept_ratio, vacc)."""
    twists = np.ascontiguousarray(twists, dtype=np.float64).reshape(-1, 3)
    p = sys.cparams()
    R = np.ascontiguousarray(R, dtype=np.float64)
    init = X is None
    Xa = np.zeros((W, sys.n_elec, 3)) if init else np.array(X, dtype=np.float64, copy=True)
    acc = np.zeros((W, 3 + 9 * sys.N))
    vacc = np.zeros(W)
    ca = ChainArgs(W, n_sweeps, n_warmup, measure_every, int(init), int(forces), md_step, 0, sigma, seed)
    na = C.c_longlong(0); nt = C.c_longlong(0)
    rc = lib().orc_vmc_twists(C.byref(p), _ptr(R), C.byref(ca), twists.shape[0], _ptr(twists), _ptr(Xa), _ptr(acc),
                              _ptr(vacc), C.byref(na), C.byref(nt))
    if rc != 0:
        raise ValueError("walkers not a multiple of the twists")
    return Xa, acc, (na.value / nt.value if nt.value else 0.0), vacc


LV_ADOPTED, LV_FAST, LV_NOROGNA = 0, 1, 2


def langevin(R, Rprev, f, S, Sprev, T, delta, alpha, xi, noise_correction=False, box=0.0, scheme=LV_ADOPTED):
    R = np.ascontiguousarray(R, dtype=np.float64).ravel()
    n = R.size
    arr = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (Rprev, f, S, Sprev, xi)]
    out = np.zeros(n)
    rc = lib().orc_langevin(n, _ptr(R), _ptr(arr[0]), _ptr(arr[1]), _ptr(arr[2]), _ptr(arr[3]), T, delta,
                            alpha, _ptr(arr[4]), int(noise_correction), box, int(scheme), _ptr(out))
    if rc != 0:
        raise ValueError("S is not positive definite")
    return out


def langevin_first_predict(R, S, T, delta, xi):
    """First simplified scheme, predict half: y = R + sqrt(2 T D) z, <z z^T> = S^{-1}."""
    R = np.ascontiguousarray(R, dtype=np.float64).ravel()
    S, xi = (np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (S, xi))
    y = np.zeros(R.size)
    if lib().orc_langevin_first_predict(R.size, _ptr(R), _ptr(S), T, delta, _ptr(xi), _ptr(y)) != 0:
        raise ValueError("S is not positive definite")
    return y


def langevin_first_correct(R, f, S, Sy, y, delta, box=0.0):
    """First simplified scheme, correct half: R' = y + D S^{-1} f - 1/2 S^{-1} (S(y) - S)(y - R)."""
    R = np.ascontiguousarray(R, dtype=np.float64).ravel()
    f, S, Sy, y = (np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (f, S, Sy, y))
    out = np.zeros(R.size)
    if lib().orc_langevin_first_correct(R.size, _ptr(R), _ptr(f), _ptr(S), _ptr(Sy), _ptr(y), delta, box,
                                        _ptr(out)) != 0:
        raise ValueError("S is not positive definite")
    return out


def langevin_noise(seed, md_step, n):
    xi = np.zeros(n)
    lib().orc_langevin_noise(seed, md_step, n, _ptr(xi))
    return xi


def num_threads() -> int:
    return lib().orc_num_threads()


# ---- rotating-spring toy model (SI, "A simple toy model") ----
TOY_PLAIN, TOY_STANDARD, TOY_FIRST, TOY_FAST, TOY_ADOPTED, TOY_NOROGNA = range(6)
TOY_S_G, TOY_S_HG = 0, 1
TOY_SCHEMES = {"plain": TOY_PLAIN, "standard": TOY_STANDARD, "first": TOY_FIRST, "fast": TOY_FAST,
               "adopted": TOY_ADOPTED, "norogna": TOY_NOROGNA}


def toy_args(scheme=TOY_ADOPTED, s_mode=TOY_S_G, *, k=2.0, a=1.4, T=0.01, delta=0.05, lam=0.1, mu=0.5,
             alpha=0.2, n_steps=1000, n_burn=0, seed=1) -> ToyArgs:
    """Toy-model parameters; defaults are the SI's figure (k = 2, a = 1.4, T = 0.01,
    mu = 1/2, alpha = 0.2) with the printed G_lambda at lambda = 1/10."""
    return ToyArgs(k, a, T, delta, lam, mu, alpha, scheme, s_mode, n_steps, n_burn, seed)


def toy_eval(args: ToyArgs, x: float, y: float) -> dict:
    o = np.zeros(17)
    lib().orc_toy_eval(C.byref(args), x, y, _ptr(o))
    return dict(U=o[0], f=o[1:3].copy(), S=o[3:7].reshape(2, 2).copy(), Sinv=o[7:11].reshape(2, 2).copy(),
                H=o[11:15].reshape(2, 2).copy(), Gamma=o[15:17].copy())


def toy_step(args: ToyArgs, R, Rp, xi) -> np.ndarray:
    R, Rp, xi = (np.ascontiguousarray(v, dtype=np.float64) for v in (R, Rp, xi))
    out = np.zeros(2)
    if lib().orc_toy_step(C.byref(args), _ptr(R), _ptr(Rp), _ptr(xi), _ptr(out)) != 0:
        raise ValueError("S is not positive definite")
    return out


def toy_run(args: ToyArgs, xy0) -> np.ndarray:
    """Trajectories from xy0 [n][2]; returns [n][7] = x, y, sum U, sum U^2, sum |R|,
    angle travelled, status (sums over the positions after steps n_burn..n_steps-1)."""
    xy0 = np.ascontiguousarray(xy0, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((xy0.shape[0], 7))
    lib().orc_toy_run(C.byref(args), xy0.shape[0], _ptr(xy0), _ptr(out))
    return out


def toy_run_ids(args: ToyArgs, ids, xy0) -> np.ndarray:
    """toy_run for selected trajectories of a larger run (ids = their indices there)."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    xy0 = np.ascontiguousarray(xy0, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((len(ids), 7))
    lib().orc_toy_run_ids(C.byref(args), len(ids), ids.ctypes.data_as(C.POINTER(C.c_int)), _ptr(xy0), _ptr(out))
    return out


def toy_noise(seed, traj, step) -> np.ndarray:
    xi = np.zeros(2)
    lib().orc_toy_noise(seed, traj, step, _ptr(xi))
    return xi
