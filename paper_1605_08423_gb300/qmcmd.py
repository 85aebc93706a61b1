"""Python binding of libqmcmd.so (include/qmcmd.h): argument marshalling only.

Every step of the energy / force / covariance path and of the Langevin step
runs in the library's CUDA kernels; this module converts numpy arrays and
torch tensors to pointers and turns error codes into exceptions.  There is
no CPU fallback: if the compiled library is missing or no GPU is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libqmcmd.so")

QMC_FP64, QMC_MIXED = 0, 1
QMC_S_IDENTITY, QMC_S_COV, QMC_S_EMPIRICAL = 0, 1, 2
NKERNEL = 9
QMC_OPT_TENSOR_CORES, QMC_OPT_TC_ADJOINT, QMC_OPT_INTEGRATOR, QMC_OPT_NOISE_CORRECTION = 1, 2, 3, 4
QMC_OPT_RECOMPUTE = 5
QMC_RECOMPUTE_FP64, QMC_RECOMPUTE_NEWTON = 0, 1
QMC_OPT_WALKER_OFFSET = 6
HA_PER_BOHR3_IN_GPA = 29421.02648438959    # 1 hartree / bohr^3 in GPa (CODATA)
QMC_LV_ADOPTED, QMC_LV_FAST, QMC_LV_NOROGNA = 0, 1, 2
QMC_TOY_PLAIN, QMC_TOY_STANDARD, QMC_TOY_FIRST, QMC_TOY_FAST, QMC_TOY_ADOPTED, QMC_TOY_NOROGNA = range(6)
QMC_TOY_S_G, QMC_TOY_S_HG = 0, 1
QMC_TOY_NOUT = 7
TOY_SCHEMES = {"plain": QMC_TOY_PLAIN, "standard": QMC_TOY_STANDARD, "first": QMC_TOY_FIRST,
               "fast": QMC_TOY_FAST, "adopted": QMC_TOY_ADOPTED, "norogna": QMC_TOY_NOROGNA}


class QMCError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("n_protons", C.c_int32), ("n_gauss", C.c_int32), ("n_walkers", C.c_int32), ("n_sweeps", C.c_int32),
        ("n_warmup", C.c_int32), ("n_warmup_cont", C.c_int32), ("measure_every", C.c_int32),
        ("recompute_every", C.c_int32), ("precision", C.c_int32), ("ewald_mmax", C.c_int32),
        ("L", C.c_double), ("b_ee", C.c_double), ("b_ep", C.c_double), ("ewald_kappa", C.c_double),
        ("sigma", C.c_double), ("seed", C.c_uint64),
        ("zeta", C.POINTER(C.c_double)), ("coeff", C.POINTER(C.c_double)),
        ("zeta_j", C.c_double), ("fj", C.POINTER(C.c_double)),
        ("n_twist", C.c_int32), ("pad_twist", C.c_int32), ("twist", C.POINTER(C.c_double)),
    ]


class Served(C.Structure):
    _fields_ = [("traj", C.c_int), ("status", C.c_int), ("E", C.c_double), ("E_err", C.c_double),
                ("n_samples", C.c_double), ("accept", C.c_double), ("f", C.POINTER(C.c_double)),
                ("cov", C.POINTER(C.c_double)), ("R_next", C.POINTER(C.c_double)),
                ("latency_ms", C.c_double), ("wait_ms", C.c_double), ("run_ms", C.c_double),
                ("gpu_start_ms", C.c_double), ("gpu_end_ms", C.c_double)]


class Result(C.Structure):
    _fields_ = [("E", C.c_double), ("E_err", C.c_double), ("f", C.POINTER(C.c_double)),
                ("cov", C.POINTER(C.c_double)), ("n_samples", C.c_double), ("accept", C.c_double)]


class ToyParams(C.Structure):
    _fields_ = [("k", C.c_double), ("a", C.c_double), ("T", C.c_double), ("delta", C.c_double),
                ("lam", C.c_double), ("mu", C.c_double), ("alpha", C.c_double),
                ("scheme", C.c_int32), ("s_mode", C.c_int32), ("n_steps", C.c_int32), ("n_burn", C.c_int32),
                ("seed", C.c_uint64)]


_dp = C.POINTER(C.c_double)
_lib = None


def lib():
    """Load libqmcmd.so (built by __graft_entry__.build() / paper_1605_08423_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1605_08423_gb300.build` "
                               "(the CUDA library is the only implementation of this path)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.qmc_init.argtypes = [C.POINTER(Params), _dp, C.POINTER(vp)]
        L.qmc_destroy.argtypes = [vp]
        L.qmc_destroy.restype = None
        L.qmc_footprint_bytes.argtypes = [C.POINTER(Params)]
        L.qmc_footprint_bytes.restype = C.c_size_t
        L.qmc_set_stream.argtypes = [vp, vp]
        L.qmc_sync.argtypes = [vp]
        L.qmc_energy_forces.argtypes = [vp, _dp, C.POINTER(Result)]
        L.qmc_energy_forces_device.argtypes = [vp, vp, vp]
        L.langevin_step.argtypes = [vp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_int, C.c_double]
        L.langevin_step_device.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, C.c_int, C.c_double]
        L.qmc_set_empirical_s.argtypes = [vp, C.c_double, C.c_double]
        L.qmc_twist_partial_device.argtypes = [vp, vp, vp]
        L.qmc_twist_combine_device.argtypes = [vp, vp, C.c_int, vp]
        L.qmc_empirical_s.argtypes = [vp, _dp, _dp]
        L.qmc_empirical_s_device.argtypes = [vp, vp, vp]
        L.langevin_first_predict.argtypes = [vp, _dp, _dp, _dp, C.c_double, C.c_double]
        L.langevin_first_correct.argtypes = [vp, _dp, _dp]
        L.qmc_eval_config.argtypes = [vp, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.qmc_get_walkers.argtypes = [vp, _dp]
        L.qmc_set_walkers.argtypes = [vp, _dp]
        L.qmc_get_accumulators.argtypes = [vp, _dp]
        L.qmc_set_md_step.argtypes = [vp, C.c_uint32]
        L.qmc_set_profiling.argtypes = [vp, C.c_int]
        L.qmc_set_option.argtypes = [vp, C.c_int, C.c_int]
        L.qmc_kernel_times.argtypes = [vp, C.c_int, _dp, C.POINTER(C.c_longlong)]
        L.qmc_langevin_step_static.argtypes = [C.c_int, vp, vp, vp, vp, vp, C.c_double, C.c_double, C.c_int,
                                               C.c_double, C.c_uint64, C.c_uint32, C.c_double, vp]
        L.qmc_checkpoint_size.argtypes = [vp]
        L.qmc_checkpoint_size.restype = C.c_size_t
        L.qmc_checkpoint_save.argtypes = [vp, vp]
        L.qmc_checkpoint_load.argtypes = [vp, vp]
        L.qmc_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(vp)]
        L.qmc_server_destroy.argtypes = [vp]
        L.qmc_server_destroy.restype = None
        L.qmc_server_add_trajectory.argtypes = [vp, C.POINTER(Params), _dp, C.c_double, C.c_double, C.c_int,
                                                C.POINTER(C.c_int)]
        L.qmc_server_submit.argtypes = [vp, C.c_int, C.POINTER(C.c_longlong)]
        L.qmc_server_progress.argtypes = [vp]
        L.qmc_server_fetch.argtypes = [vp, C.c_longlong, C.POINTER(Served)]
        L.qmc_server_stats.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.qmc_pressure.argtypes = [vp, C.c_double, _dp]
        L.qmc_pressure_device.argtypes = [vp, C.c_double, vp]
        L.qmc_shard_sample_device.argtypes = [vp, vp, vp]
        L.qmc_shard_reduce_device.argtypes = [vp, vp, vp, vp]
        L.qmc_shard_finish_device.argtypes = [vp, vp, vp, vp, C.c_longlong]
        L.qmc_launch_count.argtypes = [vp]
        L.qmc_launch_count.restype = C.c_longlong
        L.qmc_kernel_name.argtypes = [C.c_int]
        L.qmc_kernel_name.restype = C.c_char_p
        L.qmc_toy_langevin.argtypes = [C.POINTER(ToyParams), C.c_int, _dp, _dp]
        L.qmc_toy_langevin_device.argtypes = [C.POINTER(ToyParams), C.c_int, vp, vp, vp]
        L.qmc_strerror.argtypes = [C.c_int]
        L.qmc_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().qmc_strerror(code).decode()


def _chk(rc: int, what: str):
    if rc != 0:
        raise QMCError(rc, what)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


@dataclass
class Config:
    """Parameters of one system handle (mirrors qmc_params)."""
    N: int
    L: float
    zeta: np.ndarray
    coeff: np.ndarray
    walkers: int
    sweeps: int
    warmup: int = 20
    warmup_cont: int = 5
    measure_every: int = 1
    recompute_every: int = 1
    precision: int = QMC_FP64
    mmax: int = 6
    b_ee: float = 1.0
    b_ep: float = 1.0
    kappa: float | None = None
    sigma: float = 0.3
    seed: int = 1
    zeta_j: float = 0.7933844         # exponent of the e-e-n-n Jastrow orbitals
    fj: np.ndarray | None = None      # [N][N] symmetric e-e-n-n Jastrow coefficients (FP64 form), or None
    twists: np.ndarray | None = None  # [K][3] twist vectors (twisted boundary conditions, FP64 form), or None

    @classmethod
    def from_workload(cls, wl: "synth.Workload", precision=QMC_FP64, **over):
        kw = dict(N=wl.N, L=wl.L, zeta=np.array(wl.zeta), coeff=wl.C, walkers=wl.walkers, sweeps=wl.sweeps,
                  warmup=wl.warmup, measure_every=wl.measure_every, recompute_every=wl.recompute_every,
                  precision=precision, sigma=wl.sigma, seed=wl.seed)
        kw.update(over)
        return cls(**kw)

    def cparams(self) -> Params:
        self._z = _f64(self.zeta)
        self._c = _f64(self.coeff)
        kappa = 5.0 / self.L if self.kappa is None else self.kappa
        self._fj = None if self.fj is None else _f64(np.asarray(self.fj).reshape(self.N, self.N))
        self._tw = None if self.twists is None else _f64(np.asarray(self.twists).reshape(-1, 3))
        return Params(self.N, len(self._z), self.walkers, self.sweeps, self.warmup, self.warmup_cont,
                      self.measure_every, self.recompute_every, self.precision, self.mmax, self.L, self.b_ee,
                      self.b_ep, kappa, self.sigma, self.seed, _p(self._z), _p(self._c), self.zeta_j,
                      _p(self._fj) if self._fj is not None else C.cast(None, _dp),
                      0 if self._tw is None else self._tw.shape[0], 0,
                      _p(self._tw) if self._tw is not None else C.cast(None, _dp))


def footprint_bytes(cfg: Config) -> int:
    p = cfg.cparams()
    return int(lib().qmc_footprint_bytes(C.byref(p)))


class QMCSystem:
    """One handle of libqmcmd: resident walkers + tables of one system."""

    def __init__(self, cfg: Config, R):
        self.cfg = cfg
        self.N = cfg.N
        self._h = C.c_void_p()
        p = cfg.cparams()
        _chk(lib().qmc_init(C.byref(p), _p(_f64(R)), C.byref(self._h)), "qmc_init")

    def close(self):
        if self._h:
            lib().qmc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ host API
    def energy_forces(self, R) -> dict:
        N3 = 3 * self.N
        f = np.zeros(N3)
        S = np.zeros((N3, N3))
        r = Result(0.0, 0.0, _p(f), _p(S), 0.0, 0.0)
        _chk(lib().qmc_energy_forces(self._h, _p(_f64(R)), C.byref(r)), "qmc_energy_forces")
        return dict(E=r.E, E_err=r.E_err, f=f, S=S, Nc=r.n_samples, accept=r.accept)

    def langevin_step(self, R, f, S, T_kelvin, delta, s_mode=QMC_S_COV, alpha=0.0) -> np.ndarray:
        Rn = _f64(R).copy().ravel()
        Sa = _f64(S) if S is not None else np.zeros(1)
        _chk(lib().langevin_step(self._h, _p(Rn), _p(_f64(f)), _p(Sa), T_kelvin, delta, s_mode, alpha),
             "langevin_step")
        return Rn

    # twists sharded over processes (device tensors, asynchronous): see TwistGroup
    def twist_partial_device(self, out_dev, part_dev):
        _chk(lib().qmc_twist_partial_device(self._h, C.c_void_p(out_dev.data_ptr()), C.c_void_p(part_dev.data_ptr())),
             "qmc_twist_partial_device")

    def twist_combine_device(self, part_dev, K_total: int, out_dev):
        _chk(lib().qmc_twist_combine_device(self._h, C.c_void_p(part_dev.data_ptr()), int(K_total),
                                            C.c_void_p(out_dev.data_ptr())), "qmc_twist_combine_device")

    def set_empirical_s(self, lam: float = 0.0, mu: float = 0.5):
        """Parameters of S = H + mu I for s_mode QMC_S_EMPIRICAL (lam <= 0: Thomas-Fermi length)."""
        _chk(lib().qmc_set_empirical_s(self._h, float(lam), float(mu)), "qmc_set_empirical_s")

    def empirical_s(self, R) -> np.ndarray:
        """S = H + mu I at nuclei R ([3N][3N]; the screened-Coulomb proton pair Hessian)."""
        S = np.zeros((3 * self.N, 3 * self.N))
        _chk(lib().qmc_empirical_s(self._h, _p(_f64(R)), _p(S)), "qmc_empirical_s")
        return S

    def eval_config(self, X, R) -> dict:
        X = _f64(X)
        nc = X.shape[0]
        lp = np.zeros(nc); el = np.zeros(nc)
        dl = np.zeros((nc, self.N, 3)); de = np.zeros((nc, self.N, 3))
        _chk(lib().qmc_eval_config(self._h, nc, _p(X), _p(_f64(R)), _p(lp), _p(el), _p(dl), _p(de)),
             "qmc_eval_config")
        return dict(lnpsi=lp, el=el, dlnpsi=dl, del_=de)

    def pressure(self, T_kelvin: float = 0.0) -> dict:
        """Virial pressure of the last energy_forces call (hartree / bohr^3):
        P (electrons + classical nuclei at T_kelvin), its error bar, the
        electronic part, <V_L> and <T_L>."""
        o = np.zeros(5)
        _chk(lib().qmc_pressure(self._h, float(T_kelvin), _p(o)), "qmc_pressure")
        return dict(P=o[0], P_err=o[1], P_el=o[2], V=o[3], T=o[4])

    def pressure_device(self, T_kelvin, out_dev):
        """The same into a float64 cuda tensor [5] (asynchronous)."""
        _chk(lib().qmc_pressure_device(self._h, float(T_kelvin), C.c_void_p(out_dev.data_ptr())),
             "qmc_pressure_device")

    def walkers(self) -> np.ndarray:
        X = np.zeros((self.cfg.walkers, self.N, 3))
        _chk(lib().qmc_get_walkers(self._h, _p(X)), "qmc_get_walkers")
        return X

    def set_walkers(self, X):
        _chk(lib().qmc_set_walkers(self._h, _p(_f64(X))), "qmc_set_walkers")

    def accumulators(self) -> np.ndarray:
        a = np.zeros((self.cfg.walkers, 3 + 9 * self.N))
        _chk(lib().qmc_get_accumulators(self._h, _p(a)), "qmc_get_accumulators")
        return a

    def set_md_step(self, m: int):
        _chk(lib().qmc_set_md_step(self._h, m), "qmc_set_md_step")

    # ------------------------------------------------------------------ device API (torch tensors)
    def set_stream(self, stream_handle: int | None):
        _chk(lib().qmc_set_stream(self._h, C.c_void_p(stream_handle or 0)), "qmc_set_stream")

    def energy_forces_device(self, R_dev, out_dev):
        """R_dev: float64 cuda tensor [N,3]; out_dev: float64 cuda tensor [4+3N+9N^2] (asynchronous)."""
        _chk(lib().qmc_energy_forces_device(self._h, C.c_void_p(R_dev.data_ptr()), C.c_void_p(out_dev.data_ptr())),
             "qmc_energy_forces_device")

    def langevin_first_predict(self, R, f, S, T_kelvin, delta) -> np.ndarray:
        """First simplified scheme, predict half: returns y (S(R), f(R) kept in the handle)."""
        y = _f64(R).copy().ravel()
        _chk(lib().langevin_first_predict(self._h, _p(y), _p(_f64(f)), _p(_f64(S)), T_kelvin, delta),
             "langevin_first_predict")
        return y

    def langevin_first_correct(self, y, S_y) -> np.ndarray:
        """First simplified scheme, correct half: returns R' given S at the predicted point."""
        Rn = _f64(y).copy().ravel()
        _chk(lib().langevin_first_correct(self._h, _p(Rn), _p(_f64(S_y))), "langevin_first_correct")
        return Rn

    def langevin_step_device(self, R_dev, f_dev, S_dev, T_kelvin, delta, s_mode=QMC_S_COV, alpha=0.0):
        _chk(lib().langevin_step_device(self._h, C.c_void_p(R_dev.data_ptr()), C.c_void_p(f_dev.data_ptr()),
                                        C.c_void_p(S_dev.data_ptr() if S_dev is not None else 0), T_kelvin, delta,
                                        s_mode, alpha), "langevin_step_device")

    def sync(self):
        _chk(lib().qmc_sync(self._h), "qmc_sync")

    def set_tensor_cores(self, on: bool):
        _chk(lib().qmc_set_option(self._h, QMC_OPT_TENSOR_CORES, int(on)), "qmc_set_option")

    def set_integrator(self, scheme: int):
        """QMC_LV_ADOPTED (default), QMC_LV_FAST or QMC_LV_NOROGNA for later Langevin steps."""
        _chk(lib().qmc_set_option(self._h, QMC_OPT_INTEGRATOR, int(scheme)), "qmc_set_option")

    def set_noise_correction(self, on: bool):
        _chk(lib().qmc_set_option(self._h, QMC_OPT_NOISE_CORRECTION, int(on)), "qmc_set_option")

    def set_recompute(self, mode: int):
        """QMC_RECOMPUTE_FP64 (default; FP64 Gauss-Jordan) or QMC_RECOMPUTE_NEWTON (mixed form
        only; one Newton-Schulz step with a compensated residual)."""
        _chk(lib().qmc_set_option(self._h, QMC_OPT_RECOMPUTE, int(mode)), "qmc_set_option")

    def set_walker_offset(self, w0: int):
        """Philox stream of walker 0 (walker sharding); places the walkers again."""
        _chk(lib().qmc_set_option(self._h, QMC_OPT_WALKER_OFFSET, int(w0)), "qmc_set_option")

    # walker-sharded reduction (device tensors, asynchronous): see ShardGroup
    def shard_sample_device(self, R_dev, sums_dev):
        _chk(lib().qmc_shard_sample_device(self._h, C.c_void_p(R_dev.data_ptr()), C.c_void_p(sums_dev.data_ptr())),
             "qmc_shard_sample_device")

    def shard_reduce_device(self, sums_dev, out_dev, gram_dev):
        _chk(lib().qmc_shard_reduce_device(self._h, C.c_void_p(sums_dev.data_ptr()), C.c_void_p(out_dev.data_ptr()),
                                           C.c_void_p(gram_dev.data_ptr())), "qmc_shard_reduce_device")

    def shard_finish_device(self, sums_dev, gram_dev, out_dev, walkers_total: int):
        _chk(lib().qmc_shard_finish_device(self._h, C.c_void_p(sums_dev.data_ptr()), C.c_void_p(gram_dev.data_ptr()),
                                           C.c_void_p(out_dev.data_ptr()), int(walkers_total)),
             "qmc_shard_finish_device")

    def set_tc_adjoint(self, on: bool):
        """Orbital force terms in the separate tensor-core kernel (True) or in
        the SIMT measure kernel (False); effective while tensor cores are on."""
        _chk(lib().qmc_set_option(self._h, QMC_OPT_TC_ADJOINT, int(on)), "qmc_set_option")

    def set_profiling(self, on: bool):
        _chk(lib().qmc_set_profiling(self._h, int(on)), "qmc_set_profiling")

    def checkpoint(self) -> bytes:
        n = int(lib().qmc_checkpoint_size(self._h))
        buf = (C.c_ubyte * n)()
        _chk(lib().qmc_checkpoint_save(self._h, buf), "qmc_checkpoint_save")
        return bytes(buf)

    def restore(self, blob: bytes):
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        _chk(lib().qmc_checkpoint_load(self._h, buf), "qmc_checkpoint_load")

    def launch_count(self) -> int:
        return int(lib().qmc_launch_count(self._h))

    def kernel_times(self) -> dict:
        ms = np.zeros(NKERNEL)
        ln = (C.c_longlong * NKERNEL)()
        _chk(lib().qmc_kernel_times(self._h, NKERNEL, _p(ms), ln), "qmc_kernel_times")
        return {lib().qmc_kernel_name(k).decode(): (float(ms[k]), int(ln[k])) for k in range(NKERNEL)}


def langevin_step_static(R_dev, Rprev_dev, f_dev, S_dev, Sprev_dev, T_kelvin, delta, s_mode, alpha, seed, step,
                         box, stream_handle=0):
    """qmc_langevin_step_static on float64 CUDA tensors (R_dev updated in place).
    For callers that cannot allocate device memory: the call allocates nothing."""
    n3 = R_dev.numel()
    ptr = lambda t: C.c_void_p(t.data_ptr() if t is not None else 0)
    _chk(lib().qmc_langevin_step_static(n3, ptr(R_dev), ptr(Rprev_dev), ptr(f_dev), ptr(S_dev), ptr(Sprev_dev),
                                        T_kelvin, delta, s_mode, alpha, seed, step, box,
                                        C.c_void_p(stream_handle or 0)), "qmc_langevin_step_static")


def toy_params(scheme=QMC_TOY_ADOPTED, s_mode=QMC_TOY_S_G, *, k=2.0, a=1.4, T=0.01, delta=0.05, lam=0.1, mu=0.5,
               alpha=0.2, n_steps=1000, n_burn=0, seed=1) -> ToyParams:
    """Parameters of the rotating-spring toy model (defaults: the SI's figure, k = 2,
    a = 1.4, T = 0.01, mu = 1/2, alpha = 0.2, printed G_lambda at lambda = 1/10)."""
    return ToyParams(k, a, T, delta, lam, mu, alpha, scheme, s_mode, n_steps, n_burn, seed)


def toy_langevin(p: ToyParams, xy0) -> np.ndarray:
    """qmc_toy_langevin on host arrays: xy0 [n][2] -> out [n][QMC_TOY_NOUT].
    Trajectories stopped by an indefinite S keep their status column; the call
    then raises QMCError(QMC_ERR_NOT_PD) with the array attached as .out."""
    xy0 = _f64(np.asarray(xy0).reshape(-1, 2))
    out = np.zeros((xy0.shape[0], QMC_TOY_NOUT))
    rc = lib().qmc_toy_langevin(C.byref(p), xy0.shape[0], _p(xy0), _p(out))
    if rc != 0:
        err = QMCError(rc, "qmc_toy_langevin")
        err.out = out
        raise err
    return out


def toy_langevin_device(p: ToyParams, xy0_dev, out_dev, stream_handle=0):
    """qmc_toy_langevin_device on float64 CUDA tensors ([n][2] in, [n][QMC_TOY_NOUT] out)."""
    n = xy0_dev.shape[0]
    _chk(lib().qmc_toy_langevin_device(C.byref(p), n, C.c_void_p(xy0_dev.data_ptr()),
                                       C.c_void_p(out_dev.data_ptr()), C.c_void_p(stream_handle or 0)),
         "qmc_toy_langevin_device")


class Server:
    """Continuous-batching request loop (qmc_server_*): one MD step per request."""

    def __init__(self, hbm_budget_bytes: int, max_active: int):
        self._s = C.c_void_p()
        _chk(lib().qmc_server_create(int(hbm_budget_bytes), int(max_active), C.byref(self._s)), "qmc_server_create")
        self._N = {}

    def close(self):
        if self._s:
            lib().qmc_server_destroy(self._s)
            self._s = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_trajectory(self, cfg: Config, R0, T_kelvin, delta, s_mode=QMC_S_COV) -> int:
        p = cfg.cparams()
        tid = C.c_int()
        _chk(lib().qmc_server_add_trajectory(self._s, C.byref(p), _p(_f64(R0)), T_kelvin, delta, s_mode,
                                             C.byref(tid)), "qmc_server_add_trajectory")
        self._N[tid.value] = cfg.N
        return tid.value

    def submit(self, traj: int) -> int:
        t = C.c_longlong()
        _chk(lib().qmc_server_submit(self._s, traj, C.byref(t)), "qmc_server_submit")
        return t.value

    def progress(self) -> int:
        rc = lib().qmc_server_progress(self._s)
        if rc < 0:
            raise QMCError(rc, "qmc_server_progress")
        return rc

    def fetch(self, ticket: int, traj: int):
        """Finished request as a dict, or None while it is pending."""
        N3 = 3 * self._N[traj]
        f = np.zeros(N3); S = np.zeros((N3, N3)); Rn = np.zeros(N3)
        o = Served(0, 0, 0.0, 0.0, 0.0, 0.0, _p(f), _p(S), _p(Rn), 0.0, 0.0, 0.0, -1.0, -1.0)
        rc = lib().qmc_server_fetch(self._s, ticket, C.byref(o))
        if rc < 0:
            raise QMCError(rc, "qmc_server_fetch")
        if rc == 0:
            return None
        return dict(traj=o.traj, status=o.status, E=o.E, E_err=o.E_err, Nc=o.n_samples, accept=o.accept, f=f,
                    S=S, R_next=Rn, latency_ms=o.latency_ms, wait_ms=o.wait_ms, run_ms=o.run_ms,
                    gpu_start_ms=o.gpu_start_ms, gpu_end_ms=o.gpu_end_ms)

    def stats(self) -> dict:
        st = (C.c_longlong * 8)()
        _chk(lib().qmc_server_stats(self._s, st), "qmc_server_stats")
        keys = ["resident_bytes", "resident", "active", "queued", "evictions", "completed", "admissions", "budget"]
        return dict(zip(keys, list(st)))


def unpack_out(out: np.ndarray, N: int) -> dict:
    """Split the device output vector [E, E_err, N_c, accept, f(3N), S(3N*3N)]."""
    N3 = 3 * N
    return dict(E=out[0], E_err=out[1], Nc=out[2], accept=out[3], f=out[4:4 + N3],
                S=out[4 + N3:4 + N3 + N3 * N3].reshape(N3, N3))


def energy_forces_function():
    """torch.autograd.Function whose forward is the VMC energy E(R) and whose
    backward returns dE/dR = -f (the library's Hellmann-Feynman + Pulay force)."""
    import torch

    class EnergyForces(torch.autograd.Function):
        @staticmethod
        def forward(ctx, R, system):
            out = system.energy_forces(R.detach().cpu().numpy().reshape(-1, 3))
            f = torch.as_tensor(out["f"], dtype=R.dtype, device=R.device).reshape(R.shape)
            ctx.save_for_backward(f)
            return torch.as_tensor(out["E"], dtype=R.dtype, device=R.device)

        @staticmethod
        def backward(ctx, grad_out):
            (f,) = ctx.saved_tensors
            return -f * grad_out, None

    return EnergyForces


def shard_sizes(walkers_total: int, world: int) -> list[int]:
    """Walkers per process when walkers_total is split over `world` processes
    (consecutive slices, the first walkers_total % world one larger)."""
    base, extra = divmod(int(walkers_total), int(world))
    return [base + (1 if r < extra else 0) for r in range(world)]


def twist_slice(twists, rank: int, world: int) -> np.ndarray:
    """The consecutive share of a twist list ([K][3], K a multiple of world) that
    process `rank` of `world` samples in a TwistGroup."""
    t = np.asarray(twists, dtype=np.float64).reshape(-1, 3)
    if t.shape[0] % world:
        raise ValueError(f"{t.shape[0]} twists do not split evenly over {world} processes")
    k = t.shape[0] // world
    return t[rank * k:(rank + 1) * k]


class TwistGroup:
    """One twist-averaged energy/force evaluation with the twist mesh split over
    the processes of a torch.distributed group (one GPU each): each process's
    handle samples its own slice of the twists (twist_slice), with the same
    walkers per twist everywhere, so the sampling exchanges nothing; one
    all-reduce then sums the processes' weighted averages (qmc_twist_partial),
    and every process ends with the average over all twists
    (qmc_twist_combine), the result one handle over the whole mesh would give
    up to the order of the FP64 sums.  `system` is the process's QMCSystem (or
    any object with energy_forces_device, the twist_* methods and N)."""

    def __init__(self, system, K_total: int, group=None):
        import torch
        import torch.distributed as dist
        self.system, self.group, self.dist = system, group, dist
        self.K_total = int(K_total)
        N = system.N
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        if dev == "cuda" and hasattr(system, "set_stream"):
            system.set_stream(torch.cuda.current_stream().cuda_stream or 1)
        self.part = torch.zeros(4 + 3 * N + 9 * N * N, dtype=torch.float64, device=dev)

    def energy_forces_device(self, R_dev, out_dev):
        """out_dev: [E, E_err, N_c, accept, f(3N), S(3N x 3N)], the layout of qmc_energy_forces_device."""
        self.system.energy_forces_device(R_dev, out_dev)
        self.system.twist_partial_device(out_dev, self.part)
        self.dist.all_reduce(self.part, op=self.dist.ReduceOp.SUM, group=self.group)
        self.system.twist_combine_device(self.part, self.K_total, out_dev)


class ShardGroup:
    """One energy/force evaluation with the walkers split over the processes of
    a torch.distributed group (one GPU each): each process holds a consecutive
    slice of the walker population (its handle's walker offset is the slice's
    first walker), and the reduction exchanges two buffers per evaluation --
    the column sums of the per-walker accumulators, then the sums of the
    per-walker deviations about the global mean (the covariance S) -- by
    all-reduce.  Every process ends with the E, f, S the single handle over all
    walkers would give (up to the order of the FP64 sums) and applies the same
    Langevin step.  `system` is the process's QMCSystem (or any object with the
    shard_* methods and N); the buffers are tensors on its device.  The
    collectives run on torch's current stream, so the handle is put on that
    stream too (its kernels and the all-reduces are then ordered)."""

    def __init__(self, system, walkers_total: int, group=None):
        import torch
        import torch.distributed as dist
        self.system, self.group, self.dist = system, group, dist
        self.walkers_total = int(walkers_total)
        N = system.N
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        if dev == "cuda" and hasattr(system, "set_stream"):
            # torch's default stream has handle 0, which qmc_set_stream reads as
            # "the handle's own stream": name the legacy default stream (1) instead
            system.set_stream(torch.cuda.current_stream().cuda_stream or 1)
        self.sums = torch.zeros(3 + 9 * N + 3, dtype=torch.float64, device=dev)
        self.gram = torch.zeros(1 + 9 * N * N, dtype=torch.float64, device=dev)

    def energy_forces_device(self, R_dev, out_dev):
        """out_dev: [E, E_err, N_c, accept, f(3N), S(3N x 3N)], the layout of qmc_energy_forces_device."""
        op = self.dist.ReduceOp.SUM
        self.system.shard_sample_device(R_dev, self.sums)
        self.dist.all_reduce(self.sums, op=op, group=self.group)
        self.system.shard_reduce_device(self.sums, out_dev, self.gram)
        self.dist.all_reduce(self.gram, op=op, group=self.group)
        self.system.shard_finish_device(self.sums, self.gram, out_dev, self.walkers_total)
