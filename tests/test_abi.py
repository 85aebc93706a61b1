"""Host-side checks of the C ABI (no GPU needed): the library loads and exports
every function declared in include/qmcmd.h, struct layouts agree with the
binding, and argument validation happens before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1605_08423_gb300 import build as gbuild
from paper_1605_08423_gb300 import qmcmd as q
from paper_1605_08423_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "qmcmd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return q.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "qmc_init" in names and "langevin_step" in names and "qmc_energy_forces" in names
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layouts_match_header(lib):
    # qmc_params: 10 int32, 5 double, uint64, 2 pointers, then the e-e-n-n Jastrow double and pointer,
    # then the twists: 2 int32 and a pointer
    assert C.sizeof(q.Params) == 10 * 4 + 5 * 8 + 8 + 2 * 8 + 8 + 8 + 2 * 4 + 8
    assert q.Params.twist.offset == C.sizeof(q.Params) - 8
    assert C.sizeof(q.Result) == 6 * 8
    # qmc_served: 2 int, 4 double, 3 pointers, 5 double
    assert C.sizeof(q.Served) == 2 * 4 + 4 * 8 + 3 * 8 + 5 * 8


def test_invalid_parameters_rejected_without_gpu(lib):
    wl = synth.workload("h16", walkers=2)
    cfg = q.Config.from_workload(wl, walkers=1)
    assert q.footprint_bytes(cfg) == 0            # invalid -> 0
    cfg_ok = q.Config.from_workload(wl)
    assert q.footprint_bytes(cfg_ok) > 0
    odd = q.Config.from_workload(wl)
    odd.N = 15
    h = C.c_void_p()
    rc = lib.qmc_init(C.byref(odd.cparams()), (C.c_double * 48)(), C.byref(h))
    assert rc == -1
    assert q.strerror(-7) == "singular Slater matrix"
    # the e-e-n-n Jastrow term: both forms, positive exponent
    fj = np.eye(wl.N) * 0.1
    assert q.footprint_bytes(q.Config.from_workload(wl, fj=fj)) > 0
    assert q.footprint_bytes(q.Config.from_workload(wl, fj=fj, precision=q.QMC_MIXED)) > 0
    assert q.footprint_bytes(q.Config.from_workload(wl, fj=fj, zeta_j=0.0)) == 0
    # f must be exactly symmetric: the kernels read its row a as its column a
    A = np.random.default_rng(3).uniform(-0.3, 0.3, (wl.N, wl.N))
    assert q.footprint_bytes(q.Config.from_workload(wl, fj=0.5 * (A + A.T))) > 0
    assert q.footprint_bytes(q.Config.from_workload(wl, fj=A)) == 0
    h = C.c_void_p()
    asym = q.Config.from_workload(wl, fj=A)
    assert lib.qmc_init(C.byref(asym.cparams()), (C.c_double * 48)(), C.byref(h)) == -1


def test_twist_parameters_validated_without_gpu(lib):
    wl = synth.workload("h16", walkers=8)
    tw = synth.monkhorst_pack(2)[:4]
    assert q.footprint_bytes(q.Config.from_workload(wl, twists=tw)) > q.footprint_bytes(q.Config.from_workload(wl))
    assert q.footprint_bytes(q.Config.from_workload(wl, twists=tw, precision=q.QMC_MIXED)) == 0   # FP64 only
    assert q.footprint_bytes(q.Config.from_workload(wl, twists=tw[:3])) == 0     # W not a multiple of K
    assert q.footprint_bytes(q.Config.from_workload(wl, walkers=4, twists=tw)) == 0   # fewer than 2 per twist
    assert q.footprint_bytes(q.Config.from_workload(wl, twists=tw, fj=np.eye(wl.N) * 0.1)) > 0   # with U_{3+4}
    bad = tw.copy()
    bad[1, 2] = np.nan
    assert q.footprint_bytes(q.Config.from_workload(wl, twists=bad)) == 0


def test_acceleration_matrix_modes(lib):
    assert (q.QMC_S_IDENTITY, q.QMC_S_COV, q.QMC_S_EMPIRICAL) == (0, 1, 2)
    src = open(os.path.join(ROOT, "include", "qmcmd.h")).read()
    assert "QMC_S_EMPIRICAL = 2" in src
    assert lib.qmc_set_empirical_s(None, 0.7, 0.5) == -1      # no handle
    assert lib.qmc_empirical_s(None, None, None) == -1


def test_recompute_option_values(lib):
    assert q.QMC_OPT_RECOMPUTE == 5 and (q.QMC_RECOMPUTE_FP64, q.QMC_RECOMPUTE_NEWTON) == (0, 1)
    assert lib.qmc_set_option(None, q.QMC_OPT_RECOMPUTE, 0) == -1      # no handle


def test_footprint_scales_with_walkers(lib):
    wl = synth.workload("h64")
    a = q.footprint_bytes(q.Config.from_workload(wl, walkers=1000))
    b = q.footprint_bytes(q.Config.from_workload(wl, walkers=2000))
    assert 1.8 < b / a < 2.1


def test_toy_parameters_validated_without_gpu(lib):
    # qmc_toy_params: 7 doubles, 4 int32, uint64
    assert C.sizeof(q.ToyParams) == 7 * 8 + 4 * 4 + 8
    xy0 = (C.c_double * 4)()
    out = (C.c_double * 14)()
    bad = [dict(delta=0.0), dict(lam=0.0), dict(T=-1.0), dict(alpha=-0.1), dict(n_steps=-1),
           dict(n_steps=3, n_burn=4), dict(scheme=6), dict(scheme=-1), dict(s_mode=2)]
    for kw in bad:
        p = q.toy_params(**kw)
        assert lib.qmc_toy_langevin(C.byref(p), 2, xy0, out) == -1, kw
        assert lib.qmc_toy_langevin_device(C.byref(p), 2, None, None, None) == -1, kw
    p = q.toy_params()
    assert lib.qmc_toy_langevin(C.byref(p), -1, xy0, out) == -1
    assert lib.qmc_toy_langevin(C.byref(p), 2, None, out) == -1
    assert lib.qmc_toy_langevin(C.byref(p), 0, None, None) == 0      # nothing to do
