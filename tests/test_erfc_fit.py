"""The erfc approximation of the mixed-form real-space Ewald sum: the
coefficients in the CUDA source are the committed fit, and their FP32
evaluation is within 4e-7 of erfc(x) exp(x^2) on the range the kernel uses."""
import os
import re

import numpy as np
import pytest

pytest.importorskip("scipy")
from paper_1605_08423_gb300 import fit_erfc

SRC = os.path.join(os.path.dirname(fit_erfc.__file__), "csrc", "common.cuh")


def _source_coefficients():
    body = open(SRC).read()
    body = body[body.index("erfc_scaled_fit("):]
    body = body[:body.index("return e * t * p;")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    # Horner order: highest degree first, each later one added as p * t + c
    signs = re.findall(r"p \* t ([-+]) (\d\.\d+e[-+]\d+)f", body)
    hi = vals[0]
    rest = [float(v) * (1.0 if sg == "+" else -1.0) for sg, v in signs]
    return np.array(list(reversed([hi] + rest)))


def test_source_matches_fit():
    c_src = _source_coefficients()
    c_fit = fit_erfc.fit()
    assert len(c_src) == fit_erfc.DEGREE + 1
    assert np.allclose(c_src, c_fit.astype(np.float32).astype(np.float64), rtol=2e-7, atol=1e-9)


def test_fp32_accuracy():
    assert fit_erfc.fp32_max_rel_error(_source_coefficients()) < 4e-7


def test_reference_points():
    # erfc(x) = e t P(t) at a few x against math.erfc
    import math
    c = _source_coefficients()
    for x in (0.0, 0.3, 1.0, 2.0, 3.5, 4.0):
        t = 1.0 / (1.0 + 0.5 * x)
        val = math.exp(-x * x) * t * np.polynomial.Polynomial(c)(t)
        assert abs(val - math.erfc(x)) <= 3e-7 * math.erfc(x)
