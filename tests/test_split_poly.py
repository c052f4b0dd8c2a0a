"""The FP32 tree walk evaluates the TreePM short-range factor
T(x) = erfc(x) + (2/sqrt(pi)) x exp(-x^2) as exp(-x^2) Q(x) with a fitted
polynomial (paper Sec. 2.1: the tree part of the Gaussian split).  Check the
coefficients compiled into walk.cu are the generator's, and that the FP32
evaluation meets its error bound against scipy's erfc on the walk's range."""
import math
import os
import re
import sys

import numpy as np
from scipy.special import erfc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_05328_gb300", "csrc")
sys.path.insert(0, CSRC)

import gen_split_poly as G  # noqa: E402


def compiled_coefficients():
    src = open(os.path.join(CSRC, "walk.cu")).read()
    body = re.search(r"kSplitPoly\[12\] = \{([^}]*)\}", src).group(1)
    return np.array([float(v.strip().rstrip("f")) for v in body.split(",")])


def test_coefficients_match_generator():
    coef, _, _ = G.fit()
    assert np.allclose(compiled_coefficients(), coef, rtol=1e-8, atol=0)


def test_fp32_split_factor_error():
    coef = compiled_coefficients()
    x = np.linspace(0.0, G.X_MAX, 20001)
    q32 = G.eval_fp32(coef, x).astype(np.float64)
    t_poly = np.exp(-x * x) * q32
    t_true = erfc(x) + 2 / math.sqrt(math.pi) * x * np.exp(-x * x)
    assert np.max(np.abs(t_poly / t_true - 1)) < 5e-7
