"""Generate the FP32 polynomial of the TreePM short-range factor used by the
tree walk (walk.cu).

T(x) = erfc(x) + (2 / sqrt(pi)) x exp(-x^2),  x = r / (2 r_s),
is written as T = exp(-x^2) Q(x) with Q(x) = erfcx(x) + 2 x / sqrt(pi), a smooth
function on [0, X_MAX].  Q is fitted with a Chebyshev least-squares fit in
t = 2 x / X_MAX - 1 and converted to a power series in t, evaluated with
Horner's rule in FP32 on the device.  Prints the C initialiser and the worst
relative error of the FP32 evaluation against scipy's erfcx.
"""
import numpy as np
from numpy.polynomial import chebyshev as Ch
from scipy.special import erfcx

X_MAX = 2.5  # covers r_cut / r_s <= 5
DEG = 11


def fit():
    xs = np.linspace(0.0, X_MAX, 40001)
    q = erfcx(xs) + 2 * xs / np.sqrt(np.pi)
    t = xs / X_MAX * 2 - 1
    return Ch.cheb2poly(Ch.chebfit(t, q, DEG)), xs, q


def eval_fp32(coef, xs):
    tf = (xs.astype(np.float32) * np.float32(2 / X_MAX) - np.float32(1)).astype(np.float32)
    v = np.float32(coef[-1])
    for ck in coef[::-1][1:]:
        v = (v * tf + np.float32(ck)).astype(np.float32)
    return v


if __name__ == "__main__":
    coef, xs, q = fit()
    err = np.abs(eval_fp32(coef, xs) / q - 1).max()
    print("// Q(t) power-series coefficients, t = 2 x / %.1f - 1; FP32 rel. error %.2e" % (X_MAX, err))
    print("__constant__ float kSplitPoly[%d] = {%s};" % (DEG + 1, ", ".join("%.9ef" % c for c in coef)))
