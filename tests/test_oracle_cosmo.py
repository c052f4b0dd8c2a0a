"""Pins of the oracle's background cosmology and time tables (oracle/cosmo.c).

Closed forms: Einstein-de Sitter and de Sitter integrals; an independent ODE
integration of the linear growth equation; the sigma8 normalisation re-done
with scipy quadrature.  R_lc is the comoving distance of the lightcone (paper
Sec. 1 footnote, Fig. 1)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

import oracle as O

C_H0 = 2997.92458


def eds():
    return O.params(omega_m=1.0, omega_l=0.0)


@pytest.mark.parametrize("a0,a1", [(0.02, 0.03), (0.1, 0.5), (0.5, 1.0)])
def test_eds_drift_kick(a0, a1):
    P = eds()
    assert O.drift_factor(P, a0, a1) == pytest.approx(2 * (a0 ** -0.5 - a1 ** -0.5), rel=1e-13)
    assert O.kick_factor(P, a0, a1) == pytest.approx(2 * (a1 ** 0.5 - a0 ** 0.5), rel=1e-13)


@pytest.mark.parametrize("a", [0.02, 0.3, 0.9])
def test_eds_chi_growth(a):
    P = eds()
    assert O.chi(P, a) == pytest.approx(2 * C_H0 * (1 - math.sqrt(a)), rel=1e-13)
    assert O.growth(P, a) == pytest.approx(a, rel=1e-13)
    assert O.growth_rate(P, a) == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("a", [0.05, 0.5])
def test_de_sitter_chi(a):
    P = O.params(omega_m=0.0, omega_l=1.0)
    assert O.chi(P, a) == pytest.approx(C_H0 * (1 / a - 1), rel=1e-13)


def test_lcdm_growth_matches_ode():
    """Linear growth: D'' + (3/a + E'/E) D' - 1.5 Om / (a^5 E^2) D = 0, started
    in the matter era with D = a; compared after normalising at a = 1."""
    P = O.params()
    om, ol = 0.3, 0.7

    def E(a):
        return math.sqrt(om / a ** 3 + ol)

    def dE(a):
        return -1.5 * om / a ** 4 / E(a)

    def rhs(a, y):
        D, dD = y
        return [dD, -(3 / a + dE(a) / E(a)) * dD + 1.5 * om / (a ** 5 * E(a) ** 2) * D]

    a0 = 1e-4
    sol = solve_ivp(rhs, (a0, 1.0), [a0, 1.0], rtol=1e-12, atol=1e-16, dense_output=True)
    d1 = sol.sol(1.0)[0]
    for a in (0.02, 0.1, 0.5, 0.8):
        D, dD = sol.sol(a)
        assert O.growth(P, a) == pytest.approx(D / d1, rel=1e-6)
        assert O.growth_rate(P, a) == pytest.approx(a * dD / D, rel=1e-6)


def test_sigma8_normalisation_scipy():
    """sigma(8 Mpc/h) recomputed from the oracle's P(k) with scipy quad."""
    P = O.params(sigma8=0.8)

    def w(x):
        return 3 * (math.sin(x) - x * math.cos(x)) / x ** 3

    amp = O.lib().dzso_power_amplitude(O.byref(P))

    def integrand(lnk):
        k = math.exp(lnk)
        pk = amp * O.lib().dzso_power_shape(O.byref(P), k)
        return k ** 3 * pk * w(8 * k) ** 2 / (2 * math.pi ** 2)

    s2 = quad(integrand, math.log(1e-5), math.log(50.0), limit=500, epsabs=0, epsrel=1e-10)[0]
    assert math.sqrt(s2) == pytest.approx(0.8, rel=1e-6)
    # the oracle's own top-hat sigma(r): sigma8 at 8 Mpc/h, and the same
    # integral at another radius
    assert O.sigma_r(P, 8.0) == pytest.approx(0.8, rel=1e-6)

    def integrand4(lnk):
        k = math.exp(lnk)
        return k ** 3 * amp * O.lib().dzso_power_shape(O.byref(P), k) * w(4 * k) ** 2 / (2 * math.pi ** 2)

    s4 = quad(integrand4, math.log(1e-5), math.log(100.0), limit=500, epsabs=0, epsrel=1e-10)[0]
    assert O.sigma_r(P, 4.0) == pytest.approx(math.sqrt(s4), rel=1e-6)


def test_bbks_shape():
    """P(k) / k^ns -> A at small k (T -> 1), and the transfer function
    suppresses small scales (Bardeen et al. 1986)."""
    P = O.params()
    k = 1e-9
    assert O.power(P, k) / k ** 0.96 == pytest.approx(O.power(P, 2 * k) / (2 * k) ** 0.96, rel=1e-6)
    assert O.power(P, 10.0) < O.power(P, 0.02)


def test_tables_structure():
    P = O.params(nsteps=96)
    T = O.tables(P)
    a = T["a"]
    assert a[0] == pytest.approx(1 / 50, rel=1e-15)
    assert a[-1] == 1.0
    dl = np.diff(np.log(a))
    assert np.allclose(dl, math.log(50) / 96, rtol=1e-12)
    # the two half kicks add up to the full-step kick
    for n in (0, 40, 95):
        assert T["kick1"][n] + T["kick2"][n] == pytest.approx(O.kick_factor(P, a[n], a[n + 1]), rel=1e-13)
        assert T["drift"][n] == pytest.approx(O.drift_factor(P, a[n], a[n + 1]), rel=1e-15)
    # SWEEP: R runs from the box corner to 0, proportional to chi(a)
    assert T["rlc"][0] == pytest.approx(math.sqrt(3) * 64 / 2, rel=1e-15)
    assert T["rlc"][-1] == 0.0
    assert np.all(np.diff(T["rlc"]) < 0)
    chis = np.array([O.chi(P, x) for x in a])
    assert np.allclose(T["rlc"], T["rlc"][0] * chis / chis[0], rtol=1e-13)
    assert np.array_equal(T["rlat"], np.floor(T["rlc"] / 64 * 2.0 ** 32).astype(np.uint64))


def test_tables_physical_mode():
    P = O.params(n1d=32, box=1024.0, rlc_mode=1)
    T = O.tables(P)
    rmax = math.sqrt(3) * 1024 / 2
    chis = np.array([O.chi(P, x) for x in T["a"]])
    assert np.allclose(T["rlc"], np.minimum(chis, rmax), rtol=1e-15)
    # the lightcone enters the 1024 Mpc/h box at z ~ 0.3 (chi(z=0.3) ~ 870 Mpc/h)
    inside = T["a"][T["rlc"] < rmax]
    z_entry = 1 / inside[0] - 1
    assert 0.2 < z_entry < 0.32
