"""Pins of the oracle's Carnahan-Starling thermodynamics (oracle/eos.py).

Every check compares the oracle with something other than itself: the
critical-point ratios printed in the paper, the hard-sphere virial
coefficients, the Carnahan-Starling free energy (a different closed form from
which p and the chemical potential follow), and mean-field scaling near T_c.
"""
import os

import numpy as np
import pytest

from oracle import eos

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    return vals


# ---- Carnahan-Starling free energy per volume, written independently of Eq. EOS:
# f(rho) = rho R T [ln rho - 1 + (4 eta - 3 eta^2)/(1 - eta)^2] - a rho^2, eta = b rho/4
def cs_free_energy(rho, T, a, b, R):
    eta = b * rho / 4.0
    return rho * R * T * (np.log(rho) - 1.0 + (4 * eta - 3 * eta**2) / (1 - eta) ** 2) - a * rho**2


def cs_mu(rho, T, a, b, R):
    """Chemical potential df/drho of the free energy above (standard CS result)."""
    eta = b * rho / 4.0
    return R * T * (np.log(rho) + (8 * eta - 9 * eta**2 + 3 * eta**3) / (1 - eta) ** 3) - 2 * a * rho


@pytest.mark.parametrize("a", [0.25, 0.5])
def test_critical_ratios_match_paper(a):
    """Sec. IV prints a ~ 3.8533 p_c/rho_c^2, b ~ 0.5218/rho_c, R ~ 2.7864 p_c/(rho_c T_c)."""
    g = golden()
    b, R = g["b"], g["R"]
    rho_c, T_c, p_c = eos.critical_point(a, b, R)
    # the paper gives these to 4-5 digits with "approximately"; 5e-4 relative
    assert a * rho_c**2 / p_c == pytest.approx(g["a_rhoc2_over_pc"], rel=5e-4)
    assert b * rho_c == pytest.approx(g["b_rhoc"], rel=5e-4)
    assert R * rho_c * T_c / p_c == pytest.approx(g["R_rhoc_Tc_over_pc"], rel=5e-4)


def test_critical_point_is_inflection_with_zero_slope():
    """dp/drho and d2p/drho2 vanish at (rho_c, T_c): checked by finite differences of p."""
    a, b, R = 0.25, 4.0, 1.0
    rho_c, T_c, p_c = eos.critical_point(a, b, R)
    h = 1e-4 * rho_c
    p = lambda r: float(eos.p_eos(r, T_c, a, b, R))
    d1 = (p(rho_c + h) - p(rho_c - h)) / (2 * h)
    d2 = (p(rho_c + h) - 2 * p(rho_c) + p(rho_c - h)) / h**2
    scale1 = p_c / rho_c
    scale2 = p_c / rho_c**2
    assert abs(d1) < 1e-6 * scale1
    assert abs(d2) < 1e-6 * scale2
    # just above T_c the isotherm is monotone; just below it has a loop
    rr = np.linspace(0.5 * rho_c, 1.5 * rho_c, 2001)
    assert np.all(np.diff(eos.p_eos(rr, 1.001 * T_c, a, b, R)) > 0)
    assert np.any(np.diff(eos.p_eos(rr, 0.999 * T_c, a, b, R)) < 0)


def test_eos_equals_free_energy_route():
    """p = rho mu - f from the CS free energy equals Eq. EOS as coded."""
    a, b, R, T = 0.25, 4.0, 1.0, 0.02
    rho = np.linspace(0.005, 0.6, 200)
    p_thermo = rho * cs_mu(rho, T, a, b, R) - cs_free_energy(rho, T, a, b, R)
    np.testing.assert_allclose(eos.p_eos(rho, T, a, b, R), p_thermo, rtol=1e-11, atol=1e-15)


def test_hard_sphere_virial_coefficients():
    """Z = p_rep/(rho R T) of the CS term expands as 1 + 4 eta + 10 eta^2 + ... (exact B2, B3)."""
    a, b, R, T = 0.0, 4.0, 1.0, 1.0
    for eta in [1e-3, 2e-3]:
        rho = 4 * eta / b
        Z = float(eos.p_eos(rho, T, a, b, R)) / (rho * R * T)
        assert (Z - 1) / eta == pytest.approx(4.0, rel=5 * eta)
        assert (Z - 1 - 4 * eta) / eta**2 == pytest.approx(10.0, rel=5 * eta)


@pytest.mark.parametrize("Tr", [0.6, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95, 0.99])
def test_maxwell_equal_chemical_potential(Tr):
    """Eqs. MaxwellRule are equivalent to equal pressure and equal chemical potential
    (Sec. IV, after Eq. Pressures_MaxwellRule); mu comes from the free energy."""
    a, b, R = 0.25, 4.0, 1.0
    rho_c, T_c, p_c = eos.critical_point(a, b, R)
    T = Tr * T_c
    rv, rl, ps = eos.maxwell(T, a, b, R)
    assert rv < rho_c < rl
    assert float(eos.p_eos(rv, T, a, b, R)) == pytest.approx(ps, rel=1e-12)
    assert float(eos.p_eos(rl, T, a, b, R)) == pytest.approx(ps, rel=1e-12)
    mu_scale = R * T
    assert abs(cs_mu(rv, T, a, b, R) - cs_mu(rl, T, a, b, R)) < 1e-11 * mu_scale


def test_maxwell_invariant_in_a_at_equal_reduced_temperature():
    """p and R T both scale with a at fixed T/T_c, so reduced coexistence is a-independent."""
    out = []
    for a in [0.25, 0.5, 1.0]:
        _, T_c, _ = eos.critical_point(a, 4.0, 1.0)
        out.append(eos.maxwell(0.8 * T_c, a, 4.0, 1.0))
    for o in out[1:]:
        assert o[0] == pytest.approx(out[0][0], rel=1e-10)
        assert o[1] == pytest.approx(out[0][1], rel=1e-10)


def test_mean_field_exponent_near_critical_point():
    """rho_l - rho_v ~ (1 - T/T_c)^(1/2) for a van der Waals-type EOS."""
    a, b, R = 0.25, 4.0, 1.0
    _, T_c, _ = eos.critical_point(a, b, R)
    d = []
    for eps in [1e-4, 4e-4]:
        rv, rl, _ = eos.maxwell((1 - eps) * T_c, a, b, R)
        d.append(rl - rv)
    assert d[0] / d[1] == pytest.approx(0.5, rel=2e-3)


@pytest.mark.parametrize("Tr", [0.7, 0.85, 0.95])
def test_spinodals_are_extrema(Tr):
    a, b, R = 0.25, 4.0, 1.0
    rho_c, T_c, _ = eos.critical_point(a, b, R)
    T = Tr * T_c
    sv, sl = eos.spinodals(T, a, b, R)
    rv, rl, _ = eos.maxwell(T, a, b, R)
    assert rv < sv < rho_c < sl < rl
    p = lambda r: float(eos.p_eos(r, T, a, b, R))
    for s, sign in [(sv, +1), (sl, -1)]:
        h = 1e-3 * s
        # a local maximum (sign +1) or minimum (sign -1)
        assert sign * (p(s) - p(s + h)) > 0 and sign * (p(s) - p(s - h)) > 0
        assert abs((p(s + 1e-6 * s) - p(s - 1e-6 * s)) / (2e-6 * s)) < 1e-7 * abs(p(s)) / s + 1e-12


def test_branch_density_inverts_eos():
    a, b, R = 0.25, 4.0, 1.0
    _, T_c, _ = eos.critical_point(a, b, R)
    T = 0.8 * T_c
    rv, rl, ps = eos.maxwell(T, a, b, R)
    assert eos.branch_density(ps, T, a, b, R, "vapour") == pytest.approx(rv, rel=1e-12)
    assert eos.branch_density(ps, T, a, b, R, "liquid") == pytest.approx(rl, rel=1e-12)
