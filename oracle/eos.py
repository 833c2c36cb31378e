"""Carnahan-Starling thermodynamics in FP64 (oracle; test infrastructure only).

Follows Sec. IV of Czelusniak, Cabezas Gomez & Wagner (arXiv 2301.12869):

* Eq. EOS            p = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2,
                     with eta = b rho / 4.
* critical point     the state where dp/drho = d2p/drho2 = 0 (the paper quotes
                     its consequences a ~ 3.8533 p_c/rho_c^2, b ~ 0.5218/rho_c,
                     R ~ 2.7864 p_c/(rho_c T_c) after Eq. EOS).
* spinodals          the local maximum and minimum of p(rho) at fixed T
                     (Sec. V, the "lines of unconditional instability").
* Eqs. MaxwellRule   int_{rho_v}^{rho_l} (p_i - p(rho, T)) drho / rho^2 = 0 with
                     p(rho_v) = p(rho_l) = p_i.

Only this module and ``oracle.lbm`` implement the oracle's arithmetic; nothing
here is shared with the CUDA library, which carries its own host-side solver.
Library primitives used as steps: ``numpy.polynomial`` (polynomial products,
derivatives and roots) and ``numpy.polynomial.legendre.leggauss`` (quadrature
nodes). Everything else is written out.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import Polynomial

__all__ = [
    "p_eos",
    "dp_drho",
    "critical_point",
    "spinodals",
    "branch_density",
    "maxwell",
    "maxwell_integral",
]

# N(eta) = eta (1 + eta + eta^2 - eta^3) and D(eta) = (1 - eta)^3, so that
# p = (4 R T / b) N / D - a (4 eta / b)^2.  (Eq. EOS with rho = 4 eta / b.)
_N = Polynomial([0.0, 1.0, 1.0, 1.0, -1.0])
_D = Polynomial([1.0, -1.0]) ** 3
# A = N' D - N D' is the numerator of (N/D)' = A / D^2.
_A = _N.deriv() * _D - _N * _D.deriv()


def p_eos(rho, T, a, b, R):
    """Carnahan-Starling pressure, Eq. EOS (Sec. IV), element-wise in FP64."""
    rho = np.asarray(rho, dtype=np.float64)
    eta = b * rho / 4.0
    return rho * R * T * (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3 - a * rho**2


def dp_drho(rho, T, a, b, R):
    """(dp/drho)_T of Eq. EOS: R T (N/D)'(eta) - 2 a rho, written via A/D^2."""
    rho = np.asarray(rho, dtype=np.float64)
    eta = b * rho / 4.0
    return R * T * _A(eta) / _D(eta) ** 2 - 2.0 * a * rho


def critical_point(a, b, R):
    """Critical point of Eq. EOS: dp/drho = 0 and d2p/drho2 = 0.

    Writing p = (4RT/b) F(eta) - a rho^2 with F = N/D, the two conditions are
    R T F'(eta) = 2 a rho and (b/4) R T F''(eta) = 2 a. Their ratio removes T
    and leaves F'(eta) = eta F''(eta), i.e. the polynomial
    A D - eta (A' D - 2 A D') = 0 on 0 < eta < 1 (multiplied by D^3 > 0).
    Returns (rho_c, T_c, p_c).
    """
    q = _A * _D - Polynomial([0.0, 1.0]) * (_A.deriv() * _D - 2.0 * _A * _D.deriv())
    roots = [r.real for r in q.roots() if abs(r.imag) < 1e-12 and 0.0 < r.real < 1.0]
    if len(roots) != 1:
        raise ValueError(f"expected one critical root in (0,1), got {roots}")
    eta_c = _bisect(lambda e: float(q(e)), roots[0] - 1e-6, roots[0] + 1e-6)
    # F'' = (A' D - 2 A D') / D^3
    fpp = (_A.deriv()(eta_c) * _D(eta_c) - 2.0 * _A(eta_c) * _D.deriv()(eta_c)) / _D(eta_c) ** 3
    rho_c = 4.0 * eta_c / b
    T_c = 8.0 * a / (b * R * fpp)
    p_c = float(p_eos(rho_c, T_c, a, b, R))
    return rho_c, T_c, p_c


def spinodals(T, a, b, R):
    """Densities of the local maximum (vapour side) and minimum (liquid side)
    of p(rho) at fixed T < T_c (Sec. V). Returns (rho_s_vapour, rho_s_liquid).

    dp/drho = 0 is R T A(eta) - (8 a / b) eta D(eta)^2 = 0 after multiplying by
    D^2 > 0; its two roots in (0, 1) are polished by bisection on dp/drho.
    """
    poly = R * T * _A - (8.0 * a / b) * Polynomial([0.0, 1.0]) * _D**2
    # A(1) = 0 and D(1) = 0, so eta = 1 (the packing limit, not a state) is a
    # root of the multiplied-out polynomial; only 0 < eta < 0.99 is physical.
    roots = sorted(r.real for r in poly.roots() if abs(r.imag) < 1e-9 and 0.0 < r.real < 0.99)
    if len(roots) != 2:
        raise ValueError(f"T={T} is not below the critical temperature (spinodal roots {roots})")
    out = []
    for r in roots:
        rho0 = 4.0 * r / b
        h = 1e-7 * rho0
        out.append(_bisect(lambda x: float(dp_drho(x, T, a, b, R)), rho0 - h, rho0 + h))
    return out[0], out[1]


def branch_density(p, T, a, b, R, branch):
    """Inverse of Eq. EOS on a stable/metastable branch (Sec. IV, Eq. Inverse_EOS).

    ``branch`` is "vapour" (0 < rho < spinodal maximum) or "liquid" (spinodal
    minimum < rho < 4/b). p(rho) increases monotonically on both, so the root
    is found by bisection.
    """
    rs_v, rs_l = spinodals(T, a, b, R)
    f = lambda x: float(p_eos(x, T, a, b, R)) - p
    if branch == "vapour":
        return _bisect(f, 1e-300, rs_v)
    if branch == "liquid":
        return _bisect(f, rs_l, (4.0 / b) * (1.0 - 1e-12))
    raise ValueError(branch)


_GL_X, _GL_W = np.polynomial.legendre.leggauss(256)


def maxwell_integral(p_i, rho_v, rho_l, T, a, b, R):
    """Left side of Eq. Integral_MaxwellRule by 256-point Gauss-Legendre."""
    half = 0.5 * (rho_l - rho_v)
    rho = 0.5 * (rho_l + rho_v) + half * _GL_X
    return half * float(np.sum(_GL_W * (p_i - p_eos(rho, T, a, b, R)) / rho**2))


def maxwell(T, a, b, R):
    """Coexistence state of Eqs. MaxwellRule at temperature T < T_c.

    For a trial interface pressure p_i between the spinodal pressures, rho_v and
    rho_l are the vapour- and liquid-branch roots of p(rho) = p_i
    (Eq. Pressures_MaxwellRule). The integral of Eq. Integral_MaxwellRule grows
    monotonically with p_i (its derivative is int drho/rho^2 > 0), so p_i is
    found by bisection. Returns (rho_v, rho_l, p_sat).
    """
    rs_v, rs_l = spinodals(T, a, b, R)
    p_max = float(p_eos(rs_v, T, a, b, R))
    p_min = float(p_eos(rs_l, T, a, b, R))
    lo = max(p_min, 0.0) + 1e-14 * abs(p_max)
    hi = p_max * (1.0 - 1e-13)

    def integral(p_i):
        rv = _bisect(lambda x: float(p_eos(x, T, a, b, R)) - p_i, 1e-300, rs_v)
        rl = _bisect(lambda x: float(p_eos(x, T, a, b, R)) - p_i, rs_l, (4.0 / b) * (1.0 - 1e-12))
        return maxwell_integral(p_i, rv, rl, T, a, b, R), rv, rl

    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if not (lo < mid < hi):
            break
        val, _, _ = integral(mid)
        if val > 0.0:
            hi = mid
        else:
            lo = mid
    p_sat = 0.5 * (lo + hi)
    _, rho_v, rho_l = integral(p_sat)
    return rho_v, rho_l, p_sat


def _bisect(f, lo, hi):
    """Plain bisection to the last representable midpoint; f(lo), f(hi) must differ in sign."""
    flo, fhi = f(lo), f(hi)
    if flo == 0.0:
        return lo
    if fhi == 0.0:
        return hi
    if (flo > 0.0) == (fhi > 0.0):
        raise ValueError(f"no sign change on [{lo}, {hi}]: {flo}, {fhi}")
    for _ in range(2000):
        mid = 0.5 * (lo + hi)
        if not (lo < mid < hi):
            break
        fm = f(mid)
        if fm == 0.0:
            return mid
        if (fm > 0.0) == (flo > 0.0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)
