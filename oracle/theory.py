"""Sharp-interface theory of the steady one-dimensional column, FP64 (test infrastructure only).

Sec. IV ("Minimal one dimensional system", "Theoretical solution") and Appendix A: at
rest (u = 0) the steady column obeys dp/dy = F_g,y(rho) (Eq. Momentum_Balance_TS) with a
linear temperature profile (Eq. Temp_Profile, constant kappa). In the sharp-interface
limit the interface at height h_i joins the Maxwell coexistence state at T(h_i)
(Eqs. MaxwellRule); above it the vapour branch and below it the liquid branch of Eq. EOS
are followed with the pressure integrated by explicit Euler steps of size dh
(Appendix A): going up p(h + dh) = p(h) + F_g,y(rho(h)) dh, going down
p(h - dh) = p(h) - F_g,y(rho(h)) dh, and rho = rho_EOS(p, T) on the branch
(Eq. Inverse_EOS). The interface height is the one whose profile has the prescribed mean
density (Sec. IV: "adapt the location of the interface until the desired average density
is achieved"), found by bisection (the mean falls monotonically as h_i falls). A branch
that runs out - the pressure leaves the range between the spinodal pressure and the
branch's other end - means no stable solution exists (the paper's criterion for a new
phase to form).

Geometry reading: the walls sit at y = 0 and y = H of a continuous coordinate; with
halfway bounce-back, node j of an ny-row lattice sits at y = j + 1/2 and H = ny. The wall
temperatures T_bot, T_top are the values at y = 0 and y = H. Gravity: F_g,y = rho g_y
(Eq. Gravity_1) or (rho - <rho>) g_y (Eq. Gravity_2), g_y < 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import eos


@dataclass
class Column:
    """Set-up of the 1-D problem (lattice units)."""

    H: float          # distance between the walls
    T_bot: float
    T_top: float
    mean_rho: float   # prescribed <rho>
    g_y: float        # gravity (negative: downward)
    form: int         # 1: rho g, 2: (rho - <rho>) g
    a: float = 0.5
    b: float = 4.0
    R: float = 1.0


@dataclass
class Solution:
    h_i: float        # interface height
    T_i: float
    p_i: float
    rho_v_i: float
    rho_l_i: float
    y_l: np.ndarray   # liquid: integration points from 0 up to h_i, increasing
    rho_l: np.ndarray
    p_l: np.ndarray
    y_v: np.ndarray   # vapour: from h_i up to H
    rho_v: np.ndarray
    p_v: np.ndarray


class NoSolution(Exception):
    """A branch reached its end: no stable sharp-interface solution (Sec. IV)."""

    def __init__(self, where, y):
        super().__init__(f"{where} branch ends at y = {y:.4f}")
        self.where = where
        self.y = y


def temperature(c: Column, y):
    """Eq. Temp_Profile with T(0) = T_bot and T(H) = T_top."""
    return c.T_bot + (c.T_top - c.T_bot) * np.asarray(y, dtype=np.float64) / c.H


def force(c: Column, rho):
    return c.g_y * (rho if c.form == 1 else rho - c.mean_rho)


def _branch_rho(c: Column, p, T, branch, guess):
    """rho_EOS(p, T) on a branch (Eq. Inverse_EOS), or None when p lies outside the branch's
    range. Newton from the neighbouring point's density while it stays close and on a rising
    part of the isotherm; otherwise the exact route: the spinodals bound the branch and
    bisection finds the root."""
    x = guess
    for _ in range(20):
        fx = float(eos.p_eos(x, T, c.a, c.b, c.R)) - p
        d = float(eos.dp_drho(x, T, c.a, c.b, c.R))
        if not d > 0.0:
            break
        xn = x - fx / d
        if not (0.8 * guess < xn < 1.25 * guess):
            break
        if abs(xn - x) <= 1e-13 * x:  # quadratic convergence: the next step is at rounding level
            return xn
        x = xn
    rs_v, rs_l = eos.spinodals(T, c.a, c.b, c.R)
    if branch == "vapour":
        if p <= 0.0 or p >= float(eos.p_eos(rs_v, T, c.a, c.b, c.R)):
            return None
    elif p <= float(eos.p_eos(rs_l, T, c.a, c.b, c.R)):
        return None
    return eos.branch_density(p, T, c.a, c.b, c.R, branch)


def integrate(c: Column, h_i, dh):
    """Profile for the interface at h_i (Appendix A); raises NoSolution."""
    T_i = float(temperature(c, h_i))
    rho_v, rho_l, p_i = eos.maxwell(T_i, c.a, c.b, c.R)
    phases = {}
    for branch, direction, end in (("vapour", 1.0, c.H), ("liquid", -1.0, 0.0)):
        y, rho, p = h_i, (rho_v if branch == "vapour" else rho_l), p_i
        ys, rs, ps = [y], [rho], [p]
        while (end - y) * direction > 0.0:
            step = min(dh, abs(end - y))
            p = p + direction * force(c, rho) * step
            y = y + direction * step
            rho = _branch_rho(c, p, float(temperature(c, y)), branch, rho)
            if rho is None:
                raise NoSolution(branch, y)
            ys.append(y)
            rs.append(rho)
            ps.append(p)
        order = slice(None) if direction > 0 else slice(None, None, -1)
        phases[branch] = (np.array(ys)[order], np.array(rs)[order], np.array(ps)[order])
    (yl, rl, pl), (yv, rv, pv) = phases["liquid"], phases["vapour"]
    return Solution(h_i, T_i, p_i, rho_v, rho_l, yl, rl, pl, yv, rv, pv)


def mean_density(sol: Solution, H):
    """(1/H) times the integral of rho over [0, H] (trapezoid rule in each phase)."""
    return (np.trapezoid(sol.rho_l, sol.y_l) + np.trapezoid(sol.rho_v, sol.y_v)) / H


def _mean_or_failure(c, h_i, dh):
    try:
        return mean_density(integrate(c, h_i, dh), c.H), None
    except NoSolution as e:
        return None, e


def solve(c: Column, dh=0.02, tol=1e-10, scan=64):
    """Interface height whose profile has mean density c.mean_rho. Interface heights whose
    profile runs off a branch are not candidates: a coarse scan of `scan` heights brackets
    the prescribed mean between two candidates with profiles, then bisection (the mean
    rises with h_i) narrows it. Raises NoSolution when no candidate profile brackets the
    prescribed mean: the failure of the nearest candidate without a profile is reported."""
    hs = (np.arange(scan) + 0.5) * c.H / scan
    res = [_mean_or_failure(c, h, dh) for h in hs]
    for k in range(scan - 1):
        (m0, _), (m1, _) = res[k], res[k + 1]
        if m0 is not None and m1 is not None and m0 <= c.mean_rho <= m1:
            lo, hi = hs[k], hs[k + 1]
            break
    else:
        # no bracket: report the branch failure nearest to where the mean would be met
        valid = [(h, m) for h, (m, _) in zip(hs, res) if m is not None]
        fails = [(h, e) for h, (_, e) in zip(hs, res) if e is not None]
        if not fails:
            raise ValueError("mean density outside the range of one-interface columns")
        if valid:
            side_hi = all(m < c.mean_rho for _, m in valid)
            ref = max(h for h, _ in valid) if side_hi else min(h for h, _ in valid)
            raise min(fails, key=lambda he: abs(he[0] - ref))[1]
        raise fails[len(fails) // 2][1]
    while hi - lo > tol * c.H:
        mid = 0.5 * (lo + hi)
        m, e = _mean_or_failure(c, mid, dh)
        if m is None:
            raise e
        if m > c.mean_rho:
            hi = mid
        else:
            lo = mid
    return integrate(c, 0.5 * (lo + hi), dh)


def at_nodes(sol: Solution, ny, offset=0.5):
    """rho and p at the nodes y = j + offset of an ny-row lattice, by linear interpolation
    within each phase: offset 1/2 with halfway bounce-back walls (H = ny), 0 with wet-node
    walls on the rows 0 and ny - 1 (H = ny - 1)."""
    yc = np.arange(ny) + offset
    liq = yc < sol.h_i
    rho = np.where(liq, np.interp(yc, sol.y_l, sol.rho_l), np.interp(yc, sol.y_v, sol.rho_v))
    p = np.where(liq, np.interp(yc, sol.y_l, sol.p_l), np.interp(yc, sol.y_v, sol.p_v))
    return rho, p
