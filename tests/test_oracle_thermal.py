"""Pins of the energy-equation oracle (oracle/thermal.py): exactness of the stencils on
polynomials, the steady linear conduction profile of Eq. Temp_Profile, the discrete decay
rate of a diffusing Fourier mode through Heun's RK2, and the C-S (dp/dT)_rho."""
import numpy as np
import pytest

from oracle import eos, lbm, thermal

A, B, R = 0.25, 4.0, 1.0
RHO_C, T_C, P_C = eos.critical_point(A, B, R)


def params(nx, ny):
    return lbm.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=0.8 * T_C)


def test_dp_dT_matches_finite_difference_of_eos():
    p = params(1, 1)
    rho = np.linspace(0.01, 0.4, 40)
    h = 1e-7 * T_C
    fd = (eos.p_eos(rho, p.T + h, A, B, R) - eos.p_eos(rho, p.T - h, A, B, R)) / (2 * h)
    np.testing.assert_allclose(thermal.dp_dT(rho, p), fd, rtol=1e-7)


def test_linear_conduction_profile_is_steady():
    """With u = 0 and T linear between T_bot and T_top at the wall positions, every term
    of Eq. Energy_Equation vanishes (Eq. Temp_Profile)."""
    ny, nx = 30, 6
    th = thermal.Thermal(T_bot=0.95 * T_C, T_top=0.80 * T_C)
    T = thermal.linear_profile(ny, nx, th.T_bot, th.T_top)
    rho = np.full((ny, nx), 0.2)
    z = np.zeros_like(rho)
    r = thermal.rate(T, rho, z, z, params(nx, ny), th)
    assert np.max(np.abs(r)) < 1e-18
    np.testing.assert_array_equal(thermal.energy_step(T, rho, z, z, params(nx, ny), th), T)


def test_stencils_exact_on_linear_and_quadratic_fields():
    ny, nx = 12, 10
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    phi = 0.3 + 0.02 * Y
    pad = thermal.with_ghosts(phi, lambda r: 2 * (0.3 - 0.01) - r, lambda r: 2 * (0.3 + 0.02 * (ny - 0.5)) - r)
    gx, gy = thermal.gradient(pad)
    np.testing.assert_allclose(gy, 0.02, rtol=1e-13)
    np.testing.assert_allclose(gx, 0.0, atol=1e-16)
    # quadratic in y on interior rows: the lattice Laplacian of q y^2 is 2 q
    q = 1e-3
    phi = q * Y**2
    pad = thermal.with_ghosts(phi, lambda r: r * 0 + q, lambda r: r * 0 + q * ny**2)
    lap = thermal.laplacian(pad)
    np.testing.assert_allclose(lap[1:-1], 2 * q, rtol=1e-12)
    # divergence of u = (alpha x, beta y) away from the periodic seam and the walls
    ux = 1e-3 * X
    uy = 2e-3 * Y
    uxp = thermal.with_ghosts(ux, lambda r: r, lambda r: r)
    uyp = thermal.with_ghosts(uy, lambda r: r - 2e-3, lambda r: r + 2e-3)
    div = thermal.divergence(uxp, uyp)
    np.testing.assert_allclose(div[1:-1, 1:-1], 3e-3, rtol=1e-12)


def test_diffusing_mode_decays_at_the_discrete_rate():
    """u = 0, uniform rho: a mode cos(k x) decays each Heun step by 1 + z + z^2/2 with
    z = D lambda(k), D = kappa/(rho c_v), lambda(k) = (2/cs^2) sum_i w_i (cos(k c_ix) - 1).
    Checked on the middle row of 9, out of reach of the wall ghosts for both stages."""
    nx, ny = 32, 9
    T0, amp, rho0 = 0.8 * T_C, 1e-3 * T_C, 0.1
    th = thermal.Thermal(c_v=5.0, kappa=0.02, T_bot=T0, T_top=T0)
    k = 2 * np.pi * 3 / nx
    mode = np.cos(k * np.arange(nx, dtype=float))
    T = T0 + amp * mode[None, :] * np.ones((ny, 1))
    rho = np.full_like(T, rho0)
    z = np.zeros_like(T)
    lam = 2 / lbm.CS2 * sum(lbm.W[i] * (np.cos(k * lbm.C[i, 0]) - 1) for i in range(9))
    zz = th.kappa / (rho0 * th.c_v) * lam
    Tn = thermal.energy_step(T, rho, z, z, params(nx, ny), th)
    sel = np.abs(mode) > 0.5
    np.testing.assert_allclose((Tn[4, sel] - T0) / (amp * mode[sel]), 1 + zz + zz**2 / 2, rtol=1e-10)


def test_zou_he_walls_hold_the_wall_temperatures():
    """Wet-node walls: the wall rows keep T_bot, T_top, and the linear profile between the
    wall nodes is steady at rest (every term of Eq. Energy_Equation vanishes)."""
    from dataclasses import replace

    p = replace(params(6, 14), wall="zou-he")
    th = thermal.Thermal(T_bot=0.9 * T_C, T_top=0.8 * T_C)
    T = thermal.linear_profile(14, 6, th.T_bot, th.T_top, wall="zou-he")
    assert np.all(T[0] == th.T_bot) and np.all(T[-1] == th.T_top)
    rho = np.full((14, 6), 0.2)
    z = np.zeros((14, 6))
    np.testing.assert_allclose(thermal.rate(T, rho, z, z, p, th), 0.0, atol=1e-18)
    rng = np.random.default_rng(2)
    T2 = thermal.energy_step(T, rho, 1e-3 * rng.random((14, 6)), 1e-3 * rng.random((14, 6)), p, th)
    assert np.all(T2[0] == th.T_bot) and np.all(T2[-1] == th.T_top)


def test_first_step_advances_T_with_the_fields_of_its_own_time_level():
    """Coupling order (the paper gives none): T^n advances with rho^n and u^n. From rest at
    uniform density and temperature those are rho0 and, by Eq. Momentum with no momentum,
    u = F / (2 rho0) = g / 2 at every node (F = rho0 g; uniform psi exerts no Shan-Chen
    force) - so the first step's T must be the Heun update with exactly these hand-built
    fields, and not the one with the velocity after the step."""
    nx, ny = 6, 10
    rho0, gy = 0.3, -1e-3
    p = lbm.Params(nx=nx, ny=ny, a=A, b=B, R=R, T=0.9 * T_C, g=(0.0, gy), form=1)
    th = thermal.Thermal(T_bot=0.9 * T_C, T_top=0.9 * T_C)
    T = np.full((ny, nx), 0.9 * T_C)
    fstar = lbm.init_state(np.full((ny, nx), rho0))
    f1, T1 = thermal.thermal_step(fstar, T, p, th)
    rho = np.full((ny, nx), rho0)
    want = thermal.energy_step(T, rho, np.zeros_like(rho), np.full_like(rho, 0.5 * gy), p, th)
    np.testing.assert_allclose(T1, want, rtol=0, atol=1e-15)
    # not vacuous: the wall ghosts u(-1) = -u(0) make div u and so the update non-zero there,
    # and the velocity after the step (about 3 g / 2 in the bulk) gives another update
    assert np.max(np.abs(T1 - T)) > 1e-7
    mac1 = lbm.macroscopic(f1, p)
    other = thermal.energy_step(T, mac1.rho, mac1.u[0], mac1.u[1], p, th)
    assert np.max(np.abs(other - T1)) > 1e-7
