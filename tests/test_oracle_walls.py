"""Pins of the oracle's two wall treatments against the closed form of a body-force-driven
channel (plane Poiseuille flow): a single-phase, uniform-density lattice (psi uniform, so
F_int = 0) driven by g_x between the walls reaches u_x(y) = g_x d1 d2 / (2 nu) with
nu = (tau_nu - 1/2)/3 and d1, d2 the distances to the two walls.
* halfway bounce-back: walls at y = -1/2 and ny - 1/2; exact for the MRT/TRT "magic"
  combination (tau_nu - 1/2)(tau_q - 1/2) = 3/16 (Ginzburg's wall-location condition);
* Zou-He wet nodes: walls on the nodes 0 and ny - 1 (u = 0 there by construction)."""
import numpy as np
import pytest

from oracle import eos
from oracle import lbm as olbm

A, B, R = 0.25, 4.0, 1.0
RHO_C, T_C, _ = eos.critical_point(A, B, R)


def channel(wall, ny, tau_q, steps):
    p = olbm.Params(nx=4, ny=ny, a=A, b=B, R=R, T=1.5 * T_C, g=(1e-6, 0.0), form=1, tau_q=tau_q, wall=wall)
    f = olbm.init_state(np.full((ny, 4), 0.1))
    for _ in range(steps):
        f = olbm.step(f, p)
    mac = olbm.macroscopic(f, p)
    return p, mac


def test_bounce_back_channel_is_exact_at_the_magic_combination():
    ny = 10
    p, mac = channel("bounce-back", ny, 0.875, 6000)
    y = np.arange(ny) + 0.5
    nu = (p.tau_nu - 0.5) / 3.0
    want = p.g[0] / (2.0 * nu) * y * (ny - y)
    np.testing.assert_allclose(mac.u[0][:, 0], want, rtol=1e-9)
    assert np.max(np.abs(mac.u[1])) < 1e-15
    np.testing.assert_allclose(mac.rho, 0.1, rtol=1e-11)  # rounding drift of 6000 steps


def test_zou_he_channel_has_walls_on_the_nodes():
    ny = 11
    p, mac = channel("zou-he", ny, 1.0, 6000)
    y = np.arange(ny, dtype=float)
    nu = (p.tau_nu - 0.5) / 3.0
    want = p.g[0] / (2.0 * nu) * y * (ny - 1 - y)
    assert np.max(np.abs(mac.u[0][:, 0] - want)) <= 1e-9 * np.max(want)
    assert np.max(np.abs(mac.u[0][[0, -1]])) <= 1e-15
    assert np.max(np.abs(mac.u[1])) < 1e-14


def test_zou_he_wall_nodes_have_zero_velocity_each_step():
    """Under gravity along y (both forms) and a non-equilibrium start, every step's wall
    nodes carry u = 0 including the half force (the defining property), and F_int = 0."""
    rng = np.random.default_rng(3)
    for form in (1, 2):
        p = olbm.Params(nx=4, ny=12, a=A, b=B, R=R, T=0.85 * T_C, g=(3e-6, -2e-5), form=form, wall="zou-he")
        rho0 = np.linspace(0.28, 0.04, 12)[:, None] * np.ones((1, 4))
        f = olbm.init_state(rho0) * (1.0 + 1e-3 * (rng.random((9, 12, 4)) - 0.5))
        for _ in range(5):
            mac = olbm.macroscopic(f, p)
            assert np.max(np.abs(mac.u[0][[0, -1]])) < 1e-16
            assert np.max(np.abs(mac.u[1][[0, -1]])) < 1e-16
            f = olbm.step(f, p)
