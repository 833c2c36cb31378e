"""Energy equation of the thermal variant, FP64 oracle (test infrastructure only).

Sec. III, Eq. Energy_Equation:

    dT/dt = -u . grad T + (1/(rho c_v)) div(kappa grad T) - (T/(rho c_v)) (dp_EOS/dT)_rho div u

with constant kappa (the paper's choice, Sec. IV), so div(kappa grad T) = kappa lap T,
and (dp_EOS/dT)_rho = rho R Z(eta) for the Carnahan-Starling EOS of Eq. EOS,
Z = (1 + eta + eta^2 - eta^3) / (1 - eta)^3, eta = b rho / 4.

Readings (the paper names the stencil family and the Runge-Kutta scheme without
printing them; each is listed in the design notes):
* second-order isotropic central differences weighted with the D2Q9 lattice
  weights: d_a phi = (1/cs^2) sum_i w_i c_ia phi(x + c_i) and
  lap phi = (2/cs^2) sum_i w_i (phi(x + c_i) - phi(x));
* Heun's second-order Runge-Kutta with the lattice time step dt = 1, rho and u
  held fixed during the step;
* the energy update of a time step advances T^n with rho^n and u^n, the density and
  the half-force velocity that step itself forms from the streamed populations (with
  the force of T^n): every field of the right-hand side at the time level of T^n, an
  explicit step of the coupled system;
* walls: T = T_bot on the wall below row 0 and T_top above row ny-1 (half a link
  beyond the last rows, as for the populations), by ghost rows
  T(-1) = 2 T_bot - T(0), T(ny) = 2 T_top - T(ny-1); velocity ghosts vanish at the
  wall the same way (u(-1) = -u(0)); x is periodic. With Zou-He wet-node walls the
  walls are the rows 0 and ny-1 themselves: T is held at T_bot and T_top there and only
  the rows between are advanced (the wall nodes' velocity is zero by construction).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass

import numpy as np

from . import lbm

C = lbm.C
W = lbm.W
CS2 = lbm.CS2


@dataclass
class Thermal:
    """Energy-equation parameters: c_v = 5 and kappa = 0.02 in the paper (Sec. IV)."""

    c_v: float = 5.0
    kappa: float = 0.02
    T_bot: float = 0.0
    T_top: float = 0.0


def dp_dT(rho, p):
    """(dp_EOS/dT) at fixed rho for Eq. EOS: rho R Z(eta)."""
    eta = p.b * rho / 4.0
    return rho * p.R * (1.0 + eta + eta**2 - eta**3) / (1.0 - eta) ** 3


def with_ghosts(phi, low, high):
    """Pad phi[y, x] with one ghost row below and above: phi(-1) = low(phi(0)),
    phi(ny) = high(phi(ny-1))."""
    return np.vstack([low(phi[:1]), phi, high(phi[-1:])])


def neighbour(padded, i):
    """phi(x + c_i) for every node of the unpadded lattice (x periodic)."""
    cx, cy = int(C[i, 0]), int(C[i, 1])
    ny = padded.shape[0] - 2
    rows = padded[1 + cy : 1 + cy + ny]
    return np.roll(rows, -cx, axis=1)


def gradient(padded):
    gx = sum(W[i] * C[i, 0] * neighbour(padded, i) for i in range(9)) / CS2
    gy = sum(W[i] * C[i, 1] * neighbour(padded, i) for i in range(9)) / CS2
    return gx, gy


def laplacian(padded):
    centre = padded[1:-1]
    return 2.0 / CS2 * sum(W[i] * (neighbour(padded, i) - centre) for i in range(9))


def divergence(ux_p, uy_p):
    return sum(W[i] * (C[i, 0] * neighbour(ux_p, i) + C[i, 1] * neighbour(uy_p, i)) for i in range(9)) / CS2


def rate(T, rho, ux, uy, p, th):
    """Right-hand side of Eq. Energy_Equation on the lattice (zero on wet-node wall rows)."""
    if p.wall == "zou-he":
        Tp = with_ghosts(T, lambda r: r, lambda r: r)  # ghosts unused: the wall rows do not move
    else:
        Tp = with_ghosts(T, lambda r: 2.0 * th.T_bot - r, lambda r: 2.0 * th.T_top - r)
    uxp = with_ghosts(ux, lambda r: -r, lambda r: -r)
    uyp = with_ghosts(uy, lambda r: -r, lambda r: -r)
    gx, gy = gradient(Tp)
    lap = laplacian(Tp)
    div_u = divergence(uxp, uyp)
    out = -(ux * gx + uy * gy) + th.kappa / (rho * th.c_v) * lap - T * dp_dT(rho, p) / (rho * th.c_v) * div_u
    if p.wall == "zou-he":
        out[0] = 0.0
        out[-1] = 0.0
    return out


def energy_step(T, rho, ux, uy, p, th):
    """Heun's RK2 with dt = 1 (wet-node walls: the wall rows take T_bot and T_top, which may
    have changed since the last step)."""
    k1 = rate(T, rho, ux, uy, p, th)
    k2 = rate(T + k1, rho, ux, uy, p, th)
    out = T + 0.5 * (k1 + k2)
    if p.wall == "zou-he":
        out[0] = th.T_bot
        out[-1] = th.T_top
    return out


def thermal_step(fstar, T, p, th):
    """One time step of the thermal variant: the LBM step with the local temperature in
    Eq. EOS, and the energy update of T with the rho and u of that step (time level n)."""
    pT = dataclasses.replace(p, T=T)
    mac = lbm.macroscopic(fstar, pT)
    f_new = lbm.step(fstar, pT)
    return f_new, energy_step(T, mac.rho, mac.u[0], mac.u[1], p, th)


def linear_profile(ny, nx, T_bot, T_top, wall="bounce-back"):
    """Steady conduction profile between the walls (Eq. Temp_Profile with constant kappa):
    linear in y with T = T_bot at y = -1/2 and T_top at y = ny - 1/2 (bounce-back), or at the
    wall nodes y = 0 and ny - 1 (Zou-He)."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    if wall == "zou-he":
        return T_bot + (T_top - T_bot) * y / (ny - 1)
    return T_bot + (T_top - T_bot) * (y + 0.5) / ny
