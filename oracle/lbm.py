"""FP64 CPU oracle of one D2Q9 pseudopotential LBM time step (test infrastructure only).

Written from Sec. III of Czelusniak, Cabezas Gomez & Wagner (arXiv 2301.12869),
in the order and notation of the paper. Array layout: populations f[i, y, x]
(i = 0..8 in the order of Eq. VelocitySet), fields rho[y, x]; x is periodic,
y is bounded by two walls.

One step (``step``) maps the post-collision populations f* of the previous
step to the next f*:

 1. pull streaming, left side of Eq. LBE: f_i(x, y) = f*_i(x - c_ix, y - c_iy),
    x periodic; a link that would come from outside 0 <= y < ny is reflected at
    the wall half a lattice unit beyond the last row (halfway bounce-back):
    f_i(x, y) = f*_opp(i)(x, y);
 2. rho = sum_i f_i (Eq. Density);
 3. psi(rho) by Eq. InteractionPotential with p_EOS of Eq. EOS and c = 1;
 4. <rho> = mean of rho over all nodes, same step (Eq. Gravity_2);
 5. F_int by Eq. ShanChenForce, set to zero on the first and last rows
    (the rows next to the walls: "interaction force at the boundaries set
    equal to zero", Sec. III);
 6. F_g = rho g (Eq. Gravity_1) or (rho - <rho>) g (Eq. Gravity_2);
    F = F_int + F_g (Sec. III);
 7. rho u = sum_i f_i c_i + F/2 (Eq. Momentum);
 8. m = M f, m_eq = M f_eq(rho, u) with f_eq of Eq. EquilibriumDistribution
    evaluated population by population and transformed by the matrix product;
 9. the source vector S~ of Eq. LiFS (right-hand side);
10. m* = m - Lambda (m - m_eq) + (I - Lambda/2) S~  (Eqs. LBE, OperatorMRT, LiFS),
    f* = M^-1 m*, with M^-1 obtained by Gauss-Jordan elimination of M.

Readings where the paper is silent (each listed in the design notes):
* the walls are halfway bounce-back and F_int = 0 on the two wall-adjacent
  rows (the paper uses Zou-He wet nodes);
* G = -1 and c = 1 in Eq. InteractionPotential (the paper does not print G);
* if 2 (p_EOS - rho c_s^2) / (G c^2) < 0 the state is non-physical: psi is set
  to 0 there and the node is reported in the ``nonphysical`` mask;
* sigma |F_int|^2 / psi^2 is taken as printed where psi != 0; where psi = 0
  its continuous extension G^2 |sum_i w(|c_i|^2) psi(x + c_i) c_i|^2 is used
  (F_int is proportional to psi(x), so the ratio stays finite), and on the wall
  rows, where F_int is zero by the boundary rule, the term is zero.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .eos import p_eos

# ---------------------------------------------------------------- Eq. VelocitySet
C = np.array(
    [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)],
    dtype=np.int64,
)
# weights w_i and sound speed (text after Eq. EquilibriumDistribution)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
CS2 = 1.0 / 3.0
# opposite direction of each velocity: c_opp(i) = -c_i
OPP = np.array([int(np.flatnonzero((C == -C[i]).all(axis=1))[0]) for i in range(9)])
# Shan-Chen weights w(|c_i|^2): w(1) = 1/3, w(2) = 1/12 (text after Eq. ShanChenForce)
W_SC = np.array([0.0] + [1 / 3] * 4 + [1 / 12] * 4, dtype=np.float64)

# ---------------------------------------------------------------- Eq. MatrixMRT
M = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1],
    ],
    dtype=np.float64,
)


def gauss_jordan_inverse(A):
    """Inverse of a square matrix by Gauss-Jordan elimination with partial pivoting."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    aug = np.hstack([A, np.eye(n)])
    for col in range(n):
        piv = col + int(np.argmax(np.abs(aug[col:, col])))
        if aug[piv, col] == 0.0:
            raise ValueError("singular matrix")
        aug[[col, piv]] = aug[[piv, col]]
        aug[col] /= aug[col, col]
        for row in range(n):
            if row != col:
                aug[row] -= aug[row, col] * aug[col]
    return aug[:, n:]


MINV = gauss_jordan_inverse(M)


@dataclass
class Params:
    """Parameters of one column / domain (all lattice units).

    ``T`` is the absolute temperature; ``g`` = (g_x, g_y) is the gravitational
    acceleration (the paper's downward g > 0 is g_y = -g here); ``form`` is 1
    for Eq. Gravity_1 and 2 for Eq. Gravity_2. The relaxation times are named
    as in Eq. RelaxationMatrix; the paper sets all of them to 1 and
    sigma = 1.385 (Sec. IV, "Comparison between theoretical solution and LBM").
    """

    nx: int
    ny: int
    a: float = 0.25
    b: float = 4.0
    R: float = 1.0
    T: float = 0.0
    G: float = -1.0
    sigma: float = 1.385
    tau_rho: float = 1.0
    tau_e: float = 1.0
    tau_varsigma: float = 1.0
    tau_j: float = 1.0
    tau_q: float = 1.0
    tau_nu: float = 1.0
    g: tuple = (0.0, 0.0)
    form: int = 1
    wall: str = "bounce-back"   # or "zou-he" (wet-node walls on rows 0 and ny-1, Sec. III)

    def Lambda(self):
        """Eq. RelaxationMatrix."""
        return np.diag(
            1.0
            / np.array(
                [
                    self.tau_rho,
                    self.tau_e,
                    self.tau_varsigma,
                    self.tau_j,
                    self.tau_q,
                    self.tau_j,
                    self.tau_q,
                    self.tau_nu,
                    self.tau_nu,
                ],
                dtype=np.float64,
            )
        )


# ---------------------------------------------------------------- building blocks
def equilibrium(rho, ux, uy):
    """Eq. EquilibriumDistribution, population by population:
    f_i^eq = w_i (rho + c_ia rho u_a / cs^2 + (c_ia c_ib - cs^2 d_ab) rho u_a u_b / (2 cs^4)).
    """
    feq = np.empty((9,) + np.shape(rho), dtype=np.float64)
    u = (ux, uy)
    for i in range(9):
        lin = sum(C[i, al] * rho * u[al] for al in range(2)) / CS2
        quad = 0.0
        for al in range(2):
            for be in range(2):
                quad = quad + (C[i, al] * C[i, be] - CS2 * (al == be)) * rho * u[al] * u[be]
        feq[i] = W[i] * (rho + lin + quad / (2.0 * CS2**2))
    return feq


def stream(fstar):
    """Pull streaming of Eq. LBE with periodic x and halfway bounce-back walls in y.

    f_i(x, y) = f*_i(x - c_ix, y - c_iy); when y - c_iy falls outside the
    lattice the link crosses a wall, and the population that left (x, y) towards
    that wall comes back reversed: f_i(x, y) = f*_opp(i)(x, y).
    """
    f = np.empty_like(fstar)
    for i in range(9):
        cx, cy = int(C[i, 0]), int(C[i, 1])
        # shifted[y, x] = f*_i(x - c_ix, y): periodic shift along x
        shifted = np.roll(fstar[i], cx, axis=1)
        if cy == 0:
            f[i] = shifted
        elif cy == 1:
            f[i, 1:] = shifted[:-1]          # from row y - 1
            f[i, 0] = fstar[OPP[i], 0]       # link from below the bottom wall
        else:
            f[i, :-1] = shifted[1:]          # from row y + 1
            f[i, -1] = fstar[OPP[i], -1]     # link from above the top wall
    return f


def zou_he(f, p, mean_rho):
    """Wet-node no-slip walls on rows 0 and ny - 1 (Sec. III cites Zou and He for the solid
    walls): after streaming, the populations that would enter each wall node from outside
    (bottom: c_y = +1, i = 2, 5, 6; top: c_y = -1, i = 4, 7, 8) are set so that the node's
    velocity of Eq. Momentum - including the half force - vanishes, with the non-equilibrium
    part of the normal population bounced back (f_2 - f_2^eq = f_4 - f_4^eq at u = 0).
    At the wall nodes F_int = 0 (Sec. III boundary rule), so F = F_g, whose rho dependence
    makes the wall density the solution of a linear equation: bottom
    rho = K - F_y/2, K = f0 + f1 + f3 + 2 (f4 + f7 + f8); top rho = K + F_y/2,
    K = f0 + f1 + f3 + 2 (f2 + f5 + f6). Modifies f in place."""
    gx, gy = p.g
    for row, sgn in ((0, 1.0), (-1, -1.0)):
        q = f[:, row]
        if sgn > 0:
            K = q[0] + q[1] + q[3] + 2.0 * (q[4] + q[7] + q[8])
        else:
            K = q[0] + q[1] + q[3] + 2.0 * (q[2] + q[5] + q[6])
        # rho (1 + sgn gy / 2) = K (form 1); = K + sgn <rho> gy / 2 (form 2)
        if p.form == 1:
            rho = K / (1.0 + sgn * 0.5 * gy)
            base = rho
        else:
            rho = (K + sgn * 0.5 * mean_rho * gy) / (1.0 + sgn * 0.5 * gy)
            base = rho - mean_rho
        Fx, Fy = base * gx, base * gy
        d13 = q[1] - q[3]
        if sgn > 0:
            q[2] = q[4]
            q[5] = q[7] - 0.5 * d13 - 0.25 * (Fx + Fy)
            q[6] = q[8] + 0.5 * d13 + 0.25 * (Fx - Fy)
        else:
            q[4] = q[2]
            q[7] = q[5] + 0.5 * d13 + 0.25 * (Fx + Fy)
            q[8] = q[6] - 0.5 * d13 + 0.25 * (Fy - Fx)
    return f


def density(f):
    """Eq. Density."""
    return f.sum(axis=0)


def interaction_potential(rho, p):
    """Eq. InteractionPotential with c = 1: psi = sqrt(2 (p_EOS - rho cs^2) / G).

    Returns (psi, nonphysical) where ``nonphysical`` marks nodes whose radicand
    is negative or not finite (psi is set to 0 there).
    """
    radicand = 2.0 * (p_eos(rho, p.T, p.a, p.b, p.R) - rho * CS2) / p.G
    bad = ~(radicand >= 0.0)
    psi = np.sqrt(np.where(bad, 0.0, radicand))
    return psi, bad


def shan_chen_sum(psi):
    """S_a(x) = sum_i w(|c_i|^2) psi(x + c_i) c_ia on rows 1..ny-2, zero on rows 0, ny-1."""
    ny, _ = psi.shape
    Sx = np.zeros_like(psi)
    Sy = np.zeros_like(psi)
    for i in range(1, 9):
        cx, cy = int(C[i, 0]), int(C[i, 1])
        nb = np.roll(psi, -cx, axis=1)       # nb[y, x] = psi(x + c_ix, y)
        rows = nb[1 + cy : ny - 1 + cy]      # psi(x + c_i) for y = 1..ny-2
        Sx[1:-1] += W_SC[i] * rows * cx
        Sy[1:-1] += W_SC[i] * rows * cy
    return Sx, Sy


def shan_chen_force(psi, G):
    """Eq. ShanChenForce, F_a = -G psi(x) S_a(x); zero on the wall-adjacent rows."""
    Sx, Sy = shan_chen_sum(psi)
    return -G * psi * Sx, -G * psi * Sy


def gravity(rho, mean_rho, p):
    """Eq. Gravity_1 (form 1: rho g) or Eq. Gravity_2 (form 2: (rho - <rho>) g)."""
    if p.form == 1:
        base = rho
    elif p.form == 2:
        base = rho - mean_rho
    else:
        raise ValueError(f"gravity form {p.form}")
    return base * p.g[0], base * p.g[1]


def velocity(f, rho, Fx, Fy):
    """Eq. Momentum: rho u = sum_i f_i c_i + F/2."""
    jx = np.tensordot(C[:, 0].astype(np.float64), f, axes=1)
    jy = np.tensordot(C[:, 1].astype(np.float64), f, axes=1)
    return (jx + 0.5 * Fx) / rho, (jy + 0.5 * Fy) / rho


def sigma_ratio(Fint_x, Fint_y, psi, Sx, Sy, G):
    """|F_int|^2 / psi^2 of Eq. LiFS, with the continuous extension where psi = 0."""
    Fint2 = Fint_x**2 + Fint_y**2
    safe = np.where(psi != 0.0, psi, 1.0)
    return np.where(psi != 0.0, Fint2 / safe**2, G * G * (Sx**2 + Sy**2))


def li_source(ux, uy, Fx, Fy, ratio, p):
    """Right-hand side S~ of Eq. LiFS, one 9-vector per node (moment order of M)."""
    uF = ux * Fx + uy * Fy
    S = np.empty((9,) + np.shape(ux), dtype=np.float64)
    S[0] = 0.0
    S[1] = 6.0 * uF + p.sigma * ratio / (p.tau_e - 0.5)
    S[2] = -6.0 * uF - p.sigma * ratio / (p.tau_varsigma - 0.5)
    S[3] = Fx
    S[4] = -Fx
    S[5] = Fy
    S[6] = -Fy
    S[7] = 2.0 * (ux * Fx - uy * Fy)
    S[8] = ux * Fy + uy * Fx
    return S


def collide(f, feq, S, p):
    """Eqs. OperatorMRT and LiFS in moment space:
    m* = m - Lambda (m - m_eq) + (I - Lambda/2) S~,  f* = M^-1 m*."""
    shape = f.shape
    Lam = p.Lambda()
    m = M @ f.reshape(9, -1)
    meq = M @ feq.reshape(9, -1)
    mstar = m - Lam @ (m - meq) + (np.eye(9) - 0.5 * Lam) @ S.reshape(9, -1)
    return (MINV @ mstar).reshape(shape)


# ---------------------------------------------------------------- the step
@dataclass
class Macro:
    """Fields of one step, as computed between streaming and collision."""

    f: np.ndarray
    rho: np.ndarray
    psi: np.ndarray
    mean_rho: float
    Fint: tuple
    Fg: tuple
    F: tuple
    u: tuple
    ratio: np.ndarray
    nonphysical: np.ndarray = field(default=None)


def macroscopic(fstar, p, mean_rho=None):
    """Steps 1-7: stream the stored f* and evaluate rho, psi, <rho>, forces and u.

    ``mean_rho`` overrides the domain mean of Eq. Gravity_2 for a caller that
    passes a patch cut out of a larger domain (whose mean it computed itself).
    """
    f = stream(fstar)
    if p.wall == "zou-he":
        # <rho> of Eq. Gravity_2: the mass of the stored state (the wall nodes' densities
        # are rebuilt below; with bounce-back the two definitions coincide)
        if mean_rho is None:
            mean_rho = float(np.sum(fstar)) / fstar[0].size
        zou_he(f, p, mean_rho)
    elif p.wall != "bounce-back":
        raise ValueError(f"wall {p.wall}")
    rho = density(f)
    psi, bad = interaction_potential(rho, p)
    if mean_rho is None:
        mean_rho = float(np.mean(rho))
    Sx, Sy = shan_chen_sum(psi)
    Fint = (-p.G * psi * Sx, -p.G * psi * Sy)
    Fg = gravity(rho, mean_rho, p)
    F = (Fint[0] + Fg[0], Fint[1] + Fg[1])
    u = velocity(f, rho, F[0], F[1])
    ratio = sigma_ratio(Fint[0], Fint[1], psi, Sx, Sy, p.G)
    # wall rows: F_int = 0 there by the boundary rule, so the sigma term vanishes
    ratio[0] = 0.0
    ratio[-1] = 0.0
    bad = bad | ~np.isfinite(rho) | (rho <= 0.0)
    return Macro(f, rho, psi, mean_rho, Fint, Fg, F, u, ratio, bad)


def step(fstar, p, mean_rho=None):
    """One full time step: returns the new post-collision populations f*."""
    mac = macroscopic(fstar, p, mean_rho)
    feq = equilibrium(mac.rho, mac.u[0], mac.u[1])
    S = li_source(mac.u[0], mac.u[1], mac.F[0], mac.F[1], mac.ratio, p)
    return collide(mac.f, feq, S, p)


def run(fstar, p, nsteps):
    """nsteps successive steps."""
    for _ in range(nsteps):
        fstar = step(fstar, p)
    return fstar


def init_state(rho0):
    """Initial state f* = f_eq(rho0, u = 0)."""
    rho0 = np.asarray(rho0, dtype=np.float64)
    z = np.zeros_like(rho0)
    return equilibrium(rho0, z, z)


def rest_state(rho, p, mean_rho=None):
    """Stored (post-collision) populations of a lattice at rest with the density field rho:
    an initialisation, no counterpart in the paper (which gives only the density profile of
    its initial state). The forces of Eqs. ShanChenForce and Gravity_1 / Gravity_2 follow
    from rho; the populations before the collision have the moments of the rest equilibrium
    f_eq(rho, 0) (Eq. EquilibriumDistribution) except the momentum, which is -F/2, so that
    the velocity of Eq. Momentum vanishes; then one collision (Eqs. OperatorMRT, LiFS). Its
    momentum is +F/2 (a collision adds F), and with every tau = 1 the state is
    m* = m_eq(rho, 0) + S~(u = 0, F)/2, which a steady state of the method satisfies."""
    rho = np.asarray(rho, dtype=np.float64)
    if mean_rho is None:
        mean_rho = float(np.mean(rho))
    psi, _ = interaction_potential(rho, p)
    Sx, Sy = shan_chen_sum(psi)
    Fint = (-p.G * psi * Sx, -p.G * psi * Sy)
    Fg = gravity(rho, mean_rho, p)
    F = (Fint[0] + Fg[0], Fint[1] + Fg[1])
    z = np.zeros_like(rho)
    m = M @ equilibrium(rho, z, z).reshape(9, -1)
    m[3] = -0.5 * F[0].ravel()  # j_x (moment order of Eq. MatrixMRT)
    m[5] = -0.5 * F[1].ravel()  # j_y
    f_pre = (MINV @ m).reshape((9,) + rho.shape)
    ux, uy = velocity(f_pre, rho, F[0], F[1])  # zero up to rounding
    ratio = sigma_ratio(Fint[0], Fint[1], psi, Sx, Sy, p.G)
    ratio[0] = 0.0
    ratio[-1] = 0.0
    S = li_source(ux, uy, F[0], F[1], ratio, p)
    return collide(f_pre, equilibrium(rho, ux, uy), S, p)


# ---------------------------------------------------------------- diagnostics
def mass(fstar):
    """Total mass sum_x sum_i f*_i (equal to sum_x rho after streaming)."""
    return float(np.sum(fstar))


def residual(rho_now, rho_prev):
    """max_x |rho_t(x) - rho_{t-1}(x)|."""
    return float(np.max(np.abs(rho_now - rho_prev)))


def interface_height(rho, rho_mid):
    """First height y (linear interpolation on the x-averaged profile, from the
    bottom) where rho crosses rho_mid; NaN if it never does."""
    prof = rho.mean(axis=1)
    for y in range(len(prof) - 1):
        lo, hi = prof[y], prof[y + 1]
        if (lo - rho_mid) * (hi - rho_mid) <= 0.0 and lo != hi:
            return y + (rho_mid - lo) / (hi - lo)
    return float("nan")


def normal_pressure(rho_col, p):
    """Normal pressure p_yy of Eq. GeneralPressureTensor for an x-uniform profile.

    With no x dependence, (d_g psi)(d_g psi) = psi'^2, psi lap psi = psi psi'' and
    psi d_y d_y psi = psi psi'', so with c = 1
    p_yy = p_EOS + sigma G^2/6 psi'^2 + G/12 psi psi'' + G/6 psi psi''.
    Derivatives by central differences (Sec. IV); returned on rows 1..ny-2.
    """
    rho_col = np.asarray(rho_col, dtype=np.float64)
    peos = p_eos(rho_col, p.T, p.a, p.b, p.R)
    psi = np.sqrt(2.0 * (peos - rho_col * CS2) / p.G)
    d1 = 0.5 * (psi[2:] - psi[:-2])
    d2 = psi[2:] - 2.0 * psi[1:-1] + psi[:-2]
    pc = psi[1:-1]
    return (
        peos[1:-1]
        + p.sigma * p.G**2 / 6.0 * d1**2
        + p.G / 12.0 * pc * d2
        + p.G / 6.0 * pc * d2
    )
