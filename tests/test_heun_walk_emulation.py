"""CPU emulation of the energy-equation walk of csrc/lbm_thermal.cu (heun_strip_kernel), lanes as
array entries, against the oracle's Heun step (Eq. Energy_Equation).

The emulation restates the kernel's algorithm - the lane layouts (one FP64 column, or a
pair of FP32 columns, per lane; two halo columns at each warp edge; x periodic, narrow
lattices wrapping more than once), warp shuffles (a lane at the warp's end keeps its own
value), the row window of one strip (input rows loaded two ahead, k1 and T* one row behind
the input, k2 two rows behind), the wall ghosts and wet-node wall rows, and the stencil
weights applied to T and T* - in FP64, and checks every node against
oracle.thermal.energy_step and that every node is written exactly once. It shares no code
with the oracle and none with the library; the GPU tests check the kernel itself.
"""
import itertools

import numpy as np
import pytest

from oracle import lbm as olbm
from oracle import thermal as oth

LANES = 32
ROWS, WARPS, AHEAD = 8, 8, 2  # the kernel's strip height, warps per CTA, rows loaded ahead


def shfl_up(v):
    """Lane l receives lane l - 1's value; lane 0 keeps its own (__shfl_up_sync)."""
    return np.concatenate([v[:1], v[:-1]])


def shfl_down(v):
    """Lane l receives lane l + 1's value; the last lane keeps its own (__shfl_down_sync)."""
    return np.concatenate([v[1:], v[-1:]])


class Lanes:
    """Values of a warp: shape (32, W), W columns per lane (1: FP64 layout, 2: FP32 pairs)."""

    def __init__(self, width):
        self.width = width

    def _edges(self, v):
        # the columns next to the lane's own: the left lane's last, the right lane's first
        return shfl_up(v[:, -1]), shfl_down(v[:, 0])

    def neighbours(self, v):
        """(centre, left neighbour, right neighbour) of every column of every lane."""
        left, right = self._edges(v)
        if self.width == 1:
            return v, left[:, None], right[:, None]
        return v, np.stack([left, v[:, 0]], 1), np.stack([v[:, 1], right], 1)

    def xdiff(self, v):
        """v(x + 1) - v(x - 1)."""
        c, l, r = self.neighbours(v)
        return r - l

    def xsum(self, v):
        """v(x + 1) + v(x - 1)."""
        c, l, r = self.neighbours(v)
        return r + l


def weights(P, U, V, centre):
    """Stencil weights of one node row: axis neighbours P - U c_x - V c_y, diagonals a quarter."""
    q, p, m = 0.25 * P, 0.25 * (U + V), 0.25 * (U - V)
    return dict(c=centre, e=P - U, w=P + U, n=P - V, s=P + V, ne=q - p, nw=q + m, se=q - m, sw=q + p)


def apply(a, south, centre, north):
    """L(phi) from phi on the rows below, at and above (each a (centre, left, right) triple)."""
    return (a["c"] * centre[0] + a["e"] * centre[2] + a["w"] * centre[1] + a["nw"] * north[1] + a["sw"] * south[1]) + \
           (a["n"] * north[0] + a["s"] * south[0] + a["ne"] * north[2] + a["se"] * south[2])


def walk(nx, ny, walls, Tin, rho, ux, uy, R, b, c_v, kappa, T_bot, T_top, width):
    """One Heun step of the energy equation as the kernel's grid of warps computes it."""
    lanes = Lanes(width)
    own_cols = LANES * width - 4
    Tout = np.full((ny, nx), np.nan)
    writes = np.zeros((ny, nx), dtype=int)
    b4, kP, kZ = b / 4.0, 2.0 * kappa / (3.0 * c_v), R / c_v
    two_bot, two_top = 2.0 * T_bot, 2.0 * T_top
    strips = (ny + ROWS - 1) // ROWS
    grid_x, grid_y = (nx + own_cols - 1) // own_cols, (strips + WARPS - 1) // WARPS
    rel = width * np.arange(LANES) - 2  # each lane's first column from the warp's first owned one
    zero = np.zeros((LANES, width))
    for bx, by, wy in itertools.product(range(grid_x), range(grid_y), range(WARPS)):
        x0 = bx * own_cols
        x = (x0 + rel) % nx
        assert width == 1 or np.all(x % 2 == 0)  # a pair never straddles the periodic seam
        own = (rel >= 0) & (rel < own_cols) & (x0 + rel < nx)
        cols = x[:, None] + np.arange(width)[None, :]
        ya = (by * WARPS + wy) * ROWS
        if ya >= ny:
            continue
        yb = min(ya + ROWS, ny)

        def fetch(q):
            real = 0 <= q < ny
            ghost = not walls and q in (-1, ny)
            if q <= yb + 1 and (real or ghost):
                row = q if real else (0 if q < 0 else ny - 1)
                return [Tin[row][cols], ux[row][cols], uy[row][cols], rho[row][cols] if real else zero]
            return [zero] * 4

        ring = [fetch(ya - 2 + d) for d in range(AHEAD)]
        t = [lanes.neighbours(zero)] * 3            # T rows q-2, q-1, q
        s = [lanes.neighbours(zero)] * 3            # T* rows q-3, q-2, q-1
        du, vc, sv = [zero] * 3, [zero] * 3, [zero] * 3
        U, P, Z = [zero] * 2, [zero] * 2, [zero] * 2
        w_prev, k1_prev = weights(zero, zero, zero, zero), zero
        for it in range(ROWS + 4):
            q = ya - 2 + it
            tq, uq, vq, rq = ring[it % AHEAD]
            if it + AHEAD < ROWS + 4:
                ring[it % AHEAD] = fetch(q + AHEAD)
            Pq = Zq = zero
            if not walls and q in (-1, ny):  # ghost rows beyond the walls
                tq = (two_bot if q < 0 else two_top) - tq
                uq, vq = -uq, -vq
            elif 0 <= q < ny:
                eta = b4 * rq
                om = 1.0 - eta
                Pq = kP / rq
                Zq = kZ * (eta * (eta * om + 1.0) + 1.0) / om**3
            t = t[1:] + [lanes.neighbours(tq)]
            du = du[1:] + [lanes.xdiff(uq)]
            vc = vc[1:] + [vq]
            sv = sv[1:] + [lanes.xsum(vq)]
            U, P, Z = [U[1], uq / 3.0], [P[1], Pq], [Z[1], Zq]
            r1 = q - 1  # first stage
            w_now, k1 = weights(zero, zero, zero, zero), zero
            if it >= 1 and 0 <= r1 < ny and not (walls and r1 in (0, ny - 1)):
                div = (du[1] + (vc[2] - vc[0])) / 3.0 + ((du[2] + du[0]) + (sv[2] - sv[0])) / 12.0
                w_now = weights(P[0], U[0], vc[1] / 3.0, -5.0 * P[0] - Z[0] * div)
                k1 = apply(w_now, t[0], t[1], t[2])
            s = s[1:] + [lanes.neighbours(t[1][0] + k1)]
            if not walls and r1 == 0:
                s[1] = tuple(two_bot - v for v in s[2])
            if not walls and r1 == ny:
                s[2] = tuple(two_top - v for v in s[1])
            r2 = q - 2  # second stage and the update
            if it >= 2 and ya <= r2 < yb:
                if walls and r2 in (0, ny - 1):
                    new = np.full((LANES, width), 0.5 * (two_bot if r2 == 0 else two_top))
                else:
                    new = 0.5 * (k1_prev + apply(w_prev, s[0], s[1], s[2])) + t[0][0]
                for lane in np.nonzero(own)[0]:
                    Tout[r2, cols[lane]] = new[lane]
                    writes[r2, cols[lane]] += 1
            w_prev, k1_prev = w_now, k1
    assert np.all(writes == 1), (writes.min(), writes.max())
    return Tout


@pytest.mark.parametrize("width", [1, 2])
def test_walk_matches_oracle_energy_step(width):
    rng = np.random.default_rng(5 + width)
    worst = 0.0
    for nx in (4, 12, 28, 60, 64, 68, 128):
        for ny in (1, 2, 3, 4, 7, 8, 9, 17, 66):
            for walls in (False, True):
                if walls and ny < 3:
                    continue
                R, b, c_v, kappa, T_bot, T_top = 1.0, 4.0, 5.0, 0.02, 0.090, 0.076
                T = 0.08 + 0.01 * rng.random((ny, nx))
                rho = 0.02 + 0.3 * rng.random((ny, nx))
                ux = 1e-2 * rng.standard_normal((ny, nx))
                uy = 1e-2 * rng.standard_normal((ny, nx))
                p = olbm.Params(nx=nx, ny=ny, a=0.25, b=b, R=R, T=0.08, wall="zou-he" if walls else "bounce-back")
                th = oth.Thermal(c_v=c_v, kappa=kappa, T_bot=T_bot, T_top=T_top)
                want = oth.energy_step(T, rho, ux, uy, p, th)
                got = walk(nx, ny, walls, T, rho, ux, uy, R, b, c_v, kappa, T_bot, T_top, width)
                worst = max(worst, float(np.max(np.abs(got - want))))
    assert worst < 1e-15
