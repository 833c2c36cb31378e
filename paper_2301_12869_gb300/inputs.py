"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module draws the initial density fields of the liquid-column workloads
and holds none of the method's arithmetic: the coexistence densities rho_l and
rho_v are arguments (a caller gets them from its own Maxwell solver), and the
only randomness is a counter-based generator, SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), keyed on
(seed, x, y) so that any node's draw can be regenerated on its own.

Recipe of the column inputs (the paper's Sec. IV set-up: liquid below, vapour
above, a planar interface): rho0(y) = (rho_l + rho_v)/2 - (rho_l - rho_v)/2 *
tanh(2 (y - y0) / W) with W = 5 and y0 = liquid_rows - 1/2, optionally plus
uniform noise U(-amp, amp) on the rows |y - y0| <= band.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20230130

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output for state = seed + (counter + 1) * golden gamma (uint64 wrap)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_field(seed: int, nx: int, ny: int, stream: int = 0) -> np.ndarray:
    """U[0, 1) doubles on an ny x nx grid; node (x, y) uses counter (stream, y, x)."""
    y, x = np.meshgrid(np.arange(ny, dtype=np.uint64), np.arange(nx, dtype=np.uint64), indexing="ij")
    counter = (np.uint64(stream) << np.uint64(48)) + y * np.uint64(nx) + x
    bits = splitmix64(counter, seed) >> np.uint64(11)          # top 53 bits
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def column_rho0(nx, ny, rho_l, rho_v, liquid_rows, width=5.0, noise_amp=0.0, noise_band=None, seed=DEFAULT_SEED):
    """Initial density field rho0[y, x] of a liquid column under vapour (FP64).

    liquid_rows: the interface sits at y0 = liquid_rows - 1/2.
    noise_amp:   amplitude of seeded uniform noise added on |y - y0| <= noise_band
                 (default band 2 * width).
    """
    y0 = liquid_rows - 0.5
    y = np.arange(ny, dtype=np.float64)[:, None]
    prof = 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (y - y0) / width)
    rho0 = np.repeat(prof, nx, axis=1)
    if noise_amp:
        band = 2.0 * width if noise_band is None else noise_band
        u = uniform_field(seed, nx, ny)
        mask = np.abs(y - y0) <= band
        rho0 = rho0 + np.where(mask, noise_amp * (2.0 * u - 1.0), 0.0)
    return np.ascontiguousarray(rho0)


def batched_columns(n, seed=DEFAULT_SEED, heights=(64, 128, 256, 512, 1024)):
    """Per-column parameters of the batched workload (seeded):
    H ~ U{heights}, T/T_c ~ U[0.70, 0.95], |g| log-uniform in [1e-6, 1e-4] (g_y < 0),
    gravity form 1 or 2 with p = 0.5, liquid fraction ~ U[0.3, 0.7]."""
    u = uniform_field(seed, 5, n, stream=7)
    H = np.array(heights)[np.minimum((u[:, 0] * len(heights)).astype(int), len(heights) - 1)]
    Tr = 0.70 + 0.25 * u[:, 1]
    g = -(10.0 ** (-6.0 + 2.0 * u[:, 2]))
    form = np.where(u[:, 3] < 0.5, 1, 2)
    frac = 0.3 + 0.4 * u[:, 4]
    return [
        dict(ny=int(H[k]), Tr=float(Tr[k]), gy=float(g[k]), form=int(form[k]), liquid_fraction=float(frac[k]))
        for k in range(n)
    ]


#: D2Q9 lattice weights in the velocity order (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)
LATTICE_WEIGHTS = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def perturbed_populations(rho0, amp, seed=DEFAULT_SEED):
    """Non-equilibrium test populations f[i, y, x] = w_i rho0 (1 + amp (2 U_i - 1)), U_i seeded
    per (i, y, x). Drawn data only: not an equilibrium of the method."""
    rho0 = np.asarray(rho0, dtype=np.float64)
    ny, nx = rho0.shape
    f = np.empty((9, ny, nx))
    for i in range(9):
        u = uniform_field(seed, nx, ny, stream=100 + i)
        f[i] = LATTICE_WEIGHTS[i] * rho0 * (1.0 + amp * (2.0 * u - 1.0))
    return f


def mlp_draws(seed: int = DEFAULT_SEED, width: int = 128, n_in: int = 5) -> dict:
    """U[0, 1) draws for the warm-start network's initial weights (shapes of W1 (width x
    n_in), W2, W3 (width x width) and w4 (width)), one SplitMix64 stream per array."""
    shapes = {"W1": (width, n_in), "W2": (width, width), "W3": (width, width), "w4": (width,)}
    out = {}
    for s, (name, shape) in enumerate(shapes.items()):
        n = int(np.prod(shape))
        counter = (np.uint64(200 + s) << np.uint64(48)) + np.arange(n, dtype=np.uint64)
        bits = splitmix64(counter, seed) >> np.uint64(11)
        out[name] = (bits.astype(np.float64) * (1.0 / 9007199254740992.0)).reshape(shape)
    return out


def minibatch_indices(n: int, batch: int, step: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Sample indices of minibatch `step`: SplitMix64(step * batch + i) mod n, i < batch
    (sampling with replacement)."""
    counter = np.uint64(step) * np.uint64(batch) + np.arange(batch, dtype=np.uint64)
    return (splitmix64(counter, seed) % np.uint64(n)).astype(np.int64)
