"""GPU parity of the thermal variant (Sec. III, Eq. Energy_Equation) against the FP64 oracle.

The handle is created with thermal = 1: psi uses R T(x) of the temperature field, and
after every LBM step the field is advanced by Heun's RK2 on the energy equation with that
step's rho and u. The oracle is oracle.thermal.thermal_step. Tolerances:
* FP64: per-step checks |df|, |dT| <= 1e-14 as for the isothermal path. Two FP64
  oracles that differ only in the summation order of the finite-difference stencils
  drift apart by 2e-16 (f) and 2e-17 (T) over 1000 steps on this kind of column, so the
  300-step run is held to 1e-12.
* FP32: populations as in the isothermal FP32 checks, 1e-6 sqrt(n) + 1e-6; the same bound
  on T, whose Heun update rounds a handful of terms of size <= T to FP32 per step.
"""
import math
import os

import numpy as np
import pytest

from oracle import eos
from oracle import lbm as olbm
from oracle import thermal as oth
from paper_2301_12869_gb300 import _build, inputs, lbm

pytestmark = pytest.mark.gpu

A, B, R = 0.25, 4.0, 1.0
RHO_C, T_C, P_C = eos.critical_point(A, B, R)


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


def thermal_params(nx, ny, precision, T_bot=0.92, T_top=0.80, **kw):
    kw.setdefault("a", A)
    return lbm.make_params(nx, ny, 0.5 * (T_bot + T_top) * T_C, precision, thermal=1, T_bot=T_bot * T_C,
                           T_top=T_top * T_C, **kw)


def oracle_of(p):
    op = olbm.Params(nx=p.nx, ny=p.ny, a=p.a, b=p.b, R=p.R, T=p.T, G=p.G, sigma=p.sigma, tau_rho=p.tau_rho,
                     tau_e=p.tau_e, tau_varsigma=p.tau_varsigma, tau_j=p.tau_j, tau_q=p.tau_q, tau_nu=p.tau_nu,
                     g=(p.gx, p.gy), form=p.gravity_form)
    return op, oth.Thermal(c_v=p.c_v, kappa=p.kappa, T_bot=p.T_bot, T_top=p.T_top)


def column(nx, ny, Tr=0.86, liquid=None):
    rv, rl, _ = eos.maxwell(Tr * T_C, A, B, R)
    return inputs.column_rho0(nx, ny, rl, rv, ny // 2 if liquid is None else liquid, width=3.0)


def start(p, rho0, amp=1e-3, T0=None):
    """Handle with seeded non-equilibrium populations (so u != 0 from the first step) and
    the given temperature field (default: the linear profile set by lbm_init)."""
    h = lbm.lbm_init(p, rho0)
    f0 = inputs.perturbed_populations(rho0, amp)
    lbm.lbm_set_state(h, f0)
    if T0 is not None:
        lbm.lbm_set_temperature(h, np.ascontiguousarray(T0))
    T = np.empty((p.ny, p.nx))
    lbm.lbm_get_temperature(h, T)
    return h, f0, T


def read(h, p):
    f = np.empty((9, p.ny, p.nx))
    T = np.empty((p.ny, p.nx))
    lbm.lbm_get_state(h, f)
    lbm.lbm_get_temperature(h, T)
    return f, T


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_initial_field_is_the_conduction_profile(precision):
    p = thermal_params(8, 40, precision)
    h = lbm.lbm_init(p, column(8, 40))
    try:
        T = np.empty((40, 8))
        lbm.lbm_get_temperature(h, T)
        want = oth.linear_profile(40, 8, p.T_bot, p.T_top)
        tol = 1e-15 if precision == "fp64" else 1e-7
        np.testing.assert_allclose(T, want, rtol=0, atol=tol)
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("nx, ny, form, taus", [
    (8, 24, 1, {}),
    (8, 24, 2, {}),
    (8, 24, 1, dict(tau_e=0.8, tau_varsigma=1.1, tau_q=1.2, tau_nu=0.7)),
    (200, 20, 2, {}),  # two FP64 x bands (128 + 72): band edges and a ragged tail
])
def test_fp64_steps_match_oracle(nx, ny, form, taus):
    p = thermal_params(nx, ny, "fp64", form=form, g=(0.0, -5e-5), **taus)
    op, th = oracle_of(p)
    h, f, T = start(p, column(nx, ny))
    try:
        for n in range(5):
            f, T = oth.thermal_step(f, T, op, th)
            lbm.lbm_step(h, 1)
            fg, Tg = read(h, p)
            assert np.max(np.abs(fg - f)) <= 1e-14, n
            assert np.max(np.abs(Tg - T)) <= 1e-14, n
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("nx, ny, form, wall", [
    (6, 17, 2, lbm.LBM_WALL_BOUNCE_BACK),   # 6 columns wrapped over a warp; a one-row second strip
    (30, 33, 2, lbm.LBM_WALL_ZOU_HE),       # two columns past a warp's 28 owned; <rho> in the wall closure
    (40, 3, 1, lbm.LBM_WALL_BOUNCE_BACK),   # three rows: both wall ghosts within one short walk
    (64, 4, 2, lbm.LBM_WALL_ZOU_HE),        # two fluid rows between the wall nodes
    (58, 48, 1, lbm.LBM_WALL_ZOU_HE),       # three full strips over two warps and two columns, rho g
])
def test_fp64_energy_walk_edges_match_oracle(nx, ny, form, wall):
    """The Heun strip walk at its edges, with rho and u stored by the step: lattices
    narrower than a warp (x wraps within it), a column block just past a warp's, a
    few rows (both wall ghosts inside one walk), strips ending one row past a boundary,
    and Zou-He walls with (rho - <rho>) g in the wall closure."""
    p = thermal_params(nx, ny, "fp64", form=form, g=(2e-6, -5e-5), wall=wall)
    op, th = oracle_of(p)
    op.wall = "zou-he" if wall == lbm.LBM_WALL_ZOU_HE else "bounce-back"
    h, f, T = start(p, column(nx, ny, liquid=max(1, ny // 2)))
    try:
        for n in range(6):
            f, T = oth.thermal_step(f, T, op, th)
            lbm.lbm_step(h, 1)
            fg, Tg = read(h, p)
            assert np.max(np.abs(fg - f)) <= 1e-14, n
            assert np.max(np.abs(Tg - T)) <= 1e-14, n
        assert lbm.lbm_status(h) == lbm.LBM_OK
    finally:
        lbm.lbm_destroy(h)


def test_fp64_300_steps_match_oracle():
    nx, ny = 8, 48
    p = thermal_params(nx, ny, "fp64", g=(0.0, -5e-5))
    op, th = oracle_of(p)
    h, f, T = start(p, column(nx, ny))
    try:
        for _ in range(300):
            f, T = oth.thermal_step(f, T, op, th)
        lbm.lbm_step(h, 300)
        fg, Tg = read(h, p)
        assert np.max(np.abs(fg - f)) <= 1e-12
        assert np.max(np.abs(Tg - T)) <= 1e-12
        # the field moved away from the initial profile: the check is not vacuous
        assert np.max(np.abs(T - oth.linear_profile(ny, nx, p.T_bot, p.T_top))) > 1e-4
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("nx", [24, 520])  # 520: the default FP32 tile plus a ragged band
def test_fp32_matches_oracle(nx):
    ny, steps = 32, 40
    p = thermal_params(nx, ny, "fp32", g=(0.0, -5e-5))
    op, th = oracle_of(p)
    h, f, T = start(p, column(nx, ny))
    try:
        # the FP32 start state is the rounded one: take it as the oracle's start too
        f, _ = read(h, p)
        for _ in range(steps):
            f, T = oth.thermal_step(f, T, op, th)
        lbm.lbm_step(h, steps)
        fg, Tg = read(h, p)
        tol = 1e-6 * math.sqrt(steps) + 1e-6
        assert np.max(np.abs(fg - f)) <= tol
        assert np.max(np.abs(Tg - T)) <= tol
    finally:
        lbm.lbm_destroy(h)


def test_user_temperature_field_and_moments():
    """A seeded non-uniform T field set through the ABI drives psi; lbm_moments then
    evaluates rho and u with that field, as the oracle's macroscopic step does."""
    nx, ny = 8, 24
    p = thermal_params(nx, ny, "fp64", form=2, g=(0.0, -2e-5))
    op, th = oracle_of(p)
    T0 = oth.linear_profile(ny, nx, p.T_bot, p.T_top) * (1.0 + 0.02 * (inputs.uniform_field(5, nx, ny) - 0.5))
    h, f, T = start(p, column(nx, ny), T0=T0)
    try:
        np.testing.assert_array_equal(T, T0)
        for _ in range(3):
            f, T = oth.thermal_step(f, T, op, th)
        lbm.lbm_step(h, 3)
        rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
        lbm.lbm_moments(h, rho, ux, uy)
        from dataclasses import replace

        mac = olbm.macroscopic(f, replace(op, T=T))
        np.testing.assert_allclose(rho, mac.rho, rtol=0, atol=1e-14)
        np.testing.assert_allclose(ux, mac.u[0], rtol=0, atol=1e-14)
        np.testing.assert_allclose(uy, mac.u[1], rtol=0, atol=1e-14)
    finally:
        lbm.lbm_destroy(h)


def test_uniform_field_first_step_equals_isothermal_step():
    """With T(x) = T everywhere the thermal step's populations are the isothermal ones
    (R T(x) = R T exactly in FP64)."""
    nx, ny = 8, 24
    p = thermal_params(nx, ny, "fp64", T_bot=0.86, T_top=0.86)
    q = lbm.make_params(nx, ny, p.T, "fp64", a=A)
    rho0 = column(nx, ny)
    h, _, _ = start(p, rho0, T0=np.full((ny, nx), p.T))
    g = lbm.lbm_init(q, rho0)
    try:
        lbm.lbm_set_state(g, inputs.perturbed_populations(rho0, 1e-3))
        lbm.lbm_step(h, 1)
        lbm.lbm_step(g, 1)
        fh, _ = read(h, p)
        fg = np.empty_like(fh)
        lbm.lbm_get_state(g, fg)
        np.testing.assert_array_equal(fh, fg)
    finally:
        lbm.lbm_destroy(h)
        lbm.lbm_destroy(g)


def test_isothermal_handle_has_no_temperature_field():
    p = lbm.make_params(8, 16, 0.85 * T_C, "fp64", a=A)
    h = lbm.lbm_init(p, column(8, 16))
    try:
        with pytest.raises(lbm.LbmError, match="isothermal"):
            lbm.lbm_get_temperature(h, np.empty((16, 8)))
        q = thermal_params(8, 16, "fp64")
        with pytest.raises(lbm.LbmError, match="thermal"):
            lbm.lbm_set_params(h, q)
    finally:
        lbm.lbm_destroy(h)


def test_workspace_size_in_a_fresh_process():
    """lbm_workspace_bytes called before any handle exists (so before the kernels' shared
    memory limits are set) gives the size lbm_init then requires, for every precision and
    both variants, on the sizes of the thermal and single-domain workloads."""
    import subprocess
    import sys

    code = (
        "import numpy as np, torch\n"
        "from paper_2301_12869_gb300 import lbm\n"
        "lbm.load()\n"
        "Tc = lbm.lbm_critical_point(0.25, 4.0, 1.0)[1]\n"
        "for prec in ('fp32', 'fp64'):\n"
        "    for th in (0, 1):\n"
        "        for nx, ny in ((512, 2048), (1024, 512)):\n"
        "            p = lbm.make_params(nx, ny, 0.85 * Tc, prec, a=0.25, thermal=th, T_bot=0.9 * Tc, T_top=0.8 * Tc)\n"
        "            lat = lbm.Lattice(p, torch.full((ny, nx), 0.1, dtype=torch.float64, device='cuda'))\n"
        "            lat.close()\n"
        "print('ok')\n"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().endswith("ok")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_thermal_handle_keeps_a_thermal_tile(precision):
    p = thermal_params(16, 16, precision)
    h = lbm.lbm_init(p, column(16, 16))
    try:
        with pytest.raises(lbm.LbmError, match="no thermal or Zou-He kernels"):
            lbm.lbm_set_tiling(h, 1)
        assert lbm.lbm_autotune(h, 2)[0] == 0
        lbm.lbm_step(h, 2)
        assert lbm.lbm_status(h) == 0
    finally:
        lbm.lbm_destroy(h)


def test_full_size_thermal_column_sampled():
    """The 512 x 2048 FP32 heated column of the thermal workload (bench.py's set-up, default
    tile: the launch configuration it times): one thermal step - fused LBM step storing
    rho and u, Heun step - after 20, checked on sampled columns against the oracle run on a
    24-column strip around each column (full height, so the walls are exact; one thermal step
    reaches 6 columns, the strip's periodic seams are 12 away)."""
    import dataclasses

    import bench

    p, rho0, _ = bench.thermal_setup("fp32", lbm, inputs)
    op, th = oracle_of(p)
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_step(h, 20)
        f_t, T_t = read(h, p)
        lbm.lbm_step(h, 1)
        f_n, T_n = read(h, p)
        assert lbm.lbm_status(h) == 0
    finally:
        lbm.lbm_destroy(h)
    nx = p.nx
    q = dataclasses.replace(op, nx=24)
    worst_f = worst_T = 0.0
    for x in (0, 1, 255, 256, 300, nx - 1):
        cols = [(x + d) % nx for d in range(-12, 12)]
        fo, To = oth.thermal_step(np.ascontiguousarray(f_t[:, :, cols]), np.ascontiguousarray(T_t[:, cols]), q, th)
        worst_f = max(worst_f, float(np.max(np.abs(f_n[:, :, x] - fo[:, :, 12]))))
        worst_T = max(worst_T, float(np.max(np.abs(T_n[:, x] - To[:, 12]))))
    assert worst_f <= 2e-6, worst_f
    assert worst_T <= 2e-6, worst_T
    assert np.max(np.abs(T_n - T_t)) > 0  # the field moved: the check is not vacuous
