"""Steady LBM columns against the sharp-interface theory (oracle/theory.py) in the set-up of
the paper's comparison (Sec. IV, Fig. Example_Pressure_Profile): h = 100,
<rho> = 1.3344 rho_c, g = 2e-5, a = 0.5, tau = 1, sigma = 1.385, both gravity forms, at the
uniform temperature T_med = 0.75 T_c (the thermal column with Delta T = 0.2 T_c does not
settle with the energy-equation discretisation as read: an odd-even mode grows, see the
design notes).

The theory has a sharp interface at Maxwell coexistence; the lattice Boltzmann interface is
a few nodes wide and the model's own coexistence densities deviate from the Maxwell rule
by a temperature-dependent amount (the "method's known deviation"). That deviation is
measured on the same column at g = 0; with gravity, bulk nodes - 8 or more from the
interface and 3 or more from a wall - must match the theory within it plus 1 %, the
interface height within one node and the normal pressure within 1 % (form 1) / 10 %
(form 2: the paper reports a constant offset of about 5 %).
"""
import os

import numpy as np
import pytest

from oracle import eos, theory
from oracle import lbm as olbm
from paper_2301_12869_gb300 import _build, inputs, lbm

pytestmark = pytest.mark.gpu

A, B, R = 0.5, 4.0, 1.0
RHO_C, T_C, P_C = eos.critical_point(A, B, R)
NY, NX = 100, 4


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


def steady(form, T, g, mean, h_i, rv, rl):
    rho0 = inputs.column_rho0(NX, NY, rl, rv, int(round(h_i)))
    rho0 *= mean / rho0.mean()
    p = lbm.make_params(NX, NY, T, "fp64", a=A, form=form, g=(0.0, g))
    h = lbm.lbm_init(p, rho0)
    try:
        res = np.inf
        for _ in range(100):
            lbm.lbm_step(h, 2000)
            lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)
            lbm.lbm_step(h, 1)
            res = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)[0]
            if res < 1e-13:
                break
        assert res < 1e-13
        rho = np.empty((NY, NX))
        lbm.lbm_moments(h, rho)
    finally:
        lbm.lbm_destroy(h)
    return rho[:, 0]


def deviation_at(T):
    """Relative deviation of the model's bulk densities from the Maxwell rule at g = 0 and
    temperature T (liquid, vapour): the method's known coexistence error there."""
    rv, rl, _ = eos.maxwell(T, A, B, R)
    mean = 1.3344 * RHO_C
    h_i = NY * (mean - rv) / (rl - rv)
    r = steady(1, T, 0.0, mean, h_i, rv, rl)
    y = np.arange(NY) + 0.5
    bulk = (np.abs(y - h_i) >= 8) & (y >= 3) & (y <= NY - 3)
    d_l = np.max(np.abs(r[bulk & (y < h_i)] / rl - 1))
    d_v = np.max(np.abs(r[bulk & (y > h_i)] / rv - 1))
    print(f"g = 0, T/T_c = {T / T_C:.2f}: liquid {d_l:.2e}, vapour {d_v:.2e} from Maxwell")
    return d_l, d_v


@pytest.fixture(scope="module")
def coexistence_deviation():
    return deviation_at(0.75 * T_C)


@pytest.fixture(scope="module")
def cold_deviation():
    """At the coldest wall temperature of the thermal example (0.65 T_c), where the vapour's
    deviation is largest (it grows as T falls)."""
    return deviation_at(0.65 * T_C)


@pytest.mark.parametrize("form", [1, 2])
def test_steady_column_matches_theory(form, coexistence_deviation):
    T, g, mean = 0.75 * T_C, -2e-5, 1.3344 * RHO_C
    c = theory.Column(H=float(NY), T_bot=T, T_top=T, mean_rho=mean, g_y=g, form=form, a=A, b=B, R=R)
    sol = theory.solve(c, dh=0.05, tol=1e-9, scan=16)
    rho_th, p_th = theory.at_nodes(sol, NY)
    rv, rl = sol.rho_v_i, sol.rho_l_i
    r = steady(form, T, g, mean, sol.h_i, rv, rl)
    y = np.arange(NY) + 0.5
    bulk = (np.abs(y - sol.h_i) >= 8) & (y >= 3) & (y <= NY - 3)
    liq, vap = bulk & (y < sol.h_i), bulk & (y > sol.h_i)
    e_l = np.max(np.abs(r[liq] / rho_th[liq] - 1))
    e_v = np.max(np.abs(r[vap] / rho_th[vap] - 1))
    mid = 0.5 * (rv + rl)
    k = int(np.nonzero((r[:-1] - mid) * (r[1:] - mid) <= 0)[0][0])
    y_lbm = y[k] + (r[k] - mid) / (r[k] - r[k + 1])
    # normal pressure of the LBM profile (Eq. GeneralPressureTensor, central differences)
    pyy = olbm.normal_pressure(r, olbm.Params(nx=NX, ny=NY, a=A, b=B, R=R, T=T, g=(0.0, g), form=form))
    e_p = np.max(np.abs(pyy[bulk[1:-1]] / p_th[1:-1][bulk[1:-1]] - 1))
    print(f"form {form}: liquid {e_l:.2e}, vapour {e_v:.2e}, interface {y_lbm:.3f} vs {sol.h_i:.3f}, p_yy {e_p:.2e}")
    d_l, d_v = coexistence_deviation
    assert e_l <= d_l + 0.01
    assert e_v <= d_v + 0.01
    assert abs(y_lbm - sol.h_i) <= 1.0
    assert e_p <= (0.01 if form == 1 else 0.10)


@pytest.mark.parametrize("form", [1, 2])
def test_steady_thermal_column_matches_theory(form, coexistence_deviation, cold_deviation):
    """The paper's first worked example with its own walls: Zou-He wet nodes on rows 0 and
    100 (h = 100, 101 nodes, Sec. IV) holding T_bot = 0.85 T_c and T_top = 0.65 T_c, the
    energy equation live (c_v = 5, kappa = 0.02). Run to a per-step change of 1e-11; bulk
    densities against the theory within the model's coexistence deviation plus 1 % - for
    the liquid the larger of its values at 0.75 T_c and 0.65 T_c, for the vapour its value
    at the coldest wall (0.65 T_c), which bounds the vapour's over the column; with
    Eq. Gravity_2 the vapour margin is the ~5 % offset the paper reports for that form - the
    interface within one node, and T linear to 1e-6 relative (u = 0 at rest)."""
    ny = 101
    T_bot, T_top, g, mean = 0.85 * T_C, 0.65 * T_C, -2e-5, 1.3344 * RHO_C
    c = theory.Column(H=float(ny - 1), T_bot=T_bot, T_top=T_top, mean_rho=mean, g_y=g, form=form, a=A, b=B, R=R)
    sol = theory.solve(c, dh=0.05, tol=1e-9, scan=16)
    rho_th, _ = theory.at_nodes(sol, ny, offset=0.0)
    rho0 = inputs.column_rho0(NX, ny, sol.rho_l_i, sol.rho_v_i, int(round(sol.h_i)))
    rho0 *= mean / rho0.mean()
    p = lbm.make_params(NX, ny, 0.75 * T_C, "fp64", a=A, form=form, g=(0.0, g), thermal=1, T_bot=T_bot, T_top=T_top,
                        wall=lbm.LBM_WALL_ZOU_HE)
    h = lbm.lbm_init(p, rho0)
    try:
        res = np.inf
        for _ in range(60):
            lbm.lbm_step(h, 49999)
            lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)
            lbm.lbm_step(h, 1)
            res = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)[0]
            if res < 1e-11:
                break
        rho = np.empty((ny, NX))
        T = np.empty((ny, NX))
        lbm.lbm_moments(h, rho)
        lbm.lbm_get_temperature(h, T)
    finally:
        lbm.lbm_destroy(h)
    r, y = rho[:, 0], np.arange(ny, dtype=float)
    bulk = (np.abs(y - sol.h_i) >= 8) & (y >= 3) & (y <= ny - 4)
    liq, vap = bulk & (y < sol.h_i), bulk & (y > sol.h_i)
    e_l = np.max(np.abs(r[liq] / rho_th[liq] - 1))
    e_v = np.max(np.abs(r[vap] / rho_th[vap] - 1))
    mid = 0.5 * (sol.rho_v_i + sol.rho_l_i)
    k = int(np.nonzero((r[:-1] - mid) * (r[1:] - mid) <= 0)[0][0])
    y_lbm = y[k] + (r[k] - mid) / (r[k] - r[k + 1])
    T_dev = np.max(np.abs(T[:, 0] / (T_bot + (T_top - T_bot) * y / (ny - 1)) - 1))
    print(f"thermal form {form}: res {res:.1e}, liquid {e_l:.2e}, vapour {e_v:.2e}, interface {y_lbm:.3f} vs "
          f"{sol.h_i:.3f}, T dev {T_dev:.1e}")
    assert res < 1e-11
    assert e_l <= max(coexistence_deviation[0], cold_deviation[0]) + 0.01
    # Eq. Gravity_2: the paper reports a constant offset of about 5 % between LBM and theory
    # (Sec. IV, pressure profile), which the nearly ideal vapour's density follows
    assert e_v <= cold_deviation[1] + (0.01 if form == 1 else 0.05)
    assert abs(y_lbm - sol.h_i) <= 1.0
    assert T_dev <= 1e-6
