"""GPU parity of the Zou-He wet-node walls (lbm_params.wall = LBM_WALL_ZOU_HE) against the
FP64 oracle (oracle/lbm.py, wall = "zou-he"), and the closed-form channel flow for both wall
treatments. Tolerances as in test_gpu_parity.py: FP64 1e-14 per step over a few steps, FP32
1e-6 sqrt(n) + 1e-6."""
import dataclasses
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


def oracle_params(p):
    return olbm.Params(nx=p.nx, ny=p.ny, a=p.a, b=p.b, R=p.R, T=p.T, G=p.G, sigma=p.sigma, tau_rho=p.tau_rho,
                       tau_e=p.tau_e, tau_varsigma=p.tau_varsigma, tau_j=p.tau_j, tau_q=p.tau_q, tau_nu=p.tau_nu,
                       g=(p.gx, p.gy), form=p.gravity_form,
                       wall="zou-he" if p.wall == lbm.LBM_WALL_ZOU_HE else "bounce-back")


def column(nx, ny, Tr=0.85):
    rv, rl, _ = eos.maxwell(Tr * T_C, A, B, R)
    return inputs.column_rho0(nx, ny, rl, rv, ny // 2, width=3.0)


def state(h, p):
    f = np.empty((9, p.ny, p.nx))
    lbm.lbm_get_state(h, f)
    return f


@pytest.mark.parametrize("nx, ny, form, g, taus", [
    (4, 12, 1, (0.0, -2e-5), {}),
    (4, 12, 2, (3e-6, -2e-5), {}),
    (6, 9, 1, (1e-5, -5e-5), dict(tau_e=0.8, tau_varsigma=1.1, tau_q=1.2, tau_nu=0.7)),
    (200, 10, 2, (0.0, -1e-4), {}),  # two FP64 x bands with a ragged one
])
def test_fp64_zou_he_steps_match_oracle(nx, ny, form, g, taus):
    p = lbm.make_params(nx, ny, 0.85 * T_C, "fp64", a=A, form=form, g=g, wall=lbm.LBM_WALL_ZOU_HE, **taus)
    op = oracle_params(p)
    rho0 = column(nx, ny)
    f = inputs.perturbed_populations(rho0, 1e-3)
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_set_state(h, f)
        for n in range(5):
            f = olbm.step(f, op)
            lbm.lbm_step(h, 1)
            assert np.max(np.abs(state(h, p) - f)) <= 1e-14, n
        rho, ux, uy = (np.empty((ny, nx)) for _ in range(3))
        lbm.lbm_moments(h, rho, ux, uy)
        mac = olbm.macroscopic(f, op)
        np.testing.assert_allclose(rho, mac.rho, rtol=0, atol=1e-14)
        np.testing.assert_allclose(uy, mac.u[1], rtol=0, atol=1e-13)
        assert np.max(np.abs(uy[[0, -1]])) < 1e-15  # the wall nodes are at rest
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("nx", [24, 520])
def test_fp32_zou_he_matches_oracle(nx):
    ny, steps = 16, 40
    p = lbm.make_params(nx, ny, 0.85 * T_C, "fp32", a=A, form=2, g=(0.0, -3e-5), wall=lbm.LBM_WALL_ZOU_HE)
    op = oracle_params(p)
    h = lbm.lbm_init(p, column(nx, ny))
    try:
        f = state(h, p)
        for _ in range(steps):
            f = olbm.step(f, op)
        lbm.lbm_step(h, steps)
        assert np.max(np.abs(state(h, p) - f)) <= 1e-6 * math.sqrt(steps) + 1e-6
    finally:
        lbm.lbm_destroy(h)


def test_thermal_zou_he_matches_oracle():
    nx, ny = 8, 20
    p = lbm.make_params(nx, ny, 0.85 * T_C, "fp64", a=A, form=1, g=(0.0, -2e-5), wall=lbm.LBM_WALL_ZOU_HE, thermal=1,
                        T_bot=0.9 * T_C, T_top=0.8 * T_C)
    op = oracle_params(p)
    th = oth.Thermal(c_v=p.c_v, kappa=p.kappa, T_bot=p.T_bot, T_top=p.T_top)
    rho0 = column(nx, ny)
    # the wet-node walls hold T_bot and T_top; the initial field is linear between them
    h0 = lbm.lbm_init(p, rho0)
    T0 = np.empty((ny, nx))
    lbm.lbm_get_temperature(h0, T0)
    lbm.lbm_destroy(h0)
    np.testing.assert_allclose(T0, oth.linear_profile(ny, nx, p.T_bot, p.T_top, wall="zou-he"), rtol=0, atol=1e-15)
    f = inputs.perturbed_populations(rho0, 1e-3)
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_set_state(h, f)
        T = np.empty((ny, nx))
        lbm.lbm_get_temperature(h, T)
        for n in range(5):
            f, T = oth.thermal_step(f, T, op, th)
            lbm.lbm_step(h, 1)
            Tg = np.empty((ny, nx))
            lbm.lbm_get_temperature(h, Tg)
            assert np.max(np.abs(state(h, p) - f)) <= 1e-14, n
            assert np.max(np.abs(Tg - T)) <= 1e-14, n
            assert np.all(Tg[0] == p.T_bot) and np.all(Tg[-1] == p.T_top)
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("wall, tau_q, precision", [
    (lbm.LBM_WALL_BOUNCE_BACK, 0.875, "fp64"), (lbm.LBM_WALL_ZOU_HE, 1.0, "fp64"), (lbm.LBM_WALL_ZOU_HE, 1.0, "fp32"),
])
def test_channel_flow_closed_form(wall, tau_q, precision):
    """Single-phase uniform density driven by g_x: u_x = g d1 d2 / (2 nu), walls at -1/2 and
    ny - 1/2 for bounce-back (exact at (tau_nu - 1/2)(tau_q - 1/2) = 3/16), on the nodes
    0 and ny - 1 for Zou-He."""
    ny = 12
    p = lbm.make_params(8, ny, 1.5 * T_C, precision, a=A, g=(1e-6, 0.0), wall=wall, tau_q=tau_q)
    h = lbm.lbm_init(p, np.full((ny, 8), 0.1))
    try:
        lbm.lbm_step(h, 8000)
        ux = np.empty((ny, 8))
        lbm.lbm_moments(h, None, ux, None)
    finally:
        lbm.lbm_destroy(h)
    nu = (p.tau_nu - 0.5) / 3.0
    y = np.arange(ny) + (0.5 if wall == lbm.LBM_WALL_BOUNCE_BACK else 0.0)
    H = ny if wall == lbm.LBM_WALL_BOUNCE_BACK else ny - 1
    want = p.gx / (2 * nu) * y * (H - y)
    tol = 1e-9 if precision == "fp64" else 1e-4  # FP32: rounding of populations ~1e-8 vs u ~1e-4
    assert np.max(np.abs(ux[:, 0] - want)) <= tol * np.max(want)


def test_zou_he_handles_keep_variant_zero_and_batches_need_three_rows():
    p = lbm.make_params(16, 12, 0.85 * T_C, "fp32", a=A, wall=lbm.LBM_WALL_ZOU_HE)
    h = lbm.lbm_init(p, column(16, 12))
    try:
        with pytest.raises(lbm.LbmError, match="Zou-He"):
            lbm.lbm_set_tiling(h, 1)
    finally:
        lbm.lbm_destroy(h)
    with pytest.raises(lbm.LbmError, match="ny >= 3"):
        lbm.lbm_batch_init(p, [dict(ny=2, T=0.85 * T_C, form=1)], np.full(16 * 2, 0.1))


def test_changed_wall_temperature_reaches_the_wall_rows():
    """lbm_set_params with a new T_top: the next step's wall row holds it (as the oracle's)."""
    nx, ny = 8, 12
    p = lbm.make_params(nx, ny, 0.85 * T_C, "fp64", a=A, wall=lbm.LBM_WALL_ZOU_HE, thermal=1, T_bot=0.9 * T_C,
                        T_top=0.8 * T_C)
    h = lbm.lbm_init(p, column(nx, ny))
    try:
        lbm.lbm_step(h, 3)
        f = state(h, p)
        T = np.empty((ny, nx))
        lbm.lbm_get_temperature(h, T)
        p.T_top = 0.75 * T_C
        lbm.lbm_set_params(h, p)
        lbm.lbm_step(h, 1)
        Tg = np.empty((ny, nx))
        lbm.lbm_get_temperature(h, Tg)
        op = oracle_params(p)
        th = oth.Thermal(c_v=p.c_v, kappa=p.kappa, T_bot=p.T_bot, T_top=p.T_top)
        _, Tw = oth.thermal_step(f, T, op, th)
        assert np.all(Tg[-1] == 0.75 * T_C)
        assert np.max(np.abs(Tg - Tw)) <= 1e-14
    finally:
        lbm.lbm_destroy(h)
