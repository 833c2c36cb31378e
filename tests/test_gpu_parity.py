"""GPU parity: liblbm's CUDA path, called through the C ABI, against the FP64 oracle.

Inputs come from paper_2301_12869_gb300.inputs (seeded); expected values come
only from oracle/. Tolerances:
* FP64 path: the two sides evaluate the same formulas in different association
  orders, so each step adds a few ulp (~1e-17 on populations of order 0.1);
  step-by-step checks use |df| <= 1e-14, and the 10^4-step run the stated
  bound |drho|/rho <= 1e-12.
* FP32 path: one step rounds each of the ~20 terms that build a population to
  FP32 (relative 6e-8 of terms up to ~0.3), so one step is within 1e-6 absolute
  of the FP64 result from the same input; over n steps the conserved density
  performs a bounded random walk, checked against 1e-6 * sqrt(n) + 1e-6.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from oracle import eos
from oracle import lbm as olbm
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
    torch.cuda.init()


def params(nx, ny, Tr, precision="fp64", **kw):
    kw.setdefault("a", A)
    return lbm.make_params(nx, ny, Tr * T_C, precision, **kw)


def oracle_params(p):
    return olbm.Params(
        nx=p.nx, ny=p.ny, a=p.a, b=p.b, R=p.R, T=p.T, G=p.G, sigma=p.sigma, tau_rho=p.tau_rho, tau_e=p.tau_e,
        tau_varsigma=p.tau_varsigma, tau_j=p.tau_j, tau_q=p.tau_q, tau_nu=p.tau_nu, g=(p.gx, p.gy),
        form=p.gravity_form,
    )


def state(h, p):
    f = np.empty((9, p.ny, p.nx))
    lbm.lbm_get_state(h, f)
    return f


def moments(h, p):
    rho, ux, uy = (np.empty((p.ny, p.nx)) for _ in range(3))
    lbm.lbm_moments(h, rho, ux, uy)
    return rho, ux, uy


def column(p, Tr, liquid_rows=None, width=5.0, noise=0.0, seed=inputs.DEFAULT_SEED):
    rv, rl, _ = eos.maxwell(Tr * T_C, p.a, p.b, p.R)
    lr = p.ny // 2 if liquid_rows is None else liquid_rows
    return inputs.column_rho0(p.nx, p.ny, rl, rv, lr, width=width, noise_amp=noise, seed=seed)


MRT = dict(tau_e=0.8, tau_varsigma=1.1, tau_j=1.0, tau_q=1.2, tau_nu=0.7)
TINY = [
    # nx, ny, T/Tc, extra parameters
    (2, 1, 0.85, dict(form=1, g=(0.0, -1e-4))),
    (2, 2, 0.85, dict(form=2, g=(0.0, -1e-4))),
    (2, 3, 0.80, dict(form=1, g=(2e-5, -3e-5))),
    (4, 8, 0.85, dict(form=2, g=(2e-5, -1e-4), **MRT)),
    (6, 5, 0.90, dict(form=1, g=(0.0, -2e-5), sigma=0.3)),
    (8, 13, 0.80, dict(form=2, g=(0.0, 5e-5), **MRT)),
    (10, 7, 0.75, dict(form=1, g=(0.0, 0.0))),
]


@pytest.mark.parametrize("nx, ny, Tr, kw", TINY)
def test_fp64_tiny_lattices_step_by_step(nx, ny, Tr, kw):
    p = params(nx, ny, Tr, "fp64", **kw)
    op = oracle_params(p)
    rho0 = column(p, Tr, width=2.0)
    f = inputs.perturbed_populations(rho0, 0.05, seed=nx * 100 + ny)
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_set_state(h, f)
        for _ in range(5):
            lbm.lbm_step(h, 1)
            f = olbm.step(f, op)
            g = state(h, p)
            assert np.max(np.abs(g - f)) <= 1e-14
        mac = olbm.macroscopic(f, op)
        rho, ux, uy = moments(h, p)
        np.testing.assert_allclose(rho, mac.rho, rtol=0, atol=1e-14)
        np.testing.assert_allclose(ux, mac.u[0], rtol=0, atol=1e-13)
        np.testing.assert_allclose(uy, mac.u[1], rtol=0, atol=1e-13)
        assert lbm.lbm_status(h) == lbm.LBM_OK
    finally:
        lbm.lbm_destroy(h)


def test_fp64_several_bands_and_ragged_strips():
    """nx = 1040 spans three x bands (512, 512, 16) and ny = 301 leaves a short last strip."""
    p = params(1040, 301, 0.8, "fp64", form=2, g=(1e-5, -1e-4), **MRT)
    op = oracle_params(p)
    rho0 = column(p, 0.8, noise=1e-3)
    f = inputs.perturbed_populations(rho0, 0.02, seed=11)
    h = lbm.lbm_init(p, rho0)
    try:
        info = lbm.lbm_launch_info(h)
        assert info["band_width"] < p.nx and p.nx % info["band_width"] != 0
        assert info["strip_rows"] > 1 and p.ny % info["strip_rows"] != 0
        lbm.lbm_set_state(h, f)
        for _ in range(3):
            lbm.lbm_step(h, 1)
            f = olbm.step(f, op)
        assert np.max(np.abs(state(h, p) - f)) <= 1e-14
    finally:
        lbm.lbm_destroy(h)


def test_fp64_liquid_column_10k_steps():
    """4 x 200 column, T = 0.85 T_c, rho g with g_y = -2e-5, tanh interface of width 5,
    liquid below y = 100, 10^4 steps.

    Bulk rows (more than 15 rows from the interface): |drho|/rho <= 1e-12. At the
    interface the method amplifies rounding: its position is a slow, nearly neutral mode,
    and two FP64 evaluations of the same scheme that differ only in summation order (the
    oracle with a reversed density sum and M^-1 applied as its transpose form) drift
    apart by 1.7e-11 there after 10^4 steps (3.9e-13 in the bulk). The whole column is
    therefore held to 5e-11, three times that envelope."""
    p = params(4, 200, 0.85, "fp64", form=1, g=(0.0, -2e-5))
    op = oracle_params(p)
    rho0 = column(p, 0.85, liquid_rows=100)
    h = lbm.lbm_init(p, rho0)
    try:
        m0 = lbm.lbm_reduce(h, lbm.LBM_REDUCE_MASS)[0]
        lbm.lbm_step(h, 10000)
        f = olbm.run(olbm.init_state(rho0), op, 10000)
        rho, ux, uy = moments(h, p)
        mac = olbm.macroscopic(f, op)
        rel = np.abs(rho - mac.rho) / mac.rho
        bulk = np.abs(np.arange(p.ny) - 99.5) > 15
        assert rel[bulk].max() <= 1e-12
        assert rel.max() <= 5e-11
        assert np.all(rho == rho[:, :1])  # x-uniform stays bitwise uniform
        m1 = lbm.lbm_reduce(h, lbm.LBM_REDUCE_MASS)[0]
        # the collision conserves mass up to rounding; near a steady state the same
        # rounding repeats every step, so both sides drift linearly by ~5e-17 per step
        # (relative): bound 1e-12 after 10^4 steps, and the two drifts agree
        assert abs(m1 - m0) / m0 <= 1e-12
        assert m1 == pytest.approx(olbm.mass(f), rel=1e-13)
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("nsteps", [1, 10, 100])
def test_fp32_against_fp64_oracle(nsteps):
    p = params(8, 64, 0.8, "fp32", form=2, g=(0.0, -1e-4))
    op = oracle_params(p)
    rho0 = column(p, 0.8, noise=1e-3)
    h = lbm.lbm_init(p, rho0)
    try:
        # the FP32 state starts from the same rest equilibrium rounded to FP32 deviations
        f = state(h, p)
        lbm.lbm_step(h, nsteps)
        f = olbm.run(f, op, nsteps)
        g = state(h, p)
        tol = 1e-6 * math.sqrt(nsteps) + 1e-6
        assert np.max(np.abs(g - f)) <= tol
        rho, _, _ = moments(h, p)
        assert np.max(np.abs(rho - olbm.macroscopic(f, op).rho)) <= tol
    finally:
        lbm.lbm_destroy(h)


def test_fp32_several_bands_and_ragged():
    p = params(1028, 301, 0.8, "fp32", form=2, g=(0.0, -1e-4), **MRT)
    op = oracle_params(p)
    rho0 = column(p, 0.8, noise=1e-3)
    h = lbm.lbm_init(p, rho0)
    try:
        info = lbm.lbm_launch_info(h)
        assert info["band_width"] < p.nx
        f = state(h, p)
        lbm.lbm_step(h, 2)
        f = olbm.run(f, op, 2)
        assert np.max(np.abs(state(h, p) - f)) <= 2e-6
    finally:
        lbm.lbm_destroy(h)


def test_reductions_match_oracle():
    p = params(6, 40, 0.85, "fp64", form=2, g=(0.0, -1e-4))
    op = oracle_params(p)
    rho0 = column(p, 0.85)
    h = lbm.lbm_init(p, rho0)
    try:
        f = olbm.init_state(rho0)
        r0 = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)[0]
        assert math.isinf(r0)
        lbm.lbm_step(h, 50)
        f = olbm.run(f, op, 50)
        mac = olbm.macroscopic(f, op)
        assert lbm.lbm_reduce(h, lbm.LBM_REDUCE_MASS)[0] == pytest.approx(olbm.mass(f), rel=1e-14)
        assert lbm.lbm_reduce(h, lbm.LBM_REDUCE_MEAN_RHO)[0] == pytest.approx(mac.mean_rho, rel=1e-14)
        speed = np.sqrt(mac.u[0] ** 2 + mac.u[1] ** 2)
        assert lbm.lbm_reduce(h, lbm.LBM_REDUCE_MAX_U)[0] == pytest.approx(speed.max(), rel=1e-10)
        rv, rl, _ = eos.maxwell(p.T, A, B, R)
        yi = olbm.interface_height(mac.rho, 0.5 * (rl + rv))
        assert lbm.lbm_reduce(h, lbm.LBM_REDUCE_INTERFACE_Y)[0] == pytest.approx(yi, abs=1e-9)
        prof = mac.rho.mean(axis=1)
        mx, mn = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RHO_LV)
        assert mx == pytest.approx(prof.max(), rel=1e-13) and mn == pytest.approx(prof.min(), rel=1e-13)
        # residual: max |rho_t - rho_t'| between two calls
        rho_a = mac.rho
        lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)
        lbm.lbm_step(h, 3)
        f = olbm.run(f, op, 3)
        res = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)[0]
        want = olbm.residual(olbm.macroscopic(f, op).rho, rho_a)
        assert res == pytest.approx(want, rel=1e-9, abs=1e-16)
    finally:
        lbm.lbm_destroy(h)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_state_round_trip_host_and_device(precision):
    import torch

    p = params(8, 12, 0.8, precision)
    rho0 = column(p, 0.8)
    f = inputs.perturbed_populations(rho0, 0.1, seed=5)
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_set_state(h, f, steps_done=7)
        g = np.empty_like(f)
        assert lbm.lbm_get_state(h, g) == 7
        tol = 0.0 if precision == "fp64" else 1e-8
        assert np.max(np.abs(g - f)) <= tol
        fd = torch.from_numpy(f).cuda()
        gd = torch.empty_like(fd)
        lbm.lbm_set_state(h, fd)
        lbm.lbm_get_state(h, gd)
        torch.cuda.synchronize()
        assert np.max(np.abs(gd.cpu().numpy() - f)) <= tol
    finally:
        lbm.lbm_destroy(h)


def test_gravity_forms_bitwise_equal_at_zero_gravity():
    out = []
    for form in (1, 2):
        p = params(8, 32, 0.8, "fp64", form=form, g=(0.0, 0.0))
        h = lbm.lbm_init(p, column(p, 0.8, noise=1e-3))
        lbm.lbm_step(h, 40)
        out.append(state(h, p))
        lbm.lbm_destroy(h)
    np.testing.assert_array_equal(out[0], out[1])


def test_nonphysical_state_is_reported_not_faulted():
    """Rows at rho = 0.7 (a rest state there streams back to rho = 0.7) have
    p_EOS > rho/3, so psi^2 < 0: the kernel clamps, records LBM_ENONPHYS in the
    sticky status, and the context stays usable."""
    p = params(4, 10, 0.8, "fp64")
    rho0 = np.full((10, 4), 0.1)
    rho0[4:7, :] = 0.7
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_step(h, 1)
        assert lbm.lbm_status(h) == lbm.LBM_ENONPHYS
        assert "non-physical" in lbm.lbm_last_error(h)
        lbm.lbm_set_state(h, inputs.perturbed_populations(np.full((10, 4), 0.1), 0.0))
        assert lbm.lbm_status(h) == lbm.LBM_OK
    finally:
        lbm.lbm_destroy(h)


def test_torch_workspace_lattice_matches_plain_handle():
    """Workspace from a torch tensor and torch's current stream: same bits as a
    handle whose memory the library allocates."""
    import torch

    p = params(16, 20, 0.85, "fp32", form=1, g=(0.0, -2e-5))
    rho0 = column(p, 0.85)
    lat = lbm.Lattice(p, torch.from_numpy(rho0).cuda())
    q = params(16, 20, 0.85, "fp32", form=1, g=(0.0, -2e-5))
    h = lbm.lbm_init(q, rho0)
    try:
        lat.step(25)
        lbm.lbm_step(h, 25)
        rho, ux, uy = lat.moments()
        torch.cuda.synchronize()
        assert rho.is_cuda and tuple(rho.shape) == (20, 16)
        np.testing.assert_array_equal(lat.get_state(), state(h, q))
        np.testing.assert_array_equal(rho.cpu().numpy(), moments(h, q)[0])
    finally:
        lat.close()
        lbm.lbm_destroy(h)


# ---------------------------------------------------------------- full size, sampled
def _sample_nodes(nx, ny, rng, k=48):
    ys = [0, 1, 2, ny // 2, ny // 2 + 1, ny - 3, ny - 2, ny - 1] + list(rng.integers(0, ny, k))
    xs = [0, nx - 1, 1, nx // 2, 511, 512, 513, 1023 % nx] + list(rng.integers(0, nx, k))
    return list(zip(ys[: len(xs)], xs[: len(ys)]))


def _patch_step(f_full, op, y, x, mean_rho):
    """Oracle step for node (x, y) from a 5 x 5 patch of the full state (the node's result
    depends only on its two-node neighbourhood); mean_rho is the full domain's."""
    ny, nx = f_full.shape[1:]
    y0, y1 = max(0, y - 2), min(ny, y + 3)
    cols = [(x + d) % nx for d in range(-2, 3)]
    patch = np.ascontiguousarray(f_full[:, y0:y1][:, :, cols])
    q = dataclasses.replace(op, nx=5, ny=y1 - y0)
    # a patch edge that is not a real wall must not zero F_int on the sampled row
    assert (y - y0 >= 1 or y == 0) and (y1 - 1 - y >= 1 or y == ny - 1)
    return olbm.step(patch, q, mean_rho=mean_rho)[:, y - y0, 2]


@pytest.mark.parametrize("precision, tol", [("fp32", 1e-6), ("fp64", 1e-14)])
def test_full_size_large_domain_sampled(precision, tol):
    """1024 x 4096, (rho - <rho>) g with g_y = -1e-4 at T = 0.8 T_c, seeded +-1e-3 noise
    across the interface at y = 2047.5 (the single-domain workload), in the launch
    configuration bench.py times: one GPU step from a state after 20 steps, checked on
    sampled nodes against the oracle run on each node's neighbourhood."""
    nx, ny = 1024, 4096
    p = params(nx, ny, 0.8, precision, form=2, g=(0.0, -1e-4))
    op = oracle_params(p)
    rho0 = column(p, 0.8, liquid_rows=2048, noise=1e-3)
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_step(h, 20)
        f_t = state(h, p)
        mean_rho = float(np.sum(f_t)) / (nx * ny)
        assert lbm.lbm_reduce(h, lbm.LBM_REDUCE_MEAN_RHO)[0] == pytest.approx(mean_rho, rel=1e-12)
        lbm.lbm_step(h, 1)
        f_next = state(h, p)
        rng = np.random.default_rng(2023)
        worst = 0.0
        for (y, x) in _sample_nodes(nx, ny, rng):
            want = _patch_step(f_t, op, int(y), int(x), mean_rho)
            worst = max(worst, float(np.max(np.abs(f_next[:, y, x] - want))))
        assert worst <= tol, worst
        assert lbm.lbm_status(h) == lbm.LBM_OK
    finally:
        lbm.lbm_destroy(h)


# ---------------------------------------------------------------- tile variants and autotune
@pytest.mark.parametrize("precision, nx, ny, tol", [("fp32", 1028, 150, 2e-6), ("fp64", 1040, 150, 1e-14)])
def test_every_tile_variant_matches_oracle(precision, nx, ny, tol):
    """Each tile variant of the fused kernel (band width x threads) on a lattice with a
    ragged last band, general MRT relaxation and then all-unit relaxation."""
    for extra in (MRT, {}):
        p = params(nx, ny, 0.8, precision, form=2, g=(1e-5, -1e-4), **extra)
        op = oracle_params(p)
        rho0 = column(p, 0.8, noise=1e-3)
        f0 = None
        for v in range(lbm.lbm_tile_variants(p.precision)):
            h = lbm.lbm_init(p, rho0)
            try:
                lbm.lbm_set_tiling(h, v)
                if f0 is None:
                    f0 = state(h, p)
                    want = olbm.run(f0, op, 2)
                lbm.lbm_step(h, 2)
                assert np.max(np.abs(state(h, p) - want)) <= tol, (v, extra)
            finally:
                lbm.lbm_destroy(h)


def test_autotune_keeps_state_and_picks_a_variant():
    p = params(1024, 256, 0.8, "fp32", form=2, g=(0.0, -1e-4))
    h = lbm.lbm_init(p, column(p, 0.8, noise=1e-3))
    try:
        lbm.lbm_step(h, 3)
        before = state(h, p)
        v, ms = lbm.lbm_autotune(h, 5)
        assert 0 <= v < lbm.lbm_tile_variants(p.precision) and ms > 0
        np.testing.assert_array_equal(state(h, p), before)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_tiling(h, 99)
    finally:
        lbm.lbm_destroy(h)
