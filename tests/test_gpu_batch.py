"""GPU tests of the batched-column runner (lbm_batch_*) against the FP64 oracle.

Each column of a batch is an independent nx x ny_c lattice with its own height,
temperature, gravity and gravity form; every column is checked against the
oracle run on that column alone. Tolerances as in test_gpu_parity.py: FP64
1e-14 per step for a few steps, FP32 1e-6 sqrt(n) + 1e-6.
"""
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
NX = 4


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


def make_columns(n, seed, heights=(8, 16, 24, 32, 48, 64)):
    rng = np.random.default_rng(seed)
    cols, rhos = [], []
    for c in range(n):
        ny = int(heights[c % len(heights)])
        Tr = float(rng.uniform(0.72, 0.92))
        gy = -float(10 ** rng.uniform(-6, -4))
        form = 1 + (c % 2)
        frac = float(rng.uniform(0.3, 0.7))
        rv, rl, _ = eos.maxwell(Tr * T_C, A, B, R)
        rho0 = inputs.column_rho0(NX, ny, rl, rv, max(1, int(round(frac * ny))), width=3.0)
        cols.append(dict(ny=ny, T=Tr * T_C, gx=0.0, gy=gy, form=form))
        rhos.append(rho0)
    return cols, rhos


def batch_params(precision, **kw):
    kw.setdefault("a", A)
    return lbm.make_params(NX, 8, 0.8 * T_C, precision, **kw)


def oracle_column(col, p):
    return olbm.Params(nx=NX, ny=col["ny"], a=A, b=B, R=R, T=col["T"], G=p.G, sigma=p.sigma, tau_rho=p.tau_rho,
                       tau_e=p.tau_e, tau_varsigma=p.tau_varsigma, tau_j=p.tau_j, tau_q=p.tau_q, tau_nu=p.tau_nu,
                       g=(col["gx"], col["gy"]), form=col["form"],
                       wall="zou-he" if p.wall == lbm.LBM_WALL_ZOU_HE else "bounce-back")


def split_state(f_all, cols):
    out, off = [], 0
    for col in cols:
        n = 9 * NX * col["ny"]
        out.append(f_all[off:off + n].reshape(9, col["ny"], NX))
        off += n
    return out


@pytest.mark.parametrize("precision, steps, tol, taus", [
    ("fp64", 7, 1e-14, {}),
    ("fp64", 7, 1e-14, dict(tau_e=0.8, tau_varsigma=1.1, tau_q=1.2, tau_nu=0.7)),
    ("fp32", 50, 1e-6 * math.sqrt(50) + 1e-6, {}),
    # double-float: ~2^-46 relative per operation, a few hundred operations per node and step
    ("dd", 7, 1e-12, {}),
    ("dd", 7, 1e-12, dict(tau_e=0.8, tau_varsigma=1.1, tau_q=1.2, tau_nu=0.7)),
])
def test_every_column_matches_oracle(precision, steps, tol, taus):
    cols, rhos = make_columns(24, seed=3)
    p = batch_params(precision, **taus)
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        total = sum(9 * NX * c["ny"] for c in cols)
        f0 = np.empty(total)
        lbm.lbm_batch_get_state(b, f0)
        lbm.lbm_batch_run(b, 0.0, steps, check_every=1000)
        f1 = np.empty(total)
        lbm.lbm_batch_get_state(b, f1)
        st, res, status = lbm.lbm_batch_results(b, len(cols))
        assert np.all(st == steps) and np.all(status == 0)
        for col, g0, g1 in zip(cols, split_state(f0, cols), split_state(f1, cols)):
            want = olbm.run(g0, oracle_column(col, p), steps)
            assert np.max(np.abs(g1 - want)) <= tol, col
    finally:
        lbm.lbm_batch_destroy(b)


@pytest.mark.parametrize("precision, tol", [
    ("fp64", 1e-13),
    ("fp32", 1e-6 * math.sqrt(32) + 1e-6),
    ("dd", 1e-11),
])
@pytest.mark.parametrize("threads", [128, 256, 512])
def test_tall_columns_match_oracle(precision, tol, threads):
    """The heights of the batched workload up to 1024 rows in one batch: the dynamic shared
    memory is sized by the tallest column and a 128-thread CTA carries 32 nodes per thread.
    Every column, after 32 steps, against the oracle run on that column alone."""
    heights = (1024, 512, 256, 64, 1024, 128, 256, 512, 1024, 256)
    cols, rhos = make_columns(len(heights), seed=31, heights=heights)
    p = batch_params(precision)
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        lbm.lbm_batch_set_threads(b, threads)
        total = sum(9 * NX * c["ny"] for c in cols)
        f0, f1 = np.empty(total), np.empty(total)
        lbm.lbm_batch_get_state(b, f0)
        lbm.lbm_batch_run(b, 0.0, 32, check_every=1000)
        lbm.lbm_batch_get_state(b, f1)
        st, _, status = lbm.lbm_batch_results(b, len(cols))
        assert np.all(st == 32) and np.all(status == 0)
        for col, g0, g1 in zip(cols, split_state(f0, cols), split_state(f1, cols)):
            want = olbm.run(g0, oracle_column(col, p), 32)
            assert np.max(np.abs(g1 - want)) <= tol, col
    finally:
        lbm.lbm_batch_destroy(b)


@pytest.mark.parametrize("precision, steps, tol, taus", [
    ("fp64", 7, 1e-14, {}),
    ("fp64", 7, 1e-14, dict(tau_e=0.8, tau_varsigma=1.1, tau_q=1.2, tau_nu=0.7)),
    ("fp32", 50, 1e-6 * math.sqrt(50) + 1e-6, {}),
    ("dd", 7, 1e-12, {}),
])
def test_zou_he_columns_match_oracle(precision, steps, tol, taus):
    """The paper's wet-node walls (Sec. III) in the batch kernel: every column against the
    oracle's Zou-He column, both gravity forms, heights 8..64 (and one of 3 rows, the
    smallest the closure allows)."""
    cols, rhos = make_columns(13, seed=41)
    cols[-1]["ny"] = 3
    rhos[-1] = np.full((3, NX), 0.15)
    p = batch_params(precision, wall=lbm.LBM_WALL_ZOU_HE, **taus)
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        total = sum(9 * NX * c["ny"] for c in cols)
        f0, f1 = np.empty(total), np.empty(total)
        lbm.lbm_batch_get_state(b, f0)
        lbm.lbm_batch_run(b, 0.0, steps, check_every=1000)
        lbm.lbm_batch_get_state(b, f1)
        st, _, status = lbm.lbm_batch_results(b, len(cols))
        assert np.all(st == steps) and np.all(status == 0)
        for col, g0, g1 in zip(cols, split_state(f0, cols), split_state(f1, cols)):
            want = olbm.run(g0, oracle_column(col, p), steps)
            assert np.max(np.abs(g1 - want)) <= tol, col
    finally:
        lbm.lbm_batch_destroy(b)


def test_zou_he_batch_column_equals_single_lattice_handle():
    """Zou-He columns of a batch run to a residual target equal lbm_step on the same column
    (FP64), and the batch's moments match the handle's."""
    cols, rhos = make_columns(3, seed=43, heights=(40, 24))
    p = batch_params("fp64", wall=lbm.LBM_WALL_ZOU_HE)
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        lbm.lbm_batch_run(b, 0.0, 500, check_every=1000)
        f = np.empty(sum(9 * NX * c["ny"] for c in cols))
        lbm.lbm_batch_get_state(b, f)
        rho_b = np.empty(sum(NX * c["ny"] for c in cols))
        lbm.lbm_batch_moments(b, rho=rho_b)
        off = 0
        for col, rho0, g in zip(cols, rhos, split_state(f, cols)):
            q = lbm.make_params(NX, col["ny"], col["T"], "fp64", a=A, form=col["form"], g=(col["gx"], col["gy"]),
                                wall=lbm.LBM_WALL_ZOU_HE)
            h = lbm.lbm_init(q, rho0)
            lbm.lbm_step(h, 500)
            fh = np.empty((9, col["ny"], NX))
            lbm.lbm_get_state(h, fh)
            rh = np.empty((col["ny"], NX))
            lbm.lbm_moments(h, rh)
            lbm.lbm_destroy(h)
            assert np.max(np.abs(fh - g)) <= 1e-13
            assert np.max(np.abs(rh.ravel() - rho_b[off:off + rh.size])) <= 1e-13
            off += rh.size
    finally:
        lbm.lbm_batch_destroy(b)


def test_column_seconds_bound_by_the_run():
    """lbm_batch_column_seconds: every column's device time is positive, no longer than the
    run that contains it, summed over runs and carried over by lbm_batch_convert."""
    cols, rhos = make_columns(40, seed=47)
    b = lbm.lbm_batch_init(batch_params("fp32"), cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        t1 = lbm.lbm_batch_run(b, 0.0, 300, check_every=100)
        s1 = lbm.lbm_batch_column_seconds(b, len(cols))
        assert np.all(s1 > 0) and np.all(s1 <= t1 * 1.001 + 1e-5)
        t2 = lbm.lbm_batch_run(b, 0.0, 300, check_every=100)
        s2 = lbm.lbm_batch_column_seconds(b, len(cols))
        assert np.all(s2 > s1) and np.all(s2 - s1 <= t2 * 1.001 + 1e-5)
        bc = lbm.lbm_batch_convert(b, lbm.LBM_FP64)
        try:
            assert np.array_equal(lbm.lbm_batch_column_seconds(bc, len(cols)), s2)
        finally:
            lbm.lbm_batch_destroy(bc)
    finally:
        lbm.lbm_batch_destroy(b)


def test_batch_column_equals_single_lattice_handle():
    """The batch runner and lbm_step give the same state for the same column (FP64)."""
    cols, rhos = make_columns(3, seed=9, heights=(40,))
    p = batch_params("fp64")
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        lbm.lbm_batch_run(b, 0.0, 300, check_every=1000)
        f = np.empty(sum(9 * NX * c["ny"] for c in cols))
        lbm.lbm_batch_get_state(b, f)
        for col, rho0, g in zip(cols, rhos, split_state(f, cols)):
            q = lbm.make_params(NX, col["ny"], col["T"], "fp64", a=A, form=col["form"], g=(col["gx"], col["gy"]))
            h = lbm.lbm_init(q, rho0)
            lbm.lbm_step(h, 300)
            fh = np.empty((9, col["ny"], NX))
            lbm.lbm_get_state(h, fh)
            lbm.lbm_destroy(h)
            assert np.max(np.abs(fh - g)) <= 1e-13
    finally:
        lbm.lbm_batch_destroy(b)


def test_residual_target_and_precision_continuation():
    """FP32 to its rounding floor, then FP64 to 1e-10: every column reaches the target,
    and the final profiles agree with an FP64-only run to the FP32 path's accuracy."""
    cols, rhos = make_columns(8, seed=5, heights=(16, 24))
    rho_all = np.concatenate([r.ravel() for r in rhos])
    b32 = lbm.lbm_batch_init(batch_params("fp32"), cols, rho_all)
    b64 = lbm.lbm_batch_init(batch_params("fp64"), cols, rho_all)
    try:
        lbm.lbm_batch_run(b32, 1e-6, 200000, check_every=100)
        st32, res32, _ = lbm.lbm_batch_results(b32, len(cols))
        assert np.all(res32 <= 1e-6)
        b = lbm.lbm_batch_convert(b32, lbm.LBM_FP64)
        try:
            lbm.lbm_batch_run(b, 1e-10, 400000, check_every=100)
            st, res, status = lbm.lbm_batch_results(b, len(cols))
            assert np.all(res <= 1e-10) and np.all(status == 0)
            assert np.all(st >= st32)
            lbm.lbm_batch_run(b64, 1e-10, 400000, check_every=100)
            _, res64, _ = lbm.lbm_batch_results(b64, len(cols))
            assert np.all(res64 <= 1e-10)
            n = rho_all.size
            r1, r2 = np.empty(n), np.empty(n)
            lbm.lbm_batch_moments(b, rho=r1)
            lbm.lbm_batch_moments(b64, rho=r2)
            # both are steady states of the same columns: equal to the FP32 mass error
            assert np.max(np.abs(r1 - r2)) <= 1e-5
        finally:
            lbm.lbm_batch_destroy(b)
    finally:
        lbm.lbm_batch_destroy(b32)
        lbm.lbm_batch_destroy(b64)


def test_batch_moments_match_oracle():
    cols, rhos = make_columns(6, seed=11)
    p = batch_params("fp64")
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        lbm.lbm_batch_run(b, 0.0, 20, check_every=1000)
        total = sum(NX * c["ny"] for c in cols)
        f = np.empty(9 * total)
        lbm.lbm_batch_get_state(b, f)
        rho, ux, uy = np.empty(total), np.empty(total), np.empty(total)
        lbm.lbm_batch_moments(b, rho, ux, uy)
        off = 0
        for col, g in zip(cols, split_state(f, cols)):
            n = NX * col["ny"]
            mac = olbm.macroscopic(g, oracle_column(col, p))
            np.testing.assert_allclose(rho[off:off + n].reshape(col["ny"], NX), mac.rho, rtol=0, atol=1e-14)
            np.testing.assert_allclose(uy[off:off + n].reshape(col["ny"], NX), mac.u[1], rtol=0, atol=1e-13)
            off += n
    finally:
        lbm.lbm_batch_destroy(b)


def test_batch_rejects_oversized_columns():
    p = batch_params("fp64")
    with pytest.raises(lbm.LbmError, match="shared memory"):
        lbm.lbm_batch_init(p, [dict(ny=4000, T=0.8 * T_C, form=1)], np.full(4 * 4000, 0.1))


def test_fp32_columns_stop_at_their_rounding_floor():
    """With a target below FP32 reach, lbm_batch_run_stall stops each FP32 column once ten
    checks have not lowered its residual by 1 %: well before max_steps, at a floor of a few
    1e-9 to a few 1e-8 (the FP64-evaluated change per step of the FP32 state)."""
    cols, rhos = make_columns(8, seed=21, heights=(16, 24))
    b = lbm.lbm_batch_init(batch_params("fp32"), cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        lbm.lbm_batch_run_stall(b, 1e-13, 400000, 100, 10)
        st, res, status = lbm.lbm_batch_results(b, len(cols))
        assert np.all(status == 0)
        assert np.all(st < 400000)
        assert np.all((res > 1e-10) & (res < 1e-7))
    finally:
        lbm.lbm_batch_destroy(b)


def test_extrapolation_reaches_the_same_steady_states_in_fewer_steps():
    """lbm_batch_set_acceleration: FP64 columns run to 1e-10 with extrapolation every five
    checks reach the steady states of the plain iteration in fewer steps in total. The two
    are compared at 1e-5: the slow modes decay as damped oscillations, whose per-step change
    dips towards zero at every turning point, so a run can meet "per-step change <= 1e-10"
    while still ~1e-6 from its fixed point (as the warm-start comparison also allows)."""
    cols, rhos = make_columns(24, seed=31, heights=(32, 48, 64))
    rho = np.concatenate([r.ravel() for r in rhos])
    out = []
    for checks in (0, 5):
        b = lbm.lbm_batch_init(batch_params("fp64"), cols, rho)
        try:
            if checks:
                lbm.lbm_batch_set_acceleration(b, checks)
            lbm.lbm_batch_run(b, 1e-10, 300000, 100)
            st, res, status = lbm.lbm_batch_results(b, len(cols))
            r = np.empty(rho.size)
            lbm.lbm_batch_moments(b, rho=r)
            out.append((st, res, status, r))
        finally:
            lbm.lbm_batch_destroy(b)
    (st0, res0, s0, r0), (st1, res1, s1, r1) = out
    ok = (res0 <= 1e-10) & (res1 <= 1e-10) & (s0 == 0) & (s1 == 0)
    assert ok.sum() >= 0.9 * len(cols)
    assert np.sum(st1[ok]) < 0.8 * np.sum(st0[ok])
    off = np.cumsum([0] + [NX * c["ny"] for c in cols])
    for c in np.nonzero(ok)[0]:
        assert np.max(np.abs(r1[off[c]:off[c + 1]] - r0[off[c]:off[c + 1]])) <= 1e-5, c


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-14), ("fp32", 1e-6 * math.sqrt(40) + 1e-6), ("dd", 1e-12)])
def test_every_block_size_matches_oracle(precision, tol):
    """128, 256 and 512 threads per column CTA: the oracle's states after 40 steps (the
    block size changes only the order of the FP64 mass partials)."""
    cols, rhos = make_columns(10, seed=21, heights=(8, 24, 64, 150))
    p = batch_params(precision)
    total = sum(9 * NX * c["ny"] for c in cols)
    for threads in (128, 256, 512):
        b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
        try:
            lbm.lbm_batch_set_threads(b, threads)
            f0 = np.empty(total)
            lbm.lbm_batch_get_state(b, f0)
            lbm.lbm_batch_run(b, 0.0, 40, check_every=1000)
            f1 = np.empty(total)
            lbm.lbm_batch_get_state(b, f1)
            for col, g0, g1 in zip(cols, split_state(f0, cols), split_state(f1, cols)):
                want = olbm.run(g0, oracle_column(col, p), 40)
                assert np.max(np.abs(g1 - want)) <= tol * (1 if precision == "fp32" else 40), (threads, col)
        finally:
            lbm.lbm_batch_destroy(b)


def test_autotune_keeps_the_fastest_block_size_and_leaves_the_state():
    cols, rhos = make_columns(64, seed=22, heights=(32, 64, 96))
    b = lbm.lbm_batch_init(batch_params("fp32"), cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        lbm.lbm_batch_run(b, 0.0, 30, check_every=10)
        total = sum(9 * NX * c["ny"] for c in cols)
        f0 = np.empty(total)
        lbm.lbm_batch_get_state(b, f0)
        st0, res0, _ = lbm.lbm_batch_results(b, len(cols))
        best, times = lbm.lbm_batch_autotune(b, steps=50)
        assert sorted(times) == [128, 256, 512] and all(t > 0 for t in times.values())
        assert best == min(times, key=times.get)
        f1 = np.empty(total)
        lbm.lbm_batch_get_state(b, f1)
        st1, res1, _ = lbm.lbm_batch_results(b, len(cols))
        np.testing.assert_array_equal(f1, f0)
        np.testing.assert_array_equal(st1, st0)
        np.testing.assert_array_equal(res1, res0)
        # the tuned batch still runs (the graph is recaptured for the kept block size)
        lbm.lbm_batch_run(b, 0.0, 10, check_every=5)
        assert np.all(lbm.lbm_batch_results(b, len(cols))[0] == 40)
        with pytest.raises(lbm.LbmError, match="128, 256 or 512"):
            lbm.lbm_batch_set_threads(b, 64)
    finally:
        lbm.lbm_batch_destroy(b)


def test_double_float_continuation_reaches_fp64_steady_states():
    """FP32 to 1e-6, then double-float (FP32-pair) arithmetic to 1e-10: every column reaches
    the target and ends where the plain FP64 run does (to the FP32 path's 1e-5, as in the
    FP64 continuation); a double-float batch also runs on to 1e-12, well below any FP32
    rounding floor (~1e-8)."""
    cols, rhos = make_columns(8, seed=5, heights=(16, 24))
    rho_all = np.concatenate([r.ravel() for r in rhos])
    b32 = lbm.lbm_batch_init(batch_params("fp32"), cols, rho_all)
    b64 = lbm.lbm_batch_init(batch_params("fp64"), cols, rho_all)
    bdd = lbm.lbm_batch_init(batch_params("dd"), cols, rho_all)
    try:
        lbm.lbm_batch_run(b32, 1e-6, 200000, check_every=100)
        b = lbm.lbm_batch_convert(b32, lbm.LBM_DOUBLE_FLOAT)
        try:
            lbm.lbm_batch_run(b, 1e-10, 400000, check_every=100)
            _, res, status = lbm.lbm_batch_results(b, len(cols))
            assert np.all(res <= 1e-10) and np.all(status == 0)
            lbm.lbm_batch_run(b64, 1e-10, 400000, check_every=100)
            n = rho_all.size
            r1, r2 = np.empty(n), np.empty(n)
            lbm.lbm_batch_moments(b, rho=r1)
            lbm.lbm_batch_moments(b64, rho=r2)
            assert np.max(np.abs(r1 - r2)) <= 1e-5
        finally:
            lbm.lbm_batch_destroy(b)
        lbm.lbm_batch_run(bdd, 1e-12, 600000, check_every=100)
        _, resdd, sdd = lbm.lbm_batch_results(bdd, len(cols))
        assert np.all(resdd <= 1e-12) and np.all(sdd == 0)
    finally:
        lbm.lbm_batch_destroy(b32)
        lbm.lbm_batch_destroy(b64)
        lbm.lbm_batch_destroy(bdd)


@pytest.mark.parametrize("precision, tol", [("fp64", 1e-13), ("fp32", 1e-6 * math.sqrt(30) + 1e-6), ("dd", 1e-11)])
def test_stated_column_set_sampled(precision, tol):
    """The time-to-steady block's column set as stated - 4096 seeded columns, H in {64, 128,
    256, 512, 1024} - in its launch configuration (autotuned block size, extrapolation on for
    FP32 and double-float as that block runs them): 30 steps of every column, then
    sampled columns of every height against the oracle run on each column alone."""
    import bench

    cols, rho = bench.column_set(4096, bench.SEED, bench.STEADY_HEIGHTS, lbm, inputs)
    cols = [dict(c, gx=0.0) for c in cols]
    p = lbm.make_params(4, 8, 0.8 * T_C, precision, a=A, b=B, R=R)
    b = lbm.lbm_batch_init(p, cols, rho)
    try:
        lbm.lbm_batch_autotune(b, 5)
        if precision != "fp64":
            lbm.lbm_batch_set_acceleration(b, bench.ACCEL_CHECKS)  # no snapshot within 30 steps
        total = sum(9 * NX * c["ny"] for c in cols)
        f0, f1 = np.empty(total), np.empty(total)
        lbm.lbm_batch_get_state(b, f0)
        lbm.lbm_batch_run(b, 0.0, 30, check_every=1000)
        lbm.lbm_batch_get_state(b, f1)
    finally:
        lbm.lbm_batch_destroy(b)
    g0s, g1s = split_state(f0, cols), split_state(f1, cols)
    hs = np.array([c["ny"] for c in cols])
    rng = np.random.default_rng(79)
    picks = [int(rng.choice(np.nonzero(hs == H)[0])) for H in bench.STEADY_HEIGHTS for _ in range(2)]
    for c in [0, len(cols) - 1] + picks:
        want = olbm.run(g0s[c], oracle_column(cols[c], p), 30)
        assert np.max(np.abs(g1s[c] - want)) <= tol, (c, cols[c]["ny"])


@pytest.mark.parametrize("precision, tol", [("fp32", 1e-6 * math.sqrt(30) + 1e-6), ("dd", 1e-11)])
def test_full_size_column_set_sampled(precision, tol):
    """The columns workload's 1024 seeded columns (H in {64, 128}) in its launch
    configuration (block size from the autotuner): 30 steps of every column, sampled columns
    checked against the oracle run on each column alone."""
    import bench

    cols, rho = bench.column_set(1024, bench.SEED, (64, 128), lbm, inputs)
    cols = [dict(c, gx=0.0) for c in cols]
    p = lbm.make_params(4, 8, 0.8 * T_C, precision, a=A, b=B, R=R)
    b = lbm.lbm_batch_init(p, cols, rho)
    try:
        lbm.lbm_batch_autotune(b, 20)
        total = sum(9 * NX * c["ny"] for c in cols)
        f0, f1 = np.empty(total), np.empty(total)
        lbm.lbm_batch_get_state(b, f0)
        lbm.lbm_batch_run(b, 0.0, 30, check_every=1000)
        lbm.lbm_batch_get_state(b, f1)
    finally:
        lbm.lbm_batch_destroy(b)
    g0s, g1s = split_state(f0, cols), split_state(f1, cols)
    rng = np.random.default_rng(77)
    for c in [0, 1, 511, 1023] + list(rng.integers(0, len(cols), 4)):
        want = olbm.run(g0s[c], oracle_column(cols[c], p), 30)
        assert np.max(np.abs(g1s[c] - want)) <= tol, (c, cols[c])


@pytest.mark.parametrize("precision, tol, taus", [
    ("fp64", 1e-14, {}),
    ("fp64", 1e-14, dict(tau_e=0.8, tau_varsigma=1.1, tau_q=1.2, tau_nu=0.7)),
    ("fp32", 2e-6, {}),
    ("dd", 1e-12, {}),
])
def test_rest_state_matches_oracle(precision, tol, taus):
    """lbm_batch_rest_state on every column of a mixed batch (heights 3 .. 1024, both gravity
    forms, own T and g) against the oracle's rest_state of the column's stored density."""
    heights = (8, 24, 64, 256, 1024, 3)
    cols, rhos = make_columns(12, seed=41, heights=heights)
    p = batch_params(precision, **taus)
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        total = sum(9 * NX * c["ny"] for c in cols)
        f0 = np.empty(total)
        lbm.lbm_batch_get_state(b, f0)
        lbm.lbm_batch_rest_state(b)
        f1 = np.empty(total)
        lbm.lbm_batch_get_state(b, f1)
        _, _, status = lbm.lbm_batch_results(b, len(cols))
        assert np.all(status == 0)
        for col, g0, g1 in zip(cols, split_state(f0, cols), split_state(f1, cols)):
            want = olbm.rest_state(g0.sum(axis=0), oracle_column(col, p))
            assert np.max(np.abs(g1 - want)) <= tol, col
    finally:
        lbm.lbm_batch_destroy(b)


def test_rest_state_of_a_steady_density_starts_at_the_steady_state():
    """Columns run in FP64 to a per-step change of 1e-12, then restarted from their converged
    density: from the rest state of that density they are back below 1e-10 at the first
    check (100 steps), while the rest equilibrium f_eq(rho, 0) of the same density
    (lbm_batch_init alone) takes 900 - 8000 steps - the slow transient every equilibrium
    start pays comes from the missing forcing terms, not from the density."""
    import torch

    cols, rhos = make_columns(8, seed=17, heights=(16, 24, 32))
    p = batch_params("fp64")
    b = lbm.lbm_batch_init(p, cols, np.concatenate([r.ravel() for r in rhos]))
    try:
        lbm.lbm_batch_run(b, 1e-12, 400000, 100)
        _, res, status = lbm.lbm_batch_results(b, len(cols))
        assert np.all(res <= 1e-12) and np.all(status == 0)
        rho = torch.empty(sum(NX * c["ny"] for c in cols), dtype=torch.float64, device="cuda")
        lbm.lbm_batch_moments(b, rho=rho)
    finally:
        lbm.lbm_batch_destroy(b)
    steps = {}
    for rest in (False, True):
        bb = lbm.lbm_batch_init(p, cols, rho)
        try:
            if rest:
                lbm.lbm_batch_rest_state(bb)
            lbm.lbm_batch_run(bb, 1e-10, 400000, 100)
            st, res, status = lbm.lbm_batch_results(bb, len(cols))
            assert np.all(res <= 1e-10) and np.all(status == 0)
            steps[rest] = st
        finally:
            lbm.lbm_batch_destroy(bb)
    assert np.all(steps[True] == 100)
    assert np.all(steps[False] >= 500)
