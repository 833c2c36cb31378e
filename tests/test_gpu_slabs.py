"""Slabs of one domain (lbm_slab_*) on one GPU against the single-domain step.

The ranks of the multi-GPU path are host threads of one process here, each driving its
own ``partition.SlabLattice``; a thread comm hands the ghost rows and the mass sums from
thread to thread with a barrier (host-side tensor copies on the one CUDA stream the
threads share, ordered by the barrier - no kernel waits on another). After K steps the
slabs' own rows must equal lbm_step on the whole domain: bit for bit up to the summation
order of <rho> (Eq. Gravity_2), so 1e-13 in FP64 and the FP32 bound 1e-6 in FP32.
"""
import os
import threading

import numpy as np
import pytest

from paper_2301_12869_gb300 import _build, inputs, lbm, partition

pytestmark = pytest.mark.gpu

A, B, R = 0.25, 4.0, 1.0
W = inputs.LATTICE_WEIGHTS


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


class ThreadComm:
    """The comm of partition.exchange_halos / SlabLattice for ranks that are threads."""

    def __init__(self, world):
        self.world = world
        self.box = {}
        self.barrier = threading.Barrier(world, timeout=120)

    def rank_view(self, rank):
        import torch

        comm = self

        class View:
            def exchange(self, sends, recvs=None):
                for peer, t in sends.items():
                    comm.box[(rank, peer)] = t.clone()
                comm.barrier.wait()
                out = {peer: comm.box[(peer, rank)] for peer in sends}
                comm.barrier.wait()
                if recvs is not None:
                    for peer in out:
                        recvs[peer].copy_(out[peer])
                    return recvs
                return out

            def sum_(self, t):
                return self._reduce(t, lambda a, b: a + b)

            def max_(self, t):
                return self._reduce(t, torch.maximum)

            def _reduce(self, t, op):
                comm.box[("red", rank)] = t.clone()
                comm.barrier.wait()
                total = comm.box[("red", 0)].clone()
                for r in range(1, comm.world):
                    total = op(total, comm.box[("red", r)])
                comm.barrier.wait()
                t.copy_(total)
                return t

        return View()


def run_slabs(p, rho0, world, steps):
    import torch

    plan = partition.SlabPlan(p.ny, world)
    comm = ThreadComm(world)
    out, errors = {}, []

    def rank_main(r):
        try:
            sl = plan[r]
            rho_own = torch.from_numpy(np.ascontiguousarray(rho0[sl.y0:sl.y0 + sl.ny_own])).cuda()
            lat = partition.SlabLattice(p, sl, rho_own, comm.rank_view(r))
            lat.step(steps)
            torch.cuda.synchronize()
            out[r] = (partition.own_rows(lat.state, sl).double().cpu().numpy(), lat.status_code())
        except Exception as exc:  # noqa: BLE001 - re-raised in the main thread
            errors.append(exc)
            comm.barrier.abort()

    threads = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    if errors:
        raise errors[0]
    assert all(out[r][1] == lbm.LBM_OK for r in range(world))
    return plan.gather([out[r][0] for r in range(world)])


@pytest.mark.parametrize("precision, nx, ny, world, form, wall, tol", [
    ("fp64", 64, 48, 2, 2, lbm.LBM_WALL_BOUNCE_BACK, 1e-13),
    ("fp64", 64, 47, 3, 2, lbm.LBM_WALL_ZOU_HE, 1e-13),
    ("fp64", 32, 9, 3, 1, lbm.LBM_WALL_BOUNCE_BACK, 1e-13),   # 3-row slabs
    ("fp32", 1028, 300, 2, 2, lbm.LBM_WALL_BOUNCE_BACK, 1e-6),  # two x bands, a ragged one
    ("fp32", 512, 203, 4, 1, lbm.LBM_WALL_ZOU_HE, 1e-6),
])
def test_slabs_equal_the_single_domain(precision, nx, ny, world, form, wall, tol):
    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    T = 0.8 * Tc
    rv, rl, _ = lbm.lbm_coexistence(A, B, R, T)
    rho0 = inputs.column_rho0(nx, ny, rl, rv, ny // 2, noise_amp=1e-3)
    rho_ref = 0.0 if precision == "fp64" else float(rho0.mean())
    p = lbm.make_params(nx, ny, T, precision, a=A, b=B, R=R, form=form, g=(1e-6, -1e-4), rho_ref=rho_ref, wall=wall)
    steps = 40
    got = run_slabs(p, rho0, world, steps)
    h = lbm.lbm_init(p, rho0)
    try:
        lbm.lbm_step(h, steps)
        f = np.empty((9, ny, nx))
        lbm.lbm_get_state(h, f)
    finally:
        lbm.lbm_destroy(h)
    want = f - W[:, None, None] * rho_ref
    assert np.max(np.abs(got - want)) <= tol


def test_slab_arguments_are_checked():
    import torch

    p = lbm.make_params(16, 10, 0.02, "fp64", a=A)
    with pytest.raises(lbm.LbmError, match="outside"):
        lbm.lbm_slab_partials(p, lbm.make_slab(8, 4))
    with pytest.raises(lbm.LbmError, match="at least 2 rows"):
        lbm.lbm_slab_partials(p, lbm.make_slab(0, 1))
    s = lbm.make_slab(0, 5)
    f = torch.zeros((9, 9, 16), dtype=torch.float64, device="cuda")
    part = torch.zeros(lbm.lbm_slab_partials(p, s), dtype=torch.float64, device="cuda")
    part2 = torch.zeros_like(part)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(lbm.LbmError, match="distinct"):
        lbm.lbm_slab_step(p, s, f, f, part, part2, st)
    with pytest.raises(lbm.LbmError, match="distinct"):
        lbm.lbm_slab_step(p, s, f, torch.zeros_like(f), part, part, st)
    with pytest.raises(ValueError, match="CUDA"):
        lbm.lbm_slab_step(p, s, f.cpu(), f, part, part2, st)
    with pytest.raises(lbm.LbmError, match="part_out holds"):  # fewer partial slots than CTAs
        lbm.lbm_slab_step(p, s, f, torch.zeros_like(f), part, part2[:1], st)
    off = torch.zeros(f.numel() + 1, dtype=torch.float64, device="cuda")[1:]  # 8 bytes past a boundary
    with pytest.raises(lbm.LbmError, match="16-byte"):  # refused on the host: nothing is launched
        lbm.lbm_slab_step(p, s, off, torch.zeros_like(f), part, part2, st)


@pytest.mark.parametrize("precision, nx, ny", [("fp32", 1024, 4096), ("fp64", 1024, 4096), ("fp32", 64, 40)])
def test_whole_domain_slab_plans_like_a_handle(precision, nx, ny):
    """One slab over the whole domain, asked first in a fresh plan: as many CTAs (= partial
    sums) as the handle's grid for the same lattice - the plan is made after the step
    kernels' shared-memory limit is set (their occupancy depends on it)."""
    p = lbm.make_params(nx, ny, 0.02, precision, a=A)
    n = lbm.lbm_slab_partials(p, lbm.make_slab(0, ny))
    h = lbm.lbm_init(p, np.full((ny, nx), 0.1))
    try:
        assert n == lbm.lbm_launch_info(h)["grid"]
    finally:
        lbm.lbm_destroy(h)
