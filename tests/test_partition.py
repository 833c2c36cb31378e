"""The multi-GPU partitions on CPU: gloo ranks on 127.0.0.1, the oracle as each rank's step.

* Columns: every rank runs its share (``partition.column_shares``) of a column set; the
  gathered states equal a single-process run of all columns bit for bit (the columns are
  independent, so no data crosses ranks).
* Slabs of one domain: every rank holds its rows plus HALO ghost rows on each side,
  steps them with the oracle using the mean density summed over all ranks (Eq. Gravity_2)
  and refreshes its ghost rows by ``partition.exchange_halos``; after K steps the gathered
  domain equals the single-domain oracle to 1e-14 (summation order of the mean only).
  This checks the exchange plan (which rows go where, HALO deep) and the global mean.
"""
import os
import socket
import sys

import numpy as np
import pytest

from oracle import eos
from oracle import lbm as olbm
from paper_2301_12869_gb300 import inputs, partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
A = 0.25
RHO_C, T_C, _ = eos.critical_point(A, 4.0, 1.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_column_shares_cover_and_balance():
    rng = np.random.default_rng(3)
    heights = rng.choice([64, 128, 256, 512, 1024], size=4096)
    for world in (1, 2, 3, 8):
        shares = partition.column_shares(heights, world)
        allc = np.concatenate(shares)
        assert np.array_equal(np.sort(allc), np.arange(heights.size))
        load = np.array([heights[s].sum() for s in shares])
        assert load.max() - load.min() <= heights.max()


def test_slab_plan_rows_and_neighbours():
    for ny, world in ((4096, 8), (23, 3), (4, 2), (17, 1)):
        plan = partition.SlabPlan(ny, world)
        assert sum(s.ny_own for s in plan.slabs) == ny
        assert plan[0].y0 == 0 and plan[0].wall_below and plan[world - 1].wall_above
        for a, b in zip(plan.slabs, plan.slabs[1:]):
            assert b.y0 == a.y0 + a.ny_own and a.upper == b.rank and b.lower == a.rank
        assert min(s.ny_own for s in plan.slabs) >= partition.HALO
    with pytest.raises(ValueError):
        partition.SlabPlan(3, 2)


def _domain(nx, ny, form, wall):
    rv, rl, _ = eos.maxwell(0.8 * T_C, A, 4.0, 1.0)
    rho0 = inputs.column_rho0(nx, ny, rl, rv, ny // 2, width=3.0, noise_amp=1e-3, seed=5)
    p = olbm.Params(nx=nx, ny=ny, a=A, T=0.8 * T_C, g=(1e-6, -1e-4), form=form, wall=wall)
    return olbm.init_state(rho0), p


def _slab_rank(rank, world, port, q, nx, ny, steps, form, wall):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import dataclasses

    import torch
    import torch.distributed as dist

    from oracle import lbm as olbm_
    from paper_2301_12869_gb300 import partition as part

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = part.TorchComm(dist)
        f0, p = _domain(nx, ny, form, wall)
        plan = part.SlabPlan(ny, world)
        sl = plan[rank]
        buf = torch.zeros((9, sl.rows, nx), dtype=torch.float64)
        part.own_rows(buf, sl)[:] = torch.from_numpy(f0[:, sl.y0:sl.y0 + sl.ny_own])
        part.exchange_halos(buf, sl, comm)
        a = part.HALO if sl.wall_below else 0
        b = part.HALO + sl.ny_own if sl.wall_above else sl.rows
        sub_p = dataclasses.replace(p, ny=b - a)
        for _ in range(steps):
            # <rho> of Eq. Gravity_2 over the whole domain: each rank's own stored mass, summed
            mass = part.own_rows(buf, sl).sum().reshape(1).clone()
            comm.sum_(mass)
            new = olbm_.step(buf[:, a:b].numpy(), sub_p, mean_rho=float(mass[0]) / (nx * ny))
            part.own_rows(buf, sl)[:] = torch.from_numpy(new[:, part.HALO - a:part.HALO - a + sl.ny_own])
            part.exchange_halos(buf, sl, comm)
        q.put((rank, part.own_rows(buf, sl).numpy().copy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world, ny, form, wall", [
    (2, 24, 2, "bounce-back"),
    (2, 24, 1, "zou-he"),
    (3, 17, 2, "zou-he"),     # uneven slabs, one of them interior
    (3, 9, 2, "bounce-back"),  # the thinnest slabs: 3 rows each
])
def test_slabs_with_halo_exchange_equal_the_single_domain(world, ny, form, wall):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    nx, steps = 8, 12
    procs = [ctx.Process(target=_slab_rank, args=(r, world, port, q, nx, ny, steps, form, wall))
             for r in range(world)]
    for pr in procs:
        pr.start()
    parts = dict(q.get(timeout=300) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    got = partition.SlabPlan(ny, world).gather([parts[r] for r in range(world)])
    f0, p = _domain(nx, ny, form, wall)
    want = olbm.run(f0, p, steps)
    assert np.max(np.abs(got - want)) <= 1e-14


def _column_rank(rank, world, port, q, ncols):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2301_12869_gb300 import partition as part

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cols = _columns(ncols)
        share = part.column_shares([c[1].ny for c in cols], world)[rank]
        q.put((rank, {int(c): olbm.run(cols[c][0], cols[c][1], 20) for c in share}))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _columns(n):
    out = []
    for c, gen in enumerate(inputs.batched_columns(n, seed=11)):
        ny = gen["ny"] // 16  # heights 4..64: the same mix, small enough for the oracle
        T = gen["Tr"] * T_C
        rv, rl, _ = eos.maxwell(T, A, 4.0, 1.0)
        rho0 = inputs.column_rho0(4, ny, rl, rv, max(1, int(round(gen["liquid_fraction"] * ny))), width=3.0)
        out.append((olbm.init_state(rho0), olbm.Params(nx=4, ny=ny, a=A, T=T, g=(0.0, gen["gy"]), form=gen["form"])))
    return out


def test_column_partition_over_two_ranks_equals_one_process():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_column_rank, args=(r, 2, port, q, 12)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = {}
    shares = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for _, d in shares:
        assert not set(d) & set(got)  # disjoint
        got.update(d)
    cols = _columns(12)
    assert sorted(got) == list(range(12))
    for c, (f0, p) in enumerate(cols):
        assert np.array_equal(got[c], olbm.run(f0, p, 20))
