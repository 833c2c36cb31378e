"""Work partitions across GPUs (one process per GPU) for the two workloads that shard.

* Independent columns (the batched liquid columns of Sec. IV): disjoint column sets, no
  exchange at all. ``column_shares`` balances the ranks by lattice nodes (a column's
  cost per step is proportional to its nodes, 4 H), longest first onto the least loaded
  rank.
* One large domain: horizontal slabs of rows. A step of Eq. LBE pulls from the rows one
  link below and above, and the Shan-Chen force (Eq. ShanChenForce) needs psi of the rows
  next to a node, so a slab's first row depends on the post-collision populations of the
  two rows below it, and its last row on the two rows above. Each slab therefore keeps
  HALO = 2 ghost rows on each side, refreshed from its neighbours after every step, and
  Eq. Gravity_2 needs the mean density of the whole domain: one sum over all ranks per
  step (``SlabPlan`` and ``exchange_halos``).

Host logic only: which rows and columns live where and which rows travel to which rank.
The arithmetic of a step stays in the library's kernels (or, in tests, in the oracle).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

HALO = 2  # ghost rows per side of a slab


def column_shares(heights, world):
    """Per rank, the sorted indices of its columns: a disjoint cover of range(len(heights))
    balanced by nodes (greedy longest-processing-time on the heights)."""
    heights = np.asarray(heights, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    load = np.zeros(world, dtype=np.int64)
    shares = [[] for _ in range(world)]
    for c in np.argsort(-heights, kind="stable"):
        r = int(np.argmin(load))
        shares[r].append(int(c))
        load[r] += int(heights[c])
    return [np.array(sorted(s), dtype=np.int64) for s in shares]


@dataclass(frozen=True)
class Slab:
    """Rows [y0, y0 + ny_own) of an ny_total-row domain, stored with HALO ghost rows below
    and above: buffer row j holds domain row y0 - HALO + j. lower / upper: the neighbour
    ranks (None at a wall)."""

    rank: int
    y0: int
    ny_own: int
    ny_total: int
    lower: int | None
    upper: int | None

    @property
    def rows(self):
        """Buffer rows (own rows plus both halos)."""
        return self.ny_own + 2 * HALO

    @property
    def wall_below(self):
        return self.lower is None

    @property
    def wall_above(self):
        return self.upper is None


class SlabPlan:
    """Rows of an ny_total-row domain split into `world` slabs of near-equal height
    (at least HALO rows each, so that a slab's halo comes from its direct neighbour)."""

    def __init__(self, ny_total, world):
        if world < 1:
            raise ValueError("world must be >= 1")
        if ny_total < HALO * world:
            raise ValueError(f"{ny_total} rows cannot give {world} slabs of at least {HALO} rows")
        base, extra = divmod(ny_total, world)
        self.ny_total = ny_total
        self.world = world
        self.slabs = []
        y = 0
        for r in range(world):
            n = base + (1 if r < extra else 0)
            self.slabs.append(Slab(rank=r, y0=y, ny_own=n, ny_total=ny_total,
                                   lower=r - 1 if r > 0 else None, upper=r + 1 if r + 1 < world else None))
            y += n

    def __getitem__(self, rank):
        return self.slabs[rank]

    def gather(self, parts):
        """The whole domain [..., ny_total, nx] from every rank's own rows (arrays shaped
        [..., ny_own, nx], in rank order)."""
        return np.concatenate(parts, axis=-2)


def own_rows(buf, slab):
    """View of a slab buffer [..., rows, nx] restricted to its own rows."""
    return buf[..., HALO:HALO + slab.ny_own, :]


def exchange_halos(buf, slab, comm, bufs=None):
    """Refresh the ghost rows of a slab buffer (torch tensor [9, rows, nx] holding the
    post-collision populations of the last step) from the neighbours: the lowest HALO own
    rows go to the lower neighbour's upper halo, the highest HALO own rows to the upper
    neighbour's lower halo, and the halos are filled from what the neighbours send.
    comm.exchange(sends, recvs), sends = {peer: contiguous tensor}, returns {peer: tensor} of
    the same shapes (into recvs when given). bufs: optional preallocated
    {("send" | "recv", peer): tensor [9, HALO, nx]}. A slab at a wall leaves that halo
    untouched (the step applies the wall)."""
    sends, recvs = {}, None
    edges = []
    if slab.lower is not None:
        edges.append((slab.lower, HALO))
    if slab.upper is not None:
        edges.append((slab.upper, slab.ny_own))
    for peer, row in edges:
        if bufs is None:
            sends[peer] = buf[:, row:row + HALO, :].contiguous()
        else:
            sends[peer] = bufs[("send", peer)]
            sends[peer].copy_(buf[:, row:row + HALO, :])
    if bufs is not None:
        recvs = {peer: bufs[("recv", peer)] for peer, _ in edges}
    recv = comm.exchange(sends, recvs) if recvs is not None else comm.exchange(sends)
    if slab.lower is not None:
        buf[:, 0:HALO, :] = recv[slab.lower]
    if slab.upper is not None:
        top = HALO + slab.ny_own
        buf[:, top:top + HALO, :] = recv[slab.upper]
    return buf


class TorchComm:
    """Point-to-point row exchange and scalar sums over torch.distributed (NCCL between GPUs,
    gloo on CPU): sends and receives of one exchange are posted together
    (batch_isend_irecv), so neighbours cannot deadlock on their order."""

    def __init__(self, dist):
        self.dist = dist

    def exchange(self, sends, recvs=None):
        import torch

        dist = self.dist
        if recvs is None:
            recvs = {peer: torch.empty_like(t) for peer, t in sends.items()}
        ops = []
        for peer, t in sends.items():
            ops.append(dist.P2POp(dist.isend, t, peer))
            ops.append(dist.P2POp(dist.irecv, recvs[peer], peer))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        return recvs

    def sum_(self, t):
        """In-place element-wise sum of a tensor over all ranks."""
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t

    def max_(self, t):
        """In-place element-wise max of a tensor over all ranks."""
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t


class SlabLattice:
    """One rank's slab of a domain on the current GPU. Buffers are torch CUDA tensors, every
    step is the library's slab step (lbm_slab_step) on torch's current stream, and `comm`
    carries the two exchanges a step needs: the domain's mass (the slabs' FP64 partials,
    added element-wise over ranks, for Eq. Gravity_2) and the ghost rows
    (``exchange_halos``). The partials vectors have the largest rank's length (a max over
    ranks at set-up), zero beyond a rank's own count.

    params: lbm_params of the whole domain (p.ny = all rows; p.rho_ref the same on every
    rank); slab: this rank's ``Slab``; rho0_own: its rows of the initial density, a torch
    CUDA tensor [ny_own, nx] of float64."""

    def __init__(self, params, slab, rho0_own, comm):
        import torch

        from . import lbm

        self._lbm, self._torch = lbm, torch
        self.p, self.slab, self.comm = params, slab, comm
        self.s = lbm.make_slab(slab.y0, slab.ny_own)
        dtype = torch.float32 if params.precision == lbm.LBM_FP32 else torch.float64
        self.f = [torch.zeros((9, slab.rows, params.nx), dtype=dtype, device="cuda") for _ in range(2)]
        self.cur = 0
        count = torch.tensor([float(lbm.lbm_slab_partials(params, self.s))], dtype=torch.float64, device="cuda")
        comm.max_(count)
        npart = int(count.item())
        self.part = [torch.zeros(npart, dtype=torch.float64, device="cuda") for _ in range(2)]
        self.status = torch.zeros(1, dtype=torch.int32, device="cuda")
        stream = self._stream()
        lbm.lbm_slab_init(params, self.s, rho0_own.contiguous(), self.f[0], stream)
        lbm.lbm_slab_mass(params, self.s, self.f[0], self.part[0], stream)
        # ghost-row exchange buffers, allocated once
        self.bufs = {}
        for peer in (slab.lower, slab.upper):
            if peer is not None:
                for kind in ("send", "recv"):
                    self.bufs[(kind, peer)] = torch.empty((9, HALO, params.nx), dtype=dtype, device="cuda")
        comm.sum_(self.part[0])
        exchange_halos(self.f[0], slab, comm, self.bufs)
        self.steps = 0
        # the step's library call with its arguments marshalled once (the buffers never move)
        import ctypes

        lib = lbm.load()
        self._call = lib.lbm_slab_step
        self._pp, self._sp = ctypes.byref(params), ctypes.byref(self.s)
        self._ptr = {"f": [t.data_ptr() for t in self.f], "part": [t.data_ptr() for t in self.part], "npart": npart,
                     "status": self.status.data_ptr()}

    def _stream(self):
        return self._torch.cuda.current_stream().cuda_stream

    @property
    def state(self):
        """The current buffer [9, rows, nx] (deviations f_i - w_i rho_ref)."""
        return self.f[self.cur]

    def step(self, n=1):
        lbm, stream = self._lbm, self._stream()
        pf, pp, npart = self._ptr["f"], self._ptr["part"], self._ptr["npart"]
        for _ in range(n):
            c = self.cur
            rc = self._call(self._pp, self._sp, pf[c], pf[1 - c], pp[c], npart, pp[1 - c], npart, self._ptr["status"],
                            stream)
            if rc != lbm.LBM_OK:
                lbm._check(rc)
            self.cur ^= 1
            self.comm.sum_(self.part[self.cur])
            exchange_halos(self.f[self.cur], self.slab, self.comm, self.bufs)
            self.steps += 1

    @property
    def mass(self):
        """sum(rho - rho_ref) over the whole domain of the current state (host float; the
        partials are copied back and added on the host in index order)."""
        return float(np.sum(self.part[self.cur].cpu().numpy()))

    def snapshot(self):
        return self.state.clone(), self.part[self.cur].clone()

    def restore(self, snap):
        f, m = snap
        self.state.copy_(f)
        self.part[self.cur].copy_(m)

    def status_code(self):
        """LBM_OK, or LBM_ENONPHYS / LBM_ETIMEOUT from the status bits of this rank's steps."""
        st = int(self.status.item())
        if st & 2:
            return self._lbm.LBM_ETIMEOUT
        if st & 1:
            return self._lbm.LBM_ENONPHYS
        return self._lbm.LBM_OK


class SingleComm:
    """The comm of a single rank (one slab = the whole domain): nothing to exchange."""

    def exchange(self, sends, recvs=None):
        if sends:
            raise ValueError("a single rank has no neighbours")
        return {}

    def sum_(self, t):
        return t

    def max_(self, t):
        return t
