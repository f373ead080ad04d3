"""Row-strip domain decomposition of one simulation over several ranks.

The paper runs one simulation per GPU (Sect. 3.2).  A domain larger than one
GPU's memory is split here into strips of whole rows, one per rank.  Each
rank's simulation covers its own rows plus ``o`` rows of overlap on each
side that meets another strip (its window), with that window's slice of the
DEM, release and boundary inflow.  Every step:

1. each rank steps its whole window (the CFL step of Sect. 2.2, from the
   agreed maximum wave speed);
2. each rank sends its first ``o`` own rows to the rank below and its last
   ``o`` own rows to the rank above, and receives theirs into its overlap;
3. the ranks agree on the largest wave speed of their own rows (a max
   all-reduce of one double), which sets the next step's time step.

A stage reads the state and the bed geometry up to two cells away (the
minmod slopes of a face's two cells, each from its two neighbours).  The
geometry of a window's last row comes from a bed extrapolated past the
window and differs from the undecomposed one, so with o = 2 x (stages per
step) + 1 every value an own cell's step reads is exact.  The own rows
therefore evolve bit for bit as in the undecomposed run, and the maximum
over all own rows is the undecomposed one (the speeds of the overlap do not
count: its last row sees the extrapolated bed).  Cells of the overlap that
are farther from the own rows go wrong during the step and are overwritten
at its end.

The window's sides inside the domain get the transmissive rule (their
values do not matter); the others keep the domain's boundary conditions.
An inflow segment on the west or east side must not be cut by a window
edge, since its ghost state depends on its full width.

Engines: ``GpuStrip`` runs a strip on this process's GPU through the C-ABI
(``moses_set_owned_rows``, ``moses_get_rows_device``,
``moses_set_rows_device``, ``moses_set_max_speed``).  Anything with the same
methods can stand in (the tests use the FP64 oracle on CPU ranks).
Communicators: ``TorchComm`` over ``torch.distributed`` (NCCL for CUDA
tensors, gloo for CPU tensors), ``LocalComm`` for all strips in one
process.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def overlap_rows(params: dict) -> int:
    """Rows of overlap a strip needs on each inner side: two per stage of
    the step (the stencil's reach) and the window's last row, whose bed
    geometry is not the undecomposed one."""
    stages = 3 if int(params.get("rk", 2)) == 3 else 2
    return 2 * stages + 1


@dataclass(frozen=True)
class StripPlan:
    rank: int
    world: int
    ny: int
    own0: int  # own rows [own0, own1) of the domain
    own1: int
    win0: int  # window rows [win0, win1) of the domain
    win1: int
    o: int

    @property
    def own_local(self):
        """Own rows in the window's numbering."""
        return self.own0 - self.win0, self.own1 - self.win0


def plan(ny: int, world: int, o: int) -> list[StripPlan]:
    """Rows as even as possible over `world` strips; each strip must own at
    least `o` rows (so that one neighbour owns the whole overlap)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(ny, world)
    if world > 1 and base < o:
        raise ValueError(f"{ny} rows over {world} strips leaves fewer than {o} rows for a strip")
    out, j = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        own0, own1 = j, j + n
        j = own1
        win0 = own0 - o if r > 0 else 0
        win1 = own1 + o if r < world - 1 else ny
        out.append(StripPlan(r, world, ny, own0, own1, win0, win1, o))
    return out


def strip_config(cfg: dict, p: StripPlan) -> dict:
    """The workload dict of one strip's window (DEM, release and velocities
    sliced; inner sides transmissive; the inflow where the window holds it)."""
    rows = slice(p.win0, p.win1)
    out = dict(cfg)
    for k in ("dem", "h", "phi_s", "vx_s", "vy_s", "vx_f", "vy_f"):
        if cfg.get(k) is not None:
            out[k] = np.ascontiguousarray(np.asarray(cfg[k], dtype=np.float64)[rows])
    bc = list(cfg["params"]["bc"])
    if p.win0 > 0:
        bc[2] = 1
    if p.win1 < p.ny:
        bc[3] = 1
    out["params"] = dict(cfg["params"], bc=tuple(bc))
    out["inflow"] = None
    f = cfg.get("inflow")
    if f:
        side = f["side"]
        if side == 2 and p.win0 == 0 or side == 3 and p.win1 == p.ny:
            out["inflow"] = f
        elif side in (0, 1) and f["i0"] < p.win1 and p.win0 < f["i1"]:
            if not (p.win0 <= f["i0"] and f["i1"] <= p.win1):
                raise ValueError("an inflow segment crosses a strip window's edge: choose another split")
            out["inflow"] = dict(f, i0=f["i0"] - p.win0, i1=f["i1"] - p.win0)
    return out


class GpuStrip:
    """One strip on this process's GPU (moses.Sim through the C-ABI)."""

    def __init__(self, cfg: dict, p: StripPlan, precision=None, stream=None):
        import torch

        from . import moses
        self.p = p
        self.sim = moses.from_config(strip_config(cfg, p), precision=moses.FP64 if precision is None else precision,
                                     stream=stream)
        self.sim.set_owned_rows(*p.own_local)
        self._torch = torch

    def get_rows(self, j0: int, n: int):
        t = self._torch.empty((self.sim.row_planes, n, self.sim.nx), dtype=self._torch.float64, device="cuda")
        self.sim.get_rows_device(j0, n, t.data_ptr())
        return t

    def set_rows(self, j0: int, n: int, rows):
        assert rows.is_cuda and rows.dtype == self._torch.float64 and rows.is_contiguous()
        self.sim.set_rows_device(j0, n, rows.data_ptr())

    def step(self):
        self.sim.step(1)

    def max_speed(self) -> float:
        return self.sim.max_speed()

    def set_max_speed(self, amax: float):
        self.sim.set_max_speed(amax)

    def own_state(self) -> np.ndarray:
        a, b = self.p.own_local
        return self.sim.get_conserved()[:, a:b]

    def budget(self) -> dict:
        return self.sim.budget()


class LocalComm:
    """Every strip in this process: the exchange is a copy, the maximum a max."""

    def __init__(self, strips):
        self.strips = list(strips)

    def run(self, nsteps: int):
        agree_max(self.strips, max(s.max_speed() for s in self.strips))
        for _ in range(nsteps):
            for s in self.strips:
                s.step()
            sends = [outgoing(s) for s in self.strips]
            for r, s in enumerate(self.strips):
                lo = sends[r - 1]["hi"] if r > 0 else None
                hi = sends[r + 1]["lo"] if r + 1 < len(self.strips) else None
                incoming(s, lo, hi)
            agree_max(self.strips, max(s.max_speed() for s in self.strips))


class TorchComm:
    """One strip per rank of a torch.distributed process group; row buffers
    and the maximum live on `device` (cuda for NCCL, cpu for gloo)."""

    def __init__(self, strip, device="cuda", group=None):
        import torch
        import torch.distributed as dist
        self.s, self.dev, self.group = strip, device, group
        self.torch, self.dist = torch, dist

    def _max(self, v: float) -> float:
        t = self.torch.tensor([v], dtype=self.torch.float64, device=self.dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def _exchange(self):
        s, dist = self.s, self.dist
        r, w = s.p.rank, s.p.world
        send = outgoing(s)
        shape = lambda t: (t.shape[0], s.p.o, t.shape[2])  # noqa: E731
        ref = send["lo"] if send["lo"] is not None else send["hi"]
        recv_lo = self.torch.empty(shape(ref), dtype=ref.dtype, device=ref.device) if r > 0 else None
        recv_hi = self.torch.empty(shape(ref), dtype=ref.dtype, device=ref.device) if r + 1 < w else None
        ops = []
        if r > 0:
            ops += [dist.P2POp(dist.isend, send["lo"], r - 1, self.group), dist.P2POp(dist.irecv, recv_lo, r - 1, self.group)]
        if r + 1 < w:
            ops += [dist.P2POp(dist.isend, send["hi"], r + 1, self.group), dist.P2POp(dist.irecv, recv_hi, r + 1, self.group)]
        if ops:
            for q in dist.batch_isend_irecv(ops):
                q.wait()
        incoming(s, recv_lo, recv_hi)

    def run(self, nsteps: int):
        self.s.set_max_speed(self._max(self.s.max_speed()))
        for _ in range(nsteps):
            self.s.step()
            self._exchange()
            self.s.set_max_speed(self._max(self.s.max_speed()))


def outgoing(s) -> dict:
    """The rows a strip sends: its first o own rows down, its last o own rows up."""
    a, b = s.p.own_local
    o = s.p.o
    return {"lo": s.get_rows(a, o) if s.p.rank > 0 else None,
            "hi": s.get_rows(b - o, o) if s.p.rank + 1 < s.p.world else None}


def incoming(s, lo, hi):
    """The neighbours' own rows into this strip's overlap below and above."""
    a, b = s.p.own_local
    o = s.p.o
    if lo is not None:
        s.set_rows(a - o, o, lo)
    if hi is not None:
        s.set_rows(b, o, hi)


def agree_max(strips, amax: float):
    for s in strips:
        s.set_max_speed(amax)
