"""Row strips of one grid over several processes, one GPU each (a grid too large for one GPU).

The checkerboard of Sect. 3.3 is cut into bands of rows, one per strip.  Each half-sweep of
a colour updates every strip's own gap sites of that colour; the sites of one colour depend
only on the other colour, so after a half-sweep a strip needs nothing from its neighbours
but their boundary rows.  The driver below therefore runs, per sweep of Algorithm 2:

    colour 0 on every strip -> exchange boundary rows -> colour 1 -> exchange boundary rows
    -> sum the strips' accepted energy changes and acceptance counts -> control step

and every strip applies the same control step to the same totals, so they keep one window,
one slope test and one sweep counter.  The random numbers are drawn from counters of the
whole grid's site indices, so the strips together make exactly the updates of one process
on the whole grid.  Every step of the method runs in the library's kernels (the strip
entry points of mpr.h); this module only moves rows and totals between strips:

* ``LocalComm``: all strips in this process (tests, or several strips on one GPU);
* ``DistComm``: one strip per process over ``torch.distributed`` (NCCL between GPUs: send /
  recv of the boundary rows, all-reduce of the totals; gloo on the CPU).

The compute side of a strip is an object with the methods of ``GpuStrip``.
"""
from __future__ import annotations

import numpy as np

from . import mpr


def partition(H: int, n: int):
    """Own rows [y0, y1) of n strips of an H-row grid, about equal, every strip after the
    first beginning at an odd row (its block then begins one row above, at an even row)."""
    if n < 1 or H < 2 * n:
        raise ValueError("need at least two rows per strip")
    bounds = [0]
    for k in range(1, n):
        b = ((k * H) // n) | 1
        if b <= bounds[-1] + 1:
            b = bounds[-1] + 2
        bounds.append(b)
    bounds.append(H)
    if any(b1 - b0 < 1 for b0, b1 in zip(bounds, bounds[1:])):
        raise ValueError("strips too thin for this many ranks")
    return list(zip(bounds[:-1], bounds[1:]))


def block(y0: int, y1: int, H: int):
    """(row0, Hb): the block of a strip with own rows [y0, y1) -- those rows and one row of
    each neighbouring strip."""
    row0 = y0 - 1 if y0 > 0 else 0
    end = y1 + 1 if y1 < H else H
    return row0, end - row0


class GpuStrip:
    """One strip on this process's GPU: the library's strip context."""

    def __init__(self, z, mask, y0: int, y1: int, H: int, params=None, stream=None):
        import torch
        self.torch = torch
        self.row0, self.Hb = block(y0, y1, H)
        self.H, self.W = H, int(z.shape[1])
        self.z = z[self.row0:self.row0 + self.Hb].contiguous()
        self.mask = mask[self.row0:self.row0 + self.Hb].contiguous()
        self.params = params if params is not None else mpr.mpr_default_params()
        self.stream = stream
        self.own = (y0 - self.row0, y1 - self.row0)
        self.ctx = None
        dev = self.z.device
        self.totals = torch.zeros(2, dtype=torch.float64, device=dev)

    def extremes(self):
        return mpr.mpr_strip_extremes(self.z, self.mask, self.W, self.Hb, self.row0, self.H, self.stream)

    def init(self, zmin: float, zmax: float):
        self.ctx = mpr.mpr_strip_init(self.z, self.mask, self.W, self.Hb, self.row0, self.H, zmin, zmax,
                                      self.params, self.stream)
        n = mpr.mpr_strip_row_bytes(self.ctx)
        dev = self.z.device
        self.out_rows = [self.torch.empty(n, dtype=self.torch.uint8, device=dev) for _ in range(2)]
        self.in_rows = [self.torch.empty(n, dtype=self.torch.uint8, device=dev) for _ in range(2)]

    def pairs(self):
        return mpr.mpr_strip_pairs(self.ctx)

    def temperature(self, e_s: float) -> float:
        return mpr.mpr_strip_temperature(self.ctx, e_s)

    def set_temperature(self, T: float):
        mpr.mpr_set_T(self.ctx, T)

    def energy(self) -> float:
        return mpr.mpr_strip_energy(self.ctx)

    def gaps(self) -> int:
        return mpr.mpr_strip_gaps(self.ctx)

    def begin(self, phase: int, H_total: float = 0.0, P_total: float = 0.0):
        mpr.mpr_strip_begin(self.ctx, phase, H_total, P_total)

    def half_sweep(self, color: int, phase: int):
        mpr.mpr_strip_half_sweep(self.ctx, color, phase, self.totals)

    def partials(self):
        return self.totals

    def vec(self, values):
        """Host values as a vector of the totals' kind (for the reductions across strips)."""
        return self.totals.new_tensor([float(v) for v in values])

    def control(self, totals, phase: int) -> bool:
        return mpr.mpr_strip_control(self.ctx, totals, phase, want_stop=phase == 0)

    def first_row(self):
        mpr.mpr_strip_row(self.ctx, 0, self.out_rows[0])
        return self.out_rows[0]

    def last_row(self):
        mpr.mpr_strip_row(self.ctx, 1, self.out_rows[1])
        return self.out_rows[1]

    def recv_buffers(self):
        return self.in_rows

    def set_above(self, buf):
        mpr.mpr_strip_row(self.ctx, 2, buf)

    def set_below(self, buf):
        mpr.mpr_strip_row(self.ctx, 3, buf)

    def predict(self, M: int):
        out = self.torch.empty_like(self.z)
        mpr.mpr_strip_predict(self.ctx, M, out)
        return out[self.own[0]:self.own[1]]

    def state(self):
        phi = self.torch.empty_like(self.z)
        mpr.mpr_get_state(self.ctx, phi)
        return phi[self.own[0]:self.own[1]]

    def close(self):
        if self.ctx is not None:
            mpr.mpr_free(self.ctx)
            self.ctx = None


class LocalComm:
    """Every strip of the grid in this process: rows are copied between neighbouring strips,
    totals added in strip order."""

    def __init__(self, strips):
        self.strips = strips

    def sum(self, values):
        t = values[0].clone() if hasattr(values[0], "clone") else values[0].copy()
        for v in values[1:]:
            t += v
        return t

    def min(self, values):
        return min(values)

    def max(self, values):
        return max(values)

    def exchange(self):
        s = self.strips
        for k in range(len(s) - 1):
            s[k + 1].set_above(s[k].last_row())
            s[k].set_below(s[k + 1].first_row())


class DistComm:
    """One strip per process over torch.distributed (rank k owns strip k of world_size)."""

    def __init__(self, strip, dist):
        self.strips = [strip]
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def _reduce(self, values, op):
        import torch
        v = values[0]
        t = v.clone() if isinstance(v, torch.Tensor) else torch.as_tensor(np.asarray(v, dtype=np.float64)).clone()
        if self.dist.get_backend() == "nccl" and not t.is_cuda:
            t = t.cuda()
        self.dist.all_reduce(t, op=op)
        if isinstance(v, torch.Tensor):
            return t
        return float(t) if np.ndim(v) == 0 else t.cpu().numpy()

    def sum(self, values):
        return self._reduce(values, self.dist.ReduceOp.SUM)

    def min(self, values):
        return self._reduce(values, self.dist.ReduceOp.MIN)

    def max(self, values):
        return self._reduce(values, self.dist.ReduceOp.MAX)

    def exchange(self):
        s = self.strips[0]
        below, above = s.recv_buffers()
        reqs = []
        if self.rank > 0:
            reqs.append(self.dist.isend(s.first_row(), self.rank - 1))
            reqs.append(self.dist.irecv(above, self.rank - 1))
        if self.rank + 1 < self.world:
            reqs.append(self.dist.isend(s.last_row(), self.rank + 1))
            reqs.append(self.dist.irecv(below, self.rank + 1))
        for r in reqs:
            r.wait()
        if self.rank > 0:
            s.set_above(above)
        if self.rank + 1 < self.world:
            s.set_below(below)


def fill(comm, M: int, T: float | None = None, relax: bool = True):
    """Algorithm 2 on a grid cut into the strips of ``comm``: Eq. 1 with the whole grid's
    extremes, T-hat from the whole grid's e_s (Eq. 4; or the given T), the relaxation of
    step 5 (unless relax is False), M equilibrium sweeps and the estimates.  Returns, per
    local strip, its own rows' estimates, and the relaxation's sweep count."""
    strips = comm.strips
    ex = [s.extremes() for s in strips]
    zmin = comm.min([e[0] for e in ex])
    zmax = comm.max([e[1] for e in ex])
    for s in strips:
        s.init(zmin, zmax)
    comm.exchange()
    if T is None:
        pc = comm.sum([s.vec(s.pairs()) for s in strips])
        sc, n = float(pc[0]), float(pc[1])
        if n == 0:
            raise mpr.MprError(mpr.MPR_ENOPAIRS, "no nearest-neighbour sample pairs")
        for s in strips:
            T = s.temperature(-sc / n)
    else:
        for s in strips:
            s.set_temperature(T)
    sweeps = 0
    if relax:
        HP = comm.sum([s.vec((s.energy(), float(s.gaps()))) for s in strips])
        for s in strips:
            s.begin(0, float(HP[0]), float(HP[1]))
        stop = False
        while not stop:
            _sweep(comm, 0)
            tot = comm.sum([s.partials() for s in strips])
            stops = [s.control(tot, 0) for s in strips]
            stop = stops[0]
            sweeps += 1
    P = comm.sum([s.vec((0.0, float(s.gaps()))) for s in strips])
    for s in strips:
        s.begin(1, 0.0, float(P[1]))
    for _ in range(M):
        _sweep(comm, 1)
        tot = comm.sum([s.partials() for s in strips])
        for s in strips:
            s.control(tot, 1)
    return [s.predict(M) for s in strips], sweeps


def _sweep(comm, phase):
    for color in (0, 1):
        for s in comm.strips:
            s.half_sweep(color, phase)
        comm.exchange()


__all__ = ["partition", "block", "GpuStrip", "LocalComm", "DistComm", "fill"]
