"""Sharding over several ranks: row slabs of one grid, and independent grids.

The paper gives each processing element one tile with a halo (Sec. IV-A) and
swaps halos between neighbours before every step (Sec. IV-B to IV-D).  Here
each rank owns a band of full-width rows and keeps ``G = radius * S`` ghost
rows above and below it; ranks swap those rows once every ``S`` steps (one
temporal block) and advance ``S`` steps in between with the CUDA library's
``stencil_slab_step``.  The slab geometry comes from the C ABI
(``stencil_slab_geometry`` / ``stencil_slab_create``); this module only moves
rows between ranks and marshals arguments.

Communication: one point-to-point send and receive per neighbour and block
(``torch.distributed.batch_isend_irecv``): NCCL on GPUs; with the gloo
backend, CUDA rows are staged through host memory.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import check

_TAG_UP, _TAG_DOWN = 11, 12  # rows travelling to the rank above / below


def partition(ny: int, world: int) -> list[tuple[int, int]]:
    """Balanced contiguous row bands [y0, y1) of an ny-row grid, one per rank."""
    if world < 1 or ny < world:
        raise ValueError(f"cannot split {ny} rows over {world} ranks")
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((y, y + n))
        y += n
    return out


def lpt_partition(costs, world: int) -> list[list[int]]:
    """Independent grids over `world` ranks: longest processing time first.

    Each grid (cost = its point-steps, ny * nx * T) goes, largest first, to the
    rank with the least assigned cost so far (ties to the lower rank).  The
    busiest rank carries at most 4/3 of the best possible maximum (Graham's
    bound); no grid is split and no rank exchanges anything, so a batch of
    many grids runs as one Batch per rank with no collective.  Returns the
    grid indices of each rank in increasing order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def geometry(ny: int, nx: int, y0: int, y1: int, radius: int, boundary: str,
             steps_per_exchange: int) -> dict:
    """The slab's layout from the C ABI (host only; no GPU needed)."""
    from . import BOUNDARIES
    info = _capi.stencil_slab_info_t()
    check(_capi.load().stencil_slab_geometry(int(ny), int(nx), int(y0), int(y1), int(radius),
                                             BOUNDARIES[boundary], int(steps_per_exchange),
                                             ctypes.byref(info)), "stencil_slab_geometry")
    return {f: getattr(info, f) for f, _ in info._fields_}


class HaloExchange:
    """Swaps the ghost rows of one rank's slab buffer with its two neighbours.

    ``geom`` is this rank's slab geometry (see :func:`geometry`).  The rank
    above rank p is p-1 and the one below p+1 (wrapping for the periodic
    rule); under the zero rule the first and last rank have no neighbour on
    the grid's edge.  With one rank and the periodic rule the slab is its own
    neighbour and the rows are copied locally.
    """

    def __init__(self, geom: dict, rank: int, world: int, group=None):
        self.g = geom
        self.rank, self.world, self.group = rank, world, group
        periodic = geom["boundary"] == _capi.STENCIL_BOUNDARY_PERIODIC
        self.up = (rank - 1) % world if (periodic or rank > 0) else None
        self.down = (rank + 1) % world if (periodic or rank < world - 1) else None
        if (self.up is None) != (geom["ghost_above"] == 0) or (self.down is None) != (geom["ghost_below"] == 0):
            raise ValueError("slab geometry does not match the rank layout")

    def exchange(self, buf) -> None:
        """Fill buf's ghost rows with the neighbours' current boundary rows."""
        import torch
        import torch.distributed as dist
        g, G = self.g, self.g["ghost_depth"]
        rows = lambda a: buf[a:a + G]  # noqa: E731
        if self.world == 1:
            if self.up is not None:  # periodic, one rank: the slab wraps onto itself
                rows(g["recv_above_row"]).copy_(rows(g["send_below_row"]))
                rows(g["recv_below_row"]).copy_(rows(g["send_above_row"]))
            return
        stage = buf.is_cuda and dist.get_backend(self.group) == "gloo"
        sends, recvs = [], []
        if self.up is not None:
            sends.append((rows(g["send_above_row"]), self.up, _TAG_UP))
            recvs.append((rows(g["recv_above_row"]), self.up, _TAG_DOWN))
        if self.down is not None:
            sends.append((rows(g["send_below_row"]), self.down, _TAG_DOWN))
            recvs.append((rows(g["recv_below_row"]), self.down, _TAG_UP))
        # Post every send before every receive, in the same order on all ranks:
        # sends [up, down], receives [from below, from above] pair up message by
        # message even when the two neighbours are the same rank (two ranks,
        # periodic rule).
        recvs.sort(key=lambda r: 0 if r[2] == _TAG_UP else 1)
        if stage:
            torch.cuda.current_stream().synchronize()
            sbufs = [(t.cpu(), peer, tag) for t, peer, tag in sends]
            rbufs = [(torch.empty(t.shape, dtype=t.dtype), peer, tag) for t, peer, tag in recvs]
        else:
            sbufs, rbufs = sends, recvs
        ops = [dist.P2POp(dist.isend, t, peer, self.group, tag) for t, peer, tag in sbufs]
        ops += [dist.P2POp(dist.irecv, t, peer, self.group, tag) for t, peer, tag in rbufs]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        if stage:
            for (dst, _, _), (src, _, _) in zip(recvs, rbufs):
                dst.copy_(src, non_blocking=False)


class SlabSweep:
    """This rank's share of a T-step sweep of one ny x nx grid.

    Each rank constructs one with the same global arguments; ``load`` takes
    the rank's owned rows (or the whole grid, from which they are sliced),
    ``run(T)`` advances T steps with an exchange before every block of at
    most ``steps_per_exchange`` steps, ``owned()`` is a view of the result.
    """

    def __init__(self, ny: int, nx: int, weights, steps_per_exchange: int, boundary: str = "zero",
                 dtype: str = "f32", rank: int | None = None, world: int | None = None, group=None,
                 device=None, **plan_options):
        import torch
        import torch.distributed as dist
        from . import BOUNDARIES, COMPUTES, DTYPES, KERNELS, LOADS
        if rank is None or world is None:
            if dist.is_available() and dist.is_initialized():
                rank, world = dist.get_rank(group), dist.get_world_size(group)
            else:
                rank, world = 0, 1
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
        d = w.shape[0]
        if w.ndim != 2 or w.shape[1] != d or d % 2 != 1:
            raise ValueError(f"weights must be (2r+1, 2r+1), got {w.shape}")
        self.radius = d // 2
        self.shape = (int(ny), int(nx))
        self.rank, self.world = rank, world
        self.y0, self.y1 = partition(ny, world)[rank]
        opt = _capi.stencil_options_t(COMPUTES[plan_options.pop("compute", "auto")],
                                      KERNELS[plan_options.pop("kernel", "stream")],
                                      int(plan_options.pop("tb_depth", 0)),
                                      int(plan_options.pop("threads", 0)),
                                      int(plan_options.pop("tile_rows", 0)),
                                      int(bool(plan_options.pop("autotune", False))), 0, 0, 0,
                                      LOADS[plan_options.pop("load", "auto")])
        if plan_options:
            raise TypeError(f"unknown options {sorted(plan_options)}")
        lib = _capi.load()
        h = ctypes.c_void_p()
        check(lib.stencil_slab_create(ctypes.byref(h), int(ny), int(nx), self.y0, self.y1, self.radius,
                                      w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), DTYPES[dtype],
                                      BOUNDARIES[boundary], int(steps_per_exchange), ctypes.byref(opt)),
              "stencil_slab_create")
        self._h = h
        info = _capi.stencil_slab_info_t()
        check(lib.stencil_slab_info(h, ctypes.byref(info)), "stencil_slab_info")
        self.geom = {f: getattr(info, f) for f, _ in info._fields_}
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buf = torch.zeros((self.geom["buffer_rows"], nx), dtype=tdt, device=dev)
        self.halo = HaloExchange(self.geom, rank, world, group)
        self.S = int(steps_per_exchange)

    def owned(self):
        a = self.geom["ghost_above"]
        return self.buf[a:a + self.y1 - self.y0]

    def load(self, x) -> None:
        """Set the owned rows from x: the owned rows themselves or the whole grid."""
        x = x.to(self.buf.device, self.buf.dtype)
        if tuple(x.shape) == self.shape and self.y1 - self.y0 != self.shape[0]:
            x = x[self.y0:self.y1]
        self.owned().copy_(x)

    def step(self, steps: int) -> None:
        """stencil_slab_step on the current stream: `steps` <= S steps, no exchange."""
        import torch
        stream = int(torch.cuda.current_stream(self.buf.device).cuda_stream)
        check(_capi.load().stencil_slab_step(self._h, self.buf.data_ptr(), int(steps), stream),
              "stencil_slab_step")

    def run(self, T: int) -> None:
        """Advance the owned rows T steps (exchange, then up to S steps, repeated)."""
        t = 0
        while t < T:
            s = min(self.S, T - t)
            self.halo.exchange(self.buf)
            self.step(s)
            t += s

    def status(self) -> None:
        check(_capi.load().stencil_plan_status(_capi.load().stencil_slab_plan(self._h)), "stencil_plan_status")

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _capi.load().stencil_slab_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["partition", "lpt_partition", "geometry", "HaloExchange", "SlabSweep"]
