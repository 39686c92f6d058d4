"""Row-slab halo exchange on CPU ranks (gloo): the communication half of the
multi-GPU path (paper Sec. IV-A tiles with halos, Sec. IV-B..D halo swaps).

Each rank owns a band of rows of one grid plus radius*S ghost rows on each
side; ranks swap ghost rows with paper_2605_07954_gb300.slab.HaloExchange
before every block of S steps, and advance the block with the FP64 oracle on
the slab buffer (in place of the GPU kernel).  The gathered owned rows must
equal the single-domain oracle run bit for bit: the exchange, the slab
geometry from the C ABI (stencil_slab_geometry, which needs no GPU) and the
claim that S steps on the buffer keep every owned row exact are checked
together.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # pattern, boundary, ny, nx, S, T
    ("box9", "zero", 48, 20, 3, 10),
    ("box9", "periodic", 48, 20, 4, 9),
    ("star13", "zero", 54, 17, 3, 7),
    ("star13", "periodic", 54, 17, 2, 7),
    ("heat5", "periodic", 30, 9, 5, 11),
]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2605_07954_gb300 import inputs, slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        results = []
        for name, boundary, ny, nx, S, T in CASES:
            W = inputs.pattern_weights(name)
            r = W.shape[0] // 2
            u0 = inputs.field(ny, nx).astype(np.float64)
            y0, y1 = slab.partition(ny, world)[rank]
            geom = slab.geometry(ny, nx, y0, y1, r, boundary, S)
            buf = torch.zeros((geom["buffer_rows"], nx), dtype=torch.float64)
            a = geom["ghost_above"]
            buf[a:a + y1 - y0] = torch.from_numpy(u0[y0:y1])
            halo = slab.HaloExchange(geom, rank, world)
            t = 0
            while t < T:
                s = min(S, T - t)
                halo.exchange(buf)
                buf = torch.from_numpy(oracle.sweep_f64(buf.numpy(), W, s, boundary))
                t += s
            results.append(buf[a:a + y1 - y0].numpy().copy())
        q.put((rank, results))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_match_single_domain_bitwise(world, oracle):
    from paper_2605_07954_gb300 import build, inputs
    build.build()
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for i, (name, boundary, ny, nx, S, T) in enumerate(CASES):
        W = inputs.pattern_weights(name)
        ref = oracle.sweep_f64(inputs.field(ny, nx).astype(np.float64), W, T, boundary)
        full = np.concatenate([got[r][i] for r in range(world)], axis=0)
        assert np.array_equal(full, ref), (name, boundary, world)


def test_partition_and_geometry():
    from paper_2605_07954_gb300 import build, slab
    build.build()
    assert slab.partition(10, 3) == [(0, 4), (4, 7), (7, 10)]
    g = slab.geometry(64, 16, 0, 32, 3, "zero", 4)
    assert (g["ghost_above"], g["ghost_below"], g["buffer_rows"]) == (0, 12, 44)
    assert (g["send_below_row"], g["recv_below_row"]) == (20, 32)
    g = slab.geometry(64, 16, 32, 64, 3, "periodic", 4)
    assert (g["ghost_above"], g["ghost_below"], g["buffer_rows"]) == (12, 12, 56)
    assert (g["send_above_row"], g["send_below_row"], g["recv_above_row"], g["recv_below_row"]) == (12, 32, 0, 44)
    # a slab thinner than the ghost depth cannot be fed by one neighbour
    from paper_2605_07954_gb300._capi import StencilError
    with pytest.raises(StencilError):
        slab.geometry(64, 16, 0, 8, 3, "zero", 4)
    with pytest.raises(StencilError):
        slab.geometry(64, 16, 10, 8, 1, "zero", 4)


def test_lpt_partition_balances_the_batch():
    """The 256-grid batch over 1..8 ranks: every grid on exactly one rank, the
    busiest rank within Graham's 4/3 bound of the lower bound max(mean, largest)."""
    from paper_2605_07954_gb300 import inputs, slab
    sides, _ = inputs.batch_spec(256)
    costs = [int(s) * int(s) * 200 for s in sides]
    for world in (1, 2, 3, 4, 8):
        parts = slab.lpt_partition(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(256))
        loads = [sum(costs[i] for i in p) for p in parts]
        lower = max(sum(costs) / world, max(costs))
        assert max(loads) <= 4 / 3 * lower
    # by hand: 5 -> r0, 4 -> r1, 3 -> r1 (4 < 5), 2 -> r0 (5 < 7), 1 -> r0 (7 = 7, lower rank)
    assert slab.lpt_partition([5, 1, 4, 2, 3], 2) == [[0, 1, 3], [2, 4]]
