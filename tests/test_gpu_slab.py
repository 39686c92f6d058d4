"""Row slabs on the GPU: stencil_slab_step with ghost rows from neighbouring
slabs (paper Sec. IV-A tiles with halos, Sec. IV-B..D halo swaps).

Several slabs of one grid, exchanged either in one process (rows copied
between the slabs' buffers) or between two processes over torch.distributed
(gloo, both on cuda:0: they do not wait on each other inside any kernel), must
reproduce the single-domain stencil_run of the streaming kernel bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2605_07954_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07954_gb300 import build
    build.build()


def _single(u0, W, T, boundary, dtype=torch.float32, **opts):
    from paper_2605_07954_gb300 import Plan
    x = torch.from_numpy(u0).to(dtype).cuda()
    dt = {torch.float32: "f32", torch.bfloat16: "bf16"}[dtype]
    p = Plan(x.shape[0], x.shape[1], W, dtype=dt, boundary=boundary, kernel="stream", **opts)
    y = p.run(x, T)
    torch.cuda.synchronize()
    p.close()
    return y


def _local_exchange(slabs):
    """Copy every slab's boundary rows into its neighbours' ghost rows."""
    world = len(slabs)
    for r, s in enumerate(slabs):
        g, G = s.geom, s.geom["ghost_depth"]
        if g["ghost_above"]:
            up = slabs[(r - 1) % world]
            s.buf[g["recv_above_row"]:g["recv_above_row"] + G] = \
                up.buf[up.geom["send_below_row"]:up.geom["send_below_row"] + G]
        if g["ghost_below"]:
            dn = slabs[(r + 1) % world]
            s.buf[g["recv_below_row"]:g["recv_below_row"] + G] = \
                dn.buf[dn.geom["send_above_row"]:dn.geom["send_above_row"] + G]


@pytest.mark.parametrize("name,boundary,world,S,T", [
    ("box9", "zero", 3, 8, 40),
    ("box9", "periodic", 2, 8, 37),
    ("star13", "zero", 4, 4, 22),
    ("star13", "periodic", 3, 6, 30),
    ("heat5", "zero", 2, 16, 64),
])
def test_slabs_in_one_process_bitwise(name, boundary, world, S, T):
    from paper_2605_07954_gb300.slab import SlabSweep
    W = inputs.pattern_weights(name)
    ny, nx = 1000, 1024
    u0 = inputs.field(ny, nx)
    ref = _single(u0, W, T, boundary)
    x = torch.from_numpy(u0).cuda()
    slabs = [SlabSweep(ny, nx, W, S, boundary, rank=r, world=world) for r in range(world)]
    for s in slabs:
        s.load(x)
    t = 0
    while t < T:
        st = min(S, T - t)
        _local_exchange(slabs)
        for s in slabs:
            s.step(st)
        t += st
    torch.cuda.synchronize()
    for s in slabs:
        s.status()
    got = torch.cat([s.owned() for s in slabs], dim=0)
    assert torch.equal(got, ref), (name, boundary, world)
    for s in slabs:
        s.close()


def test_single_slab_periodic_wraps_onto_itself():
    """One rank, periodic rule: the slab's ghost rows are its own far rows."""
    from paper_2605_07954_gb300.slab import SlabSweep
    W = inputs.pattern_weights("star13")
    u0 = inputs.field(300, 256)
    s = SlabSweep(300, 256, W, 5, "periodic", rank=0, world=1)
    s.load(torch.from_numpy(u0).cuda())
    s.run(23)
    torch.cuda.synchronize()
    assert torch.equal(s.owned(), _single(u0, W, 23, "periodic"))
    s.close()


def test_slabs_bf16_same_launch_depths():
    """BF16 storage rounds once per launch: with blocks of 16 steps at depth 8
    (two launches per block) the slabs match the single-domain run bit for bit."""
    from paper_2605_07954_gb300.slab import SlabSweep
    W = inputs.pattern_weights("box9")
    ny, nx, S, T = 512, 768, 16, 64
    u0 = inputs.field(ny, nx)
    ref = _single(u0, W, T, "zero", torch.bfloat16, tb_depth=8)
    x = torch.from_numpy(u0).to(torch.bfloat16).cuda()
    slabs = [SlabSweep(ny, nx, W, S, "zero", dtype="bf16", rank=r, world=2, tb_depth=8) for r in range(2)]
    for s in slabs:
        s.load(x)
    for _ in range(T // S):
        _local_exchange(slabs)
        for s in slabs:
            s.step(S)
    torch.cuda.synchronize()
    got = torch.cat([s.owned() for s in slabs], dim=0)
    assert torch.equal(got, ref)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2605_07954_gb300 import inputs
    from paper_2605_07954_gb300.slab import SlabSweep
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = []
        for name, boundary, S, T in (("box9", "zero", 8, 24), ("star13", "periodic", 4, 18)):
            W = inputs.pattern_weights(name)
            s = SlabSweep(640, 512, W, S, boundary)
            s.load(torch.from_numpy(inputs.field(640, 512)).cuda())
            s.run(T)
            torch.cuda.synchronize()
            s.status()
            out.append(s.owned().cpu().numpy().copy())
            s.close()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu_bitwise():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for i, (name, boundary, S, T) in enumerate((("box9", "zero", 8, 24), ("star13", "periodic", 4, 18))):
        W = inputs.pattern_weights(name)
        ref = _single(inputs.field(640, 512), W, T, boundary).cpu().numpy()
        full = np.concatenate([got[0][i], got[1][i]], axis=0)
        assert np.array_equal(full, ref), name
