"""Slab split along y on CPU: the row split, the neighbours, and the face trade of
`slab.halo_exchange` between world_size 2 and 3 gloo ranks.

Each rank holds rows [y0, y1) of a random 24 x 17 lattice and advances them with the
oracle's own step (Eq. 1), periodic within the slab; after each step the ranks trade,
through `halo_exchange`, the populations that crossed a face. The oracle holds
pre-collision populations f(x, t), so a step taken periodically within the slab
leaves, in its bottom row, the populations with c_y = +1 (i = 2, 5, 6) that came from
its own top row; in the whole lattice they come from the top row of the slab below,
which is exactly what the slab below holds in its own bottom row after its periodic
step. So the bottom row's i = 2, 5, 6 go up and are replaced by the slab below's, and
the top row's i = 4, 7, 8 go down (the CUDA path trades the same slots one pull
earlier: the top row's 2, 5, 6 and the bottom row's 4, 7, 8 of its post-collision
buffer). After 20 steps the slabs put together equal the oracle's single-lattice run
bit for bit, and the summed diagnostics equal the whole lattice's.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, STEPS, THETA, TAU, MODEL = 24, 17, 20, 1.0 / 3.0, 0.8, 3


def test_slab_rows_cover_the_lattice_evenly():
    from paper_2602_21242_gb300.slab import slab_rows

    for ny in (1, 2, 7, 17, 64):
        for k in range(1, min(ny, 9) + 1):
            rows = [slab_rows(ny, k, j) for j in range(k)]
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            sizes = [b - a for a, b in rows]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab_rows(3, 4, 0)
    with pytest.raises(ValueError):
        slab_rows(8, 2, 2)


def test_neighbours_are_periodic():
    from paper_2602_21242_gb300.slab import neighbours

    assert neighbours(0, 3) == (2, 1)
    assert neighbours(2, 3) == (1, 0)
    assert neighbours(0, 1) == (0, 0)
    assert neighbours(1, 2) == (0, 0)


def test_face_populations_are_those_crossing_y():
    from oracle.oracle import CX, CY
    from paper_2602_21242_gb300.slab import DOWN_POPS, UP_POPS

    assert sorted(UP_POPS) == [i for i in range(9) if CY[i] == 1]
    assert sorted(DOWN_POPS) == [i for i in range(9) if CY[i] == -1]
    # each face buffer lists c_x = 0, +1, -1 in that order
    assert [int(CX[i]) for i in UP_POPS] == [0, 1, -1]
    assert [int(CX[i]) for i in DOWN_POPS] == [0, -1, 1]


def _worker(rank, world, port, f0, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2602_21242_gb300.slab import DOWN_POPS, UP_POPS, global_diagnostics, halo_exchange, slab_rows

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        y0, y1 = slab_rows(NY, world, rank)
        f = np.array(f0[:, y0:y1, :])
        up, down = list(UP_POPS), list(DOWN_POPS)
        bufs = [torch.empty(3 * NX, dtype=torch.float64) for _ in range(4)]
        for _ in range(STEPS):
            f = O.run(f, THETA, TAU, MODEL, 1)
            bufs[0].copy_(torch.from_numpy(f[up, 0, :].reshape(-1)))
            bufs[1].copy_(torch.from_numpy(f[down, -1, :].reshape(-1)))
            halo_exchange(*bufs)
            f[up, 0, :] = bufs[2].numpy().reshape(3, NX)
            f[down, -1, :] = bufs[3].numpy().reshape(3, NX)
        diag = global_diagnostics(O.diagnostics(f), torch.device("cpu"))
        out.put((rank, y0, y1, f, diag))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_slabs_equal_the_single_lattice_run(oracle, world):
    import torch.multiprocessing as mp

    from paper_2602_21242_gb300 import flows

    f0 = flows.random_populations(NX, NY, seed=2602 + world, spread=0.2)
    ref = oracle.run(f0, THETA, TAU, MODEL, STEPS)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + (os.getpid() * 7 + world) % 900
    procs = [ctx.Process(target=_worker, args=(r, world, port, f0, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in range(world)), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    whole = np.empty_like(ref)
    for _, y0, y1, f, _ in got:
        whole[:, y0:y1, :] = f
    assert np.array_equal(whole, ref)
    want = oracle.diagnostics(ref)
    for *_, diag in got:
        assert diag[4] == 0
        np.testing.assert_allclose(diag[:4], want[:4], rtol=1e-13, atol=1e-13 * abs(want[0]))


def test_single_rank_exchange_returns_the_buffers():
    import torch

    from paper_2602_21242_gb300.slab import halo_exchange

    bufs = [torch.arange(6, dtype=torch.float64) + 10 * k for k in range(4)]
    halo_exchange(*bufs)
    assert torch.equal(bufs[2], bufs[0]) and torch.equal(bufs[3], bufs[1])
