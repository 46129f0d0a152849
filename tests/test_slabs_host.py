"""The row-slab decomposition on the CPU: the partition against the
library's, and the ghost-row exchange between processes (gloo ranks, one
slab per rank): after one exchange every ghost row equals the global row it
stands for, the stencil chain of one step (pulled populations, density,
mu, grad mu) evaluated on a slab's own rows from its stored rows alone
equals the whole-lattice evaluation, and the per-slab statistics reduced
across ranks equal the whole lattice's."""
import os
import socket

import numpy as np
import pytest

from paper_2012_11075_gb300 import slabs, wblbe

CX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)


@pytest.mark.parametrize("ny,nslabs", [(3, 1), (8, 2), (64, 3), (257, 5), (4096, 8), (16, 4)])
def test_partition_matches_the_library(ny, nslabs):
    r = slabs.rows(ny, nslabs)
    assert r == wblbe.slab_rows(ny, nslabs)
    assert r[0] == 0 and r[-1] == ny and all(b - a >= slabs.GHOST for a, b in zip(r, r[1:]))
    assert all(v % 2 == 0 for v in r[1:-1])
    p = slabs.plan(ny, nslabs)
    for k, q in enumerate(p):
        assert q["lower_rows"] == [(q["y0"] - 3 + j) % ny for j in range(3)]
        assert q["upper_rows"] == [(q["y0"] + q["n"] + j) % ny for j in range(3)]
        # the ghost rows are owned rows of the named neighbours
        lo, up = p[q["lower_from"]], p[q["upper_from"]]
        assert all(lo["y0"] <= g < lo["y0"] + lo["n"] for g in q["lower_rows"])
        assert all(up["y0"] <= g < up["y0"] + up["n"] for g in q["upper_rows"])


@pytest.mark.parametrize("ny,nslabs", [(5, 2), (7, 2), (8, 3), (0, 1)])
def test_partition_refuses_thin_slabs(ny, nslabs):
    with pytest.raises(ValueError):
        slabs.rows(ny, nslabs)
    if ny > 0:
        with pytest.raises(wblbe.WblbeError):
            wblbe.slab_rows(ny, nslabs)


def _chain(A, kappa=0.0128, beta=0.01, rho_l=1.0, rho_g=0.2):
    """Pulled populations, density, mu and 12 grad(mu) of one step from the
    stored post-collision rows A[9][rows][nx], rows treated as periodic (so
    on a slab only rows 3 .. rows - 4 are meaningful)."""
    f = np.stack([np.roll(A[i], (CY[i], CX[i]), axis=(0, 1)) for i in range(9)])
    rho = f.sum(axis=0)
    r = lambda dy, dx: np.roll(rho, (-dy, -dx), axis=(0, 1))
    lap = (4 * (r(0, 1) + r(0, -1) + r(1, 0) + r(-1, 0)) + r(1, 1) + r(1, -1) + r(-1, 1)
           + r(-1, -1) - 20 * rho) / 6
    a, b = rho - rho_l, rho - rho_g
    mu = 2 * beta * a * b * (a + b) - kappa * lap
    m = lambda dy, dx: np.roll(mu, (-dy, -dx), axis=(0, 1))
    gx = 4 * (m(0, 1) - m(0, -1)) + (m(1, 1) - m(-1, -1)) + (m(-1, 1) - m(1, -1))
    gy = 4 * (m(1, 0) - m(-1, 0)) + (m(1, 1) - m(-1, -1)) - (m(-1, 1) - m(1, -1))
    return rho, mu, gx, gy


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, ny, nx, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(11)
        glob = 0.05 + 0.1 * rng.random((9, ny, nx))            # every rank builds the same
        rows = slabs.stored_rows(ny, world, rank)
        q = slabs.plan(ny, world)[rank]
        local = np.full((9, len(rows), nx), np.nan)
        local[:, 3:3 + q["n"], :] = glob[:, q["y0"]:q["y0"] + q["n"], :]
        slabs.exchange_between_ranks(local, ny, world, rank, dist)
        ghosts_ok = bool(np.array_equal(local, glob[:, rows, :]))
        rho_l, mu_l, gx_l, gy_l = _chain(local)
        rho_g, mu_g, gx_g, gy_g = _chain(glob)
        own = slice(3, 3 + q["n"])
        sel = slice(q["y0"], q["y0"] + q["n"])
        chain_ok = all(np.array_equal(a[own], b[sel]) for a, b in
                       ((rho_l, rho_g), (mu_l, mu_g), (gx_l, gx_g), (gy_l, gy_g)))
        # statistics of the owned rows, reduced across the ranks
        part = torch.tensor([rho_l[own].sum()], dtype=torch.float64)
        hi = torch.tensor([np.abs(gx_l[own]).max(), mu_l[own].max()], dtype=torch.float64)
        lo = torch.tensor([mu_l[own].min()], dtype=torch.float64)
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        dist.all_reduce(hi, op=dist.ReduceOp.MAX)
        dist.all_reduce(lo, op=dist.ReduceOp.MIN)
        stats_ok = (abs(part.item() - rho_g.sum()) <= 1e-12 * rho_g.sum()
                    and hi[0].item() == np.abs(gx_g).max() and hi[1].item() == mu_g.max()
                    and lo[0].item() == mu_g.min())
        out.put((rank, ghosts_ok, chain_ok, bool(stats_ok)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ny,nx", [(2, 23, 17), (3, 30, 8)])
def test_gloo_ranks_exchange_ghost_rows(world, ny, nx):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ny, nx, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    assert all(r[1] and r[2] and r[3] for r in res), res


def test_single_slab_exchange_wraps_onto_itself():
    ny, nx = 9, 5
    rng = np.random.default_rng(3)
    glob = rng.random((9, ny, nx))
    local = np.full((9, ny + 6, nx), np.nan)
    local[:, 3:3 + ny] = glob
    slabs.exchange_between_ranks(local, ny, 1, 0, dist=None)
    assert np.array_equal(local, glob[:, slabs.stored_rows(ny, 1, 0), :])
