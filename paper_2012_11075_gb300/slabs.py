"""Row-slab decomposition of one lattice: the partition and the ghost-row
exchange plan, and the exchange itself between processes.

One step of Eq. D2Q9 at a node reads post-collision populations of the
previous step within GHOST = 3 nodes (pulled populations, then the
densities that mu and grad mu need, Sec. II).  A slab of rows [y0, y0 + n)
is stored with GHOST ghost rows on each side (stored row b holds global row
y0 - GHOST + b, so the owned rows are stored rows [GHOST, GHOST + n)); after
every step each slab sends its first GHOST owned rows to the slab below
(that slab's upper ghosts) and its last GHOST owned rows to the slab above
(its lower ghosts), periodically.  Full rows are exchanged, so the corner
values that diagonal directions pull come with them.

The library (wblbe_slabs_*) runs all slabs of a lattice on one device with
this partition and exchange; ``exchange_between_ranks`` carries the same
plan between processes with torch.distributed point-to-point messages (one
slab per rank), which is how the plan is exercised across ranks on the CPU.
"""
from __future__ import annotations

import numpy as np

GHOST = 3


def rows(ny: int, nslabs: int) -> list:
    """First global row of every slab (length nslabs + 1, last = ny):
    near-equal runs with boundaries on even rows (the FP32 stochastic
    rounding draws one hash per pair of rows 2j, 2j + 1).  Every slab must
    own at least GHOST rows."""
    if ny < 1 or nslabs < 1:
        raise ValueError("need ny >= 1 and nslabs >= 1")
    out = [0] + [(k * ny // nslabs) & ~1 for k in range(1, nslabs)] + [ny]
    if any(b - a < GHOST for a, b in zip(out, out[1:])):
        raise ValueError(f"every slab needs at least {GHOST} rows (ny = {ny}, nslabs = {nslabs})")
    return out


def plan(ny: int, nslabs: int) -> list:
    """For every slab k: its rows and where its ghost rows come from.
    lower_from / upper_from: the slab indices (periodic) whose owned rows
    fill the lower / upper ghost rows; lower_rows / upper_rows: those global
    rows, in stored order."""
    r = rows(ny, nslabs)
    out = []
    for k in range(nslabs):
        y0, y1 = r[k], r[k + 1]
        out.append({
            "y0": y0, "n": y1 - y0,
            "lower_from": (k - 1) % nslabs,
            "lower_rows": [(y0 - GHOST + j) % ny for j in range(GHOST)],
            "upper_from": (k + 1) % nslabs,
            "upper_rows": [(y1 + j) % ny for j in range(GHOST)],
        })
    return out


def stored_rows(ny: int, nslabs: int, k: int) -> list:
    """Global row held by every stored row of slab k (ghosts included)."""
    p = plan(ny, nslabs)[k]
    return [(p["y0"] - GHOST + b) % ny for b in range(p["n"] + 2 * GHOST)]


def exchange_between_ranks(local: np.ndarray, ny: int, nslabs: int, rank: int, dist) -> None:
    """Refresh the ghost rows of this rank's slab (slab index = rank) from the
    neighbouring ranks' owned rows, in place.  local: array whose second-last
    axis holds the slab's stored rows (n + 2 GHOST), e.g. [9][rows][nx]
    populations; every rank calls this at the same step.  dist: an
    initialised torch.distributed (any backend able to send host tensors,
    e.g. gloo), one rank per slab."""
    import torch

    p = plan(ny, nslabs)[rank]
    n = p["n"]
    if local.shape[-2] != n + 2 * GHOST:
        raise ValueError(f"slab {rank} stores {n + 2 * GHOST} rows, got {local.shape[-2]}")
    first = np.ascontiguousarray(local[..., GHOST:2 * GHOST, :])     # to the slab below
    last = np.ascontiguousarray(local[..., n:n + GHOST, :])          # to the slab above
    if nslabs == 1:
        local[..., :GHOST, :] = last
        local[..., n + GHOST:, :] = first
        return
    below, above = p["lower_from"], p["upper_from"]
    got_lower = torch.empty(first.shape, dtype=torch.from_numpy(first).dtype)
    got_upper = torch.empty(first.shape, dtype=torch.from_numpy(first).dtype)
    # tag 0: rows travelling upwards (a slab's last rows), tag 1: downwards
    reqs = [dist.isend(torch.from_numpy(last), dst=above, tag=0),
            dist.isend(torch.from_numpy(first), dst=below, tag=1),
            dist.irecv(got_lower, src=below, tag=0),
            dist.irecv(got_upper, src=above, tag=1)]
    for r in reqs:
        r.wait()
    local[..., :GHOST, :] = got_lower.numpy()
    local[..., n + GHOST:, :] = got_upper.numpy()
