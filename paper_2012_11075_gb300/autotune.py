"""Autotuner of the batched persistent kernel's launch configuration.

For a given case mix it times candidate (tile_x, rows_per_tile,
steps_per_launch) triples on the device, through the batch's own advance()
(so the per-launch checks are part of the cost), and keeps the one with the
highest lattice-update rate.  Winners are cached in a JSON file keyed by the
GPU name, precision, scheme and a size-class signature of the mix
(``WBLBE_TUNE_CACHE`` overrides the cache path).
"""
from __future__ import annotations

import json
import math
import os
import time
from pathlib import Path

# strip width x rows per tile x steps per launch; 1-16 steps per launch and
# 16-row tiles were never chosen on the benchmark mix (the per-launch host
# check, the launch tail and the halo rows weigh too much)
DEFAULT_CANDIDATES = [(tx, rows, k) for tx in (64, 128, 256) for rows in (32, 64, 128)
                      for k in (32, 64, 128)]


def cache_path() -> Path:
    env = os.environ.get("WBLBE_TUNE_CACHE")
    if env:
        return Path(env)
    return Path(__file__).resolve().parent / "_lib" / "tune_cache.json"


def size_class(shapes) -> str:
    """Histogram of log2(nodes) over the mix, as a short key."""
    hist = {}
    for nx, ny in shapes:
        b = int(math.log2(max(nx * ny, 1)))
        hist[b] = hist.get(b, 0) + 1
    total = sum(hist.values())
    return ",".join(f"{b}:{round(100 * c / total)}" for b, c in sorted(hist.items()))


def cache_key(gpu: str, precision: int, scheme: int, shapes) -> str:
    return f"{gpu}|p{precision}|s{scheme}|{size_class(shapes)}"


def load_cache() -> dict:
    p = cache_path()
    if p.exists():
        try:
            return json.loads(p.read_text())
        except (OSError, ValueError):
            return {}
    return {}


def store_cache(key: str, entry: dict):
    p = cache_path()
    p.parent.mkdir(parents=True, exist_ok=True)
    data = load_cache()
    data[key] = entry
    tmp = p.with_suffix(f".{os.getpid()}.tmp")
    tmp.write_text(json.dumps(data, indent=1, sort_keys=True))
    os.replace(tmp, p)


def tune(batch, shapes, gpu_name: str, candidates=None, launches: int = 3,
         use_cache: bool = True, sync=None) -> dict:
    """Pick the fastest configuration for the cases resident in ``batch``
    (their lattice shapes are ``shapes``); the batch is left configured with
    it.  Timing advances the resident cases.  Returns the winning entry
    (config and measured rate of every candidate).  If the cases stop before
    any candidate could be timed, the first candidate is kept, uncached."""
    key = cache_key(gpu_name, batch.precision, batch.scheme, shapes)
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            batch.set_config(*hit["config"])
            return dict(hit, cached=True)
    nodes = sum(nx * ny for nx, ny in shapes)
    rates = {}
    for cand in (candidates or DEFAULT_CANDIDATES):
        batch.set_config(*cand)
        batch.advance(1)                     # warm-up: retile, graph capture
        if sync:
            sync()
        t0 = time.perf_counter()
        batch.advance(launches)
        if sync:
            sync()
        dt = time.perf_counter() - t0
        running = batch.counts()["running"]
        if running == 0 or dt <= 0:
            break
        rates[f"{cand[0]}x{cand[1]}x{cand[2]}"] = nodes * cand[2] * launches / dt / 1e6
    cands = list(candidates or DEFAULT_CANDIDATES)
    if not rates:
        batch.set_config(*cands[0])
        return {"config": list(cands[0]), "mlups": None, "candidates": {}, "cached": False}
    best = max(rates, key=rates.get)
    cfg = tuple(int(v) for v in best.split("x"))
    batch.set_config(*cfg)
    entry = {"config": list(cfg), "mlups": rates[best], "candidates": rates}
    if use_cache:
        store_cache(key, entry)
    return dict(entry, cached=False)
