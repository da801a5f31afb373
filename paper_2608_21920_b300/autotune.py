"""Autotuner of the launch geometry: tile size (dual cells per block) and
threads per block of the push kernel, chosen by timing the push kernel live
(CUDA events on the launching stream) on the caller's own workload."""
from __future__ import annotations

import itertools

import torch

from .gap import Gap


def tune(params, precision="fp32", tiles=(128, 256, 512), threads=(128, 256), variants=(0, 1, 4, 5),
         steps=6, warmup=2, verbose=False):
    """Returns (best (tile, threads, variant), {(tile, threads, variant): ms per push launch})."""
    times = {}
    for tile, thr, var in itertools.product(tiles, threads, variants):
        g = Gap(params, precision=precision, tile=tile, threads=thr, variant=var)
        g.step(warmup)
        g.profile(True)
        g.step(steps)
        ms, n, _ = g.profile(False)
        times[(tile, thr, var)] = ms / max(n, 1)
        if verbose:
            print(f"tile {tile:5d} threads {thr:4d} variant {var}: {times[(tile, thr, var)]:.3f} ms/push", flush=True)
        g.close()
        del g
        torch.cuda.empty_cache()
    best = min(times, key=times.get)
    return best, times
