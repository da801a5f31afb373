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


def tune_step(params, precision="fp32", tiles=(64, 128, 256), threads=(128, 256), rebins=(32, 64),
              steps=60, warmup=20, graph_chunk=20, verbose=False):
    """Whole-step objective for batched runs with QED (where the push kernel is
    the general one and the photon, injection and compaction launches weigh
    in): each (tile, threads, rebin_every) is timed over `steps` graph-replayed
    steps.  Returns (best (tile, threads, rebin_every), {geometry: ms per step})."""
    times = {}
    s = torch.cuda.Stream()
    for tile, thr, rb in itertools.product(tiles, threads, rebins):
        g = Gap(params, precision=precision, tile=tile, threads=thr, rebin_every=rb)
        with torch.cuda.stream(s):
            g.step(warmup, graph_chunk=graph_chunk)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            g.step(steps, graph_chunk=graph_chunk)
            e1.record(s)
        e1.synchronize()
        times[(tile, thr, rb)] = e0.elapsed_time(e1) / steps
        if verbose:
            print(f"tile {tile:5d} threads {thr:4d} rebin {rb:3d}: {times[(tile, thr, rb)]:.3f} ms/step", flush=True)
        g.close()
        del g
        torch.cuda.empty_cache()
    best = min(times, key=times.get)
    return best, times
