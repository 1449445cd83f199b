"""Autotuner of the batched solve's launch shape.

For a batch it times every candidate (storage format x right-hand sides per
SpMM chunk x blocks per SM x step form: textbook or single-reduction CG) on a
short run of the real launch -- the same
kernel, a fixed number of CG steps with the stopping test disabled -- and
keeps the fastest per step.  Results are cached per batch signature (the
sorted mesh sizes), in memory and optionally in a JSON file.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import torch

from . import fe

FORMATS = ("bcrs3", "sell")
KRHS = (1, 2, 4)
BLOCKS_PER_SM = (0, 2)   # 0: as many as fit
METHODS = (fe.BATCH_TEXTBOOK, fe.BATCH_SINGLE_REDUCTION)


@dataclass
class Choice:
    fmt: str
    krhs: int
    blocks_per_sm: int
    ms_per_step: float
    method: int = fe.BATCH_TEXTBOOK


_cache: dict = {}


def signature(sizes) -> str:
    return ",".join(str(n) for n in sorted(int(n) for n in sizes))


def tune(batch: "fe.Batch", steps: int = 24, repeats: int = 2, cache_file: str | None = None,
         candidates=None) -> Choice:
    key = signature(batch.sizes)
    if key in _cache:
        return _cache[key]
    if cache_file and os.path.exists(cache_file):
        with open(cache_file) as f:
            disk = json.load(f)
        if key in disk:
            _cache[key] = Choice(**disk[key])
            return _cache[key]
    work = batch.workspace()
    best = None
    cands = candidates or [(f, k, b, m) for f in FORMATS for k in KRHS for b in BLOCKS_PER_SM
                           for m in METHODS]
    for cand in cands:
        fmt, krhs, bps = cand[:3]
        method = cand[3] if len(cand) > 3 else fe.BATCH_TEXTBOOK
        mats = batch.mats_for(fmt)
        try:
            plan = fe.fe_cg_batched_plan(mats, batch.b, batch.x, krhs, work, blocks_per_sm=bps,
                                         method=method)
        except fe.FeError:
            continue
        times = []
        for _ in range(repeats):
            batch.reset()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fe.fe_cg_batched_launch(plan, 0.0, steps)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) / steps)
        t = min(times)
        if best is None or t < best.ms_per_step:
            best = Choice(fmt, krhs, bps, t, method)
    batch.reset()
    if best is None:
        raise RuntimeError("no batched launch shape fits this batch")
    _cache[key] = best
    if cache_file:
        disk = {}
        if os.path.exists(cache_file):
            with open(cache_file) as f:
                disk = json.load(f)
        disk[key] = best.__dict__
        with open(cache_file, "w") as f:
            json.dump(disk, f, indent=1)
    return best
