"""Autotuner of the batched apply's launch shape.

The batched kernel sweeps a group of subdomains of one system in lockstep
(their levels merged), and how many to group trades steps per CTA against
shared memory (vectors of every grouped subdomain and right-hand side) and
ring depth.  ``tune_group`` builds the batch for each candidate group size,
times the batched apply with CUDA events (L2 flushed between launches, as the
bench does) and returns the fastest.  Every candidate computes the same
result; only the speed differs.
"""
from __future__ import annotations

import torch

from . import pslr


def _time_apply(bt, prec, steps, warmup, flush):
    dtype = torch.float64 if prec == pslr.PSLR_FP64 else torch.float32
    b = torch.rand(bt.info["n_total"], dtype=dtype, device="cuda")
    z = torch.empty_like(b)
    for _ in range(warmup):
        bt.apply(b, z)
    bt.sync()
    st = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        bt.apply(b, z)
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    bt.sync()
    ms.sort()
    return ms[len(ms) // 2]


def tune_group(systems, nrhs, prec=pslr.PSLR_FP32, candidates=(1, 2, 4, 6, 8), steps=5, warmup=2,
               flush_bytes=512 << 20):
    """Time the batched apply of ``systems`` (set-up :class:`pslr.Pslr`
    contexts with their low-rank terms) for each requested group size and
    return ``(best_group, table)``; ``table`` maps each request to
    ``(effective group, ms per apply)`` (a request larger than shared memory
    allows is reduced by the library)."""
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device="cuda")
    k = 0 if prec == pslr.PSLR_FP64 else 1
    table = {}
    for g in candidates:
        bt = pslr.Batch(systems, nrhs, group=g)
        try:
            table[g] = (bt.info["group"][k], _time_apply(bt, prec, steps, warmup, flush))
        finally:
            bt.close()
    best = min(table, key=lambda g: table[g][1])
    return best, table
